// k_grad.cu -- adjoint of simus_rf (vector-Jacobian product), FP32 on the CUDA cores.
//
// With drf = dL/drf and Lambda_q(e,t) = H_q sum_j drf[t][e][j] e^{-2 pi i q j / Nt} (the
// adjoint of the inverse DFT and of the transfer factor), dL = Re sum Lambda dRF_q.  Per
// bin q and scatterer s, with c_te = W e^{i w dtau} and G_e = sum_mu g (Eq. 33):
//   P_t = sum_e c_te G_e,   A_t = sum_e Lambda_te G_e      (and the same with dG/dX, dG/dZ)
//   dL/dR_s      += Re sum_t A_t P_t
//   dL/dX_s      += R_s Re sum_t (A_t Px_t + P_t Ax_t),   dL/dZ_s likewise
//   B_q(t,e)     += R_s A_t G_e,   dL/d dtau_te = Re sum_q i w_q c_te B_q(t,e).
// Green's terms and their derivatives are recomputed here, never stored across calls.
//
// Kernels: k_adjoint_dft (Lambda), k_grad (per tile of QB bins x chunk of scatterers,
// groups of SB scatterers: generation -> contraction -> B accumulation; per-bin-tile
// partial gradients and per-chunk partial B, reduced in a fixed order afterwards),
// k_grad_reduce_scat, k_grad_delays.
#include <algorithm>

#include "green.cuh"
#include "simus_internal.h"

namespace simus {

namespace {
constexpr int kGThreads = 256;
constexpr int kGQB = 2;     // bins per tile
constexpr int kGSB = 8;     // scatterers per group
}  // namespace

// lam[t][k][e] = H_k sum_j drf[t][e][j] exp(-2 pi i ((q_lo + k) j mod Nt) / Nt).
// Thread per bin and CB channels; samples staged in shared memory.
template <int CB, int JB>
__global__ void __launch_bounds__(256)
k_adjoint_dft(const float *__restrict__ drf, int N, int n_chan, int nq, int q_lo, int nt,
              const float2 *__restrict__ H, float2 *__restrict__ lam) {
    __shared__ float ds[JB][CB];
    const int tid = threadIdx.x;
    const int k = blockIdx.x * 256 + tid;
    const int c0 = blockIdx.y * CB;
    const int q = q_lo + (k < nq ? k : 0);
    const float wstep = -6.283185307179586f / (float)nt;
    const int half = nt / 2;
    float ar[CB], ai[CB];
#pragma unroll
    for (int c = 0; c < CB; ++c) ar[c] = ai[c] = 0.f;
    int m = 0;   // q * j mod Nt at j = jb
    for (int jb = 0; jb < nt; jb += JB) {
        __syncthreads();
        for (int i = tid; i < JB * CB; i += 256) {
            int cc = i / JB, jj = i - cc * JB;
            int c = c0 + cc, j = jb + jj;
            ds[jj][cc] = (c < n_chan && j < nt) ? drf[(size_t)c * nt + j] : 0.f;
        }
        __syncthreads();
        const int jend = min(JB, nt - jb);
        for (int jj = 0; jj < jend; ++jj) {
            int mm = m > half ? m - nt : m;
            float s, co;
            sincos_a(wstep * (float)mm, s, co);     // exp(-2 pi i m / Nt) = co + i s
#pragma unroll
            for (int c = 0; c < CB; ++c) {
                float v = ds[jj][c];
                ar[c] = fmaf(v, co, ar[c]);
                ai[c] = fmaf(v, s, ai[c]);
            }
            m += q;
            if (m >= nt) m -= nt;
        }
    }
    if (k < nq) {
        const float2 h = H[k];
#pragma unroll
        for (int c = 0; c < CB; ++c) {
            int cc = c0 + c;
            if (cc < n_chan) {
                int t = cc / N, e = cc - t * N;
                lam[((size_t)t * nq + k) * N + e] =
                    make_float2(h.x * ar[c] - h.y * ai[c], h.x * ai[c] + h.y * ar[c]);
            }
        }
    }
}

template <bool NARROW>
__global__ void __launch_bounds__(kGThreads, 1)
k_grad(const GreenConst gc, const SubElem *__restrict__ sub_g, const float *__restrict__ xg,
       const float *__restrict__ zg, const float *__restrict__ rcg, int64_t S, int64_t chunk_len,
       int T, const float2 *__restrict__ cw, const float2 *__restrict__ lam,
       float *__restrict__ gpart /*[3][n_qtiles][S]*/, int n_qtiles,
       float2 *__restrict__ bpart /*[n_chunks][T][nq][N]*/) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = gc.N, nu = gc.nu, M = gc.M, nq = gc.nq;
    const int tid = threadIdx.x;
    constexpr int QB = kGQB, SB = kGSB;
    float4 *sc = reinterpret_cast<float4 *>(smem_raw);              // [SB] (x, 0, z, R)
    SubElem *sub = reinterpret_cast<SubElem *>(sc + SB);            // [M]
    float2 *cwt = reinterpret_cast<float2 *>(sub + M);              // [QB][T][N]
    float2 *lat = cwt + QB * T * N;                                 // [QB][T][N]
    float2 *Bt = lat + QB * T * N;                                  // [QB][T][N]
    float2 *Gt = Bt + QB * T * N;                                   // [3][QB][SB][N]
    float2 *RA = Gt + 3 * QB * SB * N;                              // [QB][SB][T]
    float *sg = reinterpret_cast<float *>(RA + QB * SB * T);        // [3][QB*SB*T]
    const int nit = QB * SB * T;

    const int qt = blockIdx.x, chunk = blockIdx.y;
    const int k0 = qt * QB;
    const int64_t s_begin = (int64_t)chunk * chunk_len;
    const int64_t s_end = min(S, s_begin + chunk_len);

    for (int i = tid; i < M; i += kGThreads) sub[i] = sub_g[i];
    for (int i = tid; i < QB * T * N; i += kGThreads) {
        int j = i / (T * N), r = i - j * T * N, t = r / N, e = r - t * N, k = k0 + j;
        bool ok = k < nq;
        cwt[i] = ok ? cw[((size_t)t * nq + k) * N + e] : make_float2(0.f, 0.f);
        lat[i] = ok ? lam[((size_t)t * nq + k) * N + e] : make_float2(0.f, 0.f);
        Bt[i] = make_float2(0.f, 0.f);
    }
    const float q0 = (float)(gc.q_lo + k0);
    const size_t plane = (size_t)QB * SB * N;

    for (int64_t sb = s_begin; sb < s_end; sb += SB) {
        __syncthreads();
        if (tid < SB) {
            int64_t s = sb + tid;
            sc[tid] = s < s_end ? make_float4(xg[s], 0.f, zg[s], rcg[s]) : make_float4(0.f, 0.f, 1.f, 0.f);
        }
        __syncthreads();

        // 1. G, dG/dX, dG/dZ tiles
        for (int pr = tid; pr < SB * N; pr += kGThreads) {
            const int s = pr / N, e = pr - s * N;
            const float4 ps = sc[s];
            float2 G[QB], GX[QB], GZ[QB];
#pragma unroll
            for (int j = 0; j < QB; ++j) G[j] = GX[j] = GZ[j] = make_float2(0.f, 0.f);
            for (int mu = 0; mu < nu; ++mu) {
                const SubElem se = sub[e * nu + mu];
                const PairSetup P = pair_setup<false>(gc, se, ps.x, 0.f, ps.z, q0);
                const PairGrad Q = pair_grad(gc, se, ps.x, ps.z, P);
#pragma unroll
                for (int j = 0; j < QB; ++j) {
                    const float q = q0 + (float)j;
                    const float amp = (gc.two_d ? rsqrt_a(P.rh) : gc.h * P.inv_r) *
                                      ex2_a(-q * gc.att2 * P.rh);
                    float2 g, gx, gz;
                    green_grad_term<NARROW>(gc, P, Q, q, amp, g, gx, gz);
                    G[j].x += g.x; G[j].y += g.y;
                    GX[j].x += gx.x; GX[j].y += gx.y;
                    GZ[j].x += gz.x; GZ[j].y += gz.y;
                }
            }
#pragma unroll
            for (int j = 0; j < QB; ++j) {
                const size_t o = ((size_t)j * SB + s) * N + e;
                Gt[o] = G[j];
                Gt[plane + o] = GX[j];
                Gt[2 * plane + o] = GZ[j];
            }
        }
        __syncthreads();

        // 2. contractions per (bin, scatterer, transmit)
        for (int it = tid; it < QB * SB * T; it += kGThreads) {
            const int j = it / (SB * T), r = it - j * SB * T, s = r / T, t = r - s * T;
            const float2 *g0 = Gt + ((size_t)j * SB + s) * N;
            const float2 *g1 = g0 + plane, *g2 = g0 + 2 * plane;
            const float2 *c = cwt + ((size_t)j * T + t) * N;
            const float2 *l = lat + ((size_t)j * T + t) * N;
            float Pr = 0, Pi = 0, Ar = 0, Ai = 0, Pxr = 0, Pxi = 0, Axr = 0, Axi = 0,
                  Pzr = 0, Pzi = 0, Azr = 0, Azi = 0;
            for (int e = 0; e < N; ++e) {
                const float2 cc = c[e], ll = l[e], a = g0[e], bx = g1[e], bz = g2[e];
                Pr = fmaf(cc.x, a.x, fmaf(-cc.y, a.y, Pr));
                Pi = fmaf(cc.x, a.y, fmaf(cc.y, a.x, Pi));
                Ar = fmaf(ll.x, a.x, fmaf(-ll.y, a.y, Ar));
                Ai = fmaf(ll.x, a.y, fmaf(ll.y, a.x, Ai));
                Pxr = fmaf(cc.x, bx.x, fmaf(-cc.y, bx.y, Pxr));
                Pxi = fmaf(cc.x, bx.y, fmaf(cc.y, bx.x, Pxi));
                Axr = fmaf(ll.x, bx.x, fmaf(-ll.y, bx.y, Axr));
                Axi = fmaf(ll.x, bx.y, fmaf(ll.y, bx.x, Axi));
                Pzr = fmaf(cc.x, bz.x, fmaf(-cc.y, bz.y, Pzr));
                Pzi = fmaf(cc.x, bz.y, fmaf(cc.y, bz.x, Pzi));
                Azr = fmaf(ll.x, bz.x, fmaf(-ll.y, bz.y, Azr));
                Azi = fmaf(ll.x, bz.y, fmaf(ll.y, bz.x, Azi));
            }
            const float R = sc[s].w;
            sg[it] = Ar * Pr - Ai * Pi;                                             // dL/dR
            sg[nit + it] = R * ((Ar * Pxr - Ai * Pxi) + (Pr * Axr - Pi * Axi));     // dL/dX
            sg[2 * nit + it] = R * ((Ar * Pzr - Ai * Pzi) + (Pr * Azr - Pi * Azi)); // dL/dZ
            RA[((size_t)j * SB + s) * T + t] = make_float2(R * Ar, R * Ai);
        }
        __syncthreads();

        // 3. B_q(t, e) += sum_s R_s A_t G_e ; per-scatterer gradients of this bin tile
        for (int i = tid; i < QB * T * N; i += kGThreads) {
            const int j = i / (T * N), r = i - j * T * N, t = r / N, e = r - t * N;
            float2 b = Bt[i];
            for (int s = 0; s < SB; ++s) {
                const float2 ra = RA[((size_t)j * SB + s) * T + t];
                const float2 a = Gt[((size_t)j * SB + s) * N + e];
                b.x = fmaf(ra.x, a.x, fmaf(-ra.y, a.y, b.x));
                b.y = fmaf(ra.x, a.y, fmaf(ra.y, a.x, b.y));
            }
            Bt[i] = b;
        }
        if (tid < 3 * SB) {       // fixed-order sum over (bin, transmit): reproducible
            const int which = tid / SB, s = tid - which * SB;
            float acc = 0.f;
            for (int j = 0; j < QB; ++j)
                for (int t = 0; t < T; ++t) acc += sg[which * nit + (j * SB + s) * T + t];
            if (sb + s < s_end)
                gpart[(size_t)which * n_qtiles * S + (size_t)qt * S + (sb + s)] = acc;
        }
    }
    __syncthreads();
    for (int i = tid; i < QB * T * N; i += kGThreads) {
        const int j = i / (T * N), r = i - j * T * N, t = r / N, e = r - t * N, k = k0 + j;
        if (k < nq) bpart[(((size_t)chunk * T + t) * nq + k) * N + e] = Bt[i];
    }
}

// g[s] = sum over bin tiles of gpart[which][qt][s] (fixed order).
__global__ void k_grad_reduce_scat(const float *__restrict__ gpart, int n_qtiles, int64_t S,
                                   float *__restrict__ g_rc, float *__restrict__ g_x,
                                   float *__restrict__ g_z) {
    const size_t pl = (size_t)n_qtiles * S;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S;
         s += (int64_t)gridDim.x * blockDim.x) {
        float a = 0.f, b = 0.f, c = 0.f;
        for (int q = 0; q < n_qtiles; ++q) {
            a += gpart[(size_t)q * S + s];
            b += gpart[pl + (size_t)q * S + s];
            c += gpart[2 * pl + (size_t)q * S + s];
        }
        if (g_rc) g_rc[s] = a;
        if (g_x) g_x[s] = b;
        if (g_z) g_z[s] = c;
    }
}

// g_delays[t][e] = Re sum_k i w_k c_te(k) sum_chunk B[chunk][t][k][e].
__global__ void k_grad_delays(const float2 *__restrict__ bpart, int n_chunks, int T, int N, int nq,
                              int q_lo, double df, const float2 *__restrict__ cw,
                              float *__restrict__ gd) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T * N) return;
    const int t = i / N, e = i - t * N;
    double acc = 0.0;
    for (int k = 0; k < nq; ++k) {
        float br = 0.f, bi = 0.f;
        for (int c = 0; c < n_chunks; ++c) {
            const float2 b = bpart[(((size_t)c * T + t) * nq + k) * N + e];
            br += b.x;
            bi += b.y;
        }
        const float2 cc = cw[((size_t)t * nq + k) * N + e];
        const double w = 6.283185307179586 * (double)(q_lo + k) * df;
        // Re(i w c B) = -w Im(c B)
        acc += -w * (double)(cc.x * bi + cc.y * br);
    }
    gd[i] = (float)acc;
}

GradGeom grad_geometry(const simus_plan *p, int T, int64_t S) {
    GradGeom g{};
    g.ok = (int64_t)T * p->N <= 2048;
    g.n_qtiles = (p->nq + kGQB - 1) / kGQB;
    int64_t want = (int64_t)p->num_sms * 4;
    int64_t chunks = std::max<int64_t>(1, (want + g.n_qtiles - 1) / g.n_qtiles);
    chunks = std::min<int64_t>(chunks, std::max<int64_t>(1, S / (kGSB * 16)));
    int64_t len = (S + chunks - 1) / chunks;
    len = ((len + kGSB - 1) / kGSB) * kGSB;
    g.chunk_len = std::max<int64_t>(len, kGSB);
    g.n_chunks = (int)((S + g.chunk_len - 1) / g.chunk_len);
    g.smem = sizeof(float4) * kGSB + sizeof(SubElem) * p->M
           + sizeof(float2) * (size_t)kGQB * T * p->N * 3
           + sizeof(float2) * (size_t)3 * kGQB * kGSB * p->N
           + sizeof(float2) * (size_t)kGQB * kGSB * T + sizeof(float) * 3 * kGQB * kGSB * T;
    g.ok = g.ok && g.smem <= 227 * 1024;
    return g;
}

int launch_adjoint_dft(const simus_plan *p, const float *drf, int T, float2 *lam, cudaStream_t st) {
    constexpr int CB = 8, JB = 256;
    const int n_chan = T * p->N;
    dim3 grid((p->nq + 255) / 256, (n_chan + CB - 1) / CB);
    k_adjoint_dft<CB, JB><<<grid, 256, 0, st>>>(drf, p->N, n_chan, p->nq, p->q_lo, p->nt, p->d_H, lam);
    count_launches(1);
    return check_cuda(cudaGetLastError(), "k_adjoint_dft launch");
}

int launch_grad(const simus_plan *p, const GradGeom &g, const simus_scat *sc, int T,
                const float2 *cw, const float2 *lam, float *gpart, float2 *bpart, cudaStream_t st) {
    auto kern = p->gc.narrow == 1 ? k_grad<true> : k_grad<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
    if (e != cudaSuccess) return check_cuda(e, "k_grad smem attribute");
    dim3 grid(g.n_qtiles, g.n_chunks);
    kern<<<grid, kGThreads, g.smem, st>>>(p->gc, p->d_sub, sc->x, sc->z, sc->rc, sc->n, g.chunk_len,
                                          T, cw, lam, gpart, g.n_qtiles, bpart);
    count_launches(1);
    return check_cuda(cudaGetLastError(), "k_grad launch");
}

int launch_grad_finish(const simus_plan *p, const GradGeom &g, int T, int64_t S, const float *gpart,
                       const float2 *bpart, const float2 *cw, float *g_rc, float *g_x, float *g_z,
                       float *g_delays, cudaStream_t st) {
    if (g_rc || g_x || g_z) {
        int blocks = (int)std::min<int64_t>((S + 255) / 256, (int64_t)p->num_sms * 8);
        k_grad_reduce_scat<<<std::max(blocks, 1), 256, 0, st>>>(gpart, g.n_qtiles, S, g_rc, g_x, g_z);
        count_launches(1);
        int rc = check_cuda(cudaGetLastError(), "k_grad_reduce_scat launch");
        if (rc) return rc;
    }
    if (g_delays) {
        const int n = T * p->N;
        k_grad_delays<<<(n + 127) / 128, 128, 0, st>>>(bpart, g.n_chunks, T, p->N, p->nq, p->q_lo,
                                                      p->gc.df, cw, g_delays);
        count_launches(1);
        return check_cuda(cudaGetLastError(), "k_grad_delays launch");
    }
    return SIMUS_OK;
}

}  // namespace simus
