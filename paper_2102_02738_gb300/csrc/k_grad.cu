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
constexpr int kGThreads = 384;  // 12 warps: the register budget of the generation allows it
constexpr int kGQB = 2;     // bins per tile
constexpr int kGSBMax = 16; // scatterers per group (16, or 8 where shared memory is short)
constexpr int kGRT = 2;     // transmits per thread in the contraction (register block)

// Threads sharing one (bin, scatterer, transmit pair) item of the contraction along the
// elements (1, 2, 4 or 8): as many as keep two items per thread or fewer.
__host__ __device__ inline int grad_ks(int SB, int T) {
    const int items = kGQB * SB * ((T + kGRT - 1) / kGRT);
    int ks = 1;
    while (ks < 8 && items * ks * 2 <= kGThreads) ks *= 2;
    return ks;
}
// Row stride (complex values) of the G, dG/dX, dG/dZ tiles: N rounded up to ks mod 16, so
// that the rows of consecutive scatterers start 2 ks words apart and the ks lanes of an item
// (elements e, e + 1, ...) and the items of the next scatterer fall in distinct banks.
__host__ __device__ inline int grad_row(int N, int ks) {
    return N + (((ks - N) % 16) + 16) % 16;
}
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

// Shared-memory rows of N complex values are padded to Nr = N + 1 (weights, adjoint
// spectra) or NrG (Green's tiles) so that rows of different transmits or scatterers start
// in different banks.  The sub-element records are held as two float4 planes indexed
// [mu][e] (centroid; normal and rotated centroid), so that the threads of a warp, which
// take consecutive elements, read consecutive 16-byte words instead of 32-byte records
// nu apart.  TAB: delta and d delta/dr from the plan's cubic pieces (staged after the other
// tiles; the derivative of the piece in its variable times dx/dr), and the phase and
// absorption of the tile's second bin from the first by one phasor step; points within
// ~2 mm of a sub-element, outside the table, take the direct four-Gaussian form.
template <bool NARROW, bool TAB>
__global__ void __launch_bounds__(kGThreads, 1)
k_grad(const GreenConst gc, const SubElem *__restrict__ sub_g, const float *__restrict__ xg,
       const float *__restrict__ zg, const float *__restrict__ rcg, int64_t S, int64_t chunk_len,
       int T, int SB, const float2 *__restrict__ cw, const float2 *__restrict__ lam,
       float *__restrict__ gpart /*[3][n_qtiles][S]*/, int n_qtiles,
       float2 *__restrict__ bpart /*[n_chunks][T][nq][N]*/, const float4 *__restrict__ dtab) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = gc.N, nu = gc.nu, M = gc.M, nq = gc.nq, Nr = N + 1;
    const int tid = threadIdx.x;
    constexpr int QB = kGQB;
    const int ks = grad_ks(SB, T);
    const int NrG = grad_row(N, ks);
    float4 *sc = reinterpret_cast<float4 *>(smem_raw);              // [SB] (x, 0, z, R)
    float4 *subA = sc + kGSBMax;                                     // [nu][N] xh, xl, zh, zl
    float4 *subB = subA + M;                                        // [nu][N] cpsi, spsi, l0, z0
    float2 *cwt = reinterpret_cast<float2 *>(subB + M);             // [QB][T][Nr]
    float2 *lat = cwt + QB * T * Nr;                                // [QB][T][Nr]
    float2 *Bt = lat + QB * T * Nr;                                 // [QB][T][N]
    float2 *Gt = Bt + QB * T * N;                                   // [3][QB][SB][NrG]
    float2 *RA = Gt + 3 * QB * SB * NrG;                            // [QB][SB][T]
    float *sg = reinterpret_cast<float *>(RA + QB * SB * T);        // [3][QB*SB*T]
    const int nit = QB * SB * T;
    float4 *tabs = reinterpret_cast<float4 *>(sg + 3 * nit);        // [2 tab_n] (TAB)

    const int qt = blockIdx.x, chunk = blockIdx.y;
    const int k0 = qt * QB;
    const int64_t s_begin = (int64_t)chunk * chunk_len;
    const int64_t s_end = min(S, s_begin + chunk_len);

    if (TAB)
        for (int i = tid; i < 2 * gc.tab_n; i += kGThreads) tabs[i] = dtab[i];
    for (int i = tid; i < M; i += kGThreads) {          // global [e][mu] -> shared [mu][e]
        const float4 *r = reinterpret_cast<const float4 *>(sub_g + i);
        const int e = i / nu, mu = i - e * nu;
        subA[mu * N + e] = r[0];
        subB[mu * N + e] = r[1];
    }
    for (int i = tid; i < QB * T * N; i += kGThreads) {
        int j = i / (T * N), r = i - j * T * N, t = r / N, e = r - t * N, k = k0 + j;
        bool ok = k < nq;
        const int o = (j * T + t) * Nr + e;
        cwt[o] = ok ? cw[((size_t)t * nq + k) * N + e] : make_float2(0.f, 0.f);
        lat[o] = ok ? lam[((size_t)t * nq + k) * N + e] : make_float2(0.f, 0.f);
        Bt[i] = make_float2(0.f, 0.f);
    }
    const float q0 = (float)(gc.q_lo + k0);
    // contraction work: (bin, scatterer, pair of transmits) items, each split over ks
    // threads along the elements when there are fewer items than threads
    const int TB = (T + kGRT - 1) / kGRT;
    const int items = QB * SB * TB;
    const int units = items * ks;
    const size_t plane = (size_t)QB * SB * NrG;

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
                SubElem se;
                reinterpret_cast<float4 *>(&se)[0] = subA[mu * N + e];
                reinterpret_cast<float4 *>(&se)[1] = subB[mu * N + e];
                const PairSetup P = pair_setup<false>(gc, se, ps.x, 0.f, ps.z, q0);
                const PairGrad Q = pair_grad(gc, se, ps.x, ps.z, P);
                if (TAB) {
                    // E = exp((i k - k_a) r) / r at q0 from the exact phase reduction, then
                    // E <- E w, w = exp(-k_a r df / c) exp(2 pi i frac(u)) (as phase_run,
                    // without the obliquity, which the derivative keeps apart)
                    const float amp0 = gc.h * P.inv_r * ex2_a(-q0 * gc.att2 * P.rh);
                    float sn, cs;
                    sincos_a(6.283185307179586f * df_frac_mul(q0, P.u), sn, cs);
                    float Er = amp0 * cs, Ei = amp0 * sn, wr = 0.f, wi = 0.f;
                    if (QB > 1) {
                        sincospif(2.0f * ((P.u.h - rintf(P.u.h)) + P.u.l), &sn, &cs);
                        wr = P.mstep * cs;
                        wi = P.mstep * sn;
                    }
                    const float kt = P.kap * gc.tab_inv_dx, t0 = gc.tab_x0 * gc.tab_inv_dx;
                    const float dxdr = gc.tab_inv_dx * gc.kh * gc.h2 * Q.rr2;   // per bin
#pragma unroll
                    for (int j = 0; j < QB; ++j) {
                        const float q = q0 + (float)j;
                        const float tt = fmaf(q, kt, -t0);
                        const float fl = floorf(fminf(fmaxf(tt, 0.0f), (float)gc.tab_n - 0.5f));
                        const int i = (int)fl;
                        const float u = tt - fl;
                        float dr_, di_, ddr, ddi;
                        if (u >= 0.0f && u <= 1.0f) {
                            const float4 lo = tabs[2 * i], hi = tabs[2 * i + 1];
                            const float2 d = cubic_piece(lo, hi, u);
                            dr_ = d.x;
                            di_ = d.y;
                            // d/du of the piece: c1 + u (2 c2 + 3 c3 u)
                            const float sc = q * dxdr;
                            ddr = fmaf(u, fmaf(3.0f * u, hi.z, 2.0f * hi.x), lo.z) * sc;
                            ddi = fmaf(u, fmaf(3.0f * u, hi.w, 2.0f * hi.y), lo.w) * sc;
                        } else {
                            delta_and_dr(gc, P, Q, q, dr_, di_, ddr, ddi);
                        }
                        float2 g, gx, gz;
                        green_grad_assemble<NARROW>(gc, P, Q, q, Er, Ei, dr_, di_, ddr, ddi, g, gx, gz);
                        G[j].x += g.x; G[j].y += g.y;
                        GX[j].x += gx.x; GX[j].y += gx.y;
                        GZ[j].x += gz.x; GZ[j].y += gz.y;
                        if (j + 1 < QB) {
                            const float nr = fmaf(Er, wr, -Ei * wi);
                            Ei = fmaf(Er, wi, Ei * wr);
                            Er = nr;
                        }
                    }
                } else {
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
            }
#pragma unroll
            for (int j = 0; j < QB; ++j) {
                const size_t o = ((size_t)j * SB + s) * NrG + e;
                Gt[o] = G[j];
                Gt[plane + o] = GX[j];
                Gt[2 * plane + o] = GZ[j];
            }
        }
        __syncthreads();

        // 2. contractions per (bin, scatterer, transmit): P = C.G, A = L.G and the same
        // with dG/dX, dG/dZ, as a register-blocked product (one scatterer, kGRT transmits)
        for (int base = 0; base < units; base += kGThreads) {
            const int w = base + tid;
            const bool act = w < units;
            const int it = act ? w / ks : 0, part = w - (w / ks) * ks;
            const int j = it / (SB * TB), r = it - j * SB * TB, s = r / TB, tb = r - s * TB;
            const int t0 = tb * kGRT;
            const float2 *g0 = Gt + ((size_t)j * SB + s) * NrG;
            const float2 *g1 = g0 + plane, *g2 = g0 + 2 * plane;
            const float2 *cr[kGRT], *lr[kGRT];
#pragma unroll
            for (int dt = 0; dt < kGRT; ++dt) {
                const int t = min(t0 + dt, T - 1);          // past T: a duplicate, discarded
                cr[dt] = cwt + ((size_t)j * T + t) * Nr;
                lr[dt] = lat + ((size_t)j * T + t) * Nr;
            }
            // acc[dt][type][0: C, 1: L][re, im]
            float acc[kGRT][3][2][2];
#pragma unroll
            for (int dt = 0; dt < kGRT; ++dt)
#pragma unroll
                for (int y = 0; y < 3; ++y)
#pragma unroll
                    for (int c = 0; c < 2; ++c) acc[dt][y][c][0] = acc[dt][y][c][1] = 0.f;
#pragma unroll 2
            for (int e = part; e < N; e += ks) {
                const float2 a[3] = {g0[e], g1[e], g2[e]};
#pragma unroll
                for (int dt = 0; dt < kGRT; ++dt) {
                    const float2 cc = cr[dt][e], ll = lr[dt][e];
#pragma unroll
                    for (int y = 0; y < 3; ++y) {
                        acc[dt][y][0][0] = fmaf(cc.x, a[y].x, fmaf(-cc.y, a[y].y, acc[dt][y][0][0]));
                        acc[dt][y][0][1] = fmaf(cc.x, a[y].y, fmaf(cc.y, a[y].x, acc[dt][y][0][1]));
                        acc[dt][y][1][0] = fmaf(ll.x, a[y].x, fmaf(-ll.y, a[y].y, acc[dt][y][1][0]));
                        acc[dt][y][1][1] = fmaf(ll.x, a[y].y, fmaf(ll.y, a[y].x, acc[dt][y][1][1]));
                    }
                }
            }
            for (int o = 1; o < ks; o <<= 1) {              // ks adjacent lanes share an item
#pragma unroll
                for (int dt = 0; dt < kGRT; ++dt)
#pragma unroll
                    for (int y = 0; y < 3; ++y)
#pragma unroll
                        for (int c = 0; c < 2; ++c) {
                            acc[dt][y][c][0] += __shfl_xor_sync(0xffffffffu, acc[dt][y][c][0], o);
                            acc[dt][y][c][1] += __shfl_xor_sync(0xffffffffu, acc[dt][y][c][1], o);
                        }
            }
            if (act && part == 0) {
                const float R = sc[s].w;
#pragma unroll
                for (int dt = 0; dt < kGRT; ++dt) {
                    const int t = t0 + dt;
                    if (t < T) {
                        const float Pr = acc[dt][0][0][0], Pi = acc[dt][0][0][1];
                        const float Ar = acc[dt][0][1][0], Ai = acc[dt][0][1][1];
                        const float Pxr = acc[dt][1][0][0], Pxi = acc[dt][1][0][1];
                        const float Axr = acc[dt][1][1][0], Axi = acc[dt][1][1][1];
                        const float Pzr = acc[dt][2][0][0], Pzi = acc[dt][2][0][1];
                        const float Azr = acc[dt][2][1][0], Azi = acc[dt][2][1][1];
                        const int o = (j * SB + s) * T + t;
                        sg[o] = Ar * Pr - Ai * Pi;                                             // dL/dR
                        sg[nit + o] = R * ((Ar * Pxr - Ai * Pxi) + (Pr * Axr - Pi * Axi));     // dL/dX
                        sg[2 * nit + o] = R * ((Ar * Pzr - Ai * Pzi) + (Pr * Azr - Pi * Azi)); // dL/dZ
                        RA[o] = make_float2(R * Ar, R * Ai);
                    }
                }
            }
        }
        __syncthreads();

        // 3. B_q(t, e) += sum_s R_s A_t G_e (four elements per thread, 32 apart, so that
        // a warp reads 32 consecutive elements of a row); per-scatterer gradients of this
        // bin tile
        const int NC = (N + 127) >> 7;                      // chunks of 128 elements
        for (int i = tid; i < QB * T * NC * 32; i += kGThreads) {
            const int l = i & 31, jt = i >> 5;
            const int jc = jt / NC, c = jt - jc * NC;
            const int j = jc / T, t = jc - j * T;
            const int e0 = c * 128 + l;
            float2 b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) b[u] = make_float2(0.f, 0.f);
            for (int s = 0; s < SB; ++s) {
                const float2 ra = RA[((size_t)j * SB + s) * T + t];
                const float2 *g = Gt + ((size_t)j * SB + s) * NrG + e0;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (e0 + 32 * u < N) {
                        const float2 a = g[32 * u];
                        b[u].x = fmaf(ra.x, a.x, fmaf(-ra.y, a.y, b[u].x));
                        b[u].y = fmaf(ra.x, a.y, fmaf(ra.y, a.x, b[u].y));
                    }
                }
            }
            float2 *bt = Bt + ((size_t)j * T + t) * N + e0;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (e0 + 32 * u < N) { bt[32 * u].x += b[u].x; bt[32 * u].y += b[u].y; }
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

// g_delays[t][e] = Re sum_k i w_k c_te(k) sum_chunk B[chunk][t][k][e].  A block takes 32
// consecutive channels (t, e) x 16 slices of the bins (k = slice, slice + 16, ...): the
// threads of a warp read 32 consecutive elements of one (chunk, t, k) row, and the slices'
// FP64 partial sums are added in a fixed order (reproducible).
constexpr int kGdCh = 32, kGdSl = 16;
__global__ void __launch_bounds__(kGdCh * kGdSl)
k_grad_delays(const float2 *__restrict__ bpart, int n_chunks, int T, int N, int nq, int q_lo,
              double df, const float2 *__restrict__ cw, float *__restrict__ gd) {
    __shared__ double part[kGdSl][kGdCh];
    const int l = threadIdx.x % kGdCh, sl = threadIdx.x / kGdCh;
    const int i = blockIdx.x * kGdCh + l;
    double acc = 0.0;
    if (i < T * N) {
        const int t = i / N, e = i - t * N;
        for (int k = sl; k < nq; k += kGdSl) {
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
    }
    part[sl][l] = acc;
    __syncthreads();
    if (sl == 0 && i < T * N) {
        double a = 0.0;
        for (int j = 0; j < kGdSl; ++j) a += part[j][l];
        gd[i] = (float)a;
    }
}

GradGeom grad_geometry(const simus_plan *p, int T, int64_t S) {
    GradGeom g{};
    g.ok = (int64_t)T * p->N <= 2048;
    g.n_qtiles = (p->nq + kGQB - 1) / kGQB;
    const size_t Nr = (size_t)p->N + 1;
    const int tab_full = (p->d_dtab && p->delta_table && !p->probe.two_d) ? p->gc.tab_n : 0;
    auto smem_for = [&](int SB, int tab_n) {
        return sizeof(float4) * kGSBMax + sizeof(SubElem) * p->M
             + sizeof(float2) * (size_t)kGQB * T * Nr * 2 + sizeof(float2) * (size_t)kGQB * T * p->N
             + sizeof(float2) * (size_t)3 * kGQB * SB * grad_row(p->N, grad_ks(SB, T))
             + sizeof(float2) * (size_t)kGQB * SB * T + sizeof(float) * 3 * kGQB * SB * T
             + 2 * sizeof(float4) * (size_t)tab_n;
    };
    // 16-scatterer groups with the delta table, else without it, else 8-scatterer groups
    const size_t lim = 227 * 1024;
    g.tab = tab_full > 0 && smem_for(kGSBMax, tab_full) <= lim;
    g.SB = (g.tab || smem_for(kGSBMax, 0) <= lim) ? kGSBMax : 8;
    if (g.SB == 8) g.tab = tab_full > 0 && smem_for(8, tab_full) <= lim;
    const int tab_n = g.tab ? tab_full : 0;
    int64_t want = (int64_t)p->num_sms * 8;
    int64_t chunks = std::max<int64_t>(1, (want + g.n_qtiles - 1) / g.n_qtiles);
    chunks = std::min<int64_t>(chunks, std::max<int64_t>(1, S / (g.SB * 16)));
    int64_t len = (S + chunks - 1) / chunks;
    len = ((len + g.SB - 1) / g.SB) * g.SB;
    g.chunk_len = std::max<int64_t>(len, g.SB);
    g.n_chunks = (int)((S + g.chunk_len - 1) / g.chunk_len);
    g.smem = smem_for(g.SB, tab_n);
    g.ok = g.ok && g.smem <= lim;
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
    auto kern = p->gc.narrow == 1 ? (g.tab ? k_grad<true, true> : k_grad<true, false>)
                                  : (g.tab ? k_grad<false, true> : k_grad<false, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
    if (e != cudaSuccess) return check_cuda(e, "k_grad smem attribute");
    dim3 grid(g.n_qtiles, g.n_chunks);
    kern<<<grid, kGThreads, g.smem, st>>>(p->gc, p->d_sub, sc->x, sc->z, sc->rc, sc->n, g.chunk_len,
                                          T, g.SB, cw, lam, gpart, g.n_qtiles, bpart, p->d_dtab);
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
        k_grad_delays<<<(n + kGdCh - 1) / kGdCh, kGdCh * kGdSl, 0, st>>>(bpart, g.n_chunks, T, p->N, p->nq,
                                                                       p->q_lo, p->gc.df, cw, g_delays);
        count_launches(1);
        return check_cuda(cudaGetLastError(), "k_grad_delays launch");
    }
    return SIMUS_OK;
}

}  // namespace simus
