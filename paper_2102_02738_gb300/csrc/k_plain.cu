// k_plain.cu -- plain FP32 path: Green's terms (Eq. 17/20/39/40), transmit sum (Eq. 29)
// and receive sum over scatterers (Eq. 30-33) on the CUDA cores, one transmit per
// grid z-slice (Green's terms recomputed for every transmit).
//
// Block tile: QB consecutive kept bins x one chunk of scatterers x all N elements.
// For each group of SB scatterers the block
//   1. generates G_e(q, s, e) = sum_mu g(q, s, (e, mu)) for the QB x SB x N tile into
//      shared memory (thread per (s, e) pair; the per-pair geometry is amortised over
//      the QB bins),
//   2. forms P(q, s) = sum_e C(q, e) G_e(q, s, e) (warp per (q, s), shuffle reduction),
//      scaled by R_s,
//   3. accumulates RF_q(e) += sum_s G_e(q, s, e) R_s P(q, s) in shared memory.
// The chunk's partial spectrum is written to part[chunk][t][e][k]; chunks are summed
// in a fixed order by the reduction kernel, so results are bitwise reproducible.
#include <algorithm>

#include "green.cuh"
#include "simus_internal.h"

namespace simus {

static constexpr int kPlainThreads = 256;
// Bins per block tile.  With the elevation factor (3-D model) 8 bins, three blocks per SM:
// occupancy hides the latency of the per-bin δ-table loads (planewave-linear-128 17.5 ->
// 17.0 ms against 16 bins at two blocks); without it (2-D model) 16 bins, two blocks per
// SM, which amortise the geometry setup over more of the cheaper bins (11.4 against 12.1 ms).
static constexpr int kPlainQB3D = 8;
static constexpr int kPlainQB2D = 16;

// C[t][k][e] = W_te exp(i 2 pi frac(q df dtau_te)), q = q_lo + k, reduced in FP64.
__global__ void k_tx_weights(int T, int N, int nq, int q_lo, double df,
                             const float *__restrict__ delays, const float *__restrict__ apod,
                             float2 *__restrict__ cw) {
    int64_t total = (int64_t)T * nq * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int e = (int)(i % N);
        int64_t r = i / N;
        int k = (int)(r % nq);
        int t = (int)(r / nq);
        double v = (double)delays[t * N + e] * df;        // cycles per bin
        double ph = (double)(q_lo + k) * v;
        ph -= rint(ph);
        float s, c;
        sincospif((float)(2.0 * ph), &s, &c);
        float w = apod[t * N + e];
        cw[i] = make_float2(w * c, w * s);
    }
}

int launch_tx_weights(const simus_plan *p, const simus_tx *tx, float2 *cw, cudaStream_t st) {
    int64_t total = (int64_t)tx->n_tx * p->nq * p->N;
    int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)p->num_sms * 8);
    k_tx_weights<<<blocks, 256, 0, st>>>(tx->n_tx, p->N, p->nq, p->q_lo, p->gc.df, tx->delays,
                                         tx->apod, cw);
    count_launches(1);
    return check_cuda(cudaGetLastError(), "k_tx_weights launch");
}

// TAB: delta/h at Y = 0 from the plan's table of cubic pieces (read through the read-only
// cache; relative error <= 2.3e-6), evaluated directly outside the table.
template <int QB, bool HAS_Y, bool NARROW, bool TAB>
__global__ void __launch_bounds__(kPlainThreads, QB <= 8 ? 3 : 2)
k_plain_rf(const GreenConst gc, const SubElem *__restrict__ sub_g, const float *__restrict__ xg,
           const float *__restrict__ yg, const float *__restrict__ zg,
           const float *__restrict__ rcg, int64_t S, int64_t chunk_len, int SB, int T,
           const float2 *__restrict__ cw, float2 *__restrict__ part,
           const float4 *__restrict__ dtab) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = gc.N, nu = gc.nu, M = gc.M, nq = gc.nq;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float4 *sc = reinterpret_cast<float4 *>(smem_raw);             // [SB] (x, y, z, R)
    float4 *subA = sc + SB;                                        // [nu][N] xh, xl, zh, zl
    float4 *subB = subA + M;                                       // [nu][N] cpsi, spsi, l0, z0
    float2 *cwt = reinterpret_cast<float2 *>(subB + M);            // [QB][N]
    float2 *acc = cwt + QB * N;                                    // [QB][N]
    float2 *RP = acc + QB * N;                                     // [QB][SB]
    float2 *Gt = RP + QB * SB;                                     // [QB][SB][N]

    const int k0 = blockIdx.x * QB;
    const int chunk = blockIdx.y, t = blockIdx.z;
    const int64_t s_begin = (int64_t)chunk * chunk_len;
    const int64_t s_end = min(S, s_begin + chunk_len);

    for (int i = tid; i < M; i += kPlainThreads) {      // global [e][mu] -> shared [mu][e]
        const float4 *rec = reinterpret_cast<const float4 *>(sub_g + i);
        const int e = i / nu, mu = i - e * nu;
        subA[mu * N + e] = rec[0];
        subB[mu * N + e] = rec[1];
    }
    for (int i = tid; i < QB * N; i += kPlainThreads) {
        int j = i / N, e = i - j * N, k = k0 + j;
        cwt[i] = k < nq ? cw[((size_t)t * nq + k) * N + e] : make_float2(0.f, 0.f);
        acc[i] = make_float2(0.f, 0.f);
    }
    const float q0 = (float)(gc.q_lo + k0);

    for (int64_t sb = s_begin; sb < s_end; sb += SB) {
        __syncthreads();  // previous group done with sc, RP, Gt
        if (tid < SB) {
            int64_t s = sb + tid;
            sc[tid] = s < s_end ? make_float4(xg[s], HAS_Y ? yg[s] : 0.f, zg[s], rcg[s])
                                : make_float4(0.f, 0.f, 1.f, 0.f);   // padding: R = 0
        }
        __syncthreads();

        // 1. Green's tile
        for (int pr = tid; pr < SB * N; pr += kPlainThreads) {
            int s = pr / N, e = pr - s * N;
            float4 ps = sc[s];
            float2 G[QB];
#pragma unroll
            for (int j = 0; j < QB; ++j) G[j] = make_float2(0.f, 0.f);
            for (int mu = 0; mu < nu; ++mu) {
                SubElem se;
                reinterpret_cast<float4 *>(&se)[0] = subA[mu * N + e];
                reinterpret_cast<float4 *>(&se)[1] = subB[mu * N + e];
                PairSetup P = pair_setup<HAS_Y>(gc, se, ps.x, ps.y, ps.z, q0);
                PhaseRun R = phase_run(P, q0);
                const float kt = TAB ? P.kap * gc.tab_inv_dx : 0.0f;
                const float t0 = TAB ? gc.tab_x0 * gc.tab_inv_dx : 0.0f;
#pragma unroll
                for (int j = 0; j < QB; ++j) {
                    const float q = q0 + (float)j;
                    const float m = sinc_f<NARROW>(q * P.xb);
                    float2 d;
                    if (TAB) {
                        const float tt = fmaf(q, kt, -t0);
                        const float fl = floorf(fminf(fmaxf(tt, 0.0f), (float)gc.tab_n - 0.5f));
                        const int i = (int)fl;
                        const float u = tt - fl;
                        d = cubic_piece(__ldg(dtab + 2 * i), __ldg(dtab + 2 * i + 1), u);
                        if (!(u >= 0.0f && u <= 1.0f)) d = delta_f<false>(gc, P, q);   // r < ~2 mm
                    } else {
                        d = delta_f<HAS_Y>(gc, P, q);
                    }
                    const float er = R.zr * m, ei = R.zi * m;
                    G[j].x = fmaf(er, d.x, fmaf(-ei, d.y, G[j].x));
                    G[j].y = fmaf(er, d.y, fmaf(ei, d.x, G[j].y));
                    const float nzr = fmaf(R.zr, R.wr, -R.zi * R.wi);
                    R.zi = fmaf(R.zr, R.wi, R.zi * R.wr);
                    R.zr = nzr;
                }
            }
#pragma unroll
            for (int j = 0; j < QB; ++j) Gt[(j * SB + s) * N + e] = G[j];
        }
        __syncthreads();

        // 2. transmit sum (Eq. 29) times R_s
        for (int pi = warp; pi < QB * SB; pi += kPlainThreads / 32) {
            int j = pi / SB, s = pi - j * SB;
            const float2 *g = Gt + (j * SB + s) * N;
            const float2 *c = cwt + j * N;
            float pr = 0.f, pim = 0.f;
            for (int e = lane; e < N; e += 32) {
                float2 cc = c[e], gg = g[e];
                pr = fmaf(cc.x, gg.x, fmaf(-cc.y, gg.y, pr));
                pim = fmaf(cc.x, gg.y, fmaf(cc.y, gg.x, pim));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                pr += __shfl_xor_sync(0xffffffffu, pr, o);
                pim += __shfl_xor_sync(0xffffffffu, pim, o);
            }
            if (lane == 0) {
                float R = sc[s].w;
                RP[pi] = make_float2(R * pr, R * pim);
            }
        }
        __syncthreads();

        // 3. receive sum over the group's scatterers (Eq. 30-33)
        for (int i = tid; i < QB * N; i += kPlainThreads) {
            int j = i / N, e = i - j * N;
            float2 a = acc[i];
            for (int s = 0; s < SB; ++s) {
                float2 gg = Gt[(j * SB + s) * N + e], rp = RP[j * SB + s];
                a.x = fmaf(gg.x, rp.x, fmaf(-gg.y, rp.y, a.x));
                a.y = fmaf(gg.x, rp.y, fmaf(gg.y, rp.x, a.y));
            }
            acc[i] = a;
        }
    }
    __syncthreads();
    for (int i = tid; i < QB * N; i += kPlainThreads) {
        int e = i / QB, j = i - e * QB, k = k0 + j;
        if (k < nq) part[(((size_t)chunk * T + t) * N + e) * nq + k] = acc[j * N + e];
    }
}

static size_t plain_smem(const simus_plan *p, int QB, int SB) {
    return sizeof(float4) * SB + sizeof(SubElem) * p->M + sizeof(float2) * (size_t)QB * p->N * 2
         + sizeof(float2) * (size_t)QB * SB + sizeof(float2) * (size_t)QB * SB * p->N;
}

PlainGeom plain_geometry(const simus_plan *p, int T, int64_t S) {
    PlainGeom g{};
    g.QB = p->gc.two_d ? kPlainQB2D : kPlainQB3D;
    const int per_sm = g.QB <= 8 ? 3 : 2;     // resident blocks per SM (launch bounds)
    // scatterers per group: G tile within 64 KB, pairs a multiple of the block if possible
    int sb_max = std::max(1, 8192 / (g.QB * p->N));
    int SB = sb_max;
    for (int s = 1; s <= sb_max; ++s)
        if ((s * p->N) % kPlainThreads == 0) { SB = s; break; }
    g.SB = std::min(SB, 8);
    g.n_qtiles = (p->nq + g.QB - 1) / g.QB;
    // enough blocks for ~8 waves of resident blocks, chunks of at least 4 groups (a few
    // hundred scatterers then still fill the GPU: 0.113 -> 0.089 ms for 200 scatterers
    // at 64 elements, against 8 groups)
    int64_t want = (int64_t)p->num_sms * per_sm * 8;
    int64_t per_tx = std::max<int64_t>(1, want / std::max<int64_t>(1, (int64_t)g.n_qtiles * T));
    int64_t min_chunk = (int64_t)g.SB * 4;
    int64_t chunks = std::max<int64_t>(1, std::min<int64_t>(per_tx, (S + min_chunk - 1) / min_chunk));
    int64_t len = (S + chunks - 1) / chunks;
    len = ((len + g.SB - 1) / g.SB) * g.SB;
    g.chunk_len = std::max<int64_t>(len, g.SB);
    g.n_chunks = (int)((S + g.chunk_len - 1) / g.chunk_len);
    if (g.n_chunks < 1) g.n_chunks = 1;
    g.smem = plain_smem(p, g.QB, g.SB);
    return g;
}

using PlainKernel = void (*)(const GreenConst, const SubElem *, const float *, const float *,
                             const float *, const float *, int64_t, int64_t, int, int,
                             const float2 *, float2 *, const float4 *);

template <int QB>
static PlainKernel plain_kernel(bool has_y, bool narrow, bool tab) {
    return has_y ? (narrow ? k_plain_rf<QB, true, true, false> : k_plain_rf<QB, true, false, false>)
         : tab   ? (narrow ? k_plain_rf<QB, false, true, true> : k_plain_rf<QB, false, false, true>)
                 : (narrow ? k_plain_rf<QB, false, true, false> : k_plain_rf<QB, false, false, false>);
}

int launch_plain(const simus_plan *p, const PlainGeom &g, const simus_scat *sc, int T,
                 const float2 *cw, float2 *part, cudaStream_t st) {
    dim3 grid(g.n_qtiles, g.n_chunks, T);
    const bool has_y = sc->y != nullptr, narrow = p->gc.narrow == 1;
    const bool tab = !has_y && p->d_dtab && p->gc.tab_n > 0 && p->delta_table;
    if (g.QB != kPlainQB3D && g.QB != kPlainQB2D) return fail(SIMUS_ERR_ARG, "plain tile of %d bins", g.QB);
    const PlainKernel kern = g.QB == kPlainQB3D ? plain_kernel<kPlainQB3D>(has_y, narrow, tab)
                                                : plain_kernel<kPlainQB2D>(has_y, narrow, tab);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)g.smem);
    if (e != cudaSuccess) return check_cuda(e, "k_plain_rf smem attribute");
    kern<<<grid, kPlainThreads, g.smem, st>>>(p->gc, p->d_sub, sc->x, sc->y, sc->z, sc->rc, sc->n,
                                               g.chunk_len, g.SB, T, cw, part, p->d_dtab);
    count_launches(1);
    return check_cuda(cudaGetLastError(), "k_plain_rf launch");
}

}  // namespace simus
