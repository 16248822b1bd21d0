// k_tc.cu -- batched path on the tcgen05 tensor cores: one persistent launch over the
// work items of any number of simulations.
//
// The Green's tile G_e(q, s, e) of a bin q and a tile of 128 scatterers is generated once
// in FP32 (Eq. 17/20/39/40, sub-element sum of Eq. 33), rounded to FP16 (or BF16) in
// shared memory, and feeds two complex contractions written as real GEMMs:
//
//   transmit sum (Eq. 29)   P[s][t]  = sum_e G[s][e] C_q[t][e]
//       A  = [Re G | Im G]                      128 x 2Np   (rows s, K over e), K-major
//       B1 rows 2t   = [ Re C_t | -Im C_t ]     nN x 2Np    (per bin, TMA bulk copy)
//       B1 rows 2t+1 = [ Im C_t |  Re C_t ]
//       D1 columns (2t, 2t+1) = (Re P, Im P)    FP32 in tensor memory
//   reflection + receive sum (Eq. 30-32)   RF_q[e][t] += sum_s G[s][e] R_s P[s][t]
//       A^T read from the same tile as an MN-major operand: M = e (in halves of 128 when
//       Np > 128), K = (s | s) over the Re G and Im G halves -- no transposed copy
//       B2 rows 2t   = [ Re P' | -Im P' ],  rows 2t+1 = [ Im P' | Re P' ],  P' = R_s P,
//       stored MN-major so that one thread's transmits are contiguous
//       D2[bin][half] columns (2t, 2t+1) = (Re RF, Im RF), accumulated over every
//       scatterer tile of the work item in tensor memory.
//
// Work: a unit is one (simulation, transmit group); a work item is QB bins x a chunk of
// scatterer tiles of one unit.  One CTA per SM (512 threads) takes items from a global
// counter until none are left.  With two tile buffers ("pair"), bins are generated two at
// a time so that the per-(scatterer, sub-element) geometry -- double-float distance and
// phase rate -- is shared by both.  Per bin: MMA1 -> read P from tensor memory, scale by
// R_s, write B2 -> MMA2.  All waits are bounded; on a timeout the CTA records an error
// code, waits for its own bulk copy, frees its tensor memory and returns.
#include <algorithm>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "green.cuh"
#include "simus_internal.h"
#include "tcgen05.cuh"

namespace simus {

namespace {
constexpr int kThreads = 512;
constexpr int kSB = 128;          // scatterers per tile
constexpr int kMaxWait = 1 << 22; // polls before a wait is declared timed out
constexpr size_t kHeader = 128;   // mbarriers, tensor-memory slot, flags, item index

template <bool BF16>
__device__ __forceinline__ uint16_t h16(float v) {
    if (BF16) return __bfloat16_as_ushort(__float2bfloat16_rn(v));
    return __half_as_ushort(__float2half_rn(v));
}
template <bool BF16>
__device__ __forceinline__ uint32_t h16x2(float lo, float hi) {
    return (uint32_t)h16<BF16>(lo) | ((uint32_t)h16<BF16>(hi) << 16);
}

// delta / h from the table of cubic pieces: interval i holds c0..c3 (complex) of
// c0 + c1 u + c2 u^2 + c3 u^3, u = t - i, t = (x - x0) / dx (two float4 per interval).
__device__ __forceinline__ float2 cubic_piece(const float4 &lo, const float4 &hi, float u) {
    return make_float2(fmaf(u, fmaf(u, fmaf(u, hi.z, hi.x), lo.z), lo.x),
                       fmaf(u, fmaf(u, fmaf(u, hi.w, hi.y), lo.w), lo.y));
}

// Sub-element sums (Eq. 33) of the Green's terms of elements e0 and e0 + 1 for one
// scatterer at the NB consecutive bins qA, qA + 1, ...: two independent evaluation chains
// side by side, so that each warp has twice the instruction-level parallelism, and one
// geometry setup per (scatterer, sub-element) for all NB bins.  An element past N is
// evaluated on element N - 1 with zero amplitude (no branch).  With the delta table, bin
// qA picks the cubic piece and the later bins reuse it: bin qA + b moves u by b kap/dx,
// small except within a few mm of the sub-element, where (|u| check) delta is evaluated
// directly instead.  o[c][b] = (Re, Im) of element e0 + c at bin qA + b.
template <int NB, bool TAB, bool HAS_Y, bool NARROW, bool LINEAR>
__device__ __forceinline__ void gen_two(const GreenConst &gc, const SubElem *sub,
                                        const float4 *tabs, const float4 &ps, int e0, float qA,
                                        float (&o)[2][NB][2]) {
    const int N = gc.N, nu = gc.nu;
    const float w0 = e0 < N ? 1.0f : 0.0f, w1 = e0 + 1 < N ? 1.0f : 0.0f;
    const int b0 = min(e0, N - 1) * nu, b1 = min(e0 + 1, N - 1) * nu;
    const float t0 = gc.tab_x0 * gc.tab_inv_dx, tmax = (float)gc.tab_n - 0.5f;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < NB; ++b) o[c][b][0] = o[c][b][1] = 0.0f;
    for (int mu = 0; mu < nu; ++mu) {
        PairSetup P[2];
        P[0] = pair_setup_f32<HAS_Y, LINEAR>(gc, sub[b0 + mu], ps.x, ps.y, ps.z, qA);
        P[1] = pair_setup_f32<HAS_Y, LINEAR>(gc, sub[b1 + mu], ps.x, ps.y, ps.z, qA);
        P[0].amp0 *= w0;
        P[1].amp0 *= w1;
        float kt[2] = {0.0f, 0.0f}, u[2] = {0.0f, 0.0f};
        int ti[2] = {0, 0};
        bool ok = TAB;
        if (TAB) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                kt[c] = P[c].kap * gc.tab_inv_dx;
                const float t = fmaf(qA, kt[c], -t0);
                const float fl = floorf(fminf(fmaxf(t, 0.0f), tmax));
                ti[c] = (int)fl;
                u[c] = t - fl;
                const float ue = fmaf((float)(NB - 1), kt[c], u[c]);
                ok = ok && u[c] >= 0.0f && u[c] <= 1.0f && ue >= -0.25f && ue <= 1.25f;
            }
        }
        float4 lo[2], hi[2];            // the pieces (index clamped: always a valid load)
        if (TAB) {
#pragma unroll
            for (int c = 0; c < 2; ++c) { lo[c] = tabs[2 * ti[c]]; hi[c] = tabs[2 * ti[c] + 1]; }
        }
        // phase, absorption and sinc directivity of every bin (common to both delta forms)
        float er[2][NB], ei[2][NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const float q = qA + (float)b;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const float fr = df_frac_mul(q, P[c].u);
                float sn, cs;
                sincos_a(6.283185307179586f * fr, sn, cs);
                float amp = P[c].amp0;
                if (b >= 1) amp *= P[c].mstep;
                if (b >= 2) amp *= P[c].mstep;
                const float m = amp * sinc_f<NARROW>(q * P[c].xb);
                er[c][b] = cs * m;
                ei[c][b] = sn * m;
            }
        }
        float2 d[2][NB];
        if (TAB) {
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int b = 0; b < NB; ++b) d[c][b] = cubic_piece(lo[c], hi[c], fmaf((float)b, kt[c], u[c]));
        }
        if (!ok) {
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int b = 0; b < NB; ++b) d[c][b] = delta_f<HAS_Y>(gc, P[c], qA + (float)b);
        }
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                o[c][b][0] += er[c][b] * d[c][b].x - ei[c][b] * d[c][b].y;
                o[c][b][1] += er[c][b] * d[c][b].y + ei[c][b] * d[c][b].x;
            }
    }
}

// One generation pass over a scatterer tile: every (scatterer, group of 8 elements) item
// at bins qA .. qA + NB - 1, written as FP16/BF16 rows of the K-major tiles A0 (bin qA)
// and A1 (bin qA + 1); a third bin goes to tensor memory (its row s in lane s, Re of the
// 8 elements packed in columns st + 4 eg .. + 3, Im at st + Np/2 + 4 eg) until A0 is free.
// The lane rule holds by construction: item it has s = it mod 128 = 32 (warp mod 4) + lane.
template <int NB, bool TAB, bool HAS_Y, bool BF16, bool NARROW, bool LINEAR>
__device__ __forceinline__ void gen_tiles(const GreenConst &gc, const SubElem *sub,
                                          const float4 *tabs, const float4 *sc, int Np,
                                          float qA, unsigned char *A0, unsigned char *A1,
                                          uint32_t stash, int tid) {
    const int K1 = 2 * Np;
    const int n_groups = Np >> 3;
    for (int it = tid; it < kSB * n_groups; it += kThreads) {
        const int s = it & (kSB - 1), eg = it >> 7;
        const float4 ps = sc[s];
        uint32_t pk[NB][2][4];
#pragma unroll
        for (int jp = 0; jp < 4; ++jp) {
            float o[2][NB][2];
            gen_two<NB, TAB, HAS_Y, NARROW, LINEAR>(gc, sub, tabs, ps, eg * 8 + 2 * jp, qA, o);
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                pk[b][0][jp] = h16x2<BF16>(o[0][b][0], o[1][b][0]);
                pk[b][1][jp] = h16x2<BF16>(o[0][b][1], o[1][b][1]);
            }
        }
        *reinterpret_cast<uint4 *>(A0 + tc::kmajor_offset(s, eg * 8, K1)) =
            make_uint4(pk[0][0][0], pk[0][0][1], pk[0][0][2], pk[0][0][3]);
        *reinterpret_cast<uint4 *>(A0 + tc::kmajor_offset(s, Np + eg * 8, K1)) =
            make_uint4(pk[0][1][0], pk[0][1][1], pk[0][1][2], pk[0][1][3]);
        if (NB >= 2) {
            *reinterpret_cast<uint4 *>(A1 + tc::kmajor_offset(s, eg * 8, K1)) =
                make_uint4(pk[NB > 1][0][0], pk[NB > 1][0][1], pk[NB > 1][0][2], pk[NB > 1][0][3]);
            *reinterpret_cast<uint4 *>(A1 + tc::kmajor_offset(s, Np + eg * 8, K1)) =
                make_uint4(pk[NB > 1][1][0], pk[NB > 1][1][1], pk[NB > 1][1][2], pk[NB > 1][1][3]);
        }
        if (NB == 3) {
            const uint32_t ta = stash + ((uint32_t)(s & ~31) << 16) + 4u * eg;
            tc::tmem_st4(ta, pk[NB - 1][0][0], pk[NB - 1][0][1], pk[NB - 1][0][2], pk[NB - 1][0][3]);
            tc::tmem_st4(ta + (uint32_t)(Np >> 1), pk[NB - 1][1][0], pk[NB - 1][1][1], pk[NB - 1][1][2],
                         pk[NB - 1][1][3]);
        }
    }
    if (NB == 3) tc::tmem_wait_st();
}

// Move the stashed third bin from tensor memory into tile buffer A (same item-to-thread
// map as gen_tiles, so every thread reads back the lanes and columns it wrote).
__device__ __forceinline__ void unstash_tile(int Np, unsigned char *A, uint32_t stash, int tid) {
    const int K1 = 2 * Np;
    const int n_groups = Np >> 3;
    for (int it = tid; it < kSB * n_groups; it += kThreads) {
        const int s = it & (kSB - 1), eg = it >> 7;
        const uint32_t ta = stash + ((uint32_t)(s & ~31) << 16) + 4u * eg;
        uint32_t re[4], im[4];
        tc::tmem_ld4(ta, re);
        tc::tmem_ld4(ta + (uint32_t)(Np >> 1), im);
        tc::tmem_wait_ld();
        *reinterpret_cast<uint4 *>(A + tc::kmajor_offset(s, eg * 8, K1)) = make_uint4(re[0], re[1], re[2], re[3]);
        *reinterpret_cast<uint4 *>(A + tc::kmajor_offset(s, Np + eg * 8, K1)) = make_uint4(im[0], im[1], im[2], im[3]);
    }
}

// shared memory a unit needs after the header
size_t unit_smem(int Np, int nN, int pair, int M, int tab_n) {
    const size_t a = (size_t)kSB * 2 * Np * 2;
    return (pair ? 2 : 1) * a + (size_t)nN * 2 * Np * 2 + (size_t)nN * 256 * 2
         + sizeof(float4) * kSB + sizeof(SubElem) * M + 2 * sizeof(float4) * tab_n;
}
}  // namespace

// B1 images of one simulation: per kept bin and transmit group g, the nN x 2Np K-major
// operand of the transmit GEMM for transmits g TG .. g TG + TG - 1 (image [k][g]),
//   row 2t: (Re C, -Im C), row 2t+1: (Im C, Re C), C = W exp(i 2 pi frac(q df dtau)).
template <bool BF16>
__global__ void k_tc_weights(int T, int G, int TG, int N, int Np, int nN, int nq, int q_lo,
                             double df, const float *__restrict__ delays,
                             const float *__restrict__ apod, uint16_t *__restrict__ img) {
    const int K = 2 * Np;
    const int64_t per_img = (int64_t)nN * K;
    const int64_t total = per_img * G * nq;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t kg = i / per_img;
        int k = (int)(kg / G), g = (int)(kg % G);
        int r = (int)(i % per_img);
        int n = r / K, kk = r % K;
        int tl = n >> 1;
        int t = g * TG + tl;
        int e = kk < Np ? kk : kk - Np;
        float v = 0.f;
        if (tl < TG && t < T && e < N) {
            double ph = (double)(q_lo + k) * ((double)delays[t * N + e] * df);
            ph -= rint(ph);
            float s, c;
            sincospif((float)(2.0 * ph), &s, &c);
            float w = apod[t * N + e];
            float cr = w * c, ci = w * s;
            bool first_half = kk < Np;
            v = (n & 1) ? (first_half ? ci : cr) : (first_half ? cr : -ci);
        }
        img[(size_t)kg * per_img + tc::kmajor_offset(n, kk, K) / 2] = h16<BF16>(v);
    }
}

template <bool HAS_Y, bool BF16, bool NARROW, bool LINEAR>
__global__ void __launch_bounds__(kThreads, 1)
k_tc_rf(const TcUnit *__restrict__ units, int n_units, int64_t n_items, int *counter, int *err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    __shared__ TcUnit U;                  // the current item's unit

    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);          // 3 mbarriers
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + 24);
    int *abort_flag = reinterpret_cast<int *>(smem + 28);
    long long *s_item = reinterpret_cast<long long *>(smem + 32);
    int *s_unit = reinterpret_cast<int *>(smem + 40);
    unsigned char *dyn = smem + kHeader;
    const uint32_t mbar_b1 = tc::smem_u32(&bars[0]);
    const uint32_t mbar1 = tc::smem_u32(&bars[1]);
    const uint32_t mbar2 = tc::smem_u32(&bars[2]);

    if (tid == 0) {
        tc::mbar_init(mbar_b1, 1);
        tc::mbar_init(mbar1, 1);
        tc::mbar_init(mbar2, 1);
        tc::fence_mbar_init();
        *abort_flag = 0;
        *s_unit = -1;
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(tslot), 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;

    uint32_t ph_b1 = 0, ph1 = 0, ph2 = 0;
    bool pending2 = false;     // an MMA2 commit not yet waited for
    bool aborted = false;
    bool b1_inflight = false;  // thread 0: a bulk copy into B1 not yet waited for
    int cur_unit = -1;

    auto wait_all = [&](uint32_t mbar, uint32_t parity) -> bool {
        if (!tc::mbar_wait_bounded(mbar, parity, kMaxWait)) atomicExch(abort_flag, 1);
        __syncthreads();
        return *abort_flag == 0;
    };

    while (!aborted) {
        // ---- next work item (dynamic: heavier units come first in the item order)
        if (tid == 0) {
            long long it = atomicAdd(counter, 1);
            *s_item = it;
            if (it < n_items) {
                int lo = 0, hi = n_units - 1;     // last unit with item0 <= it
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (units[mid].item0 <= it) lo = mid; else hi = mid - 1;
                }
                *s_unit = lo;
            }
        }
        __syncthreads();
        const long long item = *s_item;
        if (item >= n_items) break;
        const int ui = *s_unit;
        if (ui != cur_unit) {
            if (pending2) {   // the previous unit's MMA2 may still read the tile buffers
                if (!wait_all(mbar2, ph2)) { aborted = true; break; }
                ph2 ^= 1;
                pending2 = false;
            }
            const int nw = (int)(sizeof(TcUnit) / 4);
            for (int i = tid; i < nw; i += kThreads)
                reinterpret_cast<int *>(&U)[i] = reinterpret_cast<const int *>(&units[ui])[i];
            __syncthreads();
        }
        const GreenConst gc = U.gc;   // register copy: the per-pair setup reads it often
        const int N = gc.N, nu = gc.nu, M = gc.M, nq = gc.nq;
        const int Np = U.Np, nN = U.nN, TG = U.TG, QB = U.QB, mh = U.mh, pair = U.pair;
        const int G = U.G, T = U.T;
        const int K1 = 2 * Np;
        const size_t abytes = (size_t)kSB * K1 * 2;
        unsigned char *A0 = dyn;
        unsigned char *A1 = A0 + (pair ? abytes : 0);
        unsigned char *B1 = A0 + (pair ? 2 : 1) * abytes;
        unsigned char *B2 = B1 + (size_t)nN * K1 * 2;
        float4 *sc = reinterpret_cast<float4 *>(B2 + (size_t)nN * 256 * 2);
        SubElem *sub = reinterpret_cast<SubElem *>(sc + kSB);
        float4 *tabs = reinterpret_cast<float4 *>(sub + M);               // delta table
        const bool use_tab = !HAS_Y && gc.tab_n > 0;
        const uint32_t abuf0 = tc::smem_u32(A0), abuf1 = tc::smem_u32(A1);
        const uint32_t b1s = tc::smem_u32(B1), b2s = tc::smem_u32(B2);
        const uint32_t idesc1 = tc::idesc_f16(128, nN, BF16);
        const uint32_t idesc2 = idesc1 | (1u << 15) | (1u << 16);   // A and B MN-major
        const uint32_t b1_bytes = (uint32_t)nN * K1 * 2;
        if (ui != cur_unit) {
            for (int i = tid; i < M; i += kThreads) sub[i] = U.sub[i];
            if (use_tab)
                for (int i = tid; i < 2 * gc.tab_n; i += kThreads) tabs[i] = U.dtab[i];
            cur_unit = ui;
            __syncthreads();
        }
        auto issue_b1 = [&](int k, int g) {   // weights of bin k, transmit group g
            if (tid == 0) {
                tc::mbar_arrive_expect_tx(mbar_b1, b1_bytes);
                tc::bulk_g2s(b1s, U.b1img + ((size_t)k * G + g) * nN * K1, b1_bytes, mbar_b1);
                b1_inflight = true;
            }
        };

        const int64_t li = item - U.item0;
        const int bt = (int)(li % U.n_btiles), chunk = (int)(li / U.n_btiles);
        const int k0 = bt * QB;
        const int64_t tile0 = (int64_t)chunk * U.tiles_per_chunk;
        const int64_t tile1 = std::min<int64_t>(tile0 + U.tiles_per_chunk, U.n_tiles);
        const int step = pair + 1;                        // bins per generation pass
        const uint32_t stash = tmem + (uint32_t)(nN * (1 + QB * G * mh));   // third bin's tile
        for (int64_t tile = tile0; tile < tile1 && !aborted; ++tile) {
            for (int bp = 0; bp < QB && !aborted; bp += step) {
                const int nb = min(step, QB - bp);
                const int kA = min(k0 + bp, nq - 1);   // bins past the end repeat the last
                issue_b1(kA, 0);                        // (their outputs are discarded)
                if (pending2) {   // tile buffers and B2 still read by the last MMA2
                    if (!wait_all(mbar2, ph2)) { aborted = true; break; }
                    ph2 ^= 1;
                    pending2 = false;
                }
                if (bp == 0) {    // new scatterer tile
                    for (int i = tid; i < kSB; i += kThreads) {
                        int64_t s = tile * kSB + i;
                        sc[i] = s < U.S ? make_float4(U.x[s], (HAS_Y && U.y) ? U.y[s] : 0.f, U.z[s], U.rc[s])
                                        : make_float4(0.f, 0.f, 1.f, 0.f);
                    }
                    __syncthreads();
                }
                // ---- Green's tiles of bins kA (buffer A0), kA + 1 (A1), kA + 2 (stash)
                const float qA = (float)(gc.q_lo + kA);
                const bool tab = !HAS_Y && use_tab;
                if (nb == 3) {
                    if (tab) gen_tiles<3, !HAS_Y, HAS_Y, BF16, NARROW, LINEAR>(gc, sub, tabs, sc, Np, qA, A0, A1, stash, tid);
                    else gen_tiles<3, false, HAS_Y, BF16, NARROW, LINEAR>(gc, sub, tabs, sc, Np, qA, A0, A1, stash, tid);
                } else if (nb == 2) {
                    if (tab) gen_tiles<2, !HAS_Y, HAS_Y, BF16, NARROW, LINEAR>(gc, sub, tabs, sc, Np, qA, A0, A1, stash, tid);
                    else gen_tiles<2, false, HAS_Y, BF16, NARROW, LINEAR>(gc, sub, tabs, sc, Np, qA, A0, A1, stash, tid);
                } else {
                    if (tab) gen_tiles<1, !HAS_Y, HAS_Y, BF16, NARROW, LINEAR>(gc, sub, tabs, sc, Np, qA, A0, A1, stash, tid);
                    else gen_tiles<1, false, HAS_Y, BF16, NARROW, LINEAR>(gc, sub, tabs, sc, Np, qA, A0, A1, stash, tid);
                }
                tc::fence_proxy_async_smem();
                tc::fence_before_sync();
                __syncthreads();
                tc::fence_after_sync();

                // every bin of the pass, every transmit group: MMA1 -> P' -> MMA2
                for (int si = 0; si < nb * G && !aborted; ++si) {
                    const int bi_ = si / G, g = si - bi_ * G;
                    const int TGg = min(TG, T - g * TG);      // transmits of this group
                    const uint32_t abase = bi_ == 1 ? abuf1 : abuf0;
                    if (bi_ == 2 && g == 0) {
                        // the third bin into A0: every MMA2 of the first bin (the last
                        // readers of A0) completed before the second bin's first P'
                        unstash_tile(Np, A0, stash, tid);
                        tc::fence_proxy_async_smem();
                        tc::fence_before_sync();
                        __syncthreads();
                        tc::fence_after_sync();
                    }
                    // ---- MMA1: D1 = A * B1^T
                    if (tid == 0) {
                        if (!tc::mbar_wait_bounded(mbar_b1, ph_b1, kMaxWait)) {
                            atomicExch(abort_flag, 1);
                        } else {
                            b1_inflight = false;
                            tc::fence_after_sync();
                            for (int j = 0; j < K1 / 16; ++j) {
                                uint64_t ad = tc::smem_desc(abase + 256 * j, 128, 16 * K1);
                                uint64_t bd = tc::smem_desc(b1s + 256 * j, 128, 16 * K1);
                                tc::mma_f16(tmem, ad, bd, idesc1, j > 0);
                            }
                            tc::mma_commit(mbar1);
                        }
                    }
                    ph_b1 ^= 1;
                    if (!wait_all(mbar1, ph1)) { aborted = true; break; }
                    ph1 ^= 1;
                    tc::fence_after_sync();
                    if (si + 1 < nb * G) {                     // B1 is free again
                        const int sn = si + 1;
                        issue_b1(min(k0 + bp + sn / G, nq - 1), sn % G);
                    }
                    if (pending2) {                            // B2 still read by MMA2
                        if (!wait_all(mbar2, ph2)) { aborted = true; break; }
                        ph2 ^= 1;
                        pending2 = false;
                    }
                    // ---- P' = R_s P -> B2, MN-major (the 8 transmit rows of a core matrix
                    // are contiguous for one scatterer): row 2t = (Re P' | -Im P'), row
                    // 2t+1 = (Im P' | Re P') over K = (s | 128 + s), four 16-byte stores
                    // per thread and 8 transmits
                    {
                        const int sp = warp & 3, cc = warp >> 2;
                        const int s = sp * 32 + lane;
                        const float R = sc[s].w;
                        for (int c0 = cc * 16; c0 < nN; c0 += 64) {
                            float v[16];
                            tc::tmem_ld16(tmem + ((uint32_t)(sp * 32) << 16) + (uint32_t)c0, v);
                            uint32_t w0[8], w1[8];
#pragma unroll
                            for (int i = 0; i < 8; ++i) {
                                const int t = (c0 >> 1) + i;
                                float pr = 0.f, pi = 0.f;
                                if (t < TGg) { pr = R * v[2 * i]; pi = R * v[2 * i + 1]; }
                                w0[i] = h16x2<BF16>(pr, pi);
                                w1[i] = h16x2<BF16>(-pi, pr);
                            }
                            const uint32_t nrow = (uint32_t)(nN >> 3);
                            unsigned char *q0 = B2 + ((((uint32_t)(s >> 3) * nrow + (uint32_t)(c0 >> 3)) << 7) + ((s & 7) << 4));
                            unsigned char *q1 = q0 + ((16u * nrow) << 7);        // k = 128 + s
                            *reinterpret_cast<uint4 *>(q0) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
                            *reinterpret_cast<uint4 *>(q0 + 128) = make_uint4(w0[4], w0[5], w0[6], w0[7]);
                            *reinterpret_cast<uint4 *>(q1) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
                            *reinterpret_cast<uint4 *>(q1 + 128) = make_uint4(w1[4], w1[5], w1[6], w1[7]);
                        }
                    }
                    tc::fence_proxy_async_smem();
                    tc::fence_before_sync();
                    __syncthreads();
                    tc::fence_after_sync();
                    // ---- MMA2: D2[bin][half] (+)= A^T * B2^T, A^T the MN-major view of
                    // the tile: k-slice j covers scatterers 16 (j mod 8) .. +15 of the Re
                    // (j < 8) or Im (j >= 8) half.  In the no-swizzle MN-major form the
                    // leading byte offset is the stride between K-adjacent core matrices
                    // (scatterer groups, 16 K1 bytes) and the stride byte offset the one
                    // between MN-adjacent core matrices (element groups, 128 bytes).
                    if (tid == 0) {
                        for (int h = 0; h < mh; ++h) {
                            const uint32_t d2 = tmem + (uint32_t)(nN * (1 + ((bp + bi_) * G + g) * mh + h));
                            for (int j = 0; j < 16; ++j) {
                                const uint32_t a0 = abase + (uint32_t)((2 * (j & 7)) * 16 * K1)
                                                  + (uint32_t)((j >> 3) * (Np / 8) * 128) + (uint32_t)(h * 16 * 128);
                                uint64_t ad = tc::smem_desc(a0, 16 * K1, 128);
                                uint64_t bd = tc::smem_desc(b2s + (uint32_t)(32 * nN * j), 16 * nN, 128);
                                tc::mma_f16(d2, ad, bd, idesc2, (j > 0 || tile > tile0) ? 1u : 0u);
                            }
                        }
                        tc::mma_commit(mbar2);
                    }
                    pending2 = true;
                }
            }
        }
        if (aborted) break;
        if (pending2) {
            if (!wait_all(mbar2, ph2)) { aborted = true; break; }
            ph2 ^= 1;
            pending2 = false;
        }
        tc::fence_after_sync();
        // ---- partial spectra of this item: part[chunk][g TG + t][e][k]
        {
            const int sp = warp & 3, cc = warp >> 2;
            for (int bg = 0; bg < QB * G; ++bg) {
                const int b = bg / G, g = bg - b * G;
                const int k = k0 + b;
                const int TGg = min(TG, T - g * TG);
                for (int h = 0; h < mh; ++h) {
                    const int e = 128 * h + sp * 32 + lane;
                    for (int c0 = cc * 16; c0 < nN; c0 += 64) {
                        float v[16];
                        tc::tmem_ld16(tmem + ((uint32_t)(sp * 32) << 16) +
                                          (uint32_t)(nN * (1 + bg * mh + h) + c0), v);
                        if (k < nq && e < N) {
#pragma unroll
                            for (int i = 0; i < 8; ++i) {
                                const int t = (c0 >> 1) + i;
                                if (t < TGg)
                                    U.part[(((size_t)chunk * T + g * TG + t) * N + e) * nq + k] =
                                        make_float2(v[2 * i], v[2 * i + 1]);
                            }
                        }
                    }
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    if (*abort_flag && tid == 0) {
        atomicExch(err, SIMUS_ERR_TIMEOUT);
        if (b1_inflight) tc::mbar_wait_bounded(mbar_b1, ph_b1, kMaxWait);   // own copy in flight
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// Shape of one simulation on this kernel.  Transmit groups as large as the tensor
// memory (512 columns: D1 + QB * mh D2 slices of nN columns) and shared memory allow;
// two tile buffers when they fit; chunk sizes from the simulation's share of the work.
TcShape tc_shape(const simus_plan *p, int T, int64_t S, double work_share, int items_per_sm) {
    TcShape g{};
    g.Np = (p->N + 7) & ~7;
    if (g.Np > 256) return g;
    g.mh = g.Np > 128 ? 2 : 1;
    const size_t limit = 227 * 1024 - kHeader - 1024;
    const int tab_full = (p->delta_table && p->d_dtab) ? p->gc.tab_n : 0;
    // Three bins per generation pass (two tile buffers and a tensor-memory stash), else
    // two (two buffers), else one, with at most two transmit groups when bins share a
    // pass; the delta table where it still fits beside them; tensor memory holds D1,
    // QB * G * mh accumulator slices of nN columns and the stash.
    for (int mode = p->pair_mode; mode >= 0 && !g.ok; --mode) {
        if (mode == 2 && g.mh != 1) continue;        // the stash holds one 128-column tile
        const int per = mode + 1;                    // bins per generation pass
        const int stash = mode == 2 ? g.Np : 0;      // tensor-memory columns of the stash
        for (int tb = 0; tb < 2 && !g.ok; ++tb) {
            const int tab_n = tb ? 0 : tab_full;
            if (tb && !tab_full) break;
            for (int TG = std::min(T, 120); TG >= 1 && !g.ok; TG = (TG > 8 ? TG - 8 : TG - 1)) {
                const int nN = ((2 * TG + 15) / 16) * 16;
                const int G = (T + TG - 1) / TG;
                if (mode && G > 2) break;
                const int qb = (512 - nN - stash) / (nN * G * g.mh);
                if (qb < per) continue;
                const size_t sm = unit_smem(g.Np, nN, mode ? 1 : 0, p->M, tab_n);
                if (sm > limit) continue;
                g.ok = true;
                g.TG = TG; g.nN = nN; g.pair = mode; g.n_groups = G; g.tab_n = tab_n;
                g.QB = std::min(std::max(p->max_bins, per), qb);
                g.QB -= g.QB % per;
                g.smem = sm + kHeader;
            }
        }
    }
    if (!g.ok) return g;
    g.n_btiles = (p->nq + g.QB - 1) / g.QB;
    g.n_tiles = std::max<int64_t>(1, (S + kSB - 1) / kSB);
    int64_t chunks;
    if (work_share >= 0.999 && p->chunks > 0) {
        chunks = std::min<int64_t>(p->chunks, g.n_tiles);
    } else if (work_share >= 0.999) {
        // one simulation: the chunk count minimising the modelled makespan
        // ceil(items / SMs) * tiles per item, items = bin tiles * chunks
        const int64_t per = (int64_t)g.n_btiles;
        double best = 1e300;
        chunks = 1;
        for (int64_t c = 1; c <= std::min<int64_t>(g.n_tiles, 64); ++c) {
            const int64_t waves = (per * c + p->num_sms - 1) / p->num_sms;
            const int64_t tiles = (g.n_tiles + c - 1) / c;
            const double span = (double)waves * tiles * (1.0 + 0.002 * c);   // small cost per chunk
            if (span < best) { best = span; chunks = c; }
        }
    } else {
        // part of a batch: this simulation's share of ~items_per_sm items per SM; the
        // dynamic work counter balances the rest
        const double want = std::max(1.0, work_share * items_per_sm * p->num_sms);
        chunks = (int64_t)std::ceil(want / (double)g.n_btiles);
        chunks = std::max<int64_t>(1, std::min<int64_t>(chunks, std::max<int64_t>(1, g.n_tiles / 2)));
    }
    g.tiles_per_chunk = (int)((g.n_tiles + chunks - 1) / chunks);
    g.n_chunks = (int)((g.n_tiles + g.tiles_per_chunk - 1) / g.tiles_per_chunk);
    g.b1_bytes = (size_t)p->nq * g.n_groups * g.nN * 2 * g.Np * 2;
    return g;
}

template <bool HAS_Y, bool BF16>
static auto pick_tc(bool narrow, bool linear) {
    return narrow ? (linear ? k_tc_rf<HAS_Y, BF16, true, true> : k_tc_rf<HAS_Y, BF16, true, false>)
                  : (linear ? k_tc_rf<HAS_Y, BF16, false, true> : k_tc_rf<HAS_Y, BF16, false, false>);
}

int launch_tc_units(const TcUnit *h_units, const TcUnit *d_units, int n_units, int64_t n_items,
                    size_t smem, bool bf16, bool has_y, bool narrow, bool linear, int num_sms,
                    int *counter, int *err, cudaStream_t st) {
    for (int u = 0; u < n_units; ++u) {
        const TcUnit &U = h_units[u];
        int64_t total = (int64_t)U.gc.nq * U.G * U.nN * 2 * U.Np;
        int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms * 16);
        if (bf16)
            k_tc_weights<true><<<blocks, 256, 0, st>>>(U.T, U.G, U.TG, U.gc.N, U.Np, U.nN, U.gc.nq,
                                                       U.gc.q_lo, U.gc.df, U.delays, U.apod, U.b1img);
        else
            k_tc_weights<false><<<blocks, 256, 0, st>>>(U.T, U.G, U.TG, U.gc.N, U.Np, U.nN, U.gc.nq,
                                                        U.gc.q_lo, U.gc.df, U.delays, U.apod, U.b1img);
        count_launches(1);
        int rc = check_cuda(cudaGetLastError(), "k_tc_weights launch");
        if (rc) return rc;
    }
    auto kern = has_y ? (bf16 ? pick_tc<true, true>(narrow, linear) : pick_tc<true, false>(narrow, linear))
                      : (bf16 ? pick_tc<false, true>(narrow, linear) : pick_tc<false, false>(narrow, linear));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return check_cuda(e, "k_tc_rf smem attribute");
    const int grid = (int)std::min<int64_t>(n_items, num_sms);
    kern<<<grid, kThreads, smem, st>>>(d_units, n_units, n_items, counter, err);
    count_launches(1);
    return check_cuda(cudaGetLastError(), "k_tc_rf launch");
}

}  // namespace simus
