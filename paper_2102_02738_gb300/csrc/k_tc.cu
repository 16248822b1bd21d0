// k_tc.cu -- batched path on the tcgen05 tensor cores.
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
//       A^T read from the same tile as an MN-major operand: M = e, K = (s | s) over
//       the Re G and Im G halves -- no second copy of the tile
//       B2 rows 2t   = [ Re P' | -Im P' ],  rows 2t+1 = [ Im P' | Re P' ],  P' = R_s P
//       D2[bin] columns (2t, 2t+1) = (Re RF, Im RF), accumulated over every scatterer
//       tile of the work item in tensor memory.
//
// One CTA per SM (512 threads, persistent over work items = (tile of QB bins, chunk of
// scatterer tiles)).  Bins are generated in pairs into two tile buffers so that the
// per-(scatterer, sub-element) geometry -- double-float distance and phase rate -- is
// shared by both bins.  Per bin: MMA1 -> read P from tensor memory, scale by R_s, write
// B2 -> MMA2.  All waits are bounded; on a timeout the CTA records an error code, waits
// for its own bulk copy, frees its tensor memory and returns.
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

template <bool BF16>
__device__ __forceinline__ uint16_t h16(float v) {
    if (BF16) return __bfloat16_as_ushort(__float2bfloat16_rn(v));
    return __half_as_ushort(__float2half_rn(v));
}
template <bool BF16>
__device__ __forceinline__ uint32_t h16x2(float lo, float hi) {
    return (uint32_t)h16<BF16>(lo) | ((uint32_t)h16<BF16>(hi) << 16);
}
}  // namespace

// B1 images: per kept bin, the nN x 2Np K-major operand of the transmit GEMM,
//   row 2t: (Re C, -Im C), row 2t+1: (Im C, Re C), C = W exp(i 2 pi frac(q df dtau)).
template <bool BF16>
__global__ void k_tc_weights(int T, int N, int Np, int nN, int nq, int q_lo, double df,
                             const float *__restrict__ delays, const float *__restrict__ apod,
                             uint16_t *__restrict__ img) {
    const int K = 2 * Np;
    const int64_t per_bin = (int64_t)nN * K;
    const int64_t total = per_bin * nq;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int k = (int)(i / per_bin);
        int r = (int)(i % per_bin);
        int n = r / K, kk = r % K;
        int t = n >> 1;
        int e = kk < Np ? kk : kk - Np;
        float v = 0.f;
        if (t < T && e < N) {
            double ph = (double)(q_lo + k) * ((double)delays[t * N + e] * df);
            ph -= rint(ph);
            float s, c;
            sincospif((float)(2.0 * ph), &s, &c);
            float w = apod[t * N + e];
            float cr = w * c, ci = w * s;
            bool first_half = kk < Np;
            v = (n & 1) ? (first_half ? ci : cr) : (first_half ? cr : -ci);
        }
        img[(size_t)k * per_bin + tc::kmajor_offset(n, kk, K) / 2] = h16<BF16>(v);
    }
}

struct TcParams {
    GreenConst gc;
    const SubElem *sub;
    const float *x, *y, *z, *rc;
    int64_t S;
    int T, Np, nN, QB;
    int n_btiles;          // bin tiles of QB bins
    int n_chunks;          // scatterer chunks
    int tiles_per_chunk;   // scatterer tiles (of 128) per chunk
    int n_items;           // n_btiles * n_chunks
    const uint16_t *b1img; // [nq][nN * 2Np]
    float2 *part;          // [n_chunks][T][N][nq]
    int *err;              // error flag
};

template <bool HAS_Y, bool BF16, bool NARROW, bool LINEAR>
__global__ void __launch_bounds__(kThreads, 1) k_tc_rf(const TcParams P) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const GreenConst &gc = P.gc;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = gc.N, nu = gc.nu, M = gc.M, nq = gc.nq;
    const int Np = P.Np, nN = P.nN, T = P.T, QB = P.QB;
    const int K1 = 2 * Np;
    const size_t abytes = (size_t)kSB * K1 * 2;

    // shared-memory carve-up (all offsets multiples of 128 bytes)
    unsigned char *A0 = smem;                              // bin buffer 0: 128 x K1
    unsigned char *A1 = A0 + abytes;                       // bin buffer 1
    unsigned char *B1 = A1 + abytes;                       // nN x K1
    unsigned char *B2 = B1 + (size_t)nN * K1 * 2;          // nN x 256
    float4 *sc = reinterpret_cast<float4 *>(B2 + (size_t)nN * 256 * 2);   // [128]
    SubElem *sub = reinterpret_cast<SubElem *>(sc + kSB);                  // [M]
    uint64_t *bars = reinterpret_cast<uint64_t *>(sub + M);                // 3 mbarriers
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 3);
    int *abort_flag = reinterpret_cast<int *>(tslot + 1);

    const uint32_t abuf[2] = {tc::smem_u32(A0), tc::smem_u32(A1)};
    const uint32_t b1s = tc::smem_u32(B1), b2s = tc::smem_u32(B2);
    const uint32_t mbar_b1 = tc::smem_u32(&bars[0]);
    const uint32_t mbar1 = tc::smem_u32(&bars[1]);
    const uint32_t mbar2 = tc::smem_u32(&bars[2]);

    for (int i = tid; i < M; i += kThreads) sub[i] = P.sub[i];
    if (tid == 0) {
        tc::mbar_init(mbar_b1, 1);
        tc::mbar_init(mbar1, 1);
        tc::mbar_init(mbar2, 1);
        tc::fence_mbar_init();
        *abort_flag = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(tslot), 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t idesc1 = tc::idesc_f16(128, nN, BF16);
    const uint32_t idesc2 = idesc1 | (1u << 15);          // A operand MN-major
    const uint32_t b1_bytes = (uint32_t)nN * K1 * 2;

    uint32_t ph_b1 = 0, ph1 = 0, ph2 = 0;
    bool pending2 = false;     // an MMA2 commit not yet waited for
    bool aborted = false;
    bool b1_inflight = false;  // thread 0: a bulk copy into B1 not yet waited for

    auto wait_all = [&](uint32_t mbar, uint32_t parity) -> bool {
        if (!tc::mbar_wait_bounded(mbar, parity, kMaxWait)) atomicExch(abort_flag, 1);
        __syncthreads();
        return *abort_flag == 0;
    };
    auto issue_b1 = [&](int k) {
        if (tid == 0) {
            tc::mbar_arrive_expect_tx(mbar_b1, b1_bytes);
            tc::bulk_g2s(b1s, P.b1img + (size_t)k * nN * K1, b1_bytes, mbar_b1);
            b1_inflight = true;
        }
    };

    for (int item = blockIdx.x; item < P.n_items && !aborted; item += gridDim.x) {
        const int bt = item % P.n_btiles, chunk = item / P.n_btiles;
        const int k0 = bt * QB;
        const int64_t tile0 = (int64_t)chunk * P.tiles_per_chunk;
        const int64_t n_tiles_total = (P.S + kSB - 1) / kSB;
        const int64_t tile1 = std::min<int64_t>(tile0 + P.tiles_per_chunk, n_tiles_total);
        for (int64_t tile = tile0; tile < tile1 && !aborted; ++tile) {
            for (int bp = 0; bp < QB && !aborted; bp += 2) {
                const int nb = min(2, QB - bp);
                const int kA = min(k0 + bp, nq - 1);       // bins past the end repeat the last
                const int kB = min(k0 + bp + 1, nq - 1);   // (their outputs are discarded)
                issue_b1(kA);
                if (pending2) {   // both tile buffers and B2 still read by the last MMA2
                    if (!wait_all(mbar2, ph2)) { aborted = true; break; }
                    ph2 ^= 1;
                    pending2 = false;
                }
                if (bp == 0) {    // new scatterer tile
                    for (int i = tid; i < kSB; i += kThreads) {
                        int64_t s = tile * kSB + i;
                        sc[i] = s < P.S ? make_float4(P.x[s], HAS_Y ? P.y[s] : 0.f, P.z[s], P.rc[s])
                                        : make_float4(0.f, 0.f, 1.f, 0.f);
                    }
                    __syncthreads();
                }
                // ---- Green's tiles of bins kA (buffer 0) and kB (buffer 1): items (s, 8 elements)
                const float qA = (float)(gc.q_lo + kA), qB = (float)(gc.q_lo + kB);
                const int n_groups = Np >> 3;
                for (int it = tid; it < kSB * n_groups; it += kThreads) {
                    const int s = it & (kSB - 1), eg = it >> 7;
                    const float4 ps = sc[s];
                    float ar[8], ai[8], br[8], bi[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int e = eg * 8 + j;
                        float xr = 0.f, xi = 0.f, yr = 0.f, yi = 0.f;
                        if (e < N) {
                            for (int mu = 0; mu < nu; ++mu) {
                                const PairSetup pa =
                                    pair_setup<HAS_Y, LINEAR>(gc, sub[e * nu + mu], ps.x, ps.y, ps.z, qA);
                                const float2 g = green_term<HAS_Y, NARROW>(gc, pa, qA, pa.amp0);
                                xr += g.x;
                                xi += g.y;
                                if (nb == 2) {
                                    const float2 h = green_term<HAS_Y, NARROW>(gc, pa, qB, pa.amp0 * pa.mstep);
                                    yr += h.x;
                                    yi += h.y;
                                }
                            }
                        }
                        ar[j] = xr; ai[j] = xi; br[j] = yr; bi[j] = yi;
                    }
                    *reinterpret_cast<uint4 *>(A0 + tc::kmajor_offset(s, eg * 8, K1)) =
                        make_uint4(h16x2<BF16>(ar[0], ar[1]), h16x2<BF16>(ar[2], ar[3]),
                                   h16x2<BF16>(ar[4], ar[5]), h16x2<BF16>(ar[6], ar[7]));
                    *reinterpret_cast<uint4 *>(A0 + tc::kmajor_offset(s, Np + eg * 8, K1)) =
                        make_uint4(h16x2<BF16>(ai[0], ai[1]), h16x2<BF16>(ai[2], ai[3]),
                                   h16x2<BF16>(ai[4], ai[5]), h16x2<BF16>(ai[6], ai[7]));
                    if (nb == 2) {
                        *reinterpret_cast<uint4 *>(A1 + tc::kmajor_offset(s, eg * 8, K1)) =
                            make_uint4(h16x2<BF16>(br[0], br[1]), h16x2<BF16>(br[2], br[3]),
                                       h16x2<BF16>(br[4], br[5]), h16x2<BF16>(br[6], br[7]));
                        *reinterpret_cast<uint4 *>(A1 + tc::kmajor_offset(s, Np + eg * 8, K1)) =
                            make_uint4(h16x2<BF16>(bi[0], bi[1]), h16x2<BF16>(bi[2], bi[3]),
                                       h16x2<BF16>(bi[4], bi[5]), h16x2<BF16>(bi[6], bi[7]));
                    }
                }
                tc::fence_proxy_async_smem();
                tc::fence_before_sync();
                __syncthreads();
                tc::fence_after_sync();

                for (int bi_ = 0; bi_ < nb && !aborted; ++bi_) {
                    const uint32_t abase = abuf[bi_];
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
                    if (bi_ + 1 < nb) issue_b1(kB);           // B1 is free again
                    if (pending2) {                            // B2 still read by MMA2
                        if (!wait_all(mbar2, ph2)) { aborted = true; break; }
                        ph2 ^= 1;
                        pending2 = false;
                    }
                    // ---- P' = R_s P -> B2
                    {
                        const int sp = warp & 3, cc = warp >> 2;
                        const int s = sp * 32 + lane;
                        const float R = sc[s].w;
                        for (int c0 = cc * 16; c0 < nN; c0 += 64) {
                            float v[16];
                            tc::tmem_ld16(tmem + ((uint32_t)(sp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
                            for (int i = 0; i < 8; ++i) {
                                const int t = (c0 >> 1) + i;
                                float pr = 0.f, pi = 0.f;
                                if (t < T) { pr = R * v[2 * i]; pi = R * v[2 * i + 1]; }
                                const int n0 = 2 * t;
                                *reinterpret_cast<uint16_t *>(B2 + tc::kmajor_offset(n0, s, 256)) = h16<BF16>(pr);
                                *reinterpret_cast<uint16_t *>(B2 + tc::kmajor_offset(n0, 128 + s, 256)) = h16<BF16>(-pi);
                                *reinterpret_cast<uint16_t *>(B2 + tc::kmajor_offset(n0 + 1, s, 256)) = h16<BF16>(pi);
                                *reinterpret_cast<uint16_t *>(B2 + tc::kmajor_offset(n0 + 1, 128 + s, 256)) = h16<BF16>(pr);
                            }
                        }
                    }
                    tc::fence_proxy_async_smem();
                    tc::fence_before_sync();
                    __syncthreads();
                    tc::fence_after_sync();
                    // ---- MMA2: D2[bin] (+)= A^T * B2^T, A^T the MN-major view of the tile:
                    // k-slice j covers scatterers 16 (j mod 8) .. +15 of the Re (j < 8) or
                    // Im (j >= 8) half.  In the no-swizzle MN-major form the leading byte
                    // offset is the stride between K-adjacent core matrices (scatterer
                    // groups, 16 K1 bytes) and the stride byte offset the one between
                    // MN-adjacent core matrices (element groups, 128 bytes).
                    if (tid == 0) {
                        const uint32_t d2 = tmem + (uint32_t)(nN * (1 + bp + bi_));
                        for (int j = 0; j < 16; ++j) {
                            const uint32_t a0 = abase + (uint32_t)((2 * (j & 7)) * 16 * K1)
                                              + (uint32_t)((j >> 3) * (Np / 8) * 128);
                            uint64_t ad = tc::smem_desc(a0, 16 * K1, 128);
                            uint64_t bd = tc::smem_desc(b2s + 256 * j, 128, 4096);
                            tc::mma_f16(d2, ad, bd, idesc2, (j > 0 || tile > tile0) ? 1u : 0u);
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
        // ---- partial spectra of this item: part[chunk][t][e][k]
        {
            const int sp = warp & 3, cc = warp >> 2;
            const int e = sp * 32 + lane;
            for (int b = 0; b < QB; ++b) {
                const int k = k0 + b;
                for (int c0 = cc * 16; c0 < nN; c0 += 64) {
                    float v[16];
                    tc::tmem_ld16(tmem + ((uint32_t)(sp * 32) << 16) + (uint32_t)(nN * (1 + b) + c0), v);
                    if (k < nq && e < N) {
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int t = (c0 >> 1) + i;
                            if (t < T)
                                P.part[(((size_t)chunk * T + t) * N + e) * nq + k] =
                                    make_float2(v[2 * i], v[2 * i + 1]);
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
        atomicExch(P.err, SIMUS_ERR_TIMEOUT);
        if (b1_inflight) tc::mbar_wait_bounded(mbar_b1, ph_b1, kMaxWait);   // own copy in flight
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

TcGeom tc_geometry(const simus_plan *p, int T, int64_t S) {
    TcGeom g{};
    g.Np = (p->N + 7) & ~7;
    g.nN = ((2 * T + 15) / 16) * 16;
    g.ok = p->N <= 128 && g.nN <= 256;
    if (!g.ok) return g;
    g.QB = std::max(1, std::min(4, (512 - g.nN) / g.nN));
    if (g.QB == 3) g.QB = 2;   // bins go in pairs
    g.n_btiles = (p->nq + g.QB - 1) / g.QB;
    const int64_t n_tiles = std::max<int64_t>(1, (S + kSB - 1) / kSB);
    // chunks: enough items for ~4 per SM, chunks of at least 4 scatterer tiles
    int64_t want_items = (int64_t)p->num_sms * 4;
    int64_t chunks = std::max<int64_t>(1, want_items / g.n_btiles);
    chunks = std::min<int64_t>(chunks, std::max<int64_t>(1, n_tiles / 4));
    g.tiles_per_chunk = (int)((n_tiles + chunks - 1) / chunks);
    g.n_chunks = (int)((n_tiles + g.tiles_per_chunk - 1) / g.tiles_per_chunk);
    g.n_items = g.n_btiles * g.n_chunks;
    g.grid = (int)std::min<int64_t>(g.n_items, p->num_sms);
    g.b1_bytes = (size_t)p->nq * g.nN * 2 * g.Np * 2;
    g.smem = 2 * (size_t)kSB * 2 * g.Np * 2 + (size_t)g.nN * 2 * g.Np * 2
           + (size_t)g.nN * 256 * 2 + sizeof(float4) * kSB + sizeof(SubElem) * p->M + 64;
    g.ok = g.smem <= 227 * 1024;
    return g;
}

template <bool HAS_Y, bool BF16>
static auto pick_tc(bool narrow, bool linear) {
    return narrow ? (linear ? k_tc_rf<HAS_Y, BF16, true, true> : k_tc_rf<HAS_Y, BF16, true, false>)
                  : (linear ? k_tc_rf<HAS_Y, BF16, false, true> : k_tc_rf<HAS_Y, BF16, false, false>);
}

int launch_tc(const simus_plan *p, const TcGeom &g, const simus_tx *tx, const simus_scat *sc,
              uint16_t *b1img, float2 *part, int *err, cudaStream_t st) {
    const bool bf16 = p->path == SIMUS_PATH_TC_BF16;
    {
        int64_t total = (int64_t)p->nq * g.nN * 2 * g.Np;
        int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)p->num_sms * 16);
        if (bf16)
            k_tc_weights<true><<<blocks, 256, 0, st>>>(tx->n_tx, p->N, g.Np, g.nN, p->nq, p->q_lo,
                                                       p->gc.df, tx->delays, tx->apod, b1img);
        else
            k_tc_weights<false><<<blocks, 256, 0, st>>>(tx->n_tx, p->N, g.Np, g.nN, p->nq, p->q_lo,
                                                        p->gc.df, tx->delays, tx->apod, b1img);
        count_launches(1);
        int rc = check_cuda(cudaGetLastError(), "k_tc_weights launch");
        if (rc) return rc;
    }
    TcParams P;
    P.gc = p->gc;
    P.sub = p->d_sub;
    P.x = sc->x; P.y = sc->y; P.z = sc->z; P.rc = sc->rc;
    P.S = sc->n;
    P.T = tx->n_tx; P.Np = g.Np; P.nN = g.nN; P.QB = g.QB;
    P.n_btiles = g.n_btiles; P.n_chunks = g.n_chunks; P.tiles_per_chunk = g.tiles_per_chunk;
    P.n_items = g.n_items;
    P.b1img = b1img; P.part = part; P.err = err;
    const bool has_y = sc->y != nullptr, narrow = p->gc.narrow != 0, linear = p->probe.radius <= 0;
    auto kern = has_y ? (bf16 ? pick_tc<true, true>(narrow, linear) : pick_tc<true, false>(narrow, linear))
                      : (bf16 ? pick_tc<false, true>(narrow, linear) : pick_tc<false, false>(narrow, linear));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
    if (e != cudaSuccess) return check_cuda(e, "k_tc_rf smem attribute");
    kern<<<g.grid, kThreads, g.smem, st>>>(P);
    count_launches(1);
    return check_cuda(cudaGetLastError(), "k_tc_rf launch");
}

}  // namespace simus
