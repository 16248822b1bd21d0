// k_tc.cu -- batched path on the tcgen05 tensor cores.
//
// The Green's tile G_e(q, s, e) of one bin q and one tile of 128 scatterers is generated
// once in FP32 (Eq. 17/20/39/40, sub-element sum of Eq. 33), rounded to FP16 (or BF16)
// in shared memory, and feeds two complex contractions written as real GEMMs:
//
//   transmit sum (Eq. 29)   P[s][t]  = sum_e G[s][e] C_q[t][e]
//       A1 = [Re G | Im G]                      128 x 2Np   (rows s, K over e)
//       B1 rows 2t   = [ Re C_t | -Im C_t ]     nN x 2Np    (prepared per bin, TMA bulk copy)
//       B1 rows 2t+1 = [ Im C_t |  Re C_t ]
//       D1 columns (2t, 2t+1) = (Re P, Im P)    in tensor memory, FP32
//   reflection + receive sum (Eq. 30-32)   RF_q[e][t] += sum_s G[s][e] R_s P[s][t]
//       A2 = [Re G^T | Im G^T]                  128 x 256   (rows e, K over s)
//       B2 rows 2t   = [ Re P' | -Im P' ],  rows 2t+1 = [ Im P' | Re P' ],  P' = R_s P
//       D2[bin] columns (2t, 2t+1) = (Re RF, Im RF), accumulated over every scatterer
//       tile of the work item in tensor memory.
//
// One CTA per SM (512 threads, persistent over work items = (tile of QB bins, chunk of
// scatterer tiles)).  Per bin and scatterer tile: generate -> MMA1 -> read P, scale by
// R_s, write B2 -> MMA2.  All waits are bounded; on a timeout the CTA records an error
// code, frees its tensor memory and returns.
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

template <bool BF16> struct H16;
template <> struct H16<false> {
    using T = __half;
    static __device__ __forceinline__ T cvt(float v) { return __float2half_rn(v); }
    static __device__ __forceinline__ uint16_t bits(float v) { return __half_as_ushort(__float2half_rn(v)); }
};
template <> struct H16<true> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ T cvt(float v) { return __float2bfloat16_rn(v); }
    static __device__ __forceinline__ uint16_t bits(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }
};
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
        img[(size_t)k * per_bin + tc::kmajor_offset(n, kk, K) / 2] = H16<BF16>::bits(v);
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

template <bool HAS_Y, bool BF16, bool NARROW>
__global__ void __launch_bounds__(kThreads, 1) k_tc_rf(const TcParams P) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const GreenConst &gc = P.gc;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = gc.N, nu = gc.nu, M = gc.M, nq = gc.nq;
    const int Np = P.Np, nN = P.nN, T = P.T, QB = P.QB;
    const int K1 = 2 * Np;

    // shared-memory carve-up (all offsets multiples of 128 bytes)
    unsigned char *A1 = smem;                              // 128 x K1
    unsigned char *A2 = A1 + (size_t)kSB * K1 * 2;         // 128 x 256
    unsigned char *B1 = A2 + (size_t)128 * 256 * 2;        // nN x K1
    unsigned char *B2 = B1 + (size_t)nN * K1 * 2;          // nN x 256
    float4 *sc = reinterpret_cast<float4 *>(B2 + (size_t)nN * 256 * 2);   // [128]
    SubElem *sub = reinterpret_cast<SubElem *>(sc + kSB);                  // [M]
    uint64_t *bars = reinterpret_cast<uint64_t *>(sub + M);                // 3 mbarriers
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 3);
    int *abort_flag = reinterpret_cast<int *>(tslot + 1);

    const uint32_t a1s = tc::smem_u32(A1), a2s = tc::smem_u32(A2);
    const uint32_t b1s = tc::smem_u32(B1), b2s = tc::smem_u32(B2);
    const uint32_t mbar_b1 = tc::smem_u32(&bars[0]);
    const uint32_t mbar1 = tc::smem_u32(&bars[1]);
    const uint32_t mbar2 = tc::smem_u32(&bars[2]);

    for (int i = tid; i < M; i += kThreads) sub[i] = P.sub[i];
    // A2 rows >= Np are padding: zero once (the generation writes rows < Np)
    for (int i = tid; i < (128 - Np) * 256 / 8; i += kThreads)
        reinterpret_cast<uint4 *>(A2 + (size_t)Np * 256 * 2)[i] = make_uint4(0, 0, 0, 0);
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
    const uint32_t idesc = tc::idesc_f16(128, nN, BF16);
    const uint32_t b1_bytes = (uint32_t)nN * K1 * 2;

    uint32_t ph_b1 = 0, ph1 = 0, ph2 = 0;
    bool pending2 = false;
    bool aborted = false;
    bool b1_inflight = false;   // thread 0: a bulk copy into B1 not yet waited for

    auto wait_all = [&](uint32_t mbar, uint32_t parity) -> bool {
        if (!tc::mbar_wait_bounded(mbar, parity, kMaxWait)) atomicExch(abort_flag, 1);
        __syncthreads();
        return *abort_flag == 0;
    };

    for (int item = blockIdx.x; item < P.n_items && !aborted; item += gridDim.x) {
        const int bt = item % P.n_btiles, chunk = item / P.n_btiles;
        const int k0 = bt * QB;
        const int64_t tile0 = (int64_t)chunk * P.tiles_per_chunk;
        const int64_t n_tiles_total = (P.S + kSB - 1) / kSB;
        const int64_t tile1 = std::min<int64_t>(tile0 + P.tiles_per_chunk, n_tiles_total);
        for (int64_t tile = tile0; tile < tile1 && !aborted; ++tile) {
            // scatterer tile (all MMAs reading the previous one are complete: see below)
            if (pending2) {
                if (!wait_all(mbar2, ph2)) { aborted = true; break; }
                ph2 ^= 1;
                pending2 = false;
            }
            for (int i = tid; i < kSB; i += kThreads) {
                int64_t s = tile * kSB + i;
                sc[i] = s < P.S ? make_float4(P.x[s], HAS_Y ? P.y[s] : 0.f, P.z[s], P.rc[s])
                                : make_float4(0.f, 0.f, 1.f, 0.f);
            }
            __syncthreads();
            for (int b = 0; b < QB && !aborted; ++b) {
                const int k = min(k0 + b, nq - 1);   // bins past the end repeat the last (discarded)
                const float q = (float)(gc.q_lo + k);
                if (tid == 0) {
                    tc::mbar_arrive_expect_tx(mbar_b1, b1_bytes);
                    tc::bulk_g2s(b1s, P.b1img + (size_t)k * nN * K1, b1_bytes, mbar_b1);
                    b1_inflight = true;
                }
                if (pending2) {   // A2 / B2 still read by the previous MMA2
                    if (!wait_all(mbar2, ph2)) { aborted = true; break; }
                    ph2 ^= 1;
                    pending2 = false;
                }
                // ---- Green's tile: item (s, group of 8 elements)
                const int n_groups = Np >> 3;
                for (int it = tid; it < kSB * n_groups; it += kThreads) {
                    const int s = it & (kSB - 1), eg = it >> 7;
                    const float4 ps = sc[s];
                    float gr[8], gi[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int e = eg * 8 + j;
                        float ar = 0.f, ai = 0.f;
                        if (e < N) {
                            for (int mu = 0; mu < nu; ++mu) {
                                PairSetup ps_ = pair_setup<HAS_Y>(gc, sub[e * nu + mu], ps.x, ps.y, ps.z, q);
                                float2 g = green_term<HAS_Y, NARROW>(gc, ps_, q, ps_.amp0);
                                ar += g.x;
                                ai += g.y;
                            }
                        }
                        gr[j] = ar;
                        gi[j] = ai;
                    }
                    uint32_t pr[4], pim[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        pr[j] = (uint32_t)H16<BF16>::bits(gr[2 * j]) | ((uint32_t)H16<BF16>::bits(gr[2 * j + 1]) << 16);
                        pim[j] = (uint32_t)H16<BF16>::bits(gi[2 * j]) | ((uint32_t)H16<BF16>::bits(gi[2 * j + 1]) << 16);
                    }
                    *reinterpret_cast<uint4 *>(A1 + tc::kmajor_offset(s, eg * 8, K1)) =
                        make_uint4(pr[0], pr[1], pr[2], pr[3]);
                    *reinterpret_cast<uint4 *>(A1 + tc::kmajor_offset(s, Np + eg * 8, K1)) =
                        make_uint4(pim[0], pim[1], pim[2], pim[3]);
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int e = eg * 8 + j;
                        *reinterpret_cast<uint16_t *>(A2 + tc::kmajor_offset(e, s, 256)) = H16<BF16>::bits(gr[j]);
                        *reinterpret_cast<uint16_t *>(A2 + tc::kmajor_offset(e, 128 + s, 256)) = H16<BF16>::bits(gi[j]);
                    }
                }
                tc::fence_proxy_async_smem();
                tc::fence_before_sync();
                __syncthreads();
                tc::fence_after_sync();
                // ---- MMA1: D1 = A1 * B1^T
                if (tid == 0) {
                    bool ok = tc::mbar_wait_bounded(mbar_b1, ph_b1, kMaxWait);
                    if (!ok) atomicExch(abort_flag, 1);
                    else {
                        b1_inflight = false;
                        tc::fence_after_sync();
                        for (int j = 0; j < K1 / 16; ++j) {
                            uint64_t ad = tc::smem_desc(a1s + 256 * j, 128, 16 * K1);
                            uint64_t bd = tc::smem_desc(b1s + 256 * j, 128, 16 * K1);
                            tc::mma_f16(tmem, ad, bd, idesc, j > 0);
                        }
                        tc::mma_commit(mbar1);
                    }
                }
                ph_b1 ^= 1;
                if (!wait_all(mbar1, ph1)) { aborted = true; break; }
                ph1 ^= 1;
                tc::fence_after_sync();
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
                            *reinterpret_cast<uint16_t *>(B2 + tc::kmajor_offset(n0, s, 256)) = H16<BF16>::bits(pr);
                            *reinterpret_cast<uint16_t *>(B2 + tc::kmajor_offset(n0, 128 + s, 256)) = H16<BF16>::bits(-pi);
                            *reinterpret_cast<uint16_t *>(B2 + tc::kmajor_offset(n0 + 1, s, 256)) = H16<BF16>::bits(pi);
                            *reinterpret_cast<uint16_t *>(B2 + tc::kmajor_offset(n0 + 1, 128 + s, 256)) = H16<BF16>::bits(pr);
                        }
                    }
                }
                tc::fence_proxy_async_smem();
                tc::fence_before_sync();
                __syncthreads();
                tc::fence_after_sync();
                // ---- MMA2: D2[b] (+)= A2 * B2^T
                if (tid == 0) {
                    const uint32_t d2 = tmem + (uint32_t)(nN * (1 + b));
                    for (int j = 0; j < 16; ++j) {
                        uint64_t ad = tc::smem_desc(a2s + 256 * j, 128, 4096);
                        uint64_t bd = tc::smem_desc(b2s + 256 * j, 128, 4096);
                        tc::mma_f16(d2, ad, bd, idesc, (j > 0 || tile > tile0) ? 1u : 0u);
                    }
                    tc::mma_commit(mbar2);
                }
                pending2 = true;
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
    g.smem = (size_t)kSB * 2 * g.Np * 2 + 128 * 256 * 2 + (size_t)g.nN * 2 * g.Np * 2
           + (size_t)g.nN * 256 * 2 + sizeof(float4) * kSB + sizeof(SubElem) * p->M + 64;
    g.ok = g.smem <= 227 * 1024;
    return g;
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
    const bool has_y = sc->y != nullptr;
    const bool narrow = p->gc.narrow != 0;
    auto kern = has_y ? (bf16 ? (narrow ? k_tc_rf<true, true, true> : k_tc_rf<true, true, false>)
                              : (narrow ? k_tc_rf<true, false, true> : k_tc_rf<true, false, false>))
                      : (bf16 ? (narrow ? k_tc_rf<false, true, true> : k_tc_rf<false, true, false>)
                              : (narrow ? k_tc_rf<false, false, true> : k_tc_rf<false, false, false>));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
    if (e != cudaSuccess) return check_cuda(e, "k_tc_rf smem attribute");
    kern<<<g.grid, kThreads, g.smem, st>>>(P);
    count_launches(1);
    return check_cuda(cudaGetLastError(), "k_tc_rf launch");
}

}  // namespace simus
