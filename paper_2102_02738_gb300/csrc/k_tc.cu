// k_tc.cu -- batched path on the tcgen05 tensor cores: one persistent launch over the
// work items of any number of simulations.
//
// The Green's tile G_e(q, s, e) of a bin q and a tile of 128 scatterers is generated once
// in FP32 (Eq. 17/20/39/40, sub-element sum of Eq. 33), rounded to FP16 (or split into BF16
// leading parts and remainders, three products per GEMM) in shared memory, and feeds two
// complex contractions written as real GEMMs:
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

#include "k_tc_kernel.cuh"

namespace simus {

namespace {
template <bool BF16>
__device__ __forceinline__ uint16_t h16(float v) {
    if (BF16) return __bfloat16_as_ushort(__float2bfloat16_rn(v));
    return __half_as_ushort(__float2half_rn(v));
}

// shared memory a unit needs after the header (split BF16: the tile's remainders in a
// second buffer, B1 and B2 doubled)
size_t unit_smem(int Np, int nN, int nbuf, int M, int tab_n, bool split) {
    const size_t a = (size_t)kSB * 2 * Np * 2;
    const size_t ops = split ? 2 : 1;
    return (split ? 2 : nbuf) * a + ops * ((size_t)nN * 2 * Np * 2 + (size_t)nN * 256 * 2)
         + sizeof(float4) * kSB + sizeof(float4) * M + 2 * sizeof(float4) * tab_n;
}
}  // namespace

// B1 images of one simulation: per kept bin and transmit group g, the nN x 2Np K-major
// operand of the transmit GEMM for transmits g TG .. g TG + TG - 1 (image [k][g]),
//   row 2t: (Re C, -Im C), row 2t+1: (Im C, Re C), C = W exp(i 2 pi frac(q df dtau)).
// BF16 images are split: the BF16 leading parts, then the BF16 remainders C - hi.
// One thread per complex weight (transmit slot, element) of an image, writing its four
// entries; blockIdx.y strides over the images.
template <bool BF16>
__device__ __forceinline__ void put_weight(uint16_t *im, int per_img, uint32_t o, float v) {
    im[o] = h16<BF16>(v);
    if (BF16) im[o + per_img] = h16<true>(v - __bfloat162float(__float2bfloat16_rn(v)));
}
template <bool BF16>
__global__ void k_tc_weights(int T, int G, int TG, int N, int Np, int nN, int nq, int q_lo,
                             double df, const float *__restrict__ delays,
                             const float *__restrict__ apod, uint16_t *__restrict__ img) {
    const int K = 2 * Np, per_img = nN * K, n_w = (nN / 2) * Np;
    constexpr int kOps = BF16 ? 2 : 1;
    for (int kg = blockIdx.y; kg < nq * G; kg += gridDim.y) {
        const int k = kg / G, g = kg - k * G;
        uint16_t *im = img + (size_t)kg * kOps * per_img;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_w; i += gridDim.x * blockDim.x) {
            const int tl = i / Np, e = i - tl * Np;
            const int t = g * TG + tl;
            float cr = 0.f, ci = 0.f;
            if (tl < TG && t < T && e < N) {
                double ph = (double)(q_lo + k) * ((double)delays[t * N + e] * df);
                ph -= rint(ph);
                float s, c;
                sincospif((float)(2.0 * ph), &s, &c);
                const float w = apod[t * N + e];
                cr = w * c;
                ci = w * s;
            }
            const int n = 2 * tl;
            put_weight<BF16>(im, per_img, tc::kmajor_offset(n, e, K) / 2, cr);
            put_weight<BF16>(im, per_img, tc::kmajor_offset(n, Np + e, K) / 2, -ci);
            put_weight<BF16>(im, per_img, tc::kmajor_offset(n + 1, e, K) / 2, ci);
            put_weight<BF16>(im, per_img, tc::kmajor_offset(n + 1, Np + e, K) / 2, cr);
        }
    }
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
    // BF16 operands are split into leading parts and remainders: one logical tile buffer
    // (the remainders take the second), stash slots of 2 Np columns, at most two bins per
    // pass (the packed leading parts and remainders of three bins exceed the registers)
    const bool split = p->path == SIMUS_PATH_TC_BF16;
    const int ops = split ? 2 : 1;
    // Preference, measured on the ragged batch: the delta table first (without it the
    // generation costs about 1.5 times as much); then more bins per generation pass
    // (3, 2, 1: sharing one geometry setup); then fewer transmit groups (each group
    // repeats MMA1, P' and MMA2 over the whole tile: one group with one tile buffer beat
    // two groups with two buffers by 11-16 %); then two shared-memory tile buffers over
    // one.  Bins past the buffers wait in tensor-memory stash slots of Np columns; at most
    // two transmit groups when bins share a pass; tensor memory holds D1, QB * G * mh
    // accumulator slices of nN columns and the stash.
    for (int tb = 0; tb < 2 && !g.ok; ++tb) {
        const int tab_n = tb ? 0 : tab_full;
        if (tb && !tab_full) break;
        for (int per = 3; per >= 1 && !g.ok; --per) {
            if (per > p->pair_mode + 1) continue;
            if (split && per > 2) continue;
            for (int nbuf = std::min(per, 2); nbuf >= 1; --nbuf) {
                if (split && nbuf != 1) continue;
                if (nbuf > p->tile_buffers) continue;
                const int stash = (per - nbuf) * g.Np * ops;   // tensor-memory columns of the stash
                // transmit-group sizes, largest first: FP16 steps down by 8; split BF16
                // (whose operands fill shared memory at smaller groups) takes the largest
                // size of each group count, ceil(T / G)
                for (int TG = std::min(T, 120), G0 = 1; TG >= 1;
                     TG = split ? (G0 < T ? (T + G0) / (G0 + 1) : 0) : (TG > 8 ? TG - 8 : TG - 1), ++G0) {
                    const int nN = ((2 * TG + 15) / 16) * 16;
                    const int G = (T + TG - 1) / TG;
                    if (per > 1 && G > 2) break;
                    if (g.ok && G >= g.n_groups) break;           // not fewer groups than found
                    if (nN > 256 || nN + stash > 512) continue;   // (an M = 128 MMA takes N <= 256)
                    const int qb = (512 - nN - stash) / (nN * G * g.mh);
                    if (qb < per) continue;
                    const size_t sm = unit_smem(g.Np, nN, nbuf, p->M + p->nu, tab_n, split);
                    if (sm > limit) continue;
                    g.ok = true;
                    g.TG = TG; g.nN = nN; g.pair = per - 1; g.nbuf = nbuf; g.n_groups = G;
                    g.tab_n = tab_n;
                    g.QB = std::min(std::max(p->max_bins, per), qb);
                    g.QB -= g.QB % per;
                    g.smem = sm + kHeader;
                    break;
                }
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
    g.b1_bytes = (size_t)p->nq * g.n_groups * g.nN * 2 * g.Np * 2 * ops;
    return g;
}


// One block waits for the second phase of an mbarrier that expects one arrival that
// never comes; the bounded wait gives up and the error flag is set as in k_tc_rf.
__global__ void k_selftest_timeout(int max_polls, int *err) {
    __shared__ uint64_t bar;
    const uint32_t mbar = tc::smem_u32(&bar);
    if (threadIdx.x == 0) {
        tc::mbar_init(mbar, 1);
        tc::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !tc::mbar_wait_bounded(mbar, 0, max_polls)) atomicExch(err, SIMUS_ERR_TIMEOUT);
}

int launch_selftest_timeout(int max_polls, int *err, cudaStream_t st) {
    k_selftest_timeout<<<1, 32, 0, st>>>(max_polls, err);
    count_launches(1);
    return check_cuda(cudaGetLastError(), "k_selftest_timeout launch");
}

int launch_tc_units(const TcUnit *h_units, const TcUnit *d_units, int n_units, int64_t n_items,
                    size_t smem, bool bf16, bool has_y, int sinc_mode, bool linear, int num_sms,
                    int *counter, int *err, cudaStream_t st) {
    for (int u = 0; u < n_units; ++u) {
        const TcUnit &U = h_units[u];
        const int n_w = (U.nN / 2) * U.Np;
        const dim3 blocks((n_w + 255) / 256, (unsigned)std::min<int64_t>((int64_t)U.gc.nq * U.G, 65535));
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
    // BF16 operands always go through the split (leading part + remainder) kernels
    const TcKernelFn kern = has_y ? (sinc_mode == 1 ? tc_kernel_y1_narrow(linear, bf16) : tc_kernel_y1_wide(linear, bf16))
                                  : (sinc_mode == 1 ? tc_kernel_y0_narrow(linear, bf16)
                                                    : (sinc_mode == 2 ? tc_kernel_y0_mid(linear, bf16)
                                                                      : tc_kernel_y0_wide(linear, bf16)));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return check_cuda(e, "k_tc_rf smem attribute");
    const int grid = (int)std::min<int64_t>(n_items, num_sms);
    kern<<<grid, kThreads, smem, st>>>(d_units, n_units, n_items, counter, err, bf16 ? 1 : 0);
    count_launches(1);
    return check_cuda(cudaGetLastError(), "k_tc_rf launch");
}

}  // namespace simus
