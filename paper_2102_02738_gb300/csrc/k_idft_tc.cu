// k_idft_tc.cu -- the inverse DFT of Eq. 1 on the tensor cores, for the tensor-core path.
//
//   rf[c][j] = Re sum_k X[c][k] exp(-2 pi i q_k j / Nt) = sum_k (Re X cos phi + Im X sin phi),
//   phi = 2 pi (q_k j mod Nt) / Nt,
//
// is a real matrix product rf^T = B A^T with B[j][2k + (0, 1)] = (cos phi, sin phi)
// (samples x 2 nq) and A[c][2k + (0, 1)] = (Re X, Im X) (channels x 2 nq).  Both operands
// are carried as BF16 leading parts and remainders, hi = bf16(v), rem = bf16(v - hi), and
// each K step forms hi hi' + hi rem' + rem hi' (the dropped rem rem' is 2^-16 relative), so
// the product keeps the FP32 range and about 16 significant bits.
//
// Operands are stored pre-blocked: for a tile of R rows (128 samples or 256 channels) and a
// chunk of 32 K values, one contiguous block per part in the no-swizzle K-major
// core-matrix layout of tcgen05.cuh, so that one 1-D bulk copy moves it.  One CTA (128
// threads) per tile of 128 samples x 256 channels: four shared-memory stages of (twiddle
// hi, rem, spectrum hi, rem), filled by bulk copies on full barriers and released by
// tcgen05.commit on empty barriers; thread 0 issues 6 MMAs (M 128, N 256, K 16) per chunk
// into a 256-column tensor-memory accumulator, whose lanes are samples, so that the
// epilogue's stores run along the RF rows.  Every wait is bounded.
#include <algorithm>
#include <cuda_bf16.h>

#include "simus_internal.h"
#include "tcgen05.cuh"

namespace simus {

namespace {
constexpr int kIBM = 128, kIBN = 256, kIKC = 32;      // samples, channels, K per chunk
constexpr int kIStages = 4;
constexpr int kIThreads = 128;
constexpr int kIMaxWait = 1 << 22;
constexpr uint32_t kITwBytes = kIBM * kIKC * 2, kISpBytes = kIBN * kIKC * 2;   // one part
constexpr uint32_t kIStageBytes = 2 * kITwBytes + 2 * kISpBytes;
constexpr size_t kISmem = 1024 + (size_t)kIStages * kIStageBytes;
static_assert(kISmem <= 232448, "k_idft_tc stages exceed the shared memory of a CTA");

// hi, rem of a pair of values as two packed BF16 pairs
__device__ __forceinline__ void split_pair(float a, float b, uint32_t &hi, uint32_t &rem) {
    const __nv_bfloat16 ah = __float2bfloat16_rn(a), bh = __float2bfloat16_rn(b);
    const __nv_bfloat16 ar = __float2bfloat16_rn(a - __bfloat162float(ah));
    const __nv_bfloat16 br = __float2bfloat16_rn(b - __bfloat162float(bh));
    hi = (uint32_t)__bfloat16_as_ushort(ah) | ((uint32_t)__bfloat16_as_ushort(bh) << 16);
    rem = (uint32_t)__bfloat16_as_ushort(ar) | ((uint32_t)__bfloat16_as_ushort(br) << 16);
}

// Word w (4 bytes: K values 2k, 2k + 1 of one row) of an R x kIKC block in the K-major
// core-matrix layout: its row r and pair index kp (K value 2 kp) within the block.
__device__ __forceinline__ void block_word(int w, int &r, int &kp) {
    const int core = w >> 5, in = w & 31;               // 32 words per 128-byte core matrix
    r = (core / (kIKC / 8)) * 8 + (in >> 2);
    kp = (core % (kIKC / 8)) * 4 + (in & 3);
}
}  // namespace

size_t idft_tc_twiddle_bytes(int nt, int nq) {
    const size_t njt = (size_t)(nt + kIBM - 1) / kIBM, nkc = ((size_t)2 * nq + kIKC - 1) / kIKC;
    return njt * nkc * 2 * kITwBytes;
}
size_t idft_tc_operand_bytes(int n_chan, int nq) {
    const size_t nct = (size_t)(n_chan + kIBN - 1) / kIBN, nkc = ((size_t)2 * nq + kIKC - 1) / kIKC;
    return nct * nkc * 2 * kISpBytes;
}

// Twiddles, blocked: block (jt, kc) holds samples jt kIBM .. + kIBM - 1 and K values
// kc kIKC .. + kIKC - 1 as two parts (hi, rem) of kITwBytes; samples past nt and K values
// past 2 nq are zero.  One thread per word (one sample, one bin: cos and sin).
__global__ void k_idft_twiddles(int nq, int q_lo, int nt, int nkc, int njt, uint32_t *__restrict__ tw) {
    constexpr int W = kITwBytes / 4;
    const int64_t total = (int64_t)njt * nkc * W;
    const int half = nt / 2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int w = (int)(i % W);
        const int64_t blk = i / W;                      // jt nkc + kc
        const int kc = (int)(blk % nkc), jt = (int)(blk / nkc);
        int r, kp;
        block_word(w, r, kp);
        const int j = jt * kIBM + r, k = kc * (kIKC / 2) + kp;
        float s = 0.f, c = 0.f;
        if (j < nt && k < nq) {
            int m = (int)(((int64_t)(q_lo + k) * j) % nt);
            if (m > half) m -= nt;                       // angle in (-pi, pi]
            sincospif(2.0f * (float)m / (float)nt, &s, &c);
        }
        uint32_t hi, rem;
        split_pair(c, s, hi, rem);
        tw[blk * 2 * W + w] = hi;
        tw[(blk * 2 + 1) * W + w] = rem;
    }
}

// Spectra X[c][k] (complex, c < n_chan) into blocks of kIBN channels, like the twiddles.
__global__ void k_idft_operand(const float2 *__restrict__ spec, int n_chan, int nq, int nkc, int nct,
                               uint32_t *__restrict__ sp) {
    constexpr int W = kISpBytes / 4;
    const int64_t total = (int64_t)nct * nkc * W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int w = (int)(i % W);
        const int64_t blk = i / W;                      // ct nkc + kc
        const int kc = (int)(blk % nkc), ct = (int)(blk / nkc);
        int r, kp;
        block_word(w, r, kp);
        const int c = ct * kIBN + r, k = kc * (kIKC / 2) + kp;
        const float2 x = (c < n_chan && k < nq) ? spec[(size_t)c * nq + k] : make_float2(0.f, 0.f);
        uint32_t hi, rem;
        split_pair(x.x, x.y, hi, rem);
        sp[blk * 2 * W + w] = hi;
        sp[(blk * 2 + 1) * W + w] = rem;
    }
}

// rf[c][j] for the tile blockIdx.x (128 samples) x blockIdx.y (256 channels).
__global__ void __launch_bounds__(kIThreads, 1)
k_idft_tc(const uint32_t *__restrict__ tw, const uint32_t *__restrict__ sp, int n_chan, int nt, int nkc,
          float *__restrict__ rf, int *err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    // header: full[kIStages], empty[kIStages], done mbarriers, tensor-memory slot, abort flag
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + 8 * (2 * kIStages + 1));
    int *abort_flag = reinterpret_cast<int *>(smem + 8 * (2 * kIStages + 1) + 4);
    unsigned char *stage0 = smem + 1024;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int jt = blockIdx.x, ct = blockIdx.y;
    if (tid == 0) {
        for (int i = 0; i < 2 * kIStages + 1; ++i) tc::mbar_init(tc::smem_u32(&bars[i]), 1);
        tc::fence_mbar_init();
        *abort_flag = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(tslot), 256);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;

    if (tid == 0) {
        const uint32_t idesc = tc::idesc_f16(kIBM, kIBN, true);
        const char *twb = reinterpret_cast<const char *>(tw) + (size_t)jt * nkc * 2 * kITwBytes;
        const char *spb = reinterpret_cast<const char *>(sp) + (size_t)ct * nkc * 2 * kISpBytes;
        auto load = [&](int kc, int s) {       // chunk kc's four parts into stage s
            unsigned char *st = stage0 + (size_t)s * kIStageBytes;
            const uint32_t fb = tc::smem_u32(&bars[s]);
            tc::mbar_arrive_expect_tx(fb, kIStageBytes);
            tc::bulk_g2s(tc::smem_u32(st), twb + (size_t)kc * 2 * kITwBytes, 2 * kITwBytes, fb);
            tc::bulk_g2s(tc::smem_u32(st + 2 * kITwBytes), spb + (size_t)kc * 2 * kISpBytes, 2 * kISpBytes, fb);
        };
        bool ok = true;
        int issued[kIStages], taken[kIStages];           // loads per stage issued / waited for
        for (int s = 0; s < kIStages; ++s) {
            issued[s] = taken[s] = 0;
            if (s < nkc) { load(s, s); issued[s] = 1; }
        }
        for (int kc = 0; kc < nkc; ++kc) {
            const int s = kc % kIStages;
            if (!tc::mbar_wait_bounded(tc::smem_u32(&bars[s]), (uint32_t)((kc / kIStages) & 1), kIMaxWait)) {
                ok = false;
                break;
            }
            ++taken[s];
            tc::fence_after_sync();
            const uint32_t a = tc::smem_u32(stage0 + (size_t)s * kIStageBytes);
            const uint64_t ah = tc::smem_desc(a, 128, 16 * kIKC);
            const uint64_t ar = tc::smem_desc(a + kITwBytes, 128, 16 * kIKC);
            const uint64_t bh = tc::smem_desc(a + 2 * kITwBytes, 128, 16 * kIKC);
            const uint64_t br = tc::smem_desc(a + 2 * kITwBytes + kISpBytes, 128, 16 * kIKC);
#pragma unroll
            for (int q = 0; q < kIKC / 16; ++q) {      // K steps of 16: 256 bytes, 16 units
                const uint64_t d = 16ull * q;
                tc::mma_f16(tmem, ah + d, bh + d, idesc, (kc > 0 || q > 0) ? 1u : 0u);
                tc::mma_f16(tmem, ah + d, br + d, idesc, 1u);
                tc::mma_f16(tmem, ar + d, bh + d, idesc, 1u);
            }
            tc::mma_commit(tc::smem_u32(&bars[kIStages + s]));
            // the previous chunk's stage takes the chunk kIStages after it, once its MMAs
            // are done (this chunk's MMAs are queued behind them meanwhile)
            const int kp = kc - 1, kn = kc - 1 + kIStages;
            if (kp >= 0 && kn < nkc) {
                const int sp_ = kp % kIStages;
                if (!tc::mbar_wait_bounded(tc::smem_u32(&bars[kIStages + sp_]), (uint32_t)((kp / kIStages) & 1),
                                           kIMaxWait)) {
                    ok = false;
                    break;
                }
                load(kn, sp_);
                ++issued[sp_];
            }
        }
        tc::mma_commit(tc::smem_u32(&bars[2 * kIStages]));   // every MMA issued, also after a timeout
        if (!ok) {
            atomicExch(abort_flag, 1);
            for (int s = 0; s < kIStages; ++s)           // this CTA's copies still in flight
                for (int u = taken[s]; u < issued[s]; ++u)
                    tc::mbar_wait_bounded(tc::smem_u32(&bars[s]), (uint32_t)(u & 1), kIMaxWait);
        }
    }
    __syncthreads();
    const bool mma_done = tc::mbar_wait_bounded(tc::smem_u32(&bars[2 * kIStages]), 0, kIMaxWait);
    const bool done = mma_done && *abort_flag == 0;
    if (!done && tid == 0) atomicExch(err, SIMUS_ERR_TIMEOUT);
    tc::fence_after_sync();
    if (done) {    // warp w holds samples 32 w .. + 31 (tensor-memory lanes); columns: channels
        const int j = jt * kIBM + warp * 32 + lane;
        for (int c0 = 0; c0 < kIBN; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            const int cb = ct * kIBN + c0;
            if (j < nt) {
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (cb + i < n_chan) rf[(size_t)(cb + i) * nt + j] = v[i];
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

int build_idft_tc_twiddles(const simus_plan *p, void *tw, cudaStream_t st) {
    const int njt = (p->nt + kIBM - 1) / kIBM, nkc = (2 * p->nq + kIKC - 1) / kIKC;
    const int64_t words = (int64_t)njt * nkc * (kITwBytes / 4);
    const int blocks = (int)std::min<int64_t>((words + 255) / 256, (int64_t)p->num_sms * 16);
    k_idft_twiddles<<<blocks, 256, 0, st>>>(p->nq, p->q_lo, p->nt, nkc, njt, reinterpret_cast<uint32_t *>(tw));
    count_launches(1);
    return check_cuda(cudaGetLastError(), "k_idft_twiddles launch");
}

int launch_idft_tc(const simus_plan *p, const float2 *spec, int n_chan, float *rf, void *blocks_ws,
                   cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_idft_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kISmem);
    if (e != cudaSuccess) return check_cuda(e, "k_idft_tc smem attribute");
    const int njt = (p->nt + kIBM - 1) / kIBM, nct = (n_chan + kIBN - 1) / kIBN;
    const int nkc = (2 * p->nq + kIKC - 1) / kIKC;
    if (nct > 65535) return fail(SIMUS_ERR_UNSUPPORTED, "tensor-core iDFT: %d channels", n_chan);
    uint32_t *spb = reinterpret_cast<uint32_t *>(blocks_ws);
    const int64_t words = (int64_t)nct * nkc * (kISpBytes / 4);
    const int blocks = (int)std::min<int64_t>((words + 255) / 256, (int64_t)p->num_sms * 16);
    k_idft_operand<<<blocks, 256, 0, st>>>(spec, n_chan, p->nq, nkc, nct, spb);
    k_idft_tc<<<dim3(njt, nct), kIThreads, kISmem, st>>>(reinterpret_cast<const uint32_t *>(p->d_idft_tw), spb,
                                                           n_chan, p->nt, nkc, rf, p->d_err);
    count_launches(2);
    return check_cuda(cudaGetLastError(), "k_idft_tc launch");
}

}  // namespace simus
