// k_order.cu -- a simulation's scatterers reordered by their distance to the array before
// the tensor-core launch.
//
// The RF is a sum over scatterers (Eq. 30-32), so their order changes only the rounding.
// In distance order the 128-scatterer tiles hold scatterers at similar depth: those within
// a few mm of the array, whose sub-element pairs leave the delta table's first piece or the
// table itself (Eq. 16 evaluated directly), are gathered in a few tiles instead of making
// warps of every tile take those paths while the rest of the CTA waits at the barrier after
// generation.
//
// A stable counting sort into kOrdBuckets buckets of 0.5 mm (the last one open): per-block
// bucket counts (blocks of 1,024 scatterers or more), one prefix pass, and one warp per
// block placing its scatterers in their input order (the lanes of one bucket ranked with __match_any_sync), so the order is the
// same on every call.
#include <algorithm>

#include "simus_internal.h"

namespace simus {

namespace {
constexpr int kOrdBuckets = 256;
constexpr int kOrdMaxBlocks = 1024;

// scatterers per block: 1,024, or more (a multiple of 32) so that at most kOrdMaxBlocks
// blocks share the prefix pass; the order does not depend on it
int order_chunk(int64_t S) {
    const int64_t c = ((S + kOrdMaxBlocks - 1) / kOrdMaxBlocks + 31) / 32 * 32;
    return (int)std::max<int64_t>(1024, c);
}

// distance bucket of a scatterer: to the arc of radius R about (0, -R) (convex), to the
// line z = 0 (linear, R = 0)
__device__ __forceinline__ int depth_bucket(float x, float z, float R) {
    const float d = R > 0.0f ? fabsf(hypotf(x, z + R) - R) : fabsf(z);
    return min(kOrdBuckets - 1, (int)(d * 2000.0f));
}
}  // namespace

// hist[b][k]: scatterers of block b's chunk in bucket k
__global__ void __launch_bounds__(256)
k_order_hist(const float *__restrict__ x, const float *__restrict__ z, int64_t S, int chunk, float R,
             int *__restrict__ hist) {
    __shared__ int cnt[kOrdBuckets];
    for (int k = threadIdx.x; k < kOrdBuckets; k += blockDim.x) cnt[k] = 0;
    __syncthreads();
    const int64_t b0 = (int64_t)blockIdx.x * chunk, b1 = min(S, b0 + chunk);
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) atomicAdd(&cnt[depth_bucket(x[i], z[i], R)], 1);
    __syncthreads();
    for (int k = threadIdx.x; k < kOrdBuckets; k += blockDim.x)
        hist[(size_t)blockIdx.x * kOrdBuckets + k] = cnt[k];
}

// offs[b][k] = first output position of block b's scatterers of bucket k (buckets in
// order, blocks in order within a bucket); one block, thread k owns bucket k
__global__ void __launch_bounds__(kOrdBuckets)
k_order_scan(const int *__restrict__ hist, int nblk, int *__restrict__ offs) {
    __shared__ int base[kOrdBuckets];
    const int k = threadIdx.x;
    int run = 0;
    for (int b = 0; b < nblk; ++b) {
        offs[(size_t)b * kOrdBuckets + k] = run;
        run += hist[(size_t)b * kOrdBuckets + k];
    }
    base[k] = run;
    __syncthreads();
    if (k == 0) {                // exclusive prefix of the bucket totals
        int acc = 0;
        for (int j = 0; j < kOrdBuckets; ++j) {
            const int t = base[j];
            base[j] = acc;
            acc += t;
        }
    }
    __syncthreads();
    for (int b = 0; b < nblk; ++b) offs[(size_t)b * kOrdBuckets + k] += base[k];
}

// one warp per block: its chunk in slices of 32 in input order, each scatterer written at
// its bucket's running position plus its rank among the slice's lanes of that bucket
__global__ void __launch_bounds__(32)
k_order_scatter(const float *__restrict__ x, const float *__restrict__ y, const float *__restrict__ z,
                const float *__restrict__ rc, int64_t S, int chunk, float R, const int *__restrict__ offs,
                float *__restrict__ xo, float *__restrict__ yo, float *__restrict__ zo,
                float *__restrict__ rco) {
    __shared__ int pos[kOrdBuckets];
    const int lane = threadIdx.x;
    for (int k = lane; k < kOrdBuckets; k += 32) pos[k] = offs[(size_t)blockIdx.x * kOrdBuckets + k];
    __syncwarp();
    const int64_t b0 = (int64_t)blockIdx.x * chunk, b1 = min(S, b0 + chunk);
    const unsigned below = (1u << lane) - 1u;
    for (int64_t s0 = b0; s0 < b1; s0 += 32) {
        const int64_t i = s0 + lane;
        const bool valid = i < b1;
        float xv = 0.f, zv = 0.f;
        if (valid) { xv = x[i]; zv = z[i]; }
        const int key = valid ? depth_bucket(xv, zv, R) : kOrdBuckets + lane;   // idle lanes: own keys
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        const int rank = __popc(peers & below);
        if (valid) {
            const int p = pos[key] + rank;
            xo[p] = xv;
            zo[p] = zv;
            rco[p] = rc[i];
            if (y) yo[p] = y[i];
        }
        __syncwarp();
        if (valid && rank == 0) pos[key] += __popc(peers);     // the bucket's lowest lane
        __syncwarp();
    }
}

size_t order_scratch_bytes(int64_t S) {
    const int chunk = order_chunk(S);
    const int64_t nblk = (S + chunk - 1) / chunk;
    return sizeof(int) * (size_t)nblk * kOrdBuckets * 2;
}

int launch_order(const simus_scat *in, float R, int *scratch, float *xo, float *yo, float *zo,
                 float *rco, cudaStream_t st) {
    const int64_t S = in->n;
    const int chunk = order_chunk(S);
    const int nblk = (int)((S + chunk - 1) / chunk);
    int *hist = scratch, *offs = scratch + (size_t)nblk * kOrdBuckets;
    k_order_hist<<<nblk, 256, 0, st>>>(in->x, in->z, S, chunk, R, hist);
    k_order_scan<<<1, kOrdBuckets, 0, st>>>(hist, nblk, offs);
    k_order_scatter<<<nblk, 32, 0, st>>>(in->x, in->y, in->z, in->rc, S, chunk, R, offs, xo, in->y ? yo : nullptr,
                                         zo, rco);
    count_launches(3);
    return check_cuda(cudaGetLastError(), "scatterer order launch");
}

}  // namespace simus
