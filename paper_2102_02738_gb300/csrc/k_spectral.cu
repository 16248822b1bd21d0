// k_spectral.cu -- chunk reduction with the transfer factor (Eq. 28, Eq. 34) and the
// inverse DFT to RF time signals (Eq. 1 convention), both on the CUDA cores in FP32.
#include <algorithm>

#include "simus_internal.h"

namespace simus {

// spec[i] = H[i % nq] * sum_c part[c][i], chunks summed in index order.
__global__ void k_reduce_spectrum(const float2 *__restrict__ part, int n_chunks, int64_t n_per,
                                  int nq, const float2 *__restrict__ H,
                                  float2 *__restrict__ spec) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_per;
         i += (int64_t)gridDim.x * blockDim.x) {
        float sx = 0.f, sy = 0.f;
        for (int c = 0; c < n_chunks; ++c) {
            float2 v = part[(size_t)c * n_per + i];
            sx += v.x;
            sy += v.y;
        }
        float2 h = H[i % nq];
        spec[i] = make_float2(h.x * sx - h.y * sy, h.x * sy + h.y * sx);
    }
}

int launch_reduce_spectrum(const simus_plan *p, const float2 *part, int n_chunks, int n_chan,
                           float2 *spec, cudaStream_t st) {
    int64_t n_per = (int64_t)n_chan * p->nq;
    int blocks = (int)std::min<int64_t>((n_per + 255) / 256, (int64_t)p->num_sms * 16);
    k_reduce_spectrum<<<blocks, 256, 0, st>>>(part, n_chunks, n_per, p->nq, p->d_H, spec);
    count_launches(1);
    return check_cuda(cudaGetLastError(), "k_reduce_spectrum launch");
}

// rf[c][j] = Re sum_k spec[c][k] exp(-2 pi i ((q_lo + k) j mod Nt) / Nt).
// Thread per sample j and CB channels; bins staged through shared memory in chunks of
// KB; the twiddle index m = q j mod Nt advances by j per bin (exact integers), and the
// angle 2 pi m / Nt is taken in (-pi, pi] before the hardware sine/cosine.
template <int CB, int KB>
__global__ void __launch_bounds__(256)
k_idft(const float2 *__restrict__ spec, int n_chan, int nq, int q_lo, int nt,
       float *__restrict__ rf) {
    __shared__ float2 xs[KB][CB];
    const int tid = threadIdx.x;
    const int j = blockIdx.x * 256 + tid;
    const int c0 = blockIdx.y * CB;
    const float wstep = -6.283185307179586f / (float)nt;
    float acc[CB];
#pragma unroll
    for (int c = 0; c < CB; ++c) acc[c] = 0.f;
    const int jj = j < nt ? j : 0;                 // idle threads of the last tile
    int m = (int)(((int64_t)q_lo * jj) % nt);
    const int half = nt / 2;
    for (int kb = 0; kb < nq; kb += KB) {
        __syncthreads();
        for (int i = tid; i < KB * CB; i += 256) {
            int cc = i / KB, kk = i - cc * KB;
            int c = c0 + cc, k = kb + kk;
            xs[kk][cc] = (c < n_chan && k < nq) ? spec[(size_t)c * nq + k] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        int kend = min(KB, nq - kb);
        for (int kk = 0; kk < kend; ++kk) {
            int mm = m > half ? m - nt : m;
            float s, co;
            __sincosf(wstep * (float)mm, &s, &co);
#pragma unroll
            for (int c = 0; c < CB; ++c) {
                float2 x = xs[kk][c];
                acc[c] = fmaf(x.x, co, fmaf(-x.y, s, acc[c]));
            }
            m += jj;
            if (m >= nt) m -= nt;
        }
    }
    if (j < nt) {
#pragma unroll
        for (int c = 0; c < CB; ++c)
            if (c0 + c < n_chan) rf[(size_t)(c0 + c) * nt + j] = acc[c];
    }
}

int launch_idft(const simus_plan *p, const float2 *spec, int n_chan, float *rf, cudaStream_t st) {
    constexpr int CB = 8, KB = 256;
    dim3 grid((p->nt + 255) / 256, (n_chan + CB - 1) / CB);
    k_idft<CB, KB><<<grid, 256, 0, st>>>(spec, n_chan, p->nq, p->q_lo, p->nt, rf);
    count_launches(1);
    return check_cuda(cudaGetLastError(), "k_idft launch");
}

}  // namespace simus
