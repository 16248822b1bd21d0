// k_pfield.cu -- RMS pressure field (Eq. 22, Eq. 41-42) on the CUDA cores, FP32.
//
//   P(X, w_j) = P_Tx(w_j) sum_n W_n g_n(X, w_j) exp(i w_j dtau_n),
//   P_RMS(X)  = sqrt(dw sum_j |P(X, w_j)|^2),   w_j = (j + 1/2) dw,  dw = 2 w_c / N_f.
// Since only |P|^2 enters, the pulse contributes |P_Tx|^2 = |S_P|^2 S_T per frequency.
// The midpoint frequencies are f_j = (j + 1/2) df with df = 2 fc / N_f, so the Green's
// machinery runs with half-integer "bin indices" q = j + 1/2 and that df.
//
// Thread per field point and chunk of frequencies; frequencies in runs of QB (phase
// recurrence over the run), all sub-elements accumulated per run, then |.|^2 weighted and
// summed; with several chunks their partial sums are added in a fixed order afterwards.  Frequencies
// whose |P_Tx|^2 is below 1e-12 of its maximum are skipped (their share of the sum is
// below 1e-12 N_f relative).
#include <algorithm>

#include "green.cuh"
#include "simus_internal.h"

namespace simus {

namespace {
constexpr int kPThreads = 256;
constexpr int kPQB = 8;
}  // namespace

// wt[t][jj][e] = W_te exp(i 2 pi frac((j0 + jj + 1/2) df dtau_te)), FP64 phase reduction.
__global__ void k_pfield_weights(int T, int N, int nf, int j0, double df,
                                 const float *__restrict__ delays, const float *__restrict__ apod,
                                 float2 *__restrict__ wt) {
    const int64_t total = (int64_t)T * nf * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(i % N);
        const int64_t r = i / N;
        const int jj = (int)(r % nf), t = (int)(r / nf);
        double ph = ((double)(j0 + jj) + 0.5) * ((double)delays[t * N + e] * df);
        ph -= rint(ph);
        float s, c;
        sincospif((float)(2.0 * ph), &s, &c);
        const float w = apod[t * N + e];
        wt[i] = make_float2(w * c, w * s);
    }
}

// TAB: delta/h at Y = 0 from the plan's table of cubic pieces (read-only cache; relative
// error <= 2.3e-6), evaluated directly within ~2 mm of a sub-element.
template <bool HAS_Y, bool NARROW, bool TAB>
__global__ void __launch_bounds__(kPThreads, 2)
k_pfield(const GreenConst gc, const SubElem *__restrict__ sub_g, const float *__restrict__ xg,
         const float *__restrict__ yg, const float *__restrict__ zg, int64_t npts, int nf, int j0,
         const float2 *__restrict__ wt, const float *__restrict__ ptx2, float dw,
         float *__restrict__ prms, const float4 *__restrict__ dtab, int fchunk,
         float *__restrict__ ppart) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = gc.N, nu = gc.nu, M = gc.M;
    const int tid = threadIdx.x, t = blockIdx.y;
    SubElem *sub = reinterpret_cast<SubElem *>(smem_raw);      // [M]
    float2 *wtt = reinterpret_cast<float2 *>(sub + M);         // [QB][N]
    for (int i = tid; i < M; i += kPThreads) sub[i] = sub_g[i];

    const int64_t i = blockIdx.x * (int64_t)kPThreads + tid;
    const bool live = i < npts;
    const float xs = live ? xg[i] : 0.f, zs = live ? zg[i] : 1.f;
    const float ys = (HAS_Y && live) ? yg[i] : 0.f;
    // frequency chunk blockIdx.z: [jbeg, jend) of the nf midpoints (a multiple of kPQB)
    const int jbeg = min(nf, (int)blockIdx.z * fchunk), jend = min(nf, jbeg + fchunk);
    float power = 0.f;
    for (int jb = jbeg; jb < jend; jb += kPQB) {
        __syncthreads();
        for (int k = tid; k < kPQB * N; k += kPThreads) {
            const int jj = k / N, e = k - jj * N;
            wtt[k] = jb + jj < jend ? wt[((size_t)t * nf + jb + jj) * N + e] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        const float q0 = (float)(j0 + jb) + 0.5f;
        float ar[kPQB], ai[kPQB];
#pragma unroll
        for (int j = 0; j < kPQB; ++j) ar[j] = ai[j] = 0.f;
        for (int n = 0; n < M; ++n) {
            const int e = n / nu;
            PairSetup P = pair_setup<HAS_Y>(gc, sub[n], xs, ys, zs, q0);
            PhaseRun R = phase_run(P, q0);
            const float kt = TAB ? P.kap * gc.tab_inv_dx : 0.0f;
            const float t0 = TAB ? gc.tab_x0 * gc.tab_inv_dx : 0.0f;
#pragma unroll
            for (int j = 0; j < kPQB; ++j) {
                const float q = q0 + (float)j;
                const float m = sinc_f<NARROW>(q * P.xb);
                float2 d;
                if (TAB) {
                    const float tt = fmaf(q, kt, -t0);
                    const float fl = floorf(fminf(fmaxf(tt, 0.0f), (float)gc.tab_n - 0.5f));
                    const int ii = (int)fl;
                    const float u = tt - fl;
                    d = cubic_piece(__ldg(dtab + 2 * ii), __ldg(dtab + 2 * ii + 1), u);
                    if (!(u >= 0.0f && u <= 1.0f)) d = delta_f<false>(gc, P, q);
                } else {
                    d = delta_f<HAS_Y>(gc, P, q);
                }
                const float er = R.zr * m, ei = R.zi * m;
                const float gr = er * d.x - ei * d.y, gi = er * d.y + ei * d.x;
                const float2 w = wtt[j * N + e];
                ar[j] = fmaf(w.x, gr, fmaf(-w.y, gi, ar[j]));
                ai[j] = fmaf(w.x, gi, fmaf(w.y, gr, ai[j]));
                const float nzr = fmaf(R.zr, R.wr, -R.zi * R.wi);
                R.zi = fmaf(R.zr, R.wi, R.zi * R.wr);
                R.zr = nzr;
            }
        }
#pragma unroll
        for (int j = 0; j < kPQB; ++j)
            if (jb + j < jend) power = fmaf(ptx2[jb + j], ar[j] * ar[j] + ai[j] * ai[j], power);
    }
    if (!live) return;
    if (ppart) ppart[((size_t)blockIdx.z * gridDim.y + t) * npts + i] = power;   // partial sum
    else prms[(size_t)t * npts + i] = sqrtf(dw * power);
}

// prms[t][i] = sqrt(dw sum_c ppart[c][t][i]), chunks summed in a fixed order.
__global__ void k_pfield_finish(const float *__restrict__ ppart, int n_chunks, int64_t n,
                                float dw, float *__restrict__ prms) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float a = 0.f;
        for (int c = 0; c < n_chunks; ++c) a += ppart[(size_t)c * n + i];
        prms[i] = sqrtf(dw * a);
    }
}

// Frequency chunks (a multiple of kPQB midpoints each): the count minimising the modelled
// makespan, waves of resident blocks x (midpoints per chunk + the per-chunk geometry setup,
// about two midpoints' work), so that the last wave is not a small remainder (with one
// chunk per 150 midpoints the L11-5v grid ran 2.08 waves of two blocks per SM and its SMs
// were active 79 % of the time).
using PfieldKernel = void (*)(const GreenConst, const SubElem *, const float *, const float *,
                              const float *, int64_t, int, int, const float2 *, const float *,
                              float, float *, const float4 *, int, float *);

static PfieldKernel pfield_kernel(const simus_plan *p, const GreenConst &gc, bool has_y) {
    const bool narrow = gc.narrow == 1;
    const bool tab = !has_y && p->d_dtab && gc.tab_n > 0;
    return has_y ? (narrow ? k_pfield<true, true, false> : k_pfield<true, false, false>)
         : tab   ? (narrow ? k_pfield<false, true, true> : k_pfield<false, false, true>)
                 : (narrow ? k_pfield<false, true, false> : k_pfield<false, false, false>);
}

static size_t pfield_smem(const simus_plan *p) {
    return sizeof(SubElem) * p->M + sizeof(float2) * (size_t)kPQB * p->N;
}

static void pfield_split(const simus_plan *p, PfieldKernel kern, int T, int64_t npts, int nf,
                         int &n_fc, int &fchunk) {
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, kPThreads, pfield_smem(p)) != cudaSuccess)
        bps = 1;
    const int64_t slots = (int64_t)p->num_sms * std::max(bps, 1);
    const int64_t pblocks = ((npts + kPThreads - 1) / kPThreads) * T;
    n_fc = 1;
    fchunk = (nf + kPQB - 1) / kPQB * kPQB;
    double best = 1e300;
    for (int n = 1; n <= 64; ++n) {
        const int fc = ((nf + n - 1) / n + kPQB - 1) / kPQB * kPQB;
        const int ne = (nf + fc - 1) / fc;
        if (ne != n) continue;                     // the same split as a smaller n
        const int64_t waves = (pblocks * ne + slots - 1) / slots;
        const double cost = (double)waves * (fc + 2);
        if (cost < best) { best = cost; n_fc = ne; fchunk = fc; }
    }
}

int pfield_fchunks(const simus_plan *p, const GreenConst &gc, int T, int64_t npts, int nf, bool has_y) {
    const PfieldKernel kern = pfield_kernel(p, gc, has_y);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pfield_smem(p));
    int n_fc, fchunk;
    pfield_split(p, kern, T, npts, nf, n_fc, fchunk);
    return n_fc;
}

int launch_pfield(const simus_plan *p, const GreenConst &gc, const simus_tx *tx, int64_t npts,
                  const float *x, const float *y, const float *z, int nf, int j0, float2 *wt,
                  const float *ptx2, float dw, float *prms, float *ppart, cudaStream_t st) {
    const int T = tx->n_tx;
    {
        int64_t total = (int64_t)T * nf * p->N;
        int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)p->num_sms * 8);
        k_pfield_weights<<<std::max(blocks, 1), 256, 0, st>>>(T, p->N, nf, j0, gc.df, tx->delays,
                                                               tx->apod, wt);
        count_launches(1);
        int rc = check_cuda(cudaGetLastError(), "k_pfield_weights launch");
        if (rc) return rc;
    }
    const size_t smem = pfield_smem(p);
    const PfieldKernel kern = pfield_kernel(p, gc, y != nullptr);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return check_cuda(e, "k_pfield smem attribute");
    int n_fc, fchunk;
    pfield_split(p, kern, T, npts, nf, n_fc, fchunk);
    dim3 grid((unsigned)((npts + kPThreads - 1) / kPThreads), T, n_fc);
    kern<<<grid, kPThreads, smem, st>>>(gc, p->d_sub, x, y, z, npts, nf, j0, wt, ptx2, dw, prms,
                                        p->d_dtab, fchunk, n_fc > 1 ? ppart : nullptr);
    count_launches(1);
    int rc = check_cuda(cudaGetLastError(), "k_pfield launch");
    if (rc || n_fc == 1) return rc;
    const int64_t n = (int64_t)T * npts;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)p->num_sms * 8);
    k_pfield_finish<<<blocks, 256, 0, st>>>(ppart, n_fc, n, dw, prms);
    count_launches(1);
    return check_cuda(cudaGetLastError(), "k_pfield_finish launch");
}

}  // namespace simus
