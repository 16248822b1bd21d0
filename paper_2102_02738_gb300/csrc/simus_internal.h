// simus_internal.h -- structures shared by the host API and the kernels of the CUDA
// library (not part of the C ABI).
#pragma once

#include <cstdint>
#include <vector>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/simus.h"

namespace simus {

// Per-plan constants of the Green's term, passed to kernels by value.  Bin q has
// frequency f_q = q * df; every per-bin quantity is stored "per unit q".
struct GreenConst {
    int32_t N;        // elements
    int32_t nu;       // sub-elements per element
    int32_t M;        // nu * N
    int32_t q_lo;     // first kept bin
    int32_t nq;       // number of kept bins
    int32_t nt;       // RF samples
    int32_t baffle;   // SIMUS_BAFFLE_*
    int32_t two_d;    // 1: 2-D model (Section V): amplitude 1/sqrt(r), delta = 1
    float Kh, Kl;     // df / c as a double-float [cycles per metre per bin]
    float k1;         // 2 pi df / c [rad per metre per bin]
    float k1b;        // k1 * b / nu: sinc argument per bin per unit sin(theta)
    float kh;         // k1 / 2: Im(alpha_g) per bin per unit (1/R_f - 1/r)
    float inv_rf;     // 1 / R_f (0 without lens)
    float att2;       // (alpha_dB / 8.69) * df * 1e-4 * log2(e): base-2 absorption per bin per metre
    float zeta;       // Eq. 39
    float h;          // element height (delta is evaluated as h * f(h^2 alpha))
    float h2;         // h^2
    int32_t narrow;   // sinc range at every kept bin: 1 |k b / nu| <= 3.2, 2 <= 4.6, 0 beyond
    int32_t tab_n;    // intervals of the delta table (0: none)
    float tab_x0;     // delta table: first abscissa of x = h^2 (k/2)(1/R_f - 1/r)
    float tab_inv_dx; // 1 / spacing
    double df;        // fs / nt [Hz]
};

// Sub-element record: centroid as double-float pairs and the normal's angle.
struct __align__(16) SubElem {
    float xh, xl, zh, zl;   // x_c = xh + xl, z_c = zh + zl
    float cpsi, spsi;       // normal (sin psi, cos psi); local frame rotation
    float l0, z0;           // the centroid rotated into that frame (x_c cpsi - z_c spsi,
                            // x_c spsi + z_c cpsi), for the FP32 setup of the TC path
};

}  // namespace simus

struct simus_plan {
    simus_probe probe;
    simus_medium medium;
    int32_t nt = 0, path = 0, nu = 0, N = 0, M = 0, q_lo = 0, q_hi = 0, nq = 0;
    int device = 0;
    int num_sms = 0;
    simus::GreenConst gc{};
    simus::SubElem *d_sub = nullptr;  // [M]
    float2 *d_H = nullptr;            // [nq] transfer S_P S_T at the kept bins
    int *d_err = nullptr;             // device-side error flag (bounded waits)
    float4 *d_dtab = nullptr;         // [2 gc.tab_n] delta/h cubic pieces
    float4 *d_dtab_q = nullptr;       // [2 gc.tab_n] the same as quadratic pieces (FP16 tensor-core kernels)
    void *d_idft_tw = nullptr;        // blocked BF16 twiddles of the tensor-core iDFT (tensor-core paths)
    void *d_work = nullptr;           // workspace
    size_t work_bytes = 0;
    void *h_stage = nullptr;          // pinned host staging of work descriptors
    size_t h_stage_bytes = 0;
    cudaEvent_t ev_stage = nullptr;   // recorded after the staging copy; guards reuse
    bool stage_pending = false;
    int items_per_sm = 4;             // tensor-core path tuning (simus_tuning)
    int max_bins = 4;
    int pair_mode = 2;
    int delta_table = 1;
    int tile_buffers = 2;
    int depth_order = 1;              // tensor-core path: scatterers reordered by depth first
    int tensor_idft = 1;              // tensor-core path: iDFT on the tensor cores (if d_idft_tw)
    int chunks = 0;
    bool profiling = false;
    bool stage_used[SIMUS_N_STAGES] = {};
    cudaEvent_t ev[2 * SIMUS_N_STAGES] = {};
};

namespace simus {

// Workspace helper: returns a device pointer with at least `bytes`, growing the
// plan's workspace (synchronising the device before a reallocation).
int workspace(simus_plan *plan, size_t bytes, void **ptr);

// Host part of a plan (validation, nu, kept bins, Green's constants; no device work)
// and its two tables (sub-element records [M], transfer values [nq]).
int plan_setup_host(const simus_probe *probe, const simus_medium *medium, int32_t n_samples,
                    int32_t path, simus_plan *p);
void plan_fill_tables(const simus_plan *p, SubElem *sub, float2 *H);
// Cubic Hermite table of delta/h over the x = h^2 Im(alpha_g - B_g/h^2) reachable by the
// plan's bins for scatterers at least 2 mm from a sub-element (spacing 0.5, relative error
// <= 2.3e-6), as power-basis pieces (two float4 per interval); sets gc.tab_x0, tab_inv_dx,
// tab_n = intervals (0 if it would exceed 2048); tab_q: the quadratic through each interval's
// ends and midpoint in the same layout (c3 = 0; relative error <= 1.9e-5), for the FP16
// tensor-core kernels.
void plan_delta_table(simus_plan *p, std::vector<float4> &tab, std::vector<float4> &tab_q);
GreenConst green_const(const simus_probe &pr, const simus_medium &md, int N, int nu, double df,
                       double q_max);

// RMS pressure field (Eq. 22, Eq. 41-42) on midpoint frequencies (j0 + jj + 1/2) gc.df,
// jj < nf; wt: workspace [T][nf][N]; ptx2: device [nf] = |P_Tx|^2.
// The frequencies are split into pfield_fchunks() chunks (chosen with the occupancy of the
// kernel variant that has_y and gc select); ppart: workspace [chunks][T][npts] for their
// partial sums (unused for one chunk).
int pfield_fchunks(const simus_plan *p, const GreenConst &gc, int T, int64_t npts, int nf, bool has_y);
int launch_pfield(const simus_plan *p, const GreenConst &gc, const simus_tx *tx, int64_t npts,
                  const float *x, const float *y, const float *z, int nf, int j0, float2 *wt,
                  const float *ptx2, float dw, float *prms, float *ppart, cudaStream_t st);

// Tracing: an NVTX range around each entry point (visible to Nsight tools, free
// otherwise), events around a stage (no-ops unless profiling is enabled) and the
// process-wide launch counter.
struct NvtxScope {
    explicit NvtxScope(const char *name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope &) = delete;
    NvtxScope &operator=(const NvtxScope &) = delete;
};
void stage_begin(simus_plan *plan, int stage, cudaStream_t st);
void stage_end(simus_plan *plan, int stage, cudaStream_t st);
void count_launches(int n);

// Error reporting (thread-local message).
int fail(int code, const char *fmt, ...);
int check_cuda(cudaError_t e, const char *what);

// ---- kernel launchers (each returns SIMUS_OK or an error code) ----------------
// Transmit weights C[t][k][e] = W_te exp(i w_q dtau_te), q = q_lo + k.
int launch_tx_weights(const simus_plan *p, const simus_tx *tx, float2 *cw, cudaStream_t st);

// Plain FP32 path: partial spectra part[chunk][t][e][k] (no transfer factor).
struct PlainGeom { int QB, SB, n_qtiles, n_chunks; int64_t chunk_len; size_t smem; };
PlainGeom plain_geometry(const simus_plan *p, int T, int64_t S);
int launch_plain(const simus_plan *p, const PlainGeom &g, const simus_scat *sc, int T,
                 const float2 *cw, float2 *part, cudaStream_t st);
// Plain FP32 path for T >= 2: the Green's tile generated once per bin and contracted
// against every transmit (k_plain_mt.cu); SB = 0 when its operands do not fit shared
// memory (T N beyond ~6,000).  Same partial-spectrum layout as launch_plain.
PlainGeom plain_mt_geometry(const simus_plan *p, int T, int64_t S);
int launch_plain_mt(const simus_plan *p, const PlainGeom &g, const simus_scat *sc, int T,
                    const float2 *cw, float2 *part, cudaStream_t st);

// Batched tensor-core path (FP16 / BF16 operands, FP32 accumulation).
// A simulation ("unit") is cut into work items of QB bins x tiles_per_chunk scatterer
// tiles; its transmits are contracted in G groups of TG inside every item, so that the
// Green's tile is generated once whatever the number of transmits.  The shapes are
// chosen per simulation so that one CTA's operands fit shared memory and its
// accumulators (D1 + QB G mh slices of nN columns) fit the 512 tensor-memory columns.
struct TcShape {
    bool ok;
    int Np;              // elements padded to 8 (<= 256)
    int TG, n_groups;    // transmits per group, groups
    int nN;              // GEMM N of a group: 2 TG padded to 16
    int mh;              // receive GEMM M-halves: 1 (Np <= 128) or 2
    int pair;            // bins per generation pass - 1 (0, 1, 2)
    int nbuf;            // shared-memory tile buffers (1, 2); the other bins of a pass
                         // wait in tensor-memory stash slots
    int tab_n;           // delta-table intervals staged in shared memory (0: direct delta)
    int QB;              // bins per work item
    int n_btiles;
    int64_t n_tiles;     // scatterer tiles of 128
    int tiles_per_chunk, n_chunks;
    size_t smem;         // dynamic shared memory of the kernel for this shape
    size_t b1_bytes;     // B1 operand images of one group: nq * nN * 2Np * 2
};
// items_per_sm: target number of work items per SM over the whole launch (tuning).
TcShape tc_shape(const simus_plan *p, int T, int64_t S, double work_share, int items_per_sm);
// Scatterers of one simulation in distance-to-array order (k_order.cu): out arrays of
// in->n floats (yo only when in->y), scratch of order_scratch_bytes(in->n).
size_t order_scratch_bytes(int64_t S);
int launch_order(const simus_scat *in, float R, int *scratch, float *xo, float *yo, float *zo,
                 float *rco, cudaStream_t st);

// One simulation, as the kernel reads it.
struct TcUnit {
    GreenConst gc;
    const SubElem *sub;
    const float4 *dtab;           // delta/h pieces [2 gc.tab_n]: quadratic for FP16, cubic for split
                                  // BF16 (gc.tab_n = 0: direct)
    const float *x, *y, *z, *rc;
    const float *delays, *apod;   // of the whole simulation, [T][N]
    int64_t S, n_tiles;
    int T, G, TG;                 // simulation transmits, transmit groups, group size
    int Np, nN, QB, mh, pair;
    int n_btiles, n_chunks, tiles_per_chunk;
    int nbuf;                     // shared-memory tile buffers
    int64_t item0;                // first global item of this unit
    uint16_t *b1img;              // [nq][G][nN * 2Np]
    float2 *part;                 // [n_chunks][T][N][nq] of the simulation
};
// Launch the B1 image kernels of every unit and the persistent tensor-core kernel over
// all items.  d_units: device copy of units (n_units), counter: zeroed device int.
int launch_tc_units(const TcUnit *h_units, const TcUnit *d_units, int n_units, int64_t n_items,
                    size_t smem, bool bf16, bool has_y, int sinc_mode, bool linear, int num_sms,
                    int *counter, int *err, cudaStream_t st);

// Failure-detection self-test: a bounded wait on a barrier phase nothing completes.
int launch_selftest_timeout(int max_polls, int *err, cudaStream_t st);

// Adjoint (gradient) path, FP32.
struct GradGeom {
    bool ok;             // T * N <= 2048 and the shared-memory tiles fit
    int n_qtiles, n_chunks;
    int SB;              // scatterers per group (16, or 8 where shared memory is short)
    bool tab;            // delta from the plan's table (staged in shared memory)
    int64_t chunk_len;
    size_t smem;
};
GradGeom grad_geometry(const simus_plan *p, int T, int64_t S);
int launch_adjoint_dft(const simus_plan *p, const float *drf, int T, float2 *lam, cudaStream_t st);
int launch_grad(const simus_plan *p, const GradGeom &g, const simus_scat *sc, int T,
                const float2 *cw, const float2 *lam, float *gpart, float2 *bpart, cudaStream_t st);
int launch_grad_finish(const simus_plan *p, const GradGeom &g, int T, int64_t S, const float *gpart,
                       const float2 *bpart, const float2 *cw, float *g_rc, float *g_x, float *g_z,
                       float *g_delays, cudaStream_t st);

// Sum partial spectra over chunks and multiply by H: spec[c][k] (c = t * N + e).
int launch_reduce_spectrum(const simus_plan *p, const float2 *part, int n_chunks, int n_chan,
                           float2 *spec, cudaStream_t st);

// rf[c][j] = Re sum_k spec[c][k] e^{-2 pi i (q_lo + k) j / Nt}.
int launch_idft(const simus_plan *p, const float2 *spec, int n_chan, float *rf, cudaStream_t st);
// The same on the tensor cores (split-BF16 operands, FP32 accumulation): spectra blocked
// into blocks_ws (idft_tc_operand_bytes), then one GEMM with p->d_idft_tw, which
// build_idft_tc_twiddles fills (idft_tc_twiddle_bytes).
size_t idft_tc_twiddle_bytes(int nt, int nq);
size_t idft_tc_operand_bytes(int n_chan, int nq);
int build_idft_tc_twiddles(const simus_plan *p, void *tw, cudaStream_t st);
int launch_idft_tc(const simus_plan *p, const float2 *spec, int n_chan, float *rf, void *blocks_ws,
                   cudaStream_t st);

}  // namespace simus
