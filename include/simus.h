/*
 * simus.h -- C ABI of the GB300 (sm_103a) SIMUS RF library.
 *
 * The library evaluates the linear frequency-domain model of Garcia, "SIMUS: an
 * open-source simulator for medical ultrasound imaging. Part I: theory & examples"
 * (arXiv:2102.02738):
 *   - Green's term of one sub-element (Eq. 17/19/20 with Eq. 39 and Eq. 40),
 *   - array field / transmit sum (Eq. 22, Eq. 29),
 *   - reciprocity receive term, scatterer sum and sub-element sum (Eq. 30-33),
 *   - RF spectrum S_P S_T P^e (Eq. 28, Eq. 34) and its inverse DFT to time signals (Eq. 1),
 *   - RMS pressure field (Eq. 41-42).
 *
 * Conventions (SI units throughout): x azimuth, y elevation, z depth; the array is
 * centred at x = 0 (convex arrays: centre of curvature at (0, -radius)); t = 0 is the
 * firing of an element with zero delay; the exp(-i w t) time convention of Eq. 1.
 *
 * Ownership: every array argument is caller-owned DEVICE memory (float32, contiguous,
 * 4-byte aligned) unless stated otherwise; the library never frees it.  A plan owns
 * its constant tables and a workspace that grows on demand and is freed by
 * simus_plan_destroy.
 *
 * Errors: calls return SIMUS_OK (0) or a negative SIMUS_ERR_* code and never throw
 * across the ABI; simus_last_error() returns a message for the calling thread's last
 * failure.  Arguments are validated on the host before any launch.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 * stream).  Calls enqueue their kernels on it and return without synchronising; the
 * outputs are valid once the stream reaches that point.  A plan must not be used by
 * two calls that overlap in time (its workspace is shared).
 */
#ifndef SIMUS_H
#define SIMUS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SIMUS_OK 0
#define SIMUS_ERR_ARG (-1)         /* invalid argument (message says which)          */
#define SIMUS_ERR_CUDA (-2)        /* a CUDA runtime call or a launch failed         */
#define SIMUS_ERR_OOM (-3)         /* device allocation of the workspace failed      */
#define SIMUS_ERR_TIMEOUT (-4)     /* a bounded device wait gave up                  */
#define SIMUS_ERR_UNSUPPORTED (-5) /* valid request the library does not implement   */

/* Contraction path chosen at plan creation.
 *   PLAIN_F32 : Green's terms and every contraction in FP32 on the CUDA cores; with
 *               several transmits a Green's tile is generated once per bin and
 *               contracted against every transmit where its operands fit shared memory
 *               (T N up to ~6,000), otherwise it is recomputed for each transmit.
 *   TC_F16    : Green's terms generated once per (bin, scatterer, element) in FP32,
 *               rounded to FP16, and both contractions (transmit sum Eq. 29 and
 *               receive sum Eq. 32) run on the tcgen05 tensor cores with FP32
 *               accumulation in tensor memory.
 *   TC_BF16   : as TC_F16 with BF16 operands, each FP32 value carried as a BF16 leading
 *               part and a BF16 remainder and each GEMM formed as three products
 *               (hi hi' + hi rem' + rem hi'), which keeps ~16 significant bits; arrays of
 *               up to 176 elements (wider ones return SIMUS_ERR_UNSUPPORTED). */
#define SIMUS_PATH_PLAIN_F32 0
#define SIMUS_PATH_TC_F16 1
#define SIMUS_PATH_TC_BF16 2

/* Baffle of Eq. 39. */
#define SIMUS_BAFFLE_SOFT 0
#define SIMUS_BAFFLE_RIGID 1
#define SIMUS_BAFFLE_IMPEDANCE 2

/* Transmit pulse window (Section III). */
#define SIMUS_PULSE_RECT 0 /* Eq. 25: rectangular-windowed sine              */
#define SIMUS_PULSE_HANN 1 /* the same sine under a Hann window of width T   */

/* Uniform linear or convex 1-D probe (Section II, Fig. 2, Eq. 21, Eq. 24). */
typedef struct simus_probe {
    int32_t n_elements; /* N >= 1                                                   */
    int32_t n_sub;      /* nu sub-elements per element; 0 = Eq. 21 with lambda_min at
                           the upper -6 dB edge c / (fc (1 + frac_bw / 2))             */
    int32_t baffle;     /* SIMUS_BAFFLE_*                                            */
    int32_t two_d;      /* 0: 3-D model (Eq. 17, elevation factor delta of Eq. 16);
                           1: the 2-D x-z model of Section V (Eq. 36-38): Green's term
                           exp(i(k + i k_a) r)/sqrt(r) D(theta, k), height and
                           elev_focus unused, scatterer and field-point y must be NULL */
    double pitch;       /* p [m] > 0                                                 */
    double width;       /* element width 2b [m], 0 < width <= pitch                   */
    double height;      /* element height h [m] > 0 (3-D)                              */
    double elev_focus;  /* elevation focus R_f [m] > 0; +INFINITY = no lens           */
    double radius;      /* convex radius of curvature [m]; 0 = linear array           */
    double fc;          /* centre frequency [Hz] > 0                                  */
    double frac_bw;     /* pulse-echo fractional bandwidth w_b / w_c, in (0, 2)       */
    double zeta;        /* medium / baffle impedance ratio (SIMUS_BAFFLE_IMPEDANCE)   */
} simus_probe;

/* Homogeneous medium and sampling (Section III, Eq. 40). */
typedef struct simus_medium {
    double c;            /* speed of sound [m/s] > 0                                  */
    double alpha_db;     /* attenuation [dB/cm/MHz] >= 0, linear in f (Eq. 40)        */
    double fs;           /* RF sampling frequency [Hz] > 0                            */
    int32_t pulse;       /* SIMUS_PULSE_*                                             */
    int32_t reserved;    /* must be 0                                                 */
    double pulse_cycles; /* n_lambda of Eq. 25 > 0                                    */
} simus_medium;

/* Transmit sequence (Eq. 20, Eq. 22): per-element delays and apodisation. */
typedef struct simus_tx {
    int32_t n_tx;        /* T >= 1                                                    */
    int32_t reserved;
    const float *delays; /* device [T][N] seconds, delay dtau of each element          */
    const float *apod;   /* device [T][N] apodisation W of each element               */
} simus_tx;

/* Point scatterers (Section IV-A), structure of arrays. */
typedef struct simus_scat {
    int64_t n;           /* S >= 0                                                    */
    const float *x;      /* device [S] azimuth [m]                                    */
    const float *y;      /* device [S] elevation [m], or NULL for y = 0               */
    const float *z;      /* device [S] depth [m]                                      */
    const float *rc;     /* device [S] reflection coefficients R_s                    */
} simus_scat;

/* Read-only description of a plan. */
typedef struct simus_plan_info {
    int32_t n_elements;  /* N                                                         */
    int32_t n_sub;       /* nu actually used (Eq. 21 resolved)                        */
    int32_t n_samples;   /* Nt                                                        */
    int32_t path;        /* SIMUS_PATH_*                                              */
    int32_t q_lo, q_hi;  /* kept frequency bins f_q = q fs / Nt, q in [q_lo, q_hi]     */
    int32_t n_bins;      /* q_hi - q_lo + 1                                           */
    int32_t reserved;
    double df;           /* bin spacing fs / Nt [Hz]                                  */
} simus_plan_info;

typedef struct simus_plan simus_plan;

/* Create a plan: resolves nu (Eq. 21), the sub-element centroids (Eq. 24; convex: on
 * the arc, centre of curvature (0, -radius), pitch measured along the arc), the
 * kept frequency bins -- the contiguous range of 1 <= q < Nt/2 on which the transfer
 * magnitude |S_P S_T| (Eq. 25-28, Eq. 34) is at least 1e-5 of its maximum -- and the
 * transfer values H_q = S_P(w_q) S_T(w_q).  n_samples is the RF length Nt (>= 8).
 * Host-only apart from uploading the tables to the current device; plans of the
 * tensor-core paths also build the inverse DFT's twiddles on that device (one kernel,
 * then a device synchronisation): ceil(Nt/128) * ceil(2 n_bins/32) * 16 KiB of device
 * memory held by the plan (none where that would exceed 1 GiB: their iDFT then runs on
 * the CUDA cores).  All of it is freed by simus_plan_destroy.
 * Returns SIMUS_ERR_ARG on invalid parameters, SIMUS_ERR_CUDA/OOM on upload failure. */
int simus_plan_create(const simus_probe *probe, const simus_medium *medium,
                      int32_t n_samples, int32_t path, simus_plan **out);

/* Destroy a plan and its device memory (synchronises the device first). NULL is ok. */
void simus_plan_destroy(simus_plan *plan);

/* Fill *info. */
int simus_plan_get_info(const simus_plan *plan, simus_plan_info *info);

/* An even RF length covering the longest two-way path: the smallest even
 * Nt >= fs (2 r_max / c + tau_max + 8 / fc), where r_max bounds the distance from any
 * sub-element to any scatterer and tau_max the largest transmit delay.  Host only.
 * Returns Nt, or SIMUS_ERR_ARG. */
int32_t simus_default_nt(const simus_probe *probe, const simus_medium *medium,
                         double r_max, double tau_max);

/* RF signals (Eq. 29-34, then rf[t][e][j] = Re sum_q X_q e^{-2 pi i q j / Nt} over the
 * kept bins, the exp(-i w t) convention of Eq. 1, no scale factor).
 * rf: device [T][N][Nt] float32, fully overwritten.  Scatterers with cos(theta) <= 0
 * for a sub-element receive D = 0 from it (behind the aperture).  S = 0 gives zeros. */
int simus_rf(simus_plan *plan, const simus_tx *tx, const simus_scat *scat, float *rf,
             void *stream);

/* RF spectra before the inverse DFT: spec[t][e][k] = X_{q_lo + k}(e, t) = S_P S_T P^e
 * (Eq. 33-34) as interleaved (re, im) float32, device [T][N][n_bins][2]. */
int simus_rf_spectrum(simus_plan *plan, const simus_tx *tx, const simus_scat *scat,
                      float *spec, void *stream);

/* RMS pressure field (Eq. 22, Eq. 41-42) of each transmit at each point:
 * P(X, w) = S_P sqrt(S_T) sum_n W_n g_n(X) e^{i w dtau_n},
 * prms[t][i] = sqrt(dw sum_j |P(X_i, w_j)|^2), w_j = (j + 1/2) dw, dw = 2 w_c / n_freq,
 * j = 0..n_freq-1 (midpoint sum over [0, 2 w_c]).  x, y (or NULL), z: device [n_pts];
 * prms: device [T][n_pts] float32. */
int simus_pfield(simus_plan *plan, const simus_tx *tx, int64_t n_pts, const float *x,
                 const float *y, const float *z, int32_t n_freq, float *prms, void *stream);

/* Number of midpoint frequencies of Eq. 42 for points within r_max of every
 * sub-element and delays up to tau_max: N_f = ceil(2 w_c / dw_max) with
 * dw_max = 2 pi / (r_max / c + tau_max).  Host only. */
int32_t simus_pfield_nfreq(const simus_probe *probe, const simus_medium *medium,
                           double r_max, double tau_max);

/* Gradient of a loss through simus_rf (not in the paper): given drf = dL/drf,
 * device [T][N][Nt], writes the vector-Jacobian products
 *   g_rc[s] = dL/dR_s, g_x[s] = dL/dx_s, g_z[s] = dL/dz_s (device [S]) and
 *   g_delays[t][e] = dL/d dtau_{t,e} (device [T][N]);
 * any output may be NULL.  Green's terms are recomputed, not stored.  Requires
 * scat->y == NULL (scatterers in the azimuth plane); FP32 on the CUDA cores. */
int simus_rf_grad(simus_plan *plan, const simus_tx *tx, const simus_scat *scat,
                  const float *drf, float *g_rc, float *g_x, float *g_z, float *g_delays,
                  void *stream);

/* Many independent simulations in one persistent launch: simulation i uses plans[i],
 * tx[i], scat[i] and writes rf[i] (device [T_i][N_i][Nt_i]).  All plans must share
 * one path.  Work is scheduled over (simulation, bin tile, scatterer chunk) items. */
int simus_batch_rf(int32_t n_sims, simus_plan *const *plans, const simus_tx *tx,
                   const simus_scat *scat, float *const *rf, void *stream);

/* As simus_batch_rf, but writes each simulation's RF spectrum before the inverse DFT
 * (Eq. 33-34), as simus_rf_spectrum does: spec[i] is device [T_i][N_i][n_bins_i][2]
 * float32 (interleaved re, im).  The work split over the launch is the same as
 * simus_batch_rf's for the same batch. */
int simus_batch_rf_spectrum(int32_t n_sims, simus_plan *const *plans, const simus_tx *tx,
                            const simus_scat *scat, float *const *spec, void *stream);

/* Wait for all work queued on the plan's device, then report a failure that an earlier
 * asynchronous call on this plan met on the device: SIMUS_ERR_TIMEOUT if a bounded wait
 * inside a kernel gave up (that call's outputs are invalid; the flag is then cleared),
 * SIMUS_ERR_CUDA for an asynchronous CUDA error, else SIMUS_OK. */
int simus_plan_check(simus_plan *plan);

/* Failure-detection self-test (a diagnostic; the paper has no counterpart).  Enqueues one
 * block that waits, with the same bounded mbarrier wait the tensor-core kernel uses, for a
 * barrier phase that nothing ever completes; the wait gives up after max_polls polls
 * (1 <= max_polls <= 2^24; each poll may suspend the thread for a short, hardware-defined
 * time) and records SIMUS_ERR_TIMEOUT in the plan's error flag, exactly as a stalled
 * tensor-core work item would.  The next simus_plan_check then returns SIMUS_ERR_TIMEOUT
 * (and clears the flag) and the device stays usable.  Returns SIMUS_ERR_ARG for a NULL
 * plan or max_polls out of range, SIMUS_ERR_CUDA if the launch fails, else SIMUS_OK. */
int simus_plan_selftest_timeout(simus_plan *plan, int32_t max_polls, void *stream);

/* Per-stage timing of the calls made on a plan (tracing).  With profiling enabled,
 * each entry point records CUDA events around its kernels on the call's stream;
 * simus_plan_get_timings waits for them and writes the durations in milliseconds of
 * the LAST call's stages to ms[0..SIMUS_N_STAGES-1] (0 for stages the call did not
 * run).  Stages: 0 transmit weights, 1 Green's terms + contraction, 2 chunk reduction
 * with the transfer factor, 3 inverse DFT, 4 pfield, 5 adjoint DFT, 6 gradient,
 * 7 other. */
#define SIMUS_N_STAGES 8
int simus_plan_set_profiling(simus_plan *plan, int32_t enable);
int simus_plan_get_timings(simus_plan *plan, float *ms);

/* Launch shapes of the tensor-core path (tuning; results do not depend on them beyond
 * FP32 summation order, except delta_table, which trades the direct Eq. 16-18 evaluation
 * for a cubic Hermite table of relative error <= 2.3e-6).  A field < 0 (chunks: <= 0)
 * selects the library's default; simus_plan_get_tuning reports the values in force.
 *   items_per_sm  batches: work items per SM the scatterer chunking aims at (default 4)
 *   max_bins      frequency bins per work item, upper bound (default 4; tensor memory
 *                 may allow fewer)
 *   pair          bins generated per pass from one geometry setup, minus one: 2 three
 *                 (two shared-memory tile buffers and a tensor-memory stash; default),
 *                 1 two (two buffers), 0 one; the largest that fits at most this
 *   delta_table   1: delta from the table where Y = 0 (default), 0: direct evaluation
 *   tile_buffers  shared-memory buffers for the Green's tiles of a pass, at most: 2 (the
 *                 default) or 1 (later bins of a pass wait in the tensor-memory stash)
 *   chunks        single simulations: scatterer chunks per bin tile (default: chosen by a
 *                 makespan model over the SMs)
 *   depth_order   1: each simulation's scatterers are copied in order of their distance
 *                 to the array into the workspace before the launch (default; the sum
 *                 over scatterers is the same up to rounding, and tiles of similar depth
 *                 take the same delta-table paths), 0: the caller's order
 *   tensor_idft   1: the inverse DFT of Eq. 1 runs on the tensor cores as a product of
 *                 split-BF16 operands (each value a BF16 leading part and a BF16
 *                 remainder, three products, FP32 accumulation; about 2^-16 relative per
 *                 term) where the plan holds its twiddles (plans whose blocked twiddles
 *                 take at most 1 GiB; default), 0: on the CUDA cores in FP32
 * The project's autotuner (paper_2102_02738_gb300/autotune.py) times candidates through
 * these calls and caches the fastest per problem shape.
 * Returns SIMUS_ERR_ARG for a NULL plan or values out of range (max_bins > 64,
 * items_per_sm > 1024, chunks > 65536, pair > 2, delta_table > 1, tile_buffers > 2,
 * depth_order > 1, tensor_idft > 1). */
typedef struct simus_tuning {
    int32_t items_per_sm;
    int32_t max_bins;
    int32_t pair;
    int32_t delta_table;
    int32_t chunks;
    int32_t tile_buffers;
    int32_t depth_order;
    int32_t tensor_idft;
} simus_tuning;
int simus_plan_set_tuning(simus_plan *plan, const simus_tuning *tuning);
int simus_plan_get_tuning(const simus_plan *plan, simus_tuning *tuning);

/* Number of kernels this library has launched in the process so far (tracing). */
int64_t simus_kernel_launches(void);

/* ---- Allocation-free RF (the paper has no counterpart; an interface for callers) -----
 * simus_rf_noalloc computes what simus_rf computes on a SIMUS_PATH_PLAIN_F32 plan built
 * from the same probe, medium and n_samples, without allocating device memory.  It is
 * for callers that cannot allocate: latency-critical loops that must not enter an
 * allocator (which may synchronise the device), and plug-ins whose host application
 * owns the device memory.  Such callers cannot create a plan, so the probe and medium are
 * passed directly; the caller still passes the input and output arrays (device memory,
 * as for simus_rf).  Every temporary lives in one fixed device array of
 * SIMUS_NOALLOC_SCRATCH_BYTES that each device loading the library holds until the
 * process exits; problems whose temporaries (sub-element table, transfer values,
 * transmit weights T*bins*N*8 bytes, spectrum T*N*bins*8 bytes and at least one partial
 * spectrum of the same size) do not fit are rejected with SIMUS_ERR_ARG before any
 * device work.  The first call on each device resolves the array's address
 * (cudaGetSymbolAddress) with that device current.  The call uploads its two small
 * tables from host memory with stream-ordered copies, so it cannot be recorded into a
 * CUDA graph (a replay would read whatever a later call left in that host memory): a
 * stream that is being captured is rejected with SIMUS_ERR_ARG before any device work.
 * All calls share the array and each keeps the previous call's contents; calls whose
 * kernels overlap on the GPU race on it (host threads are serialised, streams are not).
 * No cudaMalloc, cudaFree or allocating library routine is called. */
#define SIMUS_NOALLOC_SCRATCH_BYTES (32u << 20)
int simus_rf_noalloc(const simus_probe *probe, const simus_medium *medium, int32_t n_samples,
                     const simus_tx *tx, const simus_scat *scat, float *rf, void *stream);

/* Message of the calling thread's last error ("" if none). */
const char *simus_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SIMUS_H */
