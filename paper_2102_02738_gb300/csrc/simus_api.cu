// simus_api.cu -- host side of the C ABI (include/simus.h): argument validation, the
// plan (sub-element geometry, kept bins, transfer values, Green's constants), the
// workspace, and the launch sequence of each entry point.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "simus_internal.h"

using namespace simus;

namespace {

thread_local char g_err[512] = "";
std::atomic<int64_t> g_launches{0};

inline double sinc_d(double x) { return x == 0.0 ? 1.0 : std::sin(x) / x; }

// Eq. 26-27: two-way transducer response.
double transducer(const simus_probe &pr, double w) {
    const double wc = 2.0 * M_PI * pr.fc, wb = pr.frac_bw * wc;
    const double p = std::log(126.0) / std::log(2.0 * wc / wb);
    return std::exp(-std::log(2.0) * std::pow(2.0 * std::fabs(w - wc) / wb, p));
}

// Eq. 25 (and its Hann-windowed variant): pulse spectrum as (re, im).
void pulse(const simus_probe &pr, const simus_medium &md, double w, double &re, double &im) {
    const double wc = 2.0 * M_PI * pr.fc, T = md.pulse_cycles / pr.fc;
    auto rect = [&](double v) { return sinc_d(T * (v - wc) / 2.0) - sinc_d(T * (v + wc) / 2.0); };
    double s = rect(w);   // S_P = i * s
    if (md.pulse == SIMUS_PULSE_HANN) {
        const double dw = 2.0 * M_PI / T;
        s = 0.5 * s + 0.25 * rect(w + dw) + 0.25 * rect(w - dw);
    }
    re = 0.0;
    im = s;
}

int validate_probe(const simus_probe *pr, const simus_medium *md) {
    if (!pr || !md) return fail(SIMUS_ERR_ARG, "probe and medium must not be NULL");
    if (pr->n_elements < 1 || pr->n_elements > 4096)
        return fail(SIMUS_ERR_ARG, "n_elements=%d outside [1, 4096]", pr->n_elements);
    if (pr->n_sub < 0 || pr->n_sub > 64) return fail(SIMUS_ERR_ARG, "n_sub=%d outside [0, 64]", pr->n_sub);
    if (!(pr->pitch > 0) || !(pr->width > 0) || pr->width > pr->pitch * (1 + 1e-12))
        return fail(SIMUS_ERR_ARG, "need 0 < width <= pitch (width=%g pitch=%g)", pr->width, pr->pitch);
    if (pr->two_d != 0 && pr->two_d != 1) return fail(SIMUS_ERR_ARG, "two_d must be 0 or 1");
    if (!pr->two_d && !(pr->height > 0)) return fail(SIMUS_ERR_ARG, "height must be > 0");
    if (!pr->two_d && !(pr->elev_focus > 0)) return fail(SIMUS_ERR_ARG, "elev_focus must be > 0 or +inf");
    if (!(pr->radius >= 0) || std::isinf(pr->radius)) return fail(SIMUS_ERR_ARG, "radius must be finite and >= 0");
    if (!(pr->fc > 0) || std::isinf(pr->fc)) return fail(SIMUS_ERR_ARG, "fc must be > 0");
    if (!(pr->frac_bw > 0) || !(pr->frac_bw < 2)) return fail(SIMUS_ERR_ARG, "frac_bw must be in (0, 2)");
    if (pr->baffle < 0 || pr->baffle > 2) return fail(SIMUS_ERR_ARG, "baffle must be 0, 1 or 2");
    if (pr->baffle == SIMUS_BAFFLE_IMPEDANCE && !(pr->zeta >= 0))
        return fail(SIMUS_ERR_ARG, "zeta must be >= 0");
    if (!(md->c > 0) || std::isinf(md->c)) return fail(SIMUS_ERR_ARG, "c must be > 0");
    if (!(md->alpha_db >= 0) || std::isinf(md->alpha_db)) return fail(SIMUS_ERR_ARG, "alpha_db must be >= 0");
    if (!(md->fs > 0) || std::isinf(md->fs)) return fail(SIMUS_ERR_ARG, "fs must be > 0");
    if (md->pulse != SIMUS_PULSE_RECT && md->pulse != SIMUS_PULSE_HANN)
        return fail(SIMUS_ERR_ARG, "pulse must be 0 (rect) or 1 (Hann)");
    if (!(md->pulse_cycles > 0) || std::isinf(md->pulse_cycles))
        return fail(SIMUS_ERR_ARG, "pulse_cycles must be > 0");
    return SIMUS_OK;
}

int resolve_nsub(const simus_probe &pr, const simus_medium &md) {
    if (pr.n_sub > 0) return pr.n_sub;
    const double lambda_min = md.c / (pr.fc * (1.0 + pr.frac_bw / 2.0));   // Eq. 21
    return std::max(1, (int)std::ceil(pr.width / lambda_min));
}

// True while the calling thread's current entry point enqueues on a capturing stream:
// then only capture-safe CUDA calls are made (no pointer queries, no event queries).
thread_local bool g_capturing = false;

void note_capture(void *stream) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    g_capturing = cudaStreamIsCapturing(reinterpret_cast<cudaStream_t>(stream), &cs) == cudaSuccess &&
                  cs != cudaStreamCaptureStatusNone;
}

// Sets the flag for the duration of one entry point.
struct CaptureScope {
    explicit CaptureScope(void *stream) { note_capture(stream); }
    ~CaptureScope() { g_capturing = false; }
};

int check_device_ptr(const void *ptr, const char *name, bool allow_null = false) {
    if (!ptr) return allow_null ? SIMUS_OK : fail(SIMUS_ERR_ARG, "%s must not be NULL", name);
    if (g_capturing) return SIMUS_OK;
    cudaPointerAttributes a{};
    cudaError_t e = cudaPointerGetAttributes(&a, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SIMUS_ERR_ARG, "%s: not a CUDA pointer (%s)", name, cudaGetErrorString(e));
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return fail(SIMUS_ERR_ARG, "%s must be device memory", name);
    return SIMUS_OK;
}

int validate_tx(const simus_plan *p, const simus_tx *tx) {
    if (!tx) return fail(SIMUS_ERR_ARG, "tx must not be NULL");
    if (tx->n_tx < 1 || tx->n_tx > 65535) return fail(SIMUS_ERR_ARG, "n_tx=%d outside [1, 65535]", tx->n_tx);
    int rc;
    if ((rc = check_device_ptr(tx->delays, "tx.delays"))) return rc;
    if ((rc = check_device_ptr(tx->apod, "tx.apod"))) return rc;
    (void)p;
    return SIMUS_OK;
}

int validate_scat(const simus_scat *sc, int two_d) {
    if (!sc) return fail(SIMUS_ERR_ARG, "scat must not be NULL");
    if (two_d && sc->y) return fail(SIMUS_ERR_ARG, "scat.y must be NULL for a 2-D probe (x-z model)");
    if (sc->n < 0 || sc->n > (int64_t)1 << 34) return fail(SIMUS_ERR_ARG, "scat.n=%lld out of range", (long long)sc->n);
    if (sc->n == 0) return SIMUS_OK;
    int rc;
    if ((rc = check_device_ptr(sc->x, "scat.x"))) return rc;
    if ((rc = check_device_ptr(sc->y, "scat.y", true))) return rc;
    if ((rc = check_device_ptr(sc->z, "scat.z"))) return rc;
    if ((rc = check_device_ptr(sc->rc, "scat.rc"))) return rc;
    return SIMUS_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

int use_plan_device(const simus_plan *p) {
    return check_cuda(cudaSetDevice(p->device), "cudaSetDevice");
}

}  // namespace

namespace simus {

int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int check_cuda(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return SIMUS_OK;
    return fail(e == cudaErrorMemoryAllocation ? SIMUS_ERR_OOM : SIMUS_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

void stage_begin(simus_plan *plan, int stage, cudaStream_t st) {
    if (!plan->profiling) return;
    plan->stage_used[stage] = true;
    cudaEventRecord(plan->ev[2 * stage], st);
}

void stage_end(simus_plan *plan, int stage, cudaStream_t st) {
    if (!plan->profiling) return;
    cudaEventRecord(plan->ev[2 * stage + 1], st);
}

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int workspace(simus_plan *plan, size_t bytes, void **ptr) {
    if (bytes > plan->work_bytes) {
        if (g_capturing)
            return fail(SIMUS_ERR_ARG, "workspace must grow: make a warm-up call before stream capture");
        if (plan->d_work) {
            cudaError_t e = cudaDeviceSynchronize();
            if (e != cudaSuccess) return check_cuda(e, "workspace sync");
            cudaFree(plan->d_work);
            plan->d_work = nullptr;
            plan->work_bytes = 0;
        }
        size_t want = align256(bytes + bytes / 8);
        cudaError_t e = cudaMalloc(&plan->d_work, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(SIMUS_ERR_OOM, "workspace of %zu bytes: %s", want, cudaGetErrorString(e));
        }
        plan->work_bytes = want;
    }
    *ptr = plan->d_work;
    return SIMUS_OK;
}

// Host part of a plan: validation, nu (Eq. 21), kept bins and the Green's constants.
// Fills every field of *p except the device pointers, the device and the SM count.
int plan_setup_host(const simus_probe *probe, const simus_medium *medium, int32_t n_samples,
                    int32_t path, simus_plan *p) {
    int rc = validate_probe(probe, medium);
    if (rc) return rc;
    if (n_samples < 8 || n_samples > (1 << 24))
        return fail(SIMUS_ERR_ARG, "n_samples=%d outside [8, 2^24]", n_samples);
    if (path < SIMUS_PATH_PLAIN_F32 || path > SIMUS_PATH_TC_BF16)
        return fail(SIMUS_ERR_ARG, "unknown path %d", path);
    p->probe = *probe;
    p->medium = *medium;
    p->nt = n_samples;
    p->path = path;
    p->N = probe->n_elements;
    p->nu = resolve_nsub(*probe, *medium);
    p->M = p->nu * p->N;
    if (p->M > 8192) return fail(SIMUS_ERR_ARG, "nu * N = %d > 8192", p->M);

    // Kept bins: contiguous range where |S_P S_T| >= 1e-5 max over 1 <= q < Nt/2.
    const double df = medium->fs / n_samples;
    const int q_max = (n_samples - 1) / 2;
    auto mag = [&](int q) {
        double w = 2.0 * M_PI * q * df, re, im;
        pulse(*probe, *medium, w, re, im);
        return std::hypot(re, im) * transducer(*probe, w);
    };
    double hmax = 0.0;
    for (int q = 1; q <= q_max; ++q) hmax = std::max(hmax, mag(q));
    int lo = -1, hi = -1;
    for (int q = 1; q <= q_max; ++q)
        if (mag(q) >= 1e-5 * hmax) { if (lo < 0) lo = q; hi = q; }
    if (lo < 0) return fail(SIMUS_ERR_ARG, "no frequency bin above threshold (Nt too small?)");
    p->q_lo = lo;
    p->q_hi = hi;
    p->nq = hi - lo + 1;
    if ((double)hi * n_samples > 16777216.0 * 64)
        return fail(SIMUS_ERR_ARG, "bin index too large for the exact phase reduction");

    p->gc = green_const(*probe, *medium, p->N, p->nu, df, hi);
    p->gc.q_lo = lo;
    p->gc.nq = p->nq;
    p->gc.nt = n_samples;
    return SIMUS_OK;
}

// Green's constants for bin spacing df (frequency of "bin" q is q df; q may be
// fractional), with the narrow-sinc flag valid for bins up to q_max.
GreenConst green_const(const simus_probe &pr, const simus_medium &md, int N, int nu, double df,
                       double q_max) {
    const simus_probe *probe = &pr;
    const simus_medium *medium = &md;
    const double b = probe->width / 2.0;
    GreenConst gc{};
    gc.N = N; gc.nu = nu; gc.M = N * nu;
    gc.baffle = probe->baffle;
    const double K = df / medium->c;                       // cycles per metre per bin
    gc.Kh = (float)K;
    gc.Kl = (float)(K - (double)gc.Kh);
    gc.k1 = (float)(2.0 * M_PI * K);
    gc.k1b = (float)(2.0 * M_PI * K * b / nu);
    gc.kh = (float)(M_PI * K);
    gc.inv_rf = std::isinf(probe->elev_focus) ? 0.f : (float)(1.0 / probe->elev_focus);
    // Eq. 40: k_a = alpha_dB / 8.69 * f * 1e-4 per metre; base 2 per bin.
    gc.att2 = (float)(medium->alpha_db / 8.69 * df * 1e-4 / std::log(2.0));
    gc.zeta = (float)probe->zeta;
    gc.two_d = probe->two_d;
    gc.h = probe->two_d ? 1.0f : (float)probe->height;          // 2-D: no delta (Section V)
    gc.h2 = probe->two_d ? 0.0f : (float)(probe->height * probe->height);
    if (probe->two_d) gc.inv_rf = 0.0f;
    const double x_max = (2.0 * M_PI * K * b / nu) * q_max;   // largest |k b sin(theta) / nu|
    gc.narrow = x_max <= 3.19 ? 1 : (x_max <= 4.59 ? 2 : 0);
    gc.df = df;
    return gc;
}

void plan_delta_table(simus_plan *p, std::vector<float4> &tab, std::vector<float4> &tab_q) {
    // Eq. 15-16 at Y = 0 in the rescaled variable: delta/h = sum_g A_g sqrt(pi / (B_g + i x))
    static const double Ar[4] = {0.187, 0.288, 0.187, 0.288}, Ai[4] = {0.275, -1.954, -0.275, 1.954};
    static const double Br[4] = {4.558, 8.598, 4.558, 8.598}, Bi[4] = {-25.59, -7.924, 25.59, 7.924};
    GreenConst &gc = p->gc;
    gc.tab_n = 0;
    tab.clear();
    tab_q.clear();
    if (p->probe.two_d) return;   // no elevation factor in 2-D
    const double kx = M_PI * gc.df / p->medium.c * p->probe.height * p->probe.height;  // x per bin per (1/m)
    const double inv_rf = std::isinf(p->probe.elev_focus) ? 0.0 : 1.0 / p->probe.elev_focus;
    const double inv_r_max = 1.0 / 2e-3;
    double xs[4] = {p->q_lo * kx * inv_rf, p->q_hi * kx * inv_rf,
                    p->q_lo * kx * (inv_rf - inv_r_max), p->q_hi * kx * (inv_rf - inv_r_max)};
    const double xlo = std::min(0.0, *std::min_element(xs, xs + 4));
    const double xhi = std::max(0.0, *std::max_element(xs, xs + 4));
    const double dx = 0.5;
    const double x0 = std::floor(xlo) - 1.0;
    int n = (int)std::ceil((xhi - x0) / dx) + 3;   // nodes; n - 1 intervals
    if (n > 2049) return;
    // per node: Re f, Im f, Re f' dx, Im f' dx; and f at the interval midpoints
    std::vector<double> f(4 * n), fm(2 * n);
    auto eval = [&](double x, double *out) {
        double fr = 0, fi = 0, dr = 0, di = 0;
        for (int g = 0; g < 4; ++g) {
            // a = B + i x; f += A sqrt(pi) a^{-1/2}; df/dx += A sqrt(pi) (-1/2) a^{-3/2} i
            const double ar = Br[g], ai = Bi[g] + x;
            const double m = std::hypot(ar, ai);
            const double w = std::sqrt((m + ar) / 2.0), v = ai / (2.0 * w);      // sqrt(a) = w + i v
            const double ir = w / m, ii = -v / m;                                // a^{-1/2}
            const double pr = (ir * ar + ii * ai) / (m * m), pim = (ii * ar - ir * ai) / (m * m);  // a^{-3/2}
            const double cr = Ar[g] * std::sqrt(M_PI), ci = Ai[g] * std::sqrt(M_PI);
            fr += cr * ir - ci * ii;
            fi += cr * ii + ci * ir;
            // (-1/2) i a^{-3/2} = (0.5 pim, -0.5 pr)
            const double qr = 0.5 * pim, qi = -0.5 * pr;
            dr += cr * qr - ci * qi;
            di += cr * qi + ci * qr;
        }
        out[0] = fr; out[1] = fi; out[2] = dr * dx; out[3] = di * dx;
    };
    for (int j = 0; j < n; ++j) {
        double v[4];
        eval(x0 + j * dx, &f[4 * j]);
        eval(x0 + (j + 0.5) * dx, v);
        fm[2 * j] = v[0];
        fm[2 * j + 1] = v[1];
    }
    // interval j: the cubic Hermite interpolant in u = (x - x_j) / dx as power-basis
    // coefficients c0 + c1 u + c2 u^2 + c3 u^3 (complex), two float4 per interval
    tab.resize(2 * (n - 1));
    for (int j = 0; j + 1 < n; ++j) {
        double c[4][2];
        for (int k = 0; k < 2; ++k) {
            const double f0 = f[4 * j + k], f1 = f[4 * j + 4 + k];
            const double d0 = f[4 * j + 2 + k], d1 = f[4 * j + 6 + k];
            c[0][k] = f0;
            c[1][k] = d0;
            c[2][k] = 3.0 * (f1 - f0) - 2.0 * d0 - d1;
            c[3][k] = 2.0 * (f0 - f1) + d0 + d1;
        }
        tab[2 * j] = make_float4((float)c[0][0], (float)c[0][1], (float)c[1][0], (float)c[1][1]);
        tab[2 * j + 1] = make_float4((float)c[2][0], (float)c[2][1], (float)c[3][0], (float)c[3][1]);
    }
    // the quadratic through the interval's ends and midpoint, c0 + c1 u + c2 u^2, in the
    // same layout (c3 = 0): relative error <= 1.9e-5 inside an interval, <= 3e-4 half an
    // interval beyond it (FP16 operands round at 2.4e-4)
    tab_q.resize(2 * (n - 1));
    for (int j = 0; j + 1 < n; ++j) {
        double c[3][2];
        for (int k = 0; k < 2; ++k) {
            const double f0 = f[4 * j + k], f1 = f[4 * j + 4 + k], fh = fm[2 * j + k];
            c[0][k] = f0;
            c[1][k] = -3.0 * f0 + 4.0 * fh - f1;
            c[2][k] = 2.0 * f0 - 4.0 * fh + 2.0 * f1;
        }
        tab_q[2 * j] = make_float4((float)c[0][0], (float)c[0][1], (float)c[1][0], (float)c[1][1]);
        tab_q[2 * j + 1] = make_float4((float)c[2][0], (float)c[2][1], 0.0f, 0.0f);
    }
    n = n - 1;
    gc.tab_n = n;
    gc.tab_x0 = (float)x0;
    gc.tab_inv_dx = (float)(1.0 / dx);
}

// The plan's tables: sub-element records (Eq. 24; convex: arc of radius R about (0, -R))
// into sub[M], transfer values H_q = S_P S_T (Eq. 25-28, Eq. 34) into H[nq].
void plan_fill_tables(const simus_plan *p, SubElem *sub, float2 *H) {
    const simus_probe &probe = p->probe;
    for (int k = 0; k < p->nq; ++k) {
        double w = 2.0 * M_PI * (p->q_lo + k) * p->gc.df, re, im;
        pulse(probe, p->medium, w, re, im);
        double st = transducer(probe, w);
        H[k] = make_float2((float)(re * st), (float)(im * st));
    }
    const double b = probe.width / 2.0;
    const int N = p->N, nu = p->nu;
    for (int e = 0; e < N; ++e)
        for (int mu = 0; mu < nu; ++mu) {
            double xc, zc, psi;
            const double off = b / nu * (2.0 * mu - nu + 1);
            if (probe.radius > 0) {
                const double R = probe.radius;
                psi = (e - (N - 1) / 2.0) * probe.pitch / R + off / R;
                xc = R * std::sin(psi);
                zc = R * std::cos(psi) - R;
            } else {
                psi = 0.0;
                xc = probe.pitch / 2.0 * (2.0 * (e + 1) - N - 1) + off;
                zc = 0.0;
            }
            SubElem &s = sub[e * nu + mu];
            s.xh = (float)xc;
            s.xl = (float)(xc - (double)s.xh);
            s.zh = (float)zc;
            s.zl = (float)(zc - (double)s.zh);
            s.cpsi = (float)std::cos(psi);
            s.spsi = (float)std::sin(psi);
            s.l0 = (float)(xc * std::cos(psi) - zc * std::sin(psi));
            s.z0 = (float)(xc * std::sin(psi) + zc * std::cos(psi));
        }
}

}  // namespace simus

extern "C" {

const char *simus_last_error(void) { return g_err; }

int32_t simus_default_nt(const simus_probe *probe, const simus_medium *medium, double r_max,
                         double tau_max) {
    int rc = validate_probe(probe, medium);
    if (rc) return rc;
    if (!(r_max >= 0) || !(tau_max >= 0) || std::isinf(r_max) || std::isinf(tau_max))
        return fail(SIMUS_ERR_ARG, "r_max and tau_max must be finite and >= 0");
    double n = std::ceil(medium->fs * (2.0 * r_max / medium->c + tau_max + 8.0 / probe->fc));
    if (n > 1e8) return fail(SIMUS_ERR_ARG, "RF length %g too large", n);
    int32_t nt = (int32_t)n;
    return nt + (nt & 1);
}

int32_t simus_pfield_nfreq(const simus_probe *probe, const simus_medium *medium, double r_max,
                           double tau_max) {
    int rc = validate_probe(probe, medium);
    if (rc) return rc;
    if (!(r_max > 0) || !(tau_max >= 0) || std::isinf(r_max) || std::isinf(tau_max))
        return fail(SIMUS_ERR_ARG, "need r_max > 0 and tau_max >= 0");
    const double wc = 2.0 * M_PI * probe->fc;
    const double dw_max = 2.0 * M_PI / (r_max / medium->c + tau_max);   // Eq. 42 step rule
    double n = std::ceil(2.0 * wc / dw_max);
    if (n > 1e7) return fail(SIMUS_ERR_ARG, "frequency count %g too large", n);
    return (int32_t)n;
}

int simus_plan_create(const simus_probe *probe, const simus_medium *medium, int32_t n_samples,
                      int32_t path, simus_plan **out) {
    NvtxScope nvtx_scope("simus_plan_create");
    if (!out) return fail(SIMUS_ERR_ARG, "out must not be NULL");
    *out = nullptr;
    simus_plan *p = new simus_plan();
    int rc = plan_setup_host(probe, medium, n_samples, path, p);
    if (rc) { delete p; return rc; }
    std::vector<SubElem> sub(p->M);
    std::vector<float2> H(p->nq);
    plan_fill_tables(p, sub.data(), H.data());
    std::vector<float4> dtab, dtab_q;
    plan_delta_table(p, dtab, dtab_q);

    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess && !dtab.empty()) e = cudaMalloc(&p->d_dtab, sizeof(float4) * dtab.size());
    if (e == cudaSuccess && !dtab.empty())
        e = cudaMemcpy(p->d_dtab, dtab.data(), sizeof(float4) * dtab.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !dtab_q.empty()) e = cudaMalloc(&p->d_dtab_q, sizeof(float4) * dtab_q.size());
    if (e == cudaSuccess && !dtab_q.empty())
        e = cudaMemcpy(p->d_dtab_q, dtab_q.data(), sizeof(float4) * dtab_q.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_sub, sizeof(SubElem) * p->M);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_H, sizeof(float2) * p->nq);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(p->d_sub, sub.data(), sizeof(SubElem) * p->M, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_H, H.data(), sizeof(float2) * p->nq, cudaMemcpyHostToDevice);
    // tensor-core paths: the iDFT's twiddles, blocked for the tensor cores, when they take
    // at most 1 GiB (larger problems keep the CUDA-core iDFT)
    const size_t tw_b = idft_tc_twiddle_bytes(p->nt, p->nq);
    int trc = SIMUS_OK;
    if (e == cudaSuccess && p->path != SIMUS_PATH_PLAIN_F32 && tw_b <= ((size_t)1 << 30)) {
        e = cudaMalloc(&p->d_idft_tw, tw_b);
        if (e == cudaSuccess) trc = build_idft_tc_twiddles(p, p->d_idft_tw, nullptr);
        if (e == cudaSuccess && !trc) e = cudaDeviceSynchronize();
    }
    if (trc) {
        simus_plan_destroy(p);
        return trc;
    }
    if (e != cudaSuccess) {
        int r = check_cuda(e, "plan upload");
        cudaGetLastError();
        simus_plan_destroy(p);
        return r;
    }
    *out = p;
    return SIMUS_OK;
}

void simus_plan_destroy(simus_plan *plan) {
    if (!plan) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(plan->device);
    cudaDeviceSynchronize();
    for (auto &e : plan->ev)
        if (e) cudaEventDestroy(e);
    if (plan->ev_stage) cudaEventDestroy(plan->ev_stage);
    if (plan->h_stage) cudaFreeHost(plan->h_stage);
    cudaFree(plan->d_sub);
    cudaFree(plan->d_H);
    cudaFree(plan->d_err);
    cudaFree(plan->d_dtab);
    cudaFree(plan->d_dtab_q);
    cudaFree(plan->d_idft_tw);
    cudaFree(plan->d_work);
    cudaSetDevice(cur);
    delete plan;
}

int simus_plan_check(simus_plan *plan) {
    if (!plan) return fail(SIMUS_ERR_ARG, "plan must not be NULL");
    int rc = use_plan_device(plan);
    if (rc) return rc;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return check_cuda(e, "asynchronous error");
    int flag = 0;
    e = cudaMemcpy(&flag, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return check_cuda(e, "reading the device error flag");
    if (flag) {
        cudaMemset(plan->d_err, 0, sizeof(int));
        return fail(SIMUS_ERR_TIMEOUT, "a bounded device wait gave up (code %d); outputs invalid", flag);
    }
    return SIMUS_OK;
}

int simus_plan_selftest_timeout(simus_plan *plan, int32_t max_polls, void *stream) {
    if (!plan) return fail(SIMUS_ERR_ARG, "plan must not be NULL");
    if (max_polls < 1 || max_polls > (1 << 24)) return fail(SIMUS_ERR_ARG, "max_polls outside [1, 2^24]");
    int rc = use_plan_device(plan);
    if (rc) return rc;
    return launch_selftest_timeout(max_polls, plan->d_err, reinterpret_cast<cudaStream_t>(stream));
}

int simus_plan_set_profiling(simus_plan *plan, int32_t enable) {
    if (!plan) return fail(SIMUS_ERR_ARG, "plan must not be NULL");
    int rc = use_plan_device(plan);
    if (rc) return rc;
    if (enable && !plan->ev[0]) {
        for (auto &e : plan->ev) {
            cudaError_t err = cudaEventCreate(&e);
            if (err != cudaSuccess) return check_cuda(err, "cudaEventCreate");
        }
    }
    plan->profiling = enable != 0;
    return SIMUS_OK;
}

int simus_plan_set_tuning(simus_plan *plan, const simus_tuning *t) {
    if (!plan || !t) return fail(SIMUS_ERR_ARG, "plan and tuning must not be NULL");
    if (t->items_per_sm > 1024 || t->max_bins > 64 || t->chunks > 65536 || t->pair > 2 ||
        t->delta_table > 1 || t->tile_buffers > 2 || t->depth_order > 1 || t->tensor_idft > 1)
        return fail(SIMUS_ERR_ARG, "tuning value out of range");
    plan->items_per_sm = t->items_per_sm > 0 ? t->items_per_sm : 4;
    plan->max_bins = t->max_bins > 0 ? t->max_bins : 4;
    plan->pair_mode = t->pair >= 0 ? t->pair : 2;
    plan->delta_table = t->delta_table >= 0 ? t->delta_table : 1;
    plan->chunks = t->chunks > 0 ? t->chunks : 0;
    plan->tile_buffers = t->tile_buffers > 0 ? t->tile_buffers : 2;
    plan->depth_order = t->depth_order >= 0 ? t->depth_order : 1;
    plan->tensor_idft = t->tensor_idft >= 0 ? t->tensor_idft : 1;
    return SIMUS_OK;
}

int simus_plan_get_tuning(const simus_plan *plan, simus_tuning *t) {
    if (!plan || !t) return fail(SIMUS_ERR_ARG, "plan and tuning must not be NULL");
    *t = simus_tuning{};
    t->items_per_sm = plan->items_per_sm;
    t->max_bins = plan->max_bins;
    t->pair = plan->pair_mode;
    t->delta_table = plan->delta_table;
    t->chunks = plan->chunks;
    t->tile_buffers = plan->tile_buffers;
    t->depth_order = plan->depth_order;
    t->tensor_idft = plan->tensor_idft;
    return SIMUS_OK;
}

int simus_plan_get_timings(simus_plan *plan, float *ms) {
    if (!plan || !ms) return fail(SIMUS_ERR_ARG, "plan and ms must not be NULL");
    for (int i = 0; i < SIMUS_N_STAGES; ++i) {
        ms[i] = 0.f;
        if (!plan->profiling || !plan->stage_used[i]) continue;
        cudaError_t e = cudaEventSynchronize(plan->ev[2 * i + 1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[i], plan->ev[2 * i], plan->ev[2 * i + 1]);
        if (e != cudaSuccess) return check_cuda(e, "stage timing");
    }
    return SIMUS_OK;
}

int64_t simus_kernel_launches(void) { return g_launches.load(); }

int simus_plan_get_info(const simus_plan *plan, simus_plan_info *info) {
    if (!plan || !info) return fail(SIMUS_ERR_ARG, "plan and info must not be NULL");
    std::memset(info, 0, sizeof(*info));
    info->n_elements = plan->N;
    info->n_sub = plan->nu;
    info->n_samples = plan->nt;
    info->path = plan->path;
    info->q_lo = plan->q_lo;
    info->q_hi = plan->q_hi;
    info->n_bins = plan->nq;
    info->df = plan->gc.df;
    return SIMUS_OK;
}

}  // extern "C"

namespace {

// Workspace layout of one RF call: [weights | partial spectra | spectrum (simus_rf)].
// Plain FP32 path of one simulation in p's workspace [weights | partials | spectrum]:
// the spectrum goes to spec_out if given (else to the workspace), the time signals to rf
// if given.
int plain_run(simus_plan *p, const simus_tx *tx, const simus_scat *sc, float2 *spec_out,
              float *rf, cudaStream_t st) {
    const int T = tx->n_tx, n_chan = T * p->N;
    const PlainGeom gm = plain_mt_geometry(p, T, sc->n);   // several transmits: one tile per bin
    const bool mt = gm.SB > 0;
    const PlainGeom g = mt ? gm : plain_geometry(p, T, sc->n);
    const size_t w_b = align256(sizeof(float2) * (size_t)T * p->nq * p->N);
    const size_t part_b = align256(sizeof(float2) * (size_t)g.n_chunks * n_chan * p->nq);
    const size_t spec_b = spec_out ? 0 : align256(sizeof(float2) * (size_t)n_chan * p->nq);
    void *ws;
    int rc;
    if ((rc = workspace(p, w_b + part_b + spec_b, &ws))) return rc;
    char *base = reinterpret_cast<char *>(ws);
    float2 *cw = reinterpret_cast<float2 *>(base);
    float2 *part = reinterpret_cast<float2 *>(base + w_b);
    float2 *spec = spec_out ? spec_out : reinterpret_cast<float2 *>(base + w_b + part_b);
    stage_begin(p, 0, st);
    if ((rc = launch_tx_weights(p, tx, cw, st))) return rc;
    stage_end(p, 0, st);
    stage_begin(p, 1, st);
    if ((rc = mt ? launch_plain_mt(p, g, sc, T, cw, part, st) : launch_plain(p, g, sc, T, cw, part, st)))
        return rc;
    stage_end(p, 1, st);
    stage_begin(p, 2, st);
    if ((rc = launch_reduce_spectrum(p, part, g.n_chunks, n_chan, spec, st))) return rc;
    stage_end(p, 2, st);
    if (!rf) return SIMUS_OK;
    stage_begin(p, 3, st);
    rc = launch_idft(p, spec, n_chan, rf, st);
    stage_end(p, 3, st);
    return rc;
}

// Tensor-core path of n simulations in one persistent launch; temporaries in owner's
// workspace [unit descriptors | work counter | B1 images | partials | spectra].  Each
// simulation's spectrum goes to specs[i] if given, its time signals to rfs[i] if given.
// Simulations with no scatterer get zero outputs.
int tc_execute(simus_plan *owner, int n, simus_plan *const *plans, const simus_tx *txs,
               const simus_scat *scs, float2 *const *specs, float *const *rfs, cudaStream_t st) {
    std::vector<int> live;
    double total = 0.0;
    for (int i = 0; i < n; ++i) {
        const simus_plan *p = plans[i];
        const int n_chan = txs[i].n_tx * p->N;
        if (scs[i].n == 0) {
            int rc = specs && specs[i]
                ? check_cuda(cudaMemsetAsync(specs[i], 0, sizeof(float2) * (size_t)n_chan * p->nq, st), "memset")
                : SIMUS_OK;
            if (!rc && rfs && rfs[i])
                rc = check_cuda(cudaMemsetAsync(rfs[i], 0, sizeof(float) * (size_t)n_chan * p->nt, st), "memset");
            if (rc) return rc;
            continue;
        }
        live.push_back(i);
        total += (double)p->nq * (double)scs[i].n * p->M * txs[i].n_tx;
    }
    if (live.empty()) return SIMUS_OK;
    const int nl = (int)live.size();
    std::vector<TcShape> sh(nl);
    size_t smem = 0;
    int n_units = 0;
    bool has_y = false, linear = true;
    int sinc_rank = 0;   // sinc range of the launch: 0 |x| <= 3.2, 1 |x| <= 4.6, 2 any
    for (int j = 0; j < nl; ++j) {
        const int i = live[j];
        const simus_plan *p = plans[i];
        const double w = (double)p->nq * (double)scs[i].n * p->M * txs[i].n_tx / total;
        sh[j] = tc_shape(p, txs[i].n_tx, scs[i].n, w, owner->items_per_sm);
        if (!sh[j].ok)
            return fail(SIMUS_ERR_UNSUPPORTED, "tensor-core path: simulation %d (N=%d, nu=%d) does not fit",
                        i, p->N, p->nu);
        smem = std::max(smem, sh[j].smem);
        n_units += 1;
        has_y = has_y || scs[i].y != nullptr;
        sinc_rank = std::max(sinc_rank, p->gc.narrow == 1 ? 0 : (p->gc.narrow == 2 ? 1 : 2));
        linear = linear && p->probe.radius <= 0;
    }
    // workspace
    const size_t units_b = align256(sizeof(TcUnit) * n_units);
    size_t off = units_b + 256;
    std::vector<size_t> b1_off(n_units), part_off(nl), spec_off(nl), ord_off(nl), idft_off(nl);
    {
        int u = 0;
        for (int j = 0; j < nl; ++j)
            { b1_off[u] = off; off += align256(sh[j].b1_bytes); ++u; }
        for (int j = 0; j < nl; ++j) {
            const simus_plan *p = plans[live[j]];
            part_off[j] = off;
            off += align256(sizeof(float2) * (size_t)sh[j].n_chunks * txs[live[j]].n_tx * p->N * p->nq);
        }
        for (int j = 0; j < nl; ++j) {
            const simus_plan *p = plans[live[j]];
            spec_off[j] = off;
            if (!(specs && specs[live[j]])) off += align256(sizeof(float2) * (size_t)txs[live[j]].n_tx * p->N * p->nq);
        }
        // spectra blocked for the tensor-core iDFT: one region for the largest, as the
        // simulations' iDFTs run one after another on the stream
        size_t idft_b = 0;
        for (int j = 0; j < nl; ++j) {
            const int i = live[j];
            const simus_plan *p = plans[i];
            idft_off[j] = 0;
            if (!(rfs && rfs[i]) || !p->tensor_idft || !p->d_idft_tw) continue;
            idft_off[j] = off;
            idft_b = std::max(idft_b, align256(idft_tc_operand_bytes(txs[i].n_tx * p->N, p->nq)));
        }
        off += idft_b;
        // scatterers in distance order: x, y (when given), z, R and the sort's scratch
        for (int j = 0; j < nl; ++j) {
            const int i = live[j];
            ord_off[j] = 0;
            if (!plans[i]->depth_order || scs[i].n > (int64_t)INT32_MAX) continue;
            ord_off[j] = off;
            const size_t a = align256(sizeof(float) * (size_t)scs[i].n);
            off += (scs[i].y ? 4 : 3) * a + align256(order_scratch_bytes(scs[i].n));
        }
    }
    void *ws;
    int rc;
    if ((rc = workspace(owner, off, &ws))) return rc;
    char *base = reinterpret_cast<char *>(ws);
    TcUnit *d_units = reinterpret_cast<TcUnit *>(base);
    int *counter = reinterpret_cast<int *>(base + units_b);

    // unit descriptors in pinned staging (the previous call's copy must have read it)
    const size_t need = sizeof(TcUnit) * n_units;
    // While capturing, the caller has completed the previous (warm-up) call before
    // starting the capture, so the staging buffer is free.
    if (owner->stage_pending && g_capturing) owner->stage_pending = false;
    if (owner->stage_pending) {   // query first: a completed copy needs no wait
        if (cudaEventQuery(owner->ev_stage) != cudaSuccess &&
            (rc = check_cuda(cudaEventSynchronize(owner->ev_stage), "staging event")))
            return rc;
        owner->stage_pending = false;
    }
    if (need > owner->h_stage_bytes) {
        if (g_capturing)
            return fail(SIMUS_ERR_ARG, "stream capture needs a completed warm-up call of the same batch first");
        if (owner->h_stage) cudaFreeHost(owner->h_stage);
        owner->h_stage = nullptr;
        owner->h_stage_bytes = 0;
        if ((rc = check_cuda(cudaMallocHost(&owner->h_stage, need * 2), "pinned staging"))) return rc;
        owner->h_stage_bytes = need * 2;
    }
    if (!owner->ev_stage &&
        (rc = check_cuda(cudaEventCreateWithFlags(&owner->ev_stage, cudaEventDisableTiming), "event")))
        return rc;
    TcUnit *hu = reinterpret_cast<TcUnit *>(owner->h_stage);
    std::vector<std::pair<double, int>> order;
    {
        int u = 0;
        for (int j = 0; j < nl; ++j) {
            const int i = live[j];
            const simus_plan *p = plans[i];
            const TcShape &s = sh[j];
            TcUnit U{};
            U.gc = p->gc;
            U.sub = p->d_sub;
            // FP16 kernels evaluate the quadratic pieces, the split-BF16 ones the cubic
            U.dtab = owner->path == SIMUS_PATH_TC_BF16 ? p->d_dtab : p->d_dtab_q;
            U.gc.tab_n = s.tab_n;
            U.x = scs[i].x; U.y = scs[i].y; U.z = scs[i].z; U.rc = scs[i].rc;
            if (ord_off[j]) {   // the reordered copies (filled below, before the launch)
                const size_t a = align256(sizeof(float) * (size_t)scs[i].n);
                float *o = reinterpret_cast<float *>(base + ord_off[j]);
                U.x = o;
                U.z = reinterpret_cast<float *>(base + ord_off[j] + a);
                U.rc = reinterpret_cast<float *>(base + ord_off[j] + 2 * a);
                U.y = scs[i].y ? reinterpret_cast<float *>(base + ord_off[j] + 3 * a) : nullptr;
            }
            U.delays = txs[i].delays; U.apod = txs[i].apod;
            U.S = scs[i].n; U.n_tiles = s.n_tiles;
            U.T = txs[i].n_tx; U.G = s.n_groups; U.TG = s.TG;
            U.Np = s.Np; U.mh = s.mh; U.pair = s.pair; U.nbuf = s.nbuf; U.QB = s.QB; U.nN = s.nN;
            U.n_btiles = s.n_btiles; U.n_chunks = s.n_chunks; U.tiles_per_chunk = s.tiles_per_chunk;
            U.b1img = reinterpret_cast<uint16_t *>(base + b1_off[u]);
            U.part = reinterpret_cast<float2 *>(base + part_off[j]);
            hu[u] = U;
            order.push_back({(double)s.QB * s.tiles_per_chunk * s.Np * p->nu, u});
            ++u;
        }
    }
    // heaviest items first; item0 = prefix of item counts in that order
    std::stable_sort(order.begin(), order.end(), [](auto &a, auto &b) { return a.first > b.first; });
    std::vector<TcUnit> sorted(n_units);
    int64_t n_items = 0;
    for (int k = 0; k < n_units; ++k) {
        sorted[k] = hu[order[k].second];
        sorted[k].item0 = n_items;
        n_items += (int64_t)sorted[k].n_btiles * sorted[k].n_chunks;
    }
    std::copy(sorted.begin(), sorted.end(), hu);
    if ((rc = check_cuda(cudaMemcpyAsync(d_units, hu, need, cudaMemcpyHostToDevice, st), "upload units"))) return rc;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs == cudaStreamCaptureStatusNone) {
        if ((rc = check_cuda(cudaEventRecord(owner->ev_stage, st), "staging event"))) return rc;
        owner->stage_pending = true;
    }
    if ((rc = check_cuda(cudaMemsetAsync(counter, 0, sizeof(int), st), "memset counter"))) return rc;
    stage_begin(owner, 1, st);
    for (int j = 0; j < nl; ++j) {
        if (!ord_off[j]) continue;
        const int i = live[j];
        const size_t a = align256(sizeof(float) * (size_t)scs[i].n);
        char *o = base + ord_off[j];
        float *yo = scs[i].y ? reinterpret_cast<float *>(o + 3 * a) : nullptr;
        int *scratch = reinterpret_cast<int *>(o + (scs[i].y ? 4 : 3) * a);
        if ((rc = launch_order(&scs[i], (float)plans[i]->probe.radius, scratch, reinterpret_cast<float *>(o), yo,
                               reinterpret_cast<float *>(o + a), reinterpret_cast<float *>(o + 2 * a), st)))
            return rc;
    }
    rc = launch_tc_units(hu, d_units, n_units, n_items, smem, owner->path == SIMUS_PATH_TC_BF16, has_y,
                         sinc_rank == 0 ? 1 : (sinc_rank == 1 ? 2 : 0), linear, owner->num_sms,
                         counter, owner->d_err, st);
    stage_end(owner, 1, st);
    if (rc) return rc;
    stage_begin(owner, 2, st);
    for (int j = 0; j < nl; ++j) {
        const int i = live[j];
        simus_plan *p = plans[i];
        const int n_chan = txs[i].n_tx * p->N;
        float2 *spec = specs && specs[i] ? specs[i] : reinterpret_cast<float2 *>(base + spec_off[j]);
        if ((rc = launch_reduce_spectrum(p, reinterpret_cast<float2 *>(base + part_off[j]), sh[j].n_chunks,
                                         n_chan, spec, st)))
            return rc;
    }
    stage_end(owner, 2, st);
    if (!rfs) return SIMUS_OK;
    stage_begin(owner, 3, st);
    for (int j = 0; j < nl; ++j) {
        const int i = live[j];
        if (!rfs[i]) continue;
        simus_plan *p = plans[i];
        float2 *spec = specs && specs[i] ? specs[i] : reinterpret_cast<float2 *>(base + spec_off[j]);
        rc = idft_off[j] ? launch_idft_tc(p, spec, txs[i].n_tx * p->N, rfs[i], base + idft_off[j], st)
                         : launch_idft(p, spec, txs[i].n_tx * p->N, rfs[i], st);
        if (rc) return rc;
    }
    stage_end(owner, 3, st);
    return SIMUS_OK;
}

}  // namespace

extern "C" {

int simus_rf_spectrum(simus_plan *plan, const simus_tx *tx, const simus_scat *scat, float *spec,
                      void *stream) {
    NvtxScope nvtx_scope("simus_rf_spectrum");
    CaptureScope capture_scope(stream);
    if (!plan) return fail(SIMUS_ERR_ARG, "plan must not be NULL");
    for (bool &u : plan->stage_used) u = false;
    int rc;
    if ((rc = use_plan_device(plan))) return rc;
    if ((rc = validate_tx(plan, tx))) return rc;
    if ((rc = validate_scat(scat, plan->probe.two_d))) return rc;
    if ((rc = check_device_ptr(spec, "spec"))) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (scat->n == 0)
        return check_cuda(cudaMemsetAsync(spec, 0, sizeof(float2) * (size_t)tx->n_tx * plan->N * plan->nq, st),
                          "memset spectrum");
    float2 *sp = reinterpret_cast<float2 *>(spec);
    if (plan->path == SIMUS_PATH_PLAIN_F32) return plain_run(plan, tx, scat, sp, nullptr, st);
    return tc_execute(plan, 1, &plan, tx, scat, &sp, nullptr, st);
}

int simus_rf(simus_plan *plan, const simus_tx *tx, const simus_scat *scat, float *rf,
             void *stream) {
    NvtxScope nvtx_scope("simus_rf");
    CaptureScope capture_scope(stream);
    if (!plan) return fail(SIMUS_ERR_ARG, "plan must not be NULL");
    for (bool &u : plan->stage_used) u = false;
    int rc;
    if ((rc = use_plan_device(plan))) return rc;
    if ((rc = validate_tx(plan, tx))) return rc;
    if ((rc = validate_scat(scat, plan->probe.two_d))) return rc;
    if ((rc = check_device_ptr(rf, "rf"))) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int n_chan = tx->n_tx * plan->N;
    if (scat->n == 0)
        return check_cuda(cudaMemsetAsync(rf, 0, sizeof(float) * (size_t)n_chan * plan->nt, st),
                          "memset rf");
    if (plan->path == SIMUS_PATH_PLAIN_F32) return plain_run(plan, tx, scat, nullptr, rf, st);
    return tc_execute(plan, 1, &plan, tx, scat, nullptr, &rf, st);
}

int simus_pfield(simus_plan *plan, const simus_tx *tx, int64_t n_pts, const float *x,
                 const float *y, const float *z, int32_t n_freq, float *prms, void *stream) {
    NvtxScope nvtx_scope("simus_pfield");
    CaptureScope capture_scope(stream);
    if (!plan) return fail(SIMUS_ERR_ARG, "plan must not be NULL");
    for (bool &u : plan->stage_used) u = false;
    int rc;
    if ((rc = use_plan_device(plan))) return rc;
    if ((rc = validate_tx(plan, tx))) return rc;
    if (n_pts < 0 || n_pts > ((int64_t)1 << 31)) return fail(SIMUS_ERR_ARG, "n_pts out of range");
    if (n_freq < 1 || n_freq > 1000000) return fail(SIMUS_ERR_ARG, "n_freq=%d outside [1, 1e6]", n_freq);
    if (n_pts == 0) return SIMUS_OK;
    if ((rc = check_device_ptr(x, "x")) || (rc = check_device_ptr(y, "y", true)) ||
        (rc = check_device_ptr(z, "z")) || (rc = check_device_ptr(prms, "prms")))
        return rc;
    if (plan->probe.two_d && y) return fail(SIMUS_ERR_ARG, "y must be NULL for a 2-D probe (x-z model)");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const double df = 2.0 * plan->probe.fc / n_freq;            // midpoint grid of Eq. 42 (R8)
    const double dw = 2.0 * M_PI * df;
    // |P_Tx|^2 = |S_P|^2 S_T (Eq. 28); keep the contiguous range above 1e-12 of the maximum
    std::vector<float> p2(n_freq);
    double pmax = 0.0;
    for (int j = 0; j < n_freq; ++j) {
        double w = 2.0 * M_PI * (j + 0.5) * df, re, im;
        pulse(plan->probe, plan->medium, w, re, im);
        double v = (re * re + im * im) * transducer(plan->probe, w);
        p2[j] = (float)v;
        pmax = std::max(pmax, v);
    }
    int j_lo = -1, j_hi = -1;
    for (int j = 0; j < n_freq; ++j)
        if (p2[j] >= 1e-12 * pmax) { if (j_lo < 0) j_lo = j; j_hi = j; }
    if (j_lo < 0) return fail(SIMUS_ERR_ARG, "empty transmit spectrum");
    const int nf = j_hi - j_lo + 1;
    GreenConst gc = green_const(plan->probe, plan->medium, plan->N, plan->nu, df, j_hi + 0.5);
    if (plan->d_dtab && plan->delta_table) {   // the delta table's abscissa is physical (x), not a bin index
        gc.tab_n = plan->gc.tab_n;
        gc.tab_x0 = plan->gc.tab_x0;
        gc.tab_inv_dx = plan->gc.tab_inv_dx;
    }
    const int T = tx->n_tx;
    const size_t wt_b = align256(sizeof(float2) * (size_t)T * nf * plan->N);
    const size_t p2_b = align256(sizeof(float) * nf);
    const int n_fc = pfield_fchunks(plan, gc, T, n_pts, nf, y != nullptr);
    const size_t pp_b = n_fc > 1 ? align256(sizeof(float) * (size_t)n_fc * T * n_pts) : 0;
    void *ws;
    if ((rc = workspace(plan, wt_b + p2_b + pp_b, &ws))) return rc;
    float2 *wt = reinterpret_cast<float2 *>(ws);
    float *d_p2 = reinterpret_cast<float *>(reinterpret_cast<char *>(ws) + wt_b);
    float *ppart = n_fc > 1 ? reinterpret_cast<float *>(reinterpret_cast<char *>(ws) + wt_b + p2_b) : nullptr;
    if ((rc = check_cuda(cudaMemcpyAsync(d_p2, p2.data() + j_lo, sizeof(float) * nf,
                                         cudaMemcpyHostToDevice, st), "upload |P_Tx|^2")))
        return rc;
    stage_begin(plan, 4, st);
    rc = launch_pfield(plan, gc, tx, n_pts, x, y, z, nf, j_lo, wt, d_p2, (float)dw, prms, ppart, st);
    stage_end(plan, 4, st);
    return rc;
}

int simus_rf_grad(simus_plan *plan, const simus_tx *tx, const simus_scat *scat, const float *drf,
                  float *g_rc, float *g_x, float *g_z, float *g_delays, void *stream) {
    NvtxScope nvtx_scope("simus_rf_grad");
    CaptureScope capture_scope(stream);
    if (!plan) return fail(SIMUS_ERR_ARG, "plan must not be NULL");
    for (bool &u : plan->stage_used) u = false;
    int rc;
    if ((rc = use_plan_device(plan))) return rc;
    if ((rc = validate_tx(plan, tx))) return rc;
    if ((rc = validate_scat(scat, plan->probe.two_d))) return rc;
    if (scat->y) return fail(SIMUS_ERR_ARG, "simus_rf_grad needs scatterers in the azimuth plane (y == NULL)");
    if ((rc = check_device_ptr(drf, "drf"))) return rc;
    if ((rc = check_device_ptr(g_rc, "g_rc", true)) || (rc = check_device_ptr(g_x, "g_x", true)) ||
        (rc = check_device_ptr(g_z, "g_z", true)) || (rc = check_device_ptr(g_delays, "g_delays", true)))
        return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int T = tx->n_tx;
    const int64_t S = scat->n;
    if (S == 0) {
        if (g_delays)
            return check_cuda(cudaMemsetAsync(g_delays, 0, sizeof(float) * (size_t)T * plan->N, st),
                              "memset g_delays");
        return SIMUS_OK;
    }
    GradGeom g = grad_geometry(plan, T, S);
    if (!g.ok) return fail(SIMUS_ERR_UNSUPPORTED, "simus_rf_grad needs T * N <= 2048 (T=%d, N=%d)", T, plan->N);
    const size_t tab = align256(sizeof(float2) * (size_t)T * plan->nq * plan->N);
    const size_t gp = align256(sizeof(float) * 3 * (size_t)g.n_qtiles * S);
    const size_t bp = align256(sizeof(float2) * (size_t)g.n_chunks * T * plan->nq * plan->N);
    void *ws;
    if ((rc = workspace(plan, 2 * tab + gp + bp, &ws))) return rc;
    char *base = reinterpret_cast<char *>(ws);
    float2 *cw = reinterpret_cast<float2 *>(base);
    float2 *lam = reinterpret_cast<float2 *>(base + tab);
    float *gpart = reinterpret_cast<float *>(base + 2 * tab);
    float2 *bpart = reinterpret_cast<float2 *>(base + 2 * tab + gp);
    stage_begin(plan, 0, st);
    if ((rc = launch_tx_weights(plan, tx, cw, st))) return rc;
    stage_end(plan, 0, st);
    stage_begin(plan, 5, st);
    if ((rc = launch_adjoint_dft(plan, drf, T, lam, st))) return rc;
    stage_end(plan, 5, st);
    stage_begin(plan, 6, st);
    if ((rc = launch_grad(plan, g, scat, T, cw, lam, gpart, bpart, st))) return rc;
    stage_end(plan, 6, st);
    stage_begin(plan, 7, st);
    rc = launch_grad_finish(plan, g, T, S, gpart, bpart, cw, g_rc, g_x, g_z, g_delays, st);
    stage_end(plan, 7, st);
    return rc;
}

}  // extern "C"

namespace {

// Shared body of simus_batch_rf (rf != NULL) and simus_batch_rf_spectrum (spec != NULL).
int batch_run(const char *name, int32_t n_sims, simus_plan *const *plans, const simus_tx *tx,
              const simus_scat *scat, float *const *rf, float *const *spec, void *stream) {
    NvtxScope nvtx_scope(name);
    CaptureScope capture_scope(stream);
    float *const *out = rf ? rf : spec;
    if (n_sims < 0 || (n_sims > 0 && (!plans || !tx || !scat || !out)))
        return fail(SIMUS_ERR_ARG, "invalid batch arguments");
    if (n_sims == 0) return SIMUS_OK;
    int rc;
    for (int i = 0; i < n_sims; ++i) {
        if (!plans[i]) return fail(SIMUS_ERR_ARG, "plans[%d] is NULL", i);
        if (plans[i]->path != plans[0]->path || plans[i]->device != plans[0]->device)
            return fail(SIMUS_ERR_ARG, "all plans of a batch must share path and device (plan %d)", i);
        for (bool &u : plans[i]->stage_used) u = false;
    }
    if ((rc = use_plan_device(plans[0]))) return rc;
    for (int i = 0; i < n_sims; ++i) {
        if ((rc = validate_tx(plans[i], &tx[i])) || (rc = validate_scat(&scat[i], plans[i]->probe.two_d)) ||
            (rc = check_device_ptr(out[i], rf ? "rf[i]" : "spec[i]")))
            return fail(rc, "simulation %d: %s", i, simus_last_error());
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (plans[0]->path == SIMUS_PATH_PLAIN_F32) {
        for (int i = 0; i < n_sims; ++i) {
            const size_t n_chan = (size_t)tx[i].n_tx * plans[i]->N;
            float2 *sp = spec ? reinterpret_cast<float2 *>(spec[i]) : nullptr;
            if (scat[i].n == 0)
                rc = check_cuda(rf ? cudaMemsetAsync(rf[i], 0, sizeof(float) * n_chan * plans[i]->nt, st)
                                   : cudaMemsetAsync(sp, 0, sizeof(float2) * n_chan * plans[i]->nq, st),
                                "memset output");
            else
                rc = plain_run(plans[i], &tx[i], &scat[i], sp, rf ? rf[i] : nullptr, st);
            if (rc) return rc;
        }
        return SIMUS_OK;
    }
    if (rf) return tc_execute(plans[0], n_sims, plans, tx, scat, nullptr, rf, st);
    std::vector<float2 *> sp(n_sims);
    for (int i = 0; i < n_sims; ++i) sp[i] = reinterpret_cast<float2 *>(spec[i]);
    return tc_execute(plans[0], n_sims, plans, tx, scat, sp.data(), nullptr, st);
}

}  // namespace

extern "C" {

int simus_batch_rf(int32_t n_sims, simus_plan *const *plans, const simus_tx *tx,
                   const simus_scat *scat, float *const *rf, void *stream) {
    return batch_run("simus_batch_rf", n_sims, plans, tx, scat, rf, nullptr, stream);
}

int simus_batch_rf_spectrum(int32_t n_sims, simus_plan *const *plans, const simus_tx *tx,
                            const simus_scat *scat, float *const *spec, void *stream) {
    return batch_run("simus_batch_rf_spectrum", n_sims, plans, tx, scat, nullptr, spec, stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// simus_rf_noalloc: the plain FP32 RF computation with no device allocation.
//
// Some callers cannot allocate device memory: latency-critical loops that must never
// enter the allocator (which can synchronise the device), and plug-ins hosted by an
// application that owns the whole device memory pool.  They cannot create a plan
// either, so this entry point takes the probe and medium directly and keeps every
// temporary -- sub-element table, transfer values, transmit weights, per-chunk partial
// spectra and the spectrum -- in one file-scope device array of fixed size.
//
// The array exists once per device that loads the library and lives until the process
// exits.  Host code cannot use the array's name as a device address, so the first call
// on each device (with that device current) resolves the address with
// cudaGetSymbolAddress and caches it.  The two small tables are uploaded from host
// memory by stream-ordered copies; a captured copy would read that host memory when the
// graph is replayed, after later calls have overwritten it, so a stream under capture is
// refused before anything else is done.  Every call shares the array: calls that
// overlap on the GPU (other streams, or other host threads whose kernels are still
// running) race on it.  Calls from several host threads are serialised on the host.
// Nothing in the array must start at zero: every buffer is fully written before it is
// read.
// ---------------------------------------------------------------------------------
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[SIMUS_NOALLOC_SCRATCH_BYTES];

constexpr int kNoallocMaxDevices = 64;
constexpr int kNoallocMaxSub = 2048;     // nu * N
constexpr int kNoallocMaxBins = 16384;   // kept bins
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kNoallocMaxDevices] = {};
int g_noalloc_sms[kNoallocMaxDevices] = {};
SubElem g_noalloc_sub[kNoallocMaxSub];   // host staging of the tables (no allocation)
float2 g_noalloc_H[kNoallocMaxBins];

}  // namespace

extern "C" int simus_rf_noalloc(const simus_probe *probe, const simus_medium *medium,
                                int32_t n_samples, const simus_tx *tx, const simus_scat *scat,
                                float *rf, void *stream) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    int dev = 0, rc;
    {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if ((rc = check_cuda(cudaStreamIsCapturing(reinterpret_cast<cudaStream_t>(stream), &cs),
                             "cudaStreamIsCapturing")))
            return rc;
        if (cs != cudaStreamCaptureStatusNone)
            return fail(SIMUS_ERR_ARG, "simus_rf_noalloc cannot run under stream capture: its table "
                                       "uploads read host memory that later calls overwrite");
    }
    if ((rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice"))) return rc;
    if (dev < 0 || dev >= kNoallocMaxDevices)
        return fail(SIMUS_ERR_ARG, "device %d beyond the %d this entry point serves", dev, kNoallocMaxDevices);
    if (!g_noalloc_addr[dev]) {   // once per device, with that device current
        void *addr = nullptr;
        if ((rc = check_cuda(cudaGetSymbolAddress(&addr, g_noalloc_scratch), "cudaGetSymbolAddress")))
            return rc;
        if ((rc = check_cuda(cudaDeviceGetAttribute(&g_noalloc_sms[dev], cudaDevAttrMultiProcessorCount, dev),
                             "SM count")))
            return rc;
        g_noalloc_addr[dev] = addr;
    }

    simus_plan plan;   // host-only description; its table pointers point into the scratch
    if ((rc = plan_setup_host(probe, medium, n_samples, SIMUS_PATH_PLAIN_F32, &plan))) return rc;
    plan.device = dev;
    plan.num_sms = g_noalloc_sms[dev];
    if (plan.M > kNoallocMaxSub || plan.nq > kNoallocMaxBins)
        return fail(SIMUS_ERR_ARG, "simus_rf_noalloc serves nu*N <= %d and <= %d kept bins (got %d, %d)",
                    kNoallocMaxSub, kNoallocMaxBins, plan.M, plan.nq);
    if ((rc = validate_tx(&plan, tx))) return rc;
    if ((rc = validate_scat(scat, plan.probe.two_d))) return rc;
    if ((rc = check_device_ptr(rf, "rf"))) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int T = tx->n_tx, n_chan = T * plan.N;
    if (scat->n == 0)
        return check_cuda(cudaMemsetAsync(rf, 0, sizeof(float) * (size_t)n_chan * plan.nt, st), "memset rf");

    // scratch layout: [sub | H | weights | spectrum | partials (as many chunks as fit)]
    const size_t sub_b = align256(sizeof(SubElem) * plan.M);
    const size_t h_b = align256(sizeof(float2) * plan.nq);
    const size_t cw_b = align256(sizeof(float2) * (size_t)T * plan.nq * plan.N);
    const size_t spec_b = align256(sizeof(float2) * (size_t)n_chan * plan.nq);
    const size_t per_chunk = sizeof(float2) * (size_t)n_chan * plan.nq;
    const size_t fixed = sub_b + h_b + cw_b + spec_b;
    if (fixed + per_chunk > SIMUS_NOALLOC_SCRATCH_BYTES)
        return fail(SIMUS_ERR_ARG,
                    "problem needs at least %zu bytes of scratch, more than the fixed %u of "
                    "simus_rf_noalloc (use simus_rf with a plan)",
                    fixed + per_chunk, (unsigned)SIMUS_NOALLOC_SCRATCH_BYTES);
    const int64_t max_chunks = (int64_t)((SIMUS_NOALLOC_SCRATCH_BYTES - fixed) / per_chunk);

    PlainGeom g = plain_geometry(&plan, T, scat->n);
    if (g.n_chunks > max_chunks) {
        int64_t len = (scat->n + max_chunks - 1) / max_chunks;
        len = ((len + g.SB - 1) / g.SB) * g.SB;
        g.chunk_len = len;
        g.n_chunks = (int)((scat->n + len - 1) / len);
    }

    char *base = reinterpret_cast<char *>(g_noalloc_addr[dev]);
    SubElem *d_sub = reinterpret_cast<SubElem *>(base);
    float2 *d_H = reinterpret_cast<float2 *>(base + sub_b);
    float2 *cw = reinterpret_cast<float2 *>(base + sub_b + h_b);
    float2 *spec = reinterpret_cast<float2 *>(base + sub_b + h_b + cw_b);
    float2 *part = reinterpret_cast<float2 *>(base + fixed);

    plan_fill_tables(&plan, g_noalloc_sub, g_noalloc_H);
    // pageable source: the copies have read the host staging when these calls return
    if ((rc = check_cuda(cudaMemcpyAsync(d_sub, g_noalloc_sub, sizeof(SubElem) * plan.M,
                                         cudaMemcpyHostToDevice, st), "upload sub-elements")))
        return rc;
    if ((rc = check_cuda(cudaMemcpyAsync(d_H, g_noalloc_H, sizeof(float2) * plan.nq,
                                         cudaMemcpyHostToDevice, st), "upload transfer values")))
        return rc;
    plan.d_sub = d_sub;
    plan.d_H = d_H;
    if ((rc = launch_tx_weights(&plan, tx, cw, st))) return rc;
    if ((rc = launch_plain(&plan, g, scat, T, cw, part, st))) return rc;
    if ((rc = launch_reduce_spectrum(&plan, part, g.n_chunks, n_chan, spec, st))) return rc;
    return launch_idft(&plan, spec, n_chan, rf, st);
}
