/*
 * simus_oracle.c -- plain FP64 CPU oracle of the SIMUS linear frequency-domain model
 * (D. Garcia, "SIMUS: an open-source simulator for medical ultrasound imaging.
 *  Part I: theory & examples", arXiv:2102.02738).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the CUDA
 * library is checked against.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load it; the product path never does.  It shares no
 * code, header, table or constant with the CUDA library: the paper's constants are
 * typed here a second time on purpose.
 *
 * Every routine follows one equation of the paper, in FP64, in the paper's order and
 * notation, with no blocking, fusion or reordering beyond what the equation states.
 * OpenMP only splits independent frequency bins (or scatterers) across host cores.
 *
 * Readings of points the paper leaves open (each one also listed in the design notes):
 *   R1  sinc is the unnormalised sin(x)/x (forced by the integral of Eq. 10).
 *   R2  a sub-element of an element of width 2b split in nu has half-width b/nu in
 *       D(theta,k) (Eq. 21, Eq. 24 space the centroids by 2b/nu).
 *   R3  constant prefactors (kb/(i pi), rho c, v0) are dropped: Eq. 22 and Eq. 32 are
 *       used literally with P_Tx = S_P sqrt(S_T) (Eq. 28) and RF = sqrt(S_T) P (Eq. 34).
 *   R4  frequency grid of the RF signals: f_q = q fs / Nt; the kept bins are the
 *       contiguous range of 1 <= q < Nt/2 whose transfer magnitude |S_P S_T| is at
 *       least 1e-5 of its maximum over that range.
 *   R5  time signals: rf[j] = Re sum_q X_q exp(-2 pi i q j / Nt), no scale factor; the
 *       sign follows the exp(-i omega t) convention of Eq. 1.
 *   R6  D = 0 for points behind a (sub-)element (cos(theta) <= 0).
 *   R7  convex probe: centre of curvature (0,-R); element e at arc angle
 *       psi_e = (e-(N+1)/2) p / R; sub-elements on the arc at psi_e + (b/nu)(2mu-nu+1)/R;
 *       theta measured from the local normal (sin psi, cos psi).
 *   R8  Eq. 42: midpoint sum f_j = (j+1/2) 2 fc / N_f, j = 0..N_f-1, dw = 2 w_c / N_f,
 *       |P|^2 for the complex P.
 *   R9  lambda_min of Eq. 21 is c / (fc (1 + bw/2)), the upper -6 dB edge.
 *   R10 Eq. 23 is used as printed: r_n includes Y^2, and beta, gamma of Eq. 14 are
 *       evaluated with that r_n.
 *   R11 Hann pulse: window 0.5(1+cos(2 pi t/T)) on [-T/2,T/2] applied to the sine of
 *       Eq. 25, i.e. S_P^Hann(w) = S_P(w)/2 + S_P(w+2pi/T)/4 + S_P(w-2pi/T)/4.
 *   R14 2-D mode (Section V, Eq. 36-38): the Green's term is exp(i(k + i k_a) r)/sqrt(r)
 *       * D(theta, k), with the constants sqrt(2b), 2b and the sqrt(k) inside P_Tx dropped
 *       as in R3 (P_Tx stays S_P sqrt(S_T)); h and R_f play no part and Y must be 0.
 *
 * Gradients (oracle_rf_grad) are not in the paper; they are the exact derivative of
 * the model above and are pinned by central finite differences of oracle_rf.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* Problem description (Section II, Fig. 2; Section III; Section VI). */
typedef struct {
    int32_t n_elements;   /* N */
    int32_t n_sub;        /* nu; 0 selects Eq. 21 */
    int32_t baffle;       /* 0 soft, 1 rigid, 2 finite impedance (Eq. 39) */
    int32_t pulse;        /* 0 rectangular window (Eq. 25), 1 Hann window (R11) */
    int32_t n_samples;    /* Nt, RF samples per channel */
    int32_t two_d;        /* 1: the 2-D model of Section V (R14), 0: 3-D */
    double pitch;         /* p [m] */
    double width;         /* 2b [m] */
    double height;        /* h [m] */
    double elev_focus;    /* R_f [m]; +inf: no elevation lens */
    double radius;        /* convex radius of curvature [m]; 0: linear array */
    double fc;            /* centre frequency [Hz] */
    double frac_bw;       /* pulse-echo fractional bandwidth, w_b / w_c */
    double zeta;          /* impedance ratio of Eq. 39 */
    double c;             /* speed of sound [m/s] */
    double alpha_db;      /* attenuation [dB/cm/MHz] (Eq. 40) */
    double fs;            /* RF sampling frequency [Hz] */
    double pulse_cycles;  /* n_lambda of Eq. 25 */
} oracle_params;

/* Eq. 18: the four-Gaussian coefficients, third and fourth the conjugates of the first
 * two. */
static const double A_RE[4] = {0.187, 0.288, 0.187, 0.288};
static const double A_IM[4] = {0.275, -1.954, -0.275, 1.954};
static const double B_RE[4] = {4.558, 8.598, 4.558, 8.598};
static const double B_IM[4] = {-25.59, -7.924, 25.59, 7.924};

void oracle_gaussian_coefficients(double *a_re, double *a_im, double *b_re, double *b_im)
{
    for (int g = 0; g < 4; ++g) {
        a_re[g] = A_RE[g]; a_im[g] = A_IM[g]; b_re[g] = B_RE[g]; b_im[g] = B_IM[g];
    }
}

static double sinc(double x) /* R1 */
{
    return x == 0.0 ? 1.0 : sin(x) / x;
}

/* Eq. 26-27 (Appendix B): generalised-Gaussian transducer response, two-way. */
double oracle_transducer_response(const oracle_params *p, double w)
{
    double wc = 2.0 * M_PI * p->fc;
    double wb = p->frac_bw * wc;
    double pexp = log(126.0) / log(2.0 * wc / wb);
    return exp(-log(2.0) * pow(2.0 * fabs(w - wc) / wb, pexp));
}

/* Eq. 25: spectrum of the windowed sine, T = n_lambda / fc; Hann variant by R11. */
static cplx rect_pulse(double wc, double T, double w)
{
    return I * (sinc(T * (w - wc) / 2.0) - sinc(T * (w + wc) / 2.0));
}

cplx oracle_pulse_spectrum_c(const oracle_params *p, double w)
{
    double wc = 2.0 * M_PI * p->fc;
    double T = p->pulse_cycles / p->fc;
    if (p->pulse == 1) {
        double dw = 2.0 * M_PI / T;
        return 0.5 * rect_pulse(wc, T, w) + 0.25 * rect_pulse(wc, T, w + dw)
             + 0.25 * rect_pulse(wc, T, w - dw);
    }
    return rect_pulse(wc, T, w);
}

void oracle_pulse_spectrum(const oracle_params *p, double w, double *re, double *im)
{
    cplx s = oracle_pulse_spectrum_c(p, w);
    *re = creal(s); *im = cimag(s);
}

/* Eq. 28 and Eq. 34 (R3): transmit spectrum S_P sqrt(S_T), receive response sqrt(S_T);
 * the RF spectrum carries their product S_P S_T. */
static cplx transfer(const oracle_params *p, double w)
{
    return oracle_pulse_spectrum_c(p, w) * oracle_transducer_response(p, w);
}

void oracle_transfer(const oracle_params *p, double w, double *re, double *im)
{
    cplx h = transfer(p, w);
    *re = creal(h); *im = cimag(h);
}

/* Eq. 21 with R9. */
int32_t oracle_nsub(const oracle_params *p)
{
    if (p->n_sub > 0) return p->n_sub;
    double lambda_min = p->c / (p->fc * (1.0 + p->frac_bw / 2.0));
    int32_t nu = (int32_t)ceil(p->width / lambda_min);
    return nu < 1 ? 1 : nu;
}

/* R4: kept frequency bins [q_lo, q_hi]. Returns their number. */
int32_t oracle_bins(const oracle_params *p, int32_t *q_lo, int32_t *q_hi)
{
    int32_t nt = p->n_samples;
    int32_t q_max = (nt - 1) / 2; /* largest q with q < Nt/2 */
    double hmax = 0.0;
    for (int32_t q = 1; q <= q_max; ++q) {
        double h = cabs(transfer(p, 2.0 * M_PI * q * p->fs / nt));
        if (h > hmax) hmax = h;
    }
    int32_t lo = -1, hi = -1;
    for (int32_t q = 1; q <= q_max; ++q) {
        double h = cabs(transfer(p, 2.0 * M_PI * q * p->fs / nt));
        if (h >= 1e-5 * hmax) {
            if (lo < 0) lo = q;
            hi = q;
        }
    }
    *q_lo = lo; *q_hi = hi;
    return lo < 0 ? 0 : hi - lo + 1;
}

/* Eq. 24 (linear array) and R7 (convex array): centroid (xc, zc) and normal angle psi
 * of each of the nu N sub-elements, numbered n = 1..nu N from left to right. */
void oracle_centroids(const oracle_params *p, double *xc, double *zc, double *psi)
{
    int32_t N = p->n_elements, nu = oracle_nsub(p);
    double b = p->width / 2.0;
    for (int32_t n = 1; n <= nu * N; ++n) {
        int32_t e = (n + nu - 1) / nu;     /* ceil(n / nu): element of sub-element n */
        int32_t mu = (n - 1) % nu;         /* (n-1) mod nu */
        if (p->radius <= 0.0) {
            xc[n - 1] = p->pitch / 2.0 * (2.0 * e - N - 1) + b / nu * (2.0 * mu - nu + 1);
            zc[n - 1] = 0.0;
            psi[n - 1] = 0.0;
        } else {
            double R = p->radius;
            double ang = (e - (N + 1) / 2.0) * p->pitch / R + b / nu * (2.0 * mu - nu + 1) / R;
            xc[n - 1] = R * sin(ang);
            zc[n - 1] = R * cos(ang) - R;
            psi[n - 1] = ang;
        }
    }
}

/* Eq. 14-16: elevation factor delta(y, r, k) by the Gaussian superposition model. */
cplx oracle_delta_c(const oracle_params *p, double k, double y, double r)
{
    double h = p->height;
    double inv_rf = isinf(p->elev_focus) ? 0.0 : 1.0 / p->elev_focus;
    cplx beta = -I * k * y / r;
    cplx gamma = I * k * y * y / (2.0 * r);
    cplx delta = 0.0;
    for (int g = 0; g < 4; ++g) {
        cplx A = A_RE[g] + I * A_IM[g];
        cplx B = B_RE[g] + I * B_IM[g];
        cplx alpha = B / (h * h) + I * k / 2.0 * (inv_rf - 1.0 / r);
        delta += A * csqrt(M_PI / alpha) * cexp(beta * beta / (4.0 * alpha) + gamma);
    }
    return delta;
}

void oracle_delta(const oracle_params *p, double k, double y, double r, double *re, double *im)
{
    cplx d = oracle_delta_c(p, k, y, r);
    *re = creal(d); *im = cimag(d);
}

/* Eq. 10 and Eq. 39, with R1, R2, R6: directivity of a (sub-)element of half-width bh. */
double oracle_directivity(const oracle_params *p, double k, double bh, double sin_t, double cos_t)
{
    if (cos_t <= 0.0) return 0.0;
    double d = sinc(k * bh * sin_t);
    if (p->baffle == 0) return d * cos_t;
    if (p->baffle == 1) return d;
    return d * cos_t / (cos_t + p->zeta);
}

/* Geometry of one scatterer seen from sub-element n (Eq. 23 and R7, R10). */
typedef struct {
    double dx, dz, rho, r, lx, lz, sin_t, cos_t, cpsi, spsi;
} geom;

static geom geometry(double xc, double zc, double psi, double X, double Y, double Z)
{
    geom G;
    G.dx = X - xc;
    G.dz = Z - zc;
    G.rho = sqrt(G.dx * G.dx + G.dz * G.dz);
    G.r = sqrt(G.dx * G.dx + Y * Y + G.dz * G.dz);
    G.cpsi = cos(psi);
    G.spsi = sin(psi);
    G.lx = G.dx * G.cpsi - G.dz * G.spsi;
    G.lz = G.dx * G.spsi + G.dz * G.cpsi;
    G.sin_t = G.lx / G.rho;
    G.cos_t = G.lz / G.rho;
    return G;
}

/* Eq. 40: amplitude absorption k_a = (alpha_dB / 8.69) k c / (2 pi 1e4). */
static double absorption(const oracle_params *p, double k)
{
    return p->alpha_db / 8.69 * k * p->c / (2.0 * M_PI * 1e4);
}

/* Eq. 17/19 with Eq. 39 and Eq. 40: the Green's term of sub-element n at frequency f,
 *   g = exp(i (k + i k_a) r) / r * D(theta, k) * delta(Y, r, k);
 * in 2-D (Eq. 36, R14) g = exp(i (k + i k_a) r) / sqrt(r) * D(theta, k). */
static cplx green(const oracle_params *p, int32_t nu, double f, double xc, double zc,
                  double psi, double X, double Y, double Z)
{
    double k = 2.0 * M_PI * f / p->c;
    double ka = absorption(p, k);
    geom G = geometry(xc, zc, psi, X, Y, Z);
    double D = oracle_directivity(p, k, p->width / 2.0 / nu, G.sin_t, G.cos_t);
    if (D == 0.0) return 0.0;
    if (p->two_d) return cexp(I * (k + I * ka) * G.r) / sqrt(G.r) * D;
    return cexp(I * (k + I * ka) * G.r) / G.r * D * oracle_delta_c(p, k, Y, G.r);
}

void oracle_green(const oracle_params *p, double f, double X, double Y, double Z, int32_t n,
                  double *re, double *im)
{
    int32_t nu = oracle_nsub(p), M = nu * p->n_elements;
    double *xc = malloc(sizeof(double) * 3 * M);
    oracle_centroids(p, xc, xc + M, xc + 2 * M);
    cplx g = green(p, nu, f, xc[n], xc[M + n], xc[2 * M + n], X, Y, Z);
    free(xc);
    *re = creal(g); *im = cimag(g);
}

/* Eq. 29-34: RF spectrum X_q(e, t) of every element e and transmit t at the listed bins.
 *   P(X_s, w)      = sum_n W_n exp(i w dtau_n) g_ns                      (Eq. 29)
 *   P^se_m         = sum_s R_s P(X_s, w) g_ms                            (Eq. 30-32)
 *   P^e            = sum_{mu} P^se_{(e,mu)}                              (Eq. 33)
 *   X_q(e, t)      = S_P S_T P^e                                         (Eq. 34, R3)
 * delays/apod: [T][N]; scatterers x, y, z, R: [S] (y may be NULL for Y = 0);
 * out: [T][N][nq] complex as interleaved (re, im). */
void oracle_rf_spectrum(const oracle_params *p, int32_t T, const double *delays,
                        const double *apod, int64_t S, const double *x, const double *y,
                        const double *z, const double *R, int32_t nq, const int32_t *qlist,
                        double *out)
{
    int32_t N = p->n_elements, nu = oracle_nsub(p), M = nu * N;
    double *cen = malloc(sizeof(double) * 3 * M);
    oracle_centroids(p, cen, cen + M, cen + 2 * M);
    const double *xc = cen, *zc = cen + M, *psi = cen + 2 * M;

#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t iq = 0; iq < nq; ++iq) {
        double f = (double)qlist[iq] * p->fs / p->n_samples;
        double w = 2.0 * M_PI * f;
        cplx *g = malloc(sizeof(cplx) * M);
        cplx *P = malloc(sizeof(cplx) * T);
        cplx *Pse = calloc((size_t)T * M, sizeof(cplx));
        cplx *Wn = malloc(sizeof(cplx) * (size_t)T * M);
        for (int32_t t = 0; t < T; ++t)
            for (int32_t n = 0; n < M; ++n) {
                int32_t e = n / nu;   /* W_n = W_ceil(n/nu), dtau_n = dtau_ceil(n/nu) */
                Wn[(size_t)t * M + n] = apod[t * N + e] * cexp(I * w * delays[t * N + e]);
            }
        for (int64_t s = 0; s < S; ++s) {
            double Ys = y ? y[s] : 0.0;
            for (int32_t n = 0; n < M; ++n)
                g[n] = green(p, nu, f, xc[n], zc[n], psi[n], x[s], Ys, z[s]);
            for (int32_t t = 0; t < T; ++t) {
                cplx acc = 0.0;
                for (int32_t n = 0; n < M; ++n) acc += Wn[(size_t)t * M + n] * g[n];
                P[t] = acc;
            }
            for (int32_t t = 0; t < T; ++t)
                for (int32_t m = 0; m < M; ++m)
                    Pse[(size_t)t * M + m] += R[s] * P[t] * g[m];
        }
        cplx H = transfer(p, w);
        for (int32_t t = 0; t < T; ++t)
            for (int32_t e = 0; e < N; ++e) {
                cplx Pe = 0.0;
                for (int32_t mu = 0; mu < nu; ++mu) Pe += Pse[(size_t)t * M + e * nu + mu];
                cplx X = H * Pe;
                size_t o = (((size_t)t * N + e) * nq + iq) * 2;
                out[o] = creal(X);
                out[o + 1] = cimag(X);
            }
        free(g); free(P); free(Pse); free(Wn);
    }
    free(cen);
}

/* R5: direct inverse DFT of the kept bins, rf[c][j] = Re sum_q X[c][q] e^{-2 pi i q j/Nt};
 * (q j) mod Nt is reduced exactly in integers before the trigonometric call. */
void oracle_idft(int32_t n_chan, int32_t nt, int32_t nq, const int32_t *qlist,
                 const double *X, double *rf)
{
#pragma omp parallel for schedule(static)
    for (int32_t c = 0; c < n_chan; ++c) {
        for (int32_t j = 0; j < nt; ++j) {
            double acc = 0.0;
            for (int32_t iq = 0; iq < nq; ++iq) {
                int64_t m = ((int64_t)qlist[iq] * j) % nt;
                double ph = -2.0 * M_PI * (double)m / nt;
                cplx Xq = X[((size_t)c * nq + iq) * 2] + I * X[((size_t)c * nq + iq) * 2 + 1];
                acc += creal(Xq * cexp(I * ph));
            }
            rf[(size_t)c * nt + j] = acc;
        }
    }
}

/* RF time signals of every element and transmit (Eq. 32-34 then R5): rf [T][N][Nt]. */
int32_t oracle_rf(const oracle_params *p, int32_t T, const double *delays, const double *apod,
                  int64_t S, const double *x, const double *y, const double *z,
                  const double *R, double *rf)
{
    int32_t q_lo, q_hi;
    int32_t nq = oracle_bins(p, &q_lo, &q_hi);
    int32_t N = p->n_elements;
    if (nq <= 0) {
        memset(rf, 0, sizeof(double) * (size_t)T * N * p->n_samples);
        return 0;
    }
    int32_t *qlist = malloc(sizeof(int32_t) * nq);
    for (int32_t i = 0; i < nq; ++i) qlist[i] = q_lo + i;
    double *X = malloc(sizeof(double) * 2 * (size_t)T * N * nq);
    oracle_rf_spectrum(p, T, delays, apod, S, x, y, z, R, nq, qlist, X);
    oracle_idft(T * N, p->n_samples, nq, qlist, X, rf);
    free(X); free(qlist);
    return nq;
}

/* Eq. 42 step (R8): the number of midpoint frequencies for points at distance at most
 * r_max from every sub-element and transmit delays at most tau_max:
 *   dw_max = 2 pi / (r_max / c + tau_max),  N_f = ceil(2 w_c / dw_max). */
int32_t oracle_pfield_nfreq(const oracle_params *p, double r_max, double tau_max)
{
    double wc = 2.0 * M_PI * p->fc;
    double dw_max = 2.0 * M_PI / (r_max / p->c + tau_max);
    return (int32_t)ceil(2.0 * wc / dw_max);
}

/* Eq. 22 and Eq. 41-42 (R3, R8): RMS pressure of each transmit at each point,
 *   P(X, w)   = S_P sqrt(S_T) sum_n W_n g_n(X) exp(i w dtau_n)
 *   P_RMS(X)  = sqrt(dw sum_j |P(X, w_j)|^2),  w_j = (j + 1/2) dw,  dw = 2 w_c / N_f.
 * prms: [T][npts]. */
void oracle_pfield(const oracle_params *p, int32_t T, const double *delays, const double *apod,
                   int64_t npts, const double *x, const double *y, const double *z,
                   int32_t nf, double *prms)
{
    int32_t N = p->n_elements, nu = oracle_nsub(p), M = nu * N;
    double *cen = malloc(sizeof(double) * 3 * M);
    oracle_centroids(p, cen, cen + M, cen + 2 * M);
    double wc = 2.0 * M_PI * p->fc;
    double dw = 2.0 * wc / nf;

#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < npts; ++i) {
        double Y = y ? y[i] : 0.0;
        for (int32_t t = 0; t < T; ++t) {
            double sum = 0.0;
            for (int32_t j = 0; j < nf; ++j) {
                double w = (j + 0.5) * dw;
                double f = w / (2.0 * M_PI);
                cplx Ptx = oracle_pulse_spectrum_c(p, w) * sqrt(oracle_transducer_response(p, w));
                cplx P = 0.0;
                for (int32_t n = 0; n < M; ++n) {
                    int32_t e = n / nu;
                    P += apod[t * N + e]
                       * green(p, nu, f, cen[n], cen[M + n], cen[2 * M + n], x[i], Y, z[i])
                       * cexp(I * w * delays[t * N + e]);
                }
                P *= Ptx;
                sum += creal(P) * creal(P) + cimag(P) * cimag(P);
            }
            prms[(size_t)t * npts + i] = sqrt(dw * sum);
        }
    }
    free(cen);
}

/* ---------------------------------------------------------------------------------
 * Gradient of L through rf (not in the paper): vector-Jacobian product of oracle_rf.
 *
 * With drf = dL/drf [T][N][Nt] and Lambda_q(e,t) = S_P S_T sum_j drf e^{-2 pi i q j/Nt},
 *   dL = Re sum_{q,t,e} Lambda_q(e,t) dP^e_q(e,t).
 * Writing G_e = sum_mu g_(e,mu), c_te = W_te e^{i w dtau_te}, P_t = sum_e c_te G_e and
 * A_t = sum_e Lambda(e,t) G_e (all at one bin q and scatterer s):
 *   dL/dR_s        = Re sum_{q,t} A_t P_t
 *   dL/dX_s        = R_s Re sum_{q,t} (A_t sum_e c_te dG_e/dX + P_t sum_e Lambda dG_e/dX)
 *   dL/dZ_s        likewise with d/dZ
 *   dL/ddtau_te    = Re sum_{q,s} R_s A_t G_e i w c_te
 * with dg/dX, dg/dZ the exact derivatives of Eq. 17/19/39/40 (Y = 0 and Y != 0).
 * ------------------------------------------------------------------------------- */

/* sinc'(x) = (cos x - sinc x) / x, 0 at x = 0. */
static double dsinc(double x)
{
    if (fabs(x) < 1e-4) return -x / 3.0 + x * x * x / 30.0;
    return (cos(x) - sin(x) / x) / x;
}

/* g and its derivatives with respect to the scatterer's X and Z. */
static void green_grad(const oracle_params *p, int32_t nu, double f, double xc, double zc,
                       double psi, double X, double Y, double Z, cplx *g, cplx *gx, cplx *gz)
{
    double k = 2.0 * M_PI * f / p->c;
    double ka = absorption(p, k);
    double bh = p->width / 2.0 / nu;
    geom G = geometry(xc, zc, psi, X, Y, Z);
    if (G.cos_t <= 0.0) { *g = *gx = *gz = 0.0; return; }

    /* E(r) = exp(i (k + i ka) r) / r and dE/dr; 2-D: / sqrt(r), no delta (R14) */
    cplx E, dE;
    if (p->two_d) {
        E = cexp(I * (k + I * ka) * G.r) / sqrt(G.r);
        dE = E * (I * k - ka - 0.5 / G.r);
    } else {
        E = cexp(I * (k + I * ka) * G.r) / G.r;
        dE = E * (I * k - ka - 1.0 / G.r);
    }

    /* delta(r) and d delta / dr (Eq. 14-16 differentiated in r) */
    double h = p->height;
    double inv_rf = isinf(p->elev_focus) ? 0.0 : 1.0 / p->elev_focus;
    double r = G.r;
    cplx beta = -I * k * Y / r, dbeta = I * k * Y / (r * r);
    cplx gamma = I * k * Y * Y / (2.0 * r), dgamma = -I * k * Y * Y / (2.0 * r * r);
    cplx delta = 0.0, ddelta = 0.0;
    if (p->two_d) delta = 1.0;
    for (int gg = 0; gg < 4 && !p->two_d; ++gg) {
        cplx A = A_RE[gg] + I * A_IM[gg];
        cplx B = B_RE[gg] + I * B_IM[gg];
        cplx alpha = B / (h * h) + I * k / 2.0 * (inv_rf - 1.0 / r);
        cplx dalpha = I * k / (2.0 * r * r);
        cplx phi = beta * beta / (4.0 * alpha) + gamma;
        cplx dphi = 2.0 * beta * dbeta / (4.0 * alpha)
                  - beta * beta * dalpha / (4.0 * alpha * alpha) + dgamma;
        cplx term = A * csqrt(M_PI / alpha) * cexp(phi);
        delta += term;
        ddelta += term * (dphi - dalpha / (2.0 * alpha));
    }

    /* D(sin theta, cos theta) and its partial derivatives */
    double u = k * bh * G.sin_t;
    double s0 = sinc(u), s1 = dsinc(u) * k * bh;   /* d sinc / d sin_t */
    double ob, dob;                                /* obliquity and d/d cos_t */
    if (p->baffle == 0) { ob = G.cos_t; dob = 1.0; }
    else if (p->baffle == 1) { ob = 1.0; dob = 0.0; }
    else { ob = G.cos_t / (G.cos_t + p->zeta); dob = p->zeta / ((G.cos_t + p->zeta) * (G.cos_t + p->zeta)); }
    double D = s0 * ob;
    double dD_dsin = s1 * ob, dD_dcos = s0 * dob;

    double rho = G.rho, rho3 = rho * rho * rho;
    double dsin_dx = G.cpsi / rho - G.lx * G.dx / rho3;
    double dcos_dx = G.spsi / rho - G.lz * G.dx / rho3;
    double dsin_dz = -G.spsi / rho - G.lx * G.dz / rho3;
    double dcos_dz = G.cpsi / rho - G.lz * G.dz / rho3;
    double dD_dx = dD_dsin * dsin_dx + dD_dcos * dcos_dx;
    double dD_dz = dD_dsin * dsin_dz + dD_dcos * dcos_dz;
    double dr_dx = G.dx / r, dr_dz = G.dz / r;

    *g = E * D * delta;
    *gx = (dE * delta + E * ddelta) * D * dr_dx + E * delta * dD_dx;
    *gz = (dE * delta + E * ddelta) * D * dr_dz + E * delta * dD_dz;
}

void oracle_green_grad(const oracle_params *p, double f, double X, double Y, double Z, int32_t n,
                       double *out /* g, dg/dX, dg/dZ as (re, im) pairs */)
{
    int32_t nu = oracle_nsub(p), M = nu * p->n_elements;
    double *cen = malloc(sizeof(double) * 3 * M);
    oracle_centroids(p, cen, cen + M, cen + 2 * M);
    cplx g, gx, gz;
    green_grad(p, nu, f, cen[n], cen[M + n], cen[2 * M + n], X, Y, Z, &g, &gx, &gz);
    free(cen);
    out[0] = creal(g); out[1] = cimag(g);
    out[2] = creal(gx); out[3] = cimag(gx);
    out[4] = creal(gz); out[5] = cimag(gz);
}

/* VJP of oracle_rf. Any of g_R, g_x, g_z, g_delay may be NULL. */
void oracle_rf_grad(const oracle_params *p, int32_t T, const double *delays, const double *apod,
                    int64_t S, const double *x, const double *y, const double *z,
                    const double *R, const double *drf, double *g_R, double *g_x,
                    double *g_z, double *g_delay)
{
    int32_t N = p->n_elements, nu = oracle_nsub(p), M = nu * N, nt = p->n_samples;
    int32_t q_lo, q_hi;
    int32_t nq = oracle_bins(p, &q_lo, &q_hi);
    if (g_R) memset(g_R, 0, sizeof(double) * S);
    if (g_x) memset(g_x, 0, sizeof(double) * S);
    if (g_z) memset(g_z, 0, sizeof(double) * S);
    if (g_delay) memset(g_delay, 0, sizeof(double) * (size_t)T * N);
    if (nq <= 0) return;

    double *cen = malloc(sizeof(double) * 3 * M);
    oracle_centroids(p, cen, cen + M, cen + 2 * M);

    /* Lambda_q(e,t) = S_P S_T sum_j drf[t][e][j] exp(-2 pi i q j / Nt) */
    cplx *Lam = malloc(sizeof(cplx) * (size_t)nq * T * N);
#pragma omp parallel for schedule(static)
    for (int32_t iq = 0; iq < nq; ++iq) {
        int32_t q = q_lo + iq;
        cplx H = transfer(p, 2.0 * M_PI * q * p->fs / nt);
        for (int32_t c = 0; c < T * N; ++c) {
            cplx acc = 0.0;
            for (int32_t j = 0; j < nt; ++j) {
                int64_t m = ((int64_t)q * j) % nt;
                acc += drf[(size_t)c * nt + j] * cexp(-2.0 * M_PI * I * (double)m / nt);
            }
            Lam[(size_t)iq * T * N + c] = H * acc;
        }
    }

    double *gd_all = calloc((size_t)T * N, sizeof(double));
#pragma omp parallel
    {
        cplx *g = malloc(sizeof(cplx) * M), *gx = malloc(sizeof(cplx) * M), *gz = malloc(sizeof(cplx) * M);
        cplx *Ge = malloc(sizeof(cplx) * N), *Gx = malloc(sizeof(cplx) * N), *Gz = malloc(sizeof(cplx) * N);
        cplx *cte = malloc(sizeof(cplx) * (size_t)T * N);
        double *gd = calloc((size_t)T * N, sizeof(double));
#pragma omp for schedule(dynamic, 4)
        for (int64_t s = 0; s < S; ++s) {
            double Ys = y ? y[s] : 0.0;
            double aR = 0.0, ax = 0.0, az = 0.0;
            for (int32_t iq = 0; iq < nq; ++iq) {
                double f = (double)(q_lo + iq) * p->fs / nt;
                double w = 2.0 * M_PI * f;
                for (int32_t n = 0; n < M; ++n)
                    green_grad(p, nu, f, cen[n], cen[M + n], cen[2 * M + n], x[s], Ys, z[s],
                               &g[n], &gx[n], &gz[n]);
                for (int32_t e = 0; e < N; ++e) {
                    Ge[e] = Gx[e] = Gz[e] = 0.0;
                    for (int32_t mu = 0; mu < nu; ++mu) {
                        Ge[e] += g[e * nu + mu]; Gx[e] += gx[e * nu + mu]; Gz[e] += gz[e * nu + mu];
                    }
                }
                for (int32_t t = 0; t < T; ++t)
                    for (int32_t e = 0; e < N; ++e)
                        cte[t * N + e] = apod[t * N + e] * cexp(I * w * delays[t * N + e]);
                const cplx *L = Lam + (size_t)iq * T * N;
                for (int32_t t = 0; t < T; ++t) {
                    cplx P = 0, A = 0, Px = 0, Ax = 0, Pz = 0, Az = 0;
                    for (int32_t e = 0; e < N; ++e) {
                        P += cte[t * N + e] * Ge[e];
                        A += L[t * N + e] * Ge[e];
                        Px += cte[t * N + e] * Gx[e];
                        Ax += L[t * N + e] * Gx[e];
                        Pz += cte[t * N + e] * Gz[e];
                        Az += L[t * N + e] * Gz[e];
                    }
                    aR += creal(A * P);
                    ax += R[s] * creal(A * Px + P * Ax);
                    az += R[s] * creal(A * Pz + P * Az);
                    for (int32_t e = 0; e < N; ++e)
                        gd[t * N + e] += creal(R[s] * A * Ge[e] * I * w * cte[t * N + e]);
                }
            }
            if (g_R) g_R[s] = aR;
            if (g_x) g_x[s] = ax;
            if (g_z) g_z[s] = az;
        }
#pragma omp critical
        for (int32_t i = 0; i < T * N; ++i) gd_all[i] += gd[i];
        free(g); free(gx); free(gz); free(Ge); free(Gx); free(Gz); free(cte); free(gd);
    }
    if (g_delay) memcpy(g_delay, gd_all, sizeof(double) * (size_t)T * N);
    free(gd_all); free(Lam); free(cen);
}
