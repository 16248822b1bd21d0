// k_grad.cu -- adjoint of simus_rf (vector-Jacobian product), FP32 on the CUDA cores.
//
// With drf = dL/drf and Lambda_q(e,t) = H_q sum_j drf[t][e][j] e^{-2 pi i q j / Nt} (the
// adjoint of the inverse DFT and of the transfer factor), dL = Re sum Lambda dRF_q.  Per
// bin q and scatterer s, with c_te = W e^{i w dtau} and G_e = sum_mu g (Eq. 33):
//   P_t = sum_e c_te G_e,   A_t = sum_e Lambda_te G_e
//   dL/dR_s      += Re sum_t A_t P_t
//   dL/dX_s      += R_s Re sum_t (A_t Px_t + P_t Ax_t)   (Px, Ax: the same sums of dG/dX)
//                 = R_s Re sum_e dG_e/dX W_e,   W_e = sum_t (A_t c_te + P_t Lambda_te),
//   dL/dZ_s likewise with dG/dZ,
//   B_q(t,e)     += R_s A_t G_e,   dL/d dtau_te = Re sum_q i w_q c_te B_q(t,e).
// The second form of dL/dX needs two contractions of the Green's tile (P, A) and one of
// the transmit weights (W) instead of six of the three tiles.  Green's terms and their
// derivatives are recomputed here, never stored across calls.
//
// Kernels: k_adjoint_dft (Lambda), k_grad (per tile of QB bins x chunk of scatterers,
// groups of SB scatterers: generation -> P, A -> W and B accumulation; per-bin-tile
// partial gradients and per-chunk partial B, reduced in a fixed order afterwards),
// k_grad_reduce_scat, k_grad_delays.
#include <algorithm>

#include "green.cuh"
#include "simus_internal.h"

namespace simus {

namespace {
constexpr int kGThreads = 384;  // 12 warps: the register budget of the generation allows it
constexpr int kGWarps = kGThreads / 32;
constexpr int kGQB = 2;     // bins per tile
// the Green's tiles follow QB T N complex values of B and take 16-byte stores of element
// pairs: an even QB keeps them on a 16-byte boundary for every T and N
static_assert(kGQB % 2 == 0, "k_grad's Green's tiles need an even number of bins per tile");
constexpr int kGSBMax = 16; // scatterers per group (16, or 8 where shared memory is short)

// P, A products: an item is (bin, 4 scatterers, 2 transmits) with both weight sets (32
// accumulators); ks threads (1, 2, 4 or 8) share an item along the elements, as many as
// keep every item's threads within 384.
__host__ __device__ inline int grad_ks(int SB, int T) {
    const int items = kGQB * (SB / 4) * ((T + 1) / 2);
    int ks = 1;
    while (ks < 8 && items * ks * 2 <= kGThreads) ks *= 2;
    return ks;
}
// Row strides (complex values): Green's tiles N rounded up to 2 mod 4 (the rows of
// scatterers four apart, read by one P, A load, start in different bank halves); weight
// and adjoint-spectrum rows N rounded up to 4 mod 8 (the rows of transmits two apart,
// read by one P, A load, start 16 words apart).
__host__ __device__ inline int grad_row(int N) { return N + (((2 - N) % 4) + 4) % 4; }
__host__ __device__ inline int grad_wrow(int N) { return N + (((4 - N) % 8) + 8) % 8; }

// Halve n live values across the lanes xor o: lanes with bit o clear keep the lower half,
// the others the upper half, each summed with its partner's copy.
template <int NV, int O>
__device__ __forceinline__ void halve_lanes(float (&v)[32], int lane) {
    const bool up = (lane & O) != 0;
#pragma unroll
    for (int i = 0; i < NV / 2; ++i) {
        const float send = up ? v[i] : v[i + NV / 2];
        const float keep = up ? v[i + NV / 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
    }
}
// Sum the 32 accumulators of a P, A item over its KS lanes (consecutive lanes, part =
// lane mod KS): afterwards part p holds the values p (32/KS) .. + 32/KS - 1 in v[0..].
template <int KS>
__device__ __forceinline__ void reduce_item(float (&v)[32], int lane) {
    if (KS >= 8) halve_lanes<32, 4>(v, lane);
    if (KS >= 4) halve_lanes<(KS >= 8 ? 16 : 32), 2>(v, lane);
    if (KS >= 2) halve_lanes<(KS >= 8 ? 8 : (KS >= 4 ? 16 : 32)), 1>(v, lane);
}
}  // namespace

// lam[t][k][e] = H_k sum_j drf[t][e][j] exp(-2 pi i ((q_lo + k) j mod Nt) / Nt).
// Thread per bin and CB channels; samples staged in shared memory.
template <int CB, int JB>
__global__ void __launch_bounds__(256)
k_adjoint_dft(const float *__restrict__ drf, int N, int n_chan, int nq, int q_lo, int nt,
              const float2 *__restrict__ H, float2 *__restrict__ lam) {
    __shared__ float ds[JB][CB];
    const int tid = threadIdx.x;
    const int k = blockIdx.x * 256 + tid;
    const int c0 = blockIdx.y * CB;
    const int q = q_lo + (k < nq ? k : 0);
    const float wstep = -6.283185307179586f / (float)nt;
    const int half = nt / 2;
    float ar[CB], ai[CB];
#pragma unroll
    for (int c = 0; c < CB; ++c) ar[c] = ai[c] = 0.f;
    int m = 0;   // q * j mod Nt at j = jb
    for (int jb = 0; jb < nt; jb += JB) {
        __syncthreads();
        for (int i = tid; i < JB * CB; i += 256) {
            int cc = i / JB, jj = i - cc * JB;
            int c = c0 + cc, j = jb + jj;
            ds[jj][cc] = (c < n_chan && j < nt) ? drf[(size_t)c * nt + j] : 0.f;
        }
        __syncthreads();
        const int jend = min(JB, nt - jb);
        for (int jj = 0; jj < jend; ++jj) {
            int mm = m > half ? m - nt : m;
            float s, co;
            sincos_a(wstep * (float)mm, s, co);     // exp(-2 pi i m / Nt) = co + i s
#pragma unroll
            for (int c = 0; c < CB; ++c) {
                float v = ds[jj][c];
                ar[c] = fmaf(v, co, ar[c]);
                ai[c] = fmaf(v, s, ai[c]);
            }
            m += q;
            if (m >= nt) m -= nt;
        }
    }
    if (k < nq) {
        const float2 h = H[k];
#pragma unroll
        for (int c = 0; c < CB; ++c) {
            int cc = c0 + c;
            if (cc < n_chan) {
                int t = cc / N, e = cc - t * N;
                lam[((size_t)t * nq + k) * N + e] =
                    make_float2(h.x * ar[c] - h.y * ai[c], h.x * ai[c] + h.y * ar[c]);
            }
        }
    }
}

// ---------------------------------------------------------------------------------
// Generation of two elements at once (delta table, Y = 0): elements 2p and 2p + 1 of a
// scatterer in the .x and .y halves of packed FP32 pairs (green.cuh), the same
// double-float geometry, phase reduction and derivative terms as pair_setup, pair_grad
// and green_grad_assemble, each FP32 operation of both one f32x2 instruction; the SFU
// operations, the table pieces (rows differ per element) and the direct-delta fallback stay
// per element.  Sub-element records of element pairs, pair p and sub-element mu at
// [3 (p nu + mu)]: (x_h, x_h', x_l, x_l'), (z_h, z_h', z_l, z_l'), (cos psi, cos psi',
// sin psi, sin psi'), the last element repeated for odd N.
__device__ __forceinline__ float2 sinc_poly32_2(float2 x) {
    const float2 s = mul2(x, x);
    float2 p = fma2(dup2(1.3530106150e-10f), s, dup2(-2.4705910363e-08f));
    p = fma2(p, s, dup2(2.7533500506e-06f));
    p = fma2(p, s, dup2(-1.9840424160e-04f));
    p = fma2(p, s, dup2(8.3333190001e-03f));
    p = fma2(p, s, dup2(-1.6666665754e-01f));
    return fma2(p, s, dup2(9.9999999903e-01f));
}
__device__ __forceinline__ float2 dsinc_poly2(float2 x) {   // 2 x p'(x^2), as dsinc_poly
    const float2 s = mul2(x, x);
    float2 p = fma2(dup2(6.0f * 1.3530106150e-10f), s, dup2(5.0f * -2.4705910363e-08f));
    p = fma2(p, s, dup2(4.0f * 2.7533500506e-06f));
    p = fma2(p, s, dup2(3.0f * -1.9840424160e-04f));
    p = fma2(p, s, dup2(2.0f * 8.3333190001e-03f));
    p = fma2(p, s, dup2(-1.6666665754e-01f));
    return mul2(mul2(dup2(2.0f), x), p);
}

template <bool NARROW>
__device__ __forceinline__ void grad_gen_pair(const GreenConst &gc, const float4 *subP,
                                              const float4 *tabs, float xs, float zs, int p,
                                              float q0, float2 (&Gr)[kGQB], float2 (&Gi)[kGQB],
                                              float2 (&Xr)[kGQB], float2 (&Xi)[kGQB],
                                              float2 (&Zr)[kGQB], float2 (&Zi)[kGQB]) {
    const int nu = gc.nu;
    const float t0 = gc.tab_x0 * gc.tab_inv_dx, tmax = (float)gc.tab_n - 0.5f;
    const float cdx = gc.tab_inv_dx * gc.kh * gc.h2;           // dx/dr per bin times r^2
#pragma unroll
    for (int j = 0; j < kGQB; ++j)
        Gr[j] = Gi[j] = Xr[j] = Xi[j] = Zr[j] = Zi[j] = make_float2(0.f, 0.f);
    const float2 xs2 = dup2(xs), zs2 = dup2(zs);
    for (int mu = 0; mu < nu; ++mu) {
        const float4 RA = subP[3 * (p * nu + mu)], RB = subP[3 * (p * nu + mu) + 1],
                     RC = subP[3 * (p * nu + mu) + 2];
        const float2 xh = make_float2(RA.x, RA.y), xl = make_float2(RA.z, RA.w);
        const float2 zh = make_float2(RB.x, RB.y), zl = make_float2(RB.z, RB.w);
        const float2 cp = make_float2(RC.x, RC.y), sp = make_float2(RC.z, RC.w);
        // pair_setup: double-float distance and phase rate
        const df2x dx = df_sub_f2(xs2, xh, xl), dz = df_sub_f2(zs2, zh, zl);
        df2x r2 = df_add2(df_sqr2(dx), df_sqr2(dz));
        const bool v0 = r2.h.x > 1e-24f, v1 = r2.h.y > 1e-24f;   // on a centroid: dropped
        if (!v0) { r2.h.x = 1.0f; r2.l.x = 0.0f; }
        if (!v1) { r2.h.y = 1.0f; r2.l.y = 0.0f; }
        const float2 rr = make_float2(rsqrt_a(r2.h.x), rsqrt_a(r2.h.y));
        const float2 rh0 = mul2(r2.h, rr);
        const float2 rl0 = mul2(add2(fma2(neg2(rh0), rh0, r2.h), r2.l), mul2(dup2(0.5f), rr));
        const df2x r = fast_two_sum2(rh0, rl0);
        const df2x u = df_mul2(r, df2x{dup2(gc.Kh), dup2(gc.Kl)});
        const float2 lx = fma2(dx.h, cp, neg2(mul2(dz.h, sp))), lz = fma2(dx.h, sp, mul2(dz.h, cp));
        const float2 sin_t = mul2(lx, rr), cos_t = mul2(lz, rr);
        float2 ob0 = gc.baffle == SIMUS_BAFFLE_SOFT ? cos_t
                   : (gc.baffle == SIMUS_BAFFLE_RIGID ? dup2(1.0f)
                      : make_float2(cos_t.x / (cos_t.x + gc.zeta), cos_t.y / (cos_t.y + gc.zeta)));
        if (!(cos_t.x > 0.0f) || !v0) ob0.x = 0.0f;        // behind the aperture (Eq. 39 reading)
        if (!(cos_t.y > 0.0f) || !v1) ob0.y = 0.0f;
        const float2 sa = mul2(dup2(-gc.att2), r.h);
        const float2 mstep = make_float2(ex2_a(sa.x), ex2_a(sa.y));
        const float2 xb = mul2(dup2(gc.k1b), sin_t);
        const float2 kap = mul2(dup2(gc.kh * gc.h2), sub2(dup2(gc.inv_rf), rr));
        // pair_grad: FP32 offsets and the derivatives of r, sin and cos theta
        const float2 dxf = sub2(sub2(xs2, xh), xl), dzf = sub2(sub2(zs2, zh), zl);
        const float2 lx2 = fma2(dxf, cp, neg2(mul2(dzf, sp))), lz2 = fma2(dxf, sp, mul2(dzf, cp));
        const float2 st = mul2(lx2, rr), ct = mul2(lz2, rr);
        const float2 drdx = mul2(dxf, rr), drdz = mul2(dzf, rr);
        const float2 dsdx = mul2(fma2(neg2(st), drdx, cp), rr);
        const float2 dcdx = mul2(fma2(neg2(ct), drdx, sp), rr);
        const float2 dsdz = mul2(fma2(neg2(st), drdz, neg2(sp)), rr);
        const float2 dcdz = mul2(fma2(neg2(ct), drdz, cp), rr);
        float2 ob, dob;
        if (gc.baffle == SIMUS_BAFFLE_SOFT) {
            ob = ct;
            dob = dup2(1.0f);
        } else if (gc.baffle == SIMUS_BAFFLE_RIGID) {
            ob = dup2(1.0f);
            dob = dup2(0.0f);
        } else {
            const float d0 = 1.0f / (ct.x + gc.zeta), d1 = 1.0f / (ct.y + gc.zeta);
            ob = make_float2(ct.x * d0, ct.y * d1);
            dob = make_float2(gc.zeta * d0 * d0, gc.zeta * d1 * d1);
        }
        if (!(ct.x > 0.0f) || !(ob0.x != 0.0f)) { ob.x = 0.0f; dob.x = 0.0f; }
        if (!(ct.y > 0.0f) || !(ob0.y != 0.0f)) { ob.y = 0.0f; dob.y = 0.0f; }
        const float2 rr2 = mul2(rr, rr);
        // bins: E = exp((i k - k_a) r) / r (the obliquity kept apart), phase reduced exactly
        // at every bin, absorption stepped by exp(-k_a r df / c)
        const float2 ea = mul2(dup2(-q0 * gc.att2), r.h);
        float2 amp = mul2(mul2(dup2(gc.h), rr), make_float2(ex2_a(ea.x), ex2_a(ea.y)));
        const float2 kt = mul2(kap, dup2(gc.tab_inv_dx));
        const float2 dxdr = mul2(dup2(cdx), rr2);
#pragma unroll
        for (int j = 0; j < kGQB; ++j) {
            const float q = q0 + (float)j;
            if (j > 0) amp = mul2(amp, mstep);
            const float2 ph = mul2(dup2(6.283185307179586f), df_frac_mul2(dup2(q), u));
            float2 sn, cs;
            sincos_a(ph.x, sn.x, cs.x);
            sincos_a(ph.y, sn.y, cs.y);
            const float2 Er = mul2(amp, cs), Ei = mul2(amp, sn);
            // delta / h and d(delta / h)/dr per element: the table piece, else Eq. 16-18
            const float2 tt = fma2(dup2(q), kt, dup2(-t0));
            float dv[2][4];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const float tc = c ? tt.y : tt.x;
                const float fl = floorf(fminf(fmaxf(tc, 0.0f), tmax));
                const int i = (int)fl;
                const float uu = tc - fl;
                if (uu >= 0.0f && uu <= 1.0f) {
                    const float4 lo = tabs[2 * i], hi = tabs[2 * i + 1];
                    const float2 d = cubic_piece(lo, hi, uu);
                    const float sc = q * (c ? dxdr.y : dxdr.x);
                    dv[c][0] = d.x;
                    dv[c][1] = d.y;
                    dv[c][2] = fmaf(uu, fmaf(3.0f * uu, hi.z, 2.0f * hi.x), lo.z) * sc;
                    dv[c][3] = fmaf(uu, fmaf(3.0f * uu, hi.w, 2.0f * hi.y), lo.w) * sc;
                } else {
                    PairSetup P;
                    PairGrad Q;
                    P.kap = c ? kap.y : kap.x;
                    Q.rr2 = c ? rr2.y : rr2.x;
                    delta_and_dr(gc, P, Q, q, dv[c][0], dv[c][1], dv[c][2], dv[c][3]);
                }
            }
            const float2 dr = make_float2(dv[0][0], dv[1][0]), di = make_float2(dv[0][1], dv[1][1]);
            const float2 ddr = make_float2(dv[0][2], dv[1][2]), ddi = make_float2(dv[0][3], dv[1][3]);
            // green_grad_assemble
            const float2 x = mul2(dup2(q), xb);
            float2 scv, dsc;
            if (NARROW) {
                scv = sinc_poly32_2(x);
                dsc = dsinc_poly2(x);
            } else {
                scv = make_float2(sinc_f<0>(x.x), sinc_f<0>(x.y));
                dsc = make_float2(dsinc_wide(x.x), dsinc_wide(x.y));
            }
            const float2 D = mul2(scv, ob);
            const float2 dDs = mul2(mul2(dsc, dup2(q * gc.k1b)), ob), dDc = mul2(scv, dob);
            const float2 dDx = fma2(dDs, dsdx, mul2(dDc, dcdx));
            const float2 dDz = fma2(dDs, dsdz, mul2(dDc, dcdz));
            // d/dr of exp(-k_a r) / r: -k_a - 1/r (3-D)
            const float2 a = sub2(dup2(-q * gc.att2 * 0.69314718055994531f), rr);
            const float bq = q * gc.k1;
            const float2 Qr = add2(fma2(a, dr, mul2(dup2(-bq), di)), ddr);
            const float2 Qi = add2(fma2(a, di, mul2(dup2(bq), dr)), ddi);
            const float2 Vr = fma2(Er, dr, neg2(mul2(Ei, di))), Vi = fma2(Er, di, mul2(Ei, dr));
            const float2 Wr = fma2(Er, Qr, neg2(mul2(Ei, Qi))), Wi = fma2(Er, Qi, mul2(Ei, Qr));
            const float2 Dx = mul2(D, drdx), Dz = mul2(D, drdz);
            Gr[j] = fma2(Vr, D, Gr[j]);
            Gi[j] = fma2(Vi, D, Gi[j]);
            Xr[j] = fma2(Wr, Dx, fma2(Vr, dDx, Xr[j]));
            Xi[j] = fma2(Wi, Dx, fma2(Vi, dDx, Xi[j]));
            Zr[j] = fma2(Wr, Dz, fma2(Vr, dDz, Zr[j]));
            Zi[j] = fma2(Wi, Dz, fma2(Vi, dDz, Zi[j]));
        }
    }
}

// Shared-memory rows of N complex values are padded to Nr = N + 1 (weights, adjoint
// spectra) or NrG (Green's tiles) so that rows of different transmits or scatterers start
// in different banks.  The sub-element records are held as two float4 planes indexed
// [mu][e] (centroid; normal and rotated centroid), so that the threads of a warp, which
// take consecutive elements, read consecutive 16-byte words instead of 32-byte records
// nu apart.  TAB: delta and d delta/dr from the plan's cubic pieces (staged after the other
// tiles; the derivative of the piece in its variable times dx/dr); points within ~2 mm of
// a sub-element, outside the table, take the direct four-Gaussian form.  The phase of
// every bin is reduced exactly (double-float q u) and its absorption is the previous
// bin's times exp(-k_a r df / c).
template <bool NARROW, bool TAB>
__global__ void __launch_bounds__(kGThreads, 1)
k_grad(const GreenConst gc, const SubElem *__restrict__ sub_g, const float *__restrict__ xg,
       const float *__restrict__ zg, const float *__restrict__ rcg, int64_t S, int64_t chunk_len,
       int T, int SB, const float2 *__restrict__ cw, const float2 *__restrict__ lam,
       float *__restrict__ gpart /*[3][n_qtiles][S]*/, int n_qtiles,
       float2 *__restrict__ bpart /*[n_chunks][T][nq][N]*/, const float4 *__restrict__ dtab) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = gc.N, nu = gc.nu, M = gc.M, nq = gc.nq;
    const int Nr = grad_wrow(N), NrG = grad_row(N);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int QB = kGQB;
    const int ks = grad_ks(SB, T);
    const int NCH = (N + 63) >> 6;                                  // 64-element chunks
    const int nit = QB * SB * T;
    float4 *sc = reinterpret_cast<float4 *>(smem_raw);              // [SB] (x, 0, z, R)
    float4 *subA = sc + kGSBMax;                                     // [nu][N] xh, xl, zh, zl
    float4 *subB = subA + M;                                        // [nu][N] cpsi, spsi, l0, z0
    float4 *AP = subB + M + 3 * nu;                                 // [QB][SB][T] (A_t, P_t)
    float2 *cwt = reinterpret_cast<float2 *>(AP + nit);             // [QB][T][Nr]
    float2 *lat = cwt + QB * T * Nr;                                // [QB][T][Nr]
    float2 *Bt = lat + QB * T * Nr;                                 // [QB][T][N]
    float2 *Gt = Bt + QB * T * N;                                   // [3][QB][SB][NrG]
    float *sg = reinterpret_cast<float *>(Gt + 3 * QB * SB * NrG);  // [QB][SB][T] Re A_t P_t
    float *xz = sg + nit;                                           // [2][QB][SB][NCH]
    float4 *tabs = reinterpret_cast<float4 *>(xz + ((2 * QB * SB * NCH + 3) & ~3));  // (TAB)

    const int qt = blockIdx.x, chunk = blockIdx.y;
    const int k0 = qt * QB;
    const int64_t s_begin = (int64_t)chunk * chunk_len;
    const int64_t s_end = min(S, s_begin + chunk_len);

    if (TAB)
        for (int i = tid; i < 2 * gc.tab_n; i += kGThreads) tabs[i] = dtab[i];
    if (TAB) {          // element-pair records for grad_gen_pair (in place of the planes)
        const int np = ((N + 1) >> 1) * nu;
        for (int i = tid; i < np; i += kGThreads) {
            const int pp = i / nu, mu = i - pp * nu;
            const SubElem a = sub_g[min(2 * pp, N - 1) * nu + mu], b = sub_g[min(2 * pp + 1, N - 1) * nu + mu];
            subA[3 * i] = make_float4(a.xh, b.xh, a.xl, b.xl);
            subA[3 * i + 1] = make_float4(a.zh, b.zh, a.zl, b.zl);
            subA[3 * i + 2] = make_float4(a.cpsi, b.cpsi, a.spsi, b.spsi);
        }
    } else {
        for (int i = tid; i < M; i += kGThreads) {      // global [e][mu] -> shared [mu][e]
            const float4 *r = reinterpret_cast<const float4 *>(sub_g + i);
            const int e = i / nu, mu = i - e * nu;
            subA[mu * N + e] = r[0];
            subB[mu * N + e] = r[1];
        }
    }
    for (int i = tid; i < QB * T * N; i += kGThreads) {
        int j = i / (T * N), r = i - j * T * N, t = r / N, e = r - t * N, k = k0 + j;
        bool ok = k < nq;
        const int o = (j * T + t) * Nr + e;
        cwt[o] = ok ? cw[((size_t)t * nq + k) * N + e] : make_float2(0.f, 0.f);
        lat[o] = ok ? lam[((size_t)t * nq + k) * N + e] : make_float2(0.f, 0.f);
        Bt[i] = make_float2(0.f, 0.f);
    }
    const float q0 = (float)(gc.q_lo + k0);
    const size_t plane = (size_t)QB * SB * NrG;
    // P, A items: (bin, 4 scatterers, 2 transmits), ks threads each
    const int TB = (T + 1) >> 1, SB4 = SB >> 2;
    const int units = QB * SB4 * TB * ks;
    // W and B work, one warp per unit: W units (bin, 4 scatterers, 64 elements), then B
    // units (bin, 4 transmits, 64 elements); two elements per lane, 32 apart
    const int nW = QB * SB4 * NCH, nWB = nW + QB * ((T + 3) >> 2) * NCH;

    for (int64_t sb = s_begin; sb < s_end; sb += SB) {
        __syncthreads();
        if (tid < SB) {
            int64_t s = sb + tid;
            sc[tid] = s < s_end ? make_float4(xg[s], 0.f, zg[s], rcg[s]) : make_float4(0.f, 0.f, 1.f, 0.f);
        }
        __syncthreads();

        // 1. G, dG/dX, dG/dZ tiles: two elements per item with the delta table
        if (TAB) {
            const int NP = (N + 1) >> 1;
            for (int pr = tid; pr < SB * NP; pr += kGThreads) {
                const int s = pr / NP, pp = pr - s * NP;
                const float4 ps = sc[s];
                float2 Gr[QB], Gi[QB], Xr[QB], Xi[QB], Zr[QB], Zi[QB];
                grad_gen_pair<NARROW>(gc, subA, tabs, ps.x, ps.z, pp, q0, Gr, Gi, Xr, Xi, Zr, Zi);
                const int e0 = 2 * pp;
#pragma unroll
                for (int j = 0; j < QB; ++j) {
                    const size_t o = ((size_t)j * SB + s) * NrG + e0;
                    if (e0 + 1 < N) {   // (o even: 16-byte stores of both elements)
                        *reinterpret_cast<float4 *>(Gt + o) = make_float4(Gr[j].x, Gi[j].x, Gr[j].y, Gi[j].y);
                        *reinterpret_cast<float4 *>(Gt + plane + o) = make_float4(Xr[j].x, Xi[j].x, Xr[j].y, Xi[j].y);
                        *reinterpret_cast<float4 *>(Gt + 2 * plane + o) = make_float4(Zr[j].x, Zi[j].x, Zr[j].y, Zi[j].y);
                    } else {
                        Gt[o] = make_float2(Gr[j].x, Gi[j].x);
                        Gt[plane + o] = make_float2(Xr[j].x, Xi[j].x);
                        Gt[2 * plane + o] = make_float2(Zr[j].x, Zi[j].x);
                    }
                }
            }
        }
        for (int pr = tid; pr < (TAB ? 0 : SB * N); pr += kGThreads) {
            const int s = pr / N, e = pr - s * N;
            const float4 ps = sc[s];
            float2 G[QB], GX[QB], GZ[QB];
#pragma unroll
            for (int j = 0; j < QB; ++j) G[j] = GX[j] = GZ[j] = make_float2(0.f, 0.f);
            for (int mu = 0; mu < nu; ++mu) {
                SubElem se;
                reinterpret_cast<float4 *>(&se)[0] = subA[mu * N + e];
                reinterpret_cast<float4 *>(&se)[1] = subB[mu * N + e];
                const PairSetup P = pair_setup<false>(gc, se, ps.x, 0.f, ps.z, q0);
                const PairGrad Q = pair_grad(gc, se, ps.x, ps.z, P);
                if (TAB) {
                    // E = exp((i k - k_a) r) / r (without the obliquity, which the
                    // derivative keeps apart): phase reduced exactly at every bin,
                    // absorption stepped by exp(-k_a r df / c)
                    float amp = gc.h * P.inv_r * ex2_a(-q0 * gc.att2 * P.rh);
                    const float kt = P.kap * gc.tab_inv_dx, t0 = gc.tab_x0 * gc.tab_inv_dx;
                    const float dxdr = gc.tab_inv_dx * gc.kh * gc.h2 * Q.rr2;   // per bin
#pragma unroll
                    for (int j = 0; j < QB; ++j) {
                        const float q = q0 + (float)j;
                        if (j > 0) amp *= P.mstep;
                        float sn, cs;
                        sincos_a(6.283185307179586f * df_frac_mul(q, P.u), sn, cs);
                        const float Er = amp * cs, Ei = amp * sn;
                        const float tt = fmaf(q, kt, -t0);
                        const float fl = floorf(fminf(fmaxf(tt, 0.0f), (float)gc.tab_n - 0.5f));
                        const int i = (int)fl;
                        const float u = tt - fl;
                        float dr_, di_, ddr, ddi;
                        if (u >= 0.0f && u <= 1.0f) {
                            const float4 lo = tabs[2 * i], hi = tabs[2 * i + 1];
                            const float2 d = cubic_piece(lo, hi, u);
                            dr_ = d.x;
                            di_ = d.y;
                            // d/du of the piece: c1 + u (2 c2 + 3 c3 u)
                            const float sc = q * dxdr;
                            ddr = fmaf(u, fmaf(3.0f * u, hi.z, 2.0f * hi.x), lo.z) * sc;
                            ddi = fmaf(u, fmaf(3.0f * u, hi.w, 2.0f * hi.y), lo.w) * sc;
                        } else {
                            delta_and_dr(gc, P, Q, q, dr_, di_, ddr, ddi);
                        }
                        float2 g, gx, gz;
                        green_grad_assemble<NARROW>(gc, P, Q, q, Er, Ei, dr_, di_, ddr, ddi, g, gx, gz);
                        G[j].x += g.x; G[j].y += g.y;
                        GX[j].x += gx.x; GX[j].y += gx.y;
                        GZ[j].x += gz.x; GZ[j].y += gz.y;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < QB; ++j) {
                        const float q = q0 + (float)j;
                        const float amp = (gc.two_d ? rsqrt_a(P.rh) : gc.h * P.inv_r) *
                                          ex2_a(-q * gc.att2 * P.rh);
                        float2 g, gx, gz;
                        green_grad_term<NARROW>(gc, P, Q, q, amp, g, gx, gz);
                        G[j].x += g.x; G[j].y += g.y;
                        GX[j].x += gx.x; GX[j].y += gx.y;
                        GZ[j].x += gz.x; GZ[j].y += gz.y;
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < QB; ++j) {
                const size_t o = ((size_t)j * SB + s) * NrG + e;
                Gt[o] = G[j];
                Gt[plane + o] = GX[j];
                Gt[2 * plane + o] = GZ[j];
            }
        }
        __syncthreads();


        // 2. P_t = sum_e c_te G_e and A_t = sum_e L_te G_e for 4 scatterers x 2 transmits
        // per item: 8 loads and 64 FMA per element; the item's ks partial sums are halved
        // across its lanes, so that each lane ends with whole (A_t, P_t) records
        // (an item's ks lanes are consecutive and units is a multiple of ks, so a lane
        // past the end belongs to a wholly idle item: it runs item 0 and stores nothing)
        for (int base = 0; base < units && base + warp * 32 < units; base += kGThreads) {
            const int w = base + tid;
            const bool act = w < units;
            const int it = act ? w / ks : 0, part = w - (w / ks) * ks;
            const int j = it / (SB4 * TB), r = it - j * SB4 * TB, s4 = r / TB, tb = r - s4 * TB;
            const int s0 = 4 * s4, t0 = 2 * tb;
            const float2 *g0 = Gt + ((size_t)j * SB + s0) * NrG;
            const float2 *cr[2], *lr[2];
#pragma unroll
            for (int dt = 0; dt < 2; ++dt) {
                const int t = min(t0 + dt, T - 1);          // past T: a duplicate, discarded
                cr[dt] = cwt + ((size_t)j * T + t) * Nr;
                lr[dt] = lat + ((size_t)j * T + t) * Nr;
            }
            // v[((si 2 + dt) 2 + w) 2 + (re, im)], w = 0: P (weights c), 1: A (spectra L)
            float v[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = 0.f;
#pragma unroll 2
            for (int e = part; e < N; e += ks) {
                float2 g[4];
#pragma unroll
                for (int si = 0; si < 4; ++si) g[si] = g0[si * NrG + e];
#pragma unroll
                for (int dt = 0; dt < 2; ++dt) {
                    const float2 cc = cr[dt][e], ll = lr[dt][e];
#pragma unroll
                    for (int si = 0; si < 4; ++si) {
                        float *o = v + (si * 2 + dt) * 4;
                        o[0] = fmaf(cc.x, g[si].x, fmaf(-cc.y, g[si].y, o[0]));
                        o[1] = fmaf(cc.x, g[si].y, fmaf(cc.y, g[si].x, o[1]));
                        o[2] = fmaf(ll.x, g[si].x, fmaf(-ll.y, g[si].y, o[2]));
                        o[3] = fmaf(ll.x, g[si].y, fmaf(ll.y, g[si].x, o[3]));
                    }
                }
            }
            switch (ks) {
                case 8: reduce_item<8>(v, lane); break;
                case 4: reduce_item<4>(v, lane); break;
                case 2: reduce_item<2>(v, lane); break;
                default: break;
            }
            // this lane's records: (si, dt) pairs a = part (8/ks) + m
            const int nrec = 8 / ks;
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                if (m < nrec) {
                    const int a = part * nrec + m, si = a >> 1, t = t0 + (a & 1);
                    if (act && t < T) {
                        const float Pr = v[4 * m], Pi = v[4 * m + 1];
                        const float Ar = v[4 * m + 2], Ai = v[4 * m + 3];
                        const int o = (j * SB + s0 + si) * T + t;
                        AP[o] = make_float4(Ar, Ai, Pr, Pi);
                        sg[o] = Ar * Pr - Ai * Pi;                 // dL/dR term
                    }
                }
            }
        }
        __syncthreads();

        // 3. W and B units (one warp each)
        for (int u = warp; u < nWB; u += kGWarps) {
            if (u < nW) {
                // W_e = sum_t (A_t c_te + P_t L_te) for 4 scatterers x 2 elements per lane,
                // then Re sum_e dG_e/dX W_e and Re sum_e dG_e/dZ W_e over the warp
                const int j = u / (SB4 * NCH), r = u - j * SB4 * NCH, s4 = r / NCH, ch = r - s4 * NCH;
                const int s0 = 4 * s4;
                int ec[2];
                bool ev[2];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int e = ch * 64 + lane + 32 * i;
                    ev[i] = e < N;
                    ec[i] = min(e, N - 1);                  // clamped: inside the rows
                }
                const float4 *ap = AP + (j * SB + s0) * T;
                const float2 *cj = cwt + (size_t)j * T * Nr, *lj = lat + (size_t)j * T * Nr;
                float w[4][2][2];
#pragma unroll
                for (int si = 0; si < 4; ++si)
#pragma unroll
                    for (int i = 0; i < 2; ++i) w[si][i][0] = w[si][i][1] = 0.f;
                for (int t = 0; t < T; ++t) {
                    float4 a[4];
#pragma unroll
                    for (int si = 0; si < 4; ++si) a[si] = ap[si * T + t];
                    const float2 c0 = cj[t * Nr + ec[0]], c1 = cj[t * Nr + ec[1]];
                    const float2 l0 = lj[t * Nr + ec[0]], l1 = lj[t * Nr + ec[1]];
#pragma unroll
                    for (int si = 0; si < 4; ++si) {
                        // (Ar, Ai, Pr, Pi) = a[si]
                        w[si][0][0] = fmaf(a[si].x, c0.x, fmaf(-a[si].y, c0.y, fmaf(a[si].z, l0.x, fmaf(-a[si].w, l0.y, w[si][0][0]))));
                        w[si][0][1] = fmaf(a[si].x, c0.y, fmaf(a[si].y, c0.x, fmaf(a[si].z, l0.y, fmaf(a[si].w, l0.x, w[si][0][1]))));
                        w[si][1][0] = fmaf(a[si].x, c1.x, fmaf(-a[si].y, c1.y, fmaf(a[si].z, l1.x, fmaf(-a[si].w, l1.y, w[si][1][0]))));
                        w[si][1][1] = fmaf(a[si].x, c1.y, fmaf(a[si].y, c1.x, fmaf(a[si].z, l1.y, fmaf(a[si].w, l1.x, w[si][1][1]))));
                    }
                }
                float v[32];   // v[si]: X, v[4 + si]: Z (the rest unused)
#pragma unroll
                for (int si = 0; si < 4; ++si) {
                    const size_t ro = ((size_t)j * SB + s0 + si) * NrG;
                    float x = 0.f, z = 0.f;
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const float2 gx = Gt[plane + ro + ec[i]], gz = Gt[2 * plane + ro + ec[i]];
                        if (ev[i]) {
                            x = fmaf(gx.x, w[si][i][0], fmaf(-gx.y, w[si][i][1], x));
                            z = fmaf(gz.x, w[si][i][0], fmaf(-gz.y, w[si][i][1], z));
                        }
                    }
                    v[si] = x;
                    v[4 + si] = z;
                }
#pragma unroll
                for (int o = 16; o >= 8; o >>= 1)
#pragma unroll
                    for (int i = 0; i < 8; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
                halve_lanes<8, 4>(v, lane);
                halve_lanes<4, 2>(v, lane);
                halve_lanes<2, 1>(v, lane);
                if (lane < 8) {    // lane p holds value p: X (p < 4) or Z of scatterer s0 + p mod 4
                    const int which = lane >> 2, si = lane & 3;
                    xz[which * QB * SB * NCH + (j * SB + s0 + si) * NCH + ch] = v[0];
                }
            } else {
                // B_q(t, e) += sum_s A_t (R_s G_e) for 4 transmits x 2 elements per lane
                const int b = u - nW, nT4 = (T + 3) >> 2;
                const int j = b / (nT4 * NCH), r = b - j * nT4 * NCH, t4 = r / NCH, ch = r - t4 * NCH;
                const int t0 = 4 * t4;
                int ec[2];
                bool ev[2];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int e = ch * 64 + lane + 32 * i;
                    ev[i] = e < N;
                    ec[i] = min(e, N - 1);
                }
                int tc[4];
#pragma unroll
                for (int ti = 0; ti < 4; ++ti) tc[ti] = min(t0 + ti, T - 1);
                float acc[4][2][2];
#pragma unroll
                for (int ti = 0; ti < 4; ++ti)
#pragma unroll
                    for (int i = 0; i < 2; ++i) acc[ti][i][0] = acc[ti][i][1] = 0.f;
                for (int s = 0; s < SB; ++s) {
                    const float R = sc[s].w;
                    const float2 *grow = Gt + ((size_t)j * SB + s) * NrG;
                    float2 rg[2];
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const float2 x = grow[ec[i]];
                        rg[i] = make_float2(R * x.x, R * x.y);
                    }
                    const float4 *ap = AP + (j * SB + s) * T;
#pragma unroll
                    for (int ti = 0; ti < 4; ++ti) {
                        const float2 a = *reinterpret_cast<const float2 *>(ap + tc[ti]);   // A_t
#pragma unroll
                        for (int i = 0; i < 2; ++i) {
                            acc[ti][i][0] = fmaf(a.x, rg[i].x, fmaf(-a.y, rg[i].y, acc[ti][i][0]));
                            acc[ti][i][1] = fmaf(a.x, rg[i].y, fmaf(a.y, rg[i].x, acc[ti][i][1]));
                        }
                    }
                }
#pragma unroll
                for (int ti = 0; ti < 4; ++ti) {
                    if (t0 + ti < T) {
                        float2 *bt = Bt + ((size_t)j * T + t0 + ti) * N;
#pragma unroll
                        for (int i = 0; i < 2; ++i)
                            if (ev[i]) {
                                bt[ec[i]].x += acc[ti][i][0];
                                bt[ec[i]].y += acc[ti][i][1];
                            }
                    }
                }
            }
        }
        __syncthreads();
        if (tid < 3 * SB) {       // fixed-order sums over bins and transmits / chunks
            const int which = tid / SB, s = tid - which * SB;
            float acc = 0.f;
            if (which == 0) {
                for (int j = 0; j < QB; ++j)
                    for (int t = 0; t < T; ++t) acc += sg[(j * SB + s) * T + t];
            } else {
                const float *x = xz + (which - 1) * QB * SB * NCH;
                for (int j = 0; j < QB; ++j)
                    for (int ch = 0; ch < NCH; ++ch) acc += x[(j * SB + s) * NCH + ch];
                acc *= sc[s].w;
            }
            if (sb + s < s_end)
                gpart[(size_t)which * n_qtiles * S + (size_t)qt * S + (sb + s)] = acc;
        }
    }
    __syncthreads();
    for (int i = tid; i < QB * T * N; i += kGThreads) {
        const int j = i / (T * N), r = i - j * T * N, t = r / N, e = r - t * N, k = k0 + j;
        if (k < nq) bpart[(((size_t)chunk * T + t) * nq + k) * N + e] = Bt[i];
    }
}

// g[s] = sum over bin tiles of gpart[which][qt][s] (fixed order).
__global__ void k_grad_reduce_scat(const float *__restrict__ gpart, int n_qtiles, int64_t S,
                                   float *__restrict__ g_rc, float *__restrict__ g_x,
                                   float *__restrict__ g_z) {
    const size_t pl = (size_t)n_qtiles * S;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S;
         s += (int64_t)gridDim.x * blockDim.x) {
        float a = 0.f, b = 0.f, c = 0.f;
        for (int q = 0; q < n_qtiles; ++q) {
            a += gpart[(size_t)q * S + s];
            b += gpart[pl + (size_t)q * S + s];
            c += gpart[2 * pl + (size_t)q * S + s];
        }
        if (g_rc) g_rc[s] = a;
        if (g_x) g_x[s] = b;
        if (g_z) g_z[s] = c;
    }
}

// g_delays[t][e] = Re sum_k i w_k c_te(k) sum_chunk B[chunk][t][k][e].  A block takes 32
// consecutive channels (t, e) x 16 slices of the bins (k = slice, slice + 16, ...): the
// threads of a warp read 32 consecutive elements of one (chunk, t, k) row, and the slices'
// FP64 partial sums are added in a fixed order (reproducible).
constexpr int kGdCh = 32, kGdSl = 16;
__global__ void __launch_bounds__(kGdCh * kGdSl)
k_grad_delays(const float2 *__restrict__ bpart, int n_chunks, int T, int N, int nq, int q_lo,
              double df, const float2 *__restrict__ cw, float *__restrict__ gd) {
    __shared__ double part[kGdSl][kGdCh];
    const int l = threadIdx.x % kGdCh, sl = threadIdx.x / kGdCh;
    const int i = blockIdx.x * kGdCh + l;
    double acc = 0.0;
    if (i < T * N) {
        const int t = i / N, e = i - t * N;
        for (int k = sl; k < nq; k += kGdSl) {
            float br = 0.f, bi = 0.f;
            for (int c = 0; c < n_chunks; ++c) {
                const float2 b = bpart[(((size_t)c * T + t) * nq + k) * N + e];
                br += b.x;
                bi += b.y;
            }
            const float2 cc = cw[((size_t)t * nq + k) * N + e];
            const double w = 6.283185307179586 * (double)(q_lo + k) * df;
            // Re(i w c B) = -w Im(c B)
            acc += -w * (double)(cc.x * bi + cc.y * br);
        }
    }
    part[sl][l] = acc;
    __syncthreads();
    if (sl == 0 && i < T * N) {
        double a = 0.0;
        for (int j = 0; j < kGdSl; ++j) a += part[j][l];
        gd[i] = (float)a;
    }
}

GradGeom grad_geometry(const simus_plan *p, int T, int64_t S) {
    GradGeom g{};
    g.ok = (int64_t)T * p->N <= 2048;
    g.n_qtiles = (p->nq + kGQB - 1) / kGQB;
    const int tab_full = (p->d_dtab && p->delta_table && !p->probe.two_d) ? p->gc.tab_n : 0;
    auto smem_for = [&](int SB, int tab_n) {
        const size_t nit = (size_t)kGQB * SB * T, nch = (size_t)(p->N + 63) / 64;
        return sizeof(float4) * kGSBMax + sizeof(SubElem) * p->M + 3 * sizeof(float4) * p->nu
             + sizeof(float4) * nit
             + sizeof(float2) * (size_t)kGQB * T * grad_wrow(p->N) * 2
             + sizeof(float2) * (size_t)kGQB * T * p->N
             + sizeof(float2) * (size_t)3 * kGQB * SB * grad_row(p->N)
             + sizeof(float) * nit + sizeof(float) * ((2 * kGQB * SB * nch + 3) & ~(size_t)3)
             + 2 * sizeof(float4) * (size_t)tab_n;
    };
    // 16-scatterer groups with the delta table, else without it, else 8-scatterer groups
    const size_t lim = 227 * 1024;
    g.tab = tab_full > 0 && smem_for(kGSBMax, tab_full) <= lim;
    g.SB = (g.tab || smem_for(kGSBMax, 0) <= lim) ? kGSBMax : 8;
    if (g.SB == 8) g.tab = tab_full > 0 && smem_for(8, tab_full) <= lim;
    const int tab_n = g.tab ? tab_full : 0;
    int64_t want = (int64_t)p->num_sms * 8;
    int64_t chunks = std::max<int64_t>(1, (want + g.n_qtiles - 1) / g.n_qtiles);
    chunks = std::min<int64_t>(chunks, std::max<int64_t>(1, S / (g.SB * 16)));
    int64_t len = (S + chunks - 1) / chunks;
    len = ((len + g.SB - 1) / g.SB) * g.SB;
    g.chunk_len = std::max<int64_t>(len, g.SB);
    g.n_chunks = (int)((S + g.chunk_len - 1) / g.chunk_len);
    g.smem = smem_for(g.SB, tab_n);
    g.ok = g.ok && g.smem <= lim;
    return g;
}

int launch_adjoint_dft(const simus_plan *p, const float *drf, int T, float2 *lam, cudaStream_t st) {
    constexpr int CB = 8, JB = 256;
    const int n_chan = T * p->N;
    dim3 grid((p->nq + 255) / 256, (n_chan + CB - 1) / CB);
    k_adjoint_dft<CB, JB><<<grid, 256, 0, st>>>(drf, p->N, n_chan, p->nq, p->q_lo, p->nt, p->d_H, lam);
    count_launches(1);
    return check_cuda(cudaGetLastError(), "k_adjoint_dft launch");
}

int launch_grad(const simus_plan *p, const GradGeom &g, const simus_scat *sc, int T,
                const float2 *cw, const float2 *lam, float *gpart, float2 *bpart, cudaStream_t st) {
    auto kern = p->gc.narrow == 1 ? (g.tab ? k_grad<true, true> : k_grad<true, false>)
                                  : (g.tab ? k_grad<false, true> : k_grad<false, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
    if (e != cudaSuccess) return check_cuda(e, "k_grad smem attribute");
    dim3 grid(g.n_qtiles, g.n_chunks);
    kern<<<grid, kGThreads, g.smem, st>>>(p->gc, p->d_sub, sc->x, sc->z, sc->rc, sc->n, g.chunk_len,
                                          T, g.SB, cw, lam, gpart, g.n_qtiles, bpart, p->d_dtab);
    count_launches(1);
    return check_cuda(cudaGetLastError(), "k_grad launch");
}

int launch_grad_finish(const simus_plan *p, const GradGeom &g, int T, int64_t S, const float *gpart,
                       const float2 *bpart, const float2 *cw, float *g_rc, float *g_x, float *g_z,
                       float *g_delays, cudaStream_t st) {
    if (g_rc || g_x || g_z) {
        int blocks = (int)std::min<int64_t>((S + 255) / 256, (int64_t)p->num_sms * 8);
        k_grad_reduce_scat<<<std::max(blocks, 1), 256, 0, st>>>(gpart, g.n_qtiles, S, g_rc, g_x, g_z);
        count_launches(1);
        int rc = check_cuda(cudaGetLastError(), "k_grad_reduce_scat launch");
        if (rc) return rc;
    }
    if (g_delays) {
        const int n = T * p->N;
        k_grad_delays<<<(n + kGdCh - 1) / kGdCh, kGdCh * kGdSl, 0, st>>>(bpart, g.n_chunks, T, p->N, p->nq,
                                                                       p->q_lo, p->gc.df, cw, g_delays);
        count_launches(1);
        return check_cuda(cudaGetLastError(), "k_grad_delays launch");
    }
    return SIMUS_OK;
}

}  // namespace simus
