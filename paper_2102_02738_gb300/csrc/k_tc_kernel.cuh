// k_tc_kernel.cuh -- the persistent tensor-core kernel k_tc_rf and its device helpers.
// Included by the translation units that instantiate it (k_tc_rf_*.cu, one per group of
// template arguments, compiled in parallel) and by k_tc.cu for the shared constants.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "green.cuh"
#include "simus_internal.h"
#include "tcgen05.cuh"

namespace simus {

namespace {
constexpr int kThreads = 512;
constexpr int kSB = 128;          // scatterers per tile
constexpr int kMaxWait = 1 << 22; // polls before a wait is declared timed out
constexpr size_t kHeader = 128;   // mbarriers, tensor-memory slot, flags, item index

// FP16 or BF16 (bf16 is uniform over a launch) pair of halves, lo in the low 16 bits
__device__ __forceinline__ uint32_t h16x2(bool bf16, float lo, float hi) {
    if (bf16) {
        const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<const uint32_t *>(&v);
    }
    const __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// Two FP32 values as BF16 leading parts (hi) and BF16 remainders (rem = v - hi, rounded):
// hi + rem carries 16 significant bits, and a product of two such pairs formed as
// hi hi' + hi rem' + rem hi' misses only rem rem' (relative 2^-16) and the remainders'
// own roundings (2^-17 each).
__device__ __forceinline__ void bf16_split2(float a, float b, uint32_t &hi, uint32_t &rem) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 r = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    rem = *reinterpret_cast<const uint32_t *>(&r);
}



// Sub-element records of element pairs for gen_two2 (Y = 0): pair p = elements 2p, 2p + 1
// (the last element repeated for odd N), sub-element mu at [2 (p nu + mu)], two float4 with
// the pair's values side by side: linear arrays (-x_h, -x_h', -x_l, -x_l'), (0, 0, 0, 0);
// convex arrays (cos psi, cos psi', sin psi, sin psi'), (-l0, -l0', -z0, -z0').
__device__ __forceinline__ void paired_sub(const SubElem &a, const SubElem &b, bool linear,
                                           float4 &A, float4 &B) {
    if (linear) {
        A = make_float4(-a.xh, -b.xh, -a.xl, -b.xl);
        B = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        A = make_float4(a.cpsi, b.cpsi, a.spsi, b.spsi);
        B = make_float4(-a.l0, -b.l0, -a.z0, -b.z0);
    }
}

// sinc(x) of both halves by the short fits (MODE 1, 2); MODE 0 per half.
template <int MODE>
__device__ __forceinline__ float2 sinc_short2(float2 x) {
    if (MODE == 1) {
        const float2 s = mul2(x, x);
        float2 p = fma2(dup2(2.1803757591e-06f), s, dup2(-1.9345620240e-04f));
        p = fma2(p, s, dup2(8.3155957982e-03f));
        p = fma2(p, s, dup2(-1.6664430499e-01f));
        return fma2(p, s, dup2(9.9999547005e-01f));
    }
    if (MODE == 2) {
        const float2 s = mul2(x, x);
        float2 p = fma2(dup2(-1.6607067721e-08f), s, dup2(2.5681124498e-06f));
        p = fma2(p, s, dup2(-1.9642902771e-04f));
        p = fma2(p, s, dup2(8.3237346262e-03f));
        p = fma2(p, s, dup2(-1.6664959490e-01f));
        return fma2(p, s, dup2(9.9999505281e-01f));
    }
    return make_float2(sinc_short<0>(x.x), sinc_short<0>(x.y));
}

// Sub-element sums (Eq. 33) of the Green's terms of elements e0 and e0 + 1 for one
// scatterer at the NB consecutive bins qA, qA + 1, ...: the two elements' evaluation chains
// in the .x and .y halves of packed FP32 pairs (green.cuh), each FP32 operation of both
// chains one f32x2 instruction, and one geometry setup per (scatterer, sub-element) for all
// NB bins.  The SFU operations, the table pieces (rows differ per chain) and the range
// checks stay per chain.  An element past N is evaluated on element N - 1 with zero
// amplitude (no branch).
// - Geometry in FP32 (local coordinates from the rotated centroid, r^2 with Y^2 where
//   HAS_Y, one Newton step on r; absolute error ~ulp(0.1 m), relative error of r ~1e-7:
//   a phase error below 3e-4 rad at the highest bin, under the 2^-11 rounding of the FP16
//   operands) with the phase rate u = r df / c an exact double-float product: the phase is
//   reduced exactly at bin qA, the later bins advance the phasor by one bin's phase and
//   absorption.
// - At Y = 0 with the table (TAB), bin qA picks the piece and the later bins reuse it: bin
//   qA + b moves u by b kap/dx, small except within a few mm of the sub-element; up to half
//   an interval outside the piece it is extrapolated, beyond that the bin takes its own
//   piece, and outside the table delta is evaluated directly (Eq. 16).  QUAD: the table
//   holds quadratic pieces (the FP16 kernels), else cubic ones (split BF16).
// - HAS_Y: delta of Eq. 14 with the exponential factors (delta_y2), accumulated bin by bin.
// sub: paired records (paired_sub).  (ore, oim)[b]: Re, Im of both elements at bin qA + b.
template <int NB, bool TAB, int SINC, bool LINEAR, bool QUAD, bool HAS_Y>
__device__ __forceinline__ void gen_two2(const GreenConst &gc, const float4 *sub,
                                         const float4 *tabs, const float4 &ps, int e0, float qA,
                                         float2 (&ore)[NB], float2 (&oim)[NB]) {
    const int N = gc.N, nu = gc.nu;
    const float2 wv = make_float2(e0 < N ? 1.0f : 0.0f, e0 + 1 < N ? 1.0f : 0.0f);
    const int pb = (min(e0, N - 1) >> 1) * nu;
    const float t0 = gc.tab_x0 * gc.tab_inv_dx, tmax = (float)gc.tab_n - 0.5f;
#pragma unroll
    for (int b = 0; b < NB; ++b) ore[b] = oim[b] = make_float2(0.0f, 0.0f);
    const float2 xs2 = dup2(ps.x), zs2 = dup2(ps.z);
    for (int mu = 0; mu < nu; ++mu) {
        const float4 A = sub[2 * (pb + mu)];
        float2 lx, lz;
        if (LINEAR) {
            lx = add2(add2(xs2, make_float2(A.x, A.y)), make_float2(A.z, A.w));
            lz = zs2;
        } else {
            const float4 B = sub[2 * (pb + mu) + 1];
            const float2 cp = make_float2(A.x, A.y), sp = make_float2(A.z, A.w);
            lx = fma2(xs2, cp, fma2(dup2(-ps.z), sp, make_float2(B.x, B.y)));
            lz = fma2(xs2, sp, fma2(zs2, cp, make_float2(B.z, B.w)));
        }
        float2 rho2 = fma2(lx, lx, mul2(lz, lz));
        float2 r2 = HAS_Y ? add2(rho2, dup2(ps.y * ps.y)) : rho2;
        const bool v0 = r2.x > 1e-24f, v1 = r2.y > 1e-24f;   // a scatterer on a centroid is dropped
        if (!v0) r2.x = rho2.x = 1.0f;
        if (!v1) r2.y = rho2.y = 1.0f;
        const float2 rr = make_float2(rsqrt_a(r2.x), rsqrt_a(r2.y));
        // the azimuth angle from the in-plane distance (Y != 0), else from r
        const float2 irho = HAS_Y ? make_float2(rsqrt_a(rho2.x), rsqrt_a(rho2.y)) : rr;
        const float2 r0 = mul2(r2, rr);
        const float2 rh = fma2(fma2(neg2(r0), r0, r2), mul2(dup2(0.5f), rr), r0);
        const float2 uh = mul2(rh, dup2(gc.Kh));
        const float2 ul = fma2(rh, dup2(gc.Kl), fma2(rh, dup2(gc.Kh), neg2(uh)));
        const float2 sin_t = mul2(lx, irho), cos_t = mul2(lz, irho);
        float2 ob = gc.baffle == SIMUS_BAFFLE_SOFT ? cos_t
                  : (gc.baffle == SIMUS_BAFFLE_RIGID ? dup2(1.0f)
                     : make_float2(cos_t.x / (cos_t.x + gc.zeta), cos_t.y / (cos_t.y + gc.zeta)));
        if (!(cos_t.x > 0.0f) || !v0) ob.x = 0.0f;          // behind the aperture (Eq. 39 reading)
        if (!(cos_t.y > 0.0f) || !v1) ob.y = 0.0f;
        const float2 ea = mul2(dup2(-qA * gc.att2), rh);
        const float2 a1 = gc.two_d ? make_float2(rsqrt_a(rh.x), rsqrt_a(rh.y)) : mul2(dup2(gc.h), rr);
        const float2 amp0 = mul2(mul2(mul2(a1, ob), make_float2(ex2_a(ea.x), ex2_a(ea.y))), wv);
        const float2 sa = mul2(dup2(-gc.att2), rh);
        const float2 mstep = make_float2(ex2_a(sa.x), ex2_a(sa.y));
        const float2 xb = mul2(dup2(gc.k1b), sin_t);
        const float2 kap = mul2(dup2(gc.kh * gc.h2), add2(dup2(gc.inv_rf), neg2(rr)));

        float2 kt = make_float2(0.f, 0.f), u = make_float2(0.f, 0.f), tq = make_float2(0.f, 0.f);
        int ti[2] = {0, 0};
        bool ok = TAB, far = false;
        if (TAB) {
            kt = mul2(kap, dup2(gc.tab_inv_dx));
            tq = fma2(dup2(qA), kt, dup2(-t0));
            const float fl0 = floorf(fminf(fmaxf(tq.x, 0.0f), tmax));
            const float fl1 = floorf(fminf(fmaxf(tq.y, 0.0f), tmax));
            ti[0] = (int)fl0;
            ti[1] = (int)fl1;
            u = add2(tq, make_float2(-fl0, -fl1));
            const float2 ue = fma2(dup2((float)(NB - 1)), kt, u);   // the last bin's u
            ok = u.x >= 0.0f && u.x <= 1.0f && u.y >= 0.0f && u.y <= 1.0f;
            far = !(ue.x >= -0.5f && ue.x <= 1.5f) || !(ue.y >= -0.5f && ue.y <= 1.5f);
        }
        float4 lo[2], hi[2];
        if (TAB) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                lo[c] = tabs[2 * ti[c]];
                if (QUAD) {   // c2 only
                    const float2 h = reinterpret_cast<const float2 *>(tabs)[2 * (2 * ti[c] + 1)];
                    hi[c] = make_float4(h.x, h.y, 0.f, 0.f);
                } else {
                    hi[c] = tabs[2 * ti[c] + 1];
                }
            }
        }
        // phase seed at the first bin (exact reduction of q u), then the phasor step
        float2 zr, zi, wr = make_float2(0.f, 0.f), wi = make_float2(0.f, 0.f);
        {
            const float2 q2 = dup2(qA);
            const float2 a = mul2(q2, uh);
            const float2 e = fma2(q2, ul, fma2(q2, uh, neg2(a)));
            const float2 fr = add2(add2(a, make_float2(-rintf(a.x), -rintf(a.y))), e);
            const float2 ph = mul2(dup2(6.283185307179586f), fr);
            float2 sn, cs;
            sincos_a(ph.x, sn.x, cs.x);
            sincos_a(ph.y, sn.y, cs.y);
            zr = mul2(amp0, cs);
            zi = mul2(amp0, sn);
            if (NB > 1) {
                const float2 fu = add2(add2(uh, make_float2(-rintf(uh.x), -rintf(uh.y))), ul);
                const float2 ps2 = mul2(dup2(6.283185307179586f), fu);
                sincos_a(ps2.x, sn.x, cs.x);
                sincos_a(ps2.y, sn.y, cs.y);
                wr = mul2(mstep, cs);
                wi = mul2(mstep, sn);
            }
        }
        float2 er[NB], ei[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const float2 m = sinc_short2<SINC>(mul2(dup2(qA + (float)b), xb));
            er[b] = mul2(zr, m);
            ei[b] = mul2(zi, m);
            if (b + 1 < NB) {
                const float2 nzr = fma2(zr, wr, neg2(mul2(zi, wi)));
                zi = fma2(zr, wi, mul2(zi, wr));
                zr = nzr;
            }
        }
        float2 d[2][NB];
        if (TAB) {
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const float2 ub = fma2(dup2((float)b), kt, u);
                d[0][b] = QUAD ? quad_piece(lo[0], make_float2(hi[0].x, hi[0].y), ub.x) : cubic_piece(lo[0], hi[0], ub.x);
                d[1][b] = QUAD ? quad_piece(lo[1], make_float2(hi[1].x, hi[1].y), ub.y) : cubic_piece(lo[1], hi[1], ub.y);
            }
        }
        if (TAB && NB > 1 && far) {
            // a later bin moved more than half an interval past its piece (scatterers a few
            // mm from the sub-element): it takes its own piece
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int b = 1; b < NB; ++b) {
                    const float ktc = c ? kt.y : kt.x, uc = c ? u.y : u.x, tqc = c ? tq.y : tq.x;
                    const float ub = fmaf((float)b, ktc, uc);
                    if (!(ub >= -0.5f && ub <= 1.5f)) {
                        const float tb = fmaf((float)b, ktc, tqc);
                        const float fl = floorf(fminf(fmaxf(tb, 0.0f), tmax));
                        const int i = (int)fl;
                        const float v = tb - fl;
                        d[c][b] = QUAD ? quad_piece(tabs[2 * i], reinterpret_cast<const float2 *>(tabs)[2 * (2 * i + 1)], v)
                                       : cubic_piece(tabs[2 * i], tabs[2 * i + 1], v);
                        ok = ok && v >= 0.0f && v <= 1.0f;
                    }
                }
        }
        if (HAS_Y) {   // Eq. 14 with the exponential factors, both chains as packed pairs,
                       // accumulated bin by bin
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                float2 dre, dim;
                delta_y2(gc, kap, dup2(ps.y), rr, qA + (float)b, dre, dim);
                ore[b] = fma2(er[b], dre, fma2(neg2(ei[b]), dim, ore[b]));
                oim[b] = fma2(er[b], dim, fma2(ei[b], dre, oim[b]));
            }
            continue;
        }
        if (!ok) {   // outside the table (within ~2 mm of the sub-element): Eq. 16 directly
            PairSetup P;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                P.kap = c ? kap.y : kap.x;
#pragma unroll
                for (int b = 0; b < NB; ++b) d[c][b] = delta_f<false>(gc, P, qA + (float)b);
            }
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const float2 dre = make_float2(d[0][b].x, d[1][b].x), dim = make_float2(d[0][b].y, d[1][b].y);
            ore[b] = fma2(er[b], dre, fma2(neg2(ei[b]), dim, ore[b]));
            oim[b] = fma2(er[b], dim, fma2(ei[b], dre, oim[b]));
        }
    }
}

// One generation pass over a scatterer tile: every (scatterer, group of 8 elements) item
// at bins qA .. qA + NB - 1.  Bin 0 goes as FP16/BF16 rows of the K-major tile A0, bin 1
// to A1 when there are two shared-memory tile buffers (nbuf = 2); every further bin goes
// to a tensor-memory stash slot (slot i at columns stash + i Np: row s in lane s, Re of the
// 8 elements packed in columns 4 eg .. + 3, Im at Np/2 + 4 eg) until a buffer is free.
// The lane rule holds by construction: item it has s = it mod 128 = 32 (warp mod 4) + lane.
// Split BF16 (split, one logical buffer, at most two bins per pass): bin 0's leading parts
// go to A0 and its remainders to A1; a stash slot is 2 Np columns, the remainders at + Np.
template <int NB, int NBUF, bool TAB, bool HAS_Y, int SINC, bool LINEAR, bool SPLIT>
__device__ __forceinline__ void gen_tiles(const GreenConst &gc, const float4 *sub,
                                          const float4 *tabs, const float4 *sc, int Np,
                                          float qA, unsigned char *A0, unsigned char *A1,
                                          uint32_t stash, bool bf16, int tid) {
    constexpr int nbuf = NBUF < NB ? NBUF : NB;
    constexpr bool split = NB < 3 && SPLIT;       // (three-bin passes are never split)
    const int K1 = 2 * Np;
    const int n_groups = Np >> 3;
    const uint32_t sstride = split ? 2u * Np : (uint32_t)Np;
    for (int it = tid; it < kSB * n_groups; it += kThreads) {
        const int s = it & (kSB - 1), eg = it >> 7;
        const float4 ps = sc[s];
        uint32_t pk[NB][2][4], pr[NB][2][4];
#pragma unroll
        for (int jp = 0; jp < 4; ++jp) {
            float o[2][NB][2];
            {
                float2 ore[NB], oim[NB];
                gen_two2<NB, TAB, SINC, LINEAR, !SPLIT, HAS_Y>(gc, sub, tabs, ps, eg * 8 + 2 * jp, qA, ore, oim);
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    o[0][b][0] = ore[b].x; o[1][b][0] = ore[b].y;
                    o[0][b][1] = oim[b].x; o[1][b][1] = oim[b].y;
                }
            }
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                if (split) {
                    bf16_split2(o[0][b][0], o[1][b][0], pk[b][0][jp], pr[b][0][jp]);
                    bf16_split2(o[0][b][1], o[1][b][1], pk[b][1][jp], pr[b][1][jp]);
                } else {
                    pk[b][0][jp] = h16x2(bf16, o[0][b][0], o[1][b][0]);
                    pk[b][1][jp] = h16x2(bf16, o[0][b][1], o[1][b][1]);
                }
            }
        }
        const uint32_t ta = stash + ((uint32_t)(s & ~31) << 16) + 4u * eg;
        const uint32_t o_re = tc::kmajor_offset(s, eg * 8, K1), o_im = tc::kmajor_offset(s, Np + eg * 8, K1);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if (b < nbuf) {
                unsigned char *A = b ? A1 : A0;
                *reinterpret_cast<uint4 *>(A + o_re) = make_uint4(pk[b][0][0], pk[b][0][1], pk[b][0][2], pk[b][0][3]);
                *reinterpret_cast<uint4 *>(A + o_im) = make_uint4(pk[b][1][0], pk[b][1][1], pk[b][1][2], pk[b][1][3]);
                if (split) {
                    *reinterpret_cast<uint4 *>(A1 + o_re) = make_uint4(pr[b][0][0], pr[b][0][1], pr[b][0][2], pr[b][0][3]);
                    *reinterpret_cast<uint4 *>(A1 + o_im) = make_uint4(pr[b][1][0], pr[b][1][1], pr[b][1][2], pr[b][1][3]);
                }
            } else {
                const uint32_t ts = ta + (uint32_t)(b - nbuf) * sstride;
                tc::tmem_st4(ts, pk[b][0][0], pk[b][0][1], pk[b][0][2], pk[b][0][3]);
                tc::tmem_st4(ts + (uint32_t)(Np >> 1), pk[b][1][0], pk[b][1][1], pk[b][1][2], pk[b][1][3]);
                if (split) {
                    tc::tmem_st4(ts + (uint32_t)Np, pr[b][0][0], pr[b][0][1], pr[b][0][2], pr[b][0][3]);
                    tc::tmem_st4(ts + (uint32_t)(Np + (Np >> 1)), pr[b][1][0], pr[b][1][1], pr[b][1][2], pr[b][1][3]);
                }
            }
        }
    }
    if (NB > nbuf) tc::tmem_wait_st();
}

// Move a stashed bin from tensor memory into tile buffer A (same item-to-thread map as
// gen_tiles, so every thread reads back the lanes and columns it wrote); split BF16: the
// remainders (slot + Np) into Ar.
__device__ __forceinline__ void unstash_tile(int Np, unsigned char *A, unsigned char *Ar, bool split,
                                             uint32_t slot, int tid) {
    const int K1 = 2 * Np;
    const int n_groups = Np >> 3;
    for (int it = tid; it < kSB * n_groups; it += kThreads) {
        const int s = it & (kSB - 1), eg = it >> 7;
        const uint32_t ta = slot + ((uint32_t)(s & ~31) << 16) + 4u * eg;
        const uint32_t o_re = tc::kmajor_offset(s, eg * 8, K1), o_im = tc::kmajor_offset(s, Np + eg * 8, K1);
        uint32_t re[4], im[4];
        tc::tmem_ld4(ta, re);
        tc::tmem_ld4(ta + (uint32_t)(Np >> 1), im);
        tc::tmem_wait_ld();
        *reinterpret_cast<uint4 *>(A + o_re) = make_uint4(re[0], re[1], re[2], re[3]);
        *reinterpret_cast<uint4 *>(A + o_im) = make_uint4(im[0], im[1], im[2], im[3]);
        if (split) {
            tc::tmem_ld4(ta + (uint32_t)Np, re);
            tc::tmem_ld4(ta + (uint32_t)(Np + (Np >> 1)), im);
            tc::tmem_wait_ld();
            *reinterpret_cast<uint4 *>(Ar + o_re) = make_uint4(re[0], re[1], re[2], re[3]);
            *reinterpret_cast<uint4 *>(Ar + o_im) = make_uint4(im[0], im[1], im[2], im[3]);
        }
    }
}

}  // namespace

// SPLIT: BF16 operands as leading parts + remainders, three products per GEMM (bf16
// must then be 1); otherwise FP16 (bf16 = 0) or plain BF16 (bf16 = 1) operands.
template <bool HAS_Y, int SINC, bool LINEAR, bool SPLIT>
__global__ void __launch_bounds__(kThreads, 1)
k_tc_rf(const TcUnit *__restrict__ units, int n_units, int64_t n_items, int *counter, int *err,
        int bf16) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    __shared__ TcUnit U;                  // the current item's unit

    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);          // 3 mbarriers
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + 24);
    int *abort_flag = reinterpret_cast<int *>(smem + 28);
    long long *s_item = reinterpret_cast<long long *>(smem + 32);
    int *s_unit = reinterpret_cast<int *>(smem + 40);
    unsigned char *dyn = smem + kHeader;
    const uint32_t mbar_b1 = tc::smem_u32(&bars[0]);
    const uint32_t mbar1 = tc::smem_u32(&bars[1]);
    const uint32_t mbar2 = tc::smem_u32(&bars[2]);

    if (tid == 0) {
        tc::mbar_init(mbar_b1, 1);
        tc::mbar_init(mbar1, 1);
        tc::mbar_init(mbar2, 1);
        tc::fence_mbar_init();
        *abort_flag = 0;
        *s_unit = -1;
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(tslot), 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;

    uint32_t ph_b1 = 0, ph1 = 0, ph2 = 0;
    bool pending2 = false;     // an MMA2 commit not yet waited for
    bool aborted = false;
    bool b1_inflight = false;  // thread 0: a bulk copy into B1 not yet waited for
    int cur_unit = -1;

    auto wait_all = [&](uint32_t mbar, uint32_t parity) -> bool {
        if (!tc::mbar_wait_bounded(mbar, parity, kMaxWait)) atomicExch(abort_flag, 1);
        __syncthreads();
        return *abort_flag == 0;
    };

    while (!aborted) {
        // ---- next work item (dynamic: heavier units come first in the item order)
        if (tid == 0) {
            long long it = atomicAdd(counter, 1);
            *s_item = it;
            if (it < n_items) {
                int lo = 0, hi = n_units - 1;     // last unit with item0 <= it
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (units[mid].item0 <= it) lo = mid; else hi = mid - 1;
                }
                *s_unit = lo;
            }
        }
        __syncthreads();
        const long long item = *s_item;
        if (item >= n_items) break;
        const int ui = *s_unit;
        if (ui != cur_unit) {
            if (pending2) {   // the previous unit's MMA2 may still read the tile buffers
                if (!wait_all(mbar2, ph2)) { aborted = true; break; }
                ph2 ^= 1;
                pending2 = false;
            }
            const int nw = (int)(sizeof(TcUnit) / 4);
            for (int i = tid; i < nw; i += kThreads)
                reinterpret_cast<int *>(&U)[i] = reinterpret_cast<const int *>(&units[ui])[i];
            __syncthreads();
        }
        const GreenConst gc = U.gc;   // register copy: the per-pair setup reads it often
        const int N = gc.N, M = gc.M, nq = gc.nq;
        const int Np = U.Np, nN = U.nN, TG = U.TG, QB = U.QB, mh = U.mh, pair = U.pair;
        const int G = U.G, T = U.T, nbuf = U.nbuf;
        const int K1 = 2 * Np;
        const size_t abytes = (size_t)kSB * K1 * 2;
        // split BF16: every operand as leading part + remainder; the remainders of the
        // tile in A1, of B1 and B2 right after their leading parts
        constexpr bool split = SPLIT;
        const int nops = split ? 2 : 1;
        unsigned char *A0 = dyn;
        unsigned char *A1 = A0 + (nbuf == 2 || split ? abytes : 0);
        unsigned char *B1 = A0 + (split ? 2 : nbuf) * abytes;
        const uint32_t b1_part = (uint32_t)nN * K1 * 2, b2_part = (uint32_t)nN * 256 * 2;
        unsigned char *B2 = B1 + (size_t)nops * b1_part;
        float4 *sc = reinterpret_cast<float4 *>(B2 + (size_t)nops * b2_part);
        float4 *sub = sc + kSB;        // paired sub-element records
        float4 *tabs = sub + M + gc.nu;                                    // delta table
        const bool use_tab = !HAS_Y && gc.tab_n > 0;
        const uint32_t abuf0 = tc::smem_u32(A0), abuf1 = tc::smem_u32(A1);
        const uint32_t b1s = tc::smem_u32(B1), b2s = tc::smem_u32(B2);
        const uint32_t idesc1 = tc::idesc_f16(128, nN, bf16 != 0);
        const uint32_t idesc2 = idesc1 | (1u << 15) | (1u << 16);   // A and B MN-major
        const uint32_t b1_bytes = nops * b1_part;
        if (ui != cur_unit) {
            {
                const int nu = gc.nu, np = ((N + 1) >> 1) * nu;
                for (int i = tid; i < np; i += kThreads) {
                    const int pp = i / nu, mu = i - pp * nu;
                    const int ea = min(2 * pp, N - 1), eb = min(2 * pp + 1, N - 1);
                    paired_sub(U.sub[ea * nu + mu], U.sub[eb * nu + mu], LINEAR, sub[2 * i], sub[2 * i + 1]);
                }
            }
            if (use_tab)
                for (int i = tid; i < 2 * gc.tab_n; i += kThreads) tabs[i] = U.dtab[i];
            cur_unit = ui;
            __syncthreads();
        }
        auto issue_b1 = [&](int k, int g) {   // weights of bin k, transmit group g
            if (tid == 0) {
                tc::mbar_arrive_expect_tx(mbar_b1, b1_bytes);
                tc::bulk_g2s(b1s, U.b1img + ((size_t)k * G + g) * nops * nN * K1, b1_bytes, mbar_b1);
                b1_inflight = true;
            }
        };

        const int64_t li = item - U.item0;
        const int bt = (int)(li % U.n_btiles), chunk = (int)(li / U.n_btiles);
        const int k0 = bt * QB;
        const int64_t tile0 = (int64_t)chunk * U.tiles_per_chunk;
        const int64_t tile1 = std::min<int64_t>(tile0 + U.tiles_per_chunk, U.n_tiles);
        const int step = pair + 1;                        // bins per generation pass
        const uint32_t stash = tmem + (uint32_t)(nN * (1 + QB * G * mh));   // stash slots of Np columns
        const uint32_t sstride = (uint32_t)(nops * Np);                     // (2 Np when split)
        for (int64_t tile = tile0; tile < tile1 && !aborted; ++tile) {
            for (int bp = 0; bp < QB && !aborted; bp += step) {
                const int nb = min(step, QB - bp);
                const int kA = min(k0 + bp, nq - 1);   // bins past the end repeat the last
                issue_b1(kA, 0);                        // (their outputs are discarded)
                if (pending2) {   // tile buffers and B2 still read by the last MMA2
                    if (!wait_all(mbar2, ph2)) { aborted = true; break; }
                    ph2 ^= 1;
                    pending2 = false;
                }
                if (bp == 0) {    // new scatterer tile
                    for (int i = tid; i < kSB; i += kThreads) {
                        int64_t s = tile * kSB + i;
                        sc[i] = s < U.S ? make_float4(U.x[s], (HAS_Y && U.y) ? U.y[s] : 0.f, U.z[s], U.rc[s])
                                        : make_float4(0.f, 0.f, 1.f, 0.f);
                    }
                    __syncthreads();
                }
                // ---- Green's tiles of bins kA .. kA + nb - 1 (buffers A0, A1, then the stash)
                const float qA = (float)(gc.q_lo + kA);
                const bool tab = !HAS_Y && use_tab;
#define SIMUS_GEN(NB_, NBUF_)                                                                     \
    do {                                                                                          \
        if (tab) gen_tiles<NB_, NBUF_, !HAS_Y, HAS_Y, SINC, LINEAR, SPLIT>(gc, sub, tabs, sc, Np, qA, A0, A1, stash, bf16 != 0, tid); \
        else gen_tiles<NB_, NBUF_, false, HAS_Y, SINC, LINEAR, SPLIT>(gc, sub, tabs, sc, Np, qA, A0, A1, stash, bf16 != 0, tid);     \
    } while (0)
                if (nb == 3) {
                    if (nbuf == 2) SIMUS_GEN(3, 2); else SIMUS_GEN(3, 1);
                } else if (nb == 2) {
                    if (nbuf == 2) SIMUS_GEN(2, 2); else SIMUS_GEN(2, 1);
                } else {
                    SIMUS_GEN(1, 1);
                }
#undef SIMUS_GEN
                tc::fence_proxy_async_smem();
                tc::fence_before_sync();
                __syncthreads();
                tc::fence_after_sync();

                // every bin of the pass, every transmit group: MMA1 -> P' -> MMA2
                for (int si = 0; si < nb * G && !aborted; ++si) {
                    const int bi_ = si / G, g = si - bi_ * G;
                    const int TGg = min(TG, T - g * TG);      // transmits of this group
                    // a stashed bin goes to buffer (bi_ - nbuf) mod nbuf: with two buffers
                    // the third bin into A0, whose last reader (MMA2 of the first bin)
                    // completed before the second bin's first P'; with one buffer every
                    // later bin into A0 once the previous bin's MMA2 has completed
                    const int buf = bi_ < nbuf ? bi_ : (bi_ - nbuf) % nbuf;
                    const uint32_t abase = buf ? abuf1 : abuf0;
                    if (bi_ >= nbuf && g == 0) {
                        if (nbuf == 1 && pending2) {
                            if (!wait_all(mbar2, ph2)) { aborted = true; break; }
                            ph2 ^= 1;
                            pending2 = false;
                        }
                        unstash_tile(Np, buf ? A1 : A0, A1, split, stash + (uint32_t)(bi_ - nbuf) * sstride, tid);
                        tc::fence_proxy_async_smem();
                        tc::fence_before_sync();
                        __syncthreads();
                        tc::fence_after_sync();
                    }
                    // ---- MMA1: D1 = A * B1^T
                    if (tid == 0) {
                        if (!tc::mbar_wait_bounded(mbar_b1, ph_b1, kMaxWait)) {
                            atomicExch(abort_flag, 1);
                        } else {
                            b1_inflight = false;
                            tc::fence_after_sync();
                            // K1 / 16 <= 32 steps of 256 bytes (16 in the descriptors'
                            // address field); unrolled so that the issuing thread does not
                            // recompute descriptors between MMAs
                            const uint64_t ad0 = tc::smem_desc(abase, 128, 16 * K1);
                            const uint64_t bd0 = tc::smem_desc(b1s, 128, 16 * K1);
                            const int nk = K1 / 16;
                            if (!split) {
#pragma unroll
                                for (int j = 0; j < 32; ++j) {
                                    if (j >= nk) break;
                                    tc::mma_f16(tmem, ad0 + 16ull * j, bd0 + 16ull * j, idesc1, j > 0 ? 1u : 0u);
                                }
                            } else {
                                // (A + A_r)(B + B_r) without A_r B_r: three products
                                const uint64_t adr = tc::smem_desc(abuf1, 128, 16 * K1);
                                const uint64_t bdr = tc::smem_desc(b1s + b1_part, 128, 16 * K1);
#pragma unroll
                                for (int j = 0; j < 32; ++j) {
                                    if (j >= nk) break;
                                    tc::mma_f16(tmem, ad0 + 16ull * j, bd0 + 16ull * j, idesc1, j > 0 ? 1u : 0u);
                                    tc::mma_f16(tmem, ad0 + 16ull * j, bdr + 16ull * j, idesc1, 1u);
                                    tc::mma_f16(tmem, adr + 16ull * j, bd0 + 16ull * j, idesc1, 1u);
                                }
                            }
                            tc::mma_commit(mbar1);
                        }
                    }
                    ph_b1 ^= 1;
                    if (!wait_all(mbar1, ph1)) { aborted = true; break; }
                    ph1 ^= 1;
                    tc::fence_after_sync();
                    if (si + 1 < nb * G) {                     // B1 is free again
                        const int sn = si + 1;
                        issue_b1(min(k0 + bp + sn / G, nq - 1), sn % G);
                    }
                    if (pending2) {                            // B2 still read by MMA2
                        if (!wait_all(mbar2, ph2)) { aborted = true; break; }
                        ph2 ^= 1;
                        pending2 = false;
                    }
                    // ---- P' = R_s P -> B2, MN-major (the 8 transmit rows of a core matrix
                    // are contiguous for one scatterer): row 2t = (Re P' | -Im P'), row
                    // 2t+1 = (Im P' | Re P') over K = (s | 128 + s), four 16-byte stores
                    // per thread and 8 transmits
                    {
                        const int sp = warp & 3, cc = warp >> 2;
                        const int s = sp * 32 + lane;
                        const float R = sc[s].w;
                        for (int c0 = cc * 16; c0 < nN; c0 += 64) {
                            float v[16];
                            tc::tmem_ld16(tmem + ((uint32_t)(sp * 32) << 16) + (uint32_t)c0, v);
                            uint32_t w0[8], w1[8], r0[8], r1[8];
#pragma unroll
                            for (int i = 0; i < 8; ++i) {
                                const int t = (c0 >> 1) + i;
                                float pr = 0.f, pi = 0.f;
                                if (t < TGg) { pr = R * v[2 * i]; pi = R * v[2 * i + 1]; }
                                if (split) {
                                    bf16_split2(pr, pi, w0[i], r0[i]);
                                    bf16_split2(-pi, pr, w1[i], r1[i]);
                                } else {
                                    w0[i] = h16x2(bf16 != 0, pr, pi);
                                    w1[i] = h16x2(bf16 != 0, -pi, pr);
                                }
                            }
                            const uint32_t nrow = (uint32_t)(nN >> 3);
                            unsigned char *q0 = B2 + ((((uint32_t)(s >> 3) * nrow + (uint32_t)(c0 >> 3)) << 7) + ((s & 7) << 4));
                            unsigned char *q1 = q0 + ((16u * nrow) << 7);        // k = 128 + s
                            *reinterpret_cast<uint4 *>(q0) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
                            *reinterpret_cast<uint4 *>(q0 + 128) = make_uint4(w0[4], w0[5], w0[6], w0[7]);
                            *reinterpret_cast<uint4 *>(q1) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
                            *reinterpret_cast<uint4 *>(q1 + 128) = make_uint4(w1[4], w1[5], w1[6], w1[7]);
                            if (split) {                               // remainders at B2 + b2_part
                                *reinterpret_cast<uint4 *>(q0 + b2_part) = make_uint4(r0[0], r0[1], r0[2], r0[3]);
                                *reinterpret_cast<uint4 *>(q0 + b2_part + 128) = make_uint4(r0[4], r0[5], r0[6], r0[7]);
                                *reinterpret_cast<uint4 *>(q1 + b2_part) = make_uint4(r1[0], r1[1], r1[2], r1[3]);
                                *reinterpret_cast<uint4 *>(q1 + b2_part + 128) = make_uint4(r1[4], r1[5], r1[6], r1[7]);
                            }
                        }
                    }
                    tc::fence_proxy_async_smem();
                    tc::fence_before_sync();
                    __syncthreads();
                    tc::fence_after_sync();
                    // ---- MMA2: D2[bin][half] (+)= A^T * B2^T, A^T the MN-major view of
                    // the tile: k-slice j covers scatterers 16 (j mod 8) .. +15 of the Re
                    // (j < 8) or Im (j >= 8) half.  In the no-swizzle MN-major form the
                    // leading byte offset is the stride between K-adjacent core matrices
                    // (scatterer groups, 16 K1 bytes) and the stride byte offset the one
                    // between MN-adjacent core matrices (element groups, 128 bytes).
                    // Descriptor steps in 16-byte units: k-slice j starts 2 (j mod 8) 16 K1
                    // bytes (scatterer groups) plus (j / 8) 16 Np bytes (Im half) into the
                    // tile, and 32 nN j bytes into B2.
                    if (tid == 0) {
                        const uint64_t sa = (uint64_t)(2 * K1), sim = (uint64_t)Np, sb = (uint64_t)(2 * nN);
                        const uint32_t acc0 = tile > tile0 ? 1u : 0u;
                        const uint64_t bd0 = tc::smem_desc(b2s, 16 * nN, 128);
                        const uint64_t bdr = tc::smem_desc(b2s + b2_part, 16 * nN, 128);
                        for (int h = 0; h < mh; ++h) {
                            const uint32_t d2 = tmem + (uint32_t)(nN * (1 + ((bp + bi_) * G + g) * mh + h));
                            const uint64_t ad0 = tc::smem_desc(abase + (uint32_t)(h * 16 * 128), 16 * K1, 128);
                            if (!split) {
#pragma unroll
                                for (int j = 0; j < 16; ++j)
                                    tc::mma_f16(d2, ad0 + (uint64_t)(j & 7) * sa + (uint64_t)(j >> 3) * sim,
                                                bd0 + (uint64_t)j * sb, idesc2, j > 0 ? 1u : acc0);
                            } else {
                                const uint64_t adr = tc::smem_desc(abuf1 + (uint32_t)(h * 16 * 128), 16 * K1, 128);
#pragma unroll
                                for (int j = 0; j < 16; ++j) {
                                    const uint64_t ka = (uint64_t)(j & 7) * sa + (uint64_t)(j >> 3) * sim;
                                    tc::mma_f16(d2, ad0 + ka, bd0 + (uint64_t)j * sb, idesc2, j > 0 ? 1u : acc0);
                                    tc::mma_f16(d2, ad0 + ka, bdr + (uint64_t)j * sb, idesc2, 1u);
                                    tc::mma_f16(d2, adr + ka, bd0 + (uint64_t)j * sb, idesc2, 1u);
                                }
                            }
                        }
                        tc::mma_commit(mbar2);
                    }
                    pending2 = true;
                }
            }
        }
        if (aborted) break;
        if (pending2) {
            if (!wait_all(mbar2, ph2)) { aborted = true; break; }
            ph2 ^= 1;
            pending2 = false;
        }
        tc::fence_after_sync();
        // ---- partial spectra of this item: part[chunk][g TG + t][e][k]
        {
            const int sp = warp & 3, cc = warp >> 2;
            for (int bg = 0; bg < QB * G; ++bg) {
                const int b = bg / G, g = bg - b * G;
                const int k = k0 + b;
                const int TGg = min(TG, T - g * TG);
                for (int h = 0; h < mh; ++h) {
                    const int e = 128 * h + sp * 32 + lane;
                    for (int c0 = cc * 16; c0 < nN; c0 += 64) {
                        float v[16];
                        tc::tmem_ld16(tmem + ((uint32_t)(sp * 32) << 16) +
                                          (uint32_t)(nN * (1 + bg * mh + h) + c0), v);
                        if (k < nq && e < N) {
#pragma unroll
                            for (int i = 0; i < 8; ++i) {
                                const int t = (c0 >> 1) + i;
                                if (t < TGg)
                                    U.part[(((size_t)chunk * T + g * TG + t) * N + e) * nq + k] =
                                        make_float2(v[2 * i], v[2 * i + 1]);
                            }
                        }
                    }
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    if (*abort_flag && tid == 0) {
        atomicExch(err, SIMUS_ERR_TIMEOUT);
        if (b1_inflight) tc::mbar_wait_bounded(mbar_b1, ph_b1, kMaxWait);   // own copy in flight
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}


using TcKernelFn = void (*)(const TcUnit *, int, int64_t, int *, int *, int);
// Instantiations, one translation unit each (see k_tc_rf_*.cu); split: the split-BF16
// kernels (k_tc_rf_bf16_*.cu).
TcKernelFn tc_kernel_y0_narrow(bool linear, bool split);
TcKernelFn tc_kernel_y0_mid(bool linear, bool split);
TcKernelFn tc_kernel_y0_wide(bool linear, bool split);
TcKernelFn tc_kernel_y1_narrow(bool linear, bool split);
TcKernelFn tc_kernel_y1_wide(bool linear, bool split);
TcKernelFn tc_kernel_bf16_y0_narrow(bool linear);
TcKernelFn tc_kernel_bf16_y0_mid(bool linear);
TcKernelFn tc_kernel_bf16_y0_wide(bool linear);
TcKernelFn tc_kernel_bf16_y1_narrow(bool linear);
TcKernelFn tc_kernel_bf16_y1_wide(bool linear);

}  // namespace simus
