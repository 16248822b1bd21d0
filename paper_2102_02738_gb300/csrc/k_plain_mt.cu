// k_plain_mt.cu -- plain FP32 path for several transmits: the Green's tile of a group of
// scatterers is generated once per bin and contracted against every transmit, instead
// of being regenerated per transmit.
//
// Block tile: QB (4 or 2) consecutive kept bins x one chunk of scatterers x all N elements x
// all T transmits, as large as shared memory allows.  For each group of SB scatterers the
// block
//   1. generates G_e(q, s, e) = sum_mu g(q, s, (e, mu)) (Eq. 17/20/33/39/40) for the
//      QB x SB x N tile into shared memory, one geometry setup (double-float distance
//      and phase rate) per (scatterer, sub-element) for all QB bins;
//   2. forms P_t(q, s) = sum_e C_t(q, e) G_e(q, s, e) (Eq. 29) as a register-blocked
//      product (two scatterers x two transmits per thread) and scales it by R_s;
//   3. accumulates RF_q(t, e) += sum_s G_e(q, s, e) R_s P_t(q, s) (Eq. 30-32) in shared
//      memory (four elements per thread).
// Rows of N complex values are padded to N + 1 so that rows start in different banks.
// Sub-element records sit in shared memory as two float4 planes indexed [mu][e], so that
// a warp, whose threads take consecutive elements, reads consecutive 16-byte words.
// The chunk's partial spectrum goes to part[chunk][t][e][k]; chunks are summed in a fixed
// order by the reduction kernel, so results are bitwise reproducible.
#include <algorithm>
#include <type_traits>

#include "green.cuh"
#include "simus_internal.h"

namespace simus {

namespace {
constexpr int kMtThreads = 384;
constexpr int kMtQBMax = 4;     // bins per tile (4, or 2 for many transmits)
constexpr int kMtSBMax = 32;    // scatterers per group (32, 16 or 8: what shared memory allows)
}  // namespace

// Green's terms of elements 2p and 2p + 1 of one scatterer at the QB bins (Y = 0), the two
// elements in the .x and .y halves of packed FP32 pairs (pair_setup2): the phase reduced
// exactly at every bin, the absorption stepped per bin, delta per element (table piece or
// Eq. 16).  Gr[j], Gi[j]: (Re, Re') and (Im, Im') of G_e at bin q0 + j.
template <int QB, int SINC, bool TAB>
__device__ __forceinline__ void mt_gen_pair(const GreenConst &gc, const float4 *subP,
                                            const float4 *__restrict__ dtab, float xs, float zs,
                                            int p, float q0, float2 (&Gr)[QB], float2 (&Gi)[QB]) {
    const int nu = gc.nu;
    const float t0 = TAB ? gc.tab_x0 * gc.tab_inv_dx : 0.0f, tmax = (float)gc.tab_n - 0.5f;
#pragma unroll
    for (int j = 0; j < QB; ++j) Gr[j] = Gi[j] = make_float2(0.f, 0.f);
    for (int mu = 0; mu < nu; ++mu) {
        const PairSetup2 P = pair_setup2(gc, subP + 3 * (p * nu + mu), xs, zs, q0);
        float2 amp = P.amp0;
        const float2 kt = TAB ? mul2(P.kap, dup2(gc.tab_inv_dx)) : make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < QB; ++j) {
            const float q = q0 + (float)j;
            const float2 ph = mul2(dup2(6.283185307179586f), df_frac_mul2(dup2(q), P.u));
            float2 sn, cs;
            sincos_a(ph.x, sn.x, cs.x);
            sincos_a(ph.y, sn.y, cs.y);
            const float2 m = mul2(amp, sinc_f2<SINC>(mul2(dup2(q), P.xb)));
            float dv[2][2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                PairSetup Pc;
                Pc.kap = c ? P.kap.y : P.kap.x;
                float2 d;
                if (TAB) {
                    const float tt = fmaf(q, c ? kt.y : kt.x, -t0);
                    const float fl = floorf(fminf(fmaxf(tt, 0.0f), tmax));
                    const int i = (int)fl;
                    const float u = tt - fl;
                    d = cubic_piece(__ldg(dtab + 2 * i), __ldg(dtab + 2 * i + 1), u);
                    if (!(u >= 0.0f && u <= 1.0f)) d = delta_f<false>(gc, Pc, q);   // r < ~2 mm
                } else {
                    d = delta_f<false>(gc, Pc, q);
                }
                dv[c][0] = d.x;
                dv[c][1] = d.y;
            }
            const float2 dre = make_float2(dv[0][0], dv[1][0]), dim = make_float2(dv[0][1], dv[1][1]);
            const float2 er = mul2(cs, m), ei = mul2(sn, m);
            Gr[j] = fma2(er, dre, fma2(neg2(ei), dim, Gr[j]));
            Gi[j] = fma2(er, dim, fma2(ei, dre, Gi[j]));
            amp = mul2(amp, P.mstep);
        }
    }
}

// TAB: delta/h at Y = 0 from the plan's table of cubic pieces (read-only cache; relative
// error <= 2.3e-6), evaluated directly outside the table.
template <int QB, bool HAS_Y, int SINC, bool TAB>
__global__ void __launch_bounds__(kMtThreads, 1)
k_plain_mt(const GreenConst gc, const SubElem *__restrict__ sub_g, const float *__restrict__ xg,
           const float *__restrict__ yg, const float *__restrict__ zg,
           const float *__restrict__ rcg, int64_t S, int64_t chunk_len, int SB, int T,
           const float2 *__restrict__ cw, float2 *__restrict__ part,
           const float4 *__restrict__ dtab) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = gc.N, nu = gc.nu, M = gc.M, nq = gc.nq, Nr = N + 1;
    const int tid = threadIdx.x;
    float4 *sc = reinterpret_cast<float4 *>(smem_raw);              // [kMtSBMax] (x, y, z, R)
    float4 *subA = sc + kMtSBMax;                                   // [nu][N] xh, xl, zh, zl
    float4 *subB = subA + M;                                        // [nu][N] cpsi, spsi, l0, z0
    float2 *cwt = reinterpret_cast<float2 *>(subB + M + 3 * nu);    // [QB][T][Nr]
    float2 *rft = cwt + QB * T * Nr;                                // [QB][T][N]
    float2 *Gt = rft + QB * T * N;                                  // [QB][SB][Nr]
    float2 *RP = Gt + QB * SB * Nr;                                 // [QB][SB][T]

    const int qt = blockIdx.x, chunk = blockIdx.y;
    const int k0 = qt * QB;
    const int64_t s_begin = (int64_t)chunk * chunk_len;
    const int64_t s_end = min(S, s_begin + chunk_len);

    if (!HAS_Y) {       // element-pair records for mt_gen_pair (in place of the planes)
        const int np = ((N + 1) >> 1) * nu;
        for (int i = tid; i < np; i += kMtThreads) {
            const int pp = i / nu, mu = i - pp * nu;
            pair_records(sub_g[min(2 * pp, N - 1) * nu + mu], sub_g[min(2 * pp + 1, N - 1) * nu + mu],
                         subA + 3 * i);
        }
    } else {
        for (int i = tid; i < M; i += kMtThreads) {     // global [e][mu] -> shared [mu][e]
            const float4 *rec = reinterpret_cast<const float4 *>(sub_g + i);
            const int e = i / nu, mu = i - e * nu;
            subA[mu * N + e] = rec[0];
            subB[mu * N + e] = rec[1];
        }
    }
    for (int i = tid; i < QB * T * N; i += kMtThreads) {
        const int j = i / (T * N), r = i - j * T * N, t = r / N, e = r - t * N, k = k0 + j;
        cwt[(j * T + t) * Nr + e] = k < nq ? cw[((size_t)t * nq + k) * N + e] : make_float2(0.f, 0.f);
        rft[i] = make_float2(0.f, 0.f);
    }
    const float q0 = (float)(gc.q_lo + k0);
    // contraction work: (bin, scatterer pair, transmit pair) items, each split over ks
    // threads along the elements when there are fewer items than threads
    const int SP = (SB + 1) >> 1, TP = (T + 1) >> 1;
    const int items = QB * SP * TP;
    int ks = 1;
    while (ks < 8 && items * ks * 2 <= kMtThreads) ks *= 2;
    const int units = items * ks;
    const int NC = (N + 127) >> 7;       // chunks of 128 elements

    for (int64_t sb = s_begin; sb < s_end; sb += SB) {
        __syncthreads();
        if (tid < SB) {
            const int64_t s = sb + tid;
            sc[tid] = s < s_end ? make_float4(xg[s], HAS_Y ? yg[s] : 0.f, zg[s], rcg[s])
                                : make_float4(0.f, 0.f, 1.f, 0.f);
        }
        __syncthreads();

        // 1. Green's tile of the QB bins (at Y = 0 two elements per item)
        if (!HAS_Y) {
            const int NP = (N + 1) >> 1;
            for (int pr = tid; pr < SB * NP; pr += kMtThreads) {
                const int s = pr / NP, pp = pr - s * NP;
                const float4 ps = sc[s];
                float2 Gr[QB], Gi[QB];
                mt_gen_pair<QB, SINC, TAB>(gc, subA, dtab, ps.x, ps.z, pp, q0, Gr, Gi);
                const int e0 = 2 * pp;
#pragma unroll
                for (int j = 0; j < QB; ++j) {
                    float2 *o = Gt + (j * SB + s) * Nr + e0;
                    o[0] = make_float2(Gr[j].x, Gi[j].x);
                    if (e0 + 1 < N) o[1] = make_float2(Gr[j].y, Gi[j].y);
                }
            }
        }
        for (int pr = tid; pr < (HAS_Y ? SB * N : 0); pr += kMtThreads) {
            const int s = pr / N, e = pr - s * N;
            const float4 ps = sc[s];
            float2 G[QB];
#pragma unroll
            for (int j = 0; j < QB; ++j) G[j] = make_float2(0.f, 0.f);
            for (int mu = 0; mu < nu; ++mu) {
                SubElem se;
                reinterpret_cast<float4 *>(&se)[0] = subA[mu * N + e];
                reinterpret_cast<float4 *>(&se)[1] = subB[mu * N + e];
                const PairSetup P = pair_setup<HAS_Y>(gc, se, ps.x, ps.y, ps.z, q0);
                float amp = P.amp0;
                const float kt = TAB ? P.kap * gc.tab_inv_dx : 0.0f;
                const float t0 = TAB ? gc.tab_x0 * gc.tab_inv_dx : 0.0f;
#pragma unroll
                for (int j = 0; j < QB; ++j) {
                    const float q = q0 + (float)j;
                    const float fr = df_frac_mul(q, P.u);
                    float sn, cs;
                    sincos_a(6.283185307179586f * fr, sn, cs);
                    const float m = amp * sinc_f<SINC>(q * P.xb);
                    float2 d;
                    if (TAB) {
                        const float tt = fmaf(q, kt, -t0);
                        const float fl = floorf(fminf(fmaxf(tt, 0.0f), (float)gc.tab_n - 0.5f));
                        const int i = (int)fl;
                        const float u = tt - fl;
                        d = cubic_piece(__ldg(dtab + 2 * i), __ldg(dtab + 2 * i + 1), u);
                        if (!(u >= 0.0f && u <= 1.0f)) d = delta_f<false>(gc, P, q);   // r < ~2 mm
                    } else {
                        d = delta_f<HAS_Y>(gc, P, q);
                    }
                    const float er = cs * m, ei = sn * m;
                    G[j].x += er * d.x - ei * d.y;
                    G[j].y += er * d.y + ei * d.x;
                    amp *= P.mstep;
                }
            }
#pragma unroll
            for (int j = 0; j < QB; ++j) Gt[(j * SB + s) * Nr + e] = G[j];
        }
        __syncthreads();

        // 2. P_t = sum_e C_t G_e for two scatterers x two transmits per item, then R_s P
        for (int base = 0; base < units; base += kMtThreads) {
            const int w = base + tid;
            const bool act = w < units;
            const int it = act ? w / ks : 0, part_ = w - (w / ks) * ks;
            const int j = it / (SP * TP), r = it - j * SP * TP, sp = r / TP, tp = r - sp * TP;
            const int s0 = 2 * sp, t0 = 2 * tp;
            const float2 *g[2], *c[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                g[u] = Gt + (j * SB + min(s0 + u, SB - 1)) * Nr;        // past the group /
                c[u] = cwt + (j * T + min(t0 + u, T - 1)) * Nr;         // T: duplicates, dropped
            }
            float acc[2][2][2];   // [scatterer][transmit][re, im]
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b) acc[a][b][0] = acc[a][b][1] = 0.f;
#pragma unroll 4
            for (int e = part_; e < N; e += ks) {
                const float2 ga = g[0][e], gb = g[1][e], ca = c[0][e], cb = c[1][e];
                acc[0][0][0] = fmaf(ca.x, ga.x, fmaf(-ca.y, ga.y, acc[0][0][0]));
                acc[0][0][1] = fmaf(ca.x, ga.y, fmaf(ca.y, ga.x, acc[0][0][1]));
                acc[0][1][0] = fmaf(cb.x, ga.x, fmaf(-cb.y, ga.y, acc[0][1][0]));
                acc[0][1][1] = fmaf(cb.x, ga.y, fmaf(cb.y, ga.x, acc[0][1][1]));
                acc[1][0][0] = fmaf(ca.x, gb.x, fmaf(-ca.y, gb.y, acc[1][0][0]));
                acc[1][0][1] = fmaf(ca.x, gb.y, fmaf(ca.y, gb.x, acc[1][0][1]));
                acc[1][1][0] = fmaf(cb.x, gb.x, fmaf(-cb.y, gb.y, acc[1][1][0]));
                acc[1][1][1] = fmaf(cb.x, gb.y, fmaf(cb.y, gb.x, acc[1][1][1]));
            }
            for (int o = 1; o < ks; o <<= 1) {              // ks adjacent lanes share an item
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int b = 0; b < 2; ++b) {
                        acc[a][b][0] += __shfl_xor_sync(0xffffffffu, acc[a][b][0], o);
                        acc[a][b][1] += __shfl_xor_sync(0xffffffffu, acc[a][b][1], o);
                    }
            }
            if (act && part_ == 0) {
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int b = 0; b < 2; ++b)
                        if (s0 + a < SB && t0 + b < T) {
                            const float R = sc[s0 + a].w;
                            RP[(j * SB + s0 + a) * T + t0 + b] = make_float2(R * acc[a][b][0], R * acc[a][b][1]);
                        }
            }
        }
        __syncthreads();

        // 3. RF_q(t, e) += sum_s G_e R_s P_t, four elements per thread 32 apart (a warp
        // reads 32 consecutive elements of a row)
        for (int i = tid; i < QB * T * NC * 32; i += kMtThreads) {
            const int l = i & 31, jt = i >> 5;
            const int jc = jt / NC, c = jt - jc * NC;
            const int j = jc / T, t = jc - j * T;
            const int e0 = c * 128 + l;
            float2 a[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = make_float2(0.f, 0.f);
            for (int s = 0; s < SB; ++s) {
                const float2 rp = RP[(j * SB + s) * T + t];
                const float2 *gg = Gt + (j * SB + s) * Nr + e0;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (e0 + 32 * u < N) {
                        const float2 v = gg[32 * u];
                        a[u].x = fmaf(v.x, rp.x, fmaf(-v.y, rp.y, a[u].x));
                        a[u].y = fmaf(v.x, rp.y, fmaf(v.y, rp.x, a[u].y));
                    }
                }
            }
            float2 *rr = rft + (j * T + t) * N + e0;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (e0 + 32 * u < N) { rr[32 * u].x += a[u].x; rr[32 * u].y += a[u].y; }
        }
    }
    __syncthreads();
    for (int i = tid; i < QB * T * N; i += kMtThreads) {   // bins fastest: runs of QB in part
        const int j = i % QB, r = i / QB, e = r % N, t = r / N, k = k0 + j;
        if (k < nq) part[(((size_t)chunk * T + t) * N + e) * nq + k] = rft[(j * T + t) * N + e];
    }
}

static size_t plain_mt_smem(const simus_plan *p, int T, int QB, int SB) {
    const size_t Nr = (size_t)p->N + 1;
    return sizeof(float4) * kMtSBMax + sizeof(SubElem) * p->M + 3 * sizeof(float4) * p->nu
         + sizeof(float2) * (size_t)QB * T * (Nr + p->N) + sizeof(float2) * (size_t)QB * SB * Nr
         + sizeof(float2) * (size_t)QB * SB * T;
}

PlainGeom plain_mt_geometry(const simus_plan *p, int T, int64_t S) {
    PlainGeom g{};
    g.SB = 0;
    if (T < 2) return g;
    // the largest tile (bins first, then scatterers per group) whose operands fit
    for (int qb = kMtQBMax; qb >= 2 && !g.SB; qb /= 2)
        for (int sb = kMtSBMax; sb >= 8 && !g.SB; sb /= 2)
            if (plain_mt_smem(p, T, qb, sb) <= 227 * 1024) { g.QB = qb; g.SB = sb; }
    if (!g.SB) return g;
    g.n_qtiles = (p->nq + g.QB - 1) / g.QB;
    // about eight blocks per SM in total (a short last wave), chunks of at least eight groups
    const int64_t want = (int64_t)p->num_sms * 8;
    int64_t chunks = std::max<int64_t>(1, (want + g.n_qtiles - 1) / g.n_qtiles);
    chunks = std::min<int64_t>(chunks, std::max<int64_t>(1, S / ((int64_t)g.SB * 8)));
    int64_t len = (S + chunks - 1) / chunks;
    len = ((len + g.SB - 1) / g.SB) * g.SB;
    g.chunk_len = std::max<int64_t>(len, g.SB);
    g.n_chunks = (int)((S + g.chunk_len - 1) / g.chunk_len);
    g.smem = plain_mt_smem(p, T, g.QB, g.SB);
    return g;
}

int launch_plain_mt(const simus_plan *p, const PlainGeom &g, const simus_scat *sc, int T,
                    const float2 *cw, float2 *part, cudaStream_t st) {
    const bool has_y = sc->y != nullptr;
    const int mode = p->gc.narrow;
    const bool tab = !has_y && p->d_dtab && p->gc.tab_n > 0 && p->delta_table;
    auto pick = [&](auto qb, auto hy) {
        constexpr int QB = decltype(qb)::value;
        constexpr bool HY = decltype(hy)::value;
        if (!HY && tab)
            return mode == 1 ? k_plain_mt<QB, HY, 1, !HY> : (mode == 2 ? k_plain_mt<QB, HY, 2, !HY> : k_plain_mt<QB, HY, 0, !HY>);
        return mode == 1 ? k_plain_mt<QB, HY, 1, false> : (mode == 2 ? k_plain_mt<QB, HY, 2, false> : k_plain_mt<QB, HY, 0, false>);
    };
    using Q2 = std::integral_constant<int, 2>;
    using Q4 = std::integral_constant<int, 4>;
    auto kern = g.QB == 4 ? (has_y ? pick(Q4{}, std::true_type{}) : pick(Q4{}, std::false_type{}))
                          : (has_y ? pick(Q2{}, std::true_type{}) : pick(Q2{}, std::false_type{}));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
    if (e != cudaSuccess) return check_cuda(e, "k_plain_mt smem attribute");
    dim3 grid(g.n_qtiles, g.n_chunks);
    kern<<<grid, kMtThreads, g.smem, st>>>(p->gc, p->d_sub, sc->x, sc->y, sc->z, sc->rc, sc->n,
                                          g.chunk_len, g.SB, T, cw, part, p->d_dtab);
    count_launches(1);
    return check_cuda(cudaGetLastError(), "k_plain_mt launch");
}

}  // namespace simus
