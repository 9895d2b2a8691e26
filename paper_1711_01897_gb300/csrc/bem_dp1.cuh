// Local 3 x 3 matrices of element pairs for piecewise linear bases (Sec. 3.3,
// Algorithm "Integral Evaluation": the kernel is evaluated once per pair of
// quadrature points and combined with the basis function values of every
// pair of local dofs).  The local basis functions of a triangle are the
// barycentric coordinates of its stored vertices; QuadRule::wl[p][a] holds
// w_p lambda_a(p) for the regular rule, so that
//   L[alpha][beta] = |T_a||T_b| / (4 pi) sum_p sum_q wl[p][alpha] wl[q][beta] K(x_p, y_q).
// MODE 0 returns one row (alpha = fix) as out[beta], MODE 1 one column
// (beta = fix) as out[alpha], MODE 2 all nine as out[3 alpha + beta].
// Header-only, used by the DP1 kernels and the ACA.
#pragma once

#include "bem_device.cuh"

namespace bem {

template <int MODE>
struct Dp1Out {
    static constexpr int N = MODE == 2 ? 9 : 3;
};

// wl[q][fix] with q a compile-time index: selects among three parameter-space
// constants instead of indexing the kernel parameter at run time
__device__ __forceinline__ float wlf_at(const QuadRule &R, int q, int fix)
{
    return fix == 0 ? R.wlf[q][0] : (fix == 1 ? R.wlf[q][1] : R.wlf[q][2]);
}
__device__ __forceinline__ double wl_at(const QuadRule &R, int q, int fix)
{
    return fix == 0 ? R.wl[q][0] : (fix == 1 ? R.wl[q][1] : R.wl[q][2]);
}

// ---- FP64 (Laplace and Helmholtz) -------------------------------------------
template <int OP, bool CPLX, int MODE>
__device__ __forceinline__ void dp1_fp64(const TriD &a, const TriD &b, const QuadRule &R, double k,
                                         int fix, C2 *out)
{
    constexpr int NO = Dp1Out<MODE>::N;
    C2 acc[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) acc[o] = {0.0, 0.0};
#pragma unroll 1
    for (int p = 0; p < NQ; ++p) {
        C2 s[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const double d0 = a.q[p][0] - b.q[q][0], d1 = a.q[p][1] - b.q[q][1],
                         d2 = a.q[p][2] - b.q[q][2];
            const double r2 = fma(d0, d0, fma(d1, d1, d2 * d2));
            const double ri = rsqrt_fp64(r2);
            double amp;
            if (OP == 0) amp = ri;
            else if (OP == 1) amp = (d0 * b.n[0] + d1 * b.n[1] + d2 * b.n[2]) * ri * ri * ri;
            else amp = -(d0 * a.n[0] + d1 * a.n[1] + d2 * a.n[2]) * ri * ri * ri;
            C2 G = {amp, 0.0};
            if (CPLX) {
                const double r = r2 * ri;
                double sn, cs;
                sincos(k * r, &sn, &cs);
                if (OP == 0) {
                    G = {amp * cs, amp * sn};
                } else {
                    const double kr = k * r;
                    G = {amp * (cs + kr * sn), amp * (sn - kr * cs)};  // exp(ikr)(1 - ikr)
                }
            }
            if (MODE == 1) {
                const double wq = wl_at(R, q, fix);
                s[0].re = fma(wq, G.re, s[0].re);
                if (CPLX) s[0].im = fma(wq, G.im, s[0].im);
            } else {
#pragma unroll
                for (int be = 0; be < 3; ++be) {
                    s[be].re = fma(R.wl[q][be], G.re, s[be].re);
                    if (CPLX) s[be].im = fma(R.wl[q][be], G.im, s[be].im);
                }
            }
        }
        if (MODE == 0) {
            const double wp = fix == 0 ? R.wl[p][0] : (fix == 1 ? R.wl[p][1] : R.wl[p][2]);
#pragma unroll
            for (int be = 0; be < 3; ++be) {
                acc[be].re = fma(wp, s[be].re, acc[be].re);
                acc[be].im = fma(wp, s[be].im, acc[be].im);
            }
        } else if (MODE == 1) {
#pragma unroll
            for (int al = 0; al < 3; ++al) {
                acc[al].re = fma(R.wl[p][al], s[0].re, acc[al].re);
                acc[al].im = fma(R.wl[p][al], s[0].im, acc[al].im);
            }
        } else {
#pragma unroll
            for (int al = 0; al < 3; ++al)
#pragma unroll
                for (int be = 0; be < 3; ++be) {
                    acc[3 * al + be].re = fma(R.wl[p][al], s[be].re, acc[3 * al + be].re);
                    acc[3 * al + be].im = fma(R.wl[p][al], s[be].im, acc[3 * al + be].im);
                }
        }
    }
    const double sc = a.area * b.area * kInv4Pi;
#pragma unroll
    for (int o = 0; o < NO; ++o) out[o] = {acc[o].re * sc, acc[o].im * sc};
}

// ---- mixed precision, Laplace --------------------------------------------
// As entry_mixed_laplace: geometry relative to the centroids, 6-term FP32
// partial sums per test point folded into float-float accumulators.
template <int OP, int MODE>
__device__ __forceinline__ void dp1_mixed_laplace(const TriF &a, const TriF &b, const QuadRule &R,
                                                  int fix, C2 *out)
{
    constexpr int NO = Dp1Out<MODE>::N;
    float D[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) D[c] = (a.ch[c] - b.ch[c]) + (a.cl[c] - b.cl[c]);
    float cq[NQ];
    if (OP == 2) {
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            cq[q] = -((D[0] - b.q[q][0]) * a.n[0] + (D[1] - b.q[q][1]) * a.n[1] +
                      (D[2] - b.q[q][2]) * a.n[2]);
    }
    FF acc[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) acc[o] = {0.f, 0.f};
    // trial points and their basis weights as packed pairs (q, q + 1): two
    // evaluations per packed instruction (as entry_mixed_laplace_ff); each
    // partial sum in two lanes, joined after the trial points
    constexpr int NS = MODE == 1 ? 1 : 3;
    f32x2 bq[NQ / 2][3], wq[NQ / 2][NS], cq2[NQ / 2];
#pragma unroll
    for (int h = 0; h < NQ / 2; ++h) {
#pragma unroll
        for (int c = 0; c < 3; ++c) bq[h][c] = x2_pack(b.q[2 * h][c], b.q[2 * h + 1][c]);
        if (MODE == 1) {
            wq[h][0] = x2_pack(wlf_at(R, 2 * h, fix), wlf_at(R, 2 * h + 1, fix));
        } else {
#pragma unroll
            for (int be = 0; be < NS; ++be) wq[h][be] = x2_pack(R.wlf[2 * h][be], R.wlf[2 * h + 1][be]);
        }
        cq2[h] = OP == 2 ? x2_pack(cq[2 * h], cq[2 * h + 1]) : 0ull;
    }
#pragma unroll
    for (int p = 0; p < NQ; ++p) {
        const float Dp0 = D[0] + a.q[p][0], Dp1 = D[1] + a.q[p][1], Dp2 = D[2] + a.q[p][2];
        const f32x2 P0 = x2_pack(Dp0, Dp0), P1 = x2_pack(Dp1, Dp1), P2 = x2_pack(Dp2, Dp2);
        f32x2 s2[NS];
#pragma unroll
        for (int be = 0; be < NS; ++be) s2[be] = 0ull;
#pragma unroll
        for (int h = 0; h < NQ / 2; ++h) {
            const f32x2 d0 = x2_sub(P0, bq[h][0]), d1 = x2_sub(P1, bq[h][1]), d2 = x2_sub(P2, bq[h][2]);
            float r0, r1;
            x2_unpack(x2_fma(d0, d0, x2_fma(d1, d1, x2_mul(d2, d2))), r0, r1);
            f32x2 G = x2_pack(rsqrt_ftz(r0), rsqrt_ftz(r1));
            if (OP != 0) G = x2_mul(x2_mul(G, G), G);
            if (OP == 2) G = x2_mul(cq2[h], G);
#pragma unroll
            for (int be = 0; be < NS; ++be) s2[be] = x2_fma(wq[h][be], G, s2[be]);
        }
        float s[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int be = 0; be < NS; ++be) s[be] = x2_sum(s2[be]);
        if (OP == 1) {
            const float dn = Dp0 * b.n[0] + Dp1 * b.n[1] + Dp2 * b.n[2];
#pragma unroll
            for (int be = 0; be < 3; ++be) s[be] *= dn;
        }
        if (MODE == 0) {
            const float wp = wlf_at(R, p, fix);
#pragma unroll
            for (int be = 0; be < 3; ++be) ff_add(acc[be], wp * s[be]);
        } else if (MODE == 1) {
#pragma unroll
            for (int al = 0; al < 3; ++al) ff_add(acc[al], R.wlf[p][al] * s[0]);
        } else {
#pragma unroll
            for (int al = 0; al < 3; ++al)
#pragma unroll
                for (int be = 0; be < 3; ++be) ff_add(acc[3 * al + be], R.wlf[p][al] * s[be]);
        }
    }
    const FF sab = ff_mul(a.s, b.s);
#pragma unroll
    for (int o = 0; o < NO; ++o) {
        const FF r = ff_mul(acc[o], sab);
        out[o] = {f2d_exact(r.hi) + f2d_exact(r.lo), 0.0};
    }
}

// ---- mixed precision, Helmholtz --------------------------------------------
// As entry_mixed_helmholtz: exp(ikr) = exp(ik R0) exp(ik (r - R0)), the large
// phase from the float-float centroid distance in FP64, the small one per
// point pair in FP32.
template <int OP, int MODE>
__device__ __forceinline__ void dp1_mixed_helmholtz(const TriF &a, const TriF &b, const QuadRule &R,
                                                    float kf, double k, int fix, C2 *out)
{
    constexpr int NO = Dp1Out<MODE>::N;
    float Dh[3], Dl[3], D[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float s, e;
        ff_two_diff(a.ch[c], b.ch[c], s, e);
        Dh[c] = s;
        Dl[c] = e + (a.cl[c] - b.cl[c]);
        D[c] = Dh[c] + Dl[c];
    }
    FF r02 = {0.f, 0.f};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        FF sq = ff_mul({Dh[c], 0.f}, {Dh[c], 0.f});
        ff_add(r02, sq.hi);
        ff_add(r02, sq.lo);
        ff_add(r02, 2.f * Dh[c] * Dl[c]);
    }
    const float R0 = sqrtf(r02.hi);
    const FF R0sq = ff_mul({R0, 0.f}, {R0, 0.f});
    const float R0lo = ((r02.hi - R0sq.hi) - R0sq.lo + r02.lo) / (2.f * R0);
    const double ph = k * ((double)R0 + (double)R0lo);
    const double nrev = rint(ph * (0.5 / CUDART_PI));
    const float th = (float)fma(-nrev, 2.0 * CUDART_PI, ph);
    float s0, c0;
    sincosf(th, &s0, &c0);
    float cq[NQ];
    if (OP == 2) {
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            cq[q] = (D[0] - b.q[q][0]) * a.n[0] + (D[1] - b.q[q][1]) * a.n[1] +
                    (D[2] - b.q[q][2]) * a.n[2];
    }
    FF are[NO], aim[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) are[o] = aim[o] = {0.f, 0.f};
#pragma unroll
    for (int p = 0; p < NQ; ++p) {
        const float Dp0 = D[0] + a.q[p][0], Dp1 = D[1] + a.q[p][1], Dp2 = D[2] + a.q[p][2];
        const float dny = (OP == 1) ? (Dp0 * b.n[0] + Dp1 * b.n[1] + Dp2 * b.n[2]) : 0.f;
        float sre[3] = {0.f, 0.f, 0.f}, sim[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const float e0 = a.q[p][0] - b.q[q][0], e1 = a.q[p][1] - b.q[q][1],
                        e2 = a.q[p][2] - b.q[q][2];
            const float d0 = D[0] + e0, d1 = D[1] + e1, d2 = D[2] + e2;
            const float r2 = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
            const float ri = rsqrt_ftz(r2);
            const float r = r2 * ri;
            const float dr2 =
                fmaf(e0, 2.f * D[0] + e0, fmaf(e1, 2.f * D[1] + e1, e2 * (2.f * D[2] + e2)));
            const float phi = kf * dr2 * rcp_ftz(r + R0);
            float sp, cp;
            sincos_ftz(phi, &sp, &cp);
            float fr, fi, amp;
            if (OP == 0) {
                amp = ri;
                fr = cp;
                fi = sp;
            } else {
                const float kr = kf * r;
                fr = fmaf(kr, sp, cp);
                fi = fmaf(-kr, cp, sp);
                const float nf = (OP == 1) ? dny : -cq[q];
                amp = nf * ri * ri * ri;
            }
            const float gr = amp * fr, gi = amp * fi;
            if (MODE == 1) {
                const float wq = wlf_at(R, q, fix);
                sre[0] = fmaf(wq, gr, sre[0]);
                sim[0] = fmaf(wq, gi, sim[0]);
            } else {
#pragma unroll
                for (int be = 0; be < 3; ++be) {
                    sre[be] = fmaf(R.wlf[q][be], gr, sre[be]);
                    sim[be] = fmaf(R.wlf[q][be], gi, sim[be]);
                }
            }
        }
        if (MODE == 0) {
            const float wp = wlf_at(R, p, fix);
#pragma unroll
            for (int be = 0; be < 3; ++be) {
                ff_add(are[be], wp * sre[be]);
                ff_add(aim[be], wp * sim[be]);
            }
        } else if (MODE == 1) {
#pragma unroll
            for (int al = 0; al < 3; ++al) {
                ff_add(are[al], R.wlf[p][al] * sre[0]);
                ff_add(aim[al], R.wlf[p][al] * sim[0]);
            }
        } else {
#pragma unroll
            for (int al = 0; al < 3; ++al)
#pragma unroll
                for (int be = 0; be < 3; ++be) {
                    ff_add(are[3 * al + be], R.wlf[p][al] * sre[be]);
                    ff_add(aim[3 * al + be], R.wlf[p][al] * sim[be]);
                }
        }
    }
    const double sc = ff_to_double(ff_mul(a.s, b.s));
    const double cr = (double)c0, ci = (double)s0;
#pragma unroll
    for (int o = 0; o < NO; ++o) {
        const double xr = ff_to_double(are[o]) * sc, xi = ff_to_double(aim[o]) * sc;
        out[o] = {fma(xr, cr, -xi * ci), fma(xr, ci, xi * cr)};
    }
}

// ---- dispatch on the precision, like RegularEntry ----------------------------
template <int OP, bool CPLX, int PREC>
struct LocalEntry;

template <int OP, bool CPLX>
struct LocalEntry<OP, CPLX, 0> {
    using Tri = TriD;
    static __device__ __forceinline__ void load(const DevGeom &g, int64_t p, Tri &t)
    {
        load_trid(g, p, t);
    }
    static __device__ __forceinline__ void ids(const DevGeom &g, int64_t p, int v[3])
    {
        load_ids_soa(g, p, v);
    }
    template <int MODE>
    static __device__ __forceinline__ void eval(const Tri &a, const Tri &b, const QuadRule &R,
                                                double k, int fix, C2 *out)
    {
        dp1_fp64<OP, CPLX, MODE>(a, b, R, k, fix, out);
    }
};

template <int OP, bool CPLX>
struct LocalEntry<OP, CPLX, 1> {
    using Tri = TriF;
    static __device__ __forceinline__ void load(const DevGeom &g, int64_t p, Tri &t)
    {
        load_trif(g, p, t);
    }
    static __device__ __forceinline__ void ids(const DevGeom &g, int64_t p, int v[3])
    {
        load_ids_tile(g, p, v);
    }
    template <int MODE>
    static __device__ __forceinline__ void eval(const Tri &a, const Tri &b, const QuadRule &R,
                                                double k, int fix, C2 *out)
    {
        if (!CPLX) dp1_mixed_laplace<OP, MODE>(a, b, R, fix, out);
        else dp1_mixed_helmholtz<OP, MODE>(a, b, R, (float)k, k, fix, out);
    }
};

}  // namespace bem
