// Device helpers shared by the kernels: geometry access, float-float
// accumulation and the per-entry quadrature of the regular and singular
// rules.  Header-only; every .cu file gets its own copy.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>

#include "bem_internal.h"

namespace bem {

constexpr double kInv4Pi = 0.25 / CUDART_PI;

struct C2 {
    double re, im;
};

__device__ __forceinline__ C2 cadd(C2 a, C2 b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ C2 csub(C2 a, C2 b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ C2 cmul(C2 a, C2 b)
{
    return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
__device__ __forceinline__ C2 cconjmul(C2 a, C2 b)  // conj(a) * b
{
    return {fma(a.re, b.re, a.im * b.im), fma(a.re, b.im, -a.im * b.re)};
}
__device__ __forceinline__ double cabs2(C2 a) { return fma(a.re, a.re, a.im * a.im); }

// ---- single-instruction FP32 approximations (PTX ISA) ---------------------
// The .ftz forms are one MUFU instruction each; the non-ftz library forms add
// subnormal handling that no regular-pair quadrature operand needs (r^2 and
// r + R0 are bounded away from zero).  PTX ISA bounds: rsqrt.approx and
// rcp.approx have maximum relative error 2^-23 (rcp: 1 ulp); sin.approx and
// cos.approx have maximum absolute error 2^-20.5 for |x| <= 100 pi.
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_ftz(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ void sincos_ftz(float x, float *s, float *c)
{
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(*s) : "f"(x));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(*c) : "f"(x));
}

// ---- float-float accumulation (Knuth's TwoSum) ---------------------------
struct FF {
    float hi, lo;
};

__device__ __forceinline__ void ff_add(FF &a, float x)
{
    float s = __fadd_rn(a.hi, x);
    float bp = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    a.hi = s;
    a.lo = __fadd_rn(a.lo, e);
}

// Exact product a*b as float-float (FMA error term).
__device__ __forceinline__ FF ff_mul(FF a, FF b)
{
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return {p, e};
}

// Exact widening of a finite float to double from its IEEE-754 fields, on
// the integer pipe (the FP64 pipe is the scarce unit on this part).
__device__ __forceinline__ double f2d_exact(float f)
{
    unsigned b = __float_as_uint(f);
    unsigned e = (b >> 23) & 0xffu;
    if (e == 0u) return 0.0;  // zero (subnormal partial sums do not occur)
    unsigned hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
    unsigned lo = b << 29;
    return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ double ff_to_double(FF a) { return f2d_exact(a.hi) + f2d_exact(a.lo); }

// ---- packed pairs of FP32 values ---------------------------------------
// PTX .f32x2 arithmetic (sm_100-family parts): one instruction applies the
// operation to both 32-bit halves, each rounded as the scalar form (.rn), so
// two quadrature terms take the issue slot of one.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 x2_pack(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void x2_unpack(f32x2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 x2_sub(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 x2_mul(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 x2_fma(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ float x2_sum(f32x2 v)
{
    float lo, hi;
    x2_unpack(v, lo, hi);
    return lo + hi;
}

// 1/sqrt(q) in FP64 for a positive normal q (the FP64 quadratures: r^2 of a
// regular pair or of a Sauter-Schwab node, never zero).  Newton's iteration
// y <- y + y (1/2 - (q/2) y^2) from an FP32 seed: q is reduced exactly to
// q' = q 2^-2k in [1, 4), the float of q' built from its fields (23 mantissa
// bits, truncated) on the integer pipe, the seed taken by rsqrt.approx.f32
// (relative error at most 2^-22.9, PTX ISA), so the seed's relative error is
// below 2^-22.3, and one step in FP64 leaves 1.5 e^2 + rounding < 2^-43.7
// (about 7e-14); the result is scaled back by 2^-k in its exponent.  Three
// FP64 operations.
__device__ __forceinline__ double rsqrt_fp64(double q)
{
    const long long b = __double_as_longlong(q);
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    const int k = e >> 1;  // floor(e / 2)
    const long long bq = b - ((long long)(2 * k) << 52);
    const unsigned hi = (unsigned)(bq >> 32), lo = (unsigned)bq;
    const unsigned fb = ((unsigned)(127 + e - 2 * k) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    double y = f2d_exact(rsqrt_ftz(__uint_as_float(fb)));
    const double h = __longlong_as_double(bq - (1ll << 52));  // q' / 2
    y = fma(y, fma(-h, y * y, 0.5), y);
    return __longlong_as_double(__double_as_longlong(y) - ((long long)k << 52));
}

// ---- triangle views -------------------------------------------------------
struct TriF {           // mixed-precision view
    float ch[3], cl[3];
    float q[NQ][3];     // quadrature points relative to the centroid
    float n[3];
    FF s;               // area / sqrt(4 pi)
};

struct TriD {           // FP64 view
    double q[NQ][3];
    double n[3];
    double area;
};

// tiled load: field k of triangle p at a fixed offset 128 k bytes from one
// address; coalesced when neighbouring lanes read neighbouring triangles and
// a single line per field when all lanes read the same triangle
__device__ __forceinline__ const float *tile_of(const DevGeom &g, int64_t p)
{
    return g.tq + ((p >> 5) << 10) + (p & 31);
}

__device__ __forceinline__ void load_trif(const DevGeom &g, int64_t p, TriF &t)
{
    const float *f = tile_of(g, p);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        t.ch[c] = __ldg(f + 32 * (kFCh + c));
        t.cl[c] = __ldg(f + 32 * (kFCl + c));
        t.n[c] = __ldg(f + 32 * (kFN + c));
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c) t.q[q][c] = __ldg(f + 32 * (kFQ + 3 * q + c));
    t.s.hi = __ldg(f + 32 * kFS);
    t.s.lo = __ldg(f + 32 * (kFS + 1));
}

// The same view from 20 of the tile's fields: the second orbit's points are
// rho21 times the first orbit's (QuadRule::rho21f), which saves a third of
// the loads of a triangle where loads, not arithmetic, are scarce.
__device__ __forceinline__ void load_trif_compact(const DevGeom &g, int64_t p, TriF &t, float rho)
{
    const float *f = tile_of(g, p);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        t.ch[c] = __ldg(f + 32 * (kFCh + c));
        t.cl[c] = __ldg(f + 32 * (kFCl + c));
        t.n[c] = __ldg(f + 32 * (kFN + c));
    }
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            t.q[q][c] = __ldg(f + 32 * (kFQ + 3 * q + c));
            t.q[3 + q][c] = rho * t.q[q][c];
        }
    t.s.hi = __ldg(f + 32 * kFS);
    t.s.lo = __ldg(f + 32 * (kFS + 1));
}

__device__ __forceinline__ void load_ids_tile(const DevGeom &g, int64_t p, int v[3])
{
    const float *f = tile_of(g, p);
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = __float_as_int(__ldg(f + 32 * (kFId + c)));
}

__device__ __forceinline__ void load_trid(const DevGeom &g, int64_t p, TriD &t)
{
    const int64_t n = g.nt;
#pragma unroll
    for (int c = 0; c < 3; ++c) t.n[c] = __ldg(g.nrm + c * n + p);
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c) t.q[q][c] = __ldg(g.qp + (q * 3 + c) * n + p);
    t.area = __ldg(g.area + p);
}

__device__ __forceinline__ void load_ids_soa(const DevGeom &g, int64_t p, int v[3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = __ldg(g.tri + c * g.nt + p);
}

// number of vertices two triangles share
__device__ __forceinline__ int count_shared(const int a[3], const int b[3])
{
    int s = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) s += (a[i] == b[j]);
    return s;
}

// ---- regular entries, mixed precision (Laplace) --------------------------
// A_ij = |T_i||T_j|/(4 pi) sum_p sum_q w_p w_q K(x_p - y_q), with
// K = 1/r (SLP), d.n_y/r^3 (DLP), -d.n_x/r^3 (ADLP), d = x - y.
// Geometry relative to the centroids: d = (c_i - c_j) + (dx_p - dy_q); the
// points lie in their triangle's plane, so d.n_y depends on p only and
// d.n_x on q only.  Each test point's 6-term FP32 sum (for the single layer,
// each orbit's 18-term sum) is folded into a float-float accumulator.
template <int OP>
__device__ __forceinline__ FF entry_mixed_laplace_ff(const TriF &a, const TriF &b,
                                                     const float *__restrict__ w)
{
    float D[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) D[c] = (a.ch[c] - b.ch[c]) + (a.cl[c] - b.cl[c]);
    float cq[NQ];
    if (OP == 2) {
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            cq[q] = -w[q] * ((D[0] - b.q[q][0]) * a.n[0] + (D[1] - b.q[q][1]) * a.n[1] +
                             (D[2] - b.q[q][2]) * a.n[2]);
    }
    FF acc = {0.f, 0.f};
    // the trial points (and their weights) as packed pairs (q, q + 1): two
    // Green's-function evaluations per packed instruction, one rsqrt each;
    // each sum is kept in two lanes (even and odd q) and joined at its end
    f32x2 bq[NQ / 2][3], wq[NQ / 2];
#pragma unroll
    for (int h = 0; h < NQ / 2; ++h) {
#pragma unroll
        for (int c = 0; c < 3; ++c) bq[h][c] = x2_pack(b.q[2 * h][c], b.q[2 * h + 1][c]);
        wq[h] = OP == 2 ? x2_pack(cq[2 * h], cq[2 * h + 1]) : x2_pack(w[2 * h], w[2 * h + 1]);
    }
    if constexpr (OP == 0) {
        // Single layer: every term is positive, and the three test points of
        // an orbit of the rule share one weight, so each orbit's 18 terms are
        // summed in FP32 (relative error at most 17 u, u = 2^-24), scaled
        // once, and the two orbit sums joined in float-float
        f32x2 so[2] = {0ull, 0ull};
#pragma unroll
        for (int p = 0; p < NQ; ++p) {
            const f32x2 P0 = x2_pack(D[0] + a.q[p][0], D[0] + a.q[p][0]);
            const f32x2 P1 = x2_pack(D[1] + a.q[p][1], D[1] + a.q[p][1]);
            const f32x2 P2 = x2_pack(D[2] + a.q[p][2], D[2] + a.q[p][2]);
            f32x2 s = so[p / 3];
#pragma unroll
            for (int h = 0; h < NQ / 2; ++h) {
                const f32x2 d0 = x2_sub(P0, bq[h][0]), d1 = x2_sub(P1, bq[h][1]), d2 = x2_sub(P2, bq[h][2]);
                float r0, r1;
                x2_unpack(x2_fma(d0, d0, x2_fma(d1, d1, x2_mul(d2, d2))), r0, r1);
                s = x2_fma(wq[h], x2_pack(rsqrt_ftz(r0), rsqrt_ftz(r1)), s);
            }
            so[p / 3] = s;
        }
        acc.hi = w[0] * x2_sum(so[0]);
        ff_add(acc, w[3] * x2_sum(so[1]));
    } else {
#pragma unroll
        for (int p = 0; p < NQ; ++p) {
            float Dp0 = D[0] + a.q[p][0], Dp1 = D[1] + a.q[p][1], Dp2 = D[2] + a.q[p][2];
            const f32x2 P0 = x2_pack(Dp0, Dp0), P1 = x2_pack(Dp1, Dp1), P2 = x2_pack(Dp2, Dp2);
            f32x2 s2 = 0ull;
#pragma unroll
            for (int h = 0; h < NQ / 2; ++h) {
                const f32x2 d0 = x2_sub(P0, bq[h][0]), d1 = x2_sub(P1, bq[h][1]), d2 = x2_sub(P2, bq[h][2]);
                float r0, r1;
                x2_unpack(x2_fma(d0, d0, x2_fma(d1, d1, x2_mul(d2, d2))), r0, r1);
                const f32x2 ri = x2_pack(rsqrt_ftz(r0), rsqrt_ftz(r1));
                s2 = x2_fma(wq[h], x2_mul(x2_mul(ri, ri), ri), s2);
            }
            float s = x2_sum(s2);
            if (OP == 1) s *= Dp0 * b.n[0] + Dp1 * b.n[1] + Dp2 * b.n[2];
            ff_add(acc, w[p] * s);
        }
    }
    // (acc.hi + acc.lo) * |T_i||T_j|/(4 pi) in float-float
    return ff_mul(acc, ff_mul(a.s, b.s));
}

// The same entry widened to FP64 with one FP64 addition (the float halves are
// widened on the integer pipe).
template <int OP>
__device__ __forceinline__ double entry_mixed_laplace(const TriF &a, const TriF &b,
                                                      const float *__restrict__ w)
{
    const FF r = entry_mixed_laplace_ff<OP>(a, b, w);
    return f2d_exact(r.hi) + f2d_exact(r.lo);
}

// ---- lower-order rules of the distance classes (Laplace) -----------------
// Admissible blocks far enough apart for their class use NP = 3, the
// symmetric degree-2 rule at barycentric (2/3, 1/6, 1/6) and permutations
// (weights 1/3), or NP = 1, the centroid rule.  The degree-2 points are the
// stored offsets of the degree-4 rule's second orbit scaled by beta3
// (QuadRule), so the tiles need no new fields.
template <int NP>
__device__ __forceinline__ void low_points(const TriF &a, float beta, float q[NP][3])
{
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
        for (int c = 0; c < 3; ++c) q[p][c] = NP == 1 ? 0.f : beta * a.q[3 + p][c];
}

template <int OP, int NP>
__device__ __forceinline__ double entry_mixed_laplace_low(const TriF &a, const TriF &b, float beta)
{
    float aq[NP][3], bq[NP][3];
    low_points<NP>(a, beta, aq);
    low_points<NP>(b, beta, bq);
    const float w = 1.f / (float)NP;
    float D[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) D[c] = (a.ch[c] - b.ch[c]) + (a.cl[c] - b.cl[c]);
    float cq[NP];
    if (OP == 2) {
#pragma unroll
        for (int q = 0; q < NP; ++q)
            cq[q] = -w * ((D[0] - bq[q][0]) * a.n[0] + (D[1] - bq[q][1]) * a.n[1] +
                          (D[2] - bq[q][2]) * a.n[2]);
    }
    FF acc = {0.f, 0.f};
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        float Dp0 = D[0] + aq[p][0], Dp1 = D[1] + aq[p][1], Dp2 = D[2] + aq[p][2];
        float s = 0.f;
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            float d0 = Dp0 - bq[q][0], d1 = Dp1 - bq[q][1], d2 = Dp2 - bq[q][2];
            float ri = rsqrt_ftz(fmaf(d0, d0, fmaf(d1, d1, d2 * d2)));
            if (OP == 0) s = fmaf(w, ri, s);
            else if (OP == 1) s = fmaf(w, ri * ri * ri, s);
            else s = fmaf(cq[q], ri * ri * ri, s);
        }
        if (OP == 1) s *= Dp0 * b.n[0] + Dp1 * b.n[1] + Dp2 * b.n[2];
        ff_add(acc, w * s);
    }
    const FF r = ff_mul(acc, ff_mul(a.s, b.s));
    return f2d_exact(r.hi) + f2d_exact(r.lo);
}

// largest distance of a quadrature point from the centroid
__device__ __forceinline__ float trif_rad(const TriF &a)
{
    float r2 = 0.f;
#pragma unroll
    for (int p = 0; p < NQ; ++p)
        r2 = fmaxf(r2, fmaf(a.q[p][0], a.q[p][0], fmaf(a.q[p][1], a.q[p][1], a.q[p][2] * a.q[p][2])));
    return sqrtf(r2);
}

// ---- regular entries, FP64 (Laplace and Helmholtz) -----------------------
template <int OP, bool CPLX>
__device__ __forceinline__ C2 entry_fp64(const TriD &a, const TriD &b, const double *__restrict__ w,
                                         double k)
{
    C2 acc = {0.0, 0.0};
#pragma unroll 1
    for (int p = 0; p < NQ; ++p) {
        C2 s = {0.0, 0.0};
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            double d0 = a.q[p][0] - b.q[q][0], d1 = a.q[p][1] - b.q[q][1],
                   d2 = a.q[p][2] - b.q[q][2];
            double r2 = fma(d0, d0, fma(d1, d1, d2 * d2));
            double ri = rsqrt_fp64(r2);
            double amp;  // real factor multiplying exp(ikr)
            if (OP == 0) amp = ri;
            else if (OP == 1) amp = (d0 * b.n[0] + d1 * b.n[1] + d2 * b.n[2]) * ri * ri * ri;
            else amp = -(d0 * a.n[0] + d1 * a.n[1] + d2 * a.n[2]) * ri * ri * ri;
            if (!CPLX) {
                s.re = fma(w[q], amp, s.re);
            } else {
                double r = r2 * ri, sn, cs;
                sincos(k * r, &sn, &cs);
                if (OP == 0) {
                    s.re = fma(w[q] * amp, cs, s.re);
                    s.im = fma(w[q] * amp, sn, s.im);
                } else {
                    // exp(ikr)(ikr - 1)(-d.n_y) = exp(ikr)(1 - ikr) d.n_y (DLP);
                    // likewise for ADLP with d.n_x: amp already holds -/+ d.n
                    double kr = k * r;
                    double fr = cs + kr * sn;   // Re[exp(ikr)(1 - ikr)]
                    double fi = sn - kr * cs;   // Im[exp(ikr)(1 - ikr)]
                    s.re = fma(w[q] * amp, fr, s.re);
                    s.im = fma(w[q] * amp, fi, s.im);
                }
            }
        }
        acc.re = fma(w[p], s.re, acc.re);
        acc.im = fma(w[p], s.im, acc.im);
    }
    double sc = a.area * b.area * kInv4Pi;
    return {acc.re * sc, acc.im * sc};
}

// ---- regular entries, mixed precision (Helmholtz) ------------------------
// exp(ikr) = exp(ik R0) exp(ik (r - R0)) with R0 the centroid distance.  R0
// and its phase are formed in float-float and reduced modulo 2 pi, so the
// large phase k R0 keeps an absolute error far below 1e-6; the small phase
// k (r - R0) = k e.(2D + e)/(r + R0), e = dx_p - dy_q, is evaluated per point.
__device__ __forceinline__ void ff_two_diff(float a, float b, float &s, float &e)
{
    s = __fsub_rn(a, b);
    float bp = __fsub_rn(a, s);
    e = __fadd_rn(__fsub_rn(a, __fadd_rn(s, bp)), __fsub_rn(bp, b));
}

template <int OP>
__device__ __forceinline__ C2 entry_mixed_helmholtz(const TriF &a, const TriF &b,
                                                    const float *__restrict__ w, float kf,
                                                    double k)
{
    // centroid difference in float-float
    float Dh[3], Dl[3], D[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float s, e;
        ff_two_diff(a.ch[c], b.ch[c], s, e);
        Dh[c] = s;
        Dl[c] = e + (a.cl[c] - b.cl[c]);
        D[c] = Dh[c] + Dl[c];
    }
    // R0^2 = |D|^2 in float-float, then R0 = sqrt with one Newton correction
    FF r02 = {0.f, 0.f};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        FF sq = ff_mul({Dh[c], 0.f}, {Dh[c], 0.f});
        ff_add(r02, sq.hi);
        ff_add(r02, sq.lo);
        ff_add(r02, 2.f * Dh[c] * Dl[c]);
    }
    float R0 = sqrtf(r02.hi);
    FF R0sq = ff_mul({R0, 0.f}, {R0, 0.f});
    float R0lo = ((r02.hi - R0sq.hi) - R0sq.lo + r02.lo) / (2.f * R0);
    // phase k R0 in FP64 from the float-float radius (two FP64 ops), reduced
    double ph = k * ((double)R0 + (double)R0lo);
    double nrev = rint(ph * (0.5 / CUDART_PI));
    float th = (float)fma(-nrev, 2.0 * CUDART_PI, ph);
    float s0, c0;
    sincosf(th, &s0, &c0);
    float R0f = R0;
    float cq[NQ];
    if (OP == 2) {
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            cq[q] = (D[0] - b.q[q][0]) * a.n[0] + (D[1] - b.q[q][1]) * a.n[1] +
                    (D[2] - b.q[q][2]) * a.n[2];
    }
    FF are = {0.f, 0.f}, aim = {0.f, 0.f};
#pragma unroll
    for (int p = 0; p < NQ; ++p) {
        float Dp0 = D[0] + a.q[p][0], Dp1 = D[1] + a.q[p][1], Dp2 = D[2] + a.q[p][2];
        float dny = (OP == 1) ? (Dp0 * b.n[0] + Dp1 * b.n[1] + Dp2 * b.n[2]) : 0.f;
        float sre = 0.f, sim = 0.f;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            float e0 = a.q[p][0] - b.q[q][0], e1 = a.q[p][1] - b.q[q][1], e2 = a.q[p][2] - b.q[q][2];
            float d0 = D[0] + e0, d1 = D[1] + e1, d2 = D[2] + e2;
            float r2 = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
            float ri = rsqrt_ftz(r2);
            float r = r2 * ri;
            float dr2 = fmaf(e0, 2.f * D[0] + e0, fmaf(e1, 2.f * D[1] + e1, e2 * (2.f * D[2] + e2)));
            float phi = kf * dr2 * rcp_ftz(r + R0f);
            float sp, cp;
            sincos_ftz(phi, &sp, &cp);
            float fr, fi, amp;
            if (OP == 0) {
                amp = w[q] * ri;
                fr = cp;
                fi = sp;
            } else {
                // exp(i phi)(1 - ikr) times the normal factor
                float kr = kf * r;
                fr = fmaf(kr, sp, cp);
                fi = fmaf(-kr, cp, sp);
                float nf = (OP == 1) ? dny : -cq[q];
                amp = w[q] * nf * ri * ri * ri;
            }
            sre = fmaf(amp, fr, sre);
            sim = fmaf(amp, fi, sim);
        }
        ff_add(are, w[p] * sre);
        ff_add(aim, w[p] * sim);
    }
    double sc = ff_to_double(ff_mul(a.s, b.s));
    double xr = ff_to_double(are) * sc, xi = ff_to_double(aim) * sc;
    double cr = (double)c0, ci = (double)s0;
    return {fma(xr, cr, -xi * ci), fma(xr, ci, xi * cr)};
}

// ---- one regular entry, dispatched on the precision ------------------------
// Views are loaded by the caller so that a row (or column) reuses its fixed
// triangle.
template <int OP, bool CPLX, int PREC>
struct RegularEntry;

template <int OP, bool CPLX>
struct RegularEntry<OP, CPLX, 0> {  // FP64
    using Tri = TriD;
    static __device__ __forceinline__ void load(const DevGeom &g, int64_t p, Tri &t)
    {
        load_trid(g, p, t);
    }
    static __device__ __forceinline__ void load_compact(const DevGeom &g, int64_t p, Tri &t,
                                                        const QuadRule &)
    {
        load_trid(g, p, t);
    }
    static __device__ __forceinline__ void load_scattered(const DevGeom &g, int64_t p, Tri &t)
    {
        load_trid(g, p, t);
    }
    static __device__ __forceinline__ void ids(const DevGeom &g, int64_t p, int v[3])
    {
        load_ids_soa(g, p, v);
    }
    static __device__ __forceinline__ C2 eval(const Tri &a, const Tri &b, const QuadRule &R,
                                              double k)
    {
        return entry_fp64<OP, CPLX>(a, b, R.w, k);
    }
    // the plain FP64 form keeps the 6-point rule for every block
    static __device__ __forceinline__ C2 eval_rule(const Tri &a, const Tri &b, const QuadRule &R,
                                                   double k, int)
    {
        return eval(a, b, R, k);
    }
};

template <int OP, bool CPLX>
struct RegularEntry<OP, CPLX, 1> {  // mixed
    using Tri = TriF;
    static __device__ __forceinline__ void load(const DevGeom &g, int64_t p, Tri &t)
    {
        load_trif(g, p, t);
    }
    static __device__ __forceinline__ void load_compact(const DevGeom &g, int64_t p, Tri &t,
                                                        const QuadRule &R)
    {
        load_trif_compact(g, p, t, R.rho21f);
    }
    static __device__ __forceinline__ void load_scattered(const DevGeom &g, int64_t p, Tri &t)
    {
        load_trif(g, p, t);
    }
    static __device__ __forceinline__ void ids(const DevGeom &g, int64_t p, int v[3])
    {
        load_ids_tile(g, p, v);
    }
    static __device__ __forceinline__ C2 eval(const Tri &a, const Tri &b, const QuadRule &R,
                                              double k)
    {
        if (!CPLX) return {entry_mixed_laplace<OP>(a, b, R.wf), 0.0};
        return entry_mixed_helmholtz<OP>(a, b, R.wf, (float)k, k);
    }
    // the block's distance-class rule (Laplace; Helmholtz keeps the 6-point
    // rule, whose lower-order error is set by k h rather than by distance)
    static __device__ __forceinline__ C2 eval_rule(const Tri &a, const Tri &b, const QuadRule &R,
                                                   double k, int rule)
    {
        if constexpr (!CPLX) {
            if (rule == kRule3) return {entry_mixed_laplace_low<OP, 3>(a, b, R.beta3f), 0.0};
            if (rule == kRule1) return {entry_mixed_laplace_low<OP, 1>(a, b, R.beta3f), 0.0};
        }
        return eval(a, b, R, k);
    }
};

// ---- Sauter-Schwab vertex orders --------------------------------------------
// Vertex orders of the panel parametrisations chi(x^) = P0 + x1 (P1 - P0) +
// x2 (P2 - P1):  identical - stored order for both; edge - test starts at the
// shared edge in its cyclic order, trial takes the same two vertices first;
// vertex - both start at the shared vertex and continue cyclically.
template <int CASE>
__device__ __forceinline__ void singular_order(const int ta[3], const int tb[3], int oa[3],
                                               int ob[3])
{
    if (CASE == 3) {
        for (int i = 0; i < 3; ++i) {
            oa[i] = i;
            ob[i] = 0;
            for (int j = 0; j < 3; ++j)
                if (tb[j] == ta[i]) ob[i] = j;
        }
    } else if (CASE == 2) {
        int p = 0;
        for (int q = 0; q < 3; ++q) {
            bool s0 = false, s1 = false;
            for (int j = 0; j < 3; ++j) {
                s0 |= tb[j] == ta[q];
                s1 |= tb[j] == ta[(q + 1) % 3];
            }
            if (s0 && s1) {
                p = q;
                break;
            }
        }
        oa[0] = p;
        oa[1] = (p + 1) % 3;
        oa[2] = (p + 2) % 3;
        ob[0] = ob[1] = ob[2] = 0;
        for (int j = 0; j < 3; ++j) {
            if (tb[j] == ta[oa[0]]) ob[0] = j;
            else if (tb[j] == ta[oa[1]]) ob[1] = j;
            else ob[2] = j;
        }
    } else {
        int p = 0, q = 0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                if (ta[i] == tb[j]) {
                    p = i;
                    q = j;
                }
        for (int i = 0; i < 3; ++i) {
            oa[i] = (p + i) % 3;
            ob[i] = (q + i) % 3;
        }
    }
}


}  // namespace bem
