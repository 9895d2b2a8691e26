// Persistent ACA kernel templates, shared by the P0 (one dof per triangle)
// and DP1 (three local dofs per triangle) translation units.  See
// kernels_aca.cu for the algorithm and its readings.
#pragma once

#include <algorithm>
#include <type_traits>

#include "bem_dp1.cuh"

namespace bem {
namespace {

constexpr int kAcaThreads = 256;
constexpr int kWarps = kAcaThreads / 32;
constexpr int kSmallCap = 8192;  // largest max(m, n) a single warp may take

// 1/a by Newton-Raphson (r <- r + r (1 - a r)) from a single-precision
// seed: the seed comes from the top 32 bits of a and the hardware's
// approximate FP32 reciprocal, and two FP64 steps take its ~2^-20 relative
// error to rounding level.  Four FP64 operations instead of a full division;
// values outside the FP32 exponent range fall back to the division.
__device__ __forceinline__ double recip(double a)
{
    const int hi = __double2hiint(a);
    const int e = (hi >> 20) & 0x7ff;
    if (e < 1023 - 120 || e > 1023 + 120) return 1.0 / a;
    const unsigned fb = ((unsigned)hi & 0x80000000u) | ((unsigned)(e - 896) << 23) |
                        (((unsigned)hi & 0xfffffu) << 3);
    float r0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(__uint_as_float(fb)));
    double r = f2d_exact(r0);
    r = fma(r, fma(-a, r, 1.0), r);
    r = fma(r, fma(-a, r, 1.0), r);
    return r;
}

// A float from the high word of a double, scaled by 2^-E on the integer
// pipe (the FP64 pipe, conversions included, is the scarce unit on this
// part): the exponent is rebased by B = (896 + E) << 20 and the 20 mantissa
// bits of the high word kept (relative error below 2^-20); magnitudes below
// the float range flush to zero and above it saturate near 2^127.
__device__ __forceinline__ float hiword_to_float(unsigned h, unsigned B)
{
    const unsigned x = h & 0x7fffffffu;
    const unsigned y = (min(max(x, B), B + (254u << 20)) - B) << 3;
    return __uint_as_float(y | (h & 0x80000000u));
}

__device__ __forceinline__ float hi_to_float(double a, unsigned B)
{
    const unsigned h = (unsigned)__double2hiint(a);
    const unsigned x = h & 0x7fffffffu;
    const unsigned y = (min(max(x, B), B + (254u << 20)) - B) << 3;
    return __uint_as_float(y | (h & 0x80000000u));
}

template <bool CPLX>
struct VT;

template <>
struct VT<false> {
    using T = double;
    static __device__ __forceinline__ T from(C2 v) { return v.re; }
    static __device__ __forceinline__ T zero() { return 0.0; }
    static __device__ __forceinline__ double mag(T a) { return fabs(a); }
    // key ordered like |a|; mag_of_key recovers |a|
    static __device__ __forceinline__ long long key(T a)
    {
        return __double_as_longlong(a) & 0x7fffffffffffffffll;  // |a| without FP64 work
    }
    static __device__ __forceinline__ double mag_of_key(long long k)
    {
        return __longlong_as_double(k);
    }
    // key of 1e-14 * |pivot| for the vanishing test
    static __device__ __forceinline__ long long vanish_key(long long maxkey)
    {
        return __double_as_longlong(1e-14 * __longlong_as_double(maxkey));
    }
    static __device__ __forceinline__ double abs2(T a) { return a * a; }
    static __device__ __forceinline__ T fnma(T a, T b, T c) { return fma(-a, b, c); }  // c - a b
    static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
    static __device__ __forceinline__ T inv(T a) { return recip(a); }
    static __device__ __forceinline__ T dotc(T a, T b, T acc) { return fma(a, b, acc); }  // conj(a) b
    static __device__ __forceinline__ double re_mul(T a, T b) { return a * b; }
    static __device__ __forceinline__ T shfl_down(T a, int o, unsigned mask = 0xffffffffu,
                                                  int width = 32)
    {
        return __shfl_down_sync(mask, a, o, width);
    }
    static __device__ __forceinline__ T add(T a, T b) { return a + b; }
    // floor(log2 |a|) from a key
    static __device__ __forceinline__ int key_exp2(long long k) { return (int)((k >> 52) & 0x7ff) - 1023; }
    // conj(a) b accumulated in FP32, both factors scaled by 2^-E (B of hi_to_float)
    using F = float;
    static __device__ __forceinline__ F zerof() { return 0.f; }
    static __device__ __forceinline__ F dotf(T a, T b, unsigned B, F acc)
    {
        return fmaf(hi_to_float(a, B), hi_to_float(b, B), acc);
    }
    static __device__ __forceinline__ T fromf(F a) { return (double)a; }
    static __device__ __forceinline__ F tof(T a, unsigned B) { return hi_to_float(a, B); }
    // from memory: only the high word is loaded
    static __device__ __forceinline__ F tofp(const T *p, unsigned B)
    {
        return hiword_to_float(reinterpret_cast<const unsigned *>(p)[1], B);
    }
    static __device__ __forceinline__ F fdot(F a, F b, F acc) { return fmaf(a, b, acc); }  // conj(a) b
    static __device__ __forceinline__ F addf(F a, F b) { return a + b; }
    static __device__ __forceinline__ float re_mulf(F a, F b) { return a * b; }
    static __device__ __forceinline__ F shfl_xorf(F a, int d, unsigned mask)
    {
        return __shfl_xor_sync(mask, a, d);
    }
};

template <>
struct VT<true> {
    using T = double2;
    static __device__ __forceinline__ T from(C2 v) { return make_double2(v.re, v.im); }
    static __device__ __forceinline__ T zero() { return make_double2(0.0, 0.0); }
    static __device__ __forceinline__ double mag(T a) { return hypot(a.x, a.y); }
    static __device__ __forceinline__ long long key(T a)
    {
        return __double_as_longlong(fma(a.x, a.x, a.y * a.y));
    }
    static __device__ __forceinline__ double mag_of_key(long long k)
    {
        return sqrt(__longlong_as_double(k));
    }
    static __device__ __forceinline__ long long vanish_key(long long maxkey)
    {
        return __double_as_longlong(1e-28 * __longlong_as_double(maxkey));  // squares
    }
    static __device__ __forceinline__ double abs2(T a) { return fma(a.x, a.x, a.y * a.y); }
    static __device__ __forceinline__ T fnma(T a, T b, T c)
    {
        return make_double2(c.x - fma(a.x, b.x, -a.y * b.y), c.y - fma(a.x, b.y, a.y * b.x));
    }
    static __device__ __forceinline__ T mul(T a, T b)
    {
        return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
    }
    static __device__ __forceinline__ T inv(T a)
    {
        double d = recip(fma(a.x, a.x, a.y * a.y));
        return make_double2(a.x * d, -a.y * d);
    }
    static __device__ __forceinline__ T dotc(T a, T b, T acc)
    {
        return make_double2(acc.x + fma(a.x, b.x, a.y * b.y), acc.y + fma(a.x, b.y, -a.y * b.x));
    }
    static __device__ __forceinline__ double re_mul(T a, T b) { return fma(a.x, b.x, -a.y * b.y); }
    static __device__ __forceinline__ T shfl_down(T a, int o, unsigned mask = 0xffffffffu,
                                                  int width = 32)
    {
        return make_double2(__shfl_down_sync(mask, a.x, o, width),
                            __shfl_down_sync(mask, a.y, o, width));
    }
    static __device__ __forceinline__ T add(T a, T b) { return make_double2(a.x + b.x, a.y + b.y); }
    // the key is |a|^2
    static __device__ __forceinline__ int key_exp2(long long k)
    {
        return ((int)((k >> 52) & 0x7ff) - 1023) >> 1;
    }
    using F = float2;
    static __device__ __forceinline__ F zerof() { return make_float2(0.f, 0.f); }
    static __device__ __forceinline__ F dotf(T a, T b, unsigned B, F acc)
    {
        const float ax = hi_to_float(a.x, B), ay = hi_to_float(a.y, B);
        const float bx = hi_to_float(b.x, B), by = hi_to_float(b.y, B);
        return make_float2(fmaf(ax, bx, fmaf(ay, by, acc.x)), fmaf(ax, by, fmaf(-ay, bx, acc.y)));
    }
    static __device__ __forceinline__ T fromf(F a) { return make_double2(a.x, a.y); }
    static __device__ __forceinline__ F tof(T a, unsigned B)
    {
        return make_float2(hi_to_float(a.x, B), hi_to_float(a.y, B));
    }
    static __device__ __forceinline__ F tofp(const T *p, unsigned B)
    {
        const unsigned *w = reinterpret_cast<const unsigned *>(p);
        return make_float2(hiword_to_float(w[1], B), hiword_to_float(w[3], B));
    }
    static __device__ __forceinline__ F fdot(F a, F b, F acc)  // conj(a) b + acc
    {
        return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y)));
    }
    static __device__ __forceinline__ F addf(F a, F b) { return make_float2(a.x + b.x, a.y + b.y); }
    static __device__ __forceinline__ float re_mulf(F a, F b) { return fmaf(a.x, b.x, -a.y * b.y); }
    static __device__ __forceinline__ F shfl_xorf(F a, int d, unsigned mask)
    {
        return make_float2(__shfl_xor_sync(mask, a.x, d), __shfl_xor_sync(mask, a.y, d));
    }
};

// ---- groups: a whole CTA or a single warp ---------------------------------
struct RedScratch {
    double v[kWarps];
    long long k[kWarps];
    int64_t i[kWarps];
    double s0[kWarps], s1[kWarps];
};

__device__ __forceinline__ void warp_argmax(double &v, int64_t &idx)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_down_sync(0xffffffffu, v, o);
        int64_t oi = __shfl_down_sync(0xffffffffu, idx, o);
        if (ov > v || (ov == v && oi < idx)) {
            v = ov;
            idx = oi;
        }
    }
    v = __shfl_sync(0xffffffffu, v, 0);
    idx = __shfl_sync(0xffffffffu, idx, 0);
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return __shfl_sync(0xffffffffu, v, 0);
}

// argmax on integer keys: for non-negative doubles the IEEE bit pattern
// orders like the value, so the comparisons stay off the FP64 pipe
__device__ __forceinline__ void warp_argmax_key(long long &key, int64_t &idx)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        long long ok = __shfl_down_sync(0xffffffffu, key, o);
        int64_t oi = __shfl_down_sync(0xffffffffu, idx, o);
        if (ok > key || (ok == key && oi < idx)) {
            key = ok;
            idx = oi;
        }
    }
    key = __shfl_sync(0xffffffffu, key, 0);
    idx = __shfl_sync(0xffffffffu, idx, 0);
}

// W consecutive lanes of a warp working on one block (W = 32: the whole
// warp; 16 or 8: two or four blocks per warp).  Reductions are shuffle trees
// within the group's lanes; mask names them, so that the groups of a warp may
// part ways when their blocks need different numbers of steps.
template <int W>
struct SubGroup {
    static constexpr bool kShuffle = true;
    static constexpr int kWidth = W;
    int lane;        // 0 .. W - 1
    unsigned mask;   // the group's lanes in the warp
    __device__ int rank() const { return lane; }
    __device__ int size() const { return W; }
    __device__ void sync() const { __syncwarp(mask); }
    __device__ void argmax_key(long long &key, int64_t &idx) const
    {
#pragma unroll
        for (int o = W / 2; o > 0; o >>= 1) {
            long long ok = __shfl_down_sync(mask, key, o, W);
            int64_t oi = __shfl_down_sync(mask, idx, o, W);
            if (ok > key || (ok == key && oi < idx)) {
                key = ok;
                idx = oi;
            }
        }
        key = __shfl_sync(mask, key, 0, W);
        idx = __shfl_sync(mask, idx, 0, W);
    }
    __device__ double sum(double a) const
    {
#pragma unroll
        for (int o = W / 2; o > 0; o >>= 1) a += __shfl_down_sync(mask, a, o, W);
        return __shfl_sync(mask, a, 0, W);
    }
    template <class V>
    __device__ typename V::T shfl_down(typename V::T a, int o) const
    {
        return V::shfl_down(a, o, mask, W);
    }
    __device__ double shfl_idx(double a, int src) const { return __shfl_sync(mask, a, src, W); }
    // butterfly sum: every lane gets the same bits
    __device__ float sumf(float a) const
    {
#pragma unroll
        for (int o = W / 2; o > 0; o >>= 1) a += __shfl_xor_sync(mask, a, o);
        return a;
    }
};

// The FP64 form of the dot-product members of VT (the interface
// group_col_dots reads: F, zerof, tofp, fdot, addf, shfl_xorf, re_mulf), for
// the norm of the mixed path when its dot products stay FP64 (BEM_MIXED):
// values are loaded whole, B is unused.
template <bool CPLX>
struct DotF64;

template <>
struct DotF64<false> {
    using F = double;
    static __device__ __forceinline__ F zerof() { return 0.0; }
    static __device__ __forceinline__ F tofp(const double *p, unsigned) { return *p; }
    static __device__ __forceinline__ F fdot(F a, F b, F acc) { return fma(a, b, acc); }
    static __device__ __forceinline__ F addf(F a, F b) { return a + b; }
    static __device__ __forceinline__ double re_mulf(F a, F b) { return a * b; }
    static __device__ __forceinline__ F shfl_xorf(F a, int d, unsigned mask)
    {
        return __shfl_xor_sync(mask, a, d);
    }
};

template <>
struct DotF64<true> {
    using F = double2;
    static __device__ __forceinline__ F zerof() { return make_double2(0.0, 0.0); }
    static __device__ __forceinline__ F tofp(const double2 *p, unsigned) { return *p; }
    static __device__ __forceinline__ F fdot(F a, F b, F acc)  // conj(a) b + acc
    {
        return make_double2(fma(a.x, b.x, fma(a.y, b.y, acc.x)), fma(a.x, b.y, fma(-a.y, b.x, acc.y)));
    }
    static __device__ __forceinline__ F addf(F a, F b) { return make_double2(a.x + b.x, a.y + b.y); }
    static __device__ __forceinline__ double re_mulf(F a, F b) { return fma(a.x, b.x, -a.y * b.y); }
    static __device__ __forceinline__ F shfl_xorf(F a, int d, unsigned mask)
    {
        return make_double2(__shfl_xor_sync(mask, a.x, d), __shfl_xor_sync(mask, a.y, d));
    }
};

// Dot products <x_l, x_k> for the NC factor columns l0 .. l0 + NC - 1 (those
// below ncol) of a group of W lanes: lanes stride over the rows (coalesced),
// each holding NC accumulators and forming the float of x_k[r] once; a
// butterfly reduce-scatter over the low log2(NC) lane bits leaves lane t
// with column l0 + bitrev(t mod NC), summed over the lanes of its NC-lane
// set, and xor rounds over the higher bits complete the group sum.  cols:
// the first column of the chunk that holds l0 and of the next chunk (stride
// ld between the columns of a chunk), q0 = l0 mod KCHUNK (nonzero only when
// NC < KCHUNK); xk: column k.
template <class V, class D, int NC, int W>
__device__ __forceinline__ typename D::F group_col_dots(const typename V::T *c0, const typename V::T *c1,
                                                        int64_t ld, const typename V::T *xk, int len,
                                                        int nvalid, unsigned B, int t, unsigned mask,
                                                        int q0)
{
    using F = typename D::F;
    F acc[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) acc[q] = D::zerof();
#pragma unroll 2
    for (int r = t; r < len; r += W) {
        const F x = D::tofp(xk + r, B);
#pragma unroll
        for (int q = 0; q < NC; ++q)
            if (q < nvalid) {
                const int qc = q0 + q;  // column within the chunk pair
                const typename V::T *c = (qc < KCHUNK ? c0 : c1) + (int64_t)(qc % KCHUNK) * ld;
                acc[q] = D::fdot(D::tofp(c + r, B), x, acc[q]);
            }
    }
#pragma unroll
    for (int d = 1, n = NC / 2; n >= 1; d <<= 1, n >>= 1) {
        const bool up = (t & d) != 0;
#pragma unroll
        for (int q = 0; q < n; ++q) {
            const F send = up ? acc[q] : acc[q + n];
            const F keep = up ? acc[q + n] : acc[q];
            acc[q] = D::addf(keep, D::shfl_xorf(send, d, mask));
        }
    }
#pragma unroll
    for (int d = NC; d < W; d <<= 1) acc[0] = D::addf(acc[0], D::shfl_xorf(acc[0], d, mask));
    return acc[0];
}

// The FP64 form (BEM_MIXED) with the group's lanes split in two halves: the
// lower W/2 lanes form <u_l, u_k> over the m rows, the upper W/2 lanes
// <v_l, v_k> over the n columns, each half striding over its own vector with
// NC accumulators.  The reduce-scatter and the xor rounds stay within a half,
// so each lane reduces one set of NC sums over W/2 lanes instead of two sets
// over W (fewer FP64 additions, the scarce pipe, and no idle lanes in the
// tails of short columns); one shuffle across the halves then pairs each
// column's two dot products.  Every NC-lane set of the group returns
// re <u_l,u_k><v_l,v_k> of column l = l0 + bitrev(t mod NC) (bitwise the same
// in both halves).  u0 / u1: first column of the chunk holding l0 and of the
// next chunk (U columns at stride m, V columns at KCHUNK * m + stride n).
template <class V, class D, int NC, int W>
__device__ __forceinline__ double group_col_dots_split(const typename V::T *u0, const typename V::T *u1,
                                                      const typename V::T *uk, const typename V::T *vk,
                                                      int64_t m, int64_t n, int nvalid, int t, unsigned mask,
                                                      int q0)
{
    using F = typename D::F;
    constexpr int H = W / 2;
    static_assert(NC <= H, "a half holds every column of the set");
    const bool vside = t >= H;
    const int64_t ld = vside ? n : m;
    const typename V::T *c0 = vside ? u0 + (int64_t)KCHUNK * m : u0;
    const typename V::T *c1 = vside ? u1 + (int64_t)KCHUNK * m : u1;
    const typename V::T *xk = vside ? vk : uk;
    const int len = (int)ld, h = t & (H - 1);
    F acc[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) acc[q] = D::zerof();
#pragma unroll 2
    for (int r = h; r < len; r += H) {
        const F x = D::tofp(xk + r, 0u);
#pragma unroll
        for (int q = 0; q < NC; ++q)
            if (q < nvalid) {
                const int qc = q0 + q;
                const typename V::T *c = (qc < KCHUNK ? c0 : c1) + (int64_t)(qc % KCHUNK) * ld;
                acc[q] = D::fdot(D::tofp(c + r, 0u), x, acc[q]);
            }
    }
#pragma unroll
    for (int d = 1, nh = NC / 2; nh >= 1; d <<= 1, nh >>= 1) {
        const bool up = (t & d) != 0;
#pragma unroll
        for (int q = 0; q < nh; ++q) {
            const F send = up ? acc[q] : acc[q + nh];
            const F keep = up ? acc[q + nh] : acc[q];
            acc[q] = D::addf(keep, D::shfl_xorf(send, d, mask));
        }
    }
#pragma unroll
    for (int d = NC; d < H; d <<= 1) acc[0] = D::addf(acc[0], D::shfl_xorf(acc[0], d, mask));
    return D::re_mulf(acc[0], D::shfl_xorf(acc[0], H, mask));
}

template <int NC>
__device__ __forceinline__ int bitrev_low(int t)
{
    int c = 0;
#pragma unroll
    for (int b = 1, v = NC / 2; v >= 1; b <<= 1, v >>= 1)
        if (t & b) c += v;
    return c;
}
using WarpGroup = SubGroup<32>;

struct CtaGroup {
    static constexpr bool kShuffle = false;
    RedScratch *red;
    __device__ int rank() const { return threadIdx.x; }
    __device__ int size() const { return blockDim.x; }
    __device__ int warp() const { return threadIdx.x >> 5; }
    __device__ int nwarps() const { return blockDim.x >> 5; }
    __device__ void sync() const { __syncthreads(); }
    __device__ void argmax(double &v, int64_t &idx) const
    {
        warp_argmax(v, idx);
        int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        if (l == 0) {
            red->v[w] = v;
            red->i[w] = idx;
        }
        __syncthreads();
        v = red->v[0];
        idx = red->i[0];
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
            double ov = red->v[q];
            int64_t oi = red->i[q];
            if (ov > v || (ov == v && oi < idx)) {
                v = ov;
                idx = oi;
            }
        }
        __syncthreads();
    }
    __device__ void argmax_key(long long &key, int64_t &idx) const
    {
        warp_argmax_key(key, idx);
        int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        if (l == 0) {
            red->k[w] = key;
            red->i[w] = idx;
        }
        __syncthreads();
        key = red->k[0];
        idx = red->i[0];
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
            long long ok = red->k[q];
            int64_t oi = red->i[q];
            if (ok > key || (ok == key && oi < idx)) {
                key = ok;
                idx = oi;
            }
        }
        __syncthreads();
    }
    __device__ void sum2(double &a, double &b) const
    {
        a = warp_sum(a);
        b = warp_sum(b);
        int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        if (l == 0) {
            red->s0[w] = a;
            red->s1[w] = b;
        }
        __syncthreads();
        a = 0.0;
        b = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            a += red->s0[q];
            b += red->s1[q];
        }
        __syncthreads();
    }
    __device__ double sum(double a) const
    {
        double b = 0.0;
        sum2(a, b);
        return a;
    }
};

// Per-group shared state, for blocks of rank at most CAP (the rank cap
// min(m, n, KMAX) of the blocks the group takes).
template <bool CPLX, int CAP = KMAX>
struct GroupSmem {
    static constexpr int kCap = CAP, kChunks = (CAP + KCHUNK - 1) / KCHUNK;
    typename VT<CPLX>::T cu[CAP];   // (u_l)_i of the current row / (v_l)_j of the column
    int64_t chunk[kChunks];
    int64_t scal;                   // broadcast slot
    double uv2;                     // ||u_k||^2 ||v_k||^2 of the current step
    int fail;
};

// Shared bytes per warp: one full-rank group, or two groups for blocks of at
// most kSub16Max rows, or four for at most kSub8Max rows.
template <bool CPLX>
struct GroupArea {
    static constexpr size_t a = sizeof(GroupSmem<CPLX, KMAX>),
                            b = 2 * sizeof(GroupSmem<CPLX, kSub16Max>),
                            c = 4 * sizeof(GroupSmem<CPLX, kSub8Max>);
    static constexpr size_t bytes = ((a > b ? (a > c ? a : c) : (b > c ? b : c)) + 15) / 16 * 16;
};

// DOF = 1: a dof per triangle (P0).  DOF = 3: the three local dofs of each
// triangle (DP1); block ranges are dof ranges, dof 3 t + a of the cluster
// order is local basis function a of triangle t, and one element pair gives a
// requested row's (or column's) three entries of that triangle pair.
// One regular entry of a P0 block: with RULES the block's distance-class rule
// (a separate instantiation, so that trees without lower-order classes run
// the plain 6-point code), else the 6-point rule.
template <bool RULES, class E>
__device__ __forceinline__ C2 eval_entry(const typename E::Tri &a, const typename E::Tri &b,
                                         const QuadRule &R, double k, int rule)
{
    if constexpr (RULES) return E::eval_rule(a, b, R, k, rule);
    else return E::eval(a, b, R, k);
}

template <class Grp, int OP, bool CPLX, int PREC, int DOF = 1, bool RULES = false, class SM>
__device__ void aca_block(const Grp &G, const DevGeom &g, const QuadRule &R, double k, double eps,
                          FarBlock *blk, FarChunks *chk, typename VT<CPLX>::T *pool, Pool *P,
                          SM &S, unsigned *Z, typename VT<CPLX>::T *part)
{
    using V = VT<CPLX>;
    using T = typename V::T;
    using E = RegularEntry<OP, CPLX, (PREC != 0 ? 1 : 0)>;
    const int64_t tb = blk->tb, sb = blk->sb;
    const int64_t m = blk->te - tb, n = blk->se - sb;
    const int rule = blk->rule;  // the block's distance class (P0 Laplace entries)
    const int t = G.rank(), GS = G.size();
    const int64_t kmin = m < n ? m : n;
    const int kcap = (int)(kmin < SM::kCap ? kmin : SM::kCap);
    const int64_t zwords = (m + 31) >> 5;
    for (int64_t w = t; w < zwords; w += GS) Z[w] = 0u;
    for (int c = t; c < SM::kChunks; c += GS) S.chunk[c] = -1;
    if (t == 0) S.fail = 0;
    G.sync();

    int kk = 0, status = 0;
    int nalloc = 0;  // chunks allocated so far (same value in every thread)
    int64_t nZ = 0, i = 0, entries = 0;
    double normS2 = 0.0;
    const double eps2 = eps * eps;
    long long maxkey = 0, vkey = 0;  // largest pivot so far, and 1e-14 of it, as keys
    auto Uat = [&](int l, int64_t r) -> T * {
        return pool + S.chunk[l / KCHUNK] + (int64_t)(l % KCHUNK) * m + r;
    };
    auto Vat = [&](int l, int64_t j) -> T * {
        return pool + S.chunk[l / KCHUNK] + (int64_t)KCHUNK * m + (int64_t)(l % KCHUNK) * n + j;
    };

    for (;;) {
        // factor storage for column kk; the decision uses only values that
        // every thread of the group holds, so the barrier below is uniform
        if (kk < kcap && kk / KCHUNK >= nalloc) {
            if (t == 0) {
                unsigned long long need = (unsigned long long)(m + n) * KCHUNK;
                unsigned long long off = atomicAdd(&P->top, need);
                if (off + need > P->cap) {
                    P->overflow = 1;
                    S.fail = 1;
                } else {
                    S.chunk[kk / KCHUNK] = (int64_t)off;
                }
            }
            G.sync();
            if (S.fail) {
                status = 2;
                break;
            }
            ++nalloc;
        }
        long long ukey = -1;
        int64_t br = m, bj = 0;
        if constexpr (DOF == 1) {
            // The selected row i of R_{k-1} (a_{i,:} - sum_l (u_l)_i v_l),
            // then, after the pivot, the selected column bj (a_{:,bj} -
            // sum_l (v_l)_bj u_l): two passes of one loop body, so that the
            // quadrature is compiled once per work shape (a smaller hot code
            // footprint); each entry loads both triangles, the fixed one by a
            // load that is the same for every lane.
            // The pivot's reciprocal scales u_k as the column pass stores it
            // (u_k v_k^T is the same rank-one term as with v_k scaled, and
            // no separate pass over the row is needed); the keys that pick
            // the next row are taken before the scaling.
            bool vanished = false, capped = false;
            long long bkey = -1;
            T pinv = V::zero();
#pragma unroll 1
            for (int ph = 0; ph < 2; ++ph) {
                const bool col = ph != 0;
                if (!col) {
                    for (int l = t; l < kk; l += GS) S.cu[l] = *Uat(l, i);
                } else {
                    G.sync();
                    pinv = V::inv(*Vat(kk, bj));
                    for (int l = t; l < kk; l += GS) S.cu[l] = *Vat(l, bj);
                }
                G.sync();
                const int64_t len = col ? m : n;
                const int64_t a0 = col ? tb : tb + i, da = col ? 1 : 0;
                const int64_t b0 = col ? sb + bj : sb, db = col ? 0 : 1;
                // factor column l of this pass: U_l (column pass) or V_l (row pass)
                const int64_t xoff = col ? 0 : (int64_t)KCHUNK * m, xld = col ? m : n;
                const bool store = col || kk < kcap;
                long long best = -1;
                int64_t bidx = col ? m : 0;
                // the single layer is symmetric (A_rj = A_jr): both passes
                // evaluate (fixed triangle, varying triangle), the fixed one
                // loaded once into registers; the other operators load both
                // triangles of every entry in their own roles
                constexpr bool kSym = OP == 0;
                typename E::Tri tf;
                if constexpr (kSym) E::load_compact(g, col ? b0 : a0, tf, R);
                for (int64_t e = t; e < len; e += GS) {
                    typename E::Tri ta, tq;
                    if constexpr (kSym) {
                        E::load_compact(g, col ? a0 + e : b0 + e, tq, R);
                    } else {
                        E::load_compact(g, a0 + da * e, ta, R);
                        E::load_compact(g, b0 + db * e, tq, R);
                    }
                    T a = V::from((eval_entry<RULES, E>(kSym ? tf : ta, tq, R, k, rule)));
                    for (int l = 0; l < kk; ++l)
                        a = V::fnma(S.cu[l],
                                    pool[S.chunk[l / KCHUNK] + xoff + (int64_t)(l % KCHUNK) * xld + e], a);
                    if (store)
                        pool[S.chunk[kk / KCHUNK] + xoff + (int64_t)(kk % KCHUNK) * xld + e] =
                            col ? V::mul(a, pinv) : a;
                    // the column pass looks for the next row among the unused ones
                    if (!col || !((Z[e >> 5] >> (e & 31)) & 1u)) {
                        long long ky = V::key(a);
                        if (ky > best) {  // e increases, so ties keep the lowest index
                            best = ky;
                            bidx = e;
                        }
                    }
                }
                entries += len;
                G.argmax_key(best, bidx);
                if (col) {
                    ukey = best;
                    br = bidx;
                    break;
                }
                bkey = best;
                bj = bidx;
                if (t == 0) Z[i >> 5] |= 1u << (i & 31);
                ++nZ;
                if (bkey == 0 || bkey <= vkey) {
                    vanished = true;
                    break;
                }
                if (kk == kcap) {
                    capped = true;
                    break;
                }
                if (bkey > maxkey) {
                    maxkey = bkey;
                    vkey = V::vanish_key(maxkey);
                }
            }
            if (vanished) {
                if (nZ == m) break;
                G.sync();
                if (t == 0) {
                    int64_t r = 0;
                    while (r < m && (Z[r >> 5] >> (r & 31)) & 1u) ++r;
                    S.scal = r;
                }
                G.sync();
                i = S.scal;
                continue;
            }
            if (capped) {
                status = 1;
                break;
            }
            G.sync();
        } else {
            // selected row of R_{k-1}: a_{i,:} - sum_l (u_l)_i v_l
            for (int l = t; l < kk; l += GS) S.cu[l] = *Uat(l, i);
            G.sync();
            long long bkey = -1;
            using L = LocalEntry<OP, CPLX, (PREC != 0 ? 1 : 0)>;
            typename L::Tri ti;
            L::load(g, tb / 3 + i / 3, ti);
            const int alpha = (int)(i % 3);
            for (int64_t jt = t; jt < n / 3; jt += GS) {
                typename L::Tri tj;
                L::load(g, sb / 3 + jt, tj);
                C2 v[3];
                L::template eval<0>(ti, tj, R, k, alpha, v);
#pragma unroll
                for (int be = 0; be < 3; ++be) {
                    const int64_t j = 3 * jt + be;
                    T a = V::from(v[be]);
                    for (int l = 0; l < kk; ++l) a = V::fnma(S.cu[l], *Vat(l, j), a);
                    if (kk < kcap) *Vat(kk, j) = a;
                    long long ky = V::key(a);
                    if (ky > bkey) {  // j increases, so ties keep the lowest index
                        bkey = ky;
                        bj = j;
                    }
                }
            }
        entries += n;
        G.argmax_key(bkey, bj);
        if (t == 0) Z[i >> 5] |= 1u << (i & 31);
        ++nZ;
        if (bkey == 0 || bkey <= vkey) {
            if (nZ == m) break;
            G.sync();
            if (t == 0) {
                int64_t r = 0;
                while (r < m && (Z[r >> 5] >> (r & 31)) & 1u) ++r;
                S.scal = r;
            }
            G.sync();
            i = S.scal;
            continue;
        }
        if (kk == kcap) {
            status = 1;
            break;
        }
        if (bkey > maxkey) {
            maxkey = bkey;
            vkey = V::vanish_key(maxkey);
        }
        G.sync();
        const T piv = *Vat(kk, bj);
        const T pinv = V::inv(piv);
        G.sync();
        for (int64_t j = t; j < n; j += GS) *Vat(kk, j) = V::mul(*Vat(kk, j), pinv);
        // selected column of R_{k-1}: a_{:,j} - sum_l (v_l)_j u_l
        for (int l = t; l < kk; l += GS) S.cu[l] = *Vat(l, bj);
        G.sync();
            using L = LocalEntry<OP, CPLX, (PREC != 0 ? 1 : 0)>;
            typename L::Tri tj;
            L::load(g, sb / 3 + bj / 3, tj);
            const int beta = (int)(bj % 3);
            for (int64_t rt = t; rt < m / 3; rt += GS) {
                typename L::Tri tr;
                L::load(g, tb / 3 + rt, tr);
                C2 v[3];
                // the single-layer kernel is symmetric: column beta of the
                // local matrix of (T_r, T_j) is row beta of (T_j, T_r), so the
                // row evaluator serves both (one quadrature body in the
                // kernel instead of two)
                if constexpr (OP == 0) L::template eval<0>(tj, tr, R, k, beta, v);
                else L::template eval<1>(tr, tj, R, k, beta, v);
#pragma unroll
                for (int al = 0; al < 3; ++al) {
                    const int64_t r = 3 * rt + al;
                    T a = V::from(v[al]);
                    for (int l = 0; l < kk; ++l) a = V::fnma(S.cu[l], *Uat(l, r), a);
                    *Uat(kk, r) = a;
                    if (!((Z[r >> 5] >> (r & 31)) & 1u)) {
                        long long ky = V::key(a);
                        if (ky > ukey) {
                            ukey = ky;
                            br = r;
                        }
                    }
                }
            }
            entries += m;
            G.argmax_key(ukey, br);
            G.sync();
        }
        // ||S_k||_F^2 grows by 2 Re sum_{l<k} <u_k,u_l><v_k,v_l> + ||u_k||^2 ||v_k||^2.
        // Every thread forms the dot products of one column l <= k over one
        // segment of the rows (and of v_l over one segment of the columns);
        // the segments of each l are combined in shared memory, and one group
        // sum gives the increment.  FP64 work: (k+1)(m+n) multiply-adds plus
        // (k+1) * segments additions.
        double incr = 0.0, uv2 = 0.0;
        const int ncol = kk + 1;
        // BEM_MIXED_SP (PREC 2): the dot products in FP32 from floats formed
        // on the integer pipe (hi_to_float), the factor that carries the
        // pivots' magnitude scaled by 2^-E with 2^E the largest pivot so far,
        // so that its squares and products stay in the float range (the
        // other factor is divided by its pivot, the largest entry of its row,
        // and is O(1)); each product is rescaled by 2^2E in FP64.  The norm
        // feeds only the stopping test, whose threshold a relative error of
        // ~1e-6 moves by as much.  FP64 dot products in BEM_MIXED and BEM_FP64.
        unsigned Bu = 896u << 20, Bv = 896u << 20;
        double unscale = 1.0;
        if constexpr (PREC == 2) {
            int E = V::key_exp2(maxkey);
            E = E < -500 ? -500 : (E > 500 ? 500 : E);
            // P0: u_k carries 1/pivot (|u| = O(1)), v_k the pivot's scale;
            // DP1: v_k is divided by the pivot (|v| <= 1), u_k is not
            if constexpr (DOF == 1) Bv = (unsigned)(896 + E) << 20;
            else Bu = (unsigned)(896 + E) << 20;
            unscale = __longlong_as_double((long long)(1023 + 2 * E) << 52);
        }
        // <u_l, u_k> and <v_l, v_k> over segment sgi of nseg
        auto seg_dots = [&](int l, int sgi, int nseg, T &iu, T &iv) {
            const T *ul = Uat(l, 0), *uk = Uat(kk, 0);
            const T *vl = Vat(l, 0), *vk = Vat(kk, 0);
            const int mi = (int)m, ni = (int)n;
            const int r0 = (mi * sgi) / nseg, r1 = (mi * (sgi + 1)) / nseg;
            const int j0 = (ni * sgi) / nseg, j1 = (ni * (sgi + 1)) / nseg;
            if constexpr (PREC == 2) {
                typename V::F fu = V::zerof(), fv = V::zerof();
                for (int r = r0; r < r1; ++r) fu = V::dotf(ul[r], uk[r], Bu, fu);
                for (int j = j0; j < j1; ++j) fv = V::dotf(vl[j], vk[j], Bv, fv);
                iu = V::fromf(fu);
                iv = V::fromf(fv);
            } else {
                for (int r = r0; r < r1; ++r) iu = V::dotc(ul[r], uk[r], iu);
                for (int j = j0; j < j1; ++j) iv = V::dotc(vl[j], vk[j], iv);
            }
        };
        if constexpr (Grp::kShuffle && PREC != 0) {
            // columns in register groups of NC (group_col_dots), the same
            // register footprint in both forms: BEM_MIXED_SP sums FP32
            // products (scaled) and rescales the increment once; BEM_MIXED
            // keeps the dot products and their sums in FP64
            constexpr bool kF32 = PREC == 2;
            using D = std::conditional_t<kF32, V, DotF64<CPLX>>;
            using S_t = std::conditional_t<kF32, float, double>;
            constexpr int NC = kF32 ? (CPLX ? 4 : 8) : (CPLX ? 2 : 4);
            constexpr int W = Grp::kWidth;
            static_assert(KCHUNK == 4 && NC <= 2 * KCHUNK && NC <= W &&
                              (NC % KCHUNK == 0 || KCHUNK % NC == 0), "column groups span two chunks");
            S_t incr_s = 0, uv2_s = 0;
            const T *uk = Uat(kk, 0), *vk = Vat(kk, 0);
            for (int l0 = 0; l0 < ncol; l0 += NC) {
                const int nv = ncol - l0 < NC ? ncol - l0 : NC;
                const int q0 = NC < KCHUNK ? l0 % KCHUNK : 0;
                const T *u0 = pool + S.chunk[l0 / KCHUNK];
                const T *u1 = q0 + nv > KCHUNK ? pool + S.chunk[l0 / KCHUNK + 1] : u0;
                S_t pr;
                if constexpr (kF32) {
                    const typename D::F su =
                        group_col_dots<V, D, NC, W>(u0, u1, m, uk, (int)m, nv, Bu, t, G.mask, q0);
                    const typename D::F sv =
                        group_col_dots<V, D, NC, W>(u0 + (int64_t)KCHUNK * m, u1 + (int64_t)KCHUNK * m, n, vk,
                                                    (int)n, nv, Bv, t, G.mask, q0);
                    pr = D::re_mulf(su, sv);
                } else {
                    pr = group_col_dots_split<V, D, NC, W>(u0, u1, uk, vk, m, n, nv, t, G.mask, q0);
                }
                const int c = l0 + bitrev_low<NC>(t % NC);
                // FP32: lanes below NC hold the group's columns once, and a
                // group sum follows.  FP64 (the scarce pipe): every NC-lane set
                // holds all NC columns, so a butterfly over the low log2(NC)
                // lane bits completes the sum in each lane, and ||u_k||^2
                // ||v_k||^2 is read from a lane that holds column k
                if ((!kF32 || t < NC) && c < ncol) {
                    if (c == kk) {
                        incr_s += pr;
                        uv2_s = pr;
                    } else {
                        incr_s += S_t(2) * pr;
                    }
                }
            }
            if constexpr (kF32) {
                incr = (double)G.sumf(incr_s) * unscale;
                uv2 = (double)G.sumf(uv2_s) * unscale;
            } else {
#pragma unroll
                for (int d = 1; d < NC; d <<= 1) incr_s += __shfl_xor_sync(G.mask, incr_s, d);
                incr = incr_s;
                const int last_l0 = (ncol - 1) / NC * NC;
                uv2 = G.shfl_idx(uv2_s, bitrev_low<NC>(kk - last_l0));
            }
        } else if constexpr (Grp::kShuffle) {
            // power-of-two segments per column, summed by shuffle trees
            // within the group's lanes
            double uv2_lane = 0.0;
            int last_l0 = 0;
            for (int l0 = 0; l0 < ncol; l0 += GS) {
                last_l0 = l0;
                const int kc = (ncol - l0) < GS ? (ncol - l0) : GS;
                int nseg = 1;
                while (nseg * 2 * kc <= GS) nseg *= 2;
                T iu = V::zero(), iv = V::zero();
                if (t < kc * nseg) seg_dots(l0 + t % kc, t / kc, nseg, iu, iv);
                for (int off = nseg / 2; off >= 1; off >>= 1) {
                    iu = V::add(iu, G.template shfl_down<V>(iu, off * kc));
                    iv = V::add(iv, G.template shfl_down<V>(iv, off * kc));
                }
                if (t < kc) {
                    const double pr = V::re_mul(iu, iv) * unscale;
                    if (l0 + t == kk) {
                        incr += pr;
                        uv2_lane = pr;
                    } else {
                        incr += 2.0 * pr;
                    }
                }
            }
            incr = G.sum(incr);
            uv2 = G.shfl_idx(uv2_lane, kk - last_l0);
        } else {
            for (int l0 = 0; l0 < ncol; l0 += GS) {
                const int kc = (ncol - l0) < GS ? (ncol - l0) : GS;
                const int nseg = GS / kc;
                T iu = V::zero(), iv = V::zero();
                if (t < kc * nseg) seg_dots(l0 + t % kc, t / kc, nseg, iu, iv);
                part[t] = iu;
                part[GS + t] = iv;
                G.sync();
                if (t < kc) {
                    T su = part[t], sv = part[GS + t];
                    for (int q = 1; q < nseg; ++q) {
                        su = V::add(su, part[q * kc + t]);
                        sv = V::add(sv, part[GS + q * kc + t]);
                    }
                    const double pr = V::re_mul(su, sv) * unscale;
                    if (l0 + t == kk) {
                        incr += pr;          // ||u_k||^2 ||v_k||^2
                        S.uv2 = pr;
                    } else {
                        incr += 2.0 * pr;
                    }
                }
                G.sync();
            }
            incr = G.sum(incr);
            uv2 = S.uv2;  // written before the last barrier above
        }
        normS2 += incr;
        ++kk;
        // ||u_k|| ||v_k|| <= eps ||S_k||_F, compared in squares
        if (uv2 <= eps2 * normS2) break;
        if (kk == kmin || nZ == m) break;
        i = br;
    }
    G.sync();
    if (t == 0) {
        blk->rank = kk;
        blk->status = status;
        blk->entries = entries;
    }
    for (int c = t; c < NCHUNK; c += GS) chk->c[c] = c < SM::kChunks ? S.chunk[c] : -1;
    G.sync();
}

// One block per lane: the same algorithm, run sequentially by one thread for
// a block with max(m, n) <= kTinyMax.  A warp takes 32 such blocks at once, so
// every FP64 instruction of the (uniform-within-a-block) pivoting and norm
// arithmetic serves 32 blocks, and no reductions are needed.
constexpr int kTinyMax = 64;

template <int OP, bool CPLX, int PREC, bool RULES = false>
__device__ void aca_lane(const DevGeom &g, const QuadRule &R, double k, double eps,
                         FarBlock *blk, FarChunks *chk, typename VT<CPLX>::T *pool, Pool *P)
{
    using V = VT<CPLX>;
    using T = typename V::T;
    using E = RegularEntry<OP, CPLX, (PREC != 0 ? 1 : 0)>;
    const int64_t tb = blk->tb, sb = blk->sb;
    const int m = (int)(blk->te - tb), n = (int)(blk->se - sb);
    const int rule = blk->rule;
    const int kmin = m < n ? m : n;
    const int kcap = kmin < KMAX ? kmin : KMAX;
    int64_t chunk[NCHUNK];
#pragma unroll
    for (int c = 0; c < NCHUNK; ++c) chunk[c] = -1;
    int kk = 0, nalloc = 0, status = 0, nZ = 0, i = 0;
    int64_t entries = 0;
    unsigned long long Z = 0ull;
    double normS2 = 0.0, maxpiv = 0.0;
    const double eps2 = eps * eps;
    auto Uat = [&](int l, int r) -> T * {
        return pool + chunk[l / KCHUNK] + (int64_t)(l % KCHUNK) * m + r;
    };
    auto Vat = [&](int l, int j) -> T * {
        return pool + chunk[l / KCHUNK] + (int64_t)KCHUNK * m + (int64_t)(l % KCHUNK) * n + j;
    };
    for (;;) {
        if (kk < kcap && kk / KCHUNK >= nalloc) {
            unsigned long long need = (unsigned long long)(m + n) * KCHUNK;
            unsigned long long off = atomicAdd(&P->top, need);
            if (off + need > P->cap) {
                P->overflow = 1;
                status = 2;
                break;
            }
            chunk[nalloc++] = (int64_t)off;
        }
        // selected row of R_{k-1}
        typename E::Tri ti;
        E::load_scattered(g, tb + i, ti);
        long long bkey = -1;
        int bj = 0;
        for (int j = 0; j < n; ++j) {
            typename E::Tri tj;
            E::load_scattered(g, sb + j, tj);
            T a = V::from((eval_entry<RULES, E>(ti, tj, R, k, rule)));
            for (int l = 0; l < kk; ++l) a = V::fnma(*Uat(l, i), *Vat(l, j), a);
            if (kk < kcap) *Vat(kk, j) = a;
            long long ky = V::key(a);
            if (ky > bkey) {
                bkey = ky;
                bj = j;
            }
        }
        entries += n;
        Z |= 1ull << i;
        ++nZ;
        const double vmax = V::mag_of_key(bkey);
        if (vmax == 0.0 || vmax <= 1e-14 * maxpiv) {
            if (nZ == m) break;
            i = __ffsll((long long)~Z) - 1;  // smallest unused row
            continue;
        }
        if (kk == kcap) {
            status = 1;
            break;
        }
        if (vmax > maxpiv) maxpiv = vmax;
        const T pinv = V::inv(*Vat(kk, bj));
        for (int j = 0; j < n; ++j) *Vat(kk, j) = V::mul(*Vat(kk, j), pinv);
        // selected column of R_{k-1}
        typename E::Tri tj;
        E::load_scattered(g, sb + bj, tj);
        long long ukey = -1;
        int br = m;
        for (int r = 0; r < m; ++r) {
            typename E::Tri tr;
            E::load_scattered(g, tb + r, tr);
            T a = V::from((eval_entry<RULES, E>(tr, tj, R, k, rule)));
            for (int l = 0; l < kk; ++l) a = V::fnma(*Vat(l, bj), *Uat(l, r), a);
            *Uat(kk, r) = a;
            if (!((Z >> r) & 1ull)) {
                long long ky = V::key(a);
                if (ky > ukey) {
                    ukey = ky;
                    br = r;
                }
            }
        }
        entries += m;
        // ||S_k||_F^2 increment: 2 Re sum_{l<k} <u_k,u_l><v_k,v_l> + ||u_k||^2 ||v_k||^2
        // (BEM_MIXED_SP: FP32 dot products as in aca_block)
        double incr = 0.0, uv2 = 0.0;
        unsigned Bu = 0u;
        double unscale = 1.0;
        if constexpr (PREC == 2) {
            int E = (int)((__double_as_longlong(maxpiv) >> 52) & 0x7ff) - 1023;
            E = E < -500 ? -500 : (E > 500 ? 500 : E);
            Bu = (unsigned)(896 + E) << 20;
            unscale = __longlong_as_double((long long)(1023 + 2 * E) << 52);
        }
        const T *uk = Uat(kk, 0), *vk = Vat(kk, 0);
        for (int l = 0; l <= kk; ++l) {
            const T *ul = Uat(l, 0), *vl = Vat(l, 0);
            T iu = V::zero(), iv = V::zero();
            if constexpr (PREC == 2) {
                typename V::F fu = V::zerof(), fv = V::zerof();
                for (int r = 0; r < m; ++r) fu = V::dotf(ul[r], uk[r], Bu, fu);
                for (int j = 0; j < n; ++j) fv = V::dotf(vl[j], vk[j], 896u << 20, fv);
                iu = V::fromf(fu);
                iv = V::fromf(fv);
            } else {
                for (int r = 0; r < m; ++r) iu = V::dotc(ul[r], uk[r], iu);
                for (int j = 0; j < n; ++j) iv = V::dotc(vl[j], vk[j], iv);
            }
            const double pr = V::re_mul(iu, iv) * unscale;
            if (l == kk) {
                uv2 = pr;
                incr += pr;
            } else {
                incr += 2.0 * pr;
            }
        }
        normS2 += incr;
        ++kk;
        if (uv2 <= eps2 * normS2) break;
        if (kk == kmin || nZ == m) break;
        i = br;
    }
    blk->rank = kk;
    blk->status = status;
    blk->entries = entries;
#pragma unroll
    for (int c = 0; c < NCHUNK; ++c) chk->c[c] = chunk[c];
}

// The job of work item i and the block's index in that job's arrays.
// (nullptr for an item that names no block of the launch's jobs: skipped)
__device__ __forceinline__ const AcaJob *item_job(const AcaWork &w, int64_t i, int64_t &idx)
{
    if (!w.items) {
        idx = i;
        return w.jobs;
    }
    const int64_t it = w.items[i];
    idx = it & ((int64_t(1) << kItemShift) - 1);
    const int64_t j = it >> kItemShift;
    if (j < 0 || j >= w.n_jobs) return nullptr;
    const AcaJob *J = w.jobs + j;
    return idx < J->n_far ? J : nullptr;
}

// Blocks of the half- and quarter-warp shapes, W lanes each, 32 / W per
// warp: the warp takes that many consecutive blocks of the shape's queue.
template <int W, int OP, bool CPLX, int PREC, int DOF, bool RULES>
__device__ __forceinline__ void aca_subgroups(const AcaWork &w, const QuadRule &R, int64_t first,
                                              int64_t count, unsigned *counter,
                                              unsigned char *area, unsigned *zwarp)
{
    using SM = GroupSmem<CPLX, W == 16 ? kSub16Max : kSub8Max>;
    SM *gs = reinterpret_cast<SM *>(area);
    using T = typename VT<CPLX>::T;
    constexpr int NG = 32 / W;
    constexpr int ZW = (W == 16 ? kSub16Max : kSub8Max) / 32 + 1;  // row-mask words per block
    static_assert(NG * ZW <= 8, "row masks of the groups of a warp");
    const int lane = threadIdx.x & 31, gi = lane / W;
    const SubGroup<W> sg{lane % W, (W == 32 ? 0xffffffffu : ((1u << W) - 1u)) << (W * gi)};
    for (;;) {
        int64_t b0 = 0;
        if (lane == 0) b0 = (int64_t)atomicAdd(counter, (unsigned)NG);
        b0 = __shfl_sync(0xffffffffu, b0, 0);
        if (b0 >= count) break;
        const int64_t b = b0 + gi;
        int64_t idx = 0;
        const AcaJob *J = b < count ? item_job(w, first + b, idx) : nullptr;
        if (J) {
            aca_block<SubGroup<W>, OP, CPLX, PREC, DOF, RULES>(
                sg, J->g, R, J->k, J->eps, J->far + idx, J->chunks + idx, (T *)J->pool, J->P, gs[gi],
                zwarp + gi * ZW, nullptr);
        }
        __syncwarp();
    }
}

template <int OP, bool CPLX, int PREC, int DOF, bool RULES = false>
__global__ void __launch_bounds__(kAcaThreads, 2)
k_aca(AcaWork w, QuadRule R, int zwords_small, AcaQueue *Q)
{
    using T = typename VT<CPLX>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ RedScratch red;
    __shared__ __align__(16) unsigned char garea[kWarps][GroupArea<CPLX>::bytes];
    __shared__ T part[2 * kAcaThreads];
    __shared__ int64_t s_b;
    const int64_t n_big = w.n[kShapeCta], n_small = w.n[kShapeWarp];
    // row bitmasks: the whole region for a CTA-wide block, then one slice of
    // zwords_small words per warp for the warp-sized and smaller blocks
    unsigned *zbig = reinterpret_cast<unsigned *>(smem_raw);
    // phase 1: large blocks, one CTA each
    CtaGroup cg{&red};
    for (;;) {
        if (threadIdx.x == 0) s_b = (int64_t)atomicAdd(&Q->next_big, 1u);
        __syncthreads();
        int64_t b = s_b;
        __syncthreads();
        if (b >= n_big) break;
        int64_t idx;
        const AcaJob *J = item_job(w, b, idx);
        if (!J) continue;
        aca_block<CtaGroup, OP, CPLX, PREC, DOF, RULES>(cg, J->g, R, J->k, J->eps, J->far + idx,
                                                        J->chunks + idx, (T *)J->pool, J->P,
                                                        *reinterpret_cast<GroupSmem<CPLX> *>(garea[0]),
                                                        zbig, part);
    }
    // phase 2: blocks of a warp each
    const int wi = threadIdx.x >> 5;
    unsigned *zwarp = zbig + (int64_t)wi * zwords_small;
    WarpGroup wg{(int)(threadIdx.x & 31), 0xffffffffu};
    for (;;) {
        int64_t b = 0;
        if (wg.lane == 0) b = (int64_t)atomicAdd(&Q->next_small, 1u);
        b = __shfl_sync(0xffffffffu, b, 0);
        if (b >= n_small) break;
        int64_t idx;
        const AcaJob *J = item_job(w, n_big + b, idx);
        if (!J) continue;
        aca_block<WarpGroup, OP, CPLX, PREC, DOF, RULES>(wg, J->g, R, J->k, J->eps, J->far + idx,
                                                         J->chunks + idx, (T *)J->pool, J->P,
                                                         *reinterpret_cast<GroupSmem<CPLX> *>(garea[wi]),
                                                         zwarp, part + 64 * wi);
    }
    // phases 3 and 4: two blocks per warp on 16 lanes each, then four on 8
    // lanes each (P0 only; the host puts no DP1 block in these shapes)
    if constexpr (DOF == 1) {
        const int64_t f3 = n_big + n_small, f4 = f3 + w.n[kShapeHalf];
        aca_subgroups<16, OP, CPLX, PREC, DOF, RULES>(w, R, f3, w.n[kShapeHalf], &Q->next_w16,
                                                      garea[wi], zwarp);
        aca_subgroups<8, OP, CPLX, PREC, DOF, RULES>(w, R, f4, w.n[kShapeQuarter], &Q->next_w8,
                                                     garea[wi], zwarp);
    }
    // phase 5: tiny blocks, 32 per warp, one per lane (P0 only)
    if constexpr (DOF == 1) {
        const int64_t f5 = n_big + n_small + w.n[kShapeHalf] + w.n[kShapeQuarter];
        const int64_t n_tiny = w.n[kShapeLane];
        for (;;) {
            int64_t b0 = 0;
            if (wg.lane == 0) b0 = (int64_t)atomicAdd(&Q->next_tiny, 32u);
            b0 = __shfl_sync(0xffffffffu, b0, 0);
            if (b0 >= n_tiny) break;
            const int64_t b = b0 + wg.lane;
            int64_t idx = 0;
            const AcaJob *J = b < n_tiny ? item_job(w, f5 + b, idx) : nullptr;
            if (J) {
                aca_lane<OP, CPLX, PREC, RULES>(J->g, R, J->k, J->eps, J->far + idx,
                                                J->chunks + idx, (T *)J->pool, J->P);
            }
            __syncwarp();
        }
    }
}

template <int OP, bool CPLX, int PREC, int DOF, bool RULES = false>
cudaError_t aca_launch(const AcaWork &w, const QuadRule &R, AcaQueue *Q, int num_sms,
                       cudaStream_t st)
{
    // row masks: a CTA block's, or per warp a slice of at least 8 words (the
    // sub-warp groups of a warp)
    const int64_t zw_big = (w.max_m_big + 31) / 32;
    const int64_t zw_small = std::max<int64_t>((w.max_m_small + 31) / 32, 8);
    int64_t words = zw_big > kWarps * zw_small ? zw_big : kWarps * zw_small;
    size_t dyn = (size_t)(words > 0 ? words : 1) * sizeof(unsigned);
    auto kern = k_aca<OP, CPLX, PREC, DOF, RULES>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dyn);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kAcaThreads, dyn);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)num_sms * per_sm;
    if (w.max_ctas > 0 && grid > w.max_ctas) grid = w.max_ctas;
    kern<<<(unsigned)grid, kAcaThreads, dyn, st>>>(w, R, (int)zw_small, Q);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

}  // namespace bem
