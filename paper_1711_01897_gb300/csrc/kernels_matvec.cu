// H-matrix product y = P (Near x~ + sum_b U_b (V_b^T x~_sigma)), x~ = P^T x:
// gather into cluster order, t_b = V_b^T x~ for every admissible block, then
// one warp per leaf cluster sums its rows of all dense and low-rank blocks in
// a fixed order (no atomics, deterministic), and a scatter back.
#include "bem_device.cuh"

namespace bem {

namespace {

constexpr int kMvThreads = 256;

template <typename T>
__global__ void k_gather(int64_t n, const int32_t *__restrict__ perm, const T *__restrict__ x,
                         T *__restrict__ xt)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) xt[p] = x[perm[p]];
}

template <typename T>
__global__ void k_scatter(int64_t n, const int32_t *__restrict__ perm, const T *__restrict__ yt,
                          T *__restrict__ y)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) y[perm[p]] = yt[p];
}

__device__ __forceinline__ double madd(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ double2 madd(double2 a, double2 b, double2 c)
{
    return make_double2(c.x + fma(a.x, b.x, -a.y * b.y), c.y + fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double zero_of(double) { return 0.0; }
__device__ __forceinline__ double2 zero_of(double2) { return make_double2(0.0, 0.0); }
__device__ __forceinline__ double shdown(double v, int o)
{
    return __shfl_down_sync(0xffffffffu, v, o);
}
__device__ __forceinline__ double2 shdown(double2 v, int o)
{
    return make_double2(__shfl_down_sync(0xffffffffu, v.x, o), __shfl_down_sync(0xffffffffu, v.y, o));
}
__device__ __forceinline__ double add(double a, double b) { return a + b; }
__device__ __forceinline__ double2 add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

__device__ __forceinline__ double shxor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double2 shxor(double2 v, int o)
{
    return make_double2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}

// k_far_vtx: lanes per block, and columns of V summed per pass (two chunks)
constexpr int kVtxGroup = 8;
constexpr int kVtxCols = 2 * KCHUNK;

// t_b[l] = sum_j (v_l)_j x~_{sigma_b + j}.  A group of kVtxGroup lanes per
// admissible block with n <= kMatvecLongCol (longer columns go to
// k_far_vtx_long), the groups striding over the block list.  A chunk stores
// its KCHUNK columns of V contiguously, so the group's lanes read 64
// consecutive bytes of each column per step; each pass sums kVtxCols columns
// (eight loads in flight per lane, x~_j read once for all of them), and the
// eight partial sums are reduced inside the group by a transposing butterfly:
// the exchanges over lane bits 2, 1, 0 halve the values a lane holds (4, 2,
// 1 of them), after which lane g of the group holds the sum of column g.
template <typename T>
__global__ void __launch_bounds__(kMvThreads)
k_far_vtx(const FarBlock *__restrict__ far, const FarChunks *__restrict__ chunks, int64_t nfar,
          const int64_t *__restrict__ toff, const T *__restrict__ pool,
          const T *__restrict__ xt, T *__restrict__ tbuf)
{
    const int g = threadIdx.x & (kVtxGroup - 1);
    const int64_t grp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kVtxGroup;
    const int64_t ngrp = ((int64_t)gridDim.x * blockDim.x) / kVtxGroup;
    const bool h4 = g & 4, h2 = g & 2, h1 = g & 1;
    // every lane of a warp runs the same number of iterations, so that the
    // shuffles below always see the full warp
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) / kVtxGroup;
    const int64_t iters = nfar > gw ? (nfar - gw + ngrp - 1) / ngrp : 0;
    for (int64_t k = 0; k < iters; ++k) {
        const int64_t b = grp + k * ngrp;
        int rank = 0;
        int64_t m = 0, n = 0, sb = 0;
        if (b < nfar) {
            const FarBlock &B = far[b];
            rank = B.rank;
            m = B.te - B.tb;
            n = B.se - B.sb;
            sb = B.sb;
            if (n > kMatvecLongCol) rank = 0;
        }
        const int64_t *ch = b < nfar ? chunks[b].c : nullptr;
        T *t = b < nfar ? tbuf + toff[b] : nullptr;
        const T *x = xt + sb;
        // the group's largest rank is its own; passes run while any group of
        // the warp has columns left
        int wr = rank;
#pragma unroll
        for (int o = 8; o < 32; o <<= 1) wr = max(wr, __shfl_xor_sync(0xffffffffu, wr, o));
        for (int l0 = 0; l0 < wr; l0 += kVtxCols) {
            T s[kVtxCols];
#pragma unroll
            for (int q = 0; q < kVtxCols; ++q) s[q] = zero_of(T{});
            if (l0 < rank) {
                const T *v0 = pool + ch[l0 / KCHUNK] + KCHUNK * m;
                const T *v1 = l0 + KCHUNK < rank ? pool + ch[l0 / KCHUNK + 1] + KCHUNK * m : v0;
#pragma unroll 1
                for (int64_t j = g; j < n; j += kVtxGroup) {
                    const T xj = x[j];
#pragma unroll
                    for (int q = 0; q < KCHUNK; ++q) {
                        if (l0 + q < rank) s[q] = madd(v0[q * n + j], xj, s[q]);
                        if (l0 + KCHUNK + q < rank)
                            s[KCHUNK + q] = madd(v1[q * n + j], xj, s[KCHUNK + q]);
                    }
                }
            }
            T r4[4], r2[2];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const T keep = h4 ? s[4 + i] : s[i], send = h4 ? s[i] : s[4 + i];
                r4[i] = add(keep, shxor(send, 4));
            }
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const T keep = h2 ? r4[2 + i] : r4[i], send = h2 ? r4[i] : r4[2 + i];
                r2[i] = add(keep, shxor(send, 2));
            }
            const T w = add(h1 ? r2[1] : r2[0], shxor(h1 ? r2[0] : r2[1], 1));
            if (l0 + g < rank) t[l0 + g] = w;
        }
    }
}

// The same for complex factors, where the product is bound by the FP64 pipe
// (four multiply-adds per 16 bytes): one lane per (block, column) pair; the
// lane finds its block by binary search in the rank offsets and sums the
// column sequentially, so every FP64 instruction of the warp is useful and no
// reductions are needed.  Columns longer than kMatvecLongCol go to
// k_far_vtx_long.  A block of rank 0 owns no item (it is skipped by the search).
template <typename T>
__global__ void k_far_vtx_cols(const FarBlock *__restrict__ far,
                               const FarChunks *__restrict__ chunks, int64_t nfar,
                               const int64_t *__restrict__ toff, const T *__restrict__ pool,
                               const T *__restrict__ xt, T *__restrict__ tbuf)
{
    const int64_t total = toff[nfar];
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < total;
         it += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = nfar - 1;  // last block with toff[b] <= it
        while (lo < hi) {
            int64_t mid = (lo + hi + 1) >> 1;
            if (toff[mid] <= it) lo = mid;
            else hi = mid - 1;
        }
        const FarBlock &B = far[lo];
        const int64_t m = B.te - B.tb, n = B.se - B.sb;
        if (n > kMatvecLongCol) continue;
        const int l = (int)(it - toff[lo]);
        const T *v = pool + chunks[lo].c[l / KCHUNK] + (int64_t)KCHUNK * m + (int64_t)(l % KCHUNK) * n;
        const T *x = xt + B.sb;
        T s = zero_of(T{});
        for (int64_t j = 0; j < n; ++j) s = madd(v[j], x[j], s);
        tbuf[it] = s;
    }
}

// Long columns: one warp per (block, column) of the blocks with
// n > kMatvecLongCol; loff is the prefix sum of their ranks (loff[nids] total).
template <typename T>
__global__ void k_far_vtx_long(const FarBlock *__restrict__ far,
                               const FarChunks *__restrict__ chunks, const int64_t *__restrict__ ids,
                               int64_t nids, const int64_t *__restrict__ loff,
                               const int64_t *__restrict__ toff, const T *__restrict__ pool,
                               const T *__restrict__ xt, T *__restrict__ tbuf)
{
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t total = loff[nids];
    for (int64_t it = warp; it < total; it += nw) {
        int64_t lo = 0, hi = nids - 1;
        while (lo < hi) {
            int64_t mid = (lo + hi + 1) >> 1;
            if (loff[mid] <= it) lo = mid;
            else hi = mid - 1;
        }
        const int64_t b = ids[lo];
        const int l = (int)(it - loff[lo]);
        const FarBlock &B = far[b];
        const int64_t m = B.te - B.tb, n = B.se - B.sb;
        const T *v = pool + chunks[b].c[l / KCHUNK] + (int64_t)KCHUNK * m + (int64_t)(l % KCHUNK) * n;
        T s = zero_of(T{});
        for (int64_t j = lane; j < n; j += 32) s = madd(v[j], xt[B.sb + j], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s = add(s, shdown(s, o));
        if (lane == 0) tbuf[toff[b] + l] = s;
    }
}

// Prefix sum of the ranks of the long-column blocks: one CTA, chunks of
// 1024 with a carried total.
constexpr int kLongScan = 1024;

__global__ void __launch_bounds__(kLongScan)
k_long_offsets(const FarBlock *__restrict__ far, const int64_t *__restrict__ ids, int64_t nids,
               int64_t *__restrict__ loff)
{
    __shared__ int64_t wt[32];
    __shared__ int64_t carry;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t q0 = 0; q0 < nids; q0 += kLongScan) {
        const int64_t q = q0 + threadIdx.x;
        const int64_t v = q < nids ? (int64_t)far[ids[q]].rank : 0;
        int64_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wt[w] = x;
        __syncthreads();
        if (w == 0) {
            int64_t t = wt[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int64_t y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            wt[lane] = t;
        }
        __syncthreads();
        const int64_t c = carry;
        const int64_t ex = c + (w > 0 ? wt[w - 1] : 0) + x - v;
        if (q < nids) loff[q] = ex;
        __syncthreads();
        if (threadIdx.x == 0) carry = c + wt[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) loff[nids] = carry;
}

// Rows of one leaf cluster: items >= 0 are admissible blocks, items < 0 are
// dense blocks (-1 - id); every listed block's row range contains the leaf.
// The product costs one FP64 multiply-add per 8 bytes (real), more than this
// part's FP64 rate sustains at HBM speed, so the kernel is built to keep the
// FP64 lanes full: a warp per leaf, its lanes kLeafRowLanes rows x
// kLeafSlices column slices.  The leaf's columns (the rank columns of its
// admissible blocks and the columns of its dense blocks, in list order) are
// dealt round-robin to the slices; each lane keeps NS rows (rows q, q + 4,
// ...) in registers, so a leaf of 20 rows uses every lane; a butterfly over
// the slice bits adds the slices in a fixed order (deterministic, no
// atomics).  Leaves above 32 rows are taken in 32-row chunks.
constexpr int kLeafRowLanes = 4, kLeafSlices = 32 / kLeafRowLanes, kLeafChunk = 32;

template <typename T, int NS>
__device__ __forceinline__ void leaf_chunk(int64_t rb, int mrow, int64_t i0, int64_t i1,
                                           const int64_t *__restrict__ items,
                                           const FarBlock *__restrict__ far,
                                           const FarChunks *__restrict__ chunks,
                                           const int64_t *__restrict__ toff,
                                           const T *__restrict__ pool, const T *__restrict__ tbuf,
                                           const NearBlock *__restrict__ near,
                                           const T *__restrict__ near_data,
                                           const T *__restrict__ xt, T *__restrict__ yt, int lane)
{
    const int q = lane % kLeafRowLanes, sl = lane / kLeafRowLanes;
    T acc[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) acc[i] = zero_of(T{});
    bool row_ok[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) row_ok[i] = q + kLeafRowLanes * i < mrow;
    int64_t before = 0;  // columns of the leaf's earlier items
    for (int64_t it = i0; it < i1; ++it) {
        const int64_t id = items[it];
        // this slice's first column of the item
        int c = (int)((sl - before) % kLeafSlices);
        if (c < 0) c += kLeafSlices;
        if (id >= 0) {
            const FarBlock &B = far[id];
            const int64_t m = B.te - B.tb, rr = rb - B.tb + q;
            const T *t = tbuf + toff[id];
            const int64_t *ch = chunks[id].c;
            const int nc = B.rank;
            for (; c < nc; c += kLeafSlices) {
                const T *col = pool + ch[c / KCHUNK] + (int64_t)(c % KCHUNK) * m + rr;
                const T tv = t[c];
#pragma unroll
                for (int i = 0; i < NS; ++i)
                    if (row_ok[i]) acc[i] = madd(col[kLeafRowLanes * i], tv, acc[i]);
            }
            before += nc;
        } else {
            // column-major: the row lanes read consecutive entries of a column
            const NearBlock &N = near[-1 - id];
            const int64_t nc = N.se - N.sb, mr = N.te - N.tb;
            const T *a = near_data + N.off + (rb - N.tb) + q;
            for (int64_t cc = c; cc < nc; cc += kLeafSlices) {
                const T *col = a + cc * mr;
                const T xv = xt[N.sb + cc];
#pragma unroll
                for (int i = 0; i < NS; ++i)
                    if (row_ok[i]) acc[i] = madd(col[kLeafRowLanes * i], xv, acc[i]);
            }
            before += nc;
        }
    }
#pragma unroll
    for (int i = 0; i < NS; ++i)
        for (int d = kLeafRowLanes; d < 32; d <<= 1) acc[i] = add(acc[i], shxor(acc[i], d));
    if (sl == 0) {
#pragma unroll
        for (int i = 0; i < NS; ++i)
            if (row_ok[i]) yt[rb + q + kLeafRowLanes * i] = acc[i];
    }
}

template <typename T>
__global__ void __launch_bounds__(kMvThreads)
k_leaf_rows(const int64_t *__restrict__ leaf_rows, const int64_t *__restrict__ ptr,
            const int64_t *__restrict__ items, int64_t nleaf, const FarBlock *__restrict__ far,
            const FarChunks *__restrict__ chunks, const int64_t *__restrict__ toff,
            const T *__restrict__ pool, const T *__restrict__ tbuf,
            const NearBlock *__restrict__ near, const T *__restrict__ near_data,
            const T *__restrict__ xt, T *__restrict__ yt)
{
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t lf = warp; lf < nleaf; lf += nw) {
        const int64_t r0 = leaf_rows[2 * lf], r1 = leaf_rows[2 * lf + 1];
        const int64_t i0 = ptr[lf], i1 = ptr[lf + 1];
        for (int64_t rb = r0; rb < r1; rb += kLeafChunk) {
            const int mrow = (int)(r1 - rb < kLeafChunk ? r1 - rb : kLeafChunk);
            // rows per lane, the same in every lane of the warp
            switch ((mrow + kLeafRowLanes - 1) / kLeafRowLanes) {
#define BEM_LEAF(NS)                                                                              \
    case NS:                                                                                      \
        leaf_chunk<T, NS>(rb, mrow, i0, i1, items, far, chunks, toff, pool, tbuf, near, near_data, \
                          xt, yt, lane);                                                          \
        break;
                BEM_LEAF(1) BEM_LEAF(2) BEM_LEAF(3) BEM_LEAF(4)
                BEM_LEAF(5) BEM_LEAF(6) BEM_LEAF(7) BEM_LEAF(8)
#undef BEM_LEAF
                default: break;
            }
        }
    }
}

template <typename T>
cudaError_t matvec_t(int64_t n, const int32_t *perm, const T *x, T *y, T *xt, T *yt, T *tbuf,
                     const FarBlock *far, const FarChunks *chunks, int64_t nfar,
                     const int64_t *toff, const T *pool,
                     const NearBlock *near, const T *near_data, const int64_t *leaf_rows,
                     const int64_t *leaf_ptr, const int64_t *leaf_items, int64_t nleaf,
                     const int64_t *long_ids, int64_t nlong, int64_t *long_off,
                     cudaStream_t st)
{
    unsigned g1 = (unsigned)((n + kMvThreads - 1) / kMvThreads);
    k_gather<T><<<g1, kMvThreads, 0, st>>>(n, perm, x, xt);
    count_launches(1);
    if (nfar > 0) {
        int dev = 0, nsm = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if constexpr (sizeof(T) == sizeof(double))
            k_far_vtx<T><<<(unsigned)(nsm * 8), kMvThreads, 0, st>>>(far, chunks, nfar, toff, pool, xt, tbuf);
        else
            k_far_vtx_cols<T><<<(unsigned)(nsm * 8), kMvThreads, 0, st>>>(far, chunks, nfar, toff, pool,
                                                                          xt, tbuf);
        count_launches(1);
        if (nlong > 0) {
            k_far_vtx_long<T><<<(unsigned)(nsm * 8), kMvThreads, 0, st>>>(
                far, chunks, long_ids, nlong, long_off, toff, pool, xt, tbuf);
            count_launches(1);
        }
    }
    int64_t g2 = (nleaf * 32 + kMvThreads - 1) / kMvThreads;
    if (g2 > 65535) g2 = 65535;
    if (g2 > 0) {
        k_leaf_rows<T><<<(unsigned)g2, kMvThreads, 0, st>>>(leaf_rows, leaf_ptr, leaf_items, nleaf,
                                                            far, chunks, toff, pool, tbuf, near,
                                                            near_data,
                                                            xt, yt);
        count_launches(1);
    }
    k_scatter<T><<<g1, kMvThreads, 0, st>>>(n, perm, yt, y);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_long_offsets(const FarBlock *far, const int64_t *ids, int64_t nids,
                                int64_t *loff, cudaStream_t st)
{
    if (nids <= 0) return cudaSuccess;
    k_long_offsets<<<1, kLongScan, 0, st>>>(far, ids, nids, loff);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_matvec(bool cplx, int64_t n, const int32_t *perm, const void *x, void *y,
                          void *xt, void *yt, void *tbuf, const FarBlock *far,
                          const FarChunks *chunks, int64_t nfar,
                          const int64_t *toff, const void *pool_data, const NearBlock *near,
                          const void *near_data, const int64_t *leaf_rows,
                          const int64_t *leaf_ptr, const int64_t *leaf_items, int64_t nleaf,
                          const int64_t *long_ids, int64_t nlong, int64_t *long_off,
                          cudaStream_t st)
{
    if (cplx)
        return matvec_t<double2>(n, perm, (const double2 *)x, (double2 *)y, (double2 *)xt,
                                 (double2 *)yt, (double2 *)tbuf, far, chunks, nfar, toff,
                                 (const double2 *)pool_data, near, (const double2 *)near_data,
                                 leaf_rows, leaf_ptr, leaf_items, nleaf, long_ids, nlong,
                                 long_off, st);
    return matvec_t<double>(n, perm, (const double *)x, (double *)y, (double *)xt, (double *)yt,
                            (double *)tbuf, far, chunks, nfar, toff, (const double *)pool_data, near,
                            (const double *)near_data, leaf_rows, leaf_ptr, leaf_items, nleaf,
                            long_ids, nlong, long_off, st);
}

}  // namespace bem
