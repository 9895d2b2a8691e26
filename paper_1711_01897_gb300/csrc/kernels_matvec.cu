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

// t_b[l] = sum_j (v_l)_j x~_{sigma_b + j}; one warp per admissible block.
template <typename T>
__global__ void k_far_vtx(const FarBlock *__restrict__ far, int64_t nfar,
                          const int64_t *__restrict__ toff, const T *__restrict__ pool,
                          const T *__restrict__ xt, T *__restrict__ tbuf)
{
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = warp; b < nfar; b += nw) {
        const FarBlock &B = far[b];
        const int64_t m = B.te - B.tb, n = B.se - B.sb;
        const int rank = B.rank;
        for (int l = 0; l < rank; ++l) {
            const T *v = pool + B.chunk[l / KCHUNK] + (int64_t)KCHUNK * m + (int64_t)(l % KCHUNK) * n;
            T s = zero_of(T{});
            for (int64_t j = lane; j < n; j += 32) s = madd(v[j], xt[B.sb + j], s);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s = add(s, shdown(s, o));
            if (lane == 0) tbuf[toff[b] + l] = s;
        }
    }
}

// Rows of one leaf cluster: items >= 0 are admissible blocks, items < 0 are
// dense blocks (-1 - id); every listed block's row range contains the leaf.
template <typename T>
__global__ void k_leaf_rows(const int64_t *__restrict__ leaf_rows, const int64_t *__restrict__ ptr,
                            const int64_t *__restrict__ items, int64_t nleaf,
                            const FarBlock *__restrict__ far, const int64_t *__restrict__ toff,
                            const T *__restrict__ pool, const T *__restrict__ tbuf,
                            const NearBlock *__restrict__ near, const T *__restrict__ near_data,
                            const T *__restrict__ xt, T *__restrict__ yt)
{
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t lf = warp; lf < nleaf; lf += nw) {
        const int64_t r0 = leaf_rows[2 * lf], r1 = leaf_rows[2 * lf + 1];
        for (int64_t r = r0 + lane; r < r1; r += 32) {
            T acc = zero_of(T{});
            for (int64_t it = ptr[lf]; it < ptr[lf + 1]; ++it) {
                int64_t id = items[it];
                if (id >= 0) {
                    const FarBlock &B = far[id];
                    const int64_t m = B.te - B.tb, rr = r - B.tb;
                    const T *t = tbuf + toff[id];
                    for (int l = 0; l < B.rank; ++l)
                        acc = madd(pool[B.chunk[l / KCHUNK] + (int64_t)(l % KCHUNK) * m + rr], t[l], acc);
                } else {
                    const NearBlock &N = near[-1 - id];
                    const int64_t nc = N.se - N.sb, rr = r - N.tb;
                    const T *a = near_data + N.off + rr * nc;
                    for (int64_t c = 0; c < nc; ++c) acc = madd(a[c], xt[N.sb + c], acc);
                }
            }
            yt[r] = acc;
        }
    }
}

template <typename T>
cudaError_t matvec_t(int64_t n, const int32_t *perm, const T *x, T *y, T *xt, T *yt, T *tbuf,
                     const FarBlock *far, int64_t nfar, const int64_t *toff, const T *pool,
                     const NearBlock *near, const T *near_data, const int64_t *leaf_rows,
                     const int64_t *leaf_ptr, const int64_t *leaf_items, int64_t nleaf,
                     cudaStream_t st)
{
    unsigned g1 = (unsigned)((n + kMvThreads - 1) / kMvThreads);
    k_gather<T><<<g1, kMvThreads, 0, st>>>(n, perm, x, xt);
    count_launches(1);
    if (nfar > 0) {
        int64_t g = (nfar * 32 + kMvThreads - 1) / kMvThreads;
        if (g > 65535) g = 65535;
        k_far_vtx<T><<<(unsigned)g, kMvThreads, 0, st>>>(far, nfar, toff, pool, xt, tbuf);
        count_launches(1);
    }
    int64_t g2 = (nleaf * 32 + kMvThreads - 1) / kMvThreads;
    if (g2 > 65535) g2 = 65535;
    if (g2 > 0) {
        k_leaf_rows<T><<<(unsigned)g2, kMvThreads, 0, st>>>(leaf_rows, leaf_ptr, leaf_items, nleaf,
                                                            far, toff, pool, tbuf, near, near_data,
                                                            xt, yt);
        count_launches(1);
    }
    k_scatter<T><<<g1, kMvThreads, 0, st>>>(n, perm, yt, y);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_matvec(bool cplx, int64_t n, const int32_t *perm, const void *x, void *y,
                          void *xt, void *yt, void *tbuf, const FarBlock *far, int64_t nfar,
                          const int64_t *toff, const void *pool_data, const NearBlock *near,
                          const void *near_data, const int64_t *leaf_rows,
                          const int64_t *leaf_ptr, const int64_t *leaf_items, int64_t nleaf,
                          cudaStream_t st)
{
    if (cplx)
        return matvec_t<double2>(n, perm, (const double2 *)x, (double2 *)y, (double2 *)xt,
                                 (double2 *)yt, (double2 *)tbuf, far, nfar, toff,
                                 (const double2 *)pool_data, near, (const double2 *)near_data,
                                 leaf_rows, leaf_ptr, leaf_items, nleaf, st);
    return matvec_t<double>(n, perm, (const double *)x, (double *)y, (double *)xt, (double *)yt,
                            (double *)tbuf, far, nfar, toff, (const double *)pool_data, near,
                            (const double *)near_data, leaf_rows, leaf_ptr, leaf_items, nleaf, st);
}

}  // namespace bem
