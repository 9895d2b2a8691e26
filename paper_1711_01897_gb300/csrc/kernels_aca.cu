// Persistent ACA driver: every admissible block of the H-matrix is
// compressed by partially pivoted ACA (Sec. 2.1, Eq. (6)-(7), Algorithm ACA)
// inside one kernel launch.  Blocks come from two device work queues in
// descending size: a CTA works on one large block at a time; once those are
// gone, every warp takes small blocks on its own.  Entries of the requested
// rows and columns are evaluated in place by the regular quadrature
// (admissible blocks contain no pair that shares a vertex); pivot search,
// residual updates and the norm of S_k are FP64.
//
// Readings where the paper is silent (same as the oracle): i_1 = 0;
// i_{k+1} = argmax over unused rows of |(u_k)_i| (lowest index on ties); a row
// vanishes if its maximum is 0 or <= 1e-14 * the largest pivot so far, and
// then the smallest unused row is next; stop once ||u_k|| ||v_k|| <= eps
// ||S_k||_F, or k = min(m, n), or all rows used, or k = KMAX (rank cap).
#include <algorithm>

#include "aca_kernel.cuh"

namespace bem {

namespace {
}  // namespace

namespace {
__global__ void k_debug_recip(const double *__restrict__ x, double *__restrict__ y, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = recip(x[i]);
}
}  // namespace

cudaError_t launch_debug_recip(const double *x, double *y, int64_t n, cudaStream_t st)
{
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    k_debug_recip<<<(unsigned)blocks, 256, 0, st>>>(x, y, n);
    count_launches(1);
    return cudaGetLastError();
}

int aca_small_cap() { return kSmallCap; }
int aca_tiny_max() { return kTinyMax; }

// ---- after the launch: prefix sums of the ranks and device-side totals ----
namespace {
constexpr int kScanThreads = 1024, kScanPer = 1, kScanTile = kScanThreads * kScanPer;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *warp_tot, int64_t &total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    total = warp_tot[(blockDim.x >> 5) - 1];
    int64_t before = w > 0 ? warp_tot[w - 1] : 0;
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads)
k_rank_tiles(const FarBlock *__restrict__ far, const FarChunks *__restrict__ chunks, int64_t n,
             int64_t *tile_sums, AcaStats *st)
{
    __shared__ int64_t wt[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    int64_t sum = 0, ent = 0, fe = 0, k2 = 0, kmn = 0;
    int rmin = 0x7fffffff, rmax = 0, capped = 0, failed = 0;
    for (int q = 0; q < kScanPer; ++q) {
        int64_t b = base + q;
        if (b < n) {
            const FarBlock &F = far[b];
            sum += F.rank;
            ent += F.entries;
            k2 += (int64_t)F.rank * F.rank * ((F.te - F.tb) + (F.se - F.sb));
            kmn += (int64_t)F.rank * ((F.te - F.tb) + (F.se - F.sb));
            rmin = min(rmin, F.rank);
            rmax = max(rmax, F.rank);
            capped += F.status == 1;
            failed += F.status == 2;
            // a block's chunks are allocated in order: the allocated ones
            // are a prefix of its list, the rest -1
            for (int c = 0; c < NCHUNK && chunks[b].c[c] >= 0; ++c)
                fe += ((F.te - F.tb) + (F.se - F.sb)) * KCHUNK;
        }
    }
    int64_t tot = 0;
    block_exclusive_scan(sum, wt, tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
    // the CTA's totals (warp shuffles, then one warp over the warps' sums),
    // so that each CTA adds to the device totals once
    __shared__ int64_t red64[4][32];
    __shared__ int red32[4][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr int nw = kScanThreads / 32;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ent += __shfl_xor_sync(0xffffffffu, ent, o);
        fe += __shfl_xor_sync(0xffffffffu, fe, o);
        k2 += __shfl_xor_sync(0xffffffffu, k2, o);
        kmn += __shfl_xor_sync(0xffffffffu, kmn, o);
        rmin = min(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
        rmax = max(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
        capped += __shfl_xor_sync(0xffffffffu, capped, o);
        failed += __shfl_xor_sync(0xffffffffu, failed, o);
    }
    if (lane == 0) {
        red64[0][w] = ent;
        red64[1][w] = fe;
        red64[2][w] = k2;
        red64[3][w] = kmn;
        red32[0][w] = rmin;
        red32[1][w] = rmax;
        red32[2][w] = capped;
        red32[3][w] = failed;
    }
    __syncthreads();
    if (w == 0) {
        const bool on = lane < nw;
        ent = on ? red64[0][lane] : 0;
        fe = on ? red64[1][lane] : 0;
        k2 = on ? red64[2][lane] : 0;
        kmn = on ? red64[3][lane] : 0;
        rmin = on ? red32[0][lane] : 0x7fffffff;
        rmax = on ? red32[1][lane] : 0;
        capped = on ? red32[2][lane] : 0;
        failed = on ? red32[3][lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ent += __shfl_xor_sync(0xffffffffu, ent, o);
            fe += __shfl_xor_sync(0xffffffffu, fe, o);
            k2 += __shfl_xor_sync(0xffffffffu, k2, o);
            kmn += __shfl_xor_sync(0xffffffffu, kmn, o);
            rmin = min(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
            rmax = max(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
            capped += __shfl_xor_sync(0xffffffffu, capped, o);
            failed += __shfl_xor_sync(0xffffffffu, failed, o);
        }
        if (lane == 0) {
            atomicAdd(&st->entries, (unsigned long long)ent);
            atomicAdd(&st->rank_sum, (unsigned long long)tot);
            atomicAdd(&st->factor_elems, (unsigned long long)fe);
            atomicAdd(&st->k2mn, (unsigned long long)k2);
            atomicAdd(&st->rank_mn, (unsigned long long)kmn);
            atomicMin(&st->rank_min, rmin);
            atomicMax(&st->rank_max, rmax);
            if (capped) atomicAdd(&st->capped, capped);
            if (failed) atomicAdd(&st->failed, failed);
        }
    }
}

// exclusive scan of the tile sums in place, one CTA
__global__ void __launch_bounds__(kScanThreads) k_scan_tile_sums(int64_t *tile_sums, int64_t ntiles)
{
    __shared__ int64_t wt[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < ntiles; b0 += kScanThreads) {
        int64_t b = b0 + threadIdx.x;
        int64_t v = b < ntiles ? tile_sums[b] : 0;
        int64_t tot = 0;
        int64_t ex = block_exclusive_scan(v, wt, tot);
        int64_t c = carry;
        if (b < ntiles) tile_sums[b] = c + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry = c + tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kScanThreads)
k_rank_scan(const FarBlock *__restrict__ far, int64_t n, const int64_t *__restrict__ tile_off,
            int64_t *__restrict__ toff)
{
    __shared__ int64_t wt[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    int r[kScanPer];
    int64_t sum = 0;
    for (int q = 0; q < kScanPer; ++q) {
        r[q] = base + q < n ? far[base + q].rank : 0;
        sum += r[q];
    }
    int64_t tot = 0;
    int64_t ex = block_exclusive_scan(sum, wt, tot) + tile_off[blockIdx.x];
    for (int q = 0; q < kScanPer; ++q) {
        if (base + q < n) toff[base + q] = ex;
        if (base + q == n - 1) toff[n] = ex + r[q];
        ex += r[q];
    }
}
}  // namespace

int64_t aca_finish_tiles(int64_t nfar) { return (nfar + kScanTile - 1) / kScanTile + 1; }

namespace {
__global__ void k_aca_reset(Pool *P, unsigned long long cap, AcaQueue *Q, AcaStats *st)
{
    *P = Pool{0ull, cap, 0, 0};
    *Q = AcaQueue{0u, 0u, 0u, 0u};
    AcaStats z{};
    z.rank_min = 0x7fffffff;
    *st = z;
}
}  // namespace

cudaError_t launch_aca_reset(Pool *P, unsigned long long cap, AcaQueue *Q, AcaStats *st,
                             cudaStream_t s)
{
    k_aca_reset<<<1, 1, 0, s>>>(P, cap, Q, st);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_aca_finish(const FarBlock *far, const FarChunks *chunks, int64_t nfar,
                              int64_t *toff,
                              int64_t *tile_sums, AcaStats *st, cudaStream_t s)
{
    if (nfar <= 0) return cudaMemsetAsync(toff, 0, sizeof(int64_t), s);
    int64_t tiles = (nfar + kScanTile - 1) / kScanTile;
    k_rank_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(far, chunks, nfar, tile_sums, st);
    count_launches(1);
    k_scan_tile_sums<<<1, kScanThreads, 0, s>>>(tile_sums, tiles);
    count_launches(1);
    k_rank_scan<<<(unsigned)tiles, kScanThreads, 0, s>>>(far, nfar, tile_sums, toff);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_aca(const AcaWork &w, const QuadRule &rule, int op, bool cplx, int prec,
                       AcaQueue *queue, int num_sms, cudaStream_t st, int dofs, bool rules)
{
    if (dofs == 3) return launch_aca_dp1(w, rule, op, cplx, prec, queue, num_sms, st);
    if (dofs != 1) return cudaErrorInvalidValue;
    if (prec == 2) return launch_aca_sp(w, rule, op, cplx, queue, num_sms, st, rules);
    // trees with lower-order distance classes: the mixed Laplace kernels that
    // read each block's rule
    if (rules && !cplx && prec == 1) {
        if (op == 0) return aca_launch<0, false, 1, 1, true>(w, rule, queue, num_sms, st);
        if (op == 1) return aca_launch<1, false, 1, 1, true>(w, rule, queue, num_sms, st);
        if (op == 2) return aca_launch<2, false, 1, 1, true>(w, rule, queue, num_sms, st);
    }
#define BEM_ACA(O, C, Pp)                                   \
    if (op == O && cplx == C && prec == Pp)                 \
        return aca_launch<O, C, Pp, 1>(w, rule, queue, num_sms, st);
    BEM_ACA(0, false, 0) BEM_ACA(0, false, 1) BEM_ACA(0, true, 0) BEM_ACA(0, true, 1)
    BEM_ACA(1, false, 0) BEM_ACA(1, false, 1) BEM_ACA(1, true, 0) BEM_ACA(1, true, 1)
    BEM_ACA(2, false, 0) BEM_ACA(2, false, 1) BEM_ACA(2, true, 0) BEM_ACA(2, true, 1)
#undef BEM_ACA
    return cudaErrorInvalidValue;
}

}  // namespace bem
