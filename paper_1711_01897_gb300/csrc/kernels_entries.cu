// Geometry precompute, dense sub-blocks (bem_entries), the Sauter-Schwab
// singular kernel and the near-field regular kernel.
#include "bem_device.cuh"

namespace bem {

namespace {

constexpr int kGeomThreads = 256;

// Per triangle: vertices, unit normal and area (right-hand rule on the
// stored order), the 6 global quadrature points of the degree-4 rule, and the
// mixed-precision view (centroid as float-float, points relative to it).
// Sec. 3.2.1: geometry computed on the device in 1D coalesced arrays.
__global__ void __launch_bounds__(kGeomThreads)
k_geometry(const double *__restrict__ V, const int32_t *__restrict__ T,
           const int32_t *__restrict__ perm, int64_t nt, QuadRule R, int32_t *tri, double *vtx,
           double *nrm, double *area, double *qp, float *tq)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nt) return;
    int64_t t = perm ? (int64_t)perm[p] : p;
    double v[3][3];
    for (int a = 0; a < 3; ++a) {
        int32_t id = T[3 * t + a];
        tri[a * nt + p] = id;
        for (int c = 0; c < 3; ++c) {
            v[a][c] = V[3 * (int64_t)id + c];
            vtx[(3 * a + c) * nt + p] = v[a][c];
        }
    }
    double e1[3], e2[3];
    for (int c = 0; c < 3; ++c) {
        e1[c] = v[1][c] - v[0][c];
        e2[c] = v[2][c] - v[0][c];
    }
    double nn[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                    e1[0] * e2[1] - e1[1] * e2[0]};
    double len = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
    double A = 0.5 * len;
    area[p] = A;
    float *f = tq + ((p >> 5) << 10) + (p & 31);  // field k at f[32 k]
    double cen[3];
    for (int c = 0; c < 3; ++c) {
        double nc = nn[c] / len;
        nrm[c * nt + p] = nc;
        f[32 * (kFN + c)] = (float)nc;
        cen[c] = ((v[0][c] + v[1][c]) + v[2][c]) / 3.0;
        float h = (float)cen[c];
        f[32 * (kFCh + c)] = h;
        f[32 * (kFCl + c)] = (float)(cen[c] - (double)h);
        f[32 * (kFId + c)] = __int_as_float(T[3 * t + c]);
    }
    for (int q = 0; q < NQ; ++q)
        for (int c = 0; c < 3; ++c) {
            double x = v[0][c] + R.s[q] * e1[c] + R.t[q] * e2[c];
            qp[(q * 3 + c) * nt + p] = x;
            f[32 * (kFQ + 3 * q + c)] = (float)(x - cen[c]);
        }
    double s = A * rsqrt(4.0 * CUDART_PI);
    float sh = (float)s;
    f[32 * kFS] = sh;
    f[32 * (kFS + 1)] = (float)(s - (double)sh);
}

template <bool CPLX>
__device__ __forceinline__ void store_val(void *out, int64_t idx, C2 v)
{
    if (CPLX) reinterpret_cast<double2 *>(out)[idx] = make_double2(v.re, v.im);
    else reinterpret_cast<double *>(out)[idx] = v.re;
}

// Dense sub-block: thread (a, b) evaluates A(test[a], trial[b]) by the
// regular rule (Algorithm "Integral Evaluation", Sec. 3.3: one thread per
// element pair) or queues the pair for the singular kernel.
constexpr int kEntBx = 32, kEntBy = 4;

template <int OP, bool CPLX, int PREC>
__global__ void __launch_bounds__(kEntBx *kEntBy)
k_entries(DevGeom g, QuadRule R, double k, const int32_t *__restrict__ test, int64_t n_test,
          const int32_t *__restrict__ trial, int64_t n_trial, void *out, SingPair *l1,
          SingPair *l2, SingPair *l3, unsigned long long *counts, unsigned long long cap, int *err)
{
    using E = RegularEntry<OP, CPLX, PREC>;
    int64_t b = (int64_t)blockIdx.x * kEntBx + threadIdx.x;
    if (b >= n_trial) return;
    const int32_t j = trial[b];
    if (j < 0 || j >= g.nt) {
        atomicExch(err, 1);
        return;
    }
    typename E::Tri tb;  // this thread's trial triangle, fixed over its rows
    E::load(g, j, tb);
    int vj[3];
    E::ids(g, j, vj);
    for (int64_t a = (int64_t)blockIdx.y * kEntBy + threadIdx.y; a < n_test;
         a += (int64_t)gridDim.y * kEntBy) {
        int32_t i = test[a];
        if (i < 0 || i >= g.nt) {
            atomicExch(err, 1);
            continue;
        }
        int64_t dst = a * n_trial + b;
        int vi[3];
        E::ids(g, i, vi);
        const int s = count_shared(vi, vj);
        if (s > 0) {
            unsigned long long slot = atomicAdd(&counts[s - 1], 1ull);
            if (slot < cap) {
                SingPair *L = s == 1 ? l1 : (s == 2 ? l2 : l3);
                L[slot] = {i, j, dst};
            } else {
                atomicExch(err, 2);
            }
            continue;
        }
        typename E::Tri ta;
        E::load(g, i, ta);
        store_val<CPLX>(out, dst, E::eval(ta, tb, R, k));
    }
}

// Mixed precision: persistent CTAs over tiles of kTileRows test rows x 32
// trial columns.  The tile's test triangles are staged in shared memory (a
// warp copies one triangle, a field per lane), each lane holds its trial
// triangle in registers for the whole tile, and a warp evaluates one row at a
// time, reading the row's triangle with eight broadcast 128-bit loads.
constexpr int kTileThreads = 128, kTileRows = 64;
// CTAs per SM the single-layer instantiation is compiled for (measured: 7
// is 1-2 % faster than the 6 the registers allow unbounded, 8 spills)
constexpr int kSlpMinBlocks = 7;
constexpr int kRowsPerWarp = kTileRows / (kTileThreads / 32);
static_assert(kTileRows % (kTileThreads / 32) == 0 && kRowsPerWarp <= 32, "rows per warp");

// 4-byte asynchronous global -> shared copy (PTX cp.async, sm_80 and later)
__device__ __forceinline__ void cp_async4(float *smem, const float *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

__device__ __forceinline__ void push_singular(int s, int32_t i, int32_t j, int64_t dst,
                                              SingPair *l1, SingPair *l2, SingPair *l3,
                                              unsigned long long *counts, unsigned long long cap,
                                              int *err)
{
    unsigned long long slot = atomicAdd(&counts[s - 1], 1ull);
    if (slot < cap) {
        SingPair *L = s == 1 ? l1 : (s == 2 ? l2 : l3);
        L[slot] = {i, j, dst};
    } else {
        atomicExch(err, 2);
    }
}

template <int OP, bool CPLX>
__device__ __forceinline__ void
entries_tiled_body(const DevGeom &g, const QuadRule &R, double k, const int32_t *__restrict__ test,
                   int64_t n_test, const int32_t *__restrict__ trial, int64_t n_trial, void *out,
                   SingPair *l1, SingPair *l2, SingPair *l3, unsigned long long *counts,
                   unsigned long long cap, int *err)
{
    using E = RegularEntry<OP, CPLX, 1>;
    __shared__ __align__(16) float rows_s[kTileRows][kTileFields];
    __shared__ int32_t rid_s[kTileRows];
    constexpr int nw = kTileThreads / 32;
    constexpr int kBoxWarps = (kTileRows + 31) / 32;
    __shared__ float box_s[kBoxWarps][6];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    static_assert(kBoxWarps <= nw, "row boxes: one warp per 32 rows");
    const int64_t ncb = (n_trial + 31) / 32, nrb = (n_test + kTileRows - 1) / kTileRows;
    const int64_t ntiles = ncb * nrb;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t cb = tile % ncb, rb = tile / ncb;
        const int64_t a0 = rb * kTileRows;
        const int nr = (int)((n_test - a0) < kTileRows ? (n_test - a0) : kTileRows);
        __syncthreads();  // the previous tile's rows are no longer read
        // A warp stages rows w, w + nw, ...: lane t loads the id of its t-th
        // row, then the rows' fields are copied asynchronously, all in flight
        // together (one field per lane and row).
        int32_t my_id = -1;
        if (lane < kRowsPerWarp && w + lane * nw < nr) my_id = __ldg(test + a0 + w + lane * nw);
#pragma unroll 4
        for (int t = 0; t < kRowsPerWarp; ++t) {
            const int r = w + t * nw;
            const int32_t i = __shfl_sync(0xffffffffu, my_id, t);
            if (r < nr) {
                const bool ok = i >= 0 && i < g.nt;
                if (ok) cp_async4(&rows_s[r][lane], tile_of(g, i) + 32 * lane);
                else rows_s[r][lane] = 0.f;
                if (lane == 0) {
                    rid_s[r] = ok ? i : -1;
                    if (!ok) atomicExch(err, 1);
                }
            }
        }
        cp_async_wait_all();
        const int64_t b = cb * 32 + lane;
        int32_t j = -1;
        if (b < n_trial) {
            j = __ldg(trial + b);
            if (j < 0 || j >= g.nt) {
                atomicExch(err, 1);
                j = -1;
            }
        }
        TriF tb;
        int vj[3] = {-1, -1, -1};
        if (j >= 0) {
            load_trif(g, j, tb);
            load_ids_tile(g, j, vj);
        }
        __syncthreads();
        bool far_tile = false;
        // Single layer only (measured: the extra registers cost the double
        // layers more than the skipped vertex tests save)
        if constexpr (OP == 0 && !CPLX) {
        // Bounding boxes of the tile's rows and columns: a vertex lies within
        // rad / 0.7253 of its centroid (the rule's point nearest a vertex sits
        // at 0.7253 of the way from the centroid), taken as 1.4 rad.  If the
        // boxes are apart along some axis no pair of the tile shares a vertex.
        {
            float blo[3], bhi[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                blo[c] = INFINITY;
                bhi[c] = -INFINITY;
            }
            if (w < kBoxWarps) {
                const int r = threadIdx.x;
                if (r < nr && rid_s[r] >= 0) {
                    float q2 = 0.f;
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        const float *e = &rows_s[r][kFQ + 3 * q];
                        q2 = fmaxf(q2, fmaf(e[0], e[0], fmaf(e[1], e[1], e[2] * e[2])));
                    }
                    const float R = 1.4f * sqrtf(q2);
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float cc = rows_s[r][kFCh + c] + rows_s[r][kFCl + c];
                        blo[c] = cc - R;
                        bhi[c] = cc + R;
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        blo[c] = fminf(blo[c], __shfl_down_sync(0xffffffffu, blo[c], o));
                        bhi[c] = fmaxf(bhi[c], __shfl_down_sync(0xffffffffu, bhi[c], o));
                    }
                if (lane == 0)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        box_s[w][c] = blo[c];
                        box_s[w][3 + c] = bhi[c];
                    }
            }
            // columns: every warp holds the same 32 trial triangles
            float clo[3], chi[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                clo[c] = INFINITY;
                chi[c] = -INFINITY;
            }
            if (j >= 0) {
                const float R = 1.4f * trif_rad(tb);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float cc = tb.ch[c] + tb.cl[c];
                    clo[c] = cc - R;
                    chi[c] = cc + R;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    clo[c] = fminf(clo[c], __shfl_xor_sync(0xffffffffu, clo[c], o));
                    chi[c] = fmaxf(chi[c], __shfl_xor_sync(0xffffffffu, chi[c], o));
                }
            __syncthreads();
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float rlo = box_s[0][c], rhi = box_s[0][3 + c];
#pragma unroll
                for (int q = 1; q < kBoxWarps; ++q) {
                    rlo = fminf(rlo, box_s[q][c]);
                    rhi = fmaxf(rhi, box_s[q][3 + c]);
                }
                far_tile |= clo[c] > rhi || rlo > chi[c];
            }
        }
        }
        if (j < 0) continue;
        for (int r = w; r < nr; r += nw) {
            const int32_t i = rid_s[r];
            if (i < 0) continue;
            float f[kTileFields];
            const float4 *src = reinterpret_cast<const float4 *>(rows_s[r]);
#pragma unroll
            for (int v = 0; v < kTileFields / 4; ++v) {
                const float4 x = src[v];
                f[4 * v] = x.x;
                f[4 * v + 1] = x.y;
                f[4 * v + 2] = x.z;
                f[4 * v + 3] = x.w;
            }
            const int vi[3] = {__float_as_int(f[kFId]), __float_as_int(f[kFId + 1]),
                               __float_as_int(f[kFId + 2])};
            const int64_t dst = (a0 + r) * n_trial + b;
            if (!far_tile) {
                const int s = count_shared(vi, vj);
                if (s > 0) {
                    push_singular(s, i, j, dst, l1, l2, l3, counts, cap, err);
                    continue;
                }
            }
            TriF ta;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                ta.ch[c] = f[kFCh + c];
                ta.cl[c] = f[kFCl + c];
                ta.n[c] = f[kFN + c];
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q)
#pragma unroll
                for (int c = 0; c < 3; ++c) ta.q[q][c] = f[kFQ + 3 * q + c];
            ta.s.hi = f[kFS];
            ta.s.lo = f[kFS + 1];
            if constexpr (!CPLX) {
                // widened with two conversions and one addition on the FP64
                // pipe (idle in this kernel) for the single layer; on the
                // integer pipe for the double layers (measured faster each)
                const FF v = entry_mixed_laplace_ff<OP>(ta, tb, R.wf);
                if (OP == 0)
                    reinterpret_cast<double *>(out)[dst] = (double)v.hi + (double)v.lo;
                else
                    reinterpret_cast<double *>(out)[dst] = f2d_exact(v.hi) + f2d_exact(v.lo);
            } else {
                store_val<CPLX>(out, dst, E::eval(ta, tb, R, k));
            }
        }
    }
}

template <int OP, bool CPLX>
__global__ void __launch_bounds__(kTileThreads)
k_entries_tiled(DevGeom g, QuadRule R, double k, const int32_t *__restrict__ test, int64_t n_test,
                const int32_t *__restrict__ trial, int64_t n_trial, void *out, SingPair *l1,
                SingPair *l2, SingPair *l3, unsigned long long *counts, unsigned long long cap,
                int *err)
{
    entries_tiled_body<OP, CPLX>(g, R, k, test, n_test, trial, n_trial, out, l1, l2, l3, counts,
                                 cap, err);
}

// The Laplace single layer with a register bound that keeps kSlpMinBlocks
// CTAs on an SM
__global__ void __launch_bounds__(kTileThreads, kSlpMinBlocks)
k_entries_tiled_slp(DevGeom g, QuadRule R, const int32_t *__restrict__ test, int64_t n_test,
                    const int32_t *__restrict__ trial, int64_t n_trial, void *out, SingPair *l1,
                    SingPair *l2, SingPair *l3, unsigned long long *counts, unsigned long long cap,
                    int *err)
{
    entries_tiled_body<0, false>(g, R, 0.0, test, n_test, trial, n_trial, out, l1, l2, l3, counts,
                                 cap, err);
}

// ---- Sauter-Schwab singular pairs (FP64) -----------------------------------
// (vertex orders: singular_order in bem_device.cuh)
constexpr int kSingThreads = 128;
constexpr int kSingMaxPts = 6 * NGL * NGL * NGL;  // largest table (identical, helm)

// PREC 1 with real k (Laplace in BEM_MIXED_SP): the evaluations after the
// Sauter-Schwab transformation in FP32 (smooth integrands, the reduced
// distance bounded away from zero), summed in FP32 within a node row and in
// float-float outside it; the pair's geometry, its edge basis and the final
// scaling in FP64.  Otherwise (BEM_FP64, BEM_MIXED, Helmholtz) every step in
// FP64.
//
// SYM (vertex-adjacent pairs only): the rule's node set for (T_j, T_i) is that
// of (T_i, T_j) with x and y exchanged (both triangles start at the shared
// vertex, Sec. 3.2.3), so one quadrature gives A_ij and A_ji: the single
// layer is the same value (g(x, y) = g(y, x)); the double layer's transposed
// entry has the adjoint kernel's numerator (x - y).n_x over the same nodes,
// and the reverse for the adjoint double layer.  A_ij goes to pairs[pid].dest
// and A_ji to dest2[pid], each only when its offset is >= 0.
template <int CASE, int OP, bool CPLX, int PREC = 0, bool SYM = false>
__global__ void __launch_bounds__(kSingThreads)
k_singular(DevGeom g, SingTable tab, double k, const SingPair *__restrict__ pairs,
           const unsigned long long *__restrict__ dev_count, int64_t max_count, void *out,
           const int64_t *__restrict__ dest2)
{
    static_assert(!SYM || CASE == 1, "transposed pairs share nodes in the vertex case only");
    // the operator whose kernel gives the transposed entry
    constexpr int OPT = OP == 1 ? 2 : (OP == 2 ? 1 : 0);
    constexpr int NC = CASE == 3 ? 2 : (CASE == 2 ? 3 : 4);
    constexpr int ROWS = CPLX ? 5 : 6;
    constexpr bool kMix = PREC == 1 && !CPLX;
    __shared__ double s_tab[6 * kSingMaxPts];
    __shared__ float s_tabf[kMix ? 6 * kSingMaxPts : 1];
    const int npts = CPLX ? tab.n_helm : tab.n_lap;
    const double *src = CPLX ? tab.helm : tab.lap;
    for (int e = threadIdx.x; e < ROWS * npts; e += blockDim.x) {
        s_tab[e] = src[e];
        if constexpr (kMix) s_tabf[e] = (float)src[e];
    }
    __syncthreads();
    // the xi rule in FP32 and its moments (vertex case of the mixed path)
    float xf[NGL], wf[NGL];
    double sx1m = 0.0, sx2m = 0.0;
    if constexpr (kMix && CASE == 1) {
#pragma unroll
        for (int a = 0; a < NGL; ++a) {
            xf[a] = (float)tab.xi[a];
            wf[a] = (float)tab.wxi[a];
            sx1m = fma(tab.wxi[a], tab.xi[a], sx1m);
            sx2m = fma(tab.wxi[a] * tab.xi[a], tab.xi[a], sx2m);
        }
    }
    int64_t count = max_count;
    if (dev_count) {
        unsigned long long c = *dev_count;
        if ((int64_t)c < count) count = (int64_t)c;
    }
    const int64_t n = g.nt;
    for (int64_t pid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pid < count;
         pid += (int64_t)gridDim.x * blockDim.x) {
        SingPair pr = pairs[pid];
        int ta[3], tb[3];
        for (int c = 0; c < 3; ++c) {
            ta[c] = g.tri[c * n + pr.i];
            tb[c] = g.tri[c * n + pr.j];
        }
        int oa[3], ob[3];
        singular_order<CASE>(ta, tb, oa, ob);
        double Pa[3][3], Pb[3][3], nx[3], ny[3];
        for (int v = 0; v < 3; ++v)
            for (int c = 0; c < 3; ++c) {
                Pa[v][c] = g.vtx[(3 * oa[v] + c) * n + pr.i];
                Pb[v][c] = g.vtx[(3 * ob[v] + c) * n + pr.j];
            }
        for (int c = 0; c < 3; ++c) {
            nx[c] = g.nrm[c * n + pr.i];
            ny[c] = g.nrm[c * n + pr.j];
        }
        // edge basis E_i of d = x - y
        double E[4][3];
        for (int c = 0; c < 3; ++c) {
            E[0][c] = Pa[1][c] - Pa[0][c];
            E[1][c] = Pa[2][c] - Pa[1][c];
            if (CASE == 2) {
                E[2][c] = Pb[2][c] - Pb[1][c];
                E[3][c] = 0.0;
            } else if (CASE == 1) {
                E[2][c] = Pb[1][c] - Pb[0][c];
                E[3][c] = Pb[2][c] - Pb[1][c];
            } else {
                E[2][c] = E[3][c] = 0.0;
            }
        }
        double eny[4], enx[4];
        for (int i = 0; i < 4; ++i) {
            eny[i] = E[i][0] * ny[0] + E[i][1] * ny[1] + E[i][2] * ny[2];
            enx[i] = E[i][0] * nx[0] + E[i][1] * nx[1] + E[i][2] * nx[2];
        }
        C2 acc = {0.0, 0.0}, acc2 = {0.0, 0.0};
        const bool flat_zero = (CASE == 3 && OP != 0);  // d.n = 0 on one flat panel
        if constexpr (kMix && CASE == 1) {
            // the factorised vertex-adjacent rule below in FP32, with x - y
            // formed per node pair (d0 = u_a - eta2 u'_b, d1 = eta2 u_b - u'_a)
            // instead of through the expanded quadratic
            float Ef[4][3], nxf[3], nyf[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
#pragma unroll
                for (int i = 0; i < 4; ++i) Ef[i][c] = (float)E[i][c];
                nxf[c] = (float)nx[c];
                nyf[c] = (float)ny[c];
            }
            float u[NGL][3], up[NGL][3], uny[NGL], upnx[NGL], wny[NGL], wnx[NGL];
#pragma unroll
            for (int a = 0; a < NGL; ++a) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    u[a][c] = fmaf(xf[a], Ef[1][c], Ef[0][c]);
                    up[a][c] = fmaf(xf[a], Ef[3][c], Ef[2][c]);
                }
                uny[a] = u[a][0] * nyf[0] + u[a][1] * nyf[1] + u[a][2] * nyf[2];
                upnx[a] = up[a][0] * nxf[0] + up[a][1] * nxf[1] + up[a][2] * nxf[2];
                wny[a] = wf[a] * uny[a];
                wnx[a] = wf[a] * upnx[a];
            }
            // double layers: w r0^3, w r1^3 (DLP and ADLP forms share them),
            // w_b u_b.n_y r1^3 (DLP) and w_b u'_b.n_x r0^3 (ADLP)
            constexpr bool kD = OP == 1 || (SYM && OP == 2), kA = OP == 2 || (SYM && OP == 1);
            FF s = {0.f, 0.f}, s2 = {0.f, 0.f};
#pragma unroll
            for (int c = 0; c < NGL; ++c) {
                const float e2 = xf[c];
#pragma unroll
                for (int a = 0; a < NGL; ++a) {
                    float s0 = 0.f, w0 = 0.f, w1 = 0.f, d1s = 0.f, a0s = 0.f;
#pragma unroll
                    for (int b = 0; b < NGL; ++b) {
                        float d0[3], d1[3];
#pragma unroll
                        for (int m = 0; m < 3; ++m) {
                            d0[m] = fmaf(-e2, up[b][m], u[a][m]);
                            d1[m] = fmaf(e2, u[b][m], -up[a][m]);
                        }
                        const float r0 = rsqrt_ftz(fmaf(d0[0], d0[0], fmaf(d0[1], d0[1], d0[2] * d0[2])));
                        const float r1 = rsqrt_ftz(fmaf(d1[0], d1[0], fmaf(d1[1], d1[1], d1[2] * d1[2])));
                        if (OP == 0) {
                            s0 = fmaf(wf[b], r0 + r1, s0);
                        } else {
                            const float c0 = r0 * r0 * r0, c1 = r1 * r1 * r1;
                            if (kD) {
                                w0 = fmaf(wf[b], c0, w0);
                                d1s = fmaf(wny[b], c1, d1s);
                            }
                            if (kA) {
                                a0s = fmaf(wnx[b], c0, a0s);
                                w1 = fmaf(wf[b], c1, w1);
                            }
                        }
                    }
                    const float sd = kD ? fmaf(uny[a], w0, e2 * d1s) : 0.f;  // DLP form
                    const float sA = kA ? fmaf(e2, a0s, upnx[a] * w1) : 0.f;  // ADLP form
                    const float sa = OP == 0 ? s0 : (OP == 1 ? sd : sA);
                    const float wq = (wf[c] * e2) * wf[a];
                    ff_add(s, wq * sa);
                    if (SYM && OP != 0) ff_add(s2, wq * (OP == 1 ? sA : sd));
                }
            }
            acc.re = ff_to_double(s) * (OP == 0 ? sx2m : sx1m);
            acc2.re = OP == 0 ? acc.re : ff_to_double(s2) * sx1m;
        } else if (CASE == 1 && !CPLX) {
            // Vertex-adjacent Laplace pair, factorised.  Region 0 maps to
            // x - y = xi (u(eta1) - eta2 u'(eta3)), region 1 to
            // x - y = xi (eta2 u(eta3) - u'(eta1)), with u(t) = E0 + t E1 and
            // u'(t) = E2 + t E3; J = xi^3 eta2.  So |x - y|^2 / xi^2 is a
            // quadratic in eta2 with coefficients |u_a|^2, u_a.u'_b, |u'_b|^2 over
            // the 4 x 4 node pairs, and the xi sums (of xi^2 for the single
            // layer, xi for the double layers) are taken once.
            double u[NGL][3], up[NGL][3], A[NGL], Cc[NGL], B[NGL][NGL], uny[NGL], upnx[NGL];
            double sx1 = 0.0, sx2 = 0.0;
            for (int a = 0; a < NGL; ++a) {
                const double xa = tab.xi[a];
                sx1 = fma(tab.wxi[a], xa, sx1);
                sx2 = fma(tab.wxi[a] * xa, xa, sx2);
                for (int c = 0; c < 3; ++c) {
                    u[a][c] = fma(xa, E[1][c], E[0][c]);
                    up[a][c] = fma(xa, E[3][c], E[2][c]);
                }
                A[a] = u[a][0] * u[a][0] + u[a][1] * u[a][1] + u[a][2] * u[a][2];
                Cc[a] = up[a][0] * up[a][0] + up[a][1] * up[a][1] + up[a][2] * up[a][2];
                uny[a] = u[a][0] * ny[0] + u[a][1] * ny[1] + u[a][2] * ny[2];
                upnx[a] = up[a][0] * nx[0] + up[a][1] * nx[1] + up[a][2] * nx[2];
            }
            for (int a = 0; a < NGL; ++a)
                for (int b = 0; b < NGL; ++b)
                    B[a][b] = u[a][0] * up[b][0] + u[a][1] * up[b][1] + u[a][2] * up[b][2];
            // nested sums: s = sum_c w_c e2_c sum_a w_a sum_b w_b (...); the
            // double layers' per-node factors (w_b u_b.n_y, w_b u'_b.n_x) are
            // formed once
            double wny[NGL], wnx[NGL];
            for (int b = 0; b < NGL; ++b) {
                wny[b] = tab.wxi[b] * uny[b];
                wnx[b] = tab.wxi[b] * upnx[b];
            }
            // the DLP form (d.n_y / r^3: region 0 xi u_a.n_y, region 1 xi
            // eta2 u_b.n_y) and the ADLP form (-d.n_x / r^3: region 0 xi eta2
            // u'_b.n_x, region 1 xi u'_a.n_x); with SYM a double layer takes
            // both, one for each of the two entries
            constexpr bool kD = OP == 1 || (SYM && OP == 2), kA = OP == 2 || (SYM && OP == 1);
            double s = 0.0, s2 = 0.0;
            for (int c = 0; c < NGL; ++c) {
                const double e2 = tab.xi[c], m2 = -2.0 * e2, q2 = e2 * e2;
                double sc = 0.0, sc2 = 0.0;
                for (int a = 0; a < NGL; ++a) {      // eta1 node
                    double s0 = 0.0, w0 = 0.0, w1 = 0.0, d1s = 0.0, a0s = 0.0;
                    for (int b = 0; b < NGL; ++b) {  // eta3 node
                        const double q0 = fma(q2, Cc[b], fma(m2, B[a][b], A[a]));
                        const double q1 = fma(q2, A[b], fma(m2, B[b][a], Cc[a]));
                        const double r0 = rsqrt_fp64(q0), r1 = rsqrt_fp64(q1);
                        if (OP == 0) {
                            s0 = fma(tab.wxi[b], r0 + r1, s0);
                        } else {
                            const double c0 = r0 * r0 * r0, c1 = r1 * r1 * r1;
                            if (kD) {
                                w0 = fma(tab.wxi[b], c0, w0);
                                d1s = fma(wny[b], c1, d1s);
                            }
                            if (kA) {
                                a0s = fma(wnx[b], c0, a0s);
                                w1 = fma(tab.wxi[b], c1, w1);
                            }
                        }
                    }
                    const double sd = kD ? fma(uny[a], w0, e2 * d1s) : 0.0;
                    const double sA = kA ? fma(e2, a0s, upnx[a] * w1) : 0.0;
                    const double sa = OP == 0 ? s0 : (OP == 1 ? sd : sA);
                    sc = fma(tab.wxi[a], sa, sc);
                    if (SYM && OP != 0) sc2 = fma(tab.wxi[a], OP == 1 ? sA : sd, sc2);
                }
                s = fma(tab.wxi[c] * e2, sc, s);
                if (SYM && OP != 0) s2 = fma(tab.wxi[c] * e2, sc2, s2);
            }
            acc.re = s * (OP == 0 ? sx2 : sx1);
            acc2.re = OP == 0 ? acc.re : s2 * sx1;
        } else if (!flat_zero && kMix) {
            // the merged directions in FP32, summed in float-float
            float Ef[NC][3], enf[NC];
#pragma unroll
            for (int i = 0; i < NC; ++i) {
#pragma unroll
                for (int c = 0; c < 3; ++c) Ef[i][c] = (float)E[i][c];
                enf[i] = OP == 0 ? 0.f : (float)(OP == 1 ? eny[i] : enx[i]);
            }
            FF s = {0.f, 0.f};
            for (int q = 0; q < npts; ++q) {
                float cf[NC];
#pragma unroll
                for (int i = 0; i < NC; ++i) cf[i] = s_tabf[i * npts + q];
                float d[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float x = cf[0] * Ef[0][c];
#pragma unroll
                    for (int i = 1; i < NC; ++i) x = fmaf(cf[i], Ef[i][c], x);
                    d[c] = x;
                }
                const float ri = rsqrt_ftz(fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2])));
                float term;
                if (OP == 0) {
                    term = s_tabf[4 * npts + q] * ri;
                } else {
                    float dn = 0.f;
#pragma unroll
                    for (int i = 0; i < NC; ++i) dn = fmaf(cf[i], enf[i], dn);
                    if (OP == 2) dn = -dn;  // ADLP kernel has -(x - y).n_x
                    term = s_tabf[5 * npts + q] * dn * (ri * ri * ri);
                }
                ff_add(s, term);
            }
            acc.re = ff_to_double(s);
        } else if (!flat_zero) {
            for (int q = 0; q < npts; ++q) {
                double cf[NC];
#pragma unroll
                for (int i = 0; i < NC; ++i) cf[i] = s_tab[i * npts + q];
                double d[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    double x = cf[0] * E[0][c];
#pragma unroll
                    for (int i = 1; i < NC; ++i) x = fma(cf[i], E[i][c], x);
                    d[c] = x;
                }
                double r2 = fma(d[0], d[0], fma(d[1], d[1], d[2] * d[2]));
                double ri = rsqrt_fp64(r2);
                double dn = 0.0, dn2 = 0.0;
                if (OP != 0) {
#pragma unroll
                    for (int i = 0; i < NC; ++i) dn = fma(cf[i], OP == 1 ? eny[i] : enx[i], dn);
                    if (OP == 2) dn = -dn;  // ADLP kernel has -(x - y).n_x
                    if (SYM) {
                        // the transposed entry's numerator (the other form)
#pragma unroll
                        for (int i = 0; i < NC; ++i) dn2 = fma(cf[i], OPT == 1 ? eny[i] : enx[i], dn2);
                        if (OPT == 2) dn2 = -dn2;
                    }
                }
                if (!CPLX) {
                    if (OP == 0) acc.re = fma(s_tab[4 * npts + q], ri, acc.re);
                    else acc.re = fma(s_tab[5 * npts + q] * dn, ri * ri * ri, acc.re);
                } else {
                    // d = xi * dt: sum the xi axis here
                    double rt = r2 * ri, weta = s_tab[4 * npts + q];
#pragma unroll
                    for (int m = 0; m < NGL; ++m) {
                        double xi = tab.xi[m], r = xi * rt, sn, cs;
                        sincos(k * r, &sn, &cs);
                        if (OP == 0) {
                            // xi^3 J_eta exp(ikr) / (xi rt)
                            double f = tab.wxi[m] * xi * xi * weta * ri;
                            acc.re = fma(f, cs, acc.re);
                            acc.im = fma(f, sn, acc.im);
                        } else {
                            // xi^3 J_eta exp(ikr)(1 - ikr) xi dn / (xi rt)^3
                            const double f0 = tab.wxi[m] * xi * weta * ri * ri * ri;
                            const double kr = k * r;
                            const double er = fma(kr, sn, cs), ei = fma(-kr, cs, sn);
                            const double f = f0 * dn;
                            acc.re = fma(f, er, acc.re);
                            acc.im = fma(f, ei, acc.im);
                            if (SYM) {
                                const double f2 = f0 * dn2;
                                acc2.re = fma(f2, er, acc2.re);
                                acc2.im = fma(f2, ei, acc2.im);
                            }
                        }
                    }
                }
            }
        }
        double sc = 4.0 * g.area[pr.i] * g.area[pr.j] * kInv4Pi;
        if (!SYM || pr.dest >= 0) store_val<CPLX>(out, pr.dest, {acc.re * sc, acc.im * sc});
        if constexpr (SYM) {
            const int64_t d2 = dest2[pid];
            if (d2 >= 0) {
                if (OP == 0) acc2 = acc;
                store_val<CPLX>(out, d2, {acc2.re * sc, acc2.im * sc});
            }
        }
    }
}

// Near-field regular pairs: one warp per dense block, entries flattened
// column-major over the lanes (the blocks' storage order); pairs sharing a
// vertex are left to k_singular.
constexpr int kNearThreads = 128;

template <int OP, bool CPLX, int PREC>
__global__ void __launch_bounds__(kNearThreads)
k_near_regular(DevGeom g, QuadRule R, double k, const NearBlock *__restrict__ blocks,
               int64_t nblocks, void *out)
{
    using E = RegularEntry<OP, CPLX, PREC>;
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = warp; b < nblocks; b += nwarps) {
        const NearBlock B = blocks[b];
        const int m = (int)(B.te - B.tb), nn = (int)(B.se - B.sb);
        // entry e = c * m + r of the column-major block, stepped by 32
        // without division
        int c = lane / m, r = lane - c * m;
        const int dc = 32 / m, dr = 32 - dc * m;
        const int64_t tot = (int64_t)m * nn;
        for (int64_t e = lane; e < tot; e += 32) {
            // pairs that share a vertex get a value here that the singular
            // kernel, launched after this one on the same stream, overwrites
            typename E::Tri ta, tb;
            E::load(g, B.tb + r, ta);
            E::load(g, B.sb + c, tb);
            store_val<CPLX>(out, B.off + e, E::eval(ta, tb, R, k));
            c += dc;
            r += dr;
            if (r >= m) {
                r -= m;
                ++c;
            }
        }
    }
}

int num_sms_cached()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

}  // namespace

cudaError_t launch_geometry(const double *V, const int32_t *T, const int32_t *perm, int64_t nt,
                            const QuadRule &rule, void *const bufs[6], cudaStream_t st)
{
    int64_t grid = (nt + kGeomThreads - 1) / kGeomThreads;
    k_geometry<<<(unsigned)grid, kGeomThreads, 0, st>>>(
        V, T, perm, nt, rule, (int32_t *)bufs[0], (double *)bufs[1], (double *)bufs[2],
        (double *)bufs[3], (double *)bufs[4], (float *)bufs[5]);
    count_launches(1);
    return cudaGetLastError();
}

template <int OP, bool CPLX, int PREC>
static void entries_launch(const DevGeom &g, const QuadRule &R, double k, const int32_t *test,
                           int64_t n_test, const int32_t *trial, int64_t n_trial, void *out,
                           SingPair *lists[3], unsigned long long *counts,
                           unsigned long long cap, int *err, cudaStream_t st)
{
    if constexpr (PREC == 1) {
        // persistent grid: every SM filled, tiles handed out round-robin
        constexpr bool slp = OP == 0 && !CPLX;
        static int per_sm = 0;
        if (!per_sm) {
            if constexpr (slp)
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_entries_tiled_slp,
                                                              kTileThreads, 0);
            else
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_entries_tiled<OP, CPLX>,
                                                              kTileThreads, 0);
            if (per_sm < 1) per_sm = 1;
        }
        const int64_t ntiles = (n_trial + 31) / 32 * ((n_test + kTileRows - 1) / kTileRows);
        int64_t grid = (int64_t)num_sms_cached() * per_sm;
        if (grid > ntiles) grid = ntiles;
        if constexpr (slp)
            k_entries_tiled_slp<<<(unsigned)grid, kTileThreads, 0, st>>>(
                g, R, test, n_test, trial, n_trial, out, lists[0], lists[1], lists[2], counts, cap,
                err);
        else
            k_entries_tiled<OP, CPLX><<<(unsigned)grid, kTileThreads, 0, st>>>(
                g, R, k, test, n_test, trial, n_trial, out, lists[0], lists[1], lists[2], counts,
                cap, err);
        count_launches(1);
    } else {
        int64_t gx = (n_trial + kEntBx - 1) / kEntBx;
        int64_t gy = (n_test + kEntBy - 1) / kEntBy;
        if (gy > 65535) gy = 65535;
        dim3 grid((unsigned)gx, (unsigned)gy), block(kEntBx, kEntBy);
        k_entries<OP, CPLX, PREC><<<grid, block, 0, st>>>(g, R, k, test, n_test, trial, n_trial,
                                                          out, lists[0], lists[1], lists[2],
                                                          counts, cap, err);
        count_launches(1);
    }
}

#define BEM_DISPATCH(OPV, CPLXV, PRECV, CALL)                                           \
    do {                                                                                \
        if (OPV == 0 && !CPLXV && PRECV == 0) { constexpr int OP = 0; constexpr bool CPLX = false; constexpr int PREC = 0; CALL; } \
        else if (OPV == 0 && !CPLXV && PRECV == 1) { constexpr int OP = 0; constexpr bool CPLX = false; constexpr int PREC = 1; CALL; } \
        else if (OPV == 0 && CPLXV && PRECV == 0) { constexpr int OP = 0; constexpr bool CPLX = true; constexpr int PREC = 0; CALL; } \
        else if (OPV == 0 && CPLXV && PRECV == 1) { constexpr int OP = 0; constexpr bool CPLX = true; constexpr int PREC = 1; CALL; } \
        else if (OPV == 1 && !CPLXV && PRECV == 0) { constexpr int OP = 1; constexpr bool CPLX = false; constexpr int PREC = 0; CALL; } \
        else if (OPV == 1 && !CPLXV && PRECV == 1) { constexpr int OP = 1; constexpr bool CPLX = false; constexpr int PREC = 1; CALL; } \
        else if (OPV == 1 && CPLXV && PRECV == 0) { constexpr int OP = 1; constexpr bool CPLX = true; constexpr int PREC = 0; CALL; } \
        else if (OPV == 1 && CPLXV && PRECV == 1) { constexpr int OP = 1; constexpr bool CPLX = true; constexpr int PREC = 1; CALL; } \
        else if (OPV == 2 && !CPLXV && PRECV == 0) { constexpr int OP = 2; constexpr bool CPLX = false; constexpr int PREC = 0; CALL; } \
        else if (OPV == 2 && !CPLXV && PRECV == 1) { constexpr int OP = 2; constexpr bool CPLX = false; constexpr int PREC = 1; CALL; } \
        else if (OPV == 2 && CPLXV && PRECV == 0) { constexpr int OP = 2; constexpr bool CPLX = true; constexpr int PREC = 0; CALL; } \
        else { constexpr int OP = 2; constexpr bool CPLX = true; constexpr int PREC = 1; CALL; } \
    } while (0)

cudaError_t launch_entries_regular(const DevGeom &g, const QuadRule &rule, int op, double k,
                                   int prec, const int32_t *test, int64_t n_test,
                                   const int32_t *trial, int64_t n_trial, void *out,
                                   SingPair *lists[3], unsigned long long *counts,
                                   unsigned long long cap, int *err, cudaStream_t st)
{
    const bool cplx = k != 0.0;
    BEM_DISPATCH(op, cplx, (prec != 0 ? 1 : 0),
                 (entries_launch<OP, CPLX, PREC>(g, rule, k, test, n_test, trial, n_trial, out,
                                                 lists, counts, cap, err, st)));
    return cudaGetLastError();
}

template <int CASE, int OP, bool CPLX, int PREC>
static void singular_launch(const DevGeom &g, const SingTable &tab, double k, const SingPair *p,
                            const unsigned long long *dc, int64_t hc, int64_t gc, void *out,
                            cudaStream_t st, const int64_t *dest2)
{
    if (hc <= 0 || gc <= 0) return;
    // the grid covers gc pairs; its threads stride over all min(*dc, hc)
    int64_t want = (gc + kSingThreads - 1) / kSingThreads;
    int64_t cap = (int64_t)num_sms_cached() * 16;
    unsigned grid = (unsigned)(want < cap ? want : cap);
    if constexpr (CASE == 1) {
        if (dest2) {
            k_singular<CASE, OP, CPLX, PREC, true>
                <<<grid, kSingThreads, 0, st>>>(g, tab, k, p, dc, hc, out, dest2);
            count_launches(1);
            return;
        }
    }
    k_singular<CASE, OP, CPLX, PREC><<<grid, kSingThreads, 0, st>>>(g, tab, k, p, dc, hc, out, nullptr);
    count_launches(1);
}

cudaError_t launch_singular(const DevGeom &g, const SingTable *tabs, int op, double k, int prec,
                            const SingPair *pairs[3], const unsigned long long *dev_counts,
                            const int64_t host_counts[3], void *out, cudaStream_t st,
                            const int64_t *grid_counts, const int64_t *vertex_dest2)
{
    const bool cplx = k != 0.0;
    for (int c = 1; c <= 3; ++c) {
        const unsigned long long *dc = dev_counts ? dev_counts + (c - 1) : nullptr;
        const SingTable &T = tabs[c - 1];
        int64_t hc = host_counts[c - 1];
        int64_t gc = grid_counts ? grid_counts[c - 1] : hc;
        const SingPair *P = pairs[c - 1];
        // FP32 integrands only for Laplace in BEM_MIXED_SP; BEM_FP64,
        // BEM_MIXED and Helmholtz pairs stay FP64
        BEM_DISPATCH(op, cplx, (!cplx && prec == 2 ? 1 : 0), ({
                         if (c == 1) singular_launch<1, OP, CPLX, PREC>(g, T, k, P, dc, hc, gc, out, st, vertex_dest2);
                         else if (c == 2) singular_launch<2, OP, CPLX, PREC>(g, T, k, P, dc, hc, gc, out, st, nullptr);
                         else singular_launch<3, OP, CPLX, PREC>(g, T, k, P, dc, hc, gc, out, st, nullptr);
                     }));
    }
    return cudaGetLastError();
}

cudaError_t launch_near_regular(const DevGeom &g, const QuadRule &rule, int op, double k, int prec,
                                const NearBlock *blocks, int64_t nblocks, void *out,
                                cudaStream_t st)
{
    if (nblocks <= 0) return cudaSuccess;
    const bool cplx = k != 0.0;
    int64_t warps = nblocks;
    int64_t grid = (warps * 32 + kNearThreads - 1) / kNearThreads;
    int64_t cap = (int64_t)num_sms_cached() * 64;
    if (grid > cap) grid = cap;
    BEM_DISPATCH(op, cplx, (prec != 0 ? 1 : 0),
                 (k_near_regular<OP, CPLX, PREC>
                  <<<(unsigned)grid, kNearThreads, 0, st>>>(g, rule, k, blocks, nblocks, out)));
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace bem

namespace bem {
namespace {
__global__ void k_debug_rsqrt(const double *__restrict__ x, double *__restrict__ y, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = rsqrt_fp64(x[i]);
}
}  // namespace

cudaError_t launch_debug_rsqrt(const double *x, double *y, int64_t n, cudaStream_t st)
{
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    k_debug_rsqrt<<<(unsigned)blocks, 256, 0, st>>>(x, y, n);
    count_launches(1);
    return cudaGetLastError();
}
}  // namespace bem
