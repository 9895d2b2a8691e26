// Piecewise linear spaces: dense sub-blocks of element pairs
// (bem_entries_dp1), the near-field blocks of a DP1 H-matrix, and the
// Sauter-Schwab local matrices of touching pairs (FP64).  Every kernel
// produces the 3 x 3 local matrix of an element pair from one set of kernel
// evaluations (Sec. 3.3, Algorithm "Integral Evaluation").
#include "bem_dp1.cuh"

namespace bem {

namespace {

template <bool CPLX>
__device__ __forceinline__ void store_val1(void *out, int64_t idx, C2 v)
{
    if (CPLX) reinterpret_cast<double2 *>(out)[idx] = make_double2(v.re, v.im);
    else reinterpret_cast<double *>(out)[idx] = v.re;
}

template <bool CPLX>
__device__ __forceinline__ void store_local(void *out, int64_t dest, int64_t rs, int64_t cs,
                                            const C2 *v)
{
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) store_val1<CPLX>(out, dest + a * rs + b * cs, v[3 * a + b]);
}

int num_sms_dp1()
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

// Dense sub-block of element pairs: thread (a, b) evaluates the local matrix
// of (test[a], trial[b]) by the regular rule, or queues the pair for the
// singular kernel.  Output [3 n_test][3 n_trial], row 3a + alpha.
constexpr int kDp1Bx = 32, kDp1By = 4;

template <int OP, bool CPLX, int PREC>
__global__ void __launch_bounds__(kDp1Bx *kDp1By)
k_entries_dp1(DevGeom g, QuadRule R, double k, const int32_t *__restrict__ test, int64_t n_test,
              const int32_t *__restrict__ trial, int64_t n_trial, void *out, SingPairL *l1,
              SingPairL *l2, SingPairL *l3, unsigned long long *counts, unsigned long long cap,
              int *err)
{
    using E = LocalEntry<OP, CPLX, PREC>;
    const int64_t b = (int64_t)blockIdx.x * kDp1Bx + threadIdx.x;
    if (b >= n_trial) return;
    const int32_t j = trial[b];
    if (j < 0 || j >= g.nt) {
        atomicExch(err, 1);
        return;
    }
    typename E::Tri tb;
    E::load(g, j, tb);
    int vj[3];
    E::ids(g, j, vj);
    const int64_t ld = 3 * n_trial;
    for (int64_t a = (int64_t)blockIdx.y * kDp1By + threadIdx.y; a < n_test;
         a += (int64_t)gridDim.y * kDp1By) {
        const int32_t i = test[a];
        if (i < 0 || i >= g.nt) {
            atomicExch(err, 1);
            continue;
        }
        const int64_t dest = 3 * a * ld + 3 * b;
        int vi[3];
        E::ids(g, i, vi);
        const int s = count_shared(vi, vj);
        if (s > 0) {
            const unsigned long long slot = atomicAdd(&counts[s - 1], 1ull);
            if (slot < cap) {
                SingPairL *L = s == 1 ? l1 : (s == 2 ? l2 : l3);
                L[slot] = {i, j, dest, (int32_t)ld, 1};
            } else {
                atomicExch(err, 2);
            }
            continue;
        }
        typename E::Tri ta;
        E::load(g, i, ta);
        C2 v[9];
        E::template eval<2>(ta, tb, R, k, 0, v);
        store_local<CPLX>(out, dest, ld, 1, v);
    }
}

// Near-field blocks of a DP1 H-matrix: one warp per dense block, element
// pairs flattened over the lanes; every pair writes its 3 x 3 local matrix
// into the column-major block.  Touching pairs are overwritten by the
// singular kernel that follows on the same stream.
constexpr int kNearDp1Threads = 128;

template <int OP, bool CPLX, int PREC>
__global__ void __launch_bounds__(kNearDp1Threads)
k_near_dp1(DevGeom g, QuadRule R, double k, const NearBlock *__restrict__ blocks, int64_t nblocks,
           void *out)
{
    using E = LocalEntry<OP, CPLX, PREC>;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t bk = warp; bk < nblocks; bk += nwarps) {
        const NearBlock B = blocks[bk];
        const int64_t t0 = B.tb / 3, s0 = B.sb / 3;
        const int mt = (int)((B.te - B.tb) / 3), nt = (int)((B.se - B.sb) / 3);
        const int64_t ld = B.te - B.tb;   // column stride of the column-major block
        const int64_t tot = (int64_t)mt * nt;
        for (int64_t e = lane; e < tot; e += 32) {
            const int c = (int)(e / mt), r = (int)(e - (int64_t)c * mt);
            typename E::Tri ta, tb;
            E::load(g, t0 + r, ta);
            E::load(g, s0 + c, tb);
            C2 v[9];
            E::template eval<2>(ta, tb, R, k, 0, v);
            store_local<CPLX>(out, B.off + 3 * c * ld + 3 * r, 1, ld, v);
        }
    }
}

// Touching pairs (Sauter-Schwab maps, Erichsen-Sauter scheme of Sec. 3.2.3),
// FP64.  Every map is homogeneous of degree one in xi: the table lists the eta
// nodes (d / xi in the case's edge basis, the eta weight, and the reference
// points x^ / xi, y^ / xi), and the xi axis is summed here with the Jacobian
// factor xi^3.  With P_i the parametrisation's vertex order, the barycentric
// coordinates of chi(x^) are (1 - x1, x1 - x2, x2) with respect to
// (P0, P1, P2); they weight the local dofs of the stored vertices o[i].
constexpr int kSingDp1Threads = 128;
constexpr int kSingDp1MaxPts = 6 * NGL * NGL * NGL;

template <int CASE, int OP, bool CPLX>
__global__ void __launch_bounds__(kSingDp1Threads)
k_singular_dp1(DevGeom g, SingTable tab, double k, const SingPairL *__restrict__ pairs,
               const unsigned long long *__restrict__ dev_count, int64_t max_count, void *out)
{
    constexpr int NC = CASE == 3 ? 2 : (CASE == 2 ? 3 : 4);
    __shared__ double s_tab[9 * kSingDp1MaxPts];
    const int npts = tab.n_helm;
    for (int e = threadIdx.x; e < 5 * npts; e += blockDim.x) s_tab[e] = tab.helm[e];
    for (int e = threadIdx.x; e < 4 * npts; e += blockDim.x) s_tab[5 * npts + e] = tab.xy[e];
    __syncthreads();
    int64_t count = max_count;
    if (dev_count) {
        const unsigned long long c = *dev_count;
        if ((int64_t)c < count) count = (int64_t)c;
    }
    const int64_t n = g.nt;
    const bool flat_zero = (CASE == 3 && OP != 0);  // d.n = 0 on one flat panel
    for (int64_t pid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pid < count;
         pid += (int64_t)gridDim.x * blockDim.x) {
        const SingPairL pr = pairs[pid];
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
        // edge basis E_i of d = x - y (as in k_singular)
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
        // acc[i][j]: parametrisation vertices i (test) and j (trial)
        C2 acc[9];
        for (int o = 0; o < 9; ++o) acc[o] = {0.0, 0.0};
        if (!flat_zero && !CPLX) {
            // Laplace: with lambda^x = e_0 + xi beta (beta = (-X1, X1 - X2, X2))
            // and lambda^y = e_0 + xi beta' the xi integrand is a polynomial,
            // xi^p (kernel weight W) times the product of the two affine
            // factors (p = 2 single layer, 1 double layers), of degree <= p + 2,
            // which the xi rule integrates exactly; so the xi sum is taken once
            // through the moments M_p = sum_m w_m xi_m^p, and per eta node only
            // the sums of W, W beta_a, W beta'_b and W beta_a beta'_b gather.
            double S0 = 0.0, Sa[3] = {0.0, 0.0, 0.0}, Sb[3] = {0.0, 0.0, 0.0}, Sab[9];
#pragma unroll
            for (int o = 0; o < 9; ++o) Sab[o] = 0.0;
            for (int q = 0; q < npts; ++q) {
                double cf[NC];
#pragma unroll
                for (int i = 0; i < NC; ++i) cf[i] = s_tab[i * npts + q];
                const double weta = s_tab[4 * npts + q];
                const double X1 = s_tab[5 * npts + q], X2 = s_tab[6 * npts + q];
                const double Y1 = s_tab[7 * npts + q], Y2 = s_tab[8 * npts + q];
                double d[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    double x = cf[0] * E[0][c];
#pragma unroll
                    for (int i = 1; i < NC; ++i) x = fma(cf[i], E[i][c], x);
                    d[c] = x;
                }
                const double r2 = fma(d[0], d[0], fma(d[1], d[1], d[2] * d[2]));
                const double ri = rsqrt_fp64(r2);
                double W;
                if (OP == 0) {
                    W = weta * ri;
                } else {
                    double dn = 0.0;
#pragma unroll
                    for (int i = 0; i < NC; ++i) dn = fma(cf[i], OP == 1 ? eny[i] : enx[i], dn);
                    if (OP == 2) dn = -dn;  // ADLP kernel has -(x - y).n_x
                    W = weta * dn * (ri * ri * ri);
                }
                const double ba[3] = {-X1, X1 - X2, X2}, bb[3] = {-Y1, Y1 - Y2, Y2};
                S0 += W;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const double Wa = W * ba[a];
                    Sa[a] += Wa;
                    Sb[a] = fma(W, bb[a], Sb[a]);
#pragma unroll
                    for (int b = 0; b < 3; ++b) Sab[3 * a + b] = fma(Wa, bb[b], Sab[3 * a + b]);
                }
            }
            // moments of the xi rule
            const int p0 = OP == 0 ? 2 : 1;
            double M[3] = {0.0, 0.0, 0.0};
            for (int m = 0; m < NGL; ++m) {
                double xp = tab.wxi[m];
                for (int e = 0; e < p0; ++e) xp *= tab.xi[m];
                M[0] += xp;
                M[1] += xp * tab.xi[m];
                M[2] += xp * tab.xi[m] * tab.xi[m];
            }
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    double v = Sab[3 * a + b] * M[2];
                    if (a == 0) v = fma(Sb[b], M[1], v);
                    if (b == 0) v = fma(Sa[a], M[1], v);
                    if (a == 0 && b == 0) v = fma(S0, M[0], v);
                    acc[3 * a + b].re = v;
                }
        } else if (!flat_zero) {
            for (int q = 0; q < npts; ++q) {
                double cf[NC];
#pragma unroll
                for (int i = 0; i < NC; ++i) cf[i] = s_tab[i * npts + q];
                const double weta = s_tab[4 * npts + q];
                const double X1 = s_tab[5 * npts + q], X2 = s_tab[6 * npts + q];
                const double Y1 = s_tab[7 * npts + q], Y2 = s_tab[8 * npts + q];
                double d[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    double x = cf[0] * E[0][c];
#pragma unroll
                    for (int i = 1; i < NC; ++i) x = fma(cf[i], E[i][c], x);
                    d[c] = x;
                }
                const double r2 = fma(d[0], d[0], fma(d[1], d[1], d[2] * d[2]));
                const double ri = rsqrt_fp64(r2), rt = r2 * ri;
                double dn = 0.0;
                if (OP != 0) {
#pragma unroll
                    for (int i = 0; i < NC; ++i) dn = fma(cf[i], OP == 1 ? eny[i] : enx[i], dn);
                    if (OP == 2) dn = -dn;  // ADLP kernel has -(x - y).n_x
                }
#pragma unroll
                for (int m = 0; m < NGL; ++m) {
                    const double xi = tab.xi[m];
                    // kernel times xi^3 J_eta: SLP xi^2 / rt, DLP/ADLP xi dn / rt^3
                    double f = OP == 0 ? tab.wxi[m] * xi * xi * weta * ri
                                       : tab.wxi[m] * xi * weta * dn * ri * ri * ri;
                    C2 G = {f, 0.0};
                    if (CPLX) {
                        const double r = xi * rt;
                        double sn, cs;
                        sincos(k * r, &sn, &cs);
                        if (OP == 0) {
                            G = {f * cs, f * sn};
                        } else {
                            const double kr = k * r;
                            G = {f * fma(kr, sn, cs), f * fma(-kr, cs, sn)};
                        }
                    }
                    const double la[3] = {1.0 - xi * X1, xi * (X1 - X2), xi * X2};
                    const double lb[3] = {1.0 - xi * Y1, xi * (Y1 - Y2), xi * Y2};
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int b = 0; b < 3; ++b) {
                            const double w = la[a] * lb[b];
                            acc[3 * a + b].re = fma(w, G.re, acc[3 * a + b].re);
                            if (CPLX) acc[3 * a + b].im = fma(w, G.im, acc[3 * a + b].im);
                        }
                }
            }
        }
        const double sc = 4.0 * g.area[pr.i] * g.area[pr.j] * kInv4Pi;
        // parametrisation vertex i is stored vertex oa[i]
        C2 v[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                v[3 * oa[a] + ob[b]] = {acc[3 * a + b].re * sc, acc[3 * a + b].im * sc};
        store_local<CPLX>(out, pr.dest, pr.rs, pr.cs, v);
    }
}

#define BEM_DISPATCH_DP1(OPV, CPLXV, PRECV, CALL)                                           \
    do {                                                                                    \
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

template <int CASE, int OP, bool CPLX>
void singular_dp1_launch(const DevGeom &g, const SingTable &tab, double k, const SingPairL *p,
                         const unsigned long long *dc, int64_t hc, void *out, cudaStream_t st)
{
    if (hc <= 0) return;
    const int64_t want = (hc + kSingDp1Threads - 1) / kSingDp1Threads;
    const int64_t cap = (int64_t)num_sms_dp1() * 8;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    k_singular_dp1<CASE, OP, CPLX><<<grid, kSingDp1Threads, 0, st>>>(g, tab, k, p, dc, hc, out);
    count_launches(1);
}

// ---- continuous P1 and the hypersingular operator around a DP1 matrix ----
// Continuous P1 coefficients x (one per vertex) map to DP1 coefficients by
// x_dp1[3 t + a] = x[T[t][a]] (C), and a DP1 result returns to the vertices
// by the transpose, y[v] = sum of y_dp1 over the dofs of v (C^T), so that
// A_P1 = C^T A_DP1 C: the global assembly of the local matrices (Sec. 3.2.3).
template <class T>
__device__ __forceinline__ T vzero();
template <>
__device__ __forceinline__ double vzero<double>() { return 0.0; }
template <>
__device__ __forceinline__ double2 vzero<double2>() { return make_double2(0.0, 0.0); }
__device__ __forceinline__ double vaxpy(double a, double x, double y) { return fma(a, x, y); }
__device__ __forceinline__ double2 vaxpy(double a, double2 x, double2 y)
{
    return make_double2(fma(a, x.x, y.x), fma(a, x.y, y.y));
}
__device__ __forceinline__ double vadd(double a, double b) { return a + b; }
__device__ __forceinline__ double2 vadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

template <class T>
__global__ void k_p1_gather(const int32_t *__restrict__ tri, int64_t nt, const T *__restrict__ x,
                            T *__restrict__ xd)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= 3 * nt) return;
    const int64_t t = q / 3;
    const int a = (int)(q - 3 * t);
    xd[q] = x[tri[a * nt + t]];
}

template <class T>
__global__ void k_p1_scatter(const int64_t *__restrict__ vptr, const int32_t *__restrict__ vdof,
                             int64_t nv, const T *__restrict__ yd, T *__restrict__ y)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    T s = vzero<T>();
    for (int64_t q = vptr[v]; q < vptr[v + 1]; ++q) s = vadd(s, yd[vdof[q]]);
    y[v] = s;
}

// surface curl of the local basis function of vertex a on triangle t:
// n x grad lambda_a = (v_{a+1} - v_{a+2}) / (2 |T|)
__device__ __forceinline__ void curl_local(const DevGeom &g, int64_t t, int a, double c[3])
{
    const int64_t n = g.nt;
    const int a1 = (a + 1) % 3, a2 = (a + 2) % 3;
    const double s = 0.5 / g.area[t];
#pragma unroll
    for (int k = 0; k < 3; ++k) c[k] = (g.vtx[(3 * a1 + k) * n + t] - g.vtx[(3 * a2 + k) * n + t]) * s;
}

// Eq. (9), input side: xs[j] = Q_j x (the j-th component of the
// surface curl, constant on each triangle, at its three local dofs) and, for
// k != 0, xs[3 + j] = P_j x (n_j times the function).  One thread per triangle.
template <class T>
__global__ void k_hyps_in(DevGeom g, const T *__restrict__ x, T *__restrict__ xs, int nvec)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nt = g.nt;
    if (t >= nt) return;
    const int64_t nd = 3 * nt;
    T xv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) xv[a] = x[g.tri[a * nt + t]];
    T cu[3] = {vzero<T>(), vzero<T>(), vzero<T>()};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double c[3];
        curl_local(g, t, a, c);
#pragma unroll
        for (int j = 0; j < 3; ++j) cu[j] = vaxpy(c[j], xv[a], cu[j]);
    }
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int a = 0; a < 3; ++a) xs[j * nd + 3 * t + a] = cu[j];
    if (nvec == 6) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double nj = g.nrm[j * nt + t];
#pragma unroll
            for (int a = 0; a < 3; ++a) xs[(3 + j) * nd + 3 * t + a] = vaxpy(nj, xv[a], vzero<T>());
        }
    }
}

// Output side: y[v] = sum_j Q_j^T ys[j] - k^2 sum_j P_j^T ys[3 + j], one
// thread per vertex over its dofs in increasing order.
template <class T>
__global__ void k_hyps_out(const int64_t *__restrict__ vptr, const int32_t *__restrict__ vdof,
                           DevGeom g, int64_t nv, double k2, const T *__restrict__ ys, int nvec,
                           T *__restrict__ y)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const int64_t nt = g.nt, nd = 3 * nt;
    T s = vzero<T>();
    for (int64_t q = vptr[v]; q < vptr[v + 1]; ++q) {
        const int64_t d = vdof[q], t = d / 3;
        const int a = (int)(d - 3 * t);
        double c[3];
        curl_local(g, t, a, c);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const T sum3 = vadd(vadd(ys[j * nd + 3 * t], ys[j * nd + 3 * t + 1]), ys[j * nd + 3 * t + 2]);
            s = vaxpy(c[j], sum3, s);
        }
        if (nvec == 6) {
#pragma unroll
            for (int j = 0; j < 3; ++j) s = vaxpy(-k2 * g.nrm[j * nt + t], ys[(3 + j) * nd + d], s);
        }
    }
    y[v] = s;
}

}  // namespace

cudaError_t launch_entries_dp1(const DevGeom &g, const QuadRule &rule, int op, double k, int prec,
                               const int32_t *test, int64_t n_test, const int32_t *trial,
                               int64_t n_trial, void *out, SingPairL *lists[3],
                               unsigned long long *counts, unsigned long long cap, int *err,
                               cudaStream_t st)
{
    const bool cplx = k != 0.0;
    int64_t gx = (n_trial + kDp1Bx - 1) / kDp1Bx;
    int64_t gy = (n_test + kDp1By - 1) / kDp1By;
    if (gy > 65535) gy = 65535;
    const dim3 grid((unsigned)gx, (unsigned)gy), block(kDp1Bx, kDp1By);
    BEM_DISPATCH_DP1(op, cplx, prec,
                     (k_entries_dp1<OP, CPLX, PREC><<<grid, block, 0, st>>>(
                         g, rule, k, test, n_test, trial, n_trial, out, lists[0], lists[1],
                         lists[2], counts, cap, err)));
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_near_dp1(const DevGeom &g, const QuadRule &rule, int op, double k, int prec,
                            const NearBlock *blocks, int64_t nblocks, void *out, cudaStream_t st)
{
    if (nblocks <= 0) return cudaSuccess;
    const bool cplx = k != 0.0;
    int64_t grid = (nblocks * 32 + kNearDp1Threads - 1) / kNearDp1Threads;
    const int64_t cap = (int64_t)num_sms_dp1() * 64;
    if (grid > cap) grid = cap;
    BEM_DISPATCH_DP1(op, cplx, prec,
                     (k_near_dp1<OP, CPLX, PREC><<<(unsigned)grid, kNearDp1Threads, 0, st>>>(
                         g, rule, k, blocks, nblocks, out)));
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_singular_dp1(const DevGeom &g, const SingTable *tabs, int op, double k,
                                const SingPairL *pairs[3], const unsigned long long *dev_counts,
                                const int64_t host_counts[3], void *out, cudaStream_t st)
{
    const bool cplx = k != 0.0;
    for (int c = 1; c <= 3; ++c) {
        const unsigned long long *dc = dev_counts ? dev_counts + (c - 1) : nullptr;
        const SingTable &T = tabs[c - 1];
        const int64_t hc = host_counts[c - 1];
        const SingPairL *P = pairs[c - 1];
        BEM_DISPATCH_DP1(op, cplx, 0, ({
                             (void)PREC;
                             if (c == 1) singular_dp1_launch<1, OP, CPLX>(g, T, k, P, dc, hc, out, st);
                             else if (c == 2) singular_dp1_launch<2, OP, CPLX>(g, T, k, P, dc, hc, out, st);
                             else singular_dp1_launch<3, OP, CPLX>(g, T, k, P, dc, hc, out, st);
                         }));
    }
    return cudaGetLastError();
}

cudaError_t launch_p1_gather(bool cplx, const int32_t *tri, int64_t nt, const void *x, void *xd,
                             cudaStream_t st)
{
    const int64_t n = 3 * nt;
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (cplx)
        k_p1_gather<double2><<<grid, 256, 0, st>>>(tri, nt, (const double2 *)x, (double2 *)xd);
    else
        k_p1_gather<double><<<grid, 256, 0, st>>>(tri, nt, (const double *)x, (double *)xd);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_p1_scatter(bool cplx, const int64_t *vptr, const int32_t *vdof, int64_t nv,
                              const void *yd, void *y, cudaStream_t st)
{
    const unsigned grid = (unsigned)((nv + 255) / 256);
    if (cplx)
        k_p1_scatter<double2><<<grid, 256, 0, st>>>(vptr, vdof, nv, (const double2 *)yd, (double2 *)y);
    else
        k_p1_scatter<double><<<grid, 256, 0, st>>>(vptr, vdof, nv, (const double *)yd, (double *)y);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_hyps_in(bool cplx, const DevGeom &g, const void *x, void *xs, int nvec,
                           cudaStream_t st)
{
    const unsigned grid = (unsigned)((g.nt + 255) / 256);
    if (cplx)
        k_hyps_in<double2><<<grid, 256, 0, st>>>(g, (const double2 *)x, (double2 *)xs, nvec);
    else
        k_hyps_in<double><<<grid, 256, 0, st>>>(g, (const double *)x, (double *)xs, nvec);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_hyps_out(bool cplx, const int64_t *vptr, const int32_t *vdof, const DevGeom &g,
                            int64_t nv, double k, const void *ys, int nvec, void *y, cudaStream_t st)
{
    const unsigned grid = (unsigned)((nv + 255) / 256);
    if (cplx)
        k_hyps_out<double2><<<grid, 256, 0, st>>>(vptr, vdof, g, nv, k * k, (const double2 *)ys,
                                                  nvec, (double2 *)y);
    else
        k_hyps_out<double><<<grid, 256, 0, st>>>(vptr, vdof, g, nv, k * k, (const double *)ys, nvec,
                                                 (double *)y);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace bem
