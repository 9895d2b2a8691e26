/*
 * bem_oracle.c -- plain FP64 CPU oracle for P0 Galerkin BEM on flat
 * triangles and ACA-compressed hierarchical matrices, after Vater, Betcke,
 * Dilba, "Simple and efficient GPU parallelization of existing H-Matrix
 * accelerated BEM code" (arXiv 1711.01897).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * load it; the product library never does, and the two share no source,
 * header, table or generator.  Everything here is written to be read
 * against the paper, not to be fast: no blocking, no fusion, no reordering
 * beyond what a definition or algorithm states.  Rows/columns are spread
 * over threads with OpenMP only at the outermost loop.
 *
 * Pins (checked by tests/test_oracle_*.py, never by this file):
 *   - quadrature rules: polynomial exactness;
 *   - Sauter-Schwab maps: exact moments of T x T;
 *   - regular and singular entries: semi-analytic references built from the
 *     closed-form triangle potential and solid angle below, nested adaptive
 *     quadrature of the bounded Helmholtz remainder;
 *   - matrices: sphere single-layer identity, double-layer jump -1/2,
 *     symmetry, K' = K^T, Helmholtz -> Laplace as k -> 0;
 *   - tree / ACA / matvec: partition invariants, exact rank recovery,
 *     dense comparison on small meshes.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef double complex cplx;

enum { ORC_SLP = 0, ORC_DLP = 1, ORC_ADLP = 2 };

/* ------------------------------------------------------------------------ */
/* Quadrature rules                                                          */
/* ------------------------------------------------------------------------ */

/* Gauss-Legendre rule with n points on [0,1]: nodes are the roots of the
 * Legendre polynomial P_n (three-term recurrence), found by Newton's method;
 * weights 2 / ((1 - z^2) P_n'(z)^2), halved for the interval [0,1].
 * Used as the 1D factor of the 4D singular rules (Sec. 3.2, "Handling of
 * different types of integrals", scheme of Erichsen and Sauter). */
int orc_gauss_legendre01(int n, double *x, double *w)
{
    if (n < 1 || n > 128) return 1;
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 200; ++it) {
            double p0 = 1.0, p1 = z;
            if (n == 1) { p1 = z; p0 = 1.0; }
            for (int j = 2; j <= n; ++j) {
                double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            /* p1 = P_n(z), p0 = P_{n-1}(z) */
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        /* recompute derivative at the converged root */
        {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= n; ++j) {
                double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        /* z runs from near +1 downwards, so 0.5*(1-z) runs upwards */
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
    return 0;
}

/* Symmetric 6-point triangle rule of degree 4 (Sec. 3.2.1: six weights,
 * "quadrature order 4", symmetric Gauss triangle rule).  Two orbits of
 * barycentric points (a,a,1-2a) and (b,b,1-2b) with orbit weights W1, W2
 * (normalised so that all six weights sum to 1).  The four unknowns solve
 * the moment equations of the S3-invariant polynomials 1, e2, e3, e2^2 of
 * the barycentric coordinates (e2 = sum of pairwise products, e3 = product),
 * whose normalised integrals over a triangle are 1, 1/4, 1/60, 1/15.
 * Output: reference coordinates (s,t) of x = v0 + s (v1-v0) + t (v2-v0) and
 * weights w (sum 1). */
static void solve4(double A[4][4], double b[4])
{
    for (int c = 0; c < 4; ++c) {
        int p = c;
        for (int r = c + 1; r < 4; ++r)
            if (fabs(A[r][c]) > fabs(A[p][c])) p = r;
        for (int k = 0; k < 4; ++k) { double t = A[c][k]; A[c][k] = A[p][k]; A[p][k] = t; }
        { double t = b[c]; b[c] = b[p]; b[p] = t; }
        for (int r = c + 1; r < 4; ++r) {
            double f = A[r][c] / A[c][c];
            for (int k = c; k < 4; ++k) A[r][k] -= f * A[c][k];
            b[r] -= f * b[c];
        }
    }
    for (int c = 3; c >= 0; --c) {
        double s = b[c];
        for (int k = c + 1; k < 4; ++k) s -= A[c][k] * b[k];
        b[c] = s / A[c][c];
    }
}

int orc_triangle_rule_deg4(double *s, double *t, double *w)
{
    double a = 0.45, b = 0.1, W1 = 0.65, W2 = 0.35;
    for (int it = 0; it < 100; ++it) {
        double e2a = 2 * a - 3 * a * a, e2b = 2 * b - 3 * b * b;
        double e3a = a * a * (1 - 2 * a), e3b = b * b * (1 - 2 * b);
        double de2a = 2 - 6 * a, de2b = 2 - 6 * b;
        double de3a = 2 * a - 6 * a * a, de3b = 2 * b - 6 * b * b;
        double F[4] = {W1 + W2 - 1.0, W1 * e2a + W2 * e2b - 0.25,
                       W1 * e3a + W2 * e3b - 1.0 / 60.0,
                       W1 * e2a * e2a + W2 * e2b * e2b - 1.0 / 15.0};
        double J[4][4] = {{0, 0, 1, 1},
                          {W1 * de2a, W2 * de2b, e2a, e2b},
                          {W1 * de3a, W2 * de3b, e3a, e3b},
                          {W1 * 2 * e2a * de2a, W2 * 2 * e2b * de2b, e2a * e2a, e2b * e2b}};
        double d[4] = {-F[0], -F[1], -F[2], -F[3]};
        solve4(J, d);
        a += d[0]; b += d[1]; W1 += d[2]; W2 += d[3];
        if (fabs(d[0]) + fabs(d[1]) + fabs(d[2]) + fabs(d[3]) < 1e-17) break;
    }
    double orb[2] = {a, b}, ow[2] = {W1 / 3.0, W2 / 3.0};
    int k = 0;
    for (int o = 0; o < 2; ++o) {
        double q = orb[o], r = 1.0 - 2.0 * orb[o];
        /* barycentric (l0,l1,l2) -> (s,t) = (l1,l2) */
        double L[3][3] = {{q, q, r}, {q, r, q}, {r, q, q}};
        for (int m = 0; m < 3; ++m) {
            s[k] = L[m][1];
            t[k] = L[m][2];
            w[k] = ow[o];
            ++k;
        }
    }
    return 0;
}

/* Symmetric 3-point rule of degree 2 for the well-separated distance class
 * of admissible blocks (the lower of the per-class orders; the paper's own
 * rule is the 6-point one above).  One orbit (q,q,1-2q) with weights 1/3;
 * the moment of e2 (1/4) gives 3 q^2 - 2 q + 1/4 = 0, whose smaller root
 * q = 1/6 puts the points inside the triangle (the other, q = 1/2, at the
 * edge midpoints).  Output as for orc_triangle_rule_deg4. */
int orc_triangle_rule_deg2(double *s, double *t, double *w)
{
    const double a = 3.0, b = -2.0, c = 0.25;
    const double q = (-b - sqrt(b * b - 4.0 * a * c)) / (2.0 * a), r = 1.0 - 2.0 * q;
    const double L[3][3] = {{q, q, r}, {q, r, q}, {r, q, q}};
    for (int m = 0; m < 3; ++m) {
        s[m] = L[m][1];
        t[m] = L[m][2];
        w[m] = 1.0 / 3.0;
    }
    return 0;
}

/* Centroid rule (one point, degree 1) for the farthest distance class. */
int orc_triangle_rule_deg1(double *s, double *t, double *w)
{
    s[0] = t[0] = 1.0 / 3.0;
    w[0] = 1.0;
    return 0;
}

/* Conical (collapsed) product rule with n*n points: s = u, t = v (1-u),
 * Jacobian (1-u), Gauss-Legendre in u and v.  Weights normalised to sum 1.
 * Exact for total degree <= 2n-2.  Used only by the pins' reference
 * integrations and as an optional higher-order regular rule. */
int orc_triangle_rule_conical(int n, double *s, double *t, double *w)
{
    double x[128], g[128];
    if (orc_gauss_legendre01(n, x, g)) return 1;
    int k = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            s[k] = x[i];
            t[k] = x[j] * (1.0 - x[i]);
            w[k] = 2.0 * g[i] * g[j] * (1.0 - x[i]);
            ++k;
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Geometry and Green's function (Sec. 2, Eq. (1)-(3), Eq. (5))              */
/* ------------------------------------------------------------------------ */

typedef struct {
    double v[3][3];   /* vertices as stored */
    double n[3];      /* unit normal, right-hand rule on the stored order */
    double area;
} otri;

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static void tri_from_pts(const double *p0, const double *p1, const double *p2, otri *T)
{
    for (int c = 0; c < 3; ++c) {
        T->v[0][c] = p0[c];
        T->v[1][c] = p1[c];
        T->v[2][c] = p2[c];
    }
    double e1[3], e2[3], nn[3];
    for (int c = 0; c < 3; ++c) {
        e1[c] = T->v[1][c] - T->v[0][c];
        e2[c] = T->v[2][c] - T->v[0][c];
    }
    cross3(e1, e2, nn);
    double len = sqrt(dot3(nn, nn));
    T->area = 0.5 * len;
    for (int c = 0; c < 3; ++c) T->n[c] = nn[c] / len;
}

static void tri_load(const double *V, const int32_t *Tr, int64_t id, otri *T)
{
    const int32_t *t = Tr + 3 * id;
    tri_from_pts(V + 3 * (int64_t)t[0], V + 3 * (int64_t)t[1], V + 3 * (int64_t)t[2], T);
}

/* Kernel of the three operators at one point pair.
 * g(x,y) = exp(i k r) / (4 pi r), r = |x - y|            (Eq. (5))
 * SLP : g                                                  (Eq. (1))
 * DLP : dg/dn_y = exp(ikr)(ikr - 1) (y - x).n_y / (4 pi r^3)  (Eq. (2))
 * ADLP: dg/dn_x = exp(ikr)(ikr - 1) (x - y).n_x / (4 pi r^3)  (Eq. (3))
 * k = 0 gives the Laplace kernels. */
static cplx kernel(const double x[3], const double y[3], const double nx[3],
                   const double ny[3], int op, double k)
{
    double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
    double r = sqrt(dot3(d, d));
    cplx e = cexp(I * k * r);
    if (op == ORC_SLP) return e / (4.0 * M_PI * r);
    if (op == ORC_DLP) return e * (I * k * r - 1.0) * (-dot3(d, ny)) / (4.0 * M_PI * r * r * r);
    return e * (I * k * r - 1.0) * dot3(d, nx) / (4.0 * M_PI * r * r * r);
}

static void tri_point(const otri *T, double s, double t, double x[3])
{
    for (int c = 0; c < 3; ++c)
        x[c] = T->v[0][c] + s * (T->v[1][c] - T->v[0][c]) + t * (T->v[2][c] - T->v[0][c]);
}

/* ------------------------------------------------------------------------ */
/* Entries                                                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    int np;
    double s[16384], t[16384], w[16384];
} orule;

/* Regular pair: tensor Gauss rule, A_ij = |T_i||T_j| sum_p sum_q w_p w_q
 * G(x_p, y_q) with normalised weights (Sec. 3.2.3: standard Gauss triangle
 * rule for disjoint elements; Algorithm "Integral Evaluation", Sec. 3.3). */
static cplx entry_regular(const otri *Ti, const otri *Tj, int op, double k, const orule *R)
{
    cplx sum = 0;
    for (int p = 0; p < R->np; ++p) {
        double x[3];
        tri_point(Ti, R->s[p], R->t[p], x);
        for (int q = 0; q < R->np; ++q) {
            double y[3];
            tri_point(Tj, R->s[q], R->t[q], y);
            sum += R->w[p] * R->w[q] * kernel(x, y, Ti->n, Tj->n, op, k);
        }
    }
    return Ti->area * Tj->area * sum;
}

/* Sauter-Schwab maps of [0,1]^4 onto T^ x T^, T^ = {0 <= x2 <= x1 <= 1},
 * for identical (case 3), edge-adjacent (case 2) and vertex-adjacent
 * (case 1) panels (scheme of Erichsen and Sauter cited in Sec. 3.2.3).
 * Returns the Jacobian of region r at (xi, e1, e2, e3) and the two points.
 * Common edge: x2 = 0 in both parametrisations; common vertex: the origin. */
static int ss_nregions(int ncase) { return ncase == 3 ? 6 : (ncase == 2 ? 5 : 2); }

static double ss_map(int ncase, int r, double xi, double e1, double e2, double e3,
                     double xh[2], double yh[2])
{
    if (ncase == 3) {
        double J = xi * xi * xi * e1 * e1 * e2;
        switch (r) {
        case 0: xh[0] = xi; xh[1] = xi * (1 - e1 + e1 * e2);
                yh[0] = xi * (1 - e1 * e2 * e3); yh[1] = xi * (1 - e1); break;
        case 1: xh[0] = xi * (1 - e1 * e2 * e3); xh[1] = xi * (1 - e1);
                yh[0] = xi; yh[1] = xi * (1 - e1 + e1 * e2); break;
        case 2: xh[0] = xi; xh[1] = xi * e1 * (1 - e2 + e2 * e3);
                yh[0] = xi * (1 - e1 * e2); yh[1] = xi * e1 * (1 - e2); break;
        case 3: xh[0] = xi * (1 - e1 * e2); xh[1] = xi * e1 * (1 - e2);
                yh[0] = xi; yh[1] = xi * e1 * (1 - e2 + e2 * e3); break;
        case 4: xh[0] = xi * (1 - e1 * e2 * e3); xh[1] = xi * e1 * (1 - e2 * e3);
                yh[0] = xi; yh[1] = xi * e1 * (1 - e2); break;
        default: xh[0] = xi; xh[1] = xi * e1 * (1 - e2);
                 yh[0] = xi * (1 - e1 * e2 * e3); yh[1] = xi * e1 * (1 - e2 * e3); break;
        }
        return J;
    }
    if (ncase == 2) {
        double J1 = xi * xi * xi * e1 * e1, J = J1 * e2;
        switch (r) {
        case 0: xh[0] = xi; xh[1] = xi * e1 * e3;
                yh[0] = xi * (1 - e1 * e2); yh[1] = xi * e1 * (1 - e2); return J1;
        case 1: xh[0] = xi; xh[1] = xi * e1;
                yh[0] = xi * (1 - e1 * e2 * e3); yh[1] = xi * e1 * e2 * (1 - e3); return J;
        case 2: xh[0] = xi * (1 - e1 * e2); xh[1] = xi * e1 * (1 - e2);
                yh[0] = xi; yh[1] = xi * e1 * e2 * e3; return J;
        case 3: xh[0] = xi * (1 - e1 * e2 * e3); xh[1] = xi * e1 * e2 * (1 - e3);
                yh[0] = xi; yh[1] = xi * e1; return J;
        default: xh[0] = xi * (1 - e1 * e2 * e3); xh[1] = xi * e1 * (1 - e2 * e3);
                 yh[0] = xi; yh[1] = xi * e1 * e2; return J;
        }
    }
    {
        double J = xi * xi * xi * e2;
        if (r == 0) { xh[0] = xi; xh[1] = xi * e1; yh[0] = xi * e2; yh[1] = xi * e2 * e3; }
        else        { xh[0] = xi * e2; xh[1] = xi * e2 * e3; yh[0] = xi; yh[1] = xi * e1; }
        return J;
    }
}

/* Public hook for the coverage pin: integral over [0,1]^4 (n-point GL per
 * axis) of the sum over regions of J * x1^a x2^b y1^c y2^d. */
double orc_ss_moment(int ncase, int n, int a, int b, int c, int d)
{
    double x[128], g[128];
    orc_gauss_legendre01(n, x, g);
    double sum = 0;
    for (int r = 0; r < ss_nregions(ncase); ++r)
        for (int i0 = 0; i0 < n; ++i0)
            for (int i1 = 0; i1 < n; ++i1)
                for (int i2 = 0; i2 < n; ++i2)
                    for (int i3 = 0; i3 < n; ++i3) {
                        double xh[2], yh[2];
                        double J = ss_map(ncase, r, x[i0], x[i1], x[i2], x[i3], xh, yh);
                        sum += g[i0] * g[i1] * g[i2] * g[i3] * J * pow(xh[0], a) *
                               pow(xh[1], b) * pow(yh[0], c) * pow(yh[1], d);
                    }
    return sum;
}

/* Point of the panel parametrisation chi(x^) = P0 + x1 (P1 - P0) + x2 (P2 - P1)
 * which maps T^ onto the triangle (P0,P1,P2) with |det| = 2 |T|. */
static void chi(const double P[3][3], const double xh[2], double x[3])
{
    for (int c = 0; c < 3; ++c)
        x[c] = P[0][c] + xh[0] * (P[1][c] - P[0][c]) + xh[1] * (P[2][c] - P[1][c]);
}

/* Shared vertices of two triangles by vertex index. */
static int count_shared(const int32_t *a, const int32_t *b)
{
    int c = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (a[i] == b[j]) ++c;
    return c;
}

/* Vertex orderings for the singular parametrisations.
 *  identical: stored order for both panels;
 *  edge:      test P = (v[p], v[p+1], v[p+2]) with v[p], v[p+1] the shared
 *             vertices (cyclic indices); trial P0, P1 = the same two global
 *             vertices in the same order, P2 = its third vertex;
 *  vertex:    each panel starts at the shared vertex and continues
 *             cyclically in its stored order. */
static void singular_order(const int32_t *ta, const int32_t *tb, int ncase, int oa[3], int ob[3])
{
    if (ncase == 3) {
        for (int i = 0; i < 3; ++i) {
            oa[i] = i;
            for (int j = 0; j < 3; ++j)
                if (tb[j] == ta[i]) ob[i] = j;
        }
        return;
    }
    if (ncase == 2) {
        int p = 0;
        for (p = 0; p < 3; ++p) {
            int s0 = 0, s1 = 0;
            for (int j = 0; j < 3; ++j) {
                if (tb[j] == ta[p]) s0 = 1;
                if (tb[j] == ta[(p + 1) % 3]) s1 = 1;
            }
            if (s0 && s1) break;
        }
        oa[0] = p; oa[1] = (p + 1) % 3; oa[2] = (p + 2) % 3;
        for (int j = 0; j < 3; ++j) {
            if (tb[j] == ta[oa[0]]) ob[0] = j;
            else if (tb[j] == ta[oa[1]]) ob[1] = j;
            else ob[2] = j;
        }
        return;
    }
    {
        int p = 0, q = 0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                if (ta[i] == tb[j]) { p = i; q = j; }
        for (int i = 0; i < 3; ++i) { oa[i] = (p + i) % 3; ob[i] = (q + i) % 3; }
    }
}

/* Singular pair by the Sauter-Schwab transformations with n GL points per
 * axis of [0,1]^4:  A_ij = (2|T_i|)(2|T_j|) sum_regions sum_nodes w J
 * G(chi_i(x^), chi_j(y^)).  The normals stay those of the stored vertex
 * order (Sec. 3.2.3: coincident, edge- and vertex-adjacent pairs). */
static cplx entry_singular(const otri *Ti, const otri *Tj, const int32_t *ta, const int32_t *tb,
                           int ncase, int op, double k, int n)
{
    int oa[3], ob[3];
    singular_order(ta, tb, ncase, oa, ob);
    double Pa[3][3], Pb[3][3];
    for (int i = 0; i < 3; ++i)
        for (int c = 0; c < 3; ++c) {
            Pa[i][c] = Ti->v[oa[i]][c];
            Pb[i][c] = Tj->v[ob[i]][c];
        }
    double x[128], g[128];
    orc_gauss_legendre01(n, x, g);
    cplx sum = 0;
    for (int r = 0; r < ss_nregions(ncase); ++r)
        for (int i0 = 0; i0 < n; ++i0)
            for (int i1 = 0; i1 < n; ++i1)
                for (int i2 = 0; i2 < n; ++i2)
                    for (int i3 = 0; i3 < n; ++i3) {
                        double xh[2], yh[2], px[3], py[3];
                        double J = ss_map(ncase, r, x[i0], x[i1], x[i2], x[i3], xh, yh);
                        chi(Pa, xh, px);
                        chi(Pb, yh, py);
                        sum += g[i0] * g[i1] * g[i2] * g[i3] * J *
                               kernel(px, py, Ti->n, Tj->n, op, k);
                    }
    return 4.0 * Ti->area * Tj->area * sum;
}

/* Regular rule by code: 0 (or any other value <= 0) the 6-point degree-4
 * rule, -3 the 3-point degree-2 rule, -1 the centroid rule, n > 0 the
 * conical n x n rule. */
static void rule_init(orule *R, int regular_order)
{
    if (regular_order == -3) {
        R->np = 3;
        orc_triangle_rule_deg2(R->s, R->t, R->w);
    } else if (regular_order == -1) {
        R->np = 1;
        orc_triangle_rule_deg1(R->s, R->t, R->w);
    } else if (regular_order <= 0) {
        R->np = 6;
        orc_triangle_rule_deg4(R->s, R->t, R->w);
    } else {
        R->np = regular_order * regular_order;
        orc_triangle_rule_conical(regular_order, R->s, R->t, R->w);
    }
}

/* One Galerkin P0 entry of operator op (Eq. (1)-(3)) for test triangle i
 * and trial triangle j: regular pairs by the tensor Gauss rule, pairs with a
 * shared vertex by Sauter-Schwab (Sec. 3.2.3). */
static cplx entry_ij(const double *V, const int32_t *Tr, int64_t i, int64_t j, int op, double k,
                     int n_gl, const orule *R)
{
    otri Ti, Tj;
    tri_load(V, Tr, i, &Ti);
    tri_load(V, Tr, j, &Tj);
    int c = count_shared(Tr + 3 * i, Tr + 3 * j);
    if (c == 0) return entry_regular(&Ti, &Tj, op, k, R);
    return entry_singular(&Ti, &Tj, Tr + 3 * i, Tr + 3 * j, c, op, k, n_gl);
}

/* Dense sub-block out[a][b] = A(test_ids[a], trial_ids[b]) (row-major,
 * complex128).  regular_order <= 0 selects the 6-point degree-4 rule. */
int orc_entries(const double *V, const int32_t *Tr, int64_t nt, int op, double k,
                const int32_t *test_ids, int64_t n_test, const int32_t *trial_ids, int64_t n_trial,
                int n_gl, int regular_order, cplx *out, int nthreads)
{
    (void)nt;
    orule *R = (orule *)malloc(sizeof(orule));
    if (!R) return 3;
    rule_init(R, regular_order);
#ifdef _OPENMP
    /* a per-call thread count that leaves the process default untouched */
    const int nth = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nth)
#endif
    for (int64_t a = 0; a < n_test; ++a)
        for (int64_t b = 0; b < n_trial; ++b)
            out[a * n_trial + b] = entry_ij(V, Tr, test_ids[a], trial_ids[b], op, k, n_gl, R);
    free(R);
    return 0;
}

/* Entry of an explicit triangle pair given by coordinates (for pins on
 * pairs that are not part of a mesh).  shared: vertex-index triples used
 * only to classify the pair and order the singular parametrisation. */
int orc_pair_entry(const double *a9, const double *b9, const int32_t *ia, const int32_t *ib,
                   int op, double k, int n_gl, int regular_order, double *re, double *im)
{
    otri Ti, Tj;
    tri_from_pts(a9, a9 + 3, a9 + 6, &Ti);
    tri_from_pts(b9, b9 + 3, b9 + 6, &Tj);
    orule *R = (orule *)malloc(sizeof(orule));
    if (!R) return 3;
    rule_init(R, regular_order);
    int c = count_shared(ia, ib);
    cplx v = c == 0 ? entry_regular(&Ti, &Tj, op, k, R)
                    : entry_singular(&Ti, &Tj, ia, ib, c, op, k, n_gl);
    free(R);
    *re = creal(v);
    *im = cimag(v);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Piecewise linear spaces                                                   */
/* ------------------------------------------------------------------------ */

/* Local 3 x 3 matrix of an element pair for piecewise linear test and trial
 * functions (Sec. 3.3, Algorithm "Integral Evaluation": the kernel values of
 * all quadrature point pairs are combined with the basis function values of
 * every pair of local dofs).  The local basis functions of a triangle are
 * its barycentric coordinates lambda_a, a = stored vertex index; at the
 * point x = v0 + s (v1 - v0) + t (v2 - v0):  lambda = (1 - s - t, s, t).
 *   L[a][b] = int_Ti int_Tj lambda_a(x) G(x, y) lambda_b(y) dy dx.
 * Regular pairs by the tensor Gauss rule. */
static void local_regular(const otri *Ti, const otri *Tj, int op, double k, const orule *R,
                          cplx L[3][3])
{
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) L[a][b] = 0;
    for (int p = 0; p < R->np; ++p) {
        double x[3];
        tri_point(Ti, R->s[p], R->t[p], x);
        double la[3] = {1.0 - R->s[p] - R->t[p], R->s[p], R->t[p]};
        for (int q = 0; q < R->np; ++q) {
            double y[3];
            tri_point(Tj, R->s[q], R->t[q], y);
            double lb[3] = {1.0 - R->s[q] - R->t[q], R->s[q], R->t[q]};
            cplx g = R->w[p] * R->w[q] * kernel(x, y, Ti->n, Tj->n, op, k);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) L[a][b] += la[a] * lb[b] * g;
        }
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) L[a][b] *= Ti->area * Tj->area;
}

/* Singular pairs by the same Sauter-Schwab maps as entry_singular.  With the
 * panel parametrisation chi(x^) = P0 + x1 (P1 - P0) + x2 (P2 - P1), the
 * barycentric coordinates of the point with respect to (P0, P1, P2) are
 * (1 - x1, x1 - x2, x2); P_i is stored vertex o[i], so lambda_{o[i]} takes
 * the i-th of them. */
static void local_singular(const otri *Ti, const otri *Tj, const int32_t *ta, const int32_t *tb,
                           int ncase, int op, double k, int n, cplx L[3][3])
{
    int oa[3], ob[3];
    singular_order(ta, tb, ncase, oa, ob);
    double Pa[3][3], Pb[3][3];
    for (int i = 0; i < 3; ++i)
        for (int c = 0; c < 3; ++c) {
            Pa[i][c] = Ti->v[oa[i]][c];
            Pb[i][c] = Tj->v[ob[i]][c];
        }
    double x[128], g[128];
    orc_gauss_legendre01(n, x, g);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) L[a][b] = 0;
    for (int r = 0; r < ss_nregions(ncase); ++r)
        for (int i0 = 0; i0 < n; ++i0)
            for (int i1 = 0; i1 < n; ++i1)
                for (int i2 = 0; i2 < n; ++i2)
                    for (int i3 = 0; i3 < n; ++i3) {
                        double xh[2], yh[2], px[3], py[3];
                        double J = ss_map(ncase, r, x[i0], x[i1], x[i2], x[i3], xh, yh);
                        chi(Pa, xh, px);
                        chi(Pb, yh, py);
                        cplx gv = g[i0] * g[i1] * g[i2] * g[i3] * J *
                                  kernel(px, py, Ti->n, Tj->n, op, k);
                        double ba[3] = {1.0 - xh[0], xh[0] - xh[1], xh[1]};
                        double bb[3] = {1.0 - yh[0], yh[0] - yh[1], yh[1]};
                        double la[3], lb[3];
                        for (int i = 0; i < 3; ++i) {
                            la[oa[i]] = ba[i];
                            lb[ob[i]] = bb[i];
                        }
                        for (int a = 0; a < 3; ++a)
                            for (int b = 0; b < 3; ++b) L[a][b] += la[a] * lb[b] * gv;
                    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) L[a][b] *= 4.0 * Ti->area * Tj->area;
}

static void local_ij(const double *V, const int32_t *Tr, int64_t i, int64_t j, int op, double k,
                     int n_gl, const orule *R, cplx L[3][3])
{
    otri Ti, Tj;
    tri_load(V, Tr, i, &Ti);
    tri_load(V, Tr, j, &Tj);
    int c = count_shared(Tr + 3 * i, Tr + 3 * j);
    if (c == 0) local_regular(&Ti, &Tj, op, k, R, L);
    else local_singular(&Ti, &Tj, Tr + 3 * i, Tr + 3 * j, c, op, k, n_gl, L);
}

/* Discontinuous piecewise linear (DP1) entry: dof 3 t + a is lambda_a on
 * triangle t, so every entry belongs to exactly one element pair. */
static cplx entry_dp1(const double *V, const int32_t *Tr, int64_t di, int64_t dj, int op,
                      double k, int n_gl, const orule *R)
{
    cplx L[3][3];
    local_ij(V, Tr, di / 3, dj / 3, op, k, n_gl, R, L);
    return L[di % 3][dj % 3];
}

/* DP1 sub-block for triangle lists: out[3 a + alpha][3 b + beta] (row-major,
 * 3 n_test x 3 n_trial, complex128) = L(test[a], trial[b])[alpha][beta]. */
int orc_entries_dp1(const double *V, const int32_t *Tr, int64_t nt, int op, double k,
                    const int32_t *test_ids, int64_t n_test, const int32_t *trial_ids,
                    int64_t n_trial, int n_gl, int regular_order, cplx *out, int nthreads)
{
    (void)nt;
    orule *R = (orule *)malloc(sizeof(orule));
    if (!R) return 3;
    rule_init(R, regular_order);
    const int64_t ld = 3 * n_trial;
#ifdef _OPENMP
    /* a per-call thread count that leaves the process default untouched */
    const int nth = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nth)
#endif
    for (int64_t a = 0; a < n_test; ++a)
        for (int64_t b = 0; b < n_trial; ++b) {
            cplx L[3][3];
            local_ij(V, Tr, test_ids[a], trial_ids[b], op, k, n_gl, R, L);
            for (int al = 0; al < 3; ++al)
                for (int be = 0; be < 3; ++be) out[(3 * a + al) * ld + 3 * b + be] = L[al][be];
        }
    free(R);
    return 0;
}

/* Local matrix of an explicit triangle pair (coordinates + vertex-index
 * triples that classify it), for the pins. */
int orc_pair_local(const double *a9, const double *b9, const int32_t *ia, const int32_t *ib, int op,
                   double k, int n_gl, int regular_order, cplx *out9)
{
    otri Ti, Tj;
    tri_from_pts(a9, a9 + 3, a9 + 6, &Ti);
    tri_from_pts(b9, b9 + 3, b9 + 6, &Tj);
    orule *R = (orule *)malloc(sizeof(orule));
    if (!R) return 3;
    rule_init(R, regular_order);
    int c = count_shared(ia, ib);
    cplx L[3][3];
    if (c == 0) local_regular(&Ti, &Tj, op, k, R, L);
    else local_singular(&Ti, &Tj, ia, ib, c, op, k, n_gl, L);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) out9[3 * a + b] = L[a][b];
    free(R);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Closed forms used by the pins (not by the entry path above)               */
/* ------------------------------------------------------------------------ */

/* Potential of a flat triangle with unit density, Phi(x) = int_T 1/|x-y| dS_y.
 * With h the signed height of x over the plane and rho its projection, the
 * planar field F(y) = (y - rho)(sqrt(s^2+h^2) - |h|)/s^2, s = |y - rho|, has
 * divergence 1/|x-y| in the plane, so Phi is the flux of F through the three
 * edges.  On edge e with outward in-plane normal nu_e, (y-rho).nu_e = P_e is
 * constant, and with l the coordinate along the edge, R0^2 = P_e^2 + h^2,
 * R = sqrt(R0^2 + l^2):
 *   int_e P_e (R - |h|)/(P_e^2 + l^2) dl
 *     = P_e ln((R+ + l+)/(R- + l-)) - |h| [atan(P_e l/(R0^2 + |h| R))]_{l-}^{l+}. */
static double log_ratio(double Rp, double lp, double Rm, double lm, double R0sq)
{
    /* ln((Rp + lp)/(Rm + lm)) with R + l = R0^2/(R - l) for l < 0 */
    double np = lp >= 0 ? Rp + lp : R0sq / (Rp - lp);
    double nm = lm >= 0 ? Rm + lm : R0sq / (Rm - lm);
    return log(np / nm);
}

double orc_triangle_potential(const double *tri9, const double *x)
{
    otri T;
    tri_from_pts(tri9, tri9 + 3, tri9 + 6, &T);
    double h = (x[0] - T.v[0][0]) * T.n[0] + (x[1] - T.v[0][1]) * T.n[1] + (x[2] - T.v[0][2]) * T.n[2];
    double ah = fabs(h);
    double rho[3] = {x[0] - h * T.n[0], x[1] - h * T.n[1], x[2] - h * T.n[2]};
    double total = 0;
    for (int e = 0; e < 3; ++e) {
        const double *a = T.v[e], *b = T.v[(e + 1) % 3];
        double tv[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        double len = sqrt(dot3(tv, tv));
        for (int c = 0; c < 3; ++c) tv[c] /= len;
        double nu[3];
        cross3(tv, T.n, nu); /* outward for counter-clockwise order about n */
        double am[3] = {a[0] - rho[0], a[1] - rho[1], a[2] - rho[2]};
        double bm[3] = {b[0] - rho[0], b[1] - rho[1], b[2] - rho[2]};
        double P = dot3(am, nu);
        double lm = dot3(am, tv), lp = dot3(bm, tv);
        if (fabs(P) < 1e-300) continue;
        double R0sq = P * P + h * h;
        double Rm = sqrt(R0sq + lm * lm), Rp = sqrt(R0sq + lp * lp);
        total += P * log_ratio(Rp, lp, Rm, lm, R0sq);
        if (ah > 0)
            total -= ah * (atan(P * lp / (R0sq + ah * Rp)) - atan(P * lm / (R0sq + ah * Rm)));
    }
    return total;
}

/* Signed solid angle int_T (x - y).n_y / |x - y|^3 dS_y of a flat triangle
 * seen from x (van Oosterom-Strackee):  with R_a = v_a - x,
 * tan(Omega/2) = R1.(R2 x R3) / (|R1||R2||R3| + (R1.R2)|R3| + (R1.R3)|R2|
 * + (R2.R3)|R1|), and the integral equals -Omega for the right-hand normal. */
double orc_triangle_solid_angle(const double *tri9, const double *x)
{
    double R[3][3], L[3];
    for (int a = 0; a < 3; ++a) {
        for (int c = 0; c < 3; ++c) R[a][c] = tri9[3 * a + c] - x[c];
        L[a] = sqrt(dot3(R[a], R[a]));
    }
    double cr[3];
    cross3(R[1], R[2], cr);
    double num = dot3(R[0], cr);
    double den = L[0] * L[1] * L[2] + dot3(R[0], R[1]) * L[2] + dot3(R[0], R[2]) * L[1] +
                 dot3(R[1], R[2]) * L[0];
    return -2.0 * atan2(num, den);
}

/* Adaptive integration of an outer function over a triangle: compare the
 * conical rule on the triangle with the sum over its four midpoint children
 * and recurse where they differ by more than tol. */
typedef cplx (*outer_fn)(const double x[3], void *ctx);

typedef struct {
    orule R;
} adapt_rule;

static cplx rule_on(const double a[3], const double b[3], const double c[3], outer_fn f, void *ctx,
                    const orule *R)
{
    otri T;
    tri_from_pts(a, b, c, &T);
    cplx s = 0;
    for (int p = 0; p < R->np; ++p) {
        double x[3];
        tri_point(&T, R->s[p], R->t[p], x);
        s += R->w[p] * f(x, ctx);
    }
    return T.area * s;
}

static cplx adapt_tri(const double a[3], const double b[3], const double c[3], outer_fn f, void *ctx,
                      const orule *R, double tol, int depth, int maxdepth, cplx whole)
{
    double ab[3], bc[3], ca[3];
    for (int i = 0; i < 3; ++i) {
        ab[i] = 0.5 * (a[i] + b[i]);
        bc[i] = 0.5 * (b[i] + c[i]);
        ca[i] = 0.5 * (c[i] + a[i]);
    }
    cplx c0 = rule_on(a, ab, ca, f, ctx, R), c1 = rule_on(ab, b, bc, f, ctx, R);
    cplx c2 = rule_on(ca, bc, c, f, ctx, R), c3 = rule_on(ab, bc, ca, f, ctx, R);
    cplx parts = c0 + c1 + c2 + c3;
    if (cabs(parts - whole) <= tol || depth >= maxdepth) return parts;
    double t4 = 0.25 * tol;
    return adapt_tri(a, ab, ca, f, ctx, R, t4, depth + 1, maxdepth, c0) +
           adapt_tri(ab, b, bc, f, ctx, R, t4, depth + 1, maxdepth, c1) +
           adapt_tri(ca, bc, c, f, ctx, R, t4, depth + 1, maxdepth, c2) +
           adapt_tri(ab, bc, ca, f, ctx, R, t4, depth + 1, maxdepth, c3);
}

static cplx adapt_integrate(const otri *T, outer_fn f, void *ctx, const orule *R, double tol,
                            int maxdepth)
{
    cplx whole = rule_on(T->v[0], T->v[1], T->v[2], f, ctx, R);
    return adapt_tri(T->v[0], T->v[1], T->v[2], f, ctx, R, tol, 0, maxdepth, whole);
}

typedef struct {
    const otri *Tj;
    const otri *Ti;
    int op;
    double k;
    const orule *R;
    double tol;
    int maxdepth;
    const double *xo; /* current outer point */
} ctx_t;

/* Laplace inner integrals in closed form (Eq. (1)-(2), k = 0). */
static cplx inner_laplace(const double x[3], void *vctx)
{
    ctx_t *c = (ctx_t *)vctx;
    double tri9[9];
    for (int a = 0; a < 3; ++a)
        for (int d = 0; d < 3; ++d) tri9[3 * a + d] = c->Tj->v[a][d];
    if (c->op == ORC_SLP) return orc_triangle_potential(tri9, x) / (4.0 * M_PI);
    return orc_triangle_solid_angle(tri9, x) / (4.0 * M_PI);
}

/* Bounded remainder of the Helmholtz kernels, G_k - G_0. */
static cplx remainder_kernel(const double x[3], const double y[3], const double nx[3],
                             const double ny[3], int op, double k)
{
    double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
    double r = sqrt(dot3(d, d));
    if (op == ORC_SLP) {
        if (r == 0) return I * k / (4.0 * M_PI);
        return (cexp(I * k * r) - 1.0) / (4.0 * M_PI * r);
    }
    /* (exp(ikr)(ikr-1) + 1) (y-x).n_y / (4 pi r^3) */
    if (r == 0) return 0;
    cplx f = cexp(I * k * r) * (I * k * r - 1.0) + 1.0;
    double proj = op == ORC_DLP ? -dot3(d, ny) : dot3(d, nx);
    return f * proj / (4.0 * M_PI * r * r * r);
}

static cplx inner_remainder_pt(const double y[3], void *vctx)
{
    ctx_t *c = (ctx_t *)vctx;
    return remainder_kernel(c->xo, y, c->Ti->n, c->Tj->n, c->op, c->k);
}

static cplx outer_remainder(const double x[3], void *vctx)
{
    ctx_t *c = (ctx_t *)vctx;
    ctx_t in = *c;
    in.xo = x;
    return adapt_integrate(c->Tj, inner_remainder_pt, &in, c->R, c->tol, c->maxdepth);
}

/* Reference value of an entry for the pins, independent of the Gauss and
 * Sauter-Schwab rules: outer integral by adaptive subdivision of T_i, inner
 * integral of the Laplace part in closed form (potential or solid angle)
 * and, for k != 0, plus the nested adaptive integral of the bounded
 * remainder G_k - G_0.  op: SLP or DLP.  tol: absolute tolerance per level. */
int orc_reference_entry(const double *a9, const double *b9, int op, double k, int order,
                        double tol, int maxdepth, double *re, double *im)
{
    if (op != ORC_SLP && op != ORC_DLP) return 1;
    otri Ti, Tj;
    tri_from_pts(a9, a9 + 3, a9 + 6, &Ti);
    tri_from_pts(b9, b9 + 3, b9 + 6, &Tj);
    orule *R = (orule *)malloc(sizeof(orule));
    if (!R) return 3;
    rule_init(R, order);
    ctx_t c = {&Tj, &Ti, op, k, R, tol, maxdepth, NULL};
    cplx v = adapt_integrate(&Ti, inner_laplace, &c, R, tol, maxdepth);
    if (k != 0.0) {
        ctx_t c2 = c;
        c2.tol = tol / (Ti.area > 0 ? Ti.area : 1.0);
        v += adapt_integrate(&Ti, outer_remainder, &c2, R, tol, maxdepth);
    }
    free(R);
    *re = creal(v);
    *im = cimag(v);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Cluster tree and block cluster tree (Sec. 2.1; Algorithm "H-Matrix        */
/* Assembly", Sec. 4.1: "generate block cluster tree")                       */
/* ------------------------------------------------------------------------ */

/* Readings where the paper is silent:
 *  - a cluster is a contiguous range of the permutation; its bounding box is
 *    the box of its triangles' vertices;
 *  - a cluster with more than leaf_size triangles is split along the
 *    longest box axis (lowest axis on ties) at the median of the triangle
 *    centroids ((v0 + v1) + v2) / 3, ties broken by triangle index; the
 *    first floor(n/2) triangles form the left child;
 *  - inside a leaf the triangles are in increasing index order, so the
 *    permutation depends only on the cluster sets. */
static const double *g_cent; /* centroid coordinate array for qsort */
static int g_axis;

static int cmp_centroid(const void *pa, const void *pb)
{
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    double ca = g_cent[3 * (int64_t)a + g_axis], cb = g_cent[3 * (int64_t)b + g_axis];
    if (ca < cb) return -1;
    if (ca > cb) return 1;
    return (a > b) - (a < b);
}

static int cmp_index(const void *pa, const void *pb)
{
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    return (a > b) - (a < b);
}

static void cluster_bbox(const double *V, const int32_t *Tr, const int32_t *perm, int64_t b,
                         int64_t e, double *box)
{
    for (int c = 0; c < 3; ++c) { box[c] = INFINITY; box[3 + c] = -INFINITY; }
    for (int64_t q = b; q < e; ++q)
        for (int a = 0; a < 3; ++a) {
            const double *p = V + 3 * (int64_t)Tr[3 * (int64_t)perm[q] + a];
            for (int c = 0; c < 3; ++c) {
                if (p[c] < box[c]) box[c] = p[c];
                if (p[c] > box[3 + c]) box[3 + c] = p[c];
            }
        }
}

/* Builds the tree breadth-first; cluster 0 is the root.  Arrays sized
 * 2*nt.  Returns the number of clusters in *n_clusters. */
int orc_cluster_tree(const double *V, const int32_t *Tr, int64_t nt, int leaf_size,
                     int32_t *perm, int64_t *cl_begin, int64_t *cl_end, int64_t *cl_left,
                     int64_t *cl_right, double *cl_box, int64_t *n_clusters)
{
    if (leaf_size < 1 || nt < 1) return 1;
    double *cent = (double *)malloc(sizeof(double) * 3 * nt);
    if (!cent) return 3;
    for (int64_t t = 0; t < nt; ++t)
        for (int c = 0; c < 3; ++c) {
            const int32_t *tr = Tr + 3 * t;
            cent[3 * t + c] = ((V[3 * (int64_t)tr[0] + c] + V[3 * (int64_t)tr[1] + c]) +
                               V[3 * (int64_t)tr[2] + c]) / 3.0;
        }
    for (int64_t t = 0; t < nt; ++t) perm[t] = (int32_t)t;
    int64_t nc = 1, head = 0;
    cl_begin[0] = 0;
    cl_end[0] = nt;
    while (head < nc) {
        int64_t c = head++;
        int64_t b = cl_begin[c], e = cl_end[c], n = e - b;
        cluster_bbox(V, Tr, perm, b, e, cl_box + 6 * c);
        cl_left[c] = cl_right[c] = -1;
        if (n <= leaf_size) {
            /* leaf: its triangles in increasing index order */
            qsort(perm + b, (size_t)n, sizeof(int32_t), cmp_index);
            continue;
        }
        double *box = cl_box + 6 * c;
        int axis = 0;
        double ext = box[3] - box[0];
        for (int a = 1; a < 3; ++a)
            if (box[3 + a] - box[a] > ext) { ext = box[3 + a] - box[a]; axis = a; }
        g_cent = cent;
        g_axis = axis;
        qsort(perm + b, (size_t)n, sizeof(int32_t), cmp_centroid);
        int64_t mid = b + n / 2;
        cl_left[c] = nc;
        cl_begin[nc] = b; cl_end[nc] = mid; ++nc;
        cl_right[c] = nc;
        cl_begin[nc] = mid; cl_end[nc] = e; ++nc;
    }
    *n_clusters = nc;
    free(cent);
    return 0;
}

/* Admissibility (Sec. 2.1: "distance and block diameter dependent"):
 * min(diam tau, diam sigma) <= eta * dist(tau, sigma) with diam the box
 * diagonal and dist the distance between boxes; boxes that touch or overlap
 * are never admissible. */
static int admissible(const double *bt, const double *bs, double eta)
{
    double dt = sqrt((bt[3] - bt[0]) * (bt[3] - bt[0]) + (bt[4] - bt[1]) * (bt[4] - bt[1]) +
                     (bt[5] - bt[2]) * (bt[5] - bt[2]));
    double ds = sqrt((bs[3] - bs[0]) * (bs[3] - bs[0]) + (bs[4] - bs[1]) * (bs[4] - bs[1]) +
                     (bs[5] - bs[2]) * (bs[5] - bs[2]));
    double g[3];
    for (int c = 0; c < 3; ++c) {
        double g1 = bs[c] - bt[3 + c], g2 = bt[c] - bs[3 + c];
        double m = g1 > g2 ? g1 : g2;
        g[c] = m > 0 ? m : 0;
    }
    double dist = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (!(dist > 0)) return 0;
    double dmin = dt < ds ? dt : ds;
    return dmin <= eta * dist;
}

/* Block cluster tree from (root, root): an admissible pair is a far leaf;
 * otherwise a pair with a leaf cluster is a near (dense) leaf; otherwise
 * all four child pairs are visited.  Output: leaf blocks (tau, sigma,
 * admissible flag) in depth-first order.  Returns 2 if cap is too small. */
static int64_t g_nb;

static int block_rec(int64_t t, int64_t s, const int64_t *cl_left, const int64_t *cl_right,
                     const double *box, double eta, int64_t *bt, int64_t *bs, int8_t *badm,
                     int64_t cap)
{
    if (admissible(box + 6 * t, box + 6 * s, eta) || cl_left[t] < 0 || cl_left[s] < 0) {
        if (g_nb >= cap) return 2;
        bt[g_nb] = t;
        bs[g_nb] = s;
        badm[g_nb] = (int8_t)admissible(box + 6 * t, box + 6 * s, eta);
        ++g_nb;
        return 0;
    }
    int64_t ct[2] = {cl_left[t], cl_right[t]}, cs[2] = {cl_left[s], cl_right[s]};
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            int r = block_rec(ct[a], cs[b], cl_left, cl_right, box, eta, bt, bs, badm, cap);
            if (r) return r;
        }
    return 0;
}

int orc_block_tree(const int64_t *cl_left, const int64_t *cl_right, const double *cl_box,
                   double eta, int64_t *blk_tau, int64_t *blk_sigma, int8_t *blk_adm, int64_t cap,
                   int64_t *n_blocks)
{
    g_nb = 0;
    int r = block_rec(0, 0, cl_left, cl_right, cl_box, eta, blk_tau, blk_sigma, blk_adm, cap);
    *n_blocks = g_nb;
    return r;
}

/* ------------------------------------------------------------------------ */
/* ACA with partial pivoting (Sec. 2.1, Eq. (6)-(7), Algorithm ACA)          */
/* ------------------------------------------------------------------------ */

/* Entry (r, c) of a block in cluster order.  P0: dof = triangle.  DP1: the
 * dofs of the triangle at cluster position t are 3 t, 3 t + 1, 3 t + 2 (its
 * local basis functions), so a block of triangle ranges is the block of the
 * tripled dof ranges. */
static cplx block_entry(const double *V, const int32_t *Tr, const int32_t *perm, int space,
                        int64_t r, int64_t c, int op, double k, const orule *R)
{
    if (space == 0) return entry_ij(V, Tr, perm[r], perm[c], op, k, 4, R);
    return entry_dp1(V, Tr, 3 * (int64_t)perm[r / 3] + r % 3, 3 * (int64_t)perm[c / 3] + c % 3, op,
                     k, 4, R);
}

/* Regular-rule class of an admissible block (quadrature order per block
 * distance class): rho = dist(tau, sigma) / h, with dist the distance between
 * the cluster boxes (as in the admissibility test) and h the longest edge of
 * any triangle of tau or sigma.  rho >= rho1 > 0 selects the centroid rule
 * (code -1), else rho >= rho3 > 0 the 3-point rule (code -3), else the
 * 6-point rule (code 0).  Boxes: 6 doubles (lo xyz, hi xyz) per block and
 * side; ranges in cluster order through perm. */
static double longest_edge(const double *V, const int32_t *Tr, const int32_t *perm, int64_t b,
                           int64_t e)
{
    double h2 = 0.0;
    for (int64_t p = b; p < e; ++p) {
        const int32_t *tr = Tr + 3 * (int64_t)perm[p];
        for (int a = 0; a < 3; ++a) {
            const double *u = V + 3 * (int64_t)tr[a], *v = V + 3 * (int64_t)tr[(a + 1) % 3];
            double l2 = 0.0;
            for (int c = 0; c < 3; ++c) l2 += (u[c] - v[c]) * (u[c] - v[c]);
            if (l2 > h2) h2 = l2;
        }
    }
    return sqrt(h2);
}

int orc_block_rules(const double *V, const int32_t *Tr, const int32_t *perm, int64_t nblk,
                    const int64_t *tb, const int64_t *te, const int64_t *sb, const int64_t *se,
                    const double *box_t, const double *box_s, double rho3, double rho1,
                    int32_t *rules)
{
    for (int64_t b = 0; b < nblk; ++b) {
        const double *bt = box_t + 6 * b, *bs = box_s + 6 * b;
        double g2 = 0.0;
        for (int c = 0; c < 3; ++c) {
            double g1 = bs[c] - bt[3 + c], gb = bt[c] - bs[3 + c];
            double m = g1 > gb ? g1 : gb;
            if (m > 0) g2 += m * m;
        }
        const double dist = sqrt(g2);
        const double ht = longest_edge(V, Tr, perm, tb[b], te[b]);
        const double hs = longest_edge(V, Tr, perm, sb[b], se[b]);
        const double h = ht > hs ? ht : hs;
        int r = 0;
        if (rho1 > 0 && dist >= rho1 * h) r = -1;
        else if (rho3 > 0 && dist >= rho3 * h) r = -3;
        rules[b] = r;
    }
    return 0;
}

/* Readings where the paper defers or is silent:
 *  row pivot:  i_1 = 0; afterwards i_{k+1} = argmax_{i not in Z} |(u_k)_i|,
 *              lowest index on ties;
 *  vanishing:  max|v~_k| == 0 or <= 1e-14 * (largest |pivot| so far); then
 *              the next row is the smallest index not in Z;
 *  stopping:   after accepting step k, stop if ||u_k|| ||v_k|| <= eps ||S_k||_F
 *              with ||S_k||_F^2 = ||S_{k-1}||_F^2
 *                 + 2 Re sum_{l<k} <u_k,u_l><v_k,v_l> + ||u_k||^2 ||v_k||^2,
 *              or when k = min(m, n), or when Z holds all m rows.
 * Block rows are the test cluster, columns the trial cluster, as dof ranges
 * in cluster order of the space (block_entry).
 * U is m x kcap column-major, V is n x kcap column-major.  *rank = k.
 * Returns 0, or 4 if kcap was reached before the criterion held. */
int orc_aca_block(const double *V, const int32_t *Tr, const int32_t *perm, int space, int64_t tb,
                  int64_t te, int64_t sb, int64_t se, int op, double k, double eps, int kcap,
                  int regular_order, cplx *U, cplx *Vf, int *rank, int64_t *entries_evaluated)
{
    int64_t m = te - tb, n = se - sb;
    orule *R = (orule *)malloc(sizeof(orule));
    cplx *row = (cplx *)malloc(sizeof(cplx) * n);
    cplx *col = (cplx *)malloc(sizeof(cplx) * m);
    char *inZ = (char *)calloc((size_t)m, 1);
    if (!R || !row || !col || !inZ) { free(R); free(row); free(col); free(inZ); return 3; }
    rule_init(R, regular_order);
    int kk = 0, status = 0;
    int64_t nZ = 0, i = 0, evals = 0;
    double normS2 = 0, maxpiv = 0;
    int64_t kmin = m < n ? m : n;
    for (;;) {
        /* selected row of R_{k-1}: a_{i,:} - sum_l (u_l)_i v_l */
        for (int64_t j = 0; j < n; ++j) {
            cplx a = block_entry(V, Tr, perm, space, tb + i, sb + j, op, k, R);
            for (int l = 0; l < kk; ++l) a -= U[(int64_t)l * m + i] * Vf[(int64_t)l * n + j];
            row[j] = a;
        }
        evals += n;
        inZ[i] = 1;
        ++nZ;
        int64_t jk = 0;
        double vmax = -1.0;
        for (int64_t j = 0; j < n; ++j)
            if (cabs(row[j]) > vmax) { vmax = cabs(row[j]); jk = j; }
        if (vmax == 0.0 || vmax <= 1e-14 * maxpiv) {
            if (nZ == m) break;
            for (i = 0; i < m && inZ[i]; ++i) {}
            continue;
        }
        if (kk == kcap) { status = 4; break; }
        if (vmax > maxpiv) maxpiv = vmax;
        cplx piv = row[jk];
        cplx *vk = Vf + (int64_t)kk * n, *uk = U + (int64_t)kk * m;
        for (int64_t j = 0; j < n; ++j) vk[j] = row[j] / piv;
        /* selected column of R_{k-1}: a_{:,j} - sum_l (v_l)_j u_l */
        for (int64_t r = 0; r < m; ++r) {
            cplx a = block_entry(V, Tr, perm, space, tb + r, sb + jk, op, k, R);
            for (int l = 0; l < kk; ++l) a -= Vf[(int64_t)l * n + jk] * U[(int64_t)l * m + r];
            col[r] = a;
            uk[r] = a;
        }
        evals += m;
        /* Frobenius norm of S_k, updated incrementally */
        double nu2 = 0, nv2 = 0;
        for (int64_t r = 0; r < m; ++r) nu2 += creal(uk[r] * conj(uk[r]));
        for (int64_t j = 0; j < n; ++j) nv2 += creal(vk[j] * conj(vk[j]));
        double cross = 0;
        for (int l = 0; l < kk; ++l) {
            cplx iu = 0, iv = 0;
            for (int64_t r = 0; r < m; ++r) iu += conj(U[(int64_t)l * m + r]) * uk[r];
            for (int64_t j = 0; j < n; ++j) iv += conj(Vf[(int64_t)l * n + j]) * vk[j];
            cross += creal(iu * iv);
        }
        normS2 += 2.0 * cross + nu2 * nv2;
        ++kk;
        if (sqrt(nu2) * sqrt(nv2) <= eps * sqrt(normS2)) break;
        if (kk == kmin || nZ == m) break;
        /* next row: largest |(u_k)_i| among rows not yet used */
        double best = -1.0;
        int64_t bi = -1;
        for (int64_t r = 0; r < m; ++r)
            if (!inZ[r] && cabs(uk[r]) > best) { best = cabs(uk[r]); bi = r; }
        i = bi;
    }
    *rank = kk;
    if (entries_evaluated) *entries_evaluated = evals;
    free(R); free(row); free(col); free(inZ);
    return status;
}

/* ACA over a list of blocks; block b writes its factors at U + uoff[b],
 * V + voff[b] with capacity kcap[b] columns.  Parallel over blocks. */
int orc_aca_blocks(const double *V, const int32_t *Tr, const int32_t *perm, int space, int64_t nblk,
                   const int64_t *tb, const int64_t *te, const int64_t *sb, const int64_t *se,
                   int op, double k, double eps, const int32_t *kcap, const int32_t *rules,
                   const int64_t *uoff, const int64_t *voff, cplx *U, cplx *Vf, int32_t *rank,
                   int32_t *status, int64_t *entries, int nthreads)
{
#ifdef _OPENMP
    /* a per-call thread count that leaves the process default untouched */
    const int nth = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nth)
#endif
    for (int64_t b = 0; b < nblk; ++b) {
        int r = 0;
        int64_t ev = 0;
        status[b] = orc_aca_block(V, Tr, perm, space, tb[b], te[b], sb[b], se[b], op, k, eps, kcap[b],
                                  rules ? rules[b] : 0, U + uoff[b], Vf + voff[b], &r, &ev);
        rank[b] = r;
        entries[b] = ev;
    }
    return 0;
}

/* ACA on an explicit dense matrix (column-major m x n), same readings as
 * orc_aca_block; the pin for exact rank recovery uses it. */
int orc_aca_dense(const cplx *A, int64_t m, int64_t n, double eps, int kcap, cplx *U, cplx *Vf,
                  int *rank)
{
    cplx *row = (cplx *)malloc(sizeof(cplx) * n);
    char *inZ = (char *)calloc((size_t)m, 1);
    if (!row || !inZ) { free(row); free(inZ); return 3; }
    int kk = 0, status = 0;
    int64_t nZ = 0, i = 0, kmin = m < n ? m : n;
    double normS2 = 0, maxpiv = 0;
    for (;;) {
        for (int64_t j = 0; j < n; ++j) {
            cplx a = A[j * m + i];
            for (int l = 0; l < kk; ++l) a -= U[(int64_t)l * m + i] * Vf[(int64_t)l * n + j];
            row[j] = a;
        }
        inZ[i] = 1;
        ++nZ;
        int64_t jk = 0;
        double vmax = -1.0;
        for (int64_t j = 0; j < n; ++j)
            if (cabs(row[j]) > vmax) { vmax = cabs(row[j]); jk = j; }
        if (vmax == 0.0 || vmax <= 1e-14 * maxpiv) {
            if (nZ == m) break;
            for (i = 0; i < m && inZ[i]; ++i) {}
            continue;
        }
        if (kk == kcap) { status = 4; break; }
        if (vmax > maxpiv) maxpiv = vmax;
        cplx piv = row[jk];
        cplx *vk = Vf + (int64_t)kk * n, *uk = U + (int64_t)kk * m;
        for (int64_t j = 0; j < n; ++j) vk[j] = row[j] / piv;
        for (int64_t r = 0; r < m; ++r) {
            cplx a = A[jk * m + r];
            for (int l = 0; l < kk; ++l) a -= Vf[(int64_t)l * n + jk] * U[(int64_t)l * m + r];
            uk[r] = a;
        }
        double nu2 = 0, nv2 = 0, cross = 0;
        for (int64_t r = 0; r < m; ++r) nu2 += creal(uk[r] * conj(uk[r]));
        for (int64_t j = 0; j < n; ++j) nv2 += creal(vk[j] * conj(vk[j]));
        for (int l = 0; l < kk; ++l) {
            cplx iu = 0, iv = 0;
            for (int64_t r = 0; r < m; ++r) iu += conj(U[(int64_t)l * m + r]) * uk[r];
            for (int64_t j = 0; j < n; ++j) iv += conj(Vf[(int64_t)l * n + j]) * vk[j];
            cross += creal(iu * iv);
        }
        normS2 += 2.0 * cross + nu2 * nv2;
        ++kk;
        if (sqrt(nu2) * sqrt(nv2) <= eps * sqrt(normS2)) break;
        if (kk == kmin || nZ == m) break;
        double best = -1.0;
        int64_t bi = -1;
        for (int64_t r = 0; r < m; ++r)
            if (!inZ[r] && cabs(uk[r]) > best) { best = cabs(uk[r]); bi = r; }
        i = bi;
    }
    *rank = kk;
    free(row);
    free(inZ);
    return status;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
