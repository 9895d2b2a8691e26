// Internal host/device declarations of the GB300 BEM library.  Not part of
// the public ABI (include/bem.h).
#pragma once

#include <cstdint>
#include <cstddef>

#include <cuda_runtime.h>

namespace bem {

constexpr int NQ = 6;          // points of the regular triangle rule (degree 4)
constexpr int NGL = 4;         // Gauss-Legendre points per axis, singular rule
constexpr int KCHUNK = 4;      // ACA factor columns allocated at a time
constexpr int KMAX = 128;      // rank cap of one admissible block
constexpr int NCHUNK = KMAX / KCHUNK;

// Geometry of a triangle set in some order (identity for a mesh, cluster
// order for an H-matrix), structure-of-arrays in device memory.
struct DevGeom {
    int64_t nt;
    const int32_t *tri;    // [3][nt] vertex ids
    const double *vtx;     // [9][nt] v0.xyz v1.xyz v2.xyz
    const double *nrm;     // [3][nt] unit normal (right-hand rule)
    const double *area;    // [nt]
    const double *qp;      // [3*NQ][nt] quadrature points, q*3 + c
    // mixed-precision view in tiles of 32 triangles: tile t holds field f of
    // triangle 32 t + l at tq[1024 t + 32 f + l], so that a warp reading 32
    // consecutive triangles reads one 128-byte line per field and every field
    // of a triangle sits at a fixed offset from one address
    const float *tq;       // [ceil(nt / 32)][kTileFields][32]
};

// fields of a tile: centroid high part [3] and low part [3] (centroid - high),
// quadrature points minus centroid [NQ][3], unit normal [3], area/sqrt(4 pi)
// as float-float (hi, lo), vertex ids [3] stored as int bits
constexpr int kTileFields = 32;
constexpr int kFCh = 0, kFCl = 3, kFQ = 6, kFN = 6 + 3 * NQ, kFS = kFN + 3, kFId = kFS + 2;
static_assert(kFId + 3 == kTileFields, "tile fields");

// Regular rule: reference points and weights (sum 1); wl[p][a] = w_p lambda_a(p)
// with lambda = (1 - s - t, s, t) the barycentric coordinates of point p, the
// weights of the piecewise linear local basis functions.
// beta3: the scale that maps the stored points of the second orbit (indices
// 3..5, barycentric (b, b, 1 - 2b) and permutations) onto the points of the
// symmetric 3-point degree-2 rule (1/6, 1/6, 2/3): all lie on the medians, at
// 1 - 3b and 1/2 of the vertex distance from the centroid.
struct QuadRule {
    double s[NQ], t[NQ], w[NQ];
    float wf[NQ];
    double wl[NQ][3];
    float wlf[NQ][3];
    double beta3;
    float beta3f;
    // The two orbits lie on the medians: the point of orbit t with dominant
    // vertex v sits at (1 - 3 t)(v - centroid), so point 3 + m is
    // rho21 times point m ((1 - 3 b) / (1 - 3 a), points m and 3 + m sharing
    // their dominant vertex)
    double rho21;
    float rho21f;
};

// Regular rule of an admissible block (distance classes, Laplace, P0): the
// 6-point degree-4 rule, the 3-point degree-2 rule or the centroid rule.
constexpr int kRule6 = 0, kRule3 = 1, kRule1 = 2;

// Singular rule tables for one case (1 vertex-, 2 edge-adjacent, 3
// identical).  Each 4D Gauss-Legendre node of the Sauter-Schwab maps gives
// d = x - y as a combination sum_i c_i E_i of the case's edge vectors E_i.
//  lap:  nodes with the same direction c/|c|_max merged (exact for any
//        geometry); rows c0..c3 (normalised direction), w_slp = sum w J/rho,
//        w_dlp = sum w J/rho^2 with rho = |c|_max.  Used for k == 0.
//  helm: all maps are homogeneous of degree one in xi, so the table lists
//        the eta nodes (rows c0..c3 of d/xi and w_eta = weights times the
//        eta part of the Jacobian) and the xi axis is summed in the kernel.
//  xy:   for the same eta nodes, the reference points divided by xi,
//        rows X1, X2, Y1, Y2 (x^ = xi X, y^ = xi Y), for the linear basis
//        functions of the piecewise linear spaces.
struct SingTable {
    int n_lap;
    int n_helm;
    const double *lap;     // [6][n_lap]
    const double *helm;    // [5][n_helm]
    const double *xy;      // [4][n_helm]
    double xi[NGL], wxi[NGL];
};

struct SingPair {
    int32_t i, j;          // triangle ids in the mesh's own order
    int64_t dest;          // element offset of the result
};

// A touching pair of a piecewise linear matrix: its 3 x 3 local matrix goes to
// dest + alpha * rs + beta * cs (alpha, beta: stored vertex indices; rs, cs:
// the strides of the output's rows and columns).
struct SingPairL {
    int32_t i, j;
    int64_t dest;
    int32_t rs, cs;
};

struct FarBlock {
    int64_t tb, te, sb, se;         // cluster-order ranges (rows: tau)
    int32_t rank;
    int32_t status;                 // 0 ok, 1 rank cap, 2 pool overflow
    int64_t entries;                // entries evaluated by ACA
    int32_t rule;                   // kRule6 / kRule3 / kRule1 (Laplace entries)
    int32_t pad;
};

// Element offsets of a block's factor chunks (-1: not allocated), written by
// the ACA; an array parallel to the FarBlock list, kept apart so that the
// host-built block descriptors stay small.
struct FarChunks {
    int64_t c[NCHUNK];
};

// A dense (near-field) block, stored column-major: entry (r, c) at
// off + c * (te - tb) + r, so that the lanes that own consecutive rows in the
// product read consecutive addresses.
struct NearBlock {
    int64_t tb, te, sb, se;
    int64_t off;                    // element offset of the dense block
};

struct Pool {
    unsigned long long top;         // elements used
    unsigned long long cap;         // elements available
    int overflow;
    int pad;
};

// Totals of one ACA launch, reduced on the device.
struct AcaStats {
    unsigned long long entries;       // entries evaluated by all blocks
    unsigned long long rank_sum;      // = total length of the V^T x buffer
    unsigned long long factor_elems;  // elements of all allocated chunks
    unsigned long long k2mn;          // sum over blocks of rank^2 (m + n): FP64 multiply-adds
                                      // of the residual updates and norm terms
    unsigned long long rank_mn;       // sum over blocks of rank (m + n): factor elements a
                                      // product reads
    int rank_min, rank_max;
    int capped, failed;
};

struct AcaQueue {
    unsigned int next_big;
    unsigned int next_small;
    unsigned int next_tiny;
    unsigned int next_w16;
    unsigned int next_w8;
    unsigned int pad[3];
};

// Work shapes of admissible blocks (P0): a whole CTA, a warp, half a warp
// (16 lanes, two blocks per warp), a quarter warp (8 lanes, four blocks per
// warp), or one lane.  Blocks with max(m, n) <= kSub8Max rows take 8 lanes,
// <= kSub16Max 16 lanes (unless bem_tuning sends them to a CTA or a lane).
constexpr int kSub8Max = 40, kSub16Max = 80;
enum AcaShape { kShapeCta = 0, kShapeWarp = 1, kShapeHalf = 2, kShapeQuarter = 3, kShapeLane = 4 };

// One H-matrix's part of an ACA launch: its cluster-order geometry, its
// admissible blocks and their chunk tables, its factor pool, k and eps.
struct AcaJob {
    DevGeom g;
    FarBlock *far;
    FarChunks *chunks;
    void *pool;
    Pool *P;
    double k, eps;
    int64_t n_far;           // entries of far and chunks
};

// Work list of one ACA launch: the blocks of each work shape (AcaShape
// order), each shape's blocks in descending size.
// items == nullptr: item i is block i of jobs[0] (one H-matrix whose block
// array is in that order); otherwise items[i] = (job << kItemShift) | the
// block's index in that job's array (the request server's launches over
// several H-matrices).
constexpr int kItemShift = 40;
struct AcaWork {
    const AcaJob *jobs;      // device array
    const int64_t *items;    // device array or null
    int64_t n[5];            // blocks per work shape (AcaShape order; the items in that order)
    int64_t max_m_big, max_m_small;  // most rows of a CTA block, of a warp block
    int max_ctas = 0;        // > 0: at most this many CTAs (leaves SMs to other streams)
    int64_t n_jobs = 1;      // entries of jobs (items naming another job are skipped)
};

// Read-only view of a mesh and of already-initialised per-device constants,
// for entry points that must not allocate.  mesh_view fails (returns false)
// for a null mesh; consts_peek returns false if the device has none yet.
struct MeshView {
    DevGeom g;
    int device;
    int64_t nt;
    int64_t max_touch;
};
bool mesh_view(const void *mesh, MeshView *out);
bool consts_peek(int device, QuadRule *rule, const SingTable **sing);
void set_last_error(const char *msg);

// Stream value meaning "host part only" for the staged create functions.
inline cudaStream_t const kHostOnly = reinterpret_cast<cudaStream_t>(~uintptr_t(0));

// Process-wide count of kernel launches (launch accounting).
void count_launches(int64_t n);
int64_t launches_total();

// ---- launchers (defined in the .cu files) -------------------------------
cudaError_t launch_geometry(const double *V, const int32_t *T, const int32_t *perm, int64_t nt,
                            const QuadRule &rule, void *const bufs[6], cudaStream_t st);

cudaError_t launch_entries_regular(const DevGeom &g, const QuadRule &rule, int op, double k,
                                   int prec, const int32_t *test, int64_t n_test,
                                   const int32_t *trial, int64_t n_trial, void *out,
                                   SingPair *lists[3], unsigned long long *counts,
                                   unsigned long long cap, int *err, cudaStream_t st);

// Touching pairs of each case: min(dev_counts[c], host_counts[c]) pairs
// (dev_counts may be null); grid_counts[c], if given, sizes the grid instead
// of host_counts[c] (the threads stride over every pair either way).
// vertex_dest2, if given, holds per vertex-adjacent pair the offset of the
// transposed entry A_ji (or -1 for none), evaluated by the same quadrature.
cudaError_t launch_singular(const DevGeom &g, const SingTable *tabs, int op, double k, int prec,
                            const SingPair *pairs[3], const unsigned long long *dev_counts,
                            const int64_t host_counts[3], void *out, cudaStream_t st,
                            const int64_t *grid_counts = nullptr,
                            const int64_t *vertex_dest2 = nullptr);

cudaError_t launch_near_regular(const DevGeom &g, const QuadRule &rule, int op, double k, int prec,
                                const NearBlock *blocks, int64_t nblocks, void *out,
                                cudaStream_t st);

// Piecewise linear (DP1) counterparts: local 3 x 3 matrices of element pairs.
// Entries of triangle lists: out is [3 n_test][3 n_trial].
cudaError_t launch_entries_dp1(const DevGeom &g, const QuadRule &rule, int op, double k, int prec,
                               const int32_t *test, int64_t n_test, const int32_t *trial,
                               int64_t n_trial, void *out, SingPairL *lists[3],
                               unsigned long long *counts, unsigned long long cap, int *err,
                               cudaStream_t st);
cudaError_t launch_singular_dp1(const DevGeom &g, const SingTable *tabs, int op, double k,
                                const SingPairL *pairs[3], const unsigned long long *dev_counts,
                                const int64_t host_counts[3], void *out, cudaStream_t st);
// Continuous P1 around a DP1 matrix: x_dp1 = C x, y = C^T y_dp1; and the
// hypersingular operator through the DP1 single layer, Eq. (9):
// xs = (Q_1 x, Q_2 x, Q_3 x[, P_1 x, P_2 x, P_3 x]) (nvec = 3 for k = 0, else
// 6), y = sum_j Q_j^T ys_j - k^2 sum_j P_j^T ys_{3+j}.  g in the mesh's order.
cudaError_t launch_p1_gather(bool cplx, const int32_t *tri, int64_t nt, const void *x, void *xd,
                             cudaStream_t st);
cudaError_t launch_p1_scatter(bool cplx, const int64_t *vptr, const int32_t *vdof, int64_t nv,
                              const void *yd, void *y, cudaStream_t st);
cudaError_t launch_hyps_in(bool cplx, const DevGeom &g, const void *x, void *xs, int nvec,
                           cudaStream_t st);
cudaError_t launch_hyps_out(bool cplx, const int64_t *vptr, const int32_t *vdof, const DevGeom &g,
                            int64_t nv, double k, const void *ys, int nvec, void *y,
                            cudaStream_t st);
// near-field blocks in dof units (ranges are three times the triangle ranges)
cudaError_t launch_near_dp1(const DevGeom &g, const QuadRule &rule, int op, double k, int prec,
                            const NearBlock *blocks, int64_t nblocks, void *out, cudaStream_t st);

// dofs = 1: P0 (a dof per triangle); dofs = 3: DP1 (block ranges in dof
// units, three local dofs per triangle).  cplx: Helmholtz (k != 0) for every
// job of the launch; rules: the mixed Laplace kernels that read each block's
// distance class.
cudaError_t launch_aca(const AcaWork &w, const QuadRule &rule, int op, bool cplx, int prec,
                       AcaQueue *queue, int num_sms, cudaStream_t st, int dofs = 1,
                       bool rules = false);

// the P0 instantiations of BEM_MIXED_SP (kernels_aca_sp.cu: FP32 dot
// products in the norm of S_k)
cudaError_t launch_aca_sp(const AcaWork &w, const QuadRule &rule, int op, bool cplx,
                          AcaQueue *queue, int num_sms, cudaStream_t st, bool rules);

// the DP1 instantiations (kernels_aca_dp1.cu); no tiny-block class
cudaError_t launch_aca_dp1(const AcaWork &w, const QuadRule &rule, int op, bool cplx, int prec,
                           AcaQueue *queue, int num_sms, cudaStream_t st);

// y[i] = 1 / x[i] by the ACA's pivot reciprocal (diagnostic)
cudaError_t launch_debug_recip(const double *x, double *y, int64_t n, cudaStream_t st);
cudaError_t launch_debug_rsqrt(const double *x, double *y, int64_t n, cudaStream_t st);

// After an ACA launch: toff[b] = sum of ranks of blocks < b (toff[n] = total)
// and the totals in *st.  tile_sums needs aca_finish_tiles(n) entries.
int64_t aca_finish_tiles(int64_t nfar);
// Zeroes the pool header (capacity cap), the work queues and the totals.
cudaError_t launch_aca_reset(Pool *P, unsigned long long cap, AcaQueue *Q, AcaStats *st,
                             cudaStream_t s);
cudaError_t launch_aca_finish(const FarBlock *far, const FarChunks *chunks, int64_t nfar,
                              int64_t *toff,
                              int64_t *tile_sums, AcaStats *st, cudaStream_t st_);

cudaError_t launch_matvec(bool cplx, int64_t n, const int32_t *perm, const void *x, void *y,
                          void *xt, void *yt, void *tbuf, const FarBlock *far,
                          const FarChunks *chunks, int64_t nfar,
                          const int64_t *toff, const void *pool_data, const NearBlock *near,
                          const void *near_data, const int64_t *leaf_rows,
                          const int64_t *leaf_ptr, const int64_t *leaf_items, int64_t nleaf,
                          const int64_t *long_ids, int64_t nlong, int64_t *long_off,
                          cudaStream_t st);
// After an assembly: prefix sum of the ranks of the long-column blocks.
cudaError_t launch_long_offsets(const FarBlock *far, const int64_t *ids, int64_t nids,
                                int64_t *loff, cudaStream_t st);
// column length above which V^T x uses one warp per column
constexpr int64_t kMatvecLongCol = 1024;

}  // namespace bem
