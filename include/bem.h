/*
 * bem.h -- C ABI of the GB300 library for Galerkin boundary-element matrices
 * (piecewise constant P0 and piecewise linear DP1 / P1 spaces) of the 3D
 * Laplace and Helmholtz single-layer, double-layer, adjoint double-layer and
 * hypersingular operators, assembled as H-matrices with ACA
 * (Vater, Betcke, Dilba, "Simple and efficient GPU parallelization of
 * existing H-Matrix accelerated BEM code", arXiv 1711.01897).
 *
 * Conventions shared by every call
 *  - Every call returns a bem_status.  No call aborts, traps or prints.  The
 *    text of the last error of the calling thread is bem_last_error().
 *  - Handles are created and destroyed by the caller; the library copies all
 *    mesh inputs, so caller buffers may be freed after a create call.
 *  - Output buffers are owned by the caller.  A pointer argument may be host
 *    or device memory unless stated otherwise; the library detects which.
 *  - cuda_stream is a cudaStream_t (NULL = the legacy default stream).  Work
 *    with device-resident inputs and outputs is enqueued on that stream and
 *    the call returns without waiting, unless stated otherwise.  Calls with
 *    host buffers wait for their copies to finish before returning.
 *  - Rows are test functions psi_i and columns trial functions phi_j, as in
 *    [S_h]_{i,j} of Eq. (1).  Spaces (test and trial alike):
 *      BEM_P0   one basis function per triangle, its indicator
 *      BEM_DP1  three per triangle: dof 3 t + a is the barycentric coordinate
 *               of stored vertex a on triangle t, zero elsewhere
 *               (discontinuous piecewise linear)
 *      BEM_P1   one per vertex, the continuous hat function; its matrix is
 *               C^T A_DP1 C with C[3 t + a, v] = 1 where T[t][a] = v, i.e.
 *               the global assembly of the element pairs' local matrices
 *               (Sec. 3.2.3, "Global matrix assembly")
 *  - Operators (Sec. 2, Eq. (1)-(3) with g of Eq. (5), k = 0 for Laplace):
 *      BEM_SLP  single layer          int int psi_i g phi_j
 *      BEM_DLP  double layer          int int psi_i dg/dn_y phi_j
 *      BEM_ADLP adjoint double layer  int int psi_i dg/dn_x phi_j
 *      BEM_HYPS hypersingular (Eq. (4)), P1 only, applied as
 *               D = sum_j Q_j^T S Q_j - k^2 sum_j P_j^T S P_j with S the single
 *               layer on DP1, Q_j the j-th component of the surface curl and
 *               P_j the j-th normal component (Eq. (9), Sec. 5.1)
 *    Values are f64 for k == 0 and interleaved complex128 (re, im) for k != 0.
 *  - Quadrature: pairs that share no vertex use the symmetric 6-point
 *    degree-4 triangle rule in both triangles (Sec. 3.2.1, Sec. 3.2.3);
 *    pairs that share a vertex, an edge or the whole triangle use the
 *    Sauter-Schwab transformations of [0,1]^4 with 4 Gauss-Legendre points
 *    per axis (the Erichsen-Sauter scheme cited in Sec. 3.2.3), in FP64
 *    (BEM_MIXED_SP excepted, below).
 *  - Precision (Sec. 3.2.4):
 *      BEM_FP64      every quadrature, pivot, residual update and norm in FP64.
 *      BEM_MIXED     regular pairs (far field and the non-touching near
 *                    field) in FP32 with centroid-relative geometry, each
 *                    entry's quadrature sum accumulated in float-float (about
 *                    48 significant bits) and stored in FP64; FP64 for the
 *                    singular pairs, the ACA pivot search, the residual
 *                    updates and the norms of the stopping test.
 *      BEM_MIXED_SP  BEM_MIXED, plus single precision in two more places:
 *                    the dot products of the norm of S_k (they feed only the
 *                    stopping test; its accumulation stays FP64), and, for
 *                    Laplace, the Sauter-Schwab integrands after the
 *                    transformation (FP32 evaluations, float-float sums; the
 *                    pair's geometry and final scaling FP64).  P0 only
 *                    (hmat_assemble on DP1 / P1 handles returns BEM_E_ARG);
 *                    not for bem_entries_dp1.
 */
#ifndef BEM_H
#define BEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bem_mesh_s *bem_mesh;
typedef struct bem_hmat_s *bem_hmat;

enum bem_op { BEM_SLP = 0, BEM_DLP = 1, BEM_ADLP = 2, BEM_HYPS = 3 };
enum bem_space { BEM_P0 = 0, BEM_DP1 = 1, BEM_P1 = 2 };
enum bem_prec { BEM_FP64 = 0, BEM_MIXED = 1, BEM_MIXED_SP = 2 };
enum bem_status {
    BEM_OK = 0,
    BEM_E_ARG = 1,     /* invalid argument (null handle, size, enum, index) */
    BEM_E_MESH = 2,    /* mesh rejected: index out of range, zero area, NaN */
    BEM_E_OOM = 3,     /* device or host allocation failed */
    BEM_E_CUDA = 4,    /* a CUDA runtime call failed */
    BEM_E_TIMEOUT = 5, /* a bounded device-side wait ran out */
    BEM_E_STATE = 6    /* call not valid in the handle's state */
};

/* Library version, e.g. 100 for 0.1.0. */
int bem_version(void);

/* Number of CUDA kernels this library has launched in this process (all
 * devices, all handles); a monotone counter for launch accounting. */
int64_t bem_kernel_launches(void);

/* Bytes of the library's stream-ordered device memory pool on the current
 * device: *reserved = memory the pool holds from the driver, *used = memory
 * handed out and not yet freed.  Either pointer may be null.  The pool backs
 * every device buffer of meshes, trees and assemblies, so the two numbers
 * show whether a call allocated. */
int bem_memory_usage(int64_t *reserved, int64_t *used);

/* Throughputs measured on the current device by short calibration kernels
 * (independent dependency chains in every thread, best of three timed
 * launches after a warm-up, CUDA events on `cuda_stream`): the roofline
 * denominators of the units the hot path is bound by.  The paper reports no
 * such figures; this is an interface of this library only.  Rates are
 * instructions per second (one fused multiply-add counts once) and bytes per
 * second (read + write of a 1 GiB device copy).  Allocates and frees 2 GiB of
 * device memory; takes a few tens of milliseconds. */
typedef struct {
    double fp32_fma_per_s;    /* FFMA */
    double fp64_fma_per_s;    /* DFMA */
    double mufu_rsqrt_per_s;  /* rsqrt.approx.ftz.f32 */
    double mufu_sin_per_s;    /* sin.approx.ftz.f32 */
    double copy_bytes_per_s;  /* device-to-device copy by a kernel */
    int32_t sm_count;
    double clock_mhz_nominal; /* the device's reported SM clock */
    float ms[5];              /* best launch time of each kernel, in the order above */
} bem_peaks;

int bem_measure_peaks(bem_peaks *out, void *cuda_stream);

/* Diagnostic of the FP64 reciprocal that scales every ACA pivot (Eq. (7):
 * v_k = v~_k / (v~_k)_{j_k}): y[i] = 1 / x[i] computed on the device by the
 * routine the ACA kernels use (Newton-Raphson from a single-precision seed,
 * correct to rounding level; IEEE division outside the seed's exponent
 * range).  x, y: device arrays of n doubles on the current device (y may
 * alias x); x[i] finite and nonzero.  Returns after the stream is
 * synchronised. */
int bem_debug_recip(const double *x, double *y, int64_t n, void *cuda_stream);

/* Diagnostic of the FP64 reciprocal square root of the FP64 quadratures
 * (the singular pairs of Sec. 3.2.3 and the FP64 regular pairs, where the
 * kernels of Eq. (5) take 1/|x - y|): y[i] = 1 / sqrt(x[i]) by the routine
 * those kernels use (one Newton step in FP64 from a single-precision seed of
 * the mantissa reduced to [1, 4); relative error below 7e-14).  x, y: device
 * arrays of n doubles on the current device (y may alias x); x[i] positive
 * and normal (other values give unspecified results).  Returns after the
 * stream is synchronised. */
int bem_debug_rsqrt(const double *x, double *y, int64_t n, void *cuda_stream);

/* Process-wide tuning, read when a tree is built (row thresholds) and when
 * an H-matrix is assembled (graphs).  The numerical results do not depend on
 * it (up to ACA pivot near-ties, which rounding decides).
 *  warp_max_rows  admissible blocks with max(m, n) <= this are compressed by
 *                 warps, larger ones by a whole CTA (1..8192); a block of at
 *                 most 80 rows takes half a warp (two blocks per warp), of at
 *                 most 40 rows a quarter warp (four per warp)
 *  lane_max_rows  ... and those with max(m, n) <= this by one lane each,
 *                 32 blocks per warp (0 = off, at most 64)
 *  use_graphs     1: the kernel sequence of hmat_assemble is captured into a
 *                 CUDA graph per handle and replayed while op, k, aca_eps,
 *                 prec and the buffers stay the same */
typedef struct {
    int32_t warp_max_rows;
    int32_t lane_max_rows;
    int32_t use_graphs;
} bem_tuning;

int bem_set_tuning(const bem_tuning *t);
int bem_get_tuning(bem_tuning *t);

/* Regular quadrature order per distance class of the admissible blocks
 * (process-wide, read when a P0 tree is built).  The paper evaluates every
 * regular pair with one symmetric 6-point rule of degree 4 (Sec. 3.2.1); a
 * block far enough apart relative to its triangles may use a lower-order
 * rule of the same family.  With rho = dist(tau, sigma) / h -- the distance
 * between the two cluster boxes over the longest triangle edge in either
 * cluster --
 *   rho >= rho1 > 0            the centroid rule (1 point, degree 1),
 *   else rho >= rho3 > 0       the 3-point rule of degree 2 (barycentric
 *                              (2/3, 1/6, 1/6) and permutations),
 *   else                       the 6-point rule.
 * 0 switches a class off (the default: every block uses the 6-point rule).
 * The classes apply to the mixed-precision assembly of the Laplace
 * operators (k = 0) on P0 handles.  The Helmholtz entries (whose lower-order
 * error is set by k h, not by the distance), the FP64 assembly (the plain
 * form), the near field and the piecewise linear spaces keep the 6-point
 * rule.  q is copied (set) or filled (get); BEM_E_ARG for a null pointer or
 * negative or non-finite thresholds, which leave the setting unchanged. */
typedef struct {
    double rho3;
    double rho1;
} bem_quadrature;

int bem_set_quadrature(const bem_quadrature *q);
int bem_get_quadrature(bem_quadrature *q);

/* Text of the calling thread's last error ("" if none).  The pointer stays
 * valid until the next library call on this thread. */
const char *bem_last_error(void);

/* ---------------------------------------------------------------------- */
/* Meshes (Sec. 3.2.1: the whole grid is copied to the device; normals,     */
/* areas and global quadrature points are precomputed there)               */
/* ---------------------------------------------------------------------- */

/* Creates a mesh on the current CUDA device.
 *  vertices   host f64 [n_vertices][3], row-major
 *  triangles  host i32 [n_triangles][3], 0-based; the right-hand normal of
 *             the stored vertex order is n in dg/dn (outward for closed
 *             surfaces with counter-clockwise order seen from outside)
 *  out        receives the handle
 * Fails with BEM_E_MESH for an index outside [0, n_vertices), a repeated
 * vertex in a triangle, a triangle of zero area, or a non-finite coordinate;
 * BEM_E_ARG for n_vertices < 3, n_triangles < 1 or n_triangles >= 2^31.
 * Synchronous: returns after the device geometry is built. */
int bem_mesh_create(const double *vertices, int64_t n_vertices, const int32_t *triangles,
                    int64_t n_triangles, bem_mesh *out);

/* Frees a mesh.  Hierarchical matrices built on it must be destroyed first
 * (BEM_E_STATE otherwise). */
int bem_mesh_destroy(bem_mesh mesh);

/* Number of triangles; -1 for a null handle. */
int64_t bem_mesh_size(bem_mesh mesh);

/* Dense sub-block of the Galerkin matrix (Eq. (1)-(3)):
 *   out[a][b] = A(test_ids[a], trial_ids[b]),  row-major [n_test][n_trial],
 * f64 for k == 0, interleaved complex128 otherwise.  Any pairs may be
 * requested, including pairs that share vertices (evaluated by the singular
 * rule, Sec. 3.2.3, on the device).  Ids must lie in [0, n_triangles);
 * device-resident ids are checked on the device and a bad id makes the call
 * return BEM_E_ARG at its next synchronisation (the call then waits for the
 * stream).  test_ids, trial_ids and out may each be host or device memory.
 * prec: BEM_FP64, BEM_MIXED (regular pairs in FP32, singular pairs FP64) or
 * BEM_MIXED_SP (Laplace singular pairs with FP32 integrands as well).
 * Allocates stream-ordered device scratch for the list of singular pairs
 * (sized by n_test times the most triangles touching one triangle; repeated
 * trial ids that hold more touching pairs make a second, exactly sized pass).
 * Returns after the stream is synchronised. */
int bem_entries(bem_mesh mesh, int32_t op, double k, int32_t prec, const int32_t *test_ids,
                int64_t n_test, const int32_t *trial_ids, int64_t n_trial, void *out,
                void *cuda_stream);

/* The same dense sub-block as bem_entries, for callers that cannot allocate
 * device memory while they run: a process whose device memory is entirely
 * reserved by its own pool allocator (an allocation from inside this library
 * would fail or fragment that pool), or a loop where the latency or failure
 * of an allocation is not acceptable.  The paper has no counterpart; this is
 * an interface of this library only.
 *  - Allocates nothing: no cudaMalloc, cudaMallocAsync, cudaFree or
 *    allocating library routine.  The list of singular pairs lives in one
 *    file-scope device array of the library, 12 MiB plus counters, which
 *    every GPU that loads the library holds until the process exits.
 *  - test_ids, trial_ids and out must be device (or managed) memory of the
 *    mesh's device, which must be current (BEM_E_ARG for host memory or
 *    memory of another device, BEM_E_STATE for another current device).
 *  - Maximum size: the request may hold at most 262,144 singular pairs of
 *    each kind, counted as min(n_test * n_trial, n_test * T) with T the
 *    largest number of triangles that touch one triangle; larger requests
 *    return BEM_E_ARG without launching anything (use bem_entries).  Repeated
 *    trial ids can hold more touching pairs than that count: if they exceed
 *    the capacity, the call returns BEM_E_ARG after its launches and `out`
 *    is undefined.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - Every call shares the array and clears its counters first; the array
 *    keeps the last call's contents.  Calls whose work overlaps on the GPU
 *    (different streams or threads) race on it: serialise them.
 *  - Returns after the stream is synchronised, like bem_entries. */
int bem_entries_noalloc(bem_mesh mesh, int32_t op, double k, int32_t prec,
                        const int32_t *test_ids, int64_t n_test, const int32_t *trial_ids,
                        int64_t n_trial, void *out, void *cuda_stream);

/* Dense DP1 sub-block for triangle lists (Sec. 3.3, Algorithm "Integral
 * Evaluation": every combination of local dofs of an element pair):
 *   out[3 a + alpha][3 b + beta] = int_{T_i} int_{T_j} lambda_alpha g' lambda_beta,
 *   i = test_tris[a], j = trial_tris[b], row-major [3 n_test][3 n_trial],
 * with lambda the barycentric coordinates of the stored vertices and g' the
 * kernel of op (BEM_SLP, BEM_DLP or BEM_ADLP).  Same quadrature, precision
 * (BEM_FP64 or BEM_MIXED; BEM_MIXED_SP gives BEM_E_ARG), argument rules,
 * scratch and synchronisation as bem_entries; touching pairs
 * use the Sauter-Schwab rule with the basis functions at the mapped points. */
int bem_entries_dp1(bem_mesh mesh, int32_t op, double k, int32_t prec, const int32_t *test_tris,
                    int64_t n_test, const int32_t *trial_tris, int64_t n_trial, void *out,
                    void *cuda_stream);

/* ---------------------------------------------------------------------- */
/* Hierarchical matrices (Sec. 2.1; Algorithm "H-Matrix Assembly", Sec. 4.1)*/
/* ---------------------------------------------------------------------- */

/* Builds the cluster tree and the block cluster tree on the host ("purely
 * geometry-based", Sec. 4.1) and uploads them, with the geometry in cluster
 * order, to the device.
 *  leaf_size  a cluster with more triangles is split in two along the longest
 *             axis of its vertex bounding box, at the median of the triangle
 *             centroids ((v0 + v1) + v2)/3 (ties by triangle index); leaves
 *             list their triangles in increasing index order
 *  eta        a block (tau, sigma) is admissible, i.e. compressed by ACA, iff
 *             the bounding boxes are disjoint and
 *             min(diam tau, diam sigma) <= eta * dist(tau, sigma)
 *             (box diagonal and box distance); otherwise it is split, or
 *             stored dense when tau or sigma is a leaf
 * The handle keeps a reference to the mesh.  Synchronous. */
int hmat_build_tree(bem_mesh mesh, int32_t leaf_size, double eta, bem_hmat *out);

/* hmat_build_tree for a space (BEM_P0, BEM_DP1 or BEM_P1).  The piecewise
 * linear spaces use the same cluster and block trees, every triangle carrying
 * its three DP1 dofs: a block of triangle ranges is the block of the tripled
 * dof ranges (dof 3 p + a of cluster position p), so leaf_size counts
 * triangles.  BEM_P1 handles hold the DP1 matrix and apply C and C^T around
 * it in hmat_matvec.  hmat_build_tree(...) == hmat_build_tree_space(..., BEM_P0). */
int hmat_build_tree_space(bem_mesh mesh, int32_t leaf_size, double eta, int32_t space,
                          bem_hmat *out);

/* Length of the vectors of hmat_matvec: triangles (P0), 3 x triangles (DP1)
 * or vertices (P1); -1 for a null handle. */
int64_t hmat_dofs(bem_hmat hmat);

/* Assembles the H-matrix of operator op and wavenumber k on the device:
 * dense near-field blocks (regular pairs by Gauss, singular pairs by
 * Sauter-Schwab) and, for every admissible block, ACA with partial pivoting
 * (Sec. 2.1, Eq. (6)-(7), Algorithm ACA) run for all blocks by one
 * persistent kernel fed from a device work queue.  ACA readings: the first
 * row is the block's first row; later rows maximise |u_k| over unused rows
 * (lowest index on ties); a row whose maximum is 0 or at most 1e-14 times the
 * largest pivot so far "vanishes" and the smallest unused row is taken next;
 * the loop stops once ||u_k|| ||v_k|| <= aca_eps ||S_k||_F, or when k reaches
 * min(m, n) or the rank cap, or when all rows are used.
 *  op       BEM_SLP, BEM_DLP, BEM_ADLP; BEM_HYPS on BEM_P1 handles (the
 *           single layer on DP1 is assembled, the rest is applied in products)
 *  aca_eps  > 0
 *  prec     BEM_FP64, BEM_MIXED, or (P0 handles) BEM_MIXED_SP (see the top
 *           of this file)
 * May be called again on the same handle (the previous matrix is replaced).
 * Synchronous: it reads back the device status word; a bounded device wait
 * that runs out gives BEM_E_TIMEOUT. */
int hmat_assemble(bem_hmat hmat, int32_t op, double k, double aca_eps, int32_t prec,
                  void *cuda_stream);

/* y = A x for the assembled H-matrix, in the original dof order (the
 * cluster permutation is applied inside).  x and y hold `batch` vectors one
 * after another, each hmat_dofs() long (triangles, DP1 dofs 3 t + a, or
 * vertices), f64 for k == 0 and complex128 otherwise; host or device memory.
 * P1: y = C^T A_DP1 C x; BEM_HYPS: D x by Eq. (9) with three DP1
 * products for k = 0 and six otherwise.  Uses buffers owned by the handle:
 * concurrent products on one handle must be on the same stream.
 * BEM_E_STATE before hmat_assemble. */
int hmat_matvec(bem_hmat hmat, const void *x, void *y, int32_t batch, void *cuda_stream);

typedef struct {
    int64_t n_triangles;
    int64_t n_clusters;
    int64_t n_blocks_near;
    int64_t n_blocks_far;
    int64_t near_entries;        /* entries of all dense blocks */
    int64_t singular_pairs[3];   /* vertex-, edge-adjacent, identical */
    int64_t far_entries;         /* entries the ACA evaluated (rows + columns) */
    int64_t factor_bytes;        /* bytes of U, V factors (allocated 4-column chunks) */
    int64_t near_bytes;          /* bytes of the dense blocks */
    int32_t rank_min, rank_max;
    double rank_mean;
    int64_t rank_capped_blocks;  /* blocks that stopped at the rank cap */
    double time_tree_ms;         /* hmat_build_tree, host */
    double time_near_ms;         /* last assembly: near field (device) */
    double time_far_ms;          /* last assembly: ACA (device) */
    double time_near_regular_ms; /* part of time_near_ms: regular pairs */
    double time_singular_ms;     /* part of time_near_ms: singular pairs */
    int64_t aca_fp64_fma;        /* sum over admissible blocks of rank^2 (m + n): the
                                    multiply-adds of the ACA residual updates (about half,
                                    FP64) and of the norm's dot products (the other half:
                                    FP64 in BEM_FP64 and BEM_MIXED, FP32 in
                                    BEM_MIXED_SP) */
    int32_t assembled;
    int32_t op;
    double k;
    double aca_eps;
    int32_t prec;
    int32_t space;               /* BEM_P0, BEM_DP1, BEM_P1 */
    int64_t n_dofs;              /* hmat_dofs() */
    double time_tree_clusters_ms; /* parts of time_tree_ms: cluster tree, block tree, */
    double time_tree_blocks_ms;   /* block lists and touching pairs (host), and the   */
    double time_tree_lists_ms;    /* upload with the cluster-order geometry (device)  */
    double time_tree_upload_ms;
    int64_t factor_read_bytes;   /* bytes of U, V a product reads: sum of rank (m + n) */
    int64_t n_blocks_rule3;      /* admissible blocks of the 3-point and centroid classes */
    int64_t n_blocks_rule1;
    double rho3;                 /* the thresholds the tree was built with */
    double rho1;
    int64_t n_blocks_cta;        /* admissible blocks by ACA work shape (bem_tuning at tree   */
    int64_t n_blocks_warp;       /* build): a whole CTA per block, warps (a warp holds one or */
    int64_t n_blocks_lane;       /* several blocks), one lane per block                       */
    int64_t n_blocks_half_warp;  /* ... of n_blocks_warp: blocks of at most 80 rows on 16    */
    int64_t n_blocks_quarter_warp; /* lanes (two per warp), of at most 40 on 8 (four per warp) */
} bem_hmat_stats;

/* Copies statistics of the handle into *out. */
int hmat_stats(bem_hmat hmat, bem_hmat_stats *out);

/* Block list in cluster order for inspection: rows of 5 int64
 * (tau_begin, tau_end, sigma_begin, sigma_end, admissible) into host
 * `blocks` (capacity `cap` rows) and the permutation (cluster position ->
 * triangle id) into host `perm` (n_triangles).  *n_blocks receives the
 * number of blocks; BEM_E_ARG if cap is too small.  For DP1 and P1 handles
 * the ranges are DP1 dof ranges (three dofs per cluster position). */
int hmat_blocks(bem_hmat hmat, int64_t *blocks, int64_t cap, int64_t *n_blocks, int32_t *perm);

/* Copies one assembled block to host memory as a dense row-major m x n
 * array in cluster order (f64 or complex128): the near-field entries, or
 * U V^T for an admissible block; *rank receives its ACA rank (-1 for a
 * dense block).  DP1 and P1 handles: DP1 dofs, as in hmat_blocks. */
int hmat_block_dense(bem_hmat hmat, int64_t block, void *out, int32_t *rank);

/* Points per triangle of the regular rule of every block (tree order, as in
 * hmat_blocks): 6, 3 or 1 for admissible blocks (the distance classes of
 * bem_set_quadrature at tree build; 6 = the 6-point rule of Sec. 3.2.1), 0
 * for near-field blocks.  points: caller-owned host array, capacity cap >=
 * the number of blocks (hmat_blocks gives it).  BEM_E_ARG for a null handle
 * or array, or too small a capacity.  Needs no assembly and no device. */
int hmat_block_rules(bem_hmat hmat, int32_t *points, int64_t cap);

/* Row partition for assembling one H-matrix on several GPUs (the paper
 * divides its block list evenly between two GPUs, Sec. 4.1; here every part
 * owns whole block rows, balanced by estimated cost, so that no product
 * needs a reduction).  The cluster-order rows [0, n_rows) are cut into
 * n_parts ranges, only where no block's row range is cut, each range's cost
 * as near as those cuts allow to 1/n_parts of the total: m n per dense
 * block, (m + n) rank_est per admissible block, spread over its rows.
 * blocks: n_blocks rows of 5 int64 (tau_begin, tau_end, sigma_begin,
 * sigma_end, admissible) as hmat_blocks returns them; bounds: caller-owned,
 * n_parts + 1 entries (bounds[0] = 0, bounds[n_parts] = n_rows; a part may
 * be empty).  Host only; BEM_E_ARG for bad sizes or a block outside the
 * rows. */
int bem_partition_rows(const int64_t *blocks, int64_t n_blocks, int64_t n_rows, int32_t n_parts,
                       double rank_est, int64_t *bounds);

/* Part `part` (0 .. n_parts - 1) of the row partition of the P0 block tree
 * that hmat_build_tree(mesh, leaf_size, eta) would build: the same clusters
 * and blocks, keeping the blocks whose rows lie in the part's range (the
 * bem_partition_rows split with rank_est = 10).  Assembly then evaluates
 * only those blocks, and hmat_matvec returns the full-length product with
 * the rows of other parts set to zero: the products of all parts add up to
 * the product of the whole matrix, each row coming from exactly one part.
 * hmat_part_rows gives the part's cluster-order row range (hmat_blocks gives
 * the permutation).  BEM_E_ARG for a bad part. */
int hmat_build_tree_part(bem_mesh mesh, int32_t leaf_size, double eta, int32_t n_parts,
                         int32_t part, bem_hmat *out);
int hmat_part_rows(bem_hmat hmat, int64_t *row_begin, int64_t *row_end);

/* Frees the handle and its device memory. */
int hmat_destroy(bem_hmat hmat);

/* ---------------------------------------------------------------------- */
/* Request server: assembly-and-product requests for meshes of different    */
/* sizes and wavenumbers arrive over time and are served with continuous    */
/* batching.  Host threads build each request's trees; an engine admits     */
/* requests in arrival order as the HBM budget allows and runs everything   */
/* admitted since its last launch as one batch: the near fields, then ONE   */
/* persistent ACA launch over the admissible blocks of all the batch's      */
/* requests of the same kind (Algorithm ACA, Sec. 2.1, across matrices), then */
/* the products.  Requests that arrive meanwhile join the next batch, which   */
/* overlaps the running one on a second stream.  Assembled matrices stay     */
/* resident until the budget needs their bytes (least recently used first),  */
/* and a request may apply a resident matrix instead of assembling one.      */
/* (The paper runs one problem at a time; this is the library's serving      */
/* interface.)                                                               */
/* ---------------------------------------------------------------------- */

typedef struct bem_server_s *bem_server;

enum bem_server_flags { BEM_SERVER_DRY_RUN = 1 };  /* no device work (host logic only) */
enum bem_request_state {
    BEM_REQ_QUEUED = 0, BEM_REQ_PREPARING = 1, BEM_REQ_RUNNING = 2, BEM_REQ_DONE = 3,
    BEM_REQ_FAILED = 4, BEM_REQ_CANCELLED = 5
};

/* One request: mesh (copied at submit), operator, ACA settings and the host
 * vector x of the product (n_triangles f64 for k == 0, complex128 otherwise).
 * reuse > 0 makes it a product-only request: apply the resident matrix that
 * request `reuse` of this server assembled (its op, k, aca_eps and prec; the
 * mesh fields are ignored except n_triangles, the length of x).  It waits
 * while that request is still running, and fails with BEM_E_STATE if the
 * matrix is no longer resident (evicted, or its request failed). */
typedef struct {
    const double *vertices;
    int64_t n_vertices;
    const int32_t *triangles;
    int64_t n_triangles;
    int32_t op;
    double k;
    double aca_eps;
    int32_t prec;
    int32_t leaf_size;
    double eta;
    const void *x;
    double dry_run_ms;   /* duration of the simulated device work (dry-run servers) */
    int64_t reuse;       /* 0: assemble; > 0: id of the request whose matrix to apply */
} bem_request;

typedef struct {
    int32_t state;              /* bem_request_state */
    int32_t status;             /* bem_status of the request (BEM_OK while pending) */
    double t_submit_ms;         /* steady-clock times in ms */
    double t_admit_ms;
    double t_done_ms;
    int64_t reserved_bytes;     /* HBM reserved for the request while it ran */
    int64_t integrals;          /* entries evaluated: near field + ACA requests */
    double assembly_ms;         /* device time of the assembly */
    int32_t launch_requests;    /* requests whose blocks shared its ACA launch (0: none ran) */
    int32_t reused;             /* 1: applied a resident matrix, nothing assembled */
    double t_ready_ms;          /* host part (trees) done, waiting for admission */
    double t_launch_ms;         /* its batch's device work enqueued */
} bem_request_info;

typedef struct {
    int64_t submitted, completed, failed, cancelled;
    int64_t queued, running;
    int64_t reserved_bytes;      /* currently reserved: running requests + resident matrices */
    int64_t peak_reserved_bytes; /* never above the budget */
    int64_t budget_bytes;
    int64_t resident;            /* matrices kept on the device, and their bytes */
    int64_t resident_bytes;
    int64_t evictions;           /* resident matrices freed for admissions */
    int64_t reuse_hits;          /* product-only requests served from a resident matrix */
    int64_t aca_launches;        /* ACA launches run, and the requests they held in all */
    int64_t aca_launch_requests;
    int64_t max_launch_requests; /* most requests in one ACA launch */
} bem_server_stats;

/* Creates a server on the current device with `max_slots` host threads for
 * the trees (1..64); at most max_slots requests run at once.  A request is
 * admitted, in arrival order, once its device bytes (geometry, tree, dense
 * blocks, factor pool of four 4-column chunks per admissible block, vectors)
 * fit next to the running requests and resident matrices (idle resident
 * matrices are evicted, least recently used first, to make room); one that
 * alone exceeds the budget fails with BEM_E_OOM.  flags: BEM_SERVER_DRY_RUN
 * runs the host logic only (no CUDA call; reserved bytes = 1024 per
 * triangle; a batch takes the longest dry_run_ms of its requests; y = x). */
int bem_server_create(int64_t hbm_budget_bytes, int32_t max_slots, int32_t flags,
                      bem_server *out);

/* Queues a request (inputs are copied) and returns its id. */
int bem_server_submit(bem_server server, const bem_request *req, int64_t *req_id);

/* State and times of a request that has not been collected yet. */
int bem_server_poll(bem_server server, int64_t req_id, bem_request_info *info);

/* Waits up to timeout_ms (< 0: no limit) for a request to finish.  When it
 * has finished, copies its product into host `y` (may be NULL), fills *info,
 * releases the request and returns its status; otherwise returns
 * BEM_E_TIMEOUT and keeps it. */
int bem_server_wait(bem_server server, int64_t req_id, int64_t timeout_ms,
                    bem_request_info *info, void *y);

/* Cancels a request that has not been admitted yet (BEM_E_STATE once it
 * has). */
int bem_server_cancel(bem_server server, int64_t req_id);

int bem_server_stats_get(bem_server server, bem_server_stats *out);

/* Cancels queued requests, waits for running ones, joins the threads and
 * frees the resident matrices. */
int bem_server_destroy(bem_server server);

#ifdef __cplusplus
}
#endif

#endif /* BEM_H */
