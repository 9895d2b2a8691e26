// Staged creation of meshes and H-matrices (host part, then device part on a
// given stream) for the request server.  Internal; not part of the C ABI.
#pragma once

#include <functional>
#include <vector>

#include "../../include/bem.h"
#include "bem_internal.h"

namespace bem {

int mesh_create_impl(const double *vertices, int64_t n_vertices, const int32_t *triangles,
                     int64_t n_triangles, cudaStream_t st, bem_mesh *out);
int mesh_upload(bem_mesh mesh, cudaStream_t st);
void mesh_free_synced(bem_mesh mesh);
int hmat_build_tree_impl(bem_mesh mesh, int32_t leaf_size, double eta, cudaStream_t st,
                         bem_hmat *out, int32_t space = BEM_P0, int32_t n_parts = 1,
                         int32_t part = 0);
int hmat_upload(bem_hmat hmat, cudaStream_t st);
int64_t hmat_device_bytes(bem_hmat hmat, bool cplx);
void hmat_free_synced(bem_hmat hmat);

// Stages of hmat_assemble, for launches over several matrices.  Each may
// throw on a CUDA error (callers run them inside a guard); the int-returning
// ones report argument errors as a status.
int assemble_begin(bem_hmat H, int32_t op, double k, double aca_eps, int32_t prec, cudaStream_t st);
void assemble_pool(bem_hmat H, cudaStream_t st);
void enqueue_near(bem_hmat H, cudaStream_t st, bool capturing);
void enqueue_finish(bem_hmat H, cudaStream_t st, bool capturing, bool mark_aca_end = true);
int enqueue_aca_fused(const std::vector<bem_hmat> &hs, cudaStream_t st, double sm_share = 1.0,
                      void *pinned = nullptr, size_t pinned_bytes = 0);
// true if the last launch ran out of factor pool (then hmat_assemble alone
// grows the pool and repeats)
bool assemble_overflowed(bem_hmat H);
// true if the tree has admissible blocks on a lower-order regular rule
bool hmat_has_rules(bem_hmat H);
void assemble_end(bem_hmat H, cudaStream_t st);
// runs f, turning the library's internal CUDA failures and host
// allocation failures into a status
int guarded_call(const std::function<int()> &f);

}  // namespace bem
