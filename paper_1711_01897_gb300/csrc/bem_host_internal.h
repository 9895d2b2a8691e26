// Staged creation of meshes and H-matrices (host part, then device part on a
// given stream) for the request server.  Internal; not part of the C ABI.
#pragma once

#include "../../include/bem.h"
#include "bem_internal.h"

namespace bem {

int mesh_create_impl(const double *vertices, int64_t n_vertices, const int32_t *triangles,
                     int64_t n_triangles, cudaStream_t st, bem_mesh *out);
int mesh_upload(bem_mesh mesh, cudaStream_t st);
void mesh_free_synced(bem_mesh mesh);
int hmat_build_tree_impl(bem_mesh mesh, int32_t leaf_size, double eta, cudaStream_t st,
                         bem_hmat *out, int32_t space = BEM_P0);
int hmat_upload(bem_hmat hmat, cudaStream_t st);
int64_t hmat_device_bytes(bem_hmat hmat, bool cplx);
void hmat_free_synced(bem_hmat hmat);

}  // namespace bem
