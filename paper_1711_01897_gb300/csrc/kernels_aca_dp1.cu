// The persistent ACA (aca_kernel.cuh) for DP1 H-matrices: three local dofs
// per triangle, block ranges in dof units, every requested row or column
// evaluated as the matching row or column of the element pairs' local
// matrices.  A separate translation unit so that it compiles alongside the
// P0 instantiations.
#include "aca_kernel.cuh"

namespace bem {

cudaError_t launch_aca_dp1(const DevGeom &g, const QuadRule &rule, int op, double k, int prec,
                           double eps, FarBlock *blocks, FarChunks *chunks, int64_t n_big,
                           int64_t n_small, int64_t max_m_big, int64_t max_m_small,
                           void *pool_data, Pool *pool, AcaQueue *queue, int num_sms,
                           cudaStream_t st)
{
    const bool cplx = k != 0.0;
#define BEM_ACA3(O, C, Pp)                                                                    \
    if (op == O && cplx == C && prec == Pp)                                                   \
        return aca_launch<O, C, Pp, 3>(g, rule, k, eps, blocks, chunks, n_big, n_small, 0,   \
                                       max_m_big, max_m_small, pool_data, pool, queue,       \
                                       num_sms, st);
    BEM_ACA3(0, false, 0) BEM_ACA3(0, false, 1) BEM_ACA3(0, true, 0) BEM_ACA3(0, true, 1)
    BEM_ACA3(1, false, 0) BEM_ACA3(1, false, 1) BEM_ACA3(1, true, 0) BEM_ACA3(1, true, 1)
    BEM_ACA3(2, false, 0) BEM_ACA3(2, false, 1) BEM_ACA3(2, true, 0) BEM_ACA3(2, true, 1)
#undef BEM_ACA3
    return cudaErrorInvalidValue;
}

}  // namespace bem
