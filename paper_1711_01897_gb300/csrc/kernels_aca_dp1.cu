// The persistent ACA (aca_kernel.cuh) for DP1 H-matrices: three local dofs
// per triangle, block ranges in dof units, every requested row or column
// evaluated as the matching row or column of the element pairs' local
// matrices.  A separate translation unit so that it compiles alongside the
// P0 instantiations.
#include "aca_kernel.cuh"

namespace bem {

cudaError_t launch_aca_dp1(const AcaWork &w, const QuadRule &rule, int op, bool cplx, int prec,
                           AcaQueue *queue, int num_sms, cudaStream_t st)
{
    AcaWork w3 = w;
    w3.n[kShapeHalf] = w3.n[kShapeQuarter] = w3.n[kShapeLane] = 0;
#define BEM_ACA3(O, C, Pp)                                  \
    if (op == O && cplx == C && prec == Pp)                 \
        return aca_launch<O, C, Pp, 3>(w3, rule, queue, num_sms, st);
    BEM_ACA3(0, false, 0) BEM_ACA3(0, false, 1) BEM_ACA3(0, true, 0) BEM_ACA3(0, true, 1)
    BEM_ACA3(1, false, 0) BEM_ACA3(1, false, 1) BEM_ACA3(1, true, 0) BEM_ACA3(1, true, 1)
    BEM_ACA3(2, false, 0) BEM_ACA3(2, false, 1) BEM_ACA3(2, true, 0) BEM_ACA3(2, true, 1)
#undef BEM_ACA3
    return cudaErrorInvalidValue;
}

}  // namespace bem
