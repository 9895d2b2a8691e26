// The persistent ACA (aca_kernel.cuh) for P0 H-matrices in BEM_MIXED_SP:
// the norm of S_k takes its dot products in FP32 (the stopping test only);
// quadrature, pivots and residual updates as in BEM_MIXED.  A separate
// translation unit so that it compiles alongside the other instantiations.
#include "aca_kernel.cuh"

namespace bem {

cudaError_t launch_aca_sp(const AcaWork &w, const QuadRule &rule, int op, bool cplx,
                          AcaQueue *queue, int num_sms, cudaStream_t st, bool rules)
{
    if (rules && !cplx) {
        if (op == 0) return aca_launch<0, false, 2, 1, true>(w, rule, queue, num_sms, st);
        if (op == 1) return aca_launch<1, false, 2, 1, true>(w, rule, queue, num_sms, st);
        if (op == 2) return aca_launch<2, false, 2, 1, true>(w, rule, queue, num_sms, st);
    }
#define BEM_ACA_SP(O, C)                                    \
    if (op == O && cplx == C) return aca_launch<O, C, 2, 1>(w, rule, queue, num_sms, st);
    BEM_ACA_SP(0, false) BEM_ACA_SP(0, true) BEM_ACA_SP(1, false) BEM_ACA_SP(1, true)
    BEM_ACA_SP(2, false) BEM_ACA_SP(2, true)
#undef BEM_ACA_SP
    return cudaErrorInvalidValue;
}

}  // namespace bem
