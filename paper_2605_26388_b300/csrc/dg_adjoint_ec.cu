// dg_adjoint_ec.cu -- the adjoint kernel's instantiations for the two-point volume form
// (Eq. vol_split with Ranocha's flux, App. A) and the HLLC surface flux: a separate
// translation unit, so that they compile beside the Rusanov ones.
#include "dg_adjoint.cuh"

namespace dg {

cudaError_t launch_vjp_ec(int sch, int dim, int N, int fp32, const VjpArgs& a, cudaStream_t s, int* blocks) {
  switch (sch) {
    case 1: return launch_vjp_sch<1>(dim, N, fp32, a, s, blocks);
    case 2: return launch_vjp_sch<2>(dim, N, fp32, a, s, blocks);
    case 3: return launch_vjp_sch<3>(dim, N, fp32, a, s, blocks);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dg
