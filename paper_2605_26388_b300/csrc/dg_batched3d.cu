// dg_batched3d.cu -- instantiation of the batched persistent stage kernel, 3D.
#include "dg_batched.cuh"

namespace dg {

cudaError_t dispatch_batched_3d(int group_scale, int ec, int fp32, int ctas_per_sm,
                                const StageArgs* a, cudaStream_t s) {
  if (group_scale == 1) return batched_dispatch<3, 1>(ec, fp32, ctas_per_sm, a, s);
  return cudaErrorInvalidValue;
}

}  // namespace dg
