// dg_adjoint.cu -- launches of the adjoint (vector-Jacobian product) of the residual for the
// strong or weak volume form with the Rusanov flux, the fixed-order reduction of the gamma
// partials and the reverse Shu-Osher combinations; the kernel is in dg_adjoint.cuh, its
// two-point and HLLC instantiations in dg_adjoint_ec.cu.
#include "dg_adjoint.cuh"

namespace dg {

// sum of n partials in a fixed order (one block), added to *acc
__global__ void k_sum_partials(const double* part, int n, double* acc) {
  __shared__ double red[256];
  double s = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) s += part[k];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *acc += red[0];
}

int vjp_blocks(int dim, int N, long long n_elem) {
  int np = 1, nfn = 1;
  for (int l = 0; l < dim; ++l) np *= (N + 1);
  for (int l = 1; l < dim; ++l) nfn *= (N + 1);
  const int w = np > 2 * dim * nfn ? np : 2 * dim * nfn;
  const int epb = w >= 96 ? 1 : 128 / w;
  return (int)((n_elem + epb - 1) / epb);
}

cudaError_t launch_rhs_vjp(int dim, int N, int fp32, int sch, const VjpArgs& a, double* gacc, cudaStream_t s) {
  int blocks = 0;
  const cudaError_t e = sch == 0 ? launch_vjp_sch<0>(dim, N, fp32, a, s, &blocks)
                                 : launch_vjp_ec(sch, dim, N, fp32, a, s, &blocks);
  if (e != cudaSuccess || blocks == 0) return e;
  k_sum_partials<<<1, 256, 0, s>>>(a.gpart, blocks, gacc);
  return cudaGetLastError();
}

__global__ void k_combine(const CombineArgs a) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.n;
       i += (long long)gridDim.x * blockDim.x) {
    double y = 0.0;
    for (int j = 0; j < a.m; ++j) y = fma(a.c[j], a.x[j][i], y);
    a.y[i] = y;
  }
}

cudaError_t launch_combine(const CombineArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const long long want = (a.n + 255) / 256;
  const unsigned grid = (unsigned)(want < 148 * 8 ? want : 148 * 8);
  k_combine<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace dg
