// dg_kernels.cu -- dispatch of the stage kernels over (dim, degree), the time-step
// reduction and the flux probe kernel.
#include "dg_stage.cuh"

namespace dg {

int grid_cap() {
  static int cap[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148 * 16;
  if (!cap[dev]) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 148;
    cap[dev] = 16 * sms;
  }
  return cap[dev];
}

cudaError_t dispatch_stage_2d(int N, int ec, int fp32, const StageArgs* a, cudaStream_t s);
cudaError_t dispatch_stage_3d(int N, int ec, int fp32, const StageArgs* a, cudaStream_t s);
cudaError_t dispatch_batched_2d(int group_scale, int ec, int fp32, int ctas_per_sm, const StageArgs* a,
                                cudaStream_t s);
cudaError_t dispatch_batched_3d(int group_scale, int ec, int fp32, int ctas_per_sm, const StageArgs* a,
                                cudaStream_t s);

static cudaError_t dispatch(int dim, int N, int ec, int fp32, const StageArgs* a, cudaStream_t s) {
  if (dim == 2) return dispatch_stage_2d(N, ec, fp32, a, s);
  if (dim == 3) return dispatch_stage_3d(N, ec, fp32, a, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_euler_stage_batched(int dim, int ec, int fp32, int group_scale, int ctas_per_sm,
                                       const StageArgs& a, cudaStream_t s) {
  if (dim == 2) return dispatch_batched_2d(group_scale, ec, fp32, ctas_per_sm, &a, s);
  if (dim == 3) return dispatch_batched_3d(group_scale, ec, fp32, ctas_per_sm, &a, s);
  return cudaErrorInvalidValue;
}

cudaError_t prepare_euler_stage_batched(int dim, int ec, int fp32, int group_scale) {
  if (dim == 2) return dispatch_batched_2d(group_scale, ec, fp32, 0, nullptr, nullptr);
  if (dim == 3) return dispatch_batched_3d(group_scale, ec, fp32, 0, nullptr, nullptr);
  return cudaErrorInvalidValue;
}

int batched_group(int dim, int N, int group_scale) {
  int np = 1, nfn = 1;
  for (int l = 0; l < dim; ++l) np *= (N + 1);
  for (int l = 1; l < dim; ++l) nfn *= (N + 1);
  const int w = np > 2 * dim * nfn ? np : 2 * dim * nfn;  // the kernels' base group (Geo::EPB)
  const int epb = w >= 96 ? 1 : 128 / w;
  return epb * group_scale;
}

bool have_kernels(int dim, int N) {
  return (dim == 2 && N >= 1 && N <= 7) || (dim == 3 && N >= 1 && N <= 5);
}

cudaError_t launch_euler_stage(int dim, int N, int ec, int fp32, const StageArgs& a,
                               cudaStream_t s) {
  return dispatch(dim, N, ec, fp32, &a, s);
}

cudaError_t prepare_euler_stage(int dim, int N, int ec, int fp32) {
  return dispatch(dim, N, ec, fp32, nullptr, nullptr);
}

// ---------------------------------------------------------------------------------------
// Largest signal speed |u| + a (Eq. dt_hyp), FP64, as a reduction code (speed_bits): block
// maximum, then one atomicMax on the unsigned pattern.
// ---------------------------------------------------------------------------------------
template <int DIM>
__global__ void k_max_speed(const double* U, long long stride, long long base, long long n,
                            double gamma, unsigned long long* out) {
  unsigned long long lam = 0ull;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const unsigned long long b = euler_speed_bits<DIM>(U, stride, base + q, gamma);
    lam = b > lam ? b : lam;
  }
  lam = block_max_u64(lam);
  if (threadIdx.x == 0) atomicMax(out, lam);
}

cudaError_t launch_max_speed(int dim, const double* U, long long stride, long long base,
                             long long n_nodes, double gamma, unsigned long long* lam_bits,
                             cudaStream_t s) {
  if (n_nodes <= 0) return cudaSuccess;
  long long blocks = (n_nodes + 255) / 256;
  const int cap = grid_cap();
  if (blocks > cap) blocks = cap;
  if (dim == 2) k_max_speed<2><<<(int)blocks, 256, 0, s>>>(U, stride, base, n_nodes, gamma, lam_bits);
  else k_max_speed<3><<<(int)blocks, 256, 0, s>>>(U, stride, base, n_nodes, gamma, lam_bits);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Two-point flux evaluation for tests (AoS pairs).
// ---------------------------------------------------------------------------------------
template <int DIM, int L, class R>
__device__ void two_point_one(int kind, const double* uL, const double* uR, double gamma,
                              double p_ref, double* F) {
  R a[DIM + 2], b[DIM + 2], f[DIM + 2];
  double a64[DIM + 2], b64[DIM + 2];
#pragma unroll
  for (int v = 0; v < DIM + 2; ++v) {
    a64[v] = uL[v];
    b64[v] = uR[v];
    a[v] = Ar<R>::load(a64[v]);
    b[v] = Ar<R>::load(b64[v]);
  }
  const R pr = R(p_ref), gm = R(gamma), igm1 = R(1) / (gm - R(1));
  const R hgm1 = R(0.5 * (gamma - 1.0));
  const Prim<DIM, R> pa = prims<DIM>(a, pdev<DIM>(a64, a, gamma - 1.0, p_ref, hgm1), pr);
  const Prim<DIM, R> pb = prims<DIM>(b, pdev<DIM>(b64, b, gamma - 1.0, p_ref, hgm1), pr);
  if (kind < 0) ec_flux<DIM, L>(pa, pb, igm1, pr, f);
  else surface_flux<DIM, L>(kind, a, pa, b, pb, gm, igm1, pr, f);
#pragma unroll
  for (int v = 0; v < DIM + 2; ++v) F[v] = Ar<R>::widen(f[v]);
}

template <int DIM, class R>
__global__ void k_two_point(int kind, int l, int n, double gamma, double p_ref, const double* uL,
                            const double* uR, double* F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int nv = DIM + 2;
  if (l == 0) two_point_one<DIM, 0, R>(kind, uL + i * nv, uR + i * nv, gamma, p_ref, F + i * nv);
  else if (l == 1) two_point_one<DIM, 1, R>(kind, uL + i * nv, uR + i * nv, gamma, p_ref, F + i * nv);
  else if constexpr (DIM == 3) two_point_one<DIM, 2, R>(kind, uL + i * nv, uR + i * nv, gamma, p_ref, F + i * nv);
}

cudaError_t launch_two_point(int dim, int fp32, int kind, int l, int n, double gamma, double p_ref,
                             const double* uL, const double* uR, double* F, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (n + 127) / 128;
  if (dim == 2) {
    if (fp32) k_two_point<2, float><<<blocks, 128, 0, s>>>(kind, l, n, gamma, p_ref, uL, uR, F);
    else k_two_point<2, double><<<blocks, 128, 0, s>>>(kind, l, n, gamma, p_ref, uL, uR, F);
  } else {
    if (fp32) k_two_point<3, float><<<blocks, 128, 0, s>>>(kind, l, n, gamma, p_ref, uL, uR, F);
    else k_two_point<3, double><<<blocks, 128, 0, s>>>(kind, l, n, gamma, p_ref, uL, uR, F);
  }
  return cudaGetLastError();
}

}  // namespace dg
