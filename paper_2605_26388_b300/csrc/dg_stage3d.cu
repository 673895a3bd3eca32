// dg_stage3d.cu -- single-instance launches of the fused stage kernel, 3D degrees.
#include "dg_stage_ec3.cuh"

namespace dg {

template <int DIM, int N, bool EC, class R>
struct GridSize {
  static int ctas;
};
template <int DIM, int N, bool EC, class R>
int GridSize<DIM, N, EC, R>::ctas = 0;

template <int DIM, int N, bool EC, class R>
static cudaError_t prepare_one() {
  using K = EulerStage<DIM, N, EC, R>;
  cudaError_t e = cudaFuncSetAttribute(k_euler_stage<DIM, N, EC, R>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)K::smem_bytes());
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_euler_stage<DIM, N, EC, R>, K::T,
                                                    K::smem_bytes());
  if (e != cudaSuccess) return e;
  GridSize<DIM, N, EC, R>::ctas = sms * (per_sm > 0 ? per_sm : 1);
  return cudaSuccess;
}

template <int DIM, int N, bool EC, class R>
static cudaError_t launch_one(const StageArgs& a, cudaStream_t s) {
  using K = EulerStage<DIM, N, EC, R>;
  const int groups = (a.inst.n_elem + K::EPB - 1) / K::EPB;
  if (groups == 0) return cudaSuccess;
  if (GridSize<DIM, N, EC, R>::ctas == 0) {
    cudaError_t e = prepare_one<DIM, N, EC, R>();
    if (e != cudaSuccess) return e;
  }
  const int blocks = groups < GridSize<DIM, N, EC, R>::ctas ? groups : GridSize<DIM, N, EC, R>::ctas;
  k_euler_stage<DIM, N, EC, R><<<blocks, K::T, K::smem_bytes(), s>>>(a);
  return cudaGetLastError();
}

// The two-point form of elements with 64 or more nodes: the run-walking kernel (EC3).
template <int N, class R, int SPEC>
struct EC3Grid {
  static int ctas;
};
template <int N, class R, int SPEC>
int EC3Grid<N, R, SPEC>::ctas = 0;

template <int N, class R, int SPEC>
static cudaError_t prepare_ec3_s() {
  using K = EC3<N, R, SPEC>;
  cudaError_t e = cudaFuncSetAttribute(k_euler_ec3<N, R, SPEC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)K::smem_bytes());
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_euler_ec3<N, R, SPEC>, K::T, K::smem_bytes());
  if (e != cudaSuccess) return e;
  EC3Grid<N, R, SPEC>::ctas = sms * (per_sm > 0 ? per_sm : 1);
  return cudaSuccess;
}

template <int N, class R>
static cudaError_t prepare_ec3() {
  cudaError_t e = prepare_ec3_s<N, R, 0>();
  if (e == cudaSuccess) e = prepare_ec3_s<N, R, 1>();
  if (e == cudaSuccess) e = prepare_ec3_s<N, R, 2>();
  return e;
}

template <int N, class R, int SPEC>
static cudaError_t launch_ec3_s(const StageArgs& a, cudaStream_t s) {
  using K = EC3<N, R, SPEC>;
  // the runs of KRUN elements per row (a lower bound of the kernel's run count, which splits
  // the last rows into shorter runs): every CTA's first run exists
  const int nseg = (a.inst.nel[0] + K::KRUN - 1) / K::KRUN;
  const long long runs = (long long)nseg * a.inst.nel[1] * a.inst.nel[2];
  if (a.inst.n_elem == 0) return cudaSuccess;
  if (EC3Grid<N, R, SPEC>::ctas == 0) {
    cudaError_t e = prepare_ec3_s<N, R, SPEC>();
    if (e != cudaSuccess) return e;
  }
  const int blocks = runs < EC3Grid<N, R, SPEC>::ctas ? (int)runs : EC3Grid<N, R, SPEC>::ctas;
  k_euler_ec3<N, R, SPEC><<<blocks, K::T, K::smem_bytes(), s>>>(a);
  return cudaGetLastError();
}

// the plain stage update on periodic meshes with the HLLC flux (no domain faces, one surface
// flux, no RK54 sum, floor or shock flag) takes the specialisations without those branches:
// SPEC 1 for the stages that read U^n, SPEC 2 for the first stage
template <int N, class R>
static cudaError_t launch_ec3(const StageArgs& a, cudaStream_t s) {
  if (!a.inst.nonper && a.surface == 1 && a.mode == 1 && !a.acc && !a.floor_on && !a.alpha)
    return a.need_un ? launch_ec3_s<N, R, 1>(a, s) : launch_ec3_s<N, R, 2>(a, s);
  return launch_ec3_s<N, R, 0>(a, s);
}

template <int DIM, int N>
static cudaError_t launch_dn(int ec, int fp32, const StageArgs* a, cudaStream_t s) {
  constexpr bool kEC3 = DIM == 3 && N >= 3;
  if (!a) {
    if (ec) {
      if constexpr (kEC3) return fp32 ? prepare_ec3<N, float>() : prepare_ec3<N, double>();
      return fp32 ? prepare_one<DIM, N, true, float>() : prepare_one<DIM, N, true, double>();
    }
    return fp32 ? prepare_one<DIM, N, false, float>() : prepare_one<DIM, N, false, double>();
  }
  if (ec) {
    if constexpr (kEC3) return fp32 ? launch_ec3<N, float>(*a, s) : launch_ec3<N, double>(*a, s);
    return fp32 ? launch_one<DIM, N, true, float>(*a, s) : launch_one<DIM, N, true, double>(*a, s);
  }
  return fp32 ? launch_one<DIM, N, false, float>(*a, s) : launch_one<DIM, N, false, double>(*a, s);
}

cudaError_t dispatch_stage_3d(int N, int ec, int fp32, const StageArgs* a, cudaStream_t s) {
  switch (N) {
    case 1: return launch_dn<3, 1>(ec, fp32, a, s);
    case 2: return launch_dn<3, 2>(ec, fp32, a, s);
    case 3: return launch_dn<3, 3>(ec, fp32, a, s);
    case 4: return launch_dn<3, 4>(ec, fp32, a, s);
    case 5: return launch_dn<3, 5>(ec, fp32, a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace dg
