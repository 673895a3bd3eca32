// dg_peaks.cu -- arithmetic throughput of this GPU's pipes, measured with CUDA events.
//
// The stage kernels are bound by instruction issue and by the FP64 pipe rather than by
// HBM alone, so their rooflines need the measured rates of the instructions they issue.
// Each probe runs independent dependency chains (CH per thread, enough to cover the pipe
// latency) on a grid of 8 CTAs of 256 threads per SM, and times a launch after a warm-up
// launch; the result is the best of three.  No clock or device setting is touched.
#include <cuda_runtime.h>

#include "../../include/dgsem.h"

namespace {

constexpr int kThreads = 256, kCtasPerSm = 8;

template <int KIND>
struct Op;
template <>
struct Op<0> {  // FP64 fused multiply-add
  using T = double;
  static __device__ __forceinline__ T f(T a, T m, T c) { return fma(a, m, c); }
  static constexpr int per = 1;
};
template <>
struct Op<1> {  // FP64 add
  using T = double;
  static __device__ __forceinline__ T f(T a, T, T c) { return __dadd_rn(a, c); }
  static constexpr int per = 1;
};
template <>
struct Op<2> {  // FP32 fused multiply-add
  using T = float;
  static __device__ __forceinline__ T f(T a, T m, T c) { return fmaf(a, m, c); }
  static constexpr int per = 1;
};
template <>
struct Op<3> {  // packed FP32x2 fused multiply-add (two FMAs per instruction)
  using T = float2;
  static __device__ __forceinline__ T f(T a, T m, T c) { return __ffma2_rn(a, m, c); }
  static constexpr int per = 2;
};
template <>
struct Op<4> {  // FP32 approximate reciprocal (the special-function unit)
  using T = float;
  static __device__ __forceinline__ T f(T a, T, T c) {
    float r;
    asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r + c;  // keeps the chain; counted as one reciprocal (the add issues elsewhere)
  }
  static constexpr int per = 1;
};
template <>
struct Op<5> {  // FP32 add
  using T = float;
  static __device__ __forceinline__ T f(T a, T, T c) { return __fadd_rn(a, c); }
  static constexpr int per = 1;
};

template <class T> __device__ __forceinline__ T mk(float x);
template <> __device__ __forceinline__ double mk<double>(float x) { return (double)x; }
template <> __device__ __forceinline__ float mk<float>(float x) { return x; }
template <> __device__ __forceinline__ float2 mk<float2>(float x) { return make_float2(x, x + 0.5f); }
__device__ __forceinline__ float sum1(double x) { return (float)x; }
__device__ __forceinline__ float sum1(float x) { return x; }
__device__ __forceinline__ float sum1(float2 x) { return x.x + x.y; }

template <int KIND, int CH>
__global__ void __launch_bounds__(kThreads) k_alu_chain(float* sink, int iters) {
  using O = Op<KIND>;
  using T = typename O::T;
  T a[CH];
#pragma unroll
  for (int k = 0; k < CH; ++k) a[k] = mk<T>(1.0f + 1e-3f * (threadIdx.x + k));
  const T m = mk<T>(0.999999f), c = mk<T>(1e-6f);
  for (int it = 0; it < iters; ++it) {
#pragma unroll 8
    for (int r = 0; r < 8; ++r) {
#pragma unroll
      for (int k = 0; k < CH; ++k) a[k] = O::f(a[k], m, c);
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < CH; ++k) s += sum1(a[k]);
  if (s == -1.0f) sink[blockIdx.x] = s;  // never true; keeps the chains live
}

template <int KIND, int CH>
cudaError_t time_kind(int sms, int iters, double* rate) {
  float* sink = nullptr;  // never written (the guard is false), but must be a valid pointer
  cudaError_t e = cudaMalloc(&sink, sizeof(float) * sms * kCtasPerSm);
  if (e != cudaSuccess) return e;
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  const int blocks = sms * kCtasPerSm;
  k_alu_chain<KIND, CH><<<blocks, kThreads>>>(sink, iters);
  float best = 1e30f;
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
    cudaEventRecord(t0);
    k_alu_chain<KIND, CH><<<blocks, kThreads>>>(sink, iters);
    cudaEventRecord(t1);
    e = cudaEventSynchronize(t1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (ms < best) best = ms;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  cudaFree(sink);
  const double ops = (double)blocks * kThreads * iters * 8.0 * CH * Op<KIND>::per;
  *rate = ops / (best * 1e-3);
  return e;
}

}  // namespace

extern "C" DG_API dg_status dg_alu_rate(int kind, double* ops_per_s) {
  if (!ops_per_s) return DG_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DG_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return DG_ECUDA;
  // iteration counts: about 10-40 ms per launch at the rates of a B300-class part
  cudaError_t e;
  switch (kind) {
    case 0: e = time_kind<0, 4>(sms, 2000, ops_per_s); break;
    case 1: e = time_kind<1, 4>(sms, 2000, ops_per_s); break;
    case 2: e = time_kind<2, 8>(sms, 40000, ops_per_s); break;
    case 3: e = time_kind<3, 8>(sms, 20000, ops_per_s); break;
    case 4: e = time_kind<4, 8>(sms, 10000, ops_per_s); break;
    case 5: e = time_kind<5, 8>(sms, 40000, ops_per_s); break;
    default: return DG_EINVAL;
  }
  return e == cudaSuccess ? DG_OK : DG_ECUDA;
}
