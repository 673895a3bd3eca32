// dg_batched.cuh -- the batched persistent stage kernel (one launch per RK stage for many
// instances), shared by the 2D and 3D translation units.
#pragma once

#include "dg_stage.cuh"

namespace dg {

// staging buffers of the batched kernel (2: one item prefetched; 3: two)
#ifndef DG_BATCHED_PIPE
#define DG_BATCHED_PIPE 2
#endif
constexpr int kBatchedPipe = DG_BATCHED_PIPE;


// ---------------------------------------------------------------------------------------
// Batched persistent launch: one launch per RK stage for many instances of one dimension
// and uneven size and degree (1..5).  The host builds a list of work items (instance, element
// group), heaviest first; each CTA walks a strided slice of it, dispatching on the item's
// degree, and prefetches the next item's inputs (whatever its degree) while computing the
// current one.  Shared memory and threads are sized for the largest degree.
// ---------------------------------------------------------------------------------------
template <int DIM, bool EC, class R, int GS, int N = 1>
struct BMax {
  using K = EulerStage<DIM, N, EC, R, GS>;
  using Nx = BMax<DIM, EC, R, GS, N + 1>;
  static constexpr int st = cmax(K::ST_SIZE, Nx::st);
  static constexpr int r = cmax(K::R_SIZE, Nx::r);
  static constexpr int nb = cmax(K::EPB * K::NF, Nx::nb);
  static constexpr int t = cmax(K::T, Nx::t);
};
// the batched kernel covers degrees 1..5 in both dimensions
template <int DIM, bool EC, class R, int GS>
struct BMax<DIM, EC, R, GS, 6> {
  static constexpr int st = 0, r = 0, nb = 0, t = 0;
};

// PIPE staging buffers: the inputs of the next PIPE-1 items are in flight while one computes.
template <int DIM, bool EC, class R, int GS>
struct Batched {
  using M = BMax<DIM, EC, R, GS>;
  static constexpr int MST = M::st, MR = M::r, MNB = M::nb, BT = M::t;
  static constexpr int PIPE = kBatchedPipe;
  static constexpr size_t smem_bytes() {
    return sizeof(double) * PIPE * (size_t)MST + sizeof(R) * (size_t)MR + sizeof(int) * (PIPE * MNB + 4);
  }
};

template <int P>
__device__ __forceinline__ void cp_async_wait_keep() {  // all but the newest P groups done
  asm volatile("cp.async.wait_group %0;\n" ::"n"(P) : "memory");
}

#define DG_ON_DEGREE(NVAL, ...)                                               \
  switch (NVAL) {                                                             \
    case 1: { using K = EulerStage<DIM, 1, EC, R, GS>; __VA_ARGS__; } break; \
    case 2: { using K = EulerStage<DIM, 2, EC, R, GS>; __VA_ARGS__; } break; \
    case 3: { using K = EulerStage<DIM, 3, EC, R, GS>; __VA_ARGS__; } break; \
    case 4: { using K = EulerStage<DIM, 4, EC, R, GS>; __VA_ARGS__; } break; \
    case 5: { using K = EulerStage<DIM, 5, EC, R, GS>; __VA_ARGS__; } break; \
    default: break;                                                           \
  }

template <int DIM, bool EC, class R, int GS>
__global__ void __launch_bounds__(Batched<DIM, EC, R, GS>::BT, (Batched<DIM, EC, R, GS>::BT <= 128 ? (sizeof(R) == 4 ? 6 : 4) : 2))
    k_euler_stage_batched(const StageArgs A) {
  using B = Batched<DIM, EC, R, GS>;
  constexpr int P = B::PIPE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* st = reinterpret_cast<double*>(smem_raw);
  R* sm = reinterpret_cast<R*>(st + P * B::MST);
  int* nb = reinterpret_cast<int*>(sm + B::MR);
  const bool need_un = A.need_un != 0;
  const int k0 = blockIdx.x, step = gridDim.x;
  // prologue: neighbour tables and copies of the first P-1 items (slot/buffer j for item j)
  for (int j = 0; j < P - 1; ++j) {
    const int kj = k0 + j * step;
    if (kj < A.n_items) {
      const int2 item = A.items[kj];
      const InstArgs& I = A.insts[item.x];
      DG_ON_DEGREE(I.N, K::fill_nb(I, item.y, nb + j * B::MNB));
    }
  }
  __syncthreads();
  for (int j = 0; j < P - 1; ++j) {
    const int kj = k0 + j * step;
    if (kj < A.n_items) {
      const int2 item = A.items[kj];
      const InstArgs& I = A.insts[item.x];
      DG_ON_DEGREE(I.N, K::issue(A, I, K::role(), item.y, st + j * B::MST, nb + j * B::MNB, need_un));
    }
    cp_async_commit();
  }
  int it = 0;
  for (int k = k0; k < A.n_items; k += step, ++it) {
    const int b = it % P;
    const int bf = (it + P - 1) % P;  // buffer of the item fetched now (last read by item it-1)
    const int kf = k + (P - 1) * step;
    if (kf < A.n_items) {
      const int2 item = A.items[kf];
      const InstArgs& I = A.insts[item.x];
      DG_ON_DEGREE(I.N, K::fill_nb(I, item.y, nb + bf * B::MNB));
    }
    __syncthreads();  // neighbour table ready; the previous item no longer reads buffer bf
    if (kf < A.n_items) {
      const int2 item = A.items[kf];
      const InstArgs& I = A.insts[item.x];
      DG_ON_DEGREE(I.N, K::issue(A, I, K::role(), item.y, st + bf * B::MST, nb + bf * B::MNB, need_un));
    }
    cp_async_commit();
    cp_async_wait_keep<P - 1>();
    const int2 item = A.items[k];
    const InstArgs& I = A.insts[item.x];
    DG_ON_DEGREE(I.N, K::load_ops(sm, A.dv_table + I.N * (kMaxN + 1) * (kMaxN + 1), I));
    __syncthreads();  // item k's copies and operators are visible
    DG_ON_DEGREE(I.N, K::compute(A, I, sm, K::role(), item.y, st + b * B::MST, need_un));
  }
}
#undef DG_ON_DEGREE

template <int DIM, bool EC, class R, int GS>
struct BatchGrid {
  static int ctas_per_sm;
  static int sms;
};
template <int DIM, bool EC, class R, int GS>
int BatchGrid<DIM, EC, R, GS>::ctas_per_sm = 0;
template <int DIM, bool EC, class R, int GS>
int BatchGrid<DIM, EC, R, GS>::sms = 0;

template <int DIM, bool EC, class R, int GS>
static cudaError_t prepare_batched_one() {
  using B = Batched<DIM, EC, R, GS>;
  cudaError_t e = cudaFuncSetAttribute(k_euler_stage_batched<DIM, EC, R, GS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)B::smem_bytes());
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_euler_stage_batched<DIM, EC, R, GS>,
                                                    B::BT, B::smem_bytes());
  if (e != cudaSuccess) return e;
  BatchGrid<DIM, EC, R, GS>::ctas_per_sm = per_sm > 0 ? per_sm : 1;
  BatchGrid<DIM, EC, R, GS>::sms = sms;
  return cudaSuccess;
}

template <int DIM, bool EC, class R, int GS>
static cudaError_t launch_batched_one(const StageArgs* a, int ctas_per_sm, cudaStream_t s) {
  using B = Batched<DIM, EC, R, GS>;
  if (!a || BatchGrid<DIM, EC, R, GS>::sms == 0) {
    cudaError_t e = prepare_batched_one<DIM, EC, R, GS>();
    if (e != cudaSuccess || !a) return e;
  }
  if (a->n_items <= 0) return cudaSuccess;
  int per = BatchGrid<DIM, EC, R, GS>::ctas_per_sm;
  if (ctas_per_sm > 0 && ctas_per_sm < per) per = ctas_per_sm;
  int blocks = BatchGrid<DIM, EC, R, GS>::sms * per;
  if (blocks > a->n_items) blocks = a->n_items;
  k_euler_stage_batched<DIM, EC, R, GS><<<blocks, B::BT, B::smem_bytes(), s>>>(*a);
  return cudaGetLastError();
}

template <int DIM, int GS>
static cudaError_t batched_dispatch(int ec, int fp32, int ctas_per_sm, const StageArgs* a,
                                    cudaStream_t s) {
  if (ec) return fp32 ? launch_batched_one<DIM, true, float, GS>(a, ctas_per_sm, s)
                      : launch_batched_one<DIM, true, double, GS>(a, ctas_per_sm, s);
  return fp32 ? launch_batched_one<DIM, false, float, GS>(a, ctas_per_sm, s)
              : launch_batched_one<DIM, false, double, GS>(a, ctas_per_sm, s);
}

}  // namespace dg
