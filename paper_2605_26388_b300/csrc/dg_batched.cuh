// dg_batched.cuh -- the batched persistent stage kernel (one launch per RK stage for many
// instances), shared by the 2D and 3D translation units.
#pragma once

#include "dg_stage.cuh"

namespace dg {

// ---------------------------------------------------------------------------------------
// Batched persistent launch: one launch per RK stage for many instances of one dimension
// and uneven size and degree (1..5).  The host builds a list of work items (instance, element
// group), heaviest first; each CTA walks a strided slice of it, dispatching on the item's
// degree.  Shared memory and threads are sized for the largest degree.
//
// Nothing an item needs is read from global memory on the critical path: the instance
// arguments of the item three ahead are copied with cp.async into a ring of shared-memory
// slots (its index was loaded into a register one iteration earlier still), the volume
// operators of all degrees are held in shared memory for the whole launch, and the next
// item's neighbour table and coefficient tables are built from those copies before the one
// barrier per item that also publishes the current item's staged inputs.  The own state
// and U^n of the item two ahead are prefetched to L2 by lines (its group is a contiguous
// block of each variable); its neighbours' blocks are not (that measured slower).
// ---------------------------------------------------------------------------------------
template <int DIM, bool EC, class R, int GS, int N = 1>
struct BMax {
  using K = EulerStage<DIM, N, EC, R, GS>;
  using Nx = BMax<DIM, EC, R, GS, N + 1>;
  static constexpr int st = cmax(K::ST_SIZE, Nx::st);
  static constexpr int r = cmax(K::OFF_D, Nx::r);  // R area without the coefficient tables
  static constexpr int nd = cmax(K::ND, Nx::nd);
  static constexpr int nb = cmax(K::EPB * K::NF, Nx::nb);
  static constexpr int t = cmax(K::T, Nx::t);
};
// the batched kernel covers degrees 1..5 in both dimensions
template <int DIM, bool EC, class R, int GS>
struct BMax<DIM, EC, R, GS, 6> {
  static constexpr int st = 0, r = 0, nd = 0, nb = 0, t = 0;
};

template <int DIM, bool EC, class R, int GS>
struct Batched {
  using M = BMax<DIM, EC, R, GS>;
  static constexpr int MST = M::st, BT = M::t;
  static constexpr int MR = al4(M::r);                  // R area (16-byte multiple)
  static constexpr int MD = al4(M::nd);                 // one coefficient-table slot
  static constexpr int MNB = M::nb;
  static constexpr int NDV = (kMaxN + 1) * (kMaxN + 1);  // one volume operator (device table)
  // the operators of degrees 1..kMaxN packed: degree N at dv_off(N) = sum_{m=1}^{N-1} (m+1)^2,
  // (N+1)^2 values
  static __host__ __device__ constexpr int dv_off(int N) { return N * (N + 1) * (2 * N + 1) / 6 - 1; }
  static constexpr int DVS = dv_off(kMaxN + 1);
  static_assert(dv_off(1) == 0 && dv_off(2) == 4 && dv_off(kMaxN) + (kMaxN + 1) * (kMaxN + 1) == DVS,
                "packed operator offsets");
  static constexpr int RING = 4;                         // instance-argument slots (items it..it+3)
  static constexpr int ORING = 3;                        // coefficient-table slots (items it, it+1)
  static_assert(sizeof(InstArgs) % 16 == 0, "InstArgs is copied in 16-byte pieces");
  static constexpr int IA16 = (int)(sizeof(InstArgs) / 16);
  // layout: staging [2][MST] double | volume operators (packed) [DVS] double | instance
  // arguments [RING] | R area [MR] | coefficient tables [ORING][MD] | neighbours [2][MNB] int
  static constexpr size_t OFF_DV = sizeof(double) * 2 * (size_t)MST;
  static constexpr size_t OFF_IA = OFF_DV + sizeof(double) * (size_t)((DVS + 1) & ~1);
  static constexpr size_t OFF_R = OFF_IA + sizeof(InstArgs) * RING;
  static constexpr size_t OFF_OPS = OFF_R + sizeof(R) * (size_t)MR;
  static constexpr size_t OFF_NB = OFF_OPS + sizeof(R) * (size_t)ORING * MD;
  static constexpr size_t smem_bytes() { return OFF_NB + sizeof(int) * 2 * (size_t)MNB; }
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

// copy the instance arguments of item `item` into slot ia (threads 0..IA16-1, 16 bytes each)
template <class B>
__device__ __forceinline__ void copy_inst(const StageArgs& A, int2 item, InstArgs* ia) {
  const int t = threadIdx.x;
  if (t < B::IA16) {
    const char* src = reinterpret_cast<const char*>(A.insts + item.x) + 16 * t;
    char* dst = reinterpret_cast<char*>(ia) + 16 * t;
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
  }
}

template <int DIM, bool EC, class R, int GS>
__global__ void __launch_bounds__(Batched<DIM, EC, R, GS>::BT, (Batched<DIM, EC, R, GS>::BT <= 128 ? (sizeof(R) == 4 ? 6 : 4) : 2))
    k_euler_stage_batched(const StageArgs A) {
  using B = Batched<DIM, EC, R, GS>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* st = reinterpret_cast<double*>(smem_raw);
  double* sdv = reinterpret_cast<double*>(smem_raw + B::OFF_DV);
  InstArgs* sia = reinterpret_cast<InstArgs*>(smem_raw + B::OFF_IA);
  R* sm = reinterpret_cast<R*>(smem_raw + B::OFF_R);
  R* sops = reinterpret_cast<R*>(smem_raw + B::OFF_OPS);
  int* nb = reinterpret_cast<int*>(smem_raw + B::OFF_NB);
  __shared__ int2 sitem[B::RING];  // the item of each slot
  const bool need_un = A.need_un != 0;
  const int k0 = blockIdx.x, step = gridDim.x, n = A.n_items;
  const int t = threadIdx.x;
  if (k0 >= n) return;
  // volume operators of all degrees, for the whole launch
  for (int N = 1; N <= kMaxN; ++N)
    for (int q = t; q < (N + 1) * (N + 1); q += blockDim.x) sdv[B::dv_off(N) + q] = A.dv_table[N * B::NDV + q];
  // instance arguments of items 0..2 of this CTA's slice (slot j for item j)
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int kj = k0 + j * step;
    if (kj < n) {
      const int2 item = A.items[kj];
      copy_inst<B>(A, item, sia + j);
      if (t == 0) sitem[j] = item;
    }
  }
  cp_async_commit();
  // index of item 3 (its arguments are copied in iteration 0)
  int2 ahead = make_int2(0, 0);
  if (k0 + 3 * step < n) ahead = A.items[k0 + 3 * step];
  cp_async_wait_all();
  __syncthreads();
  {
    const InstArgs& I = sia[0];
    DG_ON_DEGREE(I.N, K::fill_nb(I, sitem[0].y, nb); K::load_ops(sops, sdv + B::dv_off(I.N), I));
  }
  __syncthreads();
  {
    const InstArgs& I = sia[0];
    DG_ON_DEGREE(I.N, K::issue(A, I, K::role(), sitem[0].y, st, nb, need_un));
  }
  cp_async_commit();
  int it = 0;
  for (int k = k0; k < n; k += step, ++it) {
    const int b = it & 1, s0 = it % B::RING, s1 = (it + 1) % B::RING, s3 = (it + 3) % B::RING;
    const int o0 = it % B::ORING, o1 = (it + 1) % B::ORING;
    const int kf = k + step;
    // item it+1: neighbour and coefficient tables from its copied arguments (visible since
    // the previous iteration's barrier)
    if (kf < n) {
      const InstArgs& I = sia[s1];
      DG_ON_DEGREE(I.N, K::fill_nb(I, sitem[s1].y, nb + (b ^ 1) * B::MNB);
                   K::load_ops(sops + o1 * B::MD, sdv + B::dv_off(I.N), I));
    }
    cp_async_wait_all();
    __syncthreads();  // item it's inputs, item it+1's tables and item it+2's arguments are
                      // visible; every thread has left item it-1 (its buffer, tables and
                      // argument slot are free)
    if (kf < n) {
      const InstArgs& I = sia[s1];
      DG_ON_DEGREE(I.N, K::issue(A, I, K::role(), sitem[s1].y, st + (b ^ 1) * B::MST,
                                 nb + (b ^ 1) * B::MNB, need_un));
    }
    if (k + 2 * step < n) {  // item it+2's own state towards L2 (its arguments are visible)
      const int s2 = (it + 2) % B::RING;
      const InstArgs& I2 = sia[s2];
      DG_ON_DEGREE(I2.N, K::prefetch_group(A, I2, sitem[s2].y, need_un));
    }
    const int k3 = k + 3 * step;
    if (k3 < n) {
      copy_inst<B>(A, ahead, sia + s3);
      if (t == 0) sitem[s3] = ahead;
    }
    cp_async_commit();
    if (k3 + step < n) ahead = A.items[k3 + step];  // used one iteration later
    const InstArgs& I = sia[s0];
    DG_ON_DEGREE(I.N, K::compute(A, I, sm, sops + o0 * B::MD, K::role(), sitem[s0].y, st + b * B::MST,
                                 need_un));
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
