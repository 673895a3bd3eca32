// dg_noalloc.cu -- a time-step bound for callers that cannot allocate GPU memory.
//
// dg_max_dt() needs a context, and a context allocates its state buffers and a scratch
// word with cudaMalloc.  Some callers cannot do that: code that runs inside another
// framework's memory management (a caching allocator that has already reserved the
// device's memory, where a raw cudaMalloc fails or fragments it), or a host application
// that fixes its GPU memory footprint up front and forbids allocation in its time loop.
// dg_max_dt_noalloc() gives them the same bound on a state they already hold, with the
// reduction's scratch in a fixed array that the library itself carries.
//
// The scratch is one 64-bit slot per instance in a file-scope __device__ array of
// DG_NOALLOC_MAX_INSTANCES entries (32 KiB); every GPU that loads the library holds it
// until the process exits.  All calls share it, so calls that overlap on the GPU race.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/dgsem.h"
#include "dg_device.cuh"

static __device__ __align__(256) unsigned long long g_speed_slots[DG_NOALLOC_MAX_INSTANCES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned long long* g_slots_addr[kMaxDevices] = {};  // device address, per device

// Largest |u| + a over the nodes of one instance (the Eq. dt_hyp signal speed), as the
// reduction code of dg_device.cuh (a non-finite node, or one with rho <= 0 or p <= 0, makes
// the slot report it), reduced per block and merged into *slot with one atomicMax.
template <int DIM>
__global__ void k_max_speed_slots(const double* U, long long stride, long long base, long long n,
                                  double gamma, unsigned long long* slot) {
  unsigned long long lam = 0ull;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const unsigned long long b = dg::euler_speed_bits<DIM>(U, stride, base + q, gamma);
    lam = b > lam ? b : lam;
  }
  lam = dg::block_max_u64(lam);
  if (threadIdx.x == 0) atomicMax(slot, lam);
}

dg_status reject(const char** msg, dg_status st, const char* why) {
  if (msg) *msg = why;
  return st;
}

}  // namespace

extern "C" dg_status dg_max_dt_noalloc(const dg_mesh_desc* inst, int n_inst, double gamma,
                                       const double* U, double cfl, void* cuda_stream,
                                       double* dt_out, const char** msg) {
  if (msg) *msg = "";
  if (!inst || !U || !dt_out) return reject(msg, DG_EINVAL, "null argument");
  if (n_inst < 1) return reject(msg, DG_EINVAL, "n_inst must be >= 1");
  if (n_inst > DG_NOALLOC_MAX_INSTANCES)
    return reject(msg, DG_ETOOLARGE,
                  "n_inst exceeds DG_NOALLOC_MAX_INSTANCES, the size of the static scratch array");
  if (!(gamma > 1.0) || !(cfl > 0.0)) return reject(msg, DG_EINVAL, "gamma must be > 1 and cfl > 0");
  long long total = 0;
  for (int i = 0; i < n_inst; ++i) {
    const dg_mesh_desc& m = inst[i];
    if ((m.dim != 2 && m.dim != 3) || m.dim != inst[0].dim || m.N < 1)
      return reject(msg, DG_EINVAL, "bad dim or N");
    if (m.coords)  // the bound uses the box spacing; a curved mesh's elements can be smaller
      return reject(msg, DG_EUNSUPPORTED, "curved meshes (coords != NULL) are not supported here");
    long long ne = 1, np = 1;
    for (int l = 0; l < m.dim; ++l) {
      if (m.nel[l] < 1 || !(m.hi[l] > m.lo[l])) return reject(msg, DG_EINVAL, "bad nel or box");
      ne *= m.nel[l];
      np *= (m.N + 1);
    }
    total += ne * np;
  }

  // once per device, with that device current: the device address of the scratch array
  // (its name in host code is only a host-side stand-in)
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return reject(msg, DG_ECUDA, "cudaGetDevice failed");
  if (dev < 0 || dev >= kMaxDevices) return reject(msg, DG_EUNSUPPORTED, "device index too large");
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess || sms < 1) return reject(msg, DG_ECUDA, "cudaDeviceGetAttribute failed");
  unsigned long long* slots;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_slots_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_speed_slots);
      if (e != cudaSuccess || !p) return reject(msg, DG_ECUDA, "cudaGetSymbolAddress failed");
      g_slots_addr[dev] = static_cast<unsigned long long*>(p);
    }
    slots = g_slots_addr[dev];
  }

  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the array keeps the previous call's maxima: clear the slots this call uses
  e = cudaMemsetAsync(slots, 0, sizeof(unsigned long long) * (size_t)n_inst, s);
  long long off = 0;
  for (int i = 0; i < n_inst && e == cudaSuccess; ++i) {
    const dg_mesh_desc& m = inst[i];
    long long n = 1;
    for (int l = 0; l < m.dim; ++l) n *= (long long)m.nel[l] * (m.N + 1);
    long long blocks = (n + 255) / 256;
    if (blocks > 16LL * sms) blocks = 16LL * sms;
    if (m.dim == 2) k_max_speed_slots<2><<<(int)blocks, 256, 0, s>>>(U, total, off, n, gamma, slots + i);
    else k_max_speed_slots<3><<<(int)blocks, 256, 0, s>>>(U, total, off, n, gamma, slots + i);
    e = cudaGetLastError();
    off += n;
  }
  unsigned long long bits[DG_NOALLOC_MAX_INSTANCES];
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bits, slots, sizeof(unsigned long long) * (size_t)n_inst,
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return reject(msg, DG_ECUDA, "a CUDA call failed in dg_max_dt_noalloc");

  double best = INFINITY;
  for (int i = 0; i < n_inst; ++i) {
    if (bits[i] >= dg::kSpeedNonFinite) return reject(msg, DG_ENONFINITE, "the state holds a non-finite value");
    if (bits[i] >= dg::kSpeedNonPositive)
      return reject(msg, DG_EPOSITIVITY, "the state has a node with rho <= 0 or p <= 0");
    double lam;
    std::memcpy(&lam, &bits[i], sizeof(lam));
    if (!(lam > 0.0)) return reject(msg, DG_ENONFINITE, "no positive signal speed");
    const dg_mesh_desc& m = inst[i];
    double dxmin = INFINITY;
    for (int l = 0; l < m.dim; ++l) dxmin = std::fmin(dxmin, (m.hi[l] - m.lo[l]) / m.nel[l]);
    best = std::fmin(best, cfl * dxmin / ((2 * m.N + 1) * lam));
  }
  *dt_out = best;
  return DG_OK;
}
