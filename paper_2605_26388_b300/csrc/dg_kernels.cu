// dg_kernels.cu -- fused DGSEM residual + SSP-RK3 stage kernels for sm_103a.
//
// One launch evaluates, for every element of a periodic Cartesian instance, the
// semi-discrete Euler residual of Sec. 3.1.1 -- volume term (Eq. vol_weak, or Eq. vol_split
// with Ranocha's two-point flux, App. A Eq. split_form_3D), Riemann fluxes on the element
// faces, surface lifting and Jacobian rescale (Eq. surf_int) -- and applies the Shu-Osher
// stage update of App. B in FP64, in place of the paper's five kernels and its surface
// buffer.  Thread mapping: one thread per GLL node, one or more elements per CTA.
//
// Phases per CTA (all staged through shared memory):
//   1. load the FP64 state of its element(s) (coalesced SoA reads), convert to the flux
//      precision R, compute per-node primitives (two-point form) or per-direction point
//      fluxes (strong/weak form);
//   2. volume term: strong/weak -- each node contracts the volume operator along its d
//      lines; two-point form -- for one direction at a time, every pair a<b of every line
//      is evaluated once (F# is symmetric) into a pair buffer, then each node gathers its
//      N partners with D weights in a fixed order (deterministic, no atomics);
//   3. surface: one job per (face, face node): the neighbour trace is read from global
//      memory (L2), F* = F*(U_L, U_R) is evaluated at a single call site for both
//      orientations -- so the two elements sharing a face compute bitwise-identical F*,
//      which makes the scheme exactly conservative without a shared surface buffer --
//      and the lifted jump is staged per face node;
//   4. each node gathers its face terms, forms L, and writes L or the FP64 stage update.
#include "dg_device.cuh"
#include "dg_internal.h"

namespace dg {

template <int N1>
__device__ __forceinline__ void pair_ab(int p, int& a, int& b) {
  a = 0;
  int rem = p;
  while (rem >= N1 - 1 - a) {
    rem -= N1 - 1 - a;
    ++a;
  }
  b = a + 1 + rem;
}

template <int N1>
__device__ __forceinline__ int pair_index(int a, int b) {  // a < b
  return a * N1 - (a * (a + 1)) / 2 + (b - a - 1);
}

template <int DIM, int L, class R>
__device__ __forceinline__ void surface_flux(int kind, const R* uL, const R* uR, R pdL, R pdR,
                                             R gamma, R p_ref, R* F) {
  switch (kind) {
    case 1: hllc<DIM, L>(uL, uR, pdL, pdR, gamma, p_ref, F); break;
    case 2: hll<DIM, L>(uL, uR, pdL, pdR, gamma, p_ref, F); break;
    case 3: ec_flux<DIM, L>(uL, uR, pdL, pdR, gamma - R(1), p_ref, F); break;
    default: rusanov<DIM, L>(uL, uR, pdL, pdR, gamma, p_ref, F); break;
  }
}

template <int DIM, int N, bool EC, class R>
struct EulerStage {
  using G = Geo<DIM, N>;
  static constexpr int NV = G::NV, NP = G::NP, N1 = G::N1, EPB = G::EPB, NFN = G::NFN;
  static constexpr int NLINE = G::NLINE, NPAIR = G::NPAIR, T = G::THREADS;
  // per-node staged quantities: EC -- rho, v_1..v_DIM, pd, beta = rho/p; strong/weak -- the
  // DIM point fluxes (NV each) and pd
  static constexpr int NQ = EC ? (DIM + 3) : (DIM * NV + 1);
  static constexpr int PD = EC ? (DIM + 1) : (DIM * NV);  // slot of pd
  // shared-memory layout (in units of R)
  static constexpr int OFF_U = 0;                                 // [EPB][NV][NP]
  static constexpr int OFF_Q = OFF_U + EPB * NV * NP;             // [EPB][NQ][NP]
  static constexpr int OFF_S = OFF_Q + EPB * NQ * NP;             // [EPB][2DIM][NFN][NV]
  static constexpr int OFF_X = OFF_S + EPB * 2 * DIM * NFN * NV;  // [EPB][NLINE][NPAIR][NV]
  static constexpr int OFF_D = OFF_X + (EC ? EPB * NLINE * NPAIR * NV : 0);  // [N1][N1]
  static constexpr int SMEM_ELEMS = OFF_D + N1 * N1;
  static constexpr size_t smem_bytes() { return sizeof(R) * (size_t)SMEM_ELEMS; }

  // point flux of direction L at node nd of element el from the staged state
  template <int L>
  static __device__ __forceinline__ void staged_point_flux(const R* sm, int el, int nd, R p_ref,
                                                           R* F) {
    R u[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = sm[OFF_U + (el * NV + v) * NP + nd];
    const Prim<DIM, R> q = prims<DIM>(u, sm[OFF_Q + (el * NQ + PD) * NP + nd], p_ref);
    point_flux<DIM, L>(u, q, F);
  }

  // two-point volume term of direction L for this node (EC form)
  template <int L>
  static __device__ __forceinline__ void ec_direction(R* sm, const StageArgs& A, int el, int nd,
                                                      bool active, R p_ref, R igm1, R* acc) {
    const int e0 = blockIdx.x * EPB;
    // pair phase: every pair (a<b) of every line, once
    for (int J = threadIdx.x; J < EPB * NLINE * NPAIR; J += T) {
      const int ej = J / (NLINE * NPAIR);
      const int r = J - ej * NLINE * NPAIR;
      const int q = r / NPAIR;
      const int p = r - q * NPAIR;
      if (e0 + ej >= A.n_elem) continue;
      int a, b;
      pair_ab<N1>(p, a, b);
      const int na = G::line_node(L, q, a), nb = G::line_node(L, q, b);
      const R* Q = sm + OFF_Q + ej * NQ * NP;
      R vA[DIM], vB[DIM];
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        vA[d] = Q[(1 + d) * NP + na];
        vB[d] = Q[(1 + d) * NP + nb];
      }
      R F[NV];
      ec_flux_prims<DIM, L>(Q[na], vA, Q[PD * NP + na], Q[(DIM + 2) * NP + na], Q[nb], vB,
                            Q[PD * NP + nb], Q[(DIM + 2) * NP + nb], igm1, p_ref, F);
      R* X = sm + OFF_X + ((ej * NLINE + q) * NPAIR + p) * NV;
#pragma unroll
      for (int v = 0; v < NV; ++v) X[v] = F[v];
    }
    __syncthreads();
    if (active) {
      const R s = R(A.s[L]);
      const int q = G::node_line(L, nd), i = G::node_pos(L, nd);
      const R* Dv = sm + OFF_D;
      const R* X = sm + OFF_X + (el * NLINE + q) * NPAIR * NV;
#pragma unroll
      for (int m = 0; m < N1; ++m) {
        if (m == i) continue;
        const int p = (m < i) ? pair_index<N1>(m, i) : pair_index<N1>(i, m);
        const R c = s * Dv[i * N1 + m];
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] -= c * X[p * NV + v];
      }
      // diagonal term: F#(U_i, U_i) = F(U_i); only the end nodes have D_ii != 0
      if (i == 0 || i == N) {
        R F[NV];
        staged_point_flux<L>(sm, el, nd, p_ref, F);
        const R c = s * Dv[i * N1 + i];
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] -= c * F[v];
      }
    }
    __syncthreads();  // the pair buffer is reused by the next direction
  }

  template <int L>
  static __device__ __forceinline__ void sbp_direction(const R* sm, const StageArgs& A, int el,
                                                       int nd, R* acc) {
    const R s = R(A.s[L]);
    const int q = G::node_line(L, nd), i = G::node_pos(L, nd);
    const R* Dv = sm + OFF_D;
    const R* Fq = sm + OFF_Q + (el * NQ + L * NV) * NP;
#pragma unroll
    for (int m = 0; m < N1; ++m) {
      const int n2 = G::line_node(L, q, m);
      const R c = s * Dv[i * N1 + m];
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] -= c * Fq[v * NP + n2];
    }
  }

  // one surface job in direction L: face node f of face `side` of element ej
  template <int L>
  static __device__ __forceinline__ void surface_job(R* sm, const StageArgs& A, int ej, int side,
                                                     int f, R gamma, R p_ref) {
    const int e = blockIdx.x * EPB + ej;
    const int ndo = G::line_node(L, f, side ? N : 0);
    // periodic neighbour element across this face
    int c[3];
    c[0] = e % A.nel[0];
    c[1] = (e / A.nel[0]) % A.nel[1];
    c[2] = (DIM == 3) ? e / (A.nel[0] * A.nel[1]) : 0;
    c[L] += side ? 1 : -1;
    if (c[L] < 0) c[L] += A.nel[L];
    if (c[L] >= A.nel[L]) c[L] -= A.nel[L];
    const int en = c[0] + A.nel[0] * (c[1] + A.nel[1] * c[2]);
    const int ndn = G::line_node(L, f, side ? 0 : N);
    const long long gn = A.base + (long long)en * NP + ndn;
    R own[NV], nbr[NV];
    double n64[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      own[v] = sm[OFF_U + (ej * NV + v) * NP + ndo];
      n64[v] = __ldg(A.U + v * A.stride + gn);
      nbr[v] = Ar<R>::load(n64[v]);
    }
    const R pd_own = sm[OFF_Q + (ej * NQ + PD) * NP + ndo];
    double rhoe;
    const R pd_nbr = pdev<DIM>(n64, nbr, A.gamma - 1.0, A.p_ref, rhoe);
    R uL[NV], uR[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      uL[v] = side ? own[v] : nbr[v];
      uR[v] = side ? nbr[v] : own[v];
    }
    const R pdL = side ? pd_own : pd_nbr, pdR = side ? pd_nbr : pd_own;
    R Fs[NV];
    surface_flux<DIM, L>(A.surface, uL, uR, pdL, pdR, gamma, p_ref, Fs);  // the single call site
    R Fo[NV];
    if (A.weak) {
#pragma unroll
      for (int v = 0; v < NV; ++v) Fo[v] = R(0);
    } else {
      const Prim<DIM, R> q = prims<DIM>(own, pd_own, p_ref);
      point_flux<DIM, L>(own, q, Fo);
    }
    const R lf = (side ? R(-1) : R(1)) * R(A.s[L]) * R(A.lift);
    R* S = sm + OFF_S + ((ej * 2 * DIM + 2 * L + side) * NFN + f) * NV;
#pragma unroll
    for (int v = 0; v < NV; ++v) S[v] = lf * (Fs[v] - Fo[v]);
  }

  static __device__ void run(const StageArgs& A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sm = reinterpret_cast<R*>(smem_raw);
    const int t = threadIdx.x;
    const int el = t / NP, nd = t - (t / NP) * NP;
    const int e = blockIdx.x * EPB + el;
    const bool active = (el < EPB) && (e < A.n_elem);
    const R gamma = R(A.gamma), gm1 = gamma - R(1), igm1 = R(1) / gm1, p_ref = R(A.p_ref);

    for (int k = t; k < N1 * N1; k += T) sm[OFF_D + k] = R(A.Dv[k]);

    // ---- phase 1: load, convert, stage primitives / fluxes ----
    double u64[NV], un64[NV];
    const long long g = A.base + (long long)e * NP + nd;
    if (active) {
      const bool need_un = (A.mode == 1) && (A.ca != 0.0);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        u64[v] = __ldg(A.U + v * A.stride + g);
        un64[v] = need_un ? __ldg(A.Un + v * A.stride + g) : 0.0;
      }
      R u[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        u[v] = Ar<R>::load(u64[v]);
        sm[OFF_U + (el * NV + v) * NP + nd] = u[v];
      }
      // pressure deviation from the FP64 energy; positivity of the state this stage reads
      // (rho > 0 and rho e > 0) decided in FP64
      double rhoe;
      const R pd = pdev<DIM>(u64, u, A.gamma - 1.0, A.p_ref, rhoe);
      const Prim<DIM, R> q = prims<DIM>(u, pd, p_ref);
      const bool ok = (u64[0] > 0.0) && (rhoe > 0.0);
      if (!ok) atomicOr(A.err, 2u);
      R* Q = sm + OFF_Q + el * NQ * NP;
      Q[PD * NP + nd] = pd;
      if (EC) {
        Q[nd] = q.rho;
#pragma unroll
        for (int d = 0; d < DIM; ++d) Q[(1 + d) * NP + nd] = q.v[d];
        Q[(DIM + 2) * NP + nd] = q.rho * Ar<R>::rcp(q.p);
      } else {
        R F[NV];
        point_flux<DIM, 0>(u, q, F);
#pragma unroll
        for (int v = 0; v < NV; ++v) Q[(0 * NV + v) * NP + nd] = F[v];
        point_flux<DIM, 1>(u, q, F);
#pragma unroll
        for (int v = 0; v < NV; ++v) Q[(1 * NV + v) * NP + nd] = F[v];
        if constexpr (DIM == 3) {
          point_flux<DIM, 2>(u, q, F);
#pragma unroll
          for (int v = 0; v < NV; ++v) Q[(2 * NV + v) * NP + nd] = F[v];
        }
      }
    }
    __syncthreads();

    // ---- phase 2: volume term ----
    R acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = R(0);
    if constexpr (EC) {
      ec_direction<0>(sm, A, el, nd, active, p_ref, igm1, acc);
      ec_direction<1>(sm, A, el, nd, active, p_ref, igm1, acc);
      if constexpr (DIM == 3) ec_direction<2>(sm, A, el, nd, active, p_ref, igm1, acc);
    } else {
      if (active) {
        sbp_direction<0>(sm, A, el, nd, acc);
        sbp_direction<1>(sm, A, el, nd, acc);
        if constexpr (DIM == 3) sbp_direction<2>(sm, A, el, nd, acc);
      }
    }

    // ---- phase 3: surface jobs ----
    const int e0 = blockIdx.x * EPB;
    for (int J = t; J < EPB * 2 * DIM * NFN; J += T) {
      const int ej = J / (2 * DIM * NFN);
      const int r = J - ej * 2 * DIM * NFN;
      const int face = r / NFN;
      const int f = r - face * NFN;
      if (e0 + ej >= A.n_elem) continue;
      const int l = face >> 1, side = face & 1;
      if (l == 0) surface_job<0>(sm, A, ej, side, f, gamma, p_ref);
      else if (l == 1) surface_job<1>(sm, A, ej, side, f, gamma, p_ref);
      else if constexpr (DIM == 3) surface_job<2>(sm, A, ej, side, f, gamma, p_ref);
    }
    __syncthreads();

    // ---- phase 4: gather face terms, write L or the stage update ----
    if (!active) return;
#pragma unroll
    for (int l = 0; l < DIM; ++l) {
      const int i = G::node_pos(l, nd), f = G::node_line(l, nd);
      if (i == 0) {
        const R* S = sm + OFF_S + ((el * 2 * DIM + 2 * l) * NFN + f) * NV;
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] += S[v];
      }
      if (i == N) {
        const R* S = sm + OFF_S + ((el * 2 * DIM + 2 * l + 1) * NFN + f) * NV;
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] += S[v];
      }
    }
    double res[NV];
    bool finite = true;
    if (A.mode == 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) res[v] = Ar<R>::widen(acc[v]);
    } else {
      // U^(k) = ca Un + cb (U^(k-1) + dt L), with the increment cb dt L formed in R
      const R cbdt = R(A.cb * A.dt);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const double inc = Ar<R>::widen(cbdt * acc[v]);
        double x = fma(A.cb, u64[v], inc);
        if (A.ca != 0.0) x = fma(A.ca, un64[v], x);
        res[v] = x;
      }
      if (A.rho_floor > 0.0 || A.p_floor > 0.0) {  // positivity floor (off by default)
        if (A.rho_floor > 0.0 && res[0] < A.rho_floor) res[0] = A.rho_floor;
        double kin = 0.0;
#pragma unroll
        for (int d = 0; d < DIM; ++d) kin += res[1 + d] * res[1 + d] / res[0];
        const double p = (A.gamma - 1.0) * (res[DIM + 1] - 0.5 * kin);
        if (A.p_floor > 0.0 && p < A.p_floor) res[DIM + 1] = A.p_floor / (A.gamma - 1.0) + 0.5 * kin;
      }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      finite = finite && finite64(res[v]);
      A.out[v * A.stride + g] = res[v];
    }
    if (!finite) atomicOr(A.err, 1u);
  }
};

template <int DIM, int N, bool EC, class R>
__global__ void __launch_bounds__(Geo<DIM, N>::THREADS) k_euler_stage(const StageArgs A) {
  EulerStage<DIM, N, EC, R>::run(A);
}

template <int DIM, int N, bool EC, class R>
static cudaError_t launch_one(const StageArgs& a, cudaStream_t s) {
  using K = EulerStage<DIM, N, EC, R>;
  const int blocks = (a.n_elem + K::EPB - 1) / K::EPB;
  if (blocks == 0) return cudaSuccess;
  k_euler_stage<DIM, N, EC, R><<<blocks, K::T, K::smem_bytes(), s>>>(a);
  return cudaGetLastError();
}

template <int DIM, int N, bool EC, class R>
static cudaError_t prepare_one() {
  using K = EulerStage<DIM, N, EC, R>;
  return cudaFuncSetAttribute(k_euler_stage<DIM, N, EC, R>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::smem_bytes());
}

template <int DIM, int N>
static cudaError_t launch_dn(int ec, int fp32, const StageArgs* a, cudaStream_t s) {
  if (!a) {
    if (ec) return fp32 ? prepare_one<DIM, N, true, float>() : prepare_one<DIM, N, true, double>();
    return fp32 ? prepare_one<DIM, N, false, float>() : prepare_one<DIM, N, false, double>();
  }
  if (ec) return fp32 ? launch_one<DIM, N, true, float>(*a, s) : launch_one<DIM, N, true, double>(*a, s);
  return fp32 ? launch_one<DIM, N, false, float>(*a, s) : launch_one<DIM, N, false, double>(*a, s);
}

static cudaError_t dispatch(int dim, int N, int ec, int fp32, const StageArgs* a, cudaStream_t s) {
  if (dim == 2) {
    switch (N) {
      case 1: return launch_dn<2, 1>(ec, fp32, a, s);
      case 2: return launch_dn<2, 2>(ec, fp32, a, s);
      case 3: return launch_dn<2, 3>(ec, fp32, a, s);
      case 4: return launch_dn<2, 4>(ec, fp32, a, s);
      case 5: return launch_dn<2, 5>(ec, fp32, a, s);
      case 6: return launch_dn<2, 6>(ec, fp32, a, s);
      case 7: return launch_dn<2, 7>(ec, fp32, a, s);
    }
  } else if (dim == 3) {
    switch (N) {
      case 1: return launch_dn<3, 1>(ec, fp32, a, s);
      case 2: return launch_dn<3, 2>(ec, fp32, a, s);
      case 3: return launch_dn<3, 3>(ec, fp32, a, s);
      case 4: return launch_dn<3, 4>(ec, fp32, a, s);
      case 5: return launch_dn<3, 5>(ec, fp32, a, s);
    }
  }
  return cudaErrorInvalidValue;
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
// Largest signal speed |u| + a (Eq. dt_hyp), FP64, block max then one atomicMax on the
// bit pattern (non-negative doubles order like their unsigned bit patterns).
// ---------------------------------------------------------------------------------------
template <int DIM>
__global__ void k_max_speed(const double* U, long long stride, long long base, long long n,
                            double gamma, unsigned long long* out) {
  double lam = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const double rho = U[base + q];
    double m2 = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const double m = U[(1 + d) * stride + base + q];
      m2 += m * m;
    }
    const double E = U[(DIM + 1) * stride + base + q];
    const double p = (gamma - 1.0) * (E - 0.5 * m2 / rho);
    const double sp = sqrt(m2) / rho + sqrt(gamma * p / rho);
    lam = fmax(lam, sp);
  }
  for (int o = 16; o > 0; o >>= 1) lam = fmax(lam, __shfl_xor_sync(0xffffffffu, lam, o));
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lam;
  __syncthreads();
  if (threadIdx.x < 32) {
    lam = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) lam = fmax(lam, __shfl_xor_sync(0xffffffffu, lam, o));
    if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(lam));
  }
}

cudaError_t launch_max_speed(int dim, const double* U, long long stride, long long base,
                             long long n_nodes, double gamma, unsigned long long* lam_bits,
                             cudaStream_t s) {
  if (n_nodes <= 0) return cudaSuccess;
  long long blocks = (n_nodes + 255) / 256;
  if (blocks > 148 * 16) blocks = 148 * 16;
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
  double ea, eb;
  const R pda = pdev<DIM>(a64, a, gamma - 1.0, p_ref, ea);
  const R pdb = pdev<DIM>(b64, b, gamma - 1.0, p_ref, eb);
  if (kind < 0) ec_flux<DIM, L>(a, b, pda, pdb, R(gamma) - R(1), R(p_ref), f);
  else surface_flux<DIM, L>(kind, a, b, pda, pdb, R(gamma), R(p_ref), f);
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
