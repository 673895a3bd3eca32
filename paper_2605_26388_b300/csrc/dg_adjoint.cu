// dg_adjoint.cu -- hand-written adjoint (vector-Jacobian product) of the DGSEM residual.
//
// For the strong or weak volume form (Eq. vol_weak) with the Rusanov surface flux
// (Eq. surf_int, Sec. 3.1.1), on periodic meshes or with the boundary functors of the forward
// pass (slip wall, supersonic inflow and outflow, Dirichlet), given a co-state lam this
// computes, element by element,
//   w = (dL/dU)^T lam      and      g = lam . dL/dgamma,
// without atomics: the volume part contracts lam with the transposed volume operator along
// each line and applies the transposed Euler flux Jacobian; every face node combines its own
// and its neighbour's co-state (gathered from global memory, as the forward pass gathers
// the neighbour's state) with the transposed Rusanov flux Jacobian.  Non-smooth points
// follow the forward evaluation: the larger signal speed of the Rusanov flux (the left one
// on a tie) carries the derivative, and d|x|/dx = sign(x) with sign(0) = 0.
//
// Output modes (one kernel, fused with the reverse Shu-Osher combination of App. B):
//   mode 0:  out += w                                    (dg_rhs_vjp, accumulating)
//   mode 1:  out  = bcoef (lam + dt w) [+ accin];  accupd (=|+=) acoef lam
// and the gamma contribution, weighted by gw, is reduced per CTA into gpart[blockIdx.x].
#include <cuda_runtime.h>

#include "dg_device.cuh"
#include "dg_internal.h"

namespace dg {

// (dF^l/dU)^T mu for the Euler flux F^l (Sec. 2), primitives v, p, enthalpy H = (E+p)/rho.
template <int DIM, class R>
__device__ __forceinline__ void flux_jac_t(int l, const R* v, R H, R gm1, const R* mu, R* out) {
  R mv = R(0), v2 = R(0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    mv += mu[1 + d] * v[d];
    v2 += v[d] * v[d];
  }
  const R q = gm1 * R(0.5) * v2;  // dp/drho
  R vl = R(0), mul = R(0);
#pragma unroll
  for (int d = 0; d < DIM; ++d)
    if (d == l) { vl = v[d]; mul = mu[1 + d]; }
  const R muE = mu[DIM + 1];
  out[0] = -vl * mv + mul * q + muE * vl * (q - H);
  const R t = mul + muE * vl;
#pragma unroll
  for (int k = 0; k < DIM; ++k)
    out[1 + k] = (k == l ? (mu[0] + mv + muE * H) : R(0)) + vl * mu[1 + k] - gm1 * v[k] * t;
  out[DIM + 1] = gm1 * mul + (gm1 + R(1)) * vl * muE;
}

// gradient of the signal speed s = |v_l| + c, c = sqrt(gamma p / rho), and ds/dgamma
template <int DIM, class R>
__device__ __forceinline__ void speed_grad(int l, const R* v, R rho, R p, R c, R gamma, R* g,
                                           R& dsdg) {
  const R gm1 = gamma - R(1);
  R v2 = R(0), vl = R(0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    v2 += v[d] * v[d];
    if (d == l) vl = v[d];
  }
  const R irho = Ar<R>::rcp(rho);
  const R sg = (vl > R(0)) ? R(1) : ((vl < R(0)) ? R(-1) : R(0));
  const R k = gamma * Ar<R>::rcp(R(2) * c * rho);
  const R q = gm1 * R(0.5) * v2;
  g[0] = -sg * vl * irho + k * (q - p * irho);
#pragma unroll
  for (int d = 0; d < DIM; ++d) g[1 + d] = (d == l ? sg * irho : R(0)) - k * gm1 * v[d];
  g[DIM + 1] = k * gm1;
  const R rhoe = p * Ar<R>::rcp(gm1);
  dsdg = (p + gamma * rhoe) * Ar<R>::rcp(R(2) * c * rho);
}

// per-instance metric scalars in the flux precision (no double->float conversion per thread)
template <class R> __device__ __forceinline__ R s_of(const InstArgs& I, int l);
template <> __device__ __forceinline__ double s_of<double>(const InstArgs& I, int l) { return I.s[l]; }
template <> __device__ __forceinline__ float s_of<float>(const InstArgs& I, int l) { return I.sf[l]; }
template <class R> __device__ __forceinline__ R lift_of(const InstArgs& I);
template <> __device__ __forceinline__ double lift_of<double>(const InstArgs& I) { return I.lift; }
template <> __device__ __forceinline__ float lift_of<float>(const InstArgs& I) { return I.liftf; }

template <int DIM, class R>
struct NodeState {
  R u[DIM + 2], v[DIM], rho, p, H, c, rhoe;
};

template <int DIM, class R>
__device__ __forceinline__ NodeState<DIM, R> node_state(const double* u64, R gamma) {
  NodeState<DIM, R> s;
#pragma unroll
  for (int k = 0; k < DIM + 2; ++k) s.u[k] = Ar<R>::load(u64[k]);
  s.rho = s.u[0];
  const R irho = Ar<R>::rcp(s.rho);
  R kin = R(0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    s.v[d] = s.u[1 + d] * irho;
    kin += s.u[1 + d] * s.v[d];
  }
  s.rhoe = s.u[DIM + 1] - R(0.5) * kin;
  s.p = (gamma - R(1)) * s.rhoe;
  s.H = (s.u[DIM + 1] + s.p) * irho;
  s.c = Ar<R>::sqrt(gamma * s.p * irho);
  return s;
}

// Domain face (2 l + side) that side `side` of element e in direction l lies on when that face
// carries a boundary condition, else -1.
__device__ __forceinline__ int wall_face(const InstArgs& I, int e, int l, int side) {
  const int f = 2 * l + side;
  if (I.bc[f] == 0) return -1;
  const int c = l == 0 ? e % I.nel[0] : (l == 1 ? (e / I.nel[0]) % I.nel[1] : e / (I.nel[0] * I.nel[1]));
  return (side ? c == I.nel[l] - 1 : c == 0) ? f : -1;
}

template <int DIM, int N, class R>
struct Vjp {
  using G = Geo<DIM, N>;
  static constexpr int NV = G::NV, NP = G::NP, N1 = G::N1, NFN = G::NFN, EPB = G::EPB;
  static constexpr int NF = 2 * DIM, NJS = EPB * NF * NFN;
  static constexpr int T = (((EPB * NP > NJS) ? EPB * NP : NJS) + 31) / 32 * 32;
  // shared: co-state [EPB][NV][NP], face contributions [EPB][NF][NFN][NV], D, reduction
  static constexpr int OFF_L = 0, OFF_S = EPB * NV * NP, OFF_D = OFF_S + EPB * NF * NFN * NV;
  static constexpr int R_SIZE = OFF_D + N1 * N1;
  static constexpr size_t RED_OFF = (sizeof(R) * R_SIZE + 15) / 16 * 16;  // 16-byte aligned
  static constexpr size_t smem_bytes() { return RED_OFF + sizeof(double) * 32; }

  static __device__ __forceinline__ int stride_l(int l) { return l == 0 ? 1 : (l == 1 ? N1 : N1 * N1); }
  static __device__ __forceinline__ int pos(int l, int nd) { return (nd / stride_l(l)) % N1; }
  static __device__ __forceinline__ int face_line(int l, int nd) {
    const int S = stride_l(l);
    return (nd % S) + (nd / (S * N1)) * S;
  }
  static __device__ __forceinline__ int line_node(int l, int q, int m) {
    const int S = stride_l(l);
    return (q % S) + m * S + (q / S) * S * N1;
  }
  static __device__ __forceinline__ int neighbour(const InstArgs& I, int e, int face) {
    int c[3] = {e % I.nel[0], (e / I.nel[0]) % I.nel[1], (DIM == 3) ? e / (I.nel[0] * I.nel[1]) : 0};
    const int l = face >> 1;
    int x = c[l] + ((face & 1) ? 1 : -1);
    x = x < 0 ? x + I.nel[l] : (x >= I.nel[l] ? x - I.nel[l] : x);
    if (l == 0) c[0] = x; else if (l == 1) c[1] = x; else c[2] = x;
    return c[0] + I.nel[0] * (c[1] + I.nel[1] * c[2]);
  }

  static __device__ void run(const VjpArgs& A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sm = reinterpret_cast<R*>(smem_raw);
    double* red = reinterpret_cast<double*>(smem_raw + RED_OFF);
    const InstArgs& I = A.inst;
    const int t = threadIdx.x;
    const int e0 = blockIdx.x * EPB;
    const R gamma = R(A.gamma), gm1 = gamma - R(1);
    for (int k = t; k < N1 * N1; k += T) sm[OFF_D + k] = R(A.Dv[k]);
    const int el = t / NP, nd = t - (t / NP) * NP;
    const bool active = (t < EPB * NP) && (e0 + el < I.n_elem);
    const long long gi = I.base + (long long)(e0 + el) * NP + nd;
    double gacc = 0.0;  // this thread's share of lam . dL/dgamma
    if (active) {
#pragma unroll
      for (int v = 0; v < NV; ++v) sm[OFF_L + (el * NV + v) * NP + nd] = Ar<R>::load(A.lam[v * A.stride + gi]);
    }
    __syncthreads();

    // volume: w_m = -sum_l s_l A^l(U_m)^T sum_i Dv[i][m] lam_i
    R w[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) w[v] = R(0);
    NodeState<DIM, R> ns;
    if (active) {
      double u64[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) u64[v] = A.U[v * A.stride + gi];
      ns = node_state<DIM, R>(u64, gamma);
#pragma unroll
      for (int l = 0; l < DIM; ++l) {
        const int m = pos(l, nd), q = face_line(l, nd);
        const R s = s_of<R>(I, l);
        R mu[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) mu[v] = R(0);
#pragma unroll
        for (int i = 0; i < N1; ++i) {
          const R d = sm[OFF_D + i * N1 + m];
          const int ni = line_node(l, q, i);
#pragma unroll
          for (int v = 0; v < NV; ++v) mu[v] += d * sm[OFF_L + (el * NV + v) * NP + ni];
        }
        R a[NV];
        flux_jac_t<DIM, R>(l, ns.v, ns.H, gm1, mu, a);
#pragma unroll
        for (int v = 0; v < NV; ++v) w[v] -= s * a[v];
        // dF^l/dgamma = rho e (0, e_l, v_l)
        R ml = R(0), vl = R(0);
#pragma unroll
        for (int d = 0; d < DIM; ++d)
          if (d == l) { ml = mu[1 + d]; vl = ns.v[d]; }
        gacc -= (double)(s * ns.rhoe * (ml + mu[DIM + 1] * vl));
      }
    }

    // faces: one job per face node
    for (int J = t; J < NJS; J += T) {
      const int ej = J / (NF * NFN), r = J - ej * (NF * NFN);
      const int face = r / NFN, f = r - face * NFN;
      if (e0 + ej >= I.n_elem) continue;
      const int l = face >> 1, side = face & 1;
      const int ndo = line_node(l, f, side ? N : 0);
      const long long go = I.base + (long long)(e0 + ej) * NP + ndo;
      // a domain face with a boundary condition: the exterior state of its functor (slip wall:
      // the mirror state; inflow, Dirichlet: U_b; outflow: the own state) and no neighbour
      // residual (its co-state is 0)
      const int fb = I.nonper ? wall_face(I, e0 + ej, l, side) : -1;
      const int type = fb >= 0 ? I.bc[fb] : 0;
      double uo[NV], un[NV];
      R lo[NV], ln[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        uo[v] = A.U[v * A.stride + go];
        lo[v] = sm[OFF_L + (ej * NV + v) * NP + ndo];
      }
      if (fb < 0) {
        const int en = neighbour(I, e0 + ej, face);
        const long long gn = I.base + (long long)en * NP + line_node(l, f, side ? 0 : N);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          un[v] = A.U[v * A.stride + gn];
          ln[v] = Ar<R>::load(A.lam[v * A.stride + gn]);
        }
      } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          un[v] = (type == 2 || type == 4) ? I.bcs[fb][v] : uo[v];
          ln[v] = R(0);
        }
        if (type == 1) {
#pragma unroll
          for (int d = 0; d < DIM; ++d)
            if (d == l) un[1 + d] = -uo[1 + d];
        }
      }
      const NodeState<DIM, R> so = node_state<DIM, R>(uo, gamma), sn = node_state<DIM, R>(un, gamma);
      const NodeState<DIM, R>& sL = side ? so : sn;
      const NodeState<DIM, R>& sR = side ? sn : so;
      R vlL = R(0), vlR = R(0);
#pragma unroll
      for (int d = 0; d < DIM; ++d)
        if (d == l) { vlL = sL.v[d]; vlR = sR.v[d]; }
      const R spL = Ar<R>::abs(vlL) + sL.c, spR = Ar<R>::abs(vlR) + sR.c;
      const bool left_sel = spL >= spR;
      const R lmax = left_sel ? spL : spR;
      const bool own_sel = (side == 1) ? left_sel : !left_sel;  // own is L on an upper face
      R mu[NV], dUm = R(0), dUl = R(0);  // mu = lam_own - lam_nbr; Delta = U_R - U_L
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        mu[v] = lo[v] - ln[v];
        const R dl = sR.u[v] - sL.u[v];
        dUm += mu[v] * dl;
        dUl += lo[v] * dl;
      }
      R a[NV], g[NV], dsdg;
      flux_jac_t<DIM, R>(l, so.v, so.H, gm1, mu, a);
      speed_grad<DIM, R>(l, so.v, so.rho, so.p, so.c, gamma, g, dsdg);
      const R sgn_l = side ? R(1) : R(-1);  // d F*/dU_own: +lmax/2 on the left, -lmax/2 on the right
      R ao[NV];
      if (!A.weak || type == 3) flux_jac_t<DIM, R>(l, so.v, so.H, gm1, lo, ao);
      const R s = s_of<R>(I, l);
      const R c = (side ? R(-1) : R(1)) * s * lift_of<R>(I);
      // slip wall: the exterior state M U_own also depends on U_own; its part of dF*/dU_own is
      // M (dF*/dU_ext)^T lam (M negates the normal momentum; the signal speeds tie, so the
      // left state carries the speed derivative)
      R ext[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) ext[v] = R(0);
      if (type == 1) {
        R ae[NV], ge[NV], dsdge;
        flux_jac_t<DIM, R>(l, sn.v, sn.H, gm1, lo, ae);
        speed_grad<DIM, R>(l, sn.v, sn.rho, sn.p, sn.c, gamma, ge, dsdge);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          ext[v] = R(0.5) * ae[v] - sgn_l * R(0.5) * lmax * lo[v];
          if (!own_sel) ext[v] -= R(0.5) * dUm * ge[v];
        }
#pragma unroll
        for (int d = 0; d < DIM; ++d)
          if (d == l) ext[1 + d] = -ext[1 + d];
      }
      R contrib[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        R jt = R(0.5) * a[v] + sgn_l * R(0.5) * lmax * mu[v];
        if (own_sel) jt -= R(0.5) * dUm * g[v];
        jt += ext[v];
        if (type == 2) jt = R(0);      // supersonic inflow: F* = F(U_b) does not see U_own
        if (type == 3) jt = ao[v];     // supersonic outflow: F* = F(U_own)
        contrib[v] = c * (jt - (A.weak ? R(0) : ao[v]));
      }
      R* S = sm + OFF_S + ((ej * NF + face) * NFN + f) * NV;
#pragma unroll
      for (int v = 0; v < NV; ++v) S[v] = contrib[v];
      // gamma: c lam_own . (dF*/dgamma - dF_own/dgamma), from this element's residual only
      R mlo = R(0), vlo = R(0);
#pragma unroll
      for (int d = 0; d < DIM; ++d)
        if (d == l) { mlo = lo[1 + d]; vlo = so.v[d]; }
      const R dFL = sL.rhoe * (mlo + lo[DIM + 1] * vlL), dFR = sR.rhoe * (mlo + lo[DIM + 1] * vlR);
      R dsel;
      {
        R gs[NV], dsdg_sel;
        const NodeState<DIM, R>& ssel = left_sel ? sL : sR;
        speed_grad<DIM, R>(l, ssel.v, ssel.rho, ssel.p, ssel.c, gamma, gs, dsdg_sel);
        dsel = dsdg_sel;
      }
      R dFs = R(0.5) * (dFL + dFR) - R(0.5) * dsel * dUl;
      if (type == 2) dFs = side ? dFR : dFL;  // the flux of U_b, the exterior state
      if (type == 3) dFs = side ? dFL : dFR;  // the own flux
      const R dFo = A.weak ? R(0) : so.rhoe * (mlo + lo[DIM + 1] * vlo);
      gacc += (double)(c * (dFs - dFo));
    }
    __syncthreads();

    if (active) {
#pragma unroll
      for (int l = 0; l < DIM; ++l) {
        const int i = pos(l, nd), f = face_line(l, nd);
        if (i == 0) {
          const R* S = sm + OFF_S + ((el * NF + 2 * l) * NFN + f) * NV;
#pragma unroll
          for (int v = 0; v < NV; ++v) w[v] += S[v];
        }
        if (i == N) {
          const R* S = sm + OFF_S + ((el * NF + 2 * l + 1) * NFN + f) * NV;
#pragma unroll
          for (int v = 0; v < NV; ++v) w[v] += S[v];
        }
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const long long k = v * A.stride + gi;
        const double wv = Ar<R>::widen(w[v]);
        if (A.mode == 0) {
          A.out[k] += wv;
        } else {
          const double lv = A.lam[k];
          double o = A.bcoef * (lv + A.dt * wv);
          if (A.accin) o += A.accin[k];
          if (A.accupd) A.accupd[k] = A.acc_init ? A.acoef * lv : A.accupd[k] + A.acoef * lv;
          A.out[k] = o;
        }
      }
    }
    // deterministic per-CTA reduction of the gamma contribution
    for (int o = 16; o > 0; o >>= 1) gacc += __shfl_xor_sync(0xffffffffu, gacc, o);
    if ((t & 31) == 0) red[t >> 5] = gacc;
    __syncthreads();
    if (t == 0) {
      double sum = 0.0;
      for (int k = 0; k < T / 32; ++k) sum += red[k];
      A.gpart[blockIdx.x] = A.gw * sum;
    }
  }
};

template <int DIM, int N, class R>
__global__ void __launch_bounds__(Vjp<DIM, N, R>::T) k_rhs_vjp(const VjpArgs A) {
  Vjp<DIM, N, R>::run(A);
}

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

template <int DIM, int N, class R>
static cudaError_t launch_vjp_one(const VjpArgs& a, cudaStream_t s, int* blocks_out) {
  using K = Vjp<DIM, N, R>;
  const int blocks = (a.inst.n_elem + K::EPB - 1) / K::EPB;
  if (blocks_out) *blocks_out = blocks;
  if (blocks == 0) return cudaSuccess;
  k_rhs_vjp<DIM, N, R><<<blocks, K::T, K::smem_bytes(), s>>>(a);
  return cudaGetLastError();
}

template <int DIM, int N>
static cudaError_t launch_vjp_dn(int fp32, const VjpArgs& a, cudaStream_t s, int* blocks) {
  return fp32 ? launch_vjp_one<DIM, N, float>(a, s, blocks) : launch_vjp_one<DIM, N, double>(a, s, blocks);
}

int vjp_blocks(int dim, int N, long long n_elem) {
  int np = 1, nfn = 1;
  for (int l = 0; l < dim; ++l) np *= (N + 1);
  for (int l = 1; l < dim; ++l) nfn *= (N + 1);
  const int w = np > 2 * dim * nfn ? np : 2 * dim * nfn;
  const int epb = w >= 96 ? 1 : 128 / w;
  return (int)((n_elem + epb - 1) / epb);
}

cudaError_t launch_rhs_vjp(int dim, int N, int fp32, const VjpArgs& a, double* gacc, cudaStream_t s) {
  int blocks = 0;
  cudaError_t e = cudaErrorInvalidValue;
  if (dim == 2) {
    switch (N) {
      case 1: e = launch_vjp_dn<2, 1>(fp32, a, s, &blocks); break;
      case 2: e = launch_vjp_dn<2, 2>(fp32, a, s, &blocks); break;
      case 3: e = launch_vjp_dn<2, 3>(fp32, a, s, &blocks); break;
      case 4: e = launch_vjp_dn<2, 4>(fp32, a, s, &blocks); break;
      case 5: e = launch_vjp_dn<2, 5>(fp32, a, s, &blocks); break;
      case 6: e = launch_vjp_dn<2, 6>(fp32, a, s, &blocks); break;
      case 7: e = launch_vjp_dn<2, 7>(fp32, a, s, &blocks); break;
    }
  } else if (dim == 3) {
    switch (N) {
      case 1: e = launch_vjp_dn<3, 1>(fp32, a, s, &blocks); break;
      case 2: e = launch_vjp_dn<3, 2>(fp32, a, s, &blocks); break;
      case 3: e = launch_vjp_dn<3, 3>(fp32, a, s, &blocks); break;
      case 4: e = launch_vjp_dn<3, 4>(fp32, a, s, &blocks); break;
      case 5: e = launch_vjp_dn<3, 5>(fp32, a, s, &blocks); break;
    }
  }
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
