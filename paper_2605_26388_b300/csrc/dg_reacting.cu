// dg_reacting.cu -- residual and SSP-RK3 stage of the single-temperature reacting
// Navier-Stokes equations (Sec. 2 reacting system) on periodic 3D Cartesian meshes, FP64.
//
// One stage is two launches over the elements of an instance:
//   1. k_br1_faces: BR1 gradients (Sec. 3.1.2, Eq. br1_avg) of W = (u, v, w, T) at every node
//      of the element, and the element's own viscous flux F_v^l (Eq. tau, q = -k grad T) at
//      its six faces, written to a face buffer fb[elem][face][4][(N+1)^2] (the four non-zero
//      components: three momentum rows and energy).
//   2. k_reacting_stage: the residual
//        L = -sum_l (2/dx_l) D (F^l - F_v^l)                       (strong volume form)
//            -/+ (2/dx_l)(1/w) [(F* - F^l) - ((F_v^l)* - F_v^l)]  (Eq. surf_int, Eq. br1_flux)
//            + omega                                            (Sec. 3.1.3, App. C)
//      with F* the Rusanov flux (frozen mixture sound speed), (F_v^l)* the BR1 average of the
//      own and the neighbour's face value (the latter read from the face buffer), and the
//      Arrhenius source evaluated in FP64; then the Shu-Osher stage update (App. B).
// The gradient is recomputed in launch 2 from the same inputs by the same code, so the
// neighbour's face value and the own one come from identical arithmetic.
//
// Threads: one thread per node, EPB = 128 / (N+1)^3 elements per 128-thread CTA; face work
// (6 (N+1)^2 face nodes per element) is spread over all threads of the CTA.
#include <cmath>

#include "dg_device.cuh"
#include "dg_internal.h"

namespace dg {
namespace {

constexpr int kRT = 128;

template <int N, int NS>
struct RG {
  static constexpr int N1 = N + 1, NP = N1 * N1 * N1, NFN = N1 * N1, NV = NS + 4;
  static constexpr int EPB = kRT / NP;
  static constexpr int NFJ = 6 * NFN;  // face nodes of one element
  static constexpr int NSL = NS + 1;   // concentration slots (last one holds 1.0)
  // stage kernel shared memory per element (doubles)
  static constexpr int E_US = 0;                        // U            [NV][NP]
  static constexpr int E_UT = E_US + NV * NP;           // nbr U traces [6][NV][NFN] -> lifts
  static constexpr int E_W = E_UT + 6 * NV * NFN;       // W            [4][NP]
  static constexpr int E_WT = E_W + 4 * NP;             // nbr W traces [6][4][NFN]
  static constexpr int E_FT = E_WT + 24 * NFN;          // nbr F_v      [6][4][NFN]
  static constexpr int E_FO = E_FT + 24 * NFN;          // own F_v      [6][4][NFN]
  static constexpr int E_H = E_FO + 24 * NFN;           // F^l - F_v^l  [NV][NP]
  static constexpr int E_SIZE = E_H + NV * NP;
  // per CTA: D, species table, concentration slots
  static constexpr int C_D = 0;
  static constexpr int C_SP = C_D + N1 * N1;            // R, cv, h0, scale [4][NS]
  static constexpr int C_X = C_SP + 4 * NS;             // [NSL][kRT]
  static constexpr int C_SIZE = C_X + NSL * kRT;
  static constexpr size_t stage_smem() { return sizeof(double) * (size_t)(C_SIZE + EPB * E_SIZE); }
  // gradient kernel: W [4][NP] and W traces [6][4][NFN] per element
  static constexpr int G_W = 0, G_WT = 4 * NP, G_SIZE = 4 * NP + 24 * NFN;
  static constexpr size_t grad_smem() {
    return sizeof(double) * (size_t)(N1 * N1 + 3 * NS + EPB * G_SIZE);
  }
};

template <int N1>
__device__ __forceinline__ int face_node(int l, int side, int jf) {
  const int a = jf % N1, b = jf / N1, c = side ? N1 - 1 : 0;
  return l == 0 ? c + N1 * (a + N1 * b) : (l == 1 ? a + N1 * (c + N1 * b) : a + N1 * (b + N1 * c));
}

__device__ __forceinline__ int neighbour(const int* nel, int e, int l, int dir) {
  int c[3] = {e % nel[0], (e / nel[0]) % nel[1], e / (nel[0] * nel[1])};
#pragma unroll
  for (int d = 0; d < 3; ++d)
    if (d == l) c[d] = (c[d] + dir + nel[d]) % nel[d];
  return c[0] + nel[0] * (c[1] + nel[1] * c[2]);
}

__device__ __forceinline__ double pick3(int l, double a, double b, double c) {
  return l == 0 ? a : (l == 1 ? b : c);
}

// Mixture state of one node (calorically perfect species, single temperature):
// T = (E - rho|u|^2/2 - sum rho_s h0_s) / sum rho_s cv_s, p = T sum rho_s R_s,
// frozen sound speed a^2 = (1 + sum rho_s R_s / sum rho_s cv_s) p / rho, c_p of the mixture.
struct Mx {
  double rho, v[3], T, p, a, cp;
};

template <int NS>
__device__ __forceinline__ Mx mixture(const double* u, const double* sp) {
  double rho = 0.0, rR = 0.0, rcv = 0.0, rh0 = 0.0;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    rho += u[s];
    rR = fma(u[s], sp[s], rR);
    rcv = fma(u[s], sp[NS + s], rcv);
    rh0 = fma(u[s], sp[2 * NS + s], rh0);
  }
  Mx m;
  m.rho = rho;
  const double irho = 1.0 / rho;
  double kin = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    m.v[d] = u[NS + d] * irho;
    kin = fma(u[NS + d], m.v[d], kin);
  }
  const double ircv = 1.0 / rcv;
  m.T = (u[NS + 3] - 0.5 * kin - rh0) * ircv;
  m.p = rR * m.T;
  m.a = sqrt(fma(rR, ircv, 1.0) * m.p * irho);
  m.cp = (rcv + rR) * irho;
  return m;
}

// Inviscid flux in direction l (runtime l allowed: no dynamic register indexing).
template <int NS>
__device__ __forceinline__ void inv_flux(int l, const double* u, const Mx& m, double* F) {
  const double vl = pick3(l, m.v[0], m.v[1], m.v[2]);
#pragma unroll
  for (int s = 0; s < NS; ++s) F[s] = u[s] * vl;
#pragma unroll
  for (int d = 0; d < 3; ++d) F[NS + d] = fma(u[NS + d], vl, d == l ? m.p : 0.0);
  F[NS + 3] = (u[NS + 3] + m.p) * vl;
}

// Viscous flux in direction L (compile-time) from the gradient S[q][l] of (u, v, w, T):
// tau_jL = mu (d_L u_j + d_j u_L) - (2/3) mu (div u) delta_jL, energy u . tau_L + k d_L T.
template <int L>
__device__ __forceinline__ void visc_flux(const double (&S)[4][3], const Mx& m, double mu, double kfac,
                                          double* Fv) {
  const double div = S[0][0] + S[1][1] + S[2][2];
  double work = 0.0;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    double t = mu * (S[j][L] + S[L][j]);
    if (j == L) t = fma(-2.0 / 3.0 * mu, div, t);
    Fv[j] = t;
    work = fma(m.v[j], t, work);
  }
  Fv[3] = fma(kfac * m.cp, S[3][L], work);
}

// BR1 gradient of W at node q of element slot el (Eq. br1_avg): for each direction l,
// (2/dx_l) [ sum_m D_{i_l m} W_m + (upper) (W^ - W_N)/w_N - (lower) (W^ - W_0)/w_0 ],
// W^ = (W_own + W_nbr)/2.  W: [4][NP] of the element, Wt: [6][4][NFN] neighbour traces.
template <int N>
__device__ __forceinline__ void br1_gradient(int q, const double* W, const double* Wt, const double* D,
                                             const double* s, double lift, double (&S)[4][3]) {
  constexpr int N1 = N + 1, NFN = N1 * N1;
  const int ijk[3] = {q % N1, (q / N1) % N1, q / NFN};
  constexpr int stride_l[3] = {1, N1, NFN};
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const int il = ijk[l];
    const int q0 = q - il * stride_l[l];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int m = 0; m < N1; ++m) {
      const double d = D[il * N1 + m];
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[c] = fma(d, W[c * (N1 * NFN) + q0 + m * stride_l[l]], acc[c]);
    }
    if (il == N || il == 0) {
      const int side = il == N ? 1 : 0;
      const int jf = l == 0 ? ijk[1] + N1 * ijk[2] : (l == 1 ? ijk[0] + N1 * ijk[2] : ijk[0] + N1 * ijk[1]);
      const double* wt = Wt + (2 * l + side) * 4 * NFN + jf;
      const double h = side ? 0.5 * lift : -0.5 * lift;
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[c] = fma(h, wt[c * NFN] - W[c * (N1 * NFN) + q], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) S[c][l] = s[l] * acc[c];
  }
}

template <int NS>
__device__ __forceinline__ void load_species(const MechDev* __restrict__ mech, double* sp) {
  for (int t = threadIdx.x; t < 4 * NS; t += blockDim.x) {
    const int k = t / NS, s = t % NS;
    const double* src = k == 0 ? mech->R : (k == 1 ? mech->cv : (k == 2 ? mech->h0 : mech->scale));
    sp[t] = src[s];
  }
}

// W = (u, v, w, T) and its error flags for one node state.
template <int NS>
__device__ __forceinline__ unsigned node_w(const double* u, const double* sp, double* w4, int stride,
                                           Mx* out) {
  const Mx m = mixture<NS>(u, sp);
  w4[0] = m.v[0];
  w4[stride] = m.v[1];
  w4[2 * stride] = m.v[2];
  w4[3 * stride] = m.T;
  if (out) *out = m;
  return (m.rho > 0.0 && m.T > 0.0) ? 0u : 2u;
}

// Own W and neighbour W traces (and optionally U, U traces) of the CTA's elements.
template <int N, int NS, bool KEEP_U>
__device__ __forceinline__ unsigned load_element_w(const ReactArgs& a, int e0, double* smem_el, int esz,
                                                   int off_w, int off_wt, int off_us, int off_ut,
                                                   const double* sp) {
  using G = RG<N, NS>;
  unsigned flag = 0;
  const int t = threadIdx.x;
  if (t < G::EPB * G::NP) {
    const int el = t / G::NP, q = t % G::NP, e = e0 + el;
    if (e < a.n_elem) {
      double* sm = smem_el + el * esz;
      const long long gi = a.base + (long long)e * G::NP + q;
      double u[G::NV];
#pragma unroll
      for (int v = 0; v < G::NV; ++v) {
        u[v] = a.U[v * a.stride + gi];
        if (KEEP_U) sm[off_us + v * G::NP + q] = u[v];
      }
      flag |= node_w<NS>(u, sp, sm + off_w + q, G::NP, nullptr);
    }
  }
  for (int idx = t; idx < G::EPB * G::NFJ; idx += kRT) {
    const int el = idx / G::NFJ, r = idx % G::NFJ, f = r / G::NFN, jf = r % G::NFN;
    const int e = e0 + el;
    if (e >= a.n_elem) continue;
    double* sm = smem_el + el * esz;
    const int l = f >> 1, side = f & 1;
    const int en = neighbour(a.nel, e, l, side ? 1 : -1);
    const long long gi = a.base + (long long)en * G::NP + face_node<G::N1>(l, side ^ 1, jf);
    double u[G::NV];
#pragma unroll
    for (int v = 0; v < G::NV; ++v) {
      u[v] = a.U[v * a.stride + gi];
      if (KEEP_U) sm[off_ut + (f * G::NV + v) * G::NFN + jf] = u[v];
    }
    flag |= node_w<NS>(u, sp, sm + off_wt + f * 4 * G::NFN + jf, G::NFN, nullptr);
  }
  return flag;
}

// ---------------------------------------------------------------------------------------
// Launch 1: BR1 gradients and the element's own viscous flux on its faces.
// ---------------------------------------------------------------------------------------
template <int N, int NS>
__global__ void __launch_bounds__(kRT) k_br1_faces(const ReactArgs a) {
  using G = RG<N, NS>;
  extern __shared__ double smem[];
  double* D = smem;
  double* sp = D + G::N1 * G::N1;
  double* el_base = sp + 3 * NS;
  const int t = threadIdx.x;
  for (int k = t; k < G::N1 * G::N1; k += kRT) D[k] = a.D[k];
  for (int k = t; k < 3 * NS; k += kRT) {
    const int c = k / NS, s = k % NS;
    D[G::N1 * G::N1 + k] = c == 0 ? a.mech->R[s] : (c == 1 ? a.mech->cv[s] : a.mech->h0[s]);
  }
  __syncthreads();
  const int e0 = blockIdx.x * G::EPB;
  load_element_w<N, NS, false>(a, e0, el_base, G::G_SIZE, G::G_W, G::G_WT, 0, 0, sp);
  __syncthreads();
  if (t >= G::EPB * G::NP) return;
  const int el = t / G::NP, q = t % G::NP, e = e0 + el;
  if (e >= a.n_elem) return;
  const double* sm = el_base + el * G::G_SIZE;
  double S[4][3];
  br1_gradient<N>(q, sm + G::G_W, sm + G::G_WT, D, a.s, a.lift, S);
  const int ijk[3] = {q % G::N1, (q / G::N1) % G::N1, q / G::NFN};
  if (ijk[0] != 0 && ijk[0] != N && ijk[1] != 0 && ijk[1] != N && ijk[2] != 0 && ijk[2] != N) return;
  // own mixture state again (cheap next to the gradient) for u and c_p
  double u[G::NV];
  const long long gi = a.base + (long long)e * G::NP + q;
#pragma unroll
  for (int v = 0; v < G::NV; ++v) u[v] = a.U[v * a.stride + gi];
  const Mx m = mixture<NS>(u, sp);
  double* fbe = a.fb + (size_t)e * 6 * 4 * G::NFN;
  double Fv[4];
#define DG_FACE_OUT(L)                                                                       \
  if (ijk[L] == 0 || ijk[L] == N) {                                                          \
    visc_flux<L>(S, m, a.mu, a.kfac, Fv);                                                    \
    const int jf = L == 0 ? ijk[1] + G::N1 * ijk[2]                                          \
                          : (L == 1 ? ijk[0] + G::N1 * ijk[2] : ijk[0] + G::N1 * ijk[1]);     \
    double* dst = fbe + (2 * L + (ijk[L] == N ? 1 : 0)) * 4 * G::NFN + jf;                   \
    for (int c = 0; c < 4; ++c) dst[c * G::NFN] = Fv[c];                                     \
  }
  DG_FACE_OUT(0)
  DG_FACE_OUT(1)
  DG_FACE_OUT(2)
#undef DG_FACE_OUT
}

// ---------------------------------------------------------------------------------------
// Launch 2: the fused stage.
// ---------------------------------------------------------------------------------------
template <int N, int NS>
__global__ void __launch_bounds__(kRT) k_reacting_stage(const ReactArgs a) {
  using G = RG<N, NS>;
  constexpr int N1 = G::N1, NP = G::NP, NFN = G::NFN, NV = G::NV;
  extern __shared__ double smem[];
  double* D = smem + G::C_D;
  double* sp = smem + G::C_SP;
  double* X = smem + G::C_X;
  double* el_base = smem + G::C_SIZE;
  const int t = threadIdx.x;
  for (int k = t; k < N1 * N1; k += kRT) D[k] = a.D[k];
  load_species<NS>(a.mech, sp);
  // neighbour viscous face fluxes from launch 1
  const int e0 = blockIdx.x * G::EPB;
  for (int idx = t; idx < G::EPB * 24 * NFN; idx += kRT) {
    const int el = idx / (24 * NFN), r = idx % (24 * NFN), f = r / (4 * NFN), cj = r % (4 * NFN);
    const int e = e0 + el;
    if (e >= a.n_elem) continue;
    const int l = f >> 1, side = f & 1;
    const int en = neighbour(a.nel, e, l, side ? 1 : -1);
    el_base[el * G::E_SIZE + G::E_FT + r] = a.fb[((size_t)en * 6 + (2 * l + (side ^ 1))) * 4 * NFN + cj];
  }
  __syncthreads();
  unsigned flag = load_element_w<N, NS, true>(a, e0, el_base, G::E_SIZE, G::E_W, G::E_WT, G::E_US, G::E_UT, sp);
  __syncthreads();

  const bool node_thread = t < G::EPB * NP;
  const int el = node_thread ? t / NP : 0, q = node_thread ? t % NP : 0, e = e0 + el;
  const bool active = node_thread && e < a.n_elem;
  double* sm = el_base + el * G::E_SIZE;
  const int ijk[3] = {q % N1, (q / N1) % N1, q / NFN};
  double u[NV], res[NV];
  Mx m{};
  double S[4][3];
#pragma unroll
  for (int v = 0; v < NV; ++v) res[v] = 0.0;
  if (active) {
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = sm[G::E_US + v * NP + q];
    m = mixture<NS>(u, sp);
    br1_gradient<N>(q, sm + G::E_W, sm + G::E_WT, D, a.s, a.lift, S);
  }
  // volume term, one direction at a time through the H buffer
#define DG_VOLUME_DIR(L)                                                                      \
  {                                                                                           \
    if (active) {                                                                             \
      double F[NV], Fv[4];                                                                    \
      inv_flux<NS>(L, u, m, F);                                                               \
      visc_flux<L>(S, m, a.mu, a.kfac, Fv);                                                   \
      _Pragma("unroll") for (int c = 0; c < 4; ++c) F[NS + c] -= Fv[c];                       \
      _Pragma("unroll") for (int v = 0; v < NV; ++v) sm[G::E_H + v * NP + q] = F[v];          \
      if (ijk[L] == 0 || ijk[L] == N) {                                                       \
        const int jf = L == 0 ? ijk[1] + N1 * ijk[2]                                          \
                              : (L == 1 ? ijk[0] + N1 * ijk[2] : ijk[0] + N1 * ijk[1]);        \
        double* dst = sm + G::E_FO + (2 * L + (ijk[L] == N ? 1 : 0)) * 4 * NFN + jf;          \
        _Pragma("unroll") for (int c = 0; c < 4; ++c) dst[c * NFN] = Fv[c];                   \
      }                                                                                       \
    }                                                                                         \
    __syncthreads();                                                                          \
    if (active) {                                                                             \
      constexpr int st = L == 0 ? 1 : (L == 1 ? N1 : NFN);                                    \
      const int il = ijk[L], q0 = q - il * st;                                                \
      double acc[NV];                                                                         \
      _Pragma("unroll") for (int v = 0; v < NV; ++v) acc[v] = 0.0;                            \
      _Pragma("unroll") for (int mm = 0; mm < N1; ++mm) {                                     \
        const double d = D[il * N1 + mm];                                                     \
        _Pragma("unroll") for (int v = 0; v < NV; ++v)                                        \
            acc[v] = fma(d, sm[G::E_H + v * NP + q0 + mm * st], acc[v]);                      \
      }                                                                                       \
      _Pragma("unroll") for (int v = 0; v < NV; ++v) res[v] = fma(-a.s[L], acc[v], res[v]);   \
    }                                                                                         \
    __syncthreads();                                                                          \
  }
  DG_VOLUME_DIR(0)
  DG_VOLUME_DIR(1)
  DG_VOLUME_DIR(2)
#undef DG_VOLUME_DIR

  // face jobs: Rusanov flux and the BR1 viscous interface flux; the lifted difference
  // (F* - F_own) - ((F_v)* - F_v,own) replaces the neighbour trace in place
  for (int idx = t; idx < G::EPB * G::NFJ; idx += kRT) {
    const int fel = idx / G::NFJ, r = idx % G::NFJ, f = r / NFN, jf = r % NFN;
    if (e0 + fel >= a.n_elem) continue;
    double* fs = el_base + fel * G::E_SIZE;
    const int l = f >> 1, side = f & 1;
    const int qo = face_node<N1>(l, side, jf);
    double uo[NV], un[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      uo[v] = fs[G::E_US + v * NP + qo];
      un[v] = fs[G::E_UT + (f * NV + v) * NFN + jf];
    }
    const Mx mo = mixture<NS>(uo, sp), mn = mixture<NS>(un, sp);
    double Fo[NV], Fn[NV];
    inv_flux<NS>(l, uo, mo, Fo);
    inv_flux<NS>(l, un, mn, Fn);
    const double lam = fmax(fabs(pick3(l, mo.v[0], mo.v[1], mo.v[2])) + mo.a,
                            fabs(pick3(l, mn.v[0], mn.v[1], mn.v[2])) + mn.a);
    // F* = (F_L + F_R)/2 - lam (U_R - U_L)/2; with L/R the lower/upper side of the face
    const double sgn = side ? 1.0 : -1.0;  // U_R - U_L = sgn (un - uo)
    double dlt[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double Fs = 0.5 * (Fo[v] + Fn[v]) - 0.5 * lam * sgn * (un[v] - uo[v]);
      dlt[v] = Fs - Fo[v];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
      dlt[NS + c] -= 0.5 * (fs[G::E_FT + f * 4 * NFN + c * NFN + jf] - fs[G::E_FO + f * 4 * NFN + c * NFN + jf]);
#pragma unroll
    for (int v = 0; v < NV; ++v) fs[G::E_UT + (f * NV + v) * NFN + jf] = dlt[v];
  }
  __syncthreads();
  if (!active) return;
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const int il = ijk[l];
    if (il != 0 && il != N) continue;
    const int side = il == N ? 1 : 0;
    const int jf = l == 0 ? ijk[1] + N1 * ijk[2] : (l == 1 ? ijk[0] + N1 * ijk[2] : ijk[0] + N1 * ijk[1]);
    const double c = (side ? -a.s[l] : a.s[l]) * a.lift;
    const double* ls = sm + G::E_UT + (2 * l + side) * NV * NFN + jf;
#pragma unroll
    for (int v = 0; v < NV; ++v) res[v] = fma(c, ls[v * NFN], res[v]);
  }

  // Arrhenius source (Sec. 3.1.3, Eqs. src_reaction_rate and src_omega; App. C), FP64:
  // [X_s] = rho_s 1e-6 / W_s, k_f = exp(lnA + b ln T - Ta/T), ln K_c from the five-term fit
  // in Z = 1e4/T, R_r = k_f prod [X]^nu' - (k_f / K_c) prod [X]^nu'',
  // omega_s = sum_r W_s 1e6 (nu''_s - nu'_s) R_r.
  const int nr = a.mech->nr;
  if (nr > 0) {
    const double lnT = log(m.T), invT = 1.0 / m.T;
    const double Z = 1.0e4 * invT, Zi = 1.0e-4 * m.T, lnZ = a.ln1e4 - lnT, Z2 = Z * Z;
#pragma unroll
    for (int s2 = 0; s2 < NS; ++s2) X[s2 * kRT + t] = u[s2] * sp[3 * NS + s2];
    X[NS * kRT + t] = 1.0;
    double om[NS];
#pragma unroll
    for (int s2 = 0; s2 < NS; ++s2) om[s2] = 0.0;
    for (int r = 0; r < nr; ++r) {
      const RxnDev& R = a.mech->rx[r];
      const double lkf = fma(R.b, lnT, fma(-R.Ta, invT, R.lnA));
      const double lkc = fma(R.kc[0], Zi, fma(R.kc[2], lnZ, fma(R.kc[3], Z, fma(R.kc[4], Z2, R.kc[1]))));
      const double kf = exp(lkf), kb = exp(lkf - lkc);
      const double pf = X[R.f[0] * kRT + t] * X[R.f[1] * kRT + t] * X[R.f[2] * kRT + t];
      const double pb = X[R.bk[0] * kRT + t] * X[R.bk[1] * kRT + t] * X[R.bk[2] * kRT + t];
      const double rate = fma(kf, pf, -kb * pb);
#pragma unroll
      for (int s2 = 0; s2 < NS; ++s2) om[s2] = fma(R.coef[s2], rate, om[s2]);
    }
#pragma unroll
    for (int s2 = 0; s2 < NS; ++s2) res[s2] += om[s2];
  }

  const long long gi = a.base + (long long)e * NP + q;
  bool finite = true;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double x = res[v];
    if (a.mode == 1) {
      x = fma(a.cb, u[v], a.cbdt * res[v]);
      if (a.need_un) x = fma(a.ca, a.Un[v * a.stride + gi], x);
    }
    finite = finite && finite64(x);
    a.out[v * a.stride + gi] = x;
  }
  if (!finite) flag |= 1u;
  if (flag) atomicOr(a.err, flag);
}

// Largest |u| + a and largest 1/rho over the nodes of one instance.
template <int NS>
__global__ void k_max_speed_mix(const double* U, long long stride, long long base, long long n,
                                const MechDev* __restrict__ mech, unsigned long long* out2) {
  __shared__ double sp[4 * NS];
  load_species<NS>(mech, sp);
  __syncthreads();
  double lam = 0.0, irho = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    double u[NS + 4];
#pragma unroll
    for (int v = 0; v < NS + 4; ++v) u[v] = U[v * stride + base + q];
    const Mx m = mixture<NS>(u, sp);
    lam = fmax(lam, sqrt(m.v[0] * m.v[0] + m.v[1] * m.v[1] + m.v[2] * m.v[2]) + m.a);
    irho = fmax(irho, 1.0 / m.rho);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lam = fmax(lam, __shfl_xor_sync(0xffffffffu, lam, o));
    irho = fmax(irho, __shfl_xor_sync(0xffffffffu, irho, o));
  }
  __shared__ double red[2][32];
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = lam;
    red[1][threadIdx.x >> 5] = irho;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      lam = fmax(lam, red[0][w]);
      irho = fmax(irho, red[1][w]);
    }
    atomicMax(out2, (unsigned long long)__double_as_longlong(lam));
    atomicMax(out2 + 1, (unsigned long long)__double_as_longlong(irho));
  }
}

template <int N, int NS>
cudaError_t prepare_one() {
  using G = RG<N, NS>;
  cudaError_t e = cudaFuncSetAttribute(k_reacting_stage<N, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)G::stage_smem());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_br1_faces<N, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)G::grad_smem());
  return e;
}

template <int N, int NS>
cudaError_t launch_one(const ReactArgs& a, cudaStream_t s) {
  using G = RG<N, NS>;
  if (a.n_elem <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((a.n_elem + G::EPB - 1) / G::EPB);
  k_br1_faces<N, NS><<<grid, kRT, G::grad_smem(), s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_reacting_stage<N, NS><<<grid, kRT, G::stage_smem(), s>>>(a);
  return cudaGetLastError();
}

#define DG_REACT_DISPATCH(CALL)                 \
  switch (ns * 16 + N) {                        \
    case 1 * 16 + 1: return CALL(1, 1);         \
    case 1 * 16 + 2: return CALL(2, 1);         \
    case 1 * 16 + 3: return CALL(3, 1);         \
    case 1 * 16 + 4: return CALL(4, 1);         \
    case 5 * 16 + 1: return CALL(1, 5);         \
    case 5 * 16 + 2: return CALL(2, 5);         \
    case 5 * 16 + 3: return CALL(3, 5);         \
    case 5 * 16 + 4: return CALL(4, 5);         \
    default: return cudaErrorInvalidValue;      \
  }

}  // namespace

bool have_reacting(int N, int ns) { return (ns == 1 || ns == 5) && N >= 1 && N <= kMaxReactingN; }

cudaError_t prepare_reacting(int N, int ns) {
#define DG_P(n, s) prepare_one<n, s>()
  DG_REACT_DISPATCH(DG_P)
#undef DG_P
}

cudaError_t launch_reacting(int N, int ns, const ReactArgs& a, cudaStream_t s) {
#define DG_L(n, sp) launch_one<n, sp>(a, s)
  DG_REACT_DISPATCH(DG_L)
#undef DG_L
}

cudaError_t launch_max_speed_mix(int ns, const double* U, long long stride, long long base,
                                 long long n_nodes, const MechDev* mech,
                                 unsigned long long* out2, cudaStream_t s) {
  if (n_nodes <= 0) return cudaSuccess;
  const long long want = (n_nodes + 255) / 256;
  const unsigned grid = (unsigned)(want < 148 * 16 ? want : 148 * 16);
  if (ns == 1) k_max_speed_mix<1><<<grid, 256, 0, s>>>(U, stride, base, n_nodes, mech, out2);
  else if (ns == 5) k_max_speed_mix<5><<<grid, 256, 0, s>>>(U, stride, base, n_nodes, mech, out2);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace dg
