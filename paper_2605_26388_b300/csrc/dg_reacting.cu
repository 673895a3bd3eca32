// dg_reacting.cu -- residual, SSP-RK stage and implicit source substep of the
// single-temperature reacting Navier-Stokes equations (Sec. 2 reacting system) on 3D
// Cartesian meshes, periodic or with per-face boundary conditions (slip, no-slip adiabatic and
// isothermal walls, supersonic inflow and outflow, Dirichlet: Sec. 3.1.1 boundary functors for
// the inviscid flux, Sec. 3.1.2 boundary kernels for the BR1 trace and the viscous flux).
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
//      Arrhenius source; then the Shu-Osher stage update (App. B).
// The gradient is recomputed in launch 2 from the same inputs by the same code, so the
// neighbour's face value and the own one come from identical arithmetic.
//
// Primitive cache: the mixture state of every node (u, v, w, T, p - p_ref, a, c_p in R and T
// in FP64) is computed once per stage, by the stage kernel for its output state (or by
// k_react_prims for a state that did not come from a stage), and both launches of the next
// stage read it for their own nodes and the neighbours' face traces instead of evaluating
// the FP64 mixture again (five times per node otherwise).
//
// Precision: the mixture state of every node (T, p, sound speed, c_p from the FP64 conserved
// variables), the Arrhenius source and the stage update are FP64 in both modes; gradients,
// viscous and inviscid fluxes, the Rusanov flux, the contractions and the lifts run in the
// flux type R (double, or float in the FP32-mixed mode).  The momentum flux carries
// p - p_ref (a constant shift that leaves the discrete operator unchanged, as for Euler).
//
// Threads: one thread per node, EPB = 128 / (N+1)^3 elements per 128-thread CTA; face work
// (6 (N+1)^2 face nodes per element) is spread over all threads of the CTA.
#include <cmath>

#include "dg_device.cuh"
#include "dg_internal.h"

namespace dg {
namespace {

constexpr int kRT = 128;

// Per-launch geometry.  TT: the two-temperature model (E_v appended to the state, T_v a
// gradient variable, E_v a viscous flux row).
template <int N, int NS, bool TT, class R>
struct RG {
  static constexpr int N1 = N + 1, NP = N1 * N1 * N1, NFN = N1 * N1;
  static constexpr int NV = NS + 4 + (TT ? 1 : 0);
  static constexpr int NW = TT ? 5 : 4;    // gradient variables: u, v, w, T (, T_v)
  static constexpr int NFV = NW;           // viscous face flux rows: 3 momenta, E (, E_v)
  static constexpr int NPR = NW + 2;       // staged primitives: u, v, w, T (, T_v), p - p_ref, a
  static constexpr int RPD = NW, RA = NW + 1, RCP = NW + 2, RCV = NW + 3;  // cache rows
  static constexpr int NSP = TT ? 5 : 4;   // species table rows: R, cv, h0, 1e-6/W (, theta)
  static constexpr int EPB = kRT / NP;
  static constexpr int NFJ = 6 * NFN;  // face nodes of one element
  static constexpr int NSL = NS + 1;   // concentration slots (last one holds 1.0)
  // stage kernel, per element (R)
  static constexpr int E_US = 0;                        // U            [NV][NP]
  static constexpr int E_UT = E_US + NV * NP;           // nbr U traces [6][NV][NFN] -> lifts
  static constexpr int E_P = E_UT + 6 * NV * NFN;       // primitives   [NPR][NP]
  static constexpr int E_PT = E_P + NPR * NP;           // nbr prims    [6][NPR][NFN]
  static constexpr int E_FT = E_PT + 6 * NPR * NFN;     // nbr F_v      [6][NFV][NFN]
  static constexpr int E_FO = E_FT + 6 * NFV * NFN;     // own F_v      [6][NFV][NFN]
  static constexpr int E_H = E_FO + 6 * NFV * NFN;      // F^l - F_v^l  [NV][NP]
  static constexpr int E_SIZE = E_H + NV * NP;
  // stage kernel, per CTA: species table, exp table, concentration slots (double), D (R)
  static constexpr int C_SP = 0;                        // species table [NSP][NS]
  static constexpr int C_MW = C_SP + 5 * 8;             // TT: Millikan-White A, C [2][NS][NS]
  static constexpr int C_E2 = C_MW + 2 * 8 * 8;         // 2^(j/64) [64]
  static constexpr int C_X = C_E2 + 64;                 // [NSL][kRT]
  static constexpr int C_DBL = C_X + NSL * kRT;
  static constexpr size_t stage_smem() {
    return sizeof(double) * (size_t)C_DBL + sizeof(R) * (size_t)(N1 * N1 + EPB * E_SIZE);
  }
  // gradient kernel, per element (R): primitives and trace primitives
  static constexpr int G_P = 0, G_PT = NPR * NP, G_SIZE = NPR * NP + 6 * NPR * NFN;
  static constexpr size_t grad_smem() { return sizeof(R) * (size_t)(N1 * N1 + EPB * G_SIZE); }
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

// Domain face (2 l + side) that side `side` (0 lower, 1 upper) of element e in direction l
// lies on when that face carries a boundary condition, else -1.
__device__ __forceinline__ int wall_face(const ReactArgs& a, int e, int l, int side) {
  const int f = 2 * l + side;
  if (a.bnd.bc[f] == 0) return -1;
  const int c = l == 0 ? e % a.nel[0] : (l == 1 ? (e / a.nel[0]) % a.nel[1] : e / (a.nel[0] * a.nel[1]));
  return (side ? c == a.nel[l] - 1 : c == 0) ? f : -1;
}

// exp(x) for the Arrhenius rates, after Tang's table-driven method (P. T. P. Tang, ACM TOMS
// 15(2), 1989): x = (64 m + j) ln2/64 + r with |r| <= ln2/128, exp(x) = 2^m 2^(j/64) e^r;
// e^r - 1 from its degree-5 Taylor polynomial (truncation < 4e-17 relative), 2^(j/64) from a
// 64-entry FP64 table computed on the host, 2^m added to the exponent field.  ln2/64 is
// split into a 33-bit head (n * head exact for |n| < 2^20) and a tail.  Ten FP64 operations;
// |x| >= 704 (outside the rates' range) falls back to the library function.
__device__ __forceinline__ double exp_tab(double x, const double* tab) {
  const uint32_t ah = (uint32_t)__double2hiint(x) & 0x7fffffffu;
  if (ah >= 0x40860000u) return exp(x);
  const double kShift = 6755399441055744.0;  // 1.5 * 2^52: the sum's low word holds rint(x 64/ln2)
  const double t = fma(x, 92.33248261689366, kShift);
  const int n = __double2loint(t);
  const double nd = t - kShift;
  double r = fma(-nd, 0.010830424695086549, x);
  r = fma(-nd, 1.162596423439437e-12, r);
  const double p = fma(r * r, fma(r, fma(r, fma(r, 1.0 / 120.0, 1.0 / 24.0), 1.0 / 6.0), 0.5), r);
  const double T = tab[n & 63];
  const double y = fma(T, p, T);
  return __hiloint2double(__double2hiint(y) + ((n >> 6) << 20), __double2loint(y));
}

template <class T>
__device__ __forceinline__ T pick3(int l, T a, T b, T c) {
  return l == 0 ? a : (l == 1 ? b : c);
}

// Mixture state of one node, FP64 (calorically perfect species):
// T = (E - E_v - rho|u|^2/2 - sum rho_s h0_s) / sum rho_s cv_s (E_v = 0 for one temperature),
// p = T sum rho_s R_s, frozen sound speed a^2 = (1 + sum rho_s R_s / sum rho_s cv_s) p / rho,
// c_p of the mixture; two-temperature: T_v with E_v(T_v) = E_v and c_v,v = dE_v/dT_v / rho.
struct Mx {
  double rho, v[3], T, p, a, cp, Tv, cvv;
  bool conv;  // the T_v iteration converged
};

// Two-temperature: the vibrational temperature of the partial densities u[0..NS) with
// E_v(T_v) = sum rho_s R_s theta_s / (exp(theta_s / T_v) - 1) = Ev (harmonic oscillators;
// sp: species table, row 0 R_s, row 4 theta_s), by Newton's method from x0 (the node's T_v of
// the previous stage when known; else the exact inverse for the (rho R)-weighted mean theta);
// steps are limited to a factor 2 either way (E_v grows strictly with T_v, so the iterate
// stays positive and approaches the single root); stops after a step |dT_v| <= 1e-13 T_v, at
// most 50 updates.  Also returns rho c_v,v = dE_v/dT_v (at the last iterate but one, within
// 1e-13 relative of the root's).  exp by the table-driven exp_tab (e2tab).
template <int NS>
__device__ __forceinline__ double vib_temperature(const double* u, const double* sp, double Ev, double x0,
                                                  const double* e2tab, double& dEv, bool& conv) {
  double x = x0;
  if (!(x0 > 0.0)) {
    double rR = 0.0, rRt = 0.0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const double th = sp[4 * NS + s];
      if (th > 0.0) {
        rR = fma(u[s], sp[s], rR);
        rRt = fma(u[s] * sp[s], th, rRt);
      }
    }
    x = rRt * rcp64(rR) / log1p(rRt / Ev);
  }
  conv = false;
  dEv = 0.0;
  for (int it = 0; it < 50; ++it) {
    double f = -Ev, df = 0.0;
    const double ix = rcp64(x);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const double th = sp[4 * NS + s];
      if (th > 0.0) {
        const double y = th * ix, ey = exp_tab(y, e2tab), iem = rcp64(ey - 1.0);
        const double e = u[s] * sp[s] * th * iem;
        f += e;
        df = fma(e * y * ix, ey * iem, df);
      }
    }
    dEv = df;
    double xn = fma(-f, rcp64(df), x);
    xn = fmin(fmax(xn, 0.5 * x), 2.0 * x);
    const bool done = fabs(xn - x) <= 1e-13 * x;
    x = xn;
    if (done) {
      conv = true;
      break;
    }
  }
  return x;
}

template <int NS, bool TT>
__device__ __forceinline__ Mx mixture(const double* u, const double* sp, double tv_guess = 0.0,
                                      const double* e2tab = nullptr) {
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
  const double irho = rcp64(rho);
  double kin = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    m.v[d] = u[NS + d] * irho;
    kin = fma(u[NS + d], m.v[d], kin);
  }
  const double ircv = rcp64(rcv);
  const double Ev = TT ? u[NS + 4] : 0.0;
  m.T = (u[NS + 3] - Ev - 0.5 * kin - rh0) * ircv;
  m.p = rR * m.T;
  m.a = sqrt(fma(rR, ircv, 1.0) * m.p * irho);
  m.cp = (rcv + rR) * irho;
  m.Tv = m.T;
  m.cvv = 0.0;
  m.conv = true;
  if constexpr (TT) {
    double dEv;
    m.Tv = vib_temperature<NS>(u, sp, Ev, tv_guess, e2tab, dEv, m.conv);
    m.cvv = dEv * irho;
  }
  return m;
}

// Mixture state of one node into the primitive cache (R rows u, v, w, T (, T_v), p - p_ref,
// a, c_p (, c_v,v) at stride `stride`; T (and T_v) in FP64); returns the flags: 2 -- rho <= 0
// or T <= 0 (or T_v <= 0), in FP64; 4 -- the T_v iteration did not converge.
template <int NS, bool TT, class R>
__device__ __forceinline__ unsigned write_prims(const double* u, const double* sp, double p_ref, R* P,
                                                double* T64, long long stride, long long gi,
                                                double tv_guess = 0.0, const double* e2tab = nullptr) {
  const Mx m = mixture<NS, TT>(u, sp, tv_guess, e2tab);
  constexpr int W = TT ? 5 : 4;
  P[gi] = Ar<R>::load(m.v[0]);
  P[stride + gi] = Ar<R>::load(m.v[1]);
  P[2 * stride + gi] = Ar<R>::load(m.v[2]);
  P[3 * stride + gi] = Ar<R>::load(m.T);
  if (TT) P[4 * stride + gi] = Ar<R>::load(m.Tv);
  P[W * stride + gi] = Ar<R>::load(m.p - p_ref);
  P[(W + 1) * stride + gi] = Ar<R>::load(m.a);
  P[(W + 2) * stride + gi] = Ar<R>::load(m.cp);
  if (TT) P[(W + 3) * stride + gi] = Ar<R>::load(m.cvv);
  T64[gi] = m.T;
  if (TT) T64[stride + gi] = m.Tv;
  unsigned flag = (m.rho > 0.0 && m.T > 0.0 && m.Tv > 0.0) ? 0u : 2u;
  if (!m.conv) flag |= 4u;
  return flag;
}

// Inviscid flux in direction l (runtime l: no dynamic register indexing); the momentum rows
// carry pd = p - p_ref, the energy row (E + p) v_l with p = pd + p_ref; two-temperature: the
// E_v row E_v v_l.
template <int NS, bool TT, class R>
__device__ __forceinline__ void inv_flux(int l, const R* u, R v0, R v1, R v2, R pd, R p_ref, R* F) {
  const R vl = pick3(l, v0, v1, v2);
#pragma unroll
  for (int s = 0; s < NS; ++s) F[s] = u[s] * vl;
  F[NS + 0] = u[NS + 0] * vl + (l == 0 ? pd : R(0));
  F[NS + 1] = u[NS + 1] * vl + (l == 1 ? pd : R(0));
  F[NS + 2] = u[NS + 2] * vl + (l == 2 ? pd : R(0));
  F[NS + 3] = (u[NS + 3] + (pd + p_ref)) * vl;
  if constexpr (TT) F[NS + 4] = u[NS + 4] * vl;
}

// Viscous flux in direction L (compile-time) from the gradient S[q][l] of (u, v, w, T (, T_v)):
// tau_jL = mu (d_L u_j + d_j u_L) - (2/3) mu (div u) delta_jL, energy u . tau_L + k d_L T;
// two-temperature: + k_v d_L T_v in the energy row and the E_v row k_v d_L T_v.
template <int L, int NW, class R>
__device__ __forceinline__ void visc_flux(const R (&S)[NW][3], const R* v, R mu, R kcond, R kvib, R* Fv) {
  const R div = S[0][0] + S[1][1] + S[2][2];
  R work = R(0);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    R t = mu * (S[j][L] + S[L][j]);
    if (j == L) t = t - R(2.0 / 3.0) * mu * div;
    Fv[j] = t;
    work = work + v[j] * t;
  }
  Fv[3] = work + kcond * S[3][L];
  if constexpr (NW == 5) {
    const R qv = kvib * S[4][L];
    Fv[3] = Fv[3] + qv;
    Fv[4] = qv;
  }
  (void)kvib;
}

// BR1 gradient of W at node q (Eq. br1_avg): for each direction l,
// (2/dx_l) [ sum_m D_{i_l m} W_m + (upper) (W^ - W_N)/w_N - (lower) (W^ - W_0)/w_0 ],
// W^ = (W_own + W_nbr)/2.  W: rows c = 0..NW-1 of the element's primitives (row stride NP),
// Wt: the neighbours' face-trace primitives [6][NPR][NFN].
template <int N, int NW, int NPR, class R>
__device__ __forceinline__ void br1_gradient(int q, const R* W, const R* Wt, const R* D, const R* s,
                                             R lift, R (&S)[NW][3]) {
  constexpr int N1 = N + 1, NFN = N1 * N1, NP = N1 * NFN;
  const int ijk[3] = {q % N1, (q / N1) % N1, q / NFN};
  constexpr int stride_l[3] = {1, N1, NFN};
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const int il = ijk[l];
    const int q0 = q - il * stride_l[l];
    R acc[NW];
#pragma unroll
    for (int c = 0; c < NW; ++c) acc[c] = R(0);
#pragma unroll
    for (int m = 0; m < N1; ++m) {
      const R d = D[il * N1 + m];
#pragma unroll
      for (int c = 0; c < NW; ++c) acc[c] = acc[c] + d * W[c * NP + q0 + m * stride_l[l]];
    }
    if (il == N || il == 0) {
      const int side = il == N ? 1 : 0;
      const int jf = l == 0 ? ijk[1] + N1 * ijk[2] : (l == 1 ? ijk[0] + N1 * ijk[2] : ijk[0] + N1 * ijk[1]);
      const R* wt = Wt + (2 * l + side) * NPR * NFN + jf;
      const R h = side ? R(0.5) * lift : R(-0.5) * lift;
#pragma unroll
      for (int c = 0; c < NW; ++c) acc[c] = acc[c] + h * (wt[c * NFN] - W[c * NP + q]);
    }
#pragma unroll
    for (int c = 0; c < NW; ++c) S[c][l] = s[l] * acc[c];
  }
}

// ---- curved elements (Sec. 3.1.1 metric terms; Sec. 3.1.2 BR1 on the mapped element) ----
// The node's contravariant vectors Ja[l][d] and 1/J from the metric rows (FP64, converted to
// the flux precision).
template <class R>
__device__ __forceinline__ void node_metric(const ReactArgs& a, long long gi, R (&Ja)[3][3], R& iJ) {
#pragma unroll
  for (int l = 0; l < 3; ++l)
#pragma unroll
    for (int d = 0; d < 3; ++d) Ja[l][d] = Ar<R>::load(a.met[(long long)(l * 3 + d) * a.stride + gi]);
  iJ = Ar<R>::load(a.met[9 * a.stride + gi]);
}
// The contravariant vector Ja^l of the node (one direction).
template <class R>
__device__ __forceinline__ void node_metric_dir(const ReactArgs& a, long long gi, int l, R (&ja)[3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) ja[d] = Ar<R>::load(a.met[(long long)(l * 3 + d) * a.stride + gi]);
}
// Physical gradient from the reference-space BR1 derivative (br1_gradient with s = 1):
// S_d = (1/J) sum_l Ja^l_d S_l.
template <int NW, class R>
__device__ __forceinline__ void to_physical(const R (&Ja)[3][3], R iJ, R (&S)[NW][3]) {
#pragma unroll
  for (int c = 0; c < NW; ++c) {
    R p[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) p[d] = iJ * (Ja[0][d] * S[c][0] + Ja[1][d] * S[c][1] + Ja[2][d] * S[c][2]);
#pragma unroll
    for (int d = 0; d < 3; ++d) S[c][d] = p[d];
  }
}
// Contravariant viscous flux sum_d ja_d F_v^d, formed directly: the stress tensor applied to
// ja, the work of that traction, the conduction of the temperature gradient along ja.
template <int NW, int NFV, class R>
__device__ __forceinline__ void visc_flux_contra(const R (&S)[NW][3], const R* v, R mu, R kcond, R kvib,
                                                 const R (&ja)[3], R* Fv) {
  const R div = S[0][0] + S[1][1] + S[2][2];
  const R jd = R(2.0 / 3.0) * mu * div;
  R work = R(0);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    R t = R(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) t = t + ja[d] * (mu * (S[j][d] + S[d][j]));
    t = t - jd * ja[j];
    Fv[j] = t;
    work = work + v[j] * t;
  }
  Fv[3] = work + kcond * (ja[0] * S[3][0] + ja[1] * S[3][1] + ja[2] * S[3][2]);
  if constexpr (NW == 5) {
    const R qv = kvib * (ja[0] * S[4][0] + ja[1] * S[4][1] + ja[2] * S[4][2]);
    Fv[3] = Fv[3] + qv;
    Fv[4] = qv;
  }
  (void)kvib;
}
// Contravariant inviscid flux sum_d ja_d F^d of the mixture, formed directly with the
// contravariant velocity ja . v.
template <int NS, bool TT, class R>
__device__ __forceinline__ void inv_flux_contra(const R* u, R v0, R v1, R v2, R pd, R p_ref, const R (&ja)[3],
                                                R* F) {
  const R vn = ja[0] * v0 + ja[1] * v1 + ja[2] * v2;
#pragma unroll
  for (int s = 0; s < NS; ++s) F[s] = u[s] * vn;
  F[NS + 0] = u[NS + 0] * vn + ja[0] * pd;
  F[NS + 1] = u[NS + 1] * vn + ja[1] * pd;
  F[NS + 2] = u[NS + 2] * vn + ja[2] * pd;
  F[NS + 3] = (u[NS + 3] + (pd + p_ref)) * vn;
  if constexpr (TT) F[NS + 4] = u[NS + 4] * vn;
}

// Ghost neighbour value of the viscous face flux (momentum rows, energy) at a domain face
// with normal axis L, from the element's own flux Fv and its conduction part heat = k dT/dx_L,
// such that the BR1 average (Fv + gh)/2 is the boundary's viscous flux (Sec. 3.1.2 boundary
// kernels): slip wall -- only the normal-stress row survives; no-slip adiabatic -- stress
// rows kept, energy 0; no-slip isothermal -- stress rows kept, energy = heat; inflow,
// outflow, Dirichlet -- the interior flux itself.  Two-temperature (NFV = 5): heat_v =
// k_v dT_v/dx_L; the E_v row is 0 at slip and adiabatic walls and heat_v at isothermal ones,
// whose energy row is heat + heat_v.
template <int L, int NFV, class R>
__device__ __forceinline__ void ghost_viscous_flux(int type, const R* Fv, R heat, R heat_v, R* gh) {
#pragma unroll
  for (int c = 0; c < NFV; ++c) gh[c] = Fv[c];
  if (type == 1) {
#pragma unroll
    for (int c = 0; c < NFV; ++c)
      if (c != L) gh[c] = -Fv[c];
  } else if (type == 5) {
#pragma unroll
    for (int c = 3; c < NFV; ++c) gh[c] = -Fv[c];
  } else if (type == 6) {
    gh[3] = R(2) * (heat + heat_v) - Fv[3];
    if (NFV > 4) gh[NFV - 1] = R(2) * heat_v - Fv[NFV - 1];
  }
}

// Species table rows: R, cv, h0, 1e-6/W (, theta_v).
template <int NS>
__device__ __forceinline__ void load_species(const MechDev* __restrict__ mech, double* sp, int n) {
  for (int t = threadIdx.x; t < n * NS; t += blockDim.x) {
    const int k = t / NS, s = t % NS;
    const double* src = k == 0 ? mech->R : (k == 1 ? mech->cv : (k == 2 ? mech->h0 : (k == 3 ? mech->scale : mech->theta)));
    sp[t] = src[s];
  }
}

// Species production rates omega_s of one node (Sec. 3.1.3, Eqs. src_reaction_rate and
// src_omega; App. C), FP64: k_f = exp(lnA + b ln T_a - Ta/T_a), ln K_c from the five-term fit
// in Z = 1e4/T_a, R_r = k_f prod [X]^nu' - (k_f / K_c) prod [X]^nu'',
// omega_s = sum_r W_s 1e6 (nu''_s - nu'_s) R_r, with T_a = T, or (two-temperature, reactions
// flagged ta) T_a = sqrt(T T_v).  The concentrations [X_s] sit in this thread's slots
// X[s * xs] (slot NS holds 1.0, the factor of an empty place in a product).
template <int NS, bool TT>
__device__ __forceinline__ void species_rates(const MechDev* __restrict__ mech, int nr, double T, double Tv,
                                              const double* X, int xs, const double* e2tab,
                                              double ln1e4, double (&om)[NS]) {
  const double lnT = log(T), invT = rcp64(T);
  const double Z = 1.0e4 * invT, Zi = 1.0e-4 * T, lnZ = ln1e4 - lnT, Z2 = Z * Z;
  double lnTa = lnT, invTa = invT, Za = Z, Zia = Zi, lnZa = lnZ, Za2 = Z2;
  if constexpr (TT) {
    const double Ta = sqrt(T * Tv);
    lnTa = 0.5 * (lnT + log(Tv));
    invTa = rcp64(Ta);
    Za = 1.0e4 * invTa;
    Zia = 1.0e-4 * Ta;
    lnZa = ln1e4 - lnTa;
    Za2 = Za * Za;
  }
  (void)Tv;
#pragma unroll
  for (int s = 0; s < NS; ++s) om[s] = 0.0;
  for (int r = 0; r < nr; ++r) {
    const RxnDev& Rx = mech->rx[r];
    const bool ta = TT && Rx.ta;  // uniform across the launch
    const double lt = ta ? lnTa : lnT, it = ta ? invTa : invT;
    const double z = ta ? Za : Z, zi = ta ? Zia : Zi, lz = ta ? lnZa : lnZ, z2 = ta ? Za2 : Z2;
    const double lkf = fma(Rx.b, lt, fma(-Rx.Ta, it, Rx.lnA));
    const double lkc = fma(Rx.kc[0], zi, fma(Rx.kc[2], lz, fma(Rx.kc[3], z, fma(Rx.kc[4], z2, Rx.kc[1]))));
    const double kf = exp_tab(lkf, e2tab), kb = exp_tab(lkf - lkc, e2tab);
    const double pf = X[Rx.f[0] * xs] * X[Rx.f[1] * xs] * X[Rx.f[2] * xs];
    const double pb = X[Rx.bk[0] * xs] * X[Rx.bk[1] * xs] * X[Rx.bk[2] * xs];
    const double rate = fma(kf, pf, -kb * pb);
#pragma unroll
    for (int s = 0; s < NS; ++s) om[s] = fma(Rx.coef[s], rate, om[s]);
  }
}

// Two-temperature E_v source of one node (Sec. 3.1.3 Eqs. src_vector, src_landau_teller),
// FP64: Q_T-v + sum_s omega_s e_v,s(T_v) with Q_T-v = sum rho_s (e_v,s(T) - e_v,s(T_v)) / tau_s
// over the vibrating species, tau_s = tau_MW + tau_P:
//   1 / tau_MW = (p / 1 atm) sum_r X_r exp(C_sr - A_sr T^-1/3)       (Millikan and White)
//   tau_P = k_B T / (p sigma_v c_s), sigma_v = 1e-21 (5e4 / T)^2 m^2, c_s = (8 R_s T / pi)^1/2
// (Park), X_r the mole fractions, A_sr and C_sr = A_sr B_sr + 18.42 precomputed on the host.
// sp: species table (rows R, cv, h0, 1e-6/W, theta); mw: [2][NS][NS] (A, then C).
template <int NS>
__device__ __forceinline__ double vib_source(const double* u, const double* sp, const double* mw, double T,
                                             double Tv, const double (&om)[NS], const double* e2tab) {
  double X[NS], sum = 0.0, rR = 0.0;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    X[s] = u[s] * sp[3 * NS + s];
    sum += X[s];
    rR = fma(u[s], sp[s], rR);
  }
  const double ix = rcp64(sum), invT = rcp64(T), invTv = rcp64(Tv);
  const double p = rR * T;
  const double t13 = exp_tab(-log(T) * (1.0 / 3.0), e2tab);  // T^-1/3
  const double patm = p * (1.0 / 101325.0);
  const double r5 = 5.0e4 * invT;
  const double park = 1.380649e-23 * T / (p * 1.0e-21 * r5 * r5);  // k_B T / (p sigma_v)
  double out = 0.0;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const double th = sp[4 * NS + s];
    if (th <= 0.0) continue;
    double r = 0.0;
#pragma unroll
    for (int q = 0; q < NS; ++q) r = fma(X[q], exp_tab(fma(-mw[s * NS + q], t13, mw[NS * NS + s * NS + q]), e2tab), r);
    const double tau = rcp64(patm * r * ix) + park * rsqrt(8.0 * sp[s] * T * (1.0 / 3.141592653589793));
    const double Rth = sp[s] * th;
    const double eT = Rth * rcp64(exp_tab(th * invT, e2tab) - 1.0);
    const double eTv = Rth * rcp64(exp_tab(th * invTv, e2tab) - 1.0);
    out = fma(u[s], (eT - eTv) * rcp64(tau), out);
    out = fma(om[s], eTv, out);
  }
  return out;
}

// Launch scalars in the flux precision.
template <class R>
struct RS {
  R s[3], lift, mu, kfac, p_ref;
  __device__ __forceinline__ explicit RS(const ReactArgs& a) {
    for (int l = 0; l < 3; ++l) s[l] = sel(a.s[l], a.sf[l]);
    lift = sel(a.lift, a.liftf);
    mu = sel(a.mu, a.muf);
    kfac = sel(a.kfac, a.kfacf);
    p_ref = sel(a.p_ref, a.p_reff);
  }
  static __device__ __forceinline__ R sel(double d, float f) {
    if constexpr (sizeof(R) == 4) return f; else return d;
  }
};

// Own primitives (and U in R) of the CTA's elements and the neighbours' face traces, from the
// primitive cache (rows 0..NROW-1) and, with KEEP_U, the FP64 state; the own nodes' FP64
// state is returned in u_own and (c_p, T, c_v,v, T_v) (FP64; the last two two-temperature
// only) in cpT_own.
template <int N, int NS, bool TT, class R, bool KEEP_U, int NROW>
__device__ __forceinline__ void load_element(const ReactArgs& a, int e0, R* smem_el, int esz, int off_p,
                                             int off_pt, int off_us, int off_ut, double* u_own, double* cpT_own) {
  using G = RG<N, NS, TT, R>;
  constexpr int NPR = G::NPR;
  const int t = threadIdx.x;
  const R* P = reinterpret_cast<const R*>(a.pin);
  if (t < G::EPB * G::NP) {
    const int el = t / G::NP, q = t % G::NP, e = e0 + el;
    if (e < a.n_elem) {
      R* sm = smem_el + el * esz;
      const long long gi = a.base + (long long)e * G::NP + q;
#pragma unroll
      for (int c = 0; c < NROW; ++c) sm[off_p + c * G::NP + q] = P[c * a.stride + gi];
      if (cpT_own) {
        cpT_own[0] = Ar<R>::widen(P[G::RCP * a.stride + gi]);
        cpT_own[1] = a.tin[gi];
        if (TT) {
          cpT_own[2] = Ar<R>::widen(P[G::RCV * a.stride + gi]);
          cpT_own[3] = a.tin[a.stride + gi];
        }
      }
      if (KEEP_U) {
#pragma unroll
        for (int v = 0; v < G::NV; ++v) {
          u_own[v] = a.U[v * a.stride + gi];
          sm[off_us + v * G::NP + q] = Ar<R>::load(u_own[v]);
        }
      }
    }
  }
  for (int idx = t; idx < G::EPB * G::NFJ; idx += kRT) {
    const int el = idx / G::NFJ, r = idx % G::NFJ, f = r / G::NFN, jf = r % G::NFN;
    const int e = e0 + el;
    if (e >= a.n_elem) continue;
    R* sm = smem_el + el * esz;
    const int l = f >> 1, side = f & 1;
    const int fw = a.bnd.nonper ? wall_face(a, e, l, side) : -1;
    if (fw >= 0) {
      // a domain face: a ghost trace W+ whose BR1 average (W + W+)/2 is the boundary's
      // trace of (u, v, w, T) (Sec. 3.1.2 boundary kernels); the other rows and U are the
      // element's own (the face job computes the inviscid boundary flux from them)
      const long long go = a.base + (long long)e * G::NP + face_node<G::N1>(l, side, jf);
      const int type = a.bnd.bc[fw];
      R w[NROW];
#pragma unroll
      for (int c = 0; c < NROW; ++c) w[c] = P[c * a.stride + go];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        R g = w[c];
        if (type == 1) {                        // slip wall: the mirror image
          if (c == l) g = -g;
        } else if (type == 5 || type == 6) {    // no-slip walls: velocity 0 on the wall
          if (c < 3) g = -g;
          else if (type == 6) g = R(2) * Ar<R>::load(a.bnd.bcw[fw][3]) - g;  // T = T_wall
        } else if (type == 2 || type == 4) {    // inflow, Dirichlet: W of U_b
          g = R(2) * Ar<R>::load(a.bnd.bcw[fw][c]) - g;
        }                                       // outflow: the interior trace
        sm[off_pt + (f * NPR + c) * G::NFN + jf] = g;
      }
#pragma unroll
      for (int c = 4; c < NROW; ++c) sm[off_pt + (f * NPR + c) * G::NFN + jf] = w[c];
      if (TT && NROW > 4) {  // T_v: the wall temperature at isothermal walls, U_b's at far-field
                             // faces, the interior T_v otherwise
        if (type == 2 || type == 4 || type == 6)
          sm[off_pt + (f * NPR + 4) * G::NFN + jf] = R(2) * Ar<R>::load(a.bnd.bcw[fw][6]) - w[4];
      }
      if (KEEP_U) {
#pragma unroll
        for (int v = 0; v < G::NV; ++v) sm[off_ut + (f * G::NV + v) * G::NFN + jf] = Ar<R>::load(a.U[v * a.stride + go]);
      }
      continue;
    }
    const int en = neighbour(a.nel, e, l, side ? 1 : -1);
    const long long gi = a.base + (long long)en * G::NP + face_node<G::N1>(l, side ^ 1, jf);
#pragma unroll
    for (int c = 0; c < NROW; ++c) sm[off_pt + (f * NPR + c) * G::NFN + jf] = P[c * a.stride + gi];
    if (KEEP_U) {
#pragma unroll
      for (int v = 0; v < G::NV; ++v) sm[off_ut + (f * G::NV + v) * G::NFN + jf] = Ar<R>::load(a.U[v * a.stride + gi]);
    }
  }
}

// ---------------------------------------------------------------------------------------
// Launch 1: BR1 gradients and the element's own viscous flux on its faces.
// ---------------------------------------------------------------------------------------
// CURV: a curved instance -- the reference-space derivative is mapped to the physical
// gradient with the node's contravariant vectors and 1/J, and the face flux written is the
// contravariant one, sum_d Ja^l_d F_v^d (the face's Ja^l is the same on both sides).
template <int N, int NS, bool TT, class R, bool CURV>
__global__ void __launch_bounds__(kRT) k_br1_faces(const ReactArgs a) {
  using G = RG<N, NS, TT, R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* D = reinterpret_cast<R*>(smem_raw);
  R* el_base = D + G::N1 * G::N1;
  const int t = threadIdx.x;
  for (int k = t; k < G::N1 * G::N1; k += kRT) D[k] = Ar<R>::load(a.D[k]);
  const RS<R> rs(a);
  const int e0 = blockIdx.x * G::EPB;
  double cpT[4] = {0.0, 0.0, 0.0, 0.0};
  load_element<N, NS, TT, R, false, G::NW>(a, e0, el_base, G::G_SIZE, G::G_P, G::G_PT, 0, 0, nullptr, cpT);
  __syncthreads();
  if (t >= G::EPB * G::NP) return;
  const int el = t / G::NP, q = t % G::NP, e = e0 + el;
  if (e >= a.n_elem) return;
  const int ijk[3] = {q % G::N1, (q / G::N1) % G::N1, q / G::NFN};
  if (ijk[0] != 0 && ijk[0] != N && ijk[1] != 0 && ijk[1] != N && ijk[2] != 0 && ijk[2] != N) return;
  const R* sm = el_base + el * G::G_SIZE;
  R S[G::NW][3];
  br1_gradient<N, G::NW, G::NPR, R>(q, sm + G::G_P, sm + G::G_PT, D, rs.s, rs.lift, S);
  R Ja[3][3];
  if constexpr (CURV) {
    R iJ;
    node_metric<R>(a, a.base + (long long)e * G::NP + q, Ja, iJ);
    to_physical<G::NW, R>(Ja, iJ, S);
  }
  const R v[3] = {sm[G::G_P + q], sm[G::G_P + G::NP + q], sm[G::G_P + 2 * G::NP + q]};
  const R kcond = rs.kfac * Ar<R>::load(cpT[0]);
  const R kvib = rs.kfac * Ar<R>::load(cpT[2]);
  R* fbe = reinterpret_cast<R*>(a.fb) + (size_t)e * 6 * G::NFV * G::NFN;
  R Fv[G::NFV];
#define DG_FACE_OUT(L)                                                                       \
  if (ijk[L] == 0 || ijk[L] == N) {                                                          \
    if constexpr (CURV) visc_flux_contra<G::NW, G::NFV, R>(S, v, rs.mu, kcond, kvib, Ja[L], Fv); \
    else visc_flux<L, G::NW, R>(S, v, rs.mu, kcond, kvib, Fv);                               \
    const int jf = L == 0 ? ijk[1] + G::N1 * ijk[2]                                          \
                          : (L == 1 ? ijk[0] + G::N1 * ijk[2] : ijk[0] + G::N1 * ijk[1]);     \
    R* dst = fbe + (2 * L + (ijk[L] == N ? 1 : 0)) * G::NFV * G::NFN + jf;                   \
    for (int c = 0; c < G::NFV; ++c) dst[c * G::NFN] = Fv[c];                               \
  }
  DG_FACE_OUT(0)
  DG_FACE_OUT(1)
  DG_FACE_OUT(2)
#undef DG_FACE_OUT
}

// ---------------------------------------------------------------------------------------
// Launch 2: the fused stage.
// ---------------------------------------------------------------------------------------
// CURV: a curved instance (periodic) -- the physical gradient from the node's metric, the
// contravariant fluxes sum_d Ja^l_d F^d in the volume term, the Rusanov flux along the
// contravariant normal n = Ja^l / |Ja^l| scaled by |Ja^l| at the faces, the whole transport
// residual times 1/J (Sec. 3.1.1, Eq. vol_weak with the contravariant flux; Sec. 3.1.2).
template <int N, int NS, bool TT, class R, bool CURV>
__global__ void __launch_bounds__(kRT) k_reacting_stage(const ReactArgs a) {
  using G = RG<N, NS, TT, R>;
  constexpr int N1 = G::N1, NP = G::NP, NFN = G::NFN, NV = G::NV, NFV = G::NFV, NPR = G::NPR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sp = reinterpret_cast<double*>(smem_raw) + G::C_SP;
  double* X = reinterpret_cast<double*>(smem_raw) + G::C_X;
  double* e2tab = reinterpret_cast<double*>(smem_raw) + G::C_E2;
  double* mw = reinterpret_cast<double*>(smem_raw) + G::C_MW;
  R* D = reinterpret_cast<R*>(reinterpret_cast<double*>(smem_raw) + G::C_DBL);
  R* el_base = D + N1 * N1;
  const int t = threadIdx.x;
  for (int k = t; k < N1 * N1; k += kRT) D[k] = Ar<R>::load(a.D[k]);
  load_species<NS>(a.mech, sp, G::NSP);
  for (int k = t; k < 64; k += kRT) e2tab[k] = a.mech->exp2tab[k];
  if (TT) {  // Millikan-White coefficients [A | C][s][r]
    for (int k = t; k < 2 * NS * NS; k += kRT) {
      const int w = k / (NS * NS), s2 = (k / NS) % NS, r2 = k % NS;
      mw[k] = w ? a.mech->mwC[s2][r2] : a.mech->mwA[s2][r2];
    }
  }
  // neighbour viscous face fluxes from launch 1
  const int e0 = blockIdx.x * G::EPB;
  const R* fb = reinterpret_cast<const R*>(a.fb);
  for (int idx = t; idx < G::EPB * 6 * NFV * NFN; idx += kRT) {
    const int el = idx / (6 * NFV * NFN), r = idx % (6 * NFV * NFN), f = r / (NFV * NFN), cj = r % (NFV * NFN);
    const int e = e0 + el;
    if (e >= a.n_elem) continue;
    const int l = f >> 1, side = f & 1;
    const int en = neighbour(a.nel, e, l, side ? 1 : -1);
    el_base[el * G::E_SIZE + G::E_FT + r] = fb[((size_t)en * 6 + (2 * l + (side ^ 1))) * NFV * NFN + cj];
  }
  __syncthreads();
  const RS<R> rs(a);
  double u64[NV];
  double cpT[4] = {0.0, 1.0, 0.0, 1.0};
  load_element<N, NS, TT, R, true, NPR>(a, e0, el_base, G::E_SIZE, G::E_P, G::E_PT, G::E_US, G::E_UT, u64, cpT);
  unsigned flag = 0;
  __syncthreads();

  const bool node_thread = t < G::EPB * NP;
  const int el = node_thread ? t / NP : 0, q = node_thread ? t % NP : 0, e = e0 + el;
  const bool active = node_thread && e < a.n_elem;
  R* sm = el_base + el * G::E_SIZE;
  const int ijk[3] = {q % N1, (q / N1) % N1, q / NFN};
  R u[NV], res[NV], v[3], pd = R(0), kcond = R(0), kvib = R(0);
  R S[G::NW][3];
  R Ja[3][3], iJ = R(1);
#pragma unroll
  for (int k = 0; k < NV; ++k) res[k] = R(0);
  if (active) {
#pragma unroll
    for (int k = 0; k < NV; ++k) u[k] = sm[G::E_US + k * NP + q];
#pragma unroll
    for (int d = 0; d < 3; ++d) v[d] = sm[G::E_P + d * NP + q];
    pd = sm[G::E_P + G::RPD * NP + q];
    kcond = rs.kfac * Ar<R>::load(cpT[0]);
    kvib = rs.kfac * Ar<R>::load(cpT[2]);
    br1_gradient<N, G::NW, NPR, R>(q, sm + G::E_P, sm + G::E_PT, D, rs.s, rs.lift, S);
    if constexpr (CURV) {
      node_metric<R>(a, a.base + (long long)e * NP + q, Ja, iJ);
      to_physical<G::NW, R>(Ja, iJ, S);
    }
  }
  // volume term, one direction at a time through the H buffer
#define DG_VOLUME_DIR(L)                                                                      \
  {                                                                                           \
    if (active) {                                                                             \
      R F[NV], Fv[NFV];                                                                       \
      if constexpr (CURV) {                                                                   \
        inv_flux_contra<NS, TT, R>(u, v[0], v[1], v[2], pd, rs.p_ref, Ja[L], F);              \
        visc_flux_contra<G::NW, NFV, R>(S, v, rs.mu, kcond, kvib, Ja[L], Fv);                 \
      } else {                                                                                \
        inv_flux<NS, TT, R>(L, u, v[0], v[1], v[2], pd, rs.p_ref, F);                         \
        visc_flux<L, G::NW, R>(S, v, rs.mu, kcond, kvib, Fv);                                 \
      }                                                                                       \
      _Pragma("unroll") for (int c = 0; c < NFV; ++c) F[NS + c] -= Fv[c];                     \
      _Pragma("unroll") for (int k = 0; k < NV; ++k) sm[G::E_H + k * NP + q] = F[k];          \
      if (ijk[L] == 0 || ijk[L] == N) {                                                       \
        const int jf = L == 0 ? ijk[1] + N1 * ijk[2]                                          \
                              : (L == 1 ? ijk[0] + N1 * ijk[2] : ijk[0] + N1 * ijk[1]);        \
        const int side = ijk[L] == N ? 1 : 0;                                                 \
        R* dst = sm + G::E_FO + (2 * L + side) * NFV * NFN + jf;                              \
        _Pragma("unroll") for (int c = 0; c < NFV; ++c) dst[c * NFN] = Fv[c];                 \
        const int fw = a.bnd.nonper ? wall_face(a, e, L, side) : -1;                          \
        if (fw >= 0) { /* ghost neighbour flux: (F_v + ghost)/2 is the boundary flux */       \
          R gh[NFV];                                                                          \
          ghost_viscous_flux<L, NFV, R>(a.bnd.bc[fw], Fv, kcond * S[3][L],                    \
                                        TT ? kvib * S[G::NW - 1][L] : R(0), gh);              \
          R* gd = sm + G::E_FT + (2 * L + side) * NFV * NFN + jf;                             \
          _Pragma("unroll") for (int c = 0; c < NFV; ++c) gd[c * NFN] = gh[c];                \
        }                                                                                     \
      }                                                                                       \
    }                                                                                         \
    __syncthreads();                                                                          \
    if (active) {                                                                             \
      constexpr int st = L == 0 ? 1 : (L == 1 ? N1 : NFN);                                    \
      const int il = ijk[L], q0 = q - il * st;                                                \
      R acc[NV];                                                                              \
      _Pragma("unroll") for (int k = 0; k < NV; ++k) acc[k] = R(0);                           \
      _Pragma("unroll") for (int mm = 0; mm < N1; ++mm) {                                     \
        const R d = D[il * N1 + mm];                                                          \
        _Pragma("unroll") for (int k = 0; k < NV; ++k)                                        \
            acc[k] = acc[k] + d * sm[G::E_H + k * NP + q0 + mm * st];                         \
      }                                                                                       \
      _Pragma("unroll") for (int k = 0; k < NV; ++k) res[k] = res[k] - rs.s[L] * acc[k];      \
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
    R* fs = el_base + fel * G::E_SIZE;
    const int l = f >> 1, side = f & 1;
    const int qo = face_node<N1>(l, side, jf);
    R uo[NV], un[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      uo[k] = fs[G::E_US + k * NP + qo];
      un[k] = fs[G::E_UT + (f * NV + k) * NFN + jf];
    }
    const R* po = fs + G::E_P + qo;
    const R* pn = fs + G::E_PT + f * NPR * NFN + jf;
    if constexpr (CURV) {  // periodic: the neighbour's trace; Rusanov along n = Ja^l / |Ja^l|
      R ja[3], nrm[3];
      node_metric_dir<R>(a, a.base + (long long)(e0 + fel) * NP + qo, l, ja);
      const R sj = Ar<R>::sqrt(ja[0] * ja[0] + ja[1] * ja[1] + ja[2] * ja[2]);
      const R isj = R(1) / sj;
#pragma unroll
      for (int d = 0; d < 3; ++d) nrm[d] = ja[d] * isj;
      R Fo[NV], Fn[NV];
      inv_flux_contra<NS, TT, R>(uo, po[0], po[NP], po[2 * NP], po[G::RPD * NP], rs.p_ref, nrm, Fo);
      inv_flux_contra<NS, TT, R>(un, pn[0], pn[NFN], pn[2 * NFN], pn[G::RPD * NFN], rs.p_ref, nrm, Fn);
      const R vno = nrm[0] * po[0] + nrm[1] * po[NP] + nrm[2] * po[2 * NP];
      const R vnn = nrm[0] * pn[0] + nrm[1] * pn[NFN] + nrm[2] * pn[2 * NFN];
      const R lam = Ar<R>::fmax(Ar<R>::abs(vno) + po[G::RA * NP], Ar<R>::abs(vnn) + pn[G::RA * NFN]);
      const R hl = side ? R(0.5) * lam : R(-0.5) * lam;
      R dlt[NV];
#pragma unroll
      for (int k = 0; k < NV; ++k) dlt[k] = sj * (R(0.5) * (Fn[k] - Fo[k]) - hl * (un[k] - uo[k]));
#pragma unroll
      for (int c = 0; c < NFV; ++c)
        dlt[NS + c] = dlt[NS + c] - R(0.5) * (fs[G::E_FT + f * NFV * NFN + c * NFN + jf] -
                                              fs[G::E_FO + f * NFV * NFN + c * NFN + jf]);
#pragma unroll
      for (int k = 0; k < NV; ++k) fs[G::E_UT + (f * NV + k) * NFN + jf] = dlt[k];
      continue;
    }
    R Fo[NV], Fn[NV];
    inv_flux<NS, TT, R>(l, uo, po[0], po[NP], po[2 * NP], po[G::RPD * NP], rs.p_ref, Fo);
    // the exterior state: the neighbour's trace, or at a domain face the boundary functor's
    // (Sec. 3.1.1): walls -- the mirror state; Dirichlet -- U_b; inflow -- F* = F(U_b);
    // outflow -- F* = F(U-)
    R vn[3] = {pn[0], pn[NFN], pn[2 * NFN]}, pdn = pn[G::RPD * NFN], an = pn[G::RA * NFN];
    const int fw = a.bnd.nonper ? wall_face(a, e0 + fel, l, side) : -1;
    const int type = fw >= 0 ? a.bnd.bc[fw] : 0;
    if (fw >= 0) {
      if (type == 2 || type == 4) {
#pragma unroll
        for (int k = 0; k < NV; ++k) un[k] = Ar<R>::load(a.bnd.bcu[fw][k]);
#pragma unroll
        for (int d = 0; d < 3; ++d) vn[d] = Ar<R>::load(a.bnd.bcw[fw][d]);
        pdn = Ar<R>::load(a.bnd.bcw[fw][4]);
        an = Ar<R>::load(a.bnd.bcw[fw][5]);
      } else {
#pragma unroll
        for (int k = 0; k < NV; ++k) un[k] = uo[k];
        vn[0] = po[0];
        vn[1] = po[NP];
        vn[2] = po[2 * NP];
#pragma unroll
        for (int d = 0; d < 3; ++d)
          if (d == l) {
            un[NS + d] = -uo[NS + d];
            vn[d] = -vn[d];
          }
        pdn = po[G::RPD * NP];
        an = po[G::RA * NP];
      }
    }
    inv_flux<NS, TT, R>(l, un, vn[0], vn[1], vn[2], pdn, rs.p_ref, Fn);
    const R vlo = pick3(l, po[0], po[NP], po[2 * NP]), vln = pick3(l, vn[0], vn[1], vn[2]);
    const R lam = Ar<R>::fmax(Ar<R>::abs(vlo) + po[G::RA * NP], Ar<R>::abs(vln) + an);
    // F* = (F_L + F_R)/2 - lam (U_R - U_L)/2; with L/R the lower/upper side of the face
    const R hl = side ? R(0.5) * lam : R(-0.5) * lam;  // lam/2 (U_R - U_L) = hl (un - uo)
    R dlt[NV];
    if (type == 2) {  // supersonic inflow: F* = F(U_b)
#pragma unroll
      for (int k = 0; k < NV; ++k) dlt[k] = Fn[k] - Fo[k];
    } else if (type == 3) {  // supersonic outflow: F* = F(U-)
#pragma unroll
      for (int k = 0; k < NV; ++k) dlt[k] = R(0);
    } else {
#pragma unroll
      for (int k = 0; k < NV; ++k) dlt[k] = R(0.5) * (Fn[k] - Fo[k]) - hl * (un[k] - uo[k]);
    }
#pragma unroll
    for (int c = 0; c < NFV; ++c)
      dlt[NS + c] = dlt[NS + c] - R(0.5) * (fs[G::E_FT + f * NFV * NFN + c * NFN + jf] -
                                            fs[G::E_FO + f * NFV * NFN + c * NFN + jf]);
#pragma unroll
    for (int k = 0; k < NV; ++k) fs[G::E_UT + (f * NV + k) * NFN + jf] = dlt[k];
  }
  __syncthreads();
  if (!active) return;
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const int il = ijk[l];
    if (il != 0 && il != N) continue;
    const int side = il == N ? 1 : 0;
    const int jf = l == 0 ? ijk[1] + N1 * ijk[2] : (l == 1 ? ijk[0] + N1 * ijk[2] : ijk[0] + N1 * ijk[1]);
    const R c = (side ? -rs.s[l] : rs.s[l]) * rs.lift;
    const R* ls = sm + G::E_UT + (2 * l + side) * NV * NFN + jf;
#pragma unroll
    for (int k = 0; k < NV; ++k) res[k] = res[k] + c * ls[k * NFN];
  }
  if constexpr (CURV) {
#pragma unroll
    for (int k = 0; k < NV; ++k) res[k] = res[k] * iJ;
  }
  double r64[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) r64[k] = Ar<R>::widen(res[k]);

  // Arrhenius source (Sec. 3.1.3; App. C), FP64, [X_s] = rho_s 1e-6 / W_s; left out of L
  // under the Strang split, where the implicit substep takes it
  const int nr = a.mech->nr;
  if (a.src && (nr > 0 || TT)) {
    double om[NS];
#pragma unroll
    for (int s2 = 0; s2 < NS; ++s2) om[s2] = 0.0;
    if (nr > 0) {
#pragma unroll
      for (int s2 = 0; s2 < NS; ++s2) X[s2 * kRT + t] = u64[s2] * sp[3 * NS + s2];
      X[NS * kRT + t] = 1.0;
      species_rates<NS, TT>(a.mech, nr, cpT[1], cpT[3], X + t, kRT, e2tab, a.ln1e4, om);
#pragma unroll
      for (int s2 = 0; s2 < NS; ++s2) r64[s2] += om[s2];
    }
    // two-temperature: the E_v source (Landau-Teller and the vibrational energy that
    // chemistry carries)
    if constexpr (TT) r64[NS + 4] += vib_source<NS>(u64, sp, mw, cpT[1], cpT[3], om, e2tab);
  }

  const long long gi = a.base + (long long)e * NP + q;
  bool finite = true;
  double x[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    x[k] = r64[k];
    if (a.mode == 1) {
      x[k] = fma(a.cb, u64[k], a.cbdt * r64[k]);
      if (a.need_un) x[k] = fma(a.ca, a.Un[k * a.stride + gi], x[k]);
      if (a.acc) {  // running sum of a later stage (SSP-RK54)
        double y = fma(a.acc_b, u64[k], a.acc_bdt * r64[k]);
        if (a.acc_a != 0.0) y = fma(a.acc_a, a.acc[k * a.stride + gi], y);
        a.acc[k * a.stride + gi] = y;
      }
    }
    finite = finite && finite64(x[k]);
    a.out[k * a.stride + gi] = x[k];
  }
  // the primitive cache of the new state, read by the next stage
  if (a.mode == 1 && a.pout) flag |= write_prims<NS, TT, R>(x, sp, a.p_ref, reinterpret_cast<R*>(a.pout), a.tout,
                                                            a.stride, gi, cpT[3], e2tab);
  if (!finite) flag |= 1u;
  if (flag) atomicOr(a.err, flag);
}

// The primitive cache of a state that did not come from a stage launch.
template <int NS, bool TT, class R>
__global__ void k_react_prims(const double* U, long long stride, long long base, long long n,
                              const MechDev* __restrict__ mech, double p_ref, R* P, double* T64, unsigned* err) {
  constexpr int NV = NS + 4 + (TT ? 1 : 0);
  __shared__ double sp[5 * NS];
  load_species<NS>(mech, sp, TT ? 5 : 4);
  __syncthreads();
  unsigned flag = 0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    double u[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = U[v * stride + base + q];
    flag |= write_prims<NS, TT, R>(u, sp, p_ref, P, T64, stride, base + q, 0.0, mech->exp2tab);
  }
  if (flag) atomicOr(err, flag);
}

// ---------------------------------------------------------------------------------------
// Implicit source substep of the Strang split (Sec. 3.1.3, Eqs. strang_split and
// source_residual): one thread per node advances the partial densities Y by one
// backward-Euler step of length h,  R(Y) = Y - Y^n - h omega(Y) = 0,  by Newton's method
// with rho, the momentum and E fixed.  Each Newton update takes NS + 1 evaluations of R
// (at Y and at Y + eps_k e_k, eps_k = max(1e-7 |Y_k|, 1e-12): the forward-difference
// Jacobian, column by column) and one Gauss-Jordan solve J d = R with partial pivoting, all
// in registers (the concentrations of the evaluation in a per-thread shared-memory slot
// table, indexed by the reactions' species lists).  The temperature of an iterate follows
// from the fixed internal energy e = E - |rho u|^2 / (2 rho): T = (e - sum Y h0) / sum Y cv.
// The step Y <- Y - lam d is guarded (the paper names no safeguard; a full step can
// overshoot to a negative temperature and non-finite rates for h above about 2e-5 s on air
// at 2000-8000 K): lam = 1 is halved (at most 30 times) while the new temperature leaves
// [T/2, 2T].  The iteration stops after the first full step with max |d| <= tol rho; a node
// that is still unconverged after max_it updates keeps its last iterate and sets bit 2 of
// the error word.  FP64 throughout (both precisions); the output's primitive cache is written
// in the flux type R.
// ---------------------------------------------------------------------------------------
constexpr int kCT = 128;  // threads per CTA of the implicit source kernel

// Temperature of the partial densities Y at the fixed internal energy e.
template <int NS>
__device__ __forceinline__ double temp_of(const double* Y, const double* sp, double e) {
  double rcv = 0.0, rh0 = 0.0;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    rcv = fma(Y[s], sp[NS + s], rcv);
    rh0 = fma(Y[s], sp[2 * NS + s], rh0);
  }
  return (e - rh0) * rcp64(rcv);
}

template <int NS>
__device__ __forceinline__ void be_residual(const MechDev* __restrict__ mech, int nr, const double* sp,
                                            const double (&Y)[NS], const double (&Yn)[NS], double e,
                                            double h, double* X, const double* e2tab, double ln1e4,
                                            double (&R)[NS]) {
#pragma unroll
  for (int s = 0; s < NS; ++s) X[s * kCT] = Y[s] * sp[3 * NS + s];
  const double T = temp_of<NS>(Y, sp, e);
  double om[NS];
  species_rates<NS, false>(mech, nr, T, T, X, kCT, e2tab, ln1e4, om);
#pragma unroll
  for (int s = 0; s < NS; ++s) R[s] = fma(-h, om[s], Y[s] - Yn[s]);
}

// Two-temperature residual of the unknowns y = (Y, E_v) (Sec. 3.1.3: the substep takes the
// full source vector, Eq. src_vector): T from the fixed internal energy e less E_v, T_v by
// vib_temperature from tv (updated in place: the warm start of the next evaluation),
// R = y - y^n - h (omega, Q_T-v + sum omega_s e_v,s(T_v)).  Returns T; false in ok when T or
// T_v is not positive or the T_v iteration did not converge.
template <int NS>
__device__ __forceinline__ double be_residual_tt(const MechDev* __restrict__ mech, int nr, const double* sp,
                                                 const double* mw, const double (&y)[NS + 1],
                                                 const double (&yn)[NS + 1], double e, double h, double* X,
                                                 const double* e2tab, double ln1e4, double& tv,
                                                 double (&R)[NS + 1], bool& ok) {
  const double T = temp_of<NS>(y, sp, e - y[NS]);
  double dEv;
  bool conv;
  tv = vib_temperature<NS>(y, sp, y[NS], tv, e2tab, dEv, conv);
  ok = conv && T > 0.0 && tv > 0.0;
#pragma unroll
  for (int s = 0; s < NS; ++s) X[s * kCT] = y[s] * sp[3 * NS + s];
  double om[NS];
  species_rates<NS, true>(mech, nr, T, tv, X, kCT, e2tab, ln1e4, om);
  const double Sv = vib_source<NS>(y, sp, mw, T, tv, om, e2tab);
#pragma unroll
  for (int s = 0; s < NS; ++s) R[s] = fma(-h, om[s], y[s] - yn[s]);
  R[NS] = fma(-h, Sv, y[NS] - yn[NS]);
  return T;
}

// Two-temperature implicit substep: Newton on (Y, E_v) as in k_source_implicit, the forward-
// difference Jacobian (NS + 2 residual evaluations per update), Gauss-Jordan on the
// (NS+1)^2 system, the guarded step also keeping T_v within [T_v/2, 2 T_v], convergence once
// a full step has max_s |dY_s| <= tol rho and |dE_v| <= tol e.
template <int NS, class R>
__global__ void __launch_bounds__(kCT) k_source_implicit_tt(const SourceArgs a) {
  constexpr int NU = NS + 1;
  __shared__ double sp[5 * NS];
  __shared__ double mw[2 * NS * NS];
  __shared__ double e2tab[64];
  __shared__ double Xs[(NS + 1) * kCT];
  const int t = threadIdx.x;
  load_species<NS>(a.mech, sp, 5);
  for (int k = t; k < 64; k += kCT) e2tab[k] = a.mech->exp2tab[k];
  for (int k = t; k < 2 * NS * NS; k += kCT) {
    const int w = k / (NS * NS), s2 = (k / NS) % NS, r2 = k % NS;
    mw[k] = w ? a.mech->mwC[s2][r2] : a.mech->mwA[s2][r2];
  }
  double* X = Xs + t;
  X[NS * kCT] = 1.0;
  __syncthreads();
  const long long q = blockIdx.x * (long long)kCT + t;
  if (q >= a.n) return;
  const long long gi = a.base + q;
  const int nr = a.mech->nr;
  double u[NS + 5];
#pragma unroll
  for (int v = 0; v < NS + 5; ++v) u[v] = a.U[v * a.stride + gi];
  double yn[NU], y[NU], rho = 0.0;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    yn[s] = y[s] = u[s];
    rho += u[s];
  }
  yn[NS] = y[NS] = u[NS + 4];
  const double kin = fma(u[NS], u[NS], fma(u[NS + 1], u[NS + 1], u[NS + 2] * u[NS + 2]));
  const double e = u[NS + 3] - 0.5 * kin * rcp64(rho);
  const double lim = a.tol * rho, lim_v = a.tol * e;
  double tv = a.tin ? a.tin[a.stride + gi] : 0.0;  // T_v of the input state when cached
  bool done = false;
  int it = 0;
  for (; it < a.max_it && !done; ++it) {
    double Rv[NU], J[NU][NU];
    bool ok;
    const double T0 = be_residual_tt<NS>(a.mech, nr, sp, mw, y, yn, e, a.h, X, e2tab, a.ln1e4, tv, Rv, ok);
    if (!ok) break;
    const double tv0 = tv;
#pragma unroll
    for (int k = 0; k < NU; ++k) {
      double yp[NU], Rp[NU];
#pragma unroll
      for (int s = 0; s < NU; ++s) yp[s] = y[s];
      const double eps = fmax(1e-7 * fabs(y[k]), 1e-12);
      yp[k] += eps;
      double tvp = tv0;
      bool okp;
      be_residual_tt<NS>(a.mech, nr, sp, mw, yp, yn, e, a.h, X, e2tab, a.ln1e4, tvp, Rp, okp);
      const double ie = rcp64(eps);
#pragma unroll
      for (int i = 0; i < NU; ++i) J[i][k] = (Rp[i] - Rv[i]) * ie;
    }
#pragma unroll
    for (int k = 0; k < NU; ++k) {
#pragma unroll
      for (int i = k + 1; i < NU; ++i) {
        if (fabs(J[i][k]) > fabs(J[k][k])) {
#pragma unroll
          for (int j = 0; j < NU; ++j) {
            const double tmp = J[i][j];
            J[i][j] = J[k][j];
            J[k][j] = tmp;
          }
          const double tmp = Rv[i];
          Rv[i] = Rv[k];
          Rv[k] = tmp;
        }
      }
      const double d = rcp64(J[k][k]);
#pragma unroll
      for (int j = 0; j < NU; ++j) J[k][j] *= d;
      Rv[k] *= d;
#pragma unroll
      for (int i = 0; i < NU; ++i) {
        if (i == k) continue;
        const double f = J[i][k];
#pragma unroll
        for (int j = 0; j < NU; ++j) J[i][j] = fma(-f, J[k][j], J[i][j]);
        Rv[i] = fma(-f, Rv[k], Rv[i]);
      }
    }
    double lam = 1.0, yt[NU];
    for (int k = 0; k < 30; ++k) {
#pragma unroll
      for (int s = 0; s < NU; ++s) yt[s] = fma(-lam, Rv[s], y[s]);
      const double Tt = temp_of<NS>(yt, sp, e - yt[NS]);
      double dEv, tvt = tv0;
      bool conv;
      tvt = vib_temperature<NS>(yt, sp, yt[NS], tvt, e2tab, dEv, conv);
      if (Tt >= 0.5 * T0 && Tt <= 2.0 * T0 && tvt >= 0.5 * tv0 && tvt <= 2.0 * tv0) break;
      lam *= 0.5;
    }
    bool small = lam == 1.0 && fabs(Rv[NS]) <= lim_v;
#pragma unroll
    for (int s = 0; s < NU; ++s) {
      if (s < NS) small = small && fabs(Rv[s]) <= lim;
      y[s] = yt[s];
    }
    done = small;
  }
  {
    const unsigned mask = __activemask();
    const unsigned sum = __reduce_add_sync(mask, (unsigned)it);
    if ((threadIdx.x & 31) == __ffs(mask) - 1) atomicAdd(a.updates, (unsigned long long)sum);
  }
  unsigned flag = done ? 0u : 4u;
  bool finite = true;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    u[s] = y[s];
    finite = finite && finite64(y[s]);
    a.out[s * a.stride + gi] = y[s];
  }
  u[NS + 4] = y[NS];
  finite = finite && finite64(y[NS]);
  a.out[(NS + 4) * a.stride + gi] = y[NS];
  if (a.copy_rest) {
#pragma unroll
    for (int v = NS; v < NS + 4; ++v) a.out[v * a.stride + gi] = u[v];
  }
  if (a.pout) flag |= write_prims<NS, true, R>(u, sp, a.p_ref, reinterpret_cast<R*>(a.pout), a.tout, a.stride, gi,
                                               tv, e2tab);
  if (!finite) flag |= 1u;
  if (flag) atomicOr(a.err, flag);
}

template <int NS, class R>
__global__ void __launch_bounds__(kCT) k_source_implicit(const SourceArgs a) {
  __shared__ double sp[4 * NS];
  __shared__ double e2tab[64];
  __shared__ double Xs[(NS + 1) * kCT];
  const int t = threadIdx.x;
  load_species<NS>(a.mech, sp, 4);
  for (int k = t; k < 64; k += kCT) e2tab[k] = a.mech->exp2tab[k];
  double* X = Xs + t;
  X[NS * kCT] = 1.0;
  __syncthreads();
  const long long q = blockIdx.x * (long long)kCT + t;
  if (q >= a.n) return;
  const long long gi = a.base + q;
  const int nr = a.mech->nr;
  double u[NS + 4];
#pragma unroll
  for (int v = 0; v < NS + 4; ++v) u[v] = a.U[v * a.stride + gi];
  double Yn[NS], Y[NS], rho = 0.0;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    Yn[s] = Y[s] = u[s];
    rho += u[s];
  }
  const double kin = fma(u[NS], u[NS], fma(u[NS + 1], u[NS + 1], u[NS + 2] * u[NS + 2]));
  const double e = u[NS + 3] - 0.5 * kin * rcp64(rho);
  const double lim = a.tol * rho;
  bool done = false;
  int it = 0;
  for (; it < a.max_it && !done; ++it) {
    double Rv[NS], J[NS][NS];
    be_residual<NS>(a.mech, nr, sp, Y, Yn, e, a.h, X, e2tab, a.ln1e4, Rv);
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      double Yp[NS], Rp[NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) Yp[s] = Y[s];
      const double eps = fmax(1e-7 * fabs(Y[k]), 1e-12);
      Yp[k] += eps;
      be_residual<NS>(a.mech, nr, sp, Yp, Yn, e, a.h, X, e2tab, a.ln1e4, Rp);
      const double ie = rcp64(eps);
#pragma unroll
      for (int i = 0; i < NS; ++i) J[i][k] = (Rp[i] - Rv[i]) * ie;
    }
    // Gauss-Jordan on [J | R] with partial pivoting (row swaps by compare-and-swap, so that
    // every index stays compile-time and J stays in registers)
#pragma unroll
    for (int k = 0; k < NS; ++k) {
#pragma unroll
      for (int i = k + 1; i < NS; ++i) {
        if (fabs(J[i][k]) > fabs(J[k][k])) {
#pragma unroll
          for (int j = 0; j < NS; ++j) {
            const double tmp = J[i][j];
            J[i][j] = J[k][j];
            J[k][j] = tmp;
          }
          const double tmp = Rv[i];
          Rv[i] = Rv[k];
          Rv[k] = tmp;
        }
      }
      const double d = rcp64(J[k][k]);
#pragma unroll
      for (int j = 0; j < NS; ++j) J[k][j] *= d;
      Rv[k] *= d;
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        if (i == k) continue;
        const double f = J[i][k];
#pragma unroll
        for (int j = 0; j < NS; ++j) J[i][j] = fma(-f, J[k][j], J[i][j]);
        Rv[i] = fma(-f, Rv[k], Rv[i]);
      }
    }
    // the guarded step
    const double T0 = temp_of<NS>(Y, sp, e);
    double lam = 1.0, Yt[NS];
    for (int k = 0; k < 30; ++k) {
#pragma unroll
      for (int s = 0; s < NS; ++s) Yt[s] = fma(-lam, Rv[s], Y[s]);
      const double Tt = temp_of<NS>(Yt, sp, e);
      if (Tt >= 0.5 * T0 && Tt <= 2.0 * T0) break;
      lam *= 0.5;
    }
    bool small = lam == 1.0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      // false for a non-finite update: the node then runs out of updates and is flagged
      small = small && fabs(Rv[s]) <= lim;
      Y[s] = Yt[s];
    }
    done = small;
  }
  // Newton updates of this node into the launch's counter (one atomic per converged group of
  // lanes)
  {
    const unsigned mask = __activemask();
    const unsigned sum = __reduce_add_sync(mask, (unsigned)it);
    if ((threadIdx.x & 31) == __ffs(mask) - 1) atomicAdd(a.updates, (unsigned long long)sum);
  }
  unsigned flag = done ? 0u : 4u;
  bool finite = true;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    u[s] = Y[s];
    finite = finite && finite64(Y[s]);
    a.out[s * a.stride + gi] = Y[s];
  }
  if (a.copy_rest) {
#pragma unroll
    for (int v = NS; v < NS + 4; ++v) a.out[v * a.stride + gi] = u[v];
  }
  if (a.pout) flag |= write_prims<NS, false, R>(u, sp, a.p_ref, reinterpret_cast<R*>(a.pout), a.tout, a.stride, gi);
  if (!finite) flag |= 1u;
  if (flag) atomicOr(a.err, flag);
}

// Zhang-Shu limiter of the partial densities after a stage (Sec. 4 reacting blast set-up:
// rho_s >= 0 per species; X. Zhang and C.-W. Shu, J. Comput. Phys. 229, 2010): one warp per
// element; an element with no negative nodal density (sign bits) is left at once; otherwise
// the lanes stride over its nodes and reduce, per species, the GLL-weighted mean and the
// minimum by shuffles; where a minimum is negative the nodal values contract toward
// the mean, rho_s <- m + theta (rho_s - m) with theta = m / (m - min) (the mean itself when it
// is not positive), and the changed nodes' primitive cache is rewritten.
constexpr int kLT = 128;  // threads per CTA of the limiter: four elements
template <int NS, bool TT, class R>
__global__ void __launch_bounds__(kLT) k_species_limiter(const LimiterArgs a) {
  constexpr int NV = NS + 4 + (TT ? 1 : 0);
  __shared__ double sp[5 * NS];
  __shared__ double e2tab[64];
  __shared__ double wq[(kMaxReactingN + 1) * (kMaxReactingN + 1) * (kMaxReactingN + 1)];
  load_species<NS>(a.mech, sp, TT ? 5 : 4);
  for (int k = threadIdx.x; k < 64; k += kLT) e2tab[k] = a.mech->exp2tab[k];
  // the weights once per CTA (lanes reading different parameter words serialize)
  for (int k = threadIdx.x; k < a.np; k += kLT) wq[k] = a.wq[k];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int e = blockIdx.x * (kLT / 32) + (threadIdx.x >> 5);
  if (e >= a.n_elem) return;
  const long long g0 = a.base + (long long)e * a.np;
  // a sign-bit test first (integer operations only): most elements have no negative density
  // and leave before any FP64 reduction (the FP64 pipe runs at a 64th of the FP32 rate)
  bool neg = false;
  for (int q = lane; q < a.np; q += 32) {
#pragma unroll
    for (int s = 0; s < NS; ++s) neg = neg || __double2hiint(a.U[s * a.stride + g0 + q]) < 0;
  }
  if (!__any_sync(0xffffffffu, neg)) return;
  double mean[NS], lo[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    mean[s] = 0.0;
    lo[s] = 1e300;
  }
  for (int q = lane; q < a.np; q += 32) {
    const double w = wq[q];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const double r = a.U[s * a.stride + g0 + q];
      mean[s] = fma(w, r, mean[s]);
      lo[s] = fmin(lo[s], r);
    }
  }
  bool any = false;
  double theta[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    for (int o = 16; o > 0; o >>= 1) {
      mean[s] += __shfl_xor_sync(0xffffffffu, mean[s], o);
      lo[s] = fmin(lo[s], __shfl_xor_sync(0xffffffffu, lo[s], o));
    }
    theta[s] = 1.0;
    if (lo[s] < 0.0) {
      theta[s] = mean[s] > 0.0 ? mean[s] / (mean[s] - lo[s]) : 0.0;
      any = true;
    }
  }
  if (!any) return;  // warp-uniform
  unsigned flag = 0;
  for (int q = lane; q < a.np; q += 32) {
    const long long gi = g0 + q;
    double u[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = a.U[v * a.stride + gi];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      if (theta[s] < 1.0) {
        u[s] = fma(theta[s], u[s] - mean[s], mean[s]);
        a.U[s * a.stride + gi] = u[s];
      }
    }
    if (a.pout) {
      const double tv = TT ? a.tout[a.stride + gi] : 0.0;
      flag |= write_prims<NS, TT, R>(u, sp, a.p_ref, reinterpret_cast<R*>(a.pout), a.tout, a.stride, gi, tv, e2tab);
    }
  }
  if (flag) atomicOr(a.err, flag);
}

// Element-wise math routines for the tests (see MathArgs).
__global__ void k_math_fn(const MathArgs a) {
  __shared__ double tab[64];
  for (int k = threadIdx.x; k < 64; k += blockDim.x) tab[k] = a.tab[k];
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.n;
       i += (long long)gridDim.x * blockDim.x) {
    const double x = a.x[i];
    double y;
    if (a.kind == 0) y = exp_tab(x, tab);
    else if (a.kind == 1) y = rcp64(x);
    else if (a.kind == 2) y = exp(x);
    else y = 1.0 / x;
    a.y[i] = y;
  }
}

// Largest |u| + a and largest 1/rho over the nodes of one instance.
template <int NS, bool TT>
__global__ void k_max_speed_mix(const double* U, long long stride, long long base, long long n,
                                const MechDev* __restrict__ mech, unsigned long long* out2) {
  constexpr int NV = NS + 4 + (TT ? 1 : 0);
  __shared__ double sp[4 * NS];
  load_species<NS>(mech, sp, 4);
  __syncthreads();
  // reduction codes (speed_bits): a node with a non-finite value, or with rho <= 0 or T <= 0,
  // makes the whole bound report it instead of being dropped
  unsigned long long lam = 0ull, irho = 0ull;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    double u[NV];
    bool fin = true;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      u[v] = U[v * stride + base + q];
      fin = fin && isfinite(u[v]);
    }
    if (TT) u[NS + 3] -= u[NV - 1];  // the frozen sound speed needs T only: E - E_v
    const Mx m = mixture<NS, false>(u, sp);
    const bool pos = m.rho > 0.0 && m.T > 0.0;
    const unsigned long long a = speed_bits(pos ? sqrt(m.v[0] * m.v[0] + m.v[1] * m.v[1] + m.v[2] * m.v[2]) + m.a : 0.0,
                                            fin, pos);
    const unsigned long long b = speed_bits(pos ? 1.0 / m.rho : 0.0, fin, pos);
    lam = a > lam ? a : lam;
    irho = b > irho ? b : irho;
  }
  lam = block_max_u64(lam);
  __syncthreads();  // the reduction's shared scratch is reused
  irho = block_max_u64(irho);
  if (threadIdx.x == 0) {
    atomicMax(out2, lam);
    atomicMax(out2 + 1, irho);
  }
}

template <int N, int NS, bool TT, class R, bool CURV>
cudaError_t prepare_kernels() {
  using G = RG<N, NS, TT, R>;
  cudaError_t e = cudaFuncSetAttribute(k_reacting_stage<N, NS, TT, R, CURV>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::stage_smem());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_br1_faces<N, NS, TT, R, CURV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)G::grad_smem());
  return e;
}

template <int N, int NS, bool TT, class R>
cudaError_t prepare_one() {
  cudaError_t e = prepare_kernels<N, NS, TT, R, false>();
  return e == cudaSuccess ? prepare_kernels<N, NS, TT, R, true>() : e;
}

template <int N, int NS, bool TT, class R, bool CURV>
cudaError_t launch_kernels(const ReactArgs& a, cudaStream_t s) {
  using G = RG<N, NS, TT, R>;
  const unsigned grid = (unsigned)((a.n_elem + G::EPB - 1) / G::EPB);
  k_br1_faces<N, NS, TT, R, CURV><<<grid, kRT, G::grad_smem(), s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_reacting_stage<N, NS, TT, R, CURV><<<grid, kRT, G::stage_smem(), s>>>(a);
  return cudaGetLastError();
}

template <int N, int NS, bool TT, class R>
cudaError_t launch_one(const ReactArgs& a, cudaStream_t s) {
  if (a.n_elem <= 0) return cudaSuccess;
  return a.met ? launch_kernels<N, NS, TT, R, true>(a, s) : launch_kernels<N, NS, TT, R, false>(a, s);
}

// (N, n_species, two-temperature) instantiations: one species (the non-dimensional single
// gas) and five (air), N = 1..4; the two-temperature model for air.
#define DG_REACT_DISPATCH(CALL)                          \
  switch ((tt ? 256 : 0) + ns * 16 + N) {                \
    case 1 * 16 + 1: return CALL(1, 1, false);           \
    case 1 * 16 + 2: return CALL(2, 1, false);           \
    case 1 * 16 + 3: return CALL(3, 1, false);           \
    case 1 * 16 + 4: return CALL(4, 1, false);           \
    case 5 * 16 + 1: return CALL(1, 5, false);           \
    case 5 * 16 + 2: return CALL(2, 5, false);           \
    case 5 * 16 + 3: return CALL(3, 5, false);           \
    case 5 * 16 + 4: return CALL(4, 5, false);           \
    case 256 + 5 * 16 + 1: return CALL(1, 5, true);      \
    case 256 + 5 * 16 + 2: return CALL(2, 5, true);      \
    case 256 + 5 * 16 + 3: return CALL(3, 5, true);      \
    case 256 + 5 * 16 + 4: return CALL(4, 5, true);      \
    default: return cudaErrorInvalidValue;               \
  }

}  // namespace

bool have_reacting(int N, int ns, int tt) {
  return (tt ? ns == 5 : (ns == 1 || ns == 5)) && N >= 1 && N <= kMaxReactingN;
}

cudaError_t prepare_reacting(int N, int ns, int tt, int fp32) {
#define DG_P(n, s, t) (fp32 ? prepare_one<n, s, t, float>() : prepare_one<n, s, t, double>())
  DG_REACT_DISPATCH(DG_P)
#undef DG_P
}

cudaError_t launch_reacting(int N, int ns, int tt, int fp32, const ReactArgs& a, cudaStream_t s) {
#define DG_L(n, sp, t) (fp32 ? launch_one<n, sp, t, float>(a, s) : launch_one<n, sp, t, double>(a, s))
  DG_REACT_DISPATCH(DG_L)
#undef DG_L
}

cudaError_t launch_react_prims(int ns, int tt, int fp32, const double* U, long long stride, long long base,
                               long long n_nodes, const MechDev* mech, double p_ref, void* P, double* T64,
                               unsigned* err, cudaStream_t s) {
  if (n_nodes <= 0) return cudaSuccess;
  const long long want = (n_nodes + 255) / 256;
  const unsigned grid = (unsigned)(want < grid_cap() ? want : grid_cap());
#define DG_RP(S2, T2, R2) k_react_prims<S2, T2, R2><<<grid, 256, 0, s>>>(U, stride, base, n_nodes, mech, p_ref, (R2*)P, T64, err)
  if (tt && ns == 5 && fp32) DG_RP(5, true, float);
  else if (tt && ns == 5) DG_RP(5, true, double);
  else if (tt) return cudaErrorInvalidValue;
  else if (ns == 1 && fp32) DG_RP(1, false, float);
  else if (ns == 1) DG_RP(1, false, double);
  else if (ns == 5 && fp32) DG_RP(5, false, float);
  else if (ns == 5) DG_RP(5, false, double);
  else return cudaErrorInvalidValue;
#undef DG_RP
  return cudaGetLastError();
}

cudaError_t launch_source_implicit(int ns, int tt, int fp32, const SourceArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((a.n + kCT - 1) / kCT);
  if (tt && ns == 5 && fp32) k_source_implicit_tt<5, float><<<grid, kCT, 0, s>>>(a);
  else if (tt && ns == 5) k_source_implicit_tt<5, double><<<grid, kCT, 0, s>>>(a);
  else if (tt) return cudaErrorInvalidValue;
  else if (ns == 1 && fp32) k_source_implicit<1, float><<<grid, kCT, 0, s>>>(a);
  else if (ns == 1) k_source_implicit<1, double><<<grid, kCT, 0, s>>>(a);
  else if (ns == 5 && fp32) k_source_implicit<5, float><<<grid, kCT, 0, s>>>(a);
  else if (ns == 5) k_source_implicit<5, double><<<grid, kCT, 0, s>>>(a);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_species_limiter(int ns, int tt, int fp32, const LimiterArgs& a, cudaStream_t s) {
  if (a.n_elem <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((a.n_elem + kLT / 32 - 1) / (kLT / 32));
  if (tt && ns == 5 && fp32) k_species_limiter<5, true, float><<<grid, kLT, 0, s>>>(a);
  else if (tt && ns == 5) k_species_limiter<5, true, double><<<grid, kLT, 0, s>>>(a);
  else if (tt) return cudaErrorInvalidValue;
  else if (ns == 1 && fp32) k_species_limiter<1, false, float><<<grid, kLT, 0, s>>>(a);
  else if (ns == 1) k_species_limiter<1, false, double><<<grid, kLT, 0, s>>>(a);
  else if (ns == 5 && fp32) k_species_limiter<5, false, float><<<grid, kLT, 0, s>>>(a);
  else if (ns == 5) k_species_limiter<5, false, double><<<grid, kLT, 0, s>>>(a);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_math_fn(const MathArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const long long want = (a.n + 255) / 256;
  const unsigned grid = (unsigned)(want < 148 * 8 ? want : 148 * 8);
  k_math_fn<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_max_speed_mix(int ns, int tt, const double* U, long long stride, long long base,
                                 long long n_nodes, const MechDev* mech,
                                 unsigned long long* out2, cudaStream_t s) {
  if (n_nodes <= 0) return cudaSuccess;
  const long long want = (n_nodes + 255) / 256;
  const unsigned grid = (unsigned)(want < grid_cap() ? want : grid_cap());
  if (tt && ns == 5) k_max_speed_mix<5, true><<<grid, 256, 0, s>>>(U, stride, base, n_nodes, mech, out2);
  else if (tt) return cudaErrorInvalidValue;
  else if (ns == 1) k_max_speed_mix<1, false><<<grid, 256, 0, s>>>(U, stride, base, n_nodes, mech, out2);
  else if (ns == 5) k_max_speed_mix<5, false><<<grid, 256, 0, s>>>(U, stride, base, n_nodes, mech, out2);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace dg
