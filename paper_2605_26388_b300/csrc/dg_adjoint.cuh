// dg_adjoint.cuh -- hand-written adjoint (vector-Jacobian product) of the DGSEM residual.
//
// For the Euler equations on affine meshes (Sec. 3.1.1): the strong or weak volume form
// (Eq. vol_weak) or the two-point form (Eq. vol_split with Ranocha's flux, App. A), with the
// Rusanov or HLLC surface flux (periodic, or with the boundary functors of the forward pass:
// slip wall, supersonic inflow and outflow, Dirichlet).  Given a
// co-state lam this computes, element by element,
//   w = (dL/dU)^T lam      and      g = lam . dL/dgamma,
// without atomics.  Strong/weak volume: lam contracted with the transposed volume operator
// along each line, times the transposed Euler flux Jacobian.  Two-point volume: as F# is
// symmetric, node i needs only the derivative in its first argument, against the cotangent
// Dv[i][m] lam_i + Dv[m][i] lam_m of each pair on its lines (reverse differentiation of the
// flux, the log means in their series form near equal arguments).  Faces: every face node
// combines its own and its neighbour's co-state (gathered from global memory, as the forward
// pass gathers the neighbour's state) with the transposed Rusanov flux Jacobian or the
// reverse-differentiated HLLC flux.  Non-smooth points follow the forward evaluation: the
// larger Rusanov signal speed (the left one on a tie), d|x|/dx = sign(x) with sign(0) = 0,
// HLLC's branch and the min/max of its speeds by the values.
//
// Output modes (one kernel, fused with the reverse Shu-Osher combination of App. B):
//   mode 0:  out += w                                    (dg_rhs_vjp, accumulating)
//   mode 1:  out  = bcoef (lam + dt w) [+ accin];  accupd (=|+=) acoef lam
// and the gamma contribution, weighted by gw, is reduced per CTA into gpart[blockIdx.x].
#pragma once
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

// Logarithmic mean m = (a - b)/(ln a - ln b) (App. A) and its partial derivatives.  With
// s = a + b, f = (a - b)/s, u = f^2: m = (s/2)/Fs(u), Fs(u) = atanh(f)/f = sum_k u^k/(2k+1),
// so dm/da = 1/(2 Fs) - 2 f b Fs'(u)/(s Fs^2) and dm/db = 1/(2 Fs) + 2 f a Fs'(u)/(s Fs^2):
// near a = b (u below 1e-4 in FP64, 1e-2 in FP32; five terms of the series) from those, where
// they stay accurate; otherwise from the closed forms dm/da = m (a - m)/(a (a - b)) and
// dm/db = m (m - b)/(b (a - b)).
template <class R>
__device__ __forceinline__ void log_mean_grad(R a, R b, R& m, R& da, R& db) {
  const R s = a + b, d = a - b, is = Ar<R>::rcp(s), f = d * is, u = f * f;
  const R thr = sizeof(R) == 8 ? R(1e-4) : R(1e-2);
  if (u < thr) {
    const R Fs = R(1) + u * (R(1.0 / 3.0) + u * (R(1.0 / 5.0) + u * (R(1.0 / 7.0) + u * R(1.0 / 9.0))));
    const R dF = R(1.0 / 3.0) + u * (R(2.0 / 5.0) + u * (R(3.0 / 7.0) + u * R(4.0 / 9.0)));
    const R iF = Ar<R>::rcp(Fs);
    const R k = R(2) * f * is * dF * iF * iF;
    m = R(0.5) * s * iF;
    da = R(0.5) * iF - k * b;
    db = R(0.5) * iF + k * a;
  } else {
    m = d * Ar<R>::rcp(Ar<R>::log(a) - Ar<R>::log(b));
    const R id = Ar<R>::rcp(d);
    da = m * (a - m) * Ar<R>::rcp(a) * id;
    db = m * (m - b) * Ar<R>::rcp(b) * id;
  }
}

// Reverse differentiation of Ranocha's two-point flux F#(U_a, U_b) in direction l (App. A,
// the energy component in its consistent published form) in both arguments against one
// cotangent c: ga = (dF#/dU_a)^T c, gb = (dF#/dU_b)^T c, and cg = c . dF#/dgamma (gamma enters
// through 1/((gamma-1) beta^ln) and both pressures).  A, B: the two nodes' states with their
// reciprocal densities and pressures; igm1 = 1/(gamma - 1).
template <int DIM, class R>
__device__ __forceinline__ void ec_flux_vjp(int l, const NodeState<DIM, R>& A, R irhoa, R ipa,
                                            const NodeState<DIM, R>& B, R irhob, R ipb, R gm1, R igm1,
                                            const R* c, R* ga, R* gb, R& cg) {
  constexpr int NV = DIM + 2;
  const R ba = A.rho * ipa, bb = B.rho * ipb;
  R rln, drla, drlb, bln, dbla, dblb;
  log_mean_grad<R>(A.rho, B.rho, rln, drla, drlb);
  log_mean_grad<R>(ba, bb, bln, dbla, dblb);
  R vavg[DIM], vv = R(0), val = R(0), vbl = R(0), vavl = R(0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    vavg[d] = R(0.5) * (A.v[d] + B.v[d]);
    vv += A.v[d] * B.v[d];
    if (d == l) { val = A.v[d]; vbl = B.v[d]; vavl = vavg[d]; }
  }
  const R frho = rln * vavl;
  const R ibln = Ar<R>::rcp(bln), ib = igm1 * ibln;
  const R cE = c[NV - 1];
  R cm = R(0), cl = R(0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    cm += c[1 + d] * vavg[d];
    if (d == l) cl = c[1 + d];
  }
  // F0 = frho, F_{1+d} = frho vavg_d + [d = l] (pa + pb)/2,
  // F_E = frho (ib + vv/2) + (pa vb_l + pb va_l)/2
  const R fb = c[0] + cm + cE * (ib + R(0.5) * vv);
  const R efr = cE * frho * ib;
  const R blnb = -efr * ibln;
  cg = -efr * igm1;
  const R vvb = R(0.5) * cE * frho;
  const R fr = fb * vavl;  // adjoint of rho^ln
  R pab = R(0.5) * (cE * vbl + cl), pbb = R(0.5) * (cE * val + cl);
  R vab[DIM], vbb[DIM];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const R h = R(0.5) * c[1 + d] * frho;
    vab[d] = h + vvb * B.v[d];
    vbb[d] = h + vvb * A.v[d];
    if (d == l) {
      const R t = R(0.5) * fb * rln;
      vab[d] += R(0.5) * cE * B.p + t;
      vbb[d] += R(0.5) * cE * A.p + t;
    }
  }
  // beta = rho / p
  const R bab = blnb * dbla, bbb = blnb * dblb;
  const R rab = fr * drla + bab * ipa, rbb = fr * drlb + bbb * ipb;
  pab -= bab * ba * ipa;
  pbb -= bbb * bb * ipb;
  cg += pab * A.rhoe + pbb * B.rhoe;
  // p = (gamma - 1)(E - |m|^2/(2 rho)), v = m / rho
  R v2a = R(0), v2b = R(0), vva = R(0), vvbb = R(0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    v2a += A.v[d] * A.v[d];
    v2b += B.v[d] * B.v[d];
    vva += vab[d] * A.v[d];
    vvbb += vbb[d] * B.v[d];
    ga[1 + d] = vab[d] * irhoa - pab * gm1 * A.v[d];
    gb[1 + d] = vbb[d] * irhob - pbb * gm1 * B.v[d];
  }
  ga[0] = rab + pab * gm1 * R(0.5) * v2a - vva * irhoa;
  gb[0] = rbb + pbb * gm1 * R(0.5) * v2b - vvbb * irhob;
  ga[NV - 1] = pab * gm1;
  gb[NV - 1] = pbb * gm1;
}

// Reverse differentiation of the HLLC flux F*(U_L, U_R) in direction l (Toro, Spruce and
// Speares, with the Davis/Einfeldt speeds S_L = min(u_L - a_L, u~ - a~), S_R = max(u_R + a_R,
// u~ + a~) of the Roe average): gL = (dF*/dU_L)^T mu, gR = (dF*/dU_R)^T mu and
// gg = mu . dF*/dgamma.  The branch (S_L >= 0: F_L; S* >= 0: F_L + S_L (U*_L - U_L);
// S_R > 0: F_R + S_R (U*_R - U_R); else F_R) and the min/max follow the forward values, the
// left argument on a tie, with the star state
//   U*_K = fac (1, S* e_l + tangential v_K, E_K/rho_K + (S* - u_K)(S* + p_K/(rho_K (S_K - u_K)))),
//   fac = rho_K (S_K - u_K)/(S_K - S*).
template <int DIM, class R>
__device__ void hllc_vjp(int l, const NodeState<DIM, R>& L, const NodeState<DIM, R>& Rt, R gamma, const R* mu,
                         R* gL, R* gR, R& gg) {
  constexpr int NV = DIM + 2;
  const R gm1 = gamma - R(1);
#pragma unroll
  for (int v = 0; v < NV; ++v) gL[v] = gR[v] = R(0);
  R uLn = R(0), uRn = R(0), mul = R(0);
#pragma unroll
  for (int d = 0; d < DIM; ++d)
    if (d == l) { uLn = L.v[d]; uRn = Rt.v[d]; mul = mu[1 + d]; }
  // Roe-averaged speeds
  const R sL = Ar<R>::sqrt(L.rho), sR = Ar<R>::sqrt(Rt.rho), iden = Ar<R>::rcp(sL + sR);
  R vt[DIM], v2 = R(0), vtl = R(0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    vt[d] = (sL * L.v[d] + sR * Rt.v[d]) * iden;
    v2 += vt[d] * vt[d];
    if (d == l) vtl = vt[d];
  }
  const R Ht = (sL * L.H + sR * Rt.H) * iden;
  const R at = Ar<R>::sqrt(gm1 * (Ht - R(0.5) * v2));
  const R xL1 = uLn - L.c, xL2 = vtl - at, xR1 = uRn + Rt.c, xR2 = vtl + at;
  const bool selL = xL1 <= xL2, selR = xR1 >= xR2;
  const R SL = selL ? xL1 : xL2, SR = selR ? xR1 : xR2;
  if (SL >= R(0) || !(SR > R(0))) {  // the upwind flux of one side
    const bool left = SL >= R(0);
    const NodeState<DIM, R>& K = left ? L : Rt;
    flux_jac_t<DIM, R>(l, K.v, K.H, gm1, mu, left ? gL : gR);
    gg = K.rhoe * (mul + mu[NV - 1] * (left ? uLn : uRn));
    return;
  }
  const R wL = SL - uLn, wR = SR - uRn;
  const R dd = L.rho * wL - Rt.rho * wR, idd = Ar<R>::rcp(dd);
  const R Ss = (Rt.p - L.p + L.rho * uLn * wL - Rt.rho * uRn * wR) * idd;
  const bool left = Ss >= R(0);
  const NodeState<DIM, R>& K = left ? L : Rt;
  const R SK = left ? SL : SR, uKn = left ? uLn : uRn, wK = left ? wL : wR;
  const R iq = Ar<R>::rcp(SK - Ss), fac = K.rho * wK * iq;
  const R irK = Ar<R>::rcp(K.rho), iw = Ar<R>::rcp(K.rho * wK);
  const R e = K.u[NV - 1] * irK, t = Ss - uKn, z = K.p * iw, r = Ss + z, g = e + t * r;
  // F = F_K + S_K (U* - U_K)
  R gK[NV];
  flux_jac_t<DIM, R>(l, K.v, K.H, gm1, mu, gK);
  gg = K.rhoe * (mul + mu[NV - 1] * uKn);
  R SKb = mu[0] * (fac - K.u[0]) + mu[NV - 1] * (fac * g - K.u[NV - 1]);
  R facb = SK * (mu[0] + mu[NV - 1] * g), Ssb = R(0);
  R vKb[DIM], vLb[DIM], vRb[DIM];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    vLb[d] = vRb[d] = R(0);
    const R us = fac * (d == l ? Ss : K.v[d]);
    SKb += mu[1 + d] * (us - K.u[1 + d]);
    const R ub = SK * mu[1 + d];
    if (d == l) {
      facb += ub * Ss;
      Ssb += ub * fac;
      vKb[d] = R(0);
    } else {
      facb += ub * K.v[d];
      vKb[d] = ub * fac;
    }
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) gK[v] -= SK * mu[v];
  // U*_E = fac g, g = e + t r, t = S* - u_K, r = S* + z, z = p_K/(rho_K w_K), e = E_K/rho_K
  const R gb = SK * mu[NV - 1] * fac;
  R vKlb = -gb * r, pKb = gb * t * iw, rKb = -gb * t * z * irK - gb * e * irK, EKb = gb * irK;
  R wKb = -gb * t * z * Ar<R>::rcp(wK);
  Ssb += gb * (r + t);
  // fac = rho_K w_K / (S_K - S*)
  rKb += facb * wK * iq;
  wKb += facb * K.rho * iq;
  const R qb = -facb * fac * iq;
  SKb += wKb + qb;
  vKlb -= wKb;
  Ssb -= qb;
  // S* = num / dd
  const R numb = Ssb * idd, ddb = -Ssb * Ss * idd;
  R rLb = numb * uLn * wL + ddb * wL, rRb = -numb * uRn * wR - ddb * wR;
  R pLb = -numb, pRb = numb, ELb = R(0), ERb = R(0);
  R vLlb = numb * L.rho * (wL - uLn) - ddb * L.rho;
  R vRlb = -numb * Rt.rho * (wR - uRn) + ddb * Rt.rho;
  R SLb = numb * L.rho * uLn + ddb * L.rho;
  R SRb = -numb * Rt.rho * uRn - ddb * Rt.rho;
  if (left) {
    SLb += SKb; vLlb += vKlb; pLb += pKb; rLb += rKb; ELb += EKb;
  } else {
    SRb += SKb; vRlb += vKlb; pRb += pKb; rRb += rKb; ERb += EKb;
  }
  // the wave speeds
  R aLb = R(0), aRb = R(0), atb = R(0), vtlb = R(0);
  if (selL) { vLlb += SLb; aLb -= SLb; } else { vtlb += SLb; atb -= SLb; }
  if (selR) { vRlb += SRb; aRb += SRb; } else { vtlb += SRb; atb += SRb; }
  // a~ = sqrt((gamma - 1)(H~ - |v~|^2/2))
  const R at2b = atb * R(0.5) * Ar<R>::rcp(at);
  const R Htb = at2b * gm1, v2b = -R(0.5) * at2b * gm1;
  gg += at2b * (Ht - R(0.5) * v2);
  R sLb = Htb * (L.H - Ht) * iden, sRb = Htb * (Rt.H - Ht) * iden;
  const R HLb = Htb * sL * iden, HRb = Htb * sR * iden;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const R vtb = R(2) * vt[d] * v2b + (d == l ? vtlb : R(0));
    vLb[d] += vtb * sL * iden + (d == l ? vLlb : R(0)) + (left ? vKb[d] : R(0));
    vRb[d] += vtb * sR * iden + (d == l ? vRlb : R(0)) + (left ? R(0) : vKb[d]);
    sLb += vtb * (L.v[d] - vt[d]) * iden;
    sRb += vtb * (Rt.v[d] - vt[d]) * iden;
  }
  rLb += sLb * R(0.5) * Ar<R>::rcp(sL);
  rRb += sRb * R(0.5) * Ar<R>::rcp(sR);
  // a_K = sqrt(gamma p_K / rho_K), H_K = (E_K + p_K)/rho_K
  const R irL = Ar<R>::rcp(L.rho), irR = Ar<R>::rcp(Rt.rho);
  const R kL = aLb * R(0.5) * Ar<R>::rcp(L.c) * irL, kR = aRb * R(0.5) * Ar<R>::rcp(Rt.c) * irR;
  pLb += kL * gamma + HLb * irL;
  pRb += kR * gamma + HRb * irR;
  rLb -= kL * gamma * L.p * irL + HLb * L.H * irL;
  rRb -= kR * gamma * Rt.p * irR + HRb * Rt.H * irR;
  gg += kL * L.p + kR * Rt.p;
  ELb += HLb * irL;
  ERb += HRb * irR;
  // primitives -> conserved: p = (gamma - 1)(E - |m|^2/(2 rho)), v = m / rho
  gg += pLb * L.rhoe + pRb * Rt.rhoe;
  R v2L = R(0), v2R = R(0), vvL = R(0), vvR = R(0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    v2L += L.v[d] * L.v[d];
    v2R += Rt.v[d] * Rt.v[d];
    vvL += vLb[d] * L.v[d];
    vvR += vRb[d] * Rt.v[d];
    gL[1 + d] = vLb[d] * irL - pLb * gm1 * L.v[d];
    gR[1 + d] = vRb[d] * irR - pRb * gm1 * Rt.v[d];
  }
  gL[0] = rLb + pLb * gm1 * R(0.5) * v2L - vvL * irL;
  gR[0] = rRb + pRb * gm1 * R(0.5) * v2R - vvR * irR;
  gL[NV - 1] = ELb + pLb * gm1;
  gR[NV - 1] = ERb + pRb * gm1;
  R* gKs = left ? gL : gR;
#pragma unroll
  for (int v = 0; v < NV; ++v) gKs[v] += gK[v];
}

// Domain face (2 l + side) that side `side` of element e in direction l lies on when that face
// carries a boundary condition, else -1.
__device__ __forceinline__ int wall_face(const InstArgs& I, int e, int l, int side) {
  const int f = 2 * l + side;
  if (I.bc[f] == 0) return -1;
  const int c = l == 0 ? e % I.nel[0] : (l == 1 ? (e / I.nel[0]) % I.nel[1] : e / (I.nel[0] * I.nel[1]));
  return (side ? c == I.nel[l] - 1 : c == 0) ? f : -1;
}

// SCH: bit 0 the two-point volume form (Ranocha's flux), bit 1 the HLLC surface flux; 0 is the
// strong or weak volume form with the Rusanov flux.
template <int DIM, int N, class R, int SCH = 0>
struct Vjp {
  using G = Geo<DIM, N>;
  static constexpr bool EC = (SCH & 1) != 0, HLLC = (SCH & 2) != 0;
  static constexpr int NV = G::NV, NP = G::NP, N1 = G::N1, NFN = G::NFN, EPB = G::EPB;
  static constexpr int NF = 2 * DIM, NJS = EPB * NF * NFN;
  static constexpr int T = (((EPB * NP > NJS) ? EPB * NP : NJS) + 31) / 32 * 32;
  // shared: co-state [EPB][NV][NP], face contributions [EPB][NF][NFN][NV], D, (two-point form)
  // the nodes' rho, v, rho e, 1/p, 1/rho [EPB][NV + 2][NP] and the partners' parts of the
  // pairs of one direction [EPB][NO][NV][NP], reduction
  static constexpr int NO = N1 / 2;  // pair offsets per line (cyclic ownership)
  static constexpr int OFF_L = 0, OFF_S = EPB * NV * NP, OFF_D = OFF_S + EPB * NF * NFN * NV;
  static constexpr int OFF_W = OFF_D + N1 * N1;
  static constexpr int OFF_X = OFF_W + (EC ? EPB * (NV + 2) * NP : 0);
  static constexpr int R_SIZE = OFF_X + (EC ? EPB * NO * NV * NP : 0);
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
    NodeState<DIM, R> ns;
    if (active) {
#pragma unroll
      for (int v = 0; v < NV; ++v) sm[OFF_L + (el * NV + v) * NP + nd] = Ar<R>::load(A.lam[v * A.stride + gi]);
      double u64[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) u64[v] = A.U[v * A.stride + gi];
      ns = node_state<DIM, R>(u64, gamma);
      if constexpr (EC) {
        R* W = sm + OFF_W + el * (NV + 2) * NP + nd;
        W[0] = ns.rho;
#pragma unroll
        for (int d = 0; d < DIM; ++d) W[(1 + d) * NP] = ns.v[d];
        W[(NV - 1) * NP] = ns.rhoe;
        W[NV * NP] = Ar<R>::rcp(ns.p);
        W[(NV + 1) * NP] = Ar<R>::rcp(ns.rho);
      }
    }
    __syncthreads();

    // volume: w_m = -sum_l s_l A^l(U_m)^T sum_i Dv[i][m] lam_i
    R w[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) w[v] = R(0);
    if constexpr (EC) {
      // two-point form: R_i = -s_l sum_m Dv[i][m] F#(U_i, U_m) along each line.  F# is symmetric
      // and a pair's cotangent c = Dv[i][m] lam_i + Dv[m][i] lam_m is the same from both of its
      // nodes, so each pair is reverse-differentiated once, by its owner (cyclic ownership as in
      // the forward stage: node i owns the pairs to i+1 .. i+NO, on a line of even length the
      // half-way pair belongs to the lower half): w_i -= s (dF#/dU_a)^T c, and the partner's
      // -s (dF#/dU_b)^T c passes through a shared-memory slot.  The diagonal pair (U_i, U_i),
      // whose Dv[i][i] vanishes inside the line, takes both arguments' parts with c = Dv[i][i]
      // lam_i.  Every pair's gamma derivative counts once.
      R li[NV], irhoi = R(0), ipi = R(0);
      const R igm1 = Ar<R>::rcp(gm1);
      if (active) {
        const R* Wi = sm + OFF_W + el * (NV + 2) * NP + nd;
        ipi = Wi[NV * NP];
        irhoi = Wi[(NV + 1) * NP];
#pragma unroll
        for (int v = 0; v < NV; ++v) li[v] = sm[OFF_L + (el * NV + v) * NP + nd];
      }
      R gsum = R(0);
#pragma unroll
      for (int l = 0; l < DIM; ++l) {
        const R s = s_of<R>(I, l);
        R* X = sm + OFF_X + el * NO * NV * NP;
        const int i = active ? pos(l, nd) : 0, q = active ? face_line(l, nd) : 0;
        if (active) {
          R gl = R(0);
          const R dii = sm[OFF_D + i * N1 + i];
          if (dii != R(0)) {
            R c[NV], ga[NV], gb[NV], cg;
#pragma unroll
            for (int v = 0; v < NV; ++v) c[v] = dii * li[v];
            ec_flux_vjp<DIM, R>(l, ns, irhoi, ipi, ns, irhoi, ipi, gm1, igm1, c, ga, gb, cg);
#pragma unroll
            for (int v = 0; v < NV; ++v) w[v] -= s * (ga[v] + gb[v]);
            gl += cg;
          }
#pragma unroll
          for (int o = 1; o <= NO; ++o) {
            if (2 * o == N1 && i >= N1 / 2) break;
            const int m = i + o < N1 ? i + o : i + o - N1;
            const int nm = line_node(l, q, m);
            const R* Wm = sm + OFF_W + el * (NV + 2) * NP + nm;
            NodeState<DIM, R> B;
            B.rho = Wm[0];
#pragma unroll
            for (int d = 0; d < DIM; ++d) B.v[d] = Wm[(1 + d) * NP];
            B.rhoe = Wm[(NV - 1) * NP];
            B.p = gm1 * B.rhoe;
            const R dim_ = sm[OFF_D + i * N1 + m], dmi = sm[OFF_D + m * N1 + i];
            R c[NV], ga[NV], gb[NV], cg;
#pragma unroll
            for (int v = 0; v < NV; ++v) c[v] = dim_ * li[v] + dmi * sm[OFF_L + (el * NV + v) * NP + nm];
            ec_flux_vjp<DIM, R>(l, ns, irhoi, ipi, B, Wm[(NV + 1) * NP], Wm[NV * NP], gm1, igm1, c, ga, gb, cg);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              w[v] -= s * ga[v];
              X[((o - 1) * NV + v) * NP + nm] = gb[v];
            }
            gl += cg;
          }
          gsum += s * gl;
        }
        __syncthreads();  // the partners' parts of direction l are in the slots
        if (active) {
#pragma unroll
          for (int o = 1; o <= NO; ++o) {
            const int k = i >= o ? i - o : i - o + N1;  // the owner of the pair (k, i)
            if (2 * o == N1 && k >= N1 / 2) continue;
#pragma unroll
            for (int v = 0; v < NV; ++v) w[v] -= s * X[((o - 1) * NV + v) * NP + nd];
          }
        }
        __syncthreads();  // the slots are free for the next direction
      }
      gacc -= (double)gsum;
    } else if (active) {
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
      if constexpr (HLLC) {
        // An interior face's F* enters this element's residual (c lam_own) and the neighbour's
        // (-c lam_nbr), so its part of w_own is c (dF*/dU_own)^T (lam_own - lam_nbr); its gamma
        // derivative, met from both sides' jobs with the same c (lam_own - lam_nbr), counts
        // half.  A domain face (lam_nbr = 0, no second job): slip wall and Dirichlet take the
        // HLLC flux against the mirror state / U_b (the mirror's part folded back with the
        // normal momentum negated), supersonic inflow F(U_b), outflow F(U_own).
        R mu[NV], gLv[NV], gRv[NV], gg = R(0), ao[NV], gown[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) mu[v] = lo[v] - ln[v];
        if (!A.weak || type == 3) flux_jac_t<DIM, R>(l, so.v, so.H, gm1, lo, ao);
        R mlo = R(0), vlo = R(0), vln = R(0);
#pragma unroll
        for (int d = 0; d < DIM; ++d)
          if (d == l) { mlo = lo[1 + d]; vlo = so.v[d]; vln = sn.v[d]; }
        if (type == 2 || type == 3) {
#pragma unroll
          for (int v = 0; v < NV; ++v) gown[v] = type == 3 ? ao[v] : R(0);
          gg = type == 3 ? so.rhoe * (mlo + lo[DIM + 1] * vlo) : sn.rhoe * (mlo + lo[DIM + 1] * vln);
        } else {
          hllc_vjp<DIM, R>(l, sL, sR, gamma, mu, gLv, gRv, gg);
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            gown[v] = side ? gLv[v] : gRv[v];
            if (type == 1) {
              const R ge = side ? gRv[v] : gLv[v];
              gown[v] += (v == 1 + l) ? -ge : ge;
            }
          }
        }
        const R c = (side ? R(-1) : R(1)) * s_of<R>(I, l) * lift_of<R>(I);
        R* S = sm + OFF_S + ((ej * NF + face) * NFN + f) * NV;
#pragma unroll
        for (int v = 0; v < NV; ++v) S[v] = c * (gown[v] - (A.weak ? R(0) : ao[v]));
        const R dFo = A.weak ? R(0) : so.rhoe * (mlo + lo[DIM + 1] * vlo);
        gacc += (double)(c * ((fb >= 0 ? R(1) : R(0.5)) * gg - dFo));
        continue;
      }
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

template <int DIM, int N, class R, int SCH>
__global__ void __launch_bounds__(Vjp<DIM, N, R, SCH>::T) k_rhs_vjp(const VjpArgs A) {
  Vjp<DIM, N, R, SCH>::run(A);
}

// one instance's launch of scheme SCH; *blocks_out receives the grid size
template <int DIM, int N, class R, int SCH>
static cudaError_t launch_vjp_one(const VjpArgs& a, cudaStream_t s, int* blocks_out) {
  using K = Vjp<DIM, N, R, SCH>;
  const int blocks = (a.inst.n_elem + K::EPB - 1) / K::EPB;
  if (blocks_out) *blocks_out = blocks;
  if (blocks == 0) return cudaSuccess;
  if constexpr (K::smem_bytes() > 48 * 1024) {  // above the default dynamic limit: opt in once
    static bool opted = false;
    if (!opted) {
      const cudaError_t e = cudaFuncSetAttribute(k_rhs_vjp<DIM, N, R, SCH>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::smem_bytes());
      if (e != cudaSuccess) return e;
      opted = true;
    }
  }
  k_rhs_vjp<DIM, N, R, SCH><<<blocks, K::T, K::smem_bytes(), s>>>(a);
  return cudaGetLastError();
}

template <int SCH>
static cudaError_t launch_vjp_sch(int dim, int N, int fp32, const VjpArgs& a, cudaStream_t s, int* blocks) {
#define DG_VJP_CASE(D, NN)                                                                         \
  case NN:                                                                                         \
    return fp32 ? launch_vjp_one<D, NN, float, SCH>(a, s, blocks) : launch_vjp_one<D, NN, double, SCH>(a, s, blocks);
  if (dim == 2) {
    switch (N) { DG_VJP_CASE(2, 1) DG_VJP_CASE(2, 2) DG_VJP_CASE(2, 3) DG_VJP_CASE(2, 4) DG_VJP_CASE(2, 5)
                 DG_VJP_CASE(2, 6) DG_VJP_CASE(2, 7) }
  } else if (dim == 3) {
    switch (N) { DG_VJP_CASE(3, 1) DG_VJP_CASE(3, 2) DG_VJP_CASE(3, 3) DG_VJP_CASE(3, 4) DG_VJP_CASE(3, 5) }
  }
#undef DG_VJP_CASE
  return cudaErrorInvalidValue;
}

}  // namespace dg
