// dg_shock.cu -- Hennemann-Gassner shock capturing of the Euler residual (Sec. 3.1.1 "Shock
// Indicator and Smoothing", Eq. vol_blend; App. A "Shock Capturing").
//
// Per stage and instance, around the fused stage launch:
//   1. k_hg_indicator: per element, the modal smoothness of rho p (orthonormal tensor
//      Legendre modes by three line contractions with V^{-1} in shared memory, energies of
//      the top and next-to-top shells; an FP32 filter settles the clearly smooth elements,
//      the others are evaluated in FP64), the sigmoid with threshold T and steepness s, and
//      the clipping to [alpha_min, alpha_max] -> alpha_raw;
//   2. k_hg_alpha: alpha_e = max(alpha_raw_e, alpha_raw of the face neighbours); elements with
//      alpha > 0 are appended to a list (its order does not matter: the elements are
//      independent);
//   3. (the stage launch writes the DG residual of the listed elements to a side buffer and
//      skips their update);
//   4. k_fv_blend: one CTA per listed element (persistent over the list) computes the
//      first-order FV residual on the GLL sub-cells -- the interface fluxes F*(U_i, U_{i+1})
//      and, at the element faces, F* with the neighbour's trace, evaluated exactly as the
//      stage kernel's face jobs do (same conversions and pressure deviation, same flux call
//      after the same axis relabelling), so the F* both elements of a face use agree -- and
//      forms L = (1 - alpha) L_DG + alpha R_FV and the stage update.
// The decisions (alpha_min cut, alpha > 0) are taken in FP64 in both precisions.
#include "dg_stage.cuh"

namespace dg {
namespace {

constexpr int kIT = 128;  // threads of the indicator CTA (more when one element has more nodes)

template <int DIM, int N>
struct SG {
  static constexpr int N1 = N + 1;
  static constexpr int NP = DIM == 2 ? N1 * N1 : N1 * N1 * N1;
  static constexpr int NV = DIM + 2;
  static constexpr int EPB = NP >= kIT ? 1 : kIT / NP;          // elements per indicator CTA
  static constexpr int T = ((EPB * NP + 31) / 32) * 32;          // threads per indicator CTA
  static constexpr int NLINE = NP / N1;
  static constexpr int NJ = DIM * NLINE * (N + 2);                // sub-cell interfaces
  static int stride(int l) { return l == 0 ? 1 : (l == 1 ? N1 : N1 * N1); }
};

template <int N1>
__device__ __forceinline__ int dstride(int l) {
  return l == 0 ? 1 : (l == 1 ? N1 : N1 * N1);
}

// ---- 1: indicator ----
// FP32 filter, FP64 decision: the modes, energies and E are first evaluated in FP32; an
// element whose FP32 E lies below a quarter of E_min -- the E below which the sigmoid is
// under alpha_min, so that alpha_raw is 0 -- is decided there (the FP32 error of E is many
// orders of magnitude below that margin).  If any element of the CTA is not, the CTA repeats
// the evaluation in FP64 exactly as the definition states and decides those elements from
// it.  Smooth regions thus cost FP32 arithmetic only (B300 issues FP64 at a sixtieth of the
// FP32 rate); every decision near the threshold is an FP64 one.
template <int DIM, int N>
struct IG {
  static constexpr int N1 = N + 1;
  static constexpr int NP = DIM == 2 ? N1 * N1 : N1 * N1 * N1;
  static constexpr int NPP = NP <= 32 ? 32 : (NP <= 64 ? 64 : (NP <= 128 ? 128 : 256));  // pow2 >= NP
  static constexpr int EPB = SG<DIM, N>::EPB;
  static constexpr int T = SG<DIM, N>::T;
};

// Modes of the EPB element fields in q[0] (ping-pong with q[1]): V^{-1} along each direction.
// Returns the buffer holding the result.  Every thread of the CTA must call it.
template <int DIM, int N, class F>
__device__ __forceinline__ F* to_modes(F* q0, F* q1, const F* V, int el, int nd, bool active) {
  constexpr int N1 = N + 1, NP = IG<DIM, N>::NP;
  F* src = q0;
  F* dst = q1;
#pragma unroll
  for (int l = 0; l < DIM; ++l) {
    if (active) {
      const int S = dstride<N1>(l);
      const int i = (nd / S) % N1;
      const F* line = src + el * NP + nd - i * S;
      F acc = F(0);
#pragma unroll
      for (int j = 0; j < N1; ++j) acc = fma(V[i * N1 + j], line[j * S], acc);
      dst[el * NP + nd] = acc;
    }
    __syncthreads();
    F* tmp = src;
    src = dst;
    dst = tmp;
  }
  return src;
}

// The four shell energies of every element, by a fixed-order tree in shared memory
// (deterministic): part[el][0][c] = E_tot^(N), E_tot^(N-1), E_high^(N), E_high^(N-1).
template <int DIM, int N, class F>
__device__ __forceinline__ void shell_energies(const F* m, F* part, int el, int nd, bool active) {
  constexpr int N1 = N + 1, NP = IG<DIM, N>::NP, NPP = IG<DIM, N>::NPP, EPB = IG<DIM, N>::EPB;
  const int t = threadIdx.x;
  for (int k = t; k < EPB * NPP * 4; k += blockDim.x) part[k] = F(0);
  __syncthreads();
  if (active) {
    const F mm = m[el * NP + nd];
    int mx = nd % N1;
    mx = max(mx, (nd / N1) % N1);
    if (DIM == 3) mx = max(mx, nd / (N1 * N1));
    const F e2 = mm * mm;
    F* p = part + (el * NPP + nd) * 4;
    p[0] = e2;
    p[1] = mx <= N - 1 ? e2 : F(0);
    p[2] = mx == N ? e2 : F(0);
    p[3] = mx == N - 1 ? e2 : F(0);
  }
  __syncthreads();
#pragma unroll 1
  for (int s = NPP / 2; s >= 1; s >>= 1) {
    for (int k = t; k < EPB * s * 4; k += blockDim.x) {
      const int e = k / (s * 4), r = k - e * s * 4, i = r >> 2, c = r & 3;
      part[(e * NPP + i) * 4 + c] += part[(e * NPP + i + s) * 4 + c];
    }
    __syncthreads();
  }
}

template <int DIM, int N>
__global__ void __launch_bounds__(IG<DIM, N>::T) k_hg_indicator(const ShockArgs a) {
  using G = IG<DIM, N>;
  constexpr int N1 = G::N1, NP = G::NP, NPP = G::NPP, EPB = G::EPB, NV = DIM + 2;
  __shared__ float qf[2][EPB * NP], Vf[N1 * N1], pf[EPB * NPP * 4];
  __shared__ double qd[2][EPB * NP], Vd[N1 * N1], pd[EPB * NPP * 4];
  __shared__ int need[EPB], any;
  const int t = threadIdx.x;
  for (int k = t; k < N1 * N1; k += blockDim.x) {
    Vd[k] = a.Vinv[k];
    Vf[k] = d2f_rn(a.Vinv[k]);
  }
  if (t == 0) any = 0;
  const int el = t / NP, nd = t - el * NP;
  const int e = blockIdx.x * EPB + el;
  const bool active = t < EPB * NP && e < a.inst.n_elem;
  const long long gi = a.inst.base + (long long)e * NP + nd;
  if (active) {  // rho p in FP32 for the filter
    float u[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = d2f_rz(a.U[v * a.stride + gi]);
    float m2 = 0.0f;
#pragma unroll
    for (int d = 0; d < DIM; ++d) m2 = fmaf(u[1 + d], u[1 + d], m2);
    const float p = a.pf.gm1 * (u[DIM + 1] - 0.5f * m2 * __fdividef(1.0f, u[0]));
    qf[0][el * NP + nd] = u[0] * p;
  }
  __syncthreads();
  const float* mf = to_modes<DIM, N, float>(qf[0], qf[1], Vf, el, nd, active);
  shell_energies<DIM, N, float>(mf, pf, el, nd, active);
  if (t < EPB) {
    const int ee = blockIdx.x * EPB + t;
    const float* s4 = pf + t * NPP * 4;
    const float r1 = s4[0] > 0.0f ? s4[2] / s4[0] : 0.0f;
    const float r2 = s4[1] > 0.0f ? s4[3] / s4[1] : 0.0f;
    const float E = fmaxf(r1, r2);
    need[t] = ee < a.inst.n_elem && !(E <= 0.25f * (float)a.emin) ? 1 : 0;
    if (need[t]) atomicOr(&any, 1);
  }
  __syncthreads();
  double al = 0.0;
  if (any) {  // FP64, as the definition states
    if (active) {
      double u[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) u[v] = a.U[v * a.stride + gi];
      double m2 = 0.0;
#pragma unroll
      for (int d = 0; d < DIM; ++d) m2 = fma(u[1 + d], u[1 + d], m2);
      const double p = (a.gamma - 1.0) * (u[DIM + 1] - 0.5 * m2 / u[0]);
      qd[0][el * NP + nd] = u[0] * p;
    }
    __syncthreads();
    const double* md = to_modes<DIM, N, double>(qd[0], qd[1], Vd, el, nd, active);
    shell_energies<DIM, N, double>(md, pd, el, nd, active);
    if (t < EPB && need[t]) {
      const double* s4 = pd + t * NPP * 4;
      const double r1 = s4[0] > 0.0 ? s4[2] / s4[0] : 0.0;
      const double r2 = s4[1] > 0.0 ? s4[3] / s4[1] : 0.0;
      const double E = fmax(r1, r2);
      al = 1.0 / (1.0 + exp(-(a.sharp / a.thr) * (E - a.thr)));
      if (al < a.alpha_min) al = 0.0;
      al = fmin(al, a.alpha_max);
    }
  }
  if (t < EPB && blockIdx.x * EPB + t < a.inst.n_elem) a.alpha_raw[blockIdx.x * EPB + t] = al;
}

// ---- 2: neighbourhood maximum and the list of blended elements ----
template <int DIM>
__global__ void k_hg_alpha(const ShockArgs a) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.inst.n_elem) return;
  const int* nel = a.inst.nel;
  const int c[3] = {e % nel[0], (e / nel[0]) % nel[1], DIM == 3 ? e / (nel[0] * nel[1]) : 0};
  double al = a.alpha_raw[e];
#pragma unroll
  for (int l = 0; l < DIM; ++l) {
#pragma unroll
    for (int d = -1; d <= 1; d += 2) {
      if (a.inst.nonper && boundary_face(a.inst, DIM, e, l, d > 0 ? 1 : 0) >= 0) continue;  // no neighbour
      int cc[3] = {c[0], c[1], c[2]};
      cc[l] = (cc[l] + d + nel[l]) % nel[l];
      al = fmax(al, a.alpha_raw[cc[0] + nel[0] * (cc[1] + nel[1] * cc[2])]);
    }
  }
  a.alpha[e] = al;
  if (al > 0.0) a.list[atomicAdd(a.count, 1)] = e;
}

// ---- 4: sub-cell FV residual, blend, stage update ----
template <class R> __device__ __forceinline__ const ScalarsT<R>& shs(const ShockArgs& a);
template <> __device__ __forceinline__ const ScalarsT<double>& shs<double>(const ShockArgs& a) { return a.pd; }
template <> __device__ __forceinline__ const ScalarsT<float>& shs<float>(const ShockArgs& a) { return a.pf; }

// F*(U_L, U_R) in direction l from FP64 states, as the stage kernel's face jobs evaluate it.
template <int DIM, class R>
__device__ __forceinline__ void interface_flux(const ShockArgs& a, int l, const double* L64,
                                               const double* R64, R* F) {
  constexpr int NV = DIM + 2;
  R uL0[NV], uR0[NV], uL[NV], uR[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    uL0[v] = Ar<R>::load(L64[v]);
    uR0[v] = Ar<R>::load(R64[v]);
  }
  const ScalarsT<R>& k = shs<R>(a);
  const R pdL = pdev<DIM>(L64, uL0, a.pd.gm1, a.pd.p_ref, k.hgm1);
  const R pdR = pdev<DIM>(R64, uR0, a.pd.gm1, a.pd.p_ref, k.hgm1);
  to_face_axes<DIM>(uL0, uL, l);
  to_face_axes<DIM>(uR0, uR, l);
  const Prim<DIM, R> pa = prims<DIM>(uL, pdL, k.p_ref);
  const Prim<DIM, R> pb = prims<DIM>(uR, pdR, k.p_ref);
  trace_momentum<DIM>(pa, uL);
  trace_momentum<DIM>(pb, uR);
  R Fs[NV];
  surface_flux<DIM, 0>(a.surface, uL, pa, uR, pb, k.gamma, k.igm1, k.p_ref, Fs);
  from_face_axes<DIM>(Fs, F, l);
}

// Flux at domain face fb (boundary condition) from the interior node's FP64 state, as the
// stage kernel's face jobs evaluate it; side = 1 when the interior is the left state.
template <int DIM, class R>
__device__ __forceinline__ void domain_face_flux(const ShockArgs& a, int fb, int l, int side,
                                                 const double* own64, R* F) {
  constexpr int NV = DIM + 2;
  R own0[NV], own[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) own0[v] = Ar<R>::load(own64[v]);
  const ScalarsT<R>& k = shs<R>(a);
  const R pd = pdev<DIM>(own64, own0, a.pd.gm1, a.pd.p_ref, k.hgm1);
  to_face_axes<DIM>(own0, own, l);
  const Prim<DIM, R> po = prims<DIM>(own, pd, k.p_ref);
  trace_momentum<DIM>(po, own);
  R Fs[NV];
  boundary_flux<DIM, R>(a.inst, fb, l, side, own, po, a.surface, k.gamma, k.igm1, k.p_ref, a.pd.gm1,
                        a.pd.p_ref, k.hgm1, Fs);
  from_face_axes<DIM>(Fs, F, l);
}

__device__ __forceinline__ int nbr_elem(const InstArgs& I, int dim, int e, int l, int d) {
  int c[3] = {e % I.nel[0], (e / I.nel[0]) % I.nel[1], dim == 3 ? e / (I.nel[0] * I.nel[1]) : 0};
  c[l] = (c[l] + d + I.nel[l]) % I.nel[l];
  return c[0] + I.nel[0] * (c[1] + I.nel[1] * c[2]);
}

template <int DIM, int N, class R>
__global__ void __launch_bounds__(128) k_fv_blend(const ShockArgs a) {
  using G = SG<DIM, N>;
  constexpr int N1 = G::N1, NP = G::NP, NV = G::NV, NLINE = G::NLINE, NJ = G::NJ;
  __shared__ R Fh[NJ * NV];
  const int t = threadIdx.x;
  const InstArgs& I = a.inst;
  const int n = *a.count;
  for (int k = blockIdx.x; k < n; k += gridDim.x) {
    const int e = a.list[k];
    // interface jobs: direction l, line, interface position i = 0..N+1 (between nodes i-1, i)
    for (int j = t; j < NJ; j += blockDim.x) {
      const int l = j / (NLINE * (N + 2));
      const int r = j - l * NLINE * (N + 2);
      const int line = r / (N + 2), i = r - line * (N + 2);
      const int S = dstride<N1>(l);
      const int base_nd = (line % S) + (line / S) * S * N1;  // node of position 0 on this line
      const int fb = (i == 0 || i == N + 1) && I.nonper ? boundary_face(I, DIM, e, l, i == N + 1 ? 1 : 0) : -1;
      R F[NV];
      if (fb >= 0) {  // element face on a domain boundary: the boundary functor
        const long long go = I.base + (long long)e * NP + base_nd + (i == 0 ? 0 : N) * S;
        double own64[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) own64[v] = a.U[v * a.stride + go];
        domain_face_flux<DIM, R>(a, fb, l, i == 0 ? 0 : 1, own64, F);
      } else {
        int eL = e, iL = i - 1, eR = e, iR = i;
        if (i == 0) { eL = nbr_elem(I, DIM, e, l, -1); iL = N; }
        if (i == N + 1) { eR = nbr_elem(I, DIM, e, l, +1); iR = 0; }
        const long long gL = I.base + (long long)eL * NP + base_nd + iL * S;
        const long long gR = I.base + (long long)eR * NP + base_nd + iR * S;
        double L64[NV], R64[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          L64[v] = a.U[v * a.stride + gL];
          R64[v] = a.U[v * a.stride + gR];
        }
        interface_flux<DIM, R>(a, l, L64, R64, F);
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) Fh[j * NV + v] = F[v];
    }
    __syncthreads();
    const double al = a.alpha[e];
    for (int nd = t; nd < NP; nd += blockDim.x) {
      R rfv[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) rfv[v] = R(0);
#pragma unroll
      for (int l = 0; l < DIM; ++l) {
        const int S = dstride<N1>(l);
        const int i = (nd / S) % N1;
        const int line = (nd % S) + (nd / (S * N1)) * S;
        const int j0 = (l * NLINE + line) * (N + 2) + i;  // interface i - 1/2; i + 1/2 is j0 + 1
        const R c = (sizeof(R) == 4 ? R(I.sf[l]) : R(I.s[l])) *
                    (sizeof(R) == 4 ? R(a.iwf[i]) : R(a.iw[i]));
#pragma unroll
        for (int v = 0; v < NV; ++v) rfv[v] -= c * (Fh[(j0 + 1) * NV + v] - Fh[j0 * NV + v]);
      }
      const long long gi = I.base + (long long)e * NP + nd;
      double res[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const double L = fma(al, Ar<R>::widen(rfv[v]) - a.ldg[v * a.stride + gi], a.ldg[v * a.stride + gi]);
        if (a.mode == 0) {
          res[v] = L;
        } else {
          const double u = a.U[v * a.stride + gi];
          double x = fma(a.cb, u, a.bdt * L);
          if (a.need_un) x = fma(a.ca, a.Un[v * a.stride + gi], x);
          res[v] = x;
          if (a.acc) {
            double y = fma(a.acc_b, u, a.acc_bdt * L);
            if (a.acc_a != 0.0) y = fma(a.acc_a, a.acc[v * a.stride + gi], y);
            a.acc[v * a.stride + gi] = y;
          }
        }
      }
      if (a.mode == 1 && a.floor_on) {  // the stage kernel's positivity floor
        if (a.rho_floor > 0.0 && res[0] < a.rho_floor) res[0] = a.rho_floor;
        double kin = 0.0;
#pragma unroll
        for (int d = 0; d < DIM; ++d) kin += res[1 + d] * res[1 + d] / res[0];
        const double p = (a.gamma - 1.0) * (res[DIM + 1] - 0.5 * kin);
        if (a.p_floor > 0.0 && p < a.p_floor) res[DIM + 1] = a.p_floor / (a.gamma - 1.0) + 0.5 * kin;
      }
      bool finite = true;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        finite = finite && finite64(res[v]);
        a.out[v * a.stride + gi] = res[v];
      }
      if (!finite) atomicOr(a.err, 1u);
    }
    __syncthreads();
  }
}

template <int DIM, int N>
cudaError_t indicator_dn(const ShockArgs& a, cudaStream_t s) {
  using G = IG<DIM, N>;
  if (a.inst.n_elem <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((a.inst.n_elem + G::EPB - 1) / G::EPB);
  k_hg_indicator<DIM, N><<<grid, G::T, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_hg_alpha<DIM><<<(unsigned)((a.inst.n_elem + 127) / 128), 128, 0, s>>>(a);
  return cudaGetLastError();
}

template <int DIM, int N>
cudaError_t blend_dn(int fp32, const ShockArgs& a, cudaStream_t s) {
  if (a.inst.n_elem <= 0) return cudaSuccess;
  const int want = a.inst.n_elem;
  const unsigned grid = (unsigned)(want < grid_cap() ? want : grid_cap());
  if (fp32) k_fv_blend<DIM, N, float><<<grid, 128, 0, s>>>(a);
  else k_fv_blend<DIM, N, double><<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}

#define DG_SHOCK_DISPATCH(CALL)                                                  \
  switch (dim * 16 + N) {                                                        \
    case 2 * 16 + 2: return CALL(2, 2);                                          \
    case 2 * 16 + 3: return CALL(2, 3);                                          \
    case 2 * 16 + 4: return CALL(2, 4);                                          \
    case 2 * 16 + 5: return CALL(2, 5);                                          \
    case 2 * 16 + 6: return CALL(2, 6);                                          \
    case 2 * 16 + 7: return CALL(2, 7);                                          \
    case 3 * 16 + 2: return CALL(3, 2);                                          \
    case 3 * 16 + 3: return CALL(3, 3);                                          \
    case 3 * 16 + 4: return CALL(3, 4);                                          \
    case 3 * 16 + 5: return CALL(3, 5);                                          \
    default: return cudaErrorInvalidValue;                                       \
  }

}  // namespace

bool have_shock(int dim, int N) {
  return (dim == 2 && N >= 2 && N <= 7) || (dim == 3 && N >= 2 && N <= 5);
}

cudaError_t launch_shock_indicator(int dim, int N, const ShockArgs& a, cudaStream_t s) {
#define DG_I(d, n) indicator_dn<d, n>(a, s)
  DG_SHOCK_DISPATCH(DG_I)
#undef DG_I
}

cudaError_t launch_shock_blend(int dim, int N, int fp32, const ShockArgs& a, cudaStream_t s) {
#define DG_B(d, n) blend_dn<d, n>(fp32, a, s)
  DG_SHOCK_DISPATCH(DG_B)
#undef DG_B
}

}  // namespace dg
