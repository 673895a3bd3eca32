// dg_curved.cu -- the Euler residual and stage update on curved (curvilinear) meshes
// (Sec. 3.1.1: element maps x = X(xi), metric terms Ja^l with the discrete GCL, the strong
// form Eq. vol_weak and the two-point form Eq. vol_split with averaged metrics, Eq. surf_int
// along the contravariant normal).
//
// One CTA per element, one launch per stage (per instance):
//   1. one thread per node: the FP64 state converted to the flux precision R, the pressure
//      deviation from the FP64 energy, the node's metric terms Ja^l_d and 1/J; the strong form
//      stages the contravariant fluxes Ja^l . F(U), the two-point form per-node primitives;
//   2. one thread per face node: both traces expressed in the orthonormal frame (n, t1, t2) of
//      the face's contravariant normal n = Ja^l / |Ja^l| (taken at the own node: it depends
//      only on the face's nodes, so both elements of a face use the same one), the Riemann flux
//      of direction 0 there (at a domain face with a boundary condition: the functor's flux in
//      the same frame), rotated back and scaled by |Ja^l|; minus Ja^l . F(U_own); lifted by
//      1 / (J w);
//   3. one thread per node: the volume term -(1/J) sum_l sum_m D_im Ja^l(m) . F(U_m) (strong) or
//      -(2/J) sum_l sum_m D_im {{Ja^l}} . F#(U_i, U_m) (two-point, F# in all DIM Cartesian
//      directions per pair), the lifted face terms, and L or the Shu-Osher update.
// The metric terms are computed once on the host and read per stage (DIM^2 + 1 doubles per
// node).  This path favours clarity over the Cartesian kernel's tuning (no pair sharing, no
// persistent CTAs).
#include "dg_stage.cuh"

namespace dg {
namespace {

template <int DIM, int N, bool EC, class R>
struct CG {
  static constexpr int N1 = N + 1;
  static constexpr int NP = DIM == 2 ? N1 * N1 : N1 * N1 * N1;
  static constexpr int NFN = DIM == 2 ? N1 : N1 * N1;
  static constexpr int NV = DIM + 2;
  static constexpr int NF = 2 * DIM;
  static constexpr int NJ = NF * NFN;
  static constexpr int T = ((cmax(NP, NJ) + 31) / 32) * 32;
  static constexpr int NQ = EC ? 8 : DIM * NV;  // per node: prims (EC) or contravariant fluxes
  // two-point pairs along a line: every node owns (N1-1)/2 of them (partner i+k mod N1,
  // k = 1..(N1-1)/2) and, on a line of even length, the lower half owns the k = N1/2 pair too
  static constexpr int KM = N1 / 2;
  // shared layout (R): U [NV][NP], Q [NQ][NP], pd [NP], Ja [DIM*DIM][NP], jinv [NP],
  // S [NF][NFN][NV], D [N1*N1], pair fluxes of one direction P [NP][KM][NV] (EC)
  static constexpr int O_U = 0, O_Q = O_U + NV * NP, O_PD = O_Q + NQ * NP, O_JA = O_PD + NP;
  static constexpr int O_JI = O_JA + DIM * DIM * NP, O_S = O_JI + NP, O_D = O_S + NF * NFN * NV;
  static constexpr int O_P = O_D + N1 * N1;
  static constexpr int SIZE = O_P + (EC ? NP * KM * NV : 0);
  static constexpr size_t smem() { return sizeof(R) * (size_t)SIZE; }
};

template <int N1>
__device__ __forceinline__ int cstride(int l) {
  return l == 0 ? 1 : (l == 1 ? N1 : N1 * N1);
}

// Orthonormal frame of the unit vector n: t1 (and t2 in 3D).  3D: t1 is n x e_a normalised,
// e_a the unit axis of the smallest |n_a| (the best-conditioned cross product), t2 = n x t1.
// The rotated Riemann flux does not depend on the choice of tangents (rotational invariance
// of the Euler fluxes), so any orthonormal completion gives the same F* . n.
template <int DIM, class R>
__device__ __forceinline__ void frame(const R* n, R (&t)[2][3]) {
  if constexpr (DIM == 2) {
    t[0][0] = -n[1];
    t[0][1] = n[0];
    t[0][2] = R(0);
  } else {
    int a = 0;
    if (Ar<R>::abs(n[1]) < Ar<R>::abs(n[a])) a = 1;
    if (Ar<R>::abs(n[2]) < Ar<R>::abs(n[a])) a = 2;
    const R e0 = a == 0 ? R(1) : R(0), e1 = a == 1 ? R(1) : R(0), e2 = a == 2 ? R(1) : R(0);
    const R c0 = n[1] * e2 - n[2] * e1, c1 = n[2] * e0 - n[0] * e2, c2 = n[0] * e1 - n[1] * e0;
    const R ic = Ar<R>::rcp(Ar<R>::sqrt(c0 * c0 + c1 * c1 + c2 * c2));
    t[0][0] = c0 * ic;
    t[0][1] = c1 * ic;
    t[0][2] = c2 * ic;
    t[1][0] = n[1] * t[0][2] - n[2] * t[0][1];
    t[1][1] = n[2] * t[0][0] - n[0] * t[0][2];
    t[1][2] = n[0] * t[0][1] - n[1] * t[0][0];
  }
}

template <int DIM, class R>
__device__ __forceinline__ void to_frame(const R* u, const R* n, const R (&t)[2][3], R* r) {
  constexpr int NV = DIM + 2;
  r[0] = u[0];
  r[NV - 1] = u[NV - 1];
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    const R* b = c == 0 ? n : t[c - 1];
    R acc = R(0);
#pragma unroll
    for (int d = 0; d < DIM; ++d) acc += u[1 + d] * b[d];
    r[1 + c] = acc;
  }
}

template <int DIM, int N, bool EC, class R>
__global__ void __launch_bounds__(CG<DIM, N, EC, R>::T) k_euler_curved(const StageArgs A, const double* __restrict__ met) {
  using G = CG<DIM, N, EC, R>;
  constexpr int N1 = G::N1, NP = G::NP, NFN = G::NFN, NV = G::NV;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sm = reinterpret_cast<R*>(smem_raw);
  const InstArgs& I = A.inst;
  const int e = blockIdx.x;
  const int t = threadIdx.x;
  const ScalarsT<R>& k = sc<R>(A);
  const R gamma = k.gamma, igm1 = k.igm1, p_ref = k.p_ref;
  const long long stride = A.stride;
  for (int q = t; q < N1 * N1; q += blockDim.x) sm[G::O_D + q] = Ar<R>::load(A.Dv[q]);  // plain D
  // phase 1
  if (t < NP) {
    const long long gi = I.base + (long long)e * NP + t;
    double u64[NV];
    R u[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      u64[v] = A.U[v * stride + gi];
      u[v] = Ar<R>::load(u64[v]);
      sm[G::O_U + v * NP + t] = u[v];
    }
    const R pd = pdev<DIM>(u64, u, A.pd.gm1, A.pd.p_ref, k.hgm1);
    if (!positive<DIM>(u64, u, pd, p_ref, k.margin_e, k.margin_0, A.pd.gm1)) atomicOr(A.err, 2u);
    sm[G::O_PD + t] = pd;
    R ja[DIM * DIM];
#pragma unroll
    for (int c = 0; c < DIM * DIM; ++c) {
      ja[c] = Ar<R>::load(met[c * stride + gi]);
      sm[G::O_JA + c * NP + t] = ja[c];
    }
    sm[G::O_JI + t] = Ar<R>::load(met[DIM * DIM * stride + gi]);
    const Prim<DIM, R> q = prims<DIM>(u, pd, p_ref);
    if constexpr (EC) {
      const R beta = q.rho * Ar<R>::rcp(q.p);
      const bool f32 = sizeof(R) == 4;
      sm[G::O_Q + 0 * NP + t] = q.rho;
#pragma unroll
      for (int d = 0; d < 3; ++d) sm[G::O_Q + (1 + d) * NP + t] = d < DIM ? q.v[d] : R(0);
      sm[G::O_Q + 4 * NP + t] = pd;
      sm[G::O_Q + 5 * NP + t] = beta;
      sm[G::O_Q + 6 * NP + t] = f32 ? Ar<R>::log(q.rho) : R(0);
      sm[G::O_Q + 7 * NP + t] = f32 ? Ar<R>::log(beta) : R(0);
    } else {
      R F[DIM][NV];
      point_flux<DIM, 0>(u, q, F[0]);
      point_flux<DIM, 1>(u, q, F[1]);
      if constexpr (DIM == 3) point_flux<DIM, 2>(u, q, F[2]);
#pragma unroll
      for (int l = 0; l < DIM; ++l)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          R acc = R(0);
#pragma unroll
          for (int d = 0; d < DIM; ++d) acc += ja[l * DIM + d] * F[d][v];
          sm[G::O_Q + (l * NV + v) * NP + t] = acc;
        }
    }
  }
  __syncthreads();
  // phase 2: face nodes
  if (t < G::NJ) {
    const int face = t / NFN, j = t - face * NFN, l = face >> 1, side = face & 1;
    const int S = cstride<N1>(l);
    const int line_nd = (j % S) + (j / S) * S * N1;  // node of position 0 on the face-normal line
    const int nd = line_nd + (side ? N : 0) * S;
    R own[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) own[v] = sm[G::O_U + v * NP + nd];
    const R pd_own = sm[G::O_PD + nd];
    R ja[DIM], s2 = R(0);
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      ja[d] = sm[G::O_JA + (l * DIM + d) * NP + nd];
      s2 += ja[d] * ja[d];
    }
    const R s = Ar<R>::sqrt(s2), is = Ar<R>::rcp(s);
    R n[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int d = 0; d < DIM; ++d) n[d] = ja[d] * is;
    R tv[2][3];
    frame<DIM>(n, tv);
    R ro[NV], rn[NV];
    to_frame<DIM>(own, n, tv, ro);
    const Prim<DIM, R> po = prims<DIM>(ro, pd_own, p_ref);
    // the exterior state in the frame: the neighbour's trace, or at a domain face the
    // boundary functor's (Sec. 3.1.1): slip wall -- the mirror state (normal momentum, the
    // frame's first momentum row, reversed); Dirichlet -- U_b; inflow -- F* = F(U_b) . n;
    // outflow -- F* = F(U-) . n
    const int fb = I.nonper ? boundary_face(I, DIM, e, l, side) : -1;
    const int type = fb >= 0 ? I.bc[fb] : 0;
    R pd_ext = pd_own;
    if (fb < 0 || type == 2 || type == 4) {
      double n64[NV];
      R ext[NV];
      if (fb < 0) {  // the neighbour's trace
        int c[3] = {e % I.nel[0], (e / I.nel[0]) % I.nel[1], DIM == 3 ? e / (I.nel[0] * I.nel[1]) : 0};
        c[l] = (c[l] + (side ? 1 : -1) + I.nel[l]) % I.nel[l];
        const int en = c[0] + I.nel[0] * (c[1] + I.nel[1] * c[2]);
        const long long gn = I.base + (long long)en * NP + line_nd + (side ? 0 : N) * S;
#pragma unroll
        for (int v = 0; v < NV; ++v) n64[v] = A.U[v * stride + gn];
      } else {  // the prescribed state
#pragma unroll
        for (int v = 0; v < NV; ++v) n64[v] = I.bcs[fb][v];
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) ext[v] = Ar<R>::load(n64[v]);
      pd_ext = pdev<DIM>(n64, ext, A.pd.gm1, A.pd.p_ref, k.hgm1);
      to_frame<DIM>(ext, n, tv, rn);
    } else {  // slip wall (mirror) or outflow (the own trace)
#pragma unroll
      for (int v = 0; v < NV; ++v) rn[v] = ro[v];
      if (type == 1) rn[1] = -ro[1];
    }
    const Prim<DIM, R> pn = prims<DIM>(rn, pd_ext, p_ref);
    R Fr[NV];
    if (type == 2) point_flux<DIM, 0>(rn, pn, Fr);       // supersonic inflow
    else if (type == 3) point_flux<DIM, 0>(ro, po, Fr);  // supersonic outflow
    else if (side) surface_flux<DIM, 0>(A.surface, ro, po, rn, pn, gamma, igm1, p_ref, Fr);
    else surface_flux<DIM, 0>(A.surface, rn, pn, ro, po, gamma, igm1, p_ref, Fr);
    // back to Cartesian components, scaled by |Ja^l|; minus the own contravariant flux
    R Fs[NV];
    Fs[0] = s * Fr[0];
    Fs[NV - 1] = s * Fr[NV - 1];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      R acc = Fr[1] * n[d];
#pragma unroll
      for (int cc = 1; cc < DIM; ++cc) acc += Fr[1 + cc] * tv[cc - 1][d];
      Fs[1 + d] = s * acc;
    }
    const Prim<DIM, R> qo = prims<DIM>(own, pd_own, p_ref);
    R Fd[NV];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      if (d == 0) point_flux<DIM, 0>(own, qo, Fd);
      else if (d == 1) point_flux<DIM, 1>(own, qo, Fd);
      else point_flux<DIM, DIM - 1>(own, qo, Fd);
#pragma unroll
      for (int v = 0; v < NV; ++v) Fs[v] -= ja[d] * Fd[v];
    }
    const R cf = (side ? R(-1) : R(1)) * sm[G::O_JI + nd] * liftv<R>(I);
#pragma unroll
    for (int v = 0; v < NV; ++v) sm[G::O_S + (face * NFN + j) * NV + v] = cf * Fs[v];
  }
  __syncthreads();
  // phase 3: volume terms and lifted face terms per node
  const bool node = t < NP;
  const int nd = node ? t : 0;
  R acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = R(0);
  const R jinv = sm[G::O_JI + nd];
  const R* Dv = sm + G::O_D;
  auto lifted = [&](int l, int S, int i) {
    const int jf = (nd % S) + (nd / (S * N1)) * S;
    if (i == 0)
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] += sm[G::O_S + ((2 * l) * NFN + jf) * NV + v];
    if (i == N)
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] += sm[G::O_S + ((2 * l + 1) * NFN + jf) * NV + v];
  };
  if constexpr (EC) {
    // The contracted two-point flux of a pair (i, m) is symmetric (the metric average too), so
    // each pair is evaluated once: its owner adds 2/J_i D_im F and stores F; after the barrier
    // the partner adds 2/J_m D_mi F.  The diagonal pair is the node's own.
    const R* Q = sm + G::O_Q;
    R* Pf = sm + G::O_P;
    auto pair_flux = [&](int l, int na, int nb, R* F) {
      const R va[3] = {Q[1 * NP + na], Q[2 * NP + na], Q[3 * NP + na]};
      const R vb[3] = {Q[1 * NP + nb], Q[2 * NP + nb], Q[3 * NP + nb]};
      R a[DIM];
#pragma unroll
      for (int d = 0; d < DIM; ++d)
        a[d] = R(0.5) * (sm[G::O_JA + (l * DIM + d) * NP + na] + sm[G::O_JA + (l * DIM + d) * NP + nb]);
      ec_flux_prims_n<DIM>(Q[na], va, Q[4 * NP + na], Q[5 * NP + na], Q[6 * NP + na], Q[7 * NP + na], Q[nb],
                           vb, Q[4 * NP + nb], Q[5 * NP + nb], Q[6 * NP + nb], Q[7 * NP + nb], igm1, p_ref, a,
                           F);
    };
    const R two_jinv = R(2) * jinv;
#pragma unroll 1
    for (int l = 0; l < DIM; ++l) {
      const int S = cstride<N1>(l);
      const int i = (nd / S) % N1;
      const int base = nd - i * S;
      if (node) {
        R F[NV];
        pair_flux(l, nd, nd, F);
        const R cd = two_jinv * Dv[i * N1 + i];
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] -= cd * F[v];
#pragma unroll
        for (int k = 1; k <= G::KM; ++k) {
          if (2 * k == G::N1 && i >= G::KM) continue;  // the half-way pair of an even line: lower node
          const int m = i + k < N1 ? i + k : i + k - N1;
          pair_flux(l, nd, base + m * S, F);
          const R cm = two_jinv * Dv[i * N1 + m];
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            acc[v] -= cm * F[v];
            Pf[(nd * G::KM + (k - 1)) * NV + v] = F[v];
          }
        }
      }
      __syncthreads();
      if (node) {
#pragma unroll
        for (int k = 1; k <= G::KM; ++k) {
          const int j = i - k >= 0 ? i - k : i - k + N1;  // the owner of pair (j, j + k = i)
          if (2 * k == G::N1 && j >= G::KM) continue;
          const R cm = two_jinv * Dv[i * N1 + j];
          const int nj = base + j * S;
#pragma unroll
          for (int v = 0; v < NV; ++v) acc[v] -= cm * Pf[(nj * G::KM + (k - 1)) * NV + v];
        }
        lifted(l, S, i);
      }
      if (l + 1 < DIM) __syncthreads();  // the next direction reuses the pair buffer
    }
    if (!node) return;
  } else {
    if (!node) return;
#pragma unroll
    for (int l = 0; l < DIM; ++l) {
      const int S = cstride<N1>(l);
      const int i = (nd / S) % N1;
      const int base = nd - i * S;
#pragma unroll
      for (int m = 0; m < N1; ++m) {
        const R cm = jinv * Dv[i * N1 + m];
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] -= cm * sm[G::O_Q + (l * NV + v) * NP + base + m * S];
      }
      lifted(l, S, i);
    }
  }
  const long long gi = I.base + (long long)e * NP + nd;
  double res[NV];
  if (A.mode == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) res[v] = Ar<R>::widen(acc[v]);
  } else {
    const R cbdt = k.cbdt;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double u = A.U[v * stride + gi];
      double x = fma(A.cb, u, Ar<R>::widen(cbdt * acc[v]));
      if (A.need_un) x = fma(A.ca, A.Un[v * stride + gi], x);
      res[v] = x;
      if (A.acc) {
        double y = fma(A.acc_b, u, Ar<R>::widen(k.abdt * acc[v]));
        if (A.acc_a != 0.0) y = fma(A.acc_a, A.acc[v * stride + gi], y);
        A.acc[v * stride + gi] = y;
      }
    }
  }
  bool finite = true;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    finite = finite && finite64(res[v]);
    A.out[v * stride + gi] = res[v];
  }
  if (!finite) atomicOr(A.err, 1u);
}

template <int DIM, int N, bool EC, class R>
cudaError_t curved_one(const StageArgs* a, const double* met, cudaStream_t s) {
  using G = CG<DIM, N, EC, R>;
  if (!a)
    return cudaFuncSetAttribute(k_euler_curved<DIM, N, EC, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)G::smem());
  if (a->inst.n_elem <= 0) return cudaSuccess;
  k_euler_curved<DIM, N, EC, R><<<a->inst.n_elem, G::T, G::smem(), s>>>(*a, met);
  return cudaGetLastError();
}

template <int DIM, int N>
cudaError_t curved_dn(int ec, int fp32, const StageArgs* a, const double* met, cudaStream_t s) {
  if (ec) return fp32 ? curved_one<DIM, N, true, float>(a, met, s) : curved_one<DIM, N, true, double>(a, met, s);
  return fp32 ? curved_one<DIM, N, false, float>(a, met, s) : curved_one<DIM, N, false, double>(a, met, s);
}

}  // namespace

bool have_curved(int dim, int N) { return (dim == 2 && N >= 1 && N <= 7) || (dim == 3 && N >= 1 && N <= 5); }

// a == null: set the kernel's shared-memory attribute (before the first launch, outside capture)
cudaError_t launch_curved(int dim, int N, int ec, int fp32, const StageArgs* a, const double* met,
                          cudaStream_t s) {
  switch (dim * 16 + N) {
    case 2 * 16 + 1: return curved_dn<2, 1>(ec, fp32, a, met, s);
    case 2 * 16 + 2: return curved_dn<2, 2>(ec, fp32, a, met, s);
    case 2 * 16 + 3: return curved_dn<2, 3>(ec, fp32, a, met, s);
    case 2 * 16 + 4: return curved_dn<2, 4>(ec, fp32, a, met, s);
    case 2 * 16 + 5: return curved_dn<2, 5>(ec, fp32, a, met, s);
    case 2 * 16 + 6: return curved_dn<2, 6>(ec, fp32, a, met, s);
    case 2 * 16 + 7: return curved_dn<2, 7>(ec, fp32, a, met, s);
    case 3 * 16 + 1: return curved_dn<3, 1>(ec, fp32, a, met, s);
    case 3 * 16 + 2: return curved_dn<3, 2>(ec, fp32, a, met, s);
    case 3 * 16 + 3: return curved_dn<3, 3>(ec, fp32, a, met, s);
    case 3 * 16 + 4: return curved_dn<3, 4>(ec, fp32, a, met, s);
    case 3 * 16 + 5: return curved_dn<3, 5>(ec, fp32, a, met, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dg
