// dg_stage_ec3.cuh -- the fused stage kernel of the 3D two-point (entropy-conservative) form
// for elements of 64 or more nodes (N = 3, 4, 5): one element per iteration of a persistent
// CTA, walked in runs of consecutive elements along x.
//
// Same operator as EulerStage (Sec. 3.1.1, Eq. vol_split with Ranocha's flux of App. A,
// Eq. surf_int, the Shu-Osher update of App. B), organised for the hot 3D case:
//   * each CTA walks runs of KRUN consecutive elements along x; the x-face between two
//     consecutive elements of a run is evaluated once -- by the first element as its x+ face
//     -- and carried in shared memory to the second as its x- face, so a run of KRUN elements
//     evaluates 5 + 1/KRUN faces per element instead of 6, and every thread holds one node
//     and one face job (no face-only warp).  The runs are dealt to the CTAs cyclically, so
//     the elements in flight at any time stay within a band of the mesh and the neighbours'
//     face traces are served by L2;
//   * the element's FP64 state and the five neighbour traces it needs are double-buffered
//     in shared memory with cp.async; U^n is read in the update only, straight from global
//     memory (one coalesced 8-byte load per variable);
//   * per node two 16-byte records of the two-point flux and the FP32 total energy; a face
//     job rebuilds its own trace from them (momentum as rho v on both sides of the face, so
//     the two elements of a face still feed identical bits to the single Riemann-flux call
//     site), and stores F* as one 16-byte record plus the energy component.
#pragma once

#include "dg_stage.cuh"

namespace dg {

template <int N, class R>
struct EC3 {
  using G = Geo<3, N>;
  static constexpr int NV = 5, NP = G::NP, N1 = G::N1, NFN = G::NFN;
  static constexpr int NF = 6;
  static constexpr int KRUN = 8;                 // consecutive elements along x per run
  static constexpr int NJ = 5 * NFN;             // standard face jobs: x+, y-, y+, z-, z+
  static constexpr int T = ((cmax(NP, NJ) + 31) / 32) * 32;
  static constexpr int NO = N1 / 2;              // pair offsets per direction (cyclic ownership)
  // FP64 staging (two buffers): U [NV][NP], traces of faces 1..5 [5][NV][NFN]
  static constexpr int ST_T = NV * NP;
  static constexpr int ST_SIZE = ST_T + 5 * NV * NFN;
  // flux-precision arrays
  static constexpr int XSLOT = 4 * NP + al4(NP);           // pair slot: Q4 [NP] then F_4 [NP]
  static constexpr int NS = NF + 1;                        // face slots (x+ alternates 1 / 6)
  static constexpr int OFF_Q = 0;                          // records [2][NP] Q4
  static constexpr int OFF_E = OFF_Q + 8 * NP;             // E [NP]
  static constexpr int OFF_SQ = al4(OFF_E + NP);           // face results [NS][NFN] Q4 ...
  static constexpr int OFF_SE = OFF_SQ + 4 * NS * NFN;     //   ... and their energy [NS][NFN]
  static constexpr int OFF_X = al4(OFF_SE + NS * NFN);     // pair slots [3][NO]
  static constexpr int OFF_D = OFF_X + 3 * NO * XSLOT;     // own [3][N1][NO], partner [3][N1][NO]
  static constexpr int R_SIZE = OFF_D + 2 * 3 * N1 * NO;
  static constexpr size_t smem_bytes() {
    return sizeof(double) * 2 * (size_t)ST_SIZE + sizeof(R) * (size_t)R_SIZE + sizeof(int) * 2 * NF;
  }
  // FP32: the CTAs per SM that the shared memory allows (228 KB per SM, 1 KB reserved per
  // CTA), the register budget the compiler is held to; FP64 (bound by the FP64 pipe): free
  static constexpr int MINB =
      sizeof(R) == 4 ? cmax(1, cmin(8, (int)(233472 / (smem_bytes() + 1024)))) : 1;

  struct Role {
    int nd, pos[3];           // node
    int face, f, ndo, ndn;    // standard face job (face 1..5)
    int pm[3];                // face axes -> Cartesian momentum index (1..3)
    int ndo_m, ndn_m;         // x- face job (thread < NFN): own node (i = 0), neighbour node (i = N)
  };

  template <int L>
  static __device__ __forceinline__ int line_node(int q, int m) {
    constexpr int S = G::stride(L);
    return (q % S) + m * S + (q / S) * S * N1;
  }

  static __device__ __forceinline__ Role role() {
    Role r;
    const int t = threadIdx.x;
    r.nd = t;
    r.pos[0] = t % N1;
    r.pos[1] = (t / N1) % N1;
    r.pos[2] = t / (N1 * N1);
    const int tj = t < NJ ? t : 0;
    r.face = 1 + tj / NFN;
    r.f = tj - (r.face - 1) * NFN;
    const int l = r.face >> 1, side = r.face & 1;
    if (l == 0) { r.ndn = line_node<0>(r.f, side ? 0 : N); r.ndo = line_node<0>(r.f, side ? N : 0); }
    else if (l == 1) { r.ndn = line_node<1>(r.f, side ? 0 : N); r.ndo = line_node<1>(r.f, side ? N : 0); }
    else { r.ndn = line_node<2>(r.f, side ? 0 : N); r.ndo = line_node<2>(r.f, side ? N : 0); }
#pragma unroll
    for (int k = 0; k < 3; ++k) r.pm[k] = 1 + (l + k) % 3;
    const int fm = t < NFN ? t : 0;
    r.ndo_m = line_node<0>(fm, 0);
    r.ndn_m = line_node<0>(fm, N);
    return r;
  }

  // neighbour element across face `face` of element e (periodic wrap)
  static __device__ __forceinline__ int neighbour(const InstArgs& I, int e, int face) {
    const int l = face >> 1, d = (face & 1) ? 1 : -1;
    int c[3] = {e % I.nel[0], (e / I.nel[0]) % I.nel[1], e / (I.nel[0] * I.nel[1])};
    c[l] += d;
    c[l] = c[l] < 0 ? c[l] + I.nel[l] : (c[l] >= I.nel[l] ? c[l] - I.nel[l] : c[l]);
    return c[0] + I.nel[0] * (c[1] + I.nel[1] * c[2]);
  }

  // group (element) of iteration it of this CTA: runs of KRUN dealt cyclically
  static __device__ __forceinline__ int elem_of(int it) {
    const int q = it / KRUN, m = it - q * KRUN;
    return (blockIdx.x + q * (int)gridDim.x) * KRUN + m;
  }

  static __device__ __forceinline__ void issue(const StageArgs& A, const InstArgs& I, const Role& r,
                                               int e, double* S, const int* nb) {
    const int t = threadIdx.x;
    if (t < NP) {
      const double* pu = A.U + I.base + (long long)e * NP + t;
#pragma unroll
      for (int v = 0; v < NV; ++v) cp_async8(S + v * NP + t, pu + v * A.stride);
    }
    if (t < NJ) {
      const double* pt = A.U + I.base + (long long)nb[r.face] * NP + r.ndn;
      double* st = S + ST_T + (r.face - 1) * NV * NFN + r.f;
#pragma unroll
      for (int v = 0; v < NV; ++v) cp_async8(st + v * NFN, pt + v * A.stride);
    }
  }

  static __device__ __forceinline__ void fill_nb(const InstArgs& I, int e, int* nb) {
    const int t = threadIdx.x;
    if (t < NF) nb[t] = neighbour(I, e, t);
  }

  // ---- two-point pairs (cyclic ownership, as EulerStage) ----
  static __device__ __forceinline__ const Q4<R>* rec(const R* sm) {
    return reinterpret_cast<const Q4<R>*>(sm + OFF_Q);
  }
  static __device__ __forceinline__ R* xslot(R* sm, int L, int o) { return sm + OFF_X + (L * NO + o - 1) * XSLOT; }
  static __device__ __forceinline__ const R* xslot(const R* sm, int L, int o) {
    return sm + OFF_X + (L * NO + o - 1) * XSLOT;
  }

  template <int L>
  static __device__ __forceinline__ void own_pairs(R* sm, const Role& r, const Q4<R>& ai, const Q4<R>& bi,
                                                   R igm1, R p_ref, R* acc) {
    constexpr int S = G::stride(L);
    const int nd = r.nd, i = r.pos[L];
    const R* C = sm + OFF_D + (L * N1 + i) * NO;
    const Q4<R>* Q = rec(sm);
#pragma unroll
    for (int o = 1; o <= NO; ++o) {
      if (2 * o == N1 && i >= N1 / 2) break;
      const int nj = (i + o < N1) ? nd + o * S : nd + (o - N1) * S;
      const Q4<R> aj = Q[nj], bj = Q[NP + nj];
      R F[NV];
      ec_flux_rec<3, L>(ai, bi, aj, bj, igm1, p_ref, F);
      const R c = C[o - 1];
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] -= c * F[v];
      R* X = xslot(sm, L, o);
      reinterpret_cast<Q4<R>*>(X)[nd] = Q4<R>{F[0], F[1], F[2], F[3]};
      X[4 * NP + nd] = F[4];
    }
  }

  template <int L>
  static __device__ __forceinline__ void partner_pairs(const R* sm, const Role& r, R* acc) {
    constexpr int S = G::stride(L);
    const int nd = r.nd, i = r.pos[L];
    const R* C = sm + OFF_D + 3 * N1 * NO + (L * N1 + i) * NO;
#pragma unroll
    for (int o = 1; o <= NO; ++o) {
      if (2 * o == N1 && (i >= o ? i - o : i - o + N1) >= N1 / 2) continue;
      const int nk = (i >= o) ? nd - o * S : nd + (N1 - o) * S;
      const R c = C[o - 1];
      const R* X = xslot(sm, L, o);
      const Q4<R> f = reinterpret_cast<const Q4<R>*>(X)[nk];
      acc[0] -= c * f.x;
      acc[1] -= c * f.y;
      acc[2] -= c * f.z;
      acc[3] -= c * f.w;
      acc[4] -= c * X[4 * NP + nk];
    }
  }

  // ---- face jobs ----
  // F* of face (l, side) at face node f with own node ndo, the neighbour's FP64 trace in n64
  // (Cartesian); lifted by lf and stored to face slot `slot` in Cartesian components.
  static __device__ __forceinline__ void face_flux(R* sm, const StageArgs& A, const InstArgs& I, int e, int l,
                                                   int side, int ndo, const int* pm, const double* n64,
                                                   int slot, int f) {
    const ScalarsT<R>& k = sc<R>(A);
    const R gamma = k.gamma, igm1 = k.igm1, p_ref = k.p_ref;
    const Q4<R>* Q = rec(sm);
    const R* Bo = reinterpret_cast<const R*>(Q + NP + ndo);  // (v_1, v_2, v_3, pd)
    R own[NV];
    Prim<3, R> po;
    po.rho = Q[ndo].x;
    po.irho = Ar<R>::rcp(po.rho);
#pragma unroll
    for (int d = 0; d < 3; ++d) po.v[d] = Bo[pm[d] - 1];
    po.pd = Bo[3];
    po.p = po.pd + p_ref;
    own[0] = po.rho;
    trace_momentum<3>(po, own);
    own[4] = sm[OFF_E + ndo];
    R Fs[NV];
    const int fb = I.nonper ? boundary_face(I, 3, e, l, side) : -1;
    if (fb >= 0) {
      boundary_flux<3, R>(I, fb, l, side, own, po, A.surface, gamma, igm1, p_ref, A.pd.gm1, A.pd.p_ref, k.hgm1, Fs);
    } else {
      R n0[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) n0[v] = Ar<R>::load(n64[v]);
      Prim<3, R> pn;
      pn.rho = n0[0];
      pn.irho = Ar<R>::rcp(n0[0]);
      pn.pd = pdev_i<3>(n64, n0, pn.irho, A.pd.gm1, A.pd.p_ref, k.hgm1);
      pn.p = pn.pd + p_ref;
      R vc[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) vc[d] = n0[1 + d] * pn.irho;
      pn.v[0] = l == 0 ? vc[0] : (l == 1 ? vc[1] : vc[2]);
      pn.v[1] = l == 0 ? vc[1] : (l == 1 ? vc[2] : vc[0]);
      pn.v[2] = l == 0 ? vc[2] : (l == 1 ? vc[0] : vc[1]);
      R nb[NV];
      nb[0] = pn.rho;
      trace_momentum<3>(pn, nb);
      nb[4] = n0[4];
      R uL[NV], uR[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        uL[v] = side ? own[v] : nb[v];
        uR[v] = side ? nb[v] : own[v];
      }
      const Prim<3, R>& a = side ? po : pn;
      const Prim<3, R>& b = side ? pn : po;
      surface_flux<3, 0>(A.surface, uL, a, uR, b, gamma, igm1, p_ref, Fs);  // the single call site
    }
    const R lf = (side ? R(-1) : R(1)) * sv<R>(I, l) * liftv<R>(I);
    R* Sq = sm + OFF_SQ + (slot * NFN + f) * 4;
    Sq[0] = lf * Fs[0];
#pragma unroll
    for (int d = 0; d < 3; ++d) Sq[pm[d]] = lf * Fs[1 + d];
    sm[OFF_SE + slot * NFN + f] = lf * Fs[4];
  }

  template <int L>
  static __device__ __forceinline__ void gather_slot(const R* sm, int slot, int f, R sgn, R* acc) {
    const Q4<R> q = reinterpret_cast<const Q4<R>*>(sm + OFF_SQ)[slot * NFN + f];
    acc[0] += sgn * q.x;
    acc[1] += sgn * q.y;
    acc[2] += sgn * q.z;
    acc[3] += sgn * q.w;
    acc[4] += sgn * sm[OFF_SE + slot * NFN + f];
  }

  static __device__ __forceinline__ void load_ops(R* sm, const double* Dv, const InstArgs& I) {
    for (int q = threadIdx.x; q < 2 * 3 * N1 * NO; q += blockDim.x) {
      const int part = q / (3 * N1 * NO), rem = q - part * (3 * N1 * NO);
      const int L = rem / (N1 * NO), i = (rem / NO) % N1, o = rem % NO + 1;
      const int j = part ? (i - o + N1) % N1 : (i + o) % N1;
      sm[OFF_D + q] = from64<R>(I.s[L] * Dv[i * N1 + j]);
    }
  }

  // ---- one element ----
  // xp: slot of this element's x+ face; xm: slot its x- face is read from (sgn: its sign) --
  // the previous element's x+ slot (carry, sgn -1) or slot 0 (computed here, sgn +1)
  static __device__ __forceinline__ void compute(const StageArgs& A, const InstArgs& I, R* sm, const Role& r,
                                                 int e, const double* S, bool carry, int xp, bool need_un) {
    const int t = threadIdx.x, nd = r.nd;
    const ScalarsT<R>& k = sc<R>(A);
    const R igm1 = k.igm1, p_ref = k.p_ref;
    const bool node = t < NP;
    // phase 1: convert, primitives, records
    if (node) {
      double u64[NV];
      R u[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        u64[v] = S[v * NP + nd];
        u[v] = Ar<R>::load(u64[v]);
      }
      const R irho = Ar<R>::rcp(u[0]);
      const R pd = pdev_i<3>(u64, u, irho, A.pd.gm1, A.pd.p_ref, k.hgm1);
      if (!positive<3>(u64, u, pd, p_ref, k.margin_e, k.margin_0, A.pd.gm1)) atomicOr(A.err, 2u);
      const Prim<3, R> q = prims_i<3>(u, irho, pd, p_ref);
      Q4<R>* Q = reinterpret_cast<Q4<R>*>(sm + OFF_Q);
      ec_records<3>(q, Q[nd], Q[NP + nd]);
      sm[OFF_E + nd] = u[4];
    }
    __syncthreads();
    // phase 2: own pairs; phase 3: face jobs
    R acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = R(0);
    if (node) {
      const Q4<R>* Q = rec(sm);
      const Q4<R> ai = Q[nd], bi = Q[NP + nd];
      own_pairs<0>(sm, r, ai, bi, igm1, p_ref, acc);
      own_pairs<1>(sm, r, ai, bi, igm1, p_ref, acc);
      own_pairs<2>(sm, r, ai, bi, igm1, p_ref, acc);
    }
    if (t < NJ) {
      const double* tr = S + ST_T + (r.face - 1) * NV * NFN + r.f;
      double n64[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) n64[v] = tr[v * NFN];
      const int slot = r.face == 1 ? xp : r.face;
      face_flux(sm, A, I, e, r.face >> 1, r.face & 1, r.ndo, r.pm, n64, slot, r.f);
    }
    if (!carry && t < NFN) {  // the x- face (start of a run or of an x line): its own job
      const double* pt = A.U + I.base + (long long)neighbour(I, e, 0) * NP + r.ndn_m;
      double n64[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) n64[v] = __ldg(pt + v * A.stride);
      const int pm0[3] = {1, 2, 3};
      face_flux(sm, A, I, e, 0, 0, r.ndo_m, pm0, n64, 0, t);
    }
    __syncthreads();
    // phase 4: partners' pairs, lifted faces, update
    if (!node) return;
    const long long gi = I.base + (long long)e * NP + nd;
    double un[NV];
    if (need_un) {
#pragma unroll
      for (int v = 0; v < NV; ++v) un[v] = __ldg(A.Un + v * A.stride + gi);
    }
    partner_pairs<0>(sm, r, acc);
    partner_pairs<1>(sm, r, acc);
    partner_pairs<2>(sm, r, acc);
    const int i = r.pos[0], j = r.pos[1], kk = r.pos[2];
    if (i == 0) gather_slot<0>(sm, carry ? (xp == 1 ? NF : 1) : 0, j + N1 * kk, carry ? R(-1) : R(1), acc);
    if (i == N) gather_slot<0>(sm, xp, j + N1 * kk, R(1), acc);
    if (j == 0) gather_slot<1>(sm, 2, i + N1 * kk, R(1), acc);
    if (j == N) gather_slot<1>(sm, 3, i + N1 * kk, R(1), acc);
    if (kk == 0) gather_slot<2>(sm, 4, i + N1 * j, R(1), acc);
    if (kk == N) gather_slot<2>(sm, 5, i + N1 * j, R(1), acc);

    double res[NV];
    if (A.mode == 1 && A.alpha && A.alpha[e] > 0.0) {  // shock-flagged: the DG residual only
#pragma unroll
      for (int v = 0; v < NV; ++v) A.ldg[v * A.stride + gi] = Ar<R>::widen(acc[v]);
      return;
    }
    if (A.mode == 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) res[v] = Ar<R>::widen(acc[v]);
    } else {
      const R cbdt = k.cbdt;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        double x = fma(A.cb, S[v * NP + nd], Ar<R>::widen(cbdt * acc[v]));
        if (need_un) x = fma(A.ca, un[v], x);
        res[v] = x;
      }
      if (A.acc) {
        const R abdt = k.abdt;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          double y = fma(A.acc_b, S[v * NP + nd], Ar<R>::widen(abdt * acc[v]));
          if (A.acc_a != 0.0) y = fma(A.acc_a, A.acc[v * A.stride + gi], y);
          A.acc[v * A.stride + gi] = y;
        }
      }
      if (A.floor_on) {
        if (A.rho_floor > 0.0 && res[0] < A.rho_floor) res[0] = A.rho_floor;
        double kin = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) kin += res[1 + d] * res[1 + d] / res[0];
        const double p = (A.gamma - 1.0) * (res[4] - 0.5 * kin);
        if (A.p_floor > 0.0 && p < A.p_floor) res[4] = A.p_floor / (A.gamma - 1.0) + 0.5 * kin;
      }
    }
    bool finite = true;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      finite = finite && finite64(res[v]);
      A.out[v * A.stride + gi] = res[v];
    }
    if (!finite) atomicOr(A.err, 1u);
  }

  // Persistent walk: iteration it handles element elem_of(it); its inputs were copied during
  // iteration it-1 into buffer it & 1, with its neighbour table in slot it & 1 (filled two
  // iterations ahead).  The x+ face slot alternates between 1 and 6, so that the next element
  // of the run reads the carried face while this one's slots are rewritten.
  static __device__ void run(const StageArgs& A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* st = reinterpret_cast<double*>(smem_raw);
    R* sm = reinterpret_cast<R*>(st + 2 * ST_SIZE);
    int* nb = reinterpret_cast<int*>(sm + R_SIZE);
    const InstArgs& I = A.inst;
    const Role r = role();
    load_ops(sm, A.Dv, I);
    const bool need_un = A.need_un != 0;
    const int ne = I.n_elem;
    int e = elem_of(0);
    if (e < ne) fill_nb(I, e, nb);
    if (elem_of(1) < ne) fill_nb(I, elem_of(1), nb + NF);
    __syncthreads();
    if (e < ne) issue(A, I, r, e, st, nb);
    cp_async_commit();
    for (int it = 0; e < ne; ++it) {
      const int b = it & 1;
      const int en = elem_of(it + 1), enn = elem_of(it + 2);
      cp_async_wait_all();
      __syncthreads();
      if (en < ne) issue(A, I, r, en, st + (b ^ 1) * ST_SIZE, nb + (b ^ 1) * NF);
      cp_async_commit();
      if (enn < ne) fill_nb(I, enn, nb + b * NF);  // read by the next iteration's issue
      // the x- face is carried when the previous iteration handled element e - 1 of the same
      // x line
      const bool carry = (it % KRUN) != 0 && (e % I.nel[0]) != 0;
      compute(A, I, sm, r, e, st + b * ST_SIZE, carry, b ? NF : 1, need_un);
      e = en;
    }
  }
};

template <int N, class R>
__global__ void __launch_bounds__(EC3<N, R>::T, EC3<N, R>::MINB) k_euler_ec3(const StageArgs A) {
  EC3<N, R>::run(A);
}

}  // namespace dg
