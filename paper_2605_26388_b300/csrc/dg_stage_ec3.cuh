// dg_stage_ec3.cuh -- the fused stage kernel of the 3D two-point (entropy-conservative) form
// for elements of 64 or more nodes (N = 3, 4, 5): one element per iteration of a persistent
// CTA, walked in runs of consecutive elements along x.
//
// Same operator as EulerStage (Sec. 3.1.1, Eq. vol_split with Ranocha's flux of App. A,
// Eq. surf_int, the Shu-Osher update of App. B), organised for the hot 3D case:
//   * each CTA walks runs of up to KRUN consecutive elements along x; the x-face between two
//     consecutive elements of a run is evaluated once -- by the first element as its x+ face
//     -- and carried in shared memory to the second as its x- face, so a run of KRUN elements
//     evaluates 5 + 1/KRUN faces per element instead of 6, and every thread holds one node
//     and one face job (no face-only warp);
//   * the runs are dealt to the CTAs cyclically in the element order, so that the elements
//     in flight stay within a band of the mesh and most neighbours' face traces are served
//     by L2;
//   * the element's FP64 state and the five neighbour traces it needs are copied into shared
//     memory with cp.async one iteration ahead (two buffers); U^n is read in the update only,
//     straight from global memory (one coalesced 8-byte load per variable, issued before the
//     gathers of the partners' pairs and the face terms, which cover its latency), after a
//     prefetch to L2 at the start of the element's flux phase;
//   * per node two 16-byte records of the two-point flux and the FP32 total energy; a face
//     job rebuilds its own trace from them (momentum as rho v on both sides of the face, so
//     the two elements of a face still feed identical bits to the single Riemann-flux call
//     site), and stores F* as one 16-byte record plus the energy component.
#pragma once

#include "dg_stage.cuh"

namespace dg {

// SPEC = 1, 2: the specialisations for the plain SSP-RK3 stage on periodic meshes with the
// HLLC surface flux (no domain faces, no dispatch on the surface flux, no RK54 running sum,
// positivity floor or shock flag), whose face job and update have no branch on those; SPEC 1
// for the stages that read U^n (2 and 3), SPEC 2 for the first, which does not -- the U^n
// loads and prefetch become unconditional or absent
template <int N, class R, int SPEC = 0>
struct EC3 {
  using G = Geo<3, N>;
  static constexpr int NV = 5, NP = G::NP, N1 = G::N1, NFN = G::NFN;
  static constexpr int NF = 6;
  static constexpr int KRUN = 32;                // consecutive elements along x per run
  static constexpr int NJ = 5 * NFN;             // standard face jobs: x+, y-, y+, z-, z+
  static constexpr int T = ((cmax(NP, NJ) + 31) / 32) * 32;
  static constexpr int NO = N1 / 2;              // pair offsets per direction (cyclic ownership)
  // FP64 staging, two buffers of: U [NV][NP], traces of faces 1..5 [5][NV][NFN]
  static constexpr int ST_T = NV * NP;
  static constexpr int ST_XM = ST_T + 5 * NV * NFN;  // x- trace [NV][NFN] (first element of a run)
  static constexpr int ST_SIZE = ST_XM + NV * NFN;
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
  // The CTAs per SM that the shared memory allows (228 KB per SM, 1 KB reserved per CTA),
  // the register budget the compiler is held to; FP64 (bound by the FP64 pipe) at most 3
  static constexpr int MINB =
      cmax(1, cmin(sizeof(R) == 4 ? 8 : 3, (int)(233472 / (smem_bytes() + 1024))));

  struct Role {
    int nd, pos[3];           // node
    int face, f, ndo, ndn;    // standard face job (face 1..5)
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
    const int fm = t < NFN ? t : 0;
    r.ndo_m = line_node<0>(fm, 0);
    r.ndn_m = line_node<0>(fm, N);
    return r;
  }

  // Runs: the rows of elements along x (rows in element order) split into runs of KRUN
  // elements, except the last rows -- about one run of KRUN per CTA -- which split into runs
  // of KTAIL, so that the CTAs, taking the runs in order, finish within a few elements of one
  // another.  Run q starts at element *e0 and holds *len elements; false past the last run.
  static constexpr int KTAIL = 4;
  static __device__ __forceinline__ bool run_of(const InstArgs& I, int q, int* e0, int* len, int* x0out,
                                                int* rowout) {
    const int nx = I.nel[0], nrows = I.nel[1] * I.nel[2];
    const int tail = ((int)gridDim.x * KRUN + nx - 1) / nx;
    const int ra = tail < nrows ? nrows - tail : 0;  // rows in runs of KRUN
    const int nsa = (nx + KRUN - 1) / KRUN, nsb = (nx + KTAIL - 1) / KTAIL;
    int row, x0, k;
    if (q < ra * nsa) {
      row = q / nsa;
      x0 = (q - row * nsa) * KRUN;
      k = KRUN;
    } else {
      const int qb = q - ra * nsa;
      const int rb = qb / nsb;
      row = ra + rb;
      if (row >= nrows) return false;
      x0 = (qb - rb * nsb) * KTAIL;
      k = KTAIL;
    }
    *e0 = x0 + nx * row;
    *len = min(k, nx - x0);
    *x0out = x0;
    *rowout = row;
    return true;
  }

  // A CTA's walk: its first run is run blockIdx.x; each further run is claimed from the
  // launch-wide counter A.work[0] (claim k gives run gridDim.x + k), so that the runs are
  // still taken up roughly in element order -- the elements in flight stay within a band of
  // the mesh, as with a cyclic deal -- and no CTA ends with a run more than another (without
  // a counter, runs blockIdx.x + k gridDim.x).  Position m within the run.
  // (with the x index x0 of the run's first element and the row's y and z indices, for the
  // neighbour table without divisions per element)
  struct Walk {
    int run, m, e0, len, x0, y, z;
    bool ok;
    __device__ __forceinline__ int elem() const { return ok ? e0 + m : -1; }
  };
  static __device__ __forceinline__ bool locate(const InstArgs& I, Walk& w) {
    int row = 0;
    if (!run_of(I, w.run, &w.e0, &w.len, &w.x0, &row)) return false;
    w.y = row % I.nel[1];
    w.z = row / I.nel[1];
    return true;
  }
  static __device__ __forceinline__ Walk walk_start(const InstArgs& I) {
    Walk w;
    w.run = blockIdx.x;
    w.m = 0;
    w.ok = locate(I, w);
    return w;
  }
  // the next element; at the end of a run the walk moves to run `next` (the run claimed
  // ahead) and sets *used
  static __device__ __forceinline__ Walk walk_next(const InstArgs& I, Walk w, int next, bool* used) {
    if (!w.ok) return w;
    if (w.m + 1 < w.len) {
      ++w.m;
      return w;
    }
    w.run = next;
    *used = true;
    w.m = 0;
    w.ok = locate(I, w);
    return w;
  }
  // a run index for the walk to take after `run`: claimed from the counter, or the cyclic deal
  static __device__ __forceinline__ int claim(const StageArgs& A, int run) {
    return A.work ? (int)(atomicAdd(A.work, 1u) + gridDim.x) : run + (int)gridDim.x;
  }

  // start the copies of element e's inputs into staging buffer S: its own state (issue_own),
  // the five neighbour traces of its face jobs (issue_traces; each thread copies the trace
  // values of its own face job)
  static __device__ __forceinline__ void issue_own(const StageArgs& A, const InstArgs& I, int e, double* S) {
    const int t = threadIdx.x;
    if (t < NP) {
      const double* pu = A.U + I.base + (long long)e * NP + t;
#pragma unroll
      for (int v = 0; v < NV; ++v) cp_async8(S + v * NP + t, pu + v * A.stride);
    }
  }
  static __device__ __forceinline__ void issue_traces(const StageArgs& A, const InstArgs& I, const Role& r,
                                                      double* S, const int* nb, bool first) {
    const int t = threadIdx.x;
    if (t < NJ) {
      const double* pt = A.U + I.base + (long long)nb[r.face] * NP + r.ndn;
      double* st = S + ST_T + (r.face - 1) * NV * NFN + r.f;
#pragma unroll
      for (int v = 0; v < NV; ++v) cp_async8(st + v * NFN, pt + v * A.stride);
    }
    if (first && t < NFN) {  // the first element of a run evaluates its x- face too
      const double* pt = A.U + I.base + (long long)nb[0] * NP + r.ndn_m;
#pragma unroll
      for (int v = 0; v < NV; ++v) cp_async8(S + ST_XM + v * NFN + t, pt + v * A.stride);
    }
  }

  // L2 prefetch of the lines that the copies of element e will read one or two iterations later: its
  // own state (NV x NP doubles, 128-byte lines) and, once its neighbour table nb is visible,
  // the face traces (one line per face node and variable; repeats hit the same line)
  static __device__ __forceinline__ void prefetch_own(const StageArgs& A, const InstArgs& I, int e) {
    constexpr int LPV = (NP * 8 + 127) / 128 + 1;  // lines per variable (unaligned start)
    const int t = threadIdx.x;
    if (t < NV * LPV) {
      const int v = t / LPV, q = t - v * LPV;
      const char* p0 = reinterpret_cast<const char*>(A.U + I.base + (long long)e * NP + v * A.stride);
      const char* p = p0 + 128 * q;
      const char* last = p0 + (NP * 8 - 1);
      asm volatile("prefetch.global.L2 [%0];" ::"l"(p < last ? p : last));
    }
  }
  static __device__ __forceinline__ void prefetch_traces(const StageArgs& A, const InstArgs& I, const Role& r,
                                                         const int* nb) {
    const int t = threadIdx.x;
    if (t < NJ && r.face >= 2) {
      const double* pt = A.U + I.base + (long long)nb[r.face] * NP + r.ndn;
#pragma unroll
      for (int v = 0; v < NV; ++v) asm volatile("prefetch.global.L2 [%0];" ::"l"(pt + v * A.stride));
    }
  }

  // neighbour table of the walk's element (periodic wrap), from its indices
  static __device__ __forceinline__ void fill_nb(const InstArgs& I, const Walk& w, int* nb) {
    const int t = threadIdx.x;
    if (t < NF) {
      const int nx = I.nel[0], ny = I.nel[1], nz = I.nel[2], e = w.e0 + w.m, x = w.x0 + w.m;
      const int sxy = nx * ny;
      int n;
      switch (t) {
        case 0: n = x > 0 ? e - 1 : e + (nx - 1); break;
        case 1: n = x < nx - 1 ? e + 1 : e - (nx - 1); break;
        case 2: n = w.y > 0 ? e - nx : e + nx * (ny - 1); break;
        case 3: n = w.y < ny - 1 ? e + nx : e - nx * (ny - 1); break;
        case 4: n = w.z > 0 ? e - sxy : e + sxy * (nz - 1); break;
        default: n = w.z < nz - 1 ? e + sxy : e - sxy * (nz - 1); break;
      }
      nb[t] = n;
    }
  }

  // ---- two-point pairs (cyclic ownership, as EulerStage) ----
  static __device__ __forceinline__ const Q4<R>* rec(const R* sm) {
    return reinterpret_cast<const Q4<R>*>(sm + OFF_Q);
  }
  static __device__ __forceinline__ R* xslot(R* sm, int L, int o) { return sm + OFF_X + (L * NO + o - 1) * XSLOT; }
  static __device__ __forceinline__ const R* xslot(const R* sm, int L, int o) {
    return sm + OFF_X + (L * NO + o - 1) * XSLOT;
  }

  // the NO coefficients of one (direction, position) row of a table, as one vector load when
  // NO = 2 (the row starts at an even index)
  static __device__ __forceinline__ void coefs(const R* C, R* c) {
    if constexpr (NO == 2) {
      if constexpr (sizeof(R) == 4) {
        const float2 v = *reinterpret_cast<const float2*>(C);
        c[0] = v.x;
        c[1] = v.y;
      } else {
        const double2 v = *reinterpret_cast<const double2*>(C);
        c[0] = v.x;
        c[1] = v.y;
      }
    } else {
#pragma unroll
      for (int o = 0; o < NO; ++o) c[o] = C[o];
    }
  }

  template <int L>
  static __device__ __forceinline__ void own_pairs(R* sm, const Role& r, const Q4<R>& ai, const Q4<R>& bi,
                                                   R igm1, R p_ref, R* acc) {
    constexpr int S = G::stride(L);
    const int nd = r.nd, i = r.pos[L];
    R c[NO];
    coefs(sm + OFF_D + (L * N1 + i) * NO, c);
    const Q4<R>* Q = rec(sm);
#pragma unroll
    for (int o = 1; o <= NO; ++o) {
      if (2 * o == N1 && i >= N1 / 2) break;
      const int nj = (i + o < N1) ? nd + o * S : nd + (o - N1) * S;
      const Q4<R> aj = Q[nj], bj = Q[NP + nj];
      R F[NV];
      ec_flux_rec<3, L>(ai, bi, aj, bj, igm1, p_ref, F);
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] -= c[o - 1] * F[v];
      R* X = xslot(sm, L, o);
      reinterpret_cast<Q4<R>*>(X)[nd] = Q4<R>{F[0], F[1], F[2], F[3]};
      X[4 * NP + nd] = F[4];
    }
  }

  // N = 4, FP32: all six pairs of a node (two per direction) with one warp vote for the log
  // means' quotient form, so that their six evaluations interleave in one basic block; the
  // same operations, and the same order of the accumulation, as own_pairs<0..2>
  static __device__ __forceinline__ void own_pairs_all(R* sm, const Role& r, const Q4<R>& ai, const Q4<R>& bi,
                                                       R igm1, R p_ref, R* acc) {
    const int nd = r.nd;
    const Q4<R>* Q = rec(sm);
    EcMeans m[3][2];
    int nj[3][2];
    bool lg = false;
#pragma unroll
    for (int L = 0; L < 3; ++L) {
      const int S = L == 0 ? 1 : (L == 1 ? N1 : N1 * N1);
      const int i = r.pos[L];
#pragma unroll
      for (int o = 1; o <= 2; ++o) {
        nj[L][o - 1] = (i + o < N1) ? nd + o * S : nd + (o - N1) * S;
        m[L][o - 1] = ec_log_means(ai, Q[nj[L][o - 1]]);
        lg = lg || m[L][o - 1].lg;
      }
    }
    if (__any_sync(__activemask(), lg)) {
#pragma unroll
      for (int L = 0; L < 3; ++L)
#pragma unroll
        for (int o = 1; o <= 2; ++o) ec_log_means_fix(ai, Q[nj[L][o - 1]], m[L][o - 1]);
    }
#pragma unroll
    for (int L = 0; L < 3; ++L) {
      R c[NO];
      coefs(sm + OFF_D + (L * N1 + r.pos[L]) * NO, c);
#pragma unroll
      for (int o = 1; o <= 2; ++o) {
        R F[NV];
        const Q4<R> bj = Q[NP + nj[L][o - 1]];
        if (L == 0) ec_flux_assemble<3, 0>(bi, bj, m[L][o - 1], igm1, p_ref, F);
        else if (L == 1) ec_flux_assemble<3, 1>(bi, bj, m[L][o - 1], igm1, p_ref, F);
        else ec_flux_assemble<3, 2>(bi, bj, m[L][o - 1], igm1, p_ref, F);
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] -= c[o - 1] * F[v];
        R* X = xslot(sm, L, o);
        reinterpret_cast<Q4<R>*>(X)[nd] = Q4<R>{F[0], F[1], F[2], F[3]};
        X[4 * NP + nd] = F[4];
      }
    }
  }

  template <int L>
  static __device__ __forceinline__ void partner_pairs(const R* sm, const Role& r, R* acc) {
    constexpr int S = G::stride(L);
    const int nd = r.nd, i = r.pos[L];
    R cc[NO];
    coefs(sm + OFF_D + 3 * N1 * NO + (L * N1 + i) * NO, cc);
#pragma unroll
    for (int o = 1; o <= NO; ++o) {
      if (2 * o == N1 && (i >= o ? i - o : i - o + N1) >= N1 / 2) continue;
      const int nk = (i >= o) ? nd - o * S : nd + (N1 - o) * S;
      const R c = cc[o - 1];
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
                                                   int side, int ndo, const double* n64, int slot, int f) {
    const ScalarsT<R>& k = sc<R>(A);
    const R gamma = k.gamma, igm1 = k.igm1, p_ref = k.p_ref;
    const Q4<R>* Q = rec(sm);
    const Q4<R> Ao = Q[ndo], Bo = Q[NP + ndo];  // (rho, ...), (v_1, v_2, v_3, pd)
    R own[NV];
    Prim<3, R> po;
    po.rho = Ao.x;
    po.irho = Ar<R>::rcp(po.rho);
    po.v[0] = l == 0 ? Bo.x : (l == 1 ? Bo.y : Bo.z);
    po.v[1] = l == 0 ? Bo.y : (l == 1 ? Bo.z : Bo.x);
    po.v[2] = l == 0 ? Bo.z : (l == 1 ? Bo.x : Bo.y);
    po.pd = Bo.w;
    po.p = po.pd + p_ref;
    own[0] = po.rho;
    trace_momentum<3>(po, own);
    own[4] = sm[OFF_E + ndo];
    R Fs[NV];
    int fb = -1;
    if constexpr (SPEC == 0) fb = I.nonper ? boundary_face(I, 3, e, l, side) : -1;
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
      if constexpr (SPEC >= 1) hllc<3, 0>(uL, a, uR, b, gamma, Fs);  // the single call site
      else surface_flux<3, 0>(A.surface, uL, a, uR, b, gamma, igm1, p_ref, Fs);
    }
    const R lf = (side ? R(-1) : R(1)) * sv<R>(I, l) * liftv<R>(I);
    // back to Cartesian components: face axis k is Cartesian direction (l + k) mod 3
    const R fx = l == 0 ? Fs[1] : (l == 1 ? Fs[3] : Fs[2]);
    const R fy = l == 0 ? Fs[2] : (l == 1 ? Fs[1] : Fs[3]);
    const R fz = l == 0 ? Fs[3] : (l == 1 ? Fs[2] : Fs[1]);
    reinterpret_cast<Q4<R>*>(sm + OFF_SQ)[slot * NFN + f] = Q4<R>{lf * Fs[0], lf * fx, lf * fy, lf * fz};
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

  // FP64 value of a flux-precision result that the caller checks for finiteness
  static __device__ __forceinline__ double wide(R x) {
    if constexpr (sizeof(R) == 4) return f2d_fin(x);
    else return x;
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
  // S: this element's staging buffer (copies complete)
  // ---- phase 1 (node threads): convert the staged state S, pressure deviation, records ----
  static __device__ __forceinline__ void phase1(const StageArgs& A, R* sm, const Role& r, const double* S) {
    const int nd = r.nd;
    const ScalarsT<R>& k = sc<R>(A);
    const R p_ref = k.p_ref;
    {
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
  }

  // ---- phases 2 and 3: own pairs into acc, face jobs (xp: this element's x+ face slot) ----
  static __device__ __forceinline__ void phase23(const StageArgs& A, const InstArgs& I, R* sm, const Role& r,
                                                 int e, const double* S, bool carry, int xp, bool need_un, R* acc) {
    const int t = threadIdx.x, nd = r.nd;
    const ScalarsT<R>& k = sc<R>(A);
    const R igm1 = k.igm1, p_ref = k.p_ref;
    const bool node = t < NP;
    if (need_un && node) {  // U^n, read by the update, towards L2 while the fluxes are computed
      const double* pn = A.Un + I.base + (long long)e * NP + nd;
#pragma unroll
      for (int v = 0; v < NV; ++v) asm volatile("prefetch.global.L2 [%0];" ::"l"(pn + v * A.stride));
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = R(0);
    // a thread with both roles runs them in one block, so that the compiler can interleave
    // the pair fluxes with the face flux
    auto pairs = [&]() {
      const Q4<R>* Q = rec(sm);
      const Q4<R> ai = Q[nd], bi = Q[NP + nd];
      if constexpr (sizeof(R) == 4 && N1 == 5) {
        own_pairs_all(sm, r, ai, bi, igm1, p_ref, acc);
      } else {
        own_pairs<0>(sm, r, ai, bi, igm1, p_ref, acc);
        own_pairs<1>(sm, r, ai, bi, igm1, p_ref, acc);
        own_pairs<2>(sm, r, ai, bi, igm1, p_ref, acc);
      }
    };
    auto face = [&]() {
      const double* tr = S + ST_T + (r.face - 1) * NV * NFN + r.f;
      double n64[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) n64[v] = tr[v * NFN];
      const int slot = r.face == 1 ? xp : r.face;
      face_flux(sm, A, I, e, r.face >> 1, r.face & 1, r.ndo, n64, slot, r.f);
    };
    constexpr int NB = NP < NJ ? NP : NJ;
    if (t < NB) {
      if constexpr (SPEC >= 1) {  // a branch-free face job first: it shares a basic block with
        face();                   // the pairs' log means, so their evaluations interleave
        pairs();
      } else {
        pairs();
        face();
      }
    } else {
      if (node) pairs();
      if (t < NJ) face();
    }
    if (!carry && t < NFN) {  // the x- face (start of a run): its own job, trace staged by
                              // this thread
      double n64[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) n64[v] = S[ST_XM + v * NFN + t];
      face_flux(sm, A, I, e, 0, 0, r.ndo_m, n64, 0, t);
    }
  }

  // ---- phase 4 (node threads): partners' pairs, lifted faces, update of element e ----
  static __device__ __forceinline__ void phase4(const StageArgs& A, const InstArgs& I, const R* sm, const Role& r,
                                                int e, const double* S, bool carry, int xp, bool need_un,
                                                R* acc) {
    const int nd = r.nd;
    const ScalarsT<R>& k = sc<R>(A);
    const long long gi = I.base + (long long)e * NP + nd;
    double un[NV];
    if (need_un) {
#pragma unroll
      for (int v = 0; v < NV; ++v) un[v] = __ldg(A.Un + v * A.stride + gi);
    }
    partner_pairs<0>(sm, r, acc);
    partner_pairs<1>(sm, r, acc);
    partner_pairs<2>(sm, r, acc);
    // lifted face terms: one conditional gather per direction (a node lies on at most one of
    // the two faces of a direction)
    const int i = r.pos[0], j = r.pos[1], kk = r.pos[2];
    if (i == 0 || i == N) {
      const bool lo = i == 0;
      gather_slot<0>(sm, lo ? (carry ? (xp == 1 ? NF : 1) : 0) : xp, j + N1 * kk, lo && carry ? R(-1) : R(1), acc);
    }
    if (j == 0 || j == N) gather_slot<1>(sm, j == 0 ? 2 : 3, i + N1 * kk, R(1), acc);
    if (kk == 0 || kk == N) gather_slot<2>(sm, kk == 0 ? 4 : 5, i + N1 * j, R(1), acc);

    // non-finite results are detected on the FP32 residual (a NaN or infinity anywhere in the
    // node's fluxes reaches it), so that the widenings below need no special cases
    bool finite = true;
    if constexpr (sizeof(R) == 4) {
#pragma unroll
      for (int v = 0; v < NV; ++v) finite = finite && fabsf(acc[v]) < INFINITY;
    }
    double res[NV];
    if constexpr (SPEC >= 1) {  // a plain stage update (no RK54 sum, floor or shock flag)
      const R cbdt = k.cbdt;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        double x = fma(A.cb, S[v * NP + nd], wide(cbdt * acc[v]));
        if (need_un) x = fma(A.ca, un[v], x);
        res[v] = x;
      }
    } else {
      if (A.mode == 1 && A.alpha && A.alpha[e] > 0.0) {  // shock-flagged: the DG residual only
#pragma unroll
        for (int v = 0; v < NV; ++v) A.ldg[v * A.stride + gi] = Ar<R>::widen(acc[v]);
        return;
      }
      if (A.mode == 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) res[v] = wide(acc[v]);
      } else {
        const R cbdt = k.cbdt;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          double x = fma(A.cb, S[v * NP + nd], wide(cbdt * acc[v]));
          if (need_un) x = fma(A.ca, un[v], x);
          res[v] = x;
        }
        if (A.acc) {
          const R abdt = k.abdt;
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            double y = fma(A.acc_b, S[v * NP + nd], wide(abdt * acc[v]));
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
#pragma unroll
          for (int v = 0; v < NV; ++v) finite = finite && finite64(res[v]);
        }
      }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      if constexpr (sizeof(R) == 8) finite = finite && finite64(res[v]);
      A.out[v * A.stride + gi] = res[v];
    }
    if (!finite) atomicOr(A.err, 1u);
  }

  // Persistent walk, two barriers per element.  Iteration it handles element e (the walk's
  // it-th): with e's inputs in buffer it & 1 and its records already built, it requests the
  // next element's inputs into the other buffer, runs e's pairs and face jobs, and after a
  // barrier runs e's update together with the next element's records (the update reads the
  // pair and face slots and e's buffer, the records phase writes the records from the other
  // buffer: nothing is shared), then a second barrier.  Each thread reads only the staged
  // values it copied itself, so its own cp.async waits suffice: for the next element's state
  // before the records phase, for its neighbour traces at the start of the next iteration
  // (a whole iteration after they were requested).  The
  // x+ face slot alternates between 1 and 6, so that the next element of the run reads the
  // carried face while this one's slots are rewritten.
  static __device__ void run(const StageArgs& A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* st = reinterpret_cast<double*>(smem_raw);
    R* sm = reinterpret_cast<R*>(st + 2 * ST_SIZE);
    int* nb = reinterpret_cast<int*>(sm + R_SIZE);
    const InstArgs& I = A.inst;
    const Role r = role();
    const bool node = threadIdx.x < NP;
    load_ops(sm, A.Dv, I);
    const bool need_un = SPEC == 0 ? A.need_un != 0 : SPEC == 1;
    __shared__ int s_next;  // the run claimed ahead (thread 0 writes it, after a barrier)
    const int t = threadIdx.x;
    Walk w = walk_start(I);
    if (t == 0) s_next = claim(A, w.run);
    __syncthreads();
    bool used = false;
    Walk wn = walk_next(I, w, s_next, &used);
    if (used) {  // a run of one element
      const int last = wn.run;
      __syncthreads();
      if (t == 0) s_next = claim(A, last);
      __syncthreads();
      used = false;
    }
    Walk wnn = walk_next(I, wn, s_next, &used);
    if (w.ok) fill_nb(I, w, nb);
    if (wn.ok) fill_nb(I, wn, nb + NF);
    __syncthreads();
    if (w.ok) {
      issue_own(A, I, w.elem(), st);
      issue_traces(A, I, r, st, nb, true);
    }
    cp_async_commit();
    cp_async_wait_all();
    if (w.ok && node) phase1(A, sm, r, st);
    __syncthreads();
    for (int it = 0; w.ok; ++it) {
      const int b = it & 1;
      cp_async_wait_all();  // this thread's copies of e's neighbour traces (requested an iteration ago)
      // buffer b^1 and neighbour slot b are free: their element's update and copies are done.
      // The next element's own state and its traces form two groups: the records phase below
      // waits for the first only, the traces have until the next iteration's face jobs.
      if (wn.ok) issue_own(A, I, wn.elem(), st + (b ^ 1) * ST_SIZE);
      cp_async_commit();
      if (wn.ok) issue_traces(A, I, r, st + (b ^ 1) * ST_SIZE, nb + (b ^ 1) * NF, wn.m == 0);
      cp_async_commit();
      if (wnn.ok) {
        fill_nb(I, wnn, nb + b * NF);  // read by the next iteration's issue
        // the own state three elements ahead when it lies in the same run (the walk does not
        // know the run after the claimed one); an element that starts a run gets it two ahead
        if (wnn.m == 0) prefetch_own(A, I, wnn.elem());
        if (wnn.m + 1 < wnn.len) prefetch_own(A, I, wnn.elem() + 1);
      }
      // the x- face is carried from the previous iteration, which handled element e - 1 of
      // the same run
      const int e = w.elem(), xp = b ? NF : 1;
      const bool carry = w.m != 0;
      R acc[NV];
      phase23(A, I, sm, r, e, st + b * ST_SIZE, carry, xp, need_un, acc);
      __syncthreads();  // pair and face slots complete; the records are free
      cp_async_wait_prev();  // this thread's copies of the next element's own state
      if (wnn.ok) prefetch_traces(A, I, r, nb + b * NF);  // the table is visible since the barrier
      if (used) {  // every thread has read s_next since the walk last took it: claim the next
        if (t == 0) s_next = claim(A, wnn.run);
        used = false;
      }
      if (node) {
        phase4(A, I, sm, r, e, st + b * ST_SIZE, carry, xp, need_un, acc);
        if (wn.ok) phase1(A, sm, r, st + (b ^ 1) * ST_SIZE);
      }
      __syncthreads();  // the next element's records complete; the slots and buffer b are free
      w = wn;
      wn = wnn;
      wnn = walk_next(I, wnn, s_next, &used);
    }
    // the last CTA to finish returns the counters to zero for the next launch (no CTA claims
    // after it has finished)
    if (A.work && t == 0) {
      __threadfence();
      if (atomicAdd(A.work + 1, 1u) == gridDim.x - 1) {
        A.work[0] = 0u;
        A.work[1] = 0u;
      }
    }
  }
};

template <int N, class R, int SPEC>
__global__ void __launch_bounds__(EC3<N, R, SPEC>::T, EC3<N, R, SPEC>::MINB) k_euler_ec3(const StageArgs A) {
  EC3<N, R, SPEC>::run(A);
}

}  // namespace dg
