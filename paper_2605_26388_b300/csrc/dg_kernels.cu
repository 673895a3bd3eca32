// dg_kernels.cu -- fused DGSEM residual + SSP-RK3 stage kernels for sm_103a.
//
// One launch evaluates, for every element of a periodic Cartesian instance, the
// semi-discrete Euler residual of Sec. 3.1.1 -- volume term (Eq. vol_weak, or Eq. vol_split
// with Ranocha's two-point flux, App. A Eq. split_form_3D), Riemann fluxes on the element
// faces, surface lifting and Jacobian rescale (Eq. surf_int) -- and applies the Shu-Osher
// stage update of App. B, in place of the paper's five kernels and its surface buffer.
//
// The kernel is persistent: each CTA walks a strided list of element groups (EPB elements
// per group) and double-buffers their inputs in shared memory with cp.async, so the next
// group's FP64 state, U^n and the neighbours' face traces are in flight while the current
// group computes.  Per group (all staging in shared memory):
//   1. one thread per node: convert the staged FP64 state to the flux precision R, evaluate
//      the pressure deviation from the FP64 energy, stage primitives (two-point form) or the
//      DIM point fluxes (strong/weak form);
//   2. two-point form: every pair a<b of every line of every direction is evaluated once
//      (F# is symmetric) into a pair buffer -- no atomics, fixed gather order later;
//   3. one job per face node: F* = F*(U_L, U_R) from the staged own and neighbour traces,
//      evaluated at a single call site for both orientations, so the two elements of a face
//      compute bitwise-identical F* (exact conservation without a shared surface buffer);
//   4. one thread per node: gather volume pairs (or contract the point fluxes), the lifted
//      face terms, and write L or the FP64 stage update.
#include "dg_device.cuh"
#include "dg_internal.h"

namespace dg {

// ---------------------------------------------------------------------------------------
// cp.async (global -> shared, 8-byte granules: legal for any element offset)
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_prev() {  // all but the newest group done
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}

template <int DIM, int L, class R>
__device__ __forceinline__ void surface_flux(int kind, const R* uL, const Prim<DIM, R>& a,
                                             const R* uR, const Prim<DIM, R>& b, R gamma,
                                             R igm1, R p_ref, R* F) {
  switch (kind) {
    case 1: hllc<DIM, L>(uL, a, uR, b, gamma, F); break;
    case 2: hll<DIM, L>(uL, a, uR, b, gamma, F); break;
    case 3: ec_flux<DIM, L>(a, b, igm1, p_ref, F); break;
    default: rusanov<DIM, L>(uL, a, uR, b, gamma, F); break;
  }
}

constexpr int cmax(int a, int b) { return a > b ? a : b; }

// the launch scalars in the flux precision (precomputed on the host)
template <class R>
__device__ __forceinline__ const StageArgs::ScalarsT<R>& sc(const StageArgs& A);
template <>
__device__ __forceinline__ const StageArgs::ScalarsT<double>& sc<double>(const StageArgs& A) {
  return A.pd;
}
template <>
__device__ __forceinline__ const StageArgs::ScalarsT<float>& sc<float>(const StageArgs& A) {
  return A.pf;
}

template <int DIM, int N, bool EC, class R>
struct EulerStage {
  using G = Geo<DIM, N>;
  static constexpr int NV = G::NV, NP = G::NP, N1 = G::N1, EPB = G::EPB, NFN = G::NFN;
  static constexpr int NF = 2 * DIM;                       // faces per element
  static constexpr int NJS = EPB * NF * NFN;               // face jobs per group
  static constexpr int T = ((cmax(EPB * NP, NJS) + 31) / 32) * 32;
  // Two-point pairs are assigned cyclically along each line: node i owns the pairs
  // (i, i+o mod N1) for o = 1..NO, the last offset (o = N1/2 when N1 is even) only for
  // i < N1/2, so that every unordered pair is evaluated exactly once.
  static constexpr int NO = N1 / 2;
  // per-node staged quantities: EC -- rho, v_1..v_DIM, pd, beta = rho/p; strong/weak -- the
  // DIM point fluxes (NV each) and pd
  static constexpr int NQ = EC ? (DIM + 3) : (DIM * NV + 1);
  static constexpr int PD = EC ? (DIM + 1) : (DIM * NV);
  static constexpr int NXN = EC ? DIM * NO : 0;            // pair slots per node
  // FP64 staging buffer (two of them): own U [EPB][NV][NP], U^n [EPB][NV][NP],
  // neighbour face traces [EPB][NF][NV][NFN]
  static constexpr int ST_U = 0, ST_N = EPB * NV * NP, ST_T = 2 * EPB * NV * NP;
  static constexpr int ST_SIZE = ST_T + EPB * NF * NV * NFN;
  // flux-precision arrays
  static constexpr int OFF_U = 0;                             // [EPB][NV][NP]
  static constexpr int OFF_Q = OFF_U + EPB * NV * NP;         // [EPB][NQ][NP]
  static constexpr int OFF_S = OFF_Q + EPB * NQ * NP;         // [EPB][NF][NFN][NV]
  static constexpr int OFF_X = OFF_S + EPB * NF * NFN * NV;   // [EPB][DIM][NO][NV][NP]
  static constexpr int OFF_D = OFF_X + EPB * NXN * NV * NP;   // [N1][N1]
  static constexpr int R_SIZE = OFF_D + N1 * N1;
  static constexpr size_t smem_bytes() {
    return sizeof(double) * 2 * (size_t)ST_SIZE + sizeof(R) * (size_t)R_SIZE +
           sizeof(int) * (size_t)(2 * EPB * NF + 4);
  }

  struct Smem {
    double* st;  // 2 * ST_SIZE
    R* sm;       // R_SIZE
    int* nb;     // [2][EPB * NF] neighbour element of each face
  };

  static __device__ __forceinline__ Smem carve() {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem m;
    m.st = reinterpret_cast<double*>(smem_raw);
    m.sm = reinterpret_cast<R*>(m.st + 2 * ST_SIZE);
    m.nb = reinterpret_cast<int*>(m.sm + R_SIZE);
    return m;
  }

  template <int L>
  static __device__ __forceinline__ int line_node(int q, int m) {
    constexpr int S = G::stride(L);
    return (q % S) + m * S + (q / S) * S * N1;
  }
  template <int L>
  static __device__ __forceinline__ int node_line(int nd) {
    constexpr int S = G::stride(L);
    return (nd % S) + (nd / (S * N1)) * S;
  }
  template <int L>
  static __device__ __forceinline__ int node_pos(int nd) {
    return (nd / G::stride(L)) % N1;
  }

  // neighbour element of face `face` (direction face/2, side face%2) of element e
  static __device__ __forceinline__ int neighbour(const StageArgs& A, int e, int face) {
    const int l = face >> 1;
    int cx = e % A.nel[0];
    int cy = (e / A.nel[0]) % A.nel[1];
    int cz = (DIM == 3) ? e / (A.nel[0] * A.nel[1]) : 0;
    const int d = (face & 1) ? 1 : -1;
    if (l == 0) { cx += d; cx = cx < 0 ? cx + A.nel[0] : (cx >= A.nel[0] ? cx - A.nel[0] : cx); }
    else if (l == 1) { cy += d; cy = cy < 0 ? cy + A.nel[1] : (cy >= A.nel[1] ? cy - A.nel[1] : cy); }
    else { cz += d; cz = cz < 0 ? cz + A.nel[2] : (cz >= A.nel[2] ? cz - A.nel[2] : cz); }
    return cx + A.nel[0] * (cy + A.nel[1] * cz);
  }

  // Per-thread roles, decoded once per launch.
  struct Role {
    int el, nd;             // node role (t < EPB*NP)
    int jel, face, f, ndn;  // face-job role (t < NJS): element, face, face node, neighbour node
    int ndo;                // own node of the face job
  };

  static __device__ __forceinline__ Role role() {
    Role r;
    const int t = threadIdx.x;
    r.el = t / NP;
    r.nd = t - r.el * NP;
    r.jel = t / (NF * NFN);
    const int q = t - r.jel * (NF * NFN);
    r.face = q / NFN;
    r.f = q - r.face * NFN;
    const int l = r.face >> 1, side = r.face & 1;
    if (l == 0) { r.ndn = line_node<0>(r.f, side ? 0 : N); r.ndo = line_node<0>(r.f, side ? N : 0); }
    else if (l == 1) { r.ndn = line_node<1>(r.f, side ? 0 : N); r.ndo = line_node<1>(r.f, side ? N : 0); }
    else { r.ndn = line_node<DIM - 1>(r.f, side ? 0 : N); r.ndo = line_node<DIM - 1>(r.f, side ? N : 0); }
    return r;
  }

  // start the asynchronous copies of group g into staging buffer b
  static __device__ __forceinline__ void issue(const StageArgs& A, const Smem& M, const Role& r,
                                               int g, int b, bool need_un) {
    const int t = threadIdx.x;
    double* S = M.st + b * ST_SIZE;
    const int e = g * EPB + r.el;
    if (t < EPB * NP && e < A.n_elem) {
      const long long o = A.base + (long long)e * NP + r.nd;
      const double* pu = A.U + o;
      const double* pn = A.Un + o;
      double* su = S + ST_U + r.el * NV * NP + r.nd;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        cp_async8(su + v * NP, pu + v * A.stride);
        if (need_un) cp_async8(su + (ST_N - ST_U) + v * NP, pn + v * A.stride);
      }
    }
    const int ej = g * EPB + r.jel;
    if (t < NJS && ej < A.n_elem) {
      const int en = M.nb[b * EPB * NF + r.jel * NF + r.face];
      const double* pt = A.U + A.base + (long long)en * NP + r.ndn;
      double* st = S + ST_T + ((r.jel * NF + r.face) * NV) * NFN + r.f;
#pragma unroll
      for (int v = 0; v < NV; ++v) cp_async8(st + v * NFN, pt + v * A.stride);
    }
  }

  // ---- phase 2 (EC): this node's own pairs in direction L ----
  template <int L>
  static __device__ __forceinline__ void own_pairs(R* sm, const StageArgs& A, int el, int nd,
                                                   R igm1, R p_ref, R* acc) {
    constexpr int S = G::stride(L);
    const int i = node_pos<L>(nd);
    const R s = sc<R>(A).s[L];
    const R* Dv = sm + OFF_D;
    const R* Q = sm + OFF_Q + el * NQ * NP;
    R vi[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) vi[d] = Q[(1 + d) * NP + nd];
    const R ri = Q[nd], pdi = Q[PD * NP + nd], bi = Q[(DIM + 2) * NP + nd];
    R* X = sm + OFF_X + ((el * DIM + L) * NO) * NV * NP + nd;
#pragma unroll
    for (int o = 1; o <= NO; ++o) {
      if (2 * o == N1 && i >= N1 / 2) break;
      const int j = (i + o < N1) ? i + o : i + o - N1;
      const int nj = nd + (j - i) * S;
      R vj[DIM];
#pragma unroll
      for (int d = 0; d < DIM; ++d) vj[d] = Q[(1 + d) * NP + nj];
      R F[NV];
      ec_flux_prims<DIM, L>(ri, vi, pdi, bi, Q[nj], vj, Q[PD * NP + nj], Q[(DIM + 2) * NP + nj],
                            igm1, p_ref, F);
      const R c = s * Dv[i * N1 + j];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        acc[v] -= c * F[v];
        X[((o - 1) * NV + v) * NP] = F[v];
      }
    }
  }

  // ---- phase 4 (EC): the pairs other nodes evaluated for this node, and D_ii F(U_i) ----
  template <int L>
  static __device__ __forceinline__ void partner_pairs(const R* sm, const StageArgs& A, int el,
                                                       int nd, R p_ref, R* acc) {
    constexpr int S = G::stride(L);
    const int i = node_pos<L>(nd);
    const R s = sc<R>(A).s[L];
    const R* Dv = sm + OFF_D;
    const R* X = sm + OFF_X + ((el * DIM + L) * NO) * NV * NP;
#pragma unroll
    for (int o = 1; o <= NO; ++o) {
      const int k = (i - o >= 0) ? i - o : i - o + N1;  // owner of pair (k, i) at offset o
      if (2 * o == N1 && k >= N1 / 2) continue;
      const int nk = nd + (k - i) * S;
      const R c = s * Dv[i * N1 + k];
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] -= c * X[((o - 1) * NV + v) * NP + nk];
    }
    if (i == 0 || i == N) {  // diagonal: F#(U_i, U_i) = F(U_i); only the end nodes have D_ii != 0
      R u[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) u[v] = sm[OFF_U + (el * NV + v) * NP + nd];
      const Prim<DIM, R> qq = prims<DIM>(u, sm[OFF_Q + (el * NQ + PD) * NP + nd], p_ref);
      R F[NV];
      point_flux<DIM, L>(u, qq, F);
      const R c = s * Dv[i * N1 + i];
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] -= c * F[v];
    }
  }

  // ---- phase 4 (strong/weak): contract the volume operator with the staged point fluxes ----
  template <int L>
  static __device__ __forceinline__ void contract(const R* sm, const StageArgs& A, int el, int nd,
                                                  R* acc) {
    constexpr int S = G::stride(L);
    const int i = node_pos<L>(nd);
    const R s = sc<R>(A).s[L];
    const R* Dv = sm + OFF_D;
    const R* Fq = sm + OFF_Q + (el * NQ + L * NV) * NP + nd - i * S;
#pragma unroll
    for (int m = 0; m < N1; ++m) {
      const R c = s * Dv[i * N1 + m];
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] -= c * Fq[v * NP + m * S];
    }
  }

  // Cyclic relabelling of the axes that makes direction l the first one: the Euler fluxes
  // are unchanged by a relabelling of the axes, so every face job evaluates its Riemann
  // flux with one instantiation (normal along axis 0) -- one code path for all faces, no
  // divergence between the directions of a warp.
  static __device__ __forceinline__ void to_face_axes(const R* in, R* out, int l) {
    out[0] = in[0];
    out[NV - 1] = in[NV - 1];
    if constexpr (DIM == 2) {
      out[1] = l ? in[2] : in[1];
      out[2] = l ? in[1] : in[2];
    } else {
      out[1] = l == 0 ? in[1] : (l == 1 ? in[2] : in[3]);
      out[2] = l == 0 ? in[2] : (l == 1 ? in[3] : in[1]);
      out[3] = l == 0 ? in[3] : (l == 1 ? in[1] : in[2]);
    }
  }
  static __device__ __forceinline__ void from_face_axes(const R* in, R* out, int l) {
    out[0] = in[0];
    out[NV - 1] = in[NV - 1];
    if constexpr (DIM == 2) {
      out[1] = l ? in[2] : in[1];
      out[2] = l ? in[1] : in[2];
    } else {
      out[1] = l == 0 ? in[1] : (l == 1 ? in[3] : in[2]);
      out[2] = l == 0 ? in[2] : (l == 1 ? in[1] : in[3]);
      out[3] = l == 0 ? in[3] : (l == 1 ? in[2] : in[1]);
    }
  }

  // ---- phase 3: one face node (face r.face of element r.jel) ----
  static __device__ __forceinline__ void face_job(R* sm, const double* trace, const StageArgs& A,
                                                  const Role& r, R gamma, R igm1, R p_ref) {
    const int ej = r.jel, side = r.face & 1, l = r.face >> 1;
    R own0[NV], nbr0[NV];
    double n64[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      own0[v] = sm[OFF_U + (ej * NV + v) * NP + r.ndo];
      n64[v] = trace[((ej * NF + r.face) * NV + v) * NFN + r.f];
      nbr0[v] = Ar<R>::load(n64[v]);
    }
    double rhoe;
    const R pd_own = sm[OFF_Q + (ej * NQ + PD) * NP + r.ndo];
    const R pd_nbr = pdev<DIM>(n64, nbr0, A.pd.gm1, A.pd.p_ref, rhoe);
    R own[NV], nbr[NV];
    to_face_axes(own0, own, l);
    to_face_axes(nbr0, nbr, l);
    const Prim<DIM, R> po = prims<DIM>(own, pd_own, p_ref);
    const Prim<DIM, R> pn = prims<DIM>(nbr, pd_nbr, p_ref);
    R uL[NV], uR[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      uL[v] = side ? own[v] : nbr[v];
      uR[v] = side ? nbr[v] : own[v];
    }
    const Prim<DIM, R>& a = side ? po : pn;
    const Prim<DIM, R>& b = side ? pn : po;
    R Fs[NV];
    surface_flux<DIM, 0>(A.surface, uL, a, uR, b, gamma, igm1, p_ref, Fs);  // the single call site
    if (!A.weak) {
      R Fo[NV];
      point_flux<DIM, 0>(own, po, Fo);
#pragma unroll
      for (int v = 0; v < NV; ++v) Fs[v] -= Fo[v];
    }
    R Fj[NV];
    from_face_axes(Fs, Fj, l);
    const R lf = (side ? R(-1) : R(1)) * sc<R>(A).s[l] * sc<R>(A).lift;
    R* Sx = sm + OFF_S + ((ej * NF + r.face) * NFN + r.f) * NV;
#pragma unroll
    for (int v = 0; v < NV; ++v) Sx[v] = lf * Fj[v];
  }

  template <int L>
  static __device__ __forceinline__ void gather_faces(const R* sm, int el, int nd, R* acc) {
    const int i = node_pos<L>(nd), f = node_line<L>(nd);
    if (i == 0) {
      const R* Sx = sm + OFF_S + ((el * NF + 2 * L) * NFN + f) * NV;
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] += Sx[v];
    }
    if (i == N) {
      const R* Sx = sm + OFF_S + ((el * NF + 2 * L + 1) * NFN + f) * NV;
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] += Sx[v];
    }
  }

  // ---- one element group, inputs staged in buffer b ----
  static __device__ __forceinline__ void compute(const StageArgs& A, const Smem& M, const Role& r,
                                                 int g, int b, bool need_un) {
    const int t = threadIdx.x;
    R* sm = M.sm;
    const double* SU = M.st + b * ST_SIZE + ST_U;
    const double* SN = M.st + b * ST_SIZE + ST_N;
    const double* TR = M.st + b * ST_SIZE + ST_T;
    const int e0 = g * EPB;
    const R gamma = sc<R>(A).gamma, igm1 = sc<R>(A).igm1, p_ref = sc<R>(A).p_ref;
    const int el = r.el, nd = r.nd;
    const bool active = (t < EPB * NP) && (e0 + el < A.n_elem);

    // phase 1: convert, primitives, stage
    if (active) {
      double u64[NV];
      R u[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        u64[v] = SU[(el * NV + v) * NP + nd];
        u[v] = Ar<R>::load(u64[v]);
        sm[OFF_U + (el * NV + v) * NP + nd] = u[v];
      }
      double rhoe;
      const R pd = pdev<DIM>(u64, u, A.pd.gm1, A.pd.p_ref, rhoe);
      const Prim<DIM, R> q = prims<DIM>(u, pd, p_ref);
      // positivity of the state this stage reads (rho > 0 and rho e > 0), decided on the
      // FP64 values by their sign/exponent bits
      if (!(__double2hiint(u64[0]) > 0 && __double2hiint(rhoe) > 0)) atomicOr(A.err, 2u);
      R* Q = sm + OFF_Q + el * NQ * NP;
      Q[PD * NP + nd] = pd;
      if constexpr (EC) {
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

    // phase 2: own two-point pairs (accumulated in registers, stored for the partners)
    R acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = R(0);
    if constexpr (EC) {
      if (active) {
        own_pairs<0>(sm, A, el, nd, igm1, p_ref, acc);
        own_pairs<1>(sm, A, el, nd, igm1, p_ref, acc);
        if constexpr (DIM == 3) own_pairs<2>(sm, A, el, nd, igm1, p_ref, acc);
      }
    }
    // phase 3: face jobs
    if (t < NJS && e0 + r.jel < A.n_elem) face_job(sm, TR, A, r, gamma, igm1, p_ref);
    __syncthreads();

    // phase 4: gather, then L or the stage update
    if (!active) return;
    if constexpr (EC) {
      partner_pairs<0>(sm, A, el, nd, p_ref, acc);
      partner_pairs<1>(sm, A, el, nd, p_ref, acc);
      if constexpr (DIM == 3) partner_pairs<2>(sm, A, el, nd, p_ref, acc);
    } else {
      contract<0>(sm, A, el, nd, acc);
      contract<1>(sm, A, el, nd, acc);
      if constexpr (DIM == 3) contract<2>(sm, A, el, nd, acc);
    }
    gather_faces<0>(sm, el, nd, acc);
    gather_faces<1>(sm, el, nd, acc);
    if constexpr (DIM == 3) gather_faces<2>(sm, el, nd, acc);

    const long long gi = A.base + (long long)(e0 + el) * NP + nd;
    double res[NV];
    if (A.mode == 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) res[v] = Ar<R>::widen(acc[v]);
    } else {
      // U^(k) = ca Un + cb (U^(k-1) + dt L), with the increment cb dt L formed in R
      const R cbdt = sc<R>(A).cbdt;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const double inc = Ar<R>::widen(cbdt * acc[v]);
        double x = fma(A.cb, SU[(el * NV + v) * NP + nd], inc);
        if (need_un) x = fma(A.ca, SN[(el * NV + v) * NP + nd], x);
        res[v] = x;
      }
      if (A.floor_on) {  // positivity floor (off by default)
        if (A.rho_floor > 0.0 && res[0] < A.rho_floor) res[0] = A.rho_floor;
        double kin = 0.0;
#pragma unroll
        for (int d = 0; d < DIM; ++d) kin += res[1 + d] * res[1 + d] / res[0];
        const double p = (A.gamma - 1.0) * (res[DIM + 1] - 0.5 * kin);
        if (A.p_floor > 0.0 && p < A.p_floor) res[DIM + 1] = A.p_floor / (A.gamma - 1.0) + 0.5 * kin;
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

  static __device__ void run(const StageArgs& A) {
    const Smem M = carve();
    const int t = threadIdx.x;
    const Role r = role();
    for (int k = t; k < N1 * N1; k += T) M.sm[OFF_D + k] = R(A.Dv[k]);
    const bool need_un = A.need_un != 0;
    const int ng = (A.n_elem + EPB - 1) / EPB;
    int g = blockIdx.x;
    if (g < ng && t < EPB * NF) {
      const int e = g * EPB + t / NF;
      M.nb[t] = (e < A.n_elem) ? neighbour(A, e, t % NF) : 0;
    }
    __syncthreads();
    if (g < ng) issue(A, M, r, g, 0, need_un);
    cp_async_commit();
    for (int it = 0; g < ng; g += gridDim.x, ++it) {
      const int b = it & 1;
      const int gn = g + gridDim.x;
      if (gn < ng && t < EPB * NF) {
        const int e = gn * EPB + t / NF;
        M.nb[(b ^ 1) * EPB * NF + t] = (e < A.n_elem) ? neighbour(A, e, t % NF) : 0;
      }
      __syncthreads();  // neighbour table ready; the previous group no longer reads buffer b^1
      if (gn < ng) issue(A, M, r, gn, b ^ 1, need_un);
      cp_async_commit();
      cp_async_wait_prev();
      __syncthreads();  // group g's copies (all threads') are visible
      compute(A, M, r, g, b, need_un);
    }
  }
};

template <int DIM, int N, bool EC, class R>
__global__ void __launch_bounds__(EulerStage<DIM, N, EC, R>::T) k_euler_stage(const StageArgs A) {
  EulerStage<DIM, N, EC, R>::run(A);
}

// persistent grid size per instantiation: resident CTAs per SM x SMs (set by prepare)
template <int DIM, int N, bool EC, class R>
struct GridSize {
  static int ctas;
};
template <int DIM, int N, bool EC, class R>
int GridSize<DIM, N, EC, R>::ctas = 0;

template <int DIM, int N, bool EC, class R>
static cudaError_t prepare_one() {
  using K = EulerStage<DIM, N, EC, R>;
  cudaError_t e = cudaFuncSetAttribute(k_euler_stage<DIM, N, EC, R>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)K::smem_bytes());
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_euler_stage<DIM, N, EC, R>, K::T,
                                                    K::smem_bytes());
  if (e != cudaSuccess) return e;
  GridSize<DIM, N, EC, R>::ctas = sms * (per_sm > 0 ? per_sm : 1);
  return cudaSuccess;
}

template <int DIM, int N, bool EC, class R>
static cudaError_t launch_one(const StageArgs& a, cudaStream_t s) {
  using K = EulerStage<DIM, N, EC, R>;
  const int groups = (a.n_elem + K::EPB - 1) / K::EPB;
  if (groups == 0) return cudaSuccess;
  if (GridSize<DIM, N, EC, R>::ctas == 0) {
    cudaError_t e = prepare_one<DIM, N, EC, R>();
    if (e != cudaSuccess) return e;
  }
  const int blocks = groups < GridSize<DIM, N, EC, R>::ctas ? groups : GridSize<DIM, N, EC, R>::ctas;
  k_euler_stage<DIM, N, EC, R><<<blocks, K::T, K::smem_bytes(), s>>>(a);
  return cudaGetLastError();
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
  const R pr = R(p_ref), gm = R(gamma), igm1 = R(1) / (gm - R(1));
  const Prim<DIM, R> pa = prims<DIM>(a, pdev<DIM>(a64, a, gamma - 1.0, p_ref, ea), pr);
  const Prim<DIM, R> pb = prims<DIM>(b, pdev<DIM>(b64, b, gamma - 1.0, p_ref, eb), pr);
  if (kind < 0) ec_flux<DIM, L>(pa, pb, igm1, pr, f);
  else surface_flux<DIM, L>(kind, a, pa, b, pb, gm, igm1, pr, f);
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
