// dg_stage.cuh -- the fused DGSEM residual + SSP-RK3 stage kernel (templates) for sm_103a.
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
#pragma once

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
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
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

// Cyclic relabelling of the axes that makes direction l the first one (and back): the Euler
// fluxes are unchanged by a relabelling of the axes, so every face flux is evaluated with one
// instantiation (normal along axis 0).
template <int DIM, class R>
__device__ __forceinline__ void to_face_axes(const R* in, R* out, int l) {
  constexpr int NV = DIM + 2;
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
template <int DIM, class R>
__device__ __forceinline__ void from_face_axes(const R* in, R* out, int l) {
  constexpr int NV = DIM + 2;
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

// Domain face of face `side` (0 lower, 1 upper) in direction l of element e, if that face
// carries a boundary condition; else -1.
__device__ __forceinline__ int boundary_face(const InstArgs& I, int dim, int e, int l, int side) {
  const int f = 2 * l + side;
  if (I.bc[f] == 0) return -1;
  const int c = l == 0 ? e % I.nel[0] : (l == 1 ? (e / I.nel[0]) % I.nel[1] : e / (I.nel[0] * I.nel[1]));
  (void)dim;
  return (side ? c == I.nel[l] - 1 : c == 0) ? f : -1;
}

// Boundary flux at domain face fb in face axes (Sec. 3.1.1 "Surface Fluxes", one functor per
// boundary type): own / po the interior trace and its primitives in face axes, side = 1 when
// the interior is the left state (upper face).  Slip wall: Riemann flux against the mirror
// state; supersonic inflow: F(U_b); supersonic outflow: F(U-); Dirichlet: Riemann flux
// against U_b.  The prescribed state is converted exactly as a neighbour trace is.
template <int DIM, class R>
__device__ __forceinline__ void boundary_flux(const InstArgs& I, int fb, int l, int side, const R* own,
                                              const Prim<DIM, R>& po, int kind, R gamma, R igm1,
                                              R p_ref, double gm1_64, double p_ref_64, R hgm1, R* Fs) {
  constexpr int NV = DIM + 2;
  const int type = I.bc[fb];
  if (type == 3) {  // outflow
    point_flux<DIM, 0>(own, po, Fs);
    return;
  }
  R ext[NV];
  Prim<DIM, R> pe;
  if (type == 1) {  // slip wall: the mirror state
#pragma unroll
    for (int v = 0; v < NV; ++v) ext[v] = own[v];
    ext[1] = -own[1];
    pe = prims<DIM>(ext, po.pd, p_ref);
  } else {  // inflow, Dirichlet: the prescribed state
    double b64[NV];
    R b0[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      b64[v] = I.bcs[fb][v];
      b0[v] = Ar<R>::load(b64[v]);
    }
    const R pd = pdev<DIM>(b64, b0, gm1_64, p_ref_64, hgm1);
    to_face_axes<DIM>(b0, ext, l);
    pe = prims<DIM>(ext, pd, p_ref);
    if (type == 2) {  // inflow
      point_flux<DIM, 0>(ext, pe, Fs);
      return;
    }
  }
  if (side) surface_flux<DIM, 0>(kind, own, po, ext, pe, gamma, igm1, p_ref, Fs);
  else surface_flux<DIM, 0>(kind, ext, pe, own, po, gamma, igm1, p_ref, Fs);
}

constexpr int cmax(int a, int b) { return a > b ? a : b; }
constexpr int cmin(int a, int b) { return a < b ? a : b; }
constexpr int al4(int n) { return (n + 3) & ~3; }

// the launch scalars in the flux precision (precomputed on the host)
template <class R>
__device__ __forceinline__ const ScalarsT<R>& sc(const StageArgs& A);
template <>
__device__ __forceinline__ const ScalarsT<double>& sc<double>(const StageArgs& A) {
  return A.pd;
}
template <>
__device__ __forceinline__ const ScalarsT<float>& sc<float>(const StageArgs& A) {
  return A.pf;
}
// per-instance metric scalars in the flux precision
template <class R> __device__ __forceinline__ R sv(const InstArgs& I, int l);
template <> __device__ __forceinline__ double sv<double>(const InstArgs& I, int l) { return I.s[l]; }
template <> __device__ __forceinline__ float sv<float>(const InstArgs& I, int l) { return I.sf[l]; }
template <class R> __device__ __forceinline__ R liftv(const InstArgs& I);
template <> __device__ __forceinline__ double liftv<double>(const InstArgs& I) { return I.lift; }
template <> __device__ __forceinline__ float liftv<float>(const InstArgs& I) { return I.liftf; }
template <class R> __device__ __forceinline__ R from64(double x);
template <> __device__ __forceinline__ double from64<double>(double x) { return x; }
template <> __device__ __forceinline__ float from64<float>(double x) { return d2f_rn(x); }

template <int DIM, int N, bool EC, class R, int GS = 1>
struct EulerStage {
  using G = Geo<DIM, N>;
  static constexpr int NV = G::NV, NP = G::NP, N1 = G::N1, NFN = G::NFN;
  static constexpr int EPB = G::EPB * GS;                  // elements per group
  static constexpr int NF = 2 * DIM;                       // faces per element
  static constexpr int NJS = EPB * NF * NFN;               // face jobs per group
  static constexpr int T = ((cmax(EPB * NP, NJS) + 31) / 32) * 32;
  // Two-point pairs are assigned cyclically along each line: node i owns the pairs
  // (i, i+o mod N1) for o = 1..NO, the last offset (o = N1/2 when N1 is even) only for
  // i < N1/2, so that every unordered pair is evaluated exactly once.
  static constexpr int NO = N1 / 2;
  // per-node staged quantities: EC -- the two Q4 records of the two-point flux (A, B); strong/
  // weak -- the DIM point fluxes (NV each) and pd
  static constexpr int NQ = EC ? 8 : (DIM * NV + 1);
  static constexpr int PD = DIM * NV;  // strong/weak: row of pd
  static constexpr int NXN = EC ? DIM * NO : 0;            // pair slots per node
  // FP64 staging buffer (two of them): own U [EPB][NV][NP], U^n [EPB][NV][NP],
  // neighbour face traces [EPB][NF][NV][NFN]
  static constexpr int ST_U = 0, ST_N = EPB * NV * NP, ST_T = 2 * EPB * NV * NP;
  static constexpr int ST_SIZE = ST_T + EPB * NF * NV * NFN;
  // flux-precision arrays
  // pair slot: F_0..F_3 as Q4 per node, then F_4 per node (3D), padded to 16 bytes
  static constexpr int XSLOT = 4 * NP + (NV > 4 ? al4(NP) : 0);
  static constexpr int OFF_U = 0;                                  // [EPB][NV][NP]
  static constexpr int OFF_Q = al4(OFF_U + EPB * NV * NP);         // EC: [EPB][2][NP] Q4, else [EPB][NQ][NP]
  static constexpr int OFF_S = al4(OFF_Q + EPB * NQ * NP);         // [EPB][NF][NFN][NV]
  static constexpr int OFF_X = al4(OFF_S + EPB * NF * NFN * NV);   // [EPB][DIM][NO] pair slots
  // coefficient tables, scaled by 2/dx_l: EC -- own [DIM][N1][NO] (s_l Dv_ij, j = i+o) then
  // partner [DIM][N1][NO] (s_l Dv_ik, k = i-o); strong/weak -- [DIM][N1][N1] (s_l Dv)
  static constexpr int OFF_D = OFF_X + EPB * NXN * XSLOT;
  static constexpr int ND = EC ? 2 * DIM * N1 * NO : DIM * N1 * N1;
  static constexpr int R_SIZE = OFF_D + ND;
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

  // EC records of element slot el: A[NP] then B[NP]
  static __device__ __forceinline__ Q4<R>* qa(R* sm, int el) {
    return reinterpret_cast<Q4<R>*>(sm + OFF_Q) + el * 2 * NP;
  }
  static __device__ __forceinline__ const Q4<R>* qa(const R* sm, int el) {
    return reinterpret_cast<const Q4<R>*>(sm + OFF_Q) + el * 2 * NP;
  }
  // pressure deviation of node nd of element slot el
  static __device__ __forceinline__ R pd_of(const R* sm, int el, int nd) {
    if constexpr (EC) return qa(sm, el)[NP + nd].w;
    else return sm[OFF_Q + (el * NQ + PD) * NP + nd];
  }
  // pair slot (direction L, offset o) of element slot el
  static __device__ __forceinline__ R* xslot(R* sm, int el, int L, int o) {
    return sm + OFF_X + ((el * DIM + L) * NO + (o - 1)) * XSLOT;
  }
  static __device__ __forceinline__ const R* xslot(const R* sm, int el, int L, int o) {
    return sm + OFF_X + ((el * DIM + L) * NO + (o - 1)) * XSLOT;
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

  // neighbour element of face `face` (direction face/2, side face%2) of element e
  static __device__ __forceinline__ int neighbour(const InstArgs& A, int e, int face) {
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
    int pos[3];             // position of the node along each direction
    int jel, face, f, ndn;  // face-job role (t < NJS): element, face, face node, neighbour node
    int ndo;                // own node of the face job
    int pm[3];              // face axes -> Cartesian variable index of the momentum components
  };

  static __device__ __forceinline__ Role role() {
    Role r;
    const int t = threadIdx.x;
    r.el = t / NP;
    r.nd = t - r.el * NP;
    r.pos[0] = r.nd % N1;
    r.pos[1] = (r.nd / N1) % N1;
    r.pos[2] = DIM == 3 ? r.nd / (N1 * N1) : 0;
    r.jel = t / (NF * NFN);
    const int q = t - r.jel * (NF * NFN);
    r.face = q / NFN;
    r.f = q - r.face * NFN;
    const int l = r.face >> 1, side = r.face & 1;
    if (l == 0) { r.ndn = line_node<0>(r.f, side ? 0 : N); r.ndo = line_node<0>(r.f, side ? N : 0); }
    else if (l == 1) { r.ndn = line_node<1>(r.f, side ? 0 : N); r.ndo = line_node<1>(r.f, side ? N : 0); }
    else { r.ndn = line_node<DIM - 1>(r.f, side ? 0 : N); r.ndo = line_node<DIM - 1>(r.f, side ? N : 0); }
#pragma unroll
    for (int k = 0; k < 3; ++k) r.pm[k] = 1 + (l + k) % DIM;
    return r;
  }

  // start the asynchronous copies of group g into staging buffer b
  static __device__ __forceinline__ void issue(const StageArgs& A, const InstArgs& I, const Role& r,
                                               int g, double* S, const int* nb, bool need_un) {
    const int t = threadIdx.x;
    const int e = g * EPB + r.el;
    if (t < EPB * NP && e < I.n_elem) {
      const long long o = I.base + (long long)e * NP + r.nd;
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
    if (t < NJS && ej < I.n_elem) {
      const int en = nb[r.jel * NF + r.face];
      const double* pt = A.U + I.base + (long long)en * NP + r.ndn;
      double* st = S + ST_T + ((r.jel * NF + r.face) * NV) * NFN + r.f;
#pragma unroll
      for (int v = 0; v < NV; ++v) cp_async8(st + v * NFN, pt + v * A.stride);
    }
  }

  // L2 prefetch of group g's own state and U^n (the EPB * NP consecutive values of each
  // variable, by 128-byte lines), for the batched walk two groups ahead
  static __device__ __forceinline__ void prefetch_group(const StageArgs& A, const InstArgs& I, int g,
                                                        bool need_un) {
    constexpr int LPV = (EPB * NP * 8 + 127) / 128 + 1;  // lines per variable (unaligned start)
    const int ne = min(EPB, I.n_elem - g * EPB);
    if (ne <= 0) return;
    const int bytes = ne * NP * 8;
    for (int q = threadIdx.x; q < 2 * NV * LPV; q += blockDim.x) {
      const int which = q / (NV * LPV), rem = q - which * (NV * LPV);
      if (which == 1 && !need_un) break;
      const int v = rem / LPV, l = rem - v * LPV;
      const double* base = (which ? A.Un : A.U) + I.base + (long long)g * EPB * NP + (long long)v * A.stride;
      const char* p0 = reinterpret_cast<const char*>(base);
      const char* p = p0 + 128 * l;
      const char* last = p0 + (bytes - 1);
      asm volatile("prefetch.global.L2 [%0];" ::"l"(p < last ? p : last));
    }
  }

  // ---- phase 2 (EC): this node's own pairs in direction L ----
  template <int L>
  static __device__ __forceinline__ void own_pairs(R* sm, const R* D, const Role& r, int el, R igm1, R p_ref,
                                                   R* acc) {
    constexpr int S = G::stride(L);
    const int nd = r.nd, i = r.pos[L];
    const R* C = D + (L * N1 + i) * NO;
    const Q4<R>* QA = qa(sm, el);
    const Q4<R> ai = QA[nd], bi = QA[NP + nd];
#pragma unroll
    for (int o = 1; o <= NO; ++o) {
      if (2 * o == N1 && i >= N1 / 2) break;
      const int nj = (i + o < N1) ? nd + o * S : nd + (o - N1) * S;
      const Q4<R> aj = QA[nj], bj = QA[NP + nj];
      R F[NV];
      ec_flux_rec<DIM, L>(ai, bi, aj, bj, igm1, p_ref, F);
      const R c = C[o - 1];
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] -= c * F[v];
      R* X = xslot(sm, el, L, o);
      reinterpret_cast<Q4<R>*>(X)[nd] = Q4<R>{F[0], F[1], F[2], F[3]};
      if constexpr (NV > 4) X[4 * NP + nd] = F[4];
    }
  }

  // ---- phase 4 (EC): the pairs other nodes evaluated for this node ----
  template <int L>
  static __device__ __forceinline__ void partner_pairs(const R* sm, const R* D, const Role& r, int el, R* acc) {
    constexpr int S = G::stride(L);
    const int nd = r.nd, i = r.pos[L];
    const R* C = D + DIM * N1 * NO + (L * N1 + i) * NO;
#pragma unroll
    for (int o = 1; o <= NO; ++o) {
      // owner k = i - o (mod N1) of pair (k, i) at offset o
      if (2 * o == N1 && (i >= o ? i - o : i - o + N1) >= N1 / 2) continue;
      const int nk = (i >= o) ? nd - o * S : nd + (N1 - o) * S;
      const R c = C[o - 1];
      const R* X = xslot(sm, el, L, o);
      const Q4<R> f = reinterpret_cast<const Q4<R>*>(X)[nk];
      acc[0] -= c * f.x;
      acc[1] -= c * f.y;
      acc[2] -= c * f.z;
      acc[3] -= c * f.w;
      if constexpr (NV > 4) acc[4] -= c * X[4 * NP + nk];
    }
  }

  // ---- phase 4 (strong/weak): contract the volume operator with the staged point fluxes ----
  template <int L>
  static __device__ __forceinline__ void contract(const R* sm, const R* D, const Role& r, int el, R* acc) {
    constexpr int S = G::stride(L);
    const int nd = r.nd, i = r.pos[L];
    const R* Dl = D + (L * N1 + i) * N1;
    const R* Fq = sm + OFF_Q + (el * NQ + L * NV) * NP + nd - i * S;
#pragma unroll
    for (int m = 0; m < N1; ++m) {
      const R c = Dl[m];
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

  // ---- phase 3: one face node (face r.face of element r.jel) ----
  // The own trace is read in face axes (permuted shared-memory offsets); the neighbour's
  // FP64 trace is converted and its pressure deviation formed in Cartesian order (as the
  // neighbour's own phase 1 does, so that both elements see the same bits), then relabelled.
  // The result is stored back to Cartesian components by permuted offsets.
  static __device__ __forceinline__ void face_job(R* sm, const double* trace, const StageArgs& A,
                                                  const InstArgs& I, const Role& r, int e, R gamma,
                                                  R igm1, R p_ref) {
    const int ej = r.jel, side = r.face & 1, l = r.face >> 1;
    const ScalarsT<R>& k = sc<R>(A);
    const R* Uo = sm + OFF_U + ej * NV * NP + r.ndo;
    R own[NV];
    own[0] = Uo[0];
#pragma unroll
    for (int d = 0; d < DIM; ++d) own[1 + d] = Uo[r.pm[d] * NP];
    own[NV - 1] = Uo[(NV - 1) * NP];
    const Prim<DIM, R> po = prims_i<DIM>(own, Ar<R>::rcp(own[0]), pd_of(sm, ej, r.ndo), p_ref);
    trace_momentum<DIM>(po, own);
    R Fs[NV];
    const int fb = I.nonper ? boundary_face(I, DIM, e, l, side) : -1;
    if (fb >= 0) {  // a domain face with a boundary condition
      boundary_flux<DIM, R>(I, fb, l, side, own, po, A.surface, gamma, igm1, p_ref, A.pd.gm1, A.pd.p_ref,
                            k.hgm1, Fs);
    } else {
      R nbr0[NV];
      double n64[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        n64[v] = trace[((ej * NF + r.face) * NV + v) * NFN + r.f];
        nbr0[v] = Ar<R>::load(n64[v]);
      }
      const R irn = Ar<R>::rcp(nbr0[0]);
      const R pd_nbr = pdev_i<DIM>(n64, nbr0, irn, A.pd.gm1, A.pd.p_ref, k.hgm1);
      R nbr[NV];
      to_face_axes(nbr0, nbr, l);
      const Prim<DIM, R> pn = prims_i<DIM>(nbr, irn, pd_nbr, p_ref);
      trace_momentum<DIM>(pn, nbr);
      R uL[NV], uR[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        uL[v] = side ? own[v] : nbr[v];
        uR[v] = side ? nbr[v] : own[v];
      }
      const Prim<DIM, R>& a = side ? po : pn;
      const Prim<DIM, R>& b = side ? pn : po;
      surface_flux<DIM, 0>(A.surface, uL, a, uR, b, gamma, igm1, p_ref, Fs);  // the single call site
    }
    if (!EC && !A.weak) {  // strong form: F* - F(U_own) (the two-point form's diagonal cancels it)
      R Fo[NV];
      point_flux<DIM, 0>(own, po, Fo);
#pragma unroll
      for (int v = 0; v < NV; ++v) Fs[v] -= Fo[v];
    }
    const R lf = (side ? R(-1) : R(1)) * sv<R>(I, l) * liftv<R>(I);
    R* Sx = sm + OFF_S + ((ej * NF + r.face) * NFN + r.f) * NV;
    Sx[0] = lf * Fs[0];
#pragma unroll
    for (int d = 0; d < DIM; ++d) Sx[r.pm[d]] = lf * Fs[1 + d];
    Sx[NV - 1] = lf * Fs[NV - 1];
  }

  template <int L>
  static __device__ __forceinline__ void gather_faces(const R* sm, const Role& r, int el, R* acc) {
    const int i = r.pos[L], f = node_line<L>(r.nd);
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

  // ---- one element group, inputs staged in buffer b; D: the coefficient tables (load_ops) ----
  static __device__ __forceinline__ void compute(const StageArgs& A, const InstArgs& I, R* sm, const R* D,
                                                 const Role& r, int g, const double* S,
                                                 bool need_un) {
    const int t = threadIdx.x;
    const double* SU = S + ST_U;
    const double* SN = S + ST_N;
    const double* TR = S + ST_T;
    const int e0 = g * EPB;
    const ScalarsT<R>& k = sc<R>(A);
    const R gamma = k.gamma, igm1 = k.igm1, p_ref = k.p_ref;
    const int el = r.el, nd = r.nd;
    const bool active = (t < EPB * NP) && (e0 + el < I.n_elem);

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
      const R irho = Ar<R>::rcp(u[0]);
      const R pd = pdev_i<DIM>(u64, u, irho, A.pd.gm1, A.pd.p_ref, k.hgm1);
      // positivity of the state this stage reads (rho > 0 and rho e > 0), decided on the
      // FP64 values
      if (!positive<DIM>(u64, u, pd, p_ref, k.margin_e, k.margin_0, A.pd.gm1)) atomicOr(A.err, 2u);
      const Prim<DIM, R> q = prims_i<DIM>(u, irho, pd, p_ref);
      if constexpr (EC) {
        Q4<R>* QA = qa(sm, el);
        ec_records<DIM>(q, QA[nd], QA[NP + nd]);
      } else {
        R* Q = sm + OFF_Q + el * NQ * NP;
        Q[PD * NP + nd] = pd;
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
        own_pairs<0>(sm, D, r, el, igm1, p_ref, acc);
        own_pairs<1>(sm, D, r, el, igm1, p_ref, acc);
        if constexpr (DIM == 3) own_pairs<2>(sm, D, r, el, igm1, p_ref, acc);
      }
    }
    // phase 3: face jobs
    if (t < NJS && e0 + r.jel < I.n_elem) face_job(sm, TR, A, I, r, e0 + r.jel, gamma, igm1, p_ref);
    __syncthreads();

    // phase 4: gather, then L or the stage update
    if (!active) return;
    if constexpr (EC) {
      partner_pairs<0>(sm, D, r, el, acc);
      partner_pairs<1>(sm, D, r, el, acc);
      if constexpr (DIM == 3) partner_pairs<2>(sm, D, r, el, acc);
    } else {
      contract<0>(sm, D, r, el, acc);
      contract<1>(sm, D, r, el, acc);
      if constexpr (DIM == 3) contract<2>(sm, D, r, el, acc);
    }
    gather_faces<0>(sm, r, el, acc);
    gather_faces<1>(sm, r, el, acc);
    if constexpr (DIM == 3) gather_faces<2>(sm, r, el, acc);

    const long long gi = I.base + (long long)(e0 + el) * NP + nd;
    double res[NV];
    if (A.mode == 1 && A.alpha && A.alpha[e0 + el] > 0.0) {
      // shock-flagged element: its DG residual goes to the side buffer, the blending launch
      // forms the update
#pragma unroll
      for (int v = 0; v < NV; ++v) A.ldg[v * A.stride + gi] = Ar<R>::widen(acc[v]);
      return;
    }
    if (A.mode == 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) res[v] = Ar<R>::widen(acc[v]);
    } else {
      // U^(k) = ca Un + cb U^(k-1) + beta dt L, with the increment beta dt L formed in R
      const R cbdt = k.cbdt;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const double inc = Ar<R>::widen(cbdt * acc[v]);
        double x = fma(A.cb, SU[(el * NV + v) * NP + nd], inc);
        if (need_un) x = fma(A.ca, SN[(el * NV + v) * NP + nd], x);
        res[v] = x;
      }
      if (A.acc) {  // running sum of a later stage: acc = acc_a acc + acc_b U^(k-1) + acc_beta dt L
        const R abdt = k.abdt;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          double y = fma(A.acc_b, SU[(el * NV + v) * NP + nd], Ar<R>::widen(abdt * acc[v]));
          if (A.acc_a != 0.0) y = fma(A.acc_a, A.acc[v * A.stride + gi], y);
          A.acc[v * A.stride + gi] = y;
        }
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

  static __device__ __forceinline__ void fill_nb(const InstArgs& I, int g, int* nb) {
    const int t = threadIdx.x;
    if (t < EPB * NF) {
      const int e = g * EPB + t / NF;
      nb[t] = (e < I.n_elem) ? neighbour(I, e, t % NF) : 0;
    }
  }

  // coefficient tables of instance I (volume operator Dv, row-major (N+1)^2), scaled by 2/dx_l,
  // written to D[ND]
  static __device__ __forceinline__ void load_ops(R* D, const double* Dv, const InstArgs& I) {
    for (int q = threadIdx.x; q < ND; q += blockDim.x) {
      double c;
      if constexpr (EC) {
        const int part = q / (DIM * N1 * NO), rem = q - part * (DIM * N1 * NO);
        const int L = rem / (N1 * NO), i = (rem / NO) % N1, o = rem % NO + 1;
        const int j = part ? (i - o + N1) % N1 : (i + o) % N1;
        c = I.s[L] * Dv[i * N1 + j];
      } else {
        const int L = q / (N1 * N1), rem = q - L * N1 * N1;
        c = I.s[L] * Dv[rem];
      }
      D[q] = from64<R>(c);
    }
  }

  // single-instance persistent launch: groups of A.inst, double-buffered, one barrier per
  // group outside compute().  The neighbour table of a group is filled two iterations ahead
  // (slot it & 1 holds the table of iteration it's group), so that the barrier that publishes
  // a group's copies also publishes the next group's table and frees the other buffer.
  static __device__ void run(const StageArgs& A) {
    const Smem M = carve();
    const InstArgs& I = A.inst;
    const Role r = role();
    load_ops(M.sm + OFF_D, A.Dv, I);
    const bool need_un = A.need_un != 0;
    const int ng = (I.n_elem + EPB - 1) / EPB;
    int g = blockIdx.x;
    if (g < ng) fill_nb(I, g, M.nb);
    if (g + (int)gridDim.x < ng) fill_nb(I, g + gridDim.x, M.nb + EPB * NF);
    __syncthreads();
    if (g < ng) issue(A, I, r, g, M.st, M.nb, need_un);
    cp_async_commit();
    for (int it = 0; g < ng; g += gridDim.x, ++it) {
      const int b = it & 1;
      const int gn = g + gridDim.x, gnn = gn + gridDim.x;
      cp_async_wait_all();
      __syncthreads();  // group g's copies are visible; every thread has left the previous group,
                        // so buffer b^1 and neighbour slot b are free
      if (gn < ng) issue(A, I, r, gn, M.st + (b ^ 1) * ST_SIZE, M.nb + (b ^ 1) * EPB * NF, need_un);
      cp_async_commit();
      if (gnn < ng) fill_nb(I, gnn, M.nb + b * EPB * NF);  // read by the next iteration's issue
      compute(A, I, M.sm, M.sm + OFF_D, r, g, M.st + b * ST_SIZE, need_un);
    }
  }
};

template <int DIM, int N, bool EC, class R>
__global__ void __launch_bounds__(EulerStage<DIM, N, EC, R>::T) k_euler_stage(const StageArgs A) {
  EulerStage<DIM, N, EC, R>::run(A);
}

}  // namespace dg
