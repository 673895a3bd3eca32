// dg_api.cu -- the C-ABI of include/dgsem.h: context lifecycle, operators, launches.
//
// Host side only.  The context owns three FP64 state buffers (the current state and two
// stage buffers, rotated so that no launch writes a buffer it reads; SSP-RK54 adds a fourth),
// the device error word, a scratch word for the time-step reduction, a private capture stream
// and the CUDA graph that replays three time steps (nine fused stage launches for SSP-RK3).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dgsem.h"
#include "dg_internal.h"

struct dg_ctx {
  std::vector<dg_mesh_desc> inst;
  dg_physics phys{};
  cudaStream_t stream = nullptr;     // caller's stream
  cudaStream_t cap = nullptr;        // private stream for graph capture
  int dim = 0, nv = 0;
  long long n_nodes_total = 0;
  std::vector<long long> offs;       // node offset per instance
  double* buf[4] = {nullptr, nullptr, nullptr, nullptr};  // buf[3]: SSP-RK54 only
  int cur = 0;                       // index of the buffer holding the current state
  bool rk54 = false;                 // SSP-RK54 (the state stays in buf[cur]); else SSP-RK3
  bool split = false;                // Strang-split implicit source (reacting)
  int tt = 0;                        // two-temperature model (reacting)
  unsigned* err = nullptr;
  unsigned long long* lam = nullptr;  // [0..1] time-step reductions, [2] Newton update count
  std::string msg;
  cudaGraphExec_t gexec = nullptr;   // three RK steps starting from buf[0]
  double g_dt = 0.0;
  // batched launch (several instances): work list and per-instance arguments on the device
  bool batched = false;
  dg::BatchConfig bcfg{1, 0, 0};
  dg::InstArgs* d_insts = nullptr;
  int2* d_items = nullptr;
  size_t items_cap = 0;
  int n_items = 0;
  int n_items_g1 = 0;  // items of the degrees launched with group scale 1 (the list's head)
  double* d_dv = nullptr;
  // adjoint workspace (allocated on the first adjoint call): recomputed stage states W1, W2,
  // co-state temporaries T1..T3, per-CTA gamma partials and their device accumulator
  double* adj[10] = {};               // adjoint workspace (SSP-RK54: all ten)
  double* gpart = nullptr;
  double* gacc = nullptr;
  // Navier-Stokes: mechanism (device copy), face buffer of the BR1 pass and its per-instance
  // offsets (doubles)
  bool ns = false;
  int n_species = 0;
  dg::MechDev* d_mech = nullptr;
  double* fb = nullptr;
  std::vector<long long> fb_offs;
  std::vector<dg::ReactBC> rbc;      // boundary conditions per instance (viscous equations)
  // primitive caches of the state buffers (slot 3 with SSP-RK54) and a scratch one (slot 4)
  // (flux-type rows, then the FP64 temperature), and whether each cache matches its
  // buffer's current contents
  void* pc[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  double* pT[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  bool pvalid[4] = {false, false, false, false};
  // shock capturing (Euler): per-element blending coefficients (raw and smoothed), the list
  // of blended elements and its length, the DG-residual side buffer, per-instance element
  // offsets
  // curved meshes: metric terms [dim*dim + 1][n_nodes_total] on the device, which instances
  // are curved, and their smallest element size for the time-step bound
  double* met = nullptr;
  std::vector<char> curved;
  std::vector<double> curved_dx;
  bool shock = false;
  double* alpha_raw = nullptr;
  double* alpha = nullptr;
  int* list = nullptr;
  int* count = nullptr;
  double* ldg = nullptr;
  std::vector<long long> eoffs;
};

namespace {

const char* kNullCtxMsg = "null context";

dg_status fail(dg_ctx* c, dg_status s, const std::string& m) {
  if (c) c->msg = m;
  return s;
}

dg_status cuda_fail(dg_ctx* c, cudaError_t e, const char* where) {
  return fail(c, DG_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------------------
// GLL rule and differentiation matrix (Sec. 3.1.1).  Interior nodes are the zeros of
// P_N', found by Newton's method with P_N'' from Legendre's equation
// (1-x^2) P'' = 2x P' - N(N+1) P; weights w_i = 2 / (N(N+1) P_N(x_i)^2).  The derivative
// matrix uses the closed form for Lobatto nodes:
//   D_ij = P_N(x_i) / (P_N(x_j) (x_i - x_j))  (i != j),  D_00 = -N(N+1)/4,
//   D_NN = N(N+1)/4, other diagonal entries 0.
// ---------------------------------------------------------------------------------------
void legendre_p(int N, double x, double& P, double& dP) {
  double pm = 1.0, p = x;  // P_0, P_1
  if (N == 0) { P = 1.0; dP = 0.0; return; }
  for (int k = 2; k <= N; ++k) {
    const double pn = ((2.0 * k - 1.0) * x * p - (k - 1.0) * pm) / k;
    pm = p;
    p = pn;
  }
  P = p;
  dP = (std::fabs(x) < 1.0) ? N * (pm - x * p) / (1.0 - x * x) : 0.0;
}

void gll_table(int N, double* x, double* w, double* D) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i <= N; ++i) {
    if (i == 0) { x[i] = -1.0; continue; }
    if (i == N) { x[i] = 1.0; continue; }
    double xi = -std::cos(pi * i / N);
    for (int it = 0; it < 60; ++it) {
      double P, dP;
      legendre_p(N, xi, P, dP);
      const double d2P = (2.0 * xi * dP - N * (N + 1.0) * P) / (1.0 - xi * xi);
      const double step = dP / d2P;
      xi -= step;
      if (std::fabs(step) < 1e-17) break;
    }
    x[i] = xi;
  }
  // symmetrise (the rule is symmetric about 0)
  for (int i = 0; i <= N / 2; ++i) {
    const double a = 0.5 * (x[N - i] - x[i]);
    x[i] = -a;
    x[N - i] = a;
  }
  if (N % 2 == 0) x[N / 2] = 0.0;
  std::vector<double> PN(N + 1);
  for (int i = 0; i <= N; ++i) {
    double P, dP;
    legendre_p(N, x[i], P, dP);
    PN[i] = P;
    w[i] = 2.0 / (N * (N + 1.0) * P * P);
  }
  if (D) {
    for (int i = 0; i <= N; ++i)
      for (int j = 0; j <= N; ++j)
        D[i * (N + 1) + j] = (i == j) ? 0.0 : PN[i] / (PN[j] * (x[i] - x[j]));
    D[0] = -N * (N + 1.0) / 4.0;
    D[N * (N + 1) + N] = N * (N + 1.0) / 4.0;
  }
}

dg_status check_desc(const dg_mesh_desc& m, int dim0, int equations, std::string& why) {
  const bool viscous = equations != DG_EULER;
  if (m.dim != 2 && m.dim != 3) { why = "dim must be 2 or 3"; return DG_EINVAL; }
  if (m.dim != dim0) { why = "all instances must have the same dim"; return DG_EINVAL; }
  if (m.N < 1) { why = "N must be >= 1"; return DG_EINVAL; }
  if (!dg::have_kernels(m.dim, m.N)) { why = "no kernels for this (dim, N)"; return DG_EUNSUPPORTED; }
  for (int l = 0; l < m.dim; ++l) {
    if (m.nel[l] < 1) { why = "nel must be >= 1"; return DG_EINVAL; }
    if (!(m.hi[l] > m.lo[l])) { why = "hi must exceed lo"; return DG_EINVAL; }
    if (m.periodic[l] != 1 && m.periodic[l] != 0) { why = "periodic must be 0 or 1"; return DG_EINVAL; }
    if (m.periodic[l] == 1) continue;
    for (int side = 0; side < 2; ++side) {
      const int f = 2 * l + side;
      const int top = viscous ? DG_BC_NOSLIP_ISOTHERMAL : DG_BC_DIRICHLET;
      if (m.bc[f] < DG_BC_SLIP_WALL || m.bc[f] > top) { why = "bad boundary type"; return DG_EINVAL; }
      if (viscous) {  // the prescribed states are checked against the mixture later
        if (m.bc[f] == DG_BC_NOSLIP_ISOTHERMAL &&
            !(m.bc_state[f][0] > 0.0 && std::isfinite(m.bc_state[f][0]))) {
          why = "the wall temperature must be > 0";
          return DG_EINVAL;
        }
        continue;
      }
      if (m.bc[f] == DG_BC_INFLOW || m.bc[f] == DG_BC_DIRICHLET) {
        const double* b = m.bc_state[f];
        double m2 = 0.0;
        for (int d = 0; d < m.dim; ++d) m2 += b[1 + d] * b[1 + d];
        bool ok = b[0] > 0.0 && std::isfinite(b[0]) && std::isfinite(m2) && std::isfinite(b[m.dim + 1]);
        ok = ok && b[m.dim + 1] - 0.5 * m2 / b[0] > 0.0;
        if (!ok) { why = "boundary state must have rho > 0 and p > 0"; return DG_EINVAL; }
      }
    }
  }
  const long long ne = (long long)m.nel[0] * m.nel[1] * (m.dim == 3 ? m.nel[2] : 1);
  if (ne > (1LL << 31) - 1) { why = "too many elements"; return DG_EINVAL; }
  return DG_OK;
}

// The kernels' copy of a mechanism: species data, per-reaction Arrhenius and K_c
// coefficients, the species of each side's concentration product (at most three molecules;
// index n_species stands for a factor 1) and the source coefficients W_s 1e6 (nu'' - nu').
// 2^(j/64), j = 0..63, rounded once from long double: the table of the device exp.
void fill_exp2_table(double* tab) {
  for (int j = 0; j < 64; ++j) tab[j] = (double)std::exp2((long double)j / 64.0L);
}

// tt: the two-temperature model -- vibrational temperatures (>= 0, one at least > 0), each
// reaction's controlling-temperature flag, and the Millikan-White coefficients of every
// (vibrating species s, collision partner r) pair: A_sr = 1.16e-3 mu_sr^1/2 theta_s^4/3,
// B_sr = 0.015 mu_sr^1/4 (mu_sr the reduced molar mass in g/mol), stored as A_sr and
// C_sr = A_sr B_sr + 18.42 (Millikan and White, J. Chem. Phys. 39, 1963).
dg_status pack_mechanism(const dg_mechanism& m, dg::MechDev& d, int tt, std::string& why) {
  std::memset(&d, 0, sizeof(d));
  if (m.n_species < 1 || m.n_species > DG_MAX_SPECIES || m.n_reactions < 0 ||
      m.n_reactions > DG_MAX_REACTIONS) {
    why = "species or reaction count out of range";
    return DG_EINVAL;
  }
  const int ns = m.n_species;
  d.ns = ns;
  d.nr = m.n_reactions;
  fill_exp2_table(d.exp2tab);
  for (int s = 0; s < ns; ++s) {
    if (!(m.W[s] > 0.0) || !(m.R[s] > 0.0) || !(m.cv[s] > 0.0) || !std::isfinite(m.h0[s]) ||
        !std::isfinite(m.W[s]) || !std::isfinite(m.R[s]) || !std::isfinite(m.cv[s])) {
      why = "species data must be finite with W, R, cv > 0";
      return DG_EINVAL;
    }
    d.R[s] = m.R[s];
    d.cv[s] = m.cv[s];
    d.h0[s] = m.h0[s];
    d.scale[s] = 1.0e-6 / m.W[s];
  }
  for (int r = 0; r < m.n_reactions; ++r) {
    dg::RxnDev& x = d.rx[r];
    x.lnA = m.lnA[r];
    x.b = m.b[r];
    x.Ta = m.Ta[r];
    bool ok = std::isfinite(x.lnA) && std::isfinite(x.b) && std::isfinite(x.Ta);
    for (int k = 0; k < 5; ++k) {
      x.kc[k] = m.kc[r][k];
      ok = ok && std::isfinite(x.kc[k]);
    }
    if (!ok) { why = "reaction coefficients must be finite"; return DG_EINVAL; }
    int nf = 0, nb = 0;
    for (int k = 0; k < 3; ++k) x.f[k] = x.bk[k] = ns;
    for (int s = 0; s < ns; ++s) {
      if (m.nu_f[r][s] < 0 || m.nu_b[r][s] < 0) { why = "negative stoichiometric coefficient"; return DG_EINVAL; }
      for (int k = 0; k < m.nu_f[r][s]; ++k) {
        if (nf == 3) { why = "more than 3 molecules on one side of a reaction"; return DG_EUNSUPPORTED; }
        x.f[nf++] = s;
      }
      for (int k = 0; k < m.nu_b[r][s]; ++k) {
        if (nb == 3) { why = "more than 3 molecules on one side of a reaction"; return DG_EUNSUPPORTED; }
        x.bk[nb++] = s;
      }
      x.coef[s] = m.W[s] * 1.0e6 * (double)(m.nu_b[r][s] - m.nu_f[r][s]);
    }
    if (tt) {
      if (m.ta_mode[r] != 0 && m.ta_mode[r] != 1) { why = "ta_mode must be 0 or 1"; return DG_EINVAL; }
      x.ta = m.ta_mode[r];
    }
  }
  if (tt) {
    bool any = false;
    for (int s = 0; s < ns; ++s) {
      if (!(m.theta_v[s] >= 0.0) || !std::isfinite(m.theta_v[s])) { why = "theta_v must be finite and >= 0"; return DG_EINVAL; }
      d.theta[s] = m.theta_v[s];
      any = any || m.theta_v[s] > 0.0;
    }
    if (!any) { why = "the two-temperature model needs a vibrating species"; return DG_EINVAL; }
    for (int s = 0; s < ns; ++s)
      for (int r = 0; r < ns; ++r) {
        if (!(d.theta[s] > 0.0)) continue;
        const double Ws = m.W[s] * 1.0e3, Wr = m.W[r] * 1.0e3;
        const double mu = Ws * Wr / (Ws + Wr);
        const double A = 1.16e-3 * std::sqrt(mu) * std::pow(d.theta[s], 4.0 / 3.0);
        d.mwA[s][r] = A;
        d.mwC[s][r] = A * 0.015 * std::pow(mu, 0.25) + 18.42;
      }
  }
  return DG_OK;
}

long long n_elem_of(const dg_mesh_desc& m) {
  return (long long)m.nel[0] * m.nel[1] * (m.dim == 3 ? m.nel[2] : 1);
}
int n_p_of(const dg_mesh_desc& m) {
  int n = 1;
  for (int l = 0; l < m.dim; ++l) n *= (m.N + 1);
  return n;
}

// The volume operator of degree N for this context's volume form, row-major (N+1)^2.
void volume_operator(const dg_ctx* c, int N, double* Dv, double* lift) {
  const int n1 = N + 1;
  double x[dg::kMaxN + 1], w[dg::kMaxN + 1], D[(dg::kMaxN + 1) * (dg::kMaxN + 1)];
  gll_table(N, x, w, D);
  for (int r = 0; r < n1; ++r)
    for (int k = 0; k < n1; ++k) {
      double v;
      if (c->phys.volume == DG_VOL_WEAK) v = -(w[k] / w[r]) * D[k * n1 + r];
      else if (c->phys.volume == DG_VOL_EC) v = 2.0 * D[r * n1 + k];
      else v = D[r * n1 + k];
      Dv[r * n1 + k] = v;
    }
  if (lift) *lift = 1.0 / w[0];
}

// Nodal -> orthonormal Legendre modes on the GLL nodes (Sec. 3.1.1 "Shock Indicator"; the
// Hennemann-Gassner indicator's modal decomposition): Vinv = V^{-1}, V_ij = P~_j(x_i),
// P~_j = sqrt((2j+1)/2) P_j, inverted by Gauss-Jordan in long double.
void modal_inverse(int N, double* Vinv) {
  const int n1 = N + 1;
  double x[dg::kMaxN + 1], w[dg::kMaxN + 1];
  gll_table(N, x, w, nullptr);
  long double A[dg::kMaxN + 1][2 * (dg::kMaxN + 1)];
  for (int i = 0; i < n1; ++i) {
    long double pm = 1.0L, p = x[i];  // P_0, P_1
    for (int j = 0; j < n1; ++j) {
      long double Pj;
      if (j == 0) Pj = 1.0L;
      else if (j == 1) Pj = x[i];
      else {
        const long double pn = ((2.0L * j - 1.0L) * x[i] * p - (j - 1.0L) * pm) / j;
        pm = p;
        p = pn;
        Pj = pn;
      }
      A[i][j] = std::sqrt((2.0L * j + 1.0L) / 2.0L) * Pj;
      A[i][n1 + j] = (i == j) ? 1.0L : 0.0L;
    }
  }
  for (int k = 0; k < n1; ++k) {
    int piv = k;
    for (int i = k + 1; i < n1; ++i)
      if (std::fabs(A[i][k]) > std::fabs(A[piv][k])) piv = i;
    for (int j = 0; j < 2 * n1; ++j) std::swap(A[k][j], A[piv][j]);
    const long double d = A[k][k];
    for (int j = 0; j < 2 * n1; ++j) A[k][j] /= d;
    for (int i = 0; i < n1; ++i) {
      if (i == k) continue;
      const long double f = A[i][k];
      for (int j = 0; j < 2 * n1; ++j) A[i][j] -= f * A[k][j];
    }
  }
  for (int i = 0; i < n1; ++i)
    for (int j = 0; j < n1; ++j) Vinv[i * n1 + j] = (double)A[i][n1 + j];
}

// Metric terms of a curved instance (Sec. 3.1.1: element maps interpolating the node
// coordinates, contravariant vectors Ja^l with the discrete GCL): 2D Ja^1 = (y_eta, -x_eta),
// Ja^2 = (-y_xi, x_xi); 3D the conservative curl form
// Ja^i_n = -1/2 [curl_xi (X_l grad_xi X_m - X_m grad_xi X_l)]_i, (n, m, l) cyclic; derivatives
// by D along the lines; J the determinant of dx/dxi.  Writes met[c][base + node] (c = l*dim + d,
// then 1/J at c = dim*dim) with the given node stride; returns false if some J <= 0, and the
// smallest 2 J / |Ja^l| over nodes and directions in dxmin.
bool curved_metrics_host(const dg_mesh_desc& m, double* met, long long stride, long long base,
                         double& dxmin) {
  const int dim = m.dim, N = m.N, n1 = N + 1;
  const int np = dim == 2 ? n1 * n1 : n1 * n1 * n1;
  const long long ne = n_elem_of(m);
  double x[dg::kMaxN + 1], w[dg::kMaxN + 1], D[(dg::kMaxN + 1) * (dg::kMaxN + 1)];
  gll_table(N, x, w, D);
  auto pos = [&](int q, int k) { return k == 0 ? q % n1 : (k == 1 ? (q / n1) % n1 : q / (n1 * n1)); };
  auto strd = [&](int k) { return k == 0 ? 1 : (k == 1 ? n1 : n1 * n1); };
  auto deriv = [&](const std::vector<double>& f, int k, int q) {
    const int i = pos(q, k), S = strd(k), b = q - i * S;
    double acc = 0.0;
    for (int j = 0; j < n1; ++j) acc += D[i * n1 + j] * f[b + j * S];
    return acc;
  };
  dxmin = INFINITY;
  for (long long e = 0; e < ne; ++e) {
    std::vector<std::vector<double>> X(dim, std::vector<double>(np));
    for (int d = 0; d < dim; ++d)
      for (int q = 0; q < np; ++q) X[d][q] = m.coords[((size_t)d * ne + e) * np + q];
    std::vector<double> g((size_t)np * 9, 0.0), Ja((size_t)np * 9, 0.0);  // g[q][d][k] = dx_d/dxi_k
    for (int q = 0; q < np; ++q)
      for (int d = 0; d < dim; ++d)
        for (int k = 0; k < dim; ++k) g[(size_t)q * 9 + d * 3 + k] = deriv(X[d], k, q);
    if (dim == 2) {
      for (int q = 0; q < np; ++q) {
        const double* G = &g[(size_t)q * 9];
        Ja[q * 9 + 0] = G[4];   // l = 0: ( y_eta, -x_eta)
        Ja[q * 9 + 1] = -G[1];
        Ja[q * 9 + 3] = -G[3];  // l = 1: (-y_xi,  x_xi)
        Ja[q * 9 + 4] = G[0];
      }
    } else {
      for (int n = 0; n < 3; ++n) {
        const int mm = (n + 1) % 3, ll = (n + 2) % 3;
        std::vector<std::vector<double>> V(3, std::vector<double>(np));
        for (int q = 0; q < np; ++q)
          for (int k = 0; k < 3; ++k)
            V[k][q] = X[ll][q] * g[(size_t)q * 9 + mm * 3 + k] - X[mm][q] * g[(size_t)q * 9 + ll * 3 + k];
        for (int q = 0; q < np; ++q)
          for (int i = 0; i < 3; ++i) {
            const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
            Ja[q * 9 + i * 3 + n] = -0.5 * (deriv(V[i2], i1, q) - deriv(V[i1], i2, q));
          }
      }
    }
    for (int q = 0; q < np; ++q) {
      const double* G = &g[(size_t)q * 9];
      const double J = dim == 2 ? G[0] * G[4] - G[1] * G[3]
                                : G[0] * (G[4] * G[8] - G[5] * G[7]) - G[1] * (G[3] * G[8] - G[5] * G[6]) +
                                      G[2] * (G[3] * G[7] - G[4] * G[6]);
      if (!(J > 0.0)) return false;
      const long long gi = base + e * np + q;
      for (int l = 0; l < dim; ++l) {
        double s2 = 0.0;
        for (int d = 0; d < dim; ++d) {
          met[(size_t)(l * dim + d) * stride + gi] = Ja[q * 9 + l * 3 + d];
          s2 += Ja[q * 9 + l * 3 + d] * Ja[q * 9 + l * 3 + d];
        }
        dxmin = std::fmin(dxmin, 2.0 * J / std::sqrt(s2));
      }
      met[(size_t)dim * dim * stride + gi] = 1.0 / J;
    }
  }
  return true;
}

// The kernels' copy of instance m's boundary conditions for the viscous equations: the
// prescribed states of inflow and Dirichlet faces with their (u, v, w, T, p - p_ref, a) from
// the mixture of `mech` (the kernels' closure), the wall temperature of isothermal walls.
// Two-temperature (tt): the prescribed state carries E_v, T excludes it, and T_v solves
// E_v = sum rho_s e_v,s(T_v) (bisection to the last bit; E_v grows strictly with T_v); the
// isothermal wall holds T_v at T_wall.
// False (why set) when a prescribed state is not finite or has rho <= 0 or T <= 0 (or T_v).
bool react_bc(const dg_mesh_desc& m, const dg::MechDev& mech, double p_ref, int tt, dg::ReactBC& b,
              std::string& why) {
  std::memset(&b, 0, sizeof(b));
  const int ns = mech.ns;
  for (int l = 0; l < 3; ++l) {
    if (m.periodic[l] == 1) continue;
    b.nonper = 1;
    for (int side = 0; side < 2; ++side) {
      const int f = 2 * l + side;
      b.bc[f] = m.bc[f];
      if (m.bc[f] == DG_BC_NOSLIP_ISOTHERMAL) b.bcw[f][3] = b.bcw[f][6] = m.bc_state[f][0];
      if (m.bc[f] != DG_BC_INFLOW && m.bc[f] != DG_BC_DIRICHLET) continue;
      const double* u = m.bc_state[f];
      bool ok = true;
      for (int v = 0; v < ns + 4 + tt; ++v) {
        b.bcu[f][v] = u[v];
        ok = ok && std::isfinite(u[v]);
      }
      double rho = 0.0, rR = 0.0, rcv = 0.0, rh0 = 0.0;
      for (int s = 0; s < ns; ++s) {
        rho += u[s];
        rR += u[s] * mech.R[s];
        rcv += u[s] * mech.cv[s];
        rh0 += u[s] * mech.h0[s];
      }
      ok = ok && rho > 0.0 && rcv > 0.0;
      if (ok) {
        double kin = 0.0;
        for (int d = 0; d < 3; ++d) {
          b.bcw[f][d] = u[ns + d] / rho;
          kin += u[ns + d] * b.bcw[f][d];
        }
        const double Ev = tt ? u[ns + 4] : 0.0;
        const double T = (u[ns + 3] - Ev - 0.5 * kin - rh0) / rcv, p = rR * T;
        ok = T > 0.0 && std::isfinite(T);
        b.bcw[f][3] = T;
        b.bcw[f][4] = p - p_ref;
        b.bcw[f][5] = std::sqrt((1.0 + rR / rcv) * p / rho);
        b.bcw[f][6] = T;
        if (tt) {
          auto ev = [&](double x) {
            double e = 0.0;
            for (int s = 0; s < ns; ++s)
              if (mech.theta[s] > 0.0) e += u[s] * mech.R[s] * mech.theta[s] / std::expm1(mech.theta[s] / x);
            return e;
          };
          double lo = 1e-3, hi = 1e7;
          ok = ok && Ev > 0.0 && ev(hi) > Ev;
          for (int it = 0; ok && it < 200; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            if (ev(mid) < Ev) lo = mid;
            else hi = mid;
          }
          b.bcw[f][6] = 0.5 * (lo + hi);
        }
      }
      if (!ok) {
        why = "boundary state must be finite with rho > 0 and T > 0";
        return false;
      }
    }
  }
  return true;
}

// The kernels' view of instance i.
void inst_args(const dg_ctx* c, int i, dg::InstArgs& I) {
  const dg_mesh_desc& m = c->inst[i];
  std::memset(&I, 0, sizeof(I));
  I.base = c->offs[i];
  for (int l = 0; l < m.dim; ++l) {
    if (m.periodic[l] == 1) continue;
    for (int side = 0; side < 2; ++side) {
      const int f = 2 * l + side;
      I.bc[f] = m.bc[f];
      for (int v = 0; v < 5; ++v) I.bcs[f][v] = m.bc_state[f][v];
    }
    I.nonper = 1;
  }
  for (int l = 0; l < 3; ++l) {
    I.nel[l] = (l < m.dim) ? m.nel[l] : 1;
    I.s[l] = (l < m.dim) ? 2.0 / ((m.hi[l] - m.lo[l]) / m.nel[l]) : 0.0;
    I.sf[l] = (float)I.s[l];
  }
  I.n_elem = (int)n_elem_of(m);
  I.N = m.N;
  double D[(dg::kMaxN + 1) * (dg::kMaxN + 1)];
  volume_operator(c, m.N, D, &I.lift);
  I.liftf = (float)I.lift;
}

// Coefficients of one Shu-Osher stage update (App. B), with X = U^n or a running sum:
//   out = ca X + cb U + bdt L(U)                  (bdt = beta dt)
//   acc = acc_a acc + acc_b U + acc_bdt L(U)      (only when acc is not null)
struct StageCoef {
  double ca = 0.0, cb = 0.0, bdt = 0.0;
  double* acc = nullptr;
  double acc_a = 0.0, acc_b = 0.0, acc_bdt = 0.0;
};

// Launch-wide fields (state pointers, stage coefficients, physics) and the host-precomputed
// scalars in both precisions.
void launch_args(const dg_ctx* c, dg::StageArgs& a, const double* U, const double* Un, double* out,
                 int mode, const StageCoef& k) {
  std::memset(&a, 0, sizeof(a));
  a.U = U;
  a.Un = Un;
  a.out = out;
  a.err = c->err;
  a.work = c->err + 2;
  a.stride = c->n_nodes_total;
  a.gamma = c->phys.gamma;
  a.ca = k.ca;
  a.cb = k.cb;
  a.dt = k.bdt;
  a.acc = k.acc;
  a.acc_a = k.acc_a;
  a.acc_b = k.acc_b;
  a.mode = mode;
  a.surface = c->phys.surface;
  a.weak = (c->phys.volume == DG_VOL_WEAK) ? 1 : 0;
  a.rho_floor = c->phys.rho_floor;
  a.p_floor = c->phys.p_floor;
  a.p_ref = c->phys.p_ref;
  dg::fill_scalars(a.pd, a.pf, a.gamma, a.p_ref, k.bdt, k.acc_bdt);
  a.need_un = (mode == 1 && k.ca != 0.0) ? 1 : 0;
  a.floor_on = (a.rho_floor > 0.0 || a.p_floor > 0.0) ? 1 : 0;
}

// One fused stage over all instances: mode 0 writes L(U), mode 1 the stage update.  One
// launch per instance, or one batched launch for all of them.
// Which context state buffer p is (0..3), or -1 for a caller buffer.
int buf_index(const dg_ctx* c, const double* p) {
  for (int b = 0; b < 4; ++b)
    if (p && c->buf[b] == p) return b;
  return -1;
}
constexpr int kScratch = 4;  // primitive cache slot of states that are not context buffers

// Fill primitive cache slot k (0..2: a state buffer's, 3: scratch) from state U.
dg_status fill_prims(dg_ctx* c, const double* U, int k, cudaStream_t s) {
  const int fp32 = c->phys.precision == DG_FP32_MIXED;
  for (size_t i = 0; i < c->inst.size(); ++i) {
    cudaError_t e = dg::launch_react_prims(c->n_species, c->tt, fp32, U, c->n_nodes_total, c->offs[i],
                                           n_elem_of(c->inst[i]) * n_p_of(c->inst[i]), c->d_mech,
                                           c->phys.p_ref, c->pc[k], c->pT[k], c->err, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "primitive cache launch");
  }
  return DG_OK;
}

dg_status run_stage_ns(dg_ctx* c, const double* U, const double* Un, double* out, int mode,
                       const StageCoef& k, cudaStream_t s) {
  dg::ReactArgs a;
  std::memset(&a, 0, sizeof(a));
  // the input's primitive cache: its buffer's if valid, else computed now
  const int bin = buf_index(c, U);
  const int kin = bin >= 0 ? bin : kScratch;
  if (bin < 0 || !c->pvalid[bin]) {
    dg_status st = fill_prims(c, U, kin, s);
    if (st) return st;
    if (bin >= 0) c->pvalid[bin] = true;
  }
  a.pin = c->pc[kin];
  a.tin = c->pT[kin];
  // the output's cache, written by the stage kernel when the output is a context buffer
  const int bout = buf_index(c, out);
  if (bout >= 0) {
    if (mode == 1) {
      a.pout = c->pc[bout];
      a.tout = c->pT[bout];
    }
    c->pvalid[bout] = (mode == 1);
  }
  const int bacc = buf_index(c, k.acc);
  if (bacc >= 0) c->pvalid[bacc] = false;
  a.U = U;
  a.Un = Un;
  a.out = out;
  a.err = c->err;
  a.mech = c->d_mech;
  a.stride = c->n_nodes_total;
  a.mode = mode;
  a.need_un = (mode == 1 && k.ca != 0.0) ? 1 : 0;
  a.src = c->split ? 0 : 1;
  a.ca = k.ca;
  a.cb = k.cb;
  a.cbdt = k.bdt;
  a.acc = k.acc;
  a.acc_a = k.acc_a;
  a.acc_b = k.acc_b;
  a.acc_bdt = k.acc_bdt;
  a.mu = c->phys.mu;
  a.kfac = c->phys.mu / c->phys.prandtl;
  a.p_ref = c->phys.p_ref;
  a.ln1e4 = std::log(1.0e4);
  a.muf = (float)a.mu;
  a.kfacf = (float)a.kfac;
  a.p_reff = (float)a.p_ref;
  const int fp32 = c->phys.precision == DG_FP32_MIXED;
  for (size_t i = 0; i < c->inst.size(); ++i) {
    const dg_mesh_desc& m = c->inst[i];
    a.base = c->offs[i];
    a.fb = c->fb + c->fb_offs[i];
    a.bnd = c->rbc[i];
    for (int l = 0; l < 3; ++l) {
      a.nel[l] = m.nel[l];
      a.s[l] = 2.0 / ((m.hi[l] - m.lo[l]) / m.nel[l]);
      a.sf[l] = (float)a.s[l];
    }
    a.n_elem = (int)n_elem_of(m);
    const bool curved = !c->curved.empty() && c->curved[i];
    a.met = curved ? c->met : nullptr;
    if (curved)  // the 2/dx_l of the element map are part of the metric terms
      for (int l = 0; l < 3; ++l) {
        a.s[l] = 1.0;
        a.sf[l] = 1.0f;
      }
    double x[dg::kMaxN + 1], w[dg::kMaxN + 1];
    gll_table(m.N, x, w, a.D);
    a.lift = 1.0 / w[0];
    a.liftf = (float)a.lift;
    cudaError_t e = dg::launch_reacting(m.N, c->n_species, c->tt, fp32, a, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "Navier-Stokes stage launch");
    if (mode == 1 && c->phys.species_limiter) {  // Zhang-Shu limiter of the stage's output
      dg::LimiterArgs la;
      std::memset(&la, 0, sizeof(la));
      la.U = out;
      la.pout = a.pout;
      la.tout = a.tout;
      la.err = c->err;
      la.mech = c->d_mech;
      la.stride = a.stride;
      la.base = a.base;
      la.n_elem = a.n_elem;
      la.np = n_p_of(m);
      la.p_ref = c->phys.p_ref;
      double wsum = 0.0;
      for (int q = 0; q < la.np; ++q) {
        const int i = q % (m.N + 1), j = (q / (m.N + 1)) % (m.N + 1), kk = q / ((m.N + 1) * (m.N + 1));
        la.wq[q] = w[i] * w[j] * w[kk];
        wsum += la.wq[q];
      }
      for (int q = 0; q < la.np; ++q) la.wq[q] /= wsum;
      e = dg::launch_species_limiter(c->n_species, c->tt, fp32, la, s);
      if (e != cudaSuccess) return cuda_fail(c, e, "species limiter launch");
    }
  }
  return DG_OK;
}

// Shock-capturing arguments of instance i for one stage (the stage launch's own arguments a
// supply the precomputed scalars).
void shock_args(const dg_ctx* c, int i, const dg::StageArgs& a, const StageCoef& k, dg::ShockArgs& sa) {
  std::memset(&sa, 0, sizeof(sa));
  const dg_mesh_desc& m = c->inst[i];
  sa.U = a.U;
  sa.Un = a.Un;
  sa.out = a.out;
  sa.ldg = a.mode == 1 ? c->ldg : a.out;
  sa.acc = k.acc;
  sa.acc_a = k.acc_a;
  sa.acc_b = k.acc_b;
  sa.acc_bdt = k.acc_bdt;
  sa.err = c->err;
  sa.stride = c->n_nodes_total;
  inst_args(c, i, sa.inst);
  sa.mode = a.mode;
  sa.need_un = a.need_un;
  sa.surface = c->phys.surface;
  sa.floor_on = a.floor_on;
  sa.ca = k.ca;
  sa.cb = k.cb;
  sa.bdt = k.bdt;
  sa.gamma = c->phys.gamma;
  sa.rho_floor = c->phys.rho_floor;
  sa.p_floor = c->phys.p_floor;
  sa.pd = a.pd;
  sa.pf = a.pf;
  double x[dg::kMaxN + 1], w[dg::kMaxN + 1];
  gll_table(m.N, x, w, nullptr);
  for (int j = 0; j <= m.N; ++j) {
    sa.iw[j] = 1.0 / w[j];
    sa.iwf[j] = (float)sa.iw[j];
  }
  modal_inverse(m.N, sa.Vinv);
  sa.thr = 0.5 * std::pow(10.0, -1.8 * std::pow(m.N + 1.0, 0.25));
  sa.sharp = c->phys.sharpness;
  sa.alpha_min = c->phys.alpha_min;
  sa.alpha_max = c->phys.alpha_max;
  // sigmoid(E) < alpha_min  <=>  E < T + (T/s) ln(alpha_min / (1 - alpha_min))
  sa.emin = (sa.alpha_min > 0.0 && sa.alpha_min < 1.0)
                ? sa.thr + (sa.thr / sa.sharp) * std::log(sa.alpha_min / (1.0 - sa.alpha_min))
                : -INFINITY;
  sa.alpha_raw = c->alpha_raw + c->eoffs[i];
  sa.alpha = c->alpha + c->eoffs[i];
  sa.list = c->list;
  sa.count = c->count;
}

// Indicator and neighbourhood maximum of instance i on state U (resets the list).
dg_status run_indicator(dg_ctx* c, int i, const dg::ShockArgs& sa, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(c->count, 0, sizeof(int), s);
  if (e == cudaSuccess) e = dg::launch_shock_indicator(c->inst[i].dim, c->inst[i].N, sa, s);
  return e == cudaSuccess ? DG_OK : cuda_fail(c, e, "shock indicator launch");
}

dg_status run_stage(dg_ctx* c, const double* U, const double* Un, double* out, int mode,
                    const StageCoef& k, cudaStream_t s) {
  if (c->ns) return run_stage_ns(c, U, Un, out, mode, k, s);
  const int ec = c->phys.volume == DG_VOL_EC, fp32 = c->phys.precision == DG_FP32_MIXED;
  dg::StageArgs a;
  launch_args(c, a, U, Un, out, mode, k);
  if (c->shock) {
    // per instance: indicator -> stage (blended elements only write L_DG) -> FV + blend
    for (size_t i = 0; i < c->inst.size(); ++i) {
      dg::ShockArgs sa;
      shock_args(c, (int)i, a, k, sa);
      dg_status st = run_indicator(c, (int)i, sa, s);
      if (st) return st;
      dg::StageArgs b = a;
      inst_args(c, (int)i, b.inst);
      volume_operator(c, c->inst[i].N, b.Dv, nullptr);
      b.alpha = sa.alpha;
      b.ldg = c->ldg;
      cudaError_t e = dg::launch_euler_stage(c->inst[i].dim, c->inst[i].N, ec, fp32, b, s);
      if (e == cudaSuccess) e = dg::launch_shock_blend(c->inst[i].dim, c->inst[i].N, fp32, sa, s);
      if (e != cudaSuccess) return cuda_fail(c, e, "shock-captured stage launch");
    }
    return DG_OK;
  }
  if (c->batched) {
    // one persistent launch per group-scale class: the degrees with group scale 1 (the head
    // of the work list), then those with group scale 2 (per-degree choice, 2D)
    a.insts = c->d_insts;
    a.dv_table = c->d_dv;
    cudaError_t e = cudaSuccess;
    if (c->n_items_g1 > 0) {
      a.items = c->d_items;
      a.n_items = c->n_items_g1;
      e = dg::launch_euler_stage_batched(c->dim, ec, fp32, 1, c->bcfg.ctas_per_sm, a, s);
    }
    if (e == cudaSuccess && c->n_items > c->n_items_g1) {
      a.items = c->d_items + c->n_items_g1;
      a.n_items = c->n_items - c->n_items_g1;
      e = dg::launch_euler_stage_batched(c->dim, ec, fp32, 2, c->bcfg.ctas_per_sm, a, s);
    }
    return e == cudaSuccess ? DG_OK : cuda_fail(c, e, "batched stage launch");
  }
  for (size_t i = 0; i < c->inst.size(); ++i) {
    inst_args(c, (int)i, a.inst);
    cudaError_t e;
    if (!c->curved.empty() && c->curved[i]) {  // curved instance: plain D, metric terms
      double x[dg::kMaxN + 1], w[dg::kMaxN + 1];
      gll_table(c->inst[i].N, x, w, a.Dv);
      e = dg::launch_curved(c->inst[i].dim, c->inst[i].N, ec, fp32, &a, c->met, s);
    } else {
      volume_operator(c, c->inst[i].N, a.Dv, nullptr);
      e = dg::launch_euler_stage(c->inst[i].dim, c->inst[i].N, ec, fp32, a, s);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "stage launch");
  }
  return DG_OK;
}

// (Re)build the batched work list for the current configuration: one item per element group
// of every instance, ordered heaviest first (nodes per item, then instance) or in instance
// order.  Device arrays are allocated once (sized for the smallest group) and reused.
dg_status build_batch(dg_ctx* c) {
  const int n = (int)c->inst.size();
  std::vector<dg::InstArgs> insts(n);
  for (int i = 0; i < n; ++i) inst_args(c, i, insts[i]);
  struct Item { int inst, group; long long cost; };
  std::vector<Item> items, items2;  // group scale 1, group scale 2
  for (int i = 0; i < n; ++i) {
    const int gs = dg::group_scale_of(c->bcfg, c->inst[i].N);
    const int gsz = dg::batched_group(c->dim, c->inst[i].N, gs);
    const int ng = (insts[i].n_elem + gsz - 1) / gsz;
    const long long cost = (long long)gsz * n_p_of(c->inst[i]) * (c->inst[i].N + 1);
    for (int g = 0; g < ng; ++g) (gs == 2 ? items2 : items).push_back({i, g, cost});
  }
  if (c->bcfg.order == 0) {
    auto heavier = [](const Item& x, const Item& y) { return x.cost > y.cost; };
    std::stable_sort(items.begin(), items.end(), heavier);
    std::stable_sort(items2.begin(), items2.end(), heavier);
  }
  c->n_items_g1 = (int)items.size();
  items.insert(items.end(), items2.begin(), items2.end());
  std::vector<int2> host(items.size());
  for (size_t k = 0; k < items.size(); ++k) host[k] = make_int2(items[k].inst, items[k].group);
  const size_t cap = items.size();
  if (!c->d_insts) {
    if (cudaMalloc(&c->d_insts, sizeof(dg::InstArgs) * n) != cudaSuccess) return fail(c, DG_ENOMEM, "batch");
    const int nd = (dg::kMaxN + 1) * (dg::kMaxN + 1) * (dg::kMaxN + 1);
    if (cudaMalloc(&c->d_dv, sizeof(double) * nd) != cudaSuccess) return fail(c, DG_ENOMEM, "batch");
    std::vector<double> dv(nd, 0.0);
    for (int N = 1; N <= dg::kMaxN; ++N) volume_operator(c, N, dv.data() + N * (dg::kMaxN + 1) * (dg::kMaxN + 1), nullptr);
    cudaError_t e = cudaMemcpy(c->d_dv, dv.data(), sizeof(double) * nd, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "batch operators");
  }
  if (cap > c->items_cap) {
    if (c->d_items) cudaFree(c->d_items);
    c->d_items = nullptr;
    if (cudaMalloc(&c->d_items, sizeof(int2) * cap) != cudaSuccess) return fail(c, DG_ENOMEM, "batch items");
    c->items_cap = cap;
  }
  cudaError_t e = cudaMemcpy(c->d_insts, insts.data(), sizeof(dg::InstArgs) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_items, host.data(), sizeof(int2) * cap, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(c, e, "batch upload");
  c->n_items = (int)cap;
  const int ec = c->phys.volume == DG_VOL_EC, fp32 = c->phys.precision == DG_FP32_MIXED;
  if (c->n_items_g1 > 0) e = dg::prepare_euler_stage_batched(c->dim, ec, fp32, 1);
  if (e == cudaSuccess && c->n_items > c->n_items_g1) e = dg::prepare_euler_stage_batched(c->dim, ec, fp32, 2);
  if (e != cudaSuccess) return cuda_fail(c, e, "batched kernel set-up");
  return DG_OK;
}

// ---- adjoint ----
dg_status ensure_adjoint(dg_ctx* c) {
  if (c->shock) return fail(c, DG_EUNSUPPORTED, "the adjoint has no shock capturing");
  for (const dg_mesh_desc& m : c->inst) {
    if (m.coords) return fail(c, DG_EUNSUPPORTED, "the adjoint covers affine meshes");
  }
  if (c->phys.surface != DG_SURF_RUSANOV && c->phys.surface != DG_SURF_HLLC)
    return fail(c, DG_EUNSUPPORTED, "the adjoint covers the Rusanov and HLLC surface fluxes");

  if (c->gacc) return DG_OK;
  const size_t bytes = sizeof(double) * (size_t)c->nv * c->n_nodes_total;
  int maxb = 1;
  for (const dg_mesh_desc& m : c->inst) maxb = std::max(maxb, dg::vjp_blocks(m.dim, m.N, n_elem_of(m)));
  for (int k = 0; k < (c->rk54 ? 10 : 5); ++k)
    if (cudaMalloc(&c->adj[k], bytes) != cudaSuccess) { cudaGetLastError(); return fail(c, DG_ENOMEM, "adjoint workspace"); }
  if (cudaMalloc(&c->gpart, sizeof(double) * maxb) != cudaSuccess ||
      cudaMalloc(&c->gacc, sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, DG_ENOMEM, "adjoint workspace");
  }
  if (cudaMemsetAsync(c->gacc, 0, sizeof(double), c->stream) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, DG_ECUDA, "adjoint workspace");
  }
  return DG_OK;
}

// One adjoint launch per instance (see dg::VjpArgs for the modes).
dg_status run_vjp(dg_ctx* c, const double* U, const double* lam, double* out, int mode, double bcoef,
                  double dt, const double* accin, double* accupd, int acc_init, double acoef, double gw) {
  for (size_t i = 0; i < c->inst.size(); ++i) {
    dg::VjpArgs a;
    std::memset(&a, 0, sizeof(a));
    a.U = U;
    a.lam = lam;
    a.out = out;
    a.accin = accin;
    a.accupd = accupd;
    a.acc_init = acc_init;
    a.gpart = c->gpart;
    a.stride = c->n_nodes_total;
    inst_args(c, (int)i, a.inst);
    volume_operator(c, c->inst[i].N, a.Dv, nullptr);
    a.gamma = c->phys.gamma;
    a.dt = dt;
    a.bcoef = bcoef;
    a.acoef = acoef;
    a.gw = gw;
    a.mode = mode;
    a.weak = (c->phys.volume == DG_VOL_WEAK) ? 1 : 0;
    const int sch = (c->phys.volume == DG_VOL_EC ? 1 : 0) | (c->phys.surface == DG_SURF_HLLC ? 2 : 0);
    cudaError_t e = dg::launch_rhs_vjp(c->dim, c->inst[i].N, c->phys.precision == DG_FP32_MIXED, sch, a,
                                       c->gacc, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "adjoint launch");
  }
  return DG_OK;
}

// Hand the device gamma accumulator to the host: sync, *gammabar += it, reset it.  With a
// null gammabar nothing happens (the contribution stays on the device for a later call).
dg_status read_gacc(dg_ctx* c, double* gammabar) {
  if (!gammabar) return DG_OK;
  double g = 0.0;
  cudaError_t e = cudaMemcpyAsync(&g, c->gacc, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->gacc, 0, sizeof(double), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint gamma read");
  *gammabar += g;
  return DG_OK;
}

void drop_graph(dg_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
}

const double kStageA[3] = {0.0, 0.75, 1.0 / 3.0};
const double kStageB[3] = {1.0, 0.25, 2.0 / 3.0};

StageCoef rk3_coef(int stage, double dt) {  // stage 0..2
  StageCoef k;
  k.ca = kStageA[stage];
  k.cb = kStageB[stage];
  k.bdt = kStageB[stage] * dt;
  return k;
}

// SSP-RK54 of Spiteri and Ruuth (SIAM J. Numer. Anal. 40(2), 2002), the paper's production
// integrator (App. B; it names the scheme and its SSP coefficient, not the coefficients),
// in Shu-Osher form with the published 15-digit values.  Non-zero entries only:
//   U1 = U0 + b10 dt L(U0)
//   U2 = a20 U0 + a21 U1 + b21 dt L(U1)
//   U3 = a30 U0 + a32 U2 + b32 dt L(U2)
//   U4 = a40 U0 + a43 U3 + b43 dt L(U3)
//   U5 = a52 U2 + a53 U3 + b53 dt L(U3) + a54 U4 + b54 dt L(U4)
struct Ssp54 {
  double b10, a20, a21, b21, a30, a32, b32, a40, a43, b43, a52, a53, b53, a54, b54;
};
constexpr Ssp54 kRk54 = {0.391752226571890, 0.444370493651235, 0.555629506348765,
                         0.368410593050371, 0.620101851488403, 0.379898148511597,
                         0.251891774271694, 0.178079954393132, 0.821920045606868,
                         0.544974750228521, 0.517231671970585, 0.096059710526147,
                         0.063692468666290, 0.386708617503269, 0.226007483236906};

// SSP coefficient (App. B, c~ = min alpha_ik / beta_ik over beta_ik > 0) of the context's scheme.
double ssp_coefficient(const dg_ctx* c) {
  if (!c->rk54) return 1.0;
  const Ssp54& k = kRk54;
  const double r[6] = {1.0 / k.b10, k.a21 / k.b21, k.a32 / k.b32, k.a43 / k.b43, k.a53 / k.b53,
                       k.a54 / k.b54};
  double m = r[0];
  for (double x : r) m = std::fmin(m, x);
  return m;
}

// Implicit source substep S_h (Sec. 3.1.3, Eqs. strang_split, source_residual) from U into
// out (equal pointers: in place).  Writes the output's primitive cache when out is a
// context buffer.
dg_status run_source(dg_ctx* c, const double* U, double* out, double h, cudaStream_t s) {
  dg::SourceArgs a;
  std::memset(&a, 0, sizeof(a));
  a.U = U;
  a.out = out;
  a.err = c->err;
  a.mech = c->d_mech;
  a.stride = c->n_nodes_total;
  a.h = h;
  a.max_it = c->phys.newton_max_it > 0 ? c->phys.newton_max_it : DG_NEWTON_MAX_IT;
  a.tol = c->phys.newton_tol > 0.0 ? c->phys.newton_tol : DG_NEWTON_TOL;
  a.p_ref = c->phys.p_ref;
  a.ln1e4 = std::log(1.0e4);
  a.copy_rest = (U != out) ? 1 : 0;
  a.updates = c->lam + 2;
  const int bin = buf_index(c, U);
  if (c->tt && bin >= 0 && c->pvalid[bin]) a.tin = c->pT[bin];  // warm start of T_v
  const int bout = buf_index(c, out);
  if (bout >= 0) {
    a.pout = c->pc[bout];
    a.tout = c->pT[bout];
    c->pvalid[bout] = true;
  }
  const int fp32 = c->phys.precision == DG_FP32_MIXED;
  for (size_t i = 0; i < c->inst.size(); ++i) {
    a.base = c->offs[i];
    a.n = n_elem_of(c->inst[i]) * n_p_of(c->inst[i]);
    cudaError_t e = dg::launch_source_implicit(c->n_species, c->tt, fp32, a, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "implicit source launch");
  }
  return DG_OK;
}

// One time step from buf[cur]: SSP-RK3 (the new state lands in another buffer and cur
// moves) or SSP-RK54 (the new state lands in buf[cur] again); under the Strang split
// (Eq. strang_split) wrapped in two implicit source half steps.
dg_status one_step(dg_ctx* c, double dt, cudaStream_t s) {
  dg_status st;
  if (c->split && (st = run_source(c, c->buf[c->cur], c->buf[c->cur], 0.5 * dt, s))) return st;
  if (c->rk54) {
    double* A = c->buf[c->cur];
    double* B = c->buf[(c->cur + 1) % 4];
    double* C = c->buf[(c->cur + 2) % 4];
    double* D = c->buf[(c->cur + 3) % 4];
    const Ssp54& r = kRk54;
    StageCoef k;
    k.cb = 1.0;
    k.bdt = r.b10 * dt;
    if ((st = run_stage(c, A, A, B, 1, k, s))) return st;                       // U1 -> B
    k.ca = r.a20, k.cb = r.a21, k.bdt = r.b21 * dt;
    if ((st = run_stage(c, B, A, C, 1, k, s))) return st;                       // U2 -> C
    k.ca = r.a30, k.cb = r.a32, k.bdt = r.b32 * dt;
    if ((st = run_stage(c, C, A, B, 1, k, s))) return st;                       // U3 -> B
    k.ca = r.a40, k.cb = r.a43, k.bdt = r.b43 * dt;
    k.acc = C, k.acc_a = r.a52, k.acc_b = r.a53, k.acc_bdt = r.b53 * dt;       // C: a52 U2 + a53 U3 + b53 dt L(U3)
    if ((st = run_stage(c, B, A, D, 1, k, s))) return st;                       // U4 -> D
    StageCoef k5;
    k5.ca = 1.0, k5.cb = r.a54, k5.bdt = r.b54 * dt;
    if ((st = run_stage(c, D, C, A, 1, k5, s))) return st;                      // U5 -> A
  } else {
    double* A = c->buf[c->cur];
    double* B = c->buf[(c->cur + 1) % 3];
    double* C = c->buf[(c->cur + 2) % 3];
    if ((st = run_stage(c, A, A, B, 1, rk3_coef(0, dt), s))) return st;
    if ((st = run_stage(c, B, A, C, 1, rk3_coef(1, dt), s))) return st;
    if ((st = run_stage(c, C, A, B, 1, rk3_coef(2, dt), s))) return st;
    c->cur = (c->cur + 1) % 3;
  }
  if (c->split && (st = run_source(c, c->buf[c->cur], c->buf[c->cur], 0.5 * dt, s))) return st;
  return DG_OK;
}

// Metric terms of the context's curved instances (device array met [dim*dim + 1][nodes], the
// per-instance flags and smallest spacings); euler: also set up the curved Euler kernel.
dg_status setup_curved(dg_ctx* c, const dg_mesh_desc* inst, int n_inst, long long off, bool euler) {
  const int nm = c->dim * c->dim + 1;
  std::vector<double> met((size_t)nm * off, 0.0);
  c->curved.assign(n_inst, 0);
  c->curved_dx.assign(n_inst, 0.0);
  for (int i = 0; i < n_inst; ++i) {
    if (!inst[i].coords) continue;
    c->curved[i] = 1;
    if (!curved_metrics_host(inst[i], met.data(), off, c->offs[i], c->curved_dx[i]))
      return DG_EINVAL;  // an element with J <= 0
    if (euler && dg::launch_curved(inst[i].dim, inst[i].N, c->phys.volume == DG_VOL_EC,
                                   c->phys.precision == DG_FP32_MIXED, nullptr, nullptr, nullptr) != cudaSuccess) {
      cudaGetLastError();
      return DG_ECUDA;
    }
  }
  if (cudaMalloc(&c->met, sizeof(double) * met.size()) != cudaSuccess) {
    cudaGetLastError();
    return DG_ENOMEM;
  }
  if (cudaMemcpy(c->met, met.data(), sizeof(double) * met.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return DG_ECUDA;
  }
  return DG_OK;
}

}  // namespace

extern "C" {

dg_status dg_init_mesh(const dg_mesh_desc* inst, int n_inst, const dg_physics* phys,
                       void* cuda_stream, dg_ctx** out) {
  if (!out) return DG_EINVAL;
  *out = nullptr;
  if (!inst || n_inst < 1 || !phys) return DG_EINVAL;
  std::string why;
  for (int i = 0; i < n_inst; ++i) {
    dg_status s = check_desc(inst[i], inst[0].dim, phys->equations, why);
    if (s) return s;
  }
  if (phys->equations < DG_EULER || phys->equations > DG_NS_REACTING) return DG_EINVAL;
  if (phys->volume < DG_VOL_STRONG || phys->volume > DG_VOL_EC) return DG_EINVAL;
  if (phys->surface < DG_SURF_RUSANOV || phys->surface > DG_SURF_EC) return DG_EINVAL;
  if (phys->precision != DG_FP64 && phys->precision != DG_FP32_MIXED) return DG_EINVAL;
  if (phys->equations != DG_NS_REACTING && !(phys->gamma > 1.0)) return DG_EINVAL;
  if (!std::isfinite(phys->p_ref)) return DG_EINVAL;
  if (phys->time_scheme != DG_SSPRK33 && phys->time_scheme != DG_SSPRK54) return DG_EINVAL;
  if (phys->chem_split != 0 && (phys->chem_split != 1 || phys->equations != DG_NS_REACTING))
    return DG_EINVAL;
  if (!std::isfinite(phys->newton_tol) || phys->newton_max_it > 1000) return DG_EINVAL;
  bool any_curved = false;
  for (int i = 0; i < n_inst; ++i) {
    if (!inst[i].coords) continue;
    any_curved = true;
    if (phys->shock || phys->rho_floor > 0.0 || phys->p_floor > 0.0) return DG_EUNSUPPORTED;
    if (phys->equations == DG_EULER) {
      if ((phys->volume != DG_VOL_STRONG && phys->volume != DG_VOL_EC) || !dg::have_curved(inst[i].dim, inst[i].N))
        return DG_EUNSUPPORTED;
    } else {  // viscous equations: periodic curved meshes, without the species limiter (its
              // element mean would need the Jacobian weights)
      if (phys->species_limiter) return DG_EUNSUPPORTED;
      for (int l = 0; l < inst[i].dim; ++l)
        if (!inst[i].periodic[l]) return DG_EUNSUPPORTED;
    }
  }
  dg_physics ph = *phys;  // with the shock-capturing defaults filled in
  if (ph.shock) {
    if (ph.shock != 1) return DG_EINVAL;
    if (ph.equations != DG_EULER) return DG_EUNSUPPORTED;
    for (int i = 0; i < n_inst; ++i)
      if (!dg::have_shock(inst[i].dim, inst[i].N)) return DG_EUNSUPPORTED;
    if (!(ph.alpha_min > 0.0)) ph.alpha_min = DG_ALPHA_MIN;
    if (!(ph.alpha_max > 0.0)) ph.alpha_max = DG_ALPHA_MAX;
    if (!(ph.sharpness > 0.0)) ph.sharpness = std::log(9999.0);
    if (!std::isfinite(ph.alpha_min) || !std::isfinite(ph.sharpness) || !(ph.alpha_max <= 1.0) ||
        !(ph.alpha_min <= ph.alpha_max))
      return DG_EINVAL;
  }
  const bool navier_stokes = phys->equations != DG_EULER;
  const int tt = phys->two_temperature;
  if (tt != 0 && tt != 1) return DG_EINVAL;
  if (tt && phys->equations != DG_NS_REACTING) return DG_EUNSUPPORTED;  // reacting air only
  if (phys->species_limiter != 0 && (phys->species_limiter != 1 || phys->equations == DG_EULER))
    return DG_EINVAL;  // partial densities exist for the viscous equations
  dg::MechDev mech;
  std::vector<dg::ReactBC> rbc;
  if (navier_stokes) {
    if (!(phys->mu >= 0.0) || !std::isfinite(phys->mu) || !(phys->prandtl > 0.0) ||
        !std::isfinite(phys->prandtl))
      return DG_EINVAL;
    if (phys->equations == DG_NS_REACTING) {
      if (!phys->chem) return DG_EINVAL;
      dg_status st = pack_mechanism(*phys->chem, mech, tt, why);
      if (st) return st;
    } else {
      dg_mechanism one;
      std::memset(&one, 0, sizeof(one));
      one.n_species = 1;
      one.W[0] = 1.0;
      one.R[0] = 1.0;
      one.cv[0] = 1.0 / (phys->gamma - 1.0);
      dg_status st = pack_mechanism(one, mech, 0, why);
      if (st) return st;
    }
    if (inst[0].dim != 3) return DG_EUNSUPPORTED;
    for (int i = 0; i < n_inst; ++i)
      if (!dg::have_reacting(inst[i].N, mech.ns, tt)) return DG_EUNSUPPORTED;
    rbc.resize(n_inst);
    for (int i = 0; i < n_inst; ++i)
      if (!react_bc(inst[i], mech, phys->p_ref, tt, rbc[i], why)) return DG_EINVAL;
    if (phys->volume != DG_VOL_STRONG || phys->surface != DG_SURF_RUSANOV ||
        phys->rho_floor > 0.0 || phys->p_floor > 0.0)
      return DG_EUNSUPPORTED;
  }

  dg_ctx* c = new dg_ctx();
  c->inst.assign(inst, inst + n_inst);
  c->rbc = rbc;
  c->phys = ph;
  c->stream = (cudaStream_t)cuda_stream;
  c->dim = inst[0].dim;
  c->ns = navier_stokes;
  c->n_species = navier_stokes ? mech.ns : 0;
  c->nv = navier_stokes ? mech.ns + 4 + tt : c->dim + 2;
  c->tt = tt;
  long long off = 0;
  for (int i = 0; i < n_inst; ++i) {
    c->offs.push_back(off);
    off += n_elem_of(inst[i]) * n_p_of(inst[i]);
  }
  c->n_nodes_total = off;
  c->rk54 = phys->time_scheme == DG_SSPRK54;
  c->split = phys->chem_split == 1;
  const size_t bytes = sizeof(double) * (size_t)c->nv * (size_t)off;
  for (int b = 0; b < (c->rk54 ? 4 : 3); ++b) {
    if (cudaMalloc(&c->buf[b], bytes) != cudaSuccess) {
      cudaGetLastError();
      dg_free(c);
      return DG_ENOMEM;
    }
  }
  // err[0]: the error word; err[2], err[3]: the work counters of the persistent stage
  // kernels (next run to claim, CTAs finished), zero between launches
  if (cudaMalloc(&c->err, 4 * sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&c->lam, 3 * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    dg_free(c);
    return DG_ENOMEM;
  }
  if (cudaMemset(c->err, 0, 4 * sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(c->lam, 0, 3 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemset(c->buf[0], 0, bytes) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    dg_free(c);
    return DG_ECUDA;
  }
  if (navier_stokes) {
    long long nfb = 0;
    for (int i = 0; i < n_inst; ++i) {
      c->fb_offs.push_back(nfb);
      nfb += n_elem_of(inst[i]) * 6 * (4 + tt) * (long long)(inst[i].N + 1) * (inst[i].N + 1);
    }
    if (cudaMalloc(&c->d_mech, sizeof(dg::MechDev)) != cudaSuccess ||
        cudaMalloc(&c->fb, sizeof(double) * (size_t)nfb) != cudaSuccess) {
      cudaGetLastError();
      dg_free(c);
      return DG_ENOMEM;
    }
    const size_t rsz = phys->precision == DG_FP32_MIXED ? sizeof(float) : sizeof(double);
    for (int k = 0; k < 5; ++k) {
      if (k == 3 && !c->rk54) continue;
      if (cudaMalloc(&c->pc[k], dg::react_cache_rows(tt) * rsz * (size_t)off) != cudaSuccess ||
          cudaMalloc(&c->pT[k], dg::react_t64_rows(tt) * sizeof(double) * (size_t)off) != cudaSuccess) {
        cudaGetLastError();
        dg_free(c);
        return DG_ENOMEM;
      }
    }
    if (cudaMemcpy(c->d_mech, &mech, sizeof(mech), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      dg_free(c);
      return DG_ECUDA;
    }
    for (int i = 0; i < n_inst; ++i) {
      if (dg::prepare_reacting(inst[i].N, mech.ns, tt, phys->precision == DG_FP32_MIXED) != cudaSuccess) {
        cudaGetLastError();
        dg_free(c);
        return DG_ECUDA;
      }
    }
    if (any_curved) {
      dg_status st = setup_curved(c, inst, n_inst, off, false);
      if (st) {
        dg_free(c);
        return st;
      }
    }
    *out = c;
    return DG_OK;
  }
  for (int i = 0; i < n_inst; ++i) {
    cudaError_t e = dg::prepare_euler_stage(inst[i].dim, inst[i].N, phys->volume == DG_VOL_EC,
                                            phys->precision == DG_FP32_MIXED);
    if (e != cudaSuccess) {
      dg_free(c);
      return DG_ECUDA;
    }
  }
  if (any_curved) {
    dg_status st = setup_curved(c, inst, n_inst, off, true);
    if (st) {
      dg_free(c);
      return st;
    }
    *out = c;  // curved instances are launched per instance
    return DG_OK;
  }
  if (ph.shock) {
    c->shock = true;
    long long ne = 0;
    for (int i = 0; i < n_inst; ++i) {
      c->eoffs.push_back(ne);
      ne += n_elem_of(inst[i]);
    }
    if (cudaMalloc(&c->alpha_raw, sizeof(double) * ne) != cudaSuccess ||
        cudaMalloc(&c->alpha, sizeof(double) * ne) != cudaSuccess ||
        cudaMalloc(&c->list, sizeof(int) * ne) != cudaSuccess ||
        cudaMalloc(&c->count, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&c->ldg, bytes) != cudaSuccess) {
      cudaGetLastError();
      dg_free(c);
      return DG_ENOMEM;
    }
    *out = c;  // shock-captured stages are launched per instance
    return DG_OK;
  }
  bool batchable = true;
  for (int i = 0; i < n_inst; ++i) batchable = batchable && inst[i].N <= dg::kMaxBatchedN;
  if (n_inst > 1 && batchable) {
    c->batched = true;
    dg_status st = build_batch(c);
    if (st != DG_OK) {
      dg_free(c);
      return st;
    }
  }
  *out = c;
  return DG_OK;
}

dg_status dg_state_size(const dg_ctx* c, int64_t* n_doubles, int* n_vars) {
  if (!c) return DG_EINVAL;
  if (n_doubles) *n_doubles = (int64_t)c->nv * c->n_nodes_total;
  if (n_vars) *n_vars = c->nv;
  return DG_OK;
}

dg_status dg_instance_offset(const dg_ctx* c, int i, int64_t* offset) {
  if (!c || !offset || i < 0 || i >= (int)c->inst.size()) return DG_EINVAL;
  *offset = c->offs[i];
  return DG_OK;
}

dg_status dg_set_state(dg_ctx* c, const double* U) {
  if (!c) return DG_EINVAL;
  if (!U) return fail(c, DG_EINVAL, "null state pointer");
  c->pvalid[c->cur] = false;
  const size_t bytes = sizeof(double) * (size_t)c->nv * c->n_nodes_total;
  cudaError_t e = cudaMemcpyAsync(c->buf[c->cur], U, bytes, cudaMemcpyDefault, c->stream);
  return e == cudaSuccess ? DG_OK : cuda_fail(c, e, "dg_set_state");
}

dg_status dg_get_state(const dg_ctx* c, double* U) {
  if (!c) return DG_EINVAL;
  dg_ctx* m = const_cast<dg_ctx*>(c);
  if (!U) return fail(m, DG_EINVAL, "null state pointer");
  const size_t bytes = sizeof(double) * (size_t)c->nv * c->n_nodes_total;
  cudaError_t e = cudaMemcpyAsync(U, c->buf[c->cur], bytes, cudaMemcpyDefault, c->stream);
  return e == cudaSuccess ? DG_OK : cuda_fail(m, e, "dg_get_state");
}

dg_status dg_rhs(dg_ctx* c, const double* U, double* dUdt, double t) {
  (void)t;
  if (!c) return DG_EINVAL;
  if (!U || !dUdt) return fail(c, DG_EINVAL, "null pointer");
  if (U == dUdt) return fail(c, DG_EINVAL, "U and dUdt must not overlap");
  return run_stage(c, U, U, dUdt, 0, StageCoef(), c->stream);
}

dg_status dg_rk_stage(dg_ctx* c, int stage, const double* Un, const double* Uprev, double dt,
                      double* Uout) {
  if (!c) return DG_EINVAL;
  if (stage < 1 || stage > 3) return fail(c, DG_EINVAL, "stage must be 1, 2 or 3");
  if (!Un || !Uprev || !Uout) return fail(c, DG_EINVAL, "null pointer");
  if (Uout == Un || Uout == Uprev) return fail(c, DG_EINVAL, "Uout must not alias an input");
  if (!std::isfinite(dt)) return fail(c, DG_EINVAL, "dt must be finite");
  return run_stage(c, Uprev, Un, Uout, 1, rk3_coef(stage - 1, dt), c->stream);
}

dg_status dg_rk_step(dg_ctx* c, double dt, int n_steps) {
  if (!c) return DG_EINVAL;
  if (n_steps < 0) return fail(c, DG_EINVAL, "n_steps must be >= 0");
  if (!std::isfinite(dt)) return fail(c, DG_EINVAL, "dt must be finite");
  dg_status st;
  // single steps until the current state sits in buf[0] (the graph's entry buffer)
  while (n_steps > 0 && c->cur != 0) {
    if ((st = one_step(c, dt, c->stream))) return st;
    --n_steps;
  }
  const int triples = n_steps / 3;  // three steps bring the rotation back to buf[0]
  if (triples > 0) {
    // Navier-Stokes: the graph starts from buf[0] with a valid primitive cache
    if (c->ns && !c->pvalid[0]) {
      if ((st = fill_prims(c, c->buf[0], 0, c->stream))) return st;
      c->pvalid[0] = true;
    }
    if (!c->gexec || c->g_dt != dt) {
      if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
      cudaGraph_t g;
      cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_fail(c, e, "begin capture");
      const int saved = c->cur;
      for (int k = 0; k < 3; ++k) {
        if ((st = one_step(c, dt, c->cap))) {
          cudaStreamEndCapture(c->cap, &g);
          cudaGetLastError();
          c->cur = saved;
          for (bool& v : c->pvalid) v = false;
          return st;
        }
      }
      c->cur = saved;
      e = cudaStreamEndCapture(c->cap, &g);
      if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
      e = cudaGraphInstantiate(&c->gexec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) { c->gexec = nullptr; return cuda_fail(c, e, "graph instantiate"); }
      c->g_dt = dt;
    }
    for (int k = 0; k < triples; ++k) {
      cudaError_t e = cudaGraphLaunch(c->gexec, c->stream);
      if (e != cudaSuccess) {
        for (bool& v : c->pvalid) v = false;
        return cuda_fail(c, e, "graph launch");
      }
    }
    n_steps -= 3 * triples;
  }
  while (n_steps > 0) {
    if ((st = one_step(c, dt, c->stream))) return st;
    --n_steps;
  }
  return DG_OK;
}

dg_status dg_rhs_vjp(dg_ctx* c, const double* U, const double* lam, double* Ubar, double* gammabar) {
  if (!c) return DG_EINVAL;
  if (!U || !lam || !Ubar) return fail(c, DG_EINVAL, "null pointer");
  if (Ubar == U || Ubar == lam) return fail(c, DG_EINVAL, "Ubar must not alias U or lam");
  if (c->ns) return fail(c, DG_EUNSUPPORTED, "the adjoint exists for the Euler equations");
  dg_status st = ensure_adjoint(c);
  if (st) return st;
  if ((st = run_vjp(c, U, lam, Ubar, 0, 1.0, 0.0, nullptr, nullptr, 0, 0.0, 1.0))) return st;
  return read_gacc(c, gammabar);
}

}  // extern "C"

namespace {

// Adjoint of one SSP-RK54 step (App. B, Shu-Osher form U^(i) = sum_k alpha_ik U^(k) +
// dt beta_ik L(U^(k)), U^(5) = U^{n+1}): the stages U^(1..4) are recomputed from Un, then, with
// lam^(5) = lam, for k = 4..0
//   mu_k = sum_{i>k} beta_ik lam^(i),   lam^(k) = sum_{i>k} alpha_ik lam^(i) + dt (dL/dU(U^(k)))^T mu_k
// (one VJP launch with co-state mu_k, bcoef 1 and accin = sum alpha_ik lam^(i) - mu_k, the two
// sums formed by the combination kernel), and gammabar += dt mu_k . dL/dgamma(U^(k)).
dg_status rk54_step_vjp(dg_ctx* c, const double* Un, double dt, double* lam, double* gammabar) {
  const Ssp54& k = kRk54;
  double* Us[5] = {const_cast<double*>(Un), c->adj[0], c->adj[1], c->adj[2], c->adj[3]};
  double* Lm[5] = {nullptr, c->adj[4], c->adj[5], c->adj[6], c->adj[7]};  // lam^(1..4)
  double *mu = c->adj[8], *acc = c->adj[9];
  // forward stages 1..4: U^(i) = alpha_i0 U^n + alpha_i,i-1 U^(i-1) + beta_i,i-1 dt L(U^(i-1))
  const double a_i0[5] = {0.0, 0.0, k.a20, k.a30, k.a40};
  const double a_ip[5] = {0.0, 1.0, k.a21, k.a32, k.a43};
  const double b_ip[5] = {0.0, k.b10, k.b21, k.b32, k.b43};
  dg_status st;
  for (int i = 1; i <= 4; ++i) {
    StageCoef sc;
    sc.ca = a_i0[i];
    sc.cb = a_ip[i];
    sc.bdt = b_ip[i] * dt;
    if ((st = run_stage(c, Us[i - 1], Un, Us[i], 1, sc, c->stream))) return st;
  }
  // the table's nonzero entries (i, k): alpha and beta
  double A[6][5] = {}, B[6][5] = {};
  A[1][0] = 1.0;        B[1][0] = k.b10;
  A[2][0] = k.a20;      A[2][1] = k.a21;  B[2][1] = k.b21;
  A[3][0] = k.a30;      A[3][2] = k.a32;  B[3][2] = k.b32;
  A[4][0] = k.a40;      A[4][3] = k.a43;  B[4][3] = k.b43;
  A[5][2] = k.a52;      A[5][3] = k.a53;  B[5][3] = k.b53;  A[5][4] = k.a54;  B[5][4] = k.b54;
  const long long n = (long long)c->nv * c->n_nodes_total;
  auto lam_of = [&](int i) -> const double* { return i == 5 ? lam : Lm[i]; };
  for (int kk = 4; kk >= 0; --kk) {
    dg::CombineArgs cm, ca;
    std::memset(&cm, 0, sizeof(cm));
    std::memset(&ca, 0, sizeof(ca));
    cm.y = mu;
    ca.y = acc;
    cm.n = ca.n = n;
    for (int i = kk + 1; i <= 5; ++i) {
      if (B[i][kk] != 0.0) {
        cm.x[cm.m] = lam_of(i);
        cm.c[cm.m++] = B[i][kk];
      }
      if (A[i][kk] != 0.0 || B[i][kk] != 0.0) {
        ca.x[ca.m] = lam_of(i);
        ca.c[ca.m++] = A[i][kk] - B[i][kk];
      }
    }
    cudaError_t e = dg::launch_combine(cm, c->stream);
    if (e == cudaSuccess) e = dg::launch_combine(ca, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "adjoint combination");
    double* out = kk == 0 ? lam : Lm[kk];
    if ((st = run_vjp(c, Us[kk], mu, out, 1, 1.0, dt, acc, nullptr, 0, 0.0, dt))) return st;
  }
  return read_gacc(c, gammabar);
}

}  // namespace

extern "C" {

dg_status dg_rk_step_vjp(dg_ctx* c, const double* Un, double dt, double* lam, double* gammabar) {
  if (!c) return DG_EINVAL;
  if (!Un || !lam) return fail(c, DG_EINVAL, "null pointer");
  if (Un == lam) return fail(c, DG_EINVAL, "lam must not alias Un");
  if (c->ns) return fail(c, DG_EUNSUPPORTED, "the adjoint exists for the Euler equations");
  if (!std::isfinite(dt)) return fail(c, DG_EINVAL, "dt must be finite");
  dg_status st = ensure_adjoint(c);
  if (st) return st;
  if (c->rk54) return rk54_step_vjp(c, Un, dt, lam, gammabar);
  double *W1 = c->adj[0], *W2 = c->adj[1], *T1 = c->adj[2], *T2 = c->adj[3], *T3 = c->adj[4];
  // recompute the stage states of this step
  if ((st = run_stage(c, Un, Un, W1, 1, rk3_coef(0, dt), c->stream))) return st;
  if ((st = run_stage(c, W1, Un, W2, 1, rk3_coef(1, dt), c->stream))) return st;
  // reverse Shu-Osher: U3 = 1/3 Un + 2/3 (U2 + dt L(U2)), U2 = 3/4 Un + 1/4 (U1 + dt L(U1)),
  // U1 = Un + dt L(Un)
  if ((st = run_vjp(c, W2, lam, T1, 1, kStageB[2], dt, nullptr, T2, 1, kStageA[2], kStageB[2] * dt))) return st;
  if ((st = run_vjp(c, W1, T1, T3, 1, kStageB[1], dt, nullptr, T2, 0, kStageA[1], kStageB[1] * dt))) return st;
  if ((st = run_vjp(c, Un, T3, lam, 1, kStageB[0], dt, T2, nullptr, 0, 0.0, kStageB[0] * dt))) return st;
  return read_gacc(c, gammabar);
}

dg_status dg_adjoint_gammabar(dg_ctx* c, double* gammabar) {
  if (!c) return DG_EINVAL;
  if (!gammabar) return fail(c, DG_EINVAL, "null gammabar");
  if (!c->gacc) return DG_OK;  // no adjoint call yet: nothing accumulated
  return read_gacc(c, gammabar);
}

dg_status dg_set_launch(dg_ctx* c, int mode, int group_scale, int ctas_per_sm, int order) {
  if (!c) return DG_EINVAL;
  if (mode != DG_LAUNCH_PER_INSTANCE && mode != DG_LAUNCH_BATCHED)
    return fail(c, DG_EINVAL, "mode must be DG_LAUNCH_PER_INSTANCE or DG_LAUNCH_BATCHED");
  if (c->ns && mode == DG_LAUNCH_BATCHED)
    return fail(c, DG_EUNSUPPORTED, "the batched launch exists for the Euler equations");
  if (c->shock && mode == DG_LAUNCH_BATCHED)
    return fail(c, DG_EUNSUPPORTED, "shock-captured stages are launched per instance");
  if (c->met && mode == DG_LAUNCH_BATCHED)
    return fail(c, DG_EUNSUPPORTED, "curved instances are launched per instance");
  const bool per_degree = (group_scale & DG_GROUPS_PER_DEGREE) != 0;
  if (per_degree ? (c->dim != 2 || (group_scale & ~(DG_GROUPS_PER_DEGREE | 0x3e)) != 0)
                 : (group_scale != 1 && !(group_scale == 2 && c->dim == 2)))
    return fail(c, DG_EINVAL, "group_scale must be 1 (or, in 2D, 2 or DG_GROUPS_PER_DEGREE | mask of degrees 1..5)");
  if (ctas_per_sm < 0 || (order != 0 && order != 1))
    return fail(c, DG_EINVAL, "ctas_per_sm must be >= 0 and order 0 or 1");
  if (mode == DG_LAUNCH_BATCHED)
    for (const dg_mesh_desc& m : c->inst)
      if (m.N > dg::kMaxBatchedN) return fail(c, DG_EUNSUPPORTED, "batched launches cover N <= 5");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_set_launch sync");
  drop_graph(c);
  c->bcfg = dg::BatchConfig{group_scale, ctas_per_sm, order};
  c->batched = (mode == DG_LAUNCH_BATCHED);
  if (c->batched) return build_batch(c);
  return DG_OK;
}

dg_status dg_autotune(dg_ctx* c, double dt, int n_reps, int* config_out, double* ms_out) {
  if (!c) return DG_EINVAL;
  if (!std::isfinite(dt) || n_reps < 1 || !config_out) return fail(c, DG_EINVAL, "bad autotune arguments");
  if (c->ns) return fail(c, DG_EUNSUPPORTED, "the autotuner exists for the Euler equations");
  const size_t bytes = sizeof(double) * (size_t)c->nv * c->n_nodes_total;
  double* save = nullptr;
  if (cudaMalloc(&save, bytes) != cudaSuccess) { cudaGetLastError(); return fail(c, DG_ENOMEM, "autotune copy"); }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMemcpyAsync(save, c->buf[c->cur], bytes, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  struct Cand { int mode, gs, cps, order; };
  std::vector<Cand> cands;
  cands.push_back({DG_LAUNCH_PER_INSTANCE, 1, 0, 0});
  for (int gs = 1; gs <= (c->dim == 2 ? 2 : 1); ++gs)
    for (int cps : {0, 1, 2})
      for (int order = 0; order <= 1; ++order) cands.push_back({DG_LAUNCH_BATCHED, gs, cps, order});
  const size_t n_uniform = cands.size();
  // degrees present (2D): each proper non-empty subset taking group scale 2 is a candidate of
  // the second round, with the ctas_per_sm and order of the best uniform choice
  int present = 0;
  for (const dg_mesh_desc& m : c->inst) present |= 1 << m.N;
  std::vector<int> subsets;
  if (c->dim == 2)
    for (int m = present; m > 0; m = (m - 1) & present)
      if (m != present) subsets.push_back(m);
  double best = INFINITY;
  Cand bestc = cands[0];
  dg_status st = DG_OK;
  for (size_t k = 0; k < cands.size() && e == cudaSuccess && st == DG_OK; ++k) {
    const Cand q = cands[k];  // (a copy: the list grows below)
    if ((st = dg_set_launch(c, q.mode, q.gs, q.cps, q.order)) != DG_OK) break;
    if ((st = one_step(c, dt, c->stream)) != DG_OK) break;  // warm-up
    if ((e = cudaEventRecord(e0, c->stream)) != cudaSuccess) break;
    for (int r = 0; r < n_reps && st == DG_OK; ++r) st = one_step(c, dt, c->stream);
    if (st != DG_OK) break;
    if ((e = cudaEventRecord(e1, c->stream)) != cudaSuccess) break;
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
    float ms = 0.f;
    if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
    if (ms / n_reps < best) { best = ms / n_reps; bestc = q; }
    if (k + 1 == n_uniform) {
      // per-degree group scales, with the best uniform batched choice's grid and order
      Cand base = bestc;
      if (base.mode != DG_LAUNCH_BATCHED) base = cands[1];
      for (int m : subsets) cands.push_back({DG_LAUNCH_BATCHED, DG_GROUPS_PER_DEGREE | m, base.cps, base.order});
    }
  }
  // restore the state and keep the fastest configuration
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->buf[c->cur], save, bytes, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(save);
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_autotune");
  if (st != DG_OK) return st;
  if ((st = dg_set_launch(c, bestc.mode, bestc.gs, bestc.cps, bestc.order)) != DG_OK) return st;
  config_out[0] = bestc.mode;
  config_out[1] = bestc.gs;
  config_out[2] = bestc.cps;
  config_out[3] = bestc.order;
  if (ms_out) *ms_out = best;
  return DG_OK;
}

dg_status dg_max_dt(dg_ctx* c, double cfl, double* dt_out) {
  if (!c) return DG_EINVAL;
  if (!dt_out || !(cfl > 0.0)) return fail(c, DG_EINVAL, "bad cfl or output pointer");
  double best = INFINITY;
  if (c->ns) {
    // convective bound with the frozen mixture sound speed and the diffusive bound
    // (Eq. dt_para): nu_max = mu * max(1/rho) / min(1, Pr)
    for (size_t i = 0; i < c->inst.size(); ++i) {
      const dg_mesh_desc& m = c->inst[i];
      cudaError_t e = cudaMemsetAsync(c->lam, 0, 2 * sizeof(unsigned long long), c->stream);
      if (e == cudaSuccess)
        e = dg::launch_max_speed_mix(c->n_species, c->tt, c->buf[c->cur], c->n_nodes_total, c->offs[i],
                                     n_elem_of(m) * n_p_of(m), c->d_mech, c->lam, c->stream);
      unsigned long long bits[2] = {0, 0};
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(bits, c->lam, sizeof(bits), cudaMemcpyDeviceToHost, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "dg_max_dt");
      double lam = 0.0, irho = 0.0;
      const int k0 = dg::decode_speed(bits[0], &lam), k1 = dg::decode_speed(bits[1], &irho);
      if (k0 == 1 || k1 == 1) return fail(c, DG_ENONFINITE, "the state holds a non-finite value");
      if (k0 == 2 || k1 == 2) return fail(c, DG_EPOSITIVITY, "the state has a node with rho <= 0 or T <= 0");
      if (!(lam > 0.0)) return fail(c, DG_ENONFINITE, "no positive signal speed");
      double dxmin = INFINITY;
      for (int l = 0; l < m.dim; ++l) dxmin = std::fmin(dxmin, (m.hi[l] - m.lo[l]) / m.nel[l]);
      if (!c->curved.empty() && c->curved[i]) dxmin = c->curved_dx[i];  // 2 J / |Ja^l| on curved meshes
      const double n2 = (2.0 * m.N + 1.0) * (2.0 * m.N + 1.0);
      const double nu = c->phys.mu * irho / std::fmin(1.0, c->phys.prandtl);
      const double cs = cfl * ssp_coefficient(c);
      double dt = cs * dxmin / ((2 * m.N + 1) * lam);
      if (nu > 0.0) dt = std::fmin(dt, cs * dxmin * dxmin / (n2 * nu));
      best = std::fmin(best, dt);
    }
    *dt_out = best;
    return DG_OK;
  }
  for (size_t i = 0; i < c->inst.size(); ++i) {
    const dg_mesh_desc& m = c->inst[i];
    cudaError_t e = cudaMemsetAsync(c->lam, 0, sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess)
      e = dg::launch_max_speed(m.dim, c->buf[c->cur], c->n_nodes_total, c->offs[i],
                               n_elem_of(m) * n_p_of(m), c->phys.gamma, c->lam, c->stream);
    unsigned long long bits = 0;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&bits, c->lam, sizeof(bits), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "dg_max_dt");
    double lam = 0.0;
    const int k = dg::decode_speed(bits, &lam);
    if (k == 1) return fail(c, DG_ENONFINITE, "the state holds a non-finite value");
    if (k == 2) return fail(c, DG_EPOSITIVITY, "the state has a node with rho <= 0 or p <= 0");
    if (!(lam > 0.0)) return fail(c, DG_ENONFINITE, "no positive signal speed");
    double dxmin = INFINITY;
    for (int l = 0; l < m.dim; ++l) dxmin = std::fmin(dxmin, (m.hi[l] - m.lo[l]) / m.nel[l]);
    if (!c->curved.empty() && c->curved[i]) dxmin = c->curved_dx[i];  // 2 J / |Ja^l| on curved meshes
    best = std::fmin(best, cfl * ssp_coefficient(c) * dxmin / ((2 * m.N + 1) * lam));
  }
  *dt_out = best;
  return DG_OK;
}

dg_status dg_check(dg_ctx* c) {
  if (!c) return DG_EINVAL;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_check sync");
  unsigned w = 0;
  e = cudaMemcpy(&w, c->err, sizeof(w), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(c->err, 0, sizeof(unsigned));
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_check read");
  if (w & 1u) return fail(c, DG_ENONFINITE, "a kernel produced a non-finite value");
  if (w & 2u) return fail(c, DG_EPOSITIVITY, "a kernel read a state with rho <= 0 or p <= 0");
  if (w & 4u) return fail(c, DG_ECONVERGENCE, "the implicit source Newton iteration did not converge");
  return DG_OK;
}

dg_status dg_gll(int N, double* x, double* w, double* D) {
  if (N < 1 || N > dg::kMaxN || !x || !w) return DG_EINVAL;
  gll_table(N, x, w, D);
  return DG_OK;
}

dg_status dg_two_point_flux(dg_ctx* c, int kind, int l, int n, const double* uL,
                            const double* uR, double* F) {
  if (!c) return DG_EINVAL;
  if (c->ns) return fail(c, DG_EUNSUPPORTED, "two-point fluxes exist for the Euler equations");
  if (kind < -1 || kind > DG_SURF_EC || l < 0 || l >= c->dim || n < 0 || !uL || !uR || !F)
    return fail(c, DG_EINVAL, "bad two-point flux arguments");
  cudaError_t e = dg::launch_two_point(c->dim, c->phys.precision == DG_FP32_MIXED, kind, l, n,
                                       c->phys.gamma, c->phys.p_ref, uL, uR, F, c->stream);
  return e == cudaSuccess ? DG_OK : cuda_fail(c, e, "two-point flux launch");
}

dg_status dg_source_step(dg_ctx* c, const double* U, double h, double* Uout) {
  if (!c) return DG_EINVAL;
  if (!U || !Uout) return fail(c, DG_EINVAL, "null pointer");
  if (c->phys.equations != DG_NS_REACTING)
    return fail(c, DG_EUNSUPPORTED, "the implicit source step exists for reacting mixtures");
  if (!std::isfinite(h) || h < 0.0) return fail(c, DG_EINVAL, "h must be finite and >= 0");
  return run_source(c, U, Uout, h, c->stream);
}

dg_status dg_shock_alpha(dg_ctx* c, const double* U, double* alpha_raw, double* alpha) {
  if (!c) return DG_EINVAL;
  if (!U) return fail(c, DG_EINVAL, "null pointer");
  if (!c->shock) return fail(c, DG_EUNSUPPORTED, "shock capturing is off");
  dg::StageArgs a;
  launch_args(c, a, U, U, nullptr, 0, StageCoef());
  long long ne = 0;
  for (size_t i = 0; i < c->inst.size(); ++i) {
    dg::ShockArgs sa;
    shock_args(c, (int)i, a, StageCoef(), sa);
    dg_status st = run_indicator(c, (int)i, sa, c->stream);
    if (st) return st;
    ne += n_elem_of(c->inst[i]);
  }
  cudaError_t e = cudaSuccess;
  if (alpha_raw) e = cudaMemcpyAsync(alpha_raw, c->alpha_raw, sizeof(double) * ne, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess && alpha)
    e = cudaMemcpyAsync(alpha, c->alpha, sizeof(double) * ne, cudaMemcpyDeviceToDevice, c->stream);
  return e == cudaSuccess ? DG_OK : cuda_fail(c, e, "dg_shock_alpha");
}

dg_status dg_newton_updates(dg_ctx* c, int64_t* count) {
  if (!c) return DG_EINVAL;
  if (!count) return fail(c, DG_EINVAL, "null pointer");
  unsigned long long v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, c->lam + 2, sizeof(v), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->lam + 2, 0, sizeof(v), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_newton_updates");
  *count = (int64_t)v;
  return DG_OK;
}

dg_status dg_math_fn(int kind, int64_t n, const double* x, double* y, void* cuda_stream) {
  if (kind < 0 || kind > 3 || n < 0 || (n > 0 && (!x || !y))) return DG_EINVAL;
  dg::MathArgs a;
  std::memset(&a, 0, sizeof(a));
  a.x = x;
  a.y = y;
  a.n = n;
  a.kind = kind;
  fill_exp2_table(a.tab);
  return dg::launch_math_fn(a, (cudaStream_t)cuda_stream) == cudaSuccess ? DG_OK : DG_ECUDA;
}

const char* dg_last_error(const dg_ctx* c) { return c ? c->msg.c_str() : kNullCtxMsg; }

void dg_free(dg_ctx* c) {
  if (!c) return;
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  for (int b = 0; b < 4; ++b)
    if (c->buf[b]) cudaFree(c->buf[b]);
  if (c->err) cudaFree(c->err);
  if (c->lam) cudaFree(c->lam);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->d_insts) cudaFree(c->d_insts);
  if (c->d_items) cudaFree(c->d_items);
  if (c->d_dv) cudaFree(c->d_dv);
  for (int k = 0; k < 10; ++k)
    if (c->adj[k]) cudaFree(c->adj[k]);
  if (c->gpart) cudaFree(c->gpart);
  if (c->gacc) cudaFree(c->gacc);
  if (c->d_mech) cudaFree(c->d_mech);
  if (c->fb) cudaFree(c->fb);
  if (c->met) cudaFree(c->met);
  if (c->alpha_raw) cudaFree(c->alpha_raw);
  if (c->alpha) cudaFree(c->alpha);
  if (c->list) cudaFree(c->list);
  if (c->count) cudaFree(c->count);
  if (c->ldg) cudaFree(c->ldg);
  for (int k = 0; k < 5; ++k) {
    if (c->pc[k]) cudaFree(c->pc[k]);
    if (c->pT[k]) cudaFree(c->pT[k]);
  }
  delete c;
}

}  // extern "C"
