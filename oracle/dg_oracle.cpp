// dg_oracle.cpp -- ORACLE: test infrastructure, not part of the product path.
//
// A plain, slow, FP64 CPU implementation of what the DGSEM hot path computes: the
// semi-discrete residual dU/dt = L(U) of the compressible Euler equations and of the
// single-temperature reacting Navier-Stokes equations on periodic Cartesian meshes (2D and
// 3D), its numerical fluxes, the SSP-RK3 stage update and the explicit time-step bounds.  It shares no source, header, table or helper with the CUDA
// path, and the CUDA path never loads it.  Only the test-suite, the smoke check and the
// benchmark's CPU-baseline leg may load it.
//
// Every function names the passage of the paper (arXiv 2605.26388) it follows:
//   Sec. 2           Euler equations, ideal-gas closure p = (gamma-1)(E - rho|u|^2/2)
//   Sec. 3.1.1       Eq. vol_weak (strong-form volume term), Eq. vol_split (two-point
//                    flux-differencing volume term), surface fluxes (LF / HLL), Eq. surf_int
//                    (surface lifting and Jacobian rescale)
//   App. A           Eq. split_form_3D and the Ranocha entropy-conservative two-point flux
//   Sec. 3.1.2       BR1 gradients (Eq. br1_avg), viscous stress (Eq. tau), central viscous
//                    interface flux (Eq. br1_flux), diffusive time-step bound Delta t_D
//   Sec. 3.1.3       Arrhenius source (Eqs. src_reaction_rate, src_omega)
//   App. B           SSP-RK in Shu-Osher form; convective time-step bound Delta t_C
//   Sec. 3.1.1, App. A  Hennemann-Gassner indicator, neighbourhood maximum and the DG/FV
//                    sub-cell blend (Eq. vol_blend)
//   Sec. 3.1.3       implicit source substep and Strang split (Eqs. strang_split,
//                    source_residual)
// Readings of passages the paper leaves open are marked READING below.
//
// Loops are written per element, per node, per direction, exactly in the order the
// formulas are stated; there is no blocking, fusion or reordering.  The element loop may
// run on several OpenMP threads: each element writes only its own residual, so the
// arithmetic per element is the same on one thread or many.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

// ---------------------------------------------------------------------------------------
// Problem description (the oracle's own; it mirrors nothing from the CUDA library).
// ---------------------------------------------------------------------------------------
enum { ORC_EULER = 0, ORC_NAVIER_STOKES = 1, ORC_NS_REACTING = 2 };
enum { ORC_VOL_STRONG = 0, ORC_VOL_WEAK = 1, ORC_VOL_EC = 2, ORC_VOL_CENTRAL = 3 };
enum { ORC_SURF_RUSANOV = 0, ORC_SURF_HLLC = 1, ORC_SURF_HLL = 2, ORC_SURF_EC = 3,
       ORC_SURF_CENTRAL = 4 };
// boundary condition of a domain face (0 = periodic)
enum { ORC_BC_PERIODIC = 0, ORC_BC_SLIP_WALL = 1, ORC_BC_INFLOW = 2, ORC_BC_OUTFLOW = 3,
       ORC_BC_DIRICHLET = 4, ORC_BC_NOSLIP_ADIABATIC = 5, ORC_BC_NOSLIP_ISOTHERMAL = 6 };
constexpr int ORC_MAX_VARS = 12;  // 8 species + 3 momenta + energy

}  // namespace

extern "C" {

// Reacting mixture (the oracle's own copy of the species and reaction data).
struct OrcMech {
  int n_species, n_reactions;
  double W[8], R[8], cv[8], h0[8];        // kg/mol, J/(kg K), J/(kg K), J/kg
  double lnA[32], b[32], Ta[32];          // k_f = exp(lnA + b ln T - Ta/T), cm-mol-s
  double kc[32][5];                       // ln K_c = a0/Z + a1 + a2 ln Z + a3 Z + a4 Z^2, Z = 1e4/T
  int nu_f[32][8], nu_b[32][8];           // stoichiometric coefficients nu', nu''
  double theta_v[8];                      // two-temperature: characteristic vibrational
                                          // temperature (K) of each species, 0 for atoms
  int ta_mode[32];                        // two-temperature: 1 -- the reaction's controlling
                                          // temperature is sqrt(T Tv) (dissociation), 0 -- T
};

struct OrcProblem {
  int dim;             // 2 or 3
  int N;               // polynomial degree; N+1 GLL nodes per direction
  int nel[3];          // elements per direction (nel[2] = 1 in 2D)
  double lo[3], hi[3]; // periodic box
  int equations;       // ORC_EULER or ORC_NS_REACTING
  int volume;          // ORC_VOL_*
  int surface;         // ORC_SURF_*
  double gamma;        // ratio of specific heats
  double mu, prandtl;  // viscous parameters (unused for Euler)
  double rho_floor, p_floor;  // <= 0 disables the positivity floor
  const OrcMech* mech;        // ORC_NS_REACTING: species and reactions
  int parts;                  // ORC_NS_REACTING: 1 inviscid, 2 viscous, 4 source (0 = all)
  int shock;                  // Euler: 1 = Hennemann-Gassner DG/FV blending of the residual
  double alpha_min, alpha_max, sharpness;  // blending bounds and the sigmoid's steepness s
  int bc[6];                  // per domain face x-, x+, y-, y+, z-, z+ (0 = periodic); the
                              // no-slip walls (5, 6) exist for ORC_NS_REACTING only
  double bc_state[6][12];     // INFLOW / DIRICHLET: the exterior conserved state (n_vars
                              // values); NOSLIP_ISOTHERMAL: [0] = the wall temperature
  const double* coords;       // node coordinates [d][elem][node] of a curved mesh on the same
                              // element topology (null: the Cartesian box); ORC_NS_REACTING:
                              // periodic, without the species limiter
  int two_temperature;        // ORC_NS_REACTING: 1 -- the two-temperature model (E_v appended
                              // to the state)
  int species_limiter;        // ORC_NS_REACTING: 1 -- the Zhang-Shu limiter of the partial
                              // densities after every RK stage
};

}  // extern "C"

namespace {

// ---------------------------------------------------------------------------------------
// Legendre polynomials and the Gauss-Lobatto-Legendre rule (Sec. 3.1.1: the solution lives
// on the tensor-product GLL nodes, weights w_i).  Nodes are -1, +1 and the
// roots of P_N'; weights w_i = 2 / (N (N+1) P_N(x_i)^2).  Newton iteration in long
// double on q(x) = P_{N+1}(x) - P_{N-1}(x), which vanishes exactly at the GLL nodes.
// ---------------------------------------------------------------------------------------
void legendre(int n, long double x, long double& Pn, long double& Pnm1) {
  // three-term recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}
  long double p0 = 1.0L, p1 = x;
  if (n == 0) { Pn = p0; Pnm1 = 0.0L; return; }
  for (int k = 1; k < n; ++k) {
    long double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
    p0 = p1;
    p1 = p2;
  }
  Pn = p1;
  Pnm1 = p0;
}

void gll_rule(int N, std::vector<long double>& x, std::vector<long double>& w) {
  x.assign(N + 1, 0.0L);
  w.assign(N + 1, 0.0L);
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i <= N; ++i) {
    long double xi = -cosl(pi * i / N);  // Chebyshev-Gauss-Lobatto start
    if (i == 0) xi = -1.0L;
    else if (i == N) xi = 1.0L;
    else {
      for (int it = 0; it < 100; ++it) {
        long double PN, PNm1, PNp1, tmp;
        legendre(N, xi, PN, PNm1);
        legendre(N + 1, xi, PNp1, tmp);
        long double q = PNp1 - PNm1;       // (2N+1)/... * (x^2-1) P_N'(x) up to a factor
        long double dq = (2 * N + 1) * PN; // d/dx (P_{N+1} - P_{N-1}) = (2N+1) P_N
        long double dx = q / dq;
        xi -= dx;
        if (fabsl(dx) < 1e-19L) break;
      }
    }
    x[i] = xi;
    long double PN, PNm1;
    legendre(N, xi, PN, PNm1);
    w[i] = 2.0L / (N * (N + 1) * PN * PN);
  }
}

// Lagrange differentiation matrix D_ij = l_j'(x_i) on the GLL nodes (Sec. 3.1.1: the 1D
// GLL derivative matrix D), from barycentric weights
// lambda_j = 1 / prod_{k != j} (x_j - x_k):  D_ij = (lambda_j / lambda_i) / (x_i - x_j)
// for i != j, and the diagonal by the negative row sum (derivative of a constant is 0).
void diff_matrix(int N, const std::vector<long double>& x, std::vector<long double>& D) {
  const int n = N + 1;
  std::vector<long double> lam(n, 1.0L);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) lam[j] *= (x[j] - x[k]);
  for (int j = 0; j < n; ++j) lam[j] = 1.0L / lam[j];
  D.assign(n * n, 0.0L);
  for (int i = 0; i < n; ++i) {
    long double rowsum = 0.0L;
    for (int j = 0; j < n; ++j) {
      if (i == j) continue;
      D[i * n + j] = (lam[j] / lam[i]) / (x[i] - x[j]);
      rowsum += D[i * n + j];
    }
    D[i * n + i] = -rowsum;
  }
}

// Operators of one degree, rounded to double once.
struct Ops {
  int N = 0;
  std::vector<double> x, w, D;  // D row-major: D[i*(N+1)+m]
  explicit Ops(int N_) : N(N_) {
    std::vector<long double> xl, wl, Dl;
    gll_rule(N, xl, wl);
    diff_matrix(N, xl, Dl);
    x.assign(xl.begin(), xl.end());
    w.assign(wl.begin(), wl.end());
    D.assign(Dl.begin(), Dl.end());
  }
};

// ---------------------------------------------------------------------------------------
// Euler physics (Sec. 2): U = (rho, rho u, rho v[, rho w], E), F^l the Cartesian flux in
// direction l, p = (gamma-1)(E - rho|u|^2/2), a = sqrt(gamma p / rho).
// ---------------------------------------------------------------------------------------
struct Prim {
  double rho, v[3], p;
};

Prim primitives(int dim, const double* u, double gamma) {
  Prim q;
  q.rho = u[0];
  double kin = 0.0;
  for (int d = 0; d < 3; ++d) q.v[d] = 0.0;
  for (int d = 0; d < dim; ++d) {
    q.v[d] = u[1 + d] / q.rho;
    kin += u[1 + d] * q.v[d];
  }
  q.p = (gamma - 1.0) * (u[dim + 1] - 0.5 * kin);
  return q;
}

void euler_flux(int dim, int l, const double* u, double gamma, double* F) {
  Prim q = primitives(dim, u, gamma);
  F[0] = u[1 + l];
  for (int d = 0; d < dim; ++d) F[1 + d] = u[1 + l] * q.v[d] + (d == l ? q.p : 0.0);
  F[dim + 1] = (u[dim + 1] + q.p) * q.v[l];
}

double sound_speed(const Prim& q, double gamma) { return std::sqrt(gamma * q.p / q.rho); }

// Logarithmic mean {{a}}^ln = (a_L - a_R) / (ln a_L - ln a_R) (App. A, below the Ranocha
// flux).  The paper is silent at a_L = a_R; the definition's limit there is a.  Written
// in long double, with ln a_L - ln a_R = log1p((a_L - a_R)/a_R) when the ratio is near 1,
// so that the quotient keeps full double accuracy however close a_L and a_R are.
double log_mean(double aL, double aR) {
  if (aL == aR) return aL;
  long double a = aL, b = aR;
  long double d = a - b;
  long double r = d / b;
  long double lnratio = (fabsl(r) < 0.5L) ? log1pl(r) : (logl(a) - logl(b));
  return (double)(d / lnratio);
}

// Ranocha's entropy-conservative, kinetic-energy-preserving two-point flux in direction
// e_l (App. A, Eq. split_form_3D and the flux listed after it).
// READING: the printed energy component is not consistent (F#(U,U) != F(U)); we use the
// published form  f_E = f_rho (1/((gamma-1) {{beta}}^ln) + u_L.u_R / 2)
//                      + (p_L u_{l,R} + p_R u_{l,L}) / 2,   beta = rho/p = 1/T,
// which is the unique f_E satisfying Tadmor's entropy-conservation condition given the
// printed f_rho and f_m (checked in the tests).
void ec_flux(int dim, int l, const double* uL, const double* uR, double gamma, double* F) {
  Prim L = primitives(dim, uL, gamma), R = primitives(dim, uR, gamma);
  double rho_ln = log_mean(L.rho, R.rho);
  double beta_ln = log_mean(L.rho / L.p, R.rho / R.p);
  double vavg[3], vLvR = 0.0;
  for (int d = 0; d < 3; ++d) vavg[d] = 0.5 * (L.v[d] + R.v[d]);
  for (int d = 0; d < dim; ++d) vLvR += L.v[d] * R.v[d];
  double pavg = 0.5 * (L.p + R.p);
  double frho = rho_ln * vavg[l];
  F[0] = frho;
  for (int d = 0; d < dim; ++d) F[1 + d] = frho * vavg[d] + (d == l ? pavg : 0.0);
  F[dim + 1] = frho * (1.0 / ((gamma - 1.0) * beta_ln) + 0.5 * vLvR) +
               0.5 * (L.p * R.v[l] + R.p * L.v[l]);
}

// Central two-point flux (F(U_L) + F(U_R))/2: with it the flux-differencing form equals
// the strong form (App. A, text after Eq. split_form_3D).  Test option only.
void central_flux(int dim, int l, const double* uL, const double* uR, double gamma,
                  double* F) {
  double FL[8], FR[8];
  euler_flux(dim, l, uL, gamma, FL);
  euler_flux(dim, l, uR, gamma, FR);
  for (int v = 0; v < dim + 2; ++v) F[v] = 0.5 * (FL[v] + FR[v]);
}

// Local Lax-Friedrichs (Rusanov) flux, the paper's "(local) Lax-Friedrichs" surface flux
// (Sec. 3.1.1 "Surface Fluxes"; Sec. 4 case set-ups).
// READING: dissipation speed lambda = max(|u_{l,L}| + a_L, |u_{l,R}| + a_R).
void rusanov_flux(int dim, int l, const double* uL, const double* uR, double gamma,
                  double* F) {
  Prim L = primitives(dim, uL, gamma), R = primitives(dim, uR, gamma);
  double lam = std::fmax(std::fabs(L.v[l]) + sound_speed(L, gamma),
                         std::fabs(R.v[l]) + sound_speed(R, gamma));
  double FL[8], FR[8];
  euler_flux(dim, l, uL, gamma, FL);
  euler_flux(dim, l, uR, gamma, FR);
  for (int v = 0; v < dim + 2; ++v) F[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * lam * (uR[v] - uL[v]);
}

// Roe-averaged normal velocity and sound speed, used for the Davis/Einfeldt wave-speed
// estimates of HLL and HLLC.
void roe_speeds(int dim, int l, const double* uL, const double* uR, double gamma,
                double& SL, double& SR) {
  Prim L = primitives(dim, uL, gamma), R = primitives(dim, uR, gamma);
  double sL = std::sqrt(L.rho), sR = std::sqrt(R.rho);
  double HL = (uL[dim + 1] + L.p) / L.rho, HR = (uR[dim + 1] + R.p) / R.rho;
  double vt[3], v2 = 0.0;
  for (int d = 0; d < dim; ++d) {
    vt[d] = (sL * L.v[d] + sR * R.v[d]) / (sL + sR);
    v2 += vt[d] * vt[d];
  }
  double Ht = (sL * HL + sR * HR) / (sL + sR);
  double at = std::sqrt((gamma - 1.0) * (Ht - 0.5 * v2));
  double aL = sound_speed(L, gamma), aR = sound_speed(R, gamma);
  SL = std::fmin(L.v[l] - aL, vt[l] - at);
  SR = std::fmax(R.v[l] + aR, vt[l] + at);
}

// HLL flux (Harten, Lax, van Leer), the paper's second surface-flux option (Sec. 3.1.1).
void hll_flux(int dim, int l, const double* uL, const double* uR, double gamma, double* F) {
  double SL, SR;
  roe_speeds(dim, l, uL, uR, gamma, SL, SR);
  double FL[8], FR[8];
  euler_flux(dim, l, uL, gamma, FL);
  euler_flux(dim, l, uR, gamma, FR);
  const int nv = dim + 2;
  if (SL >= 0.0) { for (int v = 0; v < nv; ++v) F[v] = FL[v]; return; }
  if (SR <= 0.0) { for (int v = 0; v < nv; ++v) F[v] = FR[v]; return; }
  for (int v = 0; v < nv; ++v)
    F[v] = (SR * FL[v] - SL * FR[v] + SL * SR * (uR[v] - uL[v])) / (SR - SL);
}

// HLLC flux (Toro, Spruce and Speares 1994) with the same Davis/Einfeldt speeds.
// READING: the paper names LF and HLL only; HLLC is the surface flux of the 3D
// Taylor-Green workload.  Branches: S_L >= 0 -> F_L; S* >= 0 -> F*_L; S_R > 0 -> F*_R;
// else F_R.  Star states U*_K = rho_K (S_K - u_K)/(S_K - S*) (1, S* e_l + tangential u,
// E_K/rho_K + (S* - u_K)(S* + p_K/(rho_K (S_K - u_K)))).
void hllc_flux(int dim, int l, const double* uL, const double* uR, double gamma, double* F) {
  double SL, SR;
  roe_speeds(dim, l, uL, uR, gamma, SL, SR);
  Prim L = primitives(dim, uL, gamma), R = primitives(dim, uR, gamma);
  double FL[8], FR[8];
  euler_flux(dim, l, uL, gamma, FL);
  euler_flux(dim, l, uR, gamma, FR);
  const int nv = dim + 2;
  double uLn = L.v[l], uRn = R.v[l];
  double Sstar = (R.p - L.p + L.rho * uLn * (SL - uLn) - R.rho * uRn * (SR - uRn)) /
                 (L.rho * (SL - uLn) - R.rho * (SR - uRn));
  auto star = [&](const Prim& K, const double* uK, double SK, double* Us) {
    double fac = K.rho * (SK - K.v[l]) / (SK - Sstar);
    Us[0] = fac;
    for (int d = 0; d < dim; ++d) Us[1 + d] = fac * (d == l ? Sstar : K.v[d]);
    Us[dim + 1] = fac * (uK[dim + 1] / K.rho +
                         (Sstar - K.v[l]) * (Sstar + K.p / (K.rho * (SK - K.v[l]))));
  };
  double Us[8];
  if (SL >= 0.0) {
    for (int v = 0; v < nv; ++v) F[v] = FL[v];
  } else if (Sstar >= 0.0) {
    star(L, uL, SL, Us);
    for (int v = 0; v < nv; ++v) F[v] = FL[v] + SL * (Us[v] - uL[v]);
  } else if (SR > 0.0) {
    star(R, uR, SR, Us);
    for (int v = 0; v < nv; ++v) F[v] = FR[v] + SR * (Us[v] - uR[v]);
  } else {
    for (int v = 0; v < nv; ++v) F[v] = FR[v];
  }
}

void surface_flux(int kind, int dim, int l, const double* uL, const double* uR, double gamma,
                  double* F) {
  switch (kind) {
    case ORC_SURF_RUSANOV: rusanov_flux(dim, l, uL, uR, gamma, F); break;
    case ORC_SURF_HLLC: hllc_flux(dim, l, uL, uR, gamma, F); break;
    case ORC_SURF_HLL: hll_flux(dim, l, uL, uR, gamma, F); break;
    case ORC_SURF_EC: ec_flux(dim, l, uL, uR, gamma, F); break;
    default: central_flux(dim, l, uL, uR, gamma, F); break;
  }
}

// ---------------------------------------------------------------------------------------
// Mesh indexing.  Element order is lexicographic with x fastest; node order within an
// element is lexicographic with i (the x index) fastest.  The state is SoA:
// U[(v * n_elem + e) * n_nodes + node].
// ---------------------------------------------------------------------------------------
struct Mesh {
  int dim, N, n1, nel[3], n_elem, n_nodes;
  double dx[3];
  explicit Mesh(const OrcProblem& P) {
    dim = P.dim;
    N = P.N;
    n1 = N + 1;
    n_elem = 1;
    n_nodes = 1;
    for (int l = 0; l < 3; ++l) {
      nel[l] = (l < dim) ? P.nel[l] : 1;
      dx[l] = (l < dim) ? (P.hi[l] - P.lo[l]) / nel[l] : 1.0;
      n_elem *= nel[l];
      if (l < dim) n_nodes *= n1;
    }
  }
  int elem(const int c[3]) const { return c[0] + nel[0] * (c[1] + nel[1] * c[2]); }
  void elem_coords(int e, int c[3]) const {
    c[0] = e % nel[0];
    c[1] = (e / nel[0]) % nel[1];
    c[2] = e / (nel[0] * nel[1]);
  }
  int node(const int ijk[3]) const { return ijk[0] + n1 * (ijk[1] + n1 * ijk[2]); }
  void node_coords(int nd, int ijk[3]) const {
    ijk[0] = nd % n1;
    ijk[1] = (nd / n1) % n1;
    ijk[2] = nd / (n1 * n1);
    if (dim == 2) ijk[2] = 0;
  }
  // periodic neighbour of element e in direction l, offset +1 or -1
  int neighbour(int e, int l, int off) const {
    int c[3];
    elem_coords(e, c);
    c[l] = (c[l] + off + nel[l]) % nel[l];
    return elem(c);
  }
};

// Boundary flux F* in direction l at domain face f (Sec. 3.1.1 "Surface Fluxes": one
// functor per boundary type; Sec. 4 set-ups: enforced weakly through the numerical flux).
// own_left: the element's own trace is the left state (upper face).  READINGS: slip wall --
// the Riemann flux against the mirror state (normal momentum reversed); supersonic inflow --
// the flux of the prescribed state itself, F^l(U_b); supersonic outflow --
// the interior state's flux F^l(U-); free-stream Dirichlet -- the Riemann flux against U_b.
void boundary_flux(const OrcProblem& P, int f, int l, const double* uown, bool own_left, double* F) {
  const int dim = P.dim, nv = dim + 2;
  double ub[8];
  switch (P.bc[f]) {
    case ORC_BC_SLIP_WALL:
      for (int v = 0; v < nv; ++v) ub[v] = uown[v];
      ub[1 + l] = -uown[1 + l];
      break;
    case ORC_BC_INFLOW:
      euler_flux(dim, l, P.bc_state[f], P.gamma, F);
      return;
    case ORC_BC_OUTFLOW:
      euler_flux(dim, l, uown, P.gamma, F);
      return;
    default:  // ORC_BC_DIRICHLET
      for (int v = 0; v < nv; ++v) ub[v] = P.bc_state[f][v];
      break;
  }
  if (own_left) surface_flux(P.surface, dim, l, uown, ub, P.gamma, F);
  else surface_flux(P.surface, dim, l, ub, uown, P.gamma, F);
}

// Whether face side (0 lower, 1 upper) of element e in direction l lies on a non-periodic
// domain face; returns that face's index or -1.
int boundary_face(const OrcProblem& P, const Mesh& M, int e, int l, int side) {
  const int f = 2 * l + side;
  if (P.bc[f] == ORC_BC_PERIODIC) return -1;
  int c[3];
  M.elem_coords(e, c);
  return (side ? c[l] == M.nel[l] - 1 : c[l] == 0) ? f : -1;
}

void load_node(const Mesh& M, int nv, const double* U, int e, int nd, double* u) {
  for (int v = 0; v < nv; ++v) u[v] = U[((size_t)v * M.n_elem + e) * M.n_nodes + nd];
}

// ---------------------------------------------------------------------------------------
// Semi-discrete Euler residual on one element (Sec. 3.1.1).
//   strong (Eq. vol_weak):     R_i = -sum_l (2/dx_l) sum_m D_{i_l m} F^l(U_m)
//   weak (by parts, SBP):      R_i =  sum_l (2/dx_l) sum_m (w_m/w_{i_l}) D_{m i_l} F^l(U_m)
//   two-point (Eq. vol_split): R_i = -sum_l (2/dx_l) 2 sum_m D_{i_l m} F#^l(U_i, U_m)
// On the affine Cartesian element J = prod_l dx_l/2 and Ja^l = J (2/dx_l) e_l, so
// (1/J) D Ja^l.F = (2/dx_l) D F^l and the averaged metric in Eq. vol_split is exact.
// Surface (Eq. surf_int): with F* = F*(U_L, U_R; e_l) computed left-to-right,
//   upper face (i_l = N):  R -= (2/dx_l)/w_N (F* - F^l(U_own))
//   lower face (i_l = 0):  R += (2/dx_l)/w_0 (F* - F^l(U_own))
// and in the weak form only F* is lifted (the volume term already carries F^l(U_own)).
// ---------------------------------------------------------------------------------------
void euler_element_residual(const OrcProblem& P, const Mesh& M, const Ops& ops,
                            const double* U, int e, double* dU) {
  const int dim = M.dim, n1 = M.n1, N = M.N, nv = dim + 2;
  const double gamma = P.gamma;
  std::vector<double> R((size_t)M.n_nodes * nv, 0.0);
  double ui[8], um[8], F[8];

  // volume term
  for (int nd = 0; nd < M.n_nodes; ++nd) {
    int ijk[3];
    M.node_coords(nd, ijk);
    load_node(M, nv, U, e, nd, ui);
    for (int l = 0; l < dim; ++l) {
      const double s = 2.0 / M.dx[l];
      const int il = ijk[l];
      for (int m = 0; m < n1; ++m) {
        int mk[3] = {ijk[0], ijk[1], ijk[2]};
        mk[l] = m;
        load_node(M, nv, U, e, M.node(mk), um);
        if (P.volume == ORC_VOL_STRONG) {
          euler_flux(dim, l, um, gamma, F);
          for (int v = 0; v < nv; ++v) R[nd * nv + v] -= s * ops.D[il * n1 + m] * F[v];
        } else if (P.volume == ORC_VOL_WEAK) {
          euler_flux(dim, l, um, gamma, F);
          for (int v = 0; v < nv; ++v)
            R[nd * nv + v] += s * (ops.w[m] / ops.w[il]) * ops.D[m * n1 + il] * F[v];
        } else {
          if (P.volume == ORC_VOL_EC) ec_flux(dim, l, ui, um, gamma, F);
          else central_flux(dim, l, ui, um, gamma, F);
          for (int v = 0; v < nv; ++v) R[nd * nv + v] -= s * 2.0 * ops.D[il * n1 + m] * F[v];
        }
      }
    }
  }

  // surface term: both faces of each direction, every face node
  const bool weak = (P.volume == ORC_VOL_WEAK);
  for (int l = 0; l < dim; ++l) {
    const double s = 2.0 / M.dx[l];
    for (int nd = 0; nd < M.n_nodes; ++nd) {
      int ijk[3];
      M.node_coords(nd, ijk);
      if (ijk[l] != N && ijk[l] != 0) continue;
      double uown[8], unbr[8], Fs[8], Fown[8];
      load_node(M, nv, U, e, nd, uown);
      euler_flux(dim, l, uown, gamma, Fown);
      if (ijk[l] == N) {  // upper face: own state is the left state
        int nk[3] = {ijk[0], ijk[1], ijk[2]};
        nk[l] = 0;
        const int fb = boundary_face(P, M, e, l, 1);
        if (fb >= 0) {
          boundary_flux(P, fb, l, uown, true, Fs);
        } else {
          load_node(M, nv, U, M.neighbour(e, l, +1), M.node(nk), unbr);
          surface_flux(P.surface, dim, l, uown, unbr, gamma, Fs);
        }
        for (int v = 0; v < nv; ++v)
          R[nd * nv + v] -= s / ops.w[N] * (Fs[v] - (weak ? 0.0 : Fown[v]));
      }
      if (ijk[l] == 0) {  // lower face: own state is the right state
        int nk[3] = {ijk[0], ijk[1], ijk[2]};
        nk[l] = N;
        const int fb = boundary_face(P, M, e, l, 0);
        if (fb >= 0) {
          boundary_flux(P, fb, l, uown, false, Fs);
        } else {
          load_node(M, nv, U, M.neighbour(e, l, -1), M.node(nk), unbr);
          surface_flux(P.surface, dim, l, unbr, uown, gamma, Fs);
        }
        for (int v = 0; v < nv; ++v)
          R[nd * nv + v] += s / ops.w[0] * (Fs[v] - (weak ? 0.0 : Fown[v]));
      }
    }
  }

  for (int nd = 0; nd < M.n_nodes; ++nd)
    for (int v = 0; v < nv; ++v)
      dU[((size_t)v * M.n_elem + e) * M.n_nodes + nd] = R[nd * nv + v];
}

// ---------------------------------------------------------------------------------------
// Hennemann-Gassner shock capturing (Sec. 3.1.1 "Shock Indicator and Smoothing" and Eq.
// vol_blend; App. A "Shock Capturing").
//
// Modes: the nodal values of the indicator field on the element are the degree-N
// interpolant's values; its coefficients in the orthonormal tensor Legendre basis
// P~_j = sqrt((2j+1)/2) P_j follow from m = V^{-1} q along every direction, with the
// Vandermonde matrix V_ij = P~_j(x_i) on the GLL nodes (inverted by Gauss-Jordan in long
// double).
// ---------------------------------------------------------------------------------------
std::vector<double> modal_matrix(int N) {
  const int n1 = N + 1;
  std::vector<long double> x, w;
  gll_rule(N, x, w);
  std::vector<long double> A((size_t)n1 * 2 * n1, 0.0L);  // [V | I]
  for (int i = 0; i < n1; ++i) {
    for (int j = 0; j < n1; ++j) {
      long double Pj, Pjm1;
      legendre(j, x[i], Pj, Pjm1);
      A[(size_t)i * 2 * n1 + j] = std::sqrt((2.0L * j + 1.0L) / 2.0L) * Pj;
    }
    A[(size_t)i * 2 * n1 + n1 + i] = 1.0L;
  }
  for (int k = 0; k < n1; ++k) {
    int piv = k;
    for (int i = k + 1; i < n1; ++i)
      if (std::fabs(A[(size_t)i * 2 * n1 + k]) > std::fabs(A[(size_t)piv * 2 * n1 + k])) piv = i;
    for (int j = 0; j < 2 * n1; ++j) std::swap(A[(size_t)k * 2 * n1 + j], A[(size_t)piv * 2 * n1 + j]);
    const long double d = A[(size_t)k * 2 * n1 + k];
    for (int j = 0; j < 2 * n1; ++j) A[(size_t)k * 2 * n1 + j] /= d;
    for (int i = 0; i < n1; ++i) {
      if (i == k) continue;
      const long double f = A[(size_t)i * 2 * n1 + k];
      for (int j = 0; j < 2 * n1; ++j) A[(size_t)i * 2 * n1 + j] -= f * A[(size_t)k * 2 * n1 + j];
    }
  }
  std::vector<double> Vinv((size_t)n1 * n1);
  for (int i = 0; i < n1; ++i)
    for (int j = 0; j < n1; ++j) Vinv[(size_t)i * n1 + j] = (double)A[(size_t)i * 2 * n1 + n1 + j];
  return Vinv;
}

// Modal coefficients m[node(i,j,k)] (mode indices in place of node indices) of one
// element's nodal field q: V^{-1} applied along direction 0, then 1, then 2.
void to_modes(const Mesh& M, const std::vector<double>& Vinv, const double* q, double* m) {
  const int n1 = M.n1;
  std::vector<double> a(q, q + M.n_nodes), b(M.n_nodes);
  for (int l = 0; l < M.dim; ++l) {
    for (int nd = 0; nd < M.n_nodes; ++nd) {
      int ijk[3];
      M.node_coords(nd, ijk);
      double acc = 0.0;
      for (int j = 0; j < n1; ++j) {
        int jk[3] = {ijk[0], ijk[1], ijk[2]};
        jk[l] = j;
        acc += Vinv[(size_t)ijk[l] * n1 + j] * a[M.node(jk)];
      }
      b[nd] = acc;
    }
    a.swap(b);
  }
  for (int nd = 0; nd < M.n_nodes; ++nd) m[nd] = a[nd];
}

// Smoothness indicator of element e: the field rho p (the paper's choice for its reacting
// and shock cases), its modes, and
//   E = max(E_high^(N) / E_tot^(N), E_high^(N-1) / E_tot^(N-1)),
// E_tot^(K) the energy of the modes with max(i,j,k) <= K, E_high^(K) of those with
// max(i,j,k) = K.  (A zero total energy gives the ratio 0.)
double smoothness(const OrcProblem& P, const Mesh& M, const std::vector<double>& Vinv,
                  const double* U, int e) {
  const int nv = M.dim + 2, N = M.N;
  std::vector<double> q(M.n_nodes), m(M.n_nodes);
  for (int nd = 0; nd < M.n_nodes; ++nd) {
    double u[8];
    load_node(M, nv, U, e, nd, u);
    Prim pr = primitives(M.dim, u, P.gamma);
    q[nd] = pr.rho * pr.p;
  }
  to_modes(M, Vinv, q.data(), m.data());
  double tot_n = 0.0, tot_nm1 = 0.0, high_n = 0.0, high_nm1 = 0.0;
  for (int nd = 0; nd < M.n_nodes; ++nd) {
    int ijk[3];
    M.node_coords(nd, ijk);
    int mx = ijk[0];
    for (int l = 1; l < M.dim; ++l) mx = std::max(mx, ijk[l]);
    const double e2 = m[nd] * m[nd];
    tot_n += e2;
    if (mx <= N - 1) tot_nm1 += e2;
    if (mx == N) high_n += e2;
    if (mx == N - 1) high_nm1 += e2;
  }
  const double r1 = tot_n > 0.0 ? high_n / tot_n : 0.0;
  const double r2 = tot_nm1 > 0.0 ? high_nm1 / tot_nm1 : 0.0;
  return std::fmax(r1, r2);
}

// Blending coefficients of all elements:
//   alpha_raw = 1 / (1 + exp(-(s/T)(E - T))),  T = 0.5 * 10^(-1.8 (N+1)^(1/4));
// READINGS (the paper names alpha_min, alpha_max and s without values): alpha_raw below
// alpha_min is set to 0 and alpha_raw is capped at alpha_max (Hennemann and Gassner's
// clipping; defaults 0.001, 0.5 and s = ln(9999), which puts alpha(E = 0) at 1e-4); then the
// face-neighbourhood maximum alpha_e = max(alpha_raw_e, alpha_raw of the 2 dim face
// neighbours), taken once over the raw values.
void shock_alpha(const OrcProblem& P, const double* U, double* alpha_raw, double* alpha) {
  Mesh M(P);
  const std::vector<double> Vinv = modal_matrix(M.N);
  const double T = 0.5 * std::pow(10.0, -1.8 * std::pow(M.N + 1.0, 0.25));
  for (int e = 0; e < M.n_elem; ++e) {
    const double E = smoothness(P, M, Vinv, U, e);
    double a = 1.0 / (1.0 + std::exp(-(P.sharpness / T) * (E - T)));
    if (a < P.alpha_min) a = 0.0;
    alpha_raw[e] = std::fmin(a, P.alpha_max);
  }
  for (int e = 0; e < M.n_elem; ++e) {
    double a = alpha_raw[e];
    for (int l = 0; l < M.dim; ++l)
      for (int off = -1; off <= 1; off += 2)
        if (boundary_face(P, M, e, l, off > 0 ? 1 : 0) < 0)  // no neighbour across a boundary
          a = std::fmax(a, alpha_raw[M.neighbour(e, l, off)]);
    alpha[e] = a;
  }
}

// First-order finite-volume residual on the GLL sub-cell grid of element e (Eq. vol_blend's
// R^FV, App. A "Shock Capturing"): along direction l node i is the centre of a sub-cell of
// reference width w_i (the sub-cell faces sit at -1 + w_0 + ... + w_{i-1}), so
//   R_i -= (2/dx_l) / w_i (f_{i+1/2} - f_{i-1/2}),
// f_{i+1/2} = F*(U_i, U_{i+1}) between nodes of the element and, at the element faces, the
// DG surface flux with the neighbour's trace (f_{-1/2} = F*(U_nbr,N, U_0),
// f_{N+1/2} = F*(U_N, U_nbr,0)).  READING: every sub-cell interface uses the context's
// surface flux (the paper asks for the same numerical flux functions as the DG surface;
// Rusanov in its cases).
void fv_element_residual(const OrcProblem& P, const Mesh& M, const Ops& ops, const double* U, int e,
                         double* dU) {
  const int dim = M.dim, N = M.N, nv = dim + 2;
  std::vector<double> R((size_t)M.n_nodes * nv, 0.0);
  for (int l = 0; l < dim; ++l) {
    const double s = 2.0 / M.dx[l];
    for (int nd = 0; nd < M.n_nodes; ++nd) {
      int ijk[3];
      M.node_coords(nd, ijk);
      const int il = ijk[l];
      double uo[8], ua[8], fm[8], fp[8];
      load_node(M, nv, U, e, nd, uo);
      int nk[3] = {ijk[0], ijk[1], ijk[2]};
      const int fl = il == 0 ? boundary_face(P, M, e, l, 0) : -1;
      if (fl >= 0) {
        boundary_flux(P, fl, l, uo, false, fm);
      } else {
        if (il == 0) {
          nk[l] = N;
          load_node(M, nv, U, M.neighbour(e, l, -1), M.node(nk), ua);
        } else {
          nk[l] = il - 1;
          load_node(M, nv, U, e, M.node(nk), ua);
        }
        surface_flux(P.surface, dim, l, ua, uo, P.gamma, fm);
      }
      const int fu = il == N ? boundary_face(P, M, e, l, 1) : -1;
      if (fu >= 0) {
        boundary_flux(P, fu, l, uo, true, fp);
      } else {
        if (il == N) {
          nk[l] = 0;
          load_node(M, nv, U, M.neighbour(e, l, +1), M.node(nk), ua);
        } else {
          nk[l] = il + 1;
          load_node(M, nv, U, e, M.node(nk), ua);
        }
        surface_flux(P.surface, dim, l, uo, ua, P.gamma, fp);
      }
      for (int v = 0; v < nv; ++v) R[nd * nv + v] -= s / ops.w[il] * (fp[v] - fm[v]);
    }
  }
  for (int nd = 0; nd < M.n_nodes; ++nd)
    for (int v = 0; v < nv; ++v) dU[((size_t)v * M.n_elem + e) * M.n_nodes + nd] = R[nd * nv + v];
}

// ---------------------------------------------------------------------------------------
// Curvilinear elements (Sec. 3.1.1: element maps x = X(xi), Jacobian J_dm = dx_d/dxi_m,
// J = det, contravariant vectors Ja^l satisfying the discrete GCL sum_l d_xi_l Ja^l = 0).
// The map is the degree-N interpolant of the given node coordinates.  Metric terms:
//   2D  Ja^1 = (y_eta, -x_eta), Ja^2 = (-y_xi, x_xi);
//   3D  the conservative curl form Ja^i_n = -1/2 [curl_xi (X_l grad_xi X_m - X_m grad_xi X_l)]_i,
//       (n, m, l) cyclic,
// derivatives by D along the lines; J = x_xi y_eta - x_eta y_xi (2D) or the determinant of
// dx/dxi (3D).  With these, d_xi-divergences of Ja^l vanish to rounding (the D's commute).
// ---------------------------------------------------------------------------------------
struct Metrics {
  std::vector<double> Ja;  // [elem][node][l][d]
  std::vector<double> J;   // [elem][node]
};

Metrics curved_metrics(const OrcProblem& P, const Mesh& M, const Ops& ops) {
  const int dim = M.dim, n1 = M.n1, np = M.n_nodes;
  Metrics G;
  G.Ja.assign((size_t)M.n_elem * np * 9, 0.0);
  G.J.assign((size_t)M.n_elem * np, 0.0);
  auto X = [&](int d, int e, int nd) { return P.coords[((size_t)d * M.n_elem + e) * np + nd]; };
  // derivative along reference direction k of a nodal field f at node nd
  auto deriv = [&](const std::vector<double>& f, int k, int nd) {
    int ijk[3];
    M.node_coords(nd, ijk);
    double acc = 0.0;
    for (int m = 0; m < n1; ++m) {
      int mk[3] = {ijk[0], ijk[1], ijk[2]};
      mk[k] = m;
      acc += ops.D[ijk[k] * n1 + m] * f[M.node(mk)];
    }
    return acc;
  };
  for (int e = 0; e < M.n_elem; ++e) {
    std::vector<std::vector<double>> x(dim, std::vector<double>(np));
    for (int d = 0; d < dim; ++d)
      for (int nd = 0; nd < np; ++nd) x[d][nd] = X(d, e, nd);
    // dx_d / dxi_k at every node
    std::vector<double> dx((size_t)np * 9);
    for (int nd = 0; nd < np; ++nd)
      for (int d = 0; d < dim; ++d)
        for (int k = 0; k < dim; ++k) dx[(size_t)nd * 9 + d * 3 + k] = deriv(x[d], k, nd);
    double* Ja = &G.Ja[(size_t)e * np * 9];
    if (dim == 2) {
      for (int nd = 0; nd < np; ++nd) {
        const double* g = &dx[(size_t)nd * 9];  // g[d*3+k] = dx_d/dxi_k
        Ja[nd * 9 + 0 * 3 + 0] = g[1 * 3 + 1];   // Ja^1 = ( y_eta, -x_eta)
        Ja[nd * 9 + 0 * 3 + 1] = -g[0 * 3 + 1];
        Ja[nd * 9 + 1 * 3 + 0] = -g[1 * 3 + 0];  // Ja^2 = (-y_xi,  x_xi)
        Ja[nd * 9 + 1 * 3 + 1] = g[0 * 3 + 0];
        G.J[(size_t)e * np + nd] = g[0] * g[4] - g[1] * g[3];
      }
    } else {
      for (int n = 0; n < 3; ++n) {
        const int m = (n + 1) % 3, l = (n + 2) % 3;
        // V_k = X_l d_k X_m - X_m d_k X_l at the nodes
        std::vector<std::vector<double>> V(3, std::vector<double>(np));
        for (int nd = 0; nd < np; ++nd)
          for (int k = 0; k < 3; ++k)
            V[k][nd] = x[l][nd] * dx[(size_t)nd * 9 + m * 3 + k] - x[m][nd] * dx[(size_t)nd * 9 + l * 3 + k];
        for (int nd = 0; nd < np; ++nd)
          for (int i = 0; i < 3; ++i) {
            const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
            const double curl = deriv(V[i2], i1, nd) - deriv(V[i1], i2, nd);
            Ja[nd * 9 + i * 3 + n] = -0.5 * curl;
          }
      }
      for (int nd = 0; nd < np; ++nd) {
        const double* g = &dx[(size_t)nd * 9];
        G.J[(size_t)e * np + nd] = g[0] * (g[4] * g[8] - g[5] * g[7]) - g[1] * (g[3] * g[8] - g[5] * g[6]) +
                                   g[2] * (g[3] * g[7] - g[4] * g[6]);
      }
    }
  }
  return G;
}

// Riemann flux in the unit direction n: the states' momenta are expressed in an orthonormal
// frame (n, t1[, t2]), the flux of direction 0 is evaluated there and its momentum rotated
// back (rotational invariance of the Euler equations).
void normal_frame(int dim, const double* n, double t[2][3]) {
  if (dim == 2) {
    t[0][0] = -n[1]; t[0][1] = n[0]; t[0][2] = 0.0;
    return;
  }
  // t1: the unit vector orthogonal to n built from the axis least aligned with n
  int a = 0;
  if (std::fabs(n[1]) < std::fabs(n[a])) a = 1;
  if (std::fabs(n[2]) < std::fabs(n[a])) a = 2;
  double e[3] = {0.0, 0.0, 0.0};
  e[a] = 1.0;
  double c[3] = {n[1] * e[2] - n[2] * e[1], n[2] * e[0] - n[0] * e[2], n[0] * e[1] - n[1] * e[0]};
  const double cn = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
  for (int d = 0; d < 3; ++d) t[0][d] = c[d] / cn;
  t[1][0] = n[1] * t[0][2] - n[2] * t[0][1];
  t[1][1] = n[2] * t[0][0] - n[0] * t[0][2];
  t[1][2] = n[0] * t[0][1] - n[1] * t[0][0];
}

void normal_riemann(int kind, int dim, const double* n, const double* uL, const double* uR, double gamma,
                    double* F) {
  const int nv = dim + 2;
  double t[2][3];
  normal_frame(dim, n, t);
  double rL[8], rR[8], Fr[8];
  rL[0] = uL[0];
  rR[0] = uR[0];
  rL[nv - 1] = uL[nv - 1];
  rR[nv - 1] = uR[nv - 1];
  for (int c = 0; c < dim; ++c) {
    const double* b = c == 0 ? n : t[c - 1];
    rL[1 + c] = 0.0;
    rR[1 + c] = 0.0;
    for (int d = 0; d < dim; ++d) {
      rL[1 + c] += uL[1 + d] * b[d];
      rR[1 + c] += uR[1 + d] * b[d];
    }
  }
  surface_flux(kind, dim, 0, rL, rR, gamma, Fr);
  F[0] = Fr[0];
  F[nv - 1] = Fr[nv - 1];
  for (int d = 0; d < dim; ++d) {
    F[1 + d] = Fr[1] * n[d];
    for (int c = 1; c < dim; ++c) F[1 + d] += Fr[1 + c] * t[c - 1][d];
  }
}

// Boundary flux along the contravariant normal n at domain face f of a curved mesh (the
// functors of boundary_flux, Sec. 3.1.1, in the face's frame): slip wall -- the Riemann flux
// against the mirror state, the velocity reflected across the wall, m - 2 (m . n) n;
// supersonic inflow -- the flux of U_b along n; supersonic outflow -- the interior flux along
// n; Dirichlet -- the Riemann flux against U_b.  own_left: the element's trace is the state
// on the lower side of the face.
void curved_boundary_flux(const OrcProblem& P, int f, const double* n, const double* uown, bool own_left,
                          double* F) {
  const int dim = P.dim, nv = dim + 2;
  double ub[8], Fd[8];
  switch (P.bc[f]) {
    case ORC_BC_INFLOW:
    case ORC_BC_OUTFLOW: {
      const double* u = P.bc[f] == ORC_BC_INFLOW ? P.bc_state[f] : uown;
      for (int v = 0; v < nv; ++v) F[v] = 0.0;
      for (int d = 0; d < dim; ++d) {
        euler_flux(dim, d, u, P.gamma, Fd);
        for (int v = 0; v < nv; ++v) F[v] += n[d] * Fd[v];
      }
      return;
    }
    case ORC_BC_SLIP_WALL: {
      double mn = 0.0;
      for (int d = 0; d < dim; ++d) mn += uown[1 + d] * n[d];
      for (int v = 0; v < nv; ++v) ub[v] = uown[v];
      for (int d = 0; d < dim; ++d) ub[1 + d] = uown[1 + d] - 2.0 * mn * n[d];
      break;
    }
    default:  // Dirichlet
      for (int v = 0; v < nv; ++v) ub[v] = P.bc_state[f][v];
      break;
  }
  if (own_left) normal_riemann(P.surface, dim, n, uown, ub, P.gamma, F);
  else normal_riemann(P.surface, dim, n, ub, uown, P.gamma, F);
}

// Residual of element e on a curved mesh (Sec. 3.1.1, Eqs. vol_weak and vol_split with the
// metric terms; Eq. surf_int):
//   strong:    R_i = -(1/J_i) sum_l sum_m D_{i_l m} Ja^l(m) . F(U_m)
//   two-point: R_i = -(2/J_i) sum_l sum_m D_{i_l m} {{Ja^l}}_{im} . F#(U_i, U_m)
//   surface:   R_i -/+ (1/(J_i w)) (|Ja^l| F*(U_L, U_R; n) - Ja^l . F(U_i)),  n = Ja^l / |Ja^l|
// on the upper / lower face of direction l, Ja^l taken at the own face node (the neighbour's
// is the same: it depends only on the face's nodes).
void curved_element_residual(const OrcProblem& P, const Mesh& M, const Ops& ops, const Metrics& G,
                             const double* U, int e, double* dU) {
  const int dim = M.dim, n1 = M.n1, N = M.N, nv = dim + 2, np = M.n_nodes;
  std::vector<double> R((size_t)np * nv, 0.0);
  auto Ja = [&](int el, int nd, int l, int d) { return G.Ja[(((size_t)el * np + nd) * 3 + l) * 3 + d]; };
  for (int nd = 0; nd < np; ++nd) {
    int ijk[3];
    M.node_coords(nd, ijk);
    double ui[8], um[8], F[8];
    load_node(M, nv, U, e, nd, ui);
    const double iJ = 1.0 / G.J[(size_t)e * np + nd];
    for (int l = 0; l < dim; ++l) {
      for (int m = 0; m < n1; ++m) {
        int mk[3] = {ijk[0], ijk[1], ijk[2]};
        mk[l] = m;
        const int nm = M.node(mk);
        load_node(M, nv, U, e, nm, um);
        const double Dim = ops.D[ijk[l] * n1 + m];
        for (int d = 0; d < dim; ++d) {
          if (P.volume == ORC_VOL_STRONG) {
            euler_flux(dim, d, um, P.gamma, F);
            for (int v = 0; v < nv; ++v) R[nd * nv + v] -= iJ * Dim * Ja(e, nm, l, d) * F[v];
          } else {
            ec_flux(dim, d, ui, um, P.gamma, F);
            const double a = 0.5 * (Ja(e, nd, l, d) + Ja(e, nm, l, d));
            for (int v = 0; v < nv; ++v) R[nd * nv + v] -= 2.0 * iJ * Dim * a * F[v];
          }
        }
      }
    }
  }
  for (int l = 0; l < dim; ++l) {
    for (int nd = 0; nd < np; ++nd) {
      int ijk[3];
      M.node_coords(nd, ijk);
      if (ijk[l] != 0 && ijk[l] != N) continue;
      const double iJ = 1.0 / G.J[(size_t)e * np + nd];
      double uown[8], unbr[8], Fs[8], Fo[8], Fd[8], n[3] = {0.0, 0.0, 0.0};
      load_node(M, nv, U, e, nd, uown);
      double s2 = 0.0;
      for (int d = 0; d < dim; ++d) s2 += Ja(e, nd, l, d) * Ja(e, nd, l, d);
      const double s = std::sqrt(s2);
      for (int d = 0; d < dim; ++d) n[d] = Ja(e, nd, l, d) / s;
      for (int v = 0; v < nv; ++v) Fo[v] = 0.0;
      for (int d = 0; d < dim; ++d) {
        euler_flux(dim, d, uown, P.gamma, Fd);
        for (int v = 0; v < nv; ++v) Fo[v] += Ja(e, nd, l, d) * Fd[v];
      }
      for (int side = 0; side < 2; ++side) {
        if (side == 1 && ijk[l] != N) continue;
        if (side == 0 && ijk[l] != 0) continue;
        const int fb = boundary_face(P, M, e, l, side);
        if (fb >= 0) {
          curved_boundary_flux(P, fb, n, uown, side == 1, Fs);
        } else {
          int nk[3] = {ijk[0], ijk[1], ijk[2]};
          nk[l] = side ? 0 : N;
          load_node(M, nv, U, M.neighbour(e, l, side ? +1 : -1), M.node(nk), unbr);
          if (side) normal_riemann(P.surface, dim, n, uown, unbr, P.gamma, Fs);
          else normal_riemann(P.surface, dim, n, unbr, uown, P.gamma, Fs);
        }
        const double c = (side ? -1.0 : 1.0) * iJ / ops.w[side ? N : 0];
        for (int v = 0; v < nv; ++v) R[nd * nv + v] += c * (s * Fs[v] - Fo[v]);
      }
    }
  }
  for (int nd = 0; nd < np; ++nd)
    for (int v = 0; v < nv; ++v) dU[((size_t)v * M.n_elem + e) * M.n_nodes + nd] = R[nd * nv + v];
}

int n_vars(const OrcProblem& P) {
  if (P.equations == ORC_NS_REACTING) return P.mech->n_species + P.dim + 1 + (P.two_temperature ? 1 : 0);
  return P.dim + 2;
}

int check_reacting_bc(const OrcProblem& P);

int check_problem(const OrcProblem& P) {
  if (P.dim != 2 && P.dim != 3) return -1;
  if (P.N < 1 || P.N > 15) return -1;
  for (int l = 0; l < P.dim; ++l)
    if (P.nel[l] < 1 || !(P.hi[l] > P.lo[l])) return -1;
  if (P.equations == ORC_NS_REACTING) {
    if (!P.mech || P.mech->n_species < 1 || P.mech->n_species > 8 || P.mech->n_reactions < 0 ||
        P.mech->n_reactions > 32)
      return -1;
    if (P.volume != ORC_VOL_STRONG || P.surface != ORC_SURF_RUSANOV) return -6;
    if (P.rho_floor > 0.0 || P.p_floor > 0.0) return -6;
    if (P.mu < 0.0 || !(P.prandtl > 0.0)) return -1;
    if (P.shock) return -6;
    if (P.coords) {  // curved meshes: periodic, without the species limiter (whose element
                     // mean would need the Jacobian weights)
      for (int f = 0; f < 2 * P.dim; ++f)
        if (P.bc[f] != ORC_BC_PERIODIC) return -6;
      if (P.species_limiter) return -6;
    }
    if (P.two_temperature) {
      if (P.two_temperature != 1) return -1;
      for (int s = 0; s < P.mech->n_species; ++s)
        if (!(P.mech->theta_v[s] >= 0.0)) return -1;
    }
    return check_reacting_bc(P);
  }
  if (P.equations != ORC_EULER || P.two_temperature) return -6;
  for (int f = 0; f < 2 * P.dim; ++f) {
    if (P.bc[f] < ORC_BC_PERIODIC || P.bc[f] > ORC_BC_DIRICHLET) return -1;  // no viscosity: no no-slip
    if ((P.bc[f] == ORC_BC_PERIODIC) != (P.bc[f ^ 1] == ORC_BC_PERIODIC)) return -1;  // pairs
    if (P.bc[f] == ORC_BC_INFLOW || P.bc[f] == ORC_BC_DIRICHLET) {
      Prim q = primitives(P.dim, P.bc_state[f], P.gamma);
      if (!(q.rho > 0.0) || !(q.p > 0.0)) return -1;
    }
  }
  if (P.coords) {  // curved meshes: strong or two-point volume form, no blending
    if (P.shock || P.rho_floor > 0.0 || P.p_floor > 0.0) return -6;
    if (P.volume != ORC_VOL_STRONG && P.volume != ORC_VOL_EC) return -6;
  }
  if (P.shock && (P.N < 2 || !(P.alpha_min >= 0.0) || !(P.alpha_max <= 1.0) ||
                  !(P.alpha_min <= P.alpha_max) || !(P.sharpness > 0.0)))
    return -1;
  return 0;
}

// ---------------------------------------------------------------------------------------
// Reacting Navier-Stokes (Sec. 2 "Thermochemical non-equilibrium", single temperature):
// U = (rho_1..rho_ns, rho u, rho v, rho w, E).  READINGS: calorically perfect species
// (Sec. 2 closure), E = sum rho_s (cv_s T + h0_s) + rho |u|^2 / 2, p = sum rho_s R_s T;
// frozen sound speed a^2 = (1 + sum rho_s R_s / sum rho_s cv_s) p / rho; no species
// diffusion; constant viscosity mu; conductivity k = mu c_p / Pr with the mixture c_p.
// Two-temperature model (Sec. 2 "Thermal nonequilibrium coupling", "Total energy and
// closure"; Sec. 3.1.3 Eqs. src_vector, src_landau_teller): E_v appended to U, cv_s the
// translational-rotational heat capacity, E_v = sum rho_s e_v,s(T_v) with harmonic
// oscillators; the vibrational mode is frozen in the sound speed; READING: conductivity of
// the vibrational mode k_v = mu c_v,v / Pr with c_v,v = (1/rho) dE_v/dT_v (the same
// Eucken-type ratio as k), and the total-energy flux carries both heat fluxes (E contains E_v).
// ---------------------------------------------------------------------------------------
struct Mix {
  double rho, v[3], T, p, a, cp, rcv;  // rcv = sum rho_s cv_s
  double Tv, Ev, cvv;                  // two-temperature: T_v, E_v, (1/rho) dE_v/dT_v
};

// Vibrational energy per unit mass of a harmonic oscillator with characteristic temperature
// theta at temperature T (Sec. 3.1.3, below Eq. src_landau_teller):
// e_v = R theta / (exp(theta / T) - 1); 0 for an atom (theta = 0).
double vib_energy(double R, double theta, double T) {
  if (theta <= 0.0) return 0.0;
  return R * theta / std::expm1(theta / T);
}

// d e_v / dT of the same oscillator.
double vib_heat(double R, double theta, double T) {
  if (theta <= 0.0) return 0.0;
  const double x = theta / T, em = std::expm1(x);
  return R * x * x * (em + 1.0) / (em * em);
}

// E_v of the partial densities rho_s at vibrational temperature T.
double vib_energy_density(const OrcMech& m, const double* rho_s, double T) {
  double Ev = 0.0;
  for (int s = 0; s < m.n_species; ++s) Ev += rho_s[s] * vib_energy(m.R[s], m.theta_v[s], T);
  return Ev;
}

// The vibrational temperature with E_v(T_v) = Ev: E_v grows strictly with T_v, so bisection
// on [1e-3, 1e7] K to the last bit finds the root (NaN when no species vibrates or Ev <= 0).
double vib_temperature(const OrcMech& m, const double* rho_s, double Ev) {
  double lo = 1e-3, hi = 1e7;
  if (!(Ev > 0.0) || !(vib_energy_density(m, rho_s, hi) > Ev)) return std::nan("");
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (vib_energy_density(m, rho_s, mid) < Ev) lo = mid;
    else hi = mid;
  }
  return 0.5 * (lo + hi);
}

Mix mixture(const OrcProblem& P, const double* u) {
  const OrcMech& m = *P.mech;
  const int ns = m.n_species, dim = P.dim;
  Mix q;
  q.rho = 0.0;
  double rR = 0.0, rcv = 0.0, rh0 = 0.0;
  for (int s = 0; s < ns; ++s) {
    q.rho += u[s];
    rR += u[s] * m.R[s];
    rcv += u[s] * m.cv[s];
    rh0 += u[s] * m.h0[s];
  }
  double kin = 0.0;
  for (int d = 0; d < 3; ++d) q.v[d] = 0.0;
  for (int d = 0; d < dim; ++d) {
    q.v[d] = u[ns + d] / q.rho;
    kin += u[ns + d] * q.v[d];
  }
  // two-temperature closure (Sec. 2 "Total energy and closure"): E = sum rho_s (cv_s T +
  // h0_s) + E_v + rho |u|^2 / 2 with cv_s the translational-rotational heat capacity
  q.Ev = P.two_temperature ? u[ns + dim + 1] : 0.0;
  q.T = (u[ns + dim] - q.Ev - 0.5 * kin - rh0) / rcv;
  q.p = rR * q.T;
  q.a = std::sqrt((1.0 + rR / rcv) * q.p / q.rho);
  q.cp = (rcv + rR) / q.rho;
  q.rcv = rcv;
  q.Tv = q.T;
  q.cvv = 0.0;
  if (P.two_temperature) {
    q.Tv = vib_temperature(m, u, q.Ev);
    for (int s = 0; s < ns; ++s) q.cvv += u[s] * vib_heat(m.R[s], m.theta_v[s], q.Tv);
    q.cvv /= q.rho;
  }
  return q;
}

// inviscid flux in direction l (Sec. 2, F_inv of the reacting system)
void mix_flux(const OrcProblem& P, int l, const double* u, double* F) {
  const int ns = P.mech->n_species, dim = P.dim;
  Mix q = mixture(P, u);
  for (int s = 0; s < ns; ++s) F[s] = u[s] * q.v[l];
  for (int d = 0; d < dim; ++d) F[ns + d] = u[ns + l] * q.v[d] + (d == l ? q.p : 0.0);
  F[ns + dim] = (u[ns + dim] + q.p) * q.v[l];
  if (P.two_temperature) F[ns + dim + 1] = u[ns + dim + 1] * q.v[l];  // E_v u_l
}

void mix_rusanov(const OrcProblem& P, int l, const double* uL, const double* uR, double* F) {
  const int nv = n_vars(P);
  Mix a = mixture(P, uL), b = mixture(P, uR);
  double lam = std::fmax(std::fabs(a.v[l]) + a.a, std::fabs(b.v[l]) + b.a);
  double FL[16], FR[16];
  mix_flux(P, l, uL, FL);
  mix_flux(P, l, uR, FR);
  for (int v = 0; v < nv; ++v) F[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * lam * (uR[v] - uL[v]);
}

// Arrhenius source (Sec. 3.1.3 and App. C, Eqs. src_reaction_rate and src_omega), single
// temperature:
// [X_s] = rho_s / W_s (mol/cm^3), R_r = k_f prod [X]^nu' - (k_f / K_c) prod [X]^nu'',
// omega_s = W_s sum_r (nu'' - nu') R_r (converted to kg m^-3 s^-1); momentum and energy 0.
void arrhenius(const OrcMech& m, int r, double T, double& kf, double& Kc) {
  const double Z = 1.0e4 / T;
  kf = std::exp(m.lnA[r] + m.b[r] * std::log(T) - m.Ta[r] / T);
  Kc = std::exp(m.kc[r][0] / Z + m.kc[r][1] + m.kc[r][2] * std::log(Z) + m.kc[r][3] * Z +
                m.kc[r][4] * Z * Z);
}

// Species production rates omega_s (kg m^-3 s^-1) of the partial densities rho_s at
// translational temperature T and vibrational temperature Tv: each reaction's rates are
// evaluated at its controlling temperature T_a (Sec. 3.1.3: sqrt(T Tv) for dissociation,
// ta_mode 1; T otherwise), k_b = k_f / K_c(T_a).  Single temperature: Tv = T.
void species_rates(const OrcMech& m, const double* rho_s, double T, double Tv, double* w) {
  const int ns = m.n_species;
  for (int s = 0; s < ns; ++s) w[s] = 0.0;
  double X[8];
  for (int s = 0; s < ns; ++s) X[s] = rho_s[s] / m.W[s] * 1.0e-6;
  for (int r = 0; r < m.n_reactions; ++r) {
    const double Ta = (m.ta_mode[r] && Tv != T) ? std::sqrt(T * Tv) : T;
    double kf, Kc;
    arrhenius(m, r, Ta, kf, Kc);
    double pf = 1.0, pb = 1.0;
    for (int s = 0; s < ns; ++s) {
      for (int k = 0; k < m.nu_f[r][s]; ++k) pf *= X[s];
      for (int k = 0; k < m.nu_b[r][s]; ++k) pb *= X[s];
    }
    const double Rr = kf * pf - kf / Kc * pb;
    for (int s = 0; s < ns; ++s) w[s] += m.W[s] * 1.0e6 * (m.nu_b[r][s] - m.nu_f[r][s]) * Rr;
  }
}

// Vibrational relaxation time tau_s (s) of molecular species s (Sec. 3.1.3, below Eq.
// src_landau_teller: the Millikan-White correlation with Park's high-temperature
// correction), at translational temperature T and pressure p (Pa) for mole fractions X.
// Millikan and White (J. Chem. Phys. 39, 1963): p tau_sr = exp(A_sr (T^-1/3 - B_sr) - 18.42)
// atm s with A_sr = 1.16e-3 mu_sr^1/2 theta_s^4/3, B_sr = 0.015 mu_sr^1/4, mu_sr the reduced
// molar mass in g/mol, and the mixture rule tau_MW = sum_r X_r / sum_r (X_r / tau_sr).
// Park (J. Thermophys. Heat Transfer 7, 1993): tau_P = 1 / (n sigma_v c_s), n = p / (k_B T)
// the number density, c_s = sqrt(8 R_s T / pi) the mean molecular speed,
// sigma_v = 1e-21 (50000 / T)^2 m^2.  READING: tau_s = tau_MW + tau_P, n the mixture's.
double relaxation_time(const OrcMech& m, int s, const double* X, double T, double p) {
  const double katm = 101325.0, kB = 1.380649e-23;
  double num = 0.0, den = 0.0;
  for (int r = 0; r < m.n_species; ++r) {
    const double Ws = m.W[s] * 1.0e3, Wr = m.W[r] * 1.0e3;  // g/mol
    const double mu = Ws * Wr / (Ws + Wr);
    const double A = 1.16e-3 * std::sqrt(mu) * std::pow(m.theta_v[s], 4.0 / 3.0);
    const double B = 0.015 * std::pow(mu, 0.25);
    const double tau_sr = std::exp(A * (std::pow(T, -1.0 / 3.0) - B) - 18.42) * katm / p;
    num += X[r];
    den += X[r] / tau_sr;
  }
  const double tau_mw = num / den;
  const double n = p / (kB * T);
  const double sigma = 1.0e-21 * (50000.0 / T) * (50000.0 / T);
  const double c = std::sqrt(8.0 * m.R[s] * T / M_PI);
  return tau_mw + 1.0 / (n * sigma * c);
}

// Landau-Teller exchange (Sec. 3.1.3 Eq. src_landau_teller):
// Q_T-v = sum over molecules rho_s (e_v,s(T) - e_v,s(Tv)) / tau_s(T, p).
double landau_teller(const OrcMech& m, const double* rho_s, const Mix& q) {
  double X[8], sum = 0.0;
  for (int s = 0; s < m.n_species; ++s) sum += (X[s] = rho_s[s] / m.W[s]);
  for (int s = 0; s < m.n_species; ++s) X[s] /= sum;
  double Q = 0.0;
  for (int s = 0; s < m.n_species; ++s) {
    if (m.theta_v[s] <= 0.0) continue;
    const double tau = relaxation_time(m, s, X, q.T, q.p);
    Q += rho_s[s] * (vib_energy(m.R[s], m.theta_v[s], q.T) - vib_energy(m.R[s], m.theta_v[s], q.Tv)) / tau;
  }
  return Q;
}

// Source vector (Sec. 3.1.3 Eq. src_vector): omega_s, no momentum or total-energy source;
// two-temperature: the E_v row Q_T-v + sum_s omega_s e_v,s(Tv).
void chem_source(const OrcProblem& P, const double* u, double* S) {
  const int nv = n_vars(P);
  for (int v = 0; v < nv; ++v) S[v] = 0.0;
  Mix q = mixture(P, u);
  species_rates(*P.mech, u, q.T, q.Tv, S);
  if (P.two_temperature) {
    const OrcMech& m = *P.mech;
    double Sv = landau_teller(m, u, q);
    for (int s = 0; s < m.n_species; ++s) Sv += S[s] * vib_energy(m.R[s], m.theta_v[s], q.Tv);
    S[nv - 1] = Sv;
  }
}

// ---------------------------------------------------------------------------------------
// Boundary conditions of the reacting Navier-Stokes system (Sec. 3.1.1 boundary functors for
// the inviscid flux; Sec. 3.1.2 "BR1 Gradient" boundary kernels for the viscous part; the
// set-up of Sec. 4's wing case: a wall is a slip wall for the inviscid flux and a no-slip
// wall for the viscous terms; every condition acts weakly, through the numerical fluxes).
// ---------------------------------------------------------------------------------------
int check_reacting_bc(const OrcProblem& P) {
  const int nv = n_vars(P);
  for (int f = 0; f < 2 * P.dim; ++f) {
    if (P.bc[f] < ORC_BC_PERIODIC || P.bc[f] > ORC_BC_NOSLIP_ISOTHERMAL) return -1;
    if ((P.bc[f] == ORC_BC_PERIODIC) != (P.bc[f ^ 1] == ORC_BC_PERIODIC)) return -1;  // pairs
    if (P.bc[f] == ORC_BC_INFLOW || P.bc[f] == ORC_BC_DIRICHLET) {
      for (int v = 0; v < nv; ++v)
        if (!std::isfinite(P.bc_state[f][v])) return -1;
      Mix q = mixture(P, P.bc_state[f]);
      if (!(q.rho > 0.0) || !(q.T > 0.0) || !(q.Tv > 0.0)) return -1;
    }
    if (P.bc[f] == ORC_BC_NOSLIP_ISOTHERMAL &&
        !(P.bc_state[f][0] > 0.0 && std::isfinite(P.bc_state[f][0])))
      return -1;
  }
  return 0;
}

// Inviscid flux F* in direction l at domain face f of the reacting system; own_left: the
// element's trace is the left state (upper face).  Every wall (slip or no-slip) is the slip
// wall here: the Rusanov flux against the mirror state (normal momentum reversed, species
// densities and energy kept); supersonic inflow: F^l(U_b); supersonic outflow: F^l(U-);
// Dirichlet: the Rusanov flux against U_b.
void mix_boundary_flux(const OrcProblem& P, int f, int l, const double* uown, bool own_left,
                       double* F) {
  const int ns = P.mech->n_species, nv = n_vars(P);
  double ub[16];
  switch (P.bc[f]) {
    case ORC_BC_INFLOW:
      mix_flux(P, l, P.bc_state[f], F);
      return;
    case ORC_BC_OUTFLOW:
      mix_flux(P, l, uown, F);
      return;
    case ORC_BC_DIRICHLET:
      for (int v = 0; v < nv; ++v) ub[v] = P.bc_state[f][v];
      break;
    default:  // slip and no-slip walls
      for (int v = 0; v < nv; ++v) ub[v] = uown[v];
      ub[ns + l] = -uown[ns + l];
      break;
  }
  if (own_left) mix_rusanov(P, l, uown, ub, F);
  else mix_rusanov(P, l, ub, uown, F);
}

// BR1 trace W^ of W = (u, v, w, T, T_v) at domain face f with normal axis l, from the
// element's own trace Wo (Sec. 3.1.2: at a no-slip adiabatic wall the velocity is zero and
// (rho, T) come from the interior; an isothermal wall also fixes T; a slip wall mirrors the
// velocity across the wall).  READINGS: the trace is the boundary's value of W itself; at a
// slip wall, the BR1 average of the interior trace and its mirror image (normal velocity 0,
// tangential velocity, T and T_v kept); an isothermal wall holds both modes at T_wall
// (T_v = T_wall), an adiabatic one keeps the interior T_v; inflow and Dirichlet: W of the
// prescribed state (the far-field Dirichlet condition); outflow: the interior trace (no
// gradient lift).  Single temperature: T_v = T throughout.
void wall_trace(const OrcProblem& P, int f, int l, const double* Wo, double* Wh) {
  switch (P.bc[f]) {
    case ORC_BC_SLIP_WALL: {
      double Wm[5] = {Wo[0], Wo[1], Wo[2], Wo[3], Wo[4]};
      Wm[l] = -Wo[l];
      for (int q = 0; q < 5; ++q) Wh[q] = 0.5 * (Wo[q] + Wm[q]);
      return;
    }
    case ORC_BC_NOSLIP_ADIABATIC:
      Wh[0] = Wh[1] = Wh[2] = 0.0;
      Wh[3] = Wo[3];
      Wh[4] = Wo[4];
      return;
    case ORC_BC_NOSLIP_ISOTHERMAL:
      Wh[0] = Wh[1] = Wh[2] = 0.0;
      Wh[3] = Wh[4] = P.bc_state[f][0];
      return;
    case ORC_BC_OUTFLOW:
      for (int q = 0; q < 5; ++q) Wh[q] = Wo[q];
      return;
    default: {  // inflow, Dirichlet
      Mix b = mixture(P, P.bc_state[f]);
      Wh[0] = b.v[0];
      Wh[1] = b.v[1];
      Wh[2] = b.v[2];
      Wh[3] = b.T;
      Wh[4] = b.Tv;
    }
  }
}

void viscous_flux(const OrcProblem& P, int l, const double* u, const double* g, double* F);

// Viscous numerical flux (F_v^l)* at domain face f with normal axis l, from the element's own
// node u and its gradient g (Sec. 3.1.2 boundary kernels: the viscous operator of a wall
// enforces no slip and, adiabatic, no heat flux).  READINGS: slip wall: the BR1 average of
// the interior flux and its mirror image -- the normal-momentum row (tau_ll) kept, the
// tangential rows and the energy (and E_v) rows 0; no-slip adiabatic wall: the interior
// stress rows, energy and E_v rows 0 (a wall at rest does no work and passes no heat);
// no-slip isothermal wall: the interior stress rows, energy k dT/dx_l + k_v dT_v/dx_l and
// E_v row k_v dT_v/dx_l (heat of both modes conducted through the wall, no work); inflow,
// outflow, Dirichlet: the interior flux (no viscous lift).
void viscous_boundary_flux(const OrcProblem& P, int f, int l, const double* u, const double* g,
                           double* F) {
  const int ns = P.mech->n_species, dim = P.dim, nv = n_vars(P);
  double Fo[16];
  viscous_flux(P, l, u, g, Fo);
  for (int v = 0; v < nv; ++v) F[v] = Fo[v];
  switch (P.bc[f]) {
    case ORC_BC_SLIP_WALL: {
      double Fm[16];
      for (int v = 0; v < nv; ++v) Fm[v] = -Fo[v];
      Fm[ns + l] = Fo[ns + l];
      for (int v = 0; v < nv; ++v) F[v] = 0.5 * (Fo[v] + Fm[v]);
      return;
    }
    case ORC_BC_NOSLIP_ADIABATIC:
      for (int v = ns + dim; v < nv; ++v) F[v] = 0.0;
      return;
    case ORC_BC_NOSLIP_ISOTHERMAL: {
      Mix q = mixture(P, u);
      F[ns + dim] = P.mu * q.cp / P.prandtl * g[3 * 3 + l];
      if (P.two_temperature) {
        const double qv = P.mu * q.cvv / P.prandtl * g[4 * 3 + l];
        F[ns + dim] += qv;
        F[ns + dim + 1] = qv;
      }
      return;
    }
    default:
      return;
  }
}

// BR1 gradient (Sec. 3.1.2 Eq. br1_avg; App. A "Viscous Volume and Interface Fluxes") of
// W = (u, v, w, T, T_v) on element e: S_l = (2/dx_l) [D W + (upper face) (W^ - W_N)/w_N
// - (lower face) (W^ - W_0)/w_0], W^ = (W_L + W_R)/2 (at a domain face: wall_trace).
// Layout G[(node * 5 + q) * 3 + l]; T_v = T in the single-temperature model.
void br1_gradient(const OrcProblem& P, const Mesh& M, const Ops& ops, const double* U, int e,
                  double* G) {
  const int dim = M.dim, n1 = M.n1, N = M.N, nv = n_vars(P);
  auto prim = [&](int el, int nd, double* W) {
    double u[16];
    load_node(M, nv, U, el, nd, u);
    Mix q = mixture(P, u);
    W[0] = q.v[0]; W[1] = q.v[1]; W[2] = q.v[2]; W[3] = q.T; W[4] = q.Tv;
  };
  for (int nd = 0; nd < M.n_nodes; ++nd) {
    int ijk[3];
    M.node_coords(nd, ijk);
    for (int q = 0; q < 5; ++q)
      for (int l = 0; l < 3; ++l) G[((size_t)(e * M.n_nodes + nd) * 5 + q) * 3 + l] = 0.0;
    for (int l = 0; l < dim; ++l) {
      const double s = 2.0 / M.dx[l];
      double acc[5] = {0, 0, 0, 0, 0}, Wm[5];
      for (int m = 0; m < n1; ++m) {
        int mk[3] = {ijk[0], ijk[1], ijk[2]};
        mk[l] = m;
        prim(e, M.node(mk), Wm);
        for (int q = 0; q < 5; ++q) acc[q] += ops.D[ijk[l] * n1 + m] * Wm[q];
      }
      double Wo[5], Wn[5], Wh[5];
      prim(e, nd, Wo);
      if (ijk[l] == N) {
        const int fb = boundary_face(P, M, e, l, 1);
        if (fb >= 0) {
          wall_trace(P, fb, l, Wo, Wh);
        } else {
          int nk[3] = {ijk[0], ijk[1], ijk[2]};
          nk[l] = 0;
          prim(M.neighbour(e, l, +1), M.node(nk), Wn);
          for (int q = 0; q < 5; ++q) Wh[q] = 0.5 * (Wo[q] + Wn[q]);
        }
        for (int q = 0; q < 5; ++q) acc[q] += (Wh[q] - Wo[q]) / ops.w[N];
      }
      if (ijk[l] == 0) {
        const int fb = boundary_face(P, M, e, l, 0);
        if (fb >= 0) {
          wall_trace(P, fb, l, Wo, Wh);
        } else {
          int nk[3] = {ijk[0], ijk[1], ijk[2]};
          nk[l] = N;
          prim(M.neighbour(e, l, -1), M.node(nk), Wn);
          for (int q = 0; q < 5; ++q) Wh[q] = 0.5 * (Wn[q] + Wo[q]);
        }
        for (int q = 0; q < 5; ++q) acc[q] -= (Wh[q] - Wo[q]) / ops.w[0];
      }
      for (int q = 0; q < 5; ++q) G[((size_t)(e * M.n_nodes + nd) * 5 + q) * 3 + l] = s * acc[q];
    }
  }
}

// viscous flux in direction l (Sec. 2 F_v; Sec. 3.1.2 Eq. tau; q = -k grad T):
// (0 for species, tau_{.l}, u . tau_{.l} + k dT/dx_l); two-temperature: the energy row adds
// k_v dT_v/dx_l and the E_v row is k_v dT_v/dx_l (q_v = -k_v grad T_v).
void viscous_flux(const OrcProblem& P, int l, const double* u, const double* g, double* F) {
  const int ns = P.mech->n_species, dim = P.dim, nv = n_vars(P);
  Mix q = mixture(P, u);
  const double mu = P.mu, k = mu * q.cp / P.prandtl;
  double div = 0.0;
  for (int d = 0; d < dim; ++d) div += g[d * 3 + d];  // du_d/dx_d
  for (int v = 0; v < nv; ++v) F[v] = 0.0;
  double work = 0.0;
  for (int j = 0; j < dim; ++j) {
    double tau = mu * (g[j * 3 + l] + g[l * 3 + j]) - (j == l ? 2.0 / 3.0 * mu * div : 0.0);
    F[ns + j] = tau;
    work += q.v[j] * tau;
  }
  F[ns + dim] = work + k * g[3 * 3 + l];
  if (P.two_temperature) {
    const double kv = mu * q.cvv / P.prandtl;
    F[ns + dim] += kv * g[4 * 3 + l];
    F[ns + dim + 1] = kv * g[4 * 3 + l];
  }
}

void reacting_element_residual(const OrcProblem& P, const Mesh& M, const Ops& ops, const double* U,
                               const double* G, int e, double* dU) {
  const int dim = M.dim, n1 = M.n1, N = M.N, nv = n_vars(P);
  const int parts = P.parts ? P.parts : 7;
  std::vector<double> R((size_t)M.n_nodes * nv, 0.0);
  auto grad = [&](int el, int nd) { return G + (size_t)(el * M.n_nodes + nd) * 15; };
  double um[16], F[16];
  for (int nd = 0; nd < M.n_nodes; ++nd) {
    int ijk[3];
    M.node_coords(nd, ijk);
    for (int l = 0; l < dim; ++l) {
      const double s = 2.0 / M.dx[l];
      for (int m = 0; m < n1; ++m) {
        int mk[3] = {ijk[0], ijk[1], ijk[2]};
        mk[l] = m;
        const int nm = M.node(mk);
        load_node(M, nv, U, e, nm, um);
        const double c = s * ops.D[ijk[l] * n1 + m];
        if (parts & 1) {
          mix_flux(P, l, um, F);
          for (int v = 0; v < nv; ++v) R[nd * nv + v] -= c * F[v];
        }
        if (parts & 2) {
          viscous_flux(P, l, um, grad(e, nm), F);
          for (int v = 0; v < nv; ++v) R[nd * nv + v] += c * F[v];
        }
      }
    }
  }
  for (int l = 0; l < dim; ++l) {
    const double s = 2.0 / M.dx[l];
    for (int nd = 0; nd < M.n_nodes; ++nd) {
      int ijk[3];
      M.node_coords(nd, ijk);
      if (ijk[l] != N && ijk[l] != 0) continue;
      double uown[16], unbr[16], Fs[16], Fo[16], Fvo[16], Fvn[16];
      load_node(M, nv, U, e, nd, uown);
      for (int side = 0; side < 2; ++side) {
        if ((side == 1 && ijk[l] != N) || (side == 0 && ijk[l] != 0)) continue;
        int nk[3] = {ijk[0], ijk[1], ijk[2]};
        nk[l] = side ? 0 : N;
        const int fb = boundary_face(P, M, e, l, side);
        const int en = M.neighbour(e, l, side ? +1 : -1), nn = M.node(nk);
        load_node(M, nv, U, en, nn, unbr);
        const double lift = s / ops.w[side ? N : 0];
        if (parts & 1) {
          if (fb >= 0) mix_boundary_flux(P, fb, l, uown, side == 1, Fs);
          else if (side) mix_rusanov(P, l, uown, unbr, Fs);
          else mix_rusanov(P, l, unbr, uown, Fs);
          mix_flux(P, l, uown, Fo);
          for (int v = 0; v < nv; ++v) R[nd * nv + v] += (side ? -lift : lift) * (Fs[v] - Fo[v]);
        }
        if (parts & 2) {  // BR1 central viscous flux (Eq. br1_flux)
          viscous_flux(P, l, uown, grad(e, nd), Fvo);
          if (fb >= 0) {
            viscous_boundary_flux(P, fb, l, uown, grad(e, nd), Fs);
          } else {
            viscous_flux(P, l, unbr, grad(en, nn), Fvn);
            for (int v = 0; v < nv; ++v) Fs[v] = 0.5 * (Fvo[v] + Fvn[v]);
          }
          for (int v = 0; v < nv; ++v) R[nd * nv + v] += (side ? lift : -lift) * (Fs[v] - Fvo[v]);
        }
      }
    }
  }
  if (parts & 4) {
    for (int nd = 0; nd < M.n_nodes; ++nd) {
      load_node(M, nv, U, e, nd, um);
      chem_source(P, um, F);
      for (int v = 0; v < nv; ++v) R[nd * nv + v] += F[v];
    }
  }
  for (int nd = 0; nd < M.n_nodes; ++nd)
    for (int v = 0; v < nv; ++v) dU[((size_t)v * M.n_elem + e) * M.n_nodes + nd] = R[nd * nv + v];
}

// ---------------------------------------------------------------------------------------
// Reacting Navier-Stokes on a curved mesh (Sec. 3.1.1 metric terms with the discrete GCL;
// Sec. 3.1.2 BR1 on the mapped element; periodic meshes).
// BR1 gradient (Step 1): the strong-form DG derivative in reference space -- along each
// reference direction l, D W plus the lifted jump (W^ - W)/w at the element's faces, W^ the
// BR1 average of Eq. br1_avg -- then mapped to physical space with the contravariant vectors
// at the node and rescaled by the inverse Jacobian:
//   S_d(i) = (1/J_i) sum_l Ja^l_d(i) [ (D_l W)_i + (face terms)_l ].
// READING: the paper says the gradient is formed by a strong-form operator and rescaled by
// 1/J after the surface contributions; the reference-space derivative mapped by Ja^l at the
// node (chain rule) is the form taken here (it equals the Cartesian operator on affine
// elements and gives a zero gradient of a constant).
// ---------------------------------------------------------------------------------------
void curved_br1_gradient(const OrcProblem& P, const Mesh& M, const Ops& ops, const Metrics& Gm,
                         const double* U, int e, double* G) {
  const int dim = M.dim, n1 = M.n1, N = M.N, nv = n_vars(P), np = M.n_nodes;
  auto prim = [&](int el, int nd, double* W) {
    double u[16];
    load_node(M, nv, U, el, nd, u);
    Mix q = mixture(P, u);
    W[0] = q.v[0]; W[1] = q.v[1]; W[2] = q.v[2]; W[3] = q.T; W[4] = q.Tv;
  };
  auto Ja = [&](int nd, int l, int d) { return Gm.Ja[(((size_t)e * np + nd) * 3 + l) * 3 + d]; };
  for (int nd = 0; nd < np; ++nd) {
    int ijk[3];
    M.node_coords(nd, ijk);
    double ref[5][3] = {};
    double Wo[5], Wn[5], Wm[5];
    prim(e, nd, Wo);
    for (int l = 0; l < dim; ++l) {
      for (int m = 0; m < n1; ++m) {
        int mk[3] = {ijk[0], ijk[1], ijk[2]};
        mk[l] = m;
        prim(e, M.node(mk), Wm);
        for (int q = 0; q < 5; ++q) ref[q][l] += ops.D[ijk[l] * n1 + m] * Wm[q];
      }
      for (int side = 0; side < 2; ++side) {
        if (ijk[l] != (side ? N : 0)) continue;
        int nk[3] = {ijk[0], ijk[1], ijk[2]};
        nk[l] = side ? 0 : N;
        prim(M.neighbour(e, l, side ? +1 : -1), M.node(nk), Wn);
        for (int q = 0; q < 5; ++q) {
          const double jump = 0.5 * (Wo[q] + Wn[q]) - Wo[q];
          ref[q][l] += (side ? 1.0 : -1.0) * jump / ops.w[side ? N : 0];
        }
      }
    }
    const double iJ = 1.0 / Gm.J[(size_t)e * np + nd];
    for (int q = 0; q < 5; ++q)
      for (int d = 0; d < 3; ++d) {
        double g = 0.0;
        if (d < dim)
          for (int l = 0; l < dim; ++l) g += Ja(nd, l, d) * ref[q][l];
        G[((size_t)(e * np + nd) * 5 + q) * 3 + d] = iJ * g;
      }
  }
}

// Rusanov flux of the mixture along the unit direction n: (F_n(U_L) + F_n(U_R))/2 -
// lambda (U_R - U_L)/2, F_n = sum_d n_d F^d, lambda = max(|u_L . n| + a_L, |u_R . n| + a_R).
void mix_rusanov_n(const OrcProblem& P, const double* n, const double* uL, const double* uR, double* F) {
  const int nv = n_vars(P), dim = P.dim;
  Mix a = mixture(P, uL), b = mixture(P, uR);
  double unL = 0.0, unR = 0.0;
  for (int d = 0; d < dim; ++d) {
    unL += a.v[d] * n[d];
    unR += b.v[d] * n[d];
  }
  const double lam = std::fmax(std::fabs(unL) + a.a, std::fabs(unR) + b.a);
  double FL[16], FR[16], Fd[16];
  for (int v = 0; v < nv; ++v) FL[v] = FR[v] = 0.0;
  for (int d = 0; d < dim; ++d) {
    mix_flux(P, d, uL, Fd);
    for (int v = 0; v < nv; ++v) FL[v] += n[d] * Fd[v];
    mix_flux(P, d, uR, Fd);
    for (int v = 0; v < nv; ++v) FR[v] += n[d] * Fd[v];
  }
  for (int v = 0; v < nv; ++v) F[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * lam * (uR[v] - uL[v]);
}

// Residual of element e on a curved mesh (Step 2 and the hyperbolic pipeline with the
// contravariant fluxes, Eqs. vol_weak, surf_int, br1_flux):
//   R_i = (1/J_i) [ - sum_l sum_m D_{i_l m} (Ftilde^l_inv - Ftilde^l_v)(m)
//                   -/+ (1/w) (|Ja^l| F*_n - Ftilde^l_inv(i))            (upper / lower face)
//                   +/- (1/w) (Ja^l . {{F_v}} - Ftilde^l_v(i)) ]        + S(U_i),
// Ftilde^l = sum_d Ja^l_d F^d, n = Ja^l / |Ja^l| at the own face node (the neighbour's face
// node has the same Ja^l: it depends on the face's nodes only).
void curved_reacting_element_residual(const OrcProblem& P, const Mesh& M, const Ops& ops, const Metrics& Gm,
                                      const double* U, const double* G, int e, double* dU) {
  const int dim = M.dim, n1 = M.n1, N = M.N, nv = n_vars(P), np = M.n_nodes;
  const int parts = P.parts ? P.parts : 7;
  std::vector<double> R((size_t)np * nv, 0.0);
  auto grad = [&](int el, int nd) { return G + (size_t)(el * np + nd) * 15; };
  auto Ja = [&](int nd, int l, int d) { return Gm.Ja[(((size_t)e * np + nd) * 3 + l) * 3 + d]; };
  // contravariant inviscid and viscous fluxes of direction l at node nd of element el with
  // the metric of own node ndm
  auto contra = [&](int l, int ndm, const double* u, const double* g, double* Fi, double* Fv) {
    double Fd[16];
    for (int v = 0; v < nv; ++v) Fi[v] = Fv[v] = 0.0;
    for (int d = 0; d < dim; ++d) {
      const double a = Ja(ndm, l, d);
      mix_flux(P, d, u, Fd);
      for (int v = 0; v < nv; ++v) Fi[v] += a * Fd[v];
      viscous_flux(P, d, u, g, Fd);
      for (int v = 0; v < nv; ++v) Fv[v] += a * Fd[v];
    }
  };
  double um[16], Fi[16], Fv[16];
  for (int nd = 0; nd < np; ++nd) {
    int ijk[3];
    M.node_coords(nd, ijk);
    for (int l = 0; l < dim; ++l)
      for (int m = 0; m < n1; ++m) {
        int mk[3] = {ijk[0], ijk[1], ijk[2]};
        mk[l] = m;
        const int nm = M.node(mk);
        load_node(M, nv, U, e, nm, um);
        contra(l, nm, um, grad(e, nm), Fi, Fv);
        const double c = ops.D[ijk[l] * n1 + m];
        for (int v = 0; v < nv; ++v) {
          if (parts & 1) R[nd * nv + v] -= c * Fi[v];
          if (parts & 2) R[nd * nv + v] += c * Fv[v];
        }
      }
  }
  for (int l = 0; l < dim; ++l)
    for (int nd = 0; nd < np; ++nd) {
      int ijk[3];
      M.node_coords(nd, ijk);
      for (int side = 0; side < 2; ++side) {
        if (ijk[l] != (side ? N : 0)) continue;
        double uown[16], unbr[16], Fs[16], Fio[16], Fvo[16], Fin[16], Fvn[16], n[3] = {0.0, 0.0, 0.0};
        load_node(M, nv, U, e, nd, uown);
        int nk[3] = {ijk[0], ijk[1], ijk[2]};
        nk[l] = side ? 0 : N;
        const int en = M.neighbour(e, l, side ? +1 : -1), nn = M.node(nk);
        load_node(M, nv, U, en, nn, unbr);
        double s2 = 0.0;
        for (int d = 0; d < dim; ++d) s2 += Ja(nd, l, d) * Ja(nd, l, d);
        const double sj = std::sqrt(s2);
        for (int d = 0; d < dim; ++d) n[d] = Ja(nd, l, d) / sj;
        contra(l, nd, uown, grad(e, nd), Fio, Fvo);
        contra(l, nd, unbr, grad(en, nn), Fin, Fvn);
        const double lift = 1.0 / ops.w[side ? N : 0];
        if (parts & 1) {
          if (side) mix_rusanov_n(P, n, uown, unbr, Fs);
          else mix_rusanov_n(P, n, unbr, uown, Fs);
          for (int v = 0; v < nv; ++v) R[nd * nv + v] += (side ? -lift : lift) * (sj * Fs[v] - Fio[v]);
        }
        if (parts & 2)
          for (int v = 0; v < nv; ++v)
            R[nd * nv + v] += (side ? lift : -lift) * (0.5 * (Fvo[v] + Fvn[v]) - Fvo[v]);
      }
    }
  for (int nd = 0; nd < np; ++nd) {
    const double iJ = 1.0 / Gm.J[(size_t)e * np + nd];
    for (int v = 0; v < nv; ++v) R[nd * nv + v] *= iJ;
  }
  if (parts & 4) {
    for (int nd = 0; nd < np; ++nd) {
      load_node(M, nv, U, e, nd, um);
      chem_source(P, um, Fi);
      for (int v = 0; v < nv; ++v) R[nd * nv + v] += Fi[v];
    }
  }
  for (int nd = 0; nd < np; ++nd)
    for (int v = 0; v < nv; ++v) dU[((size_t)v * M.n_elem + e) * np + nd] = R[nd * nv + v];
}

void residual(const OrcProblem& P, const double* U, double* dU) {
  Mesh M(P);
  Ops ops(P.N);
  if (P.equations == ORC_NS_REACTING && P.coords) {
    const Metrics Gm = curved_metrics(P, M, ops);
    std::vector<double> G((size_t)M.n_elem * M.n_nodes * 15, 0.0);
    const int parts = P.parts ? P.parts : 7;
    if (parts & 2) {
#pragma omp parallel for schedule(static)
      for (int e = 0; e < M.n_elem; ++e) curved_br1_gradient(P, M, ops, Gm, U, e, G.data());
    }
#pragma omp parallel for schedule(static)
    for (int e = 0; e < M.n_elem; ++e) curved_reacting_element_residual(P, M, ops, Gm, U, G.data(), e, dU);
    return;
  }
  if (P.equations == ORC_NS_REACTING) {
    std::vector<double> G((size_t)M.n_elem * M.n_nodes * 15, 0.0);
    const int parts = P.parts ? P.parts : 7;
    if (parts & 2) {
#pragma omp parallel for schedule(static)
      for (int e = 0; e < M.n_elem; ++e) br1_gradient(P, M, ops, U, e, G.data());
    }
#pragma omp parallel for schedule(static)
    for (int e = 0; e < M.n_elem; ++e) reacting_element_residual(P, M, ops, U, G.data(), e, dU);
    return;
  }
  if (P.coords) {  // curved mesh
    const Metrics G = curved_metrics(P, M, ops);
#pragma omp parallel for schedule(static)
    for (int e = 0; e < M.n_elem; ++e) curved_element_residual(P, M, ops, G, U, e, dU);
    return;
  }
#pragma omp parallel for schedule(static)
  for (int e = 0; e < M.n_elem; ++e) euler_element_residual(P, M, ops, U, e, dU);
  if (P.shock) {
    // Eq. vol_blend: R = (1 - alpha_e) R^DG + alpha_e R^FV per element (with the strong-form
    // DG residual this is the paper's (1 - alpha_e) F(U^-) boundary correction of F*)
    std::vector<double> araw(M.n_elem), alpha(M.n_elem);
    shock_alpha(P, U, araw.data(), alpha.data());
    const int nv = n_vars(P);
    std::vector<double> fv((size_t)nv * M.n_elem * M.n_nodes, 0.0);
#pragma omp parallel for schedule(static)
    for (int e = 0; e < M.n_elem; ++e) {
      if (alpha[e] == 0.0) continue;
      fv_element_residual(P, M, ops, U, e, fv.data());
      for (int v = 0; v < nv; ++v)
        for (int nd = 0; nd < M.n_nodes; ++nd) {
          const size_t q = ((size_t)v * M.n_elem + e) * M.n_nodes + nd;
          dU[q] = (1.0 - alpha[e]) * dU[q] + alpha[e] * fv[q];
        }
    }
  }
}

// Positivity floor (Sec. 4.1 and 4.2 set-ups: lower bounds on rho and p are applied after
// every stage).  READING: the paper does not say how; here rho is raised to
// rho_floor (momentum kept), then E is reset so that p = p_floor where p < p_floor.
void after_stage(const OrcProblem& P, double* U);
void species_limiter(const OrcProblem& P, double* U);

void positivity_floor(const OrcProblem& P, double* U) {
  if (!(P.rho_floor > 0.0) && !(P.p_floor > 0.0)) return;
  Mesh M(P);
  const int dim = M.dim, nv = dim + 2;
  const size_t stride = (size_t)M.n_elem * M.n_nodes;
  for (size_t q = 0; q < stride; ++q) {
    double u[8];
    for (int v = 0; v < nv; ++v) u[v] = U[v * stride + q];
    if (P.rho_floor > 0.0 && u[0] < P.rho_floor) u[0] = P.rho_floor;
    Prim pr = primitives(dim, u, P.gamma);
    if (P.p_floor > 0.0 && pr.p < P.p_floor) {
      double kin = 0.0;
      for (int d = 0; d < dim; ++d) kin += u[1 + d] * u[1 + d] / u[0];
      u[dim + 1] = P.p_floor / (P.gamma - 1.0) + 0.5 * kin;
    }
    for (int v = 0; v < nv; ++v) U[v * stride + q] = u[v];
  }
}

// ---------------------------------------------------------------------------------------
// Forward-mode derivatives (for checking the adjoint).  A dual number carries a value and
// one directional derivative; the residual below is the same Euler residual as above
// (strong, weak or two-point volume form; Rusanov, HLLC or EC surface flux; periodic Cartesian
// boxes), written once more over a generic scalar T so that evaluating it on duals gives L(U)
// and the directional derivative dL = (dL/dU) V + (dL/dgamma) gdot exactly (up to rounding).
// Non-smooth points: |x| has derivative sign(x) with sign(0) = 0; max(a, b) and min(a, b)
// follow the selected value, the left argument on a tie; HLLC's branch follows the values.
// ---------------------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual(double a = 0.0, double b = 0.0) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) { return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual dsqrt(Dual a) { double r = std::sqrt(a.v); return Dual(r, a.d / (2.0 * r)); }
inline Dual dabs(Dual a) { return Dual(std::fabs(a.v), (a.v > 0.0) ? a.d : (a.v < 0.0 ? -a.d : 0.0)); }
inline Dual dmax(Dual a, Dual b) { return (a.v >= b.v) ? a : b; }

template <class T>
void flux_t(int dim, int l, const T* u, T gamma, T* F) {
  T rho = u[0], kin = T(0.0), v[3];
  for (int d = 0; d < dim; ++d) {
    v[d] = u[1 + d] / rho;
    kin += u[1 + d] * v[d];
  }
  T p = (gamma - T(1.0)) * (u[dim + 1] - T(0.5) * kin);
  F[0] = u[1 + l];
  for (int d = 0; d < dim; ++d) F[1 + d] = u[1 + l] * v[d] + (d == l ? p : T(0.0));
  F[dim + 1] = (u[dim + 1] + p) * v[l];
}

template <class T>
T signal_speed_t(int dim, int l, const T* u, T gamma) {  // |u_l| + a
  T rho = u[0], kin = T(0.0);
  for (int d = 0; d < dim; ++d) kin += u[1 + d] * u[1 + d] / rho;
  T p = (gamma - T(1.0)) * (u[dim + 1] - T(0.5) * kin);
  return dabs(u[1 + l] / rho) + dsqrt(gamma * p / rho);
}

template <class T>
void rusanov_t(int dim, int l, const T* uL, const T* uR, T gamma, T* F) {
  T lam = dmax(signal_speed_t(dim, l, uL, gamma), signal_speed_t(dim, l, uR, gamma));
  T FL[8], FR[8];
  flux_t(dim, l, uL, gamma, FL);
  flux_t(dim, l, uR, gamma, FR);
  for (int v = 0; v < dim + 2; ++v) F[v] = T(0.5) * (FL[v] + FR[v]) - T(0.5) * lam * (uR[v] - uL[v]);
}

inline double val(double a) { return a; }
inline double val(const Dual& a) { return a.v; }
inline Dual dlog(Dual a) { return Dual(std::log(a.v), a.d / a.v); }
inline Dual dmin(Dual a, Dual b) { return (a.v <= b.v) ? a : b; }

// Logarithmic mean (a - b)/(ln a - ln b) (App. A) over T.  With f = (a - b)/(a + b) and
// u = f^2, ln a - ln b = 2 atanh(f), so the mean equals ((a + b)/2) / (atanh(f)/f), and
// atanh(f)/f = sum_k u^k / (2k + 1).  Near a = b (u < 1e-4) that series (eleven terms, far
// below rounding) is used: its derivative stays accurate as a -> b, where the quotient's
// derivative is a difference of two large terms; at a = b it gives the mean a and the
// derivative (da + db)/2.  Otherwise the quotient with the logarithm.
template <class T>
T log_mean_t(T a, T b) {
  const T s = a + b, f = (a - b) / s, u = f * f;
  if (val(u) < 1e-4) {
    T F = T(1.0 / 21.0);
    for (int k = 9; k >= 0; --k) F = T(1.0 / (2 * k + 1)) + u * F;
    return T(0.5) * s / F;
  }
  return (a - b) / dlog(a / b);
}

template <class T>
void prims_t(int dim, const T* u, T gamma, T* v, T& p) {
  T kin = T(0.0);
  for (int d = 0; d < dim; ++d) {
    v[d] = u[1 + d] / u[0];
    kin += u[1 + d] * v[d];
  }
  p = (gamma - T(1.0)) * (u[dim + 1] - T(0.5) * kin);
}

// Ranocha's two-point flux in direction e_l over T -- the same formula as ec_flux.
template <class T>
void ec_flux_t(int dim, int l, const T* uL, const T* uR, T gamma, T* F) {
  T vL[3], vR[3], pL, pR;
  prims_t(dim, uL, gamma, vL, pL);
  prims_t(dim, uR, gamma, vR, pR);
  const T rho_ln = log_mean_t(uL[0], uR[0]);
  const T beta_ln = log_mean_t(uL[0] / pL, uR[0] / pR);
  T vLvR = T(0.0);
  for (int d = 0; d < dim; ++d) vLvR += vL[d] * vR[d];
  const T pavg = T(0.5) * (pL + pR);
  const T frho = rho_ln * (T(0.5) * (vL[l] + vR[l]));
  F[0] = frho;
  for (int d = 0; d < dim; ++d) F[1 + d] = frho * (T(0.5) * (vL[d] + vR[d])) + (d == l ? pavg : T(0.0));
  F[dim + 1] = frho * (T(1.0) / ((gamma - T(1.0)) * beta_ln) + T(0.5) * vLvR) + T(0.5) * (pL * vR[l] + pR * vL[l]);
}

// HLLC flux over T -- the same speeds, star states and branches as hllc_flux; the branch is
// chosen on the values (min/max follow the selected argument, the left one on a tie).
template <class T>
void hllc_flux_t(int dim, int l, const T* uL, const T* uR, T gamma, T* F) {
  const int nv = dim + 2;
  T vL[3], vR[3], pL, pR;
  prims_t(dim, uL, gamma, vL, pL);
  prims_t(dim, uR, gamma, vR, pR);
  const T sL = dsqrt(uL[0]), sR = dsqrt(uR[0]);
  const T HL = (uL[dim + 1] + pL) / uL[0], HR = (uR[dim + 1] + pR) / uR[0];
  T vt[3], v2 = T(0.0);
  for (int d = 0; d < dim; ++d) {
    vt[d] = (sL * vL[d] + sR * vR[d]) / (sL + sR);
    v2 += vt[d] * vt[d];
  }
  const T Ht = (sL * HL + sR * HR) / (sL + sR);
  const T at = dsqrt((gamma - T(1.0)) * (Ht - T(0.5) * v2));
  const T aL = dsqrt(gamma * pL / uL[0]), aR = dsqrt(gamma * pR / uR[0]);
  const T SL = dmin(vL[l] - aL, vt[l] - at), SR = dmax(vR[l] + aR, vt[l] + at);
  T FL[8], FR[8];
  flux_t(dim, l, uL, gamma, FL);
  flux_t(dim, l, uR, gamma, FR);
  const T Ss = (pR - pL + uL[0] * vL[l] * (SL - vL[l]) - uR[0] * vR[l] * (SR - vR[l])) /
               (uL[0] * (SL - vL[l]) - uR[0] * (SR - vR[l]));
  auto star = [&](const T* uK, const T* vK, T pK, T SK, T* Us) {
    const T fac = uK[0] * (SK - vK[l]) / (SK - Ss);
    Us[0] = fac;
    for (int d = 0; d < dim; ++d) Us[1 + d] = fac * (d == l ? Ss : vK[d]);
    Us[dim + 1] = fac * (uK[dim + 1] / uK[0] + (Ss - vK[l]) * (Ss + pK / (uK[0] * (SK - vK[l]))));
  };
  T Us[8];
  if (val(SL) >= 0.0) {
    for (int v = 0; v < nv; ++v) F[v] = FL[v];
  } else if (val(Ss) >= 0.0) {
    star(uL, vL, pL, SL, Us);
    for (int v = 0; v < nv; ++v) F[v] = FL[v] + SL * (Us[v] - uL[v]);
  } else if (val(SR) > 0.0) {
    star(uR, vR, pR, SR, Us);
    for (int v = 0; v < nv; ++v) F[v] = FR[v] + SR * (Us[v] - uR[v]);
  } else {
    for (int v = 0; v < nv; ++v) F[v] = FR[v];
  }
}

template <class T>
void surface_flux_t(int kind, int dim, int l, const T* uL, const T* uR, T gamma, T* F) {
  if (kind == ORC_SURF_HLLC) hllc_flux_t(dim, l, uL, uR, gamma, F);
  else if (kind == ORC_SURF_EC) ec_flux_t(dim, l, uL, uR, gamma, F);
  else rusanov_t(dim, l, uL, uR, gamma, F);
}

// Eq. vol_weak (strong) or its weak form, or Eq. vol_split with Ranocha's flux, plus
// Eq. surf_int with the Rusanov, HLLC or EC flux, on element e -- the same loops as
// euler_element_residual.
template <class T>
void element_residual_t(const OrcProblem& P, const Mesh& M, const Ops& ops, const T* U, T gamma,
                        int e, T* dU) {
  const int dim = M.dim, n1 = M.n1, N = M.N, nv = dim + 2;
  std::vector<T> R((size_t)M.n_nodes * nv, T(0.0));
  auto load = [&](int el, int nd, T* u) {
    for (int v = 0; v < nv; ++v) u[v] = U[((size_t)v * M.n_elem + el) * M.n_nodes + nd];
  };
  const bool weak = (P.volume == ORC_VOL_WEAK);
  const bool ec = (P.volume == ORC_VOL_EC);
  T ui[8], um[8], F[8];
  for (int nd = 0; nd < M.n_nodes; ++nd) {
    int ijk[3];
    M.node_coords(nd, ijk);
    load(e, nd, ui);
    for (int l = 0; l < dim; ++l) {
      const double s = 2.0 / M.dx[l];
      const int il = ijk[l];
      for (int m = 0; m < n1; ++m) {
        int mk[3] = {ijk[0], ijk[1], ijk[2]};
        mk[l] = m;
        load(e, M.node(mk), um);
        if (ec) ec_flux_t(dim, l, ui, um, gamma, F);
        else flux_t(dim, l, um, gamma, F);
        const double c = ec ? 2.0 * s * ops.D[il * n1 + m]
                            : (weak ? -s * (ops.w[m] / ops.w[il]) * ops.D[m * n1 + il] : s * ops.D[il * n1 + m]);
        for (int v = 0; v < nv; ++v) R[nd * nv + v] -= T(c) * F[v];
      }
    }
  }
  for (int l = 0; l < dim; ++l) {
    const double s = 2.0 / M.dx[l];
    for (int nd = 0; nd < M.n_nodes; ++nd) {
      int ijk[3];
      M.node_coords(nd, ijk);
      if (ijk[l] != N && ijk[l] != 0) continue;
      T uown[8], unbr[8], Fs[8], Fown[8];
      load(e, nd, uown);
      flux_t(dim, l, uown, gamma, Fown);
      if (ijk[l] == N) {
        int nk[3] = {ijk[0], ijk[1], ijk[2]};
        nk[l] = 0;
        load(M.neighbour(e, l, +1), M.node(nk), unbr);
        surface_flux_t(P.surface, dim, l, uown, unbr, gamma, Fs);
        for (int v = 0; v < nv; ++v)
          R[nd * nv + v] -= T(s / ops.w[N]) * (Fs[v] - (weak ? T(0.0) : Fown[v]));
      }
      if (ijk[l] == 0) {
        int nk[3] = {ijk[0], ijk[1], ijk[2]};
        nk[l] = N;
        load(M.neighbour(e, l, -1), M.node(nk), unbr);
        surface_flux_t(P.surface, dim, l, unbr, uown, gamma, Fs);
        for (int v = 0; v < nv; ++v)
          R[nd * nv + v] += T(s / ops.w[0]) * (Fs[v] - (weak ? T(0.0) : Fown[v]));
      }
    }
  }
  for (int nd = 0; nd < M.n_nodes; ++nd)
    for (int v = 0; v < nv; ++v) dU[((size_t)v * M.n_elem + e) * M.n_nodes + nd] = R[nd * nv + v];
}

}  // namespace

// =======================================================================================
// C entry points used by the Python test harness (ctypes).  Return 0 on success and a
// negative code on a bad description; they never abort.
// =======================================================================================
extern "C" {

int orc_gll(int N, double* x, double* w) {
  if (N < 1 || N > 15) return -1;
  std::vector<long double> xl, wl;
  gll_rule(N, xl, wl);
  for (int i = 0; i <= N; ++i) { x[i] = (double)xl[i]; w[i] = (double)wl[i]; }
  return 0;
}

int orc_dmat(int N, double* D) {
  if (N < 1 || N > 15) return -1;
  std::vector<long double> xl, wl, Dl;
  gll_rule(N, xl, wl);
  diff_matrix(N, xl, Dl);
  for (int i = 0; i < (N + 1) * (N + 1); ++i) D[i] = (double)Dl[i];
  return 0;
}

int orc_nvars(const OrcProblem* P) { return n_vars(*P); }

double orc_log_mean(double a, double b) { return log_mean(a, b); }

// Point fluxes in direction l for one (left, right) pair of states, for the tests.
int orc_point_flux(int dim, int l, double gamma, const double* u, double* F) {
  euler_flux(dim, l, u, gamma, F);
  return 0;
}
int orc_two_point_flux(int kind, int dim, int l, double gamma, const double* uL,
                       const double* uR, double* F) {
  if (kind == -1) ec_flux(dim, l, uL, uR, gamma, F);
  else surface_flux(kind, dim, l, uL, uR, gamma, F);
  return 0;
}

// Arrhenius rate and equilibrium constant of reaction r at temperature T.
int orc_arrhenius(const OrcMech* m, int r, double T, double* kf, double* Kc) {
  if (!m || r < 0 || r >= m->n_reactions || !(T > 0.0)) return -1;
  arrhenius(*m, r, T, *kf, *Kc);
  return 0;
}

// Chemical source of one node state (reacting problems).
int orc_chem_source(const OrcProblem* P, const double* u, double* S) {
  if (P->equations != ORC_NS_REACTING || !P->mech) return -1;
  chem_source(*P, u, S);
  return 0;
}

// Temperature, pressure and vibrational temperature (T for the single-temperature model) of
// one node state (reacting problems).
int orc_mixture(const OrcProblem* P, const double* u, double* T, double* p, double* Tv) {
  if (P->equations != ORC_NS_REACTING || !P->mech) return -1;
  Mix q = mixture(*P, u);
  *T = q.T;
  *p = q.p;
  if (Tv) *Tv = q.Tv;
  return 0;
}

// The species limiter alone, in place (test access).
int orc_species_limiter(const OrcProblem* P, double* U) {
  int rc = check_problem(*P);
  if (rc) return rc;
  if (P->equations != ORC_NS_REACTING) return -1;
  OrcProblem Q = *P;
  Q.species_limiter = 1;
  species_limiter(Q, U);
  return 0;
}

// The Euler positivity floor alone, in place (test access).
int orc_positivity_floor(const OrcProblem* P, double* U) {
  int rc = check_problem(*P);
  if (rc) return rc;
  if (P->equations != ORC_EULER) return -1;
  positivity_floor(*P, U);
  return 0;
}

// Vibrational relaxation time of species s (two-temperature model) for mole fractions X at
// temperature T (K) and pressure p (Pa).
int orc_relaxation_time(const OrcMech* m, int s, const double* X, double T, double p, double* tau) {
  if (!m || s < 0 || s >= m->n_species || !(m->theta_v[s] > 0.0)) return -1;
  *tau = relaxation_time(*m, s, X, T, p);
  return 0;
}

// The two phases of the Navier-Stokes residual (Sec. 3.1.2), exposed so that a partitioned
// mesh can exchange the BR1 gradients of its partition faces between them (Sec. 5, face-only
// exchange): orc_br1_gradients writes the BR1 gradient of W on the listed elements into G
// (layout G[((e * n_nodes + node) * 5 + q) * 3 + l], n_elem * n_nodes * 15 doubles; rows of
// other elements untouched); orc_rhs_elements_given_gradient evaluates the residual of the
// listed elements from U and a caller-supplied G, in which the face neighbours' gradients
// must be valid at least on the shared faces' nodes.
int orc_br1_gradients(const OrcProblem* P, const double* U, const int* elems, int n, double* G) {
  int rc = check_problem(*P);
  if (rc) return rc;
  if (P->equations != ORC_NS_REACTING) return -1;
  Mesh M(*P);
  Ops ops(P->N);
  for (int k = 0; k < n; ++k)
    if (elems[k] < 0 || elems[k] >= M.n_elem) return -1;
  if (P->coords) {
    const Metrics Gm = curved_metrics(*P, M, ops);
    for (int k = 0; k < n; ++k) curved_br1_gradient(*P, M, ops, Gm, U, elems[k], G);
    return 0;
  }
  for (int k = 0; k < n; ++k) br1_gradient(*P, M, ops, U, elems[k], G);
  return 0;
}

int orc_rhs_elements_given_gradient(const OrcProblem* P, const double* U, const double* G,
                                    const int* elems, int n, double* dU) {
  int rc = check_problem(*P);
  if (rc) return rc;
  if (P->equations != ORC_NS_REACTING) return -1;
  Mesh M(*P);
  Ops ops(P->N);
  for (int k = 0; k < n; ++k)
    if (elems[k] < 0 || elems[k] >= M.n_elem) return -1;
  if (P->coords) {
    const Metrics Gm = curved_metrics(*P, M, ops);
    for (int k = 0; k < n; ++k) curved_reacting_element_residual(*P, M, ops, Gm, U, G, elems[k], dU);
    return 0;
  }
  for (int k = 0; k < n; ++k) reacting_element_residual(*P, M, ops, U, G, elems[k], dU);
  return 0;
}

// dU/dt = L(U) (Appendix B, Eq. for the semi-discrete system).
int orc_rhs(const OrcProblem* P, const double* U, double* dU) {
  int rc = check_problem(*P);
  if (rc) return rc;
  residual(*P, U, dU);
  return 0;
}

// L(U) on a list of elements only (rows of dU for other elements are left untouched);
// lets full-size problems be checked on a sample of elements.
int orc_rhs_elements(const OrcProblem* P, const double* U, const int* elems, int n, double* dU) {
  int rc = check_problem(*P);
  if (rc) return rc;
  Mesh M(*P);
  Ops ops(P->N);
  for (int k = 0; k < n; ++k) {
    if (elems[k] < 0 || elems[k] >= M.n_elem) return -1;
  }
  if (P->equations == ORC_NS_REACTING) {
    // gradients are needed on the listed elements and their face neighbours only
    std::vector<double> G((size_t)M.n_elem * M.n_nodes * 15, 0.0);
    std::vector<int> need;
    std::vector<char> mark(M.n_elem, 0);
    for (int k = 0; k < n; ++k) {
      const int e = elems[k];
      if (!mark[e]) { mark[e] = 1; need.push_back(e); }
      for (int l = 0; l < M.dim; ++l)
        for (int dir = -1; dir <= 1; dir += 2) {
          const int en = M.neighbour(e, l, dir);
          if (!mark[en]) { mark[en] = 1; need.push_back(en); }
        }
    }
    if (P->coords) {
      const Metrics Gm = curved_metrics(*P, M, ops);
#pragma omp parallel for schedule(static)
      for (int k = 0; k < (int)need.size(); ++k) curved_br1_gradient(*P, M, ops, Gm, U, need[k], G.data());
#pragma omp parallel for schedule(static)
      for (int k = 0; k < n; ++k) curved_reacting_element_residual(*P, M, ops, Gm, U, G.data(), elems[k], dU);
      return 0;
    }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < (int)need.size(); ++k) br1_gradient(*P, M, ops, U, need[k], G.data());
#pragma omp parallel for schedule(static)
    for (int k = 0; k < n; ++k) reacting_element_residual(*P, M, ops, U, G.data(), elems[k], dU);
    return 0;
  }
  if (P->coords) {
    const Metrics G = curved_metrics(*P, M, ops);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < n; ++k) curved_element_residual(*P, M, ops, G, U, elems[k], dU);
    return 0;
  }
#pragma omp parallel for schedule(static)
  for (int k = 0; k < n; ++k) euler_element_residual(*P, M, ops, U, elems[k], dU);
  if (P->shock) {  // Eq. vol_blend on the listed elements (the coefficients need the whole mesh)
    std::vector<double> araw(M.n_elem), alpha(M.n_elem);
    shock_alpha(*P, U, araw.data(), alpha.data());
    const int nv = n_vars(*P);
    std::vector<double> fv((size_t)nv * M.n_elem * M.n_nodes, 0.0);
    for (int k = 0; k < n; ++k) {
      const int e = elems[k];
      if (alpha[e] == 0.0) continue;
      fv_element_residual(*P, M, ops, U, e, fv.data());
      for (int v = 0; v < nv; ++v)
        for (int nd = 0; nd < M.n_nodes; ++nd) {
          const size_t q = ((size_t)v * M.n_elem + e) * M.n_nodes + nd;
          dU[q] = (1.0 - alpha[e]) * dU[q] + alpha[e] * fv[q];
        }
    }
  }
  return 0;
}

// Hennemann-Gassner blending coefficients of every element (before and after the
// face-neighbourhood maximum), Euler problems with shock capturing.
int orc_shock_alpha(const OrcProblem* P, const double* U, double* alpha_raw, double* alpha) {
  int rc = check_problem(*P);
  if (rc) return rc;
  if (!P->shock || P->equations != ORC_EULER) return -1;
  shock_alpha(*P, U, alpha_raw, alpha);
  return 0;
}

// The sub-cell finite-volume residual of every element alone (Euler problems).
int orc_fv_residual(const OrcProblem* P, const double* U, double* dU) {
  int rc = check_problem(*P);
  if (rc) return rc;
  if (P->equations != ORC_EULER || P->coords) return -1;
  Mesh M(*P);
  Ops ops(P->N);
  for (int e = 0; e < M.n_elem; ++e) fv_element_residual(*P, M, ops, U, e, dU);
  return 0;
}

// Metric terms of a curved mesh: Ja[elem][node][l][d] (3 x 3 per node) and J[elem][node].
int orc_metrics(const OrcProblem* P, double* Ja, double* J) {
  int rc = check_problem(*P);
  if (rc) return rc;
  if (!P->coords) return -1;
  Mesh M(*P);
  Ops ops(P->N);
  const Metrics G = curved_metrics(*P, M, ops);
  std::memcpy(Ja, G.Ja.data(), G.Ja.size() * sizeof(double));
  std::memcpy(J, G.J.data(), G.J.size() * sizeof(double));
  return 0;
}

// Orthonormal tensor-Legendre modes of one element's nodal field q ((N+1)^dim values).
int orc_modes(const OrcProblem* P, const double* q, double* m) {
  int rc = check_problem(*P);
  if (rc) return rc;
  Mesh M(*P);
  to_modes(M, modal_matrix(M.N), q, m);
  return 0;
}

// One SSP-RK3 stage in Shu-Osher form (App. B: U^(i) = sum_k alpha_ik U^(k) + dt beta_ik
// L(U^(k)); the three-stage third-order scheme of Shu and Osher, whose coefficients the
// paper cites but does not print):
//   stage 1: U1 = Un + dt L(Un)
//   stage 2: U2 = 3/4 Un + 1/4 (U1 + dt L(U1))
//   stage 3: U3 = 1/3 Un + 2/3 (U2 + dt L(U2))
// followed by the positivity floor and the species limiter when they are enabled.
int orc_rk3_stage(const OrcProblem* P, int stage, const double* Un, const double* Uprev,
                  double dt, double* Uout) {
  int rc = check_problem(*P);
  if (rc) return rc;
  if (stage < 1 || stage > 3) return -1;
  Mesh M(*P);
  const size_t n = (size_t)n_vars(*P) * M.n_elem * M.n_nodes;
  std::vector<double> L(n);
  residual(*P, Uprev, L.data());
  for (size_t q = 0; q < n; ++q) {
    if (stage == 1) Uout[q] = Un[q] + dt * L[q];
    else if (stage == 2) Uout[q] = 0.75 * Un[q] + 0.25 * (Uprev[q] + dt * L[q]);
    else Uout[q] = (1.0 / 3.0) * Un[q] + (2.0 / 3.0) * (Uprev[q] + dt * L[q]);
  }
  after_stage(*P, Uout);
  return 0;
}

// n_steps full SSP-RK3 steps, in place.
int orc_rk3(const OrcProblem* P, double* U, double dt, int n_steps) {
  int rc = check_problem(*P);
  if (rc) return rc;
  Mesh M(*P);
  const size_t n = (size_t)n_vars(*P) * M.n_elem * M.n_nodes;
  std::vector<double> U1(n), U2(n);
  for (int s = 0; s < n_steps; ++s) {
    orc_rk3_stage(P, 1, U, U, dt, U1.data());
    orc_rk3_stage(P, 2, U, U1.data(), dt, U2.data());
    orc_rk3_stage(P, 3, U, U2.data(), dt, U);
  }
  return 0;
}

}  // extern "C"

namespace {

// ---------------------------------------------------------------------------------------
// The s-stage SSP-RK scheme in Shu-Osher form (App. B):
//   U^(0) = U^n,  U^(i) = sum_{k<i} [alpha_ik U^(k) + dt beta_ik L(U^(k))],  U^{n+1} = U^(s).
// Two tables: SSP-RK33 of Shu and Osher (J. Comput. Phys. 77, 1988) and SSP-RK54 of
// Spiteri and Ruuth (SIAM J. Numer. Anal. 40(2), 2002), the paper's production integrator
// (SSP coefficient about 1.508).  The paper prints neither table; both are the published
// coefficients (SSP-RK54 to the 15 digits of its publication).  Row i holds stage i+1.
// ---------------------------------------------------------------------------------------
struct SspTable {
  int s;
  double alpha[5][5], beta[5][5];
};

SspTable ssp_table(int scheme) {
  SspTable t;
  std::memset(&t, 0, sizeof(t));
  if (scheme == 3) {
    t.s = 3;
    t.alpha[0][0] = 1.0;                           t.beta[0][0] = 1.0;
    t.alpha[1][0] = 0.75; t.alpha[1][1] = 0.25;    t.beta[1][1] = 0.25;
    t.alpha[2][0] = 1.0 / 3.0; t.alpha[2][2] = 2.0 / 3.0;  t.beta[2][2] = 2.0 / 3.0;
    return t;
  }
  t.s = 5;
  t.alpha[0][0] = 1.0;
  t.beta[0][0] = 0.391752226571890;
  t.alpha[1][0] = 0.444370493651235;
  t.alpha[1][1] = 0.555629506348765;
  t.beta[1][1] = 0.368410593050371;
  t.alpha[2][0] = 0.620101851488403;
  t.alpha[2][2] = 0.379898148511597;
  t.beta[2][2] = 0.251891774271694;
  t.alpha[3][0] = 0.178079954393132;
  t.alpha[3][3] = 0.821920045606868;
  t.beta[3][3] = 0.544974750228521;
  t.alpha[4][2] = 0.517231671970585;
  t.alpha[4][3] = 0.096059710526147;
  t.beta[4][3] = 0.063692468666290;
  t.alpha[4][4] = 0.386708617503269;
  t.beta[4][4] = 0.226007483236906;
  return t;
}

// SSP coefficient min over beta_ik > 0 of alpha_ik / beta_ik (App. B, c~).
double ssp_coefficient(const SspTable& t) {
  double c = 1e300;
  for (int i = 0; i < t.s; ++i)
    for (int k = 0; k <= i; ++k)
      if (t.beta[i][k] > 0.0) c = std::fmin(c, t.alpha[i][k] / t.beta[i][k]);
  return c;
}

// Zhang-Shu positivity limiter of the partial densities (Sec. 4 reacting blast set-up: the
// limiter keeps rho_s >= 0 per species; X. Zhang and C.-W. Shu, J. Comput. Phys. 229, 2010):
// per element and species, with the GLL-weighted element mean m and the nodal minimum
// lo, when lo < 0 every nodal value is contracted toward the mean,
//   rho_s <- m + theta (rho_s - m),  theta = m / (m - lo)  (the new minimum is 0),
// and theta = 0 (the element mean everywhere) when the mean itself is not positive.  The
// element mean of every species is unchanged; momentum and energy are untouched.
// READINGS: bound 0 (the paper states rho_s >= 0), applied after every RK stage.
void species_limiter(const OrcProblem& P, double* U) {
  if (P.equations != ORC_NS_REACTING || !P.species_limiter) return;
  Mesh M(P);
  Ops ops(P.N);
  const int ns = P.mech->n_species;
  std::vector<double> W(M.n_nodes);
  for (int nd = 0; nd < M.n_nodes; ++nd) {
    int ijk[3];
    M.node_coords(nd, ijk);
    W[nd] = 1.0;
    for (int l = 0; l < M.dim; ++l) W[nd] *= ops.w[ijk[l]];
  }
  double wsum = 0.0;
  for (int nd = 0; nd < M.n_nodes; ++nd) wsum += W[nd];
  for (int e = 0; e < M.n_elem; ++e)
    for (int s = 0; s < ns; ++s) {
      double* r = U + ((size_t)s * M.n_elem + e) * M.n_nodes;
      double mean = 0.0, lo = r[0];
      for (int nd = 0; nd < M.n_nodes; ++nd) {
        mean += W[nd] * r[nd];
        lo = std::fmin(lo, r[nd]);
      }
      mean /= wsum;
      if (!(lo < 0.0)) continue;
      const double theta = mean > 0.0 ? mean / (mean - lo) : 0.0;
      for (int nd = 0; nd < M.n_nodes; ++nd) r[nd] = mean + theta * (r[nd] - mean);
    }
}

// What follows every RK stage: the Euler positivity floor and the species limiter (each only
// when enabled).
void after_stage(const OrcProblem& P, double* U) {
  positivity_floor(P, U);
  species_limiter(P, U);
}

// One step of the table's scheme, in place; every stage state keeps its residual.  The
// positivity floor and the species limiter (when enabled) follow each stage.
void ssp_step(const OrcProblem& P, const SspTable& t, double* U, double dt) {
  Mesh M(P);
  const size_t n = (size_t)n_vars(P) * M.n_elem * M.n_nodes;
  std::vector<std::vector<double>> Us(t.s + 1, std::vector<double>(n)), Ls(t.s, std::vector<double>(n));
  std::memcpy(Us[0].data(), U, n * sizeof(double));
  for (int i = 1; i <= t.s; ++i) {
    residual(P, Us[i - 1].data(), Ls[i - 1].data());
    for (size_t q = 0; q < n; ++q) {
      double x = 0.0;
      for (int k = 0; k < i; ++k) x += t.alpha[i - 1][k] * Us[k][q] + dt * t.beta[i - 1][k] * Ls[k][q];
      Us[i][q] = x;
    }
    after_stage(P, Us[i].data());
  }
  std::memcpy(U, Us[t.s].data(), n * sizeof(double));
}

// ---------------------------------------------------------------------------------------
// Implicit source substep S_h of the Strang split (Sec. 3.1.3, Eqs. strang_split and
// source_residual), single temperature.  Per node, the partial densities Y = (rho_1..rho_ns)
// advance by one backward-Euler step of length h of the chemical source,
//   R(Y*) = Y* - Y^n - h omega(Y*) = 0,
// with rho = sum rho_s, the momentum and E held fixed (the source has no momentum or energy
// component and sum_s omega_s = 0).  READINGS: with one temperature there is no E_v row and
// no Landau-Teller term; the temperature of an iterate Y follows in closed form from the
// fixed internal energy e = E - |rho u|^2 / (2 rho^n) of the calorically perfect species,
// T(Y) = (e - sum Y_s h0_s) / sum Y_s cv_s (the paper's inner NASA-9 Newton reduces to this).
// Newton: J = dR/dY by forward differences column by column with
// eps_k = max(1e-7 |Y_k|, 1e-12); the update solves J d = R by Gauss-Jordan elimination
// (partial pivoting) and takes the step Y <- Y - lambda d.  READINGS: the paper names no
// safeguard and no stopping rule.  A full Newton step from the initial composition can
// overshoot far enough that the next iterate's temperature is negative and its rates are
// not finite (on the reacting workload once h exceeds about 2e-5 s); so lambda = 1 is halved
// (at most 30 times) while the temperature of the new iterate lies outside [T/2, 2T].
// Partial densities are not bounded below: the backward-Euler root itself can hold a
// slightly negative trace density (seen at 1e-8 of rho near equilibrium), and a positivity
// limit would stall there.  The iteration stops after the first full step (lambda = 1) with
// max_k |d_k| <= tol * rho, or after max_it updates (then the node counts as not converged).
// ---------------------------------------------------------------------------------------
// Temperature of the partial densities Y at the fixed internal energy e.
double temperature_of(const OrcMech& m, const double* Y, double e) {
  double rcv = 0.0, rh0 = 0.0;
  for (int s = 0; s < m.n_species; ++s) {
    rcv += Y[s] * m.cv[s];
    rh0 += Y[s] * m.h0[s];
  }
  return (e - rh0) / rcv;
}

void source_residual(const OrcMech& m, const double* Y, const double* Yn, double e, double h,
                     double* R) {
  const int ns = m.n_species;
  const double T = temperature_of(m, Y, e);
  double w[8];
  species_rates(m, Y, T, T, w);
  for (int s = 0; s < ns; ++s) R[s] = Y[s] - Yn[s] - h * w[s];
}

// Solve A x = b (n x n, row-major, both overwritten) by Gauss-Jordan elimination with
// partial pivoting; x is returned in b.  Returns false on a zero pivot.
bool gauss_jordan(int n, double* A, double* b) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i * n + k]) > std::fabs(A[piv * n + k])) piv = i;
    if (A[piv * n + k] == 0.0) return false;
    if (piv != k) {
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[piv * n + j]);
      std::swap(b[k], b[piv]);
    }
    const double d = A[k * n + k];
    for (int j = 0; j < n; ++j) A[k * n + j] /= d;
    b[k] /= d;
    for (int i = 0; i < n; ++i) {
      if (i == k) continue;
      const double f = A[i * n + k];
      for (int j = 0; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      b[i] -= f * b[k];
    }
  }
  return true;
}

// Two-temperature backward-Euler residual of the unknowns y = (Y_1..Y_ns, E_v) (Sec. 3.1.3:
// the implicit substep takes the full source vector, Eq. src_vector, whose E_v row is
// Q_T-v + sum omega_s e_v,s(T_v)): T from the fixed internal energy e (E minus the kinetic
// energy) less E_v, T_v from E_v; R = y - y^n - h S(y).  Returns false when T or T_v is not
// positive and finite.
bool source_residual_tt(const OrcProblem& P, const double* y, const double* yn, double e, double h,
                        double* R, double* T_out, double* Tv_out) {
  const OrcMech& m = *P.mech;
  const int ns = m.n_species;
  const double T = temperature_of(m, y, e - y[ns]);
  const double Tv = vib_temperature(m, y, y[ns]);
  if (T_out) *T_out = T;
  if (Tv_out) *Tv_out = Tv;
  if (!(T > 0.0) || !(Tv > 0.0) || !std::isfinite(T) || !std::isfinite(Tv)) return false;
  double w[8];
  species_rates(m, y, T, Tv, w);
  Mix q;
  double rR = 0.0;
  for (int s = 0; s < ns; ++s) rR += y[s] * m.R[s];
  q.T = T;
  q.Tv = Tv;
  q.p = rR * T;
  double Sv = landau_teller(m, y, q);
  for (int s = 0; s < ns; ++s) Sv += w[s] * vib_energy(m.R[s], m.theta_v[s], Tv);
  for (int s = 0; s < ns; ++s) R[s] = y[s] - yn[s] - h * w[s];
  R[ns] = y[ns] - yn[ns] - h * Sv;
  return true;
}

// One node: u (all n_vars components) in, the new partial densities (and, two-temperature,
// E_v) written to u.  Single temperature: Newton on R(Y) = Y - Y^n - h omega(Y) with T from
// the fixed internal energy.  Two-temperature: Newton on the unknowns (Y, E_v) of
// source_residual_tt; the step guard also keeps T_v within [T_v/2, 2 T_v], and convergence
// also asks |dE_v| <= tol e (e the internal energy density).  Returns the number of Newton
// updates taken, or -1 if the iteration did not converge.
int source_implicit_node(const OrcProblem& P, double* u, double h, int max_it, double tol) {
  const OrcMech& m = *P.mech;
  const int ns = m.n_species, dim = P.dim;
  double Yn[9], Y[9], rho = 0.0, kin = 0.0;
  for (int s = 0; s < ns; ++s) {
    Yn[s] = Y[s] = u[s];
    rho += u[s];
  }
  for (int d = 0; d < dim; ++d) kin += u[ns + d] * u[ns + d];
  const double e = u[ns + dim] - 0.5 * kin / rho;
  if (P.two_temperature) {
    const int n = ns + 1;
    Yn[ns] = Y[ns] = u[ns + dim + 1];
    for (int it = 1; it <= max_it; ++it) {
      double R[9], J[81], T0, Tv0;
      if (!source_residual_tt(P, Y, Yn, e, h, R, &T0, &Tv0)) break;
      for (int k = 0; k < n; ++k) {
        const double eps = std::fmax(1e-7 * std::fabs(Y[k]), 1e-12);
        double Yp[9], Rp[9];
        for (int s = 0; s < n; ++s) Yp[s] = Y[s];
        Yp[k] += eps;
        if (!source_residual_tt(P, Yp, Yn, e, h, Rp, nullptr, nullptr)) return -1;
        for (int i = 0; i < n; ++i) J[i * n + k] = (Rp[i] - R[i]) / eps;
      }
      if (!gauss_jordan(n, J, R)) return -1;
      double lam = 1.0, Yt[9];
      for (int k = 0; k < 30; ++k) {
        for (int s = 0; s < n; ++s) Yt[s] = Y[s] - lam * R[s];
        const double Tt = temperature_of(m, Yt, e - Yt[ns]);
        const double Tvt = vib_temperature(m, Yt, Yt[ns]);
        if (Tt >= 0.5 * T0 && Tt <= 2.0 * T0 && Tvt >= 0.5 * Tv0 && Tvt <= 2.0 * Tv0) break;
        lam *= 0.5;
      }
      bool small = lam == 1.0 && std::fabs(R[ns]) <= tol * e;
      for (int s = 0; s < n; ++s) {
        if (s < ns) small = small && std::fabs(R[s]) <= tol * rho;
        Y[s] = Yt[s];
      }
      if (small) {
        for (int s = 0; s < ns; ++s) u[s] = Y[s];
        u[ns + dim + 1] = Y[ns];
        return it;
      }
    }
    for (int s = 0; s < ns; ++s) u[s] = Y[s];
    u[ns + dim + 1] = Y[ns];
    return -1;
  }
  for (int it = 1; it <= max_it; ++it) {
    double R[8], J[64];
    source_residual(m, Y, Yn, e, h, R);
    for (int k = 0; k < ns; ++k) {
      const double eps = std::fmax(1e-7 * std::fabs(Y[k]), 1e-12);
      double Yp[8], Rp[8];
      for (int s = 0; s < ns; ++s) Yp[s] = Y[s];
      Yp[k] += eps;
      source_residual(m, Yp, Yn, e, h, Rp);
      for (int i = 0; i < ns; ++i) J[i * ns + k] = (Rp[i] - R[i]) / eps;
    }
    if (!gauss_jordan(ns, J, R)) return -1;
    // the step, halved while the new temperature leaves [T/2, 2T]
    const double T0 = temperature_of(m, Y, e);
    double lam = 1.0, Yt[8];
    for (int k = 0; k < 30; ++k) {
      for (int s = 0; s < ns; ++s) Yt[s] = Y[s] - lam * R[s];
      const double Tt = temperature_of(m, Yt, e);
      if (Tt >= 0.5 * T0 && Tt <= 2.0 * T0) break;
      lam *= 0.5;
    }
    bool small = lam == 1.0;
    for (int s = 0; s < ns; ++s) {
      small = small && std::fabs(R[s]) <= tol * rho;  // false for a non-finite update
      Y[s] = Yt[s];
    }
    if (small) {
      for (int s = 0; s < ns; ++s) u[s] = Y[s];
      return it;
    }
  }
  for (int s = 0; s < ns; ++s) u[s] = Y[s];
  return -1;
}

// S_h over every node of a state, in place; returns the largest iteration count, or -1.
int source_implicit(const OrcProblem& P, double* U, double h, int max_it, double tol) {
  Mesh M(P);
  const int nv = n_vars(P);
  const size_t stride = (size_t)M.n_elem * M.n_nodes;
  int worst = 0;
  for (size_t q = 0; q < stride; ++q) {
    double u[16];
    for (int v = 0; v < nv; ++v) u[v] = U[v * stride + q];
    const int it = source_implicit_node(P, u, h, max_it, tol);
    worst = (it < 0 || worst < 0) ? -1 : std::max(worst, it);
    for (int v = 0; v < nv; ++v) U[v * stride + q] = u[v];
  }
  return worst;
}

}  // namespace

extern "C" {

// The Shu-Osher table of an SSP scheme (3: SSP-RK33, 54: SSP-RK54) as 5 x 5 row-major
// alpha and beta (row i = stage i+1), its stage count and its SSP coefficient.
int orc_ssp_table(int scheme, double* alpha, double* beta, int* s, double* c) {
  if (scheme != 3 && scheme != 54) return -1;
  SspTable t = ssp_table(scheme);
  for (int i = 0; i < 5; ++i)
    for (int k = 0; k < 5; ++k) {
      alpha[i * 5 + k] = t.alpha[i][k];
      beta[i * 5 + k] = t.beta[i][k];
    }
  *s = t.s;
  *c = ssp_coefficient(t);
  return 0;
}

// n_steps steps of the SSP scheme (3 or 54) in place, by the Shu-Osher sums as written.
int orc_ssp_steps(const OrcProblem* P, int scheme, double* U, double dt, int n_steps) {
  int rc = check_problem(*P);
  if (rc) return rc;
  if (scheme != 3 && scheme != 54) return -1;
  SspTable t = ssp_table(scheme);
  for (int k = 0; k < n_steps; ++k) ssp_step(*P, t, U, dt);
  return 0;
}

// One implicit source substep S_h over a whole state, in place (reacting problems).
// *iters receives the largest Newton count over the nodes (-1: some node did not converge).
int orc_source_implicit(const OrcProblem* P, double* U, double h, int max_it, double tol, int* iters) {
  int rc = check_problem(*P);
  if (rc) return rc;
  if (P->equations != ORC_NS_REACTING || !P->mech) return -1;
  *iters = source_implicit(*P, U, h, max_it, tol);
  return 0;
}

// n_steps Strang-split steps (Eq. strang_split), in place:
//   U <- S_{dt/2}( T_dt( S_{dt/2}(U) ) ),
// T_dt one step of the SSP scheme on the residual without its source part.
int orc_strang_steps(const OrcProblem* P, int scheme, double* U, double dt, int n_steps, int max_it,
                     double tol, int* iters) {
  int rc = check_problem(*P);
  if (rc) return rc;
  if (P->equations != ORC_NS_REACTING || !P->mech || (scheme != 3 && scheme != 54)) return -1;
  OrcProblem T = *P;
  T.parts = (P->parts ? P->parts : 7) & 3;
  if (T.parts == 0) T.parts = 8;  // no transport part: the residual is zero
  SspTable t = ssp_table(scheme);
  int worst = 0;
  for (int k = 0; k < n_steps; ++k) {
    const int a = source_implicit(*P, U, 0.5 * dt, max_it, tol);
    ssp_step(T, t, U, dt);
    const int b = source_implicit(*P, U, 0.5 * dt, max_it, tol);
    worst = (a < 0 || b < 0 || worst < 0) ? -1 : std::max(worst, std::max(a, b));
  }
  *iters = worst;
  return 0;
}

// Directional derivative of the residual (forward mode, dual numbers): for the strong, weak
// or two-point (Ranocha) volume form with the Rusanov, HLLC or EC surface flux,
//   L  = L(U; gamma)      and      dL = (dL/dU) V + (dL/dgamma) gdot.
int orc_rhs_jvp(const OrcProblem* P, const double* U, const double* V, double gdot, double* L,
                double* dL) {
  int rc = check_problem(*P);
  if (rc) return rc;
  // the dual-number residual has no shock capturing, periodic boundaries and Cartesian boxes only
  if (P->shock || P->coords || P->bc[0] || P->bc[1] || P->bc[2] || P->bc[3] || P->bc[4] || P->bc[5]) return -6;
  if ((P->volume != ORC_VOL_STRONG && P->volume != ORC_VOL_WEAK && P->volume != ORC_VOL_EC) ||
      (P->surface != ORC_SURF_RUSANOV && P->surface != ORC_SURF_HLLC && P->surface != ORC_SURF_EC) ||
      P->equations != ORC_EULER)
    return -6;
  Mesh M(*P);
  Ops ops(P->N);
  const size_t n = (size_t)n_vars(*P) * M.n_elem * M.n_nodes;
  std::vector<Dual> Ud(n), Ld(n);
  for (size_t q = 0; q < n; ++q) Ud[q] = Dual(U[q], V ? V[q] : 0.0);
  const Dual g(P->gamma, gdot);
#pragma omp parallel for schedule(static)
  for (int e = 0; e < M.n_elem; ++e) element_residual_t<Dual>(*P, M, ops, Ud.data(), g, e, Ld.data());
  for (size_t q = 0; q < n; ++q) {
    if (L) L[q] = Ld[q].v;
    dL[q] = Ld[q].d;
  }
  return 0;
}

// The logarithmic mean over duals (test access): *L = {{a}}^ln and
// *dL = (d{{a}}^ln/da) da + (d{{a}}^ln/db) db.
int orc_log_mean_jvp(double a, double b, double da, double db, double* L, double* dL) {
  if (!(a > 0.0) || !(b > 0.0)) return -1;
  const Dual m = log_mean_t(Dual(a, da), Dual(b, db));
  *L = m.v;
  *dL = m.d;
  return 0;
}

// Adjoint by brute force: (dL/dU)^T lam and lam . dL/dgamma, assembled from one
// directional derivative per unknown (tiny meshes only).
int orc_rhs_vjp_brute(const OrcProblem* P, const double* U, const double* lam, double* Ubar,
                      double* gbar) {
  int rc = check_problem(*P);
  if (rc) return rc;
  // the dual-number residual has no shock capturing, periodic boundaries and Cartesian boxes only
  if (P->shock || P->coords || P->bc[0] || P->bc[1] || P->bc[2] || P->bc[3] || P->bc[4] || P->bc[5]) return -6;
  Mesh M(*P);
  const size_t n = (size_t)n_vars(*P) * M.n_elem * M.n_nodes;
  if (n > 20000) return -1;
  std::vector<double> V(n, 0.0), dL(n);
  for (size_t j = 0; j < n; ++j) {
    V[j] = 1.0;
    if ((rc = orc_rhs_jvp(P, U, V.data(), 0.0, nullptr, dL.data()))) return rc;
    V[j] = 0.0;
    double acc = 0.0;
    for (size_t i = 0; i < n; ++i) acc += lam[i] * dL[i];
    Ubar[j] = acc;
  }
  if ((rc = orc_rhs_jvp(P, U, nullptr, 1.0, nullptr, dL.data()))) return rc;
  double acc = 0.0;
  for (size_t i = 0; i < n; ++i) acc += lam[i] * dL[i];
  *gbar = acc;
  return 0;
}

// Gradient of the rollout loss J = 1/2 sum_e sum_i wq[e][i] (rho_final - target)^2, where
// rho_final is the density after n_steps SSP-RK3 steps (App. B, Shu-Osher form) of size dt
// from U0 (strong or weak volume form, Rusanov flux), with respect to every entry of U0
// (grad, layout of U0) and gamma (*ggam).  Exact forward mode: one dual-number rollout per
// direction (tiny meshes only); an independent route to what the adjoint computes in reverse.
int orc_rollout_grad(const OrcProblem* P, const double* U0, const double* target, const double* wq,
                     double dt, int n_steps, double* grad, double* ggam) {
  int rc = check_problem(*P);
  if (rc) return rc;
  // the dual-number residual has no shock capturing, periodic boundaries and Cartesian boxes only
  if (P->shock || P->coords || P->bc[0] || P->bc[1] || P->bc[2] || P->bc[3] || P->bc[4] || P->bc[5]) return -6;
  if ((P->volume != ORC_VOL_STRONG && P->volume != ORC_VOL_WEAK && P->volume != ORC_VOL_EC) ||
      (P->surface != ORC_SURF_RUSANOV && P->surface != ORC_SURF_HLLC && P->surface != ORC_SURF_EC) ||
      P->equations != ORC_EULER)
    return -6;
  Mesh M(*P);
  Ops ops(P->N);
  const size_t stride = (size_t)M.n_elem * M.n_nodes;
  const size_t n = (size_t)n_vars(*P) * stride;
  if (n > 4000 || n_steps < 0) return -1;
  std::vector<Dual> Un(n), U1(n), U2(n), L(n);
  for (size_t dir = 0; dir <= n; ++dir) {
    for (size_t q = 0; q < n; ++q) Un[q] = Dual(U0[q], q == dir ? 1.0 : 0.0);
    const Dual g(P->gamma, dir == n ? 1.0 : 0.0);
    for (int s = 0; s < n_steps; ++s) {
      for (int e = 0; e < M.n_elem; ++e) element_residual_t<Dual>(*P, M, ops, Un.data(), g, e, L.data());
      for (size_t q = 0; q < n; ++q) U1[q] = Un[q] + Dual(dt) * L[q];
      for (int e = 0; e < M.n_elem; ++e) element_residual_t<Dual>(*P, M, ops, U1.data(), g, e, L.data());
      for (size_t q = 0; q < n; ++q) U2[q] = Dual(0.75) * Un[q] + Dual(0.25) * (U1[q] + Dual(dt) * L[q]);
      for (int e = 0; e < M.n_elem; ++e) element_residual_t<Dual>(*P, M, ops, U2.data(), g, e, L.data());
      for (size_t q = 0; q < n; ++q)
        Un[q] = Dual(1.0 / 3.0) * Un[q] + Dual(2.0 / 3.0) * (U2[q] + Dual(dt) * L[q]);
    }
    double dJ = 0.0;  // dJ = sum wq (rho - target) drho
    for (size_t q = 0; q < stride; ++q) dJ += wq[q] * (Un[q].v - target[q]) * Un[q].d;
    if (dir < n) grad[dir] = dJ;
    else *ggam = dJ;
  }
  return 0;
}

// Convective time-step bound (Sec. 3.1.2 Eq. dt_hyp; App. B):
//   dt = cfl * dx_min / ((2N+1) lambda_max),  lambda_max = max over nodes of |u| + a.
// READING: |u| is the speed (vector magnitude); the SSP coefficient of SSP-RK3 is 1, so
// cfl multiplies nothing else; dx_min is the smallest element edge.
}  // extern "C"

namespace {
// READING (curved meshes): the element size in direction l is 2 J / |Ja^l| (the physical
// length of the reference interval; dx_l on the affine box), minimised over the nodes.
double curved_spacing(const OrcProblem& P, const Mesh& M) {
  Ops ops(P.N);
  const Metrics G = curved_metrics(P, M, ops);
  const size_t stride = (size_t)M.n_elem * M.n_nodes;
  double dxmin = 1e300;
  for (size_t q = 0; q < stride; ++q)
    for (int l = 0; l < M.dim; ++l) {
      double s2 = 0.0;
      for (int d = 0; d < M.dim; ++d) s2 += G.Ja[(q * 3 + l) * 3 + d] * G.Ja[(q * 3 + l) * 3 + d];
      dxmin = std::fmin(dxmin, 2.0 * G.J[q] / std::sqrt(s2));
    }
  return dxmin;
}
}  // namespace

extern "C" {

int orc_max_dt(const OrcProblem* P, const double* U, double cfl, double* dt) {
  int rc = check_problem(*P);
  if (rc) return rc;
  Mesh M(*P);
  const int dim = M.dim, nv = n_vars(*P);
  const size_t stride = (size_t)M.n_elem * M.n_nodes;
  double lam = 0.0;
  if (P->equations == ORC_NS_REACTING) {
    // reacting: frozen sound speed of the mixture for dt_C; the diffusive bound
    // (Sec. 3.1.2 Eq. dt_para; App. B) dt_D = cfl dx_min^2 / ((2N+1)^2 nu_max) with
    // nu_max = max over nodes of max(mu / rho, k / (rho c_p)) = max(mu/rho, mu/(rho Pr)).
    // READING: cfl multiplies both bounds (the SSP coefficient of SSP-RK3 is 1).
    double nu = 0.0;
    for (size_t q = 0; q < stride; ++q) {
      double u[16];
      for (int v = 0; v < nv; ++v) u[v] = U[v * stride + q];
      Mix m = mixture(*P, u);
      double speed = 0.0;
      for (int d = 0; d < dim; ++d) speed += m.v[d] * m.v[d];
      lam = std::fmax(lam, std::sqrt(speed) + m.a);
      nu = std::fmax(nu, std::fmax(P->mu / m.rho, P->mu / (m.rho * P->prandtl)));
    }
    double dxmin = M.dx[0];
    for (int l = 1; l < dim; ++l) dxmin = std::fmin(dxmin, M.dx[l]);
    if (P->coords) dxmin = curved_spacing(*P, M);  // as for the curved Euler bound below
    const double dtc = cfl * dxmin / ((2 * P->N + 1) * lam);
    const double n2 = (2.0 * P->N + 1) * (2.0 * P->N + 1);
    *dt = nu > 0.0 ? std::fmin(dtc, cfl * dxmin * dxmin / (n2 * nu)) : dtc;
    return 0;
  }
  for (size_t q = 0; q < stride; ++q) {
    double u[8];
    for (int v = 0; v < nv; ++v) u[v] = U[v * stride + q];
    Prim pr = primitives(dim, u, P->gamma);
    double speed = 0.0;
    for (int d = 0; d < dim; ++d) speed += pr.v[d] * pr.v[d];
    lam = std::fmax(lam, std::sqrt(speed) + sound_speed(pr, P->gamma));
  }
  double dxmin = M.dx[0];
  for (int l = 1; l < dim; ++l) dxmin = std::fmin(dxmin, M.dx[l]);
  if (P->coords) dxmin = curved_spacing(*P, M);
  *dt = cfl * dxmin / ((2 * P->N + 1) * lam);
  return 0;
}

}  // extern "C"
