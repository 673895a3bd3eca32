/* dgsem.h -- C-ABI of the B300 (sm_103a) DGSEM residual and SSP-RK stage library.
 *
 * The library evaluates the semi-discrete DGSEM residual of the compressible Euler
 * equations, and of the single-temperature reacting Navier-Stokes equations, on Cartesian
 * meshes (periodic, or with per-face boundary conditions) and on curved meshes (periodic
 * ones for Navier-Stokes) and advances it with the SSP-RK33 or SSP-RK54 scheme, entirely in
 * hand-written CUDA kernels (one fused kernel per RK stage for Euler; a BR1 gradient pass
 * plus one fused kernel for Navier-Stokes; one per-node kernel for the implicit chemistry
 * substep of the Strang split).  The operations follow arXiv 2605.26388:
 *   - equations and ideal-gas closure: Sec. 2;
 *   - viscous terms: BR1 lifting (Sec. 3.1.2, Eqs. br1_avg, tau, br1_flux);
 *   - finite-rate chemistry: Arrhenius source (Sec. 3.1.3, Eqs. src_reaction_rate,
 *     src_omega; App. C), in the residual or by the Strang split with a per-node
 *     backward-Euler Newton substep (Sec. 3.1.3, Eqs. strang_split, source_residual);
 *   - element-local DGSEM on (N+1)^d GLL nodes: Sec. 3.1.1 and App. A;
 *   - volume term: Eq. vol_weak (strong form; the weak form is the same operator by the
 *     SBP property) or Eq. vol_split / Eq. split_form_3D (flux differencing with the
 *     Ranocha entropy-conservative two-point flux);
 *   - surface term: Eq. surf_int with a Riemann flux (Sec. 3.1.1 "Surface Fluxes");
 *   - time integration: App. B (SSP-RK33 and SSP-RK54, Shu-Osher form) and Eq. dt_hyp
 *     (time-step bound).
 *
 * Conventions shared by every entry point:
 *   - State layout (SoA, FP64): U[v * n_nodes_total + node_offset(instance) + e * n_p + q]
 *     with v the conserved variable -- Euler: (rho, rho u, rho v[, rho w], E); Navier-Stokes:
 *     (rho_1 .. rho_ns, rho u, rho v, rho w, E) -- e the element index
 *     within its instance (lexicographic, x fastest), q the node index within the element
 *     (lexicographic, i fastest) and n_p = (N+1)^dim.  n_nodes_total is the sum over
 *     instances of n_elem * n_p.
 *   - Array arguments are owned by the caller; the library never frees them.  Unless an
 *     entry point says otherwise they are DEVICE pointers on the context's device.
 *   - Launches are asynchronous on the context's CUDA stream.  Device-side faults of the
 *     state (non-finite values, non-positive density or pressure) are recorded in a
 *     device error word and reported by dg_check(), which synchronizes the stream.
 *   - No entry point aborts, prints or traps.  Errors are returned as dg_status, with a
 *     message in dg_last_error().
 */
#ifndef DGSEM_H
#define DGSEM_H

#include <stdint.h>

#if defined(__GNUC__)
#define DG_API __attribute__((visibility("default")))
#else
#define DG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_ctx dg_ctx; /* opaque: mesh, operators, stage buffers, error word */

typedef enum {
  DG_OK = 0,
  DG_EINVAL = -1,       /* bad argument or description */
  DG_ENOMEM = -2,       /* device allocation failed */
  DG_ECUDA = -3,        /* a CUDA runtime call failed */
  DG_ENONFINITE = -4,   /* a kernel produced a non-finite value */
  DG_EPOSITIVITY = -5,  /* a kernel read a state with rho <= 0 or p <= 0 */
  DG_EUNSUPPORTED = -6, /* valid but not implemented (e.g. the adjoint on a curved mesh) */
  DG_ETOOLARGE = -7,    /* more instances than dg_max_dt_noalloc's static scratch holds */
  DG_ECONVERGENCE = -8  /* a node's Newton iteration (implicit source, or the vibrational
                        * temperature of the two-temperature model) did not converge */
} dg_status;

/* Equations.  DG_NAVIER_STOKES is the single-gas, non-dimensional case (R = 1, so T = p/rho,
 * cv = 1/(gamma-1), conductivity k = gamma mu / ((gamma-1) Pr)); DG_NS_REACTING takes its
 * species and reactions from dg_physics.chem (SI units).  Both: 3D, Cartesian, strong volume
 * form, Rusanov surface flux, no positivity floor, no shock capturing; others return
 * DG_EUNSUPPORTED. */
enum { DG_EULER = 0, DG_NAVIER_STOKES = 1, DG_NS_REACTING = 2 };
/* Volume term: strong form (Eq. vol_weak), weak form (integrated by parts; equal to the
 * strong form by SBP), or two-point flux differencing with Ranocha's EC flux
 * (Eq. vol_split). */
enum { DG_VOL_STRONG = 0, DG_VOL_WEAK = 1, DG_VOL_EC = 2 };
/* Riemann flux at element faces: local Lax-Friedrichs (Rusanov), HLLC, HLL, or Ranocha's
 * EC flux (no dissipation; used to check entropy conservation). */
enum { DG_SURF_RUSANOV = 0, DG_SURF_HLLC = 1, DG_SURF_HLL = 2, DG_SURF_EC = 3 };
/* Arithmetic: plain FP64 throughout, or FP32 volume/surface flux arithmetic with the
 * state, the RK accumulation, the pressure (from the FP64 total energy) and the
 * positivity decision kept in FP64. */
enum { DG_FP64 = 0, DG_FP32_MIXED = 1 };
/* Time integration (App. B): SSP-RK33 of Shu and Osher (SSP coefficient 1) or SSP-RK54 of
 * Spiteri and Ruuth (five stages, fourth order, SSP coefficient 1.508; the paper's
 * production integrator, with the coefficients of its publication). */
enum { DG_SSPRK33 = 0, DG_SSPRK54 = 1 };
/* Defaults of the Hennemann-Gassner blending bounds (dg_physics fields <= 0); the sigmoid's
 * steepness defaults to ln(9999), which puts the blending of a perfectly smooth element at
 * 1e-4 before the cut. */
#define DG_ALPHA_MIN 0.001
#define DG_ALPHA_MAX 0.5
/* Defaults of the implicit source substep's Newton iteration (dg_physics fields <= 0). */
#define DG_NEWTON_MAX_IT 40
#define DG_NEWTON_TOL 1e-12

/* Boundary conditions of a non-periodic domain face (Sec. 3.1.1 "Surface Fluxes": one
 * functor per boundary type; enforced weakly through the numerical flux, Sec. 4 set-ups).
 * Inviscid flux:
 *   DG_BC_SLIP_WALL  the Riemann flux against the mirror state (normal momentum reversed);
 *   DG_BC_INFLOW     supersonic inflow: the flux F^l(U_b) of the prescribed state;
 *   DG_BC_OUTFLOW    supersonic outflow: the flux F^l(U-) of the interior state;
 *   DG_BC_DIRICHLET  free stream: the Riemann flux against the prescribed state U_b;
 *   DG_BC_NOSLIP_*   as DG_BC_SLIP_WALL (Sec. 4: walls are slip walls for the inviscid flux).
 * Viscous terms (DG_NAVIER_STOKES, DG_NS_REACTING; Sec. 3.1.2 boundary kernels), the BR1
 * trace of (u, v, w, T) and the viscous numerical flux (F_v^l)* at the face:
 *   DG_BC_SLIP_WALL           trace: velocity with its normal part removed, T inherited;
 *                             flux: the normal-stress row tau_ll only (no shear, no heat);
 *   DG_BC_NOSLIP_ADIABATIC    trace: velocity 0, T inherited; flux: the interior stress
 *                             rows, energy 0 (no work, no heat through the wall);
 *   DG_BC_NOSLIP_ISOTHERMAL   trace: velocity 0, T = T_wall; flux: the interior stress rows,
 *                             energy k dT/dx_l (conduction through the wall, no work);
 *   DG_BC_INFLOW, DG_BC_DIRICHLET  trace: (u, v, w, T) of U_b; flux: the interior flux;
 *   DG_BC_OUTFLOW             trace and flux: the interior ones (no viscous lift).
 * Two-temperature model: the T_v trace is the interior's at slip and adiabatic walls and at
 * outflow faces, T_wall at isothermal walls, U_b's at inflow and Dirichlet faces; the E_v
 * flux row is 0 at slip and adiabatic walls, k_v dT_v/dx_l at isothermal walls (whose energy
 * row then carries k dT/dx_l + k_v dT_v/dx_l), the interior flux at far-field faces.
 * The no-slip walls need viscous equations (DG_EULER: DG_EINVAL). */
enum { DG_BC_SLIP_WALL = 1, DG_BC_INFLOW = 2, DG_BC_OUTFLOW = 3, DG_BC_DIRICHLET = 4,
       DG_BC_NOSLIP_ADIABATIC = 5, DG_BC_NOSLIP_ISOTHERMAL = 6 };
/* Conserved variables of one node at most: 8 species, 3 momenta, energy. */
#define DG_MAX_VARS 12

/* One Cartesian mesh instance (Sec. 3.1.1: element-wise affine map of the reference cube;
 * collocation on (N+1)^dim GLL nodes). */
typedef struct {
  int dim;          /* 2 or 3 */
  int N;            /* polynomial degree: 1..7 in 2D, 1..5 in 3D (Navier-Stokes: 1..4) */
  int nel[3];       /* elements per direction (nel[2] ignored in 2D) */
  double lo[3];     /* box lower corner */
  double hi[3];     /* box upper corner */
  int periodic[3];  /* 1: periodic in that direction; 0: the faces bc[2l] (lower) and bc[2l+1]
                     * (upper) carry boundary conditions */
  int bc[6];        /* DG_BC_* per face x-, x+, y-, y+, z-, z+ of a non-periodic direction */
  double bc_state[6][DG_MAX_VARS];  /* DG_BC_INFLOW / DG_BC_DIRICHLET: the conserved state U_b
                           * of that face in the state's variable order -- (rho, rho u, rho v
                           * [, rho w], E) for DG_EULER, (rho_1..rho_ns, rho u, rho v, rho w, E)
                           * for the viscous equations -- with rho > 0 and p > 0 (Euler) or
                           * T > 0 (viscous); DG_BC_NOSLIP_ISOTHERMAL: bc_state[f][0] = T_wall
                           * > 0 (the non-dimensional T = p/rho for DG_NAVIER_STOKES, K for
                           * DG_NS_REACTING).  Else DG_EINVAL. */
  const double* coords;   /* NULL: the affine box.  Else a curved mesh on the same element
                           * topology (Sec. 3.1.1: element maps, metric terms Ja^l with the
                           * discrete GCL): host array of the node coordinates,
                           * coords[d * n_elem * n_p + e * n_p + q], copied at dg_init_mesh.
                           * Periodic directions must map periodically; a non-periodic direction
                           * takes its boundary conditions along the faces' contravariant normal
                           * (the slip wall mirrors the velocity across it).  DG_EULER: strong
                           * or two-point volume form.  The viscous equations: periodic in every
                           * direction, no species limiter (Sec. 3.1.2 BR1 on the mapped
                           * element: the reference derivative mapped by Ja^l and 1/J).  No
                           * shock capturing, no positivity floor (else DG_EUNSUPPORTED); every
                           * element must have J > 0 (else DG_EINVAL). */
} dg_mesh_desc;

/* Species and reactions of a reacting mixture (Sec. 2 thermochemistry, single temperature;
 * Sec. 3.1.3 and App. C).  Calorically perfect species: e_s = cv_s T + h0_s, p = sum rho_s R_s T.
 * Reaction r: sum_s nu_f[r][s] X_s <-> sum_s nu_b[r][s] X_s with
 *   k_f = exp(lnA + b ln T - Ta / T)                      (cm-mol-s units),
 *   ln K_c = kc0 / Z + kc1 + kc2 ln Z + kc3 Z + kc4 Z^2,   Z = 10^4 / T,
 *   R_r = k_f prod [X]^nu_f - (k_f / K_c) prod [X]^nu_b,   [X_s] = rho_s / W_s in mol/cm^3,
 *   omega_s = 10^6 W_s sum_r (nu_b - nu_f) R_r            (kg m^-3 s^-1).
 * Compiled kernels: n_species 1 or 5; each side of a reaction has at most 3 molecules. */
#define DG_MAX_SPECIES 8
#define DG_MAX_REACTIONS 32
typedef struct dg_mechanism {
  int n_species;                      /* 1..DG_MAX_SPECIES */
  int n_reactions;                    /* 0..DG_MAX_REACTIONS */
  double W[DG_MAX_SPECIES];           /* molar mass, kg/mol */
  double R[DG_MAX_SPECIES];           /* specific gas constant, J/(kg K) */
  double cv[DG_MAX_SPECIES];          /* specific heat at constant volume, J/(kg K) */
  double h0[DG_MAX_SPECIES];          /* formation energy, J/kg */
  double lnA[DG_MAX_REACTIONS];
  double b[DG_MAX_REACTIONS];
  double Ta[DG_MAX_REACTIONS];        /* activation temperature, K */
  double kc[DG_MAX_REACTIONS][5];
  int nu_f[DG_MAX_REACTIONS][DG_MAX_SPECIES];
  int nu_b[DG_MAX_REACTIONS][DG_MAX_SPECIES];
  /* Two-temperature model only (dg_physics.two_temperature; ignored otherwise): */
  double theta_v[DG_MAX_SPECIES];     /* characteristic vibrational temperature, K (>= 0; 0 for
                                       * atoms): e_v,s(T) = R_s theta / (exp(theta / T) - 1) */
  int ta_mode[DG_MAX_REACTIONS];      /* 1: the reaction's controlling temperature is
                                       * T_a = sqrt(T T_v) (dissociation), 0: T_a = T */
} dg_mechanism;

typedef struct {
  int equations;    /* DG_EULER | DG_NAVIER_STOKES | DG_NS_REACTING */
  int volume;       /* DG_VOL_* */
  int surface;      /* DG_SURF_* */
  int precision;    /* DG_FP64 | DG_FP32_MIXED */
  double gamma;     /* ratio of specific heats (Sec. 2 closure) */
  double rho_floor; /* > 0: clamp rho after each stage (Sec. 4 set-ups); <= 0: off */
  double p_floor;   /* > 0: reset E so that p >= p_floor after each stage; <= 0: off */
  double p_ref;     /* constant subtracted from the pressure in the momentum flux, p -> p - p_ref.
                     * Leaves the discrete operator unchanged in exact arithmetic (rows of D sum
                     * to zero; F* - F(U_own) is invariant to a common constant) and keeps FP32
                     * flux arithmetic out of cancellation at low Mach number.  0 = no shift.
                     * dg_two_point_flux reports momentum fluxes with this shift applied. */
  /* Navier-Stokes only (ignored for DG_EULER): */
  double mu;        /* constant dynamic viscosity (>= 0) */
  double prandtl;   /* Prandtl number (> 0); conductivity k = mu c_p / Pr */
  const dg_mechanism* chem;  /* DG_NS_REACTING: species and reactions (copied at init) */
  /* Time integration (a zero-filled struct gives SSP-RK33 with the source in the residual): */
  int time_scheme;  /* DG_SSPRK33 | DG_SSPRK54 */
  int chem_split;   /* DG_NS_REACTING only: 0 the Arrhenius source is part of L(U); 1 Strang
                     * split (Eq. strang_split): L(U) has no source and every step is
                     * S_{dt/2} o T_dt o S_{dt/2}, S the implicit substep of dg_source_step */
  int newton_max_it;  /* implicit substep: Newton updates per node at most (<= 0: default) */
  double newton_tol;  /* stop once max_s |dY_s| <= newton_tol * rho (<= 0: default) */
  /* Shock capturing (Sec. 3.1.1 "Shock Indicator and Smoothing", Eq. vol_blend; App. A):
   * DG_EULER only, N >= 2 (N <= 7 in 2D, <= 5 in 3D), per-instance launches. */
  int shock;        /* 1: every stage blends R = (1 - alpha_e) R^DG + alpha_e R^FV per element */
  double alpha_min; /* blending below this is cut to 0 (<= 0: DG_ALPHA_MIN) */
  double alpha_max; /* blending is capped here (<= 0: DG_ALPHA_MAX) */
  double sharpness; /* steepness s of the sigmoid (<= 0: ln 9999) */
  /* Two-temperature model (Sec. 2 "Thermal nonequilibrium coupling" and "Total energy and
   * closure"; Sec. 3.1.3 Eqs. src_vector, src_reaction_rate, src_landau_teller): DG_NS_REACTING
   * with 5 species (else DG_EUNSUPPORTED).  The state gains
   * E_v, U = (rho_1..rho_ns, rho u, rho v, rho w, E, E_v); cv_s is the translational-rotational
   * heat capacity and E = sum rho_s (cv_s T + h0_s) + E_v + rho|u|^2/2; T_v solves
   * E_v = sum rho_s e_v,s(T_v) (harmonic oscillators of chem->theta_v); the E_v flux is E_v u,
   * the vibrational heat flux -k_v grad T_v (k_v = mu c_v,v / Pr, c_v,v = dE_v/dT_v / rho)
   * enters the E and E_v rows; reaction r runs at its controlling temperature (ta_mode) with
   * k_b = k_f / K_c(T_a); the E_v source is Q_T-v + sum_s omega_s e_v,s(T_v) with the
   * Landau-Teller Q_T-v = sum rho_s (e_v,s(T) - e_v,s(T_v)) / tau_s, tau_s the Millikan-White
   * relaxation time plus Park's high-temperature term.  A node whose T_v iteration does not
   * converge sets DG_ECONVERGENCE. */
  int two_temperature;  /* 0: single temperature; 1: two-temperature */
  /* Zhang-Shu positivity limiter of the partial densities (Sec. 4 reacting blast set-up:
   * rho_s >= 0 per species; DG_NAVIER_STOKES and DG_NS_REACTING, else DG_EINVAL): after every
   * RK stage, per element and species with a negative nodal value, the nodal values contract
   * toward the GLL-weighted element mean m, rho_s <- m + theta (rho_s - m), theta =
   * m / (m - min rho_s) (the mean itself when m <= 0); element means are kept, momentum and
   * energy are untouched.  One extra launch per stage. */
  int species_limiter;  /* 0: off; 1: on */
} dg_physics;

/* Build a context for n_inst instances (all of the same dim) sharing one physics
 * description.  Allocates the context-held state and stage buffers on the current CUDA
 * device.  `cuda_stream` is a cudaStream_t (NULL = legacy default stream).
 * Returns DG_EINVAL on a bad description (including a boundary type the equations do not
 * have or a bad boundary state), DG_EUNSUPPORTED on an unsupported combination (dim, N,
 * options; boundary conditions with the batched launch, curved meshes or the adjoint),
 * DG_ENOMEM if allocation fails.  *out is NULL on failure. */
DG_API dg_status dg_init_mesh(const dg_mesh_desc* inst, int n_inst, const dg_physics* phys,
                       void* cuda_stream, dg_ctx** out);

/* Total number of doubles of one state (n_vars * n_nodes_total) and n_vars. */
DG_API dg_status dg_state_size(const dg_ctx* ctx, int64_t* n_doubles, int* n_vars);

/* Node offset of instance i within a variable's slab. */
DG_API dg_status dg_instance_offset(const dg_ctx* ctx, int i, int64_t* offset);

/* Copy a state into / out of the context-held state.  U may be a device pointer or a host
 * pointer (pinned host memory gives full PCIe/C2C speed); unified addressing resolves the
 * direction.  Asynchronous on the context's stream (the host buffer must stay valid until
 * the stream reaches the copy). */
DG_API dg_status dg_set_state(dg_ctx* ctx, const double* U);
DG_API dg_status dg_get_state(const dg_ctx* ctx, double* U);

/* dUdt = L(U) at time t (the residual does not depend on t).  U and dUdt are device
 * pointers of dg_state_size() doubles and must not overlap.  Under the Strang split L has
 * no chemical source. */
DG_API dg_status dg_rhs(dg_ctx* ctx, const double* U, double* dUdt, double t);

/* One SSP-RK3 stage (App. B, Shu-Osher form) on caller buffers:
 *   stage 1: Uout = Un + dt L(Un)                       (Uprev must equal Un)
 *   stage 2: Uout = 3/4 Un + 1/4 (Uprev + dt L(Uprev))
 *   stage 3: Uout = 1/3 Un + 2/3 (Uprev + dt L(Uprev))
 * followed by the positivity floor when enabled.  Uout must not alias Un or Uprev.  The
 * stage is SSP-RK3's whatever the context's time_scheme. */
DG_API dg_status dg_rk_stage(dg_ctx* ctx, int stage, const double* Un, const double* Uprev,
                      double dt, double* Uout);

/* n_steps steps of size dt on the context-held state with the context's time_scheme:
 * SSP-RK33 (3 fused stage launches per step) or SSP-RK54 (5 launches; stage 4 also writes
 * the running sum a52 U2 + a53 U3 + b53 dt L(U3) of stage 5 into a fourth buffer).  Under
 * the Strang split each step is wrapped in two implicit source substeps of dt/2.  Steps are
 * replayed from a CUDA graph.  Asynchronous: call dg_check() to synchronize and collect
 * device-side errors. */
DG_API dg_status dg_rk_step(dg_ctx* ctx, double dt, int n_steps);

/* Adjoint of the residual (for differentiable rollouts; the paper has no adjoint -- it is the
 * exact transpose of the semi-discrete operator of the Euler equations on affine meshes:
 * the strong or weak volume form (Eq. vol_weak) or the two-point form (Eq. vol_split with
 * Ranocha's flux, App. A), with the Rusanov or HLLC flux -- periodic or with boundary
 * conditions (the functors' exterior states differentiated with the own trace: the slip
 * wall's mirror state, U_b fixed); other surface fluxes, shock capturing and curved meshes
 * return DG_EUNSUPPORTED):
 *   Ubar += (dL/dU)^T lam            (device arrays of dg_state_size() doubles)
 *   *gammabar += lam . dL/dgamma     (host double)
 * Non-smooth points follow the forward evaluation: the larger Rusanov signal speed (the left
 * one on a tie) carries the derivative, and d|u|/du = sign(u) with sign(0) = 0; the HLLC
 * flux's branch and the min/max of its wave speeds follow the values (the left argument on a
 * tie); the logarithmic means are differentiated in their series form near equal
 * arguments, where the derivative is 1/2 in each.  Ubar must not
 * alias U or lam.  Allocates the adjoint workspace on first use.  The gamma contribution is
 * added to a device accumulator of the context; with gammabar != NULL the call synchronizes
 * the stream, adds the accumulator to *gammabar and resets it; with gammabar == NULL it stays
 * on the device (no synchronization) until dg_adjoint_gammabar(). */
DG_API dg_status dg_rhs_vjp(dg_ctx* ctx, const double* U, const double* lam, double* Ubar,
                            double* gammabar);

/* Adjoint of one SSP step from Un with step dt (App. B, Shu-Osher form, the context's scheme,
 * stages recomputed from Un; SSP-RK54 reverses its five stages through the table,
 * lam^(k) = sum_i alpha_ik lam^(i) + dt (dL/dU(U^(k)))^T sum_i beta_ik lam^(i)): on entry
 * lam = dJ/dU^{n+1}, on exit lam = dJ/dU^n; *gammabar (host)
 * += dJ/dgamma through this step.  The positivity floor, if enabled, is not differentiated.
 * lam must not alias Un.  gammabar as for dg_rhs_vjp: NULL keeps the contribution in the
 * context's device accumulator and the call stays asynchronous. */
DG_API dg_status dg_rk_step_vjp(dg_ctx* ctx, const double* Un, double dt, double* lam,
                                double* gammabar);

/* Synchronize the stream and add the gamma contributions accumulated on the device by
 * adjoint calls made with gammabar == NULL to *gammabar (host); resets the accumulator. */
DG_API dg_status dg_adjoint_gammabar(dg_ctx* ctx, double* gammabar);

/* Launch modes for contexts with several instances. */
enum { DG_LAUNCH_PER_INSTANCE = 0, DG_LAUNCH_BATCHED = 1 };

/* Per-degree group scale for dg_set_launch: DG_GROUPS_PER_DEGREE | mask, bit N of mask
 * (N = 1..5) giving degree N work items of twice the base group (2D only). */
#define DG_GROUPS_PER_DEGREE 0x100

/* How a stage is launched over the context's instances (batched form; the paper runs
 * one problem at a time): one fused launch per instance, or one persistent launch per stage
 * over a work list of (instance, element group) items covering every instance -- the default
 * when n_inst > 1.  group_scale multiplies the elements per work item: 1 (or 2 in 2D) for
 * every degree, or, in 2D, DG_GROUPS_PER_DEGREE | mask for a choice per degree (the degrees
 * with scale 1 and those with scale 2 then run as two persistent launches per stage, one
 * after the other on the context's stream); ctas_per_sm caps the persistent grid (0 = as many
 * CTAs as fit); order 0 puts the heaviest items (degree, then instance) first, 1 keeps
 * instance order.  Synchronizes the stream and rebuilds the work list; DG_EINVAL on an
 * out-of-range choice.  The batched mode (and the autotuner below) exists for the Euler
 * equations; Navier-Stokes contexts return DG_EUNSUPPORTED for it. */
DG_API dg_status dg_set_launch(dg_ctx* ctx, int mode, int group_scale, int ctas_per_sm, int order);

/* Autotuner for the launch configuration: times n_reps SSP-RK3 steps of size dt for the
 * per-instance mode and every uniform batched choice (group_scale x ctas_per_sm in {0,1,2} x
 * order), then, in 2D with several degrees, every per-degree group scale (each subset of the
 * degrees present taking scale 2) with the best uniform choice's ctas_per_sm and order;
 * restores the context-held state afterwards, keeps the fastest configuration and reports it:
 * config_out[4] = {mode, group_scale, ctas_per_sm, order}, *ms_out (host, may be NULL) = its
 * time per step in ms.  Allocates one temporary state copy; synchronizes the stream. */
DG_API dg_status dg_autotune(dg_ctx* ctx, double dt, int n_reps, int* config_out, double* ms_out);

/* Convective time-step bound of Eq. dt_hyp (App. B) on the context-held state:
 *   dt = c * cfl * dx_min / ((2N+1) * max over nodes of (|u| + a)),
 * c the SSP coefficient of the context's time_scheme (1 for SSP-RK33, 1.508 for SSP-RK54),
 * taking the minimum over instances.  Navier-Stokes: a is the frozen mixture sound speed and
 * the result is min(dt_C, dt_D) with the diffusive bound of Eq. dt_para,
 *   dt_D = c * cfl * dx_min^2 / ((2N+1)^2 * max over nodes of max(mu/rho, mu/(rho Pr))).
 * A state with a non-finite value at any node returns DG_ENONFINITE, one with rho <= 0 or
 * p <= 0 (T <= 0 for Navier-Stokes) at any node DG_EPOSITIVITY; no bound is taken from the
 * other nodes.  Synchronizes the stream; *dt_out is a host double. */
DG_API dg_status dg_max_dt(dg_ctx* ctx, double cfl, double* dt_out);

/* Synchronize the context's stream, then read and clear the device error word:
 * DG_ENONFINITE or DG_EPOSITIVITY if a kernel since the last check flagged the state. */
DG_API dg_status dg_check(dg_ctx* ctx);

/* The library's own GLL nodes x[0..N], weights w[0..N] and differentiation matrix
 * D[(N+1)*(N+1)] (row-major, D[i*(N+1)+m] = l_m'(x_i)); host pointers, N in 1..7. */
DG_API dg_status dg_gll(int N, double* x, double* w, double* D);

/* Evaluate the device's two-point flux for n state pairs (device pointers, AoS n x n_vars)
 * in direction l: kind = -1 the EC volume flux, else a DG_SURF_* kind.  Uses the context's
 * precision and gamma.  Test and inspection aid (Euler contexts only). */
DG_API dg_status dg_two_point_flux(dg_ctx* ctx, int kind, int l, int n, const double* uL,
                            const double* uR, double* F);

/* The time-step bound of dg_max_dt() for callers that cannot allocate GPU memory -- for
 * example code running under another framework's caching allocator, which has already
 * reserved the device's memory, or an application that fixes its GPU footprint up front.
 * The paper has no counterpart; this is an interface convenience.  It needs no context:
 * the caller passes the instance descriptions (as for dg_init_mesh), gamma, a device
 * pointer U to a state in the library's SoA layout (instances concatenated in the order
 * given), cfl, and a cudaStream_t (NULL = legacy default stream).  *dt_out (host) receives
 * min over instances of cfl * dx_min / ((2N+1) * max(|u| + a)): the bound dg_max_dt gives a
 * Cartesian SSP-RK33 context (SSP coefficient 1; SSP-RK54 callers scale cfl by its
 * coefficient 1.508 themselves).  Curved instances (coords != NULL) return DG_EUNSUPPORTED:
 * the bound here uses the box spacing.  A non-finite value at any node returns
 * DG_ENONFINITE, rho <= 0 or p <= 0 at any node DG_EPOSITIVITY.  If msg is not NULL it
 * receives a static description of any error.
 * It calls no cudaMalloc/cudaFree: the per-instance reduction scratch is a static device
 * array of DG_NOALLOC_MAX_INSTANCES 64-bit slots inside the library, held by every GPU that
 * loads the library until exit.  n_inst above that limit returns DG_ETOOLARGE.  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress), so make that
 * first call before any stream capture.  All calls share the array and each clears the slots
 * it uses; calls that overlap on the GPU (different streams or threads) race and must be
 * serialized by the caller.  Synchronizes the stream. */
#define DG_NOALLOC_MAX_INSTANCES 4096
DG_API dg_status dg_max_dt_noalloc(const dg_mesh_desc* inst, int n_inst, double gamma,
                                   const double* U, double cfl, void* cuda_stream,
                                   double* dt_out, const char** msg);

/* Implicit source substep S_h of the Strang split (Sec. 3.1.3, Eqs. strang_split and
 * source_residual), DG_NS_REACTING contexts only.  At every node the partial densities
 * Y = (rho_1..rho_ns) take one backward-Euler step of length h >= 0 of the chemical source,
 *   Y* - Y - h omega(Y*) = 0,
 * solved by Newton's method from Y* = Y: the Jacobian by forward differences, column k with
 * the perturbation eps_k = max(1e-7 |Y*_k|, 1e-12); the update by Gauss-Jordan elimination
 * with partial pivoting; stop once max_s |dY_s| <= newton_tol * rho.  rho, the momentum and
 * E stay fixed (the source has no momentum or energy part and sum_s omega_s = 0); the
 * temperature of an iterate follows from the fixed internal energy E - |rho u|^2 / (2 rho).
 * U and Uout are device pointers of dg_state_size() doubles; they may be equal (in place)
 * but must not otherwise overlap.  A node still unconverged after newton_max_it updates
 * keeps its last iterate and makes dg_check() return DG_ECONVERGENCE.  Two-temperature
 * contexts: the unknowns are (Y, E_v) and the source is the full vector of Eq. src_vector
 * (omega_s at the controlling temperatures; E_v row Q_T-v + sum omega_s e_v,s(T_v)); T follows
 * from the fixed internal energy less E_v, T_v from E_v (by Newton's method inside each
 * evaluation); the Jacobian is (ns+1)^2; the step is also halved while T_v leaves
 * [T_v/2, 2 T_v]; convergence also needs |dE_v| <= newton_tol * (E - |rho u|^2/(2 rho)).
 * Asynchronous. */
DG_API dg_status dg_source_step(dg_ctx* ctx, const double* U, double h, double* Uout);

/* Hennemann-Gassner blending coefficients of every element for the state U (device, SoA as
 * everywhere), into alpha_raw and alpha (device arrays of the total element count, instances
 * concatenated; either may be NULL).  Per element: the field rho p at its nodes, its
 * orthonormal tensor-Legendre modes m, the smoothness
 *   E = max(E_high^(N) / E_tot^(N), E_high^(N-1) / E_tot^(N-1))
 * (E_tot^(K): energy of the modes with max index <= K; E_high^(K): with max index = K), then
 *   alpha_raw = min(alpha_max, sigmoid), sigmoid = 1 / (1 + exp(-(s/T)(E - T))), cut to 0 below
 * alpha_min, T = 0.5 * 10^(-1.8 (N+1)^(1/4)); alpha = max of alpha_raw over the element and its
 * face neighbours.  These are the coefficients every shock-captured stage computes from its
 * input state.  DG_EUNSUPPORTED unless shock capturing is on.  Asynchronous. */
DG_API dg_status dg_shock_alpha(dg_ctx* ctx, const double* U, double* alpha_raw, double* alpha);

/* Newton updates taken by all nodes in the implicit source substeps (dg_source_step and the
 * split steps of dg_rk_step) since the previous call, into *count (host); resets the count.
 * The work of a substep is proportional to it (NS + 1 evaluations of the source per update).
 * Synchronizes the stream. */
DG_API dg_status dg_newton_updates(dg_ctx* ctx, int64_t* count);

/* Element-wise device evaluation of n doubles x into y (device pointers), for testing the
 * library's own math routines against CUDA's: kind 0 the table-driven exp of the reaction
 * rates (Tang's method, 64-entry table), 1 the Newton-refined reciprocal, 2 CUDA's exp,
 * 3 CUDA's correctly rounded 1/x.  cuda_stream is a cudaStream_t (NULL = legacy default);
 * asynchronous.  Needs no context. */
DG_API dg_status dg_math_fn(int kind, int64_t n, const double* x, double* y, void* cuda_stream);

/* Measured throughput of one arithmetic instruction class on the current device, for the
 * rooflines of the stage kernels (no counterpart in the paper: a measurement utility).
 * kind: 0 FP64 fused multiply-add, 1 FP64 add, 2 FP32 fused multiply-add, 3 packed FP32x2
 * fused multiply-add (both lanes counted), 4 FP32 approximate reciprocal, 5 FP32 add.
 * *ops_per_s receives thread-level operations per second: independent dependency chains on
 * 8 CTAs of 256 threads per SM, best of three launches timed with CUDA events after a
 * warm-up launch, on the legacy default stream.  Synchronizes the device; no clock or other
 * device setting is changed.  DG_EINVAL for an unknown kind. */
DG_API dg_status dg_alu_rate(int kind, double* ops_per_s);

/* Message of the last error on this context (static string if ctx is NULL). */
DG_API const char* dg_last_error(const dg_ctx* ctx);

/* Release everything the context owns.  Safe on NULL. */
DG_API void dg_free(dg_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* DGSEM_H */
