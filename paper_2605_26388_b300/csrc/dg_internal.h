// dg_internal.h -- declarations shared by the C-ABI layer (dg_api.cu) and the kernel
// translation unit (dg_kernels.cu).  Not part of the public interface.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/dgsem.h"

namespace dg {

constexpr int kMaxN = 7;         // largest polynomial degree with compiled kernels (2D); 3D: 5
constexpr int kMaxBatchedN = 5;  // largest degree of the batched kernel

// One mesh instance as the kernels see it.
struct InstArgs {
  long long base;      // node offset of this instance in each variable's slab
  int nel[3];          // elements per direction (1 in unused directions)
  int n_elem;
  int N;
  double s[3];         // 2/dx_l
  float sf[3];
  double lift;         // 1 / w_0 (= 1 / w_N) of the GLL rule
  float liftf;
  int nonper;          // 1: some direction is not periodic
  int bc[6];           // boundary type per domain face (0: periodic)
  double bcs[6][5];    // prescribed boundary states (conserved, FP64)
};

// Launch-wide scalars in one precision, precomputed on the host so that no thread converts
// a double parameter to float (that conversion issues more slowly than an FP64 FMA on
// sm_103a) or evaluates a double comparison of a uniform flag.
template <class R>
struct ScalarsT {
  R gamma, gm1, igm1, p_ref, cbdt, abdt;
  R hgm1;                // (gamma - 1) / 2
  R margin_e, margin_0;  // positivity margin 2^-18 ((gamma - 1)|E| + |p_ref|) = margin_e |E| + margin_0
};
// Fill both precisions of the launch scalars (host).
inline void fill_scalars(ScalarsT<double>& d, ScalarsT<float>& f, double gamma, double p_ref, double cbdt,
                         double abdt) {
  const double gm1 = gamma - 1.0, s = 1.0 / 262144.0;  // 2^-18
  d.gamma = gamma;
  d.gm1 = gm1;
  d.igm1 = 1.0 / gm1;
  d.p_ref = p_ref;
  d.cbdt = cbdt;
  d.abdt = abdt;
  d.hgm1 = 0.5 * gm1;
  d.margin_e = s * gm1;
  d.margin_0 = s * (p_ref < 0.0 ? -p_ref : p_ref);
  f.gamma = (float)gamma;
  f.gm1 = (float)gamma - 1.0f;
  f.igm1 = 1.0f / f.gm1;
  f.p_ref = (float)p_ref;
  f.cbdt = (float)cbdt;
  f.abdt = (float)abdt;
  f.hgm1 = (float)d.hgm1;
  f.margin_e = (float)d.margin_e;
  f.margin_0 = (float)d.margin_0;
}

// Arguments of one fused stage launch (passed by value).
struct StageArgs {
  const double* U;     // input state U^(k-1) (or the residual's input)
  const double* Un;    // U^n (stages 2 and 3), else unused
  double* out;         // U^(k) (mode 1) or L(U) (mode 0)
  unsigned* err;       // device error word (bit 0 non-finite, bit 1 non-positive)
  unsigned* work;      // [2] work counters of a persistent launch (zero between launches), or null
  long long stride;    // per-variable stride of the SoA state (total nodes)
  double gamma;
  double ca, cb, dt;   // U^(k) = ca Un + cb U^(k-1) + (beta dt) L, beta dt in pd/pf.cbdt
  // optional second output of a stage update (the running sum of the last SSP-RK54 stage):
  // acc = acc_a acc + acc_b U^(k-1) + (acc_beta dt) L, acc_beta dt in pd/pf.abdt; null: none
  double* acc;
  double acc_a, acc_b;
  int mode;            // 0: out = L(U); 1: RK stage update
  int surface;         // DG_SURF_*
  int weak;            // 1: weak-form volume operator (surface lifts F* only)
  double rho_floor, p_floor;
  double p_ref;        // constant subtracted from the pressure in the momentum flux
  ScalarsT<double> pd;
  ScalarsT<float> pf;
  int need_un;         // mode == 1 and ca != 0
  int floor_on;        // rho_floor > 0 or p_floor > 0
  // shock capturing (mode 1): elements with alpha[e] > 0 write their DG residual to ldg and
  // leave the update to the blending launch; null alpha: no shock capturing
  const double* alpha; // per element of the instance
  double* ldg;         // state-shaped side buffer
  // single-instance launch
  InstArgs inst;
  double Dv[(kMaxN + 1) * (kMaxN + 1)];  // volume operator, row-major (N+1)^2
  // batched launch: work items (instance, element group), one volume operator per degree
  const InstArgs* insts;
  const int2* items;
  int n_items;
  const double* dv_table;  // [kMaxN + 1][(kMaxN + 1)^2]
};

// Arguments of the adjoint (vector-Jacobian product) launch over one instance.
//   mode 0:  out += w                                   (w = (dL/dU)^T lam)
//   mode 1:  out  = bcoef (lam + dt w) [+ accin];  accupd (=|+=) acoef lam
// gpart[cta] receives gw x that CTA's share of lam . dL/dgamma.
struct VjpArgs {
  const double* U;
  const double* lam;
  double* out;
  const double* accin;
  double* accupd;
  int acc_init;
  double* gpart;
  long long stride;
  InstArgs inst;
  double Dv[(kMaxN + 1) * (kMaxN + 1)];
  double gamma, dt, bcoef, acoef, gw;
  int mode, weak;
};

// y = sum_j c[j] x[j] over n doubles (m <= 5 terms; y may not alias any x): the reverse
// Shu-Osher combinations of the adjoint step.
struct CombineArgs {
  double* y;
  const double* x[5];
  double c[5];
  long long n;
  int m;
};
cudaError_t launch_combine(const CombineArgs& a, cudaStream_t s);

// Hennemann-Gassner shock capturing over one instance (Sec. 3.1.1 "Shock Indicator and
// Smoothing", Eq. vol_blend): indicator -> alpha_raw, neighbourhood maximum -> alpha and the
// list of elements with alpha > 0, then (after the stage launch) the sub-cell FV residual,
// the blend with the DG residual and the stage update of the listed elements.
struct ShockArgs {
  const double* U;       // stage input state
  const double* Un;      // X of the update (need_un)
  double* out;           // stage output (mode 1) or L (mode 0)
  const double* ldg;     // DG residual of the listed elements (mode 1: side buffer; mode 0: out)
  double* acc;           // optional running sum (see StageArgs)
  double acc_a, acc_b, acc_bdt;
  unsigned* err;
  long long stride;
  InstArgs inst;
  int mode, need_un, surface, floor_on;
  double ca, cb, bdt;
  double gamma, rho_floor, p_floor;
  ScalarsT<double> pd;
  ScalarsT<float> pf;
  double iw[kMaxN + 1];  // 1 / w_i of the GLL rule
  float iwf[kMaxN + 1];
  double Vinv[(kMaxN + 1) * (kMaxN + 1)];  // nodal -> orthonormal Legendre modes
  double thr, sharp, alpha_min, alpha_max;   // threshold T, steepness s, clipping bounds
  double emin;           // the smoothness below which the sigmoid is under alpha_min
  double* alpha_raw;     // per element of the instance
  double* alpha;
  int* list;             // elements with alpha > 0 ...
  int* count;            // ... and their number (device)
};
// The three shock-capturing launches; have_shock(dim, N) says whether they exist.
bool have_shock(int dim, int N);
cudaError_t launch_shock_indicator(int dim, int N, const ShockArgs& a, cudaStream_t s);
cudaError_t launch_shock_blend(int dim, int N, int fp32, const ShockArgs& a, cudaStream_t s);

// Launch the adjoint of the residual for one instance, then add the weighted gamma
// contribution (a deterministic sum of the per-CTA partials) to *gacc (device).
// sch: 0 the strong or weak volume form with the Rusanov flux; bit 0 the two-point form,
// bit 1 the HLLC flux (periodic meshes)
cudaError_t launch_rhs_vjp(int dim, int N, int fp32, int sch, const VjpArgs& a, double* gacc, cudaStream_t s);
// the launch of schemes 1..3 (dg_adjoint_ec.cu); *blocks receives the grid size
cudaError_t launch_vjp_ec(int sch, int dim, int N, int fp32, const VjpArgs& a, cudaStream_t s, int* blocks);
// CTAs the adjoint launch uses for an instance (size of the gpart scratch).
int vjp_blocks(int dim, int N, long long n_elem);

// Batched-launch tuning choices (picked by the autotuner).
struct BatchConfig {
  int group_scale;     // elements per work item = group scale x the kernel's base group: 1 or 2
                       // for every degree, or DG_GROUPS_PER_DEGREE | mask (bit N: degree N
                       // uses 2)
  int ctas_per_sm;     // 0 = as many as fit
  int order;           // 0 = heaviest items first, 1 = instance order
};
// The group scale of degree N under configuration b.
inline int group_scale_of(const BatchConfig& b, int N) {
  if (b.group_scale & DG_GROUPS_PER_DEGREE) return ((b.group_scale >> N) & 1) ? 2 : 1;
  return b.group_scale;
}

// Launch the fused Euler stage kernel for one instance.  Returns a CUDA error code.
cudaError_t launch_euler_stage(int dim, int N, int ec, int fp32, const StageArgs& a,
                               cudaStream_t s);

// Set the kernel attributes (dynamic shared memory) of one stage kernel; call before the
// first launch and outside stream capture.
cudaError_t prepare_euler_stage(int dim, int N, int ec, int fp32);

// A grid-stride kernel's CTA count cap: 16 CTAs per SM of the current device.
int grid_cap();

// Decode a signal-speed reduction code (see speed_bits in dg_device.cuh): 0 and *lam the
// speed; 1 a node with a non-finite value; 2 a node with rho <= 0 or p <= 0.
inline int decode_speed(unsigned long long bits, double* lam) {
  if (bits >= 0x7ff8000000000000ull) return 1;
  if (bits >= 0x7ff0000000000000ull) return 2;
  __builtin_memcpy(lam, &bits, sizeof(*lam));
  return 0;
}

// Largest signal speed |u| + a over the nodes of one instance, atomically max-ed into
// *lam_bits as a reduction code (speed_bits).
cudaError_t launch_max_speed(int dim, const double* U, long long stride, long long base,
                             long long n_nodes, double gamma, unsigned long long* lam_bits,
                             cudaStream_t s);

// Evaluate a device two-point flux for n AoS state pairs.
cudaError_t launch_two_point(int dim, int fp32, int kind, int l, int n, double gamma, double p_ref,
                             const double* uL, const double* uR, double* F, cudaStream_t s);

// Batched persistent launch over the work items in a.items (all instances of one dim).
cudaError_t launch_euler_stage_batched(int dim, int ec, int fp32, int group_scale, int ctas_per_sm,
                                       const StageArgs& a, cudaStream_t s);
// Elements per work item of the batched kernel for degree N (dim, group_scale).
int batched_group(int dim, int N, int group_scale);
// Threads per CTA and dynamic shared memory of the batched kernel.
cudaError_t prepare_euler_stage_batched(int dim, int ec, int fp32, int group_scale);

// Curved meshes: one CTA per element; met = the metric terms [DIM*DIM][nodes] (Ja^l_d at
// index l*DIM+d) then 1/J [nodes], at the state's node stride; a->Dv holds the plain D.
// a == null sets the kernel attributes (before the first launch, outside capture).
bool have_curved(int dim, int N);
cudaError_t launch_curved(int dim, int N, int ec, int fp32, const StageArgs* a, const double* met,
                          cudaStream_t s);

// Whether (dim, N) has compiled kernels.
bool have_kernels(int dim, int N);

// ---------------------------------------------------------------------------------------
// Reacting Navier-Stokes (3D): species data and reactions as the kernels read them.
// ---------------------------------------------------------------------------------------
constexpr int kMaxSpecies = 8;
constexpr int kMaxReactions = 32;
constexpr int kMaxReactingN = 4;

struct RxnDev {
  double lnA, b, Ta;
  double kc[5];                // ln K_c = kc0 / Z + kc1 + kc2 ln Z + kc3 Z + kc4 Z^2
  double coef[kMaxSpecies];    // W_s * 1e6 * (nu''_s - nu'_s): mol/(cm^3 s) -> kg/(m^3 s)
  int f[3], bk[3];             // species of the forward / backward concentration products;
                               //   index n_species stands for the factor 1
  int ta;                      // two-temperature: 1 -- rates at T_a = sqrt(T Tv), 0 -- at T
  int pad;
};

struct MechDev {
  int ns, nr;
  int pad[2];
  double R[kMaxSpecies], cv[kMaxSpecies], h0[kMaxSpecies];
  double scale[kMaxSpecies];   // 1e-6 / W_s: rho_s (kg/m^3) -> [X_s] (mol/cm^3)
  double theta[kMaxSpecies];   // two-temperature: vibrational temperature (0: atom)
  // two-temperature, Millikan-White: 1 / tau_sr = (p / 1 atm) exp(mwC[s][r] - mwA[s][r] T^-1/3)
  double mwA[kMaxSpecies][kMaxSpecies], mwC[kMaxSpecies][kMaxSpecies];
  double exp2tab[64];          // 2^(j/64), j = 0..63, for the table-driven exp of the rates
  RxnDev rx[kMaxReactions];
};

// Boundary conditions of one reacting / Navier-Stokes instance (host-filled).
struct ReactBC {
  int nonper;            // 1: some direction carries boundary conditions
  int bc[6];             // boundary type per domain face (0: periodic)
  double bcu[6][12];     // prescribed conserved state U_b (inflow, Dirichlet)
  double bcw[6][7];      // (u, v, w, T, p - p_ref, a, T_v) of U_b (inflow, Dirichlet), or
                         // (0, 0, 0, T_wall, 0, 0, T_wall) (isothermal wall); T_v = T for
                         // one temperature
};

// Arguments of the two reacting launches of one stage over one instance.
struct ReactArgs {
  const double* U;     // input state (or the residual's input)
  const double* Un;    // U^n (stages 2 and 3)
  double* out;         // stage output (mode 1) or L(U) (mode 0)
  unsigned* err;       // device error word
  void* fb;            // face buffer of this instance (flux type): [elem][face][4][(N+1)^2]
  const void* pin;     // primitive cache of U (flux type, 7 rows at `stride`) ...
  const double* tin;   //   ... and its FP64 temperature
  void* pout;          // primitive cache of the stage output (mode 1; null: not written)
  double* tout;
  const MechDev* mech; // device copy of the mechanism
  long long stride;    // per-variable stride of the SoA state
  long long base;      // node offset of the instance
  int nel[3];
  int n_elem;
  int mode;            // 0: out = L(U); 1: stage update
  int need_un;
  int src;             // 1: the Arrhenius source is part of L (0 under the Strang split)
  double s[3];         // 2 / dx_l
  double lift;         // 1 / w_0 = 1 / w_N
  double ca, cb, cbdt; // out = ca Un + cb U + cbdt L
  double* acc;         // optional second output: acc = acc_a acc + acc_b U + acc_bdt L
  double acc_a, acc_b, acc_bdt;
  double mu, kfac;     // viscosity; mu / Pr (conductivity = kfac * c_p)
  double p_ref;        // constant subtracted from the pressure in the momentum flux
  double ln1e4;        // ln 10^4 (for ln Z = ln 10^4 - ln T)
  float sf[3], liftf, muf, kfacf, p_reff;  // the same scalars for the FP32 flux arithmetic
  double D[(kMaxReactingN + 1) * (kMaxReactingN + 1)];
  ReactBC bnd;          // boundary conditions of the instance
  // curved instance (periodic): the metric terms Ja^l_d at row l*3+d, then 1/J at row 9, at
  // the state's node stride (s = 1: the 2/dx_l of a Cartesian element are in Ja^l); null:
  // Cartesian
  const double* met;
};

// Whether the reacting kernels exist for degree N, n_species and the temperature model
// (tt = 1: two-temperature).
bool have_reacting(int N, int ns, int tt);
// Kernel attributes (dynamic shared memory); call before the first launch, outside capture.
cudaError_t prepare_reacting(int N, int ns, int tt, int fp32);
// One stage (or residual) over one instance: the BR1 face pass, then the fused stage; fp32
// selects FP32 flux arithmetic (mixture, source and update stay FP64).
cudaError_t launch_reacting(int N, int ns, int tt, int fp32, const ReactArgs& a, cudaStream_t s);
// Rows of the primitive cache (flux type): u, v, w, T, p - p_ref, a, c_p; two-temperature:
// u, v, w, T, T_v, p - p_ref, a, c_p, c_v,v.  FP64 rows: T (and T_v).
inline int react_cache_rows(int tt) { return tt ? 9 : 7; }
inline int react_t64_rows(int tt) { return tt ? 2 : 1; }
// Primitive cache of the nodes [base, base + n_nodes) of a state; flags rho <= 0 or T <= 0
// (bit 1) and an unconverged T_v iteration (bit 2) in *err.
cudaError_t launch_react_prims(int ns, int tt, int fp32, const double* U, long long stride, long long base,
                               long long n_nodes, const MechDev* mech, double p_ref, void* P, double* T64,
                               unsigned* err, cudaStream_t s);
// Implicit source substep (Strang split) over the nodes [base, base + n) of a state.
struct SourceArgs {
  const double* U;     // input state
  double* out;         // output state (may equal U: each node is read, then written)
  unsigned* err;       // device error word (bit 2: a node's Newton iteration did not converge)
  const MechDev* mech;
  void* pout;          // primitive cache of the output (flux type; null: not written)
  double* tout;
  const double* tin;   // two-temperature: the FP64 cache rows of the input (T, T_v) or null;
                       //   its T_v starts the node's T_v iterations
  long long stride, base, n;
  double h;            // substep length
  double tol;          // stop when max |dY| <= tol * rho
  double p_ref, ln1e4;
  int max_it;          // Newton updates per node at most
  int copy_rest;       // 1: also copy momentum and energy (out != U)
  unsigned long long* updates;  // device counter: Newton updates taken, summed over nodes
};
cudaError_t launch_source_implicit(int ns, int tt, int fp32, const SourceArgs& a, cudaStream_t s);

// Zhang-Shu limiter of the partial densities of one instance's elements, in place, with the
// primitive cache of the changed nodes rewritten (pout/tout, when not null).
struct LimiterArgs {
  double* U;           // state (SoA), limited in place
  void* pout;          // its primitive cache (flux type) or null
  double* tout;
  unsigned* err;
  const MechDev* mech;
  long long stride, base;
  int n_elem, np;      // elements of the instance, nodes per element
  double p_ref;
  double wq[(kMaxReactingN + 1) * (kMaxReactingN + 1) * (kMaxReactingN + 1)];  // GLL weights / sum
};
cudaError_t launch_species_limiter(int ns, int tt, int fp32, const LimiterArgs& a, cudaStream_t s);

// Element-wise evaluation of a device math routine for the tests: kind 0 the library's
// table-driven exp, 1 its Newton reciprocal, 2 CUDA's exp, 3 CUDA's 1/x.
struct MathArgs {
  const double* x;
  double* y;
  long long n;
  int kind;
  double tab[64];      // 2^(j/64)
};
cudaError_t launch_math_fn(const MathArgs& a, cudaStream_t s);

// Largest |u| + a (frozen mixture sound speed) and largest 1/rho over one instance,
// atomically max-ed into out2[0] and out2[1] (bit patterns of non-negative doubles).
cudaError_t launch_max_speed_mix(int ns, int tt, const double* U, long long stride, long long base,
                                 long long n_nodes, const MechDev* mech,
                                 unsigned long long* out2, cudaStream_t s);

}  // namespace dg
