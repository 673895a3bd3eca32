"""ORACLE -- test infrastructure only, never part of the product path.

A plain, slow FP64 CPU implementation of the DGSEM residual, numerical fluxes, SSP-RK33
and SSP-RK54 steps and time-step bound of the paper's method (arXiv 2605.26388, Sec. 2,
Sec. 3.1.1, App. A, App. B), and of the reacting Navier-Stokes residual (BR1 viscous terms,
Sec. 3.1.2; Arrhenius source, Sec. 3.1.3 and App. C) with its implicit Strang-split source
substep (Sec. 3.1.3), and the Hennemann-Gassner DG/FV shock capturing of the Euler residual
(Sec. 3.1.1, Eq. vol_blend; App. A), written in C++ (``dg_oracle.cpp``) and loaded here with ctypes.  It
shares no code with the CUDA library.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.

Parity status of each function is stated in its docstring ("pinned by ..." or
"parity unpinned").
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dg_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

# enumerations of the oracle's own problem description (dg_oracle.cpp)
EULER, NAVIER_STOKES, NS_REACTING = 0, 1, 2
VOL_STRONG, VOL_WEAK, VOL_EC, VOL_CENTRAL = 0, 1, 2, 3
SURF_RUSANOV, SURF_HLLC, SURF_HLL, SURF_EC, SURF_CENTRAL = 0, 1, 2, 3, 4
BC_PERIODIC, BC_SLIP_WALL, BC_INFLOW, BC_OUTFLOW, BC_DIRICHLET = 0, 1, 2, 3, 4
BC_NOSLIP_ADIABATIC, BC_NOSLIP_ISOTHERMAL = 5, 6  # NS_REACTING only


def build(force: bool = False) -> str:
    """Compile the oracle shared library with g++ (-O2, OpenMP over elements)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-std=c++17", "-O2", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", _LIB]
        subprocess.run(cmd, check=True)
    return _LIB


class _Mech(C.Structure):
    _fields_ = [
        ("n_species", C.c_int), ("n_reactions", C.c_int),
        ("W", C.c_double * 8), ("R", C.c_double * 8), ("cv", C.c_double * 8), ("h0", C.c_double * 8),
        ("lnA", C.c_double * 32), ("b", C.c_double * 32), ("Ta", C.c_double * 32),
        ("kc", (C.c_double * 5) * 32), ("nu_f", (C.c_int * 8) * 32), ("nu_b", (C.c_int * 8) * 32),
        ("theta_v", C.c_double * 8), ("ta_mode", C.c_int * 32),
    ]


def mechanism(m: dict) -> _Mech:
    """Pack a mechanism dictionary (species data W, R, cv, h0 and, for the two-temperature
    model, theta_v; per-reaction lnA, b, Ta, kc, nu_f, nu_b and ta_mode) into the oracle's own
    structure."""
    c = _Mech()
    ns, nr = int(m["n_species"]), int(m["n_reactions"])
    c.n_species, c.n_reactions = ns, nr
    for s in range(ns):
        c.W[s], c.R[s], c.cv[s], c.h0[s] = m["W"][s], m["R"][s], m["cv"][s], m["h0"][s]
    for r in range(nr):
        c.lnA[r], c.b[r], c.Ta[r] = m["lnA"][r], m["b"][r], m["Ta"][r]
        for k in range(5):
            c.kc[r][k] = m["kc"][r][k]
        for s in range(ns):
            c.nu_f[r][s] = int(m["nu_f"][r][s])
            c.nu_b[r][s] = int(m["nu_b"][r][s])
        c.ta_mode[r] = int(m.get("ta_mode", [0] * nr)[r])
    for s in range(ns):
        c.theta_v[s] = float(m.get("theta_v", [0.0] * ns)[s])
    return c


class _Problem(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("N", C.c_int), ("nel", C.c_int * 3),
        ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("equations", C.c_int), ("volume", C.c_int), ("surface", C.c_int),
        ("gamma", C.c_double), ("mu", C.c_double), ("prandtl", C.c_double),
        ("rho_floor", C.c_double), ("p_floor", C.c_double),
        ("mech", C.POINTER(_Mech)), ("parts", C.c_int),
        ("shock", C.c_int), ("alpha_min", C.c_double), ("alpha_max", C.c_double),
        ("sharpness", C.c_double), ("bc", C.c_int * 6), ("bc_state", (C.c_double * 12) * 6),
        ("coords", C.POINTER(C.c_double)), ("two_temperature", C.c_int), ("species_limiter", C.c_int),
    ]


@dataclass
class Problem:
    """The oracle's description of one periodic Cartesian DGSEM problem."""
    dim: int
    N: int
    nel: tuple
    lo: tuple
    hi: tuple
    volume: int = VOL_STRONG
    surface: int = SURF_RUSANOV
    gamma: float = 1.4
    equations: int = EULER
    mu: float = 0.0
    prandtl: float = 0.72
    rho_floor: float = 0.0
    p_floor: float = 0.0
    mech: dict = None   # NS_REACTING: mechanism dictionary (species and reactions)
    parts: int = 0      # NS_REACTING: 1 inviscid, 2 viscous, 4 source; 0 = all
    shock: bool = False  # Euler: Hennemann-Gassner DG/FV blending
    alpha_min: float = 0.001
    alpha_max: float = 0.5
    sharpness: float = math.log(9999.0)
    bc: tuple = (0, 0, 0, 0, 0, 0)  # per domain face x-, x+, y-, y+, z-, z+; 0 = periodic
    bc_state: tuple = None          # per face: the exterior conserved state (INFLOW, DIRICHLET);
                                    # (T_wall,) for NOSLIP_ISOTHERMAL
    coords: np.ndarray = None       # node coordinates (dim, n_elem, n_nodes) of a curved mesh (reacting: periodic)
    two_temperature: bool = False   # NS_REACTING: E_v appended to the state
    species_limiter: bool = False   # NS_REACTING: Zhang-Shu limiter of rho_s after every RK stage

    @property
    def nvars(self) -> int:
        if self.equations == NS_REACTING:
            return int(self.mech["n_species"]) + self.dim + 1 + (1 if self.two_temperature else 0)
        return self.dim + 2

    @property
    def n_elem(self) -> int:
        n = 1
        for l in range(self.dim):
            n *= self.nel[l]
        return n

    @property
    def n_nodes(self) -> int:
        return (self.N + 1) ** self.dim

    @property
    def shape(self) -> tuple:
        return (self.nvars, self.n_elem, self.n_nodes)

    def _c(self) -> _Problem:
        nel = list(self.nel) + [1] * (3 - len(self.nel))
        lo = list(self.lo) + [0.0] * (3 - len(self.lo))
        hi = list(self.hi) + [1.0] * (3 - len(self.hi))
        p = _Problem(self.dim, self.N, (C.c_int * 3)(*nel), (C.c_double * 3)(*lo),
                     (C.c_double * 3)(*hi), self.equations, self.volume, self.surface,
                     self.gamma, self.mu, self.prandtl, self.rho_floor, self.p_floor)
        p.parts = self.parts
        p.two_temperature = 1 if self.two_temperature else 0
        p.species_limiter = 1 if self.species_limiter else 0
        p.shock = 1 if self.shock else 0
        p.alpha_min, p.alpha_max, p.sharpness = self.alpha_min, self.alpha_max, self.sharpness
        if self.coords is not None:
            p._coords_keep = np.ascontiguousarray(self.coords, dtype=np.float64)
            p.coords = p._coords_keep.ctypes.data_as(C.POINTER(C.c_double))
        for f in range(6):
            p.bc[f] = int(self.bc[f])
            if self.bc_state is not None and self.bc_state[f] is not None:
                for v, x in enumerate(self.bc_state[f]):
                    p.bc_state[f][v] = float(x)
        if self.mech is not None:
            p._mech_keep = mechanism(self.mech)  # kept alive with the structure
            p.mech = C.pointer(p._mech_keep)
        return p


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        pp = C.POINTER(_Problem)
        _lib.orc_gll.argtypes = [C.c_int, dp, dp]
        _lib.orc_dmat.argtypes = [C.c_int, dp]
        _lib.orc_log_mean.argtypes = [C.c_double, C.c_double]
        _lib.orc_log_mean.restype = C.c_double
        _lib.orc_point_flux.argtypes = [C.c_int, C.c_int, C.c_double, dp, dp]
        _lib.orc_two_point_flux.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, dp, dp, dp]
        _lib.orc_rhs.argtypes = [pp, dp, dp]
        _lib.orc_rhs_elements.argtypes = [pp, dp, C.POINTER(C.c_int), C.c_int, dp]
        _lib.orc_br1_gradients.argtypes = [pp, dp, C.POINTER(C.c_int), C.c_int, dp]
        _lib.orc_rhs_elements_given_gradient.argtypes = [pp, dp, dp, C.POINTER(C.c_int), C.c_int, dp]
        _lib.orc_rk3_stage.argtypes = [pp, C.c_int, dp, dp, C.c_double, dp]
        _lib.orc_rk3.argtypes = [pp, dp, C.c_double, C.c_int]
        _lib.orc_max_dt.argtypes = [pp, dp, C.c_double, dp]
        _lib.orc_rhs_jvp.argtypes = [pp, dp, dp, C.c_double, dp, dp]
        _lib.orc_rhs_vjp_brute.argtypes = [pp, dp, dp, dp, dp]
        _lib.orc_log_mean_jvp.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, dp, dp]
        _lib.orc_rollout_grad.argtypes = [pp, dp, dp, dp, C.c_double, C.c_int, dp, dp]
        _lib.orc_arrhenius.argtypes = [C.POINTER(_Mech), C.c_int, C.c_double, dp, dp]
        _lib.orc_chem_source.argtypes = [pp, dp, dp]
        _lib.orc_mixture.argtypes = [pp, dp, dp, dp, dp]
        _lib.orc_species_limiter.argtypes = [pp, dp]
        _lib.orc_positivity_floor.argtypes = [pp, dp]
        _lib.orc_relaxation_time.argtypes = [C.POINTER(_Mech), C.c_int, dp, C.c_double, C.c_double, dp]
        ip = C.POINTER(C.c_int)
        _lib.orc_shock_alpha.argtypes = [pp, dp, dp, dp]
        _lib.orc_fv_residual.argtypes = [pp, dp, dp]
        _lib.orc_modes.argtypes = [pp, dp, dp]
        _lib.orc_metrics.argtypes = [pp, dp, dp]
        _lib.orc_ssp_table.argtypes = [C.c_int, dp, dp, ip, dp]
        _lib.orc_ssp_steps.argtypes = [pp, C.c_int, dp, C.c_double, C.c_int]
        _lib.orc_source_implicit.argtypes = [pp, dp, C.c_double, C.c_int, C.c_double, ip]
        _lib.orc_strang_steps.argtypes = [pp, C.c_int, dp, C.c_double, C.c_int, C.c_int, C.c_double, ip]
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} rejected the problem (code {rc})")


def gll(N: int):
    """GLL nodes and weights (Sec. 3.1.1). Pinned by closed forms for N <= 4 and by
    exact quadrature of monomials (tests/test_oracle_operators.py)."""
    x = np.zeros(N + 1)
    w = np.zeros(N + 1)
    _check(lib().orc_gll(N, _ptr(x), _ptr(w)), "gll")
    return x, w


def dmat(N: int) -> np.ndarray:
    """GLL differentiation matrix D_ij = l_j'(x_i). Pinned by polynomial exactness, the
    SBP identity and D_00 = -N(N+1)/4."""
    D = np.zeros((N + 1) * (N + 1))
    _check(lib().orc_dmat(N, _ptr(D)), "dmat")
    return D.reshape(N + 1, N + 1)


def log_mean(a: float, b: float) -> float:
    """Logarithmic mean (a-b)/(ln a - ln b) (App. A). Pinned by a mpmath-free
    high-precision series check and by its closed-form special cases."""
    return lib().orc_log_mean(a, b)


def point_flux(dim: int, l: int, gamma: float, u) -> np.ndarray:
    """Cartesian Euler flux F^l(U) (Sec. 2)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    F = np.zeros(dim + 2)
    lib().orc_point_flux(dim, l, gamma, _ptr(u), _ptr(F))
    return F


def two_point_flux(kind: int, dim: int, l: int, gamma: float, uL, uR) -> np.ndarray:
    """Numerical two-point flux: kind = -1 Ranocha EC volume flux, else a SURF_* kind."""
    uL = np.ascontiguousarray(uL, dtype=np.float64)
    uR = np.ascontiguousarray(uR, dtype=np.float64)
    F = np.zeros(dim + 2)
    lib().orc_two_point_flux(kind, dim, l, gamma, _ptr(uL), _ptr(uR), _ptr(F))
    return F


def rhs(P: Problem, U: np.ndarray) -> np.ndarray:
    """Semi-discrete residual L(U) (Eqs. vol_weak / vol_split / surf_int). State layout
    U[var, elem, node], elements x-fastest, nodes i-fastest."""
    U = np.ascontiguousarray(U, dtype=np.float64).reshape(P.shape)
    dU = np.zeros_like(U)
    c = P._c()
    _check(lib().orc_rhs(C.byref(c), _ptr(U), _ptr(dU)), "rhs")
    return dU


def rhs_elements(P: Problem, U: np.ndarray, elems) -> np.ndarray:
    """L(U) on the listed elements only; returns an array (n_vars, len(elems), n_nodes)."""
    U = np.ascontiguousarray(U, dtype=np.float64).reshape(P.shape)
    el = np.ascontiguousarray(elems, dtype=np.int32)
    dU = np.zeros_like(U)
    c = P._c()
    _check(lib().orc_rhs_elements(C.byref(c), _ptr(U), el.ctypes.data_as(C.POINTER(C.c_int)), len(el),
                                  _ptr(dU)), "rhs_elements")
    return dU[:, el, :]


def br1_gradients(P: Problem, U: np.ndarray, elems, G=None) -> np.ndarray:
    """BR1 gradients (Sec. 3.1.2) of W = (u, v, w, T, T_v) on the listed elements, written
    into G of shape (n_elem, n_nodes, 5, 3) (a new zero array unless given); other elements'
    rows are left as they are."""
    U = np.ascontiguousarray(U, dtype=np.float64).reshape(P.shape)
    el = np.ascontiguousarray(elems, dtype=np.int32)
    if G is None:
        G = np.zeros((P.n_elem, P.n_nodes, 5, 3))
    assert G.flags.c_contiguous and G.shape == (P.n_elem, P.n_nodes, 5, 3)
    c = P._c()
    _check(lib().orc_br1_gradients(C.byref(c), _ptr(U), el.ctypes.data_as(C.POINTER(C.c_int)), len(el),
                                   _ptr(G)), "br1_gradients")
    return G


def rhs_elements_given_gradient(P: Problem, U: np.ndarray, G: np.ndarray, elems) -> np.ndarray:
    """The Navier-Stokes residual on the listed elements from U and the BR1 gradients G
    (shape (n_elem, n_nodes, 5, 3)); returns (n_vars, len(elems), n_nodes)."""
    U = np.ascontiguousarray(U, dtype=np.float64).reshape(P.shape)
    G = np.ascontiguousarray(G, dtype=np.float64)
    el = np.ascontiguousarray(elems, dtype=np.int32)
    dU = np.zeros_like(U)
    c = P._c()
    _check(lib().orc_rhs_elements_given_gradient(C.byref(c), _ptr(U), _ptr(G),
                                                 el.ctypes.data_as(C.POINTER(C.c_int)), len(el), _ptr(dU)),
           "rhs_elements_given_gradient")
    return dU[:, el, :]


def rk3_stage(P: Problem, stage: int, Un: np.ndarray, Uprev: np.ndarray, dt: float):
    """One Shu-Osher SSP-RK3 stage (App. B)."""
    Un = np.ascontiguousarray(Un, dtype=np.float64).reshape(P.shape)
    Uprev = np.ascontiguousarray(Uprev, dtype=np.float64).reshape(P.shape)
    out = np.zeros_like(Un)
    c = P._c()
    _check(lib().orc_rk3_stage(C.byref(c), stage, _ptr(Un), _ptr(Uprev), dt, _ptr(out)),
           "rk3_stage")
    return out


def rk3(P: Problem, U: np.ndarray, dt: float, n_steps: int) -> np.ndarray:
    """n_steps SSP-RK3 steps; returns the new state (the input is not modified)."""
    U = np.array(U, dtype=np.float64, order="C").reshape(P.shape)
    c = P._c()
    _check(lib().orc_rk3(C.byref(c), _ptr(U), dt, n_steps), "rk3")
    return U


def rhs_jvp(P: Problem, U: np.ndarray, V=None, gdot: float = 0.0):
    """(L(U), dL) with dL = (dL/dU) V + (dL/dgamma) gdot, by forward-mode dual numbers
    (strong, weak or two-point volume form; Rusanov, HLLC or EC surface flux; periodic
    Cartesian boxes).  Pinned by its value against rhs(), its derivative against central
    differences of rhs(), the log mean's closed-form derivative and, for the two-point form
    with the EC surface flux, the vanishing derivative of the entropy production."""
    U = np.ascontiguousarray(U, dtype=np.float64).reshape(P.shape)
    L = np.zeros_like(U)
    dL = np.zeros_like(U)
    Vp = None
    if V is not None:
        V = np.ascontiguousarray(V, dtype=np.float64).reshape(P.shape)
        Vp = _ptr(V)
    c = P._c()
    _check(lib().orc_rhs_jvp(C.byref(c), _ptr(U), Vp, gdot, _ptr(L), _ptr(dL)), "rhs_jvp")
    return L, dL


def log_mean_jvp(a: float, b: float, da: float, db: float):
    """(L, dL): the logarithmic mean of a, b (App. A) and its derivative along (da, db),
    as the dual-number residual evaluates them."""
    L, dL = np.zeros(1), np.zeros(1)
    _check(lib().orc_log_mean_jvp(a, b, da, db, _ptr(L), _ptr(dL)), "log_mean_jvp")
    return float(L[0]), float(dL[0])


def rhs_vjp_brute(P: Problem, U: np.ndarray, lam: np.ndarray):
    """((dL/dU)^T lam, lam . dL/dgamma) assembled from one JVP per unknown (tiny meshes)."""
    U = np.ascontiguousarray(U, dtype=np.float64).reshape(P.shape)
    lam = np.ascontiguousarray(lam, dtype=np.float64).reshape(P.shape)
    Ub = np.zeros_like(U)
    gb = np.zeros(1)
    c = P._c()
    _check(lib().orc_rhs_vjp_brute(C.byref(c), _ptr(U), _ptr(lam), _ptr(Ub), _ptr(gb)), "rhs_vjp_brute")
    return Ub, float(gb[0])


def max_dt(P: Problem, U: np.ndarray, cfl: float) -> float:
    """Convective time-step bound dt = cfl dx_min / ((2N+1) lambda_max) (Eq. dt_hyp)."""
    U = np.ascontiguousarray(U, dtype=np.float64).reshape(P.shape)
    out = np.zeros(1)
    c = P._c()
    _check(lib().orc_max_dt(C.byref(c), _ptr(U), cfl, _ptr(out)), "max_dt")
    return float(out[0])


def rollout_grad(P: Problem, U0: np.ndarray, target: np.ndarray, wq: np.ndarray, dt: float, n_steps: int):
    """Gradient of J = 1/2 sum wq (rho_final - target)^2 after n_steps SSP-RK3 steps from U0,
    with respect to U0 and gamma, by exact forward mode (one dual-number rollout per
    unknown; tiny meshes).  Built on the pinned dual-number residual."""
    U0 = np.ascontiguousarray(U0, dtype=np.float64).reshape(P.shape)
    target = np.ascontiguousarray(target, dtype=np.float64).reshape(P.shape[1:])
    wq = np.ascontiguousarray(wq, dtype=np.float64).reshape(P.shape[1:])
    g = np.zeros_like(U0)
    gg = C.c_double()
    c = P._c()
    _check(lib().orc_rollout_grad(C.byref(c), _ptr(U0), _ptr(target), _ptr(wq), dt, n_steps, _ptr(g),
                                  C.byref(gg)), "rollout_grad")
    return g, gg.value


def arrhenius(mech: dict, r: int, T: float):
    """Forward rate k_f = exp(lnA + b ln T - Ta/T) and equilibrium constant
    K_c = exp(a0/Z + a1 + a2 ln Z + a3 Z + a4 Z^2), Z = 1e4/T, of reaction r (Sec. 3.1.3,
    Eq. src_reaction_rate; the five-term K_c form is a reading). Pinned by a long-double
    evaluation and the hand-worked golden value in tests/golden/."""
    kf, Kc = C.c_double(), C.c_double()
    m = mechanism(mech)
    _check(lib().orc_arrhenius(C.byref(m), r, T, C.byref(kf), C.byref(Kc)), "arrhenius")
    return kf.value, Kc.value


def chem_source(P: Problem, u) -> np.ndarray:
    """Chemical source of one reacting node state (Sec. 3.1.3, Eq. src_omega). Pinned by
    mass and atom conservation, zero momentum/energy source, a zero net rate at a
    composition built to satisfy K_c, and a hand-worked single-reaction value."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    S = np.zeros(P.nvars)
    c = P._c()
    _check(lib().orc_chem_source(C.byref(c), _ptr(u), _ptr(S)), "chem_source")
    return S


def mixture(P: Problem, u):
    """Temperature and pressure of one reacting node state (calorically perfect species,
    Sec. 2 closure). Pinned by inverting the state constructor of the reacting workload."""
    T, p, _ = mixture_tt(P, u)
    return T, p


def mixture_tt(P: Problem, u):
    """(T, p, T_v) of one reacting node state; T_v = T in the single-temperature model.
    Pinned by inverting the two-temperature state constructor."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    T, p, Tv = C.c_double(), C.c_double(), C.c_double()
    c = P._c()
    _check(lib().orc_mixture(C.byref(c), _ptr(u), C.byref(T), C.byref(p), C.byref(Tv)), "mixture")
    return T.value, p.value, Tv.value


def species_limiter(P: Problem, U: np.ndarray) -> np.ndarray:
    """The Zhang-Shu limiter of the partial densities applied once to U (a copy is returned).
    Pinned by element means, the zero minimum, identity on non-negative states."""
    U = np.array(U, dtype=np.float64, order="C").reshape(P.shape)
    c = P._c()
    _check(lib().orc_species_limiter(C.byref(c), _ptr(U)), "species_limiter")
    return U


def positivity_floor(P: Problem, U: np.ndarray) -> np.ndarray:
    """The Euler positivity floor applied once to U (a copy is returned): rho raised to
    rho_floor, then E reset so that p = p_floor where p < p_floor (momentum kept).  Pinned by
    the exact floor values, untouched unfloored nodes and idempotence."""
    U = np.array(U, dtype=np.float64, order="C").reshape(P.shape)
    c = P._c()
    _check(lib().orc_positivity_floor(C.byref(c), _ptr(U)), "positivity_floor")
    return U


def relaxation_time(mech: dict, s: int, X, T: float, p: float) -> float:
    """Vibrational relaxation time (s) of molecular species s, Millikan-White with Park's
    correction (Sec. 3.1.3), for mole fractions X at temperature T (K) and pressure p (Pa)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    m = mechanism(mech)
    tau = C.c_double()
    _check(lib().orc_relaxation_time(C.byref(m), s, _ptr(X), T, p, C.byref(tau)), "relaxation_time")
    return tau.value


SSPRK33, SSPRK54 = 3, 54
NEWTON_MAX_IT, NEWTON_TOL = 40, 1e-12


def ssp_table(scheme: int):
    """(alpha, beta, s, c): the Shu-Osher table of SSP-RK33 (Shu-Osher 1988) or SSP-RK54
    (Spiteri-Ruuth 2002) as (s, s) arrays (row i = stage i+1), the stage count and the SSP
    coefficient min alpha/beta (App. B).  Pinned by the order conditions of the Butcher form
    (order 3 / 4), the convexity rules and the paper's c ~ 1.508."""
    a = np.zeros(25)
    b = np.zeros(25)
    s, c = C.c_int(), C.c_double()
    _check(lib().orc_ssp_table(scheme, _ptr(a), _ptr(b), C.byref(s), C.byref(c)), "ssp_table")
    n = s.value
    return a.reshape(5, 5)[:n, :n], b.reshape(5, 5)[:n, :n], n, c.value


def ssp_steps(P: Problem, scheme: int, U: np.ndarray, dt: float, n_steps: int) -> np.ndarray:
    """n_steps steps of SSP-RK33 or SSP-RK54 by the Shu-Osher sums (App. B); returns the new
    state.  Pinned by the temporal convergence order on a smooth problem and, for RK33, by
    agreement with the separately written rk3()."""
    U = np.array(U, dtype=np.float64, order="C").reshape(P.shape)
    c = P._c()
    _check(lib().orc_ssp_steps(C.byref(c), scheme, _ptr(U), dt, n_steps), "ssp_steps")
    return U


def source_implicit(P: Problem, U: np.ndarray, h: float, max_it: int = NEWTON_MAX_IT,
                    tol: float = NEWTON_TOL):
    """One backward-Euler substep of the chemical source of length h at every node (Sec.
    3.1.3, Eq. source_residual; Newton with a forward-difference Jacobian and Gauss-Jordan
    solves).  Returns (new state, largest Newton count; -1 = a node did not converge).
    Pinned by closed-form backward-Euler solutions of first- and second-order reactions, a
    bisection root of a temperature-coupled reaction, the O(h^2) agreement with an explicit
    Euler step, and mass and atom conservation."""
    U = np.array(U, dtype=np.float64, order="C").reshape(P.shape)
    it = C.c_int()
    c = P._c()
    _check(lib().orc_source_implicit(C.byref(c), _ptr(U), h, max_it, tol, C.byref(it)), "source_implicit")
    return U, it.value


def strang_steps(P: Problem, scheme: int, U: np.ndarray, dt: float, n_steps: int,
                 max_it: int = NEWTON_MAX_IT, tol: float = NEWTON_TOL):
    """n_steps Strang-split steps S_{dt/2} T_dt S_{dt/2} (Eq. strang_split): T_dt one SSP
    step of the residual without its source part, S the implicit source substep.  Returns
    (new state, largest Newton count).  Built from the pinned parts; with the source off it
    reduces to ssp_steps() on the transport residual (tested)."""
    U = np.array(U, dtype=np.float64, order="C").reshape(P.shape)
    it = C.c_int()
    c = P._c()
    _check(lib().orc_strang_steps(C.byref(c), scheme, _ptr(U), dt, n_steps, max_it, tol, C.byref(it)),
           "strang_steps")
    return U, it.value


def shock_alpha(P: Problem, U: np.ndarray):
    """(alpha_raw, alpha): the Hennemann-Gassner blending coefficient of every element from
    the modal smoothness of rho p, before and after the face-neighbourhood maximum (Sec.
    3.1.1 "Shock Indicator and Smoothing"; App. A "Shock Capturing").  Pinned by the modes of
    known Legendre expansions, the sigmoid's midpoint at E = T, the clipping bounds and the
    neighbourhood rule."""
    U = np.ascontiguousarray(U, dtype=np.float64).reshape(P.shape)
    a = np.zeros(P.n_elem)
    b = np.zeros(P.n_elem)
    c = P._c()
    _check(lib().orc_shock_alpha(C.byref(c), _ptr(U), _ptr(a), _ptr(b)), "shock_alpha")
    return a, b


def fv_residual(P: Problem, U: np.ndarray) -> np.ndarray:
    """The first-order sub-cell finite-volume residual alone (Eq. vol_blend's R^FV).  Pinned
    by conservation (sum_i w_i R_i telescopes to the element-face fluxes), free-stream
    preservation, first-order consistency with -div F, and monotone (no new extrema) steps
    of a jump."""
    U = np.ascontiguousarray(U, dtype=np.float64).reshape(P.shape)
    dU = np.zeros_like(U)
    c = P._c()
    _check(lib().orc_fv_residual(C.byref(c), _ptr(U), _ptr(dU)), "fv_residual")
    return dU


def modes(P: Problem, q) -> np.ndarray:
    """Orthonormal tensor-Legendre coefficients of one element's nodal field (mode index in
    place of the node index).  Pinned against expansions evaluated with numpy's Legendre
    module."""
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
    m = np.zeros_like(q)
    c = P._c()
    _check(lib().orc_modes(C.byref(c), _ptr(q), _ptr(m)), "modes")
    return m


def metrics(P: Problem):
    """(Ja, J) of a curved mesh: Ja[elem, node, l, d] (the contravariant vectors, 3 x 3 per
    node, 2D in the leading 2 x 2) and J[elem, node] (Sec. 3.1.1: 2D cross-derivative form,
    3D conservative curl form).  Pinned by the discrete GCL, the affine case and free-stream
    preservation."""
    Ja = np.zeros(P.n_elem * P.n_nodes * 9)
    J = np.zeros(P.n_elem * P.n_nodes)
    c = P._c()
    _check(lib().orc_metrics(C.byref(c), _ptr(Ja), _ptr(J)), "metrics")
    return Ja.reshape(P.n_elem, P.n_nodes, 3, 3), J.reshape(P.n_elem, P.n_nodes)
