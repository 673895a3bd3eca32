"""Thin Python binding of the C-ABI in ``include/dgsem.h`` (ctypes).

Argument marshalling only: every step of the residual and the RK stage runs in the CUDA
library ``_lib/libdgsem.so``.  PyTorch provides device memory and the CUDA stream.  There
is no CPU fallback: if the library is missing, importing :func:`lib` raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field
from typing import Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libdgsem.so")

DG_OK, DG_EINVAL, DG_ENOMEM, DG_ECUDA, DG_ENONFINITE, DG_EPOSITIVITY, DG_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
DG_ETOOLARGE, DG_ECONVERGENCE = -7, -8
NOALLOC_MAX_INSTANCES = 4096
DG_EULER, DG_NAVIER_STOKES, DG_NS_REACTING = 0, 1, 2
MAX_SPECIES, MAX_REACTIONS = 8, 32
VOL_STRONG, VOL_WEAK, VOL_EC = 0, 1, 2
SURF_RUSANOV, SURF_HLLC, SURF_HLL, SURF_EC = 0, 1, 2, 3
FP64, FP32_MIXED = 0, 1
LAUNCH_PER_INSTANCE, LAUNCH_BATCHED = 0, 1
GROUPS_PER_DEGREE = 0x100  # group_scale | (1 << N): degree N uses group scale 2
BC_PERIODIC, BC_SLIP_WALL, BC_INFLOW, BC_OUTFLOW, BC_DIRICHLET = 0, 1, 2, 3, 4
BC_NOSLIP_ADIABATIC, BC_NOSLIP_ISOTHERMAL = 5, 6
MAX_VARS = 12
SSPRK33, SSPRK54 = 0, 1
NEWTON_MAX_IT, NEWTON_TOL = 40, 1e-12
MATH_EXP_TABLE, MATH_RCP_NEWTON, MATH_EXP_CUDA, MATH_RCP_CUDA = 0, 1, 2, 3

_STATUS = {0: "DG_OK", -1: "DG_EINVAL", -2: "DG_ENOMEM", -3: "DG_ECUDA", -4: "DG_ENONFINITE",
           -5: "DG_EPOSITIVITY", -6: "DG_EUNSUPPORTED", -7: "DG_ETOOLARGE", -8: "DG_ECONVERGENCE"}

# Every entry point include/dgsem.h declares (checked by the CPU tests).
EXPORTS = ["dg_init_mesh", "dg_state_size", "dg_instance_offset", "dg_set_state", "dg_get_state",
           "dg_rhs", "dg_rk_stage", "dg_rk_step", "dg_max_dt", "dg_check", "dg_gll",
           "dg_two_point_flux", "dg_max_dt_noalloc", "dg_set_launch", "dg_autotune",
           "dg_rhs_vjp", "dg_rk_step_vjp", "dg_adjoint_gammabar", "dg_source_step", "dg_newton_updates", "dg_shock_alpha",
           "dg_math_fn", "dg_alu_rate",
           "dg_last_error", "dg_free"]


class DGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class MeshDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("N", C.c_int), ("nel", C.c_int * 3), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3), ("periodic", C.c_int * 3), ("bc", C.c_int * 6),
                ("bc_state", (C.c_double * MAX_VARS) * 6), ("coords", C.POINTER(C.c_double))]


class Mechanism(C.Structure):
    """dg_mechanism: species data and reactions of a reacting mixture."""
    _fields_ = [("n_species", C.c_int), ("n_reactions", C.c_int),
                ("W", C.c_double * MAX_SPECIES), ("R", C.c_double * MAX_SPECIES),
                ("cv", C.c_double * MAX_SPECIES), ("h0", C.c_double * MAX_SPECIES),
                ("lnA", C.c_double * MAX_REACTIONS), ("b", C.c_double * MAX_REACTIONS),
                ("Ta", C.c_double * MAX_REACTIONS), ("kc", (C.c_double * 5) * MAX_REACTIONS),
                ("nu_f", (C.c_int * MAX_SPECIES) * MAX_REACTIONS),
                ("nu_b", (C.c_int * MAX_SPECIES) * MAX_REACTIONS),
                ("theta_v", C.c_double * MAX_SPECIES), ("ta_mode", C.c_int * MAX_REACTIONS)]

    @classmethod
    def from_dict(cls, m: dict) -> "Mechanism":
        """Pack a mechanism given as a dict of plain numbers (keys n_species, n_reactions, W, R,
        cv, h0 and, for the two-temperature model, theta_v per species; lnA, b, Ta, kc (5
        each), nu_f, nu_b and ta_mode per reaction)."""
        c = cls()
        ns, nr = int(m["n_species"]), int(m["n_reactions"])
        if not (1 <= ns <= MAX_SPECIES and 0 <= nr <= MAX_REACTIONS):
            raise ValueError("species or reaction count out of range")
        c.n_species, c.n_reactions = ns, nr
        for s in range(ns):
            c.W[s], c.R[s], c.cv[s], c.h0[s] = m["W"][s], m["R"][s], m["cv"][s], m["h0"][s]
        for r in range(nr):
            c.lnA[r], c.b[r], c.Ta[r] = m["lnA"][r], m["b"][r], m["Ta"][r]
            for k in range(5):
                c.kc[r][k] = m["kc"][r][k]
            for s in range(ns):
                c.nu_f[r][s], c.nu_b[r][s] = int(m["nu_f"][r][s]), int(m["nu_b"][r][s])
            c.ta_mode[r] = int(m.get("ta_mode", [0] * nr)[r])
        for s in range(ns):
            c.theta_v[s] = float(m.get("theta_v", [0.0] * ns)[s])
        return c


class Physics(C.Structure):
    _fields_ = [("equations", C.c_int), ("volume", C.c_int), ("surface", C.c_int),
                ("precision", C.c_int), ("gamma", C.c_double), ("rho_floor", C.c_double),
                ("p_floor", C.c_double), ("p_ref", C.c_double), ("mu", C.c_double),
                ("prandtl", C.c_double), ("chem", C.POINTER(Mechanism)),
                ("time_scheme", C.c_int), ("chem_split", C.c_int), ("newton_max_it", C.c_int),
                ("newton_tol", C.c_double), ("shock", C.c_int), ("alpha_min", C.c_double),
                ("alpha_max", C.c_double), ("sharpness", C.c_double), ("two_temperature", C.c_int),
                ("species_limiter", C.c_int)]


_lib = None


def lib():
    """Load the CUDA library (raises OSError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"CUDA library not built: {LIB_PATH} (run python -m paper_2605_26388_b300.build)")
        L = C.CDLL(LIB_PATH)
        vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
        L.dg_init_mesh.argtypes = [C.POINTER(MeshDesc), ip, C.POINTER(Physics), vp, C.POINTER(vp)]
        L.dg_state_size.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int)]
        L.dg_instance_offset.argtypes = [vp, ip, C.POINTER(C.c_int64)]
        L.dg_set_state.argtypes = [vp, vp]
        L.dg_get_state.argtypes = [vp, vp]
        L.dg_rhs.argtypes = [vp, vp, vp, C.c_double]
        L.dg_rk_stage.argtypes = [vp, ip, vp, vp, C.c_double, vp]
        L.dg_rk_step.argtypes = [vp, C.c_double, ip]
        L.dg_max_dt.argtypes = [vp, C.c_double, dp]
        L.dg_check.argtypes = [vp]
        L.dg_gll.argtypes = [ip, dp, dp, dp]
        L.dg_two_point_flux.argtypes = [vp, ip, ip, ip, vp, vp, vp]
        L.dg_max_dt_noalloc.argtypes = [C.POINTER(MeshDesc), ip, C.c_double, vp, C.c_double, vp, dp,
                                         C.POINTER(C.c_char_p)]
        L.dg_set_launch.argtypes = [vp, ip, ip, ip, ip]
        L.dg_rhs_vjp.argtypes = [vp, vp, vp, vp, dp]
        L.dg_rk_step_vjp.argtypes = [vp, vp, C.c_double, vp, dp]
        L.dg_adjoint_gammabar.argtypes = [vp, dp]
        L.dg_autotune.argtypes = [vp, C.c_double, ip, C.POINTER(C.c_int), dp]
        L.dg_source_step.argtypes = [vp, vp, C.c_double, vp]
        L.dg_newton_updates.argtypes = [vp, C.POINTER(C.c_int64)]
        L.dg_shock_alpha.argtypes = [vp, vp, vp, vp]
        L.dg_math_fn.argtypes = [ip, C.c_int64, vp, vp, vp]
        L.dg_alu_rate.argtypes = [ip, dp]
        L.dg_last_error.argtypes = [vp]
        L.dg_last_error.restype = C.c_char_p
        L.dg_free.argtypes = [vp]
        L.dg_free.restype = None
        for name in EXPORTS:
            if name not in ("dg_last_error", "dg_free"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def gll(N: int):
    """The library's GLL nodes, weights and differentiation matrix (host computation)."""
    x = np.zeros(N + 1)
    w = np.zeros(N + 1)
    D = np.zeros((N + 1) * (N + 1))
    st = lib().dg_gll(N, x.ctypes.data_as(C.POINTER(C.c_double)), w.ctypes.data_as(C.POINTER(C.c_double)),
                      D.ctypes.data_as(C.POINTER(C.c_double)))
    if st != DG_OK:
        raise DGError(st, f"dg_gll({N})")
    return x, w, D.reshape(N + 1, N + 1)


@dataclass
class Mesh:
    """One Cartesian instance: periodic, or with boundary conditions bc[f] (BC_*) on the
    faces x-, x+, y-, y+, z-, z+ of a direction whose two faces are both non-periodic;
    bc_state[f] is the prescribed conserved state of an inflow or Dirichlet face, or
    (T_wall,) of an isothermal no-slip wall."""
    dim: int
    N: int
    nel: Sequence[int]
    lo: Sequence[float]
    hi: Sequence[float]
    bc: Sequence[int] = (0, 0, 0, 0, 0, 0)
    bc_state: Sequence = None
    coords: np.ndarray = None  # node coordinates (dim, n_elem, n_p) of a curved mesh

    def c(self) -> MeshDesc:
        nel = list(self.nel) + [1] * (3 - len(self.nel))
        lo = list(self.lo) + [0.0] * (3 - len(self.lo))
        hi = list(self.hi) + [1.0] * (3 - len(self.hi))
        per = [1 if self.bc[2 * l] == 0 and self.bc[2 * l + 1] == 0 else 0 for l in range(3)]
        d = MeshDesc(self.dim, self.N, (C.c_int * 3)(*nel), (C.c_double * 3)(*lo),
                     (C.c_double * 3)(*hi), (C.c_int * 3)(*per))
        for f in range(6):
            d.bc[f] = int(self.bc[f])
            if self.bc_state is not None and self.bc_state[f] is not None:
                for v, x in enumerate(self.bc_state[f]):
                    d.bc_state[f][v] = float(x)
        if self.coords is not None:
            self._coords_c = np.ascontiguousarray(self.coords, dtype=np.float64)  # read by dg_init_mesh
            if self._coords_c.size != self.dim * self.n_elem * self.n_nodes:
                raise ValueError("coords must hold dim * n_elem * n_p values")
            d.coords = self._coords_c.ctypes.data_as(C.POINTER(C.c_double))
        return d

    @property
    def n_elem(self) -> int:
        return int(np.prod(list(self.nel)[: self.dim]))

    @property
    def n_nodes(self) -> int:
        return (self.N + 1) ** self.dim


class Solver:
    """A DGSEM context: instances + physics, bound to the current CUDA stream.

    Tensors passed in and out are float64, contiguous, on the context's device, in the
    SoA layout U[var, node] (node = instance offset + elem * n_p + local node)."""

    def __init__(self, meshes, volume=VOL_STRONG, surface=SURF_RUSANOV, precision=FP64,
                 gamma=1.4, rho_floor=0.0, p_floor=0.0, p_ref=0.0, stream=None,
                 equations=DG_EULER, mu=0.0, prandtl=0.72, mechanism=None,
                 time_scheme=SSPRK33, chem_split=False, newton_max_it=0, newton_tol=0.0,
                 shock=False, alpha_min=0.0, alpha_max=0.0, sharpness=0.0, two_temperature=False,
                 species_limiter=False):
        import torch
        if isinstance(meshes, Mesh):
            meshes = [meshes]
        self.meshes = list(meshes)
        self.gamma = gamma
        arr = (MeshDesc * len(self.meshes))(*[m.c() for m in self.meshes])
        phys = Physics(equations, volume, surface, precision, gamma, rho_floor, p_floor, p_ref,
                       mu, prandtl, None, time_scheme, 1 if chem_split else 0, newton_max_it,
                       newton_tol, 1 if shock else 0, alpha_min, alpha_max, sharpness,
                       1 if two_temperature else 0, 1 if species_limiter else 0)
        self.n_elem = sum(m.n_elem for m in self.meshes)
        if mechanism is not None:
            mech = mechanism if isinstance(mechanism, Mechanism) else Mechanism.from_dict(mechanism)
            phys.chem = C.pointer(mech)  # copied by dg_init_mesh
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        st = lib().dg_init_mesh(arr, len(self.meshes), C.byref(phys), C.c_void_p(stream.cuda_stream), C.byref(h))
        if st != DG_OK:
            raise DGError(st, "dg_init_mesh")
        self._h = h
        n = C.c_int64()
        nv = C.c_int()
        self._call(lib().dg_state_size(self._h, C.byref(n), C.byref(nv)), "dg_state_size")
        self.n_doubles, self.nv = int(n.value), int(nv.value)
        self.n_nodes = self.n_doubles // self.nv
        self.offsets = []
        for i in range(len(self.meshes)):
            o = C.c_int64()
            self._call(lib().dg_instance_offset(self._h, i, C.byref(o)), "dg_instance_offset")
            self.offsets.append(int(o.value))

    # -- helpers -------------------------------------------------------------------------
    def _call(self, st: int, what: str):
        if st != DG_OK:
            msg = lib().dg_last_error(self._h if getattr(self, "_h", None) else None)
            raise DGError(st, f"{what}: {msg.decode() if msg else ''}")

    def _dev(self, t, what):
        import torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise TypeError(f"{what} must be a contiguous float64 CUDA tensor")
        if t.numel() != self.n_doubles:
            raise ValueError(f"{what} has {t.numel()} values, expected {self.n_doubles}")
        return C.c_void_p(t.data_ptr())

    @property
    def shape(self):
        return (self.nv, self.n_nodes)

    # -- entry points --------------------------------------------------------------------
    def set_state(self, U):
        """Copy a state (CUDA tensor, or host tensor / array) into the context."""
        import torch
        if isinstance(U, np.ndarray):
            U = torch.from_numpy(np.ascontiguousarray(U, dtype=np.float64))
        if U.numel() != self.n_doubles or U.dtype != torch.float64 or not U.is_contiguous():
            raise ValueError("state must be contiguous float64 with n_vars * n_nodes values")
        self._keep = U  # the copy is asynchronous; keep the source alive
        self._call(lib().dg_set_state(self._h, C.c_void_p(U.data_ptr())), "dg_set_state")

    def get_state(self, out=None):
        import torch
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        self._call(lib().dg_get_state(self._h, C.c_void_p(out.data_ptr())), "dg_get_state")
        return out

    def rhs(self, U, out=None):
        import torch
        if out is None:
            out = torch.empty_like(U)
        self._call(lib().dg_rhs(self._h, self._dev(U, "U"), self._dev(out, "dUdt"), 0.0), "dg_rhs")
        return out

    def rk_stage(self, stage: int, Un, Uprev, dt: float, out=None):
        import torch
        if out is None:
            out = torch.empty_like(Un)
        self._call(lib().dg_rk_stage(self._h, stage, self._dev(Un, "Un"), self._dev(Uprev, "Uprev"), dt,
                                     self._dev(out, "Uout")), "dg_rk_stage")
        return out

    def rk_step(self, dt: float, n_steps: int = 1):
        self._call(lib().dg_rk_step(self._h, dt, n_steps), "dg_rk_step")

    def source_step(self, U, h: float, out=None):
        """Implicit source substep S_h (see dg_source_step); out may be U (in place)."""
        import torch
        if out is None:
            out = torch.empty_like(U)
        self._call(lib().dg_source_step(self._h, self._dev(U, "U"), h, self._dev(out, "Uout")),
                   "dg_source_step")
        return out

    def shock_alpha(self, U):
        """(alpha_raw, alpha) per element for state U (see dg_shock_alpha)."""
        import torch
        a = torch.empty(self.n_elem, dtype=torch.float64, device="cuda")
        b = torch.empty_like(a)
        self._call(lib().dg_shock_alpha(self._h, self._dev(U, "U"), C.c_void_p(a.data_ptr()),
                                        C.c_void_p(b.data_ptr())), "dg_shock_alpha")
        return a, b

    def newton_updates(self) -> int:
        """Newton updates of the implicit substeps since the previous call (resets the count)."""
        n = C.c_int64()
        self._call(lib().dg_newton_updates(self._h, C.byref(n)), "dg_newton_updates")
        return int(n.value)

    def rhs_vjp(self, U, lam, Ubar=None):
        """(Ubar + (dL/dU)^T lam, lam . dL/dgamma) -- see dg_rhs_vjp."""
        import torch
        if Ubar is None:
            Ubar = torch.zeros_like(U)
        g = C.c_double(0.0)
        self._call(lib().dg_rhs_vjp(self._h, self._dev(U, "U"), self._dev(lam, "lam"), self._dev(Ubar, "Ubar"),
                                    C.byref(g)), "dg_rhs_vjp")
        return Ubar, g.value

    def rk_step_vjp(self, Un, dt: float, lam, defer: bool = False):
        """In place: lam = dJ/dU^{n+1} -> dJ/dU^n; returns dJ/dgamma through this step.  With
        defer=True the gamma contribution stays on the device (no synchronization; returns 0.0)
        until adjoint_gammabar()."""
        g = C.c_double(0.0)
        self._call(lib().dg_rk_step_vjp(self._h, self._dev(Un, "Un"), dt, self._dev(lam, "lam"),
                                        None if defer else C.byref(g)), "dg_rk_step_vjp")
        return g.value

    def adjoint_gammabar(self) -> float:
        """The gamma contributions of deferred adjoint calls (synchronizes; resets them)."""
        g = C.c_double(0.0)
        self._call(lib().dg_adjoint_gammabar(self._h, C.byref(g)), "dg_adjoint_gammabar")
        return g.value

    def set_launch(self, mode: int, group_scale: int = 1, ctas_per_sm: int = 0, order: int = 0):
        """Per-instance launches or one batched persistent launch per stage (see dg_set_launch)."""
        self._call(lib().dg_set_launch(self._h, mode, group_scale, ctas_per_sm, order), "dg_set_launch")

    def autotune(self, dt: float, n_reps: int = 2):
        """Time every launch configuration on this context, keep the fastest; returns
        ((mode, group_scale, ctas_per_sm, order), ms_per_step)."""
        cfg = (C.c_int * 4)()
        ms = C.c_double()
        self._call(lib().dg_autotune(self._h, dt, n_reps, cfg, C.byref(ms)), "dg_autotune")
        return tuple(cfg), ms.value

    def max_dt(self, cfl: float) -> float:
        out = C.c_double()
        self._call(lib().dg_max_dt(self._h, cfl, C.byref(out)), "dg_max_dt")
        return out.value

    def check(self):
        """Synchronize and raise DGError if a kernel flagged a non-finite or non-positive state."""
        self._call(lib().dg_check(self._h), "dg_check")

    def two_point_flux(self, kind: int, l: int, uL, uR, out=None):
        import torch
        n = uL.shape[0]
        if out is None:
            out = torch.empty_like(uL)
        self._call(lib().dg_two_point_flux(self._h, kind, l, n, C.c_void_p(uL.data_ptr()),
                                           C.c_void_p(uR.data_ptr()), C.c_void_p(out.data_ptr())),
                   "dg_two_point_flux")
        return out

    def close(self):
        if getattr(self, "_h", None):
            lib().dg_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def math_fn(kind: int, x, out=None):
    """The device math routine `kind` (MATH_*) applied element-wise to a float64 CUDA tensor."""
    import torch
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
        raise TypeError("x must be a contiguous float64 CUDA tensor")
    if out is None:
        out = torch.empty_like(x)
    st = lib().dg_math_fn(kind, x.numel(), C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()),
                          C.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != DG_OK:
        raise DGError(st, "dg_math_fn")
    return out
