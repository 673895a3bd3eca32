"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle's tests.

This module holds none of the method's arithmetic: it evaluates closed-form initial
conditions at given node coordinates and draws seeded random numbers.  The reference
nodes ``xi`` (GLL nodes on [-1, 1]) are passed in by the caller, so that neither side's
operator code is used by the other.

Random numbers come from splitmix64 (Steele, Lea and Flood 2014): state_k = seed +
k * 0x9E3779B97F4A7C15, then two xor-shift-multiply rounds; a uniform double on [0, 1)
is the top 53 bits times 2^-53.

State layout everywhere: ``U[var, elem, node]`` (SoA), elements lexicographic with x
fastest, nodes lexicographic with i (x index) fastest.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n consecutive splitmix64 outputs for the given seed (uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """n seeded uniforms on [lo, hi)."""
    u = (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def node_coordinates(dim: int, nel, lo, hi, xi: np.ndarray) -> np.ndarray:
    """Physical coordinates X[l, elem, node] of every GLL node of an affine Cartesian mesh
    (the element map x = lo + dx (e + (xi + 1)/2) in each direction)."""
    n1 = len(xi)
    nel = list(nel)[:dim]
    n_elem = int(np.prod(nel))
    n_nodes = n1 ** dim
    X = np.zeros((dim, n_elem, n_nodes))
    e = np.arange(n_elem)
    ec = [e % nel[0], (e // nel[0]) % nel[1]] + ([e // (nel[0] * nel[1])] if dim == 3 else [])
    nd = np.arange(n_nodes)
    nc = [nd % n1, (nd // n1) % n1] + ([nd // (n1 * n1)] if dim == 3 else [])
    for l in range(dim):
        dx = (hi[l] - lo[l]) / nel[l]
        X[l] = lo[l] + dx * (ec[l][:, None] + 0.5 * (np.asarray(xi)[nc[l]][None, :] + 1.0))
    return X


def conserved(rho, vel, p, gamma: float) -> np.ndarray:
    """Conserved Euler variables (rho, rho u, ..., E) from primitives; E from the ideal-gas
    closure p = (gamma - 1)(E - rho |u|^2 / 2) stated with the governing equations."""
    dim = len(vel)
    U = np.zeros((dim + 2,) + np.shape(rho))
    U[0] = rho
    kin = 0.0
    for d in range(dim):
        U[1 + d] = rho * vel[d]
        kin = kin + rho * vel[d] ** 2
    U[dim + 1] = p / (gamma - 1.0) + 0.5 * kin
    return U


# ------------------------------------------------------------------------------------------
# Workloads
# ------------------------------------------------------------------------------------------

def density_wave_2d(nel: int, xi: np.ndarray, gamma: float = 1.4, t: float = 0.0,
                    lo=(0.0, 0.0), hi=(2.0, 2.0)) -> np.ndarray:
    """Advected density wave rho = 1 + sin(pi (x + y - 2t))/2, u = v = 1, p = 1 on [0,2]^2
    (exact solution of the Euler equations: a pure translation)."""
    X = node_coordinates(2, (nel, nel), lo, hi, xi)
    rho = 1.0 + 0.5 * np.sin(np.pi * (X[0] + X[1] - 2.0 * t))
    one = np.ones_like(rho)
    return conserved(rho, [one, one], one, gamma)


def taylor_green_3d(nel: int, xi: np.ndarray, mach: float = 0.1, gamma: float = 1.4,
                    lo=(0.0, 0.0, 0.0), hi=None) -> np.ndarray:
    """Taylor-Green vortex (Sec. 4.2, Eq. tgv_ic) with A = 1, rho = 1:
    u = sin x cos y cos z, v = -cos x sin y cos z, w = 0,
    p = 1/(gamma Ma^2) + [cos2x cos2z + 2 cos2y + 2 cos2x + cos2y cos2z]/16."""
    if hi is None:
        hi = (2 * math.pi,) * 3
    X = node_coordinates(3, (nel, nel, nel), lo, hi, xi)
    x, y, z = X
    rho = np.ones_like(x)
    u = np.sin(x) * np.cos(y) * np.cos(z)
    v = -np.cos(x) * np.sin(y) * np.cos(z)
    w = np.zeros_like(x)
    p = 1.0 / (gamma * mach ** 2) + (np.cos(2 * x) * np.cos(2 * z) + 2 * np.cos(2 * y)
                                      + 2 * np.cos(2 * x) + np.cos(2 * y) * np.cos(2 * z)) / 16.0
    return conserved(rho, [u, v, w], p, gamma)


def fourier_field(seed: int, X: np.ndarray, lo, hi, kmax: int) -> np.ndarray:
    """Seeded smooth periodic field: sum over integer wave vectors 0 < |k|_inf, |k|_2 <= kmax
    of a_k cos(2 pi k.x/L + phi_k), a_k ~ U[-1,1] / (1 + |k|^2), scaled to max |f| = 1."""
    dim = X.shape[0]
    ks = []
    rng = range(-kmax, kmax + 1)
    if dim == 2:
        ks = [(a, b) for a in rng for b in rng if 0 < a * a + b * b <= kmax * kmax]
    else:
        ks = [(a, b, c) for a in rng for b in rng for c in rng if 0 < a * a + b * b + c * c <= kmax * kmax]
    r = uniform(seed, 2 * len(ks))
    f = np.zeros(X.shape[1:])
    for n, k in enumerate(ks):
        amp = (2.0 * r[2 * n] - 1.0) / (1.0 + sum(kk * kk for kk in k))
        phase = 2.0 * math.pi * r[2 * n + 1]
        arg = phase
        for l in range(dim):
            arg = arg + 2.0 * math.pi * k[l] * (X[l] - lo[l]) / (hi[l] - lo[l])
        f += amp * np.cos(arg)
    return f / np.max(np.abs(f))


def fourier_field_3d_tensor(seed: int, nel, xi: np.ndarray, lo, hi, kmax: int) -> np.ndarray:
    """fourier_field on a 3D Cartesian DGSEM mesh, returned as (n_elem, n_nodes): the same
    sum (same seeded amplitudes and phases, same wave vectors), evaluated as a separable
    product over the three axes, which is what makes full-size meshes affordable."""
    rng = range(-kmax, kmax + 1)
    ks = [(a, b, c) for a in rng for b in rng for c in rng if 0 < a * a + b * b + c * c <= kmax * kmax]
    r = uniform(seed, 2 * len(ks))
    nk = 2 * kmax + 1
    Ck = np.zeros((nk, nk, nk), dtype=np.complex128)
    for n, k in enumerate(ks):
        amp = (2.0 * r[2 * n] - 1.0) / (1.0 + sum(kk * kk for kk in k))
        Ck[k[0] + kmax, k[1] + kmax, k[2] + kmax] = amp * np.exp(1j * 2.0 * math.pi * r[2 * n + 1])
    n1 = len(xi)
    E = []
    for l in range(3):
        h = (hi[l] - lo[l]) / nel[l]
        x = (lo[l] + h * np.arange(nel[l])[:, None] + 0.5 * h * (np.asarray(xi)[None, :] + 1.0)).reshape(-1)
        kk = np.arange(-kmax, kmax + 1)[:, None]
        E.append(np.exp(1j * 2.0 * math.pi * kk * (x[None, :] - lo[l]) / (hi[l] - lo[l])))
    T1 = np.einsum("abc,ax->bcx", Ck, E[0])
    T2 = np.einsum("bcx,by->cyx", T1, E[1])
    F = np.einsum("cyx,cz->zyx", T2, E[2]).real
    F = F.reshape(nel[2], n1, nel[1], n1, nel[0], n1).transpose(0, 2, 4, 1, 3, 5)
    F = F.reshape(nel[0] * nel[1] * nel[2], n1 ** 3)
    return F / np.max(np.abs(F))


def acoustic_2d(nel: int, xi: np.ndarray, seed: int = 3, amp: float = 0.05, gamma: float = 1.4,
                lo=(0.0, 0.0), hi=(1.0, 1.0)) -> np.ndarray:
    """Smooth seeded acoustic perturbation at rest: rho = 1 + amp psi_rho, p = 1 + amp psi_p,
    u = v = 0, psi unit-max Fourier sums with |k| <= 4 (seeds `seed`, `seed + 100`)."""
    X = node_coordinates(2, (nel, nel), lo, hi, xi)
    rho = 1.0 + amp * fourier_field(seed, X, lo, hi, 4)
    p = 1.0 + amp * fourier_field(seed + 100, X, lo, hi, 4)
    z = np.zeros_like(rho)
    return conserved(rho, [z, z], p, gamma)


def target_density_2d(nel: int, xi: np.ndarray, seed: int = 4, amp: float = 0.05,
                      lo=(0.0, 0.0), hi=(1.0, 1.0)) -> np.ndarray:
    """Seeded target density field rho_target[elem, node] for the adjoint loss."""
    X = node_coordinates(2, (nel, nel), lo, hi, xi)
    return 1.0 + amp * fourier_field(seed, X, lo, hi, 4)


def isentropic_vortex_2d(nel: int, xi: np.ndarray, center=(0.0, 0.0), strength: float = 5.0,
                         gamma: float = 1.4, lo=(-5.0, -5.0), hi=(5.0, 5.0)) -> np.ndarray:
    """Shu's isentropic vortex on a uniform stream rho = p = 1, u = v = 1:
    du = -eps/(2 pi) e^{(1-r^2)/2} (y - yc), dv = eps/(2 pi) e^{(1-r^2)/2} (x - xc),
    T = 1 - (gamma-1) eps^2/(8 gamma pi^2) e^{1-r^2}, rho = T^{1/(gamma-1)}, p = rho T."""
    X = node_coordinates(2, (nel, nel), lo, hi, xi)
    dx = X[0] - center[0]
    dy = X[1] - center[1]
    r2 = dx * dx + dy * dy
    g = np.exp(0.5 * (1.0 - r2))
    u = 1.0 - strength / (2 * math.pi) * g * dy
    v = 1.0 + strength / (2 * math.pi) * g * dx
    T = 1.0 - (gamma - 1.0) * strength ** 2 / (8 * gamma * math.pi ** 2) * g * g
    rho = T ** (1.0 / (gamma - 1.0))
    return conserved(rho, [u, v], rho * T, gamma)


def batched_vortex_set(n_inst: int = 256, seed: int = 5, n_range=(8, 96), degrees=(2, 3, 4, 5)):
    """Seeded list of (nel, N, center) for the batched workload: nel ~ U{8..96} (nel^2
    elements), N ~ U{degrees}, vortex centre ~ U[-2.5, 2.5]^2."""
    r = uniform(seed, 4 * n_inst)
    out = []
    for i in range(n_inst):
        nel = n_range[0] + int(r[4 * i] * (n_range[1] - n_range[0] + 1))
        N = degrees[int(r[4 * i + 1] * len(degrees))]
        c = (-2.5 + 5.0 * r[4 * i + 2], -2.5 + 5.0 * r[4 * i + 3])
        out.append((nel, N, c))
    return out


def warped_coordinates(dim: int, nel, xi: np.ndarray, lo, hi, amp: float = 0.05) -> np.ndarray:
    """Node coordinates (dim, n_elem, n_nodes) of a curved periodic mesh on the box: the
    Cartesian nodes displaced by amp * L_d * prod_k sin(2 pi (x_k - lo_k) / L_k) (a phase
    per component), a periodic smooth warp of the element grid."""
    X = node_coordinates(dim, nel, lo, hi, xi)
    L = [hi[d] - lo[d] for d in range(dim)]
    Y = X.copy()
    for d in range(dim):
        w = np.ones_like(X[0])
        for k in range(dim):
            w = w * np.sin(2.0 * np.pi * (X[k] - lo[k]) / L[k] + 0.3 * d * (k == d))
        Y[d] = X[d] + amp * L[d] * w
    return Y


def blast_wave(dim: int, nel: int, xi: np.ndarray, p_in: float = 10.0, radius: float = 0.4,
               gamma: float = 1.4, L: float = 2.0) -> np.ndarray:
    """The shock-capturing workload: a blast in a periodic box [0, L]^dim -- gas at rest,
    rho = 1, p = p_in inside the ball of the given radius about the box centre and p = 1
    outside, a discontinuity at the GLL nodes (no smoothing)."""
    lo, hi = (0.0,) * dim, (L,) * dim
    X = node_coordinates(dim, (nel,) * dim, lo, hi, xi)
    r2 = sum((X[l] - 0.5 * L) ** 2 for l in range(dim))
    p = np.where(r2 < radius * radius, p_in, 1.0)
    rho = np.ones_like(p)
    return conserved(rho, [np.zeros_like(p)] * dim, p, gamma)


def perturbed(U: np.ndarray, seed: int, rel: float) -> np.ndarray:
    """U times (1 + rel * xi), xi ~ U[-1, 1] seeded per entry (a non-smooth test state)."""
    r = uniform(seed, U.size).reshape(U.shape)
    return U * (1.0 + rel * (2.0 * r - 1.0))


# ------------------------------------------------------------------------------------------
# 5-species air (N2, O2, NO, N, O): species data and a seeded reaction mechanism
# ------------------------------------------------------------------------------------------
R_UNIVERSAL = 8.314462618  # J/(mol K)
SPECIES = ("N2", "O2", "NO", "N", "O")
_W_N, _W_O = 0.0140067, 0.0159994  # kg/mol; molecules are exact sums (atom balance)
MOLAR_MASS = (2 * _W_N, 2 * _W_O, _W_N + _W_O, _W_N, _W_O)
DIATOMIC = (True, True, True, False, False)
# formation enthalpies per mole (J/mol; N2 and O2 are the references), per kg below
_H0_MOLAR = (0.0, 0.0, 90291.0, 472680.0, 249175.0)
# characteristic vibrational temperatures (K) of N2, O2, NO (harmonic oscillators; atoms 0),
# the standard values of Park's air model
THETA_V = (3395.0, 2239.0, 2817.0, 0.0, 0.0)
ATOMS_N = (2, 0, 1, 1, 0)
ATOMS_O = (0, 2, 1, 0, 1)


def air5_mechanism(seed: int = 1, lg10A=(12.0, 22.0), b=(-1.6, 0.0), Ta=(2.0e4, 1.2e5)):
    """Species properties and 17 seeded reactions (dict of plain numbers):
    r = 0..14: X + M <-> products + M for X in (N2, O2, NO) and M each of the 5 species
    (N2 -> 2N, O2 -> 2O, NO -> N + O); r = 15: N2 + O <-> NO + N; r = 16: N + O2 <-> NO + O.
    Forward rate k_f = exp(lnA + b ln T - Ta/T) with log10 A ~ U[12,22], b ~ U[-1.6,0],
    Ta ~ U[2e4,1.2e5] K (cm-mol-s units); equilibrium constant
    ln K_c = a0/Z + a1 + a2 ln Z + a3 Z + a4 Z^2, Z = 1e4/T, seeded so that |ln K_c| < 40 on
    2000-8000 K.  Calorically perfect species: c_v = 5/2 R_s (diatomic), 3/2 R_s (atomic)."""
    ns = 5
    Rs = [R_UNIVERSAL / w for w in MOLAR_MASS]
    cv = [(2.5 if d else 1.5) * r for d, r in zip(DIATOMIC, Rs)]
    h0 = [h / w for h, w in zip(_H0_MOLAR, MOLAR_MASS)]
    nu_f, nu_b = [], []
    for x, prod in ((0, (3, 3)), (1, (4, 4)), (2, (3, 4))):
        for m in range(ns):
            f = [0] * ns
            bk = [0] * ns
            f[x] += 1
            f[m] += 1
            for p_ in prod:
                bk[p_] += 1
            bk[m] += 1
            nu_f.append(f)
            nu_b.append(bk)
    nu_f.append([1, 0, 0, 0, 1]); nu_b.append([0, 0, 1, 1, 0])  # N2 + O <-> NO + N
    nu_f.append([0, 1, 0, 1, 0]); nu_b.append([0, 0, 1, 0, 1])  # N + O2 <-> NO + O
    nr = len(nu_f)
    r = uniform(seed, 8 * nr)
    lnA, bb, ta, kc = [], [], [], []
    for i in range(nr):
        lnA.append(math.log(10.0) * (lg10A[0] + (lg10A[1] - lg10A[0]) * r[8 * i]))
        bb.append(b[0] + (b[1] - b[0]) * r[8 * i + 1])
        ta.append(Ta[0] + (Ta[1] - Ta[0]) * r[8 * i + 2])
        kc.append([-1.0 + 2.0 * r[8 * i + 3], -5.0 + 10.0 * r[8 * i + 4], -1.0 + 2.0 * r[8 * i + 5],
                   -5.0 * r[8 * i + 6], -0.2 + 0.4 * r[8 * i + 7]])
    # two-temperature data: vibrational temperatures, and the controlling temperature of each
    # reaction -- sqrt(T Tv) for the 15 dissociations, T for the two exchanges
    return {"n_species": ns, "n_reactions": nr, "W": list(MOLAR_MASS), "R": Rs, "cv": cv, "h0": h0,
            "lnA": lnA, "b": bb, "Ta": ta, "kc": kc, "nu_f": nu_f, "nu_b": nu_b,
            "theta_v": list(THETA_V), "ta_mode": [1] * 15 + [0, 0]}


def reacting_conserved(rho_s, vel, T, mech: dict, Tv=None) -> np.ndarray:
    """Conserved reacting state (rho_1..rho_ns, rho u, ..., E) from partial densities, velocity
    components and temperature of calorically perfect species:
    E = sum_s rho_s (cv_s T + h0_s) + rho |u|^2 / 2.  With a vibrational temperature Tv
    (two-temperature state): E_v = sum_s rho_s R_s theta_s / (exp(theta_s / Tv) - 1) is
    appended and added to E."""
    ns = int(mech["n_species"])
    rho = sum(np.asarray(rho_s[s], dtype=np.float64) for s in range(ns))
    shape = np.shape(rho)
    U = np.zeros((ns + len(vel) + 1 + (0 if Tv is None else 1),) + shape)
    e = np.zeros(shape)
    for s in range(ns):
        U[s] = rho_s[s]
        e = e + U[s] * (mech["cv"][s] * T + mech["h0"][s])
    kin = np.zeros(shape)
    for d, v in enumerate(vel):
        U[ns + d] = rho * v
        kin = kin + v * v
    U[ns + len(vel)] = e + 0.5 * rho * kin
    if Tv is not None:
        Ev = np.zeros(shape)
        for s in range(ns):
            th = mech["theta_v"][s]
            if th > 0.0:
                Ev = Ev + U[s] * mech["R"][s] * th / np.expm1(th / Tv)
        U[ns + len(vel)] += Ev
        U[ns + len(vel) + 1] = Ev
    return U


def reacting_tgv_3d(nel: int, xi: np.ndarray, mech: dict, seed: int = 2, U0: float = 100.0,
                    p0: float = 101325.0, lo=(0.0, 0.0, 0.0), hi=None, two_temperature: bool = False):
    """The reacting workload's state (9 conserved variables rho_s, rho u, rho v, rho w, E):
    Taylor-Green velocity of amplitude U0 on [0, 2 pi]^3 m, uniform p0, temperature
    T = 5000 + 3000 phi/max|phi| K with phi a seeded Fourier sum (|k| <= 3), air mass
    fractions Y = (0.767, 0.233, 1e-10, 1e-10, 1e-10) normalised.  E from the calorically
    perfect mixture: E = sum_s rho_s (cv_s T + h0_s) + rho |u|^2 / 2, p = sum_s rho_s R_s T.
    two_temperature: a tenth variable E_v at a lagging vibrational temperature
    Tv = T (0.6 + 0.3 psi), psi a second seeded Fourier sum scaled to [-1, 1] (seed + 7), so
    Tv spans 0.3 T to 0.9 T (vibration behind the translational mode, as behind a shock)."""
    if hi is None:
        hi = (2 * math.pi,) * 3
    X = node_coordinates(3, (nel, nel, nel), lo, hi, xi)
    x, y, z = X
    T = 5000.0 + 3000.0 * fourier_field_3d_tensor(seed, (nel, nel, nel), xi, lo, hi, 3)
    Y = np.array([0.767, 0.233, 1e-10, 1e-10, 1e-10])
    Y = Y / Y.sum()
    Rmix = float(np.dot(Y, mech["R"]))
    rho = p0 / (Rmix * T)
    u = U0 * np.sin(x) * np.cos(y) * np.cos(z)
    v = -U0 * np.cos(x) * np.sin(y) * np.cos(z)
    w = np.zeros_like(x)
    Tv = None
    if two_temperature:
        Tv = T * (0.6 + 0.3 * fourier_field_3d_tensor(seed + 7, (nel, nel, nel), xi, lo, hi, 3))
    return reacting_conserved([rho * Y[s] for s in range(5)], [u, v, w], T, mech, Tv=Tv)


AIR_Y = (0.767, 0.233, 1e-10, 1e-10, 1e-10)


def reacting_tgv_viscosity(mech: dict, U0: float = 100.0, p0: float = 101325.0, T0: float = 5000.0,
                           L: float = 1.0, Re: float = 1600.0) -> float:
    """Constant viscosity of the reacting workload: mu = rho0 U0 L / Re with rho0 the density
    of the air composition at p0 and the mean temperature T0 (Re = 1600, L = 1 on the
    [0, 2 pi]^3 box)."""
    Y = np.array(AIR_Y)
    Y = Y / Y.sum()
    rho0 = p0 / (float(np.dot(Y, mech["R"])) * T0)
    return rho0 * U0 * L / Re
