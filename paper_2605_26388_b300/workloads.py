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


def perturbed(U: np.ndarray, seed: int, rel: float) -> np.ndarray:
    """U times (1 + rel * xi), xi ~ U[-1, 1] seeded per entry (a non-smooth test state)."""
    r = uniform(seed, U.size).reshape(U.shape)
    return U * (1.0 + rel * (2.0 * r - 1.0))
