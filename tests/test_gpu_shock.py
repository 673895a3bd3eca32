"""Hennemann-Gassner shock capturing on the GPU (through the C-ABI) against the oracle.

- the blending coefficients (raw and after the neighbourhood maximum) of blast states;
- the blended residual (Eq. vol_blend) in 2D and 3D, strong and two-point volume forms,
  Rusanov and HLLC, FP64 (rel-L2 <= 1e-12 per conserved quantity) and FP32-mixed (<= 1e-5);
- SSP-RK3 and SSP-RK54 steps through the blast (blended elements change every stage) against
  the oracle, conservation of every variable, and positivity where the unblended scheme fails;
- a resolved smooth state: shock capturing on gives the same bits as off;
- the blast workload at the benchmark's size: the stage residual on sampled elements.
"""
import math

import numpy as np
import pytest

from paper_2605_26388_b300 import workloads as wl

pytestmark = pytest.mark.gpu

GAMMA = 1.4


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_26388_b300 import build, dgsem
    build.build_library()
    return torch, dgsem


def dev(torch, U):
    return torch.from_numpy(np.ascontiguousarray(U.reshape(U.shape[0], -1))).cuda()


def rel(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    nv = a.shape[0]
    out = 0.0
    for g in ([0], list(range(1, nv - 1)), [nv - 1]):
        nb = np.linalg.norm(b[g])
        out = max(out, np.linalg.norm(a[g] - b[g]) / nb if nb > 0 else np.linalg.norm(a[g]))
    return out


def setup(orc, dg, dim, N, nel, vol, surf, prec=0, shock=True, **kw):
    L = 2.0
    P = orc.Problem(dim=dim, N=N, nel=(nel,) * dim, lo=(0.0,) * dim, hi=(L,) * dim, volume=vol,
                    surface=surf, gamma=GAMMA, shock=shock)
    S = dg.Solver(dg.Mesh(dim, N, (nel,) * dim, (0.0,) * dim, (L,) * dim), volume=vol, surface=surf,
                  precision=prec, gamma=GAMMA, shock=shock, **kw)
    return P, S


def blast(orc, P, seed=None):
    xi, _ = orc.gll(P.N)
    U = wl.blast_wave(P.dim, P.nel[0], xi).reshape(P.shape)
    if seed is not None:
        U = wl.perturbed(U, seed, 0.02)
    return U


CASES = [(2, 3, 12, 2, 0), (2, 4, 10, 0, 1), (2, 6, 6, 2, 1), (3, 3, 5, 2, 0), (3, 2, 6, 0, 0),
         (3, 4, 4, 2, 1)]


@pytest.mark.parametrize("dim,N,nel,vol,surf", CASES)
def test_alpha_matches_oracle(env, orc, dim, N, nel, vol, surf):
    torch, dg = env
    P, S = setup(orc, dg, dim, N, nel, vol, surf)
    U = blast(orc, P, seed=dim + N)
    raw, al = S.shock_alpha(dev(torch, U))
    oraw, oal = orc.shock_alpha(P, U)
    assert np.count_nonzero(oal) > 0
    assert np.array_equal(raw.cpu().numpy() > 0, oraw > 0)
    assert np.abs(raw.cpu().numpy() - oraw).max() <= 1e-10
    assert np.abs(al.cpu().numpy() - oal).max() <= 1e-10
    S.close()


@pytest.mark.parametrize("dim,N,nel,vol,surf", CASES)
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_blended_residual_matches_oracle(env, orc, dim, N, nel, vol, surf, prec, tol):
    torch, dg = env
    P, S = setup(orc, dg, dim, N, nel, vol, surf, prec=prec)
    U = blast(orc, P, seed=7)
    ref = orc.rhs(P, U)
    got = S.rhs(dev(torch, U)).cpu().numpy().reshape(ref.shape)
    S.check()
    assert rel(got, ref) <= tol, rel(got, ref)
    S.close()


@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 1e-5)])
def test_steps_through_the_blast(env, orc, scheme, prec, tol):
    torch, dg = env
    dim, N, nel = 2, 3, 12
    P, S = setup(orc, dg, dim, N, nel, 2, 0, prec=prec, time_scheme=scheme)
    U = blast(orc, P)
    dt = orc.max_dt(P, U, 0.3)
    n = 30
    S.set_state(dev(torch, U))
    S.rk_step(dt, n)
    S.check()
    got = S.get_state().cpu().numpy().reshape(U.shape)
    ref = orc.ssp_steps(P, 54 if scheme else 3, U, dt, n)
    assert rel(got, ref) <= tol, rel(got, ref)
    if prec == 0:
        _, w = orc.gll(N)
        W = np.multiply.outer(w, w).ravel()
        for v in range(4):
            m0, m1 = np.sum(U[v] * W), np.sum(got[v] * W)
            scale = max(np.sum(np.abs(U[v]) * W), np.sum(np.abs(got[v]) * W))  # momentum starts at 0
            assert abs(m1 - m0) <= 1e-13 * scale, v
    S.close()


def test_blast_stays_positive_only_with_shock_capturing(env, orc):
    torch, dg = env
    dim, N, nel = 2, 3, 16
    for shock in (True, False):
        P, S = setup(orc, dg, dim, N, nel, 2, 0, shock=shock)
        U = blast(orc, P)
        S.set_state(dev(torch, U))
        S.rk_step(orc.max_dt(P, U, 0.3), 200)
        if shock:
            S.check()
            V = S.get_state().cpu().numpy()
            p = 0.4 * (V[3] - 0.5 * (V[1] ** 2 + V[2] ** 2) / V[0])
            assert V[0].min() > 0 and p.min() > 0
        else:
            with pytest.raises(dg.DGError):
                S.check()
        S.close()


def test_smooth_state_gives_the_unblended_bits(env, orc):
    torch, dg = env
    dim, N, nel = 3, 3, 6
    P, S = setup(orc, dg, dim, N, nel, 2, 1)
    P0, S0 = setup(orc, dg, dim, N, nel, 2, 1, shock=False)
    xi, _ = orc.gll(N)
    X = wl.node_coordinates(dim, P.nel, P.lo, P.hi, xi)
    rho = 1.0 + 0.2 * np.sin(np.pi * X[0])
    one = np.ones_like(rho)
    U = wl.conserved(rho, [0.5 * one, 0 * one, 0 * one], one, GAMMA)
    Ud = dev(torch, U)
    assert int((S.shock_alpha(Ud)[1] > 0).sum()) == 0
    for s_ in (S, S0):
        s_.set_state(Ud)
        s_.rk_step(1e-3, 5)
    assert torch.equal(S.get_state(), S0.get_state())
    S.close()
    S0.close()


def test_unsupported_shock_choices(env, orc):
    torch, dg = env
    with pytest.raises(dg.DGError) as ei:
        dg.Solver(dg.Mesh(2, 1, (4, 4), (0.0, 0.0), (1.0, 1.0)), shock=True)
    assert ei.value.status == dg.DG_EUNSUPPORTED
    m = wl.air5_mechanism()
    with pytest.raises(dg.DGError) as ei:
        dg.Solver(dg.Mesh(3, 3, (2, 2, 2), (0.0,) * 3, (1.0,) * 3), equations=dg.DG_NS_REACTING, mu=1e-3,
                  mechanism=m, shock=True)
    assert ei.value.status == dg.DG_EUNSUPPORTED
    with pytest.raises(dg.DGError) as ei:
        dg.Solver(dg.Mesh(2, 3, (4, 4), (0.0, 0.0), (1.0, 1.0)), shock=True, alpha_min=0.6, alpha_max=0.5)
    assert ei.value.status == dg.DG_EINVAL
    meshes = [dg.Mesh(2, 3, (4, 4), (0.0, 0.0), (1.0, 1.0)), dg.Mesh(2, 3, (3, 3), (0.0, 0.0), (1.0, 1.0))]
    S = dg.Solver(meshes, shock=True)
    with pytest.raises(dg.DGError) as ei:
        S.set_launch(dg.LAUNCH_BATCHED)
    assert ei.value.status == dg.DG_EUNSUPPORTED
    U = torch.ones(S.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DGError) as ei:
        S.rhs_vjp(U, U.clone())
    assert ei.value.status == dg.DG_EUNSUPPORTED
    S.close()


def test_several_instances(env, orc):
    """Two blast instances of different size and degree in one context (per-instance
    shock-captured launches) against the oracle instance by instance."""
    torch, dg = env
    specs = [(2, 3, 10), (2, 4, 7)]
    meshes, parts, Ps = [], [], []
    for dim, N, nel in specs:
        meshes.append(dg.Mesh(dim, N, (nel, nel), (0.0, 0.0), (2.0, 2.0)))
        P = orc.Problem(dim=dim, N=N, nel=(nel, nel), lo=(0.0, 0.0), hi=(2.0, 2.0), volume=2, surface=0,
                        gamma=GAMMA, shock=True)
        Ps.append(P)
        parts.append(blast(orc, P).reshape(4, -1))
    S = dg.Solver(meshes, volume=2, surface=0, gamma=GAMMA, shock=True)
    U = np.ascontiguousarray(np.concatenate(parts, axis=1))
    got = S.rhs(torch.from_numpy(U).cuda()).cpu().numpy()
    for P, part, off in zip(Ps, parts, S.offsets):
        n = part.shape[1]
        ref = orc.rhs(P, part.reshape(P.shape))
        assert rel(got[:, off:off + n].reshape(P.shape), ref) <= 1e-12
    S.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_full_size_blast_sampled(env, orc, prec, tol):
    """The benchmark's blast workload (3D, 48^3 elements, N = 3, EC + Rusanov): one residual
    through the shock-captured launch sequence, checked on sampled elements (flagged and
    unflagged) against the oracle."""
    torch, dg = env
    dim, N, nel = 3, 3, 48
    P, S = setup(orc, dg, dim, N, nel, 2, 0, prec=prec)
    U = blast(orc, P)
    Ud = dev(torch, U)
    got = S.rhs(Ud).cpu().numpy().reshape(U.shape)
    S.check()
    oraw, oal = orc.shock_alpha(P, U)
    flagged = np.nonzero(oal)[0]
    rng = np.random.default_rng(1)
    elems = np.unique(np.concatenate([rng.choice(flagged, 40, replace=False),
                                      rng.integers(0, P.n_elem, 24), [0, P.n_elem - 1]]))
    ref = orc.rhs_elements(P, U, elems)
    assert rel(got[:, elems, :], ref) <= tol
    _, al = S.shock_alpha(Ud)
    assert np.abs(al.cpu().numpy() - oal).max() <= 1e-10
    S.close()


def test_decisions_across_the_cut(env, orc):
    """Forty elements whose smoothness E sweeps 0.05 E_min .. 20 E_min (E_min: the E where the
    sigmoid reaches alpha_min): the GPU's FP32 filter hands every element near the cut to its
    FP64 evaluation, so the cut decisions and the coefficients equal the oracle's."""
    torch, dg = env
    from numpy.polynomial import legendre as npleg
    N, n = 3, 40
    T = 0.5 * 10.0 ** (-1.8 * (N + 1) ** 0.25)
    s = math.log(9999.0)
    emin = T + T / s * math.log(0.001 / 0.999)
    Es = emin * np.geomspace(0.05, 20.0, n)
    m0 = 2.0  # mode (0, 0) of the constant 1 in 2D
    amp = m0 * np.sqrt(Es / (1.0 - Es))
    P = orc.Problem(dim=2, N=N, nel=(n, 1), lo=(0.0, 0.0), hi=(float(n), 1.0), volume=2, surface=0,
                    gamma=GAMMA, shock=True)
    S = dg.Solver(dg.Mesh(2, N, (n, 1), (0.0, 0.0), (float(n), 1.0)), volume=2, surface=0, gamma=GAMMA,
                  shock=True)
    xi, _ = orc.gll(N)
    X = wl.node_coordinates(2, P.nel, P.lo, P.hi, xi)
    e = np.floor(X[0]).astype(int).clip(0, n - 1)
    ref = 2.0 * (X[0] - e) - 1.0
    PN = npleg.legval(ref, np.eye(N + 1)[N]) * math.sqrt((2 * N + 1) / 2.0)
    p = 1.0 + amp[e] / math.sqrt(2.0) * PN
    U = wl.conserved(np.ones_like(p), [0 * p, 0 * p], p, GAMMA).reshape(P.shape)
    oraw, _ = orc.shock_alpha(P, U)
    raw, _ = S.shock_alpha(dev(torch, U))
    raw = raw.cpu().numpy()
    assert 0 < np.count_nonzero(oraw) < n
    assert np.array_equal(raw > 0, oraw > 0)
    assert np.abs(raw - oraw).max() <= 1e-10
    S.close()
