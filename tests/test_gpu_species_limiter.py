"""The Zhang-Shu limiter of the partial densities on the GPU against the oracle (Sec. 4
reacting blast set-up: rho_s >= 0 per species, after every RK stage).

- RK3 and RK54 steps of the reacting workload with negative trace densities seeded at
  random nodes: the limited steps match the oracle's (FP64 to 1e-12 per group of variables;
  FP32-mixed fluxes to 1e-6), and no partial density stays below zero in an element whose
  mean is positive;
- the two-temperature model and the Strang split take the limiter as well;
- a state without negative densities steps exactly as without the limiter."""
import numpy as np
import pytest

from paper_2605_26388_b300 import workloads as wl

pytestmark = pytest.mark.gpu

TWO_PI = 6.283185307179586


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


def groups(nv):
    g = [list(range(5)), [5, 6, 7], [8]]
    return g + ([[9]] if nv == 10 else [])


def grouped_rel(got, ref):
    out = []
    for g in groups(ref.shape[0]):
        den = np.linalg.norm(ref[g])
        out.append(np.linalg.norm(got[g] - ref[g]) / den if den > 0 else np.linalg.norm(got[g]))
    return max(out)


def negative_traces(orc, N, nel, tt=False, seed=3):
    xi, _ = orc.gll(N)
    U = wl.reacting_tgv_3d(nel, xi, wl.air5_mechanism(), two_temperature=tt).copy()
    n_el, n_nd = U.shape[1], U.shape[2]
    r = wl.uniform(seed, n_el * n_nd).reshape(n_el, n_nd)
    for s in (2, 3, 4):
        scale = 1e-4 * U[:s + 1].sum(axis=0).max() / 5
        U[s] = U[s] + np.where(r < 0.15, -scale * (1.0 + r), scale * r)
    return U


def nonnegative_where_mean_positive(orc, N, V):
    """Every element whose species mean is positive has no negative nodal value (an element
    with a negative mean holds its mean)."""
    _, w = orc.gll(N)
    W = np.einsum("i,j,k->kji", w, w, w).ravel()
    mean = V[:5] @ W / W.sum()
    low = V[:5].min(axis=2)
    tol = 1e-15 * np.abs(V[:5]).max()
    return bool(np.all((low >= -tol) | (mean <= 0)))


def setup(orc, dg, N, nel, tt=False, precision=0, p_ref=0.0, limiter=True, **kw):
    mech = wl.air5_mechanism()
    mu = wl.reacting_tgv_viscosity(mech)
    S = dg.Solver(dg.Mesh(3, N, (nel,) * 3, (0.0,) * 3, (TWO_PI,) * 3), equations=dg.DG_NS_REACTING, mu=mu,
                  prandtl=0.72, mechanism=mech, precision=precision, p_ref=p_ref, two_temperature=tt,
                  species_limiter=limiter, **kw)
    P = orc.Problem(dim=3, N=N, nel=(nel,) * 3, lo=(0.0,) * 3, hi=(TWO_PI,) * 3, equations=orc.NS_REACTING,
                    mech=mech, mu=mu, prandtl=0.72, two_temperature=tt, species_limiter=limiter)
    return S, P


@pytest.mark.parametrize("scheme", ["rk3", "rk54"])
@pytest.mark.parametrize("tt", [False, True])
def test_limited_steps_match_oracle(env, orc, scheme, tt):
    torch, dg = env
    kw = {"time_scheme": dg.SSPRK54} if scheme == "rk54" else {}
    S, P = setup(orc, dg, 3, 3, tt=tt, **kw)
    U = negative_traces(orc, 3, 3, tt=tt)
    dt = 1e-13
    S.set_state(dev(torch, U))
    S.rk_step(dt, 2)
    S.check()
    got = S.get_state().cpu().numpy().reshape(U.shape)
    ref = orc.ssp_steps(P, orc.SSPRK54 if scheme == "rk54" else orc.SSPRK33, U.copy(), dt, 2)
    assert grouped_rel(got, ref) <= 1e-12
    assert nonnegative_where_mean_positive(orc, 3, got)
    assert U[2:5].min() < 0
    S.close()


def test_full_size_limited_stage_sampled(env, orc):
    """The timed limited workload at full size (48^3 elements, N = 3, FP64, the limiter after
    every stage), with negative partial densities planted at 15% of the nodes: one SSP-RK3
    stage on sampled elements (the box's corners and 40 seeded ones) against the oracle's
    residual followed by its limiter, which is element-local and so is applied to the sampled
    elements alone (as a row of elements)."""
    torch, dg = env
    N, nel = 3, 48
    S, P = setup(orc, dg, N, nel)
    U = negative_traces(orc, N, nel)
    dt = 1e-13
    Ud = dev(torch, U)
    out = S.rk_stage(1, Ud, Ud, dt)
    S.check()
    got_all = out.cpu().numpy().reshape(U.shape)
    S.close()
    corners = [0, nel - 1, nel * (nel - 1), nel * nel - 1, nel ** 3 - 1, nel * nel * (nel - 1),
               nel * nel * (nel - 1) + nel - 1]
    elems = sorted(set(corners + [int(x * nel ** 3) for x in wl.uniform(81, 40)]))
    V = U[:, elems, :] + dt * orc.rhs_elements(P, U, elems)
    assert V[2:5].min() < 0  # the sample has work for the limiter
    Ps = orc.Problem(dim=3, N=N, nel=(len(elems), 1, 1), lo=(0.0,) * 3, hi=(TWO_PI,) * 3,
                     equations=orc.NS_REACTING, mech=P.mech, mu=P.mu, prandtl=0.72, species_limiter=1)
    ref = orc.species_limiter(Ps, V)
    got = got_all[:, elems, :]
    assert grouped_rel(got, ref) <= 1e-12
    assert nonnegative_where_mean_positive(orc, N, got)
    assert nonnegative_where_mean_positive(orc, N, got_all)


def test_fp32_mixed_limited_step(env, orc):
    torch, dg = env
    S, P = setup(orc, dg, 3, 3, precision=dg.FP32_MIXED, p_ref=101325.0)
    U = negative_traces(orc, 3, 3, seed=5)
    S.set_state(dev(torch, U))
    S.rk_step(1e-13, 2)
    S.check()
    got = S.get_state().cpu().numpy().reshape(U.shape)
    ref = orc.ssp_steps(P, orc.SSPRK33, U.copy(), 1e-13, 2)
    assert grouped_rel(got, ref) <= 1e-6
    assert nonnegative_where_mean_positive(orc, 3, got)
    S.close()


def test_split_steps_with_the_limiter(env, orc):
    torch, dg = env
    S, P = setup(orc, dg, 2, 3, chem_split=True, time_scheme=dg.SSPRK54)
    U = negative_traces(orc, 2, 3, seed=9)
    U[2:5] = np.abs(U[2:5])  # the implicit substep needs non-negative densities to start from
    dt = 1e-8
    S.set_state(dev(torch, U))
    S.rk_step(dt, 2)
    S.check()
    got = S.get_state().cpu().numpy().reshape(U.shape)
    ref, _ = orc.strang_steps(P, orc.SSPRK54, U.copy(), dt, 2)
    assert grouped_rel(got, ref) <= 1e-9
    S.close()


def test_limiter_leaves_positive_states_alone(env, orc):
    torch, dg = env
    xi, _ = orc.gll(3)
    U = wl.reacting_tgv_3d(3, xi, wl.air5_mechanism())
    outs = []
    for lim in (True, False):
        S, _ = setup(orc, dg, 3, 3, limiter=lim)
        S.set_state(dev(torch, U))
        S.rk_step(1e-13, 3)
        S.check()
        outs.append(S.get_state().cpu().numpy())
        S.close()
    assert np.array_equal(outs[0], outs[1])
