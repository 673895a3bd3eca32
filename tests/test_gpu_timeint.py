"""SSP-RK54, the implicit source substep and the Strang split on the GPU (through the
C-ABI) against the oracle, plus the library's own exp and reciprocal against CUDA's.

- SSP-RK54 steps (App. B): Euler 2D/3D, strong and EC forms, FP64 (rel-L2 <= 1e-12 after
  100 steps) and FP32-mixed (<= 1e-5); batched launches bit-equal to per-instance ones;
  graph-replayed steps bit-equal to single steps; the reacting path (source in L);
  the time-step bound scaled by the scheme's SSP coefficient;
- the implicit source substep S_h (Sec. 3.1.3, Eq. source_residual) against the oracle on
  the reacting workload and against the closed-form backward-Euler solution of a
  first-order reaction; in place equals out of place; mass, momentum and energy untouched;
  a Newton budget that is too small is reported as DG_ECONVERGENCE;
- the Strang split (Eq. strang_split) with SSP-RK33 and SSP-RK54 at dt = 1e-5 s (seven
  orders of magnitude above the explicit chemical limit, below the transport bound)
  against the oracle;
- the implicit substep at the benchmark's full size on sampled nodes.
Newton stops at max |dY| <= 1e-12 rho on both sides, from Jacobians that differ in
rounding, so substep results agree to a few 1e-12 rho: the bar is 1e-10 (relative to the
species group), 1e-9 after several split steps.
"""
import copy
import math

import numpy as np
import pytest

from paper_2605_26388_b300 import workloads as wl

pytestmark = pytest.mark.gpu

GAMMA = 1.4
TWO_PI = 2.0 * math.pi


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


def rel_groups(a, b, groups):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    out = 0.0
    for g in groups:
        nb = np.linalg.norm(b[g])
        out = max(out, np.linalg.norm(a[g] - b[g]) / nb if nb > 0 else np.linalg.norm(a[g]))
    return out


def euler_groups(nv):
    return [[0], list(range(1, nv - 1)), [nv - 1]]


REACT_GROUPS = [list(range(5)), [5, 6, 7], [8]]


# ---------------------------------------------------------------------------------------------
# SSP-RK54, Euler
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("vol,surf", [(0, 0), (2, 1)])
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_rk54_vortex_100_steps(env, orc, vol, surf, prec, tol):
    torch, dg = env
    nel, N = 6, 3
    P = orc.Problem(dim=2, N=N, nel=(nel, nel), lo=(-5.0, -5.0), hi=(5.0, 5.0), volume=vol, surface=surf,
                    gamma=GAMMA)
    S = dg.Solver(dg.Mesh(2, N, (nel, nel), (-5.0, -5.0), (5.0, 5.0)), volume=vol, surface=surf,
                  precision=prec, gamma=GAMMA, time_scheme=dg.SSPRK54)
    xi, _ = orc.gll(N)
    U0 = wl.isentropic_vortex_2d(nel, xi).reshape(P.shape)
    S.set_state(dev(torch, U0))
    c54 = orc.ssp_table(54)[3]
    dt = S.max_dt(0.9)
    assert abs(dt - c54 * orc.max_dt(P, U0, 0.9)) <= 1e-14 * dt
    S.rk_step(dt, 100)
    S.check()
    got = S.get_state().cpu().numpy().reshape(P.shape)
    ref = orc.ssp_steps(P, 54, U0, dt, 100)
    err = rel_groups(got, ref, euler_groups(4))
    assert err <= tol, err
    S.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_rk54_tgv_3d(env, orc, prec, tol):
    """The 3D Taylor-Green workload's discretisation (N = 4, EC volume, HLLC) on 3^3
    elements, 40 SSP-RK54 steps at 1.5 times the SSP-RK3 test step."""
    torch, dg = env
    nel, N = 3, 4
    p_ref = 1.0 / (GAMMA * 0.01)
    P = orc.Problem(dim=3, N=N, nel=(nel,) * 3, lo=(0.0,) * 3, hi=(TWO_PI,) * 3, volume=2, surface=1,
                    gamma=GAMMA)
    S = dg.Solver(dg.Mesh(3, N, (nel,) * 3, (0.0,) * 3, (TWO_PI,) * 3), volume=2, surface=1,
                  precision=prec, gamma=GAMMA, p_ref=p_ref, time_scheme=dg.SSPRK54)
    xi, _ = orc.gll(N)
    U0 = wl.taylor_green_3d(nel, xi, 0.1, GAMMA)
    dt = 1.5 * orc.max_dt(P, U0, 0.25)
    S.set_state(dev(torch, U0))
    S.rk_step(dt, 40)
    S.check()
    got = S.get_state().cpu().numpy().reshape(U0.shape)
    ref = orc.ssp_steps(P, 54, U0, dt, 40)
    err = rel_groups(got, ref, euler_groups(5))
    assert err <= tol, err
    S.close()


def test_rk54_graph_steps_equal_single_steps(env, orc):
    torch, dg = env
    nel, N = 5, 4
    S = dg.Solver(dg.Mesh(2, N, (nel, nel), (-5.0, -5.0), (5.0, 5.0)), volume=2, surface=1, gamma=GAMMA,
                  time_scheme=dg.SSPRK54)
    xi, _ = orc.gll(N)
    U0 = dev(torch, wl.isentropic_vortex_2d(nel, xi))
    S.set_state(U0)
    S.rk_step(0.02, 7)  # two graph replays of three steps and one single step
    a = S.get_state().clone()
    S.set_state(U0)
    for _ in range(7):
        S.rk_step(0.02, 1)
    S.check()
    assert torch.equal(S.get_state(), a)
    S.close()


def test_rk54_batched_equals_per_instance_and_oracle(env, orc):
    torch, dg = env
    specs = [(5, 2, (0.3, -0.2)), (3, 5, (-1.0, 0.5)), (7, 3, (0.0, 0.0)), (4, 4, (1.1, 1.2)), (1, 3, (0.2, 0.1))]
    meshes, parts = [], []
    for nel, N, c in specs:
        meshes.append(dg.Mesh(2, N, (nel, nel), (-5.0, -5.0), (5.0, 5.0)))
        xi, _ = orc.gll(N)
        parts.append(wl.isentropic_vortex_2d(nel, xi, center=c).reshape(4, -1))
    U = np.ascontiguousarray(np.concatenate(parts, axis=1))
    S = dg.Solver(meshes, volume=2, surface=0, gamma=GAMMA, time_scheme=dg.SSPRK54)
    U0 = torch.from_numpy(U).cuda()
    dt = 3e-3
    S.set_launch(dg.LAUNCH_PER_INSTANCE)
    S.set_state(U0)
    S.rk_step(dt, 30)
    ref_dev = S.get_state().clone()
    S.set_launch(dg.LAUNCH_BATCHED, 1, 0, 0)
    S.set_state(U0)
    S.rk_step(dt, 30)
    S.check()
    assert torch.equal(S.get_state(), ref_dev)
    got = ref_dev.cpu().numpy()
    for (nel, N, c), off in zip(specs, S.offsets):
        P = orc.Problem(dim=2, N=N, nel=(nel, nel), lo=(-5.0, -5.0), hi=(5.0, 5.0), volume=2, surface=0,
                        gamma=GAMMA)
        n = nel * nel * (N + 1) ** 2
        ref = orc.ssp_steps(P, 54, U[:, off:off + n].reshape(P.shape), dt, 30)
        assert rel_groups(got[:, off:off + n].reshape(P.shape), ref, euler_groups(4)) <= 1e-12
    S.close()


def test_split_needs_chemistry_and_the_scheme_is_checked(env, orc):
    torch, dg = env
    mesh = dg.Mesh(2, 3, (2, 2), (0.0, 0.0), (1.0, 1.0))
    for kw in ({"chem_split": True}, {"time_scheme": 7}):
        with pytest.raises(dg.DGError) as ei:
            dg.Solver(mesh, gamma=GAMMA, **kw)
        assert ei.value.status == dg.DG_EINVAL


# ---------------------------------------------------------------------------------------------
# Reacting: SSP-RK54 with the source in L, the implicit substep, the Strang split
# ---------------------------------------------------------------------------------------------
def reacting(orc, dg, nel, N, mech, mu, prec=0, p_ref=0.0, **kw):
    S = dg.Solver(dg.Mesh(3, N, (nel,) * 3, (0.0,) * 3, (TWO_PI,) * 3), equations=dg.DG_NS_REACTING, mu=mu,
                  prandtl=0.72, mechanism=mech, precision=prec, p_ref=p_ref, **kw)
    P = orc.Problem(dim=3, N=N, nel=(nel,) * 3, lo=(0.0,) * 3, hi=(TWO_PI,) * 3, equations=orc.NS_REACTING,
                    mech=mech, mu=mu, prandtl=0.72)
    return S, P


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-6)])
def test_reacting_rk54_with_source_in_the_residual(env, orc, prec, tol):
    torch, dg = env
    mech = wl.air5_mechanism()
    mu = wl.reacting_tgv_viscosity(mech)
    S, P = reacting(orc, dg, 3, 3, mech, mu, prec=prec, p_ref=101325.0 if prec else 0.0,
                    time_scheme=dg.SSPRK54)
    xi, _ = orc.gll(3)
    U = wl.reacting_tgv_3d(3, xi, mech)
    dt = 1e-12
    S.set_state(dev(torch, U))
    S.rk_step(dt, 50)
    S.check()
    got = S.get_state().cpu().numpy().reshape(U.shape)
    ref = orc.ssp_steps(P, 54, U, dt, 50)
    assert rel_groups(got, ref, REACT_GROUPS) <= tol
    assert np.abs(got[:5] - U[:5]).max() > 0.0
    S.close()


@pytest.mark.parametrize("h", [1e-12, 1e-9, 1e-6])
@pytest.mark.parametrize("prec", [0, 1])
def test_source_step_matches_oracle(env, orc, h, prec):
    torch, dg = env
    mech = wl.air5_mechanism()
    S, P = reacting(orc, dg, 3, 3, mech, 0.0, prec=prec, chem_split=True)
    xi, _ = orc.gll(3)
    U = wl.reacting_tgv_3d(3, xi, mech)
    Ud = dev(torch, U)
    out = S.source_step(Ud, h)
    S.check()
    ref, it = orc.source_implicit(P, U, h)
    assert it > 0
    n_nodes = U.shape[1] * U.shape[2]
    updates = S.newton_updates()
    assert n_nodes <= updates <= it * n_nodes + n_nodes  # every node takes at least one update
    assert S.newton_updates() == 0                       # the count was reset
    got = out.cpu().numpy().reshape(U.shape)
    rho = U[:5].sum(axis=0)
    assert np.abs(got[:5] - ref[:5]).max() <= 1e-10 * rho.max()
    assert np.array_equal(got[5:], U[5:])
    assert np.abs(got[:5].sum(axis=0) - rho).max() <= 1e-14 * rho.max()
    # in place gives the same bits
    inplace = Ud.clone()
    S.source_step(inplace, h, out=inplace)
    S.check()
    assert torch.equal(inplace, out)
    S.close()


def test_source_step_first_order_closed_form(env, orc):
    """N2 -> 2N at a constant rate k: rho_N2 / (1 + h k) on the GPU, without the oracle."""
    torch, dg = env
    k = 2.0e5
    m = copy.deepcopy(wl.air5_mechanism())
    m.update({"n_reactions": 1, "lnA": [math.log(k)], "b": [0.0], "Ta": [0.0],
              "kc": [[0.0, 600.0, 0.0, 0.0, 0.0]], "nu_f": [[1, 0, 0, 0, 0]], "nu_b": [[0, 0, 0, 2, 0]],
              "h0": [0.0] * 5})
    S = dg.Solver(dg.Mesh(3, 2, (2, 2, 2), (0.0,) * 3, (1.0,) * 3), equations=dg.DG_NS_REACTING, mu=0.0,
                  mechanism=m, chem_split=True)
    n = S.n_nodes
    rng = np.random.default_rng(3)
    rho = [rng.uniform(0.05, 0.3, n), np.full(n, 0.1), np.full(n, 1e-3), rng.uniform(0.0, 0.05, n),
           np.full(n, 0.02)]
    U = wl.reacting_conserved(rho, [np.full(n, 30.0)] * 3, rng.uniform(2000.0, 6000.0, n), m)
    for h in (1e-6, 1e-4):
        got = S.source_step(dev(torch, U), h).cpu().numpy()
        S.check()
        n2 = rho[0] / (1.0 + h * k)
        assert np.abs(got[0] - n2).max() <= 1e-12 * rho[0].max()
        assert np.abs(got[3] - (rho[3] + h * k * n2)).max() <= 1e-12 * rho[0].max()
    S.close()


def test_newton_budget_exhaustion_is_reported(env, orc):
    torch, dg = env
    mech = wl.air5_mechanism()
    S, P = reacting(orc, dg, 2, 2, mech, 0.0, chem_split=True, newton_max_it=1)
    xi, _ = orc.gll(2)
    U = dev(torch, wl.reacting_tgv_3d(2, xi, mech))
    S.source_step(U, 1e-7)
    with pytest.raises(dg.DGError) as ei:
        S.check()
    assert ei.value.status == dg.DG_ECONVERGENCE
    S.check()  # the error word was cleared
    S.close()


@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-6)])
def test_strang_split_at_a_large_step(env, orc, scheme, prec, tol):
    torch, dg = env
    mech = wl.air5_mechanism()
    mu = wl.reacting_tgv_viscosity(mech)
    S, P = reacting(orc, dg, 3, 3, mech, mu, prec=prec, p_ref=101325.0 if prec else 0.0,
                    time_scheme=scheme, chem_split=True)
    xi, _ = orc.gll(3)
    U = wl.reacting_tgv_3d(3, xi, mech)
    S.set_state(dev(torch, U))
    dt = 1e-5  # far above the explicit chemical limit (~1e-12 s), below the transport bound
    assert S.max_dt(1.0) > dt
    S.rk_step(dt, 3)
    S.check()
    got = S.get_state().cpu().numpy().reshape(U.shape)
    ref, it = orc.strang_steps(P, 54 if scheme else 3, U, dt, 3)
    assert it > 0
    assert rel_groups(got, ref, REACT_GROUPS) <= tol
    assert np.all(got[:5] > 0)
    S.close()


def test_source_step_full_size_sampled(env, orc):
    """The benchmark's split workload (32^3 elements, N = 3, h = 5e-6 s, half the split step):
    the substep over all 2.1 M nodes, checked against the oracle on sampled nodes."""
    torch, dg = env
    mech = wl.air5_mechanism()
    nel, N = 32, 3
    S, _ = reacting(orc, dg, nel, N, mech, wl.reacting_tgv_viscosity(mech), chem_split=True,
                    time_scheme=dg.SSPRK54)
    xi, _ = orc.gll(N)
    U = wl.reacting_tgv_3d(nel, xi, mech).reshape(9, -1)
    Ud = dev(torch, U)
    h = 5e-6
    out = S.source_step(Ud, h)
    S.check()
    got = out.cpu().numpy()
    rng = np.random.default_rng(11)
    idx = np.unique(np.concatenate([[0, U.shape[1] - 1], rng.integers(0, U.shape[1], 510)]))[:512]
    idx = np.resize(idx, 512)
    # the sampled nodes as a 8 x 8 x 1 mesh of N = 1 elements (the substep is node-local)
    Pn = orc.Problem(dim=3, N=1, nel=(8, 8, 1), lo=(0.0,) * 3, hi=(1.0,) * 3, equations=orc.NS_REACTING,
                     mech=mech, mu=0.0)
    ref, it = orc.source_implicit(Pn, np.ascontiguousarray(U[:, idx]).reshape(Pn.shape), h)
    assert it > 0
    ref = ref.reshape(9, -1)
    rho = U[:5, idx].sum(axis=0)
    assert np.abs(got[:5, idx] - ref[:5]).max() <= 1e-10 * rho.max()


# ---------------------------------------------------------------------------------------------
# The library's own math routines against CUDA's
# ---------------------------------------------------------------------------------------------
def test_table_exp_and_newton_reciprocal_against_cuda(env):
    torch, dg = env
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.uniform(-703.0, 703.0, 200000), rng.uniform(-40.0, 40.0, 200000),
                        rng.uniform(-1e-3, 1e-3, 20000),
                        [0.0, -0.0, 1e-300, -1e-300, math.log(2.0) / 128, 703.9, -703.9, 704.0, -704.0,
                         709.7, -745.0, 800.0, -800.0]])
    xd = torch.from_numpy(x).cuda()
    mine = dg.math_fn(dg.MATH_EXP_TABLE, xd).cpu().numpy()
    cuda = dg.math_fn(dg.MATH_EXP_CUDA, xd).cpu().numpy()
    fin = np.isfinite(cuda) & (cuda > 2.3e-308)
    rel = np.abs(mine[fin] - cuda[fin]) / cuda[fin]
    assert rel.max() <= 3 * 2.0 ** -52, rel.max()
    assert np.array_equal(mine[~fin], cuda[~fin])
    # reciprocal: Newton from an FP32 seed against the correctly rounded quotient
    y = np.concatenate([10.0 ** rng.uniform(-37.0, 37.0, 200000) * rng.choice([-1.0, 1.0], 200000),
                        [1.0, -1.0, 3.0, 1e-300, 1e300, 0.0, -0.0, np.inf, 2.0 ** -126, 2.0 ** 126]])
    yd = torch.from_numpy(y).cuda()
    r_mine = dg.math_fn(dg.MATH_RCP_NEWTON, yd).cpu().numpy()
    r_cuda = dg.math_fn(dg.MATH_RCP_CUDA, yd).cpu().numpy()
    ok = np.isfinite(r_cuda) & (r_cuda != 0)
    rel = np.abs(r_mine[ok] - r_cuda[ok]) / np.abs(r_cuda[ok])
    assert rel.max() <= 2 * 2.0 ** -52, rel.max()
    assert np.array_equal(r_mine[~ok], r_cuda[~ok])
