"""The N > 1 host logic on CPU: gloo ranks on 127.0.0.1.

- bench.py: the slowest rank's time is taken by every rank (max over ranks) and the
  whole-job value is all ranks' units over that time (independent replicas, weak scaling);
  the reference arm runs on rank 0 only: other ranks return without work;
- the partitioned mesh (the paper's face-only exchange, Sec. 5): each rank owns a slab of
  elements and receives only the face traces on partition faces; with them, and with every
  other foreign value poisoned (NaN), the oracle's residual on the rank's elements equals the
  single-domain residual bit for bit (2 and 3 ranks, 2D and 3D, strong and two-point volume
  forms); the exchanged volume is (N+1)^(d-1) n_v values per shared face;
- the reacting Navier-Stokes residual on the partitioned mesh (Sec. 3.1.2 BR1, Sec. 5): a
  first exchange of the state's face traces lets each rank form the BR1 gradients of its own
  elements, a second exchange of the gradients' face traces lets it form the residual; with
  both, and every other foreign value NaN, the residual equals the single-domain one bit for
  bit (single- and two-temperature air, viscous).
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms = 10.0 + 5.0 * rank                 # rank 1 is the slower one
        m = bench.max_over_ranks(ms, ws)
        v = bench.weak_value(1000.0, ws, m * 1e-3)
        assert bench.dist_env() == (ws, rank, rank)
        # the reference arm: only rank 0 would run the oracle
        class A:
            warmup, steps = 0, 0
        if rank != 0:
            assert bench.run_reference(A()) is None
        q.put((rank, m, v))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=5) for _ in range(ws))
    for rank, m, v in got:
        assert m == 15.0
        assert abs(v - 1000.0 * 2 / 15e-3) <= 1e-9 * v


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.weak_value(10.0, 1, 2.0) == 5.0


def _halo_worker(rank, ws, port, q, case):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import numpy as np
    import torch.distributed as dist
    import oracle as orc
    from paper_2605_26388_b300 import partition as pt
    from paper_2605_26388_b300 import workloads as wl
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        dim, N, nel, vol, surf = case
        lo, hi = (0.0,) * dim, (2.0,) * dim
        P = orc.Problem(dim=dim, N=N, nel=nel, lo=lo, hi=hi, volume=vol, surface=surf, gamma=1.4)
        xi, _ = orc.gll(N)
        X = wl.node_coordinates(dim, nel, lo, hi, xi)
        rho = 1.0 + 0.2 * wl.fourier_field(3, X, lo, hi, 2)
        vel = [0.3 * wl.fourier_field(4 + d, X, lo, hi, 2) for d in range(dim)]
        U = wl.conserved(rho, vel, 1.0 + 0.1 * wl.fourier_field(9, X, lo, hi, 2), 1.4).reshape(P.shape)
        parts = pt.slab_partition(nel, ws)
        own = parts[rank]
        halo = pt.shared_faces(nel, dim, parts, rank)
        Ul = np.full(P.shape, np.nan)
        Ul[:, own, :] = U[:, own, :]
        got = pt.exchange(Ul, halo, rank, ws, N, dim, dist)
        values = 0
        for p, (idx, traces) in got.items():
            pt.place_traces(Ul, halo, idx, traces, N, dim)
            values += traces.size
        Rl = orc.rhs_elements(P, Ul, own)
        Rg = orc.rhs(P, U)[:, own, :]
        ghost_elems = len(set(halo.nbr.tolist()))
        q.put((rank, bool(np.array_equal(Rl, Rg)), values, len(halo.own), ghost_elems))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws,case", [
    (2, (3, 3, (3, 2, 4), 2, 1)),   # 3D, two-point EC volume + HLLC
    (3, (3, 2, (2, 3, 3), 0, 0)),   # 3D, strong form + Rusanov, three slabs
    (2, (2, 4, (4, 4), 2, 2)),      # 2D, EC + HLL
])
def test_face_trace_exchange_reproduces_the_single_domain_residual(ws, case):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_halo_worker, args=(r, ws, port, q, case)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    dim, N, nel = case[0], case[1], case[2]
    nv = dim + 2
    for _ in range(ws):
        rank, same, values, n_faces, ghost_elems = q.get(timeout=5)
        assert same, rank
        assert values == n_faces * nv * (N + 1) ** (dim - 1)  # face-only: one trace per shared face
        assert values < ghost_elems * nv * (N + 1) ** dim      # less than whole ghost elements


def _ns_halo_worker(rank, ws, port, q, case):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import numpy as np
    import torch.distributed as dist
    import oracle as orc
    from paper_2605_26388_b300 import partition as pt
    from paper_2605_26388_b300 import workloads as wl
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        N, nel, tt = case
        dim = 3
        mech = wl.air5_mechanism()
        P = orc.Problem(dim=3, N=N, nel=(nel,) * 3, lo=(0.0,) * 3, hi=(6.283185307179586,) * 3,
                        equations=orc.NS_REACTING, mech=mech, mu=2e-3, prandtl=0.72, two_temperature=tt)
        xi, _ = orc.gll(N)
        U = wl.reacting_tgv_3d(nel, xi, mech, two_temperature=tt).reshape(P.shape)
        parts = pt.slab_partition(P.nel, ws)
        own = parts[rank]
        halo = pt.shared_faces(P.nel, dim, parts, rank)
        # exchange 1: the state's face traces
        Ul = np.full(P.shape, np.nan)
        Ul[:, own, :] = U[:, own, :]
        n1 = 0
        for p, (idx, traces) in pt.exchange(Ul, halo, rank, ws, N, dim, dist).items():
            pt.place_traces(Ul, halo, idx, traces, N, dim)
            n1 += traces.size
        # BR1 gradients of the own elements, then exchange 2: their face traces
        G = np.full((P.n_elem, P.n_nodes, 5, 3), np.nan)
        orc.br1_gradients(P, Ul, own, G)
        Gs = np.ascontiguousarray(G.reshape(P.n_elem, P.n_nodes, 15).transpose(2, 0, 1))
        n2 = 0
        for p, (idx, traces) in pt.exchange(Gs, halo, rank, ws, N, dim, dist).items():
            pt.place_traces(Gs, halo, idx, traces, N, dim)
            n2 += traces.size
        G = np.ascontiguousarray(Gs.transpose(1, 2, 0).reshape(P.n_elem, P.n_nodes, 5, 3))
        Rl = orc.rhs_elements_given_gradient(P, Ul, G, own)
        Rg = orc.rhs(P, U)[:, own, :]
        q.put((rank, bool(np.isfinite(Rl).all() and np.array_equal(Rl, Rg)), n1, n2, len(halo.own),
               P.nvars))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws,case", [
    (2, (2, 3, False)),   # single-temperature air, two slabs
    (3, (2, 3, True)),    # two-temperature air, three slabs
])
def test_two_exchanges_reproduce_the_single_domain_ns_residual(ws, case):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_ns_halo_worker, args=(r, ws, port, q, case)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    N = case[0]
    for _ in range(ws):
        rank, same, n1, n2, n_faces, nv = q.get(timeout=5)
        assert same, rank
        assert n1 == n_faces * nv * (N + 1) ** 2    # state traces
        assert n2 == n_faces * 15 * (N + 1) ** 2    # gradient traces: 5 variables x 3 directions
