"""Benchmark: RK-stage DOF-updates/s of the fused DGSEM stage on one B300.

Workload (the 3D Taylor-Green case): compressible Euler, DGSEM N = 4 (125 GLL nodes per
element), 64^3 periodic elements on [0, 2pi]^3, Taylor-Green vortex at Ma = 0.1,
Ranocha two-point flux-differencing volume term, HLLC surface flux, SSP-RK3 with a fixed
dt from the time-step bound at CFL 0.25 (CFL 0.5 is unstable in 3D).  163,840,000 DOF; a step is one SSP-RK3 step (3 fused stage
launches) = 491,520,000 DOF-updates.  The headline runs the FP32-flux / FP64-state path;
the plain FP64 path is measured beside it.

Timing: W untimed warm-up steps, then K steps replayed from a CUDA graph, bracketed by
CUDA events on the solver's stream with a device synchronize (and a barrier under
torchrun) on both sides.  The three 1.31 GB state buffers exceed the 126 MB L2, so no
flush is needed between steps.  Multi-GPU: independent replicas (the path has no data
exchange on one box), value = all ranks' DOF-updates / max time.

`--impl reference` times the plain CPU oracle (the only other place this script runs
oracle code) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NEL, N, GAMMA, MACH, CFL = 64, 4, 1.4, 0.1, 0.25
NV = 5
NP = (N + 1) ** 3
DOF = NEL ** 3 * NP * NV
BYTES_PER_DOF_UPDATE = (16 + 24 + 24) / 3.0  # stage 1 reads U^n, writes U^1; stages 2-3 read 2, write 1
WORKLOAD = "tgv3d_euler_N4_64cube_ec_hllc_ssprk3"
P_REF = 1.0 / (GAMMA * MACH ** 2)  # background pressure; the momentum flux carries p - P_REF
METRIC = "RK-stage DOF-updates/s (3D Euler DGSEM N=4, TGV Ma 0.1, EC flux differencing + HLLC; FP32-mixed vs FP64)"


def workload_config(nel, ws=1):
    """The `config` object of both arms (the workload, not a model)."""
    return {"workload": WORKLOAD if nel == 64 else f"{WORKLOAD} (profiling size {nel}^3)",
            "mesh": f"{nel}^3 periodic on [0,2pi]^3", "N": N, "dof": nel ** 3 * NP * NV,
            "cfl": CFL, "p_ref": P_REF,
            "l2": "inputs larger than L2: three state buffers of %.2f GB per replica" % (nel ** 3 * NP * NV * 8 / 1e9),
            "parallelism": f"replicas x{ws}"}

# Figures from ncu captures of the stage kernels, valid only for the kernel sources they were
# taken on: keyed by a hash of those sources (kernel_hash), and reported as null when the
# sources have changed since.  traffic_*: dram__bytes_read.sum + dram__bytes_write.sum per
# stage launch at 64^3 (mean of stages 1-3, one 1-pass capture of the full workload);
# fp64_instr: FP64 thread instructions (DFMA + DADD + DMUL) per FP64 stage launch at 64^3
# (a 32^3 capture scaled by the element count).  The commands are in profiles/.
KERNEL_SOURCES = ["dg_stage_ec3.cuh", "dg_stage.cuh", "dg_device.cuh", "dg_internal.h", "dg_stage3d.cu"]
BATCHED_SOURCES = ["dg_batched.cuh", "dg_stage.cuh", "dg_device.cuh", "dg_internal.h", "dg_batched2d.cu"]
NCU_FIGURES = {
    "35e12d0919ca11f5": {"traffic_fp32_mixed": 4.007e9, "traffic_fp64": 3.820e9, "fp64_instr": 1.6906e10},
    # the batched kernel on the 256-instance workload (BATCHED_SOURCES), group scale 1
    "9e7e12d0d272fdad": {"traffic_batched": 1.645e9},
}


def kernel_hash(sources=None):
    """Hash of a kernel's code (default: the headline stage kernel): its sources with comments
    and blank lines removed, so that an edit of a comment does not retire the ncu figures
    taken of the same code."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in sources or KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2605_26388_b300", "csrc", f)) as fh:
            text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        for line in text.splitlines():
            line = line.split("//", 1)[0].rstrip()
            if line:
                h.update(line.encode() + b"\n")
    return h.hexdigest()[:16]


def ncu_figure(key, sources=None):
    return NCU_FIGURES.get(kernel_hash(sources), {}).get(key)


def alu_peaks():
    """Measured thread-level rates of FP64 and FP32 fused multiply-adds on this GPU
    (dg_alu_rate: independent chains, CUDA events, best of three; no clock changes)."""
    import ctypes as C
    from paper_2605_26388_b300 import dgsem
    out = {}
    for kind, name in ((0, "fp64_fma_g_per_s"), (2, "fp32_fma_g_per_s")):
        r = C.c_double()
        st = dgsem.lib().dg_alu_rate(kind, C.byref(r))
        out[name] = r.value / 1e9 if st == dgsem.DG_OK else None
    out["how"] = "dg_alu_rate: 8 CTAs x 256 threads per SM of independent FMA chains, best of 3 launches"
    return out


def fp64_pipe(launch_ms, peak_g):
    """Executed FP64 instructions per second of the FP64 stage kernel against the measured
    FP64 FMA rate (each FP64 instruction counted once)."""
    instr = ncu_figure("fp64_instr")
    if instr is None or not peak_g:
        return None
    ach = instr / (launch_ms * 1e-3) / 1e9
    return {"bound": "alu", "unit": "G FP64 instr/s", "achieved": ach, "peak": peak_g, "frac": ach / peak_g,
            "peak_kind": "measured (dg_alu_rate, FP64 FMA)", "instr_per_launch": instr,
            "note": "executed FP64 instructions from ncu (not algorithmic flops)"}


# FP64 instructions (thread level: DFMA + DADD + DMUL) per Newton update of
# k_source_implicit<5,double>, from an ncu capture of one substep on the 12^3 split workload
# (2.054e9 instructions over 442003 updates); the implicit-substep kernel is unchanged since.
FP64_INSTR_PER_NEWTON_UPDATE = 2.054e9 / 442003
SPLIT_DT = 1e-5          # the split workload's step (s)
EXPLICIT_DT = 1e-13      # the explicit source's stable step on the same mechanism (s)


ALU = None  # measured ALU rates (alu_peaks), set by main


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int) -> float:
    """The largest x over all ranks of the initialised process group (x itself for one
    rank); the device of the reduction follows the backend (CUDA for NCCL, host for gloo)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(units_per_rank: float, ws: int, seconds: float) -> float:
    """Whole-job throughput of N independent replicas: all ranks' units / slowest rank's time."""
    return units_per_rank * ws / seconds


ACC_NEL, ACC_STEPS = 4, 100  # the accuracy workload: the same TGV problem on 4^3, 100 steps


def accuracy_states():
    """The accuracy workload on the GPU in both precisions: the TGV N=4 EC+HLLC problem on
    4^3 elements, 100 SSP-RK3 steps at the CFL 0.25 bound; returns (U0, dt, {precision:
    final state}) for the CPU-baseline leg to compare with the oracle."""
    import torch
    from paper_2605_26388_b300 import dgsem, workloads as wl
    x, _, _ = dgsem.gll(N)
    U0 = wl.taylor_green_3d(ACC_NEL, x, MACH, GAMMA)
    out, dt = {}, None
    for name, prec in (("fp64", dgsem.FP64), ("fp32_mixed", dgsem.FP32_MIXED)):
        S = dgsem.Solver(dgsem.Mesh(3, N, (ACC_NEL,) * 3, (0.0,) * 3, (2 * math.pi,) * 3), volume=dgsem.VOL_EC,
                         surface=dgsem.SURF_HLLC, precision=prec, gamma=GAMMA, p_ref=P_REF)
        S.set_state(torch.from_numpy(np.ascontiguousarray(U0.reshape(NV, -1))).cuda())
        dt = S.max_dt(CFL)
        S.rk_step(dt, ACC_STEPS)
        S.check()
        out[name] = S.get_state().cpu().numpy().reshape(U0.shape)
        S.close()
    return U0, dt, out


def _groups(a, b):
    a = np.asarray(a).reshape(NV, -1)
    b = np.asarray(b).reshape(NV, -1)
    return [float(np.linalg.norm(a[g] - b[g]) / np.linalg.norm(b[g])) for g in ([0], [1, 2, 3], [4])]


def oracle_sample(acc=None, seconds_hint: float = 8.0, single_core_hint: float = 4.0):
    """The CPU-baseline leg: the plain FP64 oracle on bounded samples of the same workload.
    (1) The accuracy workload (4^3, 100 SSP-RK3 steps), whose result is the reference of the
    GPU states in acc (per-group relative L2 of the final state and of the increment U_T - U_0,
    mass / momentum / energy).  (2) Full SSP-RK3 steps of the same problem on a 12^3 sub-mesh
    for about seconds_hint on all host cores, then (3) for about single_core_hint on one core
    (the OpenMP element loop restricted to one thread; same arithmetic)."""
    import ctypes as C
    import oracle
    from paper_2605_26388_b300 import workloads as wl
    oracle.build()
    xi, _ = oracle.gll(N)
    accuracy = None
    if acc is not None:
        U0, dt_acc, states = acc
        P4 = oracle.Problem(dim=3, N=N, nel=(ACC_NEL,) * 3, lo=(0.0,) * 3, hi=(2 * math.pi,) * 3,
                            volume=oracle.VOL_EC, surface=oracle.SURF_HLLC, gamma=GAMMA)
        t0 = time.perf_counter()
        ref = oracle.rk3(P4, U0, dt_acc, ACC_STEPS)
        t_acc = time.perf_counter() - t0
        accuracy = {"workload": f"TGV N=4 EC+HLLC on {ACC_NEL}^3, {ACC_STEPS} SSP-RK3 steps at CFL {CFL}, "
                                "vs the FP64 CPU oracle; relative L2 per group [mass, momentum, energy]",
                    "oracle_s": t_acc}
        for name, Ug in states.items():
            accuracy[name] = {"state": _groups(Ug, ref), "increment": _groups(Ug - U0, ref - U0)}
    nel = 12
    P = oracle.Problem(dim=3, N=N, nel=(nel,) * 3, lo=(0.0,) * 3, hi=(2 * math.pi,) * 3,
                       volume=oracle.VOL_EC, surface=oracle.SURF_HLLC, gamma=GAMMA)
    U = wl.taylor_green_3d(nel, xi, MACH, GAMMA)
    dt = oracle.max_dt(P, U, CFL)
    dof = nel ** 3 * NP * NV

    def timed(hint):
        nonlocal U
        steps, t0 = 0, time.perf_counter()
        while True:
            U = oracle.rk3(P, U, dt, 1)
            steps += 1
            if time.perf_counter() - t0 >= hint:
                return steps, time.perf_counter() - t0

    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    steps, el = timed(seconds_hint)
    single = None
    try:
        gomp = C.CDLL("libgomp.so.1")
        gomp.omp_set_num_threads(1)
        s1, el1 = timed(single_core_hint)
        gomp.omp_set_num_threads(cores)
        single = {"value": 3 * s1 * dof / el1, "unit": "DOF-updates/s", "cores": 1,
                  "sample": f"{s1} step(s) on the {nel}^3 sub-mesh, {el1:.1f} s"}
    except OSError:
        pass
    return {"value": 3 * steps * dof / el, "unit": "DOF-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"{steps} SSP-RK3 step(s) of the same TGV N=4 EC+HLLC problem on a {nel}^3 sub-mesh "
                      f"({dof} DOF), FP64, {el:.1f} s",
            "single_core": single}, accuracy


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    per_step = []
    total_dof_updates, t_all = 0.0, 0.0
    import oracle
    from paper_2605_26388_b300 import workloads as wl
    oracle.build()
    nel = 8
    P = oracle.Problem(dim=3, N=N, nel=(nel,) * 3, lo=(0.0,) * 3, hi=(2 * math.pi,) * 3,
                       volume=oracle.VOL_EC, surface=oracle.SURF_HLLC, gamma=GAMMA)
    xi, _ = oracle.gll(N)
    U = wl.taylor_green_3d(nel, xi, MACH, GAMMA)
    dt = oracle.max_dt(P, U, CFL)
    for _ in range(args.warmup):
        U = oracle.rk3(P, U, dt, 1)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        U = oracle.rk3(P, U, dt, 1)
        per_step.append(time.perf_counter() - t0)
    dof = nel ** 3 * NP * NV
    t_all = sum(per_step)
    value = 3 * dof * args.steps / t_all
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC,
            "value": value, "unit": "DOF-updates/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(NEL, 1),
            "cpu_baseline": {"value": value, "unit": "DOF-updates/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step: one SSP-RK3 step of the same problem on a {nel}^3 "
                                       f"sub-mesh ({dof} DOF), FP64, on the host cores; {args.steps} steps"},
            "e2e": {"value": value, "unit": "DOF-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    global NEL, DOF, ALU
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=None)
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-reacting", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--only", default="both", choices=["both", "fp32", "fp64", "reacting", "split", "shock", "curved", "batched", "adjoint"],
                    help="precision(s) to time, or one secondary workload alone (profiling runs)")
    ap.add_argument("--reacting-nel", type=int, default=48,
                    help="elements per direction of the reacting workload (profiling runs)")
    ap.add_argument("--no-split", action="store_true")
    ap.add_argument("--no-shock", action="store_true")
    ap.add_argument("--no-curved", action="store_true")
    ap.add_argument("--shock-nel", type=int, default=48,
                    help="elements per direction of the blast (shock-capturing) workload")
    ap.add_argument("--split-nel", type=int, default=32,
                    help="elements per direction of the split (implicit chemistry) workload")
    ap.add_argument("--nel", type=int, default=NEL, help="elements per direction (profiling runs)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
        return
    if args.only in ("reacting", "split", "shock", "curved", "batched", "adjoint"):
        import torch
        torch.cuda.set_device(dist_env()[2])
        ALU = alu_peaks()
        fn = {"reacting": run_reacting, "split": run_split, "shock": run_shock, "curved": run_curved,
              "batched": run_batched, "adjoint": run_adjoint}[args.only]
        print(json.dumps({args.only: fn(args)}), flush=True)
        return

    import torch
    NEL = args.nel
    DOF = NEL ** 3 * NP * NV
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    from paper_2605_26388_b300 import build, dgsem, workloads as wl
    build.build_library()
    x, w, _ = dgsem.gll(N)
    U0 = wl.taylor_green_3d(NEL, x, MACH, GAMMA).reshape(NV, -1)
    U0_dev = torch.from_numpy(U0).cuda()
    peak, peak_kind = measured_peaks()

    def run(precision, steps, warmup):
        S = dgsem.Solver(dgsem.Mesh(3, N, (NEL,) * 3, (0.0,) * 3, (2 * math.pi,) * 3), volume=dgsem.VOL_EC,
                         surface=dgsem.SURF_HLLC, precision=precision, gamma=GAMMA, p_ref=P_REF)
        S.set_state(U0_dev)
        dt = S.max_dt(CFL)
        S.rk_step(dt, warmup)
        S.check()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            torch.cuda.synchronize()
            barrier()
            e0.record(stream)
            S.rk_step(dt, steps)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
        S.check()
        ms = max_over_ranks(e0.elapsed_time(e1), ws)
        return S, dt, ms, clk.summary()

    fp64_steps = args.fp64_steps or max(3, args.steps // 10)
    ms32 = ms64 = None
    clk32 = clk64 = None
    if args.only in ("both", "fp32"):
        S32, dt, ms32, clk32 = run(dgsem.FP32_MIXED, args.steps, args.warmup)
        S32.close()
    if args.only in ("both", "fp64"):
        S64, dt, ms64, clk64 = run(dgsem.FP64, fp64_steps, 3)
        S64.close()

    def roofline(ms, steps, prec):
        launch_ms = ms / (3 * steps)
        alg = BYTES_PER_DOF_UPDATE * DOF  # algorithmic bytes per average launch
        ach = alg / (launch_ms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": ncu_figure("traffic_" + prec) if NEL == 64 else None, "peak_kind": peak_kind,
                "kernel": "k_euler_ec3<4," + ("float" if prec == "fp32_mixed" else "double") + ",1|2> (plain SSP-RK3 stage, periodic HLLC)",
                "avg_launch_ms": launch_ms, "alg_bytes_per_launch": alg, "kernel_hash": kernel_hash()}

    value = weak_value(3 * DOF * args.steps, ws, ms32 * 1e-3) if ms32 else None
    if args.no_e2e or ms32 is None:
        e2e = None
    else:
        e2e = run_e2e(args, U0, dt, ws, barrier)
    if rank != 0:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    ALU = alu_peaks()
    cpu = accuracy = None
    if not args.no_cpu_baseline and ws == 1:
        cpu, accuracy = oracle_sample(accuracy_states())
    batched = None if args.no_batched else run_batched(args)
    reacting = None if args.no_reacting else run_reacting(args)
    split = None if args.no_split else run_split(args)
    shock = None if args.no_shock else run_shock(args)
    curved = None if args.no_curved else run_curved(args)
    adjoint = None if args.no_adjoint else run_adjoint(args)
    fp64 = None
    if ms64:
        r64 = roofline(ms64, fp64_steps, "fp64")
        fp64 = {"value": weak_value(3 * DOF * fp64_steps, ws, ms64 * 1e-3), "unit": "DOF-updates/s", "steps": fp64_steps,
                "ms_per_step": ms64 / fp64_steps, "hbm_frac": r64["frac"], "avg_launch_ms": r64["avg_launch_ms"],
                "traffic": r64["traffic"], "bound_note": "FP64-pipe bound on B300",
                "fp64_pipe": fp64_pipe(ms64 / (3 * fp64_steps), ALU.get("fp64_fma_g_per_s")),
                "clocks": clk64}
    line = {
        "metric": METRIC,
        "value": value, "unit": "DOF-updates/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms32 / args.steps if ms32 else None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 flux / f64 state", "data": "synthetic",
        "config": dict(workload_config(NEL, ws), precision="fp32_mixed", dt=dt),
        "roofline": roofline(ms32, args.steps, "fp32_mixed") if ms32 else None,
        "clocks": clk32 if clk32 else clk64,
        "e2e": e2e,
        "gpu_launches": 3 * args.steps,
        "cpu_baseline": cpu,
        "batched": batched,
        "reacting": reacting,
        "reacting_split": split,
        "shock": shock,
        "curved": curved,
        "adjoint": adjoint,
        # last, so that a tail of the output keeps them: the paper-precision arm, the accuracy
        # of both arms and the measured ALU peaks
        "alu_peaks": ALU,
        "accuracy": accuracy,
        "fp64": fp64,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_batched(args):
    """The batched workload: 256 independent 2D Euler instances (isentropic vortex, seeded
    sizes 8^2..96^2 elements and degrees N in {2,3,4,5}), strong form + Rusanov,
    FP32-mixed.  Times K SSP-RK3 steps for per-instance launches, the default batched
    launch and the autotuned configuration (all replayed from CUDA graphs)."""
    import torch
    from paper_2605_26388_b300 import dgsem, workloads as wl
    specs = wl.batched_vortex_set(256, seed=5)
    meshes, parts = [], []
    for nel, Nd, c in specs:
        meshes.append(dgsem.Mesh(2, Nd, (nel, nel), (-5.0, -5.0), (5.0, 5.0)))
        x, _, _ = dgsem.gll(Nd)
        parts.append(wl.isentropic_vortex_2d(nel, x, center=c).reshape(4, -1))
    U = torch.from_numpy(np.ascontiguousarray(np.concatenate(parts, axis=1))).cuda()
    S = dgsem.Solver(meshes, volume=dgsem.VOL_STRONG, surface=dgsem.SURF_RUSANOV,
                     precision=dgsem.FP32_MIXED, gamma=GAMMA)
    S.set_state(U)
    dt = S.max_dt(0.5)
    dof = S.n_doubles
    steps = max(3, args.steps // 3)
    out = {"workload": "256 x 2D Euler isentropic vortex, nel in [8,96], N in {2..5}, strong + Rusanov, FP32-mixed",
           "instances": len(meshes), "elements": sum(m.n_elem for m in meshes), "dof": dof, "steps": steps}
    peak, peak_kind = measured_peaks()

    def timed(label):
        S.set_state(U)
        S.rk_step(dt, 3)
        S.check()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        S.rk_step(dt, steps)
        e1.record()
        torch.cuda.synchronize()
        S.check()
        ms = e0.elapsed_time(e1) / steps
        ach = BYTES_PER_DOF_UPDATE * dof / (ms / 3 * 1e-3) / 1e9  # per stage, all instances
        out[label] = {"ms_per_step": ms, "value": 3 * dof / (ms * 1e-3), "unit": "DOF-updates/s",
                      "hbm_frac": ach / peak}
        return ms, ach

    S.set_launch(dgsem.LAUNCH_PER_INSTANCE)
    timed("per_instance")
    S.set_launch(dgsem.LAUNCH_BATCHED, 1, 0, 0)
    timed("batched_default")
    # group scale 2 for every degree, and per degree (a second launch per stage for the
    # degrees with scale 2): the low degrees, the high degrees
    per_degree = {}
    for label, gsv in (("all_2", 2), ("N2_N3_at_2", dgsem.GROUPS_PER_DEGREE | (1 << 2) | (1 << 3)),
                       ("N4_N5_at_2", dgsem.GROUPS_PER_DEGREE | (1 << 4) | (1 << 5))):
        S.set_launch(dgsem.LAUNCH_BATCHED, gsv, 0, 0)
        ms_g, _ = timed("_tmp")
        per_degree[label] = {"ms_per_step": ms_g, "value": out.pop("_tmp")["value"]}
    out["per_degree"] = per_degree
    S.set_state(U)
    cfg, _ = S.autotune(dt, 3)
    gs = cfg[1]
    if gs & dgsem.GROUPS_PER_DEGREE:  # per-degree choice: degree N uses 2 where bit N is set
        gs = {str(n): 2 if (gs >> n) & 1 else 1 for n in sorted({m.N for m in meshes})}
    out["autotuned_config"] = {"mode": cfg[0], "group_scale": gs, "ctas_per_sm": cfg[2], "order": cfg[3]}
    ms, ach = timed("batched_autotuned")
    # the stage launch of the configuration the autotuner keeps: the same algorithmic bytes per
    # DOF-update as the headline stage (stage 1 reads U^n and writes U^1, stages 2-3 read two
    # states and write one), over the mean of the three stage launches of a step
    out["roofline"] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                       "peak_kind": peak_kind,
                       "kernel": "k_euler_stage_batched<2,strong,float>" if cfg[0] == dgsem.LAUNCH_BATCHED
                       else "k_euler_stage<2,N,strong,float> per instance",
                       "avg_launch_ms": ms / 3, "alg_bytes_per_launch": BYTES_PER_DOF_UPDATE * dof,
                       "traffic": ncu_figure("traffic_batched", BATCHED_SOURCES) if cfg[0] == dgsem.LAUNCH_BATCHED
                       and cfg[1] == 1 else None, "kernel_hash": kernel_hash(BATCHED_SOURCES)}
    S.close()
    return out


def run_reacting(args):
    """The reacting workload: 3D Navier-Stokes with 5-species air, N = 3, 48^3 elements,
    9 conserved variables, BR1 viscous terms (Re = 1600, Pr = 0.72), 17 seeded Arrhenius
    reactions evaluated in FP64, Rusanov surface flux, FP64 throughout.  dt = 1e-13 s keeps
    the explicit source below the seeded mechanism's chemical time scale; the work per
    stage does not depend on dt.  Times K SSP-RK3 steps (two launches per stage: the BR1
    face pass and the fused stage) replayed from CUDA graphs."""
    import torch
    from paper_2605_26388_b300 import dgsem, workloads as wl
    nel, n_deg = args.reacting_nel, 3
    mech = wl.air5_mechanism()
    mu = wl.reacting_tgv_viscosity(mech)
    x, _, _ = dgsem.gll(n_deg)
    U = torch.from_numpy(wl.reacting_tgv_3d(nel, x, mech).reshape(9, -1)).cuda()
    dt = 1e-13
    steps = max(3, args.steps // 10)

    def timed(precision, bc=(0,) * 6, bc_state=None, tt=False, limiter=False):
        S = dgsem.Solver(dgsem.Mesh(3, n_deg, (nel,) * 3, (0.0,) * 3, (2 * math.pi,) * 3, bc=bc, bc_state=bc_state),
                         equations=dgsem.DG_NS_REACTING, mu=mu, prandtl=0.72, mechanism=mech,
                         precision=precision, p_ref=101325.0 if precision == dgsem.FP32_MIXED else 0.0,
                         two_temperature=tt, species_limiter=limiter)
        S.set_state(U_tt if tt else U)
        S.rk_step(dt, 3)
        S.check()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        S.rk_step(dt, steps)
        e1.record()
        torch.cuda.synchronize()
        S.check()
        n = S.n_doubles
        S.close()
        return e0.elapsed_time(e1) / steps, n

    ms, dof = timed(dgsem.FP64)
    ms32, _ = timed(dgsem.FP32_MIXED)
    # the same workload in a closed box: slip, no-slip adiabatic and isothermal walls
    walls = (dgsem.BC_SLIP_WALL, dgsem.BC_NOSLIP_ISOTHERMAL, dgsem.BC_NOSLIP_ADIABATIC,
             dgsem.BC_NOSLIP_ADIABATIC, dgsem.BC_NOSLIP_ISOTHERMAL, dgsem.BC_SLIP_WALL)
    wall_T = (None, (6200.0,), None, None, (4300.0,), None)
    msw, _ = timed(dgsem.FP64, walls, wall_T)
    ms_lim, _ = timed(dgsem.FP64, limiter=True)
    # the two-temperature model on the same workload: E_v at a lagging T_v, Landau-Teller
    # exchange, dissociation at sqrt(T T_v)
    U_tt = torch.from_numpy(wl.reacting_tgv_3d(nel, x, mech, two_temperature=True).reshape(10, -1)).cuda()
    ms_tt, dof_tt = timed(dgsem.FP64, tt=True)
    ms_tt32, _ = timed(dgsem.FP32_MIXED, tt=True)
    del U_tt
    state_bytes = dof * 8
    alg = (16 + 24 + 24) / 3.0 * dof  # stage update bytes per average stage, as for Euler
    peak, kind = measured_peaks()
    return {"workload": f"3D reacting NS, 5-species air, 17 reactions, N=3, {nel}^3, BR1 Re=1600, Rusanov, FP64",
            "dof": dof, "steps": steps, "dt": dt, "ms_per_step": ms, "value": 3 * dof / (ms * 1e-3),
            "unit": "DOF-updates/s", "gpu_launches": 6 * steps,
            "hbm_fraction": {"achieved_gbs": alg / (ms / 3 * 1e-3) / 1e9, "peak": peak, "peak_kind": kind,
                             "frac": alg / (ms / 3 * 1e-3) / 1e9 / peak,
                             "note": "far below 1: the stage is bound by the FP64 pipe (chemistry exp, "
                                     "BR1 and flux arithmetic), see profiles/"},
            "state_gb": state_bytes / 1e9,
            "fp32_mixed": {"ms_per_step": ms32, "value": 3 * dof / (ms32 * 1e-3), "unit": "DOF-updates/s",
                           "note": "fluxes, gradients, viscous terms in FP32 (momentum flux shifted by "
                                   "p_ref = 101325 Pa); mixture state, Arrhenius source, update FP64"},
            "two_temperature": {"dof": dof_tt, "ms_per_step": ms_tt, "value": 3 * dof_tt / (ms_tt * 1e-3),
                                "unit": "DOF-updates/s", "cost_ratio": ms_tt / ms,
                                "fp32_mixed": {"ms_per_step": ms_tt32, "value": 3 * dof_tt / (ms_tt32 * 1e-3)},
                                "note": "10 variables (E_v); T_v by Newton per node per stage, Landau-Teller "
                                        "with Millikan-White + Park, 15 dissociations at sqrt(T T_v); FP64 "
                                        "and FP32-mixed"},
            "species_limiter": {"ms_per_step": ms_lim, "cost_ratio": ms_lim / ms,
                                "note": "FP64; Zhang-Shu limiter of the partial densities after every stage "
                                        "(one warp per element, one more launch per stage)"},
            "closed_box": {"ms_per_step": msw, "value": 3 * dof / (msw * 1e-3), "unit": "DOF-updates/s",
                           "cost_ratio": msw / ms,
                           "note": "FP64; x: slip / isothermal 6200 K, y: no-slip adiabatic, z: isothermal "
                                   "4300 K / slip (boundary functors in the BR1 pass and the stage)"}}


def run_split(args):
    """The stiff-chemistry workload: the reacting workload on 32^3 elements (N = 3, 2.1 M
    nodes) advanced by the Strang split (Eq. strang_split): SSP-RK54 transport (five BR1 +
    stage launch pairs, no source in L) between two implicit source substeps of dt/2 (one
    k_source_implicit launch each), at dt = 1e-5 s.  For comparison, the explicit path (source
    in L, SSP-RK3) is stable only below about 1e-12 s on this mechanism; it is timed at
    1e-13 s on the same mesh.  Transport in FP64 and FP32-mixed; chemistry FP64 in both.
    Steps are timed after three warm-up steps (the first substeps, far from chemical
    equilibrium, take the most Newton updates); the substep is also timed alone, with the
    Newton updates it took."""
    import torch
    from paper_2605_26388_b300 import dgsem, workloads as wl
    nel, n_deg = args.split_nel, 3
    mech = wl.air5_mechanism()
    mu = wl.reacting_tgv_viscosity(mech)
    x, _, _ = dgsem.gll(n_deg)
    U = torch.from_numpy(wl.reacting_tgv_3d(nel, x, mech).reshape(9, -1)).cuda()
    U_tt = torch.from_numpy(wl.reacting_tgv_3d(nel, x, mech, two_temperature=True).reshape(10, -1)).cuda()
    steps = max(2, args.steps // 20)
    mesh = dgsem.Mesh(3, n_deg, (nel,) * 3, (0.0,) * 3, (2 * math.pi,) * 3)

    def events():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed_steps(S, dt, k):
        e0, e1 = events()
        torch.cuda.synchronize()
        e0.record()
        S.rk_step(dt, k)
        e1.record()
        torch.cuda.synchronize()
        S.check()
        return e0.elapsed_time(e1) / k

    out = {"workload": f"3D reacting NS, 5-species air, 17 reactions, N=3, {nel}^3, BR1 Re=1600, Rusanov; "
                       "Strang split: SSP-RK54 transport + implicit backward-Euler chemistry substeps",
           "dt": SPLIT_DT, "steps": steps}
    for name, prec, tt in (("fp64", dgsem.FP64, False), ("fp32_mixed", dgsem.FP32_MIXED, False),
                           ("two_temperature_fp64", dgsem.FP64, True)):
        S = dgsem.Solver(mesh, equations=dgsem.DG_NS_REACTING, mu=mu, prandtl=0.72, mechanism=mech,
                         precision=prec, p_ref=101325.0 if prec == dgsem.FP32_MIXED else 0.0,
                         time_scheme=dgsem.SSPRK54, chem_split=True, two_temperature=tt)
        S.set_state(U_tt if tt else U)
        transport_dt = S.max_dt(1.0)
        S.rk_step(SPLIT_DT, 3)
        S.check()
        S.newton_updates()
        ms = timed_steps(S, SPLIT_DT, steps)
        upd_steps = S.newton_updates()
        V = S.get_state()
        W = torch.empty_like(V)
        reps, times = 3, []
        for _ in range(reps):  # the same substep three times: median launch time
            e0, e1 = events()
            torch.cuda.synchronize()
            e0.record()
            S.source_step(V, 0.5 * SPLIT_DT, W)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        S.check()
        chem_ms = sorted(times)[reps // 2]
        upd = S.newton_updates() // reps
        nodes = S.n_nodes
        r = {"ms_per_step": ms, "sim_seconds_per_s": SPLIT_DT / (ms * 1e-3),
             "transport_dt_bound": transport_dt, "gpu_launches_per_step": 2 * 5 + 2,
             "newton_updates_per_node_per_substep": upd_steps / (2 * steps * nodes),
             "source_substep": {"kernel": "k_source_implicit_tt<5,double>" if tt else "k_source_implicit<5,double>",
                                "ms": chem_ms, "nodes": nodes,
                                "newton_updates": upd, "updates_per_node": upd / nodes,
                                "share_of_step": 2 * chem_ms / ms}}
        peak_g = (ALU or {}).get("fp64_fma_g_per_s")
        if FP64_INSTR_PER_NEWTON_UPDATE and not tt and peak_g:
            ach = upd * FP64_INSTR_PER_NEWTON_UPDATE / (chem_ms * 1e-3) / 1e9
            r["source_substep"]["roofline"] = {
                "bound": "alu", "unit": "G FP64 instr/s", "achieved": ach, "peak": peak_g,
                "frac": ach / peak_g, "peak_kind": "measured (dg_alu_rate, FP64 FMA)",
                "instr_per_update": FP64_INSTR_PER_NEWTON_UPDATE}
        S.close()
        out[name] = r
    # the explicit path on the same mesh: source in L, SSP-RK3, at its stable step
    S = dgsem.Solver(mesh, equations=dgsem.DG_NS_REACTING, mu=mu, prandtl=0.72, mechanism=mech)
    S.set_state(U)
    S.rk_step(EXPLICIT_DT, 3)
    S.check()
    ms_exp = timed_steps(S, EXPLICIT_DT, steps)
    S.close()
    out["explicit_fp64"] = {"dt": EXPLICIT_DT, "ms_per_step": ms_exp,
                            "sim_seconds_per_s": EXPLICIT_DT / (ms_exp * 1e-3)}
    out["speedup_sim_time_fp64"] = out["fp64"]["sim_seconds_per_s"] / out["explicit_fp64"]["sim_seconds_per_s"]
    return out


def run_shock(args):
    """The shock-capturing workload: 3D Euler blast (pressure ratio 10, gas at rest) in the
    periodic box [0, 2]^3, 48^3 elements, N = 3, EC flux differencing + Rusanov, Hennemann-
    Gassner DG/FV blending in every stage (indicator + neighbourhood maximum, the fused stage
    with blended elements deferred, the sub-cell FV blend), SSP-RK3 at CFL 0.3, FP32-mixed
    and FP64.  Steps are timed after three warm-up steps, beside the same steps with shock
    capturing off (which stays finite for these few steps) for the overhead."""
    import torch
    from paper_2605_26388_b300 import dgsem, workloads as wl
    nel, n_deg = args.shock_nel, 3
    x, _, _ = dgsem.gll(n_deg)
    U = torch.from_numpy(wl.blast_wave(3, nel, x).reshape(5, -1)).cuda()
    steps = max(3, args.steps // 6)
    mesh = dgsem.Mesh(3, n_deg, (nel,) * 3, (0.0,) * 3, (2.0,) * 3)
    out = {"workload": f"3D Euler blast (p ratio 10), N=3, {nel}^3, EC + Rusanov, SSP-RK3 CFL 0.3, "
                       "Hennemann-Gassner DG/FV blending", "steps": steps, "dof": nel ** 3 * 64 * 5}
    for name, prec in (("fp32_mixed", dgsem.FP32_MIXED), ("fp64", dgsem.FP64)):
        r = {}
        for shock in (True, False):
            S = dgsem.Solver(mesh, volume=dgsem.VOL_EC, surface=dgsem.SURF_RUSANOV, precision=prec,
                             gamma=GAMMA, shock=shock)
            S.set_state(U)
            dt = S.max_dt(0.3)
            S.rk_step(dt, 3)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            S.rk_step(dt, steps)
            e1.record()
            torch.cuda.synchronize()
            try:
                S.check()
                finite = True
            except dgsem.DGError:
                if shock:
                    raise
                finite = False  # the unblended scheme may leave the physical states: timing only
            ms = e0.elapsed_time(e1) / steps
            key = "blended" if shock else "unblended"
            r[key] = {"ms_per_step": ms, "value": 3 * out["dof"] / (ms * 1e-3), "unit": "DOF-updates/s",
                      "state_valid": finite}
            if shock:
                _, al = S.shock_alpha(S.get_state())
                r["blended"]["elements_blended"] = float((al > 0).double().mean())
            S.close()
        r["overhead"] = r["blended"]["ms_per_step"] / r["unblended"]["ms_per_step"]
        out[name] = r
    return out


def run_curved(args):
    """The curved-mesh workload: the 3D Taylor-Green vortex (Ma 0.1, N = 4, EC flux
    differencing + HLLC) on a periodically warped 32^3 mesh (node displacement 5% of the box
    times a product of sines), SSP-RK3 at CFL 0.25, FP32-mixed and FP64, timed beside the
    affine Cartesian kernel on the same 32^3 problem."""
    import torch
    from paper_2605_26388_b300 import dgsem, workloads as wl
    nel = 32
    x, _, _ = dgsem.gll(N)
    lo, hi = (0.0,) * 3, (2 * math.pi,) * 3
    X = wl.warped_coordinates(3, (nel,) * 3, x, lo, hi, 0.05)
    U0 = wl.taylor_green_3d(nel, x, MACH, GAMMA).reshape(NV, -1)
    U = torch.from_numpy(U0).cuda()
    dof = nel ** 3 * NP * NV
    steps = max(3, args.steps // 6)
    out = {"workload": f"3D Euler TGV Ma 0.1, N=4, {nel}^3 warped periodic mesh, EC + HLLC, SSP-RK3",
           "dof": dof, "steps": steps}
    for name, prec in (("fp32_mixed", dgsem.FP32_MIXED), ("fp64", dgsem.FP64)):
        r = {}
        for key, coords in (("curved", X), ("cartesian", None)):
            S = dgsem.Solver(dgsem.Mesh(3, N, (nel,) * 3, lo, hi, coords=coords), volume=dgsem.VOL_EC,
                             surface=dgsem.SURF_HLLC, precision=prec, gamma=GAMMA, p_ref=P_REF)
            S.set_state(U)
            dt = S.max_dt(CFL)
            S.rk_step(dt, 3)
            S.check()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            S.rk_step(dt, steps)
            e1.record()
            torch.cuda.synchronize()
            S.check()
            ms = e0.elapsed_time(e1) / steps
            r[key] = {"ms_per_step": ms, "value": 3 * dof / (ms * 1e-3), "unit": "DOF-updates/s"}
            S.close()
        r["cost_ratio"] = r["curved"]["ms_per_step"] / r["cartesian"]["ms_per_step"]
        out[name] = r
    out["reacting"] = run_curved_reacting(args)
    return out


def run_curved_reacting(args):
    """The reacting workload's state (5-species air, N = 3, BR1 Re = 1600, 17 Arrhenius
    reactions, Rusanov) on a periodically warped 32^3 mesh, timed beside the Cartesian mesh of
    the same problem; dt = 1e-13 s (the work per stage does not depend on dt)."""
    import torch
    from paper_2605_26388_b300 import dgsem, workloads as wl
    nel, n_deg = 32, 3
    mech = wl.air5_mechanism()
    mu = wl.reacting_tgv_viscosity(mech)
    x, _, _ = dgsem.gll(n_deg)
    lo, hi = (0.0,) * 3, (2 * math.pi,) * 3
    X = wl.warped_coordinates(3, (nel,) * 3, x, lo, hi, 0.05)
    U = torch.from_numpy(wl.reacting_tgv_3d(nel, x, mech).reshape(9, -1)).cuda()
    dof = nel ** 3 * (n_deg + 1) ** 3 * 9
    steps = max(3, args.steps // 10)
    out = {"workload": f"3D reacting NS, 5-species air, N=3, {nel}^3 warped periodic mesh, BR1, Arrhenius, Rusanov",
           "dof": dof, "steps": steps, "dt": 1e-13}
    for name, prec in (("fp64", dgsem.FP64), ("fp32_mixed", dgsem.FP32_MIXED)):
        r = {}
        for key, coords in (("curved", X), ("cartesian", None)):
            S = dgsem.Solver(dgsem.Mesh(3, n_deg, (nel,) * 3, lo, hi, coords=coords), equations=dgsem.DG_NS_REACTING,
                             mu=mu, prandtl=0.72, mechanism=mech, precision=prec,
                             p_ref=101325.0 if prec == dgsem.FP32_MIXED else 0.0)
            S.set_state(U)
            S.rk_step(1e-13, 3)
            S.check()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            S.rk_step(1e-13, steps)
            e1.record()
            torch.cuda.synchronize()
            S.check()
            ms = e0.elapsed_time(e1) / steps
            r[key] = {"ms_per_step": ms, "value": 3 * dof / (ms * 1e-3), "unit": "DOF-updates/s"}
            S.close()
        r["cost_ratio"] = r["curved"]["ms_per_step"] / r["cartesian"]["ms_per_step"]
        out[name] = r
    return out


def run_adjoint(args):
    """The differentiable workload: 2D Euler, N = 4, 128^2 elements, strong form + Rusanov,
    200 SSP-RK3 steps (cfl 0.5) from a seeded acoustic state, checkpoints every 20 steps;
    gradient of the quadrature-weighted L2 density mismatch to a seeded target with respect
    to U0 and gamma through the hand-written residual/step adjoint.  Times the forward
    rollout alone (graph-replayed steps) and forward + backward, in FP64 and FP32-mixed."""
    import torch
    from paper_2605_26388_b300 import dgsem, workloads as wl
    from paper_2605_26388_b300.adjoint import rollout
    nel, n_deg, steps, every = 128, 4, 200, 20
    x, w, _ = dgsem.gll(n_deg)
    U0 = torch.from_numpy(wl.acoustic_2d(nel, x, seed=3).reshape(4, -1)).cuda()
    target = torch.from_numpy(wl.target_density_2d(nel, x, seed=4).reshape(-1)).cuda()
    jac = (1.0 / nel / 2.0) ** 2
    wq = torch.from_numpy(np.tile(np.multiply.outer(w, w).ravel(), nel * nel) * jac).cuda()
    out = {"workload": "2D Euler N=4 128^2, 200 SSP-RK3 steps, checkpoints every 20, grad of the "
                       "L2 density mismatch in U0 and gamma", "steps": steps}
    for name, prec in (("fp64", dgsem.FP64), ("fp32_mixed", dgsem.FP32_MIXED)):
        S = dgsem.Solver(dgsem.Mesh(2, n_deg, (nel, nel), (0.0, 0.0), (1.0, 1.0)), volume=dgsem.VOL_STRONG,
                         surface=dgsem.SURF_RUSANOV, precision=prec, gamma=GAMMA)
        S.set_state(U0)
        dt = S.max_dt(0.5)
        S.rk_step(dt, 3)
        S.check()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.set_state(U0)
        S.rk_step(dt, steps)
        S.check()
        t_fwd = time.perf_counter() - t0
        def grad(n):
            U = U0.clone().requires_grad_(True)
            gam = torch.tensor(GAMMA, dtype=torch.float64, requires_grad=True)
            loss = 0.5 * torch.sum(wq * (rollout(S, U, gam, dt, n, every)[0] - target) ** 2)
            loss.backward()

        grad(2 * every)  # warm-up: first use of the adjoint workspace, autograd and loss kernels
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        grad(steps)
        torch.cuda.synchronize()
        t_grad = time.perf_counter() - t0
        S.close()
        out[name] = {"forward_ms": 1e3 * t_fwd, "gradient_ms": 1e3 * t_grad,
                     "gradient_over_forward": t_grad / t_fwd,
                     "note": "gradient = checkpointed forward + segment recompute + reverse step adjoints"}
    out["tgv3d_ec_hllc"] = run_adjoint_tgv(args)
    return out


def run_adjoint_tgv(args):
    """The adjoint of the Taylor-Green scheme (3D, N = 4, two-point form + HLLC) on 32^3
    elements: one residual VJP against one residual evaluation, and one SSP-RK3 step's adjoint
    (three VJPs, two recomputed stages) against one forward step, FP64 and FP32-mixed; CUDA
    events on the solver's stream."""
    import torch
    from paper_2605_26388_b300 import dgsem, workloads as wl
    nel = 32
    x, _, _ = dgsem.gll(N)
    U0 = torch.from_numpy(wl.taylor_green_3d(nel, x, MACH, GAMMA).reshape(NV, -1)).cuda()
    out = {"workload": f"3D Euler TGV Ma {MACH}, N={N}, {nel}^3, EC + HLLC: residual VJP and SSP-RK3 step VJP"}
    for name, prec, reps in (("fp64", dgsem.FP64, 3), ("fp32_mixed", dgsem.FP32_MIXED, 10)):
        S = dgsem.Solver(dgsem.Mesh(3, N, (nel,) * 3, (0.0,) * 3, (2 * math.pi,) * 3), volume=dgsem.VOL_EC,
                         surface=dgsem.SURF_HLLC, precision=prec, gamma=GAMMA,
                         p_ref=P_REF if prec == dgsem.FP32_MIXED else 0.0)
        S.set_state(U0)
        dt = S.max_dt(CFL)
        lam = torch.rand_like(U0) - 0.5
        Ub = torch.zeros_like(U0)
        S.rhs_vjp(U0, lam, Ub)
        S.rhs(U0)
        S.rk_step(dt, 1)
        S.rk_step_vjp(U0, dt, lam.clone(), defer=True)
        S.check()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        lam_s = lam.clone()
        torch.cuda.synchronize()
        ev[0].record()
        for _ in range(reps):
            S.rhs_vjp(U0, lam, Ub)
        ev[1].record()
        for _ in range(reps):
            S.rhs(U0)
        ev[2].record()
        for _ in range(reps):
            S.rk_step_vjp(U0, dt, lam_s, defer=True)
        ev[3].record()
        S.rk_step(dt, reps)
        ev[4].record()
        torch.cuda.synchronize()
        S.adjoint_gammabar()
        S.check()
        t = [ev[k].elapsed_time(ev[k + 1]) / reps for k in range(4)]
        out[name] = {"rhs_vjp_ms": t[0], "rhs_ms": t[1], "vjp_over_rhs": t[0] / t[1], "step_vjp_ms": t[2],
                     "step_ms": t[3], "step_vjp_over_step": t[2] / t[3]}
        S.close()
    return out


def run_e2e(args, U0, dt, ws, barrier):
    """The same metric through the C-ABI with host buffers: every step uploads the state from
    pinned host memory (dg_set_state), advances one SSP-RK3 step (dg_rk_step) and reads the
    new state back (dg_get_state).  Consecutive steps alternate between two solver contexts on
    two CUDA streams, so one step's upload overlaps another's download and compute (the
    copy engines work in both directions at once); every step still moves its full input and
    result across the host link."""
    import torch
    from paper_2605_26388_b300 import dgsem

    host_in = torch.from_numpy(U0).pin_memory()
    host_out = [torch.empty_like(host_in).pin_memory() for _ in range(2)]
    streams = [torch.cuda.Stream() for _ in range(2)]
    solvers = [dgsem.Solver(dgsem.Mesh(3, N, (NEL,) * 3, (0.0,) * 3, (2 * math.pi,) * 3), volume=dgsem.VOL_EC,
                            surface=dgsem.SURF_HLLC, precision=dgsem.FP32_MIXED, gamma=GAMMA, p_ref=P_REF,
                            stream=st) for st in streams]

    def step(k):
        S = solvers[k % 2]
        S.set_state(host_in)
        S.rk_step(dt, 1)
        S.get_state(host_out[k % 2])

    for k in range(4):
        step(k)
    for S in solvers:
        S.check()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for k in range(args.e2e_steps):
        step(k)
    for S in solvers:
        S.check()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws)
    barrier()
    for S in solvers:
        S.close()
    nbytes = U0.nbytes
    # the host link's own bound: one step's upload and download moved at once, each on its own
    # stream with plain copies of the same pinned buffers (no kernels)
    dev = [torch.empty(host_in.shape, dtype=torch.float64, device="cuda") for _ in range(2)]

    def copies():
        with torch.cuda.stream(streams[0]):
            dev[0].copy_(host_in, non_blocking=True)
        with torch.cuda.stream(streams[1]):
            host_out[1].copy_(dev[1], non_blocking=True)

    copies()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        copies()
    torch.cuda.synchronize()
    link_ms = 1e3 * (time.perf_counter() - t0) / 3
    del dev
    step_ms = 1e3 * e2e_s / args.e2e_steps
    return {"value": weak_value(3 * DOF * args.e2e_steps, ws, e2e_s), "unit": "DOF-updates/s",
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "streams": 2,
            "ms_per_step": step_ms, "link_ms_per_step": link_ms, "link_frac": link_ms / step_ms,
            "note": "per step: dg_set_state from pinned host memory, one SSP-RK3 step, dg_get_state to "
                    "pinned host memory; consecutive steps alternate between two contexts/streams; "
                    "link_ms_per_step: the same upload and download as plain concurrent copies"}


if __name__ == "__main__":
    main()
