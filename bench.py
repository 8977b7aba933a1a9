"""Benchmark of the periodizing multilayer scattering solver on GB300.

Metric: layer*angle solves per second (interfaces x incidence angles solved
per second, from the first fill kernel to the Bragg amplitudes).  Workload:
the 20-interface grating (5-mode random Fourier profiles 1.5 apart, period
2 pi, layer wavenumbers U[5, 20] with one lossy layer, 120 nodes per
interface, 30 wall nodes, 60 proxies, K = 25, 3 angles one of them 1e-8 past
a Wood anomaly), plain FP64.  A step is one solve of all three angles.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun every rank solves the same stack for its own three angles
(shifted by 1e-3 rank), so per-GPU work is fixed (weak scaling); the only
collective is the max over ranks of the timing.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "layer*angle solves/s"
WORKLOAD = "20-interface random grating, 120 nodes/interface, 3 angles (Wood + 2), lossy layer 11, plain FP64"
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07  # SMs x FP64 FMA/clk/SM x 2 flop x GHz (max SM clock) = 1258.6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes (fixed launch sequence, e.g. for ncu launch skips)")
    ap.add_argument("--config3", action="store_true",
                    help="also time the 1000-interface corner grating (one solve per form, after a warm-up)")
    ap.add_argument("--corner-levels", type=int, default=2)
    ap.add_argument("--gradient", action="store_true",
                    help="also time mlqp_fd_gradient on the 20-interface stack (one shape parameter)")
    ap.add_argument("--config5", action="store_true",
                    help="also time the design gradient of the 50-interface, 16-angle stack (a few parameters)")
    ap.add_argument("--config4", action="store_true",
                    help="also time the 256-angle sweep of the 100-interface uneven stack, in chunks of 128 angles")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms, device):
    """The job's time: the largest of the ranks' times (all_reduce MAX; any
    backend, the tensor on `device`)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world_size, steps, total_ms):
    """Whole-job throughput: the units all ranks processed over the job's time."""
    return units_per_rank * world_size * steps / (total_ms / 1e3)


def problem(rank=0):
    from workloads import config2
    prob = config2()
    if rank:
        prob = prob.with_angles(prob.theta + 1e-3 * rank)
    return prob


# ---------------------------------------------------------------------------
# algorithmic work (standard complex arithmetic: one complex multiply-add =
# 8 real flops) of the block-tridiagonal sweep, per angle
# ---------------------------------------------------------------------------
def sweep_flops(n):
    """n: unknowns per interface.  Forward step t eliminates n_t columns of
    the (n_t + n_b) x (n_t + n_b + 1) augmented block (row pivoting in the
    top n_t rows); then the backward sweep (matvec + triangular solve)."""
    cm = 0
    I = len(n)
    for t in range(I):
        nt, nb = n[t], (n[t + 1] if t + 1 < I else 0)
        for j in range(nt):
            rows = nt + nb - j - 1
            cols = nt + nb + 1 - j - 1
            cm += rows * cols + rows  # rank-1 update + multipliers
        cm += nt * nb + nt * nt // 2
    return 8 * cm


def schur_flops(n, P):
    I = len(n)
    cm = 0
    for i in range(I):
        cm += n[i] * n[i] * 2 * P
        if i + 1 < I:
            cm += n[i] * n[i + 1] * P
        if i > 0:
            cm += n[i] * n[i - 1] * P
    return 8 * cm


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.p = None
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(angles=1):
    """The oracle, as it stands, on one angle of the same stack, single-threaded
    BLAS, in a child process."""
    code = (
        "import sys, time, json; sys.path.insert(0, %r)\n"
        "from workloads import config2\n"
        "from oracle import mlqp_oracle as O\n"
        "p = config2(); asm = O.Assembler(p); t = time.perf_counter()\n"
        "for a in range(%d): O.solve(p, a, asm)\n"
        "dt = time.perf_counter() - t\n"
        "print(json.dumps({'seconds': dt, 'units': p.I * %d}))\n" % (ROOT, angles, angles))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        return {"error": r.stderr[-300:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": d["units"] / d["seconds"], "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"{angles} of 3 angles of the same stack (all 20 interfaces), {d['seconds']:.1f} s"}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    K, W = args.steps, args.warmup
    code = (
        "import sys, time, json; sys.path.insert(0, %r)\n"
        "from workloads import config2\n"
        "from oracle import mlqp_oracle as O\n"
        "p = config2(); ts = []\n"
        "for s in range(%d):\n"
        "    asm = O.Assembler(p); t = time.perf_counter(); O.solve(p, s %% 3, asm); ts.append(time.perf_counter() - t)\n"
        "print(json.dumps(ts))\n" % (ROOT, K + W))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=3600)
    if r.returncode != 0:
        print(json.dumps({"impl": "reference", "unavailable": "oracle run failed: " + r.stderr[-200:]}))
        return
    ts = json.loads(r.stdout.strip().splitlines()[-1])[W:]
    total = sum(ts)
    value = 20 * K / total
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus, "steps": K, "warmup": W,
            "ms_per_step": 1e3 * total / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD + " (one angle per step)", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle",
                             "sample": "one angle of the stack per step, all 20 interfaces"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def corner_grating(mlqp, dev, levels):
    """The paper-scale corner stack (1000 trapezoidal interfaces, d = 1, graded
    panels): one timed solve per form after a warm-up, per-stage CUDA events."""
    import torch
    from workloads import config3
    out = {"workload": f"1000 trapezoidal interfaces, {levels} panel levels per corner side, one angle",
           "unit": METRIC}
    for name, prec, solver in (("fp64", mlqp.MLQP_FP64, mlqp.MLQP_SWEEP), ("mixed", mlqp.MLQP_MIXED, mlqp.MLQP_SWEEP),
                               ("mixed_cyclic", mlqp.MLQP_MIXED, mlqp.MLQP_CYCLIC)):
        prob = config3(levels=levels)
        ctx = mlqp.Context(prob, device=dev, precision=prec, block_solver=solver)
        st = [mlqp.STAGE_GEOM, mlqp.STAGE_FILL, mlqp.STAGE_LSQ, mlqp.STAGE_SCHUR, mlqp.STAGE_SWEEP,
              mlqp.STAGE_RECOVER]
        for s_ in st:
            ctx.run_stage(s_)
        ctx.check()
        torch.cuda.synchronize()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(st) + 1)]
        with torch.cuda.stream(ctx.stream):
            for q, s_ in enumerate(st):
                evs[q].record(ctx.stream)
                ctx.run_stage(s_)
            evs[-1].record(ctx.stream)
        torch.cuda.synchronize()
        ctx.check()
        ms = [evs[q].elapsed_time(evs[q + 1]) for q in range(len(st))]
        res = ctx.solve_host()
        out[name] = {"value": prob.I / (sum(ms) / 1e3), "ms_per_solve": sum(ms),
                     "stage_ms": dict(zip(["geometry", "fill", "lsq", "schur", "sweep", "recover"], ms)),
                     "flux_error": float(res["flux"][0]), "unknowns": int(sum(2 * f.N for f in prob.ifaces)),
                     "workspace_gb": ctx.ws_bytes / 1e9}
        ctx.close()
    return out


def gradient_leg(mlqp, dev, reps=3):
    """mlqp_fd_gradient on the 20-interface, 3-angle stack: dJ/dp for
    J = sum over angles and orders of |a^U_n|^2 (w = 1), p = the first cosine
    coefficient of interface 10, t = 1e-3; the base context re-solved
    (untimed) before each call; wall-clock of the synchronous call (adjoint
    pieces, base refill, four moved fills and forms), best of `reps` after a
    warm-up that captures the stage graphs."""
    import time
    from dataclasses import replace
    import numpy as np
    from workloads import config2
    from workloads.problems import Interface
    prob = config2()
    t = 1e-3

    def moved_problem(s_):
        ifs = list(prob.ifaces)
        f = ifs[9]
        a = f.a.copy()
        a[0] += s_ * t
        ifs[9] = Interface(f.y0, a, f.b.copy(), f.N)
        return replace(prob, ifaces=ifs)

    ctx = mlqp.Context(prob, device=dev)
    moved = [mlqp.Context(moved_problem(s_), device=dev) for s_ in (-2, -1, 1, 2)]
    best, solve_best, grad = float("inf"), float("inf"), None
    for r in range(reps + 1):
        t0 = time.perf_counter()
        res = ctx.solve_host()
        ts = (time.perf_counter() - t0) * 1e3
        t0 = time.perf_counter()
        grad = ctx.fd_gradient(moved, t, np.asarray(res["aU"]))
        tg = (time.perf_counter() - t0) * 1e3
        if r > 0:
            best, solve_best = min(best, tg), min(solve_best, ts)
    out = {"workload": "20-interface random grating, 3 angles, d J / d a_10[1] with J = sum |a^U_n|^2",
           "ms_per_gradient": best, "ms_per_solve_host": solve_best, "dJ_dp": float(np.sum(grad)),
           "moved_contexts": 4, "step": t}
    for m in moved:
        m.close()
    ctx.close()
    return out


def design_gradient(mlqp, dev, n_params=4):
    """The design-gradient stack (50 interfaces with 4 Fourier modes, 51
    wavenumbers, 120 nodes, 16 angles; 451 parameters in all), along
    `n_params` of its parameters (wavenumbers and coefficients of the middle
    of the stack), J = sum over angles and orders of |a^U_n|^2, t = 1e-3:
    wall-clock of the solve, of forming the sensitivities once
    (mlqp_gradient_prepare), of the first parameter (making the four moved
    contexts and capturing their graphs) and of each later one (moving them by
    mlqp_set_problem, fills and forms: mlqp_gradient_eval)."""
    import time
    from dataclasses import replace
    import numpy as np
    import torch
    from workloads import config5
    from workloads.problems import Interface
    prob = config5()
    mid = prob.I // 2
    t = 1e-3

    def moved_problem(q, s_):
        k = np.asarray(prob.k, dtype=np.complex128).copy()
        ifs = list(prob.ifaces)
        f = ifs[mid - 1 + q // 2]
        a, b = f.a.copy(), f.b.copy()
        if q % 2 == 0:
            k[mid + q // 2] += s_ * t
        else:
            a[q // 2 % len(a)] += s_ * t
        ifs[mid - 1 + q // 2] = Interface(f.y0, a, b, f.N)
        return replace(prob, k=k, ifaces=ifs)

    ctx = mlqp.Context(prob, device=dev)
    ctx.solve_host()  # captures the graphs
    t0 = time.perf_counter()
    res = ctx.solve_host()
    solve_ms = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    work = ctx.gradient_prepare(np.asarray(res["aU"]))
    torch.cuda.synchronize()
    prep_ms = (time.perf_counter() - t0) * 1e3
    moved, per, first, total = [], [], None, 0.0
    for q in range(n_params):
        t0 = time.perf_counter()
        probs = [moved_problem(q, s_) for s_ in (-2, -1, 1, 2)]
        if not moved:
            moved = [mlqp.Context(mp, device=dev) for mp in probs]
        else:
            for m, mp in zip(moved, probs):
                m.set_problem(mp)
        total += float(np.sum(ctx.gradient_eval(moved, t, work)))
        ms = (time.perf_counter() - t0) * 1e3
        if q == 0:
            first = ms
        else:
            per.append(ms)
    for m in moved:
        m.close()
    ctx.close()
    n_all = prob.I * 2 * len(prob.ifaces[0].a) + prob.I + 1
    return {"workload": "50 interfaces x 4 Fourier modes, 51 wavenumbers, 120 nodes, 16 angles",
            "parameters_total": n_all, "parameters_timed": n_params, "ms_solve_host": solve_ms,
            "ms_prepare": prep_ms, "ms_first_parameter": first,
            "ms_per_parameter": float(np.median(per)) if per else None, "sum_dJ": total}


def angle_sweep(mlqp, dev, chunk=128):
    """The batched angle sweep: 256 angles of the 100-interface stack with
    uneven node counts, solved in chunks of `chunk` angles through one
    context (mlqp_set_angles; every stage a replayed graph), in FP64 and in
    the mixed form (plain and GMRES refinement), with each mixed leg's
    backward errors and amplitude deviation from the FP64 leg; beside it, the
    plain FP64 solve of single angles."""
    import numpy as np
    import torch
    from workloads import config4
    prob = config4()
    th = np.asarray(prob.theta)
    out = {"workload": "100 interfaces, N_i in {80,...,320}, 256 angles in [-pi+0.1, -0.1]", "unit": "angles/s",
           "chunk": chunk}
    def checked(ctx, prec, omegas):
        """Status check; in the mixed form an unreached refine_tol is recorded
        (per-angle backward errors), not raised."""
        try:
            ctx.check()
        except mlqp.MlqpError as e:
            if not (prec == mlqp.MLQP_MIXED and e.status == mlqp.MLQP_ENOTCONV):
                raise
        if prec == mlqp.MLQP_MIXED and omegas is not None:
            omegas += [float(ctx.block(mlqp.BLK_REFINE, 1, a)[0]) for a in range(ctx.n_theta)]

    legs = (("fp64", mlqp.MLQP_FP64, {}),
            ("mixed", mlqp.MLQP_MIXED, dict(max_refine=20)),
            ("mixed_gmres", mlqp.MLQP_MIXED, dict(max_refine=4, refine_method=mlqp.MLQP_GMRES_IR)))
    amps = {}
    for name, prec, kw in legs:
        ctx = mlqp.Context(prob.with_angles(th[:chunk]), device=dev, precision=prec, **kw)
        tuned = ctx.autotune(mlqp.TUNE_QR)  # the QR cluster size only: tuning the block solve costs minutes here
        res = ctx.outputs()
        ctx.solve_device(res)
        checked(ctx, prec, None)
        torch.cuda.synchronize()
        omegas, amps[name] = [], []
        t0 = time.perf_counter()
        for c0 in range(0, len(th), chunk):
            ctx.set_angles(th[c0:c0 + chunk])
            ctx.solve_device(res)
            checked(ctx, prec, omegas)
            amps[name].append(torch.cat([res["aU"], res["aD"]], 1).cpu())
        el = time.perf_counter() - t0
        out[name] = {"seconds": el, "value": len(th) / el, "workspace_gb": ctx.ws_bytes / 1e9,
                     "launch_shapes": {"qr_cluster": int(tuned["qr_cluster"]), "source": "mlqp_autotune"}}
        if omegas:
            out[name]["backward_error_max"] = max(omegas)
            out[name]["angles_above_refine_tol"] = int(sum(w > 1e-15 for w in omegas))
            dev_a = torch.cat(amps[name]) - torch.cat(amps["fp64"])
            rel = (dev_a.abs().amax(1) / torch.cat(amps["fp64"]).abs().amax(1)).numpy()
            out[name]["amp_rel_diff_vs_fp64"] = {"median": float(np.median(rel)), "max": float(rel.max()),
                                                 "angles_above_1e-9": int((rel > 1e-9).sum())}
        ctx.close()
        del ctx, res
        torch.cuda.empty_cache()
    # per-angle plain FP64: one-angle contexts, a sample of 4 angles
    ctx = mlqp.Context(prob.with_angles(th[:1]), device=dev)
    ctx.solve_device()
    ctx.check()
    torch.cuda.synchronize()
    sample = th[::64][:4]
    t0 = time.perf_counter()
    for a in sample:
        ctx.set_angles([a])
        ctx.solve_device()
        ctx.check()
    el = (time.perf_counter() - t0) / len(sample)
    ctx.close()
    out["per_angle_fp64"] = {"seconds_per_angle": el, "value": 1.0 / el, "sample": f"{len(sample)} of 256 angles"}
    for name, _, _ in legs:
        out[name]["speedup_vs_per_angle_fp64"] = out[name]["value"] * el
    return out


# DRAM bytes (read + write) of the sweep kernels (k_lu_panel_cl, k_lu_prep,
# k_lu_update, k_back_*) in one step of the 20-interface 3-angle grating, from
# one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum over the
# step's sweep launches, L2 warm between launches as in the bench), with the
# launch shapes SWEEP_TRAFFIC_SHAPES.
SWEEP_TRAFFIC_BYTES = 484.9e6
SWEEP_TRAFFIC_SHAPES = {"qr_cluster": 8, "angle_groups": 3, "update_tile": 16}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", init_method="env://")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_1410_5003_gb300 import build as bld
    if rank == 0:
        bld.build()
    if ws > 1:
        torch.distributed.barrier()
    from paper_1410_5003_gb300 import mlqp
    mlqp.load()

    prob = problem(rank)
    ctx = mlqp.Context(prob, device=dev)
    # launch shapes timed on this problem (untimed setup)
    tuned = ctx.autotune() if not args.no_autotune else {"qr_cluster": 8, "angle_groups": min(4, prob.n_theta),
                                                         "update_tile": 16}
    stream = ctx.stream
    out = ctx.outputs()
    n = [2 * f.N for f in prob.ifaces]
    nth = prob.n_theta
    units = prob.I * nth
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2
    stages = [mlqp.STAGE_GEOM, mlqp.STAGE_FILL, mlqp.STAGE_LSQ, mlqp.STAGE_SCHUR, mlqp.STAGE_SWEEP,
              mlqp.STAGE_RECOVER]

    def step(evs=None):
        for q, s in enumerate(stages):
            if evs is not None:
                evs[q].record(stream)
            ctx.run_stage(s)
        if evs is not None:
            evs[len(stages)].record(stream)

    for _ in range(args.warmup):
        ctx.solve_device(out)
    ctx.check()
    launches0 = ctx.launch_count()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    per_step, per_stage = [], [0.0] * len(stages)
    all_evs = []
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.fill_(1)  # evicts the 129 MB L2 between steps (outside the events)
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(stages) + 1)]
            step(evs)
            all_evs.append(evs)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = clk.stop()
    launches = ctx.launch_count() - launches0
    for evs in all_evs:
        per_step.append(evs[0].elapsed_time(evs[-1]))
        for q in range(len(stages)):
            per_stage[q] += evs[q].elapsed_time(evs[q + 1])
    total_ms = max_over_ranks(sum(per_step), dev)
    K = args.steps
    value = job_value(units, ws, K, total_ms)
    ctx.check()

    # correctness of the timed outputs: finite amplitudes
    ctx.solve_device(out)
    ctx.check()
    ok = bool(torch.isfinite(out["aU"].real).all() and torch.isfinite(out["aD"].real).all())

    line = None
    if rank == 0:
        names = ["geometry", "fill", "lsq", "schur", "sweep", "recover"]
        stage_ms = {nm: per_stage[q] / K for q, nm in enumerate(names)}
        # dominant kernel group: the block-tridiagonal sweep (FP64 pipe)
        sw_flops = nth * sweep_flops(n)
        sw_s = stage_ms["sweep"] / 1e3
        achieved = sw_flops / sw_s / 1e12
        dominant = max(stage_ms, key=stage_ms.get)
        shapes_as_captured = all(int(tuned.get(k, -1)) == v for k, v in SWEEP_TRAFFIC_SHAPES.items())
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": K,
                "warmup": args.warmup, "ms_per_step": total_ms / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "interfaces": prob.I, "angles": nth, "nodes_per_interface": 120,
                           "unknowns_per_angle": int(sum(n)), "l2": "flushed between steps (256 MB write)",
                           "launch_shapes": {"qr_cluster": int(tuned["qr_cluster"]),
                                             "angle_groups": int(tuned["angle_groups"]),
                                             "update_tile": int(tuned.get("update_tile", 32)),
                                             "source": "defaults" if args.no_autotune else "mlqp_autotune"}},
                "stage_ms": stage_ms, "dominant_stage": dominant,
                "roofline": {"bound": "alu", "kernel": "block-tridiagonal sweep (k_lu_panel/k_lu_prep/k_lu_update)",
                             "achieved": achieved, "peak": FP64_PEAK_GFLOPS / 1e3, "unit": "TFLOP/s",
                             "frac": achieved / (FP64_PEAK_GFLOPS / 1e3),
                             "traffic": SWEEP_TRAFFIC_BYTES if shapes_as_captured else None,
                             "traffic_note": ("DRAM bytes read + written by the sweep kernels per step (3 angles), "
                                              "one ncu capture of this workload with the same launch shapes"
                                              if shapes_as_captured else
                                              "null: the tuned launch shapes differ from the ncu capture's"),
                             "algorithmic_flops_per_step": sw_flops,
                             "peak_note": "FP64 FMA pipe: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz (derived; 1.20 measured at 1995 MHz)"},
                "gpu_launches": launches, "outputs_finite": ok,
                "schur_tflops": nth * schur_flops(n, prob.params.P) / (stage_ms["schur"] / 1e3) / 1e12}
        if clocks:
            line["clocks"] = clocks
    # the mixed-precision form on the same stack: FP32 Schur / block LU (sweep, then
    # block cyclic reduction), FP64 refinement
    def time_mixed(solver):
        mctx = mlqp.Context(prob, device=dev, precision=mlqp.MLQP_MIXED, max_refine=10, refine_tol=1e-15,
                            block_solver=solver)
        mtuned = mctx.autotune() if not args.no_autotune else {}
        mout = mctx.outputs()
        for _ in range(args.warmup):
            mctx.solve_device(mout)
        mctx.check()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        mtimes = []
        with torch.cuda.stream(mctx.stream):
            for _ in range(K):
                flush.fill_(1)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(mctx.stream)
                for s_ in stages:
                    mctx.run_stage(s_)
                e1.record(mctx.stream)
                mtimes.append((e0, e1))
        torch.cuda.synchronize()
        mms = max_over_ranks(sum(a.elapsed_time(b) for a, b in mtimes), dev)
        mctx.solve_device(mout)
        mctx.check()
        ref = torch.cat([out["aU"], out["aD"]], 1)
        diff = float(torch.max(torch.abs(torch.cat([mout["aU"], mout["aD"]], 1) - ref)) / torch.max(torch.abs(ref)))
        res = {"value": units * ws * K / (mms / 1e3), "unit": METRIC, "ms_per_step": mms / K,
               "speedup_vs_fp64": (total_ms / K) / (mms / K),
               "refine_steps": [int(mctx.block(mlqp.BLK_REFINE, 1, a)[1]) for a in range(nth)],
               "backward_error": max(float(mctx.block(mlqp.BLK_REFINE, 1, a)[0]) for a in range(nth)),
               "max_rel_amp_diff_vs_fp64": diff,
               "block_solver": "sweep" if solver == mlqp.MLQP_SWEEP else "cyclic reduction",
               "launch_shapes": {k: (None if v != v else int(v)) for k, v in mtuned.items()
                                 if k in ("qr_cluster", "angle_groups", "cr_cluster_cap", "update_tile")},
               "dtype": "f32 Schur/LU + f64 refinement (fill, least squares, residuals in f64)"}
        mctx.close()
        return res

    if not args.no_mixed:
        for key, solver in (("mixed", mlqp.MLQP_SWEEP), ("mixed_cyclic", mlqp.MLQP_CYCLIC)):
            res = time_mixed(solver)
            if rank == 0:
                line[key] = res
    # e2e through the C ABI with host buffers: bind (H2D of the problem) + solve (D2H of amplitudes)
    if not args.no_e2e:
        hout = ctx.host_outputs(eta=False, pinned=True)
        for _ in range(2):
            ctx.bind()
            ctx.solve_host(out=hout)
        if ws > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(K):
            ctx.bind()
            ctx.solve_host(out=hout)
        el = max_over_ranks((time.perf_counter() - t0) * 1e3, dev)
        if rank == 0:
            d2h = sum(v.numel() * v.element_size() for v in hout.values() if v is not None) + 4
            line["e2e"] = {"value": job_value(units, ws, K, el), "unit": METRIC, "h2d_bytes_per_step": ctx.upload_bytes(),
                           "d2h_bytes_per_step": d2h}
    if args.config3 and rank == 0:
        line["config3"] = corner_grating(mlqp, dev, args.corner_levels)
    if args.config4 and rank == 0:
        line["config4"] = angle_sweep(mlqp, dev)
    if args.gradient and rank == 0:
        line["gradient"] = gradient_leg(mlqp, dev)
    if args.config5 and rank == 0:
        line["config5"] = design_gradient(mlqp, dev)
    if rank == 0:
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(1)
        print(json.dumps(line))
    ctx.close()
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
