"""The multi-GPU paths on CPU: world-size-2 gloo ranks run the host logic of
bench.py's angle sharding (each rank's problem, the job time as the maximum
over ranks, the whole-job value) and of the gradient's parameter sharding
(each rank's share of the parameters, one all_reduce of the shares), and the
reference arm under torchrun prints one line from rank 0 only.  No GPU is
involved."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob = bench.problem(rank)
        ms = 100.0 + 25.0 * rank  # this rank's (made-up) device time
        job_ms = bench.max_over_ranks(ms, torch.device("cpu"))
        value = bench.job_value(prob.I * prob.n_theta, world, 3, job_ms)
        results[rank] = (list(map(float, prob.theta)), prob.I, [f.N for f in prob.ifaces], job_ms, value)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_angles_and_take_the_slowest_time():
    world, port = 2, _free_port()
    with mp.Manager() as man:
        results = man.dict()
        mp.start_processes(_rank, args=(world, port, results), nprocs=world, start_method="spawn")
        r = dict(results)
    th0, I0, N0, ms0, v0 = r[0]
    th1, I1, N1, ms1, v1 = r[1]
    # weak scaling: the same stack per rank, its own angles (shifted by 1e-3 per rank)
    assert (I0, N0) == (I1, N1)
    assert all(abs((b - a) - 1e-3) < 1e-15 for a, b in zip(th0, th1))
    # the job's time is the slowest rank's; the value counts every rank's units
    assert ms0 == ms1 == 125.0
    assert v0 == v1 == pytest.approx(I0 * len(th0) * 2 * 3 / 0.125)


def _grad_rank(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1410_5003_gb300.diff import bragg_efficiency
        from tests.adjoint_forms import OracleContext, gradient_family
        prob, make_problem, _, _ = gradient_family()
        made = []

        def new_context(pr):
            made.append(OracleContext(pr))
            return made[-1]

        p = torch.zeros(5, dtype=torch.float64, requires_grad=True)
        J = bragg_efficiency(p, make_problem, new_context=new_context, distributed=True)
        J.backward()
        results[rank] = (float(J), p.grad.tolist(), getattr(made[0], "evals", 0))
    finally:
        dist.destroy_process_group()


def test_gradient_parameters_shard_over_two_gloo_ranks():
    """bragg_efficiency(distributed=True): rank r evaluates the parameters
    r, r + 2, ..., and one all_reduce sums the shares; both ranks end with
    the whole gradient, equal to the oracle's adjoint gradient (the ranks'
    contexts are oracle-backed stand-ins; no GPU is involved)."""
    sys.path.insert(0, ROOT)
    from oracle import mlqp_oracle as O
    from tests.adjoint_forms import gradient_family
    world, port = 2, _free_port()
    with mp.Manager() as man:
        results = man.dict()
        mp.start_processes(_grad_rank, args=(world, port, results), nprocs=world, start_method="spawn")
        r = dict(results)
    prob, _, shifted, names = gradient_family()
    ref = O.adjoint_gradient(prob, shifted, {nm: 1e-3 for nm in names})
    (J0, g0, e0), (J1, g1, e1) = r[0], r[1]
    assert J0 == J1 and g0 == g1
    assert (e0, e1) == (3, 2)  # parameters 0, 2, 4 and 1, 3
    for q, nm in enumerate(names):
        assert abs(g0[q] - ref[nm]) < 1e-9 * max(abs(ref[nm]), 1e-3), (nm, g0[q], ref[nm])


def test_reference_arm_under_torchrun_prints_from_rank_zero_only():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def _failing_grad_rank(rank, world, port, results, fail_in):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1410_5003_gb300.diff import bragg_efficiency
        from tests.adjoint_forms import OracleContext, gradient_family
        prob, make_problem, _, _ = gradient_family()
        calls = []

        def flaky_problem(pv):
            calls.append(1)
            # rank 1 fails on its first problem (forward) or on a moved one (backward)
            if rank == 1 and (fail_in == "forward" or len(calls) > 1):
                raise ValueError("make_problem failed on rank 1")
            return make_problem(pv)

        p = torch.zeros(5, dtype=torch.float64, requires_grad=True)
        try:
            J = bragg_efficiency(p, flaky_problem, new_context=OracleContext, distributed=True)
            J.backward()
            results[rank] = "ok"
        except RuntimeError as e:
            results[rank] = str(e)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("fail_in", ["forward", "backward"])
def test_gradient_failure_on_one_rank_reaches_every_rank(fail_in):
    """If one rank's problem cannot be made (an exception in make_problem, in
    the forward solve or in its share of the parameters), that rank still
    takes part in the collective, and every rank raises instead of waiting."""
    world, port = 2, _free_port()
    with mp.Manager() as man:
        results = man.dict()
        mp.start_processes(_failing_grad_rank, args=(world, port, results, fail_in), nprocs=world,
                           start_method="spawn")
        r = dict(results)
    assert "failed on 1 of 2 ranks" in r[0], r
    assert "failed on 1 of 2 ranks" in r[1], r
