"""Writes the stored oracle amplitudes that the full-size GPU parity tests
compare against.  It calls only the oracle (oracle/mlqp_oracle.py) and the
seeded problem generator (workloads/); nothing here comes from the CUDA path.

  python tests/golden/make_golden.py config3 [--jobs J]
      the 1000-interface corner grating (one angle, theta = -pi/4; 512 000
      unknowns) -> tests/golden/config3_amplitudes.json
  python tests/golden/make_golden.py config4r [--angles START:STOP:STEP] [--jobs J]
      the angle sweep's 100-interface stack at its resolved discretisation
      (config4(resolved=True)), the selected angles of the 256
      -> tests/golden/config4r_amplitudes.json

Each angle is one oracle.solve_streaming call (the oracle's plain solve with
blocks formed when the forward sweep needs them, bitwise equal to
oracle.solve).  Angles run in J worker processes (spawned, BLAS threads =
cores / J each).  The file records the amplitudes a^U_n, a^D_n (n = -K..K,
index n + K, as [re, im] pairs), the flux error of Remark r:flux, the
command and the seed of the generator.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))


def _problem(name):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from workloads import config3, config4
    if name == "config3":
        return config3()
    if name == "config4r":
        return config4(resolved=True)
    raise ValueError(name)


def _solve_one(job):
    name, a = job
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from oracle import mlqp_oracle as O
    prob = _problem(name)
    t = time.perf_counter()
    r = O.solve_streaming(prob, a)
    return dict(index=a, theta=r["theta"], aU=[[float(z.real), float(z.imag)] for z in r["aU"]],
                aD=[[float(z.real), float(z.imag)] for z in r["aD"]], flux=r["flux"],
                seconds=time.perf_counter() - t)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=["config3", "config4r"])
    ap.add_argument("--angles", default="0:256:8")
    ap.add_argument("--jobs", type=int, default=1)
    args = ap.parse_args()
    prob = _problem(args.workload)
    if args.workload == "config3":
        idx = [0]
    else:
        a, b, c = (int(v) for v in args.angles.split(":"))
        idx = list(range(a, min(b, prob.n_theta), c))
    jobs = max(1, min(args.jobs, len(idx)))
    threads = max(1, (os.cpu_count() or 1) // jobs)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = str(threads)
    t0 = time.perf_counter()
    work = [(args.workload, a) for a in idx]
    if jobs == 1:
        res = [_solve_one(w) for w in work]
    else:
        with mp.get_context("spawn").Pool(jobs) as pool:
            res = pool.map(_solve_one, work, chunksize=1)
    res.sort(key=lambda r: r["index"])
    out = {
        "workload": prob.name,
        "what": "oracle Bragg amplitudes a^U_n, a^D_n (n = -K..K at index n + K, [re, im]) and flux error per angle",
        "generator": "tests/golden/make_golden.py (oracle.mlqp_oracle.solve_streaming)",
        "command": "python tests/golden/make_golden.py " + " ".join(sys.argv[1:]),
        "seed": "numpy.random.default_rng(14105003 + config number) in workloads/problems.py",
        "I": prob.I, "K": prob.params.K, "P": prob.params.P, "Mw": prob.params.Mw, "M": prob.params.M,
        "n_nodes": [int(f.N) for f in prob.ifaces],
        "lsq_rcond": prob.params.lsq_rcond,
        "angles": [r["index"] for r in res], "theta": [r["theta"] for r in res],
        "aU": [r["aU"] for r in res], "aD": [r["aD"] for r in res], "flux": [r["flux"] for r in res],
        "cpu_seconds_per_angle": [round(r["seconds"], 1) for r in res],
        "wall_seconds": round(time.perf_counter() - t0, 1), "jobs": jobs, "blas_threads": threads,
    }
    path = os.path.join(HERE, f"{args.workload}_amplitudes.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    fl = [x for x in out["flux"] if not math.isnan(x)]
    print(f"wrote {path}: {len(res)} angle(s), max |flux error| {max(map(abs, fl)) if fl else float('nan'):.2e}, "
          f"{out['wall_seconds']} s")


if __name__ == "__main__":
    main()
