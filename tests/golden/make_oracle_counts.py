"""Write tests/golden/oracle_counts.json: full FP64 oracle solves of the benchmark workloads.

Calls only the oracle and the input generators.  The stored iteration counts let the CPU
reference arm of bench.py time a bounded sample of s-step iterations and scale it to a whole
solve, and give the GPU tests a full-size count to compare with.

Usage: python tests/golden/make_oracle_counts.py [workload ...]   (ani3d, sky3d, poisson2d)
       python tests/golden/make_oracle_counts.py --perturbed SEED workload

The second form solves with b multiplied entrywise by (1 + 1e-15 xi), xi standard normal
from the given seed, and stores the iteration count under "<key>/perturbed/<SEED>": the
spread of these counts is the oracle's own sensitivity to rounding-level changes, which
bounds how closely any other floating-point implementation can be expected to match the
count.  Several seeds may run at once; each write takes an exclusive lock on the file.
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as wl  # noqa: E402
from oracle import ekcg_ref as o  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_counts.json")

RUNS = {
    "poisson2d": dict(make=lambda: wl.poisson2d(100, 4, seed=0), s=[2], variant="sre"),
    "ani3d": dict(make=lambda: wl.ani3d(128, 32, seed=1), s=[2], variant="sre"),
    "sky3d": dict(make=lambda: wl.sky3d(96, 16, seed=2), s=[4], variant="sre"),
}


def store(key, value):
    """Merge one entry into the JSON file under an exclusive lock."""
    import fcntl
    with open(OUT + ".lock", "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        data = json.load(open(OUT)) if os.path.exists(OUT) else {}
        data[key] = value
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)


def perturbed(seed, name):
    cfg = RUNS[name]
    p = cfg["make"]()
    rng = np.random.default_rng(seed)
    b = p.b * (1.0 + 1e-15 * rng.standard_normal(p.A.n))
    for s in cfg["s"]:
        t0 = time.time()
        res = o.solve(p.A, b, p.part, p.t, s, tol=1e-8, maxit=20000, variant=cfg["variant"])
        dt = time.time() - t0
        key = f"{name}/t{p.t}/s{s}/{cfg['variant']}/sstep/fp64/perturbed/{seed}"
        store(key, dict(iters=res.iters, status=res.status, seconds=round(dt, 2)))
        print(key, res.iters, res.status, f"{dt:.1f}s", flush=True)


def main(names):
    if names and names[0] == "--perturbed":
        perturbed(int(names[1]), names[2])
        return
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        cfg = RUNS[name]
        p = cfg["make"]()
        for s in cfg["s"]:
            t0 = time.time()
            res = o.solve(p.A, p.b, p.part, p.t, s, tol=1e-8, maxit=20000,
                          variant=cfg["variant"])
            dt = time.time() - t0
            relres = float(np.linalg.norm(p.b - p.A.to_scipy() @ res.x) / np.linalg.norm(p.b))
            key = f"{name}/t{p.t}/s{s}/{cfg['variant']}/sstep/fp64"
            data[key] = dict(iters=res.iters, status=res.status, relres=relres,
                             seconds=round(dt, 2), cores=len(os.sched_getaffinity(0)),
                             hist=[float(h) for h in res.hist[:21]])
            print(key, data[key]["iters"], data[key]["status"], f"{dt:.1f}s", flush=True)
            json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["poisson2d", "ani3d", "sky3d"])
