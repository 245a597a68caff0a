"""Write tests/golden/oracle_counts.json: full FP64 oracle solves of the benchmark workloads.

Calls only the oracle and the input generators.  The stored iteration counts let the CPU
reference arm of bench.py time a bounded sample of s-step iterations and scale it to a whole
solve, and give the GPU tests a full-size count to compare with.

Usage: python tests/golden/make_oracle_counts.py [workload ...]   (ani3d, sky3d, poisson2d)
       python tests/golden/make_oracle_counts.py --s S workload       (one s of a workload)
       python tests/golden/make_oracle_counts.py --perturbed SEED workload
       python tests/golden/make_oracle_counts.py diff2d
       python tests/golden/make_oracle_counts.py --perturbed SEED diff2d   (target solve)
       python tests/golden/make_oracle_counts.py --perturbed SEED diff2d-forward | diff2d-adjoint
       python tests/golden/make_oracle_counts.py --perturbed-hist SEED diff2d-target | diff2d-forward
       python tests/golden/make_oracle_counts.py --perturbed SEED sky3d-inverse   (SEED 0: b as is)
       python tests/golden/make_oracle_counts.py --contraction-noise SEED sky3d

The diff2d form records the differentiable workload (2D diffusion 512^2, kappa = exp of a
Gaussian random field, t = 16, s = 3): the solve for the target x* (field seed 5, b = 1),
the forward solve x (field seed 4, b = 1), the adjoint solve A lambda = x - x* and the
gradient dL/dlog kappa, with iteration counts, the first 21 residual norms and the values of
x, lambda and the gradient at 256 fixed sample rows (plus their 2-norms and max-norms).

The second form solves with b multiplied entrywise by (1 + 1e-15 xi), xi standard normal
from the given seed, and stores the iteration count under "<key>/perturbed/<SEED>": the
spread of these counts is the oracle's own sensitivity to rounding-level changes, which
bounds how closely any other floating-point implementation can be expected to match the
count.  Several seeds may run at once; each write takes an exclusive lock on the file.

The "-inverse" workloads solve with A-CholQR applying its factor W R^{-1} as the product
with the explicit inverse (the paper leaves the method open; the tensor-core contraction
applies it that way) and store the counts under "<key>/inverse[/perturbed/<SEED>]".

The --perturbed-hist form runs the first 21 s-step iterations of the differentiable
workload's target or forward solve with the same perturbation of b and stores their
residual norms under "<key>/perturbed_hist/<SEED>": the iteration from which the history
itself is sensitive to rounding.
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


def diff2d_target_perturbed(seed):
    """The differentiable workload's target solve (field seed 5, b = 1) with b multiplied
    entrywise by (1 + 1e-15 xi): its iteration count under rounding-level changes."""
    N, t, s = DIFF2D_N, DIFF2D_T, DIFF2D_S
    lk_star = wl.kappa_gaussian_field2d(N, seed=5, corr=16.0)
    A = wl.stencil_matrix((N, N), kappa=np.exp(lk_star))
    part = wl.partition_boxes((N, N), t)
    rng = np.random.default_rng(seed)
    b = 1.0 + 1e-15 * rng.standard_normal(N * N)
    t0 = time.time()
    res = o.solve(A, b, part, t, s, tol=1e-8, maxit=20000, variant="sre")
    key = f"diff2d/N{N}/t{t}/s{s}/sre/sstep/fp64/target/perturbed/{seed}"
    store(key, dict(iters=res.iters, status=res.status, seconds=round(time.time() - t0, 2)))
    print(key, res.iters, flush=True)


def diff2d_perturbed(seed, which):
    """The differentiable workload's forward solve (field seed 4, b = 1) or adjoint solve
    (A lambda = x - x*, x and x* from the oracle) with the right-hand side multiplied
    entrywise by (1 + 1e-15 xi): its iteration count under rounding-level changes."""
    N, t, s = DIFF2D_N, DIFF2D_T, DIFF2D_S
    lk = wl.kappa_gaussian_field2d(N, seed=4, corr=16.0)
    A = wl.stencil_matrix((N, N), kappa=np.exp(lk))
    part = wl.partition_boxes((N, N), t)
    rhs = np.ones(N * N)
    if which == "adjoint":
        lk_star = wl.kappa_gaussian_field2d(N, seed=5, corr=16.0)
        A_star = wl.stencil_matrix((N, N), kappa=np.exp(lk_star))
        xs = o.solve(A_star, rhs, part, t, s, tol=1e-8, maxit=20000, variant="sre").x
        x = o.solve(A, rhs, part, t, s, tol=1e-8, maxit=20000, variant="sre").x
        rhs = x - xs
    rng = np.random.default_rng(seed)
    b = rhs * (1.0 + 1e-15 * rng.standard_normal(N * N))
    t0 = time.time()
    res = o.solve(A, b, part, t, s, tol=1e-8, maxit=20000, variant="sre")
    key = f"diff2d/N{N}/t{t}/s{s}/sre/sstep/fp64/{which}/perturbed/{seed}"
    store(key, dict(iters=res.iters, status=res.status, seconds=round(time.time() - t0, 2)))
    print(key, res.iters, flush=True)


def perturbed_hist(seed, which):
    """First 21 residual norms of the differentiable workload's target (field seed 5) or
    forward (field seed 4) solve, b = 1 multiplied entrywise by (1 + 1e-15 xi)."""
    N, t, s = DIFF2D_N, DIFF2D_T, DIFF2D_S
    lk = wl.kappa_gaussian_field2d(N, seed=5 if which == "target" else 4, corr=16.0)
    A = wl.stencil_matrix((N, N), kappa=np.exp(lk))
    part = wl.partition_boxes((N, N), t)
    b = 1.0 + 1e-15 * np.random.default_rng(seed).standard_normal(N * N)
    res = o.solve(A, b, part, t, s, tol=1e-8, maxit=20, variant="sre")
    key = f"diff2d/N{N}/t{t}/s{s}/sre/sstep/fp64/{which}/perturbed_hist/{seed}"
    store(key, dict(hist=[float(h) for h in res.hist[:21]]))
    print(key, flush=True)


def contraction_noise(seed, name):
    """The workload solved with b as is, but with the block inner products of the
    A-orthonormalisation (the CGS coefficients Q^T (A W) and the A-CholQR Gram W^T (A W))
    each given an error of the size a float64 dot product may have, u (|X|^T |Y|) xi with
    u = 2^-53 and xi uniform in (-1, 1) from the seed: what any float64-accurate
    implementation of those contractions with another rounding may produce.  Stores the
    iteration count under "<key>/contraction_noise/<SEED>"."""
    cfg = RUNS[name]
    p = cfg["make"]()
    rng = np.random.default_rng(1000 + seed)
    u = 2.0 ** -53

    def noisy(X, Y):
        return X.T @ Y + u * rng.uniform(-1.0, 1.0, (X.shape[1], Y.shape[1])) * (
            np.abs(X).T @ np.abs(Y))

    def a_cholqr_noisy(W, AW, breakdown_tol, deflate=False):
        R = o.cholesky_upper(noisy(W, AW), breakdown_tol)
        return o.right_solve_upper(W, R), o.right_solve_upper(AW, R)

    def cgs2_noisy(W, AW, Q, matmul):
        for _ in range(2):
            W = W - Q @ noisy(Q, AW)
            AW = matmul(W)
        return W, AW

    o.a_cholqr = a_cholqr_noisy          # this process only: the solver's A-CholQR and CGS2
    o.cgs2_against = cgs2_noisy
    for s in cfg["s"]:
        t0 = time.time()
        res = o.solve(p.A, p.b, p.part, p.t, s, tol=1e-8, maxit=20000, variant=cfg["variant"])
        dt = time.time() - t0
        key = f"{name}/t{p.t}/s{s}/{cfg['variant']}/sstep/fp64/contraction_noise/{seed}"
        store(key, dict(iters=res.iters, status=res.status, seconds=round(dt, 2)))
        print(key, res.iters, res.status, f"{dt:.1f}s", flush=True)


def perturbed(seed, name):
    if name.endswith("-inverse"):
        # A-CholQR applying its factor by the explicit inverse; seed 0 = b unperturbed
        base = name[: -len("-inverse")]
        cfg = RUNS[base]
        p = cfg["make"]()
        b = p.b if seed == 0 else p.b * (
            1.0 + 1e-15 * np.random.default_rng(seed).standard_normal(p.A.n))
        for s in cfg["s"]:
            t0 = time.time()
            with o.factor_application("inverse"):
                res = o.solve(p.A, b, p.part, p.t, s, tol=1e-8, maxit=20000,
                              variant=cfg["variant"])
            dt = time.time() - t0
            key = (f"{base}/t{p.t}/s{s}/{cfg['variant']}/sstep/fp64/inverse" +
                   ("" if seed == 0 else f"/perturbed/{seed}"))
            store(key, dict(iters=res.iters, status=res.status, seconds=round(dt, 2)))
            print(key, res.iters, res.status, f"{dt:.1f}s", flush=True)
        return
    if name == "diff2d":
        return diff2d_target_perturbed(seed)
    if name in ("diff2d-forward", "diff2d-adjoint"):
        return diff2d_perturbed(seed, name.split("-")[1])
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


DIFF2D_N, DIFF2D_T, DIFF2D_S = 512, 16, 3
DIFF2D_SAMPLES = 256


def diff2d_sample_rows(n):
    """256 fixed sample rows of the 512^2 grid (natural order), spread over the whole grid."""
    return np.unique(np.linspace(0, n - 1, DIFF2D_SAMPLES).round().astype(np.int64))


def solve_record(A, b, part, t, s):
    t0 = time.time()
    res = o.solve(A, b, part, t, s, tol=1e-8, maxit=20000, variant="sre")
    dt = time.time() - t0
    relres = float(np.linalg.norm(b - A.to_scipy() @ res.x) / np.linalg.norm(b))
    rec = dict(iters=res.iters, status=res.status, relres=relres, seconds=round(dt, 2),
               cores=len(os.sched_getaffinity(0)), hist=[float(h) for h in res.hist[:21]])
    return res, rec


def diff2d():
    """Forward, target and adjoint solves and the log-kappa gradient of the differentiable
    workload, all by the oracle."""
    N, t, s = DIFF2D_N, DIFF2D_T, DIFF2D_S
    lk = wl.kappa_gaussian_field2d(N, seed=4, corr=16.0)
    lk_star = wl.kappa_gaussian_field2d(N, seed=5, corr=16.0)
    part = wl.partition_boxes((N, N), t)
    b = np.ones(N * N)
    rows = diff2d_sample_rows(N * N)
    A_star = wl.stencil_matrix((N, N), kappa=np.exp(lk_star))
    res_star, rec_star = solve_record(A_star, b, part, t, s)
    A = wl.stencil_matrix((N, N), kappa=np.exp(lk))
    res_x, rec_x = solve_record(A, b, part, t, s)
    g = res_x.x - res_star.x
    res_l, rec_l = solve_record(A, g, part, t, s)
    grad = o.diffusion2d_grad_logkappa(lk.ravel(), N, N, res_l.x, res_x.x)

    def sample(v):
        return dict(values=[float(v[i]) for i in rows], norm2=float(np.linalg.norm(v)),
                    norminf=float(np.max(np.abs(v))))

    key = f"diff2d/N{N}/t{t}/s{s}/sre/sstep/fp64"
    rec_star.update(x=sample(res_star.x))
    rec_x.update(x=sample(res_x.x))
    rec_l.update(x=sample(res_l.x))
    store(key + "/target", rec_star)
    store(key + "/forward", rec_x)
    store(key + "/adjoint", rec_l)
    store(key + "/grad_logkappa", dict(sample(grad), rows=[int(i) for i in rows],
                                       loss=float(0.5 * g @ g)))
    print(key, rec_star["iters"], rec_x["iters"], rec_l["iters"], flush=True)


def one_s(s, name):
    cfg = RUNS[name]
    p = cfg["make"]()
    _, rec = solve_record(p.A, p.b, p.part, p.t, s)
    key = f"{name}/t{p.t}/s{s}/{cfg['variant']}/sstep/fp64"
    store(key, rec)
    print(key, rec["iters"], rec["status"], f"{rec['seconds']:.1f}s", flush=True)


def main(names):
    if names and names[0] == "--contraction-noise":
        contraction_noise(int(names[1]), names[2])
        return
    if names and names[0] == "--perturbed-hist":
        perturbed_hist(int(names[1]), names[2].split("-")[1])
        return
    if names and names[0] == "--perturbed":
        perturbed(int(names[1]), names[2])
        return
    if names and names[0] == "--s":
        one_s(int(names[1]), names[2])
        return
    if names == ["diff2d"]:
        diff2d()
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
