#!/usr/bin/env python
"""Time-to-solution of the s-step enlarged CG (arXiv:1804.10629) on GB300.

One step = one whole solve of A x = b to ||r_k|| <= 1e-8 ||r_0|| (x_0 = 0) through the C-ABI
library, with A, its partition and b already resident in device memory.  Default workload:
Ani3D-like 7-point anisotropic diffusion on a 128^3 grid (n = 2,097,152, coefficients
1, 1, 1e-3), t = 32 box subdomains, s = 2, s-step SRE-CG (Algorithm 4), float64.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle instead, on a
bounded sample of s-step iterations scaled to a whole solve by the oracle's stored
iteration count (tests/golden/oracle_counts.json).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

# FP32 ALU peak: SMs x 128 FMA per clock x 2 flop x 2.07 GHz (the SM count is read from the
# device at run time; 152 on GB300).  The FP64 FMA peak is measured live by the library's
# ekcg_fp64_fma_rate (a DFMA loop over every SM).
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
HBM_FALLBACK_GBS = 6800.0

WORKLOADS = {
    "ani3d": dict(make=lambda N: wl.ani3d(N or 128, 32, seed=1), s=2, variant="sre",
                  desc="Ani3D-like 7-point anisotropic diffusion (1,1,1e-3), t=32 boxes"),
    "sky3d": dict(make=lambda N: wl.sky3d(N or 96, 16, seed=2), s=4, variant="sre",
                  desc="Sky3D-like 7-point diffusion, coefficient 1 / 1e3 on 8^3 blocks, t=16"),
    "poisson2d": dict(make=lambda N: wl.poisson2d(N or 100, 4, seed=0), s=2, variant="sre",
                      desc="Poisson2D gallery('poisson',100), 4 strips"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ekcg", choices=["ekcg", "reference"])
    ap.add_argument("--workload", default="ani3d",
                    choices=sorted(WORKLOADS) + ["batched", "diff2d"])
    ap.add_argument("--grid", type=int, default=0, help="override the grid side (quick runs)")
    ap.add_argument("--s", type=int, default=0)
    ap.add_argument("--variant", default="")
    ap.add_argument("--basis", default="sstep")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32_ir"])
    ap.add_argument("--contraction", default="split", choices=["split", "fp64"],
                    help="float64 CGS / Gram contractions: tensor-core split products "
                         "(default) or float64 FMAs")
    ap.add_argument("--precond", default=None, choices=["ic0"],
                    help="block Jacobi split preconditioning, IC(0) blocks on 64 boxes")
    ap.add_argument("--sweep", action="store_true",
                    help="stability sweep over bases, s in {1,2,4,8} and both precisions")
    ap.add_argument("--sweep-bases", default="sstep,ca5,ca7,restructured",
                    help="comma-separated Krylov bases for --sweep")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--maxit", type=int, default=20000)
    ap.add_argument("--cpu-sample-iters", type=int, default=4,
                    help="s-step iterations of the oracle in the bench line's cpu_baseline")
    ap.add_argument("--ref-sample-iters", type=int, default=2,
                    help="s-step iterations of the oracle per step of --impl reference")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--host-loop", action="store_true",
                    help="test convergence on the host every iteration instead of inside the "
                         "CUDA graph of conditional iterations (same kernels; for profilers "
                         "that take one kernel launch at a time)")
    return ap.parse_args()


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampling (every 200 ms) during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}",
                                       f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [ln.split(",") for ln in open(self.f.name).read().splitlines() if ln.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_traffic(kernel_class):
    """DRAM bytes per algorithmic byte of a kernel class from the committed ncu record
    (profiles/dominant_kernel_traffic.json).  Each class names the source files of its
    kernels and the sha256 of their contents (in that order) at capture time; the ratio is
    used only while those files are unchanged."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "dominant_kernel_traffic.json")))
        c = rec.get("classes", {}).get(kernel_class)
        if not c:
            return None
        h = hashlib.sha256()
        for f in c["sources"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        if c.get("sha256") != h.hexdigest():
            return None
        return c.get("ratio")
    except Exception:
        return None


def roofline_and_table(prof, args, fp64_peak=None):
    """Roofline of the dominant kernel class (by device time) and the per-class table.
    float64 with float64-FMA contractions: FP64 ALU bound (alu, against the measured FMA
    rate) for the arithmetic kernels; the split-product Gram and update classes and every
    float32 kernel: the HBM bound on algorithmic bytes."""
    pk = peaks()
    hbm = pk.get("hbm_gbs")
    roof = None
    alu64 = ("spmm", "chol_inv", "xr_update", "gram_reduce", "trsm")
    if args.contraction == "fp64":
        alu64 = alu64 + ("gram", "block_update")
    if prof:
        name, d = max(prof.items(), key=lambda kv: kv[1]["ms"])
        sec = d["ms"] / 1e3
        ratio = measured_traffic(name)
        traffic = (ratio * d["bytes"] / max(d["launches"], 1)) if ratio else None
        if args.precision == "fp64" and name in alu64 and fp64_peak:
            ach = d["flops"] / sec / 1e12
            roof = {"kernel": name, "bound": "alu", "achieved": ach,
                    "peak": fp64_peak, "unit": "TFLOP/s", "frac": ach / fp64_peak,
                    "peak_source": "measured FP64 FMA rate (ekcg_fp64_fma_rate, this run)",
                    "traffic": traffic, "algorithmic_bytes_per_launch":
                        d["bytes"] / max(d["launches"], 1),
                    "launches": d["launches"], "avg_launch_ms": d["ms"] / max(d["launches"], 1)}
        elif name == "gram_df":
            # float-float Gram: bound by the FP32 pipe (10 FP32 operations per multiply-add)
            ach = d["flops"] / sec / 1e12
            roof = {"kernel": name, "bound": "alu", "achieved": ach,
                    "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP32_PEAK_TFLOPS,
                    "peak_source": "derived FP32 FMA rate: 152 SMs x 128 FMA/clk x 2 x 2.07 GHz",
                    "traffic": None, "launches": d["launches"],
                    "avg_launch_ms": d["ms"] / max(d["launches"], 1)}
        else:
            peak = hbm or HBM_FALLBACK_GBS
            ach = d["bytes"] / sec / 1e9
            roof = {"kernel": name, "bound": "hbm", "achieved": ach, "peak": peak,
                    "unit": "GB/s", "frac": ach / peak,
                    "peak_source": "of measured" if hbm else "of fallback",
                    "traffic": traffic, "algorithmic_bytes_per_launch":
                        d["bytes"] / max(d["launches"], 1),
                    "launches": d["launches"],
                    "avg_launch_ms": d["ms"] / max(d["launches"], 1)}
    table = {k: {"ms_per_step": v["ms"] / args.steps,
                 "launches_per_step": v["launches"] / args.steps,
                 "gflop_per_step": v["flops"] / args.steps / 1e9,
                 "gb_per_step": v["bytes"] / args.steps / 1e9,
                 "tflops": (v["flops"] / (v["ms"] / 1e3) / 1e12) if v["ms"] else None,
                 "gbs": (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["ms"] else None}
             for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}
    return roof, table


class CudaTimer:
    """Device time between two CUDA events recorded on the solve stream."""

    def __init__(self, stream):
        import torch
        self.stream = stream
        self.sync = torch.cuda.synchronize
        self.ev0 = torch.cuda.Event(enable_timing=True)
        self.ev1 = torch.cuda.Event(enable_timing=True)
        self.device = "cuda"

    def start(self):
        self.ev0.record(self.stream)

    def stop(self):
        self.ev1.record(self.stream)

    def ms(self):
        return self.ev0.elapsed_time(self.ev1)


def timed_solves(args, S, b, x, s, stream, dist, clocks, timer=None):
    """W warm-up solves, then K timed solves bracketed by barrier + synchronize, CUDA events
    on the solve stream, with per-launch timing off; the step time is the maximum over
    ranks.  Then one more solve with CUDA events around every launch (outside the timed
    region) gives the per-kernel-class table, scaled to K solves."""
    import torch
    timer = timer or CudaTimer(stream)
    its = []
    st = 0
    S.set_profile(False)
    for _ in range(args.warmup):
        _, it, _, st = S.solve(b, s=s, tol=args.tol, maxit=args.maxit, x=x)
        its.append(it)
    launches = 0
    prof = {}
    if dist:
        dist.barrier()
    timer.sync()
    if clocks:
        clocks.start()
    timer.start()
    for _ in range(args.steps):
        _, it, hist, st = S.solve(b, s=s, tol=args.tol, maxit=args.maxit, x=x)
        its.append(it)
        launches += S.stats()[0]
    timer.stop()
    timer.sync()
    S.set_profile(True)
    S.solve(b, s=s, tol=args.tol, maxit=args.maxit, x=x)
    timer.sync()
    for k, v in S.profile().items():
        prof[k] = {f: v[f] * args.steps for f in ("ms", "launches", "flops", "bytes")}
    S.set_profile(False)
    ck = clocks.stop() if clocks else None
    if dist:
        dist.barrier()
    ms = timer.ms() / args.steps
    if dist:
        tt = torch.tensor([ms], device=timer.device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    return {"ms": ms, "iters": its[-1], "status": st, "launches": launches, "prof": prof,
            "clocks": ck}


def run_batched(args, rank, world, dist):
    """256 independent 2D diffusion systems (grids 32^2..256^2, coefficient rectangles),
    t = 8, s = 2, solved in one persistent graph-captured launch; float64 and mixed."""
    import torch
    from paper_1804_10629_gb300 import ekcg
    probs = wl.batched_systems(count=256, nmin=32, nmax=args.grid or 256, t=8, seed=3)
    s = args.s or 2
    maxit = min(args.maxit, 4000)   # bounded: systems still above tol are reported as MAXIT
    b = torch.as_tensor(np.concatenate([p.b for p in probs]), dtype=torch.float64,
                        device="cuda")
    out = {}
    for prec in ("fp64", "fp32_ir"):
        B = ekcg.BatchedSolver(probs, 8, precision=prec, max_s=s)
        for _ in range(args.warmup):
            x, it, st = B.solve(b, s=s, tol=args.tol, maxit=maxit)
        clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0"))) if prec == "fp64" else None
        if clocks:
            clocks.start()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(args.steps):
            x, it, st = B.solve(b, s=s, tol=args.tol, maxit=maxit)
        ev1.record()
        torch.cuda.synchronize()
        ck = clocks.stop() if clocks else None
        xs = x.cpu().numpy()
        worst, o0 = 0.0, 0
        for p in probs:
            xi = xs[o0:o0 + p.A.n]
            worst = max(worst, float(np.linalg.norm(p.b - p.A.to_scipy() @ xi) /
                                     np.linalg.norm(p.b)))
            o0 += p.A.n
        out[prec] = {"ms": ev0.elapsed_time(ev1) / args.steps, "iters_max": int(it.max()),
                     "iters_sum": int(it.sum()), "status_ok": int((st == 0).sum()),
                     "worst_true_relres": worst, "launch": B.info(), "clocks": ck}
        B.close()
    if rank == 0:
        f = out["fp64"]
        line = {
            "metric": "time-to-solution @relres 1e-8 (s)", "value": f["ms"] / 1e3, "unit": "s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": f["ms"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "batched: 256 2D diffusion systems 32^2..256^2, t=8, s=2, "
                                   "one persistent graph-captured launch",
                       "maxit": maxit,
                       "parallelism": "replicas", "fp64": f, "fp32_ir": out["fp32_ir"]},
            "mixed": {"value": out["fp32_ir"]["ms"] / 1e3, "unit": "s",
                      "speedup_vs_fp64": f["ms"] / out["fp32_ir"]["ms"]},
            "gpu_launches": 3 * args.steps, "clocks": f["clocks"],
        }
        print(json.dumps(line), flush=True)
    return 0


def run_sweep(args, rank):
    """Stability sweep of s-step SRE-CG (Algorithm 4) over the Krylov basis (s-step monomial
    basis of Algorithm 4, the CA forms of Algorithms 5 and 7, the restructured basis of
    Algorithm 1), s in {1, 2, 4, 8} and both precisions, one timed solve each after a short
    warm-up.  The first row of each basis and precision fixes the iteration budget of the
    others at four times its s-step iterations (scaled by 1/s), so an unstable configuration
    ends quickly at EKCG_MAXIT or breakdown.  Per entry: s-step iterations, status, time,
    true relative residual and the relative difference of x from the float64 s = 1 solution;
    per basis and precision, the largest s that reached the tolerance."""
    import torch
    from paper_1804_10629_gb300 import ekcg
    cfg = WORKLOADS[args.workload]
    prob = cfg["make"](args.grid)
    b = torch.as_tensor(prob.b, dtype=torch.float64, device="cuda")
    Asp = prob.A.to_scipy()
    nb = float(np.linalg.norm(prob.b))
    rows, ref = [], None
    bases = [v for v in args.sweep_bases.split(",") if v]
    for basis in bases:
        for prec in ("fp64", "fp32_ir"):
            budget = None
            for s in (1, 2, 4, 8):
                maxit = args.maxit if budget is None else max(8, (4 * budget) // s)
                try:
                    S = ekcg.Solver(prob.A, prob.t, prob.part, variant="sre", basis=basis,
                                    precision=prec, max_s=s)
                except ekcg.EkcgError as e:
                    rows.append({"basis": basis, "precision": prec, "s": s,
                                 "error": str(e)})
                    continue
                x = torch.empty_like(b)
                S.solve(b, s=s, tol=args.tol, maxit=min(20, maxit), x=x)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                x, its, hist, st = S.solve(b, s=s, tol=args.tol, maxit=maxit, x=x)
                e1.record()
                torch.cuda.synchronize()
                xs = x.cpu().numpy()
                S.close()
                ok = bool(np.all(np.isfinite(xs)))
                if ref is None and ok:
                    ref = xs.copy()
                if budget is None:
                    budget = int(its) * s
                rows.append({"basis": basis, "precision": prec, "s": s, "iters": int(its),
                             "maxit": maxit, "status": int(st),
                             "seconds": e0.elapsed_time(e1) / 1e3,
                             "true_relres": float(np.linalg.norm(prob.b - Asp @ xs) / nb)
                             if ok else None,
                             "x_rel_diff_vs_fp64_s1": float(np.linalg.norm(xs - ref) /
                                                            np.linalg.norm(ref))
                             if ok and ref is not None else None})
    largest = {}
    for basis in bases:
        for prec in ("fp64", "fp32_ir"):
            good = [r["s"] for r in rows if r["basis"] == basis and r["precision"] == prec
                    and r.get("status") == 0 and r.get("true_relres") is not None
                    and r["true_relres"] <= args.tol * 1.01]
            largest[f"{basis}/{prec}"] = max(good) if good else None
    if rank == 0:
        print(json.dumps({"sweep": prob.name, "n": prob.A.n, "t": prob.t, "tol": args.tol,
                          "rows": rows, "largest_stable_s": largest}), flush=True)
    return 0


def run_diff2d(args, rank, world, dist):
    """Differentiable configuration: 2D 5-point diffusion on 512^2, log kappa a Gaussian
    random field (correlation length 16 cells), loss 0.5 ||x - x*||^2 with x* the solution
    for a second field, b = 1; one step = forward solve + adjoint solve + gradient kernels
    (dL/db and dL/dlog kappa), t = 16, s = 3, float64."""
    import torch
    from paper_1804_10629_gb300 import autograd as ag
    from paper_1804_10629_gb300 import ekcg
    N = args.grid or 512
    s = args.s or 3
    lk = wl.kappa_gaussian_field2d(N, seed=4, corr=16.0)
    lk_star = wl.kappa_gaussian_field2d(N, seed=5, corr=16.0)
    A = wl.stencil_matrix((N, N), kappa=np.exp(lk))
    part = wl.partition_boxes((N, N), 16)
    S = ekcg.Solver(A, 16, part, max_s=s)
    b = torch.ones(N * N, dtype=torch.float64, device="cuda")
    lks = torch.as_tensor(lk_star.ravel(), device="cuda")
    with torch.no_grad():
        xstar = ag.diffusion2d_solve(lks, b, S, N, N, s=s, tol=args.tol)

    def step():
        lkt = torch.as_tensor(lk.ravel(), device="cuda").clone().requires_grad_(True)
        bt = b.clone().requires_grad_(True)
        x = ag.diffusion2d_solve(lkt, bt, S, N, N, s=s, tol=args.tol)
        loss = 0.5 * ((x - xstar) ** 2).sum()
        loss.backward()
        return loss, lkt.grad, bt.grad

    for _ in range(args.warmup):
        step()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.synchronize()
    clocks.start()
    ev0.record()
    for _ in range(args.steps):
        loss, g_lk, g_b = step()
    ev1.record()
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    S.close()
    if rank == 0:
        line = {
            "metric": "time-to-solution @relres 1e-8 (s)", "value": ms / 1e3, "unit": "s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"differentiable: 2D diffusion {N}^2, log-kappa Gaussian "
                                   f"field (corr 16), forward + adjoint solve + gradients, "
                                   f"t=16, s={s}", "loss": float(loss.item()),
                       "grad_logkappa_norm": float(g_lk.norm().item()),
                       "grad_b_norm": float(g_b.norm().item()), "parallelism": "replicas"},
            "clocks": ck,
        }
        print(json.dumps(line), flush=True)
    return 0


def dist_setup(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def oracle_counts():
    p = os.path.join(ROOT, "tests", "golden", "oracle_counts.json")
    return json.load(open(p)) if os.path.exists(p) else {}


def cpu_oracle_sample(prob, s, variant, iters, gpu_iters=None, full_size=True, t_setup=None):
    """Whole-solve time of the FP64 oracle from a bounded sample: one call with no
    iteration (setup, permutation, initial residual) and one with `iters` s-step
    iterations; the difference gives the time per iteration, and the estimate is the setup
    time plus that per-iteration time times the oracle's stored iteration count
    (full-size workloads), else the GPU's."""
    from oracle import ekcg_ref as o
    if t_setup is None:   # the setup is the same work every time: measured once per run
        t0 = time.perf_counter()
        o.solve(prob.A, prob.b, prob.part, prob.t, s, tol=1e-8, maxit=0, variant=variant)
        t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    res = o.solve(prob.A, prob.b, prob.part, prob.t, s, tol=1e-8, maxit=iters, variant=variant)
    dt = time.perf_counter() - t0
    per_it = max(dt - t_setup, 0.0) / max(res.iters, 1)
    key = f"{prob.name.split('-')[0].lower()}/t{prob.t}/s{s}/{variant}/sstep/fp64"
    cnt = oracle_counts().get(key, {}).get("iters") if full_size else None
    scale_src = "oracle_counts.json" if cnt else "GPU iteration count"
    total = cnt if cnt else (gpu_iters or res.iters)
    return {"value": t_setup + per_it * total, "per_iter_s": per_it, "setup_s": t_setup,
            "iters_scaled_to": total, "scaled_by": scale_src, "sample_s": dt + t_setup,
            "sample_iters": res.iters, "cores": len(os.sched_getaffinity(0))}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    cfg = WORKLOADS[args.workload]
    prob = cfg["make"](args.grid)
    s = args.s or cfg["s"]
    variant = args.variant or cfg["variant"]
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state; warm-up steps would only burn host time
    vals, samples = [], []
    t_setup = None
    for _ in range(args.steps):
        r = cpu_oracle_sample(prob, s, variant, args.ref_sample_iters,
                              full_size=not args.grid, t_setup=t_setup)
        t_setup = r["setup_s"]
        vals.append(r["value"])
        samples.append(r)
    v = statistics.median(vals)
    line = {
        "impl": "reference", "metric": "time-to-solution @relres 1e-8 (s)", "value": v,
        "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{prob.name} n={prob.A.n} nnz={prob.A.nnz} t={prob.t} s={s} "
                               f"{variant} sstep fp64", "parallelism": "replicas"},
        "cpu_baseline": {"value": v, "unit": "s", "cores": samples[0]["cores"], "kind": "oracle",
                         "sample": f"the FP64 oracle's setup (timed once) and "
                                   f"{args.ref_sample_iters} s-step iterations per step on the "
                                   f"full workload; setup time plus the per-iteration time x "
                                   f"{samples[0]['iters_scaled_to']} iterations "
                                   f"({samples[0]['scaled_by']})"},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    rank, world, local = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1804_10629_gb300 import ekcg
    if not os.path.exists(ekcg.LIB_PATH):
        from paper_1804_10629_gb300 import build
        build.build()

    if args.sweep:
        return run_sweep(args, rank)
    if args.workload == "batched":
        return run_batched(args, rank, world, dist)
    if args.workload == "diff2d":
        return run_diff2d(args, rank, world, dist)
    cfg = WORKLOADS[args.workload]
    prob = cfg["make"](args.grid)
    s = args.s or cfg["s"]
    variant = args.variant or cfg["variant"]
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    sm_count, fp64_peak = ekcg.ekcg_fp64_fma_rate(stream.cuda_stream)
    with torch.cuda.stream(stream):
        S = ekcg.Solver(prob.A, prob.t, prob.part, variant=variant, basis=args.basis,
                        precision=args.precision, max_s=s, profile=True,
                        stream=stream.cuda_stream, max_basis_bytes=64 << 30,
                        contraction=args.contraction)
    if args.host_loop:
        S.set_device_loop(False)   # the convergence test on the host, every iteration
    if args.precond:
        # block Jacobi over 64 geometric boxes (the paper's 64 subdomains), each inside one
        # of the workload's t domains
        S.set_block_jacobi(wl.partition_boxes(prob.shape, 64))
    setup_s = time.perf_counter() - t0
    b = torch.as_tensor(prob.b, dtype=torch.float64, device="cuda")
    x = torch.empty_like(b)
    torch.cuda.synchronize()

    clocks = Clocks(local)
    r = timed_solves(args, S, b, x, s, stream, dist, clocks)
    ms_step, its, st, launches, prof, ck = (r["ms"], r["iters"], r["status"], r["launches"],
                                            r["prof"], r["clocks"])
    xs = x.cpu().numpy()
    relres = float(np.linalg.norm(prob.b - prob.A.to_scipy() @ xs) / np.linalg.norm(prob.b))

    # the same workload through the float32 inner solve with float64 refinement
    mixed = None
    if args.precision == "fp64" and not args.no_mixed and not args.precond:
        with torch.cuda.stream(stream):
            M = ekcg.Solver(prob.A, prob.t, prob.part, variant=variant, basis=args.basis,
                            precision="fp32_ir", max_s=s, profile=True,
                            stream=stream.cuda_stream, max_basis_bytes=64 << 30)
        xm = torch.empty_like(b)
        rm = timed_solves(args, M, b, xm, s, stream, dist, None)
        xmh = xm.cpu().numpy()
        rr_m = float(np.linalg.norm(prob.b - prob.A.to_scipy() @ xmh) / np.linalg.norm(prob.b))
        pk = peaks().get("hbm_gbs") or HBM_FALLBACK_GBS
        hbm = {}
        for k in ("spmm", "gram", "block_update", "gram_df"):
            d = rm["prof"].get(k)
            if d and d["ms"] > 0:
                gbs = d["bytes"] / (d["ms"] / 1e3) / 1e9
                hbm[k] = {"gbs": gbs, "frac": gbs / pk, "ms_per_step": d["ms"] / args.steps}
                if k == "gram_df":
                    tf = d["flops"] / (d["ms"] / 1e3) / 1e12
                    hbm[k]["fp32_tflops"] = tf
                    hbm[k]["fp32_frac"] = tf / FP32_PEAK_TFLOPS
        mixed = {"value": rm["ms"] / 1e3, "unit": "s", "iters": rm["iters"], "status": rm["status"],
                 "true_relres": rr_m, "speedup_vs_fp64": ms_step / rm["ms"],
                 "hbm": hbm, "hbm_peak_gbs": pk,
                 "x_rel_diff_vs_fp64": float(np.linalg.norm(xmh - xs) / np.linalg.norm(xs))}
        M.close()

    roof, kernel_table = roofline_and_table(prof, args, fp64_peak)

    # end to end through the host-buffer C-ABI call (H2D of b and D2H of x inside)
    e2e = None
    if not args.no_e2e:
        bh = np.ascontiguousarray(prob.b)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        xh, it_h, _, st_h = S.solve_host(bh, s=s, tol=args.tol, maxit=args.maxit)
        e2e_s = time.perf_counter() - t1
        e2e = {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(bh.nbytes),
               "d2h_bytes_per_step": int(xh.nbytes)}
    S.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = cpu_oracle_sample(prob, s, variant, args.cpu_sample_iters, gpu_iters=its,
                              full_size=not args.grid)
        cpu = {"value": r["value"], "unit": "s", "cores": r["cores"], "kind": "oracle",
               "sample": f"setup ({r['setup_s']:.1f} s) and {r['sample_iters']} s-step "
                         f"iterations of the FP64 oracle on the full workload "
                         f"({r['sample_s']:.1f} s in all); setup plus the per-iteration time "
                         f"x {r['iters_scaled_to']} iterations ({r['scaled_by']})"}

    if rank == 0:
        line = {
            "metric": "time-to-solution @relres 1e-8 (s)", "value": ms_step / 1e3, "unit": "s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": f"{prob.name} n={prob.A.n} nnz={prob.A.nnz} t={prob.t} "
                                   f"s={s} {variant} {args.basis} {args.precision}",
                       "contraction": ("tensor-core split products (float64-accurate)"
                                       if args.contraction == "split" else "float64 FMA"),
                       "sm_count": sm_count, "fp64_fma_tflops_measured": fp64_peak,
                       "desc": cfg["desc"], "tol": args.tol, "iters": its,
                       "true_relres": relres, "status": st,
                       "l2": "working set larger than L2 (matrix + n x t blocks)",
                       "setup_s": setup_s, "parallelism": "replicas",
                       "convergence_test": ("host, every iteration" if args.host_loop else
                                            "device, inside a CUDA graph of conditional "
                                            "iterations"),
                       "precond": ("block Jacobi, IC(0) blocks on 64 boxes" if args.precond
                                   else None),
                       "profiling": "timed solves without per-launch events; kernel table from one more solve with CUDA events around every launch"},
            "roofline": roof, "kernels": kernel_table, "gpu_launches": launches,
            "mixed": mixed,
            "e2e": e2e, "cpu_baseline": cpu, "clocks": ck,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
