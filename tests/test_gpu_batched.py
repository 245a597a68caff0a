"""Batched solves (many independent systems, one persistent graph-captured launch) against
the FP64 oracle, system by system."""
import os

import numpy as np
import pytest

import workloads as wl
from oracle import ekcg_ref as o

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1804_10629_gb300 import ekcg  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not os.path.exists(ekcg.LIB_PATH):
        from paper_1804_10629_gb300 import build
        build.build()


def small_batch(count=12, seed=11, contrast=4.0):
    return wl.batched_systems(count=count, nmin=12, nmax=40, t=8, seed=seed, contrast=contrast)


def concat(probs):
    return torch.as_tensor(np.concatenate([p.b for p in probs]), dtype=torch.float64,
                           device="cuda")


def split(x, probs):
    out, o0 = [], 0
    for p in probs:
        out.append(x[o0:o0 + p.A.n])
        o0 += p.A.n
    return out


def test_batched_fp64_matches_oracle_per_system():
    """Coefficient contrast <= 10: the oracle's iteration count is stable under
    rounding-level perturbations, so the +-1 iteration, 1e-8 x criteria apply."""
    probs = small_batch(contrast=1.0)
    B = ekcg.BatchedSolver(probs, 8, max_s=2)
    x, it, st = B.solve(concat(probs), s=2, tol=1e-8, maxit=2000)
    xs = split(x.cpu().numpy(), probs)
    for k, p in enumerate(probs):
        ref = o.solve(p.A, p.b, p.part, 8, 2, tol=1e-8, maxit=2000)
        assert st[k] == ref.status == o.OK, (k, st[k], ref.status)
        assert abs(int(it[k]) - ref.iters) <= 1, (k, it[k], ref.iters)
        assert np.linalg.norm(xs[k] - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
        rr = np.linalg.norm(p.b - p.A.to_scipy() @ xs[k]) / np.linalg.norm(p.b)
        assert rr <= 1e-8 * 1.01
    # a second call replays the captured graph and reproduces the result bitwise
    x2, it2, st2 = B.solve(concat(probs), s=2, tol=1e-8, maxit=2000)
    assert np.array_equal(x.cpu().numpy(), x2.cpu().numpy()) and np.array_equal(it, it2)
    B.close()


_REFS = {}


def oracle_refs(probs, key):
    """Oracle solves of a batch, computed once per module."""
    if key not in _REFS:
        _REFS[key] = [o.solve(p.A, p.b, p.part, p.t, 2, tol=1e-8, maxit=2000) for p in probs]
    return _REFS[key]


@pytest.mark.parametrize("threads,ctas,cluster", [(512, 1, 1), (256, 2, 1), (512, 1, 2),
                                                  (512, 1, 4), (512, 1, 8), (256, 2, 4)])
def test_batched_launch_shapes_match_oracle(threads, ctas, cluster):
    """Every launch shape -- one CTA per system, or a thread-block cluster of 2, 4 or 8 CTAs
    splitting each system's rows and reducing through distributed shared memory -- against
    the oracle, system by system (+-1 iteration, x to 1e-8); each shape reproduces its own
    result bitwise on a second call."""
    probs = small_batch(contrast=1.0)
    refs = oracle_refs(probs, "contrast1")
    B = ekcg.BatchedSolver(probs, 8, max_s=2)
    B.set_shape(threads, ctas, cluster)
    info = B.info()
    assert (info["threads"], info["ctas_per_sm"], info["cluster"]) == (threads, ctas, cluster)
    assert 1 <= info["groups"] <= len(probs)
    x, it, st = B.solve(concat(probs), s=2, tol=1e-8, maxit=2000)
    xs = split(x.cpu().numpy(), probs)
    for k, (p, ref) in enumerate(zip(probs, refs)):
        assert st[k] == ref.status == o.OK, (k, st[k], ref.status)
        assert abs(int(it[k]) - ref.iters) <= 1, (k, it[k], ref.iters)
        assert np.linalg.norm(xs[k] - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
    x2, it2, st2 = B.solve(concat(probs), s=2, tol=1e-8, maxit=2000)
    assert np.array_equal(x.cpu().numpy(), x2.cpu().numpy()) and np.array_equal(it, it2)
    B.close()


def test_batched_cluster_wider_than_system():
    """Systems with fewer rows than a cluster has CTAs (n = 6, 8, 9 with 8 CTAs per system):
    the CTAs without rows contribute zero partial sums and still take every barrier."""
    probs = []
    for k, shape in enumerate([(3, 2), (4, 2), (3, 3), (10, 10)]):
        A = wl.stencil_matrix(shape)
        rng = np.random.default_rng(30 + k)
        probs.append(wl.Problem(f"tiny-{k}", A, rng.uniform(-1, 1, A.n), 2,
                                wl.partition_boxes(shape, 2), shape))
    for cluster in (8, 1):
        B = ekcg.BatchedSolver(probs, 2, max_s=2)
        B.set_shape(512, 1, cluster)
        x, it, st = B.solve(concat(probs), s=2, tol=1e-8, maxit=200)
        xs = split(x.cpu().numpy(), probs)
        for k, p in enumerate(probs):
            ref = o.solve(p.A, p.b, p.part, 2, 2, tol=1e-8, maxit=200)
            assert st[k] == ref.status, (cluster, k, st[k], ref.status)
            assert abs(int(it[k]) - ref.iters) <= 1, (cluster, k, it[k], ref.iters)
            assert np.linalg.norm(xs[k] - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
        B.close()


def test_batched_set_shape_rejects_bad_values():
    probs = small_batch(count=2, contrast=1.0)
    B = ekcg.BatchedSolver(probs, 8, max_s=2)
    for bad in [(128, 1, 1), (512, 3, 1), (512, 1, 3), (512, 1, 16)]:
        with pytest.raises(RuntimeError):
            B.set_shape(*bad)
    assert B.info()["cluster"] == 4          # unchanged default
    B.close()


def test_batched_high_contrast_within_oracle_rounding_spread():
    """Coefficient jumps up to 1e4 (the batched configuration's recipe): s-step SRE-CG runs
    into loss of A-orthogonality and its iteration count moves by several iterations under
    1e-15 perturbations of b in the oracle itself.  The GPU count must lie within the range
    the oracle shows under three such perturbations, widened by one; every system must
    reach the tolerance in the true residual."""
    probs = small_batch(contrast=4.0)
    B = ekcg.BatchedSolver(probs, 8, max_s=2)
    x, it, st = B.solve(concat(probs), s=2, tol=1e-8, maxit=4000)
    xs = split(x.cpu().numpy(), probs)
    rng = np.random.default_rng(0)
    for k, p in enumerate(probs):
        counts = [o.solve(p.A, p.b, p.part, 8, 2, tol=1e-8, maxit=4000).iters]
        for _ in range(3):
            bb = p.b * (1 + 1e-15 * rng.standard_normal(p.A.n))
            counts.append(o.solve(p.A, bb, p.part, 8, 2, tol=1e-8, maxit=4000).iters)
        assert st[k] == 0
        assert min(counts) - 1 <= int(it[k]) <= max(counts) + 1, (k, it[k], counts)
        rr = np.linalg.norm(p.b - p.A.to_scipy() @ xs[k]) / np.linalg.norm(p.b)
        assert rr <= 1e-8 * 1.01
    B.close()


@pytest.mark.parametrize("cluster", [1, 4])
def test_batched_mixed_reaches_tolerance_and_breakdown_is_per_system(cluster):
    """Float32 inner solves converge only where kappa(A) * eps_float32 is well below 1;
    coefficient contrast <= 31 keeps kappa near 1e5 on these grids (the 1e4-contrast
    systems of the batched configuration reach kappa ~ 1e7-1e8, where float32 refinement
    stalls; they are left to the float64 batched solve)."""
    probs = small_batch(seed=12, contrast=1.5)
    bad = probs[3]
    bad.b = bad.b.copy()
    bad.b[bad.part == 5] = 0.0            # T(r_0) has a zero column: breakdown
    B = ekcg.BatchedSolver(probs, 8, precision="fp32_ir", max_s=2)
    B.set_shape(512, 1, cluster)
    x, it, st = B.solve(concat(probs), s=2, tol=1e-8, maxit=4000)
    xs = split(x.cpu().numpy(), probs)
    for k, p in enumerate(probs):
        if k == 3:
            assert st[k] == ekcg.EKCG_EBREAKDOWN
            continue
        assert st[k] == 0, (k, st[k])
        rr = np.linalg.norm(p.b - p.A.to_scipy() @ xs[k]) / np.linalg.norm(p.b)
        assert rr <= 1e-8 * 1.01, (k, rr)
    B.close()


def test_batched_mixed_high_contrast_switches_to_float64():
    """Coefficient jumps up to 1e4 (the batched configuration's recipe) push kappa(A) eps32
    towards 1, where the float32 inner solves stop reducing the float64 residual: those
    systems continue on the device in float64 from the refined iterate, and every system
    reaches the tolerance in the true residual."""
    probs = small_batch(contrast=4.0)
    B = ekcg.BatchedSolver(probs, 8, precision="fp32_ir", max_s=2)
    x, it, st = B.solve(concat(probs), s=2, tol=1e-8, maxit=8000)
    nsw = B.precision_switches()
    xs = split(x.cpu().numpy(), probs)
    for k, p in enumerate(probs):
        assert st[k] == 0, (k, st[k])
        rr = np.linalg.norm(p.b - p.A.to_scipy() @ xs[k]) / np.linalg.norm(p.b)
        assert rr <= 1e-8 * 1.01, (k, rr)
    assert 0 <= nsw <= len(probs)
    B.close()


@pytest.mark.slow
def test_batched_full_config_subset_float64():
    """Systems of the full batched configuration (256 systems, grids 32^2..256^2, jumps up to
    1e4, t = 8, s = 2, seed 3) with grid side <= 96, solved together in float64 in one
    launch: every system reaches true relres <= 1e-8, and the three smallest agree with the
    oracle within its own rounding spread.  (The largest systems need thousands of
    iterations of the short-recurrence method and minutes of one SM's FP64 rate; the
    benchmark reports them.)"""
    allp = wl.batched_systems(count=256, nmin=32, nmax=256, t=8, seed=3)
    probs = [p for p in allp if p.shape[0] <= 96]
    B = ekcg.BatchedSolver(probs, 8, max_s=2)
    x, it, st = B.solve(concat(probs), s=2, tol=1e-8, maxit=8000)
    xs = split(x.cpu().numpy(), probs)
    assert np.all(st == 0), np.nonzero(st)
    for k, p in enumerate(probs):
        rr = np.linalg.norm(p.b - p.A.to_scipy() @ xs[k]) / np.linalg.norm(p.b)
        assert rr <= 1e-8 * 1.01, (k, rr)
    rng = np.random.default_rng(1)
    for k in np.argsort([p.A.n for p in probs])[:3]:
        p = probs[k]
        counts = [o.solve(p.A, p.b, p.part, 8, 2, tol=1e-8, maxit=8000).iters]
        for _ in range(3):
            bb = p.b * (1 + 1e-15 * rng.standard_normal(p.A.n))
            counts.append(o.solve(p.A, bb, p.part, 8, 2, tol=1e-8, maxit=8000).iters)
        assert min(counts) - 1 <= int(it[k]) <= max(counts) + 1, (k, it[k], counts)
    B.close()
