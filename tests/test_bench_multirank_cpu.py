"""The N > 1 logic of bench.py (barriers around the timed steps, step time = maximum over
ranks) on two CPU ranks with the gloo backend; the solver is a host stand-in, so no GPU is
involved."""
import os
import socket
import sys
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class _Args:
    warmup, steps, tol, maxit = 3, 2, 1e-8, 10


class _WallTimer:
    device = "cpu"

    def sync(self):
        pass

    def start(self):
        self.t0 = time.perf_counter()

    def stop(self):
        self.t1 = time.perf_counter()

    def ms(self):
        return (self.t1 - self.t0) * 1e3


class _FakeSolver:
    """Sleeps a rank-dependent time per solve and reports fixed accounting."""

    def __init__(self, rank):
        self.delay = 0.02 * (rank + 1)

    def solve(self, b, s=2, tol=1e-8, maxit=10, x=None):
        time.sleep(self.delay)
        return x, 5, np.ones(6), 0

    def stats(self):
        return (11, 3)

    def profile(self):
        return {"gram": {"ms": 1.0, "launches": 2, "flops": 10.0, "bytes": 20.0}}

    def set_profile(self, on):
        self.profiling = bool(on)


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    r = bench.timed_solves(_Args(), _FakeSolver(rank), None, None, 2, None, dist, None,
                           timer=_WallTimer())
    out[rank] = (r["ms"], r["iters"], r["launches"], r["prof"]["gram"]["launches"])
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_report_the_slowest_rank_time():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    ms0, it0, l0, g0 = out[0]
    ms1, it1, l1, g1 = out[1]
    # every rank reports the maximum over ranks: rank 1 sleeps 40 ms per solve
    assert ms0 == ms1 and ms0 >= 40.0
    assert it0 == it1 == 5 and l0 == l1 == 22 and g0 == g1 == 4
