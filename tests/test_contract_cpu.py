"""CPU checks of two contracts: the benchmark's reference arm prints one JSON line with the
fields the harness reads, and the product path has no CPU fallback (without a GPU a solve
cannot start; it raises)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--grid", "16", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is False
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_no_cpu_fallback_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1804_10629_gb300 import ekcg
    if not os.path.exists(ekcg.LIB_PATH):
        from paper_1804_10629_gb300 import build
        build.build()
    A = wl.stencil_matrix((8, 8))
    part = wl.partition_boxes((8, 8), 4)
    with pytest.raises(Exception):
        ekcg.Solver(A, 4, part, max_s=2)
    # the C ABI itself reports an error rather than computing anything on the host
    with pytest.raises(ekcg.EkcgError) as e:
        ekcg.ekcg_setup(A.n, A.rowptr, A.colind, A.val, 4, part)
    assert e.value.status != ekcg.EKCG_OK
