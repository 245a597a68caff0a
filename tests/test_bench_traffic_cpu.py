"""bench.py's DRAM-traffic record (profiles/dominant_kernel_traffic.json): a class's ratio is
used only while the source files it was captured from hash to the recorded sha256."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _record(tmp_path, sources, ratio, tamper=False):
    h = hashlib.sha256()
    for f in sources:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    digest = h.hexdigest()
    if tamper:
        digest = "0" * 64
    prof = tmp_path / "profiles"
    prof.mkdir(exist_ok=True)
    json.dump({"classes": {"gram": {"ratio": ratio, "sources": sources, "sha256": digest}}},
              open(prof / "dominant_kernel_traffic.json", "w"))
    return tmp_path


def test_committed_record_matches_its_sources():
    rec = json.load(open(os.path.join(ROOT, "profiles", "dominant_kernel_traffic.json")))
    for name, c in rec["classes"].items():
        assert 0.5 < c["ratio"] < 2.0, name
        for f in c["sources"]:
            assert os.path.exists(os.path.join(ROOT, f)), f


def test_ratio_used_only_while_sources_unchanged(tmp_path, monkeypatch):
    src = ["paper_1804_10629_gb300/csrc/kernels.cuh", "paper_1804_10629_gb300/csrc/bulk.cuh"]
    # the record is read from ROOT/profiles; the sources from ROOT as well
    fake_root = _record(tmp_path, src, 1.25)
    for f in src:
        d = fake_root / os.path.dirname(f)
        d.mkdir(parents=True, exist_ok=True)
        (fake_root / f).write_bytes(open(os.path.join(ROOT, f), "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(fake_root))
    assert bench.measured_traffic("gram") == 1.25
    assert bench.measured_traffic("block_update") is None
    (fake_root / src[1]).write_bytes(b"// changed\n")
    assert bench.measured_traffic("gram") is None


def test_tampered_digest_is_ignored(tmp_path, monkeypatch):
    src = ["paper_1804_10629_gb300/csrc/kernels.cuh"]
    fake_root = _record(tmp_path, src, 1.1, tamper=True)
    d = fake_root / os.path.dirname(src[0])
    d.mkdir(parents=True, exist_ok=True)
    (fake_root / src[0]).write_bytes(open(os.path.join(ROOT, src[0]), "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(fake_root))
    assert bench.measured_traffic("gram") is None
