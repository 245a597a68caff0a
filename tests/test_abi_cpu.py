"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports every
function that include/ekcg.h declares.  No compute calls (there is no GPU here)."""
import ctypes
import os

import pytest

from paper_1804_10629_gb300 import build as bld
from paper_1804_10629_gb300 import ekcg


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(ekcg.LIB_PATH):
        bld.build()
    return ekcg.lib()


def test_every_declared_function_is_exported(lib):
    names = ekcg.header_functions()
    assert len(names) >= 14
    raw = ctypes.CDLL(ekcg.LIB_PATH)
    missing = [nm for nm in names if not hasattr(raw, nm)]
    assert not missing, missing


def test_default_opts_and_strerror_need_no_gpu(lib):
    o = ekcg.ekcg_default_opts()
    assert (o.variant, o.basis, o.orth, o.precision, o.max_s) == (0, 0, 0, 0, 8)
    assert o.breakdown_tol == 1e-14 and o.inner_tol == 1e-4 and o.max_refine == 30
    assert o.contraction == ekcg.CONTRACTION["split"]
    assert o.deflate == 0
    assert ctypes.sizeof(ekcg.ekcg_opts) == 64
    assert ekcg.strerror(0) == "ok"
    assert "breakdown" in ekcg.strerror(-3)


def test_header_documents_every_entry_point():
    txt = open(ekcg.HEADER).read()
    for nm in ekcg.header_functions():
        i = txt.index(nm + "(")
        assert "/*" in txt[max(0, i - 1500):i], nm
