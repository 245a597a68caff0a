"""Host part of the GPU block Jacobi preconditioner (IC(0) factors and solve levels, computed
in C++ by libekcg) against the oracle's IC(0) (right-looking with dropped updates, an
independent implementation), on the CPU: ekcg_block_ic0_host does no device work."""
import os

import numpy as np
import pytest

import workloads as wl
from oracle import ekcg_ref as o

ekcg = pytest.importorskip("paper_1804_10629_gb300.ekcg")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not os.path.exists(ekcg.LIB_PATH):
        from paper_1804_10629_gb300 import build
        build.build()


@pytest.mark.parametrize("shape,nb", [((12, 12), 8), ((9, 7, 5), 8), ((30, 20), 16)])
def test_block_ic0_matches_the_oracle(shape, nb):
    kap = None
    if len(shape) == 2:
        kap = wl.kappa_rectangles2d(shape[0], np.random.default_rng(3), contrast=3.0)[:shape[1]]
    A = wl.stencil_matrix(shape, kappa=kap)
    bpart = wl.partition_boxes(shape, nb)
    lval, fl, bl = ekcg.ekcg_block_ic0_host(A, bpart)
    M = o.BlockJacobi(A, bpart, "ic0")
    L = M.L_dense()
    Lg = np.zeros((A.n, A.n))
    for i in range(A.n):
        for e in range(A.rowptr[i], A.rowptr[i + 1]):
            Lg[i, A.colind[e]] = lval[e]
    np.testing.assert_allclose(Lg, L, rtol=1e-12, atol=1e-14)


def test_levels_are_a_valid_schedule():
    """Every row's forward level exceeds the levels of the rows its L equation reads, and
    its backward level exceeds those of the rows its L^T equation reads; levels are tight
    (a row with level l > 0 reads a row of level l - 1)."""
    shape = (11, 9, 4)
    A = wl.stencil_matrix(shape)
    bpart = wl.partition_boxes(shape, 4)
    lval, fl, bl = ekcg.ekcg_block_ic0_host(A, bpart)
    reads_f = [[] for _ in range(A.n)]
    reads_b = [[] for _ in range(A.n)]
    for i in range(A.n):
        for e in range(A.rowptr[i], A.rowptr[i + 1]):
            k = A.colind[e]
            if k < i and lval[e] != 0.0:
                reads_f[i].append(k)      # L_ik: row i of L y = x reads y_k
                reads_b[k].append(i)      # column k of L: row k of L^T z = y reads z_i
    for i in range(A.n):
        assert all(fl[i] > fl[k] for k in reads_f[i])
        assert all(bl[i] > bl[k] for k in reads_b[i])
        assert fl[i] == (max(fl[k] for k in reads_f[i]) + 1 if reads_f[i] else 0)
        assert bl[i] == (max(bl[k] for k in reads_b[i]) + 1 if reads_b[i] else 0)
    # a 3D box of nx x ny x nz rows has nx + ny + nz - 2 wavefront levels
    assert fl.max() + 1 == max(int(np.sum(bpart == d)) > 0 for d in range(4)) * (6 + 5 + 4 - 2)


def test_block_ic0_rejects_bad_input():
    A = wl.stencil_matrix((6, 6))
    with pytest.raises(ekcg.EkcgError):
        ekcg.ekcg_block_ic0_host(A, np.full(A.n, -1, dtype=np.int32))
