"""Seeded synthetic inputs shaped like the paper's test problems.

This module builds inputs only: SPD stencil matrices in CSR form, t-way geometric
partitions and right-hand sides.  It contains none of the solver's arithmetic, so the
oracle and the CUDA path can both take their inputs from it without sharing method code.

The paper's matrices (Section 4, Table 1) are Poisson2D = gallery('poisson',100) and four
FreeFem++ convection-diffusion matrices (Nh2D, Sky2D, Sky3D, Ani3D) partitioned with METIS.
Only Poisson2D can be rebuilt exactly; the others are replaced by stencil matrices with
the same character (skyscraper coefficient jumps, anisotropic layers, smooth random
coefficients), and METIS by geometric strips and boxes.

Matrix form (edge form of a cell-centred finite-volume diffusion operator):
    A = sum_{edges (p,q)} w_pq (e_p - e_q)(e_p - e_q)^T + sum_{boundary faces of p} w_p e_p e_p^T
with w_pq = a_axis * 2 k_p k_q / (k_p + k_q) (harmonic mean of the node coefficients) and
w_p = a_axis * k_p for a face on the Dirichlet boundary.  With k == 1 and a == 1 this is
exactly gallery('poisson', N): 4 on the diagonal and -1 off it in 2D (6 / -1 in 3D).
Nodes are numbered x fastest: node(i, j[, k]) = i + nx*(j + ny*k).
"""
from __future__ import annotations

import dataclasses
import numpy as np
import scipy.sparse as sp

__all__ = [
    "CSR", "Problem", "stencil_matrix", "kappa_skyscraper3d", "kappa_rectangles2d",
    "kappa_gaussian_field2d", "partition_strips", "partition_boxes", "box_factors",
    "rhs_uniform", "poisson2d", "ani3d", "sky3d", "diffusion2d", "batched_systems",
    "named_problem",
]


@dataclasses.dataclass
class CSR:
    """Square CSR matrix: int64 row pointers, int32 sorted column indices, float64 values."""
    n: int
    rowptr: np.ndarray
    colind: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.val, self.colind, self.rowptr), shape=(self.n, self.n))


@dataclasses.dataclass
class Problem:
    """One linear system A x = b with its t-way partition (part[i] in [0, t))."""
    name: str
    A: CSR
    b: np.ndarray
    t: int
    part: np.ndarray
    shape: tuple


def _node_index(shape):
    return np.arange(int(np.prod(shape)), dtype=np.int64).reshape(shape[::-1])


def stencil_matrix(shape, kappa=None, aniso=None) -> CSR:
    """Assemble the 5-point (2D) or 7-point (3D) diffusion matrix in edge form.

    shape: (nx, ny) or (nx, ny, nz).  kappa: node coefficients with array shape
    shape[::-1] (z, y, x ordering), default 1.  aniso: per-axis factor (x, y[, z]).
    """
    dim = len(shape)
    n = int(np.prod(shape))
    if kappa is None:
        kappa = np.ones(shape[::-1])
    kappa = np.asarray(kappa, dtype=np.float64).reshape(shape[::-1])
    if aniso is None:
        aniso = (1.0,) * dim
    idx = _node_index(shape)
    diag = np.zeros(shape[::-1])
    rows, cols, vals = [], [], []
    for ax in range(dim):
        arr_ax = dim - 1 - ax           # x is the last array axis
        a = float(aniso[ax])
        lo = [slice(None)] * dim
        hi = [slice(None)] * dim
        lo[arr_ax] = slice(0, -1)
        hi[arr_ax] = slice(1, None)
        kp, kq = kappa[tuple(lo)], kappa[tuple(hi)]
        w = a * (2.0 * kp * kq / (kp + kq))
        p, q = idx[tuple(lo)].ravel(), idx[tuple(hi)].ravel()
        rows += [p, q]
        cols += [q, p]
        vals += [-w.ravel(), -w.ravel()]
        diag[tuple(lo)] += w
        diag[tuple(hi)] += w
        # Dirichlet boundary faces on both ends of this axis
        first = [slice(None)] * dim
        last = [slice(None)] * dim
        first[arr_ax] = slice(0, 1)
        last[arr_ax] = slice(-1, None)
        diag[tuple(first)] += a * kappa[tuple(first)]
        diag[tuple(last)] += a * kappa[tuple(last)]
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    M = sp.coo_matrix((v, (r, c)), shape=(n, n)).tocsr()
    M.sort_indices()
    return CSR(n=n, rowptr=M.indptr.astype(np.int64), colind=M.indices.astype(np.int32),
               val=M.data.astype(np.float64))


def kappa_skyscraper3d(N: int, block: int = 8, high: float = 1e3) -> np.ndarray:
    """Piecewise-constant coefficient: `high` on 8^3 blocks whose block-index sum is odd, else 1."""
    g = np.arange(N) // block
    s = g[:, None, None] + g[None, :, None] + g[None, None, :]
    return np.where(s % 2 == 1, high, 1.0)


def kappa_rectangles2d(N: int, rng: np.random.Generator, nrect: int = 4,
                       contrast: float = 4.0) -> np.ndarray:
    """Background 1 plus `nrect` axis-aligned rectangles, side U{4..N/2},
    value 10^U(0, contrast) (contrast 4: jumps up to 1e4)."""
    k = np.ones((N, N))
    for _ in range(nrect):
        wx, wy = rng.integers(4, N // 2 + 1, size=2)
        x0 = rng.integers(0, N - wx + 1)
        y0 = rng.integers(0, N - wy + 1)
        k[y0:y0 + wy, x0:x0 + wx] = 10.0 ** rng.uniform(0.0, contrast)
    return k


def kappa_gaussian_field2d(N: int, seed: int, corr: float = 16.0) -> np.ndarray:
    """log-kappa field: white noise N(0,1) convolved periodically with a Gaussian of
    standard deviation `corr` cells (via FFT), normalised to mean 0 and std 1.
    Returns log kappa (the caller exponentiates)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    z = rng.standard_normal((N, N))
    f = np.fft.fftfreq(N)
    g = np.exp(-2.0 * (np.pi * corr) ** 2 * (f[:, None] ** 2 + f[None, :] ** 2))
    y = np.real(np.fft.ifft2(np.fft.fft2(z) * g))
    return (y - y.mean()) / y.std()


def partition_strips(n: int, t: int) -> np.ndarray:
    """Strip partition of the natural ordering: domain(i) = floor(i*t/n)."""
    i = np.arange(n, dtype=np.int64)
    return ((i * t) // n).astype(np.int32)


def box_factors(shape, t: int):
    """Split t (a power of two) into per-axis box counts: each factor of 2 goes to the axis
    whose current box extent is largest, ties to the lowest axis (x first)."""
    if t < 1 or (t & (t - 1)) != 0:
        raise ValueError("box partitions need t to be a power of two")
    parts = [1] * len(shape)
    m = t
    while m > 1:
        ext = [shape[a] / parts[a] for a in range(len(shape))]
        a = int(np.argmax(ext))        # argmax returns the first maximum: ties to x
        parts[a] *= 2
        m //= 2
    return tuple(parts)


def partition_boxes(shape, t: int) -> np.ndarray:
    """Box partition: box id = bx + px*(by + py*bz), b_axis = floor(i_axis * p_axis / N_axis)."""
    parts = box_factors(shape, t)
    coords = np.meshgrid(*[np.arange(N, dtype=np.int64) for N in shape[::-1]], indexing="ij")
    coords = coords[::-1]               # x, y[, z] arrays in (z, y, x) layout
    bid = np.zeros(shape[::-1], dtype=np.int64)
    mult = 1
    for ax, N in enumerate(shape):
        b = (coords[ax] * parts[ax]) // N
        bid += b * mult
        mult *= parts[ax]
    return bid.ravel().astype(np.int32)


def rhs_uniform(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """b ~ U(lo, hi), NumPy PCG64 with the given seed."""
    return np.random.Generator(np.random.PCG64(seed)).uniform(lo, hi, n)


def poisson2d(N: int = 100, t: int = 4, seed: int = 0, partition: str = "strips") -> Problem:
    A = stencil_matrix((N, N))
    part = partition_strips(A.n, t) if partition == "strips" else partition_boxes((N, N), t)
    return Problem(f"Poisson2D-{N}", A, rhs_uniform(A.n, seed), t, part, (N, N))


def ani3d(N: int = 128, t: int = 32, seed: int = 1) -> Problem:
    A = stencil_matrix((N, N, N), aniso=(1.0, 1.0, 1e-3))
    return Problem(f"Ani3D-{N}", A, rhs_uniform(A.n, seed), t, partition_boxes((N, N, N), t), (N, N, N))


def sky3d(N: int = 96, t: int = 16, seed: int = 2) -> Problem:
    A = stencil_matrix((N, N, N), kappa=kappa_skyscraper3d(N))
    return Problem(f"Sky3D-{N}", A, rhs_uniform(A.n, seed), t, partition_boxes((N, N, N), t), (N, N, N))


def diffusion2d(N: int, kappa=None, t: int = 16, seed: int = 4) -> Problem:
    A = stencil_matrix((N, N), kappa=kappa)
    return Problem(f"Diff2D-{N}", A, rhs_uniform(A.n, seed), t, partition_boxes((N, N), t), (N, N))


def batched_systems(count: int = 256, nmin: int = 32, nmax: int = 256, t: int = 8, seed: int = 3,
                    contrast: float = 4.0):
    """`count` independent 2D diffusion systems, grid side N ~ U{nmin..nmax}, four random
    coefficient rectangles each (values 10^U(0, contrast)), 4x2 box partition (t=8),
    b ~ U(-1,1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(count):
        N = int(rng.integers(nmin, nmax + 1))
        kap = kappa_rectangles2d(N, rng, contrast=contrast)
        A = stencil_matrix((N, N), kappa=kap)
        b = rng.uniform(-1.0, 1.0, A.n)
        out.append(Problem(f"batched-{k}-{N}", A, b, t, partition_boxes((N, N), t), (N, N)))
    return out


def named_problem(name: str, **kw) -> Problem:
    """Problems by name at their full sizes (or overridden sizes)."""
    if name == "poisson2d":
        return poisson2d(**kw)
    if name == "ani3d":
        return ani3d(**kw)
    if name == "sky3d":
        return sky3d(**kw)
    raise KeyError(name)
