"""Seeded synthetic inputs: SU(3) gauge fields and spinor sources.

This module only draws random numbers and builds input data. It holds none of
the method's arithmetic (no Dirac operator, no Krylov step, no sign function),
so both the CPU oracle's tests and the CUDA path's tests and benchmark draw
their inputs from here.

Canonical host layouts (row-major numpy arrays, complex128):

* gauge links ``U[t, z, y, x, nu, a, b]`` with ``nu = 0..3`` for the
  directions x, y, z, t (the paper's 1..4 of Eq. 2), ``a, b`` colour indices;
* spinors ``psi[t, z, y, x, s, c]`` with spin ``s = 0..3`` and colour
  ``c = 0..2``; flattened, the site index is ``n = x + Lx*(y + Ly*(z + Lz*t))``
  and the vector index is ``12*n + 3*s + c``.

Gauge fields follow the recipe U = exp(i eps X) with X = sum_a w_a lambda_a / 2,
lambda_a the eight Gell-Mann matrices and w_a ~ N(0, 1) drawn from
``numpy.random.default_rng(seed)`` in (t, z, y, x, nu, a) order.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gell_mann",
    "random_su3_field",
    "unit_gauge_field",
    "gaussian_source",
    "point_source",
    "ones_source",
    "random_gauge_transform",
    "lattice_shape",
]


def lattice_shape(dims):
    """(Lx, Ly, Lz, Lt) -> the canonical array shape (Lt, Lz, Ly, Lx)."""
    lx, ly, lz, lt = (int(d) for d in dims)
    return (lt, lz, ly, lx)


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3), Hermitian and traceless."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1] = -1j
    lam[1][1, 0] = 1j
    lam[2][0, 0] = 1
    lam[2][1, 1] = -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2] = -1j
    lam[4][2, 0] = 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2] = -1j
    lam[6][2, 1] = 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


def _expi_hermitian(X: np.ndarray, eps: float) -> np.ndarray:
    """exp(i*eps*X) for a stack of Hermitian 3x3 matrices, via eigh."""
    w, Q = np.linalg.eigh(X)
    ph = np.exp(1j * eps * w)
    return np.einsum("...ab,...b,...cb->...ac", Q, ph, Q.conj())


def random_su3_field(dims, eps: float, seed: int = 0) -> np.ndarray:
    """SU(3) links U = exp(i eps X), X Gaussian in su(3); shape (Lt,Lz,Ly,Lx,4,3,3)."""
    shp = lattice_shape(dims)
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(shp + (4, 8))
    X = np.einsum("...a,aij->...ij", w, gell_mann()) * 0.5
    return _expi_hermitian(X, float(eps))


def unit_gauge_field(dims) -> np.ndarray:
    """The free field U = 1 on every link."""
    shp = lattice_shape(dims)
    U = np.zeros(shp + (4, 3, 3), dtype=np.complex128)
    U[..., :, :] = np.eye(3)
    return U


def random_gauge_transform(dims, seed: int = 7) -> np.ndarray:
    """Random site-local SU(3) matrices g_n, shape (Lt,Lz,Ly,Lx,3,3)."""
    shp = lattice_shape(dims)
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(shp + (8,))
    X = np.einsum("...a,aij->...ij", w, gell_mann()) * 0.5
    return _expi_hermitian(X, 1.0)


def gaussian_source(dims, seed: int = 1) -> np.ndarray:
    """Complex Gaussian spinor: re and im each N(0,1), re drawn first."""
    shp = lattice_shape(dims) + (4, 3)
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(shp)
    im = rng.standard_normal(shp)
    return re + 1j * im


def point_source(dims, spin: int, colour: int, site=(0, 0, 0, 0)) -> np.ndarray:
    """delta at site (x, y, z, t), spin ``spin``, colour ``colour``."""
    shp = lattice_shape(dims) + (4, 3)
    b = np.zeros(shp, dtype=np.complex128)
    x, y, z, t = site
    b[t, z, y, x, spin, colour] = 1.0
    return b


def ones_source(dims) -> np.ndarray:
    """x = (1, 1, ..., 1), the source of the paper's convergence figure."""
    shp = lattice_shape(dims) + (4, 3)
    return np.ones(shp, dtype=np.complex128)


def probe_vectors(n: int, count: int, seed: int = 12345) -> np.ndarray:
    """``count`` complex Gaussian probe vectors of length n (re, im ~ N(0,1)),
    used to sketch a long result vector by a few inner products."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((count, n))
    im = rng.standard_normal((count, n))
    return re + 1j * im
