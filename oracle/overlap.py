"""The overlap operator at nonzero chemical potential (Sec. 1, Eq. 1), FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``overlap_apply``         -- D_ov(mu) x = x + gamma5 sgn(H_w(mu)) x (Eq. 1).
* ``overlap_adjoint_apply`` -- D_ov(mu)^dag x = x + sgn(H_w(mu))^dag gamma5 x,
                               with sgn(H_w(mu))^dag = sgn(H_w(mu)^dag) =
                               sgn(H_w(-mu)) (H_w(mu)^dag = H_w(-mu) from Eq. 2).
* ``overlap_dense``         -- the dense matrix 1 + gamma5 sgn(H_w(mu)) by the
                               spectral definition (Eqs. 4-6), small lattices.
* ``lr_adjoint``            -- LR deflation data of H_w(mu)^dag from those of
                               H_w(mu) (Eq. 20): left and right eigenvectors swap
                               and the eigenvalues are conjugated, so one
                               eigenvector computation serves sgn and its
                               adjoint (Sec. 5).

gamma5 = diag(1, 1, -1, -1) on the spin index of every site (chiral basis).
"""
from __future__ import annotations

import numpy as np

from . import dirac, matfunc


def gamma5_apply(x: np.ndarray) -> np.ndarray:
    """gamma5 x for a canonical spinor (..., spin 4, colour 3)."""
    y = np.array(x, dtype=np.complex128, copy=True)
    y[..., 2:, :] *= -1.0
    return y


def overlap_apply(sign_apply, x: np.ndarray) -> np.ndarray:
    """Eq. 1: x + gamma5 sgn(H_w) x, with sign_apply(x) = sgn(H_w(mu)) x."""
    return x + gamma5_apply(sign_apply(x))


def overlap_adjoint_apply(sign_apply_minus_mu, x: np.ndarray) -> np.ndarray:
    """D_ov^dag x = x + sgn(H_w(-mu)) gamma5 x, with sign_apply_minus_mu(x) =
    sgn(H_w(-mu)) x."""
    return x + sign_apply_minus_mu(gamma5_apply(x))


def overlap_dense(U: np.ndarray, mu: float, m_w: float) -> np.ndarray:
    """Dense D_ov(mu) = 1 + gamma5 sgn(H_w(mu)) (Eq. 1 with Eqs. 4-6)."""
    A = dirac.hermitian_wilson(U, mu, m_w).toarray()
    V = A.shape[0] // 12
    g5 = dirac.gamma5_matrix(V).toarray()
    return np.eye(A.shape[0]) + g5 @ matfunc.sign_eig(A)


def lr_adjoint(lam: np.ndarray, R: np.ndarray, L: np.ndarray):
    """(lam, R, L) of A (A R = R diag(lam), L^dag A = diag(lam) L^dag,
    L^dag R = I) -> the same triple for A^dag: (conj(lam), L, R)."""
    return np.conj(lam), L, R
