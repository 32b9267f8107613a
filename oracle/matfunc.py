"""Scalar and matrix sign function (Sec. 1, Eqs. 4-6), plain FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``sgn_scalar``  -- Eq. 5: sgn(z) = z / sqrt(z^2) = sgn(Re z), principal root.
* ``sign_eig``    -- Eq. 4 with f = sgn, i.e. Eq. 6: A = U diag(l) U^-1 and
                     sgn(A) = U diag(sgn Re l) U^-1.  ``sign_eig_apply`` forms
                     sgn(A) b by solving U z = b instead of inverting U.
* ``sign_newton`` -- the scaled Newton (Roberts) iteration for the matrix
                     sign (the matrix iterations Sec. 2 cites):
                     X_0 = A, X_{i+1} = (c_i X_i + X_i^{-1}/c_i)/2 with the
                     determinant scaling c_i = |det X_i|^{-1/n}.  The oracle
                     uses it only as a second, independent route in tests.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def sgn_scalar(z):
    """Eq. 5: z / sqrt(z^2) with the cut of sqrt on the negative real axis."""
    z = np.asarray(z, dtype=np.complex128)
    return z / np.sqrt(z * z)


def sign_eig(A: np.ndarray) -> np.ndarray:
    """sgn(A) = U diag(sgn(Re lambda_i)) U^{-1} (Eqs. 4 and 6), dense."""
    lam, U = sla.eig(A)
    s = np.sign(lam.real)
    return (U * s[None, :]) @ np.linalg.inv(U)


def sign_eig_apply(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    """sgn(A) b by the spectral definition (Eq. 4), via a solve with U."""
    lam, U = sla.eig(A)
    z = sla.lu_solve(sla.lu_factor(U), b)
    if z.ndim == 1:
        return U @ (np.sign(lam.real) * z)
    return U @ (np.sign(lam.real)[:, None] * z)


def sign_newton(A: np.ndarray, tol: float = None, max_iter: int = 100):
    """Scaled Newton iteration for sgn(A); returns (S, iterations)."""
    X = np.array(A, dtype=np.complex128, copy=True)
    n = X.shape[0]
    if tol is None:
        tol = 10 * n * np.finfo(float).eps
    scale = True
    for it in range(1, max_iter + 1):
        Xi = np.linalg.inv(X)
        if scale:
            _, logdet = np.linalg.slogdet(X)
            c = np.exp(-logdet / n)
        else:
            c = 1.0
        Xn = 0.5 * (c * X + Xi / c)
        diff = np.linalg.norm(Xn - X, 1)
        nrm = np.linalg.norm(Xn, 1)
        X = Xn
        if diff < 1e-2 * nrm:
            scale = False
        if diff <= tol * nrm:
            return X, it
    return X, max_iter
