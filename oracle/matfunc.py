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
                     uses it as a second, independent route in tests, and as
                     the matrix function of the projected matrices when those
                     are not diagonalisable.
* ``jordan_form``, ``fun_jordan``, ``sign_jordan`` -- the spectral definition
                     for a matrix that cannot be diagonalised (Sec. 1, after
                     Eq. 4: derived from the Cauchy integral, Eq. 3, with the
                     Jordan decomposition A = X J X^{-1}). On a Jordan block
                     J_k(l) = l I + N (N the shift, N^k = 0) the integral gives
                     f(J_k(l)) = sum_{j<k} f^{(j)}(l) / j! N^j; every derivative
                     of sgn vanishes off the imaginary axis, so
                     sgn(J_k(l)) = sgn(Re l) I_k.
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


def jordan_form(blocks) -> np.ndarray:
    """J = diag(J_{k_1}(l_1), ...) for blocks [(l_1, k_1), ...]: each block has
    l on its diagonal and ones on its superdiagonal."""
    n = sum(int(k) for _, k in blocks)
    J = np.zeros((n, n), dtype=np.complex128)
    o = 0
    for lam, k in blocks:
        for i in range(int(k)):
            J[o + i, o + i] = lam
            if i + 1 < k:
                J[o + i, o + i + 1] = 1.0
        o += int(k)
    return J


def fun_jordan(X: np.ndarray, blocks, deriv) -> np.ndarray:
    """f(A) for A = X J X^{-1}, J = jordan_form(blocks): X diag(f(J_k(l))) X^{-1}
    with f(J_k(l)) = sum_{j<k} deriv(l, j) / j! N^j, deriv(l, j) = f^{(j)}(l)."""
    n = X.shape[0]
    F = np.zeros((n, n), dtype=np.complex128)
    o = 0
    for lam, k in blocks:
        k = int(k)
        N = np.eye(k, k, 1, dtype=np.complex128)
        Nj = np.eye(k, dtype=np.complex128)
        fact = 1.0
        for j in range(k):
            if j > 0:
                Nj = Nj @ N
                fact *= j
            F[o:o + k, o:o + k] += deriv(lam, j) / fact * Nj
        o += k
    return X @ F @ np.linalg.inv(X)


def sign_jordan(X: np.ndarray, blocks) -> np.ndarray:
    """sgn(A) for A = X J X^{-1} (no eigenvalue on the imaginary axis): the
    Jordan-form definition with f = sgn, whose derivatives all vanish."""
    for lam, _ in blocks:
        if np.real(lam) == 0.0:
            raise ValueError("sgn is undefined for an eigenvalue on the imaginary axis")
    return fun_jordan(X, blocks, lambda lam, j: np.sign(np.real(lam)) if j == 0 else 0.0)
