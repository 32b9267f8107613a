"""Oracle computations of the full-size parity tests, run in spawned worker
processes (tests only).

Each job rebuilds its inputs from the seeded generators, computes the
critical eigenpairs with the oracle's sparse eigensolver (ARPACK on A^2,
Sec. 5) and the oracle's result of the same algorithm the CUDA path runs
(Eq. 19 for Schur, Eq. 22 for LR, Eq. 11 without deflation). The workers
never touch the GPU; they are started with the ``spawn`` method, so a parent
that already holds a CUDA context is safe.
"""
import numpy as np

from oracle import dirac, eigen, krylov
from paper_0710_0341_gb300 import synth


def deflated_case(dims, eps, m_w, mu, m, k, schemes, tol=1e-10):
    """Critical eigenpairs of H_w(mu) and the oracle's deflated approximations
    of sgn(H_w(mu)) b for b the complex Gaussian source (seed 1).

    Returns a dict with lam, R, L (L^dag R = I), S, T (A S = S T) and one
    oracle result per scheme in ``schemes`` ("schur", "lr")."""
    U = synth.random_su3_field(dims, eps, 0)
    A = dirac.hermitian_wilson(U, mu, m_w)
    b = synth.gaussian_source(dims, 1).ravel()
    nev = m + max(10, m // 4)
    if mu == 0.0:
        # H_w(0) is Hermitian: the left eigenvectors are the right ones (Eq. 20)
        lam, R, res = eigen._critical_right_sparse(A, m, nev, tol)
        L = R / np.einsum("ni,ni->i", R.conj(), R).conj()[None, :]
    elif "lr" in schemes:
        lam, R, L, res = eigen.critical_sparse(A, dirac.hermitian_wilson(U, -mu, m_w), m, nev, tol)
    else:
        lam, R, res = eigen._critical_right_sparse(A, m, nev, tol)
        L = None
    S, T = eigen.schur_from_right(A, R)
    out = {"lam": lam, "R": R, "L": L, "S": S, "T": T, "res": float(np.max(res))}
    if "schur" in schemes:
        out["schur"] = krylov.sign_schur(A, b, k, S, T)
    if "lr" in schemes:
        out["lr"] = krylov.sign_lr(A, b, k, R, lam, L)
    return out


def undeflated_case(dims, eps, m_w, mu, k):
    """The oracle's Eq. 11 approximation beta V_k sgn(H_k) e_1 for the complex
    Gaussian source (seed 1), with Im <b, y> / |b|^2 (zero in exact arithmetic
    at mu = 0, where H_w and H_k are Hermitian)."""
    U = synth.random_su3_field(dims, eps, 0)
    A = dirac.hermitian_wilson(U, mu, m_w)
    b = synth.gaussian_source(dims, 1).ravel()
    y = krylov.sign_arnoldi(A, b, k)
    return {"y": y, "im_ratio": float(np.vdot(b, y).imag / np.vdot(b, b).real)}
