"""Oracle computations of the full-size parity tests, run in spawned worker
processes (tests only).

Each job rebuilds its inputs from the seeded generators. The critical
eigenpairs come from the oracle's sparse eigensolver (ARPACK on A^2, Sec. 5):
the right vectors of H_w(mu) and, for LR deflation, those of
H_w(-mu) = H_w(mu)^dag as the left vectors (Eq. 20), in separate jobs so that
they run side by side. The oracle's result of the algorithm the CUDA path runs
(Eq. 19 for Schur, Eq. 22 for LR, Eq. 11 without deflation) is a second job.
The workers never touch the GPU; they are started with the ``spawn`` method,
so a parent that already holds a CUDA context is safe.
"""
import numpy as np

from oracle import dirac, eigen, krylov
from paper_0710_0341_gb300 import synth


def _operator(dims, eps, m_w, mu):
    return dirac.hermitian_wilson(synth.random_su3_field(dims, eps, 0), mu, m_w)


def right_pairs(dims, eps, m_w, mu, m, tol=1e-10):
    """The m critical eigenpairs (lambda, R) of H_w(mu) with their residuals."""
    lam, R, res = eigen._critical_right_sparse(_operator(dims, eps, m_w, mu), m, m + max(10, m // 4), tol)
    return {"lam": lam, "R": R, "res": float(np.max(res))}


def deflated_solve(dims, eps, m_w, mu, k, scheme, lam, R, L=None):
    """The oracle's deflated approximation of sgn(H_w(mu)) b (complex Gaussian
    source, seed 1): Schur (Eq. 19, Schur vectors of span(R), Eq. 13) or LR
    (Eq. 22). Returns y and, for Schur, the (S, T) it used."""
    A = _operator(dims, eps, m_w, mu)
    b = synth.gaussian_source(dims, 1).ravel()
    if scheme == "schur":
        S, T = eigen.schur_from_right(A, R)
        return {"y": krylov.sign_schur(A, b, k, S, T), "S": S, "T": T}
    return {"y": krylov.sign_lr(A, b, k, R, lam, L)}


def undeflated_case(dims, eps, m_w, mu, k):
    """The oracle's Eq. 11 approximation beta V_k sgn(H_k) e_1 for the complex
    Gaussian source (seed 1), with Im <b, y> / |b|^2 (zero in exact arithmetic
    at mu = 0, where H_w and H_k are Hermitian)."""
    A = _operator(dims, eps, m_w, mu)
    b = synth.gaussian_source(dims, 1).ravel()
    y = krylov.sign_arnoldi(A, b, k)
    return {"y": y, "im_ratio": float(np.vdot(b, y).imag / np.vdot(b, b).real)}
