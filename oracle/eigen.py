"""Critical eigenpairs for deflation (Sec. 3, Eq. 13; Sec. 4, Eq. 20; Sec. 5).

TEST INFRASTRUCTURE ONLY (see the package docstring).

"Critical" eigenvalues are those closest to the discontinuity of sgn on the
imaginary axis; the reading used throughout is the m eigenvalues of smallest
|Re lambda|, ties broken by |Im lambda| and then by index.

* ``critical_dense``   -- dense eigendecomposition (small lattices), returns
                          lambda, right eigenvectors R and left eigenvectors L
                          normalised so that L^dag R = I (Eq. 20).
* ``schur_from_right`` -- orthonormal Schur vectors S_m and upper triangular
                          T_m with A S_m = S_m T_m (Eq. 13) spanning the same
                          space as the right eigenvectors.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def critical_order(lam: np.ndarray) -> np.ndarray:
    """Indices sorting eigenvalues by |Re|, then |Im|, then index."""
    lam = np.asarray(lam)
    return np.lexsort((np.arange(lam.size), np.abs(lam.imag), np.abs(lam.real)))


def critical_dense(A: np.ndarray, m: int):
    """The m critical eigenpairs of a dense matrix, with left vectors (Eq. 20)."""
    lam, Lv, Rv = sla.eig(A, left=True, right=True)
    idx = critical_order(lam)[:m]
    lam_m = lam[idx]
    R = Rv[:, idx]
    L = Lv[:, idx]
    R = R / np.linalg.norm(R, axis=0)[None, :]
    # scale left vectors so that l_i^dag r_i = 1 (L^dag R = I for distinct lambda)
    d = np.einsum("ni,ni->i", L.conj(), R)
    L = L / d.conj()[None, :]
    return lam_m, R, L


def schur_from_right(A, R: np.ndarray):
    """Schur vectors of span(R): S orthonormal, T = S^dag A S upper triangular."""
    Q, _ = np.linalg.qr(R)
    AQ = np.column_stack([A @ Q[:, i] for i in range(Q.shape[1])])
    T0 = Q.conj().T @ AQ
    T, Z = sla.schur(T0, output="complex")
    return Q @ Z, T
