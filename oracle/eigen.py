"""Critical eigenpairs for deflation (Sec. 3, Eq. 13; Sec. 4, Eq. 20; Sec. 5).

TEST INFRASTRUCTURE ONLY (see the package docstring).

"Critical" eigenvalues are those closest to the discontinuity of sgn on the
imaginary axis; the reading used throughout is the m eigenvalues of smallest
|Re lambda|, ties broken by |Im lambda| and then by index.

* ``critical_dense``   -- dense eigendecomposition (small lattices), returns
                          lambda, right eigenvectors R and left eigenvectors L
                          normalised so that L^dag R = I (Eq. 20).
* ``critical_sparse``  -- the same for a sparse A too large for a dense
                          decomposition: ARPACK on A^2 (its eigenvalues of
                          smallest real part), Rayleigh-Ritz with A, and the
                          left vectors from A^dag (Eq. 20).
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


def _critical_right_sparse(A, m: int, nev: int, tol: float):
    """Right eigenpairs of the m critical eigenvalues of sparse A (see
    critical_sparse), sorted by critical_order, with their residual norms."""
    import scipy.sparse.linalg as spla

    N = A.shape[0]
    B = spla.LinearOperator((N, N), matvec=lambda v: A @ (A @ v), dtype=np.complex128)
    _, W = spla.eigs(B, k=nev, which="SR", ncv=min(N - 1, 2 * nev + 60), tol=tol, maxiter=100000)
    Q, _ = np.linalg.qr(W)
    AQ = np.column_stack([A @ Q[:, i] for i in range(Q.shape[1])])
    lam, Y = np.linalg.eig(Q.conj().T @ AQ)
    o = critical_order(lam)
    lam, R = lam[o], (Q @ Y)[:, o]
    # Re(lambda^2) = Re^2 - Im^2: every eigenvalue ARPACK did not return has
    # Re(lambda^2) >= theta, the largest it did return, hence Re^2 >= theta;
    # so none is more critical than the m-th kept one while Re_m^2 <= theta
    theta = float(np.max((lam * lam).real))
    if not abs(lam[m - 1].real) ** 2 <= theta:
        raise ValueError(f"nev={nev} does not bracket the {m} critical eigenvalues; increase nev")
    R = R[:, :m] / np.linalg.norm(R[:, :m], axis=0)[None, :]
    lam = lam[:m]
    res = np.linalg.norm(np.column_stack([A @ R[:, i] for i in range(m)]) - R * lam[None, :], axis=0)
    return lam, R, res


def critical_sparse(A, A_adj, m: int, nev: int | None = None, tol: float = 1e-13):
    """The m critical eigenpairs of a sparse A with left vectors (Eq. 20):
    (lambda, R, L, residual of A R = R Lambda per column). The right vectors
    are the critical eigenvectors of A from restarted Arnoldi on A^2 (ARPACK,
    scipy.sparse.linalg.eigs, smallest real part; the map lambda -> lambda^2
    makes the eigenvalues closest to the imaginary axis extremal), followed by
    a Rayleigh-Ritz step with A. The left vectors are the right eigenvectors of
    A_adj = A^dag (for H_w(mu) this is H_w(-mu)) with eigenvalue conj(lambda),
    scaled so that l_i^dag r_i = 1."""
    nev = nev or m + max(10, m // 4)
    lam, R, res = _critical_right_sparse(A, m, nev, tol)
    lamL, Lv, _ = _critical_right_sparse(A_adj, m, nev, tol)
    return lam, R, pair_left(lam, R, lamL, Lv), res


def pair_left(lam, R, lamL, Lv):
    """Left vectors for the right eigenpairs (lam, R) from the right eigenpairs
    (lamL, Lv) of A^dag: l_i is the vector with eigenvalue conj(lambda_i),
    scaled so that l_i^dag r_i = 1 (Eq. 20)."""
    m = len(lam)
    idx = [int(np.argmin(np.abs(lamL - np.conj(z)))) for z in lam]
    if len(set(idx)) != m:
        raise ValueError("left and right critical eigenvalues do not pair up")
    L = Lv[:, idx]
    d = np.einsum("ni,ni->i", L.conj(), R)
    return L / d.conj()[None, :]


def schur_from_right(A, R: np.ndarray):
    """Schur vectors of span(R): S orthonormal, T = S^dag A S upper triangular."""
    Q, _ = np.linalg.qr(R)
    AQ = np.column_stack([A @ Q[:, i] for i in range(Q.shape[1])])
    T0 = Q.conj().T @ AQ
    T, Z = sla.schur(T0, output="complex")
    return Q @ Z, T
