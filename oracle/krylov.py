"""Arnoldi function approximation with Schur and LR deflation (Secs. 2-4).

TEST INFRASTRUCTURE ONLY (see the package docstring).

``A`` is anything with ``A @ v`` (a scipy sparse matrix or a dense array);
vectors are flat complex128 arrays.  The small-matrix function f(H) is taken
by the spectral definition (Eq. 4) on the small matrix, so the oracle's small
sign is independent of the Newton iteration the CUDA path uses.

* ``arnoldi``          -- Eq. 7: A V_k = V_k H_k + beta_k v_{k+1} e_k^T,
                          v_1 = x/|x|, orthogonalised by classical
                          Gram-Schmidt applied twice (CGS2); optional fixed
                          block ``S`` against which every vector is also
                          orthogonalised (the modified Arnoldi of Eq. 14).
* ``sign_arnoldi``     -- Eq. 11: f(A) x ~ beta V_k f(H_k) e_1.
* ``sign_schur``       -- Eqs. 14-19: H = [[T, X], [0, H_k]], X = S^dag A V_k;
                          f(A)x ~ S f(T) S^dag x + (S V_k) [Y; f(H_k)] beta e_1
                          with Y from the Sylvester equation of Eq. 18.
* ``sign_schur_block`` -- Eq. 16 directly: Q f(H) Q^dag x on the full block H
                          (a second route to the same number, Eq. 17).
* ``sign_lr``          -- Eqs. 20-22: R f(Lambda) L^dag x + beta V_k f(H_k) e_1
                          on x_minus = x - R L^dag x.
* ``sign_hermitian_deflated`` -- Eq. 12 (orthonormal eigenvectors).
* ``lr_search_space``, ``best_approximation`` -- span(R_m) + K_k(A, x_minus)
                          and the orthogonal projection of the exact result
                          on a space (the comparison of Sec. 5).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .matfunc import sign_eig


def arnoldi(A, x: np.ndarray, k: int, S: np.ndarray | None = None, breakdown_tol=1e-14):
    """k steps of Arnoldi (Eq. 7), CGS2; with ``S`` the modified Arnoldi of Eq. 14.

    Returns dict with V (N x k'), H (k' x k'), beta (|x|), beta_k (H[k'+1,k']),
    v_next, X (m x k', the S-coefficients S^dag A V_k) and k' (= k unless the
    recurrence broke down on an invariant subspace).
    """
    x = np.asarray(x, dtype=np.complex128).ravel()
    N = x.size
    beta = np.linalg.norm(x)
    V = np.zeros((N, k + 1), dtype=np.complex128)
    H = np.zeros((k + 1, k), dtype=np.complex128)
    m = 0 if S is None else S.shape[1]
    X = np.zeros((m, k), dtype=np.complex128)
    V[:, 0] = x / beta
    kk = k
    for j in range(k):
        w = A @ V[:, j]
        nrm_w = np.linalg.norm(w)
        h = np.zeros(j + 1, dtype=np.complex128)
        g = np.zeros(m, dtype=np.complex128)
        for _ in range(2):  # classical Gram-Schmidt, applied twice
            if m:
                dg = S.conj().T @ w
                g += dg
            dh = V[:, : j + 1].conj().T @ w
            h += dh
            if m:
                w = w - S @ dg
            w = w - V[:, : j + 1] @ dh
        H[: j + 1, j] = h
        if m:
            X[:, j] = g
        bk = np.linalg.norm(w)
        H[j + 1, j] = bk
        if bk <= breakdown_tol * nrm_w:
            kk = j + 1
            break
        V[:, j + 1] = w / bk
    return {
        "V": V[:, :kk],
        "H": H[:kk, :kk],
        "beta": beta,
        "beta_k": H[kk, kk - 1].real,
        "v_next": V[:, kk] if kk < k + 1 else None,
        "X": X[:, :kk],
        "k": kk,
    }


def sign_arnoldi(A, x: np.ndarray, k: int, f=sign_eig):
    """Eq. 11: sgn(A) x ~ beta V_k sgn(H_k) e_1 (no deflation)."""
    r = arnoldi(A, x, k)
    F = f(r["H"])
    return r["beta"] * (r["V"] @ F[:, 0])


def sign_schur(A, x: np.ndarray, k: int, S: np.ndarray, T: np.ndarray, f=sign_eig):
    """Schur deflation, Eq. 19 with the Sylvester equation of Eq. 18 for Y."""
    x = np.asarray(x, dtype=np.complex128).ravel()
    xs = S.conj().T @ x
    x_perp = x - S @ xs  # (1 - S S^dag) x
    r = arnoldi(A, x_perp, k, S=S)
    Hk, X, V, beta = r["H"], r["X"], r["V"], r["beta"]
    fT = f(T)
    fH = f(Hk)
    # Eq. 18: T Y - Y H_k = f(T) X - X f(H_k)  <=>  T Y + Y (-H_k) = rhs
    Y = sla.solve_sylvester(T, -Hk, fT @ X - X @ fH)
    e1 = np.zeros(r["k"], dtype=np.complex128)
    e1[0] = beta
    return S @ (fT @ xs) + S @ (Y @ e1) + V @ (fH @ e1)


def sign_schur_block(A, x: np.ndarray, k: int, S: np.ndarray, T: np.ndarray, f=sign_eig):
    """Schur deflation via Eq. 16: Q f(H) Q^dag x with H the block matrix of Eq. 15."""
    x = np.asarray(x, dtype=np.complex128).ravel()
    xs = S.conj().T @ x
    x_perp = x - S @ xs
    r = arnoldi(A, x_perp, k, S=S)
    m, kk = S.shape[1], r["k"]
    H = np.zeros((m + kk, m + kk), dtype=np.complex128)
    H[:m, :m] = T
    H[:m, m:] = r["X"]
    H[m:, m:] = r["H"]
    c = np.concatenate([xs, np.eye(kk, 1, dtype=np.complex128)[:, 0] * r["beta"]])
    Q = np.concatenate([S, r["V"]], axis=1)
    return Q @ (f(H) @ c)


def sign_lr(A, x: np.ndarray, k: int, R: np.ndarray, Lam: np.ndarray, L: np.ndarray, f=sign_eig):
    """LR deflation, Eq. 22: R f(Lambda) L^dag x + beta V_k f(H_k) e_1."""
    x = np.asarray(x, dtype=np.complex128).ravel()
    g = L.conj().T @ x
    x_minus = x - R @ g  # x_ominus = x - R L^dag x (Eq. 21)
    defl = R @ (np.sign(np.asarray(Lam).real) * g)  # f = sgn on the diagonal Lambda
    if k == 0:
        return defl
    r = arnoldi(A, x_minus, k)
    F = f(r["H"])
    return defl + r["beta"] * (r["V"] @ F[:, 0])


def sign_hermitian_deflated(A, x: np.ndarray, k: int, U: np.ndarray, lam: np.ndarray, f=sign_eig):
    """Eq. 12 for Hermitian A: sum_i f(lambda_i)(u_i^dag x) u_i + f(A) x_perp."""
    x = np.asarray(x, dtype=np.complex128).ravel()
    c = U.conj().T @ x
    x_perp = x - U @ c
    r = arnoldi(A, x_perp, k)
    F = f(r["H"])
    return U @ (np.sign(np.asarray(lam).real) * c) + r["beta"] * (r["V"] @ F[:, 0])


def lr_search_space(A, x: np.ndarray, k: int, R: np.ndarray, L: np.ndarray) -> np.ndarray:
    """Basis of the space the LR approximation of Eq. 22 lies in: span(R_m)
    plus the Krylov space K_k(A, x_minus) of x_minus = x - R L^dag x (Eq. 21)."""
    x = np.asarray(x, dtype=np.complex128).ravel()
    x_minus = x - R @ (L.conj().T @ x)
    return np.concatenate([R, arnoldi(A, x_minus, k)["V"]], axis=1)


def best_approximation(Q: np.ndarray, y_exact: np.ndarray) -> np.ndarray:
    """Orthogonal projection of the exact result on span(Q) (Eq. 8 generalised)."""
    Qo, _ = np.linalg.qr(Q)
    return Qo @ (Qo.conj().T @ y_exact)
