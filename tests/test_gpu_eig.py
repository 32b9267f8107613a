"""GPU deflation setup (ovl_deflation_setup) against the oracle's dense
eigendecomposition (Secs. 3-5): the m eigenvalues of smallest |Re lambda|,
the invariant-subspace relations of Eqs. 13 and 20, and the sign function
computed with the GPU's own deflation data against the dense definition."""
import numpy as np
import pytest

from helpers import lattice, need_gpu, rel
from oracle import dirac, eigen, matfunc
from paper_0710_0341_gb300 import ovl, synth

pytestmark = pytest.mark.gpu


def _cols(X, m):
    return X.reshape(m, -1).T  # canonical spinors -> N x m


@pytest.mark.parametrize("dims,m,poly", [((2, 2, 2, 4), 12, -1), ((4, 4, 4, 4), 20, -1), ((4, 4, 4, 4), 20, 0),
                                         ((4, 4, 4, 4), 20, 15)])
def test_setup_schur_and_lr_against_dense(dims, m, poly):
    """poly: -1 the Chebyshev filter with the automatic degree, 0 plain
    restarted Arnoldi on A^2, 15 the filter with a fixed degree."""
    need_gpu()
    mu, m_w = 0.3, -1.0
    U = synth.random_su3_field(dims, 0.5, 0)
    A = dirac.hermitian_wilson(U, mu, m_w)
    Ad = A.toarray()
    lam_o, R_o, L_o = eigen.critical_dense(Ad, m + 1)
    h = lattice(dims, U)
    try:
        N = Ad.shape[0]
        shp = (m,) + synth.lattice_shape(dims) + (4, 3)
        # Schur
        ds = ovl.ovl_deflation_setup_ex(h, mu, m_w, ovl.OVL_DEFL_SCHUR, m, 1e-12, 500, poly)
        S = np.zeros(shp, complex)
        T = np.zeros(m * m, complex)
        ovl.ovl_get_deflation(ds, S, T, None, h)
        S = _cols(S, m)
        T = T.reshape(m, m, order="F")
        assert np.abs(S.conj().T @ S - np.eye(m)).max() < 1e-10
        assert np.abs(np.tril(T, -1)).max() == 0.0
        assert np.linalg.norm(Ad @ S - S @ T) < 1e-9 * np.linalg.norm(Ad, 2)
        # the same eigenvalues as the dense oracle (a gap exists after the m-th)
        assert np.abs(lam_o[m].real) - np.abs(lam_o[m - 1].real) > 1e-6
        ev = np.sort_complex(np.diag(T))
        assert np.allclose(ev, np.sort_complex(lam_o[:m]), atol=1e-10)
        # same invariant subspace as the oracle's right eigenvectors
        Qo, _ = np.linalg.qr(R_o[:, :m])
        assert np.linalg.norm(S - Qo @ (Qo.conj().T @ S)) < 1e-9
        # LR
        dl = ovl.ovl_deflation_setup_ex(h, mu, m_w, ovl.OVL_DEFL_LR, m, 1e-12, 500, poly)
        R = np.zeros(shp, complex)
        L = np.zeros(shp, complex)
        lam = np.zeros(m, complex)
        ovl.ovl_get_deflation(dl, R, lam, L, h)
        R, L = _cols(R, m), _cols(L, m)
        assert np.abs(L.conj().T @ R - np.eye(m)).max() < 1e-9
        assert np.linalg.norm(Ad @ R - R * lam) < 1e-9 * np.linalg.norm(Ad, 2) * np.sqrt(m)
        assert np.linalg.norm(L.conj().T @ Ad - lam[:, None] * L.conj().T) < 1e-8 * np.linalg.norm(L)
        assert np.allclose(np.sort_complex(lam), np.sort_complex(lam_o[:m]), atol=1e-10)
        r, mv = ovl.ovl_deflation_stats(dl)
        assert r >= 1 and mv >= 1
        # the sign function with the GPU's own deflation data
        b = synth.gaussian_source(dims, 1)
        ystar = matfunc.sign_eig_apply(Ad, b.ravel())
        y = np.zeros((2,) + b.shape, complex)
        k = 200 if N > 1000 else N - m  # the small lattice: the whole complement of Omega_m
        ovl.ovl_sign_apply(h, [dict(mu=mu, m_w=m_w, k=k)] * 2, [ds, dl], np.stack([b, b]), y)
        tol = 1e-8
        assert rel(y[0], ystar) < tol, rel(y[0], ystar)
        assert rel(y[1], ystar) < tol, rel(y[1], ystar)
        ovl.ovl_destroy_deflation(ds)
        ovl.ovl_destroy_deflation(dl)
    finally:
        ovl.ovl_destroy_lattice(h)
