"""GPU overlap operator D_ov(mu) = 1 + gamma5 sgn(H_w(mu)) (Sec. 1, Eq. 1) and
its adjoint, through the C ABI, against the oracle.

Parity: the oracle's identical algorithm (same k, same deflation vectors) at
1e-10 (the FP64-mode bar of the sign function). End to end on 2^4 with a
Krylov space near the full dimension: the Ginsparg-Wilson relation
gamma5 D + D gamma5 = D gamma5 D and <a, D b> = <D^dag a, b> (the adjoint from
the swapped LR data of ovl_deflation_adjoint) to 1e-9.
"""
import numpy as np
import pytest

from helpers import canon_cols, lattice, need_gpu, rel
from oracle import dirac, eigen, krylov, overlap
from paper_0710_0341_gb300 import ovl, synth

pytestmark = pytest.mark.gpu

DIMS = (2, 2, 2, 4)


def _data(dims, mu, m_w, m):
    U = synth.random_su3_field(dims, 0.5, 0)
    A = dirac.hermitian_wilson(U, mu, m_w)
    lam, R, L = eigen.critical_dense(A.toarray(), m)
    S, T = eigen.schur_from_right(A, R)
    return U, A, S, T, lam, R, L


def _lr(h, mu, m_w, lam, R, L, dims):
    return ovl.ovl_set_deflation(h, mu, m_w, ovl.OVL_DEFL_LR, R.shape[1], canon_cols(R, dims),
                                 np.ascontiguousarray(lam), canon_cols(L, dims))


def _schur(h, mu, m_w, S, T, dims):
    return ovl.ovl_set_deflation(h, mu, m_w, ovl.OVL_DEFL_SCHUR, S.shape[1], canon_cols(S, dims),
                                 np.asfortranarray(T).ravel(order="F").copy(), None)


def _sh(f):
    return lambda v: f(v.ravel()).reshape(v.shape)


def test_overlap_forward_and_adjoint_match_oracle():
    need_gpu()
    mu, m_w, k = 0.3, -1.0, 40
    U, A, S, T, lam, R, L = _data(DIMS, mu, m_w, 12)
    Am = dirac.hermitian_wilson(U, -mu, m_w)
    x = synth.gaussian_source(DIMS, 3)
    h = lattice(DIMS, U)
    try:
        ds = _schur(h, mu, m_w, S, T, DIMS)
        dl = _lr(h, mu, m_w, lam, R, L, DIMS)
        y = np.zeros((3,) + x.shape, complex)
        infos = ovl.ovl_overlap_apply(h, [dict(mu=mu, m_w=m_w, k=k)] * 3, [None, ds, dl], np.stack([x] * 3), y)
        assert all(i["status"] == 0 for i in infos)
        ref = [overlap.overlap_apply(_sh(lambda v: krylov.sign_arnoldi(A, v, k)), x),
               overlap.overlap_apply(_sh(lambda v: krylov.sign_schur(A, v, k, S, T)), x),
               overlap.overlap_apply(_sh(lambda v: krylov.sign_lr(A, v, k, R, lam, L)), x)]
        for i in range(3):
            assert rel(y[i], ref[i]) < 1e-10, (i, rel(y[i], ref[i]))
        # adjoint: LR data of H_w(-mu) by swapping, and no deflation
        dla = ovl.ovl_deflation_adjoint(dl)
        ya = np.zeros((2,) + x.shape, complex)
        ovl.ovl_overlap_apply(h, [dict(mu=mu, m_w=m_w, k=k)] * 2, [dla, None], np.stack([x] * 2), ya, adjoint=True)
        lam2, R2, L2 = overlap.lr_adjoint(lam, R, L)
        ra = overlap.overlap_adjoint_apply(_sh(lambda v: krylov.sign_lr(Am, v, k, R2, lam2, L2)), x)
        rn = overlap.overlap_adjoint_apply(_sh(lambda v: krylov.sign_arnoldi(Am, v, k)), x)
        assert rel(ya[0], ra) < 1e-10, rel(ya[0], ra)
        assert rel(ya[1], rn) < 1e-10, rel(ya[1], rn)
        with pytest.raises(ovl.OvlError) as e:  # Schur data do not serve the adjoint
            ovl.ovl_deflation_adjoint(ds)
        assert e.value.code == ovl.OVL_ENOTSUP
        with pytest.raises(ovl.OvlError) as e:  # deflation of H_w(mu) used for H_w(-mu)
            ovl.ovl_overlap_apply(h, [dict(mu=mu, m_w=m_w, k=k)], [dl], x, ya[0], adjoint=True)
        assert e.value.code == ovl.OVL_EINVAL
        for d in (ds, dl, dla):
            ovl.ovl_destroy_deflation(d)
    finally:
        ovl.ovl_destroy_lattice(h)


def test_ginsparg_wilson_and_adjoint_end_to_end():
    need_gpu()
    dims, mu, m_w, m = (2, 2, 2, 2), 0.3, -1.0, 12
    U, A, S, T, lam, R, L = _data(dims, mu, m_w, m)
    k = A.shape[0] - m - 2
    a = synth.gaussian_source(dims, 5)
    b = synth.gaussian_source(dims, 6)
    g5 = overlap.gamma5_apply
    h = lattice(dims, U)
    try:
        dl = _lr(h, mu, m_w, lam, R, L, dims)
        dla = ovl.ovl_deflation_adjoint(dl)
        p = dict(mu=mu, m_w=m_w, k=k)

        def D(v):
            out = np.zeros_like(v)
            ovl.ovl_overlap_apply(h, [p], [dl], np.ascontiguousarray(v), out)
            return out

        def Dh(v):
            out = np.zeros_like(v)
            ovl.ovl_overlap_apply(h, [p], [dla], np.ascontiguousarray(v), out, adjoint=True)
            return out

        Db = D(b)
        gw = g5(Db) + D(g5(b)) - D(g5(Db))
        assert np.linalg.norm(gw) <= 1e-9 * np.linalg.norm(b), np.linalg.norm(gw) / np.linalg.norm(b)
        lhs = np.vdot(a.ravel(), Db.ravel())
        rhs = np.vdot(Dh(a).ravel(), b.ravel())
        assert abs(lhs - rhs) <= 1e-9 * np.linalg.norm(a) * np.linalg.norm(b), abs(lhs - rhs)
        ovl.ovl_destroy_deflation(dla)
        ovl.ovl_destroy_deflation(dl)
    finally:
        ovl.ovl_destroy_lattice(h)
