"""Pass B of the Arnoldi step (Eq. 7; the reorthogonalised column and the next
candidate) has two load paths, chosen by ovl_set_pass_b: plain register loads,
and bulk copies into a ring of shared-memory stages per warp. The arithmetic
is the same, so every result must be equal bit for bit:

* in the 48-bit and the 40-bit basis forms;
* with Schur vectors (columns addressed through the pointer table, Eq. 14),
  LR deflation (Eq. 22) and none, at uneven depths in one batch;
* on a lattice whose row count leaves a partial row block (N = 1440 =
  11 x 128 + 32) and on one where each CTA streams several row blocks
  (12^4, N = 248,832), so that the stage ring runs across blocks;
* in the deflation setup (restarted Arnoldi on the same kernels, Sec. 5).

The results themselves are held to the oracle by the other sign tests; one
case here is checked against it too."""
import numpy as np
import pytest

from helpers import lattice, need_gpu, rel
from oracle import krylov
from oracle import dirac
from paper_0710_0341_gb300 import ovl, synth

pytestmark = pytest.mark.gpu


def _both_paths(h, params, defl, b):
    out = []
    for bulk in (0, 1):
        ovl.ovl_set_pass_b(h, bulk)
        y = np.zeros_like(b)
        infos = ovl.ovl_sign_apply(h, params, defl, b, y)
        out.append((y, infos))
    ovl.ovl_set_pass_b(h, 0)
    return out


@pytest.mark.parametrize("prec", [ovl.OVL_PREC_FP64, ovl.OVL_PREC_DF40])
def test_partial_row_block_schur_lr_none_bit_identical(prec):
    need_gpu()
    dims = (3, 4, 2, 5)  # V = 120, N = 1440: the last row block holds 32 rows
    U = synth.random_su3_field(dims, 0.5, 0)
    h = lattice(dims, U, 1)
    try:
        mu, mw = 0.3, -1.0
        ds = ovl.ovl_deflation_setup(h, mu, mw, ovl.OVL_DEFL_SCHUR, 8, 1e-12, 500)
        dl = ovl.ovl_deflation_setup(h, mu, mw, ovl.OVL_DEFL_LR, 8, 1e-12, 500)
        b = np.stack([synth.gaussian_source(dims, s) for s in (1, 2, 3)])
        params = [dict(mu=mu, m_w=mw, k=k, prec=prec) for k in (40, 50, 30)]
        (y0, i0), (y1, i1) = _both_paths(h, params, [ds, dl, None], b)
        assert [i["k_used"] for i in i1] == [40, 50, 30] and all(i["status"] == 0 for i in i1)
        assert np.array_equal(y0, y1)
        if prec == ovl.OVL_PREC_FP64:  # the undeflated solve against the oracle (Eq. 11)
            A = dirac.hermitian_wilson(U, mu, mw, antiperiodic_t=True)
            ref = krylov.sign_arnoldi(A, b[2].ravel(), 30)
            assert rel(y1[2], ref) < 1e-10
        for d in (ds, dl):
            ovl.ovl_destroy_deflation(d)
    finally:
        ovl.ovl_destroy_lattice(h)


@pytest.mark.parametrize("prec", [ovl.OVL_PREC_FP64, ovl.OVL_PREC_DF40])
def test_several_row_blocks_per_cta_bit_identical(prec):
    torch = need_gpu()
    dims = (12, 12, 12, 12)  # N = 248,832: 1944 row blocks, several per CTA
    U = synth.random_su3_field(dims, 0.4, 0)
    h = lattice(dims, U)
    try:
        N, m = 12 * 12 ** 4, 10
        rng = np.random.default_rng(3)
        Q, _ = np.linalg.qr(rng.standard_normal((N, m)) + 1j * rng.standard_normal((N, m)))
        cols = np.ascontiguousarray(Q.T.reshape((m,) + synth.lattice_shape(dims) + (4, 3)))
        T = np.diag(np.linspace(0.1, 0.2, m).astype(complex))
        d = ovl.ovl_set_deflation(h, 0.2, -1.0, ovl.OVL_DEFL_SCHUR, m, cols, T.ravel(order="F").copy(), None)
        b = torch.from_numpy(np.stack([synth.gaussian_source(dims, 1)] * 2)).cuda()
        params = [dict(mu=0.2, m_w=-1.0, k=k, prec=prec) for k in (36, 28)]
        ys = []
        for bulk in (0, 1):
            ovl.ovl_set_pass_b(h, bulk)
            y = torch.zeros_like(b)
            infos = ovl.ovl_sign_apply(h, params, [d, None], b, y)
            assert all(i["status"] == 0 for i in infos)
            ys.append(y.cpu().numpy())
        assert np.array_equal(ys[0], ys[1])
        ovl.ovl_destroy_deflation(d)
    finally:
        ovl.ovl_destroy_lattice(h)


def test_deflation_setup_bit_identical_and_bad_argument():
    need_gpu()
    dims = (4, 4, 4, 4)
    h = lattice(dims, synth.random_su3_field(dims, 0.5, 0))
    try:
        res = []
        for bulk in (0, 1):
            ovl.ovl_set_pass_b(h, bulk)
            d = ovl.ovl_deflation_setup(h, 0.3, -1.0, ovl.OVL_DEFL_SCHUR, 12, 1e-12, 500)
            shp = (12,) + synth.lattice_shape(dims) + (4, 3)
            S, L, T = np.zeros(shp, complex), np.zeros(shp, complex), np.zeros(144, complex)
            ovl.ovl_get_deflation(d, S, T, L, h)
            res.append((S, T, ovl.ovl_deflation_stats(d)))
            ovl.ovl_destroy_deflation(d)
        assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
        assert res[0][2] == res[1][2]
        with pytest.raises(ovl.OvlError) as e:
            ovl.ovl_set_pass_b(h, 2)
        assert e.value.code == ovl.OVL_EINVAL
    finally:
        ovl.ovl_destroy_lattice(h)
