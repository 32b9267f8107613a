"""GPU parity of the deflated Arnoldi sign function (Secs. 2-4) against the oracle.

The CUDA path and the oracle see the same seeded inputs and, for deflation,
the same eigenvectors (computed by the oracle's dense eigensolver).
Tolerances: FP64 mode vs the oracle's identical algorithm (same k, same
deflation vectors): 1e-10 relative (the target the method's FP64 mode is
held to). Mixed modes: 1e-5 (FP32 basis: u32 = 6e-8 per entry, amplified by
the sign function's conditioning on these small lattices).
"""
import numpy as np
import pytest

from helpers import canon_cols, lattice, need_gpu, rel, to_dev
from oracle import dirac, eigen, freefield, krylov, matfunc
from paper_0710_0341_gb300 import ovl, synth

pytestmark = pytest.mark.gpu

DIMS = (2, 2, 2, 4)


def _setup(dims, eps, mu, m_w, seed=0):
    U = synth.random_su3_field(dims, eps, seed)
    A = dirac.hermitian_wilson(U, mu, m_w)
    return U, A


def _schur(A, dims, m):
    lam, R, L = eigen.critical_dense(A.toarray(), m)
    S, T = eigen.schur_from_right(A, R)
    return S, T, lam, R, L


def _defl_schur(h, mu, m_w, S, T, dims):
    return ovl.ovl_set_deflation(h, mu, m_w, ovl.OVL_DEFL_SCHUR, S.shape[1], canon_cols(S, dims),
                                 np.asfortranarray(T).ravel(order="F").copy(), None)


def _defl_lr(h, mu, m_w, lam, R, L, dims):
    return ovl.ovl_set_deflation(h, mu, m_w, ovl.OVL_DEFL_LR, R.shape[1], canon_cols(R, dims),
                                 np.ascontiguousarray(lam), canon_cols(L, dims))


@pytest.mark.parametrize("dims", [DIMS, (3, 4, 2, 5)])
def test_no_deflation_fp64(dims):
    need_gpu()
    U, A = _setup(dims, 0.5, 0.3, -1.0)
    b = synth.gaussian_source(dims, 1)
    h = lattice(dims, U)
    try:
        for k in (1, 7, 40):
            y = np.zeros_like(b)
            info = ovl.ovl_sign_apply(h, [dict(mu=0.3, m_w=-1.0, k=k)], [None], b, y)
            yo = krylov.sign_arnoldi(A, b.ravel(), k)
            assert info[0]["k_used"] == k
            assert rel(y, yo) < 1e-10, (k, rel(y, yo))
    finally:
        ovl.ovl_destroy_lattice(h)


def test_schur_and_lr_fp64():
    torch = need_gpu()
    mu, m_w = 0.3, -1.0
    U, A = _setup(DIMS, 0.5, mu, m_w)
    S, T, lam, R, L = _schur(A, DIMS, 12)
    b = synth.gaussian_source(DIMS, 1)
    h = lattice(DIMS, U)
    try:
        ds = _defl_schur(h, mu, m_w, S, T, DIMS)
        dl = _defl_lr(h, mu, m_w, lam, R, L, DIMS)
        k = 30
        bb = np.stack([b, b])
        y = np.zeros_like(bb)
        infos = ovl.ovl_sign_apply(h, [dict(mu=mu, m_w=m_w, k=k)] * 2, [ds, dl], bb, y)
        ys = krylov.sign_schur(A, b.ravel(), k, S, T)
        yl = krylov.sign_lr(A, b.ravel(), k, R, lam, L)
        assert rel(y[0], ys) < 1e-10, rel(y[0], ys)
        assert rel(y[1], yl) < 1e-10, rel(y[1], yl)
        assert infos[0]["m_used"] == 12 and infos[1]["m_used"] == 12
        # device-resident input and output give the same numbers
        bd = to_dev(torch, bb)
        yd = torch.zeros_like(bd)
        ovl.ovl_sign_apply(h, [dict(mu=mu, m_w=m_w, k=k)] * 2, [ds, dl], bd, yd)
        assert rel(yd.cpu().numpy(), y) < 1e-14
        # deflation data round trip
        S2 = np.zeros((12,) + b.shape, dtype=np.complex128)
        T2 = np.zeros(144, dtype=np.complex128)
        sch, m = ovl.ovl_get_deflation(ds, S2, T2, None, h)
        assert sch == ovl.OVL_DEFL_SCHUR and m == 12
        assert rel(S2, canon_cols(S, DIMS)) < 1e-14
        assert np.array_equal(T2.reshape(12, 12, order="F"), T)
        ovl.ovl_destroy_deflation(ds)
        ovl.ovl_destroy_deflation(dl)
    finally:
        ovl.ovl_destroy_lattice(h)


def test_uneven_batch_mixed_schemes():
    need_gpu()
    m_w = -1.0
    U = synth.random_su3_field(DIMS, 0.5, 0)
    h = lattice(DIMS, U)
    try:
        A3 = dirac.hermitian_wilson(U, 0.3, m_w)
        A1 = dirac.hermitian_wilson(U, 0.1, m_w)
        A0 = dirac.hermitian_wilson(U, 0.0, m_w)
        S, T, lam, R, L = _schur(A3, DIMS, 10)
        _, _, lam1, R1, L1 = _schur(A1, DIMS, 8)
        ds = _defl_schur(h, 0.3, m_w, S, T, DIMS)
        dl = _defl_lr(h, 0.1, m_w, lam1, R1, L1, DIMS)
        bs = [synth.gaussian_source(DIMS, s) for s in (1, 2, 3, 4)]
        params = [dict(mu=0.3, m_w=m_w, k=20), dict(mu=0.3, m_w=m_w, k=33), dict(mu=0.1, m_w=m_w, k=25),
                  dict(mu=0.0, m_w=m_w, k=41)]
        y = np.zeros((4,) + bs[0].shape, dtype=np.complex128)
        infos = ovl.ovl_sign_apply(h, params, [None, ds, dl, None], np.stack(bs), y)
        refs = [krylov.sign_arnoldi(A3, bs[0].ravel(), 20), krylov.sign_schur(A3, bs[1].ravel(), 33, S, T),
                krylov.sign_lr(A1, bs[2].ravel(), 25, R1, lam1, L1), krylov.sign_arnoldi(A0, bs[3].ravel(), 41)]
        for i in range(4):
            assert infos[i]["k_used"] == params[i]["k"]
            assert rel(y[i], refs[i]) < 1e-10, (i, rel(y[i], refs[i]))
    finally:
        ovl.ovl_destroy_lattice(h)


@pytest.mark.parametrize("prec", [ovl.OVL_PREC_MIXED, ovl.OVL_PREC_MIXED_R12])
def test_mixed_precision_several_row_blocks(prec):
    """4^4 (N = 3072: the projection kernels run several 1024-row blocks over
    Krylov columns that have no low plane): the mixed modes agree with the FP64
    mode to their FP32 bound."""
    need_gpu()
    dims, mu, m_w = (4, 4, 4, 4), 0.3, -1.0
    U = synth.random_su3_field(dims, 0.5, 0)
    b = synth.gaussian_source(dims, 1)
    h = lattice(dims, U)
    try:
        y64 = np.zeros_like(b)
        ym = np.zeros_like(b)
        ovl.ovl_sign_apply(h, [dict(mu=mu, m_w=m_w, k=120)], [None], b, y64)
        ovl.ovl_sign_apply(h, [dict(mu=mu, m_w=m_w, k=120, prec=prec)], [None], b, ym)
        assert rel(ym, y64) < 1e-5, rel(ym, y64)
    finally:
        ovl.ovl_destroy_lattice(h)


@pytest.mark.parametrize("prec,tol", [(ovl.OVL_PREC_MIXED, 1e-5), (ovl.OVL_PREC_MIXED_R12, 1e-5)])
def test_mixed_precision_bound(prec, tol):
    need_gpu()
    mu, m_w = 0.3, -1.0
    U, A = _setup(DIMS, 0.5, mu, m_w)
    S, T, lam, R, L = _schur(A, DIMS, 12)
    b = synth.gaussian_source(DIMS, 1)
    h = lattice(DIMS, U)
    try:
        ds = _defl_schur(h, mu, m_w, S, T, DIMS)
        dl = _defl_lr(h, mu, m_w, lam, R, L, DIMS)
        bb = np.stack([b, b, b])
        y = np.zeros_like(bb)
        ovl.ovl_sign_apply(h, [dict(mu=mu, m_w=m_w, k=30, prec=prec)] * 3, [ds, dl, None], bb, y)
        refs = [krylov.sign_schur(A, b.ravel(), 30, S, T), krylov.sign_lr(A, b.ravel(), 30, R, lam, L),
                krylov.sign_arnoldi(A, b.ravel(), 30)]
        for i in range(3):
            assert rel(y[i], refs[i]) < tol, (i, rel(y[i], refs[i]))
    finally:
        ovl.ovl_destroy_lattice(h)


def test_full_krylov_space_is_exact():
    need_gpu()
    dims = (2, 2, 2, 2)
    U, A = _setup(dims, 0.5, 0.3, -1.0)
    b = synth.gaussian_source(dims, 1)
    ystar = matfunc.sign_eig_apply(A.toarray(), b.ravel())
    h = lattice(dims, U)
    try:
        y = np.zeros_like(b)
        info = ovl.ovl_sign_apply(h, [dict(mu=0.3, m_w=-1.0, k=192)], [None], b, y)
        assert info[0]["k_used"] <= 192
        assert rel(y, ystar) < 1e-8, rel(y, ystar)
    finally:
        ovl.ovl_destroy_lattice(h)


def test_free_field_8x4_closed_form():
    """Full config size (8^4, N = 49152): U = 1 has a closed-form sign."""
    need_gpu()
    dims = (8, 8, 8, 8)
    U = synth.unit_gauge_field(dims)
    b = synth.gaussian_source(dims, 1)
    ystar = freefield.sign_hw_free(b, 0.3, -1.0)
    h = lattice(dims, U)
    try:
        y = np.zeros_like(b)
        ovl.ovl_sign_apply(h, [dict(mu=0.3, m_w=-1.0, k=200)], [None], b, y)
        assert rel(y, ystar) < 1e-10, rel(y, ystar)
    finally:
        ovl.ovl_destroy_lattice(h)


@pytest.mark.slow
def test_config_4x4_schur_k200_m20():
    """4^4, eps 0.5, m_w -1, mu 0.3, Gaussian source, k 200, Schur m 20, FP64:
    parity with the oracle's algorithm and accuracy against dense eig."""
    need_gpu()
    dims = (4, 4, 4, 4)
    U, A = _setup(dims, 0.5, 0.3, -1.0)
    Ad = A.toarray()
    b = synth.gaussian_source(dims, 1)
    ystar = matfunc.sign_eig_apply(Ad, b.ravel())
    lam, R, L = eigen.critical_dense(Ad, 20)
    S, T = eigen.schur_from_right(A, R)
    yo = krylov.sign_schur(A, b.ravel(), 200, S, T)
    h = lattice(dims, U)
    try:
        ds = _defl_schur(h, 0.3, -1.0, S, T, dims)
        y = np.zeros_like(b)
        ovl.ovl_sign_apply(h, [dict(mu=0.3, m_w=-1.0, k=200)], [ds], b, y)
        assert rel(y, yo) < 1e-10, rel(y, yo)
        assert rel(y, ystar) < 1e-8, rel(y, ystar)
    finally:
        ovl.ovl_destroy_lattice(h)


def test_sign_argument_errors():
    need_gpu()
    U, A = _setup(DIMS, 0.5, 0.3, -1.0)
    S, T, lam, R, L = _schur(A, DIMS, 4)
    b = synth.gaussian_source(DIMS, 1)
    h = lattice(DIMS, U)
    try:
        ds = _defl_schur(h, 0.3, -1.0, S, T, DIMS)
        y = np.zeros_like(b)
        with pytest.raises(ovl.OvlError) as e:  # deflation built for another mu
            ovl.ovl_sign_apply(h, [dict(mu=0.2, m_w=-1.0, k=10)], [ds], b, y)
        assert e.value.code == ovl.OVL_EINVAL
        with pytest.raises(ovl.OvlError) as e:  # beyond the basis limit
            ovl.ovl_sign_apply(h, [dict(mu=0.3, m_w=-1.0, k=5000)], [None], b, y)
        assert e.value.code == ovl.OVL_EINVAL
        with pytest.raises(ovl.OvlError) as e:  # one precision per batch
            ovl.ovl_sign_apply(h, [dict(mu=0.3, m_w=-1.0, k=5), dict(mu=0.3, m_w=-1.0, k=5, prec=1)],
                               [None, None], np.stack([b, b]), np.zeros((2,) + b.shape, complex))
        assert e.value.code == ovl.OVL_EINVAL
        for bad in (dict(k=0), dict(m_w=-4.0), dict(newton_fp64=7), dict(prec=9)):
            with pytest.raises(ovl.OvlError) as e:  # depth < 1, kappa infinite, unknown modes
                ovl.ovl_sign_apply(h, [dict(dict(mu=0.3, m_w=-1.0, k=5), **bad)], [None], b, y)
            assert e.value.code == ovl.OVL_EINVAL, bad
    finally:
        ovl.ovl_destroy_lattice(h)


def test_newton_double_float_matches_fp64_newton():
    """The double-float Gauss-Jordan Newton (default) and the FP64 one give the
    same sign of the projected matrix to well inside the 1e-10 parity bar."""
    need_gpu()
    mu, m_w = 0.3, -1.0
    U, A = _setup(DIMS, 0.5, mu, m_w)
    S, T, lam, R, L = _schur(A, DIMS, 12)
    b = synth.gaussian_source(DIMS, 1)
    h = lattice(DIMS, U)
    try:
        ds = _defl_schur(h, mu, m_w, S, T, DIMS)
        dl = _defl_lr(h, mu, m_w, lam, R, L, DIMS)
        bb = np.stack([b, b, b])
        y_df = np.zeros_like(bb)
        y_64 = np.zeros_like(bb)
        p = dict(mu=mu, m_w=m_w, k=60)
        i1 = ovl.ovl_sign_apply(h, [p] * 3, [ds, dl, None], bb, y_df)
        i2 = ovl.ovl_sign_apply(h, [dict(p, newton_fp64=1)] * 3, [ds, dl, None], bb, y_64)
        y_co = np.zeros_like(bb)
        i3 = ovl.ovl_sign_apply(h, [dict(p, newton_fp64=2)] * 3, [ds, dl, None], bb, y_co)
        for i in range(3):
            assert rel(y_df[i], y_64[i]) < 1e-11, (i, rel(y_df[i], y_64[i]))
            assert rel(y_co[i], y_64[i]) < 1e-11, (i, rel(y_co[i], y_64[i]))
            assert i1[i]["newton_iters"] > 0 and i2[i]["newton_iters"] > 0 and i3[i]["newton_iters"] > 0
    finally:
        ovl.ovl_destroy_lattice(h)


@pytest.mark.parametrize("ks", [(300, 460), (520,)])
def test_newton_kernels_large_projected_matrix(ks):
    """Projected matrices of order 300-520 (4^4, no deflation): at n <= 460 the
    rows fit a 16-CTA cluster's shared memory (cluster kernel), at n = 520 they
    do not (cooperative kernel). Every variant of the small sign (default with
    the Newton-Schulz finish, FP64, cooperative double-float, cluster without
    Newton-Schulz, Newton-Schulz declined and resumed by Gauss-Jordan) matches
    the oracle's Eq. 11 result and the FP64 Newton."""
    need_gpu()
    dims, mu, m_w = (4, 4, 4, 4), 0.3, -1.0
    U, A = _setup(dims, 0.5, mu, m_w)
    b = synth.gaussian_source(dims, 1)
    h = lattice(dims, U)
    try:
        bb = np.stack([b] * len(ks))
        ys = {}
        for mode in (0, 1, 2, 3, 4):
            ys[mode] = np.zeros_like(bb)
            infos = ovl.ovl_sign_apply(h, [dict(mu=mu, m_w=m_w, k=k, newton_fp64=mode) for k in ks],
                                       [None] * len(ks), bb, ys[mode])
            assert all(i["status"] == 0 and i["newton_iters"] > 0 for i in infos)
        for i, k in enumerate(ks):
            yo = krylov.sign_arnoldi(A, b.ravel(), k)
            for mode in (0, 1, 2, 3, 4):
                assert rel(ys[mode][i], yo) < 1e-10, (k, mode, rel(ys[mode][i], yo))
                assert rel(ys[mode][i], ys[1][i]) < 1e-11, (k, mode, rel(ys[mode][i], ys[1][i]))
    finally:
        ovl.ovl_destroy_lattice(h)


def test_source_in_invariant_subspace():
    """b a combination of three eigenvectors of H_w: the Krylov space is
    3-dimensional (Sec. 2), so any k >= 3 gives sgn(A) b exactly (Eqs. 4-6)."""
    need_gpu()
    mu, m_w = 0.3, -1.0
    U, A = _setup(DIMS, 0.5, mu, m_w)
    lam, Vr = np.linalg.eig(A.toarray())
    idx = [i for i in np.argsort(-np.abs(lam.real)) if abs(lam[i].real) > 0.05][:3]
    coef = np.array([1.0, 2.0, 0.5])
    b = (Vr[:, idx] @ coef).reshape(synth.lattice_shape(DIMS) + (4, 3))
    ystar = (Vr[:, idx] @ (coef * np.sign(lam[idx].real))).reshape(b.shape)
    h = lattice(DIMS, U)
    try:
        for k in (3, 12):
            y = np.zeros_like(b)
            info = ovl.ovl_sign_apply(h, [dict(mu=mu, m_w=m_w, k=k)], [None], b, y)
            assert info[0]["status"] == 0
            assert rel(y, ystar) < 1e-10, (k, rel(y, ystar))
    finally:
        ovl.ovl_destroy_lattice(h)


def test_source_in_deflated_subspace():
    """b inside span(S) (Schur) or span(R) (LR): the projected remainder x is at
    the rounding level, y comes from the deflated part alone (Eqs. 16, 22) and
    equals sgn(A) b."""
    need_gpu()
    mu, m_w = 0.3, -1.0
    U, A = _setup(DIMS, 0.5, mu, m_w)
    S, T, lam, R, L = _schur(A, DIMS, 12)
    Ad = A.toarray()
    rng = np.random.default_rng(5)
    c = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    shape = synth.lattice_shape(DIMS) + (4, 3)
    bs = (S @ c).reshape(shape)
    bl = (R @ c).reshape(shape)
    ys = matfunc.sign_eig_apply(Ad, bs.ravel()).reshape(shape)
    yl = (R @ (np.sign(lam.real) * c)).reshape(shape)
    h = lattice(DIMS, U)
    try:
        ds = _defl_schur(h, mu, m_w, S, T, DIMS)
        dl = _defl_lr(h, mu, m_w, lam, R, L, DIMS)
        y = np.zeros((2,) + shape, complex)
        infos = ovl.ovl_sign_apply(h, [dict(mu=mu, m_w=m_w, k=10)] * 2, [ds, dl], np.stack([bs, bl]), y)
        assert all(i["status"] == 0 for i in infos)
        assert infos[0]["beta"] < 1e-10 * np.linalg.norm(bs) and infos[1]["beta"] < 1e-10 * np.linalg.norm(bl)
        assert rel(y[0], ys) < 1e-10, rel(y[0], ys)
        assert rel(y[1], yl) < 1e-10, rel(y[1], yl)
    finally:
        ovl.ovl_destroy_lattice(h)


@pytest.mark.slow
def test_uneven_batch_full_size_12x4():
    """The 12^4 lattice of the 48-solve workload (N = 248832), uneven depths
    and chemical potentials in one batch: each solve equals the same solve run
    alone (the per-solve arithmetic and its reduction order do not depend on the
    batch). At mu = 0 H_w is Hermitian, so <b, y> = beta^2 e_1^dag sgn(H_k) e_1 is
    real for the approximation itself, and |y| is near |b| (sgn(H_w) is unitary)."""
    need_gpu()
    dims, m_w = (12, 12, 12, 12), -1.0
    U = synth.random_su3_field(dims, 0.4, 0)
    b = synth.gaussian_source(dims, 1)
    h = lattice(dims, U)
    try:
        params = [dict(mu=0.05, m_w=m_w, k=150), dict(mu=0.2, m_w=m_w, k=220), dict(mu=0.8, m_w=m_w, k=300),
                  dict(mu=0.0, m_w=m_w, k=300)]
        yb = np.zeros((4,) + b.shape, complex)
        infos = ovl.ovl_sign_apply(h, params, [None] * 4, np.stack([b] * 4), yb)
        assert [i["k_used"] for i in infos] == [150, 220, 300, 300]
        for i, p in enumerate(params[:3]):
            y1 = np.zeros_like(b)
            ovl.ovl_sign_apply(h, [p], [None], b, y1)
            assert rel(yb[i], y1) <= 1e-14, (i, rel(yb[i], y1))
        ip = np.vdot(b.ravel(), yb[3].ravel())
        assert abs(ip.imag) <= 1e-10 * np.linalg.norm(b) ** 2, ip  # measured 1.8e-16 |b|^2 (oracle 3.8e-18)
        assert 0.5 < np.linalg.norm(yb[3]) / np.linalg.norm(b) < 1.5
    finally:
        ovl.ovl_destroy_lattice(h)


@pytest.mark.late
@pytest.mark.parametrize("dims", [DIMS, (3, 4, 2, 5)])
def test_fp64_mode_with_double_float_stencil(dims):
    """OVL_PREC_FP64_DFSTENCIL (the FP64 mode with the stencil's arithmetic in
    double-float on the FP32 pipes) against the oracle's same algorithm at the
    FP64 mode's 1e-10 bar, for Schur, LR and no deflation in one batch, and
    within 1e-12 of the FP64 mode itself."""
    need_gpu()
    mu, m_w = 0.3, -1.0
    U, A = _setup(dims, 0.5, mu, m_w)
    S, T, lam, R, L = _schur(A, dims, 12)
    b = synth.gaussian_source(dims, 1)
    h = lattice(dims, U)
    try:
        ds = _defl_schur(h, mu, m_w, S, T, dims)
        dl = _defl_lr(h, mu, m_w, lam, R, L, dims)
        k = 60
        bb = np.stack([b, b, b])
        ys = {}
        for prec in (ovl.OVL_PREC_FP64, ovl.OVL_PREC_FP64_DFSTENCIL):
            y = np.zeros_like(bb)
            infos = ovl.ovl_sign_apply(h, [dict(mu=mu, m_w=m_w, k=k, prec=prec)] * 3, [ds, dl, None], bb, y)
            assert all(i["status"] == 0 for i in infos)
            ys[prec] = y
        refs = [krylov.sign_schur(A, b.ravel(), k, S, T), krylov.sign_lr(A, b.ravel(), k, R, lam, L),
                krylov.sign_arnoldi(A, b.ravel(), k)]
        for i in range(3):
            assert rel(ys[ovl.OVL_PREC_FP64_DFSTENCIL][i], refs[i]) < 1e-10, (i, rel(ys[3][i], refs[i]))
            assert rel(ys[ovl.OVL_PREC_FP64_DFSTENCIL][i], ys[ovl.OVL_PREC_FP64][i]) < 1e-12
        for d in (ds, dl):
            ovl.ovl_destroy_deflation(d)
    finally:
        ovl.ovl_destroy_lattice(h)


@pytest.mark.late
@pytest.mark.parametrize("dims", [DIMS, (3, 4, 2, 5)])
def test_plain_fp64_form_against_oracle(dims):
    """OVL_PREC_FP64_PLAIN (complex128 basis, FP64 products and sums in every
    pass, FP64 Gauss-Jordan Newton) against the oracle's same algorithm at
    1e-10 for Schur, LR and no deflation in one batch, k = 1 and 60, and within
    1e-11 of the 48-bit FP64 mode."""
    need_gpu()
    mu, m_w = 0.3, -1.0
    U, A = _setup(dims, 0.5, mu, m_w)
    S, T, lam, R, L = _schur(A, dims, 12)
    b = synth.gaussian_source(dims, 1)
    h = lattice(dims, U)
    try:
        ds = _defl_schur(h, mu, m_w, S, T, dims)
        dl = _defl_lr(h, mu, m_w, lam, R, L, dims)
        bb = np.stack([b, b, b])
        for k in (1, 60):
            ys = {}
            for prec in (ovl.OVL_PREC_FP64, ovl.OVL_PREC_FP64_PLAIN):
                y = np.zeros_like(bb)
                infos = ovl.ovl_sign_apply(h, [dict(mu=mu, m_w=m_w, k=k, prec=prec)] * 3, [ds, dl, None], bb, y)
                assert all(i["status"] == 0 and i["k_used"] == k for i in infos)
                ys[prec] = y
            refs = [krylov.sign_schur(A, b.ravel(), k, S, T), krylov.sign_lr(A, b.ravel(), k, R, lam, L),
                    krylov.sign_arnoldi(A, b.ravel(), k)]
            for i in range(3):
                yp = ys[ovl.OVL_PREC_FP64_PLAIN][i]
                assert rel(yp, refs[i]) < 1e-10, (k, i, rel(yp, refs[i]))
                assert rel(yp, ys[ovl.OVL_PREC_FP64][i]) < 1e-11, (k, i)
        for d in (ds, dl):
            ovl.ovl_destroy_deflation(d)
    finally:
        ovl.ovl_destroy_lattice(h)


@pytest.mark.late
@pytest.mark.parametrize("dims", [DIMS, (3, 4, 2, 5)])
def test_df40_form_against_oracle(dims):
    """OVL_PREC_DF40 (Krylov columns stored as FP32 hi + BF16 lo, about 32
    significant bits) against the oracle's same algorithm for Schur, LR and
    no deflation in one batch: the stored basis carries a relative error of
    at most 2^-33 per entry, which the tests hold to 1e-8 of the result."""
    need_gpu()
    mu, m_w = 0.3, -1.0
    U, A = _setup(dims, 0.5, mu, m_w)
    S, T, lam, R, L = _schur(A, dims, 12)
    b = synth.gaussian_source(dims, 1)
    h = lattice(dims, U)
    try:
        ds = _defl_schur(h, mu, m_w, S, T, dims)
        dl = _defl_lr(h, mu, m_w, lam, R, L, dims)
        bb = np.stack([b, b, b])
        k = 60
        y = np.zeros_like(bb)
        infos = ovl.ovl_sign_apply(h, [dict(mu=mu, m_w=m_w, k=k, prec=ovl.OVL_PREC_DF40)] * 3, [ds, dl, None], bb, y)
        assert all(i["status"] == 0 and i["k_used"] == k for i in infos)
        refs = [krylov.sign_schur(A, b.ravel(), k, S, T), krylov.sign_lr(A, b.ravel(), k, R, lam, L),
                krylov.sign_arnoldi(A, b.ravel(), k)]
        for i in range(3):
            e = rel(y[i], refs[i])
            print(f"df40 {dims} solve {i}: rel err vs oracle {e:.2e}")
            assert e < 1e-8, (i, e)
        for d in (ds, dl):
            ovl.ovl_destroy_deflation(d)
    finally:
        ovl.ovl_destroy_lattice(h)


@pytest.mark.late
@pytest.mark.parametrize("dims,m,k", [(DIMS, 12, 30), ((4, 4, 4, 4), 20, 120)])
def test_schur_sylvester_route_against_oracle(dims, m, k):
    """schur_route = 1: sgn(T) and sgn(H_k) on the two diagonal blocks, the
    coupling block from the Sylvester equation (Eq. 18), the result by Eq. 19
    -- the route the oracle's sign_schur takes (scipy's solve_sylvester) --
    within 1e-10 of the oracle, in a batch with an LR and an undeflated solve
    (which take their usual route) and equal to the block route (Eq. 16) to
    1e-11, in the 48-bit mode and in the plain FP64 form."""
    need_gpu()
    mu, m_w = 0.3, -1.0
    U, A = _setup(dims, 0.5, mu, m_w)
    S, T, lam, R, L = _schur(A, dims, m)
    b = synth.gaussian_source(dims, 1)
    h = lattice(dims, U)
    try:
        ds = _defl_schur(h, mu, m_w, S, T, dims)
        dl = _defl_lr(h, mu, m_w, lam, R, L, dims)
        bb = np.stack([b, b, b, b])
        defl = [ds, dl, None, ds]
        refs = [krylov.sign_schur(A, b.ravel(), k, S, T), krylov.sign_lr(A, b.ravel(), k, R, lam, L),
                krylov.sign_arnoldi(A, b.ravel(), k)]
        for prec in (ovl.OVL_PREC_FP64, ovl.OVL_PREC_FP64_PLAIN):
            y0 = np.zeros_like(bb)
            y1 = np.zeros_like(bb)
            ovl.ovl_sign_apply(h, [dict(mu=mu, m_w=m_w, k=k, prec=prec)] * 4, defl, bb, y0)
            infos = ovl.ovl_sign_apply(h, [dict(mu=mu, m_w=m_w, k=k, prec=prec, schur_route=1)] * 4, defl, bb, y1)
            assert all(i["status"] == 0 and i["k_used"] == k for i in infos)
            for i, ref in enumerate(refs + [refs[0]]):
                e = rel(y1[i], ref)
                print(f"sylvester route {dims} prec={prec} solve {i}: rel err vs oracle {e:.2e}, "
                      f"vs block route {rel(y1[i], y0[i]):.2e}")
                assert e < 1e-10, (prec, i, e)
                assert rel(y1[i], y0[i]) < 1e-11, (prec, i)
        for d in (ds, dl):
            ovl.ovl_destroy_deflation(d)
    finally:
        ovl.ovl_destroy_lattice(h)


@pytest.mark.late
def test_graph_replay_gives_the_eager_results():
    """ovl_set_graphs(1): the second call of a batch shape captures the
    Arnoldi loop into a CUDA graph, later calls replay it; every result equals
    the eager one bit for bit, a new shape runs eagerly again, and switching
    graphs off returns to eager launches."""
    need_gpu()
    mu, m_w = 0.3, -1.0
    U, A = _setup(DIMS, 0.5, mu, m_w)
    S, T, lam, R, L = _schur(A, DIMS, 12)
    b = synth.gaussian_source(DIMS, 1)
    h = lattice(DIMS, U)
    try:
        ds = _defl_schur(h, mu, m_w, S, T, DIMS)
        params = [dict(mu=mu, m_w=m_w, k=40), dict(mu=mu, m_w=m_w, k=25), dict(mu=0.1, m_w=m_w, k=33)]
        bb = np.stack([b, b, b])
        y0 = np.zeros_like(bb)
        ovl.ovl_sign_apply(h, params, [ds, None, None], bb, y0)
        assert ovl.ovl_set_graphs(h, 1) == 0
        for call in range(4):
            y = np.zeros_like(bb)
            ovl.ovl_sign_apply(h, params, [ds, None, None], bb, y)
            assert np.array_equal(y, y0), call
        assert ovl.ovl_set_graphs(h, -1) >= 2  # calls 3 and 4 replayed the graph
        other = [dict(p, k=p["k"] + 1) for p in params]
        ovl.ovl_sign_apply(h, other, [ds, None, None], bb, y)
        ref = [krylov.sign_schur(A, b.ravel(), 41, S, T), krylov.sign_arnoldi(A, b.ravel(), 26)]
        assert rel(y[0], ref[0]) < 1e-10 and rel(y[1], ref[1]) < 1e-10
        ovl.ovl_set_graphs(h, 0)
        y = np.zeros_like(bb)
        ovl.ovl_sign_apply(h, params, [ds, None, None], bb, y)
        assert np.array_equal(y, y0)
        ovl.ovl_destroy_deflation(ds)
    finally:
        ovl.ovl_destroy_lattice(h)
