"""GPU parity of H_w(mu) = gamma_5 D_w(mu) (Sec. 1, Eq. 2) against the oracle.

Called through the C ABI (ctypes binding). FP64 links: relative error <= 1e-13
(the same sums in another order). FP32 and 12-real links: <= 2e-6 (FP32
arithmetic: |U| = 1, 49 terms per row, u32 = 6e-8).
"""
import numpy as np
import pytest

from helpers import canon_cols, lattice, need_gpu, rel, to_dev
from oracle import dirac
from paper_0710_0341_gb300 import ovl, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,apbc", [((4, 4, 4, 4), 0), ((3, 4, 2, 5), 1), ((2, 2, 2, 2), 0), ((5, 3, 7, 6), 0)])
@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_apply_hw_fp64_and_fp32(dims, apbc, mu):
    torch = need_gpu()
    U = synth.random_su3_field(dims, 0.5, 0)
    h = lattice(dims, U, apbc)
    try:
        A = dirac.hermitian_wilson(U, mu, -1.1, antiperiodic_t=bool(apbc))
        x = np.stack([synth.gaussian_source(dims, 3), synth.gaussian_source(dims, 4)])
        ref = np.stack([dirac.apply(A, x[0]), dirac.apply(A, x[1])])
        for links, tol in ((ovl.OVL_LINKS_F64, 1e-13), (ovl.OVL_LINKS_F32, 2e-6), (ovl.OVL_LINKS_R12, 2e-6)):
            out = np.zeros_like(x)
            ovl.ovl_apply_Hw(h, mu, -1.1, x, out, 2, links)  # host pointers
            assert rel(out, ref) < tol, (links, rel(out, ref))
            xd = to_dev(torch, x)
            od = torch.zeros_like(xd)
            ovl.ovl_apply_Hw(h, mu, -1.1, xd, od, 2, links)  # device pointers
            assert rel(od.cpu().numpy(), ref) < tol
    finally:
        ovl.ovl_destroy_lattice(h)


@pytest.mark.parametrize("nrhs", [1, 10])
def test_apply_hw_fp64_8x4_multi_rhs(nrhs):
    """8^4, FP64 spinors and links, one and ten right-hand sides (the bench's
    lattice; up to 40960 site applications per launch): equal to the oracle's
    Eq. 2 to 1e-13."""
    need_gpu()
    dims = (8, 8, 8, 8)
    U = synth.random_su3_field(dims, 0.4, 0)
    h = lattice(dims, U)
    try:
        A = dirac.hermitian_wilson(U, 0.3, -1.0)
        x = np.stack([synth.gaussian_source(dims, 10 + i) for i in range(nrhs)])
        ref = np.stack([dirac.apply(A, xi) for xi in x])
        out = np.zeros_like(x)
        ovl.ovl_apply_Hw(h, 0.3, -1.0, x, out, nrhs, ovl.OVL_LINKS_F64)
        assert rel(out, ref) < 1e-13, rel(out, ref)
    finally:
        ovl.ovl_destroy_lattice(h)


def test_packed_roundtrip_and_packed_stencil():
    torch = need_gpu()
    dims = (4, 6, 2, 4)
    U = synth.random_su3_field(dims, 0.4, 1)
    h = lattice(dims, U)
    try:
        x = np.stack([synth.gaussian_source(dims, 5), synth.gaussian_source(dims, 6), synth.gaussian_source(dims, 7)])
        xd = to_dev(torch, x)
        N = x[0].size
        p64 = torch.zeros(3 * N, dtype=torch.complex128, device="cuda")
        ovl.ovl_pack_spinor(h, xd, p64, 3, ovl.OVL_VEC_F64)
        back = torch.zeros_like(xd)
        ovl.ovl_unpack_spinor(h, p64, back, 3, ovl.OVL_VEC_F64)
        assert torch.equal(back, xd)  # bit-exact permutation
        out = torch.zeros_like(p64)
        mus = [0.0, 0.25, 0.6]
        ovl.ovl_apply_Hw_packed(h, mus, -1.0, p64, out, 3, ovl.OVL_VEC_F64, ovl.OVL_LINKS_F64)
        ovl.ovl_unpack_spinor(h, out, back, 3, ovl.OVL_VEC_F64)
        for r in range(3):
            ref = dirac.apply(dirac.hermitian_wilson(U, mus[r], -1.0), x[r])
            assert rel(back[r].cpu().numpy(), ref) < 1e-13
        p32 = torch.zeros(3 * N, dtype=torch.complex64, device="cuda")
        ovl.ovl_pack_spinor(h, xd, p32, 3, ovl.OVL_VEC_F32)
        o32 = torch.zeros_like(p32)
        ovl.ovl_apply_Hw_packed(h, mus, -1.0, p32, o32, 3, ovl.OVL_VEC_F32, ovl.OVL_LINKS_R12)
        ovl.ovl_unpack_spinor(h, o32, back, 3, ovl.OVL_VEC_F32)
        for r in range(3):
            ref = dirac.apply(dirac.hermitian_wilson(U, mus[r], -1.0), x[r])
            assert rel(back[r].cpu().numpy(), ref) < 3e-6
    finally:
        ovl.ovl_destroy_lattice(h)


def test_invalid_arguments_are_rejected():
    need_gpu()
    with pytest.raises(ovl.OvlError) as e:
        ovl.ovl_create_lattice((1, 4, 4, 4))
    assert e.value.code == ovl.OVL_EINVAL
    dims = (2, 2, 2, 2)
    h = ovl.ovl_create_lattice(dims)
    try:
        x = synth.gaussian_source(dims, 1)
        with pytest.raises(ovl.OvlError) as e:  # links not set
            ovl.ovl_apply_Hw(h, 0.1, -1.0, x, np.zeros_like(x), 1, ovl.OVL_LINKS_F64)
        assert e.value.code == ovl.OVL_EINVAL
        ovl.ovl_set_links(h, synth.unit_gauge_field(dims))
        with pytest.raises(ovl.OvlError):
            ovl.ovl_apply_Hw(h, 0.1, -1.0, x, np.zeros_like(x), 1, 7)
    finally:
        ovl.ovl_destroy_lattice(h)


@pytest.mark.slow
@pytest.mark.parametrize("dims,eps,m_w", [((16, 16, 16, 32), 0.3, -1.2), ((24, 24, 24, 48), 0.3, -1.0)])
def test_apply_hw_full_size_sampled(dims, eps, m_w):
    """Full lattice sizes of the 16^3x32 and 24^3x48 workloads, one right-hand
    side (the stencil launch the bench times): H_w x at 48 sampled sites
    (corners, faces, random) against the oracle's row evaluation of Eq. 2;
    FP64 links 1e-13, FP32 and 12-real links 2e-6 of the largest entry."""
    need_gpu()
    U = synth.random_su3_field(dims, eps, 0)
    x = synth.gaussian_source(dims, 1)
    V = int(np.prod(dims))
    rng = np.random.default_rng(0)
    sites = sorted({0, V - 1, dims[0] - 1, V - dims[0], V // 2, dims[0] * dims[1] * dims[2]}
                   | {int(v) for v in rng.integers(0, V, 42)})
    ref = dirac.hermitian_wilson_rows(U, 0.2, m_w, x, sites)
    h = lattice(dims, U)
    try:
        for links, tol in ((ovl.OVL_LINKS_F64, 1e-13), (ovl.OVL_LINKS_F32, 2e-6), (ovl.OVL_LINKS_R12, 2e-6)):
            out = np.zeros_like(x)
            ovl.ovl_apply_Hw(h, 0.2, m_w, x, out, 1, links)
            got = out.reshape(-1, 4, 3)[sites]
            err = np.abs(got - ref).max() / np.abs(ref).max()
            assert err < tol, (links, err)
    finally:
        ovl.ovl_destroy_lattice(h)


@pytest.mark.late
@pytest.mark.parametrize("dims,apbc", [((4, 4, 4, 4), 0), ((3, 4, 2, 5), 1)])
def test_apply_hw_double_float_arithmetic(dims, apbc):
    """OVL_LINKS_F64DF: the FP64 data through the double-float instantiation of
    the stencil (hi + lo FP32 arithmetic) agrees with the oracle to 1e-13 and
    with the FP64 kernel to 5e-14, for several right-hand sides with their own
    mu, and is not the FP64 kernel under another name."""
    need_gpu()
    U = synth.random_su3_field(dims, 0.5, 3)
    mus = [0.0, 0.3, 0.7]
    x = np.stack([synth.gaussian_source(dims, 20 + i) for i in range(3)])
    h = lattice(dims, U, apbc)
    try:
        outs = {}
        for links in (ovl.OVL_LINKS_F64, ovl.OVL_LINKS_F64DF):
            o = np.zeros_like(x)
            for r in range(3):  # canonical entry point, one mu per call
                ovl.ovl_apply_Hw(h, mus[r], -1.0, x[r], o[r], 1, links)
            outs[links] = o
        for r in range(3):
            ref = dirac.apply(dirac.hermitian_wilson(U, mus[r], -1.0, antiperiodic_t=bool(apbc)), x[r])
            e_df = rel(outs[ovl.OVL_LINKS_F64DF][r], ref)
            d = rel(outs[ovl.OVL_LINKS_F64DF][r], outs[ovl.OVL_LINKS_F64][r])
            assert e_df < 1e-13, (r, e_df)
            assert 1e-17 < d < 5e-14, (r, d)
    finally:
        ovl.ovl_destroy_lattice(h)
