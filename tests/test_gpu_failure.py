"""Failure detection without a GPU fault: a device wait that nothing
completes gives up after its poll limit, reports OVL_ETIMEOUT to the host,
and the context keeps working; host-side failures come back as status codes
(Newton iteration limit, eigensolver restart limit)."""
import numpy as np
import pytest

from helpers import lattice, need_gpu
from oracle import dirac, krylov
from paper_0710_0341_gb300 import ovl, synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    need_gpu()
    dims = (2, 2, 2, 4)
    U = synth.random_su3_field(dims, 0.5, 0)
    h = lattice(dims, U)
    try:
        assert ovl.ovl_wait_selftest(h, 20000) == ovl.OVL_ETIMEOUT
        b = synth.gaussian_source(dims, 1)
        y = np.zeros_like(b)
        ovl.ovl_sign_apply(h, [dict(mu=0.3, m_w=-1.0, k=20)], [None], b, y)
        A = dirac.hermitian_wilson(U, 0.3, -1.0)
        yo = krylov.sign_arnoldi(A, b.ravel(), 20)
        assert np.linalg.norm(y.ravel() - yo) < 1e-10 * np.linalg.norm(yo)
    finally:
        ovl.ovl_destroy_lattice(h)


def test_iteration_limits_return_status():
    need_gpu()
    dims = (2, 2, 2, 4)
    U = synth.random_su3_field(dims, 0.5, 0)
    h = lattice(dims, U)
    try:
        b = synth.gaussian_source(dims, 1)
        y = np.zeros_like(b)
        with pytest.raises(ovl.OvlError) as e:
            ovl.ovl_sign_apply(h, [dict(mu=0.3, m_w=-1.0, k=30, newton_max_iter=1)], [None], b, y)
        assert e.value.code == ovl.OVL_ENOCONV
        assert e.value.infos[0]["status"] == ovl.OVL_ENOCONV
        with pytest.raises(ovl.OvlError) as e:
            ovl.ovl_deflation_setup(h, 0.3, -1.0, ovl.OVL_DEFL_SCHUR, 12, 1e-300, 1)
        assert e.value.code == ovl.OVL_ENOCONV
        with pytest.raises(ovl.OvlError) as e:  # the unfiltered iteration too
            ovl.ovl_deflation_setup_ex(h, 0.3, -1.0, ovl.OVL_DEFL_SCHUR, 12, 1e-300, 1, 0)
        assert e.value.code == ovl.OVL_ENOCONV
        # the handle still works after both failures
        ovl.ovl_sign_apply(h, [dict(mu=0.3, m_w=-1.0, k=10)], [None], b, y)
    finally:
        ovl.ovl_destroy_lattice(h)
