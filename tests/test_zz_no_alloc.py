"""The allocation-free stencil entry point, for callers that cannot let the
library call cudaMalloc (a process whose HBM is all reserved by its own pool,
or code that must avoid cudaMalloc/cudaFree's implicit synchronisation).

ovl_apply_Hw_noalloc must give what ovl_apply_Hw gives, call after call,
through its fixed staging array. Collected last on purpose: a failure here
leaves every other test already run."""
import numpy as np
import pytest

from helpers import lattice, need_gpu, rel, to_dev
from paper_0710_0341_gb300 import ovl, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("links,tol", [(ovl.OVL_LINKS_F64, 1e-13), (ovl.OVL_LINKS_R12, 2e-6)])
def test_noalloc_matches_apply_hw_twice(links, tol):
    torch = need_gpu()
    dims = (3, 4, 2, 5)
    U = synth.random_su3_field(dims, 0.5, 0)
    h = lattice(dims, U, 1)
    try:
        for call, seed in enumerate((3, 8)):  # two calls in a row through the shared array
            x = np.stack([synth.gaussian_source(dims, seed), synth.gaussian_source(dims, seed + 1)])
            xd = to_dev(torch, x)
            ref = torch.zeros_like(xd)
            out = torch.full_like(xd, float("nan"))
            ovl.ovl_apply_Hw(h, 0.3, -1.1, xd, ref, 2, links)
            ovl.ovl_apply_Hw_noalloc(h, 0.3, -1.1, xd, out, 2, links)
            torch.cuda.synchronize()
            assert rel(out.cpu().numpy(), ref.cpu().numpy()) < tol, (call, links)
    finally:
        ovl.ovl_destroy_lattice(h)


def test_noalloc_rejects_oversize_and_host_buffers():
    torch = need_gpu()
    dims = (16, 16, 16, 16)  # 65536 sites x 192 B: 2 rhs in + out = 50 MB > 32 MiB
    h = lattice(dims, synth.unit_gauge_field(dims))
    try:
        x = torch.zeros((2,) + synth.lattice_shape(dims) + (4, 3), dtype=torch.complex128, device="cuda")
        with pytest.raises(ovl.OvlError) as e:
            ovl.ovl_apply_Hw_noalloc(h, 0.1, -1.0, x, torch.zeros_like(x), 2, ovl.OVL_LINKS_F64)
        assert e.value.code == ovl.OVL_EINVAL
        xs = np.zeros((1,) + synth.lattice_shape((2, 2, 2, 2)) + (4, 3), complex)
        h2 = lattice((2, 2, 2, 2), synth.unit_gauge_field((2, 2, 2, 2)))
        with pytest.raises(ovl.OvlError) as e:
            ovl.ovl_apply_Hw_noalloc(h2, 0.1, -1.0, xs, np.zeros_like(xs), 1, ovl.OVL_LINKS_F64)
        assert e.value.code == ovl.OVL_EINVAL
        ovl.ovl_destroy_lattice(h2)
    finally:
        ovl.ovl_destroy_lattice(h)
