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

# late(9): after every other test, the late-marked ones included
pytestmark = [pytest.mark.gpu, pytest.mark.late(9)]


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
    small = (2, 2, 2, 2)
    h = lattice(dims, synth.unit_gauge_field(dims))
    h2 = lattice(small, synth.unit_gauge_field(small))
    try:
        x = torch.zeros((2,) + synth.lattice_shape(dims) + (4, 3), dtype=torch.complex128, device="cuda")
        with pytest.raises(ovl.OvlError) as e:
            ovl.ovl_apply_Hw_noalloc(h, 0.1, -1.0, x, torch.zeros_like(x), 2, ovl.OVL_LINKS_F64)
        assert e.value.code == ovl.OVL_EINVAL
        xs = np.zeros((1,) + synth.lattice_shape(small) + (4, 3), complex)
        with pytest.raises(ovl.OvlError) as e:
            ovl.ovl_apply_Hw_noalloc(h2, 0.1, -1.0, xs, np.zeros_like(xs), 1, ovl.OVL_LINKS_F64)
        assert e.value.code == ovl.OVL_EINVAL
    finally:
        ovl.ovl_destroy_lattice(h2)
        ovl.ovl_destroy_lattice(h)


def test_noalloc_calls_leave_free_device_memory_unchanged():
    """On a fresh handle that never ran ovl_apply_Hw (which grows the handle's
    own staging buffer): after one warm-up call, further calls change the
    device's free memory by nothing."""
    torch = need_gpu()
    dims = (4, 4, 4, 6)
    h = lattice(dims, synth.random_su3_field(dims, 0.5, 0))
    try:
        x = to_dev(torch, np.stack([synth.gaussian_source(dims, 5)] * 3))
        out = torch.zeros_like(x)
        torch.cuda.synchronize()
        ovl.ovl_apply_Hw_noalloc(h, 0.2, -1.0, x, out, 3, ovl.OVL_LINKS_F64)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for links in (ovl.OVL_LINKS_F64, ovl.OVL_LINKS_R12, ovl.OVL_LINKS_F64):
            ovl.ovl_apply_Hw_noalloc(h, 0.2, -1.0, x, out, 3, links)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    finally:
        ovl.ovl_destroy_lattice(h)


def test_noalloc_refused_while_the_lattice_stream_is_captured():
    """Each call copies a host table that is freed on return and synchronises
    the stream, which a graph cannot hold: under capture the call is refused
    with OVL_EINVAL before it issues any work, and the capture stays valid."""
    torch = need_gpu()
    dims = (2, 2, 2, 4)
    s = torch.cuda.Stream()
    h = ovl.ovl_create_lattice(dims, 0, s)
    try:
        ovl.ovl_set_links(h, np.ascontiguousarray(synth.unit_gauge_field(dims)))
        x = to_dev(torch, synth.gaussian_source(dims, 2)[None])
        out = torch.zeros_like(x)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
            with pytest.raises(ovl.OvlError) as e:
                ovl.ovl_apply_Hw_noalloc(h, 0.1, -1.0, x, out, 1, ovl.OVL_LINKS_F64)
            out.add_(1.0)  # the capture still records work after the refusal
        assert e.value.code == ovl.OVL_EINVAL
        g.replay()
        torch.cuda.synchronize()
        assert float(out.real.min()) == 1.0
    finally:
        ovl.ovl_destroy_lattice(h)
