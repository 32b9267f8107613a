"""The stencil autotuner (not in the paper): every timed candidate is a valid
launch shape for the lattice, the kept shape is the fastest candidate, and
the stencil's results are bit for bit the same with the tuned shape (the
shape only assigns sites to threads, and the cp.async-staged FP32 kernel runs
the same site arithmetic in the same order). Each candidate is also checked
on its own against the built-in shape."""
import numpy as np
import pytest

from helpers import lattice, need_gpu
from paper_0710_0341_gb300 import ovl, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,nrhs", [((8, 8, 8, 8), 2), ((12, 8, 4, 6), 1)])
def test_autotune_keeps_the_fastest_valid_shape_and_the_same_results(dims, nrhs):
    torch = need_gpu()
    U = synth.random_su3_field(dims, 0.4, 0)
    h = lattice(dims, U)
    try:
        x = torch.from_numpy(np.stack([synth.gaussian_source(dims, s) for s in range(1, nrhs + 1)])).cuda()
        before = {}
        for links in (ovl.OVL_LINKS_F64, ovl.OVL_LINKS_F32, ovl.OVL_LINKS_R12, ovl.OVL_LINKS_F64DF):
            y = torch.zeros_like(x)
            ovl.ovl_apply_Hw(h, 0.3, -1.0, x, y, nrhs, links)
            before[links] = y.cpu().numpy()
        rep = ovl.ovl_autotune(h, nrhs)
        assert rep, "no candidate timed"
        for r in rep:
            assert r["us"] > 0
            if r["tx"]:
                assert r["tpb"] == r["tx"] * r["ty"] * r["tz"] in (32, 128)
                assert dims[0] % r["tx"] == 0 and dims[1] % r["ty"] == 0 and dims[2] % r["tz"] == 0
        for fmt, links in ((ovl.OVL_VEC_F32, ovl.OVL_LINKS_R12), (ovl.OVL_VEC_F32, ovl.OVL_LINKS_F32),
                           (ovl.OVL_VEC_F64, ovl.OVL_LINKS_F64)):
            mine = [r for r in rep if r["fmt"] == fmt and r["links"] == links]
            fastest = min(mine, key=lambda r: r["us"])
            assert ovl.ovl_autotune_shape(h, fmt, links) == (fastest["tpb"], fastest["tx"], fastest["ty"],
                                                             fastest["tz"], fastest["variant"])
            if fmt == ovl.OVL_VEC_F32:  # the cp.async-staged kernel is among the FP32 candidates
                assert any(r["variant"] % 10 for r in mine) and any(r["variant"] // 10 for r in mine)
        assert ovl.ovl_autotune_shape(h, ovl.OVL_VEC_F64, ovl.OVL_LINKS_F64DF) == \
            ovl.ovl_autotune_shape(h, ovl.OVL_VEC_F64, ovl.OVL_LINKS_F64)
        for links, y0 in before.items():
            y = torch.zeros_like(x)
            ovl.ovl_apply_Hw(h, 0.3, -1.0, x, y, nrhs, links)
            assert np.array_equal(y.cpu().numpy(), y0), links
    finally:
        ovl.ovl_destroy_lattice(h)


def test_every_candidate_shape_gives_the_built_in_results():
    """Each candidate the autotuner times, set on its own with
    ovl_autotune_set_shape, gives the built-in shape's results bit for bit
    (FP32 with 18-real and 12-real links, including the cp.async-staged
    kernel, and FP64); shapes that do not fit are refused."""
    torch = need_gpu()
    dims, nrhs = (8, 8, 4, 6), 3
    h = lattice(dims, synth.random_su3_field(dims, 0.4, 0), 1)
    try:
        x = torch.from_numpy(np.stack([synth.gaussian_source(dims, s) for s in range(nrhs)])).cuda()
        ref = {}
        for links in (ovl.OVL_LINKS_F32, ovl.OVL_LINKS_R12, ovl.OVL_LINKS_F64):
            y = torch.zeros_like(x)
            ovl.ovl_apply_Hw(h, 0.3, -1.0, x, y, nrhs, links)
            ref[links] = y.cpu().numpy()
        rep = ovl.ovl_autotune(h, nrhs)
        assert any(r["variant"] for r in rep) and any(r["tx"] for r in rep)
        for r in rep:
            shape = (r["tpb"], r["tx"], r["ty"], r["tz"], r["variant"])
            ovl.ovl_autotune_set_shape(h, r["fmt"], r["links"], shape)
            y = torch.zeros_like(x)
            ovl.ovl_apply_Hw(h, 0.3, -1.0, x, y, nrhs, r["links"])
            assert np.array_equal(y.cpu().numpy(), ref[r["links"]]), shape
        for bad in ((128, 16, 4, 2, 0), (128, 0, 0, 0, 1), (64, 0, 0, 0, 0)):
            with pytest.raises(ovl.OvlError):
                ovl.ovl_autotune_set_shape(h, ovl.OVL_VEC_F64 if bad[4] else ovl.OVL_VEC_F32, ovl.OVL_LINKS_F64
                                           if bad[4] else ovl.OVL_LINKS_R12, bad)
    finally:
        ovl.ovl_destroy_lattice(h)
