"""The stencil autotuner (not in the paper): every timed candidate is a valid
launch shape for the lattice, the kept shape is the fastest candidate, and
the stencil's results are bit for bit the same with the tuned shape (the
shape only assigns sites to threads)."""
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
                                                             fastest["tz"])
        assert ovl.ovl_autotune_shape(h, ovl.OVL_VEC_F64, ovl.OVL_LINKS_F64DF) == \
            ovl.ovl_autotune_shape(h, ovl.OVL_VEC_F64, ovl.OVL_LINKS_F64)
        for links, y0 in before.items():
            y = torch.zeros_like(x)
            ovl.ovl_apply_Hw(h, 0.3, -1.0, x, y, nrhs, links)
            assert np.array_equal(y.cpu().numpy(), y0), links
    finally:
        ovl.ovl_destroy_lattice(h)
