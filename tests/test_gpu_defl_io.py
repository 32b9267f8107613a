"""Deflation data kept across processes: ovl_deflation_save / _load round trip
(the one-off eigenvector computation of Sec. 5, amortised over later runs),
and the checks that refuse a file for another operator or a damaged file."""
import os

import numpy as np
import pytest

from helpers import lattice, need_gpu, rel
from paper_0710_0341_gb300 import ovl, synth

pytestmark = pytest.mark.gpu

DIMS, MU, MW = (4, 4, 4, 4), 0.3, -1.0


@pytest.mark.parametrize("scheme", [ovl.OVL_DEFL_SCHUR, ovl.OVL_DEFL_LR])
def test_save_load_round_trip_and_refusals(tmp_path, scheme):
    need_gpu()
    U = synth.random_su3_field(DIMS, 0.5, 0)
    b = synth.gaussian_source(DIMS, 1)
    h = lattice(DIMS, U)
    try:
        d = ovl.ovl_deflation_setup(h, MU, MW, scheme, 12, 1e-12, 500)
        path = str(tmp_path / "defl.bin")
        ovl.ovl_deflation_save(d, path)
        d2 = ovl.ovl_deflation_load(h, path)
        assert ovl.ovl_deflation_stats(d2) == ovl.ovl_deflation_stats(d)
        shp = (12,) + b.shape
        S1, S2 = np.zeros(shp, complex), np.zeros(shp, complex)
        L1, L2 = np.zeros(shp, complex), np.zeros(shp, complex)
        nT = 144 if scheme == ovl.OVL_DEFL_SCHUR else 12
        T1, T2 = np.zeros(nT, complex), np.zeros(nT, complex)
        ovl.ovl_get_deflation(d, S1, T1, L1, h)
        ovl.ovl_get_deflation(d2, S2, T2, L2, h)
        assert np.array_equal(S1, S2) and np.array_equal(T1, T2) and np.array_equal(L1, L2)
        # the loaded data give the same solve, bit for bit
        y1, y2 = np.zeros_like(b), np.zeros_like(b)
        ovl.ovl_sign_apply(h, [dict(mu=MU, m_w=MW, k=60)], [d], b, y1)
        ovl.ovl_sign_apply(h, [dict(mu=MU, m_w=MW, k=60)], [d2], b, y2)
        assert rel(y2, y1) == 0.0
        # the recorded mu is enforced as for imported data
        with pytest.raises(ovl.OvlError):
            ovl.ovl_sign_apply(h, [dict(mu=0.2, m_w=MW, k=10)], [d2], b, y2)
        # other links: refused
        h2 = lattice(DIMS, synth.random_su3_field(DIMS, 0.5, 1))
        try:
            with pytest.raises(ovl.OvlError) as e:
                ovl.ovl_deflation_load(h2, path)
            assert e.value.code == ovl.OVL_EINVAL
        finally:
            ovl.ovl_destroy_lattice(h2)
        # other dims: refused
        h3 = lattice((4, 4, 4, 2), synth.random_su3_field((4, 4, 4, 2), 0.5, 0))
        try:
            with pytest.raises(ovl.OvlError):
                ovl.ovl_deflation_load(h3, path)
        finally:
            ovl.ovl_destroy_lattice(h3)
        # damaged or truncated files: refused
        raw = open(path, "rb").read()
        bad = bytearray(raw)
        bad[len(raw) // 2] ^= 1
        open(path, "wb").write(bytes(bad))
        with pytest.raises(ovl.OvlError):
            ovl.ovl_deflation_load(h, path)
        open(path, "wb").write(raw[:-100])
        with pytest.raises(ovl.OvlError):
            ovl.ovl_deflation_load(h, path)
        with pytest.raises(ovl.OvlError):
            ovl.ovl_deflation_load(h, os.path.join(str(tmp_path), "missing.bin"))
        for x in (d, d2):
            ovl.ovl_destroy_deflation(x)
    finally:
        ovl.ovl_destroy_lattice(h)
