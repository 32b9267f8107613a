"""The 16^3x32 workload at full size through the call the benchmark times:
12 spin-colour point sources at the origin in one batched ovl_sign_apply,
k = 600 (N = 1,572,864; the small sign on n = 600-640 matrices).

* Free field (U = 1): no deflation (Eq. 11), every result within 1e-9 of the
  closed-form sign in momentum space (derived from Eq. 2; pinned in the
  oracle's own tests against dense eigendecompositions).
* The synthetic field (eps 0.3, seed 0) with the GPU's own Schur deflation
  data (m = 40, Eq. 19): sgn(sgn(A) b) = b (Eq. 6) to 1e-10 for every source,
  and the sources the oracle sketch covers within 1e-9 of the oracle's
  converged y* (tests/golden/config3_ystar_sketch.json).
"""
import json
import os

import numpy as np
import pytest

from helpers import lattice, need_gpu, rel
from oracle import freefield
from paper_0710_0341_gb300 import ovl, synth

pytestmark = [pytest.mark.gpu, pytest.mark.late]

DIMS, MU, MW, K, M = (16, 16, 16, 32), 0.2, -1.2, 600, 40
SRCS = [(s, c) for s in range(4) for c in range(3)]
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config3_ystar_sketch.json")


def _sources():
    return np.stack([synth.point_source(DIMS, s, c) for s, c in SRCS])


def test_free_field_12_point_sources_against_closed_form():
    torch = need_gpu()
    b = _sources()
    h = lattice(DIMS, synth.unit_gauge_field(DIMS))
    try:
        bd = torch.from_numpy(b).cuda()
        yd = torch.zeros_like(bd)
        infos = ovl.ovl_sign_apply(h, [dict(mu=MU, m_w=MW, k=K)] * len(SRCS), [None] * len(SRCS), bd, yd)
        y = yd.cpu().numpy()
        for i in range(len(SRCS)):
            assert infos[i]["status"] == 0
            ystar = freefield.sign_hw_free(b[i], MU, MW)
            e = rel(y[i], ystar)
            assert e < 1e-9, (SRCS[i], e, infos[i]["k_used"])
    finally:
        ovl.ovl_destroy_lattice(h)


def test_synthetic_field_schur_m40_involution_and_oracle_sketch():
    torch = need_gpu()
    b = _sources()
    h = lattice(DIMS, synth.random_su3_field(DIMS, 0.3, 0))
    try:
        d = ovl.ovl_deflation_setup(h, MU, MW, ovl.OVL_DEFL_SCHUR, M, 1e-12, 1000)
        params = [dict(mu=MU, m_w=MW, k=K)] * len(SRCS)
        bd = torch.from_numpy(b).cuda()
        yd = torch.zeros_like(bd)
        zd = torch.zeros_like(bd)
        infos = ovl.ovl_sign_apply(h, params, [d] * len(SRCS), bd, yd)
        assert all(i["status"] == 0 and i["k_used"] == K and i["m_used"] == M for i in infos)
        ovl.ovl_sign_apply(h, params, [d] * len(SRCS), yd, zd)
        for i in range(len(SRCS)):
            e = float((zd[i] - bd[i]).norm() / bd[i].norm())
            assert e < 1e-10, (SRCS[i], e)
        if os.path.exists(GOLDEN):
            sk = json.load(open(GOLDEN))
            y = yd.cpu().numpy()
            n = y[0].size
            P = None
            for i, (s, c) in enumerate(SRCS):
                ref = sk.get(f"{s},{c}")
                if ref is None:
                    continue
                if P is None:
                    P = synth.probe_vectors(n, len(ref["probe_re"]))
                est = P.conj() @ y[i].ravel() - (np.array(ref["probe_re"]) + 1j * np.array(ref["probe_im"]))
                e = np.linalg.norm(est) / np.sqrt(2 * len(est)) / ref["norm"]
                samp = y[i].ravel()[ref["sample_index"]] - (np.array(ref["sample_re"]) + 1j * np.array(ref["sample_im"]))
                print(f"16^3x32 source {s},{c}: sketch error {e:.2e}, max sample error {np.abs(samp).max():.2e}")
                assert e < 1e-9, ((s, c), e)
                assert np.abs(samp).max() < 1e-9 * ref["norm"]
        ovl.ovl_destroy_deflation(d)
    finally:
        ovl.ovl_destroy_lattice(h)
