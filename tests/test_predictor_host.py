"""Host logic of the (k, m) predictor on the CPU: labels, the cost model, the
handling of an eigensolver that does not converge for one m, and the choice
of the cost-minimal (k, m), with a stand-in for the library calls."""
import math

import numpy as np
import pytest

from paper_0710_0341_gb300 import predictor


class _OvlError(RuntimeError):
    def __init__(self, infos=None):
        super().__init__("stand-in failure")
        self.infos = infos


class _FakeOvl:
    """Deflation setup fails for m = 16; the adaptive depth falls with m."""
    OVL_DEFL_SCHUR = 1
    OvlError = _OvlError

    def __init__(self, k_of_m, fail_solve=False):
        self.k_of_m = k_of_m
        self.fail_solve = fail_solve
        self.destroyed = []
        self.batches = []

    def ovl_deflation_setup(self, h, mu, m_w, scheme, m, tol, max_restarts):
        if m == 16:
            raise _OvlError()
        return ("defl", m)

    def ovl_deflation_stats(self, d):
        return (3, 1000)  # restarts, A^2 applications

    def ovl_sign_apply(self, h, params, defl, b, y):
        ms = [0 if d is None else d[1] for d in defl]
        self.batches.append(ms)
        infos = [dict(status=0, k_used=self.k_of_m[m], err_est=1e-10) for m in ms]
        if self.fail_solve:
            infos[-1] = dict(status=4, k_used=600, err_est=1e-3)
            raise _OvlError(infos)
        return infos

    def ovl_destroy_deflation(self, d):
        self.destroyed.append(d)


def test_measure_costs_and_skips_a_failed_setup(monkeypatch):
    fake = _FakeOvl({0: 200, 8: 150, 24: 100})
    monkeypatch.setattr(predictor, "ovl", fake)
    res = predictor.measure(None, 0.3, -1.0, np.zeros((2, 3)), sources=12)
    assert fake.batches == [[0, 8, 24]]  # one batch over the m whose setup converged
    by_m = {r["m"]: r for r in res}
    assert [r["m"] for r in res] == [0, 8, 16, 24]
    assert by_m[16]["ok"] is False and by_m[16]["cost"] == float("inf")
    assert by_m[0]["cost"] == 200 * (200 / 2 + 0)
    sp = predictor.setup_passes(1000, 24) / 12
    assert by_m[24]["cost"] == pytest.approx(100 * (100 / 2 + 24) + sp)
    assert sorted(fake.destroyed) == [("defl", 8), ("defl", 24)]


def test_measure_keeps_the_solves_that_finished(monkeypatch):
    fake = _FakeOvl({0: 200, 8: 150, 24: 100}, fail_solve=True)
    monkeypatch.setattr(predictor, "ovl", fake)
    res = {r["m"]: r for r in predictor.measure(None, 0.3, -1.0, np.zeros(1))}
    assert res[0]["ok"] and res[8]["ok"] and not res[24]["ok"]


def test_setup_cost_and_labels():
    # basis of at least nev + 60 and 4 nev vectors, nev = m + max(8, m/2)
    assert predictor.setup_passes(10, 8) == 10 * max(4 * 16, 16 + 60)
    assert predictor.setup_passes(10, 40) == 10 * 4 * 60
    rows = [dict(features=[0.0] * predictor.N_IN, label=[120, 8]),
            dict(features=[1.0] * predictor.N_IN, label=None),
            dict(features=[2.0] * predictor.N_IN, label=[300, 0])]
    X, T = predictor.to_xy(rows)
    assert X.shape == (2, predictor.N_IN) and X.dtype == np.float32
    assert np.allclose(T, [[math.log(120), math.log(9)], [math.log(300), 0.0]])
    assert [predictor.nearest_m(v) for v in (-3, 5, 13, 19.9, 100)] == [0, 8, 16, 16, 24]


def test_random_configs_stay_in_the_training_ranges():
    rng = np.random.default_rng(0)
    for _ in range(200):
        c = predictor.random_config(rng)
        assert 0.2 <= c["eps"] <= 0.6 and 0.0 <= c["mu"] <= 0.6 and -1.5 <= c["m_w"] <= -0.8


def test_plan_depths_start_at_the_prediction_and_cap_the_basis():
    from paper_0710_0341_gb300 import predictor

    assert predictor.plan_depths([183.0, 5.0, 900.0]) == [(180, 229), (20, 20), (700, 700)]


def test_admit_packs_solves_under_the_budget_first_fit_by_size():
    from paper_0710_0341_gb300 import predictor

    ks = [300, 100, 250, 50, 200]
    params = [dict(mu=0.1, m_w=-1.0, k=k) for k in ks]
    # a stand-in for ovl_sign_workspace_bytes: 1 byte per basis column plus 10 per solve
    ws = lambda p, d: sum(x["k"] + 1 + 10 for x in p)  # noqa: E731
    batches = predictor.admit(None, params, [None] * 5, 600, workspace=ws)
    assert sorted(i for b in batches for i in b) == list(range(5))
    assert all(ws([params[i] for i in b], None) <= 600 for b in batches)
    assert batches == [[0, 2], [1, 3, 4]]  # 300 + 250 first, then 200 + 100 + 50
    import pytest

    with pytest.raises(ValueError):
        predictor.admit(None, params, [None] * 5, 200, workspace=ws)


class _FakeOvlLR:
    """LR setup with m_max pairs; subsets imported per m; depth falls with m."""
    OVL_DEFL_LR = 2
    OvlError = _OvlError

    def __init__(self, k_of_m):
        self.k_of_m, self.imported, self.destroyed = k_of_m, [], []

    def ovl_deflation_setup(self, h, mu, m_w, scheme, m, tol, max_restarts):
        assert scheme == 2
        return ("setup", m)

    def ovl_get_deflation(self, d, R, lam, L, h):
        R[:] = np.arange(R.shape[0])[(slice(None),) + (None,) * (R.ndim - 1)]
        lam[:] = np.arange(lam.size) + 0.5
        L[:] = -R
        return 2, d[1]

    def ovl_deflation_stats(self, d):
        return (5, 3000)

    def ovl_set_deflation(self, h, mu, m_w, scheme, m, R, lam, L):
        assert R.shape[0] == m and lam.size == m and L.shape[0] == m
        assert np.array_equal(R[:, 0, 0, 0, 0, 0, 0].real, np.arange(m))  # the m most critical, in order
        self.imported.append(m)
        return ("lr", m)

    def ovl_sign_apply(self, h, params, defl, b, y):
        ms = [0 if d is None else d[1] for d in defl]
        return [dict(status=0, k_used=self.k_of_m[m], err_est=1e-10) for m in ms]

    def ovl_destroy_deflation(self, d):
        self.destroyed.append(d)


def test_measure_lr_uses_one_setup_and_its_leading_pairs(monkeypatch):
    k_of_m = {0: 400, 10: 300, 20: 250, 30: 220, 40: 210, 60: 200}
    fake = _FakeOvlLR(k_of_m)
    monkeypatch.setattr(predictor, "ovl", fake)
    dims = (2, 2, 2, 2)
    res = predictor.measure_lr(None, dims, 0.5, -1.0, np.zeros(synth_shape(dims)))
    assert fake.imported == [10, 20, 30, 40, 60]
    assert ("setup", 60) in fake.destroyed and len(fake.destroyed) == 6
    by_m = {r["m"]: r for r in res}
    sp = predictor.setup_passes(3000, 60) / 12
    assert by_m[0]["cost"] == 400 * 200
    assert by_m[30]["cost"] == pytest.approx(220 * (110 + 30) + sp * 30 / 60)
    assert all(r["ok"] for r in res)


def synth_shape(dims):
    from paper_0710_0341_gb300 import synth

    return synth.lattice_shape(dims) + (4, 3)


class _FakeOvlLattice:
    def __init__(self):
        self.created = []
        self.destroyed = 0

    def ovl_create_lattice(self, dims, *a):
        self.created.append(tuple(dims))
        return len(self.created)

    def ovl_set_links(self, h, U):
        pass

    def ovl_destroy_lattice(self, h):
        self.destroyed += 1


def test_generate_scaled_interleaves_sizes_labels_and_stops_on_time(monkeypatch, tmp_path):
    import json

    fake = _FakeOvlLattice()
    monkeypatch.setattr(predictor, "ovl", fake)
    monkeypatch.setattr(predictor.synth, "random_su3_field", lambda dims, eps, seed: np.zeros(1))
    monkeypatch.setattr(predictor.synth, "gaussian_source", lambda dims, seed: np.zeros(1))
    monkeypatch.setattr(predictor, "features", lambda h, dims, mu, m_w, b: np.full(20, float(dims[0])))
    calls = []

    def measure_lr(h, dims, mu, m_w, b):
        calls.append(dims)
        if len(calls) == 3:  # a run where no m reached the target: no label
            return [dict(m=m, k=700, ok=False, cost=float("inf"), err_est=1e-3) for m in predictor.M_GRID_LR]
        return [dict(m=m, k=300 - m, ok=True, cost=1000.0 + (m - 20) ** 2, err_est=1e-10)
                for m in predictor.M_GRID_LR]

    monkeypatch.setattr(predictor, "measure_lr", measure_lr)
    path = str(tmp_path / "runs.json")
    rows = predictor.generate_scaled(4, 2, seed=3, path=path, log=lambda s: None)
    # 6^4 first, in the proportion 4 : 2 throughout
    assert [d[0] for d in fake.created] == [6, 8, 6, 6, 8, 6]
    assert fake.destroyed == 6 and len(rows) == 6
    assert rows[2]["label"] is None
    assert all(r["label"] == [280, 20] for i, r in enumerate(rows) if i != 2)  # the cost-minimal ok entry
    assert all(0.0 <= r["config"]["mu"] <= 1.0 and list(r["config"]["dims"])[0] == r["features"][0] for r in rows)
    saved = json.load(open(path))
    assert len(saved["rows"]) == 6 and saved["m_grid"] == list(predictor.M_GRID_LR)
    # a time limit keeps the runs done so far (checked before each run): the
    # clock reads start, then per run the check and the log line
    t = iter([0.0, 0.0, 5.0, 10.0, 15.0] + [1e6] * 20)
    monkeypatch.setattr(predictor.time, "time", lambda: next(t))
    fake.created.clear()
    rows = predictor.generate_scaled(4, 2, seed=3, path=None, log=lambda s: None, seconds=100)
    assert len(rows) == 2 and [d[0] for d in fake.created] == [6, 8]
