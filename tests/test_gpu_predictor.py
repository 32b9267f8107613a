"""What the trained (k, m) predictor gains over the method without it.

Training data: paper_0710_0341_gb300/predictor_data.json, runs of the method
itself on 4^4 lattices (random eps, mu, m_w): for every deflation size of the
grid the GPU deflation setup and the adaptive depth to 1e-8, with the cost in
basis-vector passes. The network is trained on the GPU (own kernels) on the
first 3/4 of the configurations; on the held-out 1/4 the deflation size it
picks is compared with the method without it (no deflation, adaptive depth)
and with the best single fixed deflation size chosen on the training set."""
import json
import os

import numpy as np
import pytest

from helpers import need_gpu
from paper_0710_0341_gb300 import predictor

pytestmark = pytest.mark.gpu


def _cost(row, m):
    r = next(x for x in row["results"] if x["m"] == m)
    worst = max(x["cost"] for x in row["results"] if np.isfinite(x["cost"]))
    return r["cost"] if r["ok"] else 2.0 * worst  # a choice that never reached 1e-8 is penalised


def test_predictor_beats_the_method_without_it():
    need_gpu()
    if not os.path.exists(predictor.DATA):
        pytest.skip("no predictor training data")
    rows = [r for r in json.load(open(predictor.DATA))["rows"] if r["label"] is not None]
    assert len(rows) >= 16
    n_tr = (3 * len(rows)) // 4
    train, test = rows[:n_tr], rows[n_tr:]
    X, T = predictor.to_xy(train)
    p = predictor.Predictor(seed=0)
    try:
        loss = p.fit(X, T, steps=3000, lr=3e-3)
        assert np.isfinite(loss)
        Xt, Tt = predictor.to_xy(test)
        k_hat, m_hat = p.predict(Xt)
    finally:
        p.close()
    picks = [predictor.nearest_m(m) for m in m_hat]
    c_mlp = np.array([_cost(r, m) for r, m in zip(test, picks)])
    c_none = np.array([_cost(r, 0) for r in test])
    best_fixed = min(predictor.M_GRID, key=lambda m: np.mean([_cost(r, m) for r in train]))
    c_fixed = np.array([_cost(r, best_fixed) for r in test])
    c_oracle = np.array([min(_cost(r, m) for m in predictor.M_GRID) for r in test])
    print(f"held-out mean cost: predictor {c_mlp.mean():.0f}, no deflation {c_none.mean():.0f}, "
          f"best fixed m={best_fixed} {c_fixed.mean():.0f}, per-config optimum {c_oracle.mean():.0f}")
    assert c_mlp.mean() < c_none.mean()
    assert c_mlp.mean() <= 1.05 * c_fixed.mean()
    # the depth estimate sizes the basis: rarely far below the depth needed
    k_true = np.exp(Tt[:, 0])
    assert np.mean(k_hat >= 0.7 * k_true) >= 0.75
