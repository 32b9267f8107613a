"""Learned (k, m) predictor: features, training data from the method's own runs,
GPU training and prediction (not in the paper).

The network (libovl's MLP: 20 -> 64 -> 64 -> 2, FP32, own forward/backward/Adam
kernels) maps solve features to (log k, log(m + 1)):

  features = [mu, m_w, link spread, log2 V, the 16 smallest |Re theta| of the
              64 Ritz values from a 64-step Arnoldi run on the source]

Labels are the cost-minimal (k, m) over a grid of deflation sizes: for each m
the GPU computes the deflation data (ovl_deflation_setup, Schur) and runs the
adaptive depth to the target accuracy; the cost in basis-vector passes is
  k (k/2 + m) + setup_passes(m) / sources
with setup_passes = (A^2 applications) x (basis size), shared by `sources`
solves of the same operator. This module only sequences library calls and
moves arrays; every computation runs in libovl.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

from paper_0710_0341_gb300 import ovl, synth

N_IN, N_HIDDEN, N_OUT = 20, 64, 2
M_GRID = (0, 8, 16, 24)
NRITZ, NFEAT_RITZ = 64, 16
UNDER_WEIGHT = 4.0
HERE = os.path.dirname(os.path.abspath(__file__))
DATA = os.path.join(HERE, "predictor_data.json")
DATA_SCALED = os.path.join(HERE, "predictor_data_6x4_8x4.json")  # generate_scaled: 6^4 and 8^4, LR, M_GRID_LR


def features(h, dims, mu, m_w, b):
    V = int(np.prod(dims))
    spread = ovl.ovl_link_spread(h)
    th = np.zeros(NRITZ, dtype=np.complex128)
    ovl.ovl_ritz_values(h, mu, m_w, NRITZ, np.ascontiguousarray(b), th)
    re = np.sort(np.abs(th.real))[:NFEAT_RITZ]
    return np.concatenate([[mu, m_w, spread, math.log2(V)], re]).astype(np.float32)


def setup_passes(matvecs, m):
    nev = m + max(8, m // 2)
    return matvecs * max(4 * nev, nev + 60)


def measure(h, mu, m_w, b, tol=1e-8, k0=20, every=10, k_max=600, sources=12):
    """For each m of M_GRID: the adaptive depth that reaches tol and its cost."""
    grid, defl, setup, failed = [0], [None], [0.0], []
    for m in M_GRID[1:]:
        try:
            d = ovl.ovl_deflation_setup(h, mu, m_w, ovl.OVL_DEFL_SCHUR, m, 1e-12, 800)
        except ovl.OvlError:  # eigensolver did not converge: this m is not an option
            failed.append(m)
            continue
        grid.append(m)
        defl.append(d)
        setup.append(setup_passes(ovl.ovl_deflation_stats(d)[1], m) / sources)
    n = len(grid)
    bb = np.stack([b] * n)
    y = np.zeros_like(bb)
    ps = [dict(mu=mu, m_w=m_w, k=k0, adapt_every=every, k_max=k_max, tol=tol)] * n
    try:
        infos = ovl.ovl_sign_apply(h, ps, defl, bb, y)
    except ovl.OvlError as e:  # keep the solves that finished
        infos = e.infos
    out = []
    for m, inf, sc in zip(grid, infos, setup):
        k = inf["k_used"]
        ok = inf["status"] == 0 and inf["err_est"] <= tol / 10 and k < k_max
        out.append(dict(m=m, k=k, ok=bool(ok), cost=k * (k / 2 + m) + sc, err_est=inf["err_est"]))
    for m in failed:
        out.append(dict(m=m, k=k_max, ok=False, cost=float("inf"), err_est=None))
    out.sort(key=lambda r: r["m"])
    for d in defl[1:]:
        ovl.ovl_destroy_deflation(d)
    return out


def random_config(rng):
    return dict(eps=float(rng.uniform(0.2, 0.6)), mu=float(rng.uniform(0.0, 0.6)),
                m_w=float(rng.uniform(-1.5, -0.8)), seed=int(rng.integers(1 << 30)))


# Training data at scale: 6^4 and 8^4 lattices, mu in [0, 1], the m grid below.
M_GRID_LR = (0, 10, 20, 30, 40, 60)


def measure_lr(h, dims, mu, m_w, b, tol=1e-8, k0=20, every=10, k_max=700, sources=12, grid=M_GRID_LR):
    """For each m of grid: the adaptive depth that reaches tol with LR
    deflation by the m most critical pairs, all from one setup with the
    largest m; cost in basis-vector passes k (k/2 + m) plus the setup's
    passes per source, scaled by m / m_max."""
    mmax = max(grid)
    shp = (mmax,) + synth.lattice_shape(dims) + (4, 3)
    defl = [None]
    try:
        d = ovl.ovl_deflation_setup(h, mu, m_w, ovl.OVL_DEFL_LR, mmax, 1e-12, 1000)
    except ovl.OvlError:
        d = None
    setup_each = {0: 0.0}
    if d is not None:
        R = np.zeros(shp, np.complex128)
        L = np.zeros(shp, np.complex128)
        lam = np.zeros(mmax, np.complex128)
        ovl.ovl_get_deflation(d, R, lam, L, h)
        mv = ovl.ovl_deflation_stats(d)[1]
        ovl.ovl_destroy_deflation(d)
        for m in grid[1:]:
            defl.append(ovl.ovl_set_deflation(h, mu, m_w, ovl.OVL_DEFL_LR, m, np.ascontiguousarray(R[:m]),
                                              np.ascontiguousarray(lam[:m]), np.ascontiguousarray(L[:m])))
            setup_each[m] = setup_passes(mv, mmax) * (m / mmax) / sources
    ms = [0] + ([m for m in grid[1:]] if d is not None else [])
    bb = np.stack([b] * len(ms))
    y = np.zeros_like(bb)
    ps = [dict(mu=mu, m_w=m_w, k=k0, adapt_every=every, k_max=k_max, tol=tol)] * len(ms)
    try:
        infos = ovl.ovl_sign_apply(h, ps, defl, bb, y)
    except ovl.OvlError as e:
        infos = e.infos
    out = []
    for m, inf in zip(ms, infos):
        k = inf["k_used"]
        ok = inf["status"] == 0 and inf["err_est"] <= tol / 10 and k < k_max
        out.append(dict(m=m, k=k, ok=bool(ok), cost=k * (k / 2 + m) + setup_each[m], err_est=inf["err_est"]))
    for m in grid[1:]:
        if m not in ms:
            out.append(dict(m=m, k=k_max, ok=False, cost=float("inf"), err_est=None))
    out.sort(key=lambda r: r["m"])
    for x in defl[1:]:
        ovl.ovl_destroy_deflation(x)
    return out


def random_config_scaled(rng):
    """Training ranges at scale: mu ~ U[0, 1], eps ~ U[0.2, 0.6], m_w ~ U[-1.5, -0.8]."""
    return dict(eps=float(rng.uniform(0.2, 0.6)), mu=float(rng.uniform(0.0, 1.0)),
                m_w=float(rng.uniform(-1.5, -0.8)), seed=int(rng.integers(1 << 30)))


def generate_scaled(n6, n8, seed=1, path=None, log=print, seconds=None):
    """Runs of the method on 6^4 and 8^4 lattices (n6 and n8 of them,
    interleaved 6^4-first in the proportion n6 : n8): features and the
    cost-minimal (k, m) over M_GRID_LR, written to path after every run; stops
    after `seconds` (the runs done so far are kept)."""
    rng = np.random.default_rng(seed)
    rows = []
    t0 = time.time()
    plan = []
    i6 = i8 = 0
    while i6 < n6 or i8 < n8:  # interleave so that a time limit keeps both sizes
        if i8 >= n8 or (i6 < n6 and i6 * (n8 or 1) <= i8 * (n6 or 1)):
            plan.append((6, 6, 6, 6))
            i6 += 1
        else:
            plan.append((8, 8, 8, 8))
            i8 += 1
    for i, dims in enumerate(plan):
        if seconds is not None and time.time() - t0 > seconds:
            break
        cfg = dict(random_config_scaled(rng), dims=list(dims))
        U = synth.random_su3_field(dims, cfg["eps"], cfg["seed"])
        b = synth.gaussian_source(dims, cfg["seed"] + 1)
        h = ovl.ovl_create_lattice(dims)
        try:
            ovl.ovl_set_links(h, U)
            f = features(h, dims, cfg["mu"], cfg["m_w"], b)
            res = measure_lr(h, dims, cfg["mu"], cfg["m_w"], b)
        finally:
            ovl.ovl_destroy_lattice(h)
        good = [r for r in res if r["ok"]]
        best = min(good, key=lambda r: r["cost"]) if good else None
        rows.append(dict(config=cfg, features=[float(v) for v in f], results=res,
                         label=None if best is None else [best["k"], best["m"]]))
        log(f"[{i + 1}/{len(plan)}] {time.time() - t0:.0f}s {dims} label {rows[-1]['label']}")
        if path:
            json.dump({"dims": "6^4 and 8^4", "m_grid": list(M_GRID_LR), "scheme": "LR", "rows": rows},
                      open(path, "w"))
    return rows


def run_config(cfg, dims=(4, 4, 4, 4)):
    U = synth.random_su3_field(dims, cfg["eps"], cfg["seed"])
    b = synth.gaussian_source(dims, cfg["seed"] + 1)
    h = ovl.ovl_create_lattice(dims)
    try:
        ovl.ovl_set_links(h, U)
        f = features(h, dims, cfg["mu"], cfg["m_w"], b)
        res = measure(h, cfg["mu"], cfg["m_w"], b)
    finally:
        ovl.ovl_destroy_lattice(h)
    good = [r for r in res if r["ok"]]
    best = min(good, key=lambda r: r["cost"]) if good else None
    return dict(config=cfg, features=[float(v) for v in f], results=res,
                label=None if best is None else [best["k"], best["m"]])


def generate(n, seed=0, path=DATA):
    rng = np.random.default_rng(seed)
    rows = []
    t0 = time.time()
    for i in range(n):
        rows.append(run_config(random_config(rng)))
        print(f"[{i + 1}/{n}] {time.time() - t0:.0f}s label {rows[-1]['label']}", flush=True)
        json.dump({"dims": [4, 4, 4, 4], "m_grid": list(M_GRID), "rows": rows}, open(path, "w"))
    return rows


def to_xy(rows):
    rows = [r for r in rows if r["label"] is not None]
    X = np.array([r["features"] for r in rows], dtype=np.float32)
    T = np.array([[math.log(r["label"][0]), math.log(r["label"][1] + 1)] for r in rows], dtype=np.float32)
    return X, T


class Predictor:
    """Standardised features -> MLP (GPU) -> (k, m)."""

    def __init__(self, seed=0):
        self.net = ovl.ovl_mlp_create(N_IN, N_HIDDEN, N_OUT)
        npar = ovl.ovl_mlp_num_params(self.net)
        rng = np.random.default_rng(seed)
        # He initialisation drawn on the host (input data), biases zero
        theta = []
        for fan_in, fan_out in ((N_IN, N_HIDDEN), (N_HIDDEN, N_HIDDEN), (N_HIDDEN, N_OUT)):
            theta.append(rng.standard_normal(fan_in * fan_out) * math.sqrt(2.0 / fan_in))
            theta.append(np.zeros(fan_out))
        self.theta0 = np.concatenate(theta).astype(np.float32)
        assert self.theta0.size == npar
        ovl.ovl_mlp_set_params(self.net, self.theta0)
        self.mu_x = np.zeros(N_IN, np.float32)
        self.sd_x = np.ones(N_IN, np.float32)

    def fit(self, X, T, steps=3000, lr=3e-3):
        self.mu_x = X.mean(0)
        self.sd_x = X.std(0) + 1e-6
        Xs = ((X - self.mu_x) / self.sd_x).astype(np.float32)
        return ovl.ovl_mlp_train(self.net, np.ascontiguousarray(Xs), np.ascontiguousarray(T), steps, lr,
                                 UNDER_WEIGHT)

    def predict(self, X):
        Xs = ((np.atleast_2d(X) - self.mu_x) / self.sd_x).astype(np.float32)
        Y = np.zeros((Xs.shape[0], N_OUT), np.float32)
        ovl.ovl_mlp_forward(self.net, np.ascontiguousarray(Xs), Y)
        k = np.exp(Y[:, 0])
        m = np.exp(Y[:, 1]) - 1
        return k, m

    def save(self, path):
        """Weights (from the device) and the feature standardisation, as .npz."""
        theta = np.zeros(ovl.ovl_mlp_num_params(self.net), np.float32)
        ovl.ovl_mlp_get_params(self.net, theta)
        np.savez(path, theta=theta, mu_x=self.mu_x, sd_x=self.sd_x,
                 shape=np.array([N_IN, N_HIDDEN, N_OUT], np.int64))

    @classmethod
    def load(cls, path):
        z = np.load(path)
        if tuple(z["shape"]) != (N_IN, N_HIDDEN, N_OUT):
            raise ValueError(f"{path}: network shape {tuple(z['shape'])}, expected {(N_IN, N_HIDDEN, N_OUT)}")
        p = cls()
        ovl.ovl_mlp_set_params(p.net, np.ascontiguousarray(z["theta"], dtype=np.float32))
        p.mu_x, p.sd_x = z["mu_x"].astype(np.float32), z["sd_x"].astype(np.float32)
        return p

    def close(self):
        ovl.ovl_mlp_destroy(self.net)


def nearest_m(m, grid=M_GRID):
    return min(grid, key=lambda g: abs(g - m))


def plan_depths(k_pred, margin=1.25, k_floor=20, every=10, k_cap=700):
    """Adaptive depth settings from predicted depths: each solve starts its
    checks at the predicted k (rounded down to the check interval) and may run
    to margin x k (the adaptive estimate is the fallback when the prediction is
    short); the basis is sized for that k_max."""
    out = []
    for k in np.atleast_1d(k_pred):
        k0 = min(k_cap, max(k_floor, int(k) // every * every))
        out.append((k0, max(k0, min(k_cap, int(math.ceil(margin * k))))))
    return out


def admit(h, params, defl, budget_bytes, workspace=None):
    """Split the solves into batches whose device workspace (the library's
    ovl_sign_workspace_bytes for the batch) fits budget_bytes. Solves are
    taken by decreasing basis size (k_max, else k) and each goes to the first
    batch it fits in; a solve that does not fit alone raises ValueError.
    Returns lists of solve indices."""
    ws = workspace or (lambda p, d: ovl.ovl_sign_workspace_bytes(h, p, d))
    order = sorted(range(len(params)), key=lambda i: -max(params[i]["k"], params[i].get("k_max", 0)))
    batches = []
    for i in order:
        if ws([params[i]], [defl[i]]) > budget_bytes:
            raise ValueError(f"solve {i} needs more than {budget_bytes} bytes on its own")
        for bt in batches:
            if ws([params[j] for j in bt + [i]], [defl[j] for j in bt + [i]]) <= budget_bytes:
                bt.append(i)
                break
        else:
            batches.append([i])
    return [sorted(bt) for bt in batches]


if __name__ == "__main__":
    import sys

    from paper_0710_0341_gb300 import build

    build.build()
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 48
    generate(n, path=sys.argv[2] if len(sys.argv) > 2 else DATA)
