"""Reference MLP for the (k, m) predictor: plain numpy FP64 forward, loss and
backward pass (TEST INFRASTRUCTURE ONLY, see the package docstring).

Network: x (n_in) -> ReLU(W1 x + b1) (n_h) -> ReLU(W2 h1 + b2) (n_h) -> W3 h2 + b3 (n_out).
Loss over a batch of B rows: mean over rows and outputs of w * (y - t)^2 with
w = under_weight where y < t (under-prediction) and 1 otherwise.
Parameter vector order: W1 (n_h x n_in, row-major), b1, W2, b2, W3, b3.
(The paper has no learned component; this is the predictor's own definition.)
"""
import numpy as np


def unpack(theta, n_in, n_h, n_out):
    sizes = [(n_h, n_in), (n_h,), (n_h, n_h), (n_h,), (n_out, n_h), (n_out,)]
    out, o = [], 0
    for s in sizes:
        n = int(np.prod(s))
        out.append(np.asarray(theta[o:o + n], dtype=np.float64).reshape(s))
        o += n
    return out


def n_params(n_in, n_h, n_out):
    return n_h * n_in + n_h + n_h * n_h + n_h + n_out * n_h + n_out


def forward(theta, X, n_in, n_h, n_out):
    W1, b1, W2, b2, W3, b3 = unpack(theta, n_in, n_h, n_out)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0)
    return h2 @ W3.T + b3, (z1, h1, z2, h2)


def loss_grad(theta, X, T, n_in, n_h, n_out, under_weight=4.0):
    W1, b1, W2, b2, W3, b3 = unpack(theta, n_in, n_h, n_out)
    Y, (z1, h1, z2, h2) = forward(theta, X, n_in, n_h, n_out)
    B = X.shape[0]
    w = np.where(Y < T, under_weight, 1.0)
    loss = float(np.mean(w * (Y - T) ** 2))
    dY = 2.0 * w * (Y - T) / (B * n_out)
    gW3 = dY.T @ h2
    gb3 = dY.sum(0)
    dh2 = dY @ W3
    dz2 = dh2 * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (z1 > 0)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(0)
    g = np.concatenate([a.ravel() for a in (gW1, gb1, gW2, gb2, gW3, gb3)])
    return loss, g
