"""FP64 reference of the selector network and its statistics -- TEST INFRASTRUCTURE ONLY.

The selector of the library is a two-hidden-layer ReLU network (a learned stand-in for the
choice of tree depth and expansion order; it has no counterpart in arXiv 2009.00767).  This
module states, in plain numpy FP64, what its kernels compute, so that their outputs and
gradients can be checked:

* ``forward`` / ``loss_grad`` -- y = W3^T relu(W2^T relu(W1^T x + b1) + b2) + b3 per row,
  loss = (1/rows) sum_r sum_j (y_rj - t_rj)^2 and its gradient by backpropagation, with the
  parameters in the library's layout [W1 (IN x H) | b1 | W2 (H x H) | b2 | W3 (H x 2) | b3];
* ``occupancy_features`` -- for levels 3..11 of the uniform quadtree over [0, box]^2 the
  fraction of squares whose population c falls in bin floor(log2(c + 1)) (12 bins, the last
  one open), then log2(N) / 22.
"""
from __future__ import annotations

import numpy as np

LEV_MIN, LEV_MAX, BINS = 3, 11, 12
N_FEAT = (LEV_MAX - LEV_MIN + 1) * BINS + 1
N_IN = N_FEAT + 2
N_OUT = 2


def unpack(w, n_in, hidden, n_out=N_OUT):
    w = np.asarray(w, dtype=np.float64)
    o = 0
    W1 = w[o:o + n_in * hidden].reshape(n_in, hidden); o += n_in * hidden
    b1 = w[o:o + hidden]; o += hidden
    W2 = w[o:o + hidden * hidden].reshape(hidden, hidden); o += hidden * hidden
    b2 = w[o:o + hidden]; o += hidden
    W3 = w[o:o + hidden * n_out].reshape(hidden, n_out); o += hidden * n_out
    b3 = w[o:o + n_out]; o += n_out
    assert o == w.shape[0]
    return W1, b1, W2, b2, W3, b3


def forward(w, x, n_in, hidden):
    W1, b1, W2, b2, W3, b3 = unpack(w, n_in, hidden)
    x = np.asarray(x, dtype=np.float64)
    h1 = np.maximum(x @ W1 + b1, 0.0)
    h2 = np.maximum(h1 @ W2 + b2, 0.0)
    return h2 @ W3 + b3


def loss_grad(w, x, t, n_in, hidden):
    """Loss and its gradient with respect to the flat parameter vector (backpropagation)."""
    W1, b1, W2, b2, W3, b3 = unpack(w, n_in, hidden)
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    rows = x.shape[0]
    z1 = x @ W1 + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2 + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3 + b3
    loss = float(np.sum((y - t) ** 2) / rows)
    dy = 2.0 * (y - t) / rows
    dW3 = h2.T @ dy
    db3 = dy.sum(0)
    dh2 = (dy @ W3.T) * (z2 > 0)
    dW2 = h1.T @ dh2
    db2 = dh2.sum(0)
    dh1 = (dh2 @ W2.T) * (z1 > 0)
    dW1 = x.T @ dh1
    db1 = dh1.sum(0)
    return loss, np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])


def occupancy_features(xy, box=5.0):
    """The selector's 109 statistics of a particle system, by counting."""
    xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
    side = 1 << LEV_MAX
    ix = np.clip(np.floor(xy[:, 0] * float(side) / box), 0, side - 1).astype(np.int64)
    iy = np.clip(np.floor(xy[:, 1] * float(side) / box), 0, side - 1).astype(np.int64)
    feats = []
    for k in range(LEV_MIN, LEV_MAX + 1):
        sh = LEV_MAX - k
        cnt = np.bincount((iy >> sh) * (1 << k) + (ix >> sh), minlength=1 << (2 * k))
        b = np.minimum(BINS - 1, np.floor(np.log2(cnt + 1.0)).astype(np.int64))
        feats.append(np.bincount(b, minlength=BINS) / float(1 << (2 * k)))
    feats.append([np.log2(xy.shape[0]) / 22.0])
    return np.concatenate(feats)
