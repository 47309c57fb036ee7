"""Pins for the FP64 reference of the selector network and statistics (test infrastructure)."""
import numpy as np

from oracle import mlp
from paper_2009_00767_gb300 import inputs


def _params(n_in, hidden, seed):
    n = n_in * hidden + hidden + hidden * hidden + hidden + hidden * 2 + 2
    return (inputs.u01(seed, 0, n) - 0.5) * 0.6


def test_backprop_matches_central_differences():
    n_in, hidden = 7, 5
    w = _params(n_in, hidden, 1)
    x = inputs.u01(2, 0, 9 * n_in).reshape(9, n_in) - 0.3
    t = inputs.u01(3, 0, 18).reshape(9, 2)
    loss, g = mlp.loss_grad(w, x, t, n_in, hidden)
    h = 1e-6
    num = np.empty_like(w)
    for i in range(w.shape[0]):
        e = np.zeros_like(w)
        e[i] = h
        num[i] = (mlp.loss_grad(w + e, x, t, n_in, hidden)[0] - mlp.loss_grad(w - e, x, t, n_in, hidden)[0]) / (2 * h)
    assert np.max(np.abs(num - g)) <= 1e-7 * max(1.0, np.max(np.abs(g)))
    assert abs(loss - np.mean(np.sum((mlp.forward(w, x, n_in, hidden) - t) ** 2, axis=1))) < 1e-14


def test_zero_hidden_weights_give_the_output_bias():
    n_in, hidden = 4, 3
    w = np.zeros(n_in * hidden + hidden + hidden * hidden + hidden + hidden * 2 + 2)
    w[-2:] = [0.25, -1.5]
    y = mlp.forward(w, np.ones((3, n_in)), n_in, hidden)
    assert np.array_equal(y, np.tile([0.25, -1.5], (3, 1)))


def test_occupancy_features_by_hand():
    # four particles in one finest square, one far away: every level has two occupied squares
    xy = np.array([[0.001, 0.001], [0.0011, 0.0012], [0.0013, 0.001], [0.001, 0.0015], [4.9, 4.9]])
    f = mlp.occupancy_features(xy)
    assert f.shape == (mlp.N_FEAT,)
    for k in range(mlp.LEV_MIN, mlp.LEV_MAX + 1):
        row = f[(k - mlp.LEV_MIN) * mlp.BINS:(k - mlp.LEV_MIN + 1) * mlp.BINS] * (1 << (2 * k))
        want = np.zeros(mlp.BINS)
        want[0] = (1 << (2 * k)) - 2      # empty squares: log2(0 + 1) = 0
        want[1] = 1                       # one particle: log2(2) = 1
        want[2] = 1                       # four particles: floor(log2(5)) = 2
        assert np.array_equal(row, want)
    assert abs(f[-1] - np.log2(5) / 22) < 1e-15
