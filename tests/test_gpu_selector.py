"""The learned (levels, p) selector: statistics, forward, gradients against the FP64 oracle,
training, checkpoint/resume, and what the trained network gains over the fixed fallback."""
import os

import numpy as np
import pytest

from conftest import rel_l2
from paper_2009_00767_gb300 import inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MODEL = os.path.join(ROOT, "paper_2009_00767_gb300", "selector_gb300.bin")


@pytest.fixture(scope="module")
def sel():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_00767_gb300 import binding
    s = binding.Selector(hidden=16, seed=5)
    yield s
    s.close()


@pytest.mark.parametrize("fam,n", [("uniform", 70000), ("gmm", 50000), ("annulus", 30001)])
def test_features_equal_the_counting_oracle(sel, fam, n):
    import torch
    from oracle import mlp
    xy, _ = getattr(inputs, fam)(n, 1234)
    f = sel.features(torch.from_numpy(xy).to("cuda:0"))
    ref = mlp.occupancy_features(xy).astype(np.float32)
    assert np.array_equal(f, ref)


def test_forward_and_gradient_match_fp64_backprop(sel):
    from oracle import mlp
    w = sel.params().astype(np.float64)
    x = (inputs.u01(9, 0, 23 * sel.n_in).reshape(23, sel.n_in) * 1.5).astype(np.float32)
    t = (inputs.u01(9, 1, 46).reshape(23, 2) - 0.5).astype(np.float32)
    y = sel.predict(x)
    y_ref = mlp.forward(w, x.astype(np.float64), sel.n_in, sel.hidden)
    assert np.max(np.abs(y - y_ref)) <= 1e-5 * max(1.0, np.max(np.abs(y_ref)))
    loss, g = sel.loss_grad(x, t)
    loss_ref, g_ref = mlp.loss_grad(w, x.astype(np.float64), t.astype(np.float64), sel.n_in, sel.hidden)
    assert abs(loss - loss_ref) <= 1e-5 * max(1.0, loss_ref)
    assert rel_l2(g, g_ref) < 1e-4


def test_training_fits_and_resumes_from_a_checkpoint(tmp_path):
    from paper_2009_00767_gb300 import binding
    s = binding.Selector(hidden=32, seed=11)
    x = inputs.u01(21, 0, 400 * s.n_in).reshape(400, s.n_in).astype(np.float32)
    t = np.stack([np.sin(3 * x[:, 0]) + x[:, 5], x[:, 109] * x[:, 110]], 1).astype(np.float32)
    l0, _ = s.loss_grad(x, t)
    l1 = s.train(x, t, 400, lr=3e-3)
    assert l1 < 0.2 * l0
    path = str(tmp_path / "sel.bin")
    s.save(path)
    l2 = s.train(x, t, 200, lr=3e-3)
    s2 = binding.Selector(hidden=32, seed=99)
    s2.load(path)
    l2b = s2.train(x, t, 200, lr=3e-3)
    assert abs(l2b - l2) <= 1e-4 * max(1.0, l2)       # same weights, same Adam state, same steps
    s.close()
    s2.close()


@pytest.mark.skipif(not os.path.exists(MODEL), reason="no trained selector model in the package")
def test_trained_selector_beats_the_fixed_fallback():
    """Held-out systems: the learned pick meets 1e-6 (measured against the FP64 direct sum) and costs
    less in total than the fixed (levels, p) = (8, 20)."""
    from paper_2009_00767_gb300 import binding, selector
    s = binding.Selector(hidden=64, seed=1)
    s.load(MODEL)
    rows = selector.evaluate(s, range(990001, 990009))
    s.close()
    for r in rows:
        print(r)
    missed = [r for r in rows if r["err_pick"] > 1e-6]
    assert not missed, f"picks that miss 1e-6: {missed}"
    assert sum(r["ms_pick"] for r in rows) < sum(r["ms_fallback"] for r in rows)
