"""Pins for the selector network's oracle (oracle/mlp.py): the analytic
backward pass against central finite differences in float64, and closed
forms of the softmax cross-entropy."""
import numpy as np

from oracle import mlp


def test_zero_network_closed_forms():
    """All weights zero: softmax is uniform, loss = log C, the gradient of the
    last bias is (1/C - onehot(y)) averaged over the batch, every other
    gradient vanishes (ReLU of zero has zero slope here)."""
    C, B = 5, 7
    params = [np.zeros_like(p) for p in mlp.init(C)]
    rng = np.random.default_rng(0)
    X = rng.standard_normal((B, 32))
    y = rng.integers(0, C, B)
    assert abs(mlp.loss(params, X, y) - np.log(C)) < 1e-15
    g = mlp.backward(params, X, y)
    want = np.full(C, 1.0 / C) - np.bincount(y, minlength=C) / B
    assert np.allclose(g[5], want, atol=1e-15)
    for gi in g[:5]:
        assert not gi.any()


def test_backward_matches_finite_differences():
    C, B = 5, 9
    params = mlp.init(C, seed=3)
    rng = np.random.default_rng(1)
    # nudge the biases so that no pre-activation sits at the ReLU kink
    params = [p + (0.01 * rng.standard_normal(p.shape) if p.ndim == 1 else 0) for p in params]
    X = rng.standard_normal((B, 32))
    y = rng.integers(0, C, B)
    g = mlp.backward(params, X, y)
    h = 1e-6
    for pi, p in enumerate(params):
        flat = p.reshape(-1)
        for idx in rng.choice(flat.size, size=min(12, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss(params, X, y)
            flat[idx] = old - h
            lm = mlp.loss(params, X, y)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[pi].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (pi, idx, fd, an)


def test_sgd_reduces_loss_on_separable_data():
    C = 4
    rng = np.random.default_rng(2)
    X = rng.standard_normal((64, 32))
    y = np.argmax(X[:, :C], axis=1)
    params = mlp.init(C, seed=5)
    l0 = mlp.loss(params, X, y)
    for _ in range(200):
        params = mlp.sgd(params, mlp.backward(params, X, y), 0.05)
    assert mlp.loss(params, X, y) < 0.2 * l0
    assert (mlp.predict(params, X) == y).mean() > 0.9
