"""Pins for the selector network's oracle (oracle/mlp.py): the analytic
backward pass against central finite differences in float64, closed forms
of the softmax cross-entropy, of the feature standardisation and the
invariance of the network under folding the standardisation into its first
layer."""
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


def test_standardize_closed_forms():
    """Column j = a_j + b_j t with t alternating -1, +1 over an even number of
    rows: mean a_j and population deviation |b_j| exactly (the sample
    deviation would be |b_j| sqrt(n / (n - 1))); a constant column keeps the
    scale 1 and standardises to zeros; every other standardised column has
    mean 0 and population deviation 1."""
    n = 6
    t = np.array([-1.0, 1.0] * (n // 2))
    a = np.array([3.0, -2.0, 0.5, 7.0])
    b = np.array([2.0, -0.25, 4.0, 0.0])
    X = a[None, :] + b[None, :] * t[:, None]
    mu, sd, Xs = mlp.standardize(X)
    assert np.array_equal(mu, a)
    assert np.array_equal(sd, np.where(b == 0, 1.0, np.abs(b)))
    assert not Xs[:, 3].any()
    for j in range(3):
        assert np.array_equal(Xs[:, j], t * np.sign(b[j]))
    rng = np.random.default_rng(4)
    Y = rng.standard_normal((50, 32)) * 10.0 ** rng.uniform(-3, 3, 32) + rng.uniform(-50, 50, 32)
    _, _, Ys = mlp.standardize(Y)
    # rounding only: |mu| / sd reaches 5e4 here, times a few ulps
    assert np.allclose(Ys.mean(axis=0), 0.0, atol=1e-9)
    assert np.allclose(Ys.std(axis=0), 1.0, rtol=1e-9)


def test_fold_leaves_the_network_unchanged():
    """The folded network on raw rows gives the logits of the unfolded network
    on standardised rows (float64 rounding only); the deeper layers are the
    same arrays."""
    C = 5
    rng = np.random.default_rng(6)
    X = rng.standard_normal((40, 32)) * 10.0 ** rng.uniform(-2, 2, 32) + rng.uniform(-20, 20, 32)
    X[:, 11] = -4.0  # a constant feature (scale 1)
    params = mlp.init(C, seed=8)
    params = [p + (0.05 * rng.standard_normal(p.shape) if p.ndim == 1 else 0) for p in params]
    mu, sd, Xs = mlp.standardize(X)
    want = mlp.forward(params, Xs)[-1]
    folded = mlp.fold(params, mu, sd)
    got = mlp.forward(folded, X)[-1]
    assert np.allclose(got, want, rtol=1e-9, atol=1e-9 * np.abs(want).max())
    for p, q in zip(folded[2:], params[2:]):
        assert p is q
