"""Oracle for the learned precision selector's network (test infrastructure).

A plain numpy float64 multilayer perceptron 32 -> 128 -> 128 -> C with ReLU
hidden layers and a softmax cross-entropy loss averaged over the batch, its
analytic backward pass and one plain SGD step.  The GPU trains the same
network in float32 with its own kernels; tests compare the two and check this
file against central finite differences and closed forms.  The features are
standardised before training (per-feature mean and population standard
deviation over the training rows) and the scaling is then folded into the
first layer, so that the trained network takes raw features.

Parameter layout (shared in meaning with the CUDA kernels, not in code):
W1 (32 x 128), b1 (128), W2 (128 x 128), b2 (128), W3 (128 x C), b3 (C),
row-major, activations h = x @ W + b.
"""
import numpy as np

SIZES = (32, 128, 128)


def init(C, seed=0):
    """He-style uniform initialisation with a fixed seed (the GPU tests load
    these same arrays)."""
    rng = np.random.default_rng(seed)
    dims = list(SIZES) + [C]
    params = []
    for i in range(3):
        lim = np.sqrt(6.0 / dims[i])
        params.append(rng.uniform(-lim, lim, (dims[i], dims[i + 1])))
        params.append(np.zeros(dims[i + 1]))
    return params


def forward(params, X):
    W1, b1, W2, b2, W3, b3 = params
    z1 = X @ W1 + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2 + b2
    a2 = np.maximum(z2, 0.0)
    z3 = a2 @ W3 + b3
    return z1, a1, z2, a2, z3


def softmax(z):
    m = z.max(axis=1, keepdims=True)
    e = np.exp(z - m)
    return e / e.sum(axis=1, keepdims=True)


def loss(params, X, y):
    z3 = forward(params, X)[-1]
    p = softmax(z3)
    return float(-np.mean(np.log(p[np.arange(len(y)), y])))


def backward(params, X, y):
    """Gradients of the mean cross-entropy w.r.t. every parameter."""
    W1, b1, W2, b2, W3, b3 = params
    z1, a1, z2, a2, z3 = forward(params, X)
    B = X.shape[0]
    d3 = softmax(z3)
    d3[np.arange(B), y] -= 1.0
    d3 /= B
    gW3 = a2.T @ d3
    gb3 = d3.sum(axis=0)
    d2 = (d3 @ W3.T) * (z2 > 0)
    gW2 = a1.T @ d2
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2.T) * (z1 > 0)
    gW1 = X.T @ d1
    gb1 = d1.sum(axis=0)
    return [gW1, gb1, gW2, gb2, gW3, gb3]


def sgd(params, grads, lr):
    return [p - lr * g for p, g in zip(params, grads)]


def predict(params, X):
    return np.argmax(forward(params, X)[-1], axis=1)


def standardize(X, eps=1e-6):
    """Per-feature mean and population standard deviation over the rows of X
    (float64); a feature whose deviation is below eps keeps the scale 1.
    Returns mu, sd and the standardised rows (X - mu) / sd."""
    X = np.asarray(X, dtype=np.float64)
    mu = X.mean(axis=0)
    sd = X.std(axis=0)
    sd = np.where(sd < eps, 1.0, sd)
    return mu, sd, (X - mu) / sd


def fold(params, mu, sd):
    """The first layer rewritten for raw features:
    ((x - mu) / sd) W1 + b1 = x (W1 / sd[:, None]) + (b1 - (mu / sd) W1)."""
    W1, b1 = params[0], params[1]
    mu = np.asarray(mu, dtype=np.float64)
    sd = np.asarray(sd, dtype=np.float64)
    return [W1 / sd[:, None], b1 - (mu / sd) @ W1] + list(params[2:])
