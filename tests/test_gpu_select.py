"""Precision ladder, selector features and the float32 MLP kernels (C ABI)
against their oracles (oracle/features.py, oracle/mlp.py, oracle CG)."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import features as ofeat
from oracle import mlp as omlp
from tests._util import to_dev

pytestmark = pytest.mark.gpu

mps = pytest.importorskip("paper_2412_17510_gb300")
torch = pytest.importorskip("torch")


def handles(coo, levels=(1, 2, 3, 4)):
    return [mps.mpspmv_create_csr(coo.nrows, coo.ncols, coo.row, coo.col, coo.val, L, 0, val_limbs=1)
            if L in levels else None for L in (1, 2, 3, 4)]


def destroy(hs):
    for h in hs:
        if h is not None:
            mps.mpspmv_destroy(h)


def flat_params(params):
    return np.concatenate([p.reshape(-1) for p in params]).astype(np.float32)


@pytest.mark.parametrize("kind", ["laplace", "diffusion", "selector"])
def test_features_match_oracle(kind):
    if kind == "laplace":
        coo = workloads.laplacian_2d(20, 15)
        b = np.random.default_rng(0).uniform(-1, 1, coo.nrows)
    elif kind == "diffusion":
        coo = workloads.diffusion_7pt(9, 8, 7, seed=3)
        b = np.random.default_rng(1).uniform(-1, 1, coo.nrows)
    else:
        coo, b = workloads.selector_system(300, 14.0, seed=5)
    h = mps.mpspmv_create_csr(coo.nrows, coo.ncols, coo.row, coo.col, coo.val, 1, 0)
    try:
        hist = mps.mpspmv_cg_history(h, to_dev(b[None, :]), 8)
        A = oracle.coo_to_csr(coo.nrows, coo.ncols, coo.row, coo.col, coo.val, 1)
        ref_hist = ofeat.cg_history(A.indptr, A.indices.astype(np.int64), A.data[0], b, 8)
        assert np.allclose(hist, ref_hist, rtol=1e-6, atol=0)
        f = mps.mpspmv_features(h, hist)
        ref = ofeat.features(A, b)
        assert np.allclose(f, ref, rtol=2e-5, atol=2e-5), np.nonzero(~np.isclose(f, ref, rtol=2e-5, atol=2e-5))
    finally:
        mps.mpspmv_destroy(h)


def test_mlp_forward_and_gradients_match_oracle():
    C, B = 5, 48
    params = omlp.init(C, seed=2)
    rng = np.random.default_rng(4)
    params = [p + (0.05 * rng.standard_normal(p.shape) if p.ndim == 1 else 0) for p in params]
    X = rng.standard_normal((B, 32))
    y = rng.integers(0, C, B)
    p32 = [q.astype(np.float32).astype(np.float64) for q in params]
    X32 = X.astype(np.float32)
    dp = to_dev(flat_params(params))
    assert dp.numel() == mps.mpspmv_mlp_param_count(C)
    dX = to_dev(X32)
    dy = to_dev(y.astype(np.int32))
    logits = torch.empty((B, C), dtype=torch.float32, device="cuda")
    mps.mpspmv_mlp_forward(dp, C, dX, B, logits)
    ref_logits = omlp.forward(p32, X32.astype(np.float64))[-1]
    assert np.allclose(logits.cpu().numpy(), ref_logits, rtol=1e-4, atol=1e-4)
    g = torch.empty_like(dp)
    loss = mps.mpspmv_mlp_grad(dp, C, dX, dy, B, g)
    assert abs(loss - omlp.loss(p32, X32.astype(np.float64), y)) <= 1e-5 * max(1, loss)
    ref = omlp.backward(p32, X32.astype(np.float64), y)
    got = g.cpu().numpy().astype(np.float64)
    off = 0
    for r in ref:
        gg = got[off:off + r.size].reshape(r.shape)
        off += r.size
        assert np.allclose(gg, r, rtol=1e-3, atol=1e-5 * (np.abs(r).max() + 1e-12)), r.shape


def test_mlp_training_learns_separable_classes():
    C, n = 4, 512
    rng = np.random.default_rng(6)
    X = rng.standard_normal((n, 32)).astype(np.float32)
    y = np.argmax(X[:, :C], axis=1).astype(np.int32)
    dp = to_dev(flat_params(omlp.init(C, seed=1)))
    losses = mps.mpspmv_mlp_train(dp, C, to_dev(X), to_dev(y), n, 64, 60, 0.05)
    assert losses[-1] < 0.3 * losses[0]
    logits = torch.empty((n, C), dtype=torch.float32, device="cuda")
    mps.mpspmv_mlp_forward(dp, C, to_dev(X), n, logits)
    acc = (logits.argmax(dim=1).cpu().numpy() == y).mean()
    assert acc > 0.9
    # the same training in float64 on the CPU reaches a similar loss
    params = omlp.init(C, seed=1)
    for _ in range(60):
        for b0 in range(0, n, 64):
            params = omlp.sgd(params, omlp.backward(params, X[b0:b0 + 64].astype(np.float64), y[b0:b0 + 64]), 0.05)
    assert abs(omlp.loss(params, X.astype(np.float64), y) - losses[-1]) < 0.1


def test_ladder_escalates_until_the_target_is_met():
    """Laplacian 16x16 (cond ~ 1e2), rtol 1e-28: binary64 cannot reach it,
    DD can; a graded SPD system (cond ~ 1e8), rtol 1e-30: TD is the first."""
    coo = workloads.laplacian_2d(16)
    hs = handles(coo)
    try:
        b = np.random.default_rng(2).uniform(-1, 1, coo.nrows)
        x = torch.zeros((4, coo.nrows), dtype=torch.float64, device="cuda")
        st, fl, its, rr = mps.mpspmv_ladder_solve(hs, 1, to_dev(b[None, :]), x, 1e-28, 0.0, 2 * coo.nrows)
        assert st == 0 and fl == 2 and its[0] > 0 and its[1] > 0 and rr <= 1e-28
        A = oracle.coo_to_csr(coo.nrows, coo.ncols, coo.row, coo.col, coo.promoted(2), 2)
        bb = np.zeros((2, coo.nrows)); bb[0] = b
        ost, ox, oit, orr = oracle.cg(A, bb, rtol=1e-28, maxit=2 * coo.nrows)
        assert ost == 0 and orr <= 1e-28
        xd = x.cpu().numpy()
        assert not xd[2:].any()
        assert np.max(np.abs((xd[0] - ox[0]) + (xd[1] - ox[1]))) <= 1e-24 * np.abs(ox[0]).max()
    finally:
        destroy(hs)
    # graded SPD system (n = 60, cond ~ 1e8): binary64 and DD end above 1e-30
    # (oracle: true residuals 6e-13 and 7e-29), TD reaches it
    coo, b = workloads.selector_system(60, 8.0, seed=9)
    hs = handles(coo)
    try:
        x = torch.zeros((4, coo.nrows), dtype=torch.float64, device="cuda")
        st, fl, its, rr = mps.mpspmv_ladder_solve(hs, 1, to_dev(b[None, :]), x, 1e-30, 0.0, 40 * coo.nrows)
        assert st == 0 and fl == 3 and rr <= 1e-30 and its[0] > 0 and its[1] > 0 and its[2] > 0
        # starting at QD: no lower level runs
        x2 = torch.zeros_like(x)
        st2, fl2, its2, rr2 = mps.mpspmv_ladder_solve(hs, 4, to_dev(b[None, :]), x2, 1e-30, 0.0, 40 * coo.nrows)
        assert st2 == 0 and fl2 == 4 and its2[:3] == [0, 0, 0] and rr2 <= 1e-30
        # the QD solve needs fewer iterations than the TD level of the ladder
        # needed from its restart point (iterations settle as precision rises)
        A = oracle.coo_to_csr(coo.nrows, coo.ncols, coo.row, coo.col, coo.promoted(4), 4)
        bb = np.zeros((4, coo.nrows)); bb[0] = b
        ost, ox, oit, orr = oracle.cg(A, bb, rtol=1e-30, maxit=40 * coo.nrows)
        assert ost == 0 and abs(its2[3] - oit) <= max(3, 0.1 * oit)
    finally:
        destroy(hs)


def test_select_precision_maps_classes_and_solve_auto():
    """A network whose last bias favours class c selects level c + 1 (class 4,
    'none', selects QD); solve_auto starts the ladder there."""
    C = 5
    coo = workloads.laplacian_2d(12)
    hs = handles(coo)
    try:
        b = to_dev(np.random.default_rng(3).uniform(-1, 1, coo.nrows)[None, :])
        for cls, want in ((0, 1), (1, 2), (2, 3), (3, 4), (4, 4)):
            params = [np.zeros_like(p) for p in omlp.init(C)]
            params[5][cls] = 1.0
            dp = to_dev(flat_params(params))
            p, feat = mps.mpspmv_select_precision(hs, dp, C, b)
            assert p == want
            assert feat[0] == pytest.approx(np.log10(coo.nrows), rel=1e-6)
        params = [np.zeros_like(p) for p in omlp.init(C)]
        params[5][2] = 1.0
        x = torch.zeros((4, coo.nrows), dtype=torch.float64, device="cuda")
        st, ch, fl, its, rr = mps.mpspmv_solve_auto(hs, to_dev(flat_params(params)), C, b, x, 1e-30, 0.0, 1000)
        assert st == 0 and ch == 3 and fl == 3 and its[:2] == [0, 0] and rr <= 1e-30
    finally:
        destroy(hs)


def test_trained_selector_saves_ladder_iterations():
    """What the learned part gains over the method without it, and over
    constant rules: the network is trained by the float32 kernels on labels
    from the method's own batched CG solves (graded SPD systems
    A = D (L L^T + I) D, n in [40, 80], cond 10^U[8, 40], target relative
    residual 1e-30, cap 30 n per level), then 16 held-out systems are solved
    by the plain ladder from every fixed start level and by the
    selector-guided ladder.  Binary64 can never reach 1e-30 and DD does not
    on this family, so ladders that start there spend their caps; a constant
    TD start spends its cap on every system that needs QD or reaches the
    target at no level.  The selector-guided ladder needs fewer than 0.8 of
    the CG iterations of the binary64 and DD starts, no more than the TD
    start, and solves as many systems as the cold QD start.  (Ladders that
    pass through a lower level give a system 30 n more iterations, warm, so
    they can solve a system that a cold start at the top leaves at its cap.)
    A constant QD start needs the fewest iterations of all: QD's iteration
    counts are the lowest, and at these sizes an iteration costs about the
    same at every level, so the selector's choice of a lower sufficient level
    saves no time over it here; its measured times are reported by bench.py."""
    from paper_2412_17510_gb300 import selector as sel
    rng = np.random.default_rng(5)
    systems = []
    try:
        for i in range(56):
            n = int(rng.integers(40, 81))
            coo, b = workloads.selector_system(n, float(rng.uniform(8, 40)), seed=2000 + i)
            systems.append(sel.System(coo, b))
        train, held_out = systems[:40], systems[40:]
        X = sel.features(train)
        y = sel.labels(train, 1e-30, maxit_factor=30)
        assert not (y == 0).any()  # binary64 never reaches 1e-30
        params, losses, _ = sel.train(X, y, epochs=200, batch=32, lr=0.05)
        assert losses[-1] < losses[0]
        ev = sel.evaluate(held_out, params, 1e-30, maxit_factor=30)
        lad, auto = ev["ladder"], ev["selector"]
        print("held-out CG iterations / solved: " + ", ".join(
            "start %d: %d / %d" % (L0, lad[L0]["iters"], lad[L0]["solved"]) for L0 in (1, 2, 3, 4)) +
            "; selector: %d / %d (escalated %d) of %d" % (auto["iters"], auto["solved"], auto["escalated"],
                                                          len(held_out)))
        for c, f in zip(auto["chosen"], auto["final"]):
            assert f >= c >= 1
        assert auto["iters"] < 0.8 * min(lad[1]["iters"], lad[2]["iters"])
        assert auto["iters"] <= lad[3]["iters"]
        assert auto["solved"] >= lad[4]["solved"]
    finally:
        for s in systems:
            s.free()


def test_standardisation_kernels_match_the_oracle():
    """mpspmv_mlp_standardize against the oracle's standardisation
    (oracle/mlp.py, float64), and mpspmv_mlp_fold against the oracle's fold
    at the kernel's mean and deviation; the folded network on raw features
    gives the logits of the unfolded network on standardised features (float
    tolerance)."""
    C = 5
    rng = np.random.default_rng(9)
    n = 300
    X = (rng.standard_normal((n, 32)) * 10.0 ** rng.uniform(-3, 3, 32) + rng.uniform(-50, 50, 32)).astype(np.float32)
    X[:, 7] = 3.25  # a constant feature keeps sd = 1
    dX = to_dev(X)
    mu = torch.empty(32, dtype=torch.float32, device="cuda")
    sd = torch.empty(32, dtype=torch.float32, device="cuda")
    Xs = torch.empty_like(dX)
    mps.mpspmv_mlp_standardize(dX, n, mu, sd, Xs)
    torch.cuda.synchronize()
    X64 = X.astype(np.float64)
    mu_ref, sd_ref, _ = omlp.standardize(X64)
    np.testing.assert_allclose(mu.cpu().numpy(), mu_ref, rtol=1e-6, atol=1e-6 * np.abs(X64).max())
    np.testing.assert_allclose(sd.cpu().numpy(), sd_ref, rtol=1e-6)
    assert sd.cpu().numpy()[7] == 1.0
    mu_k = mu.cpu().numpy().astype(np.float64)
    sd_k = sd.cpu().numpy().astype(np.float64)
    xs_ref = (X64 - mu_k) / sd_k  # the oracle's formula at the kernel's float mean and deviation
    np.testing.assert_allclose(Xs.cpu().numpy(), xs_ref, rtol=1e-6, atol=1e-6)
    params = [p.astype(np.float32) for p in omlp.init(C, seed=4)]
    params[1] = (0.1 * rng.standard_normal(params[1].shape)).astype(np.float32)  # a non-zero b1
    dp = to_dev(flat_params(params))
    lg_std = torch.empty((n, C), dtype=torch.float32, device="cuda")
    mps.mpspmv_mlp_forward(dp, C, Xs, n, lg_std)
    mps.mpspmv_mlp_fold(dp, C, mu, sd)
    lg_raw = torch.empty((n, C), dtype=torch.float32, device="cuda")
    mps.mpspmv_mlp_forward(dp, C, dX, n, lg_raw)
    torch.cuda.synchronize()
    folded = dp.cpu().numpy()
    W1f, b1f = folded[:32 * 128].reshape(32, 128), folded[32 * 128:32 * 128 + 128]
    want = omlp.fold([p.astype(np.float64) for p in params], mu_k, sd_k)
    np.testing.assert_allclose(W1f, want[0], rtol=1e-6)
    scale = np.abs(params[1].astype(np.float64)) + np.abs(mu_k / sd_k) @ np.abs(params[0].astype(np.float64))
    assert np.all(np.abs(b1f - want[1]) <= 1e-6 * scale)
    assert np.array_equal(folded[32 * 128 + 128:], flat_params(params)[32 * 128 + 128:])  # deeper layers untouched
    a, b = lg_raw.cpu().numpy(), lg_std.cpu().numpy()
    np.testing.assert_allclose(a, b, rtol=1e-3, atol=1e-3 * np.abs(b).max())
