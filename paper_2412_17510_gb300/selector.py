"""Training and evaluation of the learned precision selector.

Host-side orchestration of C-ABI calls only: features come from
``mpspmv_cg_history`` + ``mpspmv_features``, labels from batched CG solves at
each precision (``mpspmv_batch_cg``, the method's own solves), training from
the float32 MLP kernels (``mpspmv_mlp_train``), decisions from
``mpspmv_select_precision`` / ``mpspmv_solve_auto`` and the plain ladder
(``mpspmv_ladder_solve``) stays as fallback and judge.

Classes: 0 binary64, 1 DD, 2 TD, 3 QD, 4 none (QD does not reach the target
within the iteration cap); a label is the cheapest class whose CG, from
x0 = 0, ends with a residual b - A x (recomputed in that precision) of at
most rtol ||b||.
"""
import time

import numpy as np

from . import (MPSPMV_OK, mpspmv_batch_cg, mpspmv_batch_create, mpspmv_batch_destroy, mpspmv_cg_history,
               mpspmv_create_csr, mpspmv_destroy, mpspmv_features, mpspmv_ladder_solve, mpspmv_mlp_forward,
               mpspmv_mlp_param_count, mpspmv_mlp_train, mpspmv_solve_auto)

NCLASS = 5


class System:
    """One SPD system with handles at L = 1..4 and its right-hand side;
    ``flags`` (e.g. MPSPMV_EXACT_ACC) apply to every handle."""

    def __init__(self, coo, b, flags=0):
        import torch
        self.n = coo.nrows
        self.handles = [mpspmv_create_csr(coo.nrows, coo.ncols, coo.row, coo.col, coo.val, L, flags, val_limbs=1)
                        for L in (1, 2, 3, 4)]
        self.b = torch.from_numpy(np.ascontiguousarray(b[None, :])).cuda()

    def free(self):
        for h in self.handles:
            mpspmv_destroy(h)
        self.handles = []


def features(sys_list):
    out = np.zeros((len(sys_list), 32), dtype=np.float32)
    for i, s in enumerate(sys_list):
        hist = mpspmv_cg_history(s.handles[0], s.b, 8)
        out[i] = mpspmv_features(s.handles[0], hist)
    return out


def solve_level_batched(sys_list, L, rtol, maxit):
    """Batched CG of every system at level L; returns (success mask,
    iterations, relres)."""
    import torch
    hs = [s.handles[L - 1] for s in sys_list]
    b = mpspmv_batch_create(hs, [1] * len(hs), 0)
    try:
        Bs = []
        for s in sys_list:
            B = torch.zeros((L, s.n, 1), dtype=torch.float64, device="cuda")
            B[0, :, 0] = s.b[0]
            Bs.append(B)
        Xs = [torch.zeros_like(B) for B in Bs]
        st, it, rr, ss = mpspmv_batch_cg(b, Bs, Xs, len(hs), rtol, 0.0, maxit)
        ok = (ss == MPSPMV_OK) & (rr <= rtol)
        return ok, it, rr
    finally:
        mpspmv_batch_destroy(b)


def labels(sys_list, rtol, maxit_factor=2):
    lab = np.full(len(sys_list), NCLASS - 1, dtype=np.int32)
    maxit = maxit_factor * max(s.n for s in sys_list)
    for L in (1, 2, 3, 4):
        todo = [i for i in range(len(sys_list)) if lab[i] == NCLASS - 1]
        if not todo:
            break
        ok, it, _ = solve_level_batched([sys_list[i] for i in todo], L, rtol, maxit)
        for j, i in enumerate(todo):
            # the cap is maxit_factor * n per system (one batch shares the largest)
            if ok[j] and it[j] <= maxit_factor * sys_list[i].n:
                lab[i] = L - 1
    return lab


def init_params(seed=0, C=NCLASS):
    """He-style uniform initialisation, same layout as the kernels."""
    rng = np.random.default_rng(seed)
    dims = [32, 128, 128, C]
    parts = []
    for i in range(3):
        lim = np.sqrt(6.0 / dims[i])
        parts.append(rng.uniform(-lim, lim, (dims[i], dims[i + 1])).reshape(-1))
        parts.append(np.zeros(dims[i + 1]))
    out = np.concatenate(parts).astype(np.float32)
    assert out.size == mpspmv_mlp_param_count(C)
    return out


def fold_standardisation(params, mu, sd, C=NCLASS):
    """Rewrite W1, b1 so that the network takes raw features:
    (x - mu) / sd @ W1 + b1 = x @ (W1 / sd[:, None]) + (b1 - (mu / sd) @ W1)."""
    p = params.astype(np.float64).copy()
    W1 = p[:32 * 128].reshape(32, 128)
    b1 = p[32 * 128:32 * 128 + 128]
    nb1 = b1 - (mu / sd) @ W1
    W1 /= sd[:, None]
    p[32 * 128:32 * 128 + 128] = nb1
    return p.astype(np.float32)


def train(X, y, epochs=200, batch=32, lr=0.05, seed=0, C=NCLASS):
    """Train on standardised features with the GPU kernels (plain SGD, data
    reshuffled every epoch); returns parameters for raw features, the loss
    history and (mu, sd)."""
    import torch
    mu = X.mean(axis=0)
    sd = X.std(axis=0)
    sd[sd < 1e-6] = 1.0
    Xs = ((X - mu) / sd).astype(np.float32)
    rng = np.random.default_rng(seed)
    dp = torch.from_numpy(init_params(seed, C)).cuda()
    losses = []
    for _ in range(epochs):
        perm = rng.permutation(len(y))
        dX = torch.from_numpy(np.ascontiguousarray(Xs[perm])).cuda()
        dy = torch.from_numpy(np.ascontiguousarray(y[perm].astype(np.int32))).cuda()
        losses.append(float(mpspmv_mlp_train(dp, C, dX, dy, len(y), batch, 1, lr)[0]))
    raw = fold_standardisation(dp.cpu().numpy(), mu, sd, C)
    return raw, np.array(losses), (mu, sd)


def predict(params, X, C=NCLASS):
    import torch
    dp = torch.from_numpy(np.ascontiguousarray(params)).cuda()
    lg = torch.empty((len(X), C), dtype=torch.float32, device="cuda")
    mpspmv_mlp_forward(dp, C, torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda(), len(X), lg)
    return lg.argmax(dim=1).cpu().numpy()


def evaluate(sys_list, params, rtol, maxit_factor=2, C=NCLASS):
    """Per held-out system: the plain ladder from binary64, the selector-guided
    ladder (solve_auto), each timed end to end; plus the batched selector-
    guided solve of all systems (predicted level first, failures move up a
    level in the next batch).  Returns a dict of totals."""
    import torch
    dp = torch.from_numpy(np.ascontiguousarray(params)).cuda()
    res = {"plain_s": 0.0, "auto_s": 0.0, "plain_ok": 0, "auto_ok": 0, "escalated": 0, "chosen": [], "final": []}
    for s in sys_list:
        maxit = maxit_factor * s.n
        x = torch.zeros((4, s.n), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, fl, its, rr = mpspmv_ladder_solve(s.handles, 1, s.b, x, rtol, 0.0, maxit)
        torch.cuda.synchronize()
        res["plain_s"] += time.perf_counter() - t0
        res["plain_ok"] += int(st == MPSPMV_OK)
        x.zero_()
        t0 = time.perf_counter()
        st2, ch, fl2, its2, rr2 = mpspmv_solve_auto(s.handles, dp, C, s.b, x, rtol, 0.0, maxit)
        torch.cuda.synchronize()
        res["auto_s"] += time.perf_counter() - t0
        res["auto_ok"] += int(st2 == MPSPMV_OK)
        res["escalated"] += int(fl2 > ch)
        res["chosen"].append(ch)
        res["final"].append(fl2)
    # batched, selector-guided
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X = features(sys_list)
    level = np.minimum(predict(params, X, C) + 1, 4)
    done = np.zeros(len(sys_list), dtype=bool)
    maxit = maxit_factor * max(s.n for s in sys_list)
    for L in (1, 2, 3, 4):
        idx = [i for i in range(len(sys_list)) if not done[i] and level[i] <= L]
        if not idx:
            continue
        ok, it, _ = solve_level_batched([sys_list[i] for i in idx], L, rtol, maxit)
        for j, i in enumerate(idx):
            if ok[j] and it[j] <= maxit_factor * sys_list[i].n:
                done[i] = True
    torch.cuda.synchronize()
    res["batched_auto_s"] = time.perf_counter() - t0
    res["batched_auto_ok"] = int(done.sum())
    res["n"] = len(sys_list)
    return res
