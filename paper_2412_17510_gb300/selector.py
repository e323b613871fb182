"""Training and evaluation of the learned precision selector.

Host-side orchestration of C-ABI calls only: features come from
``mpspmv_cg_history`` + ``mpspmv_features``, labels from batched CG solves at
each precision (``mpspmv_batch_cg``, the method's own solves), training from
the float32 MLP kernels (``mpspmv_mlp_train``), decisions from
``mpspmv_select_precision`` / ``mpspmv_solve_auto`` and the plain ladder
(``mpspmv_ladder_solve``) stays as the fallback and the check of the choice.

Classes: 0 binary64, 1 DD, 2 TD, 3 QD, 4 none (QD does not reach the target
within the iteration cap); a label is the cheapest class whose CG, from
x0 = 0, ends with a residual b - A x (recomputed in that precision) of at
most rtol ||b||.
"""
import time

import numpy as np

from . import (MPSPMV_OK, mpspmv_batch_cg, mpspmv_batch_create, mpspmv_batch_destroy, mpspmv_cg_history,
               mpspmv_create_csr, mpspmv_destroy, mpspmv_features, mpspmv_ladder_solve, mpspmv_mlp_fold,
               mpspmv_mlp_forward, mpspmv_mlp_param_count, mpspmv_mlp_standardize, mpspmv_mlp_train,
               mpspmv_solve_auto)

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


def train(X, y, epochs=200, batch=32, lr=0.05, seed=0, C=NCLASS):
    """Train with the GPU kernels: the features are standardised on the
    device (mpspmv_mlp_standardize), the network is trained on them by plain
    SGD with the samples reshuffled every epoch, and the standardisation is
    folded into W1 and b1 on the device (mpspmv_mlp_fold), so the returned
    parameters take raw features.  Returns (parameters, loss history,
    (mu, sd))."""
    import torch
    n = len(y)
    dX = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    mu = torch.empty(32, dtype=torch.float32, device="cuda")
    sd = torch.empty(32, dtype=torch.float32, device="cuda")
    dXs = torch.empty_like(dX)
    mpspmv_mlp_standardize(dX, n, mu, sd, dXs)
    Xs = dXs.cpu().numpy()
    rng = np.random.default_rng(seed)
    dp = torch.from_numpy(init_params(seed, C)).cuda()
    losses = []
    for _ in range(epochs):
        perm = rng.permutation(n)
        dXp = torch.from_numpy(np.ascontiguousarray(Xs[perm])).cuda()
        dy = torch.from_numpy(np.ascontiguousarray(y[perm].astype(np.int32))).cuda()
        losses.append(float(mpspmv_mlp_train(dp, C, dXp, dy, n, batch, 1, lr)[0]))
    mpspmv_mlp_fold(dp, C, mu, sd)
    return dp.cpu().numpy(), np.array(losses), (mu.cpu().numpy(), sd.cpu().numpy())


def predict(params, X, C=NCLASS):
    import torch
    dp = torch.from_numpy(np.ascontiguousarray(params)).cuda()
    lg = torch.empty((len(X), C), dtype=torch.float32, device="cuda")
    mpspmv_mlp_forward(dp, C, torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda(), len(X), lg)
    return lg.argmax(dim=1).cpu().numpy()


def batched_ladder(sys_list, start, rtol, maxit_factor=2):
    """Batched precision ladder: every system whose start level (array) is
    at most L and that is not yet solved takes part in the batched CG at
    level L, from x0 = 0; a system that falls short moves up a level.
    Returns (solved mask, total CG iterations, level that solved each system
    or 0)."""
    done = np.zeros(len(sys_list), dtype=bool)
    final = np.zeros(len(sys_list), dtype=np.int32)
    iters = 0
    maxit = maxit_factor * max(s.n for s in sys_list)
    for L in (1, 2, 3, 4):
        idx = [i for i in range(len(sys_list)) if not done[i] and start[i] <= L]
        if not idx:
            continue
        ok, it, _ = solve_level_batched([sys_list[i] for i in idx], L, rtol, maxit)
        for j, i in enumerate(idx):
            iters += int(min(it[j], maxit_factor * sys_list[i].n))
            if ok[j] and it[j] <= maxit_factor * sys_list[i].n:
                done[i] = True
                final[i] = L
    return done, iters, final


def evaluate(sys_list, params, rtol, maxit_factor=2, C=NCLASS, starts=(1, 2, 3, 4), per_system=True):
    """Time to the target on held-out systems, every strategy from x0 = 0
    and timed end to end on the host clock (device synchronised):
      plain ladder from a fixed level (one system after another,
      mpspmv_ladder_solve; start 1 is the plain binary64 -> DD -> TD -> QD
      ladder), the selector-guided ladder (mpspmv_solve_auto), and batched
      forms of both (fixed start, and the selector's level per system with
      features and inference inside the timing).  Returns a dict of totals:
      seconds, systems solved, CG iterations summed over levels, escalations
      (selector: the ladder moved above the chosen level)."""
    import torch
    dp = torch.from_numpy(np.ascontiguousarray(params)).cuda()
    res = {"n": len(sys_list), "ladder": {}, "batched_ladder": {}}
    if per_system:
        for L0 in starts:
            tot = {"s": 0.0, "solved": 0, "iters": 0}
            for s in sys_list:
                x = torch.zeros((4, s.n), dtype=torch.float64, device="cuda")
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st, fl, its, _ = mpspmv_ladder_solve(s.handles, L0, s.b, x, rtol, 0.0, maxit_factor * s.n)
                torch.cuda.synchronize()
                tot["s"] += time.perf_counter() - t0
                tot["solved"] += int(st == MPSPMV_OK)
                tot["iters"] += int(sum(its))
            res["ladder"][L0] = tot
        tot = {"s": 0.0, "solved": 0, "iters": 0, "escalated": 0, "chosen": [], "final": []}
        for s in sys_list:
            x = torch.zeros((4, s.n), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st2, ch, fl2, its2, _ = mpspmv_solve_auto(s.handles, dp, C, s.b, x, rtol, 0.0, maxit_factor * s.n)
            torch.cuda.synchronize()
            tot["s"] += time.perf_counter() - t0
            tot["solved"] += int(st2 == MPSPMV_OK)
            tot["iters"] += int(sum(its2))
            tot["escalated"] += int(fl2 > ch)
            tot["chosen"].append(ch)
            tot["final"].append(fl2)
        res["selector"] = tot
    for L0 in starts:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        done, iters, _ = batched_ladder(sys_list, np.full(len(sys_list), L0), rtol, maxit_factor)
        torch.cuda.synchronize()
        res["batched_ladder"][L0] = {"s": time.perf_counter() - t0, "solved": int(done.sum()), "iters": iters}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X = features(sys_list)
    level = np.minimum(predict(params, X, C) + 1, 4)
    done, iters, final = batched_ladder(sys_list, level, rtol, maxit_factor)
    torch.cuda.synchronize()
    res["batched_selector"] = {"s": time.perf_counter() - t0, "solved": int(done.sum()), "iters": iters,
                               "escalated": int(((final > level) & done).sum()),
                               "chosen_hist": {int(v): int((level == v).sum()) for v in np.unique(level)}}
    return res
