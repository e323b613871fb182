"""Benchmark: multiple-precision CSR SpMV throughput (Gnnz/s) on GB300, plus
complex SpMV, BiCGSTAB and the CG time-to-1e-30 comparison of the precision
ladder with the learned selector.

Timed step (``value``): y = A x in DD, TD and QD on two real matrices shaped
like the paper's SpMV workloads (arXiv 2412.17510, Section 4.1, SuiteSparse
stand-ins), repeated ``--repeat`` times per step:
  (a) 3D 27-point stencil on a 128^3 grid, non-periodic (n = 2,097,152,
      nnz = 55,742,968), off-diagonals N(0,1), diagonal = row |sum| + 1;
  (b) power-law rows, n = 1,000,000, lengths Zipf(1.5) clipped to [1, 20000]
      (nnz ~ 2.16e8), uniform distinct columns, N(0,1) values;
binary64 matrix values (P-mode results: the lower components are zero), x
with every component random, seed 0.  value = (entries multiplied in the
step) / (device time of the step).  Inputs are resident in HBM and far
larger than L2; the L2 cache is also flushed (a 512 MiB write) between
timed steps, outside the timed events.

Also in the default line (rank 0): ``complex`` (complex band SpMV, DD/QD,
both arithmetics, and BiCGSTAB to 1e-28), ``full_limb_A`` (the exact
arithmetic on matrices whose values have L random components), and
``cg_time_to_1e-30`` (plain precision ladder from every start level against
the selector-guided ladder, per system and batched, on held-out systems).

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
N > 1 runs under torch.distributed.run; every rank multiplies its own copy of
the workload (independent problems, no collective on the data path), the time
is the maximum over ranks and value counts the entries of all ranks.
"""
import argparse
import hashlib
import json
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "MP-SpMV Gnnz/s (DD/TD/QD, real/cplx), % roofline; CG time-to-1e-30 vs plain"
UNIT = "Gnnz/s"
PRECS = (2, 3, 4)
PNAME = {1: "D", 2: "DD", 3: "TD", 4: "QD"}
# binary64 operations per stored entry: one MP multiply + one MP add
# (Algorithms 2 + 1 for DD; QD sloppy mul + add; TD = QD with zero fourth
# components plus one folding addition each) -- the oracle's operation counts.
OPS_PER_ENTRY = {2: 9 + 11, 3: 124 + 88, 4: 123 + 87}
# exact accumulation (MPSPMV_EXACT_ACC): binary64 instructions per stored entry
# -- P mode (MP values): only the FMA chain of the rounded products, the
# exact products are formed on the integer pipe; binary64 data (one stored
# value plane): none, single-vector products take the wide-x form (x turned
# once per product into a W-word fixed-point number per column, one integer
# product a X per entry):
OPS_PER_ENTRY_EXACT = {2: 2, 3: 3, 4: 4}
OPS_PER_ENTRY_EXACT_D = {2: 0, 3: 0, 4: 0}
# ... and shared-memory digit updates per stored entry, the accumulation's
# own bound: in P mode an exact 106-bit product adds five 32-bit chunks, a
# rounded binary64 term three (1/3/6 exact products for DD/TD/QD); in the
# wide-x form the product a X adds W + 2 chunks (W = 4/5/7 words); each
# update an 8-byte load and an 8-byte store.
UPD_PER_ENTRY_EXACT = {2: 8, 3: 18, 4: 33}
UPD_PER_ENTRY_EXACT_D = {2: 6, 3: 7, 4: 9}
SMEM_BYTES_PER_CLK = 128  # shared-memory bandwidth per SM per clock (32 banks x 4 B)
UPD_BYTES = 16
L2_FLUSH_BYTES = 512 << 20
# oracle sample: entries per slice (about 50 ms of one Grace core each)
SLICE_ENTRIES = {2: 3000000, 3: 400000, 4: 400000}


def replica_value(local_ms, units_per_rank, world, dist=None, device="cpu"):
    """Weak scaling over independent replicas (every rank runs the same
    workload, no collective on the data path): the job's time is the slowest
    rank's, its throughput the units of all ranks over that time, in G/s.
    Returns (ms, value)."""
    ms = float(local_ms)
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, units_per_rank * world / (ms * 1e-3) / 1e9


def smem_peak_updates(clock_mhz):
    """Shared-memory digit updates per second the GPU can sustain: SMs x clock x
    bandwidth per clock / bytes per update."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return sms * clock_mhz * 1e6 * SMEM_BYTES_PER_CLK / UPD_BYTES


def make_matrices(small=False):
    if small:
        return {"stencil27_32^3": workloads.stencil_27pt(32), "powerlaw_1e5": workloads.power_law(100000)}
    return {"stencil27_128^3": workloads.stencil_27pt(128), "powerlaw_1e6_zipf1.5": workloads.power_law(1000000)}


def algorithmic_bytes(nnz, nrows, ncols, L, value_planes=None):
    """Compulsory HBM traffic of one SpMV: per entry a 4-byte column index and
    its stored value components (L, or 1 when only leading components are
    stored); per row its start offset and the L result components; x read
    once (L components per column)."""
    vp = L if value_planes is None else value_planes
    return nnz * (4 + 8 * vp) + nrows * (8 + 8 * L) + ncols * 8 * L


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def kernel_sha():
    h = hashlib.sha256()
    for f in ("spmv.cu", "mp_arith.cuh", "run_body.cuh", "fixacc.cuh", "exact_prod.cuh", "wide.cuh", "api.cu"):
        with open(os.path.join(ROOT, "paper_2412_17510_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def stored_traffic(variant):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source."""
    p = os.path.join(ROOT, "profiles", "spmv_dram_traffic.json")
    try:
        d = json.load(open(p))
    except Exception:
        return None
    if d.get("kernel_sha") != kernel_sha():
        return None
    v = d.get("variants", {}).get(variant)
    return v.get("bytes_per_launch") if v else None


# ---------------------------------------------------------------------------
# CPU oracle leg: the same sampler in both arms (bounded sample, host cores)
# ---------------------------------------------------------------------------
def _oracle_slice(args):
    """Worker: the oracle's SpMV of rows a..b-1 of one matrix at L
    components (its values promoted), x of the whole matrix; the matrix and
    x come from .npy files mapped read-only.  Returns (entries, seconds of
    the product alone)."""
    d, mname, L, a, b = args
    import oracle as orc
    ip = np.load(os.path.join(d, mname + ".indptr.npy"), mmap_mode="r")
    lo, hi = int(ip[a]), int(ip[b])
    indptr = np.array(ip[a:b + 1], dtype=np.int64) - lo
    ind = np.array(np.load(os.path.join(d, mname + ".indices.npy"), mmap_mode="r")[lo:hi], dtype=np.int32)
    vals = np.zeros((L, hi - lo))
    vals[0] = np.load(os.path.join(d, mname + ".vals.npy"), mmap_mode="r")[lo:hi]
    x = np.array(np.load(os.path.join(d, "%s.x%d.npy" % (mname, L)), mmap_mode="r"))
    A = orc.CSR(b - a, x.shape[1], indptr, ind, vals, L, False)
    t = time.perf_counter()
    orc.spmv(A, x)
    return hi - lo, time.perf_counter() - t


class OracleSampler:
    """The CPU oracle's SpMV timed on a bounded sample of the step's
    matrices, one method for both bench arms.  Per (matrix, precision):
    ``ncores`` slices of consecutive rows holding SLICE_ENTRIES[L] entries
    each (about 50 ms of one core), starting at evenly spaced rows so the
    sample spans the whole matrix (the power-law matrix's long rows sit
    wherever the draw put them).  The matrices reach the worker processes as
    .npy files mapped read-only from a temporary directory (no large
    pickles, no shared-memory segment)."""

    def __init__(self, mats, xs, ncores, slice_entries=None):
        slice_entries = slice_entries or SLICE_ENTRIES
        self.dir = tempfile.mkdtemp(prefix="mpspmv_oracle_")
        self.ncores = ncores
        self.tasks = {}
        for mname, coo in mats.items():
            ip = np.zeros(coo.nrows + 1, dtype=np.int64)
            np.cumsum(np.bincount(coo.row, minlength=coo.nrows), out=ip[1:])
            np.save(os.path.join(self.dir, mname + ".indptr.npy"), ip)
            np.save(os.path.join(self.dir, mname + ".indices.npy"), coo.col.astype(np.int32))
            np.save(os.path.join(self.dir, mname + ".vals.npy"), coo.val[0])
            starts = [int(i * coo.nrows / ncores) for i in range(ncores)] + [coo.nrows]
            for L in PRECS:
                np.save(os.path.join(self.dir, "%s.x%d.npy" % (mname, L)), xs[mname][L])
                tl = []
                for i in range(ncores):
                    a = starts[i]
                    b = int(np.searchsorted(ip, ip[a] + slice_entries[L], side="left"))
                    b = max(a + 1, min(b, starts[i + 1]))
                    if a < coo.nrows:
                        tl.append((self.dir, mname, L, a, b))
                self.tasks[(mname, L)] = tl
        self.desc = ("per (matrix, precision) %d slices of consecutive rows, each about %s entries (DD/TD/QD) and "
                     "starting at evenly spaced rows, run at once on %d spawned processes (the slowest slice "
                     "times the sample); rates combined with the GPU step's mix of entries"
                     % (ncores, [SLICE_ENTRIES[L] for L in PRECS], ncores))

    def rates(self, pool):
        """All-core entries/s per (matrix, L): the sample's entries over its
        slowest slice (the slices run concurrently)."""
        out = {}
        for key, tl in self.tasks.items():
            res = pool.map(_oracle_slice, tl, chunksize=1)
            out[key] = sum(r[0] for r in res) / max(r[1] for r in res)
        return out

    def single_rates(self, pool):
        """One-core entries/s per (matrix, L): the middle slice run alone."""
        out = {}
        for key, tl in self.tasks.items():
            e, t = pool.apply(_oracle_slice, (tl[len(tl) // 2],))
            out[key] = e / t
        return out

    def close(self):
        shutil.rmtree(self.dir, ignore_errors=True)


def cpu_rate_for_step(rates, nnz_of):
    """Aggregate oracle rate over a step with the GPU step's mix of variants."""
    tot_nnz = sum(nnz_of[v] for v in rates)
    tot_t = sum(nnz_of[v] / rates[v] for v in rates)
    return tot_nnz / tot_t


def sample_rows(coo, n=96, seed=17):
    """Rows whose results the parity report checks: n random rows plus the
    first, the last and the longest (so the bound's m is the matrix's own)."""
    counts = np.bincount(coo.row, minlength=coo.nrows)
    rng = np.random.default_rng(seed)
    pick = rng.choice(coo.nrows, min(n, coo.nrows), replace=False)
    return np.unique(np.concatenate([pick, [0, coo.nrows - 1, int(np.argmax(counts))]])).astype(np.int64)


def parity_report(mats, xs_host, rows_of, ysamp, chunk_of, sell_of=None):
    """Error of the step's results on sampled rows (part of the oracle leg):
    per arithmetic and variant, max |y - y_exact| / (8 m u (|A||x|)) over the
    sampled components against the exact value; whether the paper-order rows
    that one run holds equal the oracle's row sums bit for bit; and whether
    the exact-arithmetic rows that one thread sums (every row of a
    row-per-thread copy, sell_of[key] true, else the rows inside one run)
    equal the exact model of that arithmetic bit for bit, where their terms
    fit its window.  ysamp[(arith, matrix, L)] holds the sampled columns of y
    (L x rows); the matrices hold binary64 values."""
    import oracle
    from oracle import exact
    from oracle import exact_model
    out = {"rows_per_matrix": {m: int(len(r)) for m, r in rows_of.items()}, "max_bound_ratio": {},
           "paper_one_run_rows_bit_identical": None, "paper_one_run_rows": 0,
           "exact_model_rows_bit_identical": None, "exact_model_rows": 0}
    bit_ok = True
    model_ok = True
    for mname, coo in mats.items():
        rows = rows_of[mname]
        counts = np.bincount(coo.row, minlength=coo.nrows)
        ip = np.zeros(coo.nrows + 1, dtype=np.int64)
        np.cumsum(counts, out=ip[1:])
        mask = np.isin(coo.row, rows, kind="table")
        sub = workloads.COO(len(rows), coo.ncols, np.searchsorted(rows, coo.row[mask]), coo.col[mask],
                            coo.val[:, mask])
        for L in PRECS:
            keys = [k for k in ysamp if k[1] == mname and k[2] == L]
            if not keys:
                continue
            A = oracle.coo_to_csr(sub.nrows, sub.ncols, sub.row, sub.col, sub.promoted(L), L)
            x = xs_host[mname][L]
            ref = None
            for key in keys:
                y = ysamp[key]
                out["max_bound_ratio"].setdefault(key[0], {})["%s/%s" % (mname, PNAME[L])] = \
                    exact.bound_ratio(y, A, x)
                K = chunk_of[key]
                one = (ip[rows] // K == (ip[rows + 1] - 1) // K) & (ip[rows + 1] > ip[rows])
                if key[0] == "paper":
                    ref = oracle.spmv(A, x) if ref is None else ref
                    bit_ok = bit_ok and bool(np.array_equal(y[:, one], ref[:, one]))
                    out["paper_one_run_rows"] += int(one.sum())
                elif key[0] == "exact":
                    # binary64 values: single-vector products take the wide-x
                    # form, which the model follows step by step (every row)
                    whole = np.ones(len(rows), dtype=bool) if (sell_of or {}).get(key) else one
                    for i in np.nonzero(whole)[0]:
                        want, _ = exact_model.row_model_wide(L, A, x, int(i))
                        model_ok = model_ok and bool(np.array_equal(y[:, i], want))
                        out["exact_model_rows"] += 1
    if any(k[0] == "paper" for k in ysamp):
        out["paper_one_run_rows_bit_identical"] = bit_ok
    if out["exact_model_rows"]:
        out["exact_model_rows_bit_identical"] = model_ok
    return out


# ---------------------------------------------------------------------------
# reference arm: the oracle timed as it stands
# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import multiprocessing as mp
    ncores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    mats = make_matrices(args.small)
    xs = {m: {L: workloads.full_limb_vector(c.ncols, L, seed=0) for L in PRECS} for m, c in mats.items()}
    nnz_of = {(m, L): c.nnz for m, c in mats.items() for L in PRECS}
    sampler = OracleSampler(mats, xs, ncores)
    step_rates = []
    try:
        with ctx.Pool(ncores) as pool:
            for it in range(args.warmup + args.steps):
                rates = sampler.rates(pool)
                if it >= args.warmup:
                    step_rates.append(cpu_rate_for_step(rates, nnz_of))
    finally:
        sampler.close()
    total_nnz = sum(nnz_of.values())
    ms = [total_nnz / r * 1e3 for r in step_rates]
    value = total_nnz / (sum(ms) / len(ms) * 1e-3) / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sum(ms) / len(ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_block(mats, 1),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncores, "kind": "oracle",
                         "sample": sampler.desc + "; time scaled to one pass of the step's six products"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def config_block(mats, repeat):
    return {"workload": "real CSR SpMV y = A x in DD/TD/QD on binary64 matrix values (P-mode results: lower "
                        "components zero; exact handles keep the one non-zero value plane and use the "
                        "MP x binary64 product forms, bit-identical to full P storage): " + ", ".join(
                            "%s (n=%d, nnz=%d)" % (k, v.nrows, v.nnz) for k, v in mats.items()),
            "repeat_per_step": repeat,
            "x": "every component random, seed 0",
            "l2": "inputs larger than L2; also flushed between timed steps (512 MiB write)",
            "precisions": [PNAME[L] for L in PRECS]}


def _time_events(fn, reps, stream):
    import torch
    evs = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in evs]))


def suite_complex(mps, fp64_fma, hbm, stream, small):
    """Complex-symmetric band, half-bandwidth 48, 30% fill (n = 500,000):
    complex DD / QD SpMV, and BiCGSTAB on A + (50+10i) I to 1e-28."""
    import torch
    n = 50000 if small else 500000
    coo = workloads.complex_sym_banded(n, 48, 0.3, seed=0)
    out = {"workload": "complex-symmetric band n=%d hbw=48 fill 0.3 (nnz=%d complex)" % (n, coo.nnz)}
    for L in (2, 4):
        for sfx, fl in (("", 0), ("_exact", 16)):
            h = mps.mpspmv_create_csr(n, n, coo.row, coo.col, coo.val, L, mps.MPSPMV_COMPLEX | fl, val_limbs=1)
            vp = mps.mpspmv_get_info(h)["value_planes"]
            x = torch.from_numpy(workloads.full_limb_vector(n, L, seed=0, cplx=True)).cuda()
            y = torch.empty_like(x)
            for _ in range(3):
                mps.mpspmv_spmv(h, x, y, stream)
            ms = _time_events(lambda: mps.mpspmv_spmv(h, x, y, stream), 10, stream)
            if fl:  # four real products per complex entry
                per = OPS_PER_ENTRY_EXACT_D[L] if vp == 2 else OPS_PER_ENTRY_EXACT[L]
                upd = UPD_PER_ENTRY_EXACT_D[L] if vp == 2 else UPD_PER_ENTRY_EXACT[L]
            else:
                per, upd = OPS_PER_ENTRY[L], 0
            ops = coo.nnz * 4 * per
            byts = coo.nnz * (4 + 8 * vp) + n * (8 + 16 * L) + n * 16 * L
            troof = max(ops / fp64_fma, byts / (hbm * 1e9), coo.nnz * 4 * upd / smem_peak_updates(2070.0))
            out["spmv_%s%s" % (PNAME[L], sfx)] = {"ms": ms, "gnnz_s": coo.nnz / ms / 1e6,
                                                  "roofline_frac": troof / (ms * 1e-3)}
            mps.mpspmv_destroy(h)
    shifted = workloads.complex_sym_banded(n, 48, 0.3, seed=0, shift=50 + 10j)
    for L in (2, 4):
        for sfx, fl in (("", 0), ("_exact", 16)):
            h = mps.mpspmv_create_csr(n, n, shifted.row, shifted.col, shifted.val, L, mps.MPSPMV_COMPLEX | fl,
                                      val_limbs=1)
            xt = torch.from_numpy(workloads.full_limb_vector(n, L, seed=1, cplx=True)).cuda()
            b = torch.empty_like(xt)
            mps.mpspmv_spmv(h, xt, b, stream)
            x = torch.zeros_like(b)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, it, rr = mps.mpspmv_bicgstab(h, b, x, 1e-28, 0.0, 5000, stream)
            torch.cuda.synchronize()
            out["bicgstab_%s%s" % (PNAME[L], sfx)] = {"status": st, "iters": it, "relres": rr,
                                                      "s": time.perf_counter() - t0}
            mps.mpspmv_destroy(h)
    return out


def suite_cg(mps, stream, small, only=None, its=200):
    """CG on the SPD 7-point diffusion matrix on a 128^3 grid (kappa
    log-uniform in [0.1, 10]), a fixed number of iterations (rtol = 0; 200 by
    default), paper-order
    and exact-accumulation handles: ms per iteration, and the SpMV's ms for
    comparison (the rest is the vector kernels and the scalar steps)."""
    import torch
    N = 48 if small else 128
    coo = workloads.diffusion_7pt(N, N, N, kappa_range=(0.1, 10.0), seed=0)
    n = coo.nrows
    out = {"workload": "7-point diffusion %d^3 (n=%d, nnz=%d), %d CG iterations" % (N, n, coo.nnz, its)}
    for L in (2, 3, 4):
        for arith, fl in (("paper", 0), ("exact", 16)):
            if only and only != "%s/%s" % (PNAME[L], arith):
                continue
            h = mps.mpspmv_create_csr(n, n, coo.row, coo.col, coo.val, L, fl, val_limbs=1)
            b = torch.from_numpy(workloads.full_limb_vector(n, L, seed=1)).cuda()
            x = torch.zeros_like(b)
            y = torch.empty_like(b)
            mps.mpspmv_cg(h, b, x, 0.0, 0.0, 8, stream)  # workspace, graph warm-up
            for _ in range(3):
                mps.mpspmv_spmv(h, b, y, stream)
            spmv_ms = _time_events(lambda: mps.mpspmv_spmv(h, b, y, stream), 10, stream)
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, it, rr = mps.mpspmv_cg(h, b, x, 0.0, 0.0, its, stream)
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t0) * 1e3 / max(it, 1)
            out["cg_%s_%s" % (PNAME[L], arith)] = {"ms_per_iter": ms, "spmv_ms": spmv_ms, "iters": it,
                                                   "relres": rr, "status": st}
            mps.mpspmv_destroy(h)
            del b, x, y
    return out


def suite_product(mps, stream, small):
    """The product-type methods of Section 4.2 (BiCG, CGS, BiCGSTAB, GPBiCG)
    on a nonsymmetric band matrix: 2D convection-diffusion 300 x 300 (c = 0.5,
    n = 90,000), b = A x_true, x0 = 0, DD to 1e-25 and QD to 1e-50, paper-order
    and exact arithmetic: iterations, seconds, true relative residual."""
    import torch
    N = 100 if small else 300
    coo = workloads.convection_diffusion_2d(N, N, 0.5)
    n = coo.nrows
    out = {"workload": "convection-diffusion 2D %dx%d (n=%d, nnz=%d)" % (N, N, n, coo.nnz)}
    methods = (("bicg", mps.mpspmv_bicg), ("cgs", mps.mpspmv_cgs), ("bicgstab", mps.mpspmv_bicgstab),
               ("gpbicg", mps.mpspmv_gpbicg))
    for L, rtol in ((2, 1e-25), (4, 1e-50)):
        for arith, fl in (("paper", 0), ("exact", 16)):
            h = mps.mpspmv_create_csr(n, n, coo.row, coo.col, coo.val, L, fl | mps.MPSPMV_TRANSPOSE, val_limbs=1)
            xt = torch.from_numpy(workloads.full_limb_vector(n, L, seed=2)).cuda()
            b = torch.empty_like(xt)
            mps.mpspmv_spmv(h, xt, b, stream)
            for name, fn in methods:
                x = torch.zeros_like(b)
                fn(h, b, x, rtol, 0.0, 8, stream)  # workspace and graph warm-up
                x.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st, it, rr = fn(h, b, x, rtol, 0.0, 20000, stream)
                torch.cuda.synchronize()
                out["%s_%s_%s" % (name, PNAME[L], arith)] = {"status": st, "iters": it, "relres": rr,
                                                             "s": time.perf_counter() - t0}
            mps.mpspmv_destroy(h)
    return out


def suite_batched(mps, stream, small):
    """512 SPD 7-point diffusion matrices (kappa log-uniform in [1e-3, 1e3]),
    n log-uniform in [1e3, 2e5], k ~ U{1..32}: one graph launch of the
    batched SpMM in DD and QD (autotuned); batched CG to 1e-25 on a reduced
    set (32 matrices, n in [1e3, 1e4], k ~ U{1..8}) to keep the run short."""
    import torch
    count = 64 if small else 512
    specs = workloads.batch_specs(count, n_range=(1000, 200000), k_range=(1, 32), seed=0)
    coos = [workloads.diffusion_7pt(nx, ny, nz, seed=sd) for nx, ny, nz, k, sd in specs]
    ks = [k for *_, k, sd in specs]
    out = {"workload": "%d diffusion matrices, sum nnz %d, sum k*nnz %d" % (
        count, sum(c.nnz for c in coos), sum(c.nnz * k for c, k in zip(coos, ks)))}
    for L, fl in ((2, 0), (2, 16), (4, 0), (4, 16)):
        hs = [mps.mpspmv_create_csr(c.nrows, c.ncols, c.row, c.col, c.val, L, fl, val_limbs=1) for c in coos]
        t0 = time.perf_counter()
        b = mps.mpspmv_batch_create(hs, ks, mps.MPSPMV_BATCH_AUTOTUNE, stream)
        tune_s = time.perf_counter() - t0
        Xs = [torch.from_numpy(np.ascontiguousarray(np.broadcast_to(
            workloads.full_limb_vector(c.ncols, L, seed=i)[:, :, None], (L, c.ncols, k)))).cuda()
            for i, (c, k) in enumerate(zip(coos, ks))]
        Ys = [torch.empty((L, c.nrows, k), dtype=torch.float64, device="cuda") for c, k in zip(coos, ks)]
        for _ in range(3):
            mps.mpspmv_batch_spmm(b, Xs, Ys, stream=stream)
        ms = _time_events(lambda: mps.mpspmv_batch_spmm(b, Xs, Ys, stream=stream), 10, stream)
        work = sum(c.nnz * k for c, k in zip(coos, ks))
        K, w = mps.mpspmv_batch_get_plan(b, count)
        out["spmm_%s%s" % (PNAME[L], "_exact" if fl else "")] = {"ms_per_launch": ms, "gnnz_rhs_s": work / ms / 1e6, "autotune_s": tune_s,
                                     "K_hist": {int(v): int((K == v).sum()) for v in np.unique(K)},
                                     "w_hist": {int(v): int((w == v).sum()) for v in np.unique(w)}}
        mps.mpspmv_batch_destroy(b)
        for h in hs:
            mps.mpspmv_destroy(h)
        del Xs, Ys
    # batched CG on the reduced set
    cspecs = workloads.batch_specs(8 if small else 32, n_range=(1000, 10000), k_range=(1, 8), seed=1)
    ccoos = [workloads.diffusion_7pt(nx, ny, nz, seed=sd) for nx, ny, nz, k, sd in cspecs]
    cks = [k for *_, k, sd in cspecs]
    for L, arith in ((2, "paper"), (2, "exact"), (4, "paper"), (4, "exact")):
        fl = 16 if arith == "exact" else 0
        hs = [mps.mpspmv_create_csr(c.nrows, c.ncols, c.row, c.col, c.val, L, fl, val_limbs=1) for c in ccoos]
        b = mps.mpspmv_batch_create(hs, cks, 0, stream)
        Bs = [torch.from_numpy(np.ascontiguousarray(np.stack(
            [workloads.full_limb_vector(c.ncols, L, seed=100 + i * 40 + j) for j in range(k)], axis=-1))).cuda()
            for i, (c, k) in enumerate(zip(ccoos, cks))]
        Xs = [torch.zeros_like(B) for B in Bs]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, it, rr, ss = mps.mpspmv_batch_cg(b, Bs, Xs, sum(cks), 1e-25, 0.0, 100000, stream)
        torch.cuda.synchronize()
        out["cg_%s%s" % (PNAME[L], "_exact" if fl else "")] = {"systems": int(sum(cks)), "s": time.perf_counter() - t0, "status": st,
                                   "converged": int((ss == 0).sum()), "iters_max": int(it.max()),
                                   "iters_mean": float(it.mean()), "relres_max": float(rr.max())}
        mps.mpspmv_batch_destroy(b)
        for h in hs:
            mps.mpspmv_destroy(h)
    return out


def part_full_limb(mps, fp64_fma, hbm, stream, small, reps=10):
    """Exact arithmetic on matrices whose values have L random components
    (val_limbs = L, so every value plane is stored and the products take the
    MP x MP forms): the QD products of the step's two matrices, Gnnz/s and
    the three roofline fractions (the matrices are far larger than L2)."""
    import torch
    out = {}
    L = 4
    for mname, coo in make_matrices(small).items():
        vals = workloads.full_limb_values(coo, L, seed=7)
        h = mps.mpspmv_create_csr(coo.nrows, coo.ncols, coo.row, coo.col, vals, L, mps.MPSPMV_EXACT_ACC,
                                  val_limbs=L)
        del vals
        info = mps.mpspmv_get_info(h)
        x = torch.from_numpy(workloads.full_limb_vector(coo.ncols, L, seed=0)).cuda()
        y = torch.empty((L, coo.nrows), dtype=torch.float64, device="cuda")
        for _ in range(3):
            mps.mpspmv_spmv(h, x, y, stream)
        ms = _time_events(lambda: mps.mpspmv_spmv(h, x, y, stream), reps, stream)
        t = ms * 1e-3
        nnz = info["nnz"]
        tr = {"hbm": algorithmic_bytes(nnz, coo.nrows, coo.ncols, L, info["value_planes"]) / (hbm * 1e9),
              "fp64": nnz * OPS_PER_ENTRY_EXACT[L] / fp64_fma,
              "smem": nnz * UPD_PER_ENTRY_EXACT[L] / smem_peak_updates(2070.0)}
        out["%s/QD" % mname] = {"ms": ms, "gnnz_s": nnz / t / 1e9, "value_planes": info["value_planes"],
                                "roofline_frac": max(tr.values()) / t, "bound": max(tr, key=tr.get),
                                "fracs": {k: v / t for k, v in tr.items()}}
        mps.mpspmv_destroy(h)
        del x, y
    return out


def roof_terms(arith, L, nnz, nrows, ncols, value_planes, fp64_fma, hbm):
    """Roofline times (s) of one real product: HBM bytes, binary64 pipe,
    shared-memory digit updates (exact arithmetic only)."""
    if arith == "exact":
        one = value_planes == 1
        ops = (OPS_PER_ENTRY_EXACT_D if one else OPS_PER_ENTRY_EXACT)[L]
        upd = (UPD_PER_ENTRY_EXACT_D if one else UPD_PER_ENTRY_EXACT)[L]
    else:
        ops, upd = OPS_PER_ENTRY[L], 0
    return {"hbm": algorithmic_bytes(nnz, nrows, ncols, L, value_planes) / (hbm * 1e9),
            "fp64": nnz * ops / fp64_fma, "smem": nnz * upd / smem_peak_updates(2070.0)}


def part_powerlaw16(mps, fp64_fma, hbm, stream, small, reps=10):
    """The power-law matrix with the mean row length the configuration
    states (16): Zipf exponent 1.847 instead of 1.5, clipped to [1, 20000],
    n = 1e6 (1e5 with --small), DD/TD/QD in both arithmetics."""
    import torch
    n = 100000 if small else 1000000
    coo = workloads.power_law(n, s=1.847)
    out = {"workload": "power-law n=%d, Zipf(1.847) clipped to [1, 20000], nnz=%d (mean %.1f per row)"
                       % (n, coo.nnz, coo.nnz / n)}
    for L in PRECS:
        x = torch.from_numpy(workloads.full_limb_vector(n, L, seed=0)).cuda()
        y = torch.empty((L, n), dtype=torch.float64, device="cuda")
        for arith, fl in (("exact", mps.MPSPMV_EXACT_ACC), ("paper", 0)):
            h = mps.mpspmv_create_csr(n, n, coo.row, coo.col, coo.val, L, fl, val_limbs=1)
            info = mps.mpspmv_get_info(h)
            for _ in range(3):
                mps.mpspmv_spmv(h, x, y, stream)
            ms = _time_events(lambda: mps.mpspmv_spmv(h, x, y, stream), reps, stream)
            t = ms * 1e-3
            tr = roof_terms(arith, L, info["nnz"], n, n, info["value_planes"], fp64_fma, hbm)
            out["%s/%s" % (PNAME[L], arith)] = {"ms": ms, "gnnz_s": info["nnz"] / t / 1e9,
                                                "roofline_frac": max(tr.values()) / t, "bound": max(tr, key=tr.get),
                                                "fracs": {k: v / t for k, v in tr.items()}}
            mps.mpspmv_destroy(h)
        del x, y
    return out


def _selector_systems(sel, count, n_range, seed, flags):
    rng = np.random.default_rng(seed)
    systems = []
    for i in range(count):
        n = int(round(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1])))))
        coo, b = workloads.selector_system(n, float(rng.uniform(8, 40)), seed=1000 * (seed + 1) + i)
        systems.append(sel.System(coo, b, flags))
    return systems


def _selector_study(mps, ntrain, ntest, n_range, flags, per_system, seed=0, epochs=300):
    """Selector study on SPD systems A = D (L L^T + I) D (cond 10^U[8, 40]):
    labels from the method's own batched CG solves (cheapest of binary64 /
    DD / TD / QD whose CG reaches 1e-30 within 30 n iterations), training by
    the float32 kernels, then the held-out systems solved from x0 = 0 by the
    plain ladder from every start level and by the selector (per system and
    batched), every strategy timed end to end."""
    from paper_2412_17510_gb300 import selector as sel
    systems = _selector_systems(sel, ntrain + ntest, n_range, seed, flags)
    try:
        t0 = time.perf_counter()
        X = sel.features(systems)
        y = sel.labels(systems, 1e-30, maxit_factor=30)
        label_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        params, losses, _ = sel.train(X[:ntrain], y[:ntrain], epochs=epochs, batch=32, lr=0.05)
        train_s = time.perf_counter() - t0
        pred = sel.predict(params, X[ntrain:])
        ev = sel.evaluate(systems[ntrain:], params, 1e-30, maxit_factor=30, per_system=per_system)
    finally:
        for s in systems:
            s.free()
    out = {"systems": ntrain + ntest, "train": ntrain, "test": ntest, "n_range": list(n_range),
           "label_hist": {PNAME.get(c + 1, "none"): int((y == c).sum()) for c in range(5)},
           "label_s": label_s, "train_s": train_s, "loss_first_last": [float(losses[0]), float(losses[-1])],
           "test_accuracy": float((pred == y[ntrain:]).mean()),
           "batched": {"ladder_from_%s" % PNAME[L0]: v for L0, v in ev["batched_ladder"].items()}}
    out["batched"]["selector"] = ev["batched_selector"]
    if per_system:
        out["per_system"] = {"ladder_from_%s" % PNAME[L0]: v for L0, v in ev["ladder"].items()}
        sel_tot = dict(ev["selector"])
        sel_tot.pop("final", None)
        sel_tot["chosen_hist"] = {PNAME[c]: sel_tot["chosen"].count(c) for c in sorted(set(sel_tot["chosen"]))}
        sel_tot.pop("chosen", None)
        out["per_system"]["selector"] = sel_tot
    return out


def part_cg_time(mps, small):
    """The metric's second half, CG time to a relative residual of 1e-30:
    the plain precision ladder (binary64 -> DD -> TD -> QD, and constant
    starts at DD, TD or QD) against the learned selector's choice, one
    system after another and batched, on held-out systems (exact-
    accumulation handles, n log-uniform in [40, 160])."""
    ntrain, ntest = (60, 12) if small else (240, 24)
    return _selector_study(mps, ntrain, ntest, (40, 160), mps.MPSPMV_EXACT_ACC, per_system=True)


def suite_selector(mps, small, flags=0):
    """Selector study with both arithmetics on 360 systems (n in [40, 160])."""
    ntrain, ntest = (60, 20) if small else (300, 60)
    return _selector_study(mps, ntrain, ntest, (40, 160), flags, per_system=True)


def suite_selector_large(mps, small):
    """The largest selector study that fits a bench run: 2,000 systems with n
    log-uniform in [60, 400] (1,600 for training, 400 held out), exact
    handles; the held-out comparison is batched only."""
    ntrain, ntest = (200, 50) if small else (1600, 400)
    return _selector_study(mps, ntrain, ntest, (60, 400), mps.MPSPMV_EXACT_ACC, per_system=False, seed=3)


def suite_selector_scale(mps, small):
    """CG iterations to 1e-30 against n on the selector's family (QD, exact
    handles, cond 1e8 and 1e16, three systems each), with a cap of 100 n:
    what rules out the configured n in [1e4, 1e5]."""
    import torch
    from paper_2412_17510_gb300 import selector as sel
    out = {}
    ns = (100, 300) if small else (100, 300, 1000, 3000)
    for n in ns:
        for lc in (8.0, 16.0):
            rows = []
            for k in range(3):
                coo, b = workloads.selector_system(n, lc, seed=5000 + 10 * n + k)
                s = sel.System(coo, b, mps.MPSPMV_EXACT_ACC)
                try:
                    x = torch.zeros((4, n), dtype=torch.float64, device="cuda")
                    b4 = torch.zeros((4, n), dtype=torch.float64, device="cuda")
                    b4[0] = s.b[0]
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    st, it, rr = mps.mpspmv_cg(s.handles[3], b4, x, 1e-30, 0.0, 100 * n)
                    torch.cuda.synchronize()
                    rows.append({"status": st, "iters": it, "iters_per_n": it / n, "relres": rr,
                                 "s": time.perf_counter() - t0, "nnz": coo.nnz})
                finally:
                    s.free()
            out["n=%d,cond=1e%d" % (n, lc)] = rows
    return out


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
DEFAULT_PARTS = "complex,full_limb,powerlaw16,cg_time"
SUITE_PARTS = "cg,product,batched,selector,selector_exact,selector_large,selector_scale"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--repeat", type=int, default=8, help="passes over the six products per timed step")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--small", action="store_true", help="reduced matrices (development)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle leg")
    ap.add_argument("--only", default=None, help="run one variant, e.g. powerlaw_1e5/QD (profiling)")
    ap.add_argument("--arith", default="both", choices=["paper", "exact", "both"],
                    help="paper: the paper's DD/TD/QD operation sequences; exact: error-free products on the "
                         "integer pipe with exact integer accumulation (MPSPMV_EXACT_ACC); both: value from "
                         "exact, the paper-order step timed too")
    ap.add_argument("--cg-only", default=None,
                    help="profiling: run only the CG workload of the suite in one variant, e.g. QD/exact, and exit")
    ap.add_argument("--cg-iters", type=int, default=200, help="CG iterations of the CG workload")
    ap.add_argument("--parts", default=DEFAULT_PARTS,
                    help="default-line parts after the timed step (comma-separated; 'none' for none)")
    ap.add_argument("--suite", nargs="?", const=SUITE_PARTS, default=None,
                    help="also measure the heavier workloads (CG, product-type methods, batched, selector "
                         "studies; adds minutes); optionally a comma-separated subset")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)

    import multiprocessing as mp
    ncores = os.cpu_count() or 1
    pool = None
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank == 0 and world == 1 and not args.no_cpu and not args.only and not args.cg_only:
        # spawn the oracle workers before the first GPU call
        pool = mp.get_context("spawn").Pool(ncores)

    import torch
    import paper_2412_17510_gb300 as mps
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    if args.cg_only:
        # profiling entry: one CG variant, no timed SpMV step
        out = suite_cg(mps, torch.cuda.current_stream(), args.small, only=args.cg_only, its=args.cg_iters)
        print(json.dumps(out))
        return

    R = max(1, args.repeat)
    mats = make_matrices(args.small)
    ariths = ["exact", "paper"] if args.arith == "both" else [args.arith]
    sets = {ar: [] for ar in ariths}
    xs_host = {}
    for mname, coo in mats.items():
        xs_host[mname] = {L: workloads.full_limb_vector(coo.ncols, L, seed=0) for L in PRECS}
        for L in PRECS:
            if args.only and args.only != "%s/%s" % (mname, PNAME[L]):
                continue
            x = torch.from_numpy(xs_host[mname][L]).cuda()
            y = torch.empty((L, coo.nrows), dtype=torch.float64, device="cuda")
            for ar in ariths:
                fl = mps.MPSPMV_EXACT_ACC if ar == "exact" else 0
                h = mps.mpspmv_create_csr(coo.nrows, coo.ncols, coo.row, coo.col, coo.val, L, fl, val_limbs=1)
                info = mps.mpspmv_get_info(h)
                sets[ar].append(dict(name="%s/%s" % (mname, PNAME[L]), m=mname, L=L, h=h, x=x, y=y, info=info,
                                     nnz=info["nnz"], nrows=coo.nrows, ncols=coo.ncols, arith=ar))
    torch.cuda.synchronize()

    fp64_fma = mps.mpspmv_probe_fp64(0)
    fp64_add = mps.mpspmv_probe_fp64(1)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step(variants, evs=None, reps=1):
        k = 0
        for _ in range(reps):
            for v in variants:
                if evs:
                    evs[k][0].record(stream)
                mps.mpspmv_spmv(v["h"], v["x"], v["y"], stream)
                if evs:
                    evs[k][1].record(stream)
                k += 1

    def timed(variants, sample_clocks, reps):
        for _ in range(args.warmup):
            flush.zero_()
            step(variants, reps=reps)
        torch.cuda.synchronize()
        sampler = ClockSampler(local) if sample_clocks else None
        if sampler:
            sampler.start()
            time.sleep(0.3)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        all_evs, step_evs = [], []
        for _ in range(args.steps):
            flush.zero_()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(reps * len(variants))]
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            step(variants, evs, reps)
            s1.record(stream)
            all_evs.append(evs)
            step_evs.append((s0, s1))
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clk = sampler.stop() if sampler else None
        per_var = np.zeros(len(variants))
        for evs in all_evs:
            t = np.array([a.elapsed_time(b) for a, b in evs]).reshape(reps, len(variants))
            per_var += t.sum(axis=0)
        step_ms = [a.elapsed_time(b) for a, b in step_evs]
        return per_var / (args.steps * reps), float(np.mean(step_ms)), clk

    primary = ariths[0]
    variants = sets[primary]
    per_var, ms, clocks = timed(variants, True, R)
    # the paper-order step is about 17x slower: one pass per timed step
    other = {ar: timed(sets[ar], False, 1) for ar in ariths[1:]}
    step_nnz = R * sum(v["nnz"] for v in variants)
    ms, value = replica_value(ms, step_nnz, world, dist, device="cuda")

    def launches_of(v):
        i = v["info"]
        if v["arith"] != "exact":
            return 1 + (i["nsplit_rows"] > i["nlong_rows"]) + (i["nlong_rows"] > 0)
        inter = 1 if v["L"] > 1 else 0  # x records (wide-x form) or interleaved copy of x
        if i["sell_slots"] > 0:
            return inter + 1            # one row per thread
        finish = 1 if v["L"] > 1 else 0  # finishing pass of the staged rows (real wide-x form)
        return inter + 1 + finish + (i["nsplit_rows"] > i["nlong_rows"]) + (i["nlong_rows"] > 0)

    launches_per_step = R * sum(launches_of(v) for v in variants)

    # end to end through the host-buffer entry points (pinned host memory):
    # every product copies its x in and its y out inside the timing; the
    # products alternate between two streams, so one product's copies
    # overlap another's kernels
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    e2e_ms = []
    h2d = d2h = 0
    hosts = []
    for v in variants:
        xh = torch.from_numpy(xs_host[v["m"]][v["L"]]).pin_memory()
        yh = torch.empty((v["L"], v["nrows"]), dtype=torch.float64).pin_memory()
        hosts.append((xh, yh))
        h2d += R * xh.numel() * 8
        d2h += R * yh.numel() * 8
    torch.cuda.synchronize()
    for it in range(max(3, min(args.steps, 10)) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(R):
            for i, (v, (xh, yh)) in enumerate(zip(variants, hosts)):
                mps.mpspmv_spmv_host_async(v["h"], xh, yh, streams[i % 2])
        for s_ in streams:
            s_.synchronize()
        t1 = time.perf_counter()
        if it > 0:
            e2e_ms.append((t1 - t0) * 1e3)
    _, e2e_value = replica_value(float(np.mean(e2e_ms)), step_nnz, world, dist, device="cuda")

    hbm = 6786.2
    hbm_src = "fallback 6786.2 GB/s (MEASURED_PEAKS.json absent)"
    try:
        hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
        hbm_src = "MEASURED_PEAKS.json hbm_gbs"
    except Exception:
        pass

    smem = smem_peak_updates(clock_mhz=2070.0)

    def per_entry(v):
        """(binary64 instructions, shared-memory digit updates) per stored entry."""
        if v["arith"] != "exact":
            return OPS_PER_ENTRY[v["L"]], 0
        one = v["info"]["value_planes"] == 1
        return ((OPS_PER_ENTRY_EXACT_D if one else OPS_PER_ENTRY_EXACT)[v["L"]],
                (UPD_PER_ENTRY_EXACT_D if one else UPD_PER_ENTRY_EXACT)[v["L"]])

    def bytes_of(v):
        return algorithmic_bytes(v["nnz"], v["nrows"], v["ncols"], v["L"], v["info"]["value_planes"])

    def times_of(v):
        """Roofline times (s) of one product: HBM bytes, binary64 pipe, digit updates."""
        o, u = per_entry(v)
        return {"hbm": bytes_of(v) / (hbm * 1e9), "fp64": v["nnz"] * o / fp64_fma, "smem": v["nnz"] * u / smem}

    def breakdown_of(vs, pv):
        out = {}
        for i, w in enumerate(vs):
            t = pv[i] * 1e-3
            tr = times_of(w)
            out[w["name"]] = {"ms": pv[i], "gnnz_s": w["nnz"] / t / 1e9, "roofline_frac": max(tr.values()) / t,
                              "bound": max(tr, key=tr.get), "fracs": {k: tr[k] / t for k in tr},
                              "fp64_tinstr_s": w["nnz"] * per_entry(w)[0] / t / 1e12,
                              "hbm_gbs": bytes_of(w) / t / 1e9, "chunk": w["info"]["chunk"]}
        return out

    # roofline of the dominant kernel (largest share of the step): the
    # largest of the three roofline times decides the bound
    dom = int(np.argmax(per_var))
    v = variants[dom]
    t_s = per_var[dom] * 1e-3
    o_e, u_e = per_entry(v)
    ops, upd, byts = v["nnz"] * o_e, v["nnz"] * u_e, bytes_of(v)
    tr = times_of(v)
    which = max(tr, key=tr.get)
    if which == "fp64":
        bound, achieved, peak, unit = "alu", ops / t_s / 1e12, fp64_fma / 1e12, "T binary64 instr/s"
        src = "measured in this run by mpspmv_probe_fp64 (DFMA chains, all SMs)"
    elif which == "smem":
        bound, achieved, peak, unit = "alu", upd / t_s / 1e12, smem / 1e12, "T shared-memory digit updates/s"
        src = ("derived: SMs x 2070 MHz x %d B/clk shared-memory bandwidth / %d B per update "
               "(8-byte load + 8-byte store)" % (SMEM_BYTES_PER_CLK, UPD_BYTES))
    else:
        bound, achieved, peak, unit = "hbm", byts / t_s / 1e9, hbm, "GB/s"
        src = hbm_src
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
            "traffic": stored_traffic(v["arith"] + ":" + v["name"]),
            "kernel": "spmv run/row kernels + combine kernels, %s arithmetic, %s" % (v["arith"], v["name"]),
            "peak_source": src,
            "fracs": {k: tr[k] / t_s for k in tr},
            "hbm_peak_source": hbm_src,
            "algorithmic_ops_per_launch": ops, "algorithmic_digit_updates_per_launch": upd,
            "algorithmic_bytes_per_launch": byts, "fp64_dadd_peak_tinstr_s": fp64_add / 1e12,
            "ops_per_entry": o_e, "updates_per_entry": u_e, "value_planes": v["info"]["value_planes"]}
    breakdown = breakdown_of(variants, per_var)
    other_out = {}
    for ar, (pv, oms, _) in other.items():
        onnz = sum(w["nnz"] for w in sets[ar])
        other_out[ar] = {"value": onnz / (oms * 1e-3) / 1e9, "ms_per_step": oms, "repeat_per_step": 1,
                         "breakdown": breakdown_of(sets[ar], pv)}

    # sampled rows of every variant's result, for the parity report of the
    # oracle leg (one more product per variant, outside the timed region)
    parity = None
    samples = None
    if pool is not None:
        try:
            rows_of = {m: sample_rows(c) for m, c in mats.items()}
            samples, chunk_of, sell_of = {}, {}, {}
            for ar in ariths:
                for w in sets[ar]:
                    mps.mpspmv_spmv(w["h"], w["x"], w["y"], stream)
                    idx = torch.from_numpy(rows_of[w["m"]]).to(w["y"].device)
                    samples[(ar, w["m"], w["L"])] = w["y"].index_select(1, idx).cpu().numpy()
                    chunk_of[(ar, w["m"], w["L"])] = w["info"]["chunk"]
                    sell_of[(ar, w["m"], w["L"])] = w["info"]["sell_slots"] > 0
            torch.cuda.synchronize()
        except Exception as e:  # the report is diagnostic: it never stops the measurement
            samples, parity = None, {"error": repr(e)}

    for ar in ariths:
        for w in sets[ar]:
            mps.mpspmv_destroy(w["h"])
    del hosts
    parts_out = {}
    if rank == 0:
        del flush
        torch.cuda.empty_cache()
        parts = {"complex": lambda: suite_complex(mps, fp64_fma, hbm, stream, args.small),
                 "full_limb": lambda: part_full_limb(mps, fp64_fma, hbm, stream, args.small),
                 "powerlaw16": lambda: part_powerlaw16(mps, fp64_fma, hbm, stream, args.small),
                 "cg_time": lambda: part_cg_time(mps, args.small),
                 "cg": lambda: suite_cg(mps, stream, args.small),
                 "product": lambda: suite_product(mps, stream, args.small),
                 "batched": lambda: suite_batched(mps, stream, args.small),
                 "selector": lambda: suite_selector(mps, args.small),
                 "selector_exact": lambda: suite_selector(mps, args.small, mps.MPSPMV_EXACT_ACC),
                 "selector_large": lambda: suite_selector_large(mps, args.small),
                 "selector_scale": lambda: suite_selector_scale(mps, args.small)}
        names = [] if args.parts in ("", "none") else args.parts.split(",")
        if args.suite:
            names += [p for p in args.suite.split(",") if p not in names]
        for name in names:
            if name not in parts:
                raise SystemExit("unknown part %r" % name)
            t0 = time.perf_counter()
            parts_out[name] = parts[name]()
            parts_out[name]["wall_s"] = time.perf_counter() - t0

    cpu = None
    if pool is not None:
        if samples is not None:
            try:
                parity = parity_report(mats, xs_host, rows_of, samples, chunk_of, sell_of)
            except Exception as e:
                parity = {"error": repr(e)}
        nnz_of = {(w["m"], w["L"]): w["nnz"] for w in variants}
        t0 = time.perf_counter()
        sampler = OracleSampler(mats, xs_host, ncores)
        try:
            rates = sampler.rates(pool)
            single = sampler.single_rates(pool)
        finally:
            sampler.close()
        cpu = {"value": cpu_rate_for_step(rates, nnz_of) / 1e9, "unit": UNIT, "cores": ncores, "kind": "oracle",
               "sample": sampler.desc, "single_core_value": cpu_rate_for_step(single, nnz_of) / 1e9,
               "per_variant_all_cores": {"%s/%s" % (m, PNAME[L]): r / 1e9 for (m, L), r in rates.items()},
               "wall_s": time.perf_counter() - t0}
        pool.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_block(mats, R),
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "entry_point": "mpspmv_spmv_host_async, two streams, pinned host buffers"},
            "gpu_launches": launches_per_step * args.steps, "clocks": clocks,
            "fp64_peak_tinstr_s": {"dfma": fp64_fma / 1e12, "dadd": fp64_add / 1e12},
            "arith": primary, "breakdown": breakdown,
        }
        if other_out:
            line["other_arith"] = other_out
        if parity is not None:
            line["parity"] = parity
        for name, res in parts_out.items():
            key = {"complex": "complex", "full_limb": "full_limb_A", "powerlaw16": "powerlaw_mean16",
                   "cg_time": "cg_time_to_1e-30"}.get(name)
            if key:
                line[key] = res
            else:
                line.setdefault("suite", {})[name] = res
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
