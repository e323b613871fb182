"""Benchmark: multiple-precision CSR SpMV throughput (Gnnz/s) on GB300.

Workload (one step): y = A x in DD, TD and QD (P mode, binary64 values
promoted) on two real matrices shaped like the paper's SpMV workloads
(arXiv 2412.17510, Section 4.1, SuiteSparse stand-ins):
  (a) 3D 27-point stencil on a 128^3 grid, non-periodic (n = 2,097,152,
      nnz = 55,742,968), off-diagonals N(0,1), diagonal = row |sum| + 1;
  (b) power-law rows, n = 1,000,000, lengths Zipf(1.5) clipped to [1, 20000]
      (nnz ~ 2.17e8), uniform distinct columns, N(0,1) values;
x with every component random, seed 0.  value = (sum of nnz over the six
products) / (device time of the step).  Inputs are resident in HBM; the L2
cache is flushed (a 512 MiB write) between timed steps, outside the timed
events.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
N > 1 runs under torch.distributed.run; every rank multiplies its own copy of
the workload (independent problems, no collective on the data path), the time
is the maximum over ranks and value counts the nnz of all ranks.
"""
import argparse
import hashlib
import json
import os
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
# -- only the FMA chain of the rounded products; the exact products are
# formed on the integer pipe -- in P mode and on binary64 data (one stored
# value plane, MP x binary64 product forms):
OPS_PER_ENTRY_EXACT = {2: 2, 3: 3, 4: 4}
OPS_PER_ENTRY_EXACT_D = {2: 1, 3: 1, 4: 1}
# ... and shared-memory digit updates per stored entry, the accumulation's
# own bound: an exact 106-bit product adds five 32-bit chunks, a rounded
# binary64 term three (P mode: 1/3/6 exact products for DD/TD/QD; binary64
# data: L - 1), each update an 8-byte load and an 8-byte store.
UPD_PER_ENTRY_EXACT = {2: 8, 3: 18, 4: 33}
UPD_PER_ENTRY_EXACT_D = {2: 8, 3: 13, 4: 18}
SMEM_BYTES_PER_CLK = 128  # shared-memory bandwidth per SM per clock (32 banks x 4 B)
UPD_BYTES = 16
L2_FLUSH_BYTES = 512 << 20


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
    for f in ("spmv.cu", "mp_arith.cuh", "run_body.cuh", "fixacc.cuh", "exact_prod.cuh", "api.cu"):
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
# CPU oracle leg (bounded sample, all host cores)
# ---------------------------------------------------------------------------
def _oracle_worker(args):
    indptr, indices, data, x, L = args
    import oracle as orc
    A = orc.CSR(len(indptr) - 1, x.shape[1], indptr, indices, data, L, False)
    t = time.perf_counter()
    orc.spmv(A, x)
    return time.perf_counter() - t


def _task(ip, a, b, coo, x, L):
    """Rows a..b-1 as a small CSR over the columns they reference (x gathered
    and the column indices renumbered, so that only that part of x is sent to
    the worker)."""
    lo, hi = ip[a], ip[b]
    cols = coo.col[lo:hi]
    uniq, local = np.unique(cols, return_inverse=True)
    data = np.zeros((L, hi - lo))
    data[0] = coo.val[0, lo:hi]
    return (ip[a:b + 1] - lo, local.astype(np.int32), data, np.ascontiguousarray(x[:, uniq]), L)


def oracle_sample(mats, xs, entries_per_variant, pool, ncores):
    """Oracle throughput on a sample: for every (matrix, precision) a block of
    consecutive rows holding about entries_per_variant entries, cut into
    ncores slices run in parallel.  xs[matrix][L] is the vector.  Returns
    per-variant entries/s."""
    rates = {}
    for mname, coo in mats.items():
        ip = np.zeros(coo.nrows + 1, dtype=np.int64)
        np.add.at(ip, coo.row + 1, 1)
        ip = np.cumsum(ip)
        for L in PRECS:
            want = entries_per_variant[L]
            r0 = coo.nrows // 3
            r1 = int(np.searchsorted(ip, ip[r0] + want))
            r1 = max(r0 + 1, min(r1, coo.nrows))
            bounds = np.linspace(r0, r1, ncores + 1).astype(np.int64)
            tasks = [_task(ip, a, b, coo, xs[mname][L], L) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
            # the slices run concurrently: the sample's time is the slowest one
            dt = max(pool.map(_oracle_worker, tasks, chunksize=1))
            rates[(mname, L)] = (ip[r1] - ip[r0]) / dt
    return rates


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
                    whole = np.ones(len(rows), dtype=bool) if (sell_of or {}).get(key) else one
                    for i in np.nonzero(whole)[0]:
                        want, fits = exact_model.row_model(L, 1, A, x, int(i))
                        if fits:
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
    sample = {2: 400000, 3: 60000, 4: 60000}
    step_rates = []
    with ctx.Pool(ncores) as pool:
        for it in range(args.warmup + args.steps):
            rates = oracle_sample(mats, xs, sample, pool, ncores)
            if it >= args.warmup:
                step_rates.append(cpu_rate_for_step(rates, nnz_of))
    total_nnz = sum(nnz_of.values())
    ms = [total_nnz / r * 1e3 for r in step_rates]
    value = total_nnz / (sum(ms) / len(ms) * 1e-3) / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sum(ms) / len(ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_block(mats),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncores, "kind": "oracle",
                         "sample": "per step and per (matrix, precision) a block of consecutive rows holding "
                                   "%s entries, split over %d processes; time scaled to the full step" %
                                   (sample, ncores)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def config_block(mats):
    return {"workload": "real CSR SpMV, DD/TD/QD P mode: " + ", ".join(
        "%s (n=%d, nnz=%d)" % (k, v.nrows, v.nnz) for k, v in mats.items()),
        "x": "every component random, seed 0", "l2": "flushed between timed steps (512 MiB write)",
        "precisions": [PNAME[L] for L in PRECS]}



# ---------------------------------------------------------------------------
# --suite: the other workloads (complex SpMV + BiCGSTAB, batched SpMM + CG,
# learned selector).  Reported under "suite" in the JSON line.
# ---------------------------------------------------------------------------
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


def suite_selector(mps, small, flags=0):
    """Learned precision selector on a scaled-down system set (360 systems,
    n up to 160 rather than 1e4..1e5, so labelling stays within minutes):
    SPD systems A = D (L L^T + I) D, n log-uniform in [40, 160], cond 10^U[8, 40],
    labelled by the cheapest of binary64 / DD / TD / QD whose CG reaches
    1e-30 within 30 n iterations; train on the first ones, evaluate on the
    held-out rest against the plain ladder."""
    from paper_2412_17510_gb300 import selector as sel
    ntrain, ntest = (60, 20) if small else (300, 60)
    rng = np.random.default_rng(0)
    systems = []
    for i in range(ntrain + ntest):
        n = int(round(np.exp(rng.uniform(np.log(40), np.log(160)))))
        coo, b = workloads.selector_system(n, float(rng.uniform(8, 40)), seed=1000 + i)
        systems.append(sel.System(coo, b, flags))
    t0 = time.perf_counter()
    X = sel.features(systems)
    y = sel.labels(systems, 1e-30, maxit_factor=30)
    label_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    params, losses, _ = sel.train(X[:ntrain], y[:ntrain], epochs=300, batch=32, lr=0.05)
    train_s = time.perf_counter() - t0
    pred = sel.predict(params, X[ntrain:])
    ev = sel.evaluate(systems[ntrain:], params, 1e-30, maxit_factor=30)
    for s in systems:
        s.free()
    return {"systems": ntrain + ntest, "train": ntrain, "test": ntest,
            "label_hist": {int(c): int((y == c).sum()) for c in range(5)},
            "label_s": label_s, "train_s": train_s, "loss_first_last": [float(losses[0]), float(losses[-1])],
            "test_accuracy": float((pred == y[ntrain:]).mean()),
            "escalation_rate": ev["escalated"] / ev["n"],
            "plain_ladder_s": ev["plain_s"], "selector_ladder_s": ev["auto_s"],
            "batched_selector_s": ev["batched_auto_s"],
            "solved": {"plain": ev["plain_ok"], "selector": ev["auto_ok"], "batched_selector": ev["batched_auto_ok"]}}

# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--small", action="store_true", help="reduced matrices (development)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle leg")
    ap.add_argument("--only", default=None, help="run one variant, e.g. powerlaw_1e5/QD (profiling)")
    ap.add_argument("--arith", default="both", choices=["paper", "exact", "both"],
                    help="paper: the paper's DD/TD/QD operation sequences; exact: error-free products on the "
                         "binary64 pipe with exact integer accumulation (MPSPMV_EXACT_ACC); both: value from "
                         "exact, the paper-order step timed too")
    ap.add_argument("--cg-only", default=None,
                    help="profiling: run only the CG workload of the suite in one variant, e.g. QD/exact, and exit")
    ap.add_argument("--cg-iters", type=int, default=200, help="CG iterations of the CG workload")
    ap.add_argument("--suite", nargs="?", const="complex,cg,product,batched,selector,selector_exact", default=None,
                    help="also measure the complex, CG, product-type, batched and selector workloads (adds "
                         "minutes); "
                         "optionally a comma-separated subset")
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

    mats = make_matrices(args.small)
    ariths = ["exact", "paper"] if args.arith == "both" else [args.arith]
    sets = {ar: [] for ar in ariths}
    xs_host = {}
    xs_dev = {}
    for mname, coo in mats.items():
        xs_host[mname] = {L: workloads.full_limb_vector(coo.ncols, L, seed=0) for L in PRECS}
        for L in PRECS:
            if args.only and args.only != "%s/%s" % (mname, PNAME[L]):
                continue
            x = torch.from_numpy(xs_host[mname][L]).cuda()
            y = torch.empty((L, coo.nrows), dtype=torch.float64, device="cuda")
            xs_dev[(mname, L)] = x
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

    def step(variants, evs=None):
        for i, v in enumerate(variants):
            if evs:
                evs[i][0].record(stream)
            mps.mpspmv_spmv(v["h"], v["x"], v["y"], stream)
            if evs:
                evs[i][1].record(stream)

    def timed(variants, sample_clocks):
        for _ in range(args.warmup):
            flush.zero_()
            step(variants)
        torch.cuda.synchronize()
        sampler = ClockSampler(local) if sample_clocks else None
        if sampler:
            sampler.start()
            time.sleep(0.3)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        all_evs = []
        for _ in range(args.steps):
            flush.zero_()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in variants]
            step(variants, evs)
            all_evs.append(evs)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clk = sampler.stop() if sampler else None
        per_var = np.zeros(len(variants))
        step_ms = []
        for evs in all_evs:
            t = [a.elapsed_time(b) for a, b in evs]
            per_var += np.array(t)
            step_ms.append(sum(t))
        return per_var / args.steps, float(np.mean(step_ms)), clk

    primary = ariths[0]
    variants = sets[primary]
    per_var, ms, clocks = timed(variants, True)
    other = {ar: timed(sets[ar], False) for ar in ariths[1:]}
    step_nnz = sum(v["nnz"] for v in variants)
    ms, value = replica_value(ms, step_nnz, world, dist, device="cuda")
    def launches_of(v):
        i = v["info"]
        if v["arith"] != "exact":
            return 1 + (i["nsplit_rows"] > i["nlong_rows"]) + (i["nlong_rows"] > 0)
        inter = 1 if v["L"] > 1 else 0  # interleaved copy of x
        if i["sell_slots"] > 0:
            return inter + 1            # one row per thread
        return inter + 1 + (i["nsplit_rows"] > i["nlong_rows"]) + (i["nlong_rows"] > 0)

    launches_per_step = sum(launches_of(v) for v in variants)

    # end to end through the host-buffer entry point (pinned host memory)
    e2e_ms = []
    h2d = d2h = 0
    hosts = []
    for v in variants:
        xh = torch.from_numpy(xs_host[v["m"]][v["L"]]).pin_memory()
        yh = torch.empty((v["L"], v["nrows"]), dtype=torch.float64).pin_memory()
        hosts.append((xh, yh))
        h2d += xh.numel() * 8
        d2h += yh.numel() * 8
    for it in range(max(3, min(args.steps, 10)) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for v, (xh, yh) in zip(variants, hosts):
            mps.mpspmv_spmv_host(v["h"], xh, yh, stream)
        t1 = time.perf_counter()
        if it > 0:
            e2e_ms.append((t1 - t0) * 1e3)
    _, e2e_value = replica_value(float(np.mean(e2e_ms)), step_nnz, world, dist, device="cuda")

    hbm = 6786.2
    try:
        hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
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
                              "bound": max(tr, key=tr.get), "fp64_tinstr_s": w["nnz"] * per_entry(w)[0] / t / 1e12,
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
        src = "MEASURED_PEAKS.json hbm_gbs"
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
            "traffic": stored_traffic(v["arith"] + ":" + v["name"]),
            "kernel": "spmv run/row kernels + combine kernels, %s arithmetic, %s" % (v["arith"], v["name"]),
            "peak_source": src,
            "fracs": {k: tr[k] / t_s for k in tr},
            "algorithmic_ops_per_launch": ops, "algorithmic_digit_updates_per_launch": upd,
            "algorithmic_bytes_per_launch": byts, "fp64_dadd_peak_tinstr_s": fp64_add / 1e12,
            "ops_per_entry": o_e, "updates_per_entry": u_e, "value_planes": v["info"]["value_planes"]}
    breakdown = breakdown_of(variants, per_var)
    other_out = {}
    for ar, (pv, oms, _) in other.items():
        onnz = sum(w["nnz"] for w in sets[ar])
        other_out[ar] = {"value": onnz / (oms * 1e-3) / 1e9, "ms_per_step": oms,
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

    cpu = None
    if pool is not None:
        if samples is not None:
            try:
                parity = parity_report(mats, xs_host, rows_of, samples, chunk_of, sell_of)
            except Exception as e:
                parity = {"error": repr(e)}
        nnz_of = {(w["m"], w["L"]): w["nnz"] for w in variants}
        sample = {2: 4000000, 3: 500000, 4: 500000}
        t0 = time.perf_counter()
        rates = oracle_sample(mats, xs_host, sample, pool, ncores)
        cpu = {"value": cpu_rate_for_step(rates, nnz_of) / 1e9, "unit": UNIT, "cores": ncores, "kind": "oracle",
               "sample": "per (matrix, precision) a block of consecutive rows holding %s entries (DD/TD/QD), split "
                         "over %d spawned processes; rates combined with the GPU step's mix" % (sample, ncores),
               "wall_s": time.perf_counter() - t0}
        pool.close()

    for ar in ariths:
        for w in sets[ar]:
            mps.mpspmv_destroy(w["h"])
    suite = None
    if args.suite and rank == 0:
        del flush
        parts = {"complex": lambda: suite_complex(mps, fp64_fma, hbm, stream, args.small),
                 "cg": lambda: suite_cg(mps, stream, args.small),
                 "product": lambda: suite_product(mps, stream, args.small),
                 "batched": lambda: suite_batched(mps, stream, args.small),
                 "selector": lambda: suite_selector(mps, args.small),
                 "selector_exact": lambda: suite_selector(mps, args.small, mps.MPSPMV_EXACT_ACC)}
        suite = {}
        for name in args.suite.split(","):
            if name not in parts:
                raise SystemExit("unknown suite part %r" % name)
            suite[name] = parts[name]()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_block(mats),
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches_per_step * args.steps, "clocks": clocks,
            "fp64_peak_tinstr_s": {"dfma": fp64_fma / 1e12, "dadd": fp64_add / 1e12},
            "arith": primary, "breakdown": breakdown,
        }
        if other_out:
            line["other_arith"] = other_out
        if parity is not None:
            line["parity"] = parity
        if suite is not None:
            line["suite"] = suite
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
