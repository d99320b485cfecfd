"""Benchmark of the constant-weight PIR server answer path on GB300.

Workload (the metric's configuration): index PIR over n = 65536 rows of
8192 16-bit coefficients (1 GiB of payload, 6 GiB resident in NTT form in
the row basis), codewords of weight k = 4 and length m = 37, BFV with
N = 8192, four 54-bit primes, t = 65537; one query of 37 ciphertexts per
step.  Keys and queries are uniform residues (the distribution of RLWE keys
and ciphertexts); the answer path does the same work on them as on real
encryptions.

A step is one full answer: selection vector (product tree with
relinearisation), plain multiplication and accumulation over all rows.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun every rank answers its own
queries against its own copy of the database (queries are independent).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PIR answer DB MB/s per query (N=8192,k=4); batched vs plain; p50/p99 latency"
WL = dict(N=8192, L=4, n=65536, k=4, m=37, plen=8192, t=65537, coef_bytes=2)
WORKLOAD_NAME = ("index PIR n=65536 rows x 8192 16-bit coefficients, k=4, m=37, "
                 "BFV N=8192 L=4 (54-bit primes) t=65537, one query per step")
EXT_PRIMES = {1: 5, 2: 8, 3: 12, 4: 15, 5: 19, 6: 23, 7: 26, 8: 30}  # 30-bit primes per L


def modmul_weights(pk: dict):
    """IMAD-equivalents of one modular multiplication, from the measured
    integer rates (cwpir_measure_int_peaks): a 54-bit residue in a 64-bit
    word takes two 64 x 64 low products and one high product (Shoup or
    Barrett), a 30-bit residue two 32-bit low products and one high one;
    each product weighs the IMAD rate over its own measured rate."""
    imad = pk["imad32_per_s"]
    w54 = 2 * imad / pk["mullo64_per_s"] + imad / pk["mulhi64_per_s"]
    w30 = 2 + imad / pk["mulhi32_per_s"]
    return w54, w30


def payload_mb(rows: int) -> float:
    return rows * WL["plen"] * WL["coef_bytes"] / 1e6


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        finally:
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------------ workload
def make_inputs(seed: int = 12, rows: int | None = None, oracle_side: bool = False):
    """The workload's seeded inputs.  The primes and codewords come from the
    library's host helpers, or, for the CPU oracle's legs (oracle_side), from
    the oracle's own, so that those legs load nothing of the product."""
    from paper_2202_07569_gb300 import synthetic as syn

    if oracle_side:
        import oracle as H
        primes = H.primes
    else:
        from paper_2202_07569_gb300 import binding as H
        primes = H.default_primes
    N, L, n, k, m = WL["N"], WL["L"], rows or WL["n"], WL["k"], WL["m"]
    q = np.asarray(primes(N, L), dtype=np.uint64)
    rlk = syn.uniform_residues(syn.Stream(seed, 3), q, (L, 2), N)
    query = syn.uniform_ciphertexts(seed + 1, q, m, N)
    items = syn.payload(syn.Stream(seed, 1), n, WL["plen"], 1 << 16)
    cw = np.stack([H.map_perfect(i, m, k) for i in range(n)])
    return q, rlk, query, items, cw


def imad_per_job(kind: str, m54: float, m30: float) -> float:
    """Algorithmic work per job of a kernel class, in IMAD-equivalents:
    54-bit modular multiplications (one per butterfly, product or
    reduction) times m54, 30-bit ones times m30 (modmul_weights), and the
    scale-down's 32 x 32 products of 27-bit halves with 30-bit constants
    times 1."""
    N, L = WL["N"], WL["L"]
    K = EXT_PRIMES[L]
    logN = N.bit_length() - 1
    bf = N // 2 * logN
    if kind == "tensor":  # 3 outputs x K extension limbs, inverse transforms; 4 products
        return 3 * K * bf * m30 + 4 * N * K * m30
    if kind == "row_ntt":  # row basis of 3 primes (t = 65537, N = 8192): 3L limbs x 3
        # primes, each reduced (a 32-bit fold and Barrett step, counted as 3)
        # and transformed on 32-bit words
        return 3 * L * 3 * (bf * m30 + 3 * N)
    if kind == "relin_pm":  # row sums: one 32 x 32-bit product with the row per
        # transform coefficient; the per-group conversions and key products
        # are left out
        return 3 * L * 3 * N
    if kind == "scale":  # per coefficient of 3 polynomials, from the K extension residues
        per = (m30 * K + 3 * K          # the digits x_k; the fixed-point sums for v and G
               + L * (2 * K + 2) + m54 * L)  # the sums modulo q_j and their reductions
        return 3 * N * per
    if kind == "lift":
        return 2 * N * (m54 * L + K * 2 * L + m54 * K)
    return 0.0


# DRAM bytes (read + write) per job of each kernel class, from one ncu
# capture of the current kernels on the profiling size (4096 rows, 128
# multiplications per launch).  DRAM traffic grows in proportion to the
# jobs of a launch, so a full launch's traffic is this figure times its
# jobs.
DRAM_BYTES_PER_JOB = {
    "tensor": (79719936 + 132475392) / 128,  # k_tensor_ext, K = 15
    "scale": (188826624 + 70107136) / 128,
    "row_ntt": (108978176 + 100567296) / 128,
    # the row sums (k_rows_mac); the once-per-row-group conversions are
    # left out
    "relin_pm": (163604480 + 25714944) / 128,
}


def max_over_ranks(dist, x: float, device) -> float:
    """The largest of the ranks' values of x (x itself on one rank)."""
    if not dist:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_gpu(args, rank: int, world: int, dist, keep: bool = False):
    import torch

    from paper_2202_07569_gb300 import binding as B

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    q, rlk, query, items, cw = make_inputs(12 + rank, args.rows)
    ctx = B.Context(WL["N"], q, WL["t"], rlk)
    if args.max_jobs:
        ctx.set_option(B.OPT_MAX_JOBS, args.max_jobs)
    db = ctx.load_db(items, cw, WL["m"])
    del items
    stream = torch.cuda.current_stream()
    d_query = torch.from_numpy(query.view(np.int64)).to(f"cuda:{dev}")
    d_resp = torch.empty((2, WL["L"], WL["N"]), dtype=torch.int64, device=f"cuda:{dev}")

    def step():
        ctx.answer_device(db, d_query.data_ptr(), d_resp.data_ptr(), 0, stream.cuda_stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stats = ctx.last_stats()
    peaks = B.measure_int_peaks(dev)  # the roofline's integer denominator, this device now

    # device-timed region: per-step events on the launching stream
    ctx.set_option(B.OPT_KERNEL_TIMING, 1)
    ctx.kernel_times()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(args.steps):
            evs[i][0].record(stream)
            step()
            evs[i][1].record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    total_ms = t0.elapsed_time(t1)
    lat = sorted(a.elapsed_time(b) for a, b in evs)
    ktimes = ctx.kernel_times()
    ctx.set_option(B.OPT_KERNEL_TIMING, 0)
    if dist:
        t = torch.tensor([total_ms], device=f"cuda:{dev}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps

    # end to end through the host-buffer call (H2D of the query from pinned
    # host memory, D2H of the response inside the timed region)
    resp = np.zeros((2, WL["L"], WL["N"]), np.uint64)
    query = torch.from_numpy(query).pin_memory().numpy()
    ctx.answer(db, query)
    e2e = []
    for _ in range(max(1, min(args.steps, 3))):
        t = time.perf_counter()
        resp = ctx.answer(db, query)
        e2e.append(time.perf_counter() - t)
    e2e_s = max_over_ranks(dist, statistics.median(e2e), f"cuda:{dev}")
    h2d = query.nbytes
    d2h = resp.nbytes

    rows = cw.shape[0]
    mb = payload_mb(rows)
    out = {
        "value": world * mb / (ms_per_step / 1e3),
        "ms_per_step": ms_per_step,
        "p50_ms": lat[len(lat) // 2],
        "p99_ms": lat[min(len(lat) - 1, int(round(0.99 * (len(lat) - 1))))],
        "items_per_s": world * rows / (ms_per_step / 1e3),
        "e2e": {"value": world * mb / e2e_s, "unit": "MB/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(stats["kernel_launches"]) * args.steps,
        "stats": stats,
        "kernels": {k: {"ms": v[0] / args.steps, "launches": v[1] // max(1, args.steps)}
                    for k, v in ktimes.items() if v[1]},
        "clocks": clk.summary(),
    }
    # roofline of the dominant kernel: the class with the most time (on the
    # metric's workload "tensor" is the one kernel k_tensor_ext, "scale"
    # k_scale and "row_ntt" k_rows_ntt; "relin_pm" is the row sums and the
    # per-group conversions)
    dom = max((k for k in ktimes if ktimes[k][1]), key=lambda k: ktimes[k][0])
    ms, launches = ktimes[dom]
    jobs_per_launch = {"tensor": stats["mults"], "relin_pm": stats["rows"],
                       "row_ntt": stats["rows"], "scale": stats["mults"],
                       "lift": 0}.get(dom, 0)
    launches_per_step = launches / args.steps
    m54, m30 = modmul_weights(peaks)
    work_per_launch = imad_per_job(dom, m54, m30) * jobs_per_launch / max(1.0, launches_per_step)
    avg_launch_s = ms / launches / 1e3
    peak = peaks["imad32_per_s"] / 1e12
    achieved = work_per_launch / avg_launch_s / 1e12 if avg_launch_s > 0 else 0.0
    kernel = {"tensor": "k_tensor_ext", "scale": "k_scale", "row_ntt": "k_rows_ntt"}.get(dom)
    out["roofline"] = {"kernel": f"{dom} ({kernel})" if kernel else dom, "bound": "alu", "achieved": achieved, "peak": peak,
                       "unit": "TIMAD/s", "frac": achieved / peak if peak else None,
                       "traffic": (DRAM_BYTES_PER_JOB[dom] * jobs_per_launch
                                   / max(1.0, launches_per_step)
                                   if dom in DRAM_BYTES_PER_JOB else None),
                       "traffic_unit": "bytes per launch",
                       "peak_basis": (
                           "measured in this run (cwpir_measure_int_peaks: independent IMAD "
                           f"chains on all {peaks['sms']} SMs, CUDA events): "
                           f"{peaks['imad32_per_s'] / 1e12:.2f} T IMAD/s; work counted as "
                           f"{m54:.2f} IMAD per 54-bit and {m30:.2f} per 30-bit modular "
                           "multiplication from the measured 64-bit and high-product rates"),
                       "int_peaks_measured": peaks}
    if keep:
        return out, (ctx, db, q)
    ctx.free_db(db)
    ctx.close()
    return out, None


def run_sharded(args, rank: int, world: int, dist):
    """The metric's workload with the database's rows sharded over the
    ranks (one GPU each): every rank answers the query over its block of
    rows and the partial responses meet in one exchange (--exchange: a SUM
    all-reduce of the u64 residues then the reduction modulo q_j, or an
    all-gather then the modular sum; paper_2202_07569_gb300/shard.py).
    Total work is fixed: strong scaling.  At one rank the step is the plain
    answer plus the reduction of one partial."""
    import torch

    from paper_2202_07569_gb300 import binding as B
    from paper_2202_07569_gb300.shard import ShardedDatabase

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    q, rlk, query, items, cw = make_inputs(12, args.rows)  # same database on every rank
    ctx = B.Context(WL["N"], q, WL["t"], rlk)
    if args.max_jobs:
        ctx.set_option(B.OPT_MAX_JOBS, args.max_jobs)
    sh = ShardedDatabase(ctx, items, cw, WL["m"])
    del items
    stream = torch.cuda.current_stream()
    d_query = torch.from_numpy(query.view(np.int64)).to(f"cuda:{dev}")
    d_resp = torch.empty((2, WL["L"], WL["N"]), dtype=torch.int64, device=f"cuda:{dev}")
    for _ in range(args.warmup):
        sh.answer_device(d_query, d_resp, exchange=args.exchange)
    torch.cuda.synchronize()
    stats = ctx.last_stats()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            sh.answer_device(d_query, d_resp, exchange=args.exchange)
        t1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    total_ms = t0.elapsed_time(t1)
    if dist:
        t = torch.tensor([total_ms], device=f"cuda:{dev}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    # end to end: query from pinned host memory, response back to the host
    h_query = torch.from_numpy(query.view(np.int64)).pin_memory()
    h_resp = torch.empty((2, WL["L"], WL["N"]), dtype=torch.int64).pin_memory()
    e2e = []
    for _ in range(max(1, min(args.steps, 3))):
        if dist:
            dist.barrier()
        t = time.perf_counter()
        d_query.copy_(h_query, non_blocking=True)
        sh.answer_device(d_query, d_resp, exchange=args.exchange)
        h_resp.copy_(d_resp, non_blocking=True)
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t)
    e2e_s = max_over_ranks(dist, statistics.median(e2e), f"cuda:{dev}")
    mb = payload_mb(cw.shape[0])
    out = {
        "value": mb / (ms_per_step / 1e3),
        "ms_per_step": ms_per_step,
        "scaling": "strong",
        "items_per_s": cw.shape[0] / (ms_per_step / 1e3),
        "e2e": {"value": mb / e2e_s, "unit": "MB/s",
                "h2d_bytes_per_step": int(query.nbytes), "d2h_bytes_per_step": int(d_resp.numel() * 8)},
        "gpu_launches": (int(stats["kernel_launches"]) + 1) * args.steps,
        "stats": stats,
        "clocks": clk.summary(),
        "shard": {"rank_rows": [sh.lo, sh.hi], "world": world, "exchange": args.exchange},
    }
    sh.close()
    ctx.close()
    return out


def run_large(args):
    """Large payloads (the paper's large-payload experiment, Sec. 4): index
    PIR over n = 16384 rows with k = 2 at N = 8192, L = 4, each row s
    plaintexts of 8192 16-bit coefficients.  The selection vector is formed
    once per row and only the inner product repeats per plaintext, so DB
    MB/s grows with s.  Reported for s = 1 and s = 17 (278.5 KB per row,
    past the 268 KB where the paper finds constant-weight PIR overtaking
    MulPIR)."""
    import torch

    from paper_2202_07569_gb300 import binding as B
    from paper_2202_07569_gb300 import synthetic as syn

    N, L, n, k = 8192, 4, args.rows or 16384, 2  # --rows: a profiling size
    m = B.code_length(n, k)
    q = B.default_primes(N, L)
    rlk = syn.uniform_residues(syn.Stream(51, 3), q, (L, 2), N)
    ctx = B.Context(N, q, 65537, rlk)
    query = syn.uniform_ciphertexts(52, q, m, N)
    cw = np.stack([B.map_perfect(i, m, k) for i in range(n)])
    stream = torch.cuda.current_stream()
    d_query = torch.from_numpy(query.view(np.int64)).cuda()
    runs = []
    for sp in (1, 17):
        items = syn.payload(syn.Stream(53, sp), n, sp * N, 1 << 16)
        db = ctx.load_db(items, cw, m)
        del items
        d_resp = torch.empty((sp, 2, L, N), dtype=torch.int64, device="cuda")

        def step():
            ctx.answer_device(db, d_query.data_ptr(), d_resp.data_ptr(), 0, stream.cuda_stream)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        stats = ctx.last_stats()
        ctx.set_option(B.OPT_KERNEL_TIMING, 1)
        ctx.kernel_times()
        with ClockSampler(0) as clk:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                step()
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        kt = ctx.kernel_times()
        ctx.set_option(B.OPT_KERNEL_TIMING, 0)
        e2e = []
        h_query = torch.from_numpy(query).pin_memory().numpy()  # pinned host memory
        for _ in range(max(1, min(args.steps, 3))):
            t = time.perf_counter()
            resp = ctx.answer(db, h_query)
            e2e.append(time.perf_counter() - t)
        mb = n * sp * N * 2 / 1e6
        kernels = {kk: {"ms": v[0] / args.steps, "launches": v[1] // max(1, args.steps)}
                   for kk, v in kt.items() if v[1]}
        # the key-switch multiply-accumulate streams the database once per
        # answer: its DB bytes over its time against the measured HBM copy rate
        relin = kernels.get("relin_pm", {}).get("ms", 0.0)
        runs.append({"plaintexts_per_row": sp, "payload_kb_per_row": sp * N * 2 / 1e3,
                     "db_mb": mb, "ms_per_answer": ms, "value": mb / (ms / 1e3),
                     "e2e": {"value": mb / statistics.median(e2e), "unit": "MB/s",
                             "h2d_bytes_per_step": int(query.nbytes),
                             "d2h_bytes_per_step": int(resp.nbytes)},
                     "db_bytes_read": int(stats["db_bytes_read"]),
                     "relin_pm_db_gbs": stats["db_bytes_read"] / (relin / 1e3) / 1e9
                     if relin else None,
                     "kernels": kernels, "clocks": clk.summary()})
        ctx.free_db(db)
        del d_resp
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                            "MEASURED_PEAKS.json")))
    except OSError:
        pass
    ratio = runs[1]["ms_per_answer"] / runs[0]["ms_per_answer"]
    return {"metric": "PIR answer DB MB/s vs payload size (n=16384, k=2, N=8192)",
            "unit": "MB/s", "value": runs[-1]["value"], "runs": runs,
            "time_ratio_s17_vs_s1": ratio, "payload_ratio": 17.0,
            "hbm_peak_gbs": peaks.get("hbm_gbs"),
            "config": {"workload": "index PIR n=%d rows, k=2, m=%d, BFV N=8192 L=4, "
                                   "rows of s plaintexts of 8192 16-bit coefficients" % (n, m)}}


def run_lossy(args):
    """Keyword PIR over 64-bit keywords with the lossy mapping (App. A):
    configuration 3's shape (n = 16384 rows of 8192 16-bit coefficients,
    CW(64, 8), N = 16384, L = 7, one compressed ciphertext with c = 6), the
    keywords drawn uniformly from 2^64 -- a domain no perfect mapping into
    CW(64, 8) covers.  Keywords whose codewords collide would be selected
    together; their count is reported and they are left out."""
    import torch

    from paper_2202_07569_gb300 import binding as B
    from paper_2202_07569_gb300 import synthetic as syn

    N, L, n, k, m, c = 16384, 7, args.rows or 16384, 8, 64, 6
    q = B.default_primes(N, L)
    rlk = syn.uniform_residues(syn.Stream(61, 3), q, (L, 2), N)
    gal = {N // (1 << a) + 1: syn.uniform_residues(syn.Stream(62, a), q, (L, 2), N)
           for a in range(c)}
    ctx = B.Context(N, q, 65537, rlk, gal)
    words = syn.Stream(63).words(n)
    seen, cw, collided = set(), [], 0
    for w in words:
        pos = B.map_lossy(int(w), m, k)
        key = pos.tobytes()
        if key in seen:
            collided += 1
            continue
        seen.add(key)
        cw.append(pos)
    cw = np.stack(cw)
    items = syn.payload(syn.Stream(64), len(cw), 8192, 1 << 16)
    db = ctx.load_db(items, cw, m)
    del items
    h = -(-m // (1 << c))
    query = syn.uniform_ciphertexts(65, q, h, N)
    stream = torch.cuda.current_stream()
    d_query = torch.from_numpy(query.view(np.int64)).cuda()
    d_resp = torch.empty((2, L, N), dtype=torch.int64, device="cuda")
    for _ in range(args.warmup):
        ctx.answer_device(db, d_query.data_ptr(), d_resp.data_ptr(), c, stream.cuda_stream)
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            ctx.answer_device(db, d_query.data_ptr(), d_resp.data_ptr(), c, stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    t = time.perf_counter()
    resp = ctx.answer(db, query, c)
    e2e_s = time.perf_counter() - t
    mb = payload_mb(len(cw))
    return {"metric": "keyword PIR DB MB/s per query, 64-bit keywords, lossy mapping",
            "unit": "MB/s", "value": mb / (ms / 1e3), "ms_per_answer": ms,
            "e2e": {"value": mb / e2e_s, "unit": "MB/s", "h2d_bytes_per_step": int(query.nbytes),
                    "d2h_bytes_per_step": int(resp.nbytes)},
            "rows": len(cw), "keywords_drawn": int(n), "codeword_collisions": collided,
            "collision_probability_per_pair": 1 / math.comb(m, k),
            "clocks": clk.summary(),
            "config": {"workload": "keyword PIR n=%d rows x 8192 16-bit coefficients, "
                                   "64-bit keywords, lossy CW(64,8), BFV N=16384 L=7, c=6"
                                   % len(cw)}}


def run_folklore(args):
    """Folklore PIR against constant-weight PIR in the same engine (Sec. 4):
    n = 4096 rows of 8192 16-bit coefficients at N = 16384, L = 7; folklore
    selects each row by the plain folklore operator over ell = 12 index bits
    (12 factors, depth 4), constant-weight PIR by CW(92, 2) (one
    multiplication per row)."""
    import torch

    from paper_2202_07569_gb300 import binding as B
    from paper_2202_07569_gb300 import synthetic as syn

    N, L, n, ell = 16384, 7, args.rows or 4096, 12
    q = B.default_primes(N, L)
    rlk = syn.uniform_residues(syn.Stream(71, 3), q, (L, 2), N)
    ctx = B.Context(N, q, 65537, rlk)
    items = syn.payload(syn.Stream(72), n, 8192, 1 << 16)
    stream = torch.cuda.current_stream()
    mb = payload_mb(n)
    m2 = B.code_length(n, 2)
    dbs = {"folklore": (ctx.load_db_folklore(items, ell), ell),
           "constant_weight_k2": (ctx.load_db(items, np.stack([B.map_perfect(i, m2, 2)
                                                               for i in range(n)]), m2), m2)}
    del items
    out = {}
    for name, (db, h) in dbs.items():
        query = syn.uniform_ciphertexts(73, q, h, N)
        d_query = torch.from_numpy(query.view(np.int64)).cuda()
        d_resp = torch.empty((2, L, N), dtype=torch.int64, device="cuda")
        for _ in range(args.warmup):
            ctx.answer_device(db, d_query.data_ptr(), d_resp.data_ptr(), 0, stream.cuda_stream)
        torch.cuda.synchronize()
        stats = ctx.last_stats()
        with ClockSampler(0) as clk:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                ctx.answer_device(db, d_query.data_ptr(), d_resp.data_ptr(), 0, stream.cuda_stream)
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        out[name] = {"query_cts": h, "ms_per_answer": ms, "value": mb / (ms / 1e3),
                     "mults": int(stats["mults"]), "clocks": clk.summary()}
    return {"metric": "PIR answer DB MB/s per query: folklore vs constant-weight (k=2)",
            "unit": "MB/s", "value": out["folklore"]["value"], "runs": out,
            "slowdown_folklore_vs_cw": out["folklore"]["ms_per_answer"]
            / out["constant_weight_k2"]["ms_per_answer"],
            "config": {"workload": "index PIR n=%d rows x 8192 16-bit coefficients, BFV N=16384 "
                                   "L=7; folklore ell=12 vs CW(%d,2)" % (n, m2)}}


def run_arith(args):
    """Arithmetic constant-weight equality operator on two encrypted,
    batch-encoded operands (Sec. 4, Table arith-eq): N = 16384, L = 7,
    (n, k, m) = (2^16, 8, 19) and (2^32, 16, 36), the rows k = log2(n)/2 of
    the paper's table; one evaluation compares N pairs slot-wise.  Host
    buffers in (pinned) and out, end to end through cwpir_arith_cw_eq."""
    import torch

    from paper_2202_07569_gb300 import binding as B
    from paper_2202_07569_gb300 import synthetic as syn

    N, L = 16384, 7
    q = B.default_primes(N, L)
    rlk = syn.uniform_residues(syn.Stream(81, 3), q, (L, 2), N)
    ctx = B.Context(N, q, 65537, rlk)
    runs = []
    for logn, k, m in ((16, 8, 19), (32, 16, 36)):
        x = torch.from_numpy(syn.uniform_ciphertexts(82, q, m, N)).pin_memory().numpy()
        y = torch.from_numpy(syn.uniform_ciphertexts(83, q, m, N)).pin_memory().numpy()
        for _ in range(args.warmup):
            ctx.arith_cw_eq(m, k, x, y)
        ts = []
        for _ in range(args.steps):
            t = time.perf_counter()
            ctx.arith_cw_eq(m, k, x, y)
            ts.append(time.perf_counter() - t)
        s = statistics.median(ts)
        runs.append({"domain_bits": logn, "k": k, "m": m, "mults": m + k - 1,
                     "depth": 1 + (k - 1).bit_length(), "ms_per_evaluation": s * 1e3,
                     "comparisons_per_s": N / s, "h2d_bytes": int(x.nbytes + y.nbytes),
                     "d2h_bytes": 2 * L * N * 8})
    return {"metric": "arithmetic CW equality operator: comparisons per second (N slots per "
                      "evaluation)", "unit": "comparisons/s", "value": runs[0]["comparisons_per_s"],
            "runs": runs, "config": {"workload": "arithmetic CW operator, both operands "
                                                 "encrypted, BFV N=16384 L=7, t=65537 batching"}}


# The batching workload's four databases (configuration 4); the serving
# workload uses three of them.  name, rows, k, m, N, L, c, keyword?
SYS_SPECS = [
    ("n1024_k2", 1024, 2, 46, 8192, 4, 0, False),
    ("n4096_k2", 4096, 2, 92, 8192, 4, 0, False),
    ("n16384_k8_keyword", 16384, 8, 64, 16384, 7, 6, True),
    ("n65536_k4", 65536, 4, 37, 8192, 4, 0, False),
]


def build_system_dbs(c2=None):
    """One context per database (keys seeded per ring degree), so that each
    database's launch shape is tuned on its own; `c2` = (ctx, db, primes) of
    the metric's workload stands in for n65536_k4 (the same database
    shape).  Every database gets 16 seeded queries resident on the GPU."""
    import torch

    from paper_2202_07569_gb300 import binding as B
    from paper_2202_07569_gb300 import synthetic as syn

    dbs = []
    for i, (name, n, k, m, N, L, c, kw) in enumerate(SYS_SPECS):
        if name == "n65536_k4" and c2 is not None:
            ctx, db, q = c2
        else:
            q = B.default_primes(N, L)
            rlk = syn.uniform_residues(syn.Stream(31, N), q, (L, 2), N)
            gal = {}
            if c:
                for a in range(c):
                    g = N // (1 << a) + 1
                    gal[g] = syn.uniform_residues(syn.Stream(32, g), q, (L, 2), N)
            ctx = B.Context(N, q, 65537, rlk, gal)
            items = syn.payload(syn.Stream(33, i), n, 8192, 1 << 16)
            ids = (syn.distinct_u32(syn.Stream(34, i), n) if kw else np.arange(n, dtype=np.uint64))
            cw = np.stack([B.map_perfect(int(x), m, k) for x in ids])
            db = ctx.load_db(items, cw, m)
            del items
        h = m if c == 0 else -(-m // (1 << c))
        qs = syn.uniform_ciphertexts(35 + i, q, 16 * h, N).reshape(16, h, 2, L, N)
        dbs.append(dict(name=name, ctx=ctx, db=db, c=c, h=h, L=L, N=N, n=n, k=k, m=m,
                        nq_call=4 if N == 16384 else 16, mb=payload_mb(n), qs=qs,
                        d_qs=torch.from_numpy(qs.view(np.int64)).cuda(),
                        d_rs=torch.empty((16, 2, L, N), dtype=torch.int64, device="cuda")))
    return dbs


def _events():
    import torch

    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def run_c3(d, args):
    """The keyword workload (configuration 3): one compressed query (c = 6,
    expanded by Alg. Query Expansion) against n = 16384 rows keyed by
    32-bit keywords, k = 8, m = 64, N = 16384, L = 7.  The answer is
    data-oblivious, so present and absent keywords cost the same work; the
    queries here are uniform ciphertexts."""
    import torch

    from paper_2202_07569_gb300 import binding as B

    ctx, db, st = d["ctx"], d["db"], torch.cuda.current_stream()
    ctx.set_option(B.OPT_USE_GRAPH, 0)
    q0, r0 = d["d_qs"][0].data_ptr(), d["d_rs"][0].data_ptr()
    ctx.answer_device(db, q0, r0, d["c"], st.cuda_stream)
    torch.cuda.synchronize()
    ctx.set_option(B.OPT_KERNEL_TIMING, 1)
    ctx.kernel_times()
    steps = 3
    e0, e1 = _events()
    with ClockSampler(torch.cuda.current_device()) as clk:
        e0.record(st)
        for i in range(steps):
            ctx.answer_device(db, d["d_qs"][i].data_ptr(), d["d_rs"][i].data_ptr(), d["c"],
                              st.cuda_stream)
        e1.record(st)
        torch.cuda.synchronize()
    kt = ctx.kernel_times()
    ctx.set_option(B.OPT_KERNEL_TIMING, 0)
    status = ctx.device_status(0, st.cuda_stream)
    stats = ctx.last_stats()
    ms = e0.elapsed_time(e1) / steps
    return {"workload": "keyword PIR n=16384 rows x 8192 16-bit coefficients, 32-bit keywords, "
                        "CW(64,8), BFV N=16384 L=7, one compressed query (c=6, 1 ciphertext)",
            "ms_per_answer": ms, "value": d["mb"] / (ms / 1e3), "unit": "MB/s",
            "items_per_s": d["n"] / (ms / 1e3), "steps": steps, "device_status": status,
            "stats": stats, "clocks": clk.summary(),
            "kernels": {k: {"ms": v[0] / steps, "launches": v[1] // steps}
                        for k, v in kt.items() if v[1]}}


def run_c4_blocks(dbs, args):
    """Configuration 4: 64 queries, 16 per database, over the four resident
    databases.  plain: 64 one-query calls, each database's 16 in sequence;
    batched per database: its 16 queries in batched calls (16 at a time, 4 at
    N = 16384) replayed from a CUDA graph, the launch shape of the two small
    databases picked by the autotuner (multiplications per launch x row-group
    waves); all: the 64 queries in one forked launch sequence captured into
    one CUDA graph (one branch per database, cwpir_multi).  Every batched
    response is compared with the plain one bit for bit."""
    import torch

    from paper_2202_07569_gb300 import binding as B

    st = torch.cuda.current_stream()
    for d in dbs:
        d["ctx"].set_option(B.OPT_USE_GRAPH, 0)
        d["ctx"].answer_device(d["db"], d["d_qs"][0].data_ptr(), d["d_rs"][0].data_ptr(), d["c"],
                               st.cuda_stream)
    torch.cuda.synchronize()
    per = {}
    ev = {d["name"]: _events() for d in dbs}
    with ClockSampler(torch.cuda.current_device()) as clk_plain:
        for d in dbs:
            e0, e1 = ev[d["name"]]
            e0.record(st)
            for i in range(16):
                d["ctx"].answer_device(d["db"], d["d_qs"][i].data_ptr(), d["d_rs"][i].data_ptr(),
                                       d["c"], st.cuda_stream)
            e1.record(st)
        torch.cuda.synchronize()
    plain_total = 0.0
    plain = {}
    for d in dbs:
        ms = ev[d["name"]][0].elapsed_time(ev[d["name"]][1])
        plain_total += ms
        plain[d["name"]] = d["d_rs"].clone()
        per[d["name"]] = {"N": d["N"], "rows": d["n"], "k": d["k"], "c": d["c"],
                          "plain_ms_16": ms, "plain_launches_per_query":
                          int(d["ctx"].last_stats()["kernel_launches"])}
    # autotuner on the small databases (cheap calls); the large ones keep
    # the default launch shape
    for d in dbs:
        ctx = d["ctx"]
        ctx.set_option(B.OPT_USE_GRAPH, 1)
        if d["n"] <= 4096:
            bj, bw, bms = ctx.autotune_grid(d["db"], 16, d["d_qs"].data_ptr(), d["d_rs"].data_ptr(),
                                            [256, 512, 1024, 2048], [1, 2, 4], d["c"])
            per[d["name"]]["autotuned"] = {"max_jobs": bj, "row_group_waves": bw,
                                           "ms_per_call": bms,
                                           "grid": "jobs {256,512,1024,2048} x waves {1,2,4}"}
    same = True
    batched_total = 0.0
    launches = 0
    with ClockSampler(torch.cuda.current_device()) as clk_b:
        for d in dbs:
            ctx, nqc = d["ctx"], d["nq_call"]
            for j in range(16 // nqc):  # build and capture
                ctx.answer_batch_device(d["db"], nqc, d["d_qs"][j * nqc].data_ptr(),
                                        d["d_rs"][j * nqc].data_ptr(), d["c"], st.cuda_stream)
            torch.cuda.synchronize()
            d["d_rs"].zero_()
            e0, e1 = _events()
            e0.record(st)
            for j in range(16 // nqc):
                ctx.answer_batch_device(d["db"], nqc, d["d_qs"][j * nqc].data_ptr(),
                                        d["d_rs"][j * nqc].data_ptr(), d["c"], st.cuda_stream)
            e1.record(st)
            torch.cuda.synchronize()
            launches += (16 // nqc) * int(ctx.last_stats()["kernel_launches"])
            ms = e0.elapsed_time(e1)
            batched_total += ms
            ok = bool(torch.equal(d["d_rs"], plain[d["name"]])) and ctx.device_status(0, 0) == 0
            same &= ok
            p = per[d["name"]]
            p.update({"queries_per_call": nqc, "batched_ms_16": ms,
                      "speedup_vs_plain": p["plain_ms_16"] / ms, "identical_to_plain": ok})
            ctx.release_plans(d["db"])
    # all 64 queries in one forked sequence, one graph
    mb = B.Multi([(d["ctx"], d["db"], d["c"], 16, d["nq_call"]) for d in dbs])
    outs = [torch.zeros_like(d["d_rs"]) for d in dbs]
    qp, rp = [d["d_qs"].data_ptr() for d in dbs], [o.data_ptr() for o in outs]
    mb.answer_device(qp, rp, True, st.cuda_stream)  # capture
    torch.cuda.synchronize()
    for o in outs:
        o.zero_()
    e0, e1 = _events()
    with ClockSampler(torch.cuda.current_device()) as clk_m:
        e0.record(st)
        mb.answer_device(qp, rp, True, st.cuda_stream)
        e1.record(st)
        torch.cuda.synchronize()
    multi_ms = e0.elapsed_time(e1)
    multi_same = all(bool(torch.equal(o, plain[d["name"]])) for o, d in zip(outs, dbs))
    multi_same &= mb.status(st.cuda_stream) == 0
    mstats = mb.stats()
    mb.close()
    del outs
    for d in dbs:
        d["ctx"].set_option(B.OPT_USE_GRAPH, 0)
    total_mb = sum(16 * d["mb"] for d in dbs)
    return {"metric": "batched PIR answer DB MB/s, 64 queries over 4 resident databases",
            "value": total_mb / (multi_ms / 1e3), "unit": "MB/s",
            "ms_64_queries_one_graph": multi_ms, "ms_64_queries_batched_per_db": batched_total,
            "ms_64_queries_plain": plain_total,
            "plain_value": total_mb / (plain_total / 1e3),
            "speedup_one_graph_vs_plain": plain_total / multi_ms,
            "speedup_batched_per_db_vs_plain": plain_total / batched_total,
            "responses_identical_to_plain": bool(same and multi_same),
            "gpu_launches_one_graph": int(mstats["kernel_launches"]),
            "gpu_launches_batched_per_db": launches,
            "per_db": per,
            "clocks": {"plain": clk_plain.summary(), "batched": clk_b.summary(),
                       "one_graph": clk_m.summary()}}


def run_c5_blocks(dbs, args, rates=(0.5, 1.0, 2.0, 4.0), per_rate: int = 12):
    """Configuration 5: Poisson arrivals of index and keyword queries (2:1)
    over three resident databases (n65536_k4, n4096_k2, n16384_k8_keyword),
    served with continuous batching on two lanes per database (each its own
    stream and scratch slot, so queries of all databases overlap on the
    device); per offered rate the p50/p99 latency (submission to
    completion) and the sustained DB MB/s.  Every response is compared with
    the same query answered alone.  The rates bracket the service capacity
    of this mix (about one and a half queries per second)."""
    from paper_2202_07569_gb300 import binding as B
    from paper_2202_07569_gb300 import synthetic as syn

    by = {d["name"]: d for d in dbs}
    tg_names = ["n65536_k4", "n4096_k2", "n16384_k8_keyword"]
    targets = [(by[nm]["ctx"], by[nm]["db"], by[nm]["c"]) for nm in tg_names]
    pools = []
    for nm in tg_names:
        d = by[nm]
        qs = d["qs"][:4]
        pools.append((qs, [d["ctx"].answer(d["db"], qs[j], d["c"]) for j in range(4)]))
    srv = B.Server(targets, max_batch=4, hbm_reserve=16 << 30, lanes_per_target=2)
    mix = [0, 2, 1]  # index : keyword = 2 : 1
    results = []
    all_same = True
    st = syn.Stream(46)
    for rate in rates:
        gaps = -np.log((st.below(1 << 53, per_rate).astype(np.float64) + 0.5) / 2.0 ** 53) / rate
        sent = []
        t0 = time.perf_counter()
        t_next = t0
        for i in range(per_rate):
            t_next += gaps[i]
            delay = t_next - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tg = mix[i % 3]
            j = (i // 3) % 4
            sent.append((srv.submit(tg, pools[tg][0][j]), tg, j))
        lat, mb = [], 0.0
        by_tg = {0: [], 1: [], 2: []}
        for tk, tg, j in sent:
            status, resp, l = srv.wait(tk, tg, timeout=3600)
            all_same &= status == 1 and bool(np.array_equal(resp, pools[tg][1][j]))
            lat.append(l)
            by_tg[tg].append(l)
            mb += by[tg_names[tg]]["mb"]
        wall = time.perf_counter() - t0
        lat.sort()

        def pct(v, p):
            v = sorted(v)
            return 1e3 * v[min(len(v) - 1, int(p * (len(v) - 1) + 0.5))] if v else None

        results.append({"offered_qps": rate, "queries": per_rate, "wall_s": wall,
                        "achieved_qps": per_rate / wall, "db_mb_per_s": mb / wall,
                        "p50_ms": pct(lat, 0.5), "p99_ms": pct(lat, 0.99),
                        "p50_ms_by_db": {tg_names[t]: pct(v, 0.5) for t, v in by_tg.items()},
                        "p99_ms_by_db": {tg_names[t]: pct(v, 0.99) for t, v in by_tg.items()}})
    stats = srv.stats()
    srv.close()
    return {"metric": "served PIR: p50/p99 latency and sustained DB MB/s vs offered rate",
            "value": max(r["db_mb_per_s"] for r in results), "unit": "MB/s",
            "rates": results, "responses_identical_to_alone": bool(all_same),
            "server": stats, "max_batch": 4, "lanes_per_target": 2,
            "databases": tg_names, "mix": "index:keyword = 2:1"}


def run_c4(args):
    dbs = build_system_dbs()
    return run_c4_blocks(dbs, args)


def run_c5(args):
    dbs = build_system_dbs()
    return run_c5_blocks(dbs, args)


def cpu_baseline(rows_per_step: int | None = None, reps: int = 1):
    """The oracle as it stands, OpenMP over rows on all host cores, on a
    bounded sample of the workload's rows; returns (MB/s, cores, sample)."""
    import oracle

    cores = os.cpu_count() or 1
    q, rlk, query, items, cw = make_inputs(12, oracle_side=True)
    O = oracle.Oracle(WL["N"], q, WL["t"])
    rows = rows_per_step or 2 * cores
    times = []
    for r in range(reps):
        sel = np.arange(r * rows, (r + 1) * rows) % WL["n"]
        t = time.perf_counter()
        O.answer(items[sel], cw[sel], WL["m"], query, rlk, nthreads=cores)
        times.append(time.perf_counter() - t)
    mbps = [payload_mb(rows) / t for t in times]
    return mbps, cores, f"{rows} of {WL['n']} rows per answer (3 multiplications each)"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rows", type=int, default=0,
                    help="profiling only: answer over the first ROWS rows instead of 65536")
    ap.add_argument("--max-jobs", type=int, default=0,
                    help="multiplications per kernel launch (0 = library default)")
    ap.add_argument("--exchange", default="allreduce", choices=["allreduce", "allgather"],
                    help="exchange step of the row-sharded answer: one SUM all-reduce of the "
                         "u64 residues, or an all-gather of the partial responses")
    ap.add_argument("--no-systems", action="store_true",
                    help="only the metric's workload: skip the keyword, batching and serving "
                         "blocks that follow its timed region")
    ap.add_argument("--shard-db", action="store_true",
                    help="shard the database's rows over the ranks (strong scaling) instead of "
                         "one replica per rank")
    ap.add_argument("--workload", default="c2", choices=["c2", "c4", "c5", "large", "lossy", "folklore", "arith"],
                    help="c2: the metric's workload (default); c4: batched answering over "
                         "four databases")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as tdist

        tdist.init_process_group("nccl" if args.impl == "cuda" else "gloo")
        dist = tdist

    base = {"metric": METRIC, "unit": "MB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "rows": WL["n"], "k": WL["k"], "m": WL["m"],
                       "N": WL["N"], "L": WL["L"],
                       "payload_mb_per_query": payload_mb(WL["n"]),
                       "l2": "inputs larger than L2 (6 GiB NTT-form database, three 30-bit row primes, streamed per step)",
                       "parallelism": "one query stream per GPU (replicas)"}}

    if args.impl == "reference":
        if rank != 0:
            return
        cores = os.cpu_count() or 1
        rows = 2 * cores
        cpu_baseline(max(2, rows // 4), 1)  # warm the oracle (tables, page-in)
        mbps, cores, sample = cpu_baseline(rows, args.warmup + args.steps)
        timed = mbps[args.warmup:]
        v = statistics.mean(timed)
        line = dict(base, impl="reference", value=v,
                    ms_per_step=payload_mb(rows) / v * 1e3,
                    cpu_baseline={"value": v, "unit": "MB/s", "cores": cores, "kind": "oracle",
                                  "sample": sample},
                    e2e={"value": v, "unit": "MB/s", "h2d_bytes_per_step": 0,
                         "d2h_bytes_per_step": 0})
        print(json.dumps(line), flush=True)
        return

    from paper_2202_07569_gb300 import build as cuda_build

    if rank == 0:
        cuda_build.build()
    if dist:
        dist.barrier()
    if args.workload in ("c4", "c5", "large", "lossy", "folklore", "arith"):
        if rank == 0:
            fn = {"c4": run_c4, "c5": run_c5, "large": run_large, "lossy": run_lossy,
                  "folklore": run_folklore, "arith": run_arith}[args.workload]
            print(json.dumps(dict(fn(args), data="synthetic", n_gpus=1)), flush=True)
        return
    if args.shard_db:
        res = run_sharded(args, rank, world, dist)
        if rank == 0:
            line = dict(base, scaling="strong")
            exch = ("one SUM all-reduce of the partial responses' residues, then modulo q_j"
                    if args.exchange == "allreduce" else
                    "partial responses all-gathered and summed modulo q_j")
            line["config"] = dict(base["config"], parallelism=(
                f"database rows sharded over {world} GPU(s); {exch}"))
            if args.rows:
                line["config"]["rows"] = args.rows
            line.update(res)
            print(json.dumps(line), flush=True)
        if dist:
            dist.destroy_process_group()
        return
    systems = world == 1 and not args.no_systems and not args.rows
    res, keep = run_gpu(args, rank, world, dist, keep=systems)
    sharded = None
    if world > 1:
        # the same workload with the rows sharded over the ranks, so that a
        # multi-GPU run also exercises the exchange step (after the replicas'
        # timed region, which the line's value reports)
        sharded = run_sharded(args, rank, world, dist)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    line = dict(base)
    if args.rows:
        line["config"] = dict(base["config"], rows=args.rows,
                              workload="PROFILING SIZE, not the metric workload: " + WORKLOAD_NAME)
    if args.max_jobs:
        line["config"]["max_jobs"] = args.max_jobs
    line.update(res)
    if sharded is not None:
        line["sharded"] = {k: sharded[k] for k in ("value", "ms_per_step", "scaling", "e2e",
                                                    "gpu_launches", "clocks", "shard")}
        line["sharded"]["unit"] = "MB/s"
    if systems:
        # the other configurations on the same GPU, after the metric's timed
        # region: the keyword workload, batching over four databases and
        # serving; the metric's database serves as n65536_k4
        dbs = build_system_dbs(c2=keep)
        line["c3"] = run_c3(next(d for d in dbs if d["name"] == "n16384_k8_keyword"), args)
        line["c4"] = run_c4_blocks(dbs, args)
        c2b = line["c4"]["per_db"]["n65536_k4"]
        line["batched"] = {"workload": "the metric's database, 16 distinct queries per "
                                       "batched call replayed from a CUDA graph",
                           "ms_per_query": c2b["batched_ms_16"] / 16,
                           "plain_ms_per_query": c2b["plain_ms_16"] / 16,
                           "value": payload_mb(WL["n"]) * 16 / (c2b["batched_ms_16"] / 1e3),
                           "unit": "MB/s", "speedup_vs_plain": c2b["speedup_vs_plain"],
                           "identical_to_plain": c2b["identical_to_plain"]}
        line["c5"] = run_c5_blocks(dbs, args)
        for d in dbs:
            if d["ctx"] is not keep[0]:
                d["ctx"].close()
        keep[0].close()
    if world == 1 and not args.no_cpu_baseline:
        mbps, cores, sample = cpu_baseline(None, 1)
        line["cpu_baseline"] = {"value": mbps[0], "unit": "MB/s", "cores": cores,
                                "kind": "oracle", "sample": sample}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
