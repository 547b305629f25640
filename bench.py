#!/usr/bin/env python3
"""Benchmark of the GB300 range-SVD hot path (storage phase + query phase).

One step = one pass of the whole hot path over one synthetic workload:
  (1) compress every block of the T x n matrix (already resident in HBM) into
      the store: Gram, eigen core, U  (Section 3.2, Algorithm 1);
  (2) answer a batch of range queries from the store: Partial-SVD, stack,
      stitched core, lift  (Section 3.3, Algorithms 2-3).
`value` is the storage-phase throughput in GB/s of input (the compression
target of the workload); queries/s of the batch is reported beside it.

  python bench.py [--gpus N --steps K --warmup W --workload NAME]
  python bench.py --impl reference ...   # the FP64 CPU oracle on a bounded sample

Under torchrun each rank runs its own replica of the workload on its GPU
(weak scaling, no data-path collective); timings are max-reduced over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic  # noqa: E402

METRIC = "range-SVD queries/s, p50/p99 ms, compress GB/s vs HBM peak, at fixed rel error"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """nvidia-smi samples (200 ms) during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(values, device):
    """Max of each value over all ranks (identity when not distributed)."""
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    import torch.distributed as tdist
    if tdist.is_available() and tdist.is_initialized() and tdist.get_world_size() > 1:
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return t.tolist()


def aggregate_rate(world: int, steps: int, units_per_step_per_rank: float, max_seconds: float) -> float:
    """Whole-job throughput: every rank processes the same per-rank work (weak
    scaling); the job takes as long as the slowest rank."""
    return world * steps * units_per_step_per_rank / max_seconds


def _input_rows(w, host=False):
    A = synthetic.rows(w.series, dtype=np.float64)
    if w.dtype == "f64":
        return A
    if w.dtype == "f32":
        return A.astype(np.float32)
    return synthetic.to_bf16_bits(A).view(np.int16)


# ----------------------------------------------------------------------------
# CPU oracle (reference arm / cpu_baseline)
# ----------------------------------------------------------------------------
def oracle_sample(w, A, budget_s: float, rng_seed: int = 0):
    """Time the FP64 oracle on a bounded sample of the workload's rows A (as
    the GPU reads them): compress the first blocks until about budget_s/2 has
    passed, then answer queries drawn over the compressed sample for the
    rest.  Returns a dict of rates."""
    import oracle
    cores = os.cpu_count()
    b, n, k = w.b, w.series.n, w.k
    itemsize = {"f64": 8, "f32": 4, "bf16": 2}[w.dtype]
    blocks, nb, tc = [], 0, 0.0
    nb_max = w.series.T // b
    while nb < nb_max and tc < budget_s / 2:
        R = A[nb * b: (nb + 1) * b]
        Ab = synthetic.bf16_bits_to_f64(R.view(np.uint16)) if w.dtype == "bf16" else np.asarray(R, np.float64)
        tb = time.perf_counter()
        blocks.append(oracle.compress_block(Ab, k))   # only the oracle's work is timed
        tc += time.perf_counter() - tb
        nb += 1
    st = oracle.Store(b=b, n=n, k=k, T=nb * b, U=[x[0] for x in blocks], s=[x[1] for x in blocks],
                      Vt=[x[2] for x in blocks])
    T = nb * b
    ts, te = synthetic.queries(T, 10_000, min(w.lmin or 1_000, T), min(w.lmax or T, T), seed=rng_seed)
    t1 = time.perf_counter()
    nq = 0
    while nq < len(ts) and time.perf_counter() - t1 < budget_s / 2:
        oracle.query(st, int(ts[nq]), int(te[nq]))
        nq += 1
    tq = time.perf_counter() - t1
    return {"compress_gbps": nb * b * n * itemsize / max(tc, 1e-9) / 1e9, "blocks": nb,
            "queries_per_s": nq / max(tq, 1e-9), "queries": nq, "cores": cores,
            "compress_s": tc, "query_s": tq}


class SharedRows:
    """The workload's rows (as the GPU reads them) in a shared-memory segment,
    so that the oracle's worker processes read them without copies."""

    def __init__(self, A: np.ndarray, dtype: str):
        from multiprocessing import shared_memory
        self.shm = shared_memory.SharedMemory(create=True, size=max(A.nbytes, 1))
        np.ndarray(A.shape, dtype=A.dtype, buffer=self.shm.buf)[...] = A
        self.spec = (self.shm.name, A.shape, A.dtype.str, dtype)

    def close(self):
        self.shm.close()
        self.shm.unlink()


def _rows_from(spec, r0, r1):
    """Rows [r0, r1) of a SharedRows segment, upcast exactly to FP64."""
    from multiprocessing import shared_memory
    name, shape, dt, kind = spec
    shm = shared_memory.SharedMemory(name=name)
    try:
        A = np.ndarray(shape, dtype=np.dtype(dt), buffer=shm.buf)[r0:r1]
        if kind == "bf16":
            return synthetic.bf16_bits_to_f64(A.view(np.uint16))
        return np.array(A, dtype=np.float64)
    finally:
        shm.close()


def _pool_compress(job):
    """Worker: compress blocks [i0, i1) (b rows each, the last one possibly
    short) with the oracle; returns the factors and the seconds spent in the
    oracle itself."""
    import oracle
    spec, b, k, T, i0, i1 = job
    A = _rows_from(spec, i0 * b, min(i1 * b, T))
    out, t = [], 0.0
    for i in range(i0, i1):
        Ab = A[(i - i0) * b: min((i - i0 + 1) * b, A.shape[0])]
        t0 = time.perf_counter()
        out.append(oracle.compress_block(Ab, k))
        t += time.perf_counter() - t0
    return i0, out, t


def _pool_queries(job):
    """Worker: answer queries with the oracle until `budget` seconds pass."""
    import oracle
    st, ts, te, budget = job
    t0, nq = time.perf_counter(), 0
    while nq < len(ts) and time.perf_counter() - t0 < budget:
        oracle.query(st, int(ts[nq]), int(te[nq]))
        nq += 1
    return nq, time.perf_counter() - t0


def oracle_pool(workers: int, one_thread: bool = True):
    """A process pool (spawn) for the oracle; with one_thread each worker's
    BLAS uses one thread, so the pool's width is the cores used."""
    import multiprocessing as mp
    keep = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    if one_thread:
        for v in keep:
            os.environ[v] = "1"
    try:
        return mp.get_context("spawn").Pool(workers)
    finally:
        for v, x in keep.items():
            if x is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = x


def oracle_compress_all(pool, spec, w, T, workers):
    """Compress every block of the first T rows on the pool; returns (oracle
    store, wall seconds)."""
    import oracle
    nb = (T + w.b - 1) // w.b
    step = max(1, (nb + 4 * workers - 1) // (4 * workers))
    jobs = [(spec, w.b, w.k, T, i, min(i + step, nb)) for i in range(0, nb, step)]
    t0 = time.perf_counter()
    res = sorted(pool.map(_pool_compress, jobs), key=lambda r: r[0])
    wall = time.perf_counter() - t0
    blocks = [x for _, out, _ in res for x in out]
    st = oracle.Store(b=w.b, n=w.series.n, k=w.k, T=T, U=[x[0] for x in blocks], s=[x[1] for x in blocks],
                      Vt=[x[2] for x in blocks])
    return st, wall


def cpu_baseline_sample(spec, w, budget_s: float, cores: int):
    """The oracle as it stands, on this host: storage phase over the first
    blocks and queries over them, on one core and on `cores` cores (a spawn
    pool, one BLAS thread per worker).  Each of the four timings is bounded by
    about budget_s / 4 seconds of CPU work."""
    import oracle
    itemsize = {"f64": 8, "f32": 4, "bf16": 2}[w.dtype]
    b, n, T = w.b, w.series.n, w.series.T
    out = {}
    one = oracle_pool(1)
    try:
        nb, t, blocks = 0, 0.0, []
        while t < budget_s / 4 and nb < T // b:
            _, o, dt = one.map(_pool_compress, [(spec, b, w.k, T, nb, nb + 1)])[0]
            blocks += o
            t += dt
            nb += 1
        out["one_core"] = {"compress_gbps": nb * b * n * itemsize / t / 1e9, "blocks": nb}
        qst = oracle.Store(b=b, n=n, k=w.k, T=nb * b, U=[x[0] for x in blocks], s=[x[1] for x in blocks],
                           Vt=[x[2] for x in blocks])
        ts, te = synthetic.queries(nb * b, 2_000, min(w.lmin or 1_000, nb * b), min(w.lmax or nb * b, nb * b),
                                   seed=3)
        nq, tq = one.map(_pool_queries, [(qst, ts, te, budget_s / 4)])[0]
        out["one_core"].update({"queries_per_s": nq / tq, "queries": nq,
                                "query_lengths": [int(np.min(te - ts + 1)), int(np.max(te - ts + 1))]})
    finally:
        one.close()
    pool = oracle_pool(cores)
    try:
        nb = min(T // b, max(1, out["one_core"]["blocks"]) * cores)
        _, wall = oracle_compress_all(pool, spec, w, nb * b, cores)
        out["all_cores"] = {"compress_gbps": nb * b * n * itemsize / wall / 1e9, "blocks": nb}
        chunks = [(qst, ts[i::cores], te[i::cores], budget_s / 4) for i in range(cores)]
        t0 = time.perf_counter()
        res = pool.map(_pool_queries, chunks)
        wall = time.perf_counter() - t0
        out["all_cores"].update({"queries_per_s": sum(r[0] for r in res) / wall,
                                 "queries": sum(r[0] for r in res)})
    finally:
        pool.close()
    return out


def run_reference(args, w):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    per_step = []
    last = None
    A = _input_rows(w)
    for i in range(args.warmup + args.steps):
        r = oracle_sample(w, A, args.ref_budget, rng_seed=i)
        if i >= args.warmup:
            per_step.append(r)
        last = r
    v = statistics.mean(r["compress_gbps"] for r in per_step)
    sample = (f"per step: oracle compresses the first {last['blocks']} blocks of {w.b}x{w.series.n} "
              f"and answers {last['queries']} queries over them (~{args.ref_budget:.0f} s of CPU)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "T": w.series.T, "n": w.series.n, "b": w.b, "k": w.k,
                       "input_dtype": w.dtype},
            "queries_per_s": statistics.mean(r["queries_per_s"] for r in per_step),
            "cpu_baseline": {"value": v, "unit": "GB/s", "cores": last["cores"], "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def union_rows(ts, te):
    """Rows covered by at least one of the inclusive ranges [ts_i, te_i]."""
    order = np.argsort(ts)
    total, cur_lo, cur_hi = 0, None, None
    for i in order:
        a, z = int(ts[i]), int(te[i])
        if cur_hi is None or a > cur_hi + 1:
            if cur_hi is not None:
                total += cur_hi - cur_lo + 1
            cur_lo, cur_hi = a, z
        else:
            cur_hi = max(cur_hi, z)
    if cur_hi is not None:
        total += cur_hi - cur_lo + 1
    return total


def kernel_text_sha256(path, begin, end):
    """SHA-256 of a kernel's own source text: the slice of `path` from the
    line holding `begin` up to (not including) the one holding `end`."""
    import hashlib
    with open(os.path.join(ROOT, path), encoding="utf-8") as fh:
        text = fh.read()
    a = text.index(begin)
    b = text.index(end, a)
    return hashlib.sha256(text[a:b].encode("utf-8")).hexdigest()


def measured_traffic(name, units_per_launch):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    capture (profiles/lift_tc_traffic.json: bytes per output row, scaled by the
    launch's output rows), or None when no capture covers this kernel or the
    kernel's source text has changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "lift_tc_traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
        cur = kernel_text_sha256(rec["kernel_source"], rec["kernel_begin"], rec["kernel_end"])
    except (OSError, KeyError, ValueError):
        return None
    if rec.get("kernel") != name or rec.get("kernel_source_sha256") != cur:
        return None
    return rec["dram_bytes_per_output_row"] * units_per_launch


def kernel_model(name, w, launches_per_step, nq_total_rows, union_u_rows):
    """Compulsory bytes per launch of a kernel, for the roofline object."""
    itemsize = {"f64": 8, "f32": 4, "bf16": 2}[w.dtype]
    T, n, b, k = w.series.T, w.series.n, w.b, w.k
    if name in ("gram_compress", "form_u", "gram_lo", "project", "sketch", "check"):
        # every input byte read once per launch set
        return "hbm", T * n * itemsize / launches_per_step
    if name == "lift":
        # write every output row (k_out = k floats); read each stored U row
        # that the batch touches once (rows shared by several queries come
        # from L2 after the first read)
        return "hbm", (nq_total_rows * k * 4 + union_u_rows * k * 4) / launches_per_step
    return None, None


def run_gpu(args, w):
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    import paper_1805_00754_gb300 as zs
    from paper_1805_00754_gb300 import zoomsvd

    if args.rows:
        # smaller case of the same workload (profiling captures)
        import dataclasses
        w = dataclasses.replace(w, series=dataclasses.replace(w.series, T=args.rows))
    T, n, b, k = w.series.T, w.series.n, w.b, w.k
    itemsize = {"f64": 8, "f32": 4, "bf16": 2}[w.dtype]
    A = _input_rows(w)
    rows_dev = torch.from_numpy(A).to(f"cuda:{local}")
    in_bytes = T * n * itemsize
    if w.single_query is not None and args.nq is None:
        # the plain workload's one query (t_s, t_e)
        ts = np.array([w.single_query[0]], dtype=np.int64)
        te = np.array([w.single_query[1]], dtype=np.int64)
    else:
        nq = args.nq if args.nq is not None else w.nq
        ts, te = synthetic.queries(T, nq, w.lmin, w.lmax, seed=synthetic.SEED_BASE + 99)
    nq = len(ts)
    st = zs.Store(n=n, b=b, k=k, dtype=w.dtype, capacity_rows=T, device=local,
                  fp64_refine=(w.dtype == "bf16"))
    outs = [st.new_result(int(a), int(z), k) for a, z in zip(ts, te)]
    out_rows = int(np.sum(te - ts + 1))
    stream = torch.cuda.current_stream()

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]

    def step(e=None):
        st.reset()
        if e:
            e[0].record(stream)
        st.append(rows_dev)
        if e:
            e[1].record(stream)
        if nq:
            st.query_batch(ts, te, k, outs=outs)
        if e:
            e[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    zoomsvd.profile(True)
    zoomsvd.profile_reset()
    clocks = Clocks(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = zs.launch_count()
    for i in range(args.steps):
        step(ev[i])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = zs.launch_count() - l0
    clk = clocks.stop()
    table = zoomsvd.profile_table()
    zoomsvd.profile(False)
    tc = sum(e[0].elapsed_time(e[1]) for e in ev) / 1e3
    tq = sum(e[1].elapsed_time(e[2]) for e in ev) / 1e3
    tc, tq = reduce_max([tc, tq], f"cuda:{local}")
    K = args.steps
    compress_gbps = aggregate_rate(ws, K, in_bytes, tc) / 1e9
    qps = aggregate_rate(ws, K, nq, tq) if nq else None
    ms_step = (tc + tq) / K * 1e3

    status = st.status_counts(check=False)

    # the same batch with U left factored (Sigma, V and per-block coefficients)
    qps_fac = None
    if nq:
        fac = st.query_batch_factored(ts, te, k)          # warm (allocation, first launches)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(K):
            st.query_batch_factored(ts, te, k, out=fac)
        f1.record(stream)
        torch.cuda.synchronize()
        (tf,) = reduce_max([f0.elapsed_time(f1) / 1e3], f"cuda:{local}")
        qps_fac = aggregate_rate(ws, K, nq, tf)
        del fac

    # e2e through the C ABI from pinned host rows (H2D inside the timed region)
    e2e = None
    if not args.no_e2e:
        host = torch.from_numpy(A).pin_memory()
        sig_host = torch.empty((k,), dtype=st.fdtype).pin_memory()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        te2e = 0.0
        for i in range(args.warmup + K):
            st.reset()
            torch.cuda.synchronize()
            e0.record(stream)
            st.append(host)
            _, s_dev, _, _ = st.export_block((T - 1) // b)
            sig_host.copy_(s_dev, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            if i >= args.warmup:
                te2e += e0.elapsed_time(e1) / 1e3
        (te2e,) = reduce_max([te2e], f"cuda:{local}")
        # a plain pinned host -> device copy of the same bytes on this machine (best of 3)
        scratch = torch.empty_like(rows_dev)
        best = None
        for _ in range(3):
            e0.record(stream)
            scratch.copy_(host, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        del scratch
        e2e = {"value": aggregate_rate(ws, K, in_bytes, te2e) / 1e9, "unit": "GB/s",
               "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": k * (8 if w.dtype == "f64" else 4),
               "pinned_h2d_copy_gbps": in_bytes / (best / 1e3) / 1e9}

    # roofline of the dominant kernel
    peaks, src = _peaks()
    dom = max(table.items(), key=lambda kv: kv[1][1]) if table else None
    roof = None
    if dom:
        name, (nl, ms) = dom
        per_step = nl / K
        bound, units = kernel_model(name, w, per_step, out_rows, union_rows(ts, te))
        avg_s = ms / nl / 1e3
        if bound == "hbm":
            ach = units / avg_s / 1e9
            roof = {"kernel": name, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / peaks["hbm_gbs"], "traffic": measured_traffic(name, out_rows / per_step),
                    "peak_source": src, "avg_launch_ms": avg_s * 1e3, "launches_per_step": per_step}
        else:
            roof = {"kernel": name, "bound": "alu", "achieved": None, "peak": None, "unit": None, "frac": None,
                    "traffic": None, "avg_launch_ms": avg_s * 1e3, "launches_per_step": per_step}
    kernels = {nm: {"launches": v[0], "ms_per_step": v[1] / K} for nm, v in table.items()}

    # Theorem 3: the stored factors against the raw rows
    _, nblk, fbytes = st.info()
    space = {"factor_bytes": fbytes, "raw_bytes": in_bytes, "ratio": fbytes / in_bytes,
             "per_block": f"b*k + k + k*n = {b * k + k + k * n} factor elements"}

    plain32 = None
    if rank == 0 and not args.skip_plain and nq:
        plain32 = plain_fp32_run(st, ts, te, k)
    acc = None
    cpu = None
    if rank == 0 and (not args.skip_accuracy or not args.skip_cpu):
        cores = os.cpu_count() or 1
        shared = SharedRows(A, w.dtype)
        try:
            if not args.skip_accuracy and nq:
                pool = oracle_pool(cores)
                try:
                    ost, _ = oracle_compress_all(pool, shared.spec, w, T, cores)
                finally:
                    pool.close()
                acc = accuracy_sample(st, w, ost)
                del ost
            r = cpu_baseline_sample(shared.spec, w, args.cpu_budget, cores) if (not args.skip_cpu and ws == 1) \
                else None
        finally:
            shared.close()
        if r is not None:
            cpu = {"value": r["all_cores"]["compress_gbps"], "unit": "GB/s", "cores": cores, "kind": "oracle",
                   "sample": (f"oracle storage phase over the first {r['all_cores']['blocks']} blocks on {cores} "
                              f"worker processes (one BLAS thread each) and over {r['one_core']['blocks']} blocks "
                              f"on one; queries log-uniform over the compressed rows; "
                              f"~{args.cpu_budget:.0f} s of CPU in all"),
                   "one_core": r["one_core"], "all_cores": r["all_cores"]}
    plain = None
    if rank == 0 and not args.skip_plain and nq:
        st.close()
        del rows_dev
        torch.cuda.empty_cache()
        plain = plain_fp64_run(w, A, ts, te, local)
    rowapp = None
    if rank == 0 and not args.skip_row_append:
        rowapp = row_append_run(w, A, local)
    serving = None
    if args.serve_seconds > 0 and rank == 0:
        serving = serve_run(args.serve_seconds, local, warmup=args.serve_warmup)
    if rank == 0:
        line = {"metric": METRIC, "value": compress_gbps, "unit": "GB/s", "n_gpus": ws, "steps": K,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": {"f64": "f64", "f32": "f32", "bf16": "bf16-in/f32"}[w.dtype],
                "data": "synthetic",
                "config": {"workload": w.name, "T": T, "n": n, "b": b, "k": k, "input_dtype": w.dtype,
                           "queries_per_step": nq, "query_rows_per_step": out_rows,
                           "l2": "inputs larger than L2 (no flush needed)",
                           "parallelism": f"replicas x{ws}"},
                "queries_per_s": qps, "queries_per_s_factored": qps_fac,
                "compress_s_per_step": tc / K, "query_s_per_step": tq / K,
                "hbm_frac_compress": compress_gbps / ws / peaks["hbm_gbs"], "space": space,
                "accuracy_test": {"unconverged_blocks": status[0], "unconverged_queries": status[1],
                                  "refined_blocks": status[2], "refined_queries": status[3]},
                "accuracy": acc, "serving": serving, "row_append": rowapp,
                "plain_fp32_gpu": plain32,
                "queries_per_s_vs_plain_fp32": (qps / plain32["queries_per_s"]) if (plain32 and qps) else None,
                "plain_fp64_gpu": plain,
                "queries_per_s_vs_plain_fp64": (qps / plain["queries_per_s"]) if (plain and qps) else None,
                "comparisons": "vs_plain_fp32: equal precision (the same FP32 store, one query per call); "
                               "vs_plain_fp64: unequal precision (FP32 batched, sigma error <= 1e-4, against "
                               "FP64 one query per call, sigma error ~1e-15)",
                "roofline": roof, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk}
        print(json.dumps(line), flush=True)
    if plain is None:
        st.close()
    if dist:
        dist.destroy_process_group()


SWEEP_B = (64, 128, 256, 512, 1_024, 2_048, 4_096, 8_192, 16_384, 65_536)
SWEEP_LEN = (1_000, 10_000, 100_000)


def sweep_batch_size(L, b, k, n, itemsize=4, cap=256, budget=2 << 30):
    """Queries per timed batch of length-L ranges: at most `cap`, and few
    enough that the stacked matrices ((L / b + 2) slabs of k x n each per
    query) stay within `budget` bytes."""
    per_query = (L // b + 2) * k * n * itemsize
    return int(max(1, min(cap, budget // per_query)))


def run_sweep_b(args, w):
    """Block-size sweep (the trade-off of Fig. 7 on the synthetic workload).
    For each b: the time to compress the whole matrix (CUDA events, inputs in
    HBM), the bytes the store keeps (Theorem 3) and queries/s for batches of
    fixed-length ranges L = 1e3, 1e4, 1e5 (U materialised).  One JSON line."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1805_00754_gb300 as zs

    T, n, k = w.series.T, w.series.n, w.k
    itemsize = {"f64": 8, "f32": 4, "bf16": 2}[w.dtype]
    rows_dev = torch.from_numpy(_input_rows(w)).cuda()
    stream = torch.cuda.current_stream()
    points = []
    for b in SWEEP_B:
        st = zs.Store(n=n, b=b, k=k, dtype=w.dtype, capacity_rows=T)
        st.append(rows_dev)                      # warm-up (allocations, first launches)
        torch.cuda.synchronize()
        st.reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st.append(rows_dev)
        e1.record(stream)
        torch.cuda.synchronize()
        comp_ms = e0.elapsed_time(e1)
        _, nblk, fbytes = st.info()
        qps = {}
        for L in SWEEP_LEN:
            nq = sweep_batch_size(L, b, k, n)
            ts, te = synthetic.queries(T, nq, L, L, seed=synthetic.SEED_BASE + 7 + L)
            outs = [st.new_result(int(a), int(z), k) for a, z in zip(ts, te)]
            st.query_batch(ts, te, k, outs)      # warm-up
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(3):
                st.query_batch(ts, te, k, outs)
            e1.record(stream)
            torch.cuda.synchronize()
            qps[str(L)] = 3 * nq / (e0.elapsed_time(e1) / 1e3)
            del outs
        assert st.fault() == 0
        points.append({"b": b, "blocks": nblk, "compress_ms": comp_ms,
                       "compress_gbs": T * n * itemsize / comp_ms / 1e6, "factor_bytes": fbytes,
                       "space_vs_raw": fbytes / (T * n * itemsize), "queries_per_s": qps})
        st.close()
        torch.cuda.empty_cache()
    print(json.dumps({"sweep": "block_size", "workload": w.name, "T": T, "n": n, "k": k,
                      "dtype": w.dtype, "lengths": list(SWEEP_LEN), "points": points}))


SWEEP_XI = (0.95, 0.98, 0.99)


def run_sweep_xi(args, w, kcap=32, nq_err=8):
    """Energy-rule sweep (Eq. 1; Fig. 6 of Section 5.4 on the synthetic
    workload): for xi = 0.95, 0.98, 0.99 (ranks capped at kcap) and for the
    workload's fixed rank, the per-block ranks k_i, the space the store keeps
    (Theorem 3: sum k_i (b + n + 1) values against T n raw values), the stored
    blocks' relative squared reconstruction error, the same error of query
    results against the raw rows (nq_err ranges of the bench's lengths), the
    compression time and queries/s of the bench's batch.  One JSON line."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1805_00754_gb300 as zs
    T, n, b = w.series.T, w.series.n, w.b
    itemsize = {"f64": 8, "f32": 4, "bf16": 2}[w.dtype]
    A = _input_rows(w)
    rows_dev = torch.from_numpy(A).cuda()
    A64 = synthetic.bf16_bits_to_f64(A.view(np.uint16)) if w.dtype == "bf16" else None
    stream = torch.cuda.current_stream()
    ts, te = synthetic.queries(T, w.nq or 256, w.lmin or 1_000, w.lmax or T, seed=synthetic.SEED_BASE + 99)
    qa, qz = synthetic.queries(T, nq_err, w.lmin or 1_000, w.lmax or T, seed=synthetic.SEED_BASE + 97)
    points = []
    for xi in (None,) + SWEEP_XI:
        k = w.k if xi is None else kcap
        st = zs.Store(n=n, b=b, k=k, dtype=w.dtype, capacity_rows=T, xi=xi, fp64_refine=(w.dtype == "bf16"))
        st.append(rows_dev)
        torch.cuda.synchronize()
        st.reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st.append(rows_dev)
        e1.record(stream)
        torch.cuda.synchronize()
        comp_ms = e0.elapsed_time(e1)
        ranks, kept, en = st.block_stats()
        if xi is None:
            en = np.array([np.sum((A64 if A64 is not None else A)[i * b:(i + 1) * b].astype(np.float64) ** 2)
                           for i in range(len(ranks))])
        kq = w.k          # queries ask for the workload's rank whatever the blocks keep
        outs = [st.new_result(int(a), int(z), kq) for a, z in zip(ts, te)]
        st.query_batch(ts, te, kq, outs)
        torch.cuda.synchronize()
        e0.record(stream)
        st.query_batch(ts, te, kq, outs)
        e1.record(stream)
        torch.cuda.synchronize()
        qps = len(ts) / (e0.elapsed_time(e1) / 1e3)
        del outs
        qerr = []
        for a, z in zip(qa, qz):
            o = st.query(int(a), int(z), kq)
            torch.cuda.synchronize()
            U, S, V = (x.cpu().numpy().astype(np.float64) for x in (o.U, o.S, o.V))
            X = (A64 if A64 is not None else A)[int(a):int(z) + 1].astype(np.float64)
            R = X - (U * S[None, :]) @ V.T
            qerr.append(float(np.sum(R * R) / np.sum(X * X)))
        status = st.status_counts(check=False)
        points.append({"xi": xi, "k_cap": k, "k_i_min": int(ranks.min()), "k_i_mean": float(ranks.mean()),
                       "k_i_max": int(ranks.max()), "space_values": int(np.sum(ranks) * (b + n + 1)),
                       "space_vs_raw": float(np.sum(ranks) * (b + n + 1) / (T * n)),
                       "store_recon_err": float(1.0 - np.sum(kept) / np.sum(en)),
                       "query_recon_err_mean": float(np.mean(qerr)), "query_recon_err_max": float(np.max(qerr)),
                       "compress_ms": comp_ms, "compress_gbs": T * n * itemsize / comp_ms / 1e6,
                       "queries_per_s": qps, "unconverged": [status[0], status[1]]})
        st.close()
        torch.cuda.empty_cache()
    print(json.dumps({"sweep": "xi", "workload": w.name, "T": T, "n": n, "b": b, "dtype": w.dtype,
                      "query_lengths": [int(np.min(te - ts + 1)), int(np.max(te - ts + 1))], "points": points}))


def plain_fp64_run(w, A, ts, te, local, budget_s=4.0, acc_queries=3):
    """The same range-SVD method as a plain FP64 GPU program, one query at a
    time: an FP64 store of the same rows (FP64 CUDA-core kernels throughout),
    each query answered by its own zs_query call and synchronised before the
    next - no batching, no mixed precision.  Queries are taken in the batch's
    order until budget_s has passed."""
    import oracle
    import torch
    import paper_1805_00754_gb300 as zs
    T, n, b, k = w.series.T, w.series.n, w.b, w.k
    if w.dtype == "bf16":
        A64 = synthetic.bf16_bits_to_f64(np.asarray(A).view(np.uint16))
    else:
        A64 = np.asarray(A, dtype=np.float64)
    dev = torch.from_numpy(A64).to(f"cuda:{local}")
    st = zs.Store(n=n, b=b, k=k, dtype="f64", capacity_rows=T, device=local)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st.append(dev)
    torch.cuda.synchronize()
    tc = time.perf_counter() - t0
    del dev
    lmax = int(np.max(te - ts + 1))
    out = st.new_result(0, lmax - 1, k)
    st.query(int(ts[0]), int(te[0]), out=out)            # warm-up (first launch, plan buffers)
    torch.cuda.synchronize()
    nq, t1 = 0, time.perf_counter()
    while nq < len(ts) and time.perf_counter() - t1 < budget_s:
        st.query(int(ts[nq]), int(te[nq]), out=out)
        torch.cuda.synchronize()
        nq += 1
    tq = time.perf_counter() - t1
    # accuracy of a few short ranges against the oracle, as for the batched form
    worst = 0.0
    qa, qz = synthetic.queries(T, acc_queries, 2 * b, 20_000, seed=7)
    for a, z in zip(qa, qz):
        S, E = int(a) // b, int(z) // b
        ost = oracle.compress(A64[S * b: min((E + 1) * b, T)], b, k)
        ref = oracle.query(ost, int(a) - S * b, int(z) - S * b)
        o = st.query(int(a), int(z))
        torch.cuda.synchronize()
        s_ = o.S.cpu().numpy()
        msk = ref.s > 0
        worst = max(worst, float(np.max(np.abs(s_[msk] - ref.s[msk]) / ref.s[msk])))
    st.close()
    itemsize = {"f64": 8, "f32": 4, "bf16": 2}[w.dtype]
    return {"form": "FP64 store and kernels, one zs_query call per query, synchronised", "queries": nq,
            "queries_per_s": nq / max(tq, 1e-9), "compress_s": tc,
            "compress_gbps_of_input": T * n * itemsize / tc / 1e9, "sigma_max_rel_err": worst}


def accuracy_sample(st, w, ost, nq=8, seed=synthetic.SEED_BASE + 98):
    """Errors of GPU query results against the FP64 oracle run on the same
    (dtype-rounded) rows, at the bench's own range lengths (nq ranges drawn
    like the timed batch).  Per query: the worst relative error of sigma, the
    sine of the largest principal angle between the device's and the
    oracle's V, the truncation gap sigma_k / sigma_k+1 of the range (oracle),
    and the Wedin bound sqrt(2) |R|_F / (sigma_k - sigma_k+1) on that angle
    implied by the device pairs' residuals R against the oracle's range."""
    import oracle
    import torch
    T, b, k = w.series.T, w.b, w.k
    ts, te = synthetic.queries(T, nq, w.lmin or 1_000, w.lmax or T, seed=seed)
    per, worst_s, worst_sin = [], 0.0, 0.0
    for a, z in zip(ts, te):
        a, z = int(a), int(z)
        ref = oracle.query(ost, a, z)
        out = st.query(a, z)
        torch.cuda.synchronize()
        s = out.S.cpu().numpy().astype(np.float64)
        U = out.U.cpu().numpy().astype(np.float64)
        V = out.V.cpu().numpy().astype(np.float64)
        m = ref.s > 0
        es = float(np.max(np.abs(s[m] - ref.s[m]) / ref.s[m]))
        Q1, _ = np.linalg.qr(V[:, m])
        Q2, _ = np.linalg.qr(ref.V[:, m])
        sin = float(np.linalg.norm(Q2 - Q1 @ (Q1.T @ Q2), 2))
        # residuals against the oracle's range matrix and its full spectrum
        r = int(np.sum(m))
        AtU = np.zeros((w.series.n, r))
        AV = np.zeros((z - a + 1, r))
        G = np.zeros((w.series.n, w.series.n))
        for i in range(a // b, z // b + 1):
            lo = i * b
            Ai = (ost.U[i][max(a, lo) - lo: min(z + 1, lo + b) - lo] * ost.s[i][None, :]) @ ost.Vt[i]
            AtU += Ai.T @ U[max(a, lo) - a: min(z + 1, lo + b) - a, :r]
            AV[max(a, lo) - a: min(z + 1, lo + b) - a] = Ai @ V[:, :r]
            G += Ai.T @ Ai
        full = np.sqrt(np.maximum(np.linalg.eigvalsh(G)[::-1], 0.0))
        R2 = np.sum((AtU - V[:, :r] * s[None, :r]) ** 2) + np.sum((AV - U[:, :r] * s[None, :r]) ** 2)
        gap = full[r - 1] - full[r] if full.size > r else full[r - 1]
        wedin = float(np.sqrt(2.0 * R2) / gap) if gap > 0 else None
        per.append({"rows": z - a + 1, "sigma_rel_err": es, "v_sin": sin,
                    "gap_k": float(full[r - 1] / full[r]) if full.size > r and full[r] > 0 else None,
                    "wedin_bound": wedin})
        worst_s, worst_sin = max(worst_s, es), max(worst_sin, sin)
    return {"sigma_max_rel_err": worst_s, "v_subspace_sin_max": worst_sin, "queries": int(nq),
            "lengths": [int(np.min(te - ts + 1)), int(np.max(te - ts + 1))],
            "vs": "FP64 oracle on the same rounded rows", "per_query": per}


def plain_fp32_run(st, ts, te, k, budget_s=2.0):
    """The batched form's own FP32 store, one zs_query call per query,
    synchronised before the next: the same precision as the batch, no
    batching, no graphs."""
    import torch
    lmax = int(np.max(te - ts + 1))
    out = st.new_result(0, lmax - 1, k)
    st.query(int(ts[0]), int(te[0]), out=out)
    torch.cuda.synchronize()
    nq, t0 = 0, time.perf_counter()
    while nq < len(ts) and time.perf_counter() - t0 < budget_s:
        st.query(int(ts[nq]), int(te[nq]), out=out)
        torch.cuda.synchronize()
        nq += 1
    return {"form": "the same FP32 store, one zs_query call per query, synchronised", "queries": nq,
            "queries_per_s": nq / (time.perf_counter() - t0)}


def row_append_run(w, A, local, rows_timed: int = 256, bulk_blocks: int = 304):
    """Row-by-row storage (Algorithm 1 with truncation after every row) on the
    workload's shape: the latency of one appended row (one call per row,
    device rows, CUDA events on the caller's stream; the open block already
    holds b/2 rows, so U carries b/2 .. b/2 + rows_timed rows), and the
    throughput of folding bulk_blocks whole blocks in one call (one CTA per
    block, rows in order within each)."""
    import torch
    from paper_1805_00754_gb300 import Store
    n, b, k = w.series.n, w.b, w.k
    itemsize = {"f64": 8, "f32": 4, "bf16": 2}[w.dtype]
    nb = min(bulk_blocks, A.shape[0] // b)
    dev = torch.from_numpy(A[: nb * b]).to(f"cuda:{local}")
    st = Store(n=n, b=b, k=k, dtype=w.dtype, capacity_rows=nb * b, device=local, row_append=True)
    stream = torch.cuda.current_stream()
    try:
        half = b // 2
        st.append(dev[:half])
        torch.cuda.synchronize()
        R = min(rows_timed, b - half)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(R + 1)]
        ev[0].record(stream)
        for r in range(R):
            st.append(dev[half + r: half + r + 1])
            ev[r + 1].record(stream)
        torch.cuda.synchronize()
        lat = np.array([ev[r].elapsed_time(ev[r + 1]) * 1e3 for r in range(R)])
        st.reset()
        st.append(dev[:b])                          # warm
        torch.cuda.synchronize()
        st.reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st.append(dev)
        e1.record(stream)
        torch.cuda.synchronize()
        tb = e0.elapsed_time(e1) / 1e3
    finally:
        st.close()
    return {"per_row_us_mean": float(lat.mean()), "per_row_us_median": float(np.median(lat)),
            "per_row_us_p99": float(np.percentile(lat, 99)), "rows_timed": int(R),
            "open_block_rows_at_start": int(half),
            "bulk_blocks": int(nb), "bulk_rows_per_s": nb * b / tb, "bulk_gbps": nb * b * n * itemsize / tb / 1e9,
            "mode": "one zs_store_append call per row (device rows, one kernel each); bulk: one call, "
                    "one CTA per block"}


def serve_run(seconds: float, local: int, rate_hz: float = 20_000.0, warmup: float = 1.0):
    """Serving workload: compressed store of the serving shape, Poisson
    arrivals at rate_hz with lengths log-uniform 1e3..1e6, new blocks
    appended at 1 block/ms on another stream while queries run.  A first
    server runs `warmup` seconds of arrivals (its statistics are dropped);
    a fresh server then runs `seconds`, which are reported."""
    import torch
    import paper_1805_00754_gb300 as zs
    w = synthetic.WORKLOADS["serving_f32"]
    T, n, b, k = w.series.T, w.series.n, w.b, w.k
    extra = int((seconds + warmup) * 1000) + 32            # blocks appended during both phases
    A = synthetic.rows(w.series, dtype=np.float32)
    app = synthetic.rows(synthetic.SeriesSpec(extra * b, n, w.series.s, w.series.noise, 0.0,
                                              w.series.seed + 1), dtype=np.float32)
    st = zs.Store(n=n, b=b, k=k, dtype="f32", capacity_rows=T + extra * b, device=local)
    st.append(torch.from_numpy(A).to(f"cuda:{local}"))
    app_dev = torch.from_numpy(app).to(f"cuda:{local}")
    torch.cuda.synchronize()
    # results go to a ring arena (never read back); a slot is reused only after
    # its previous request completed
    arena_rows = 256 << 20
    arena = torch.empty((arena_rows, k), dtype=torch.float32, device=f"cuda:{local}")
    SV = torch.empty((4096, k), dtype=torch.float32, device=f"cuda:{local}")
    VV = torch.empty((4096, n, k), dtype=torch.float32, device=f"cuda:{local}")
    from paper_1805_00754_gb300 import zoomsvd
    import ctypes as C
    app_stream = torch.cuda.Stream(device=f"cuda:{local}")
    lib = zoomsvd.lib()
    state = {"appended": 0}

    def phase(dur, seed):
        sv = zs.Server(st, max_batch=512, max_inflight=3, queue_capacity=1 << 16, memory_budget=8 << 30)
        arrivals = synthetic.poisson_arrivals(rate_hz, dur, seed=seed)
        ts, te = synthetic.queries(T, len(arrivals), w.lmin, w.lmax, seed=seed + 1)
        stop = threading.Event()

        def appender():
            t0 = time.perf_counter()
            i = 0
            while not stop.is_set() and state["appended"] < extra:
                j = state["appended"]
                st.append(app_dev[j * b:(j + 1) * b], stream=app_stream)
                state["appended"] += 1
                i += 1
                d = t0 + i * 1e-3 - time.perf_counter()
                if d > 0:
                    time.sleep(d)

        th = threading.Thread(target=appender)
        pending, off = [], 0
        tick = C.c_uint64()
        arena_p, sv_p, vv_p = arena.data_ptr(), SV.data_ptr(), VV.data_ptr()
        t_start = time.perf_counter()
        th.start()
        for i, t_arr in enumerate(arrivals):
            d = t_start + t_arr - time.perf_counter()
            if d > 0:
                time.sleep(d)
            L = int(te[i] - ts[i] + 1)
            if off + L > arena_rows:
                off = 0
            res = zoomsvd.Result(arena_p + off * k * 4, k, sv_p + (i % 4096) * k * 4,
                                 vv_p + (i % 4096) * n * k * 4, k, 0)
            off += L
            if lib.zs_serve_submit(sv._h, int(ts[i]), int(te[i]), k, C.byref(res), C.byref(tick)) == 0:
                pending.append(tick.value)
        for t in pending:
            sv.wait(t, 120_000)
        stop.set()
        th.join()
        return sv.stop()

    if warmup > 0:
        phase(warmup, synthetic.SEED_BASE + 15)
    stats = phase(seconds, synthetic.SEED_BASE + 5)
    status = st.status_counts(check=False)
    st.close()
    return {"workload": "serving_f32", "offered_qps": rate_hz, "seconds": seconds, "warmup_s": warmup,
            "completed": stats["completed"], "rejected": stats["rejected"],
            "queries_per_s": stats["queries_per_s"], "p50_ms": stats["p50_ms"], "p99_ms": stats["p99_ms"],
            "max_ms": stats["max_ms"], "mean_batch": stats["mean_batch"], "appends_per_s": 1000.0,
            "unconverged": [status[0], status[1]]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="compress_f32", choices=sorted(synthetic.WORKLOADS))
    ap.add_argument("--nq", type=int, default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--ref-budget", type=float, default=6.0)
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-warmup", type=float, default=1.0)
    ap.add_argument("--skip-accuracy", action="store_true")
    ap.add_argument("--skip-row-append", action="store_true", help="skip the row-by-row storage measurement")
    ap.add_argument("--skip-plain", action="store_true", help="skip the one-query-at-a-time FP64 GPU form")
    ap.add_argument("--rows", type=int, default=0, help="use the first ROWS rows (profiling small cases)")
    ap.add_argument("--sweep-b", action="store_true",
                    help="block-size sweep (compression time, space, queries/s at 1e3/1e4/1e5 rows)")
    ap.add_argument("--sweep-xi", action="store_true",
                    help="energy-rule sweep xi = 0.95/0.98/0.99 (ranks, space, reconstruction error, rates)")
    args = ap.parse_args()
    w = synthetic.WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, w)
    elif args.sweep_b:
        run_sweep_b(args, w)
    elif args.sweep_xi:
        run_sweep_xi(args, w)
    else:
        run_gpu(args, w)


if __name__ == "__main__":
    main()
