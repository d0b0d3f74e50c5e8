"""Benchmark of the SNN hot path on one GB300 (or N independent replicas).

One step = the whole path on one synthetic batch: index build (Algorithm 1:
mean, Gram, first direction, scores, radix sort, gather) and the exact
self-join radius query (Algorithm 2: bands, scoring, FP64 decision, CSR).
Workload: the 50-cluster anisotropic mixture, n = 1,000,000 points in d = 16,
every point a query, R for ~50 neighbours per point.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
(FP64 brute force) on a bounded query sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import contextlib
import gc
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max clock
HBM_PEAK_FALLBACK = 6800.0


# DRAM bytes of one scorer launch at full size, from one-pass ncu counters
# (profiles/k_score_tc_dram_traffic_full_size.md), valid only for the scorer
# sources they were taken with (hash below); any other build reports null.
SCORER_SOURCES = ["tc_score.cu", "tc_score.cuh", "tc_common.cuh", "common.cuh", "index_struct.cuh",
                  "query_kernels.cuh"]
SCORER_TRAFFIC = {
    "sha": "4adb7edb29bdea29",
    "profile": "profiles/k_score_tc_dram_traffic_full_size.md",
    ("gmm_aniso", 1000000, "bf16"): 193561088 + 172464896,
    ("lowrank_img", 70000, "bf16"): 299913472 + 7792384,
}


def scorer_traffic(workload: str, n: int, precision: str):
    import hashlib
    h = hashlib.sha256()
    for f in SCORER_SOURCES:
        with open(os.path.join(ROOT, "paper_2212_07679_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != SCORER_TRAFFIC["sha"]:
        return None
    return SCORER_TRAFFIC.get((workload, n, precision))


@contextlib.contextmanager
def no_gc():
    """Python's cyclic garbage collector off inside a timed region (as timeit
    does): a full collection of the interpreter's objects can stall the host
    for tens of milliseconds, which would be charged to whichever step it
    lands in."""
    gc.collect()
    gc.disable()
    try:
        yield
    finally:
        gc.enable()


SPLIT_NAMES = {0: "none", 1: "bf16x2", 2: "bf16x3", 3: "fp16x2", 4: "fp16x1", 13: "e4m3x2 (3 products)",
               14: "e4m3x2 (4 products)", 16: "e4m3x3 (6 products)"}


def split_name(code: int) -> str:
    return SPLIT_NAMES.get(int(code), str(code))


def split_dtype(code: int) -> str:
    """Arithmetic the step computes in: the scorer's operand type (with its
    BF16 folded columns), FP32 accumulation and decisions, FP64 fallback."""
    code = int(code)
    if code in (3, 4):
        return "f16+bf16+f32+f64"
    if code in (1, 2):
        return "bf16+f32+f64"
    if code >= 10:
        return "e4m3+bf16+f32+f64"
    return "f32+f64"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": HBM_PEAK_FALLBACK, "bf16_tflops": 1900.0,
                "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(args):
    from paper_2212_07679_gb300 import workloads as wl
    if args.workload == "gmm_aniso":
        return wl.gmm_aniso(n=args.n) if args.n else wl.gmm_aniso()
    if args.workload == "lowrank_img":
        return wl.lowrank_img(n=args.n) if args.n else wl.lowrank_img()
    if args.workload == "blobs3d":
        return wl.blobs3d(n=args.n) if args.n else wl.blobs3d()
    if args.workload == "glove_like":
        return wl.glove_like(n=args.n) if args.n else wl.glove_like()
    if args.workload == "gmm_aniso_oos":
        n = args.n or 1_000_000
        return wl.gmm_aniso(n=n, queries=n)
    raise SystemExit(f"unknown workload {args.workload}")


def job_max_ms(local_ms: float, world: int) -> float:
    """The job's time: the largest of the ranks' timed totals (an all-reduce
    MAX over the process group; on the device for NCCL, on the host for gloo)."""
    if world <= 1:
        return float(local_ms)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, ms_step: float) -> float:
    """Units all ranks processed per second (replicas: each rank runs the whole
    workload, so the job processes world x units per step)."""
    return world * units_per_rank / (ms_step / 1e3)


def is_cosine(w):
    return w.extra.get("measure") == "cosine distance"


def workload_config(args, w, extra=None):
    kind = "self-join" if w.Q is None else "out-of-sample queries"
    cfg = {"workload": f"{w.name} {kind}", "n": w.n, "d": w.d, "queries": w.m,
           "R": w.R, "precision": args.precision, "parallelism": f"replicas{args.gpus}",
           "l2": "flushed between steps (256 MiB write)"}
    if is_cosine(w):
        cfg["workload"] = f"{w.name} cosine self-join (rows normalised inside the step)"
        cfg["cosine_distance_bound"] = w.R
        cfg["R"] = math.sqrt(2.0 * w.R)
    if extra:
        cfg.update(extra)
    return cfg


def cpu_oracle_sample(w, budget_s=15.0, seed=7, gpu_csr=None):
    """Times the FP64 brute-force oracle on a bounded random query sample.

    With ``gpu_csr`` = (offsets, indices, dist2) host arrays of the GPU
    result, the sampled rows are also compared with the oracle's: neighbour
    sets (must be identical) and the largest relative dist2 error."""
    import oracle
    rng = np.random.default_rng(seed)
    order = rng.permutation(w.m)
    P, R = w.P, w.R
    if is_cosine(w):
        # the Euclidean search on the oracle's normalised rows
        P, R = oracle.normalize_rows(w.P), oracle.radius_for_cosine_distance(w.R)
    Qall = P if w.Q is None else w.Q
    done, t_used, size = 0, 0.0, 16
    mism, max_rel, checked_pairs = 0, 0.0, 0
    while t_used < budget_s and done < w.m:
        rows = order[done:done + size]
        t0 = time.perf_counter()
        ref = oracle.brute_radius(P, Qall[rows], R)
        dt = time.perf_counter() - t0
        t_used += dt
        done += len(rows)
        if gpu_csr is not None:
            off, ids, d2 = gpu_csr
            for k, r in enumerate(rows):
                a, b = ref.offsets[k], ref.offsets[k + 1]
                ga, gb = off[r], off[r + 1]
                if gb - ga != b - a or not np.array_equal(ids[ga:gb], ref.ids[a:b]):
                    mism += 1
                    continue
                s_ref = ref.dist2[a:b].astype(np.float64)
                s_gpu = d2[ga:gb].astype(np.float64)
                rel = np.abs(s_gpu - s_ref) / np.maximum(s_ref, 1e-300)
                rel[(s_ref == 0) & (s_gpu == 0)] = 0.0
                if rel.size:
                    max_rel = max(max_rel, float(rel.max()))
                checked_pairs += b - a
        if dt < budget_s / 8:
            size *= 2
    out = {"value": done / t_used, "unit": "queries/s", "cores": oracle.oracle_threads(),
           "kind": "oracle",
           "sample": f"{done} random queries of the {w.m} against all {w.n} points "
                     f"(FP64 brute force, {t_used:.1f} s)"}
    if gpu_csr is not None:
        out["parity"] = {"rows": int(done), "pairs": int(checked_pairs),
                         "rows_with_different_sets": int(mism), "max_rel_dist2_err": max_rel}
    return out


def cpu_snn_sample(w, budget_s=8.0, seed=11, gpu_csr=None):
    """Times the paper's own method on the CPU: the oracle's plain SNN
    (Algorithms 1 and 2 in FP64 numpy, one query at a time as in Section 3.2)
    -- the full index build, then queries in random order for about
    ``budget_s`` seconds.  Query work is numpy elementwise code on one core;
    the build's SVD may use the BLAS threads.  With ``gpu_csr`` the sampled
    rows are compared with the GPU result."""
    import oracle
    P, R = w.P, w.R
    if is_cosine(w):
        P, R = oracle.normalize_rows(w.P), oracle.radius_for_cosine_distance(w.R)
    Qall = P if w.Q is None else w.Q
    t0 = time.perf_counter()
    idx = oracle.snn_index(P)
    t_index = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    order = rng.permutation(w.m)
    done, mism, t_used = 0, 0, 0.0
    while t_used < budget_s and done < w.m:
        r = int(order[done])
        t0 = time.perf_counter()
        ids, _, _, _ = oracle.snn_query(idx, Qall[r], R)
        t_used += time.perf_counter() - t0
        done += 1
        if gpu_csr is not None:
            off, gids, _ = gpu_csr
            if not np.array_equal(gids[off[r]:off[r + 1]], ids):
                mism += 1
    out = {"value": done / t_used, "unit": "queries/s", "cores": 1, "index_ms": 1e3 * t_index,
           "kind": "plain CPU SNN (Algorithms 1-2, FP64 numpy; Eq. (4) values and the direct-form decision "
                   "over each query's window)",
           "sample": f"index over all {w.n} points, then {done} random queries ({t_used:.1f} s)"}
    if gpu_csr is not None:
        out["rows_with_different_sets"] = int(mism)
    return out


# ---------------------------------------------------------------- per config
EPI_OPS_PER_PAIR = 5   # the per-pair epilogue of the low-d scorer (TMEM load, FMA, two compares, ballot)
ALU_ISSUE_TOPS = 152 * 128 * 2.070e9 / 1e12   # FP32 lanes x max clock: operations per second


def scorer_roofline(st, d, kernel_ms, precision_used, peaks, src):
    """Roofline of the scoring kernel of one query call (kernel time from the
    CUDA events around its launch).  High d: the tensor pipe (2d flop per
    scored pair).  d <= 32: the per-pair epilogue on the FP32 pipe, as the
    scoring model for low d says (the MMA is one or two k steps), with the
    tensor fraction beside it.  The FP32 scorer: 2d flop per pair on the FP32
    pipe."""
    pairs = st["band_pairs"]
    t = kernel_ms / 1e3
    flops = 2.0 * d * pairs
    peak_bf16 = float(peaks["bf16_tflops_sustained"])
    if precision_used == 0:
        ach = flops / t / 1e12
        return {"kernel": "k_score_fp32_single" if d <= 16 else "k_score_fp32_multi", "bound": "alu",
                "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP32_PEAK_TFLOPS,
                "traffic": None, "score_ms": kernel_ms,
                "algorithmic": "2d flop per scored pair (Eq. (4))",
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (derived)"}
    f8 = precision_used == 2
    peak_t = peak_bf16 * (2.0 if f8 else 1.0)
    ach_t = flops / t / 1e12
    tensor = {"kernel": "k_score_tc", "bound": "tensor", "achieved": ach_t, "peak": peak_t, "unit": "TFLOP/s",
              "frac": ach_t / peak_t, "traffic": None, "score_ms": kernel_ms,
              "algorithmic": "2d flop per scored pair (Eq. (4)); a symmetric self-join scores each "
                             "unordered pair once",
              "executed_frac": st["mma_flops_per_pair"] * pairs / t / 1e12 / peak_t,
              "mma_flops_per_pair": st["mma_flops_per_pair"],
              "peak_source": ("MEASURED_PEAKS.json bf16_tflops_sustained x 2 (e4m3 nominal ratio; %s)" % src
                              if f8 else "MEASURED_PEAKS.json bf16_tflops_sustained (%s)" % src)}
    if d > 32:
        return tensor
    ach = EPI_OPS_PER_PAIR * pairs / t / 1e12
    return {"kernel": "k_score_tc", "bound": "alu", "achieved": ach, "peak": ALU_ISSUE_TOPS,
            "unit": "Tops/s", "frac": ach / ALU_ISSUE_TOPS, "traffic": None, "score_ms": kernel_ms,
            "algorithmic": f"{EPI_OPS_PER_PAIR} FP32-pipe operations per scored pair (the low-d "
                           "epilogue: TMEM load, FMA, two compares, ballot)",
            "peak_source": "152 SMs x 128 FP32 lanes x 2.07 GHz (derived)",
            "tensor": {k: tensor[k] for k in ("achieved", "peak", "frac", "executed_frac", "unit")}}


def _timed_steps(fn, steps, warmup, flush, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ts, last = [], None
    with no_gc():
        for _ in range(steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            last = fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
    return ts, last


def _compare_rows(got_host, ref, rows):
    """Rows of a GPU CSR (host arrays) against the oracle's rows: sets must be
    identical; returns (rows with different sets, pairs, max rel dist2 error)."""
    off, ids, d2 = got_host
    mism, pairs, max_rel = 0, 0, 0.0
    for t, r in enumerate(rows):
        a, b = ref.offsets[t], ref.offsets[t + 1]
        ga, gb = off[r], off[r + 1]
        if gb - ga != b - a or not np.array_equal(ids[ga:gb], ref.ids[a:b]):
            mism += 1
            continue
        s_ref = ref.dist2[a:b].astype(np.float64)
        s_gpu = d2[ga:gb].astype(np.float64)
        rel = np.abs(s_gpu - s_ref) / np.maximum(s_ref, 1e-300)
        rel[(s_ref == 0) & (s_gpu == 0)] = 0.0
        if rel.size:
            max_rel = max(max_rel, float(rel.max()))
        pairs += b - a
    return mism, pairs, max_rel


def _oracle_rows_check(w, got_host, nrows, seed):
    """The oracle's neighbour lists of nrows random query rows (all rows when
    there are fewer), by oracle.radius_rows, compared with the GPU CSR."""
    import oracle
    rng = np.random.default_rng(seed)
    rows = np.arange(w.m) if w.m <= nrows else np.sort(rng.choice(w.m, nrows, replace=False))
    t0 = time.perf_counter()
    ref = oracle.radius_rows(w.P, w.Q, rows, w.R)
    dt = time.perf_counter() - t0
    mism, pairs, max_rel = _compare_rows(got_host, ref, rows)
    return {"rows": int(len(rows)), "pairs": int(pairs), "rows_with_different_sets": int(mism),
            "max_rel_dist2_err": max_rel, "oracle": "oracle.radius_rows (FP64 definition on every pair "
            "within a rigorous margin of R^2 of a float64 product)", "oracle_s": dt}


def _oracle_rate(w, budget_s, seed):
    """The FP64 brute-force oracle timed on a bounded query sample."""
    import oracle
    rng = np.random.default_rng(seed)
    order = rng.permutation(w.m)
    Qall = w.P if w.Q is None else w.Q
    done, used, size = 0, 0.0, 4
    while used < budget_s and done < w.m:
        rows = order[done:done + size]
        t0 = time.perf_counter()
        oracle.brute_radius(w.P, Qall[rows], w.R)
        used += time.perf_counter() - t0
        done += len(rows)
        size *= 2
    return {"value": done / used, "unit": "queries/s", "cores": oracle.oracle_threads(), "kind": "oracle",
            "sample": f"{done} random queries of the {w.m} against all {w.n} points (FP64 brute force, "
                      f"{used:.1f} s)"}


def per_config_query(args, w, label, snn, torch, flush, stream, variants=("fp32",), steps=5, warmup=3):
    """One query workload: index build + exact query per step, the 16-bit
    tensor-core path; the other precisions beside it at identical output."""
    peaks, src = load_peaks()
    X = torch.from_numpy(w.P).cuda()
    Qd = None if w.Q is None else torch.from_numpy(w.Q).cuda()

    def step(prec):
        def f():
            ix = snn.Index(X)
            return ix.query(Qd, w.R, precision=prec, stats=True)
        return f
    ts, out = _timed_steps(step("bf16"), steps, warmup, flush, stream)
    st = out.stats
    ms = float(np.median(ts))
    # index build alone, same timing rules
    tsi, _ = _timed_steps(lambda: snn.Index(X), steps, 2, flush, stream)
    directed = 2 * st["survivors"] - w.m if w.Q is None else st["survivors"]
    res = {"workload": label, "n": w.n, "d": w.d, "queries": w.m, "R": w.R,
           "value": w.m / (ms / 1e3), "unit": "queries/s", "ms_per_step": ms, "steps": steps,
           "index_build_ms": float(np.median(tsi)),
           "candidate_pairs_per_s": st["candidates"] / (ms / 1e3),
           "pairs_scored_per_s": st["band_pairs"] / (ms / 1e3),
           "tc_split": split_name(st["split_used"]), "dtype": split_dtype(st["split_used"]),
           "nnz": st["nnz"], "candidates": st["candidates"], "band_pairs": st["band_pairs"],
           "survivors": st["survivors"], "exact_fp64": st["exact_fp64"],
           "recheck_fraction": (directed - st["nnz"]) / max(1, st["candidates"]),
           "phase_ms": {k: st[k] for k in ("ms_prep", "ms_score", "ms_score_kernel", "ms_recheck", "ms_csr")},
           "roofline": scorer_roofline(st, w.d, st["ms_score_kernel"], st["precision_used"], peaks, src)}
    others = {}
    for prec in variants:
        tso, o = _timed_steps(step(prec), 3, 1, flush, stream)
        so = o.stats
        same = (torch.equal(o.offsets, out.offsets) and torch.equal(o.indices, out.indices)
                and torch.equal(o.dist2.view(torch.int32), out.dist2.view(torch.int32)))
        od = 2 * so["survivors"] - w.m if w.Q is None else so["survivors"]
        others[prec] = {"value": w.m / (np.median(tso) / 1e3), "ms_per_step": float(np.median(tso)),
                        "score_kernel_ms": so["ms_score_kernel"], "recheck_ms": so["ms_recheck"],
                        "precision_used": ["fp32", "bf16", "fp8"][so["precision_used"]],
                        "tc_split": split_name(so["split_used"]), "survivors": so["survivors"],
                        "recheck_fraction": (od - so["nnz"]) / max(1, so["candidates"]),
                        "roofline": scorer_roofline(so, w.d, so["ms_score_kernel"], so["precision_used"],
                                                    peaks, src),
                        "csr_identical": bool(same)}
        del o
    res["other_precisions"] = others
    if "fp32" in others:
        res["speedup_vs_fp32_path"] = res["value"] / others["fp32"]["value"]
    if args.cpu_baseline:
        host = (out.offsets.cpu().numpy(), out.indices.cpu().numpy(), out.dist2.cpu().numpy())
        res["parity"] = _oracle_rows_check(w, host, args.parity_rows, seed=31)
        res["max_rel_dist2_err"] = res["parity"]["max_rel_dist2_err"]
        res["cpu_baseline"] = _oracle_rate(w, args.cfg_budget, seed=32)
    del out, X, Qd
    torch.cuda.synchronize()
    return res


def per_config_ragged(args, snn, torch, flush, stream, steps=5, warmup=2):
    """Ragged batch: the batched index build of every set plus one run of the
    batched query plan per step; one index build and one query call per set
    beside it; the tuned plan's graph-replayed query phase."""
    from paper_2212_07679_gb300 import workloads as wl
    t0 = time.perf_counter()
    sets = wl.ragged_batch()
    gen_s = time.perf_counter() - t0
    Xs = [torch.from_numpy(s.P).cuda() for s in sets]
    Qs = [torch.from_numpy(s.Q).cuda() for s in sets]
    Rs = [s.R for s in sets]
    M = sum(q.shape[0] for q in Qs)
    N = sum(x.shape[0] for x in Xs)

    def make_plan(idx, prec="bf16"):
        plan = snn.BatchPlan(idx, [q.shape[0] for q in Qs], Rs, precision=prec,
                             survivor_capacity=64 * M + (1 << 20), nnz_capacity=64 * M + (1 << 20))
        plan.set_queries(Qs)
        return plan

    def step():
        idx = snn.build_batch(Xs)
        plan = make_plan(idx)
        plan.run()
        return plan.result(copy=False)

    ts, _ = _timed_steps(step, steps, warmup, flush, stream)
    tsl, _ = _timed_steps(lambda: [snn.Index(x).query(q, r, precision="bf16") for x, q, r in zip(Xs, Qs, Rs)],
                          3, 1, flush, stream)
    idx = snn.build_batch(Xs)
    plan = make_plan(idx)
    cpi, ctas, tune_ms = plan.tune()
    tuned = plan.config()

    def graph_query():
        plan.launch_graph()
        return plan.result(copy=False)
    tsg, _ = _timed_steps(graph_query, steps, 2, flush, stream)
    plan.launch_graph()
    got = plan.result()
    # the same query phase with the FP32 scorer only
    plan32 = make_plan(idx, "fp32")
    plan32.tune()

    def graph_query32():
        plan32.launch_graph()
        return plan32.result(copy=False)
    tsg32, _ = _timed_steps(graph_query32, steps, 2, flush, stream)
    plan32.close()
    ms = float(np.median(ts))
    res = {"workload": "ragged_batch (256 mixtures, batched build + one batched query)", "sets": len(sets),
           "points": N, "queries": M, "value": M / (ms / 1e3), "unit": "queries/s", "ms_per_step": ms,
           "steps": steps, "per_set_calls": {"ms_per_step": float(np.median(tsl)),
                                            "value": M / (np.median(tsl) / 1e3)},
           "query_phase_graph_ms": float(np.median(tsg)),
           "query_phase_graph_ms_fp32_scorer": float(np.median(tsg32)),
           "precision": "bf16 (tensor-core groups for the out-of-sample sets of d <= 48)",
           "tuned": {"chunks_per_item": cpi, "ctas_per_sm": ctas, "tc_groups": tuned["tc_groups"],
                     "tc_mask": tuned["tc_mask"], "from_cache": tuned["from_cache"], "tune_ms": tune_ms},
           "generation_s": gen_s}
    if args.cpu_baseline:
        import oracle
        rng = np.random.default_rng(33)
        mism, pairs, max_rel, rows_done = 0, 0, 0.0, 0
        per_set = max(1, args.parity_rows // len(sets))
        t0 = time.perf_counter()
        for t, s in enumerate(sets):
            rows = np.sort(rng.choice(s.m, min(per_set, s.m), replace=False))
            ref = oracle.radius_rows(s.P, s.Q, rows, s.R)
            g = got[t]
            host = (g.offsets.cpu().numpy(), g.indices.cpu().numpy(), g.dist2.cpu().numpy())
            a, b, c = _compare_rows(host, ref, rows)
            mism += a
            pairs += b
            max_rel = max(max_rel, c)
            rows_done += len(rows)
        res["parity"] = {"rows": rows_done, "pairs": int(pairs), "rows_with_different_sets": int(mism),
                         "max_rel_dist2_err": max_rel, "oracle_s": time.perf_counter() - t0,
                         "oracle": "oracle.radius_rows on random rows of every set"}
        res["max_rel_dist2_err"] = max_rel
    plan.close()
    del idx, Xs, Qs, got
    torch.cuda.synchronize()
    return res


def per_config_dbscan(args, snn, torch, flush, stream, steps=5, warmup=3):
    """DBSCAN on the 5e5-point 3-d particle set (eps 0.4, minPts 10): index
    build, exact self-join, core flags and union-find labels per step."""
    import oracle  # noqa: F401  (parity below only)
    from paper_2212_07679_gb300 import workloads as wl
    peaks, src = load_peaks()
    w = wl.blobs3d()
    X = torch.from_numpy(w.P).cuda()
    eps, min_pts = w.R, w.extra["min_pts"]
    ts, (labels, core) = _timed_steps(lambda: snn.dbscan(X, eps, min_pts, precision="bf16"), steps, warmup,
                                      flush, stream)
    ms = float(np.median(ts))
    # the self-join inside the step, once more with statistics
    out = snn.Index(X).query(None, eps, precision="bf16", stats=True)
    st = out.stats
    lab = labels.cpu().numpy()
    cr = core.cpu().numpy().astype(bool)
    res = {"workload": "blobs3d DBSCAN (self-join + core flags + union-find)", "n": w.n, "d": w.d,
           "eps": eps, "min_pts": min_pts, "value": w.n / (ms / 1e3), "unit": "points/s", "ms_per_step": ms,
           "steps": steps, "clusters": int(len(np.unique(lab[lab >= 0]))), "core_points": int(cr.sum()),
           "self_join": {"nnz": st["nnz"], "candidates": st["candidates"], "band_pairs": st["band_pairs"],
                         "survivors": st["survivors"],
                         "recheck_fraction": (2 * st["survivors"] - w.n - st["nnz"]) / max(1, st["candidates"]),
                         "tc_split": split_name(st["split_used"]),
                         "phase_ms": {k: st[k] for k in ("ms_prep", "ms_score", "ms_score_kernel", "ms_recheck",
                                                         "ms_csr")}},
           "roofline": scorer_roofline(st, w.d, st["ms_score_kernel"], st["precision_used"], peaks, src)}
    if args.cpu_baseline:
        import oracle
        rng = np.random.default_rng(34)
        rows = np.sort(rng.choice(w.n, args.parity_rows, replace=False))
        t0 = time.perf_counter()
        ref = oracle.radius_rows(w.P, None, rows, eps)
        host = (out.offsets.cpu().numpy(), out.indices.cpu().numpy(), out.dist2.cpu().numpy())
        mism, pairs, max_rel = _compare_rows(host, ref, rows)
        bad_core = bad_label = 0
        for t, r in enumerate(rows):
            nb = ref.row(t)[0]
            if cr[r] != (len(nb) >= min_pts):
                bad_core += 1
                continue
            core_nb = nb[cr[nb]]
            if cr[r]:
                bad_label += int(not np.all(lab[core_nb] == lab[r]))
            elif len(core_nb):
                bad_label += int(lab[r] != lab[core_nb.min()])
            else:
                bad_label += int(lab[r] != -1)
        res["parity"] = {"rows": int(len(rows)), "pairs": int(pairs), "rows_with_different_sets": int(mism),
                         "max_rel_dist2_err": max_rel, "rows_with_wrong_core_flag": int(bad_core),
                         "rows_with_wrong_label": int(bad_label), "oracle_s": time.perf_counter() - t0,
                         "oracle": "oracle.radius_rows rows; core flag = |N| >= minPts; labels checked "
                                   "against the rows' core neighbours"}
        res["max_rel_dist2_err"] = max_rel
        res["cpu_baseline"] = _oracle_rate(w, args.cfg_budget, seed=35)
    del X, out
    torch.cuda.synchronize()
    return res


def per_config_block(args, snn, torch, flush, stream):
    from paper_2212_07679_gb300 import workloads as wl
    out = {}
    t0 = time.perf_counter()
    out["cfg1_gmm_iso"] = per_config_query(args, wl.gmm_iso(), "gmm_iso: 500 queries drawn from 2,000 points",
                                           snn, torch, flush, stream)
    out["cfg3_lowrank_img"] = per_config_query(args, wl.lowrank_img(), "lowrank_img self-join", snn, torch,
                                               flush, stream, variants=("fp32", "fp8"))
    out["cfg5_blobs3d_dbscan"] = per_config_dbscan(args, snn, torch, flush, stream)
    out["cfg4_ragged_batch"] = per_config_ragged(args, snn, torch, flush, stream)
    out["wall_s"] = time.perf_counter() - t0
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = make_workload(args)
    steps = []
    for _ in range(args.warmup):
        cpu_oracle_sample(w, budget_s=2.0)
    for _ in range(args.steps):
        steps.append(cpu_oracle_sample(w, budget_s=args.ref_budget))
    qps = float(np.mean([s["value"] for s in steps]))
    line = {"impl": "reference", "metric": "exact radius queries/s & pairs scored/s: BF16+FP64 recheck vs FP32, % roofline",
            "metric_detail": "exact radius queries/s of the FP64 brute-force oracle on the host cores", "value": qps,
            "unit": "queries/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * w.m / qps, "extrapolated_from_sample": True,
            "ms_per_step_note": ("each step times the oracle on a bounded query sample; ms_per_step is the "
                                 "time all queries would take at the sampled rate"),
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, w),
            "cpu_baseline": {"value": qps, "unit": "queries/s", "cores": steps[-1]["cores"],
                             "kind": "oracle", "sample": steps[-1]["sample"]},
            "e2e": {"value": qps, "unit": "queries/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2212_07679_gb300 import snn

    w = make_workload(args)
    X_host = torch.from_numpy(w.P).pin_memory()
    X = X_host.cuda()
    Q_host = None if w.Q is None else torch.from_numpy(w.Q).pin_memory()
    Qd = None if Q_host is None else Q_host.cuda()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    # cosine workloads: rows normalised on the device inside every step, and
    # the Euclidean radius of the cosine-distance bound
    Rq = snn.radius_for_cosine_distance(w.R) if is_cosine(w) else w.R

    def index_of(Xd):
        return snn.Index(snn.normalize_rows(Xd) if is_cosine(w) else Xd)

    def step(stats=True, e_mid=None):
        ix = index_of(X)
        if e_mid is not None:
            e_mid.record(stream)
        out = ix.query(Qd, Rq, precision=args.precision, stats=stats)
        return ix, out

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    per_step, index_ms, score_ms, stats_list = [], [], [], []
    last_out = None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = snn.launch_count()
    with no_gc():
        for _ in range(args.steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            em = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            # phase events and counters, without the candidate-range count
            # (a statistics-only kernel; the count comes from one untimed
            # step below)
            ix, out = step(stats="phases", e_mid=em)
            e1.record(stream)
            e1.synchronize()
            per_step.append(e0.elapsed_time(e1))
            index_ms.append(e0.elapsed_time(em))
            score_ms.append(out.stats["ms_score_kernel"])
            stats_list.append(out.stats)
            del ix
            last_out = out
            del out
    torch.cuda.synchronize()
    launches = snn.launch_count() - launches0
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    total_ms = float(np.sum(per_step))
    ms_step = job_max_ms(total_ms, world) / args.steps
    value = whole_job_rate(w.m, world, ms_step)

    def time_precision(prec, products=None):
        # another scoring precision on the same workload, same timing rules;
        # its CSR is compared with the headline run's on the device
        if products is not None:
            os.environ["SNN_FP8_PRODUCTS"] = str(products)
        try:
            for _ in range(2):
                ix = index_of(X)
                ix.query(Qd, Rq, precision=prec)
                del ix
            times = []
            for _ in range(max(3, min(args.steps, 5))):
                flush.fill_(1)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ix = index_of(X)
                out = ix.query(Qd, Rq, precision=prec, stats=True)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
                ost = out.stats
                same = (torch.equal(out.offsets, last_out.offsets) and torch.equal(out.indices, last_out.indices)
                        and torch.equal(out.dist2.view(torch.int32), last_out.dist2.view(torch.int32)))
                del ix, out
        finally:
            if products is not None:
                os.environ.pop("SNN_FP8_PRODUCTS", None)
        oms = float(np.mean(times))
        dsurv = 2 * ost["survivors"] - w.m if w.Q is None else ost["survivors"]
        res = {"precision": prec, "value": w.m / (oms / 1e3), "unit": "queries/s",
               "ms_per_step": oms, "score_ms": ost["ms_score"], "recheck_ms": ost["ms_recheck"],
               "survivors": ost["survivors"],
               "recheck_fraction": (dsurv - ost["nnz"]) / max(1, ost["candidates"]),
               "csr_identical_to_headline": bool(same)}
        if prec == "fp8":
            res["products_per_kstep"] = products
            res["precision_used"] = ["fp32", "bf16", "fp8"][ost["precision_used"]]
            res["mma_flops_per_pair"] = ost["mma_flops_per_pair"]
        return res

    compare, fp8_variants = None, None
    if args.compare:
        compare = time_precision("fp32" if args.precision != "fp32" else "bf16")
        if args.precision == "bf16" and w.d > 55:
            fp8_variants = [time_precision("fp8", k) for k in (3, 4, 6)]

    # end to end through host buffers: pinned X in, CSR out into reused
    # pinned buffers (CSR.to_host), every step.  Serial: one step after the
    # other, each waiting for its read-back.  Pipelined (the headline e2e):
    # steps alternate between two streams, so that a step's read-back runs
    # while the next step's copy-in and compute proceed; the timed region
    # still holds every step's copy-in and read-back.  One untimed pass per
    # stream sizes the buffers.
    def e2e_step(stream, bufs, blocking):
        with torch.cuda.stream(stream):
            Xd = X_host.to("cuda", non_blocking=True)
            Qe = None if Q_host is None else Q_host.to("cuda", non_blocking=True)
            ix = snn.Index(snn.normalize_rows(Xd, stream=stream) if is_cosine(w) else Xd, stream=stream)
            out = ix.query(Qe, Rq, precision=args.precision, stream=stream)
            return out.to_host(bufs, stream=stream, blocking=blocking)

    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    hbufs = [snn.HostBuffers(), snn.HostBuffers()]
    for k in range(2):
        host = e2e_step(streams[k], hbufs[k], True)
    h2d = (X_host.numel() + (0 if Q_host is None else Q_host.numel())) * 4
    d2h = host.offsets.numel() * 8 + host.indices.numel() * 4 + host.dist2.numel() * 4
    del host
    e2e_ms = []
    with no_gc():
        for it in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_step(streams[0], hbufs[0], True)
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
    # five pipelined passes of n_pipe steps each; the median pass is
    # reported (one pass can catch a host-side stall), all five are listed
    n_pipe = max(4, min(args.steps, 8))
    pipe_passes = []
    for _ in range(5):
        with no_gc():
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for it in range(n_pipe):
                e2e_step(streams[it % 2], hbufs[it % 2], False)
            torch.cuda.synchronize()
            pipe_passes.append(1e3 * (time.perf_counter() - t0) / n_pipe)
    e2e_pipe_ms = float(np.median(pipe_passes))

    st = dict(stats_list[-1])
    _, full = step(stats=True)
    st["candidates"] = full.stats["candidates"]
    del full
    peaks, src = load_peaks()
    sm = float(np.mean(score_ms))
    # executed: pairs the kernel actually scored (the symmetric self-join
    # scores each unordered pair once); effective: the candidate pairs of
    # the per-query candidate ranges of Algorithm 2 that this replaces
    effective = 2.0 * w.d * st["candidates"] / (sm / 1e3) / 1e12
    directed_surv = 2 * st["survivors"] - w.m if w.Q is None else st["survivors"]
    # the scoring kernel's roofline (kernel time from the events around its
    # launch): the tensor pipe at high d, the per-pair epilogue on the FP32
    # pipe at d <= 32 with the tensor fraction beside it
    roofline = scorer_roofline(st, w.d, sm, st["precision_used"], peaks, src)
    roofline["effective_tflops"] = effective
    roofline["score_ms_source"] = "CUDA events around the scoring launch alone (stats.ms_score_kernel)"
    if st["precision_used"] != 0:
        used = ["fp32", "bf16", "fp8"][st["precision_used"]]
        traffic = scorer_traffic(w.name, w.n, used) if w.Q is None else None
        roofline["traffic"] = traffic
        roofline["traffic_source"] = (f"{SCORER_TRAFFIC['profile']} (dram__bytes_read.sum + "
                                      "dram__bytes_write.sum of one full-size launch)") if traffic else \
            "no full-size capture of this kernel build and workload"
    line = {
        "metric": "exact radius queries/s & pairs scored/s: BF16+FP64 recheck vs FP32, % roofline",
        "metric_detail": ("exact radius queries/s (16-bit or e4m3 tensor-core rejection, compensated FP32 "
                          "and FP64 exact decision); pairs scored/s, the FP32 path and the roofline "
                          "fraction are the other keys of this line"),
        "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": split_dtype(st.get("split_used", 0)),
        "tc_split": split_name(st.get("split_used", 0)),
        "data": "synthetic",
        "config": workload_config(args, w),
        "pairs_scored_per_s": st["band_pairs"] / (ms_step / 1e3),
        "candidate_pairs_per_s": st["candidates"] / (ms_step / 1e3),
        "nnz": st["nnz"], "candidates": st["candidates"], "band_pairs": st["band_pairs"],
        "survivors": st["survivors"], "exact_fp64": st["exact_fp64"],
        "recheck_fraction": (directed_surv - st["nnz"]) / max(1, st["candidates"]),
        "index_build_ms": float(np.mean(index_ms)),
        "phase_ms": {k: st[k] for k in ("ms_prep", "ms_score", "ms_recheck", "ms_csr")},
        "roofline": roofline,
        "clocks": clk,
        "other_precision": compare,
        "fp8_variants": fp8_variants,
        "gpu_launches": launches,
        "gpu_launches_per_step": launches / args.steps,
        "e2e": {"value": w.m / (e2e_pipe_ms / 1e3), "unit": "queries/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "ms_per_step": e2e_pipe_ms,
                "mode": f"{n_pipe} steps alternating between two streams, median of 5 passes",
                "pass_ms_per_step": pipe_passes,
                "serial": {"value": w.m / (np.median(e2e_ms) / 1e3), "ms_per_step": float(np.median(e2e_ms))}},
    }
    if args.per_config and args.workload == "gmm_aniso" and world == 1:
        # the other configurations of the benchmark, measured after the
        # headline's timed region (rank 0 only)
        line["per_config"] = per_config_block(args, snn, torch, flush, stream)
    if rank == 0:
        if args.cpu_baseline:
            csr_h = (last_out.offsets.cpu().numpy(), last_out.indices.cpu().numpy(),
                     last_out.dist2.cpu().numpy())
            line["cpu_baseline"] = cpu_oracle_sample(w, budget_s=args.ref_budget, gpu_csr=csr_h)
            line["cpu_baseline"]["cpu_snn"] = cpu_snn_sample(w, budget_s=args.ref_budget / 2,
                                                             gpu_csr=csr_h)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_ragged(args):
    """Ragged batch: 256 independent mixtures (n log-uniform in [1e3, 2e5],
    d in {2, 3, 8, 32}, 10% of each set as out-of-sample queries).  One step =
    the batched index build of every set plus one run of the batched query
    plan; the same work with one index build and one query call per set, and
    the plan's CUDA-graph replay of the query phase alone, are timed beside it."""
    import torch
    from paper_2212_07679_gb300 import snn
    from paper_2212_07679_gb300 import workloads as wl
    sets = wl.ragged_batch(n_scale=args.n / 1e5) if args.n else wl.ragged_batch()
    Xs = [torch.from_numpy(s.P).cuda() for s in sets]
    Qs = [torch.from_numpy(s.Q).cuda() for s in sets]
    Rs = [s.R for s in sets]
    M = sum(q.shape[0] for q in Qs)
    N = sum(x.shape[0] for x in Xs)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def make_plan(idx):
        plan = snn.BatchPlan(idx, [q.shape[0] for q in Qs], Rs, precision=args.precision,
                             survivor_capacity=64 * M + (1 << 20), nnz_capacity=64 * M + (1 << 20))
        plan.set_queries(Qs)
        return plan

    def step():
        idx = snn.build_batch(Xs)
        plan = make_plan(idx)
        plan.run()
        out = plan.result(copy=False)
        return idx, plan, out

    def per_set():
        return [snn.Index(x).query(q, r, precision=args.precision) for x, q, r in zip(Xs, Qs, Rs)]

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
            del r
        return float(np.mean(ts))

    for _ in range(args.warmup):
        step()
        per_set()
    torch.cuda.synchronize()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    l0 = snn.launch_count()
    ms_step = timed(step, args.steps)
    launches = snn.launch_count() - l0
    ms_loop = timed(per_set, max(3, min(args.steps, 5)))
    # query phase alone on persistent indices: tuned plan, graph replays
    idx = snn.build_batch(Xs)
    plan = make_plan(idx)
    cpi, ctas, _ = plan.tune()
    plan.launch_graph()
    plan.result(copy=False)
    torch.cuda.synchronize()

    def graph_query():
        plan.launch_graph()
        return plan.result(copy=False)
    ms_graph = timed(graph_query, max(3, args.steps))
    pidx = [snn.Index(x) for x in Xs]

    def loop_query():
        return [ix.query(q, r, precision=args.precision) for ix, q, r in zip(pidx, Qs, Rs)]
    ms_loop_query = timed(loop_query, max(3, min(args.steps, 5)))
    clk = clocks.stop()
    got = plan.result()
    # end to end: every set's points and queries from pinned host memory,
    # batched build, one plan run, every result copied into pinned buffers
    Xh = [torch.from_numpy(s.P).pin_memory() for s in sets]
    Qh = [torch.from_numpy(s.Q).pin_memory() for s in sets]
    hb = [snn.HostBuffers() for _ in sets]
    e2e_ms, d2h = [], 0
    for it in range(1 + max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xd = [x.to("cuda", non_blocking=True) for x in Xh]
        ex = snn.build_batch(xd)
        ep = snn.BatchPlan(ex, [q.shape[0] for q in Qh], Rs, precision=args.precision,
                           survivor_capacity=64 * M + (1 << 20), nnz_capacity=64 * M + (1 << 20))
        for t, q in enumerate(Qh):
            ep.queries(t).copy_(q, non_blocking=True)
        ep.run()
        outs = [o.to_host(b) for o, b in zip(ep.result(copy=False), hb)]
        torch.cuda.synchronize()
        if it > 0:
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
        d2h = sum(o.offsets.numel() * 8 + o.nnz * 8 for o in outs)
        ep.close()
        del xd, ex, ep, outs
    line = {
        "metric": "ragged batch exact radius queries/s (batched index build + one batched query)",
        "value": M / (ms_step / 1e3), "unit": "queries/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16+bf16+f32+f64" if args.precision != "fp32" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": "ragged_batch", "sets": len(sets), "points": N, "queries": M,
                   "precision": args.precision, "parallelism": "replicas1",
                   "l2": "flushed between steps (256 MiB write)"},
        "per_set_calls": {"ms_per_step": ms_loop, "value": M / (ms_loop / 1e3)},
        "query_phase": {"graph_ms": ms_graph, "graph_queries_per_s": M / (ms_graph / 1e3),
                        "per_set_calls_ms": ms_loop_query,
                        "per_set_calls_queries_per_s": M / (ms_loop_query / 1e3),
                        "tuned": dict(plan.config(), chunks_per_item=cpi, ctas_per_sm=ctas)},
        "clocks": clk, "gpu_launches": launches, "gpu_launches_per_step": launches / args.steps,
        "e2e": {"value": M / (np.median(e2e_ms) / 1e3), "unit": "queries/s",
                "h2d_bytes_per_step": int(sum(x.numel() + q.numel() for x, q in zip(Xh, Qh)) * 4),
                "d2h_bytes_per_step": int(d2h)},
    }
    if args.cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_ragged(sets, got, budget_s=args.ref_budget)
    print(json.dumps(line), flush=True)


def cpu_oracle_ragged(sets, got, budget_s=15.0, seed=11):
    """Times the FP64 brute-force oracle on a random sample of the batch's
    sets (all their queries) and compares those sets' GPU results with it."""
    import oracle
    rng = np.random.default_rng(seed)
    done_q, t_used, mism, pairs, nsets = 0, 0.0, 0, 0, 0
    for t in rng.permutation(len(sets)):
        if t_used >= budget_s:
            break
        t0 = time.perf_counter()
        ref = oracle.brute_radius(sets[t].P, sets[t].Q, sets[t].R)
        t_used += time.perf_counter() - t0
        done_q += sets[t].Q.shape[0]
        nsets += 1
        g = got[t]
        ok = (np.array_equal(g.offsets.cpu().numpy(), ref.offsets)
              and np.array_equal(g.indices.cpu().numpy(), ref.ids)
              and np.array_equal(g.dist2.cpu().numpy().view(np.uint32), ref.dist2.view(np.uint32)))
        mism += 0 if ok else 1
        pairs += len(ref.ids)
    return {"value": done_q / max(t_used, 1e-9), "unit": "queries/s", "cores": oracle.oracle_threads(),
            "kind": "oracle",
            "sample": f"all queries of {nsets} random sets of the {len(sets)} (FP64 brute force, "
                      f"{t_used:.1f} s)",
            "parity": {"sets": nsets, "pairs": int(pairs), "sets_with_different_results": int(mism)}}


def run_dbscan(args):
    """DBSCAN on top of the self-join (Section 6.4): 500,000 particle-like
    points in 3-d (200 blobs + 10% background), eps = 0.4, minPts = 10.  One
    step = index build, exact self-join, core flags, union-find labels."""
    import torch
    from paper_2212_07679_gb300 import snn
    from paper_2212_07679_gb300 import workloads as wl
    w = wl.blobs3d(n=args.n) if args.n else wl.blobs3d()
    X = torch.from_numpy(w.P).cuda()
    eps, min_pts = w.R, w.extra["min_pts"]
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        snn.dbscan(X, eps, min_pts, precision=args.precision)
    torch.cuda.synchronize()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    l0 = snn.launch_count()
    ts = []
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        labels, core = snn.dbscan(X, eps, min_pts, precision=args.precision)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    launches = snn.launch_count() - l0
    clk = clocks.stop()
    ms = float(np.mean(ts))
    # end to end: pinned points in, labels and core flags out into pinned
    # buffers, every step
    X_host = torch.from_numpy(w.P).pin_memory()
    lab_h = torch.empty(w.n, dtype=torch.int32, pin_memory=True)
    core_h = torch.empty(w.n, dtype=torch.uint8, pin_memory=True)
    e2e_ms = []
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Xd = X_host.to("cuda", non_blocking=True)
        lb, cr = snn.dbscan(Xd, eps, min_pts, precision=args.precision)
        lab_h.copy_(lb, non_blocking=True)
        core_h.copy_(cr, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
        del Xd, lb, cr
    lab = labels.cpu().numpy()
    line = {
        "metric": "DBSCAN points/s (exact eps-neighbourhoods by SNN self-join, union-find labels)",
        "value": w.n / (ms / 1e3), "unit": "points/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16+f32+f64" if args.precision == "bf16" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": "blobs3d DBSCAN", "n": w.n, "d": w.d, "eps": eps, "min_pts": min_pts,
                   "precision": args.precision, "parallelism": "replicas1",
                   "l2": "flushed between steps (256 MiB write)"},
        "clusters": int(len(np.unique(lab[lab >= 0]))), "core_points": int(core.sum().item()),
        "noise_points": int((lab < 0).sum()),
        "clocks": clk, "gpu_launches": launches, "gpu_launches_per_step": launches / args.steps,
        "e2e": {"value": w.n / (np.median(e2e_ms) / 1e3), "unit": "points/s",
                "h2d_bytes_per_step": int(X_host.numel() * 4),
                "d2h_bytes_per_step": int(w.n * 4 + w.n)},
    }
    if args.cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_sample(w, budget_s=args.ref_budget)
    print(json.dumps(line), flush=True)


def run_mips(args):
    """Inner-product threshold search (snn_inner_product_search): 10,000 queries
    against 200,000 word-vector-like rows of 100 dims, tau for ~20 results per
    query.  One step = the whole call (norms, augmentation, index build on the
    augmented rows, per-query-radius Euclidean search, exact dot-product
    decision, compaction); the FP32-pruned call is timed beside it."""
    import torch
    from paper_2212_07679_gb300 import snn
    from paper_2212_07679_gb300 import workloads as wl
    w = wl.mips_like(n=args.n) if args.n else wl.mips_like()
    P_host = torch.from_numpy(w.P).pin_memory()
    Q_host = torch.from_numpy(w.Q).pin_memory()
    P, Q = P_host.cuda(), Q_host.cuda()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed(prec, steps, stats=False):
        ts, out = [], None
        for _ in range(steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = snn.inner_product_search(P, Q, w.R, precision=prec, stats=stats)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.mean(ts)), out

    for _ in range(args.warmup):
        snn.inner_product_search(P, Q, w.R, precision=args.precision)
    torch.cuda.synchronize()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    l0 = snn.launch_count()
    ms, out = timed(args.precision, args.steps, stats=True)
    launches = snn.launch_count() - l0
    clk = clocks.stop()
    st = out.stats
    compare = None
    if args.compare:
        other = "fp32" if args.precision != "fp32" else "bf16"
        snn.inner_product_search(P, Q, w.R, precision=other)
        oms, oout = timed(other, max(3, min(args.steps, 5)))
        same = (torch.equal(oout.offsets, out.offsets) and torch.equal(oout.indices, out.indices)
                and torch.equal(oout.dist2.view(torch.int32), out.dist2.view(torch.int32)))
        compare = {"precision": other, "value": w.m / (oms / 1e3), "unit": "queries/s", "ms_per_step": oms,
                   "csr_identical_to_headline": bool(same)}
    # end to end: pinned rows in, CSR out into pinned buffers
    hb = snn.HostBuffers()
    e2e = []
    for it in range(1 + max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Pd = P_host.to("cuda", non_blocking=True)
        Qd = Q_host.to("cuda", non_blocking=True)
        host = snn.inner_product_search(Pd, Qd, w.R, precision=args.precision).to_host(hb)
        torch.cuda.synchronize()
        if it > 0:
            e2e.append(1e3 * (time.perf_counter() - t0))
        d2h = host.offsets.numel() * 8 + host.nnz * 8
        del Pd, Qd, host
    peaks, src = load_peaks()
    flops = 2.0 * (w.d + 1) * st["band_pairs"]
    achieved = flops / (ms / 1e3) / 1e12
    peak = float(peaks["bf16_tflops_sustained"])
    line = {
        "metric": "exact inner-product threshold queries/s (augmented SNN pruning, exact FP64-definition decision)",
        "value": w.m / (ms / 1e3), "unit": "queries/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"bf16": "bf16+f32+f64", "fp8": "e4m3+bf16+f32+f64"}.get(args.precision, "f32+f64"),
        "data": "synthetic",
        "config": {"workload": "mips_like inner-product threshold", "n": w.n, "d": w.d, "queries": w.m,
                   "tau": w.R, "precision": args.precision, "parallelism": "replicas1",
                   "l2": "flushed between steps (256 MiB write)"},
        "nnz": st["nnz"], "candidates": st["candidates"], "survivors": st["survivors"],
        "band_pairs": st["band_pairs"], "exact_fp64": st["exact_fp64"], "xi": st["xi"],
        "roofline": {"kernel": "whole call (augmented scoring dominant)", "bound": "tensor", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                     "peak_source": f"MEASURED_PEAKS.json bf16_tflops_sustained ({src})",
                     "algorithmic": "2 (d + 1) flop per scored augmented pair over the whole call time"},
        "other_precision": compare,
        "clocks": clk, "gpu_launches": launches, "gpu_launches_per_step": launches / args.steps,
        "e2e": {"value": w.m / (np.median(e2e) / 1e3), "unit": "queries/s",
                "h2d_bytes_per_step": int((P_host.numel() + Q_host.numel()) * 4), "d2h_bytes_per_step": int(d2h)},
    }
    if args.cpu_baseline:
        import oracle
        rng = np.random.default_rng(7)
        order = rng.permutation(w.m)
        done, t_used, size = 0, 0.0, 8
        off, ids, vals = (out.offsets.cpu().numpy(), out.indices.cpu().numpy(), out.dist2.cpu().numpy())
        mism = 0
        while t_used < args.ref_budget and done < w.m:
            rows = order[done:done + size]
            t0 = time.perf_counter()
            ref = oracle.brute_inner_product(w.P, w.Q[rows], w.R)
            t_used += time.perf_counter() - t0
            for k, r in enumerate(rows):
                a, b = ref.offsets[k], ref.offsets[k + 1]
                ga, gb = off[r], off[r + 1]
                if (gb - ga != b - a or not np.array_equal(ids[ga:gb], ref.ids[a:b])
                        or not np.array_equal(vals[ga:gb].view(np.uint32), ref.dist2[a:b].view(np.uint32))):
                    mism += 1
            done += len(rows)
            size *= 2
        line["cpu_baseline"] = {"value": done / t_used, "unit": "queries/s", "cores": 1, "kind": "oracle",
                                "sample": f"{done} random queries against all {w.n} rows (numpy FP64, {t_used:.1f} s)",
                                "parity": {"rows": int(done), "rows_with_different_results": int(mism)}}
    print(json.dumps(line), flush=True)


def run_stream(args):
    """Streaming updates (snn_index_insert / snn_index_delete) on the 10^6-point
    16-dim mixture: an index of 900,000 points takes ten insert batches of
    10,000 points; one step = one insert.  Then the self-join of the updated
    index (original centre and direction) is timed beside that of a fresh
    build on the same points, and a delete of 10,000 random ids is timed."""
    import torch
    from paper_2212_07679_gb300 import snn
    from paper_2212_07679_gb300 import workloads as wl
    w = wl.gmm_aniso(n=args.n) if args.n else wl.gmm_aniso()
    n0 = w.n - 100_000
    batch = 10_000
    X = torch.from_numpy(w.P).cuda()
    stream = torch.cuda.current_stream()

    def ev_time(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), r

    for _ in range(args.warmup):
        ix = snn.Index(X[:n0])
        ix.insert(X[n0:n0 + batch])
        del ix
    torch.cuda.synchronize()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    l0 = snn.launch_count()
    ix = snn.Index(X[:n0])
    ins = []
    for t in range(10):
        ms, _ = ev_time(lambda: ix.insert(X[n0 + t * batch:n0 + (t + 1) * batch]))
        ins.append(ms)
    launches = snn.launch_count() - l0
    clk = clocks.stop()
    # second queries of each index (the first builds the tensor-core operands)
    ix.query(None, w.R, precision=args.precision)
    q_upd, out_upd = ev_time(lambda: ix.query(None, w.R, precision=args.precision, stats=True))
    fresh = snn.Index(X)
    fresh.query(None, w.R, precision=args.precision)
    q_fresh, out_fresh = ev_time(lambda: fresh.query(None, w.R, precision=args.precision, stats=True))
    same = (torch.equal(out_upd.offsets, out_fresh.offsets) and torch.equal(out_upd.indices, out_fresh.indices)
            and torch.equal(out_upd.dist2.view(torch.int32), out_fresh.dist2.view(torch.int32)))
    rng = np.random.default_rng(5)
    ix.delete(torch.from_numpy(rng.choice(w.n, 10, replace=False).astype(np.int32)).cuda())   # warm-up
    ids = torch.from_numpy(rng.choice(ix.n, 10_000, replace=False).astype(np.int32)).cuda()
    del_ms, _ = ev_time(lambda: ix.delete(ids))
    ms = float(np.mean(ins))
    peaks, src = load_peaks()
    dp = (w.d + 3) // 4 * 4
    # every insert rewrites all per-position arrays: raw and centred rows,
    # score, id, halved norm, norm bound (read old + write merged)
    nmid = n0 + 5 * batch
    bytes_step = 2.0 * nmid * (2 * dp * 4 + 16)
    achieved = bytes_step / (ms / 1e3) / 1e9
    line = {
        "metric": "streaming insert points/s (10,000-point batches merged into a 0.9-1.0 M-point index)",
        "value": batch / (ms / 1e3), "unit": "points/s", "n_gpus": 1, "steps": 10, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "gmm_aniso streaming inserts", "n_start": n0, "batch": batch, "d": w.d,
                   "R": w.R, "precision": args.precision, "parallelism": "replicas1",
                   "l2": "inputs larger than L2 (every insert rewrites ~150 MB of index arrays)"},
        "roofline": {"kernel": "k_place (merge scatter)", "bound": "hbm", "achieved": achieved,
                     "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                     "frac": achieved / float(peaks["hbm_gbs"]), "traffic": None,
                     "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({src})",
                     "algorithmic": "per insert: read and write every per-position array of the index "
                                    "(2 x n x (2 dp x 4 + 16) B), whole insert call timed"},
        "query_after_inserts_ms": q_upd, "query_fresh_build_ms": q_fresh,
        "band_pairs_after_inserts": out_upd.stats["band_pairs"],
        "band_pairs_fresh_build": out_fresh.stats["band_pairs"],
        "csr_identical_to_fresh_build": bool(same),
        "delete_10000_ms": del_ms,
        "clocks": clk, "gpu_launches": launches, "gpu_launches_per_step": launches / 10,
    }
    print(json.dumps(line), flush=True)


def run_peaks(args):
    """Throughput probes of the arithmetic units the kernels use (tcgen05 BF16
    and e4m3 MMAs, FP32 and FP64 FMAs), each timed with CUDA events over
    `steps` launches after `warmup` launches, with clocks sampled meanwhile.
    These check the ratios the rooflines rely on (e4m3 = 2 x BF16, the FP32
    lane count x clock); the rooflines themselves keep the denominators of
    MEASURED_PEAKS.json."""
    import torch
    import bench_probes
    from paper_2212_07679_gb300 import snn  # noqa: F401
    torch.cuda.set_device(0)
    iters = {"bf16_mma": 1 << 17, "e4m3_mma": 1 << 17, "fp32_fma": 1 << 18, "fp64_fma": 1 << 12}
    for k, it in iters.items():
        for _ in range(max(1, args.warmup)):
            bench_probes.measure_peak(k, it)
    clk = ClockSampler(0)
    clk.start()
    res = {}
    for k, it in iters.items():
        res[k] = max(bench_probes.measure_peak(k, it) for _ in range(max(1, args.steps))) / 1e12
    clocks = clk.stop()
    peaks, src = load_peaks()
    line = {"metric": "probe_peak_tflops", "value": res["e4m3_mma"], "unit": "TFLOP/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "e4m3",
            "data": "synthetic", "config": {"workload": "peak_probes", "iters": iters},
            "probes_tflops": res, "e4m3_over_bf16": res["e4m3_mma"] / res["bf16_mma"],
            "bf16_probe_over_measured_burst": res["bf16_mma"] / float(peaks["bf16_tflops"]),
            "fp32_lane_clock_model_tflops": FP32_PEAK_TFLOPS, "peaks_source": src, "clocks": clocks}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="gmm_aniso")
    ap.add_argument("--n", type=int, default=0)
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "fp8"])
    ap.add_argument("--no-compare", dest="compare", action="store_false",
                    help="skip timing the other precision beside the headline one")
    ap.add_argument("--ref-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-per-config", dest="per_config", action="store_false",
                    help="skip the other configurations (default run: all of them after the headline)")
    ap.add_argument("--parity-rows", type=int, default=2000,
                    help="oracle rows sampled per configuration for the parity check")
    ap.add_argument("--cfg-budget", type=float, default=3.0,
                    help="seconds of oracle timing per configuration")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "ragged_batch":
        run_ragged(args)
    elif args.workload == "dbscan":
        run_dbscan(args)
    elif args.workload == "stream":
        run_stream(args)
    elif args.workload == "mips_like":
        run_mips(args)
    elif args.workload == "peaks":
        run_peaks(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
