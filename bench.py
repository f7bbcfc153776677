"""Benchmark of exact DTW 1-NN search on GB300 (one JSON line on stdout).

Workload: the largest single-GPU search, 1,024 queries x 100,000 candidates,
L=2,048, D=32, Sakoe-Chiba W=102 (5% of L), LB_PC K=64, seeded prototype-warp data
(100 prototypes, sigma 0.2): 26 GB of candidates resident in HBM.  A step is one
exact nearest-neighbour search of a batch of 256 of the 1,024 queries against all
100,000 candidates (the batches rotate, so four steps cover the query set):
envelopes, LB_MV, seeds, compaction, gated LB_PC / LB_TI, abandoning DTW and the
refine -- the whole hot path, all in the library's kernels.  The value is
whole-job queries/s.  No L2 flush is needed: the inputs (26 GB) are far larger
than the 129 MB L2.

Side legs measure the other workloads on the same GPU: 256 x 20,000 (L=256, D=5),
the uneven batch, the differentiable DTW pairs and the 16 x 256 search.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       [--queries M --candidates N]  (a smaller slice of the same workload, e.g. for
       a profiler capture)
Under torchrun (N > 1) every rank searches its own replica of the batch (weak
scaling, no collective on the data path); the slowest rank's time counts.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "NN queries/s & DTW cell-updates/s at exact NN; % of HBM/FP32 roofline"
WORKLOAD = synth.PROTO_1024x100000_L2048     # the headline search
SIDE = synth.PROTO_256x20000_L256            # side leg: the mid-size search
STEP_QUERIES = 256                           # queries per step (one search call)
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
SM_COUNT_NOMINAL = 152
FP32_LANES_PER_SM = 128


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extra", action="store_true", help="skip the unpruned and end-to-end legs")
    ap.add_argument("--no-few", action="store_true", help="skip the few-queries leg")
    ap.add_argument("--queries", type=int, default=0, help="queries of the workload to use (0 = all 1,024)")
    ap.add_argument("--candidates", type=int, default=0, help="candidates to use (0 = all 100,000)")
    ap.add_argument("--leg", choices=["batched", "pairs", "cascade", "few"], default=None,
                    help="run only this side leg and print its JSON (for profiler runs)")
    ap.add_argument("--workload", choices=["large", "mid"], default="large",
                    help="the search the timed steps run: the 1,024 x 100,000 headline (default) or the 256 x "
                         "20,000 one (for profiler captures of its kernels)")
    return ap.parse_args()


def _dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def job_time_ms(local_ms, dist=None, device=None):
    """The job's time: the maximum over ranks of each rank's timed milliseconds (the
    slowest replica decides); without a process group, the local time."""
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, units_per_rank_step, steps, total_ms):
    """Whole-job throughput: every rank processes its own units each step (weak
    scaling, no exchange), so the job did world * units * steps in the slowest time."""
    return world * units_per_rank_step * steps / (total_ms / 1e3)


def _config(M, N, extra=None, wl=None):
    wl = wl or WORKLOAD
    name = wl.name if (M, N) == (wl.M, wl.N) else f"{wl.name}_slice_{M}q_{N}c"
    gen = ("prototype-warp, 100 prototypes, sigma 0.2, z-normalised, seed 0" if wl is WORKLOAD else
           "prototype-warp, 20 prototypes, sigma 0.1, z-normalised, seed 0")
    c = {"workload": name, "M": M, "N": N, "L": wl.spec.L, "D": wl.spec.D, "W": wl.W, "K": wl.K,
         "queries_per_step": min(STEP_QUERIES, M),
         "step": "one exact search of a batch of the queries against all candidates; batches rotate",
         "generator": gen,
         "l2": ("not flushed: inputs (candidates N*L*D*4 bytes) larger than L2" if wl is WORKLOAD else
                "not flushed (a profiling run of the mid-size search; its side leg flushes)"),
         "parallelism": "replicas"}
    if extra:
        c.update(extra)
    return c


# ----------------------------------------------------------------- CPU oracle legs

def few_queries_leg(tc, cand, q, wl, flush, stream, Ms=(1, 2, 4, 8, 16), reps=10):
    """Searches of a few queries against the full candidate set: the LB_MV stream is
    then one pass over the candidates (HBM-bound; TMA-fed, stream-K split), the rest of
    the search is latency-bound.  Stage times come from CUDA events inside the replayed
    graph (no host gaps).  Before every call the L2 is flushed by writing a 256 MB
    buffer; in the `clean` timing a read of a second 256 MB buffer follows, so that the
    flush's dirty lines are written back before the timed call (a write-only flush leaves
    the L2 full of dirty lines, and their write-back then runs inside the LB_MV stream,
    which streams the 102 MB candidate set at the same time)."""
    import torch
    hbm = _peaks().get("hbm_gbs")
    cand_bytes = wl.N * wl.spec.L * wl.spec.D * 4
    rd = torch.ones(flush.numel(), dtype=torch.float32, device=flush.device)
    out = {"M": list(Ms), "lb_mv_us": [], "lb_mv_hbm_frac": [], "search_us": [],
           "lb_mv_us_dirty_l2": [], "lb_mv_hbm_frac_dirty_l2": []}
    for M in Ms:
        x = tc.Index(cand, wl.W, wl.K)
        qm = q[:M].contiguous()
        o = (torch.empty(M, dtype=torch.int64, device=q.device), torch.empty(M, dtype=torch.float64, device=q.device))
        for _ in range(3):
            x.nn(qm, out=o)
        torch.cuda.synchronize()
        for clean in (True, False):
            x.set_profiling(True)
            tot = 0.0
            for _ in range(reps):
                flush.zero_()
                if clean:
                    rd.amax()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                x.nn(qm, out=o)
                e1.record(stream)
                e1.synchronize()
                tot += e0.elapsed_time(e1)
            st, _ = x.stage_times()
            x.set_profiling(False)
            t_mv = (st["lb_mv"] + st["lb_rest"]) / reps / 1e3
            frac = cand_bytes / t_mv / 1e9 / hbm if hbm else None
            if clean:
                out["lb_mv_us"].append(t_mv * 1e6)
                out["lb_mv_hbm_frac"].append(frac)
                out["search_us"].append(tot / reps * 1e3)
            else:
                out["lb_mv_us_dirty_l2"].append(t_mv * 1e6)
                out["lb_mv_hbm_frac_dirty_l2"].append(frac)
        x.close()
    del rd
    out["note"] = ("lb_mv_hbm_frac: candidate bytes / LB_MV stage time / measured HBM copy bandwidth, L2 "
                   "flushed clean before each call (written, then evicted by a 256 MB read); "
                   "*_dirty_l2: the same after the write alone; search_us: whole tcdtw_nn call, profiling "
                   "events on, clean flush")
    return out


def _gen_batched_set(args):
    """One set of the uneven batch (runs in a spawned worker process)."""
    k, n_sets, M, seed, scale = args
    wl = synth.batched_sets(n_sets, M, seed, scale)[k]
    return k, wl.candidates(), wl.queries()


def batched_leg(tc, dev, reps=5):
    """The uneven batch (32 sets, L ~ U[64,1024], D ~ U{2..12}, N ~ U[1k,20k], 64
    queries each, W = 10% of L, prototype warp): tcdtw_batch_nn (graph replay) against
    the same sets searched one after another through prebuilt indexes."""
    import multiprocessing as mp
    import torch
    n_sets, M = 32, 64
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        parts = sorted(pool.map(_gen_batched_set, [(k, n_sets, M, 0, 1.0) for k in range(n_sets)]),
                       key=lambda r: r[0])
    gen_s = time.perf_counter() - t0
    wls = synth.batched_sets(n_sets, M, 0, 1.0)
    sets = [{"cand": torch.from_numpy(c).to(dev), "q": torch.from_numpy(q).to(dev), "W": w.W, "K": w.K}
            for (_, c, q), w in zip(parts, wls)]
    del parts
    out = [(torch.empty(w.M, dtype=torch.int64, device=dev), torch.empty(w.M, dtype=torch.float64, device=dev))
           for w in wls]
    n_q = sum(w.M for w in wls)
    stream = torch.cuda.current_stream()

    def timed(fn):
        fn()
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    t0 = time.perf_counter()
    tiles = tc.batch_tiles(sets)
    tune_s = time.perf_counter() - t0
    _, st = tc.batch_nn(sets, out=out, stats=True)
    l0 = tc.kernel_launches()
    b_ms = timed(lambda: tc.batch_nn(sets, out=out))
    b_launches = (tc.kernel_launches() - l0) // (reps + 2)
    got = [o[0].clone() for o in out]
    idxs = [tc.Index(s["cand"], s["W"], s["K"]) for s in sets]

    def seq():
        for x, s_, o in zip(idxs, sets, out):
            x.nn(s_["q"], out=o)
    s_ms = timed(seq)
    same = all(torch.equal(g, o[0]) for g, o in zip(got, out))
    for x in idxs:
        x.close()
    assert same, "batched and per-set searches disagree"
    del sets, out
    torch.cuda.empty_cache()
    return {"workload": f"uneven batch: {n_sets} sets x {M} queries, L~U[64,1024], D~U{{2..12}}, N~U[1k,20k], "
                        "W=10% of L, prototype warp",
            "queries": n_q, "pairs": st["pairs"], "ms_per_call": b_ms, "queries_per_s": n_q / (b_ms / 1e3),
            "dtw_cells": st["cells"], "cell_updates_per_s": st["cells"] / (b_ms / 1e3),
            "pruning_rate": 1.0 - st["dtw_started"] / st["pairs"], "kernels_per_call": int(b_launches),
            "per_set_calls_ms": s_ms, "speedup_vs_per_set_calls": s_ms / b_ms, "same_indices": same,
            "tiles_R_G": tiles, "tile_choice_s": tune_s,
            "tile_shapes_L_D_W": [[w.spec.L, w.spec.D, w.W] for w in wls],
            "generation_s": gen_s, "note": "device-resident inputs, L2 not flushed (5.8 GB of candidates >> L2); "
                                           "per-set band tiles from the single-set tuner (tiles_R_G)"}


def _fill_large_chunk(args):
    """Worker: candidate chunk c of the large workload into the shared buffer."""
    name, c, N = args
    from multiprocessing import shared_memory
    wl = WORKLOAD
    shm = shared_memory.SharedMemory(name=name)
    try:
        buf = np.ndarray((N, wl.spec.L, wl.spec.D), dtype=np.float32, buffer=shm.buf)
        lo = c * synth.CHUNK
        n = min(synth.CHUNK, N - lo)
        buf[lo:lo + n] = wl.candidates(n, lo)
    finally:
        shm.close()
    return c


def large_candidates(N, dev=None):
    """The first N candidates of the headline workload, generated by spawned workers
    (one 1,024-series chunk each) into shared memory; returned as a device tensor
    (dev given) or as a host copy."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    import torch
    wl = WORKLOAD
    L, D = wl.spec.L, wl.spec.D
    shm = shared_memory.SharedMemory(create=True, size=N * L * D * 4)
    try:
        chunks = -(-N // synth.CHUNK)
        with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1, chunks))) as pool:
            pool.map(_fill_large_chunk, [(shm.name, c, N) for c in range(chunks)])
        host = np.ndarray((N, L, D), dtype=np.float32, buffer=shm.buf)
        out = torch.from_numpy(host).to(dev) if dev is not None else host.copy()
    finally:
        shm.close()
        shm.unlink()
    return out


def pairs_leg(tc, dev, flush, reps=10):
    """The differentiable DTW distance: 1,024 pairs, L=512, D=8, W=51 (random walks).
    Forward alone (no checkpoints), and forward with band-row checkpoints plus the
    backward pass (what one autograd step costs); CUDA events, L2 flushed before every
    repetition."""
    import torch
    wl = synth.PAIRS_1024_L512
    a, b = wl.pairs()
    A, B = torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)
    P, L, D, W = wl.P, wl.L, wl.D, wl.W
    ck = torch.empty(max(1, tc.ckpt_bytes(P, L, D, W) // 4), dtype=torch.float32, device=dev)
    g = torch.ones(P, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / reps

    fwd_ms = timed(lambda: tc.dtw_pairs(A, B, W))
    fb_ms = timed(lambda: (tc.dtw_pairs(A, B, W, ck), tc.dtw_pairs_backward(A, B, W, ck, g)))
    cells = P * synth.band_cells(L, W)
    instr = cells * (2 * D + 3)
    peak = SM_COUNT_NOMINAL * FP32_LANES_PER_SM * 2070e6
    return {"workload": wl.name, "pairs": P, "forward_ms": fwd_ms, "forward_pairs_per_s": P / (fwd_ms / 1e3),
            "forward_cell_updates_per_s": cells / (fwd_ms / 1e3),
            "forward_roofline": {"bound": "alu", "achieved": instr / (fwd_ms / 1e3) / 1e12, "peak": peak / 1e12,
                                 "unit": "Tinstr/s", "frac": instr / (fwd_ms / 1e3) / peak},
            "forward_backward_ms": fb_ms, "forward_backward_pairs_per_s": P / (fb_ms / 1e3),
            "note": "forward: tcdtw_dtw_pairs without checkpoints; forward_backward: with band-row "
                    "checkpoints plus tcdtw_dtw_pairs_backward; algorithmic 2D+3 FP32 operations per band cell"}


def reverse_lb_leg(tc, cand, q, wl, flush, stream, ms_default, reps=5):
    """The candidate-side LB_MV (use_rev=1) on the benchmark search: candidate envelopes
    built once per index, the reverse bound applied to every LB_MV survivor."""
    import torch
    t0 = time.perf_counter()
    x = tc.Index(cand, wl.W, wl.K, use_rev=1)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    out = (torch.empty(wl.M, dtype=torch.int64, device=q.device),
           torch.empty(wl.M, dtype=torch.float64, device=q.device))
    _, _, st = x.nn(q, stats=True)
    for _ in range(2):
        x.nn(q, out=out)
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x.nn(q, out=out)
        e1.record(stream)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    x.close()
    ms = tot / reps
    return {"ms_per_step": ms, "queries_per_s": wl.M / (ms / 1e3), "vs_default_step": ms / ms_default,
            "pruned_rev": st["pruned_rev"], "pruned_mv": st["pruned_mv"], "dtw_started": st["dtw_started"],
            "build_s": build_s,
            "note": "tcdtw_build with use_rev=1 (candidate envelopes, 2*N*L*D floats) and the same search"}


def ti_variants_leg(tc, cand, q, wl, flush, stream, reps=3):
    """Ablation of the tight bounds on a search: each LB_TI variant (Section 4.2) and
    LB_PC (Section 5) alone behind LB_MV on every survivor (gate e = 0), and LB_MV
    alone."""
    import torch
    L = wl.spec.L
    ti = dict(use_pc=0, use_ti=1, e_ti=0.0)
    cases = [("lb_mv_only", dict(use_pc=0, use_ti=0)), ("tip_top_P5", dict(ti, P=5, ti_top=1)),
             ("tip_P5", dict(ti, P=5, ti_top=0)), ("top", dict(ti, P=L, ti_top=1)), ("basic", dict(ti, P=L, ti_top=0)),
             ("lb_pc_Lq2", dict(use_pc=1, use_ti=0, e_pc=0.0, Lq=2)), ("lb_pc_Lq3", dict(use_pc=1, use_ti=0, e_pc=0.0, Lq=3))]
    out = {}
    o = (torch.empty(wl.M, dtype=torch.int64, device=q.device), torch.empty(wl.M, dtype=torch.float64, device=q.device))
    for name, kw in cases:
        x = tc.Index(cand, wl.W, wl.K, select=0, **kw)
        _, _, st = x.nn(q, stats=True)
        for _ in range(2):
            x.nn(q, out=o)
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x.nn(q, out=o)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        x.close()
        out[name] = {"ms_per_step": tot / reps, "pruned_ti": st["pruned_ti"], "pruned_pc": st["pruned_pc"],
                     "dtw_started": st["dtw_started"], "cells": st["cells"]}
    out["note"] = ("each bound alone behind LB_MV on every survivor (gate e = 0): the LB_TI variants (P = L: no "
                   "periodic exact rows) and LB_PC with Lq = 2, 3")
    return out


def cpu_oracle_sample(Q, Cn, W, K, target_s):
    """The paper's pruned search (FP64 oracle, OpenMP over queries) on a bounded
    sample sized for about target_s seconds: a prefix of the queries, or whole passes
    over all of them when one pass is shorter; returns (queries/s, cores, sample
    description, seconds)."""
    import oracle
    cores = oracle.num_threads()
    n = min(len(Q), max(cores, 16))
    t0 = time.perf_counter()
    oracle.nn_pruned(Q[:n], Cn, W, K=K)
    t = time.perf_counter() - t0
    if t < target_s * 0.5 and n < len(Q):
        n2 = int(min(len(Q), max(n + 1, n * target_s / max(t, 1e-3))))
        t0 = time.perf_counter()
        oracle.nn_pruned(Q[:n2], Cn, W, K=K)
        t = time.perf_counter() - t0
        n = n2
    passes = 1
    if t < target_s * 0.5 and n == len(Q):
        passes = int(min(64, max(2, round(target_s / max(t, 1e-3)))))
        t0 = time.perf_counter()
        for _ in range(passes):
            oracle.nn_pruned(Q, Cn, W, K=K)
        t = time.perf_counter() - t0
    what = f"{n} of {len(Q)} queries" if passes == 1 else f"{passes} passes over all {len(Q)} queries"
    return n * passes / t, cores, f"{what} x all {len(Cn)} candidates (pruned FP64 search)", t


def cpu_brute_large_sample(nq, nc=64):
    """FP64 brute force of the largest workload (1,024 x 100,000, L=2,048, D=32, W=102)
    on the host cores: nq queries (one per core) against the first nc candidates, every
    pair's DTW, extrapolated to all 100,000 candidates."""
    import oracle
    wl = synth.PROTO_1024x100000_L2048
    Q, C = wl.queries(nq), wl.candidates(nc)
    t0 = time.perf_counter()
    oracle.nn_brute(Q, C, wl.W)
    secs = time.perf_counter() - t0
    return {"value": nq / (secs * wl.N / nc), "unit": "queries/s", "cores": len(os.sched_getaffinity(0)),
            "seconds": secs,
            "sample": f"{nq} queries x the first {nc} candidates of {wl.name}, FP64 DTW of every pair, "
                      f"extrapolated to all {wl.N} candidates"}


def cpu_brute_sample(Q, Cn, W, n):
    import oracle
    t0 = time.perf_counter()
    oracle.nn_brute(Q[:n], Cn, W)
    return n / (time.perf_counter() - t0)


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------- roofline helpers

def _peaks():
    try:
        return json.load(open(PEAKS_FILE))
    except (OSError, ValueError):
        return {}


def _profile_traffic(profile: str, pairs=None, candidates=None):
    """DRAM bytes per launch from the committed ncu summary profiles/<profile>.md, if the
    kernel source has not changed since the capture (else None): the recorded bytes per
    launch, or the recorded bytes per pair times `pairs` (a capture of a smaller launch
    of the same kernel scaled to the timed one)."""
    path = os.path.join(ROOT, "profiles", f"{profile}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    mp = re.search(r"traffic_bytes_per_pair:\s*([0-9.eE+]+)", text)
    h = re.search(r"source_sha256:\s*([0-9a-f]+)", text)
    src = re.search(r"source_file:\s*(\S+)", text)
    if not ((m or mp or re.search(r"traffic_bytes_per_candidate:", text)) and h and src):
        return None
    try:
        cur = hashlib.sha256(open(os.path.join(ROOT, src.group(1)), "rb").read()).hexdigest()
    except OSError:
        return None
    if not cur.startswith(h.group(1)):
        return None
    mc = re.search(r"traffic_bytes_per_candidate:\s*([0-9.eE+]+)", text)
    if m:
        return float(m.group(1))
    if mc:
        return float(mc.group(1)) * candidates if candidates else None
    return float(mp.group(1)) * pairs if pairs else None


# ----------------------------------------------------------------- our arm

def _roofline(stage_ms_step, st, M, N, L, D, n_sm, peaks, profile_dtw="ncu_k_dtw_nn", profile_mv="ncu_k_lb_mv"):
    """Roofline of the dominant stage of a search step: algorithmic FP32 flops of the
    stage (DTW: (3D+3) per computed band cell -- D subtractions, D multiplies, D
    additions, two minima and one addition; LB_MV: 4 per element and query) over its
    CUDA-event time, against the FP32 peak: SMs x 128 FP32 lanes x 2 flops (FMA) x
    the maximum SM clock."""
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    peak = n_sm * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12          # TFLOP/s
    dtw_s = sum(stage_ms_step.get(k, 0.0) for k in ("dtw", "seed", "seed2")) / 1e3
    mv_s = (stage_ms_step.get("lb_mv", 0.0) + stage_ms_step.get("lb_rest", 0.0)) / 1e3
    if dtw_s >= mv_s:
        flops, secs, kern = st["cells"] * (3.0 * D + 3.0), dtw_s, "k_dtw_nn"
        what = "DTW stage (seeds + survivors): (3D+3) flops per computed band cell"
        traffic = _profile_traffic(profile_dtw, st.get("dtw_started"))
    else:
        terms = st.get("mv_terms") or M * N * L * D
        flops, secs, kern = terms * 4.0, mv_s, "k_lb_mv + k_lb_mv_rest"
        what = ("LB_MV stages (prefix stream + completion of the live pairs): 4 flops per (element, pair) term "
                "summed; with early abandoning fewer terms than pairs x L x D")
        traffic = _profile_traffic(profile_mv, candidates=N)
    ach = flops / secs / 1e12
    return {"bound": "alu", "kernel": kern, "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": traffic,
            "peak_note": f"{n_sm} SMs x 128 FP32 lanes x 2 (FMA) x {sm_mhz:.0f} MHz (derived, not measured)",
            "achieved_note": what + ", per step, over its CUDA-event time inside the timed region"}


def cpu_oracle_large(Q, C_sample, N_full, W, K, target_s):
    """The oracle's pruned search (the paper's loop in FP64, OpenMP over queries, its
    default bounds) on the host cores: rounds of one query per core against the first
    len(C_sample) candidates until target_s seconds have passed (or Q is used up);
    queries/s extrapolated linearly to N_full candidates."""
    import oracle
    cores = oracle.num_threads()
    done, secs = 0, 0.0
    while done < len(Q) and secs < target_s:
        batch = Q[done:done + cores]
        t0 = time.perf_counter()
        oracle.nn_pruned(batch, C_sample, W, K=K)
        secs += time.perf_counter() - t0
        done += len(batch)
    value = done / (secs * N_full / len(C_sample))
    return value, cores, secs, done


def side_leg(tc, dev, flush, stream, a):
    """The mid-size search (256 queries x 20,000 candidates, L=256, D=5, W=26, K=16):
    step = the whole 256-query search with the L2 flushed before it (the 102 MB of
    candidates would otherwise stay in L2); stage split and roofline, unpruned GPU DTW,
    end to end, the oracle on the host cores; plus its few-query, candidate-side bound
    and LB_TI-variant legs."""
    import torch
    wl = SIDE
    Qn, Cn = wl.queries(), wl.candidates()
    cand = torch.from_numpy(Cn).to(dev)
    q = torch.from_numpy(Qn).to(dev)
    index = tc.Index(cand, wl.W, wl.K)
    out = (torch.empty(wl.M, dtype=torch.int64, device=dev), torch.empty(wl.M, dtype=torch.float64, device=dev))
    for _ in range(5):
        index.nn(q, out=out)
    _, _, st = index.nn(q, stats=True)
    reps = 10
    index.set_profiling(True)
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        index.nn(q, out=out)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    stage_ms, _ = index.stage_times()
    index.set_profiling(False)
    ms = statistics.median(ts)
    stage_step = {k: v / reps for k, v in stage_ms.items()}
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    res = {"workload": wl.name, "ms_per_step": ms, "queries_per_s": wl.M / (ms / 1e3),
           "stage_ms_per_step": stage_step, "dtw_tile": index.info(), "tc_dtw_choice": _choice(index),
           "pruning": _pruning(st),
           "roofline": _roofline(stage_step, st, wl.M, wl.N, wl.spec.L, wl.spec.D, n_sm, _peaks()),
           "note": "median of 10 searches, L2 flushed before each, per-stage CUDA events"}
    # unpruned GPU DTW of every pair
    raw = tc.Index(cand, wl.W, wl.K, no_prune=1)
    ri, _ = raw.nn(q)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(2):
        ri, _ = raw.nn(q)
    e1.record(stream)
    torch.cuda.synchronize()
    raw_ms = e0.elapsed_time(e1) / 2
    raw.close()
    assert torch.equal(out[0], ri), "unpruned and pruned searches disagree"
    res["unpruned_gpu"] = {"ms_per_step": raw_ms, "queries_per_s": wl.M / (raw_ms / 1e3),
                           "speedup_of_pruning": raw_ms / ms}
    # end to end: queries from pinned host memory, results back, inside the timing
    qh = torch.from_numpy(Qn).pin_memory()
    oh = (torch.empty(wl.M, dtype=torch.int64).pin_memory(), torch.empty(wl.M, dtype=torch.float64).pin_memory())
    qd = torch.empty_like(q)
    for _ in range(3):
        qd.copy_(qh, non_blocking=True)
        i2, d2 = index.nn(qd)
        oh[0].copy_(i2, non_blocking=True)
        oh[1].copy_(d2, non_blocking=True)
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(reps):
        flush.zero_()
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        qd.copy_(qh, non_blocking=True)
        i2, d2 = index.nn(qd)
        oh[0].copy_(i2, non_blocking=True)
        oh[1].copy_(d2, non_blocking=True)
        s1.record(stream)
        s1.synchronize()
        tot += s0.elapsed_time(s1)
    res["e2e"] = {"value": wl.M * reps / (tot / 1e3), "unit": "queries/s",
                  "h2d_bytes_per_step": int(qh.numel() * 4), "d2h_bytes_per_step": int(wl.M * 16)}
    if not a.no_cpu:
        qps, cores, sample, secs = cpu_oracle_sample(Qn, Cn, wl.W, wl.K, a.cpu_seconds)
        res["cpu_baseline"] = {"value": qps, "unit": "queries/s", "cores": cores, "kind": "oracle",
                               "sample": sample, "seconds": secs}
    res["reverse_lb"] = reverse_lb_leg(tc, cand, q, wl, flush, stream, ms)
    res["ti_variants"] = ti_variants_leg(tc, cand, q, wl, flush, stream)
    if not a.no_few:
        res["few_queries"] = few_queries_leg(tc, cand, q, wl, flush, stream)
    index.close()
    del cand, q
    torch.cuda.empty_cache()
    return res, st


def _pruning(st):
    p = st["pairs"]
    return {"pairs": p, "dtw_started": st["dtw_started"], "rate": 1.0 - st["dtw_started"] / p,
            "skipped_by": {"lb_mv": st["pruned_mv"] / p, "lb_pc": st["pruned_pc"] / p, "lb_ti": st["pruned_ti"] / p},
            "dtw_abandoned": st["dtw_abandoned"], "cells": st["cells"], "refined": st["refined"],
            "refined64": st["refined64"]}


def _choice(index):
    o = index.options()
    if o["use_pc"] and o["use_ti"]:
        return "LB_MV + LB_PC + LB_TI"
    if o["use_pc"]:
        return f"LB_MV + LB_PC (e={o['e_pc']:.2f}, Lq={o['Lq']})"
    if o["use_ti"]:
        return f"LB_MV + LB_TI (e={o['e_ti']:.2f})"
    return "LB_MV alone"


def cascade_leg(tc, dev):
    """Share of DTWs each bound avoids (the synthetic analogue of the paper's skip
    columns, Table 3) on smooth 2-D circles, where the point-based bounds are much
    tighter than LB_MV: each bound alone behind LB_MV (e = 0), and TC-DTW's choice."""
    import torch
    spec = synth.SeriesSpec("circle", 96, 2, 51, sigma=0.01)
    Qn, Cn = synth.generate(spec, synth.ROLE_QUERY, 64), synth.generate(spec, synth.ROLE_CAND, 4000)
    cand, q = torch.from_numpy(Cn).to(dev), torch.from_numpy(Qn).to(dev)
    out = {"workload": "circle_64q_4000c_L96_D2_W12_K8"}
    ref = None
    for name, kw in [("lb_mv_only", dict(use_pc=0, use_ti=0)), ("lb_pc", dict(use_pc=1, use_ti=0, e_pc=0.0)),
                     ("lb_ti", dict(use_pc=0, use_ti=1, e_ti=0.0)), ("tc_dtw", dict())]:
        x = tc.Index(cand, 12, 8, select=0 if kw else 1, **kw)
        i, _, st = x.nn(q, stats=True)
        if name == "tc_dtw":
            i, _, st = x.nn(q, stats=True)       # the choice made by the first call
            out["tc_dtw_choice"] = _choice(x)
        x.close()
        ref = i if ref is None else ref
        assert torch.equal(ref, i), "bound settings disagree on the answer"
        out[name] = _pruning(st)
    return out


def run_ours(a):
    import torch
    world, rank, local = _dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2101_07731_gb300 as tc

    wl = WORKLOAD if a.workload == "large" else SIDE
    M = a.queries or wl.M
    N = a.candidates or wl.N
    B = min(STEP_QUERIES, M)
    nb = max(1, M // B)                       # batches of B queries (a ragged rest is not used)
    L, D = wl.spec.L, wl.spec.D
    t0 = time.perf_counter()
    cand = large_candidates(N, dev) if wl is WORKLOAD else torch.from_numpy(wl.candidates(N)).to(dev)
    Qn = wl.queries(M)
    gen_s = time.perf_counter() - t0
    q = torch.from_numpy(Qn).to(dev)
    batches = [q[b * B:(b + 1) * B] for b in range(nb)]
    t0 = time.perf_counter()
    index = tc.Index(cand, wl.W, wl.K)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()

    outs = [(torch.empty(B, dtype=torch.int64, device=dev), torch.empty(B, dtype=torch.float64, device=dev))
            for _ in range(nb)]
    # warm-up (untimed): the first pass over the batches also collects the counters
    st = None
    for k in range(max(a.warmup, nb)):
        b = k % nb
        if k < nb:
            _, _, s1 = index.nn(batches[b], stats=True, out=outs[b])
            st = s1 if st is None else {kk: st[kk] + s1[kk] for kk in st}
        else:
            index.nn(batches[b], out=outs[b])
    torch.cuda.synchronize()

    # ---- timed region: K steps on device-resident inputs
    index.set_profiling(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    launches0 = tc.kernel_launches()
    with ClockSampler(local) as clocks:
        barrier()
        torch.cuda.synchronize()
        for k in range(a.steps):
            b = k % nb
            ev[k][0].record(stream)
            index.nn(batches[b], out=outs[b])
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = tc.kernel_launches() - launches0
    stage_ms, _ = index.stage_times()
    index.set_profiling(False)
    step_ms = [s_.elapsed_time(e_) for s_, e_ in ev]
    total_ms = job_time_ms(sum(step_ms), dist, dev)
    ms_per_step = total_ms / a.steps
    value = job_value(world, B, a.steps, total_ms)
    stage_step = {k: v / a.steps for k, v in stage_ms.items()}
    # counters per step: st covers the nb batches (M' = nb*B queries)
    per_step = {k: v * B / (nb * B) for k, v in st.items()}
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    band = synth.band_cells(L, wl.W)
    dtw_s = (stage_step["dtw"] + stage_step["seed"] + stage_step["seed2"]) / 1e3
    res = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": _config(M, N, {"parallelism": f"replicas x{world}" if world > 1 else "single GPU"}, wl),
           "gpu_launches": int(launches),
           "step_ms": {"median": statistics.median(step_ms), "min": min(step_ms), "max": max(step_ms)},
           "cell_updates_per_s": {"computed_over_dtw_time": per_step["cells"] / dtw_s if dtw_s > 0 else None,
                                  "effective_full_band_over_step": world * B * N * band / (ms_per_step / 1e3)},
           "pruning": _pruning(st), "tc_dtw_choice": _choice(index),
           "stage_ms_per_step": stage_step, "dtw_tile": index.info(),
           "setup_s": {"generation": gen_s, "build": build_s}}
    res["clocks"] = clocks.summary()
    res["roofline"] = _roofline(stage_step, per_step, B, N, L, D, n_sm, _peaks(),
                                profile_dtw="ncu_k_dtw_nn_6_32_ring_proto_1024x100000")
    # the other large stage against the same FP32 roof
    other = dict(stage_step)
    if res["roofline"]["kernel"] == "k_dtw_nn":
        other["dtw"] = other["seed"] = other["seed2"] = 0.0
    else:
        other["lb_mv"] = other["lb_rest"] = 0.0
    res["roofline_other_stage"] = _roofline(other, per_step, B, N, L, D, n_sm, _peaks(),
                                            profile_mv="ncu_k_lb_mv_rest_tma_proto_1024x100000")
    if res["roofline"]["traffic"] is not None:
        res["roofline"]["traffic_note"] = ("DRAM bytes per pair of an ncu capture of the same kernel (the tuner's "
                                           "16,384-pair launch on a slice of the workload) x the step's DTW pairs")
    mv_s = (stage_step["lb_mv"] + stage_step["lb_rest"]) / 1e3
    if mv_s > 0:
        hbm = _peaks().get("hbm_gbs", 6790.0)
        bytes_mv = N * L * D * 4.0
        res["lb_mv_hbm"] = {"achieved_gbs": bytes_mv / mv_s / 1e9, "peak_gbs": hbm,
                            "frac": bytes_mv / mv_s / 1e9 / hbm,
                            "terms_share": per_step.get("mv_terms", 0) / (B * N * L * D),
                            "note": "candidate bytes (every element read at least once) / time of the LB_MV "
                                    "stages (prefix stream + completion); terms_share: LB_MV terms summed over "
                                    "all B x N x L x D"}

    if not a.no_extra:
        # ---- unpruned GPU DTW (the paper's default: every pair's full DTW, no bound,
        # no abandoning) on a sample of queries, and the same answers
        nu = min(8, B)
        raw = tc.Index(cand, wl.W, wl.K, no_prune=1)
        qs = batches[0][:nu]
        ri, _ = raw.nn(qs)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ri, _ = raw.nn(qs)
        e1.record(stream)
        torch.cuda.synchronize()
        raw_ms = e0.elapsed_time(e1)
        raw.close()
        assert torch.equal(ri, outs[0][0][:nu]), "unpruned and pruned searches disagree"
        raw_qps = nu / (raw_ms / 1e3)
        res["unpruned_gpu"] = {"queries_per_s": raw_qps, "ms": raw_ms, "sample": f"{nu} queries x all {N} "
                               "candidates, full band DTW of every pair (no_prune)",
                               "cell_updates_per_s": nu * N * band / (raw_ms / 1e3),
                               "speedup_of_pruning": value / world / raw_qps}
        # ---- end to end through the public API: each step copies its batch of queries
        # from pinned host memory and reads the answers back, inside the timed region
        qh = torch.from_numpy(Qn).pin_memory()
        qd = torch.empty(B, L, D, dtype=torch.float32, device=dev)
        oh = (torch.empty(B, dtype=torch.int64).pin_memory(), torch.empty(B, dtype=torch.float64).pin_memory())
        for k in range(2):
            qd.copy_(qh[(k % nb) * B:(k % nb + 1) * B], non_blocking=True)
            i2, d2 = index.nn(qd)
            oh[0].copy_(i2, non_blocking=True)
            oh[1].copy_(d2, non_blocking=True)
        torch.cuda.synchronize()
        barrier()
        tot = 0.0
        for k in range(a.steps):
            b = k % nb
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            qd.copy_(qh[b * B:(b + 1) * B], non_blocking=True)
            i2, d2 = index.nn(qd)
            oh[0].copy_(i2, non_blocking=True)
            oh[1].copy_(d2, non_blocking=True)
            s1.record(stream)
            s1.synchronize()
            tot += s0.elapsed_time(s1)
            assert torch.equal(oh[0], outs[b][0].cpu()), "end-to-end answers differ"
        tot = job_time_ms(tot, dist, dev)
        res["e2e"] = {"value": job_value(world, B, a.steps, tot), "unit": "queries/s",
                      "h2d_bytes_per_step": int(B * L * D * 4), "d2h_bytes_per_step": int(B * 16)}
    index.close()
    ns = min(N, 25000)
    C_s = cand[:ns].cpu().numpy() if (rank == 0 and world == 1 and not a.no_cpu) else None
    del cand, q, batches
    torch.cuda.empty_cache()

    if C_s is not None:
        qps, cores, secs, nqc = cpu_oracle_large(Qn[:64], C_s, N, wl.W, wl.K, a.cpu_seconds)
        res["cpu_baseline"] = {"value": qps, "unit": "queries/s", "cores": cores, "kind": "oracle",
                               "sample": f"{nqc} queries x the first {ns} of the {N} candidates (pruned FP64 "
                                         f"search, default bounds, rounds of one query per core until "
                                         f"{a.cpu_seconds:g} s), extrapolated linearly to {N} candidates",
                               "seconds": secs}
        if not a.no_extra:
            res["cpu_bruteforce"] = cpu_brute_large_sample(max(cores, 4))
        del C_s

    if not a.no_extra and world == 1:
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        side, side_st = side_leg(tc, dev, flush, stream, a)
        res["side_proto_256x20000"] = side
        # ---- latency of a small search (16 queries x 256 candidates, L=128, D=3, W=13):
        # launch-bound; repeated calls on the same buffers replay a CUDA graph
        sw = synth.RW_16x256_L128
        sc = torch.from_numpy(sw.candidates()).to(dev)
        sq = torch.from_numpy(sw.queries()).to(dev)
        small = tc.Index(sc, sw.W, sw.K)
        sout = (torch.empty(sw.M, dtype=torch.int64, device=dev), torch.empty(sw.M, dtype=torch.float64, device=dev))
        _, _, small_st = small.nn(sq, stats=True, out=sout)
        for _ in range(5):
            small.nn(sq, out=sout)
        torch.cuda.synchronize()
        reps = 50
        t0 = time.perf_counter()
        for _ in range(reps):
            small.nn(sq, out=sout)
        torch.cuda.synchronize()
        lat = (time.perf_counter() - t0) / reps
        res["small_workload"] = {"workload": sw.name, "ms_per_call": lat * 1e3, "queries_per_s": sw.M / lat,
                                 "pruning": _pruning(small_st), "tc_dtw_choice": _choice(small),
                                 "note": "host wall time per tcdtw_nn call (graph replay, synchronous)"}
        small.close()
        res["pairs"] = pairs_leg(tc, dev, flush)
        res["batched"] = batched_leg(tc, dev)
        res["cascade"] = cascade_leg(tc, dev)
        res["skip_table"] = {
            "note": "share of all query-candidate pairs whose DTW each bound avoided, per workload "
                    "(the synthetic analogue of the paper's skip columns, Table 3)",
            wl.name: res["pruning"]["skipped_by"] | {"dtw_avoided": res["pruning"]["rate"],
                                                    "tc_dtw_choice": res["tc_dtw_choice"]},
            SIDE.name: side["pruning"]["skipped_by"] | {"dtw_avoided": side["pruning"]["rate"],
                                                       "tc_dtw_choice": side["tc_dtw_choice"]},
            sw.name: res["small_workload"]["pruning"]["skipped_by"] | {
                "dtw_avoided": res["small_workload"]["pruning"]["rate"],
                "tc_dtw_choice": res["small_workload"]["tc_dtw_choice"]},
            "uneven_batch": {"dtw_avoided": res["batched"]["pruning_rate"], "tc_dtw_choice": "not applied"},
            res["cascade"]["workload"]: {k: res["cascade"][k]["rate"] for k in
                                         ("lb_mv_only", "lb_pc", "lb_ti", "tc_dtw")} |
                                        {"tc_dtw_choice": res["cascade"]["tc_dtw_choice"]}}
    if rank == 0:
        print(json.dumps(res), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ----------------------------------------------------------------- reference arm

def run_reference(a):
    """The oracle (the paper's pruned search in FP64, OpenMP over queries, its default
    bounds) timed on the host cores, on the headline workload and metric: each step
    searches one query per host core against a bounded prefix of the candidates, and
    the queries/s are extrapolated linearly to all candidates."""
    world, rank, _ = _dist_env()
    if rank != 0:
        return
    import oracle
    wl = WORKLOAD
    M = a.queries or wl.M
    N = a.candidates or wl.N
    cores = oracle.num_threads()
    nq = max(cores, 8)
    ns = min(N, 4096)
    Qn = wl.queries(min(M, max(nq * 4, nq)))
    C_s = large_candidates(ns)
    for k in range(a.warmup):
        oracle.nn_pruned(Qn[:nq], C_s, wl.W, K=wl.K)
    t0 = time.perf_counter()
    for k in range(a.steps):
        lo = (k * nq) % (len(Qn) - nq + 1)
        oracle.nn_pruned(Qn[lo:lo + nq], C_s, wl.W, K=wl.K)
    secs = time.perf_counter() - t0
    value = nq * a.steps / (secs * N / ns)
    res = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": secs / a.steps * 1e3 * N / ns, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": _config(M, N, {"parallelism": "host cores (OpenMP)"}),
           "cpu_baseline": {"value": value, "unit": "queries/s", "cores": cores, "kind": "oracle",
                            "sample": f"per step {nq} queries x the first {ns} of the {N} candidates (pruned "
                                      f"FP64 search), extrapolated linearly to {N} candidates"},
           "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(res), flush=True)


def run_leg(a):
    """One side leg alone (for profiler runs): its JSON object on stdout."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    import paper_2101_07731_gb300 as tc
    if a.leg == "batched":
        res = batched_leg(tc, dev)
    elif a.leg == "pairs":
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        res = pairs_leg(tc, dev, flush)
    elif a.leg == "few":
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        wl = SIDE
        cand = torch.from_numpy(wl.candidates()).to(dev)
        q = torch.from_numpy(wl.queries()).to(dev)
        res = {"workload": wl.name,
               "few_queries": few_queries_leg(tc, cand, q, wl, flush, torch.cuda.current_stream())}
    else:
        res = cascade_leg(tc, dev)
    print(json.dumps({"leg": a.leg, **res}), flush=True)


if __name__ == "__main__":
    args = _args()
    if args.leg:
        run_leg(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
