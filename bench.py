"""Benchmark of the spliced protein-to-genome DP on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Step = one pass of the whole device pipeline (pack, packed-int16 DP with
int32 re-run, traceback, CIGAR compaction) over the 4,096-pair workload
(protein log-normal median 350 aa; Poisson(3) introns; 1 kb flanks; half on
the reverse strand), inputs resident in HBM.  Prints one JSON line.
At N=1 the line also carries, each measured the same way with its own
autotuned launch configuration: the 20,000-pair uneven-size workload
("c3"), the genome-scale candidate regions ("c5"), the plain
one-launch-per-pair form, the anchored modes, pseudogene-aware rescoring,
serving at 2k, 10k and 50k pairs/s for 60 s each, and the CPU oracle.
Under torchrun each rank aligns its own 4,096-pair batch (weak scaling, no
collective on the data path).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Spliced-DP GCUPS + pairs/s, batched vs plain, 1 GB300; serving p50/p99 ms"
WORKLOAD = ("4096 (protein, region) pairs: protein log-normal median 350 aa (50-2000); "
            "Poisson(3) GT-AG introns, log-normal median 800 nt; 10-40% substitutions; 0-3 frameshifts; "
            "1 kb flanks at 40% GC; half reverse strand; seed 2 (+1000 per rank)")
WORKLOAD_C3 = ("20000 (protein, region) pairs, uneven sizes: protein log-uniform 20-5000 aa; introns as the "
               "4096-pair workload plus a 2% tail of 20-100 kb; regions <= 200 kb; 5% score-only decoys; "
               "seed 3 (+1000 per rank)")
WORKLOAD_C5 = ("genome-scale: 500 Mb genome (40% GC) with 20000 planted genes; 200000 proteins (10% sources, "
               "45% 50-70%-identity paralogs, 45% unrelated); host 7-mer seed + chain stand-in, top 3 chains per "
               "protein; every candidate region aligned with traceback; seed 5 (+1000 per rank)")
WORKLOAD_SEED = ("seeding and chaining: the genome-scale workload shrunk 10 times (50 Mb genome, 2000 planted genes, "
                 "20000 proteins); index of the genome, anchors and chains (Eqs. 1-3) of every protein, the first "
                 "3 chains each; seed 5")
# algorithmic integer ops per cell of the DP pass: the 27 max/add of Eq. 7 (I 3, D 3, A/B/C 2 each,
# H 15) and one running maximum for the best cell.  Traceback decisions are re-derived from the
# stored H values along the path only (by the warp that finishes a pair's last strip).
OPS_PER_CELL = 28


def rank_seed(base: int, rank: int) -> int:
    """Each rank aligns its own batch: the workload seed offset by 1000 per rank."""
    return base + 1000 * rank


def job_totals(local_units: float, local_seconds: float, dist=None, device="cpu"):
    """(units summed over ranks, slowest rank's seconds): the whole-job
    throughput is their ratio.  Without a process group, the local values."""
    if dist is None:
        return float(local_units), float(local_seconds)
    import torch

    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())


def _profile_value(key: str):
    """A number from the committed ncu summary of the DP kernel, or None
    unless that summary was taken on the current kernel source."""
    import hashlib
    import re

    try:
        src = open(os.path.join(ROOT, "paper_2210_08052_gb300", "csrc", "dp_kernel.cu"), "rb").read()
        text = open(os.path.join(ROOT, "profiles", "dp16_c2small_full.md")).read()
    except OSError:
        return None
    h = re.search(r"sha256 \(first 16 hex\): ([0-9a-f]{16})", text)
    v = re.search(key + r": ([0-9.]+)", text)
    if not h or not v or hashlib.sha256(src).hexdigest()[:16] != h.group(1):
        return None
    return float(v.group(1))


def _profiled_traffic(cells: float):
    """DRAM bytes per DP launch, from the committed ncu summary, scaled by
    cells; None unless that summary was taken on the current kernel source."""
    import hashlib
    import re

    try:
        src = open(os.path.join(ROOT, "paper_2210_08052_gb300", "csrc", "dp_kernel.cu"), "rb").read()
        text = open(os.path.join(ROOT, "profiles", "dp16_c2small_full.md")).read()
    except OSError:
        return None
    h = re.search(r"sha256 \(first 16 hex\): ([0-9a-f]{16})", text)
    b = re.search(r"traffic_bytes_per_cell: ([0-9.]+)", text)
    if not h or not b or hashlib.sha256(src).hexdigest()[:16] != h.group(1):
        return None
    return float(b.group(1)) * cells


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


class Clocks:
    """Sample nvidia-smi clocks and throttle reasons during the timed region."""

    def __init__(self, device: int):
        self.device = device
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def cpu_baseline(pairs, seconds: float = 15.0, single_core: bool = True):
    """The oracle, as it stands, on the host cores: one pair per thread,
    pairs drawn in a fixed shuffled order until the time budget is spent;
    with single_core, also one thread alone for a fifth of that time."""
    import random
    from concurrent.futures import FIRST_COMPLETED, ThreadPoolExecutor, wait

    import oracle

    oracle.build_oracle()
    cores = os.cpu_count() or 1
    idx = list(range(len(pairs)))
    random.Random(0).shuffle(idx)
    idx = [k for k in idx if pairs[k].cells <= 20_000_000]
    done_cells = 0
    n_done = 0
    t0 = time.perf_counter()
    deadline = t0 + seconds
    with ThreadPoolExecutor(max_workers=cores) as ex:
        it = iter(idx)
        futs = {}

        def submit():
            k = next(it, None)
            if k is None or time.perf_counter() > deadline:
                return False
            p = pairs[k]
            futs[ex.submit(oracle.align, p.prot, p.nt, p.strand)] = p.cells
            return True

        for _ in range(cores):
            if not submit():
                break
        while futs:
            # refill each thread as soon as its pair is done
            done, _ = wait(list(futs), return_when=FIRST_COMPLETED)
            for f in done:
                f.result()
                done_cells += futs.pop(f)
                n_done += 1
                submit()
    dt = time.perf_counter() - t0
    # one core: the same order, one pair after another, for a fifth of the time
    c1 = 0
    n1 = 0
    t1 = time.perf_counter()
    for k in idx if single_core else []:
        if time.perf_counter() - t1 > seconds / 5:
            break
        p = pairs[k]
        oracle.align(p.prot, p.nt, p.strand)
        c1 += p.cells
        n1 += 1
    d1 = time.perf_counter() - t1
    return {"value": done_cells / dt / 1e9, "unit": "GCUPS", "cores": cores, "kind": "oracle",
            "sample": f"{n_done} pairs of the workload ({done_cells / 1e9:.2f} G cells, pairs <= 20 M cells) "
                      f"in {dt:.1f} s, one pair per thread",
            "single_core": {"value": c1 / d1 / 1e9 if (single_core and d1 > 0) else None, "unit": "GCUPS",
                            "sample": f"{n1} pairs ({c1 / 1e9:.3f} G cells) in {d1:.1f} s on one thread"}}


def run_reference(args):
    """Reference arm: the oracle on the host cores, each step a bounded sample."""
    import synth

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    pairs = synth.config2()
    per_step = max(2.0, min(20.0, 90.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_baseline(pairs, per_step / 4, single_core=False)
    vals = []
    t0 = time.perf_counter()
    cb = None
    for _ in range(args.steps):
        cb = cpu_baseline(pairs, per_step, single_core=False)
        vals.append(cb["value"])
    dt = time.perf_counter() - t0
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1000 / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"kind": "oracle", "cores": cb["cores"], "sample": cb["sample"], "value": value,
                             "unit": "GCUPS"},
            "e2e": {"value": value, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def serve_once(mp, pairs, rate: float, seconds: float, device: int):
    """Open-loop Poisson arrivals at `rate` per second for `seconds`.
    Latency (submit -> result available) is recorded by the library; a
    consumer thread drains results."""
    import random

    ctx = mp.mp_dp_init(None, device)
    rng = random.Random(4)
    stop = threading.Event()
    got = [0]

    def consumer():
        while True:
            r = mp.mp_dp_wait_any(ctx, 100_000)
            if r is not None:
                got[0] += 1
            elif stop.is_set():
                break

    t = mp.mp_dp_submit(ctx, pairs[0])                 # start and warm the serving thread
    mp.mp_dp_poll(ctx, t, 30_000_000)
    mp.mp_dp_get_serve_stats(ctx, reset=True)
    th = threading.Thread(target=consumer, daemon=True)
    th.start()
    t0 = time.perf_counter()
    nxt = t0
    k = 0
    while True:
        nxt += rng.expovariate(rate)
        if nxt - t0 > seconds:
            break
        while time.perf_counter() < nxt:
            pass
        mp.mp_dp_submit(ctx, pairs[k % len(pairs)])
        k += 1
    t_sub_end = time.perf_counter()
    deadline = time.perf_counter() + 120
    while mp.mp_dp_get_serve_stats(ctx)["completed"] < k and time.perf_counter() < deadline:
        time.sleep(0.01)
    wall = time.perf_counter() - t0
    st = mp.mp_dp_get_serve_stats(ctx)
    stop.set()
    th.join(timeout=10)
    mp.mp_dp_destroy(ctx)
    return {"rate_per_s": rate, "seconds": seconds, "submitted": k, "completed": int(st["completed"]),
            "offered_per_s": k / (t_sub_end - t0), "pairs_per_s": st["completed"] / wall,
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
            "batches": int(st["batches"]), "mean_batch_pairs": st["mean_batch_pairs"]}


TUNING_KEYS = ("dp16_variant", "dp16_ctas_per_sm", "dp32_ctas_per_sm", "wide_direct", "overlap_waves", "item_order",
               "strip_w")


def load_pairs(mp, pairs):
    """A list of pairs as the C ABI takes them (host memory)."""
    src = mp.PairBatch(pairs)
    return (src, len(pairs), float(sum(p.cells for p in pairs)), sum(len(p.prot) + len(p.nt) for p in pairs),
            pairs.__getitem__)


def load_c5(mp, rank, scale=1.0, device=0):
    """Candidate regions of the genome-scale workload as zero-copy records
    into the genome and protein buffers; the generation and the host seed +
    chain stand-in are input preparation, outside every timed region."""
    import numpy as np

    import synth

    t_gen = time.perf_counter()
    gw = synth.config5(seed=rank_seed(5, rank), scale=scale)
    prep = {"genome_bp": len(gw.genome), "proteins": len(gw.prot_len), "regions": gw.n_regions,
            "regions_per_protein": gw.n_regions / len(gw.prot_len),
            "generate_and_seed_chain_s": time.perf_counter() - t_gen}
    po, pl, no, nl, st_ = gw.region_arrays()
    src = mp.RegionBatch(gw.prot_buf, po, pl, gw.genome, no, nl, st_)
    # the library sends a genome range and a protein range once when the
    # regions (proteins) share them and the ranges are shorter than the
    # records' total length
    ascii_bytes = int(pl.sum() + nl.sum())
    nz, pz = nl > 0, pl > 0
    if nz.any() and pz.any():
        nspan = int((no[nz] + nl[nz]).max() - no[nz].min())
        pspan = int((po[pz] + pl[pz]).max() - po[pz].min())
        if nspan <= int(nl.sum()) and pspan <= int(pl.sum()) and nspan + pspan < ascii_bytes:
            ascii_bytes = nspan + pspan
    workload = WORKLOAD_C5 if scale == 1.0 else WORKLOAD_C5 + f" (scaled by {scale})"
    return src, gw.n_regions, gw.cells(), ascii_bytes, gw.pair, workload, prep


def measure(mp, torch, src, n_pairs, cells, ascii_bytes, steps, warmup, device, dist, flush, mode=0, fixed=None,
            autotune=True, e2e_steps=3, budget=None):
    """Time the device-resident pipeline (inputs in HBM, L2 flushed before
    each step, CUDA events per kernel inside the library, wall time between
    barriers + device syncs) and the end-to-end call with host buffers, with
    the launch configuration the library's autotuner picks for the batch."""
    extra = {"tb_budget_bytes": budget} if budget else {}
    ctx = mp.mp_dp_init(mp.mp_dp_default_params(mode=mode, **extra), device)
    mp.mp_dp_set_timing(ctx, True)
    batch = mp.mp_dp_batch_upload(ctx, src)
    tuning = None
    if fixed:
        mp.mp_dp_set_tuning(ctx, fixed)
        tuning = {"fixed": fixed}
    elif autotune:
        # chosen on this batch, outside the timed region; the timed runs use the choice
        best, tried = mp.mp_dp_autotune(ctx, batch)
        tuning = {"chosen": best, "candidates": tried}

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    clk = Clocks(device).__enter__()         # sampler starts before the warm-up, outside the timed region
    for _ in range(warmup):
        mp.mp_dp_batch_run(ctx, batch)
        mp.mp_dp_batch_sync(ctx)
    dp_ms, rr_ms, tb_ms, tot_ms = [], [], [], []
    clk.samples.clear()
    barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        mp.mp_dp_batch_run(ctx, batch)
        mp.mp_dp_batch_sync(ctx)
        st = mp.mp_dp_get_stats(ctx)
        dp_ms.append(st["dp_ms"]); rr_ms.append(st["rerun_ms"]); tb_ms.append(st["tb_ms"])
        tot_ms.append(st["total_ms"])
    barrier()
    elapsed = time.perf_counter() - t0
    clk.__exit__()
    stats = mp.mp_dp_get_stats(ctx)
    res = mp.mp_dp_batch_download(ctx, batch, raw=True)
    mp.mp_dp_batch_free(ctx, batch)
    all_cells, t_max = job_totals(cells, elapsed, dist, "cuda")
    # ---- end to end through the C ABI with host buffers
    mp.mp_dp_set_timing(ctx, False)
    out = res
    if e2e_steps:
        mp.mp_dp_align_batch(ctx, src, raw=True)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        out = mp.mp_dp_align_batch(ctx, src, raw=True)
    barrier()
    e2e_t = max(time.perf_counter() - t0, 1e-9)
    _, e2e_t = job_totals(cells, e2e_t, dist, "cuda")
    mp.mp_dp_destroy(ctx)
    h2d = ascii_bytes + n_pairs * (72 + 4)          # sequences + pair descriptors + work order
    d2h = n_pairs * 32 + 4 + int(out["n_cigar"].sum()) * 4
    e2e = {"value": all_cells / (e2e_t / e2e_steps) / 1e9 if e2e_steps else None, "unit": "GCUPS",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
    return {"elapsed": elapsed, "t_max": t_max, "all_cells": all_cells, "steps": steps,
            "kernel_ms": {"dp_int16": statistics.mean(dp_ms), "rerun_int32": statistics.mean(rr_ms),
                          "traceback_compact": statistics.mean(tb_ms), "pipeline": statistics.mean(tot_ms)},
            "dp_ms": dp_ms, "tot_ms": tot_ms, "waves": stats["n_waves"], "code_bytes": stats["code_bytes"],
            "moved": {k: stats[k] for k in ("record_bytes", "record_read_bytes", "boundary_bytes")},
            "launches": stats["n_launches"], "n_rerun": int(((res["status"] & 1) != 0).sum()),
            "clocks": clk.summary(), "tuning": tuning, "e2e": e2e,
            "e2e_s": e2e_t / e2e_steps if e2e_steps else None}


def roofline(m, cells, torch, device, peaks):
    """Integer-issue roofline of the DP kernel: int16 lane-ops of Eq. 7 per
    cell over the kernel's time (CUDA events; for a batch of several waves
    the whole pipeline's time, since overlapped waves' DP intervals
    overlap), against N_SM x 128 lanes x 2 int16 halves x f_SM."""
    clocks = m["clocks"]
    nsm = torch.cuda.get_device_properties(device).multi_processor_count
    f_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    peak_ops = nsm * 128 * 2 * f_mhz * 1e6 / 1e12          # int16 lane-ops/s (Tops)
    dp_avg_ms = statistics.mean(m["dp_ms"]) if m["dp_ms"] else None
    time_basis = "DP kernel launch (CUDA events on its stream)"
    if m["waves"] > 1:
        dp_avg_ms = statistics.mean(m["tot_ms"]) if m["tot_ms"] else None
        time_basis = "whole pipeline (several waves)"
    achieved = cells * OPS_PER_CELL / (dp_avg_ms / 1000) / 1e12 if dp_avg_ms else None
    ips = _profile_value("instructions_per_step")
    return {"bound": "alu", "achieved": achieved, "peak": peak_ops, "unit": "Tops/s (int16 lane-ops)",
            "frac": (achieved / peak_ops) if achieved else None, "traffic": _profiled_traffic(cells),
            "ops_per_cell": OPS_PER_CELL, "time_basis": time_basis,
            "peak_basis": f"{nsm} SMs x 128 lanes x 2 int16 halves x {f_mhz:.0f} MHz (median SM clock under load)",
            "hbm_write_gbs": m["code_bytes"] / (dp_avg_ms / 1000) / 1e9 if dp_avg_ms else None,
            "bytes_by_construction": {
                "stream_written": m["code_bytes"], "records_written": m["moved"]["record_bytes"],
                "records_read_by_strips": m["moved"]["record_read_bytes"],
                "boundary_rows": m["moved"]["boundary_bytes"],
                "stream_per_cell": m["code_bytes"] / cells if cells else None,
                "basis": "counted by the library's planner for this run, per pipeline run: the H stream "
                         "(padding of the last strip and chunk and the column maxima included), the per-nt "
                         "records (written once, read by every strip of the pair, mostly from L2), the "
                         "boundary rows between strips (written and read once, mostly in L2); "
                         "'traffic' is the DRAM count of the committed ncu capture, scaled by cells"},
            "issue_frac": (cells / 64 * ips / (dp_avg_ms / 1000) / (nsm * 4 * f_mhz * 1e6))
            if (dp_avg_ms and ips) else None,
            "issue_basis": "warp-instructions per 64-cell step from the committed ncu summary x steps/s "
                           "over N_SM x 4 issue slots x f_SM",
            "hbm_peak_gbs": peaks.get("hbm_gbs")}


def with_ceilings(roof, mp, m, cells, torch, device):
    """Add the measured integer ceilings (mp_dp_op_rates): each packed
    operation's rate alone and the int16 step's arithmetic alone at full
    occupancy, and the DP kernel's fraction of the latter."""
    try:
        r = mp.mp_dp_op_rates(device if isinstance(device, int) else (device.index or 0))
    except Exception as exc:                      # reported, not fatal: the main figures stand
        roof["alu_ceilings"] = {"error": str(exc)}
        return roof
    nsm = torch.cuda.get_device_properties(device).multi_processor_count
    f_mhz = m["clocks"].get("sm_mhz") or 2070.0
    dp_ms = statistics.mean(m["tot_ms"] if m["waves"] > 1 else m["dp_ms"]) if m["dp_ms"] else None
    step_cells_s = r["step_cells_per_clk_sm"] * nsm * f_mhz * 1e6
    roof["alu_ceilings"] = {
        **{k: round(v, 3) if isinstance(v, float) else v for k, v in r.items()},
        "unit": "warp instructions per clock per SM (each operation alone); cells per clock per SM (step)",
        "step_ceiling_gcups": step_cells_s / 1e9,
        "frac_of_step_ceiling": (cells / (dp_ms / 1000) / step_cells_s) if dp_ms else None,
        "basis": "SM clocks counted in the kernels; the step ceiling is the int16 step's arithmetic on "
                 "register state at full occupancy, without records, profile loads, stream stores or waits",
    }
    return roof


def seed_chain_leg(mp, torch, device, scale=0.1, reps=3):
    """The seeding and chaining stage on the GPU through the C ABI (host
    genome and proteins in, chains out): index build and chaining timed
    separately, the median of `reps` runs each."""
    import synth

    gw = synth.config5(scale=scale, host_seeding=False)
    ctx = mp.mp_dp_init(None, device)
    t_idx, t_ch = [], []
    chains = nch = None
    for _ in range(reps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        idx = mp.mp_index_build(ctx, gw.genome)
        t1 = time.perf_counter()
        chains, nch = mp.mp_index_chain(ctx, idx, gw.prot_buf, gw.prot_off, gw.prot_len, 3)
        t2 = time.perf_counter()
        mp.mp_index_free(idx)
        t_idx.append(t1 - t0)
        t_ch.append(t2 - t1)
    # the second round over the chains' candidate regions
    wr = synth.regions_from_chains(gw, chains, nch)
    po, pl, no, nl, sd = wr.region_arrays()
    pairs = mp.RegionBatch(wr.prot_buf, po, pl, wr.genome, no, nl, sd)
    t_rf = []
    refined = None
    for _ in range(reps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        refined = mp.mp_chain_refine(ctx, pairs)
        t_rf.append(time.perf_counter() - t0)
    mp.mp_dp_destroy(ctx)
    ti, tc, tr = statistics.median(t_idx[1:]), statistics.median(t_ch[1:]), statistics.median(t_rf[1:])
    cells = float((pl.astype("float64") * nl).sum())
    return {"workload": WORKLOAD_SEED, "genome_bp": len(gw.genome), "proteins": len(gw.prot_len),
            "index_build_ms": ti * 1000, "chain_ms": tc * 1000, "genome_mb_per_s": len(gw.genome) / ti / 1e6,
            "proteins_per_s": len(gw.prot_len) / tc, "chains": int(nch.sum()),
            "refine": {"regions": wr.n_regions, "ms": tr * 1000, "regions_per_s": wr.n_regions / tr,
                       "kmer_pairs_per_s": cells / tr,
                       "chained": int((refined["n_anchors"] >= 2).sum()),
                       "what": "second chaining round: every 5-mer of each protein against every base's 5-mer "
                               "of its candidate regions (chain span and flanks), g' = 3dy - dx"},
            "unit": "wall time through the C ABI (host buffers in, chains out), median of 3 after a warm-up"}


def leg(mp, torch, name, loader, device, flush, peaks, steps=3, warmup=3, budget=None):
    """A further workload measured like the main line (its own autotuned
    configuration, device-resident value, end-to-end figure, roofline)."""
    src, n_pairs, cells, ascii_bytes, get_pair, workload, prep = loader()
    m = measure(mp, torch, src, n_pairs, cells, ascii_bytes, steps, warmup, device, None, flush, e2e_steps=2,
                budget=budget)
    if budget:
        prep = dict(prep, tb_budget_bytes=budget)
    e2e = m["e2e"]
    e2e["pairs_per_s"] = n_pairs / m["e2e_s"]
    return {"workload": workload, "value": cells / (m["t_max"] / steps) / 1e9, "unit": "GCUPS",
            "pairs_per_s": n_pairs / (m["t_max"] / steps), "ms_per_step": m["t_max"] * 1000 / steps,
            "steps": steps, "warmup": warmup, "pairs": n_pairs, "cells": cells, "waves": m["waves"], **prep,
            "kernel_ms": m["kernel_ms"], "n_rerun": m["n_rerun"], "roofline": roofline(m, cells, torch, device, peaks),
            "clocks": m["clocks"], "tuning": m["tuning"], "e2e": e2e,
            "gpu_launches": m["launches"] * steps}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip plain/serving/cpu legs")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-rates", default="2000,10000,50000")
    ap.add_argument("--legs", default="c3,c5,seed", help="further workloads measured after the main line "
                                                       "(c3: 20,000 uneven pairs; c5: genome-scale regions; seed: "
                                                       "GPU seeding and chaining); '' for none")
    ap.add_argument("--pairs", type=int, default=4096, help="first N pairs of the workload (profiling runs)")
    ap.add_argument("--skip-e2e", action="store_true", help="profiling runs: skip the end-to-end leg")
    ap.add_argument("--no-autotune", action="store_true", help="default launch configuration, no tuning runs")
    ap.add_argument("--tuning", default="", help="fixed launch configuration 'variant,ctas16,ctas32,wide_direct[,overlap_waves[,item_order]]'")
    ap.add_argument("--c5-scale", type=float, default=1.0, help="shrink the genome-scale workload (tests)")
    ap.add_argument("--mode", default="local", choices=["local", "global", "extension"],
                    help="DP mode of the main leg (profiling runs; the bench line reports local mode)")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c5", "seed"],
                    help="c2: the 4,096-pair batch (default); c3: the 20,000-pair uneven-size stress batch; "
                         "c5: the candidate regions of the genome-scale workload; seed: only the GPU seeding and "
                         "chaining of the genome-scale workload shrunk by --seed-scale (profiling runs)")
    ap.add_argument("--seed-scale", type=float, default=0.1, help="size of the seeding and chaining workload")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import numpy as np

    import synth
    import paper_2210_08052_gb300 as mp
    from paper_2210_08052_gb300 import build as mpbuild

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if args.workload == "seed":
        mpbuild.build()
        print(json.dumps({"metric": METRIC, "seed_chain": seed_chain_leg(mp, torch, local, args.seed_scale)}),
              flush=True)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0 or world == 1:
        mpbuild.build()
    if dist:
        dist.barrier()
    mpbuild.build()

    if args.workload == "c5":
        src, n_pairs, cells, ascii_bytes, get_pair, workload, prep = load_c5(mp, rank, args.c5_scale, local)
        pairs = None
    else:
        if args.workload == "c3":
            pairs = synth.config3(seed=rank_seed(3, rank))[: args.pairs if args.pairs != 4096 else None]
            workload = WORKLOAD_C3
        else:
            pairs = synth.config2(seed=rank_seed(2, rank))[: args.pairs]
            workload = WORKLOAD
        src, n_pairs, cells, ascii_bytes, get_pair = load_pairs(mp, pairs)
        prep = {}
    mode = {"local": 0, "global": 1, "extension": 2}[args.mode]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    flush.zero_()                            # first touch of the flush buffer stays outside the timed region
    torch.cuda.synchronize()
    fixed = None
    if args.tuning:
        # a fixed launch configuration: int16 build, CTAs/SM (int16, int32), wide pairs direct, then
        # optionally the wave policy, the item order and the strip width (defaults 1, 1, 0)
        vals = [int(x) for x in args.tuning.split(",")]
        vals += [1, 1, 0][max(0, len(vals) - 4):]
        fixed = dict(zip(TUNING_KEYS, vals))
    m = measure(mp, torch, src, n_pairs, cells, ascii_bytes, args.steps, args.warmup, local, dist, flush,
                mode=mode, fixed=fixed, autotune=not args.no_autotune, e2e_steps=0 if args.skip_e2e else
                max(2, min(args.steps, 3)))
    all_pairs, _ = job_totals(n_pairs, m["elapsed"], dist, "cuda")
    t_max = m["t_max"]
    gcups = m["all_cells"] / (t_max / args.steps) / 1e9
    pairs_per_s = all_pairs / (t_max / args.steps)
    host_batch = src
    e2e = m["e2e"]
    e2e["pairs_per_s"] = all_pairs / m["e2e_s"] if m["e2e_s"] else None

    if rank != 0:
        if dist:
            dist.barrier()
        return

    peaks = _peaks()
    clocks = m["clocks"]
    line = {
        "metric": METRIC, "value": gcups, "unit": "GCUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1000 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i16x2", "data": "synthetic",
        "config": {"workload": workload + ("" if mode == 0 else f" ({args.mode} mode)"), "pairs": n_pairs,
                   "cells": cells, "waves": m["waves"], **prep,
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "256 MB buffer written between timed steps; each step also writes "
                         f"{m['code_bytes'] / 1e9:.1f} GB of traceback codes"},
        "pairs_per_s": pairs_per_s,
        "kernel_ms": m["kernel_ms"],
        "n_rerun": m["n_rerun"],
        "roofline": with_ceilings(roofline(m, cells, torch, local, peaks), mp, m, cells, torch, local),
        "clocks": clocks,
        "gpu_launches": m["launches"] * args.steps,
        "tuning": m["tuning"],
        "e2e": e2e,
    }
    if not args.no_extras and world == 1:
        # plain form: one pair per kernel launch, on a sample, timed three times
        ctxp = mp.mp_dp_init(mp.mp_dp_default_params(max_pairs_per_launch=1), local)
        rng = np.random.default_rng(0)
        sample = [get_pair(int(k)) for k in rng.choice(n_pairs, 48, replace=False)]
        mp.mp_dp_align_batch(ctxp, sample[:2], raw=True)
        bp = mp.mp_dp_batch_upload(ctxp, sample)
        mp.mp_dp_batch_run(ctxp, bp)
        mp.mp_dp_batch_sync(ctxp)
        torch.cuda.synchronize()
        pc = sum(p.cells for p in sample)
        plain_g = []
        for _ in range(3):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            mp.mp_dp_batch_run(ctxp, bp)
            mp.mp_dp_batch_sync(ctxp)
            plain_g.append(pc / (time.perf_counter() - t0) / 1e9)
        mp.mp_dp_batch_free(ctxp, bp)
        mp.mp_dp_destroy(ctxp)
        plain = statistics.median(plain_g)
        # pseudogene-aware rescoring: the end-to-end call with params.exon_rescore
        ctxe = mp.mp_dp_init(mp.mp_dp_default_params(exon_rescore=1), local)
        mp.mp_dp_align_batch(ctxe, host_batch, raw=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(2):
            mp.mp_dp_align_batch(ctxe, host_batch, raw=True)
        te = (time.perf_counter() - t0) / 2
        mp.mp_dp_destroy(ctxe)
        line["exon_rescore"] = {"value": cells / te / 1e9, "unit": "GCUPS (alignment cells; end to end)",
                                "ms_per_call": te * 1000,
                                "extra_ms_over_e2e": te * 1000 - (m["e2e_s"] * 1000 if m["e2e_s"] else 0.0)}
        # anchored modes on the same batch (gap closing between anchors, and
        # extension from an anchor): device-resident inputs, pipeline time by
        # CUDA events, the L2 flushed before each timed run
        anchored = {}
        for mode, name in ((1, "global"), (2, "extension")):
            ctxa = mp.mp_dp_init(mp.mp_dp_default_params(mode=mode, autotune=1), local)
            mp.mp_dp_set_timing(ctxa, True)
            ba = mp.mp_dp_batch_upload(ctxa, src)
            for _ in range(2):                    # autotune on the first run, then a warm-up
                mp.mp_dp_batch_run(ctxa, ba)
                mp.mp_dp_batch_sync(ctxa)
            ams, ars, ads, ats = [], [], [], []
            for _ in range(2):
                flush.zero_()
                torch.cuda.synchronize()
                mp.mp_dp_batch_run(ctxa, ba)
                mp.mp_dp_batch_sync(ctxa)
                sa = mp.mp_dp_get_stats(ctxa)
                ams.append(sa["total_ms"])
                ars.append(sa["rerun_ms"])
                ads.append(sa["dp_ms"])
                ats.append(sa["tb_ms"])
            ra = mp.mp_dp_batch_download(ctxa, ba, raw=True)
            mp.mp_dp_batch_free(ctxa, ba)
            mp.mp_dp_destroy(ctxa)
            anchored[name] = {"value": cells / (statistics.mean(ams) / 1000) / 1e9, "unit": "GCUPS",
                              "pipeline_ms": statistics.mean(ams), "dp_int16_ms": statistics.mean(ads),
                              "int32_ms": statistics.mean(ars), "traceback_ms": statistics.mean(ats),
                              "pairs_with_error_status": int(((ra["status"] & 0xF0) != 0).sum())}
        line["anchored_modes"] = anchored
        line["plain"] = {"value": plain, "unit": "GCUPS", "pairs_per_s": plain * 1e9 / (pc / len(sample)),
                         "runs": plain_g, "spread": [min(plain_g), max(plain_g)],
                         "sample": f"{len(sample)} random pairs of the workload ({pc / 1e9:.3f} G cells), one "
                                   "kernel launch per pair; median of 3 timed runs, L2 flushed before each",
                         "batched_over_plain": gcups / plain}
        # the 20,000-pair uneven-size workload and the genome-scale workload,
        # each measured like the main line with its own autotuned configuration
        if args.workload == "c2" and args.legs:
            if "c3" in args.legs:
                line["c3"] = leg(mp, torch, "c3",
                                 lambda: load_pairs(mp, synth.config3(seed=rank_seed(3, rank))) + (WORKLOAD_C3, {}),
                                 local, flush, peaks)
            if "c5" in args.legs:
                # the genome-scale batch's traceback (several TB) runs in waves under the
                # budget: 150 GiB of the 280 GB on the device (the library caps it at 60% of
                # the free memory) keeps the waves few
                line["c5"] = leg(mp, torch, "c5", lambda: load_c5(mp, rank, args.c5_scale, local), local, flush,
                                 peaks, budget=150 << 30)
        if args.workload == "c2" and "seed" in args.legs:
            line["seed_chain"] = seed_chain_leg(mp, torch, local)
        # serving: open-loop Poisson arrivals at each rate
        try:
            sp = synth.serving_pairs()
            line["serving"] = [serve_once(mp, sp, float(r), args.serve_seconds, local)
                               for r in args.serve_rates.split(",")]
        except Exception as exc:  # noqa: BLE001
            line["serving"] = {"error": str(exc)}
        cpu_pairs = pairs if args.workload != "c5" else \
            [get_pair(int(k)) for k in np.random.default_rng(1).choice(n_pairs, min(n_pairs, 4000), replace=False)]
        line["cpu_baseline"] = cpu_baseline(cpu_pairs)
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()


if __name__ == "__main__":
    main()
