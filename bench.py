#!/usr/bin/env python3
"""Benchmark of the GNN track-finding hot path on one GB300 (or N replicas).

One step = one call of the whole hot path (plane sort, embedding, radius graph,
interaction network, cut, connected components) over one batch of synthetic
events of the batched workload (1000 events, tracks Poisson(150) clipped to
[20, 400], 5 % noise, embed 3-64-64-4, IN h32 K4, mean degree 12). Prints one
JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision fp32|bf16|fp8] [--workload NAME]

--impl reference times the FP64 CPU oracle on the same workload instead. The
only other place this file runs the oracle is the cpu_baseline leg (rank 0,
N = 1, after every timed region; --no-cpu-baseline turns it off): it times the
oracle on the host cores and checks GPU results against it, the headline's
and those of the extra reports (score error, decision agreement, track
metrics). No GPU number comes from the oracle.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2508_07423_gb300 import replicas, synth  # noqa: E402

METRIC = "events/s and hits/s on 1 GB300 (BF16/FP8 batched vs FP32 plain); p99 latency"
DEFAULT_WORKLOAD = "cfg3_batched_bf16"
L2_FLUSH_BYTES = 256 << 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=DEFAULT_WORKLOAD)
    p.add_argument("--precision", default=None)
    p.add_argument("--band", type=float, default=None,
                   help="re-score band |s - cut| in score units (default: the workload's)")
    p.add_argument("--events", type=int, default=None,
                   help="events per step (default: the workload's; smaller for profiling)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--profile-case", default=None,
                   choices=["headline_300ev_bf16", "headline_300ev_bf16_tuned",
                            "headline_300ev_bf16_tma", "headline_300ev_fp32", "triplets_int8_100ev",
                            "cfg4_100ev_fp8"],
                   help="run one small case for a profiler capture (no timing, no JSON line)")
    p.add_argument("--study", default=None, choices=["occupancy"],
                   help="occupancy: throughput per event-size bin instead of the headline")
    return p.parse_args()


def fp32_peak(torch, dev, pk):
    """FP32 SIMT peak (TFLOP/s) of this device: SMs (read from the device) x 128
    FP32 FMA per clock x 2 flop x the maximum SM clock."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return (sms * 128 * 2 * pk["sm_max_mhz"] * 1e6 / 1e12,
            f"derived: {sms} SMs (device query) x 128 FP32 FMA/clk x 2 x max SM clock "
            f"{pk['sm_max_mhz']:.0f} MHz ({pk['src']})")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained"),
                "sm_max_mhz": d.get("sm_max_mhz", 2070.0), "src": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0, "src": "fallback"}


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------
# roofline of one stage
# ----------------------------------------------------------------------------
def stage_work(stage: str, precision: str, N: int, E: int, h: int, K: int, D: int, embed,
               deg: float = 0.0):
    """Algorithmic work of ONE launch of `stage`: (bound, amount, unit-of-amount).

    FP32 SIMT stages are ALU bound (flops); tensor-core and gather stages are
    HBM bound (bytes). The per-unit figure (per edge / per hit) is written
    beside each stage below; amount = figure x units of one launch. `deg` is
    the batch's mean degree 2E/N (out + in edges per hit), for the messages of
    a hit subset.
    """
    sb = 4 if precision == "fp32" else 2   # state bytes per element
    if stage == "rescore_node_messages":
        # FP32 sums over the listed hits: their incident edges' FP32 rows
        # (deg per hit on average), the in-edge ids, the two list bounds, and
        # the 2h-wide FP32 message row written
        return "hbm", N * (deg * (h * 4 + 2) + 16 + 2 * h * 4), "byte"
    if stage == "rescore_node_prep":  # FP32 node encoder + projections (the embedding is reused)
        return "alu", N * 2.0 * (3 * h + h * h + 2 * h * h), "flop"
    if stage.startswith("rescore_"):  # the FP32 re-run (same kernels as the FP32 path)
        precision, stage = "fp32", stage[len("rescore_"):]
    if stage == "edge_update":
        if precision == "fp32":
            # W_e e (h x h) and the second layer (h x h); the h_src / h_dst
            # products come precomputed per hit from the node step
            return "alu", E * 2.0 * (h * h + h * h), "flop"
        # read e, h_src, h_dst rows; write e
        return "hbm", E * (4 * h * sb + 8), "byte"
    if stage == "node_messages":
        # every edge row read twice (its source's out sum, its target's in
        # sum), the in-edge ids, the list bounds; the message row written
        # (BF16 path: rounded to BF16; FP8 path and FP32: FP32)
        mb = 2 if precision == "bf16" else 4
        return "hbm", 2 * E * h * sb + 4 * E + N * (16 + 2 * h * mb), "byte"
    if stage == "node_update":
        if precision == "fp32":
            # node network (3h x h, h x h) and the two projections (2 x h x h)
            return "alu", N * 2.0 * (3 * h * h + h * h + 2 * h * h), "flop"
        # read h and the message row, write h
        mb = 2 if precision == "bf16" else 4
        return "hbm", N * (2 * h * sb + 2 * h * mb), "byte"
    if stage == "edge_encoder":
        if precision == "fp32":
            # 2 h^2 flop per edge against 3 rows of 4h bytes: memory-bound;
            # read the two projection halves P[src], P[dst], write e, indices
            return "hbm", E * (3 * h * 4 + 8), "byte"
        if precision == "bf16":
            # read the FP32 encodings h_src, h_dst (split into hi + lo BF16
            # operands on chip); write e (BF16); indices
            return "hbm", E * (2 * h * 4 + h * sb + 8), "byte"
        # read h_src, h_dst rows; write e; indices
        return "hbm", E * (3 * h * sb + 8), "byte"
    if stage == "node_prep":
        # embedding MLP (FP32 in every precision), plus the FP32 node encoder
        # (3 x h, h x h) and its two projections (2 x h x h) on the FP32 path
        macs = sum(a * b for a, b in zip(embed[:-1], embed[1:]))
        if precision == "fp32":
            macs += 3 * h + h * h + 2 * h * h
        return "alu", N * 2.0 * macs, "flop"
    if stage == "graph":
        # the embeddings read once; per edge (col, src, d2) written, col read
        # back and the in-edge id written; row pointers and in-edge pointers
        return "hbm", N * D * 4 + E * (12 + 4 + 4) + N * 8, "byte"
    if stage == "components":
        return "hbm", E * 9 + N * 16, "byte"
    return "hbm", N * 16, "byte"


# DRAM bytes (read + write) per row of the dominant kernels, from ncu
# captures of 300 events of the same workload (the re-score edge step:
# profiles/k_gnn_f32_rescore_edge_weights_in_smem_300ev.md, variant 2, steps 0
# and 1; the others: profiles/dram_traffic_edge_steps_300ev.md), averaged over
# the captured launches; scaled to this run's rows.
TRAFFIC_PER_ROW = {
    ("rescore_edge_update", "bf16"): 280.3,
    ("edge_update", "bf16"): 116.9,
    ("edge_update", "fp32"): 257.6,
}


# What the counters of the dominant kernels show (ncu --set full, same
# 300-event captures as the traffic above): the roof their work is counted
# against is not what limits them.
COUNTERS = {
    ("rescore_edge_update", "bf16"): {
        "limiter": "latency: FMA pipe 50 % active, DRAM 28 % of peak, warps active 22.6 % of 64 "
                   "(16 resident: registers and shared memory), stalls spread over shared-memory "
                   "operand loads, fixed-latency dependencies and the FMA pipe",
        "fma_pipe_active_pct": 50.1, "dram_pct_of_peak": 28.0, "warps_active_pct": 22.6,
        "source": "profiles/k_gnn_f32_rescore_edge_weights_in_smem_300ev.md"},
}


def stage_rows_per_launch(stage, launches, rows, N, E, K):
    """Mean rows (edges or hits) one launch of `stage` processes."""
    if stage == "rescore_edge_update":
        return sum(rows["edges"][1:K + 1]) / max(launches, 1)
    if stage in ("edge_update", "edge_encoder"):
        return E
    return N


def stage_amount(stage, launches, rows, precision, N, E, m):
    """Algorithmic work of `stage` over one step: (bound, amount). A re-score
    stage works on the receptive field of the band edges, a different row set
    per launch (encoders first, then step 0 .. K-1)."""
    h, K = m["hidden"], m["iters"]
    total, bound = 0.0, "hbm"
    if stage.startswith("rescore_"):
        if stage in ("rescore_edge_encoder", "rescore_node_prep"):
            sets = [(rows["hits"][0], rows["edges"][0])]
        else:
            sets = [(rows["hits"][k + 1], rows["edges"][k + 1]) for k in range(K)]
        sets = sets[:max(launches, 1)]
    else:
        sets = [(N, E)] * max(launches, 1)
    for n_k, e_k in sets:
        bound, amt, _ = stage_work(stage, precision, n_k, e_k, h, K, m["embed"][-1], m["embed"],
                                   deg=2.0 * E / max(N, 1))
        total += amt
    return bound, total


def timed_steps(torch, tr, n_ev, N, xyz, plane, offs, labels, stream, flush, steps, tracks=None):
    """Per-step CUDA-event times on `stream`, L2 flushed between steps;
    `tracks` = (event_tracks, track_off, track_hits) runs the triplet stage."""
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    with torch.cuda.stream(stream):
        for i in range(steps):
            flush.fill_(i)
            ev_s[i].record(stream)
            if tracks is None:
                tr.find_tracks(n_ev, N, xyz, plane, offs, labels, stream)
            else:
                tr.find_tracks_triplets(n_ev, N, xyz, plane, offs, labels, *tracks, stream)
            ev_e[i].record(stream)
    torch.cuda.synchronize()
    tr.sync_status(stream)
    return [s.elapsed_time(e) for s, e in zip(ev_s, ev_e)]


def quick_rate(pkg, torch, wl, batch, dev, stream, flush, steps=5, **kw):
    """events/s of another configuration on the same resident batch."""
    n_ev, N = batch.n_events, batch.n_hits
    xyz = torch.from_numpy(batch.xyz_soa()).to(dev)
    plane = torch.from_numpy(batch.plane).to(dev)
    offs = torch.from_numpy(batch.offsets).to(dev)
    labels = torch.empty(N, dtype=torch.int32, device=dev)
    tr = pkg.tracker_for_workload(wl, max_hits=N, max_events=n_ev, edges_per_hit=16,
                                  use_graph=True, **kw)
    for _ in range(3):
        tr.find_tracks(n_ev, N, xyz, plane, offs, labels, stream)
    tr.sync_status(stream)
    ms = float(np.mean(timed_steps(torch, tr, n_ev, N, xyz, plane, offs, labels, stream,
                                   flush, steps)))
    st = tr.stats()
    tr.close()
    return {"events_per_s": round(n_ev / (ms / 1e3), 1), "ms_per_step": round(ms, 4),
            "band_edges": st["band"], "rerun_events": st["rerun_events"]}


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        return run_reference(a, rank, world)

    import torch
    import paper_2508_07423_gb300 as pkg

    if a.profile_case:
        return profile_case(a.profile_case, pkg, torch)

    if a.study == "occupancy":
        torch.cuda.set_device(local)
        dev = torch.device("cuda", local)
        res = occupancy_study(pkg, torch, dev, torch.cuda.Stream(device=dev))
        if rank == 0:
            print(json.dumps({"study": "occupancy", "metric": METRIC, "unit": "events/s",
                              "data": "synthetic", "rows": res}))
        return

    wl = synth.workload(a.workload)
    precision = a.precision or wl.get("precision", "fp32")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    # each rank processes its own events (replicas over disjoint event ranges)
    first, n_ev = replicas.event_range(rank, world, a.events or wl["n_events"])
    batch = synth.workload_batch(wl, n_ev, first_event=first)
    N = batch.n_hits
    dev = torch.device("cuda", local)
    xyz = torch.from_numpy(batch.xyz_soa()).to(dev)
    plane = torch.from_numpy(batch.plane).to(dev)
    offs = torch.from_numpy(batch.offsets).to(dev)
    labels = torch.empty(N, dtype=torch.int32, device=dev)
    kw = {} if a.band is None else {"rescore_band": a.band}
    tr = pkg.tracker_for_workload(wl, precision=precision, max_hits=N, max_events=n_ev,
                                  edges_per_hit=16, use_graph=True, **kw)
    band = tr.cfg.rescore_band
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    tuned = tr.autotune(n_ev, N, xyz, plane, offs, labels, stream)
    for _ in range(max(a.warmup, 3)):
        tr.find_tracks(n_ev, N, xyz, plane, offs, labels, stream)
        tr.sync_status(stream)
    stats = tr.stats()

    # timed region: CUDA-graph replays, per-step event pairs, L2 flushed between
    # steps (outside the pairs)
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    t0 = time.perf_counter()
    step_ms = timed_steps(torch, tr, n_ev, N, xyz, plane, offs, labels, stream, flush, a.steps)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    if dist:
        dist.barrier()
    ms, total_events, hits_total = replicas.combine(dist, float(np.mean(step_ms)), n_ev, N, dev)
    value = total_events / (ms / 1e3)

    # the same steps again with per-stage events (direct launches): roofline
    tr.set_profiling(True)
    prof_ms = timed_steps(torch, tr, n_ev, N, xyz, plane, offs, labels, stream, flush, a.steps)
    stages = tr.stage_times()
    tr.set_profiling(False)
    pk = peaks()
    m = wl["model"]
    E = stats["edges"]
    dname, (dms, druns) = max(stages.items(), key=lambda kv: kv[1][0])
    rows = tr.rescore_rows()
    bound, amount = stage_amount(dname, druns // a.steps, rows, precision, N, E, m)
    launch_ms = dms / max(druns, 1)
    step_stage_ms = dms / a.steps
    f32_peak, f32_src = fp32_peak(torch, dev, pk)
    if bound == "alu":
        peak = f32_peak
        achieved = amount / (step_stage_ms / 1e3) / 1e12
        unit = "TFLOP/s"
    else:
        peak = pk["hbm_gbs"]
        achieved = amount / (step_stage_ms / 1e3) / 1e9
        unit = "GB/s"
    bpr = TRAFFIC_PER_ROW.get((dname, precision))
    traffic = (round(bpr * stage_rows_per_launch(dname, druns // a.steps, rows, N, E, m["iters"]))
               if bpr is not None and a.workload == "cfg3_batched_bf16" else None)
    # every stage with a work model: achieved rate against its roofline
    per_stage = {}
    for sname, (sms, sruns) in stages.items():
        if sname in ("rescore_field", "sort"):
            continue
        sb_, samt = stage_amount(sname, sruns // a.steps, rows, precision, N, E, m)
        st_ms = sms / a.steps
        if sb_ == "alu":
            pk_, ach, un = f32_peak, samt / (st_ms / 1e3) / 1e12, "TFLOP/s"
        else:
            pk_, ach, un = pk["hbm_gbs"], samt / (st_ms / 1e3) / 1e9, "GB/s"
        per_stage[sname] = {"ms_per_step": round(st_ms, 4), "bound": sb_, "achieved": round(ach, 2),
                            "unit": un, "frac": round(ach / pk_, 4)}
    roof = {"kernel": dname, "bound": bound, "achieved": round(achieved, 2), "peak": peak,
            "unit": unit, "frac": round(achieved / peak, 4), "traffic": traffic,
            "traffic_unit": "DRAM bytes per launch (ncu capture of 300 events scaled by rows)",
            "counters": (COUNTERS.get((dname, precision))
                         if a.workload == "cfg3_batched_bf16" else None),
            "peak_src": f32_src if bound == "alu" else pk["src"],
            "launch_ms": round(launch_ms, 4),
            "work": "algorithmic work of the stage over one step / its time per step",
            "profiled_ms_per_step": round(float(np.mean(prof_ms)), 4),
            "stage_ms_per_step": {k: round(v[0] / a.steps, 4) for k, v in stages.items()},
            "stages": per_stage}

    e2e = None if a.no_e2e else run_e2e(a, tr, batch, stream, dev, torch)
    extra = {}
    if not a.no_plain:
        extra["plain_fp32_one_event_per_launch"] = run_plain(pkg, torch, dev, stream)
        if precision != "fp32":
            extra["no_rescore"] = quick_rate(pkg, torch, wl, batch, dev, stream, flush,
                                             precision=precision, rescore_band=0.0)
        extra["fp32_batched"] = quick_rate(pkg, torch, wl, batch, dev, stream, flush,
                                           precision="fp32")
        extra["serving"] = run_serving(pkg, precision, tuned)
    plain = extra.get("plain_fp32_one_event_per_launch")

    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "events/s", "n_gpus": world,
        "steps": a.steps, "warmup": max(a.warmup, 3), "ms_per_step": round(ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "bf16": "bf16", "fp8": "e4m3"}[precision],
        "data": "synthetic",
        "hits_per_s": round(hits_total / (ms / 1e3), 1),
        "p50_step_ms": round(float(np.percentile(step_ms, 50)), 4),
        "p99_step_ms": round(float(np.percentile(step_ms, 99)), 4),
        "config": {"workload": f"{a.workload}: {wl['description']}",
                   "n_events": n_ev, "hits": N, "edges": E, "kept_edges": stats["kept"],
                   "net": f"embed {'-'.join(map(str, m['embed']))}, IN h{m['hidden']} K{m['iters']}",
                   "precision": precision, "rescore_band": round(float(band), 6),
                   "band_edges": stats["band"], "rerun_events": stats["rerun_events"],
                   "rescore_rows": rows,
                   "launch": "one CUDA graph per step (captured on first use)",
                   "autotuned_ctas_per_sm": tuned,
                   "l2": "flushed between steps (256 MiB write)",
                   "parallelism": f"replicas x{world} (disjoint events, no collective)"},
        "clocks": clk,
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": int(stats["launches"]) * a.steps,
        "batched_over_plain": (round(value / plain["events_per_s"], 2)
                               if plain and plain.get("events_per_s") else None),
        # the same ratio in hits/s (the plain path's 40-track events are
        # smaller than the headline's)
        "batched_over_plain_hits": (round(hits_total / (ms / 1e3) / plain["hits_per_s"], 2)
                                    if plain and plain.get("hits_per_s") else None),
        "wall_s_timed": round(wall, 3),
    }
    out.update(extra)
    if rank == 0 and world == 1 and not a.no_plain:
        # what the tensor pipe sustains at the narrow N of the network's
        # layers (N = hidden), against which the tensor-core kernels' own
        # tensor-pipe activity (profiles) reads
        try:
            out["tcgen05_probe_tflops"] = {
                "what": "back-to-back BF16 MMAs M=128, N=n, K=16, one issuing thread per SM",
                **{f"n{n}": round(pkg.tc_throughput(n), 1) for n in (32, 64, 128, 256)}}
        except Exception as ex:  # reported, not fatal
            out["tcgen05_probe_tflops"] = {"error": str(ex)}
        out["occupancy_study"] = {
            "what": "config-3 model, radius and noise at a fixed tracks per event, about 1.7 M "
                    "hits per batch: batched BF16 + FP32 re-score (one call, CUDA graph) against "
                    "the plain FP32 path (one event per call, 100 events)",
            "rows": occupancy_study(pkg, torch, dev, stream)}
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl, batch, labels.cpu().numpy(), tr, a.cpu_seconds)
        if not a.no_plain:
            out["cfg2_report"] = cfg2_report(pkg, torch, dev, stream)
            out["fp8_report"] = fp8_report(pkg, torch, dev, stream)
            out["fp8_trained_report"] = fp8_trained_report(pkg, torch, dev, stream)
            out["trained_report"] = trained_report(pkg, torch, dev, stream, flush)
            out["triplet_report"] = triplet_report(pkg, torch, dev, stream, flush)
            out["int8_report"] = int8_report(pkg, torch, dev, stream, flush)
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def run_serving(pkg, precision, tuning=None):
    """Config 5: Poisson arrivals at 50 k events/s, continuous batching within a
    40 GB budget; p50/p99 latency and sustained events/s. Each slot's workspace
    holds a batch of up to 256 k hits (about 150 events of this workload, over
    twice the largest batch the arrival rate forms), so 8 slots fit the budget;
    the slots apply the headline's autotuned launch configuration."""
    try:
        wl = synth.workload("cfg5_serving")
        n = wl["n_events"]
        b = synth.workload_batch(wl, n)
        arr = pkg.poisson_arrivals(n, wl["arrival_rate_hz"], wl["seeds"]["arrivals"])
        band = float(wl.get("rescore_band_score", 0.0)) if precision != "fp32" else 0.0
        cfg = pkg.make_cfg(wl["model"], wl["radius2"], k_max=wl["k_max"], precision=precision,
                           rescore_band=band, edges_per_hit=16)
        res = {}
        for name, bnd in (("rescore", band), ("no_rescore", 0.0)):
            cfg.rescore_band = bnd
            _, done, st = pkg.serve_run(synth.workload_weights(wl), cfg, b, arr, n_slots=8,
                                        max_events_per_batch=512, max_hits_per_batch=1 << 18,
                                        memory_budget_bytes=wl["memory_budget_bytes"],
                                        tuning=tuning)
            lat = (done - arr) * 1e3
            res[name] = {"p50_ms": round(float(np.percentile(lat, 50)), 3),
                         "p99_ms": round(float(np.percentile(lat, 99)), 3),
                         "sustained_events_per_s": round(n / (done.max() - arr[0]), 1),
                         "batches": st["batches"], "slots": st["slots"],
                         "slot_bytes": st["slot_bytes"],
                         "max_in_flight": st["max_in_flight"],
                         "largest_batch": st["largest_batch"]}
            if precision == "fp32":
                break
        return {"workload": f"cfg5_serving: {n} events, {wl['description']}",
                "offered_events_per_s": wl["arrival_rate_hz"], "precision": precision, **res}
    except Exception as ex:  # reported, not fatal
        return {"error": str(ex)}


def run_e2e(a, tr, batch, stream, dev, torch):
    N, n_ev = batch.n_hits, batch.n_events
    h_xyz = torch.from_numpy(batch.xyz_soa()).pin_memory()
    h_plane = torch.from_numpy(batch.plane).pin_memory()
    h_offs = torch.from_numpy(batch.offsets).pin_memory()
    h_lab = torch.empty(N, dtype=torch.int32).pin_memory()
    d_xyz = torch.empty_like(h_xyz, device=dev)
    d_plane = torch.empty_like(h_plane, device=dev)
    d_offs = torch.empty_like(h_offs, device=dev)
    d_lab = torch.empty(N, dtype=torch.int32, device=dev)
    ms = []
    with torch.cuda.stream(stream):
        for i in range(max(a.steps // 2, 3) + 2):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            d_xyz.copy_(h_xyz, non_blocking=True)
            d_plane.copy_(h_plane, non_blocking=True)
            d_offs.copy_(h_offs, non_blocking=True)
            tr.find_tracks(n_ev, N, d_xyz, d_plane, d_offs, d_lab, stream)
            h_lab.copy_(d_lab, non_blocking=True)
            e.record(stream)
            e.synchronize()
            if i >= 2:
                ms.append(s.elapsed_time(e))
    m = float(np.mean(ms))
    return {"value": round(n_ev / (m / 1e3), 1), "unit": "events/s",
            "h2d_bytes_per_step": int(h_xyz.numel() * 4 + h_plane.numel() + h_offs.numel() * 8),
            "d2h_bytes_per_step": int(N * 4), "ms_per_step": round(m, 4)}


def run_plain(pkg, torch, dev, stream):
    """cfg1: 100 distinct 40-track events, FP32, one event per call."""
    try:
        wl = synth.workload("cfg1_plain_fp32")
        b = synth.workload_batch(wl)
        tr = pkg.tracker_for_workload(wl, precision="fp32", max_hits=8192, max_events=1)
        evs = []
        for e in range(b.n_events):
            ev = b.event(e)
            evs.append((ev.n_hits, torch.from_numpy(ev.xyz_soa()).to(dev),
                        torch.from_numpy(ev.plane).to(dev), torch.from_numpy(ev.offsets).to(dev),
                        torch.empty(ev.n_hits, dtype=torch.int32, device=dev)))
        for n, x, p, o, l in evs[:5]:
            tr.find_tracks(1, n, x, p, o, l, stream)
        tr.sync_status(stream)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        with torch.cuda.stream(stream):
            s.record(stream)
            for _ in range(reps):
                for n, x, p, o, l in evs:
                    tr.find_tracks(1, n, x, p, o, l, stream)
            e.record(stream)
        e.synchronize()
        tr.sync_status(stream)
        ms = s.elapsed_time(e)
        n = reps * len(evs)
        hits = reps * sum(v[0] for v in evs)
        tr.close()
        return {"events_per_s": round(n / (ms / 1e3), 1), "hits_per_s": round(hits / (ms / 1e3), 1),
                "workload": "cfg1_plain_fp32: 100 distinct 40-track events, FP32, one event per call"}
    except Exception as ex:  # reported, not fatal
        return {"events_per_s": None, "error": str(ex)}


def compare_edges(g, ref, n_hits):
    """One event's GPU graph (`get_graph` dict) against the oracle's
    (`oracle.EventResult`) over the union of both edge sets, an edge absent on
    one side counting as not kept there: (agreeing keep decisions, size of the
    union, |score difference| on the edges both sides hold)."""
    kg = g["src"].astype(np.int64) * n_hits + g["dst"].astype(np.int64)
    ko = ref.src.astype(np.int64) * n_hits + ref.dst.astype(np.int64)
    allk = np.union1d(kg, ko)
    keep_g = np.zeros(allk.size, bool)
    keep_g[np.searchsorted(allk, kg)] = np.asarray(g["kept"]) != 0
    keep_o = np.zeros(allk.size, bool)
    keep_o[np.searchsorted(allk, ko)] = np.asarray(ref.keep) != 0
    _, ig, io = np.intersect1d(kg, ko, assume_unique=True, return_indices=True)
    sig = lambda v: 1.0 / (1.0 + np.exp(-np.asarray(v, np.float64)))
    err = np.abs(sig(np.asarray(g["logit"])[ig]) - sig(ref.logit[io]))
    return int(np.count_nonzero(keep_g == keep_o)), int(allk.size), err


class Agreement:
    """Edge-decision agreement and score error summed over events."""

    def __init__(self):
        self.agree = self.union = self.events = self.n_err = 0
        self.sum_err = self.max_err = 0.0

    def add(self, g, ref, n_hits):
        a, u, err = compare_edges(g, ref, n_hits)
        self.agree += a
        self.union += u
        self.events += 1
        if err.size:
            self.max_err = max(self.max_err, float(err.max()))
            self.sum_err += float(err.sum())
            self.n_err += err.size

    def summary(self):
        return {"events": self.events, "edges_compared": self.union,
                "edge_decision_agreement": round(self.agree / max(self.union, 1), 6),
                "decisions_differing": self.union - self.agree,
                "max_score_error": round(self.max_err, 7),
                "mean_score_error": round(self.sum_err / max(self.n_err, 1), 8)}


def oracle_events(model, batch, idx, wl, fs, threads):
    """The FP64 oracle on events `idx` of `batch`, one event per thread (the
    oracle call releases the GIL)."""
    import concurrent.futures as cf

    import oracle

    def one(e):
        ev = batch.event(e)
        return oracle.find_tracks_event(model, ev.x, ev.y, ev.z, ev.plane, wl["radius2"],
                                        wl["k_max"], wl["cut"], feat_scale=fs)
    with cf.ThreadPoolExecutor(max(1, threads)) as ex:
        return list(ex.map(one, idx))


def cpu_baseline(wl, batch, gpu_labels, tr, seconds, seconds_one_core=4.0):
    """The FP64 oracle on the host cores over a bounded sample of the same events
    (all cores, one event per thread; and one core alone on the first events),
    plus the GPU result's agreement with it on every sampled event."""
    import oracle
    from oracle import metrics
    sh = synth.shape_of(wl)
    model = oracle.Model(synth.workload_weights(wl), sh.embed, sh.hidden, sh.iters)
    import paper_2508_07423_gb300 as pkg
    fs = pkg.feat_scale_of(tr.cfg)
    cores = os.cpu_count() or 1
    # one core
    n1, h1, t1 = 0, 0, 0.0
    while t1 < seconds_one_core and n1 < batch.n_events:
        t0 = time.perf_counter()
        oracle_events(model, batch, [n1], wl, fs, 1)
        t1 += time.perf_counter() - t0
        h1 += int(batch.offsets[n1 + 1] - batch.offsets[n1])
        n1 += 1
    # all cores, `cores` events at a time until the time budget is spent
    done, hits, t_used = 0, 0, 0.0
    refs = []
    while t_used < seconds and done < batch.n_events:
        idx = list(range(done, min(done + cores, batch.n_events)))
        t0 = time.perf_counter()
        refs += oracle_events(model, batch, idx, wl, fs, cores)
        t_used += time.perf_counter() - t0
        done += len(idx)
        hits += int(batch.offsets[done] - batch.offsets[idx[0]])
    lab_ref = np.concatenate([r.labels for r in refs])
    n_s = int(batch.offsets[done])
    same = sum(np.array_equal(gpu_labels[batch.offsets[e]:batch.offsets[e + 1]],
                              lab_ref[batch.offsets[e]:batch.offsets[e + 1]]) for e in range(done))
    cg = metrics.batch_counts(gpu_labels[:n_s], batch.pid[:n_s], batch.offsets[:done + 1]).summary()
    co = metrics.batch_counts(lab_ref, batch.pid[:n_s], batch.offsets[:done + 1]).summary()
    # edge decisions on every sampled event
    ag = Agreement()
    for e in range(done):
        ag.add(tr.get_graph(e), refs[e], int(batch.offsets[e + 1] - batch.offsets[e]))
    agm = ag.summary()
    return {"value": round(done / t_used, 2), "unit": "events/s",
            "hits_per_s": round(hits / t_used, 1), "cores": cores, "kind": "oracle",
            "sample": f"first {done} of the {batch.n_events} benchmark events "
                      f"({hits} hits), FP64 C++ oracle, one event per thread",
            "one_core": {"events_per_s": round(n1 / t1, 3), "hits_per_s": round(h1 / t1, 1),
                         "sample": f"first {n1} events, one after another on one core"},
            "labels_identical_events": f"{same}/{done}",
            "track_efficiency_gpu": round(cg["efficiency"], 6),
            "track_efficiency_oracle": round(co["efficiency"], 6),
            "track_efficiency_delta_pp": round(100 * abs(cg["efficiency"] - co["efficiency"]), 4),
            "edge_decision_agreement": agm["edge_decision_agreement"],
            "edge_decision_events": agm["events"], "edges_compared": agm["edges_compared"],
            "max_score_error": agm["max_score_error"],
            "mean_score_error": agm["mean_score_error"]}


def occupancy_study(pkg, torch, dev, stream, bins=(20, 50, 100, 150, 200, 300, 400),
                    target_hits=1_700_000):
    """Occupancy scaling: events of a fixed track count per bin (config-3
    model, radius and noise), about `target_hits` hits per batch. Batched BF16
    + FP32 re-score (one call, CUDA graph) and the plain FP32 path (one event
    per call, 100 events) per bin: events/s, hits/s and the ratio."""
    wl = synth.workload("cfg3_batched_bf16")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    rows = []
    for nt in bins:
        spec = {"kind": "fixed", "n": nt}
        probe = synth.gen_batch(20, 7700 + nt, spec, wl["noise"])
        n_ev = max(20, int(target_hits / (probe.n_hits / probe.n_events)))
        b = synth.gen_batch(n_ev, 7700 + nt, spec, wl["noise"])
        band = float(wl.get("rescore_band_score", 0.0))
        xyz = torch.from_numpy(b.xyz_soa()).to(dev)
        plane = torch.from_numpy(b.plane).to(dev)
        offs = torch.from_numpy(b.offsets).to(dev)
        lab = torch.empty(b.n_hits, dtype=torch.int32, device=dev)
        tr = pkg.tracker_for_workload(wl, precision="bf16", rescore_band=band, max_hits=b.n_hits,
                                      max_events=b.n_events, edges_per_hit=16, use_graph=True)
        for _ in range(3):
            tr.find_tracks(b.n_events, b.n_hits, xyz, plane, offs, lab, stream)
        tr.sync_status(stream)
        ms = float(np.mean(timed_steps(torch, tr, b.n_events, b.n_hits, xyz, plane, offs, lab,
                                       stream, flush, 5)))
        st = tr.stats()
        tr.close()
        # plain FP32, one event per call
        trp = pkg.tracker_for_workload(wl, precision="fp32", max_hits=max(b.event(e).n_hits for e in range(100)),
                                       max_events=1, edges_per_hit=16)
        evs = []
        for e in range(min(100, b.n_events)):
            ev = b.event(e)
            evs.append((ev.n_hits, torch.from_numpy(ev.xyz_soa()).to(dev), torch.from_numpy(ev.plane).to(dev),
                        torch.from_numpy(ev.offsets).to(dev), torch.empty(ev.n_hits, dtype=torch.int32, device=dev)))
        for n_, x_, p_, o_, l_ in evs[:3]:
            trp.find_tracks(1, n_, x_, p_, o_, l_, stream)
        trp.sync_status(stream)
        s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            s_.record(stream)
            for n_, x_, p_, o_, l_ in evs:
                trp.find_tracks(1, n_, x_, p_, o_, l_, stream)
            e_.record(stream)
        e_.synchronize()
        trp.sync_status(stream)
        pms = s_.elapsed_time(e_)
        trp.close()
        plain_rate = len(evs) / (pms / 1e3)
        rate = b.n_events / (ms / 1e3)
        rows.append({"tracks": nt, "hits_per_event": round(b.n_hits / b.n_events, 1),
                     "edges_per_event": round(st["edges"] / b.n_events, 1), "events": b.n_events,
                     "batched_bf16_rescore_events_per_s": round(rate, 1),
                     "batched_hits_per_s": round(b.n_hits / (ms / 1e3), 1),
                     "band_fraction": round(st["band"] / max(st["edges"], 1), 4),
                     "rescore_edge_fraction": round(st["rescore_edges"] / max(st["edges"], 1), 4),
                     "plain_fp32_events_per_s": round(plain_rate, 1),
                     "batched_over_plain": round(rate / plain_rate, 2)})
    return rows


def cfg2_report(pkg, torch, dev, stream, reps=3):
    """Config 2: the run-3-like model (embed 3-128-128-128-8, IN h64 K8) on
    100 events of 200 tracks, FP32 vs BF16 (alone, and with the FP32 re-score
    band |s - 0.5| < 0.02): events/s with one event per call and with the 100
    events in one call, BF16 agreement with FP32, and every form against the
    FP64 oracle on all 100 events (decisions, score error, labels, track
    efficiency)."""
    try:
        import oracle
        wl = synth.workload("cfg2_run3_single")
        b = synth.workload_batch(wl)
        res = {}
        graphs, labels = {}, {}
        for name, prec, band in (("fp32", "fp32", 0.0), ("bf16", "bf16", 0.0),
                                 ("bf16_band_0.02", "bf16", 0.02)):
            tr = pkg.tracker_for_workload(wl, precision=prec, rescore_band=band, max_hits=b.n_hits,
                                          max_events=b.n_events, edges_per_hit=24, use_graph=False)
            evs = []
            for e in range(b.n_events):
                ev = b.event(e)
                evs.append((ev.n_hits, torch.from_numpy(ev.xyz_soa()).to(dev),
                            torch.from_numpy(ev.plane).to(dev), torch.from_numpy(ev.offsets).to(dev),
                            torch.empty(ev.n_hits, dtype=torch.int32, device=dev)))
            xyz = torch.from_numpy(b.xyz_soa()).to(dev)
            plane = torch.from_numpy(b.plane).to(dev)
            offs = torch.from_numpy(b.offsets).to(dev)
            lab = torch.empty(b.n_hits, dtype=torch.int32, device=dev)
            for n_, x_, p_, o_, l_ in evs[:5]:
                tr.find_tracks(1, n_, x_, p_, o_, l_, stream)
            tr.find_tracks(b.n_events, b.n_hits, xyz, plane, offs, lab, stream)
            tr.sync_status(stream)
            s1, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s2, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                s1.record(stream)
                for _ in range(reps):
                    for n_, x_, p_, o_, l_ in evs:
                        tr.find_tracks(1, n_, x_, p_, o_, l_, stream)
                e1.record(stream)
                s2.record(stream)
                for _ in range(reps):
                    tr.find_tracks(b.n_events, b.n_hits, xyz, plane, offs, lab, stream)
                e2.record(stream)
            e2.synchronize()
            tr.sync_status(stream)
            n = reps * b.n_events
            res[name] = {"one_event_per_call_events_per_s": round(n / (s1.elapsed_time(e1) / 1e3), 1),
                         "batched_events_per_s": round(n / (s2.elapsed_time(e2) / 1e3), 1)}
            graphs[name] = [tr.get_graph(e) for e in range(b.n_events)]
            labels[name] = lab.cpu().numpy()
            tr.close()
        g16, g32 = graphs["bf16"], graphs["fp32"]
        sig = lambda v: 1 / (1 + np.exp(-np.asarray(v, np.float64)))
        d = np.concatenate([np.abs(sig(a["logit"]) - sig(c["logit"])) for a, c in zip(g16, g32)])
        agree = np.mean(np.concatenate([a["kept"] == c["kept"] for a, c in zip(g16, g32)]))
        # both precisions against the FP64 oracle on every event
        from oracle import metrics
        sh = synth.shape_of(wl)
        m = oracle.Model(synth.workload_weights(wl), sh.embed, sh.hidden, sh.iters)
        fs = pkg.feat_scale_of(pkg.make_cfg(wl["model"], wl["radius2"]))
        t0 = time.perf_counter()
        refs = oracle_events(m, b, list(range(b.n_events)), wl, fs, os.cpu_count() or 1)
        t_or = time.perf_counter() - t0
        lab_ref = np.concatenate([r.labels for r in refs])
        co = metrics.batch_counts(lab_ref, b.pid, b.offsets).summary()
        vs = {}
        for prec, gs in graphs.items():
            ag = Agreement()
            for e in range(b.n_events):
                ag.add(gs[e], refs[e], int(b.offsets[e + 1] - b.offsets[e]))
            cg = metrics.batch_counts(labels[prec], b.pid, b.offsets).summary()
            vs[prec] = {**ag.summary(),
                        "labels_identical_events": int(sum(
                            np.array_equal(labels[prec][b.offsets[e]:b.offsets[e + 1]],
                                           lab_ref[b.offsets[e]:b.offsets[e + 1]])
                            for e in range(b.n_events))),
                        "track_efficiency": round(cg["efficiency"], 6),
                        "track_efficiency_delta_pp": round(100 * abs(cg["efficiency"] - co["efficiency"]), 4)}
        return {"workload": f"cfg2_run3_single: {b.n_events} events, {wl['description']}",
                "hits": int(b.n_hits), **res,
                "bf16_vs_fp32": {"max_score_error": round(float(d.max()), 6),
                                 "mean_score_error": round(float(d.mean()), 6),
                                 "edge_decision_agreement": round(float(agree), 6)},
                "vs_fp64_oracle": {"events": b.n_events, "track_efficiency_oracle": round(co["efficiency"], 6),
                                   "oracle_seconds": round(t_or, 2), **vs}}
    except Exception as ex:  # reported, not fatal
        return {"error": str(ex)}


def trained_report(pkg, torch, dev, stream, flush, steps=5, sample=100):
    """The headline's 1000 events with trained config-1 weights (the training
    tool's hinge-loss embedding and focal-loss GNN, trained on other events):
    events/s in BF16 and FP8 with the FP32 re-score band and in FP32, graph
    size and band size, and the track metrics of each against the FP64 oracle
    on the first `sample` events."""
    try:
        import oracle
        from oracle import metrics
        wl = synth.workload("cfg3_trained_bf16")
        b = synth.workload_batch(wl)
        n_ev, N = b.n_events, b.n_hits
        xyz = torch.from_numpy(b.xyz_soa()).to(dev)
        plane = torch.from_numpy(b.plane).to(dev)
        offs = torch.from_numpy(b.offsets).to(dev)
        labels = torch.empty(N, dtype=torch.int32, device=dev)
        sub = b.subset(list(range(sample)))
        nh = int(sub.n_hits)
        res = {}
        for prec in ("bf16", "fp32", "fp8"):
            tr = pkg.tracker_for_workload(wl, precision=prec, max_hits=N, max_events=n_ev,
                                          edges_per_hit=16, use_graph=True,
                                          **({"rescore_band": 0.02} if prec == "fp8" else {}))
            tuned = tr.autotune(n_ev, N, xyz, plane, offs, labels, stream)
            for _ in range(3):
                tr.find_tracks(n_ev, N, xyz, plane, offs, labels, stream)
            tr.sync_status(stream)
            ms = float(np.mean(timed_steps(torch, tr, n_ev, N, xyz, plane, offs, labels, stream,
                                           flush, steps)))
            st = tr.stats()
            lab = labels.cpu().numpy()[:nh]
            c = metrics.batch_counts(lab, sub.pid, sub.offsets).summary()
            res[prec] = {"events_per_s": round(n_ev / (ms / 1e3), 1), "ms_per_step": round(ms, 4),
                         "edges": st["edges"], "mean_degree": round(2 * st["edges"] / N, 3),
                         "kept_edges": st["kept"], "band_edges": st["band"],
                         "rerun_events": st["rerun_events"], "rescore_rows": tr.rescore_rows(),
                         "autotuned_ctas_per_sm": tuned,
                         f"metrics_first_{sample}_events": {k: round(v, 6) if isinstance(v, float) else v
                                                            for k, v in c.items()}}
            tr.close()
        sh = synth.shape_of(wl)
        model = oracle.Model(synth.workload_weights(wl), sh.embed, sh.hidden, sh.iters)
        fs = pkg.feat_scale_of(pkg.make_cfg(wl["model"], wl["radius2"]))
        cores = os.cpu_count() or 1
        t0 = time.perf_counter()
        lab_ref, ne_ref = oracle.find_tracks_batch(model, sub.x, sub.y, sub.z, sub.plane, sub.offsets,
                                                   wl["radius2"], wl["k_max"], wl["cut"],
                                                   threads=cores, feat_scale=fs)
        t_oracle = time.perf_counter() - t0
        co = metrics.batch_counts(lab_ref, sub.pid, sub.offsets).summary()
        return {"workload": f"cfg3_trained_bf16: {n_ev} events, {wl['description']}",
                "hits": int(N), **res,
                f"oracle_first_{sample}_events": {**{k: round(v, 6) if isinstance(v, float) else v
                                                     for k, v in co.items()},
                                                  "edges": int(ne_ref), "seconds": round(t_oracle, 2),
                                                  "cores": cores}}
    except Exception as ex:  # reported, not fatal
        import traceback
        return {"error": str(ex), "trace": traceback.format_exc()[-600:]}


def pair_particle_efficiency(tracks_per_event, b):
    """Efficiency over the particles that share a hit with another one (the
    close pairs), with the same matching rule as the track metrics."""
    from collections import Counter
    rec = tot = 0
    for e, trk in enumerate(tracks_per_event):
        a0, a1 = int(b.offsets[e]), int(b.offsets[e + 1])
        pid, pid2 = b.pid[a0:a1], b.pid2[a0:a1]
        nh = Counter(pid[pid >= 0].tolist()) + Counter(pid2[pid2 >= 0].tolist())
        shared = set(pid[pid2 >= 0].tolist()) | set(pid2[pid2 >= 0].tolist())
        matched = set()
        for t in trk:
            if len(t) < 3:
                continue
            v = Counter()
            for i in t:
                v[int(pid[i])] += 1
                if pid2[i] >= 0:
                    v[int(pid2[i])] += 1
            real = [(n, -p) for p, n in v.items() if p >= 0]
            if real:
                n_, p_ = max(real)
                if n_ >= 0.7 * len(t):
                    matched.add(-p_)
        for p in shared:
            if nh[p] >= 3:
                tot += 1
                rec += p in matched
    return round(rec / max(tot, 1), 6), tot


def triplet_report(pkg, torch, dev, stream, flush, steps=5, sample=50):
    """The triplet stage on 1000 events with close track pairs (trained
    config-1 model with triplet classifiers): events/s with and without the
    triplet stage (BF16 + re-score and FP32), the triplet-stage kernels' share
    of a step, and track metrics of triplet tracks against plain components,
    GPU against the FP64 oracle on the first `sample` events."""
    try:
        import oracle
        from oracle import metrics
        wl = synth.workload("cfg6_triplets")
        b = synth.workload_batch(wl)
        n_ev, N = b.n_events, b.n_hits
        xyz = torch.from_numpy(b.xyz_soa()).to(dev)
        plane = torch.from_numpy(b.plane).to(dev)
        offs = torch.from_numpy(b.offsets).to(dev)
        labels = torch.empty(N, dtype=torch.int32, device=dev)
        ev_t = torch.zeros(n_ev + 1, dtype=torch.int32, device=dev)
        t_off = torch.zeros(2 * N + 1, dtype=torch.int64, device=dev)
        t_hits = torch.zeros(8 * N, dtype=torch.int32, device=dev)
        outs = (ev_t, t_off, t_hits)
        sub = b.subset(list(range(sample)))
        nh = int(sub.n_hits)
        res = {}
        for prec in ("bf16", "fp32", "fp8"):
            tr = pkg.tracker_for_workload(wl, precision=prec, max_hits=N, max_events=n_ev,
                                          edges_per_hit=16, use_graph=True,
                                          **({"rescore_band": 0.02} if prec == "fp8" else {}))
            tuned = tr.autotune(n_ev, N, xyz, plane, offs, labels, stream)
            for _ in range(3):
                tr.find_tracks_triplets(n_ev, N, xyz, plane, offs, labels, *outs, stream)
            tr.sync_status(stream)
            ms = float(np.mean(timed_steps(torch, tr, n_ev, N, xyz, plane, offs, labels, stream,
                                           flush, steps, tracks=outs)))
            st, ts = tr.stats(), tr.triplet_stats()
            tr.set_profiling(True)
            timed_steps(torch, tr, n_ev, N, xyz, plane, offs, labels, stream, flush, steps,
                        tracks=outs)
            stages = tr.stage_times()
            tr.set_profiling(False)
            lab = labels.cpu().numpy()
            et, to, th = ev_t.cpu().numpy(), t_off.cpu().numpy(), t_hits.cpu().numpy()
            tracks = [[th[to[t]:to[t + 1]] for t in range(et[e], et[e + 1])] for e in range(sample)]
            ct = metrics.batch_track_counts(tracks, sub.pid, sub.offsets, pid2=sub.pid2).summary()
            cw = metrics.batch_counts(lab[:nh], sub.pid, sub.offsets, pid2=sub.pid2).summary()
            wcc_tracks = []
            for e in range(sample):
                a0, a1 = int(sub.offsets[e]), int(sub.offsets[e + 1])
                mem = {}
                for i, l in enumerate(lab[a0:a1]):
                    mem.setdefault(int(l), []).append(i)
                wcc_tracks.append(list(mem.values()))
            tr.close()
            base = pkg.tracker_for_workload(wl, precision=prec, max_hits=N, max_events=n_ev,
                                            edges_per_hit=16, use_graph=True, triplets=False)
            base.autotune(n_ev, N, xyz, plane, offs, labels, stream)
            for _ in range(3):
                base.find_tracks(n_ev, N, xyz, plane, offs, labels, stream)
            base.sync_status(stream)
            ms0 = float(np.mean(timed_steps(torch, base, n_ev, N, xyz, plane, offs, labels,
                                            stream, flush, steps)))
            base.close()
            rnd = lambda d: {k: round(v, 6) if isinstance(v, float) else v for k, v in d.items()}
            # roofline of the triplet classifiers: tensor cores gather two BF16
            # e^K rows per triplet (HBM-bound); FP32 warp tiles do 2(2h^2 + h)
            # flop per triplet (ALU-bound)
            h = wl["model"]["hidden"]
            n_t = ts["articulations"] + ts["elbows"]
            t_ms = stages["triplet_scores"][0] / steps if "triplet_scores" in stages else 0.0
            pk = peaks()
            if prec == "fp32":
                ach = n_t * 2.0 * (2 * h * h + h) / (t_ms / 1e3) / 1e12 if t_ms else 0.0
                peak, psrc = fp32_peak(torch, dev, pk)
                roof = {"bound": "alu", "achieved": round(ach, 2), "unit": "TFLOP/s",
                        "peak": round(peak, 2), "frac": round(ach / peak, 4), "peak_src": psrc}
            else:
                ach = n_t * (2 * h * 2 + 8 + 5) / (t_ms / 1e3) / 1e9 if t_ms else 0.0
                roof = {"bound": "hbm", "achieved": round(ach, 1), "unit": "GB/s",
                        "peak": pk["hbm_gbs"], "frac": round(ach / pk["hbm_gbs"], 4)}
            res[prec] = {
                "triplet_classifier_roofline": roof,
                "events_per_s_with_triplets": round(n_ev / (ms / 1e3), 1),
                "events_per_s_without": round(n_ev / (ms0 / 1e3), 1),
                "ms_per_step": round(ms, 4), "ms_per_step_without": round(ms0, 4),
                "stage_ms_per_step": {k: round(stages[k][0] / steps, 4)
                                      for k in ("triplets", "triplet_scores", "track_build")
                                      if k in stages},
                "edges": st["edges"], "kept_edges": st["kept"], **{f"triplet_{k}": v for k, v in ts.items()},
                "autotuned_ctas_per_sm": tuned,
                f"triplet_tracks_first_{sample}_events": rnd(ct),
                f"plain_components_first_{sample}_events": rnd(cw),
                "pair_particle_efficiency_triplets": pair_particle_efficiency(tracks, sub),
                "pair_particle_efficiency_components": pair_particle_efficiency(wcc_tracks, sub)}
        sh = synth.shape_of(wl)
        model = oracle.Model(synth.workload_weights(wl), sh.embed, sh.hidden, sh.iters)
        fs = pkg.feat_scale_of(pkg.make_cfg(wl["model"], wl["radius2"]))
        t0 = time.perf_counter()
        ref = []
        for e in range(sample):
            ev = sub.event(e)
            ref.append(oracle.find_tracks_triplets_event(
                model, ev.x, ev.y, ev.z, ev.plane, wl["radius2"], wl["k_max"], wl["cut"],
                wl["triplet_cut"], feat_scale=fs).tracks)
        t_or = time.perf_counter() - t0
        co = metrics.batch_track_counts(ref, sub.pid, sub.offsets, pid2=sub.pid2).summary()
        return {"workload": f"cfg6_triplets: {n_ev} events, {wl['description']}", "hits": int(N),
                **res,
                f"oracle_triplet_tracks_first_{sample}_events": {
                    **{k: round(v, 6) if isinstance(v, float) else v for k, v in co.items()},
                    "pair_particle_efficiency": pair_particle_efficiency(ref, sub),
                    "seconds_one_core": round(t_or, 2)}}
    except Exception as ex:  # reported, not fatal
        import traceback
        return {"error": str(ex), "trace": traceback.format_exc()[-600:]}


def int8_report(pkg, torch, dev, stream, flush, steps=5, calib_events=5000, sample=100):
    """INT8 embedding (post-training quantisation, the thesis's Sec. on MLP
    quantisation) on the trained config-1 model and the headline's 1000
    events: graph size and track metrics with the FP32 embedding, the INT8
    one uncalibrated (alpha = 1) and the INT8 one after max calibration on
    `calib_events` other events; BF16 + re-score GNN in all three."""
    try:
        from oracle import metrics
        wl = synth.workload("cfg3_trained_bf16")
        b = synth.workload_batch(wl)
        n_ev, N = b.n_events, b.n_hits
        xyz = torch.from_numpy(b.xyz_soa()).to(dev)
        plane = torch.from_numpy(b.plane).to(dev)
        offs = torch.from_numpy(b.offsets).to(dev)
        labels = torch.empty(N, dtype=torch.int32, device=dev)
        sub = b.subset(list(range(sample)))
        nh = int(sub.n_hits)
        t0 = time.perf_counter()
        cal = synth.workload_batch(wl, calib_events, first_event=n_ev)
        t_gen = time.perf_counter() - t0
        cal_xyz = torch.from_numpy(cal.xyz_soa()).to(dev)
        res = {}
        alpha = None
        for name in ("fp32_embedding", "int8_uncalibrated", "int8_calibrated"):
            tr = pkg.tracker_for_workload(wl, max_hits=N, max_events=n_ev,
                                          edges_per_hit=40 if name == "int8_uncalibrated" else 16,
                                          use_graph=True, embed_int8=name != "fp32_embedding")
            if name == "int8_calibrated":
                t1 = time.perf_counter()
                alpha = tr.embed_amax(cal_xyz, stream)
                t_cal = time.perf_counter() - t1
                tr.set_embed_scales(alpha)
            tr.autotune(n_ev, N, xyz, plane, offs, labels, stream)
            for _ in range(3):
                tr.find_tracks(n_ev, N, xyz, plane, offs, labels, stream)
            tr.sync_status(stream)
            ms = float(np.mean(timed_steps(torch, tr, n_ev, N, xyz, plane, offs, labels, stream,
                                           flush, steps)))
            st = tr.stats()
            tr.set_profiling(True)
            timed_steps(torch, tr, n_ev, N, xyz, plane, offs, labels, stream, flush, steps)
            stages = tr.stage_times()
            tr.set_profiling(False)
            lab = labels.cpu().numpy()[:nh]
            c = metrics.batch_counts(lab, sub.pid, sub.offsets).summary()
            res[name] = {"events_per_s": round(n_ev / (ms / 1e3), 1), "edges": st["edges"],
                         "node_prep_ms_per_step": round(stages["node_prep"][0] / steps, 4),
                         f"metrics_first_{sample}_events": {
                             k: round(v, 6) if isinstance(v, float) else v for k, v in c.items()}}
            tr.close()
        e32 = res["fp32_embedding"]["edges"]
        for k in ("int8_uncalibrated", "int8_calibrated"):
            res[k]["edges_vs_fp32"] = round(res[k]["edges"] / e32 - 1.0, 4)
        return {"workload": f"cfg3_trained_bf16: {n_ev} events, {wl['description']}",
                "calibration": {"events": calib_events, "hits": int(cal.n_hits),
                                "method": "max |layer input| over the calibration events (GPU, FP32 embedding)",
                                "alpha": [round(float(a), 6) for a in alpha],
                                "seconds_on_gpu": round(t_cal, 3),
                                "seconds_generating_events": round(t_gen, 2)},
                "uncalibrated_alpha": 1.0, **res}
    except Exception as ex:  # reported, not fatal
        import traceback
        return {"error": str(ex), "trace": traceback.format_exc()[-600:]}


def fp8_report(pkg, torch, dev, stream, chunk=1000, bands=(0.02, 0.05), oracle_events_n=1000):
    """Config 4: FP8-E4M3 (per-channel weight scales, per-row activation
    scales, FP32 accumulate; the encoders as BF16 split-operand kernels),
    config-1 model at hidden 128, 10000 events of 200 tracks. Throughput over
    all events of FP32, FP8 and FP8 with the FP32 re-score band; decisions of
    each against FP32 and, on a seeded 1000-event subset (the first chunk),
    against the FP64 oracle (decision agreement over the union of edge sets,
    score error, identical labels, track efficiency)."""
    try:
        import oracle
        from oracle import metrics
        wl = synth.workload("cfg4_batched_fp8")
        n = wl["n_events"]
        chunks = [synth.workload_batch(wl, chunk, first_event=c) for c in range(0, n, chunk)]
        maxh = max(b.n_hits for b in chunks)
        b0 = chunks[0]
        variants = [("fp32", "fp32", 0.0), ("fp8", "fp8", 0.0)] + \
                   [(f"fp8_band_{bd}", "fp8", bd) for bd in bands]
        res, first = {}, {}
        for name, prec, band in variants:
            tr = pkg.tracker_for_workload(wl, precision=prec, rescore_band=band, max_hits=maxh,
                                          max_events=chunk, edges_per_hit=16, use_graph=True)
            ms, rows, edges = 0.0, 0, 0
            for ci, b in enumerate(chunks):
                xyz = torch.from_numpy(b.xyz_soa()).to(dev)
                plane = torch.from_numpy(b.plane).to(dev)
                offs = torch.from_numpy(b.offsets).to(dev)
                lab = torch.empty(b.n_hits, dtype=torch.int32, device=dev)
                tr.find_tracks(b.n_events, b.n_hits, xyz, plane, offs, lab, stream)
                tr.sync_status(stream)
                s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(stream):
                    s_.record(stream)
                    tr.find_tracks(b.n_events, b.n_hits, xyz, plane, offs, lab, stream)
                    e_.record(stream)
                e_.synchronize()
                tr.sync_status(stream)
                ms += s_.elapsed_time(e_)
                st = tr.stats()
                rows += st["rescore_edges"]
                edges += st["edges"]
                if ci == 0:
                    gs = [tr.get_graph(e) for e in range(b.n_events)]
                    first[name] = {"kept": [g["kept"] for g in gs], "logit": [g["logit"] for g in gs],
                                   "labels": lab.cpu().numpy()}
                    if name == "fp32":
                        first["src"] = [g["src"] for g in gs]
                        first["dst"] = [g["dst"] for g in gs]
                    first[name]["band_edges"] = st["band"]
            res[name] = {"events_per_s": round(n / (ms / 1e3), 1),
                         "ms_per_1000_events": round(ms / len(chunks), 3),
                         "rescore_rows_per_edge": round(rows / max(edges, 1), 4)}
            tr.close()
        # the plain FP32 path at this model, one event per call (100 events)
        trp = pkg.tracker_for_workload(wl, precision="fp32", max_hits=max(
            int(b0.offsets[e + 1] - b0.offsets[e]) for e in range(100)), max_events=1,
            edges_per_hit=16)
        evs = []
        for e in range(100):
            ev = b0.event(e)
            evs.append((ev.n_hits, torch.from_numpy(ev.xyz_soa()).to(dev),
                        torch.from_numpy(ev.plane).to(dev), torch.from_numpy(ev.offsets).to(dev),
                        torch.empty(ev.n_hits, dtype=torch.int32, device=dev)))
        for n_, x_, p_, o_, l_ in evs[:3]:
            trp.find_tracks(1, n_, x_, p_, o_, l_, stream)
        trp.sync_status(stream)
        s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            s_.record(stream)
            for n_, x_, p_, o_, l_ in evs:
                trp.find_tracks(1, n_, x_, p_, o_, l_, stream)
            e_.record(stream)
        e_.synchronize()
        trp.sync_status(stream)
        trp.close()
        plain = len(evs) / (s_.elapsed_time(e_) / 1e3)
        res["plain_fp32_one_event_per_call"] = {"events_per_s": round(plain, 1),
                                                "events": len(evs)}
        fp32_rate = res["fp32"]["events_per_s"]
        for name, _, _ in variants[1:]:
            res[name]["over_fp32"] = round(res[name]["events_per_s"] / fp32_rate, 3)
            res[name]["over_plain_fp32"] = round(res[name]["events_per_s"] / plain, 2)
        # decisions against the FP32 path on the first chunk (same graph: the
        # embedding is FP32 in every precision)
        k32 = np.concatenate(first["fp32"]["kept"])
        l32 = np.concatenate(first["fp32"]["logit"]).astype(np.float64)
        sig = lambda v: 1 / (1 + np.exp(-np.asarray(v, np.float64)))
        for name, _, _ in variants[1:]:
            kk = np.concatenate(first[name]["kept"])
            dd = np.abs(sig(np.concatenate(first[name]["logit"])) - sig(l32))
            res[name]["vs_fp32_first_1000_events"] = {
                "edge_decision_agreement": round(float(np.mean(kk == k32)), 6),
                "max_score_error": round(float(dd.max()), 5), "mean_score_error": round(float(dd.mean()), 6)}
        # against the FP64 oracle on the first `oracle_events_n` events
        sh = synth.shape_of(wl)
        model = oracle.Model(synth.workload_weights(wl), sh.embed, sh.hidden, sh.iters)
        fs = pkg.feat_scale_of(pkg.make_cfg(wl["model"], wl["radius2"]))
        cores = os.cpu_count() or 1
        ne = min(oracle_events_n, b0.n_events)
        t0 = time.perf_counter()
        refs = oracle_events(model, b0, list(range(ne)), wl, fs, cores)
        t_or = time.perf_counter() - t0
        lab_ref = np.concatenate([r.labels for r in refs])
        nh = int(b0.offsets[ne])
        co = metrics.batch_counts(lab_ref, b0.pid[:nh], b0.offsets[:ne + 1]).summary()
        vs = {"events": ne, "hits": nh, "oracle_seconds": round(t_or, 1), "oracle_cores": cores,
              "track_efficiency_oracle": round(co["efficiency"], 6)}
        for name, _, _ in variants:
            ag = Agreement()
            for e in range(ne):
                g = {"src": first["src"][e], "dst": first["dst"][e], "kept": first[name]["kept"][e],
                     "logit": first[name]["logit"][e]}
                ag.add(g, refs[e], int(b0.offsets[e + 1] - b0.offsets[e]))
            lab = first[name]["labels"][:nh]
            cg = metrics.batch_counts(lab, b0.pid[:nh], b0.offsets[:ne + 1]).summary()
            vs[name] = {**ag.summary(),
                        "labels_identical_events": int(sum(
                            np.array_equal(lab[b0.offsets[e]:b0.offsets[e + 1]],
                                           lab_ref[b0.offsets[e]:b0.offsets[e + 1]]) for e in range(ne))),
                        "track_efficiency": round(cg["efficiency"], 6),
                        "track_efficiency_delta_pp": round(100 * abs(cg["efficiency"] - co["efficiency"]), 4)}
        return {"workload": f"cfg4_batched_fp8: {n} events, {wl['description']}",
                "dtype": "e4m3 GNN steps and classifier (tcgen05 kind::f8f6f4); BF16 split-operand encoders",
                **res, "vs_fp64_oracle": vs}
    except Exception as ex:  # reported, not fatal
        import traceback
        return {"error": str(ex), "trace": traceback.format_exc()[-600:]}


def fp8_trained_report(pkg, torch, dev, stream, n_events=1000, oracle_n=200, reps=3):
    """Config-4 events (200 tracks, 2 % noise) with a hidden-128 model trained
    on other synthetic events (workload cfg4_trained_fp8): FP32, FP8 alone
    and FP8 with the FP32 re-score bands |s - 0.5| < 0.02 and 0.05, each timed over
    `n_events` events in one call and checked against the FP64 oracle on the
    first `oracle_n` events. With trained weights the logits sit far from the
    cut, so the band and its receptive field are small."""
    try:
        import oracle
        from oracle import metrics
        wl = synth.workload("cfg4_trained_fp8")
        b = synth.workload_batch(wl, n_events)
        xyz = torch.from_numpy(b.xyz_soa()).to(dev)
        plane = torch.from_numpy(b.plane).to(dev)
        offs = torch.from_numpy(b.offsets).to(dev)
        lab = torch.empty(b.n_hits, dtype=torch.int32, device=dev)
        res, keep = {}, {}
        for name, prec, band in (("fp32", "fp32", 0.0), ("fp8", "fp8", 0.0),
                                 ("fp8_band_0.02", "fp8", 0.02), ("fp8_band_0.05", "fp8", 0.05)):
            tr = pkg.tracker_for_workload(wl, precision=prec, rescore_band=band, max_hits=b.n_hits,
                                          max_events=b.n_events, edges_per_hit=16, use_graph=True)
            for _ in range(2):
                tr.find_tracks(b.n_events, b.n_hits, xyz, plane, offs, lab, stream)
            tr.sync_status(stream)
            s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                s_.record(stream)
                for _ in range(reps):
                    tr.find_tracks(b.n_events, b.n_hits, xyz, plane, offs, lab, stream)
                e_.record(stream)
            e_.synchronize()
            tr.sync_status(stream)
            st = tr.stats()
            res[name] = {"events_per_s": round(reps * b.n_events / (s_.elapsed_time(e_) / 1e3), 1),
                         "band_edges": st["band"], "rescore_rows_per_edge":
                             round(st["rescore_edges"] / max(st["edges"], 1), 4)}
            keep[name] = ([tr.get_graph(e) for e in range(oracle_n)], lab.cpu().numpy())
            tr.close()
        for name in ("fp8", "fp8_band_0.02", "fp8_band_0.05"):
            res[name]["over_fp32"] = round(res[name]["events_per_s"] / res["fp32"]["events_per_s"], 3)
        sh = synth.shape_of(wl)
        model = oracle.Model(synth.workload_weights(wl), sh.embed, sh.hidden, sh.iters)
        fs = pkg.feat_scale_of(pkg.make_cfg(wl["model"], wl["radius2"]))
        t0 = time.perf_counter()
        refs = oracle_events(model, b, list(range(oracle_n)), wl, fs, os.cpu_count() or 1)
        t_or = time.perf_counter() - t0
        lab_ref = np.concatenate([r.labels for r in refs])
        nh = int(b.offsets[oracle_n])
        co = metrics.batch_counts(lab_ref, b.pid[:nh], b.offsets[:oracle_n + 1]).summary()
        vs = {"events": oracle_n, "oracle_seconds": round(t_or, 1),
              "track_efficiency_oracle": round(co["efficiency"], 6)}
        for name, (gs, labs) in keep.items():
            ag = Agreement()
            for e in range(oracle_n):
                ag.add(gs[e], refs[e], int(b.offsets[e + 1] - b.offsets[e]))
            cg = metrics.batch_counts(labs[:nh], b.pid[:nh], b.offsets[:oracle_n + 1]).summary()
            vs[name] = {**ag.summary(), "track_efficiency": round(cg["efficiency"], 6),
                        "track_efficiency_delta_pp": round(100 * abs(cg["efficiency"] - co["efficiency"]), 4)}
        return {"workload": f"cfg4_trained_fp8: {n_events} events, {wl['description']}", **res,
                "vs_fp64_oracle": vs}
    except Exception as ex:  # reported, not fatal
        import traceback
        return {"error": str(ex), "trace": traceback.format_exc()[-600:]}


def profile_case(name, pkg, torch):
    """Small fixed cases for kernel captures (ncu): the first 100 events of
    config 4 in FP8 (three calls); the first 300 events of the
    headline batch (three calls, BF16 + FP32 re-score band 0.02, or FP32; the
    _tuned case autotunes first, so the captured kernels are the variants the
    autotuner keeps; the _tma case runs the BF16 edge step with TMA-staged
    tiles), or
    one triplet-stage call on 100 events of the triplet workload followed by
    the INT8 embedding (calibrated on the same 100 events) of the trained
    workload."""
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    if name == "cfg4_100ev_fp8":
        # the first 100 events of config 4 (hidden 128), FP8 without a band,
        # three calls
        wl = synth.workload("cfg4_batched_fp8")
        b = synth.workload_batch(wl, 100)
        tr = pkg.tracker_for_workload(wl, precision="fp8", rescore_band=0.0, max_hits=b.n_hits,
                                      max_events=b.n_events, edges_per_hit=16)
        for _ in range(3):
            pkg.run_batch(tr, b)
        print(name, tr.stats())
        return
    if name.startswith("headline_300ev"):
        prec = name.split("_")[2]
        wl = synth.workload("cfg3_batched_bf16")
        b = synth.workload_batch(wl, 300)
        tr = pkg.tracker_for_workload(wl, precision=prec, max_hits=b.n_hits, max_events=b.n_events,
                                      edges_per_hit=16,
                                      **({"rescore_band": 0.02} if prec != "fp32" else {}))
        xyz = torch.from_numpy(b.xyz_soa()).to(dev)
        plane = torch.from_numpy(b.plane).to(dev)
        offs = torch.from_numpy(b.offsets).to(dev)
        lab = torch.zeros(b.n_hits, dtype=torch.int32, device=dev)
        if name.endswith("_tuned"):  # the autotuner's launch configuration
            print(name, "tuning", tr.autotune(b.n_events, b.n_hits, xyz, plane, offs, lab))
        if name.endswith("_tma"):  # the BF16 edge step with TMA-staged tiles
            tr.set_tuning({"tc_edge_tma": 1})
        for _ in range(3):
            tr.find_tracks(b.n_events, b.n_hits, xyz, plane, offs, lab)
        tr.sync_status()
        print(name, tr.stats(), tr.rescore_rows())
        return
    wl = synth.workload("cfg6_triplets")
    b = synth.workload_batch(wl, 100)
    tr = pkg.tracker_for_workload(wl, max_hits=b.n_hits, max_events=b.n_events)
    pkg.run_batch_triplets(tr, b)
    print(name, "triplets", tr.triplet_stats())
    tr.close()
    wl3 = synth.workload("cfg3_trained_bf16")
    b3 = synth.workload_batch(wl3, 100)
    t3 = pkg.tracker_for_workload(wl3, max_hits=b3.n_hits, max_events=b3.n_events, embed_int8=True)
    t3.set_embed_scales(t3.embed_amax(torch.from_numpy(b3.xyz_soa()).to(dev)))
    pkg.run_batch(t3, b3)
    print(name, "int8 edges", t3.stats()["edges"])


def run_reference(a, rank, world):
    """The FP64 oracle as the reference arm: each step a bounded sample of the
    workload's events on all host cores."""
    if rank != 0:
        return
    import oracle
    wl = synth.workload(a.workload)
    sh = synth.shape_of(wl)
    model = oracle.Model(synth.workload_weights(wl), sh.embed, sh.hidden, sh.iters)
    cores = os.cpu_count() or 1
    per_step = cores
    fs = tuple(float(np.float32(v)) for v in oracle.DEFAULT_FEAT_SCALE)
    times, hits = [], 0
    for i in range(max(a.warmup, 3) + a.steps):
        b = synth.workload_batch(wl, per_step, first_event=(i * per_step) % wl["n_events"])
        t0 = time.perf_counter()
        oracle.find_tracks_batch(model, b.x, b.y, b.z, b.plane, b.offsets, wl["radius2"],
                                 wl["k_max"], wl["cut"], threads=cores, feat_scale=fs)
        dt = time.perf_counter() - t0
        if i >= max(a.warmup, 3):
            times.append(dt)
            hits += b.n_hits
    ms = 1e3 * float(np.mean(times))
    value = per_step / (ms / 1e3)
    sample = f"{per_step} events of the workload per step, one per thread, FP64 C++ oracle"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 2), "unit": "events/s",
        "n_gpus": world, "steps": a.steps, "warmup": max(a.warmup, 3),
        "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "hits_per_s": round(hits / sum(times), 1),
        "config": {"workload": f"{a.workload}: {wl['description']}", "sample": sample},
        "cpu_baseline": {"value": round(value, 2), "unit": "events/s", "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 2), "unit": "events/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


if __name__ == "__main__":
    main()
