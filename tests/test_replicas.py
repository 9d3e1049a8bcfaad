"""The multi-GPU form of the path on the CPU: two gloo ranks run replicas over
disjoint event ranges and combine only the measurement (max time, summed
events and hits), as bench.py does under torchrun with NCCL."""
import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2508_07423_gb300 import replicas, synth  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = synth.workload("cfg1_plain_fp32")
    first, n = replicas.event_range(rank, world, 2)
    b = synth.workload_batch(wl, n, first_event=first)
    local_ms = 10.0 + 2.5 * rank  # the slower rank sets the job's time
    ms, events, hits = replicas.combine(dist, local_ms, b.n_events, b.n_hits, torch.device("cpu"))
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"first": first, "n": n, "hits": int(b.n_hits), "x0": float(b.x[0]),
                   "ms": ms, "events": events, "job_hits": hits}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_disjoint_events_and_combined_measurement(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    r = [json.load(open(tmp_path / f"r{k}.json")) for k in range(world)]
    # disjoint, contiguous event ranges covering events 0..3
    assert [(x["first"], x["n"]) for x in r] == [(0, 2), (2, 2)]
    whole = synth.workload_batch(synth.workload("cfg1_plain_fp32"), 4)
    assert r[0]["x0"] == float(whole.event(0).x[0]) and r[1]["x0"] == float(whole.event(2).x[0])
    # every rank sees the job totals: slowest time, summed events and hits
    for x in r:
        assert x["ms"] == 12.5 and x["events"] == 4
        assert x["job_hits"] == r[0]["hits"] + r[1]["hits"] == whole.n_hits


def test_event_range_rejects_bad_ranks():
    assert replicas.event_range(3, 4, 250) == (750, 250)
    with pytest.raises(ValueError):
        replicas.event_range(4, 4, 10)
    assert replicas.combine(None, 3.0, 5, 7) == (3.0, 5, 7)


def test_balanced_ranges_split_by_hits():
    wl = synth.workload("cfg3_batched_bf16")
    b = synth.workload_batch(wl, 64)
    hits = np.diff(b.offsets)
    for world in (1, 2, 3, 4, 8):
        rng = replicas.balanced_ranges(hits, world)
        # contiguous, in order, every event exactly once
        assert sum(n for _, n in rng) == b.n_events
        nxt = 0
        for first, n in rng:
            if n:
                assert first == nxt
                nxt = first + n
        assert nxt == b.n_events
        # each rank's hits within one event's hits of the ideal share
        share = b.n_hits / world
        for first, n in rng:
            assert abs(int(hits[first:first + n].sum()) - share) <= hits.max()
    # a heavy event goes whole to one rank; empty events still get an owner
    assert replicas.balanced_ranges([1, 100, 1], 2) == [(0, 1), (1, 2)]
    assert replicas.balanced_ranges([0, 0, 0, 0], 2) == [(0, 2), (2, 2)]
    assert replicas.balanced_ranges([5], 3) == [(0, 0), (0, 1), (1, 0)]
