"""Serving loop with continuous batching (gnntrk_serve_run): every event's
result is the same alone and in the mix of a running server."""
import numpy as np
import pytest

import paper_2508_07423_gb300 as pkg
from paper_2508_07423_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_serving_results_equal_alone(prec):
    wl = synth.workload("cfg5_serving")
    b = synth.workload_batch(wl, 120)
    arrivals = pkg.poisson_arrivals(b.n_events, 20000.0, 7)
    band = 0.02 if prec != "fp32" else 0.0
    cfg = pkg.make_cfg(wl["model"], wl["radius2"], k_max=wl["k_max"], precision=prec,
                       rescore_band=band, edges_per_hit=24)
    # a saved launch configuration applied to every slot (results do not
    # depend on it)
    tuning = {"tc_edge_update": 2, "tc_node_update": 3} if prec == "bf16" else {"f32_edge_update": 2, "f32_encoders": 2}
    labels, done, st = pkg.serve_run(synth.workload_weights(wl), cfg, b, arrivals, n_slots=3,
                                     max_events_per_batch=32, max_hits_per_batch=1 << 16,
                                     memory_budget_bytes=8 << 30, tuning=tuning)
    assert st["failed_batches"] == 0
    assert st["batches"] < b.n_events          # events were batched together
    assert st["largest_batch"] <= 32
    assert np.all(done >= arrivals)            # no result before its request
    # each event alone through the same library
    tr = pkg.tracker_for_workload(wl, precision=prec, rescore_band=band, max_hits=1 << 14,
                                  max_events=1)
    for e in range(0, b.n_events, 7):
        ev = b.event(e)
        alone = pkg.run_batch(tr, ev)
        a = int(b.offsets[e])
        assert np.array_equal(labels[a:a + ev.n_hits], alone), e
    tr.close()


def test_serving_rejects_a_tuning_entry_out_of_range():
    wl = synth.workload("cfg5_serving")
    b = synth.workload_batch(wl, 2)
    cfg = pkg.make_cfg(wl["model"], wl["radius2"], precision="bf16")
    with pytest.raises(pkg.GnntrkError) as ei:
        pkg.serve_run(synth.workload_weights(wl), cfg, b, np.zeros(2), max_hits_per_batch=1 << 14,
                      memory_budget_bytes=1 << 30, tuning={"tc_edge_update": 99})
    assert ei.value.status == 1


def test_serving_budget_too_small_is_rejected():
    wl = synth.workload("cfg5_serving")
    b = synth.workload_batch(wl, 2)
    cfg = pkg.make_cfg(wl["model"], wl["radius2"])
    with pytest.raises(pkg.GnntrkError) as ei:
        pkg.serve_run(synth.workload_weights(wl), cfg, b, np.zeros(2), memory_budget_bytes=1000)
    assert ei.value.status == 3


def test_two_handles_from_two_host_threads():
    """Two handles (FP32 and BF16 + re-score, CUDA graphs on) driven at the same
    time from two host threads on their own streams: every call's labels equal
    the handle's own result computed alone beforehand."""
    import threading
    jobs = []
    for name, prec, n in (("cfg1_plain_fp32", "fp32", 6), ("cfg3_batched_bf16", "bf16", 8)):
        wl = synth.workload(name)
        b = synth.workload_batch(wl, n)
        tr = pkg.tracker_for_workload(wl, precision=prec, max_hits=b.n_hits,
                                      max_events=b.n_events, edges_per_hit=32, use_graph=True)
        want = pkg.run_batch(tr, b)
        xyz = torch.from_numpy(b.xyz_soa()).cuda()
        plane = torch.from_numpy(b.plane).cuda()
        offs = torch.from_numpy(b.offsets).cuda()
        labels = torch.full((b.n_hits,), -7, dtype=torch.int32, device="cuda")
        jobs.append((tr, b, want, xyz, plane, offs, labels))
    torch.cuda.synchronize()
    errors = []

    def worker(tr, b, want, xyz, plane, offs, labels):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                for it in range(6):
                    labels.fill_(-7)
                    tr.find_tracks(b.n_events, b.n_hits, xyz, plane, offs, labels, s)
                    tr.sync_status(s)
                    if not np.array_equal(labels.cpu().numpy(), want):
                        errors.append((tr.cfg.precision, it))
        except Exception as e:  # reported below, after both threads end
            errors.append(repr(e))

    threads = [threading.Thread(target=worker, args=j) for j in jobs]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for j in jobs:
        j[0].close()
    assert not errors, errors
