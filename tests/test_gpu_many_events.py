"""Batches of many events of mixed size, empty ones among them, through the
C ABI. The graph kernel and the re-score receptive-field kernel give each
event its place in the batch-wide edge array and row lists by a look-back over
the totals of all earlier events (windows of 32 events, more events than
resident blocks, blocks taking events in order by a ticket), so every event
must get exactly the graph, labels and re-score rows it would get alone."""
import numpy as np
import pytest

import oracle
import paper_2508_07423_gb300 as pkg
from paper_2508_07423_gb300 import synth
from parity import compare_event

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_EVENTS = 1200


def mixed_batch(n_events, seed):
    """Events of 0, 1, 3, 8 or 30 tracks (5 % noise): empty events, single
    hits and events of a few hundred hits, in a seeded random order."""
    rng = np.random.default_rng(seed)
    choices = np.array([0, 1, 3, 8, 30])
    parts = [synth.gen_batch(1, seed, {"kind": "fixed", "n": int(rng.choice(choices))}, 0.05,
                             first_event=i)
             for i in range(n_events)]
    return synth.concat(parts)


@pytest.fixture(scope="module")
def batch():
    b = mixed_batch(N_EVENTS, 4242)
    sizes = np.diff(b.offsets)
    assert (sizes == 0).sum() > 100 and sizes.max() > 200
    return b


def tracker(wl, b, precision, band=0.0):
    return pkg.tracker_for_workload(wl, precision=precision, rescore_band=band,
                                    max_hits=b.n_hits, max_events=b.n_events, edges_per_hit=32)


def test_many_events_fp32_match_the_oracle(batch):
    wl = synth.workload("cfg1_plain_fp32")
    sh = synth.shape_of(wl)
    model = oracle.Model(synth.workload_weights(wl), sh.embed, sh.hidden, sh.iters)
    tr = tracker(wl, batch, "fp32")
    labels = pkg.run_batch(tr, batch)
    fs = pkg.feat_scale_of(tr.cfg)
    st = tr.stats()
    n_edges = 0
    for e in range(batch.n_events):
        ev = batch.event(e)
        a = int(batch.offsets[e])
        g = tr.get_graph(e)
        n_edges += len(g["src"])
        rep = compare_event(ev, g, labels[a:a + ev.n_hits], model, wl["radius2"], wl["k_max"],
                            sh.iters, wl["cut"], fs)
        assert rep.labels_compared and rep.labels_equal, e
    assert st["edges"] == n_edges and st["events"] == batch.n_events
    tr.close()


def test_many_events_batch_equals_alone(batch):
    """A sample of events (first, last, empty neighbours, the largest) run
    alone gives the batch's graph and labels bit for bit."""
    wl = synth.workload("cfg1_plain_fp32")
    tr = tracker(wl, batch, "fp32")
    labels = pkg.run_batch(tr, batch)
    graphs = {}
    sizes = np.diff(batch.offsets)
    sample = sorted({0, 1, 31, 32, 33, 64, batch.n_events - 1, int(np.argmax(sizes))}
                    | set(np.flatnonzero(sizes == 0)[:3].tolist()))
    for e in sample:
        graphs[e] = tr.get_graph(e)
    for e in sample:
        ev = batch.event(e)
        a = int(batch.offsets[e])
        lab = pkg.run_batch(tr, ev)
        assert np.array_equal(lab, labels[a:a + ev.n_hits]), e
        g = tr.get_graph(0)
        for k in g:
            assert np.array_equal(g[k], graphs[e][k]), (e, k)
    tr.close()


def test_many_events_rescore_rows_and_logits(batch):
    """BF16 with a re-score band: band edges take the FP32 logits bit for bit
    and the row lists hold exactly the receptive field, summed over events."""
    from test_gpu_precision import receptive_field, sigmoid

    wl = synth.workload("cfg1_plain_fp32")
    band = 0.05
    out = {}
    for name, prec, bd in (("fp32", "fp32", 0.0), ("bf16", "bf16", 0.0), ("band", "bf16", band)):
        tr = tracker(wl, batch, prec, bd)
        pkg.run_batch(tr, batch)
        out[name] = ([tr.get_graph(e) for e in range(batch.n_events)], tr.stats(),
                     tr.rescore_rows())
        tr.close()
    cat = lambda gs, k: np.concatenate([g[k] for g in gs])
    l0, l1, l32 = (cat(out[n][0], "logit") for n in ("bf16", "band", "fp32"))
    inband = np.abs(sigmoid(l0) - 0.5) < band
    assert inband.any() and not inband.all()
    assert np.array_equal(l1[inband], l32[inband])
    assert np.array_equal(l1[~inband], l0[~inband])
    st = out["band"][1]
    assert st["band"] == int(inband.sum())
    re, rv = receptive_field(out["bf16"][0], band, synth.shape_of(wl).iters, batch)
    assert out["band"][2] == {"edges": re, "hits": rv}
    assert (st["rescore_edges"], st["rescore_hits"]) == (re[0], rv[0])
    # one launch per stage: sort, embedding + node encoder (2), graph, edge
    # encoder, K x (messages, node step, edge step), receptive field, FP32
    # node and edge encoders, K x 3 FP32 steps, components
    K = synth.shape_of(wl).iters
    assert st["launches"] == 1 + 2 + 1 + 1 + 3 * K + 1 + 2 + 3 * K + 1, st["launches"]
