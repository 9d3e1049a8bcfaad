"""GPU checks of the INT8 embedding (the thesis's post-training quantisation
of the embedding MLP): the max calibration against the FP64 oracle, the INT8
embedding's graph against the oracle's INT8 emulation, and the effect of
calibration on the graph size."""
import numpy as np
import pytest

import oracle
import paper_2508_07423_gb300 as pkg
from oracle import quant
from paper_2508_07423_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def feats_of(ev, fs):
    x, y, z = (np.asarray(v, np.float64) for v in (ev.x, ev.y, ev.z))
    return np.stack([np.hypot(x, y) / fs[0], np.arctan2(y, x) / fs[1], z / fs[2]],
                    1).astype(np.float32)


@pytest.fixture(scope="module")
def trained():
    wl = synth.workload("cfg3_trained_bf16")
    arrs = synth.weight_arrays(synth.workload_weights(wl))
    layers = arrs[:len(wl["model"]["embed"]) - 1]
    return wl, layers


def test_embed_amax_matches_oracle(trained):
    wl, layers = trained
    b = synth.workload_batch(wl, 20)
    tr = pkg.tracker_for_workload(wl, precision="fp32", max_hits=b.n_hits, max_events=b.n_events,
                                  embed_int8=True)
    fs = pkg.feat_scale_of(tr.cfg)
    got = tr.embed_amax(torch.from_numpy(b.xyz_soa()).cuda())
    want = quant.embed_amax(layers, feats_of(b, fs))
    assert np.allclose(got, want, rtol=2e-5, atol=0), (got, want)


def test_int8_graph_matches_oracle_emulation(trained):
    """Calibrated INT8 embedding, FP32 GNN: the edge sets and squared
    distances against the oracle's INT8 emulation. A code can differ where the
    float32 value before rounding sits on a half-integer (the features come
    from different atan2 implementations), so a few hits may move by one step:
    edges differ only near the radius or at such hits."""
    wl, layers = trained
    b = synth.workload_batch(wl, 4)
    tr = pkg.tracker_for_workload(wl, precision="fp32", max_hits=b.n_hits, max_events=b.n_events,
                                  embed_int8=True)
    fs = pkg.feat_scale_of(tr.cfg)
    alpha = tr.embed_amax(torch.from_numpy(b.xyz_soa()).cuda())
    tr.set_embed_scales(alpha)
    pkg.run_batch(tr, b)
    n_same = n_edges = n_diff = 0
    for e in range(b.n_events):
        ev = b.event(e)
        emb = quant.int8_embed(layers, alpha, feats_of(ev, fs))
        src, dst, d2 = oracle.radius_graph(ev.plane, emb, wl["radius2"], wl["k_max"])
        g = tr.get_graph(e)
        O = {(int(a), int(c)): float(d) for a, c, d in zip(src, dst, d2)}
        G = {(int(a), int(c)): float(d) for a, c, d in zip(g["src"], g["dst"], g["d2"])}
        n_edges += len(O)
        n_diff += len(set(O) ^ set(G))
        for k in set(O) & set(G):
            n_same += abs(O[k] - G[k]) <= 1e-5 * max(O[k], 0.05)
    common = n_edges - n_diff
    assert n_diff <= 0.01 * n_edges, (n_diff, n_edges)
    assert n_same >= 0.99 * common, (n_same, common)


def test_calibration_restores_the_graph(trained):
    """Uncalibrated (alpha = 1 for every layer input) the INT8 graph differs
    from the FP32 one by more than the calibrated graph does; calibrated it is
    within 10 % of the FP32 edge count."""
    wl, _ = trained
    b = synth.workload_batch(wl, 10)
    base = pkg.tracker_for_workload(wl, precision="fp32", max_hits=b.n_hits, max_events=b.n_events)
    pkg.run_batch(base, b)
    e32 = base.stats()["edges"]
    tr = pkg.tracker_for_workload(wl, precision="fp32", max_hits=b.n_hits, max_events=b.n_events,
                                  embed_int8=True)
    pkg.run_batch(tr, b)
    e_unc = tr.stats()["edges"]
    cal = synth.workload_batch(wl, 20, first_event=100)
    tr.set_embed_scales(tr.embed_amax(torch.from_numpy(cal.xyz_soa()).cuda()))
    pkg.run_batch(tr, b)
    e_cal = tr.stats()["edges"]
    assert abs(e_cal - e32) <= 0.10 * e32, (e_cal, e32)
    assert abs(e_unc - e32) > abs(e_cal - e32), (e_unc, e_cal, e32)


def test_embed_scales_validation(trained):
    wl, _ = trained
    tr = pkg.tracker_for_workload(wl, max_hits=1024, max_events=1, embed_int8=True)
    with pytest.raises(pkg.GnntrkError):
        tr.set_embed_scales([1.0, 1.0])
    with pytest.raises(pkg.GnntrkError):
        tr.set_embed_scales([1.0, 0.0, 1.0])
    plain = pkg.tracker_for_workload(wl, max_hits=1024, max_events=1)
    with pytest.raises(pkg.GnntrkError):
        plain.set_embed_scales([1.0, 1.0, 1.0])


def test_int8_wide_embedding_graph():
    """The run-3 model's embedding 3-128-128-128-8 (32-word inputs, 8-wide
    output) in INT8 against the oracle emulation."""
    wl = synth.workload("cfg2_run3_single")
    arrs = synth.weight_arrays(synth.workload_weights(wl))
    layers = arrs[:len(wl["model"]["embed"]) - 1]
    b = synth.workload_batch(wl, 2)
    tr = pkg.tracker_for_workload(wl, precision="fp32", max_hits=b.n_hits, max_events=b.n_events,
                                  embed_int8=True, edges_per_hit=32)
    fs = pkg.feat_scale_of(tr.cfg)
    alpha = tr.embed_amax(torch.from_numpy(b.xyz_soa()).cuda())
    assert np.allclose(alpha, quant.embed_amax(layers, feats_of(b, fs)), rtol=2e-5)
    tr.set_embed_scales(alpha)
    pkg.run_batch(tr, b)
    n_edges = n_diff = n_same = 0
    for e in range(b.n_events):
        ev = b.event(e)
        emb = quant.int8_embed(layers, alpha, feats_of(ev, fs))
        src, dst, d2 = oracle.radius_graph(ev.plane, emb, wl["radius2"], wl["k_max"])
        g = tr.get_graph(e)
        O = {(int(a), int(c)): float(d) for a, c, d in zip(src, dst, d2)}
        G = {(int(a), int(c)): float(d) for a, c, d in zip(g["src"], g["dst"], g["d2"])}
        n_edges += len(O)
        n_diff += len(set(O) ^ set(G))
        for k in set(O) & set(G):
            n_same += abs(O[k] - G[k]) <= 1e-5 * max(O[k], 0.05)
    assert n_edges > 1000
    assert n_diff <= 0.01 * n_edges, (n_diff, n_edges)
    assert n_same >= 0.99 * (n_edges - n_diff), (n_same, n_edges - n_diff)
