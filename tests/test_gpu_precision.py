"""Tensor-core paths (BF16 and FP8-E4M3 on tcgen05) and the FP32 re-score of
near-cut edges, through the C ABI.

The FP32 path is pinned to the FP64 oracle (test_gpu_parity.py); here the
low-precision paths are checked against it and against the oracle:
  * the graph is bit-identical (the embedding stays FP32 in every precision);
  * logit errors stay within bounds measured and derived for each format
    (BF16 keeps 8 significant bits: about 0.4 % relative per rounding, a few
    hundredths of a logit after 4 steps; E4M3 keeps 4: about 6 %);
  * edges in the re-score band take exactly the FP32 path's logit and
    decision, all others keep the tensor-core result;
  * with the re-score, BF16 (and, with a wider band, the wide models in BF16
    and FP8) agrees with the FP64 oracle on >= 99.9 % of edge decisions;
    without it the wide models miss that bar (recorded as expected failures).
"""
import math

import numpy as np
import pytest

import oracle
import paper_2508_07423_gb300 as pkg
from paper_2508_07423_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def sigmoid(v):
    return 1.0 / (1.0 + np.exp(-np.asarray(v, np.float64)))


TRACKER_ROWS = {}


def run(wl, batch, precision, band=0.0, **kw):
    tr = pkg.tracker_for_workload(wl, precision=precision, rescore_band=band,
                                  max_hits=batch.n_hits, max_events=batch.n_events,
                                  edges_per_hit=32, **kw)
    labels = pkg.run_batch(tr, batch)
    graphs = [tr.get_graph(e) for e in range(batch.n_events)]
    st = tr.stats()
    TRACKER_ROWS["rows"] = tr.rescore_rows()
    tr.close()
    return labels, graphs, st


def cat(graphs, key):
    return np.concatenate([g[key] for g in graphs])


@pytest.fixture(scope="module")
def cfg1():
    wl = synth.workload("cfg1_plain_fp32")
    b = synth.workload_batch(wl, 6)
    return wl, b, run(wl, b, "fp32")


@pytest.mark.parametrize("prec,mean_tol,max_tol,agree_min",
                         [("bf16", 0.015, 0.08, 0.995), ("fp8", 0.2, 1.0, 0.9)])
def test_tensor_core_close_to_fp32(cfg1, prec, mean_tol, max_tol, agree_min):
    wl, b, ref = cfg1
    _, g, st = run(wl, b, prec)
    for k in ("src", "dst", "d2"):
        assert np.array_equal(cat(g, k), cat(ref[1], k)), k
    d = np.abs(cat(g, "logit").astype(np.float64) - cat(ref[1], "logit"))
    assert d.mean() < mean_tol and d.max() < max_tol, (d.mean(), d.max())
    agree = np.mean(cat(g, "kept") == cat(ref[1], "kept"))
    assert agree >= agree_min, agree
    assert st["launches"] > 0


def test_rescore_band_takes_fp32_decisions(cfg1):
    wl, b, ref = cfg1
    band = 0.02
    _, g0, _ = run(wl, b, "bf16", band=0.0)
    _, g1, st = run(wl, b, "bf16", band=band)
    l0, l1, l32 = cat(g0, "logit"), cat(g1, "logit"), cat(ref[1], "logit")
    inband = np.abs(sigmoid(l0) - 0.5) < band
    assert inband.any() and not inband.all()
    assert st["band"] == int(inband.sum())
    assert st["rerun_events"] == b.n_events
    # band edges: the FP32 path's logit and decision, bit for bit
    assert np.array_equal(l1[inband], l32[inband])
    assert np.array_equal(cat(g1, "kept")[inband], cat(ref[1], "kept")[inband])
    # the others keep the tensor-core result
    assert np.array_equal(l1[~inband], l0[~inband])
    # every BF16 error is inside the band here, so decisions match FP32
    assert np.mean(cat(g1, "kept") == cat(ref[1], "kept")) >= 0.9999
    # only the receptive field of the band edges was recomputed, step by step
    re, rv = receptive_field(g0, band, synth.shape_of(wl).iters, b)
    rows = TRACKER_ROWS["rows"]
    assert rows == {"edges": re, "hits": rv}, (rows, re, rv)
    assert (st["rescore_edges"], st["rescore_hits"]) == (re[0], rv[0])
    assert re[-1] == st["band"] and 0 < re[0] < st["edges"]


def receptive_field(graphs, band, K, batch):
    """Rows an FP32 re-score of the band edges needs per step, found by walking
    the message passing backwards on the host: edge step K - 1 needs the band
    edges; node step k the endpoints of the edges of edge step k (and the hits
    of node step k + 1); edge step k - 1 every edge touching a hit of node
    step k; the encoders the endpoints of the first step's edges.
    Returns (edges, hits), index 0 the encoders, k + 1 step k."""
    edges = [0] * (K + 1)
    hits = [0] * (K + 1)
    for e, g in enumerate(graphs):
        src, dst = g["src"].astype(np.int64), g["dst"].astype(np.int64)
        E = np.abs(sigmoid(g["logit"]) - 0.5) < band
        V = np.zeros(batch.event(e).n_hits, bool)
        edges[K] += int(E.sum())
        for k in range(K - 1, -1, -1):
            V[src[E]] = True
            V[dst[E]] = True
            hits[k + 1] += int(V.sum())
            E = E | V[src] | V[dst]
            edges[k] += int(E.sum())
        V[src[E]] = True
        V[dst[E]] = True
        hits[0] += int(V.sum())
    return edges, hits


@pytest.mark.parametrize("name,prec", [("cfg2_run3_single", "bf16"), ("cfg4_batched_fp8", "fp8")])
def test_rescore_band_wide_models(name, prec):
    """h = 64 (BF16) and h = 128 (FP8): band edges take the FP32 path's logits
    bit for bit, and the re-score recomputes exactly the receptive field."""
    wl = synth.workload(name)
    b = synth.workload_batch(wl, 2)
    band = 0.05
    _, g0, _ = run(wl, b, prec, band=0.0)
    _, g1, st = run(wl, b, prec, band=band)
    rows = TRACKER_ROWS["rows"]
    _, g32, _ = run(wl, b, "fp32")
    l0, l1, l32 = cat(g0, "logit"), cat(g1, "logit"), cat(g32, "logit")
    inband = np.abs(sigmoid(l0) - 0.5) < band
    assert inband.any()
    assert np.array_equal(l1[inband], l32[inband])
    assert np.array_equal(l1[~inband], l0[~inband])
    re, rv = receptive_field(g0, band, synth.shape_of(wl).iters, b)
    assert rows == {"edges": re, "hits": rv}, (rows, re, rv)


def test_bf16_rescored_agrees_with_oracle(cfg1):
    wl, b, _ = cfg1
    labels, g, _ = run(wl, b, "bf16", band=0.02)
    sh = synth.shape_of(wl)
    m = oracle.Model(synth.workload_weights(wl), sh.embed, sh.hidden, sh.iters)
    fs = pkg.feat_scale_of(pkg.make_cfg(wl["model"], wl["radius2"]))
    agree = union = 0
    for e in range(b.n_events):
        ev = b.event(e)
        ref = oracle.find_tracks_event(m, ev.x, ev.y, ev.z, ev.plane, wl["radius2"],
                                       wl["k_max"], feat_scale=fs)
        O = {(int(s), int(t)): int(k) for s, t, k in zip(ref.src, ref.dst, ref.keep)}
        G = {(int(s), int(t)): int(k) for s, t, k in zip(g[e]["src"], g[e]["dst"], g[e]["kept"])}
        for key in set(O) | set(G):
            agree += O.get(key, 0) == G.get(key, 0)
            union += 1
    assert agree / union >= 0.999, agree / union


def test_tensor_core_batch_equals_one_event_per_call(cfg1):
    wl, b, _ = cfg1
    labels_b, g_b, _ = run(wl, b, "bf16", band=0.02)
    for e in (0, 3):
        ev = b.event(e)
        lab, g, _ = run(wl, ev, "bf16", band=0.02)
        a = int(b.offsets[e])
        assert np.array_equal(lab, labels_b[a:a + ev.n_hits])
        for k in g[0]:
            assert np.array_equal(g[0][k], g_b[e][k]), k


@pytest.mark.parametrize("name,prec,mean_tol", [
    ("cfg2_run3_single", "bf16", 0.02),
    ("cfg2_run3_single", "fp8", 0.2),
    ("cfg4_batched_fp8", "fp8", 0.2),
])
def test_wide_models_logit_error(name, prec, mean_tol):
    """Without the re-score band: same graph as FP32, logit error within the
    format's bound (BF16 8 significant bits, E4M3 4)."""
    wl = synth.workload(name)
    b = synth.workload_batch(wl, 1)
    _, g32, _ = run(wl, b, "fp32")
    _, g, _ = run(wl, b, prec)
    assert np.array_equal(g[0]["src"], g32[0]["src"])
    d = np.abs(g[0]["logit"].astype(np.float64) - g32[0]["logit"])
    assert d.mean() < mean_tol, d.mean()


@pytest.mark.parametrize("name,prec", [
    pytest.param("cfg2_run3_single", "bf16", marks=pytest.mark.xfail(
        strict=True, reason="BF16 alone at h64 K8 agrees with FP32 on about 99.5 % of the "
                            "decisions; the re-score band brings it to the bar")),
    pytest.param("cfg4_batched_fp8", "fp8", marks=pytest.mark.xfail(
        strict=True, reason="E4M3 alone at h128 agrees with FP32 on about 95.8 % of the "
                            "decisions; the re-score band brings it to the bar")),
])
def test_wide_models_without_band_miss_the_bar(name, prec):
    """Recorded gap: the low-precision forms alone do not reach 99.9 % decision
    agreement on seeded weights, whose logits crowd the cut."""
    wl = synth.workload(name)
    b = synth.workload_batch(wl, 1)
    _, g32, _ = run(wl, b, "fp32")
    _, g, _ = run(wl, b, prec)
    assert np.mean(g[0]["kept"] == g32[0]["kept"]) >= 0.999


@pytest.mark.parametrize("name,prec,band,n_events", [
    ("cfg2_run3_single", "bf16", 0.02, 8),
    ("cfg4_batched_fp8", "fp8", 0.05, 8),
    ("cfg4_trained_fp8", "fp8", 0.05, 8),
])
def test_wide_models_with_band_at_the_bar(name, prec, band, n_events):
    """With the FP32 re-score band, the wide models agree with the FP64 oracle
    on >= 99.9 % of the edge decisions (union of both edge sets) and label
    most events identically."""
    import concurrent.futures as cf
    import os
    wl = synth.workload(name)
    b = synth.workload_batch(wl, n_events)
    labels, g, _ = run(wl, b, prec, band=band)
    sh = synth.shape_of(wl)
    m = oracle.Model(synth.workload_weights(wl), sh.embed, sh.hidden, sh.iters)
    fs = pkg.feat_scale_of(pkg.make_cfg(wl["model"], wl["radius2"]))

    def one(e):
        ev = b.event(e)
        return oracle.find_tracks_event(m, ev.x, ev.y, ev.z, ev.plane, wl["radius2"],
                                        wl["k_max"], feat_scale=fs)
    with cf.ThreadPoolExecutor(min(n_events, os.cpu_count() or 1)) as ex:
        refs = list(ex.map(one, range(n_events)))
    agree = union = same = 0
    for e, ref in enumerate(refs):
        O = {(int(s), int(t)): int(k) for s, t, k in zip(ref.src, ref.dst, ref.keep)}
        G = {(int(s), int(t)): int(k) for s, t, k in zip(g[e]["src"], g[e]["dst"], g[e]["kept"])}
        for key in set(O) | set(G):
            agree += O.get(key, 0) == G.get(key, 0)
            union += 1
        same += np.array_equal(labels[b.offsets[e]:b.offsets[e + 1]], ref.labels)
    assert agree / union >= 0.999, agree / union
    assert same >= n_events // 2, same


def test_bf16_at_hidden_128_is_rejected():
    wl = synth.workload("cfg4_batched_fp8")
    with pytest.raises(pkg.GnntrkError) as ei:
        pkg.tracker_for_workload(wl, precision="bf16", max_hits=1024, max_events=1)
    assert ei.value.status == 7


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_cuda_graph_replay_matches_direct_launches(prec):
    """use_graph: the first call of a shape is captured into a CUDA graph and
    later calls replay it; replays read the current contents of the buffers."""
    wl = synth.workload("cfg3_batched_bf16")
    b1 = synth.workload_batch(wl, 8)
    b2 = synth.workload_batch(wl, 8, first_event=8)
    n = max(b1.n_hits, b2.n_hits)
    ref = []
    for b in (b1, b2):
        lab, g, _ = run(wl, b, prec, band=0.02 if prec != "fp32" else 0.0)
        ref.append((lab, g))
    tr = pkg.tracker_for_workload(wl, precision=prec, max_hits=n, max_events=8,
                                  edges_per_hit=32, use_graph=True)
    s = torch.cuda.Stream()
    xyz = torch.zeros((3, n), dtype=torch.float32, device="cuda")
    plane = torch.zeros(n, dtype=torch.uint8, device="cuda")
    offs = torch.zeros(9, dtype=torch.int64, device="cuda")
    labels = torch.zeros(n, dtype=torch.int32, device="cuda")
    for rep in range(2):
        for k, b in enumerate((b1, b2)):
            # same shape and buffers each time: captured once, then replayed
            nh = b.n_hits
            xyz2 = torch.from_numpy(b.xyz_soa())
            xyz.zero_()
            xyz.view(-1)[:3 * nh].copy_(xyz2.reshape(-1).cuda())
            plane[:nh].copy_(torch.from_numpy(b.plane).cuda())
            offs.copy_(torch.from_numpy(b.offsets).cuda())
            torch.cuda.synchronize()
            tr.find_tracks(8, nh, xyz.view(-1)[:3 * nh], plane, offs, labels, s)
            tr.sync_status(s)
            assert np.array_equal(labels[:nh].cpu().numpy(), ref[k][0])
            for e in (0, 7):
                g = tr.get_graph(e)
                for key in g:
                    assert np.array_equal(g[key], ref[k][1][e][key]), key
    tr.close()


def test_autotune_picks_a_count_and_keeps_results():
    wl = synth.workload("cfg3_batched_bf16")
    b = synth.workload_batch(wl, 16)
    lab0, g0, _ = run(wl, b, "bf16", band=0.02)
    tr = pkg.tracker_for_workload(wl, precision="bf16", rescore_band=0.02, max_hits=b.n_hits,
                                  max_events=b.n_events, edges_per_hit=32)
    xyz = torch.from_numpy(b.xyz_soa()).cuda()
    plane = torch.from_numpy(b.plane).cuda()
    offs = torch.from_numpy(b.offsets).cuda()
    labels = torch.zeros(b.n_hits, dtype=torch.int32, device="cuda")
    choice = tr.autotune(b.n_events, b.n_hits, xyz, plane, offs, labels)
    assert all(1 <= v <= 8 for k, v in choice.items() if k.startswith("tc_") and k != "tc_edge_tma"), choice
    assert choice["tc_edge_tma"] in (0, 1, 2), choice
    assert all(v in (0, 1, 2) for k, v in choice.items() if k.startswith("f32_")), choice
    tr.find_tracks(b.n_events, b.n_hits, xyz, plane, offs, labels)
    tr.sync_status()
    # launch shapes do not change any result
    assert np.array_equal(labels.cpu().numpy(), lab0)
    g = tr.get_graph(5)
    for k in g:
        assert np.array_equal(g[k], g0[5][k]), k
    # the choice re-applied without timing gives the same results again
    tr.set_tuning(choice)
    tr.find_tracks(b.n_events, b.n_hits, xyz, plane, offs, labels)
    tr.sync_status()
    assert np.array_equal(labels.cpu().numpy(), lab0)
    # restore the default launch configuration for the other tests of this process
    tr.set_tuning({})
    tr.close()


@pytest.mark.parametrize("name,prec", [("cfg1_plain_fp32", "fp32"), ("cfg2_run3_single", "fp32"),
                                       ("cfg4_batched_fp8", "fp32"), ("cfg3_batched_bf16", "bf16"),
                                       ("cfg4_batched_fp8", "fp8")])
def test_fp32_tile_variants_give_identical_results(name, prec):
    """Every FP32 variant (4 or 8 warps per block, or the edge kernels that
    copy the next tile's rows in while a tile computes) computes each row with
    the same arithmetic: labels, graphs and logits are bit-identical across
    variants, for the FP32 path and for the FP32 re-score of the tensor-core
    paths, at hidden 32, 64 and 128."""
    wl = synth.workload(name)
    b = synth.workload_batch(wl, 3)
    band = 0.02 if prec != "fp32" else 0.0
    tr = pkg.tracker_for_workload(wl, precision=prec, rescore_band=band, max_hits=b.n_hits,
                                  max_events=b.n_events, edges_per_hit=32)
    ref = None
    try:
        for v in (0, 1, 2):
            tr.set_tuning({"f32_encoders": v, "f32_node_update": v, "f32_edge_update": v})
            labels = pkg.run_batch(tr, b)
            graphs = [tr.get_graph(e) for e in range(b.n_events)]
            if ref is None:
                ref = (labels, graphs)
                if prec != "fp32":
                    assert tr.stats()["band"] > 0
                continue
            assert np.array_equal(labels, ref[0]), v
            for e in range(b.n_events):
                for k in graphs[e]:
                    assert np.array_equal(graphs[e][k], ref[1][e][k]), (v, e, k)
    finally:
        tr.set_tuning({})
        tr.close()


@pytest.mark.parametrize("n_events,band", [(12, 0.0), (12, 0.02), (1, 0.02), (-1, 0.02)])
def test_tma_edge_step_gives_identical_results(n_events, band):
    """The BF16 edge step with TMA-staged tiles (form 1: a box of 128 e rows and
    row gathers of h_src, h_dst; form 2: the same loads in a ring of tile
    buffers with producer, MMA and epilogue warps) gives bit-identical logits,
    decisions, graphs and labels to the per-thread copies (form 0), on a batch
    whose CTAs each run several tiles (every ring slot and both accumulators,
    a ragged last tile) and on one event with fewer tiles than CTAs."""
    wl = synth.workload("cfg3_batched_bf16")
    # n_events = -1: two events at the largest occupancy (400 tracks, about
    # 4500 hits and 65 k edges each)
    b = (synth.workload_batch(wl, n_events) if n_events > 0 else
         synth.gen_batch(2, 4242, {"kind": "fixed", "n": 400}, wl["noise"]))
    tr = pkg.tracker_for_workload(wl, precision="bf16", rescore_band=band, max_hits=b.n_hits,
                                  max_events=b.n_events, edges_per_hit=32)
    ref = None
    try:
        for form in (0, 1, 2):
            tr.set_tuning({"tc_edge_tma": form})
            labels = pkg.run_batch(tr, b)
            graphs = [tr.get_graph(e) for e in range(b.n_events)]
            if ref is None:
                ref = (labels, graphs)
                assert tr.stats()["edges"] > (128 * 600 if b.n_events > 1 else 0)
                continue
            assert np.array_equal(labels, ref[0])
            for e in range(b.n_events):
                for k in graphs[e]:
                    assert np.array_equal(graphs[e][k], ref[1][e][k]), (e, k)
    finally:
        tr.set_tuning({})
        tr.close()


def test_set_tuning_rejects_out_of_range_choices():
    wl = synth.workload("cfg1_plain_fp32")
    tr = pkg.tracker_for_workload(wl, max_hits=1024, max_events=2)
    for bad in ({"f32_edge_update": 3}, {"tc_edge_update": 9}, {"f32_encoders": -1},
                {"tc_edge_tma": 3}):
        with pytest.raises(pkg.GnntrkError):
            tr.set_tuning(bad)
    tr.set_tuning({})
    tr.close()


def test_device_e4m3_conversion_matches_the_oracle_codec():
    """The activation conversion of the FP8 kernels (device) against the
    oracle's brute-force E4M3 codec, including ties, saturation and an odd
    count (the last pair is half used)."""
    from oracle import quant
    dec = np.array([quant.e4m3_decode(c) for c in range(256)])
    fin = np.sort(np.unique(dec[~np.isnan(dec)]))
    mids = (fin[:-1] + fin[1:]) / 2
    rng = np.random.default_rng(23)
    vals = np.concatenate([fin, mids, [447.9, 448.0, 460.0, 1e9, -1e9],
                           rng.normal(0, 30, 4001)]).astype(np.float32)
    assert vals.size % 2 == 1
    got = pkg.e4m3_encode(torch.from_numpy(vals).cuda()).cpu().numpy()
    want = quant.e4m3_encode_array(vals.astype(np.float64))
    assert np.array_equal(got, want), np.flatnonzero(got != want)[:10]


def test_tensor_core_throughput_probe():
    """The tcgen05 throughput probe runs and reports a rate below the chip's
    dense BF16 peak (2.25 PFLOP/s nominal) that grows with N."""
    rates = [pkg.tc_throughput(n, iters=4000) for n in (32, 128)]
    assert 0 < rates[0] <= rates[1] * 1.05
    assert rates[1] < 2600.0
