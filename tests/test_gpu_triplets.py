"""GPU parity of the triplet stage (Secs. "Triplet Building" and "Track
Building") against the FP64 oracle, through the C ABI: triplet sets, triplet
scores and decisions, and the tracks, element by element."""
import math

import numpy as np
import pytest

import oracle
import paper_2508_07423_gb300 as pkg
from paper_2508_07423_gb300 import synth
from parity import SCORE_TOL, compare_event, sigmoid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def model_of(wl, blob=None):
    sh = synth.shape_of(wl)
    return oracle.Model(blob or synth.workload_weights(wl), sh.embed, sh.hidden, sh.iters)


def oracle_triplets(model, ev, ref, fs):
    """Oracle triplets of one event as {(type, A, C, B): logit}."""
    E = oracle.edge_states(model, ev.x, ev.y, ev.z, ref.src, ref.dst, fs)
    ty, e1, e2 = oracle.triplets(ev.plane, ref.src, ref.dst, ref.keep)
    tl = oracle.triplet_logits(model, ty, e1, e2, E)
    out = {}
    for t, a, b, l in zip(ty, e1, e2, tl):
        if t == 0:
            key = (0, int(ref.src[a]), int(ref.dst[a]), int(ref.dst[b]))
        elif t == 1:
            key = (1, int(ref.dst[a]), int(ref.src[a]), int(ref.dst[b]))
        else:
            key = (2, int(ref.src[a]), int(ref.dst[a]), int(ref.src[b]))
        out[key] = float(l)
    return out, (ty, e1, e2, tl)


def canon(tracks):
    return sorted(tuple(sorted(int(v) for v in t)) for t in tracks)


def gpu_triplets(tr, e):
    t = tr.get_triplets(e)
    return {(int(a), int(h[0]), int(h[1]), int(h[2])): (float(l), int(k))
            for a, h, l, k in zip(t["type"], t["hits"], t["logit"], t["kept"])}


def compare_triplet_event(tr, e, ev, g, labels, tracks, model, wl, fs):
    rep = compare_event(ev, g, labels, model, wl["radius2"], wl["k_max"], wl["model"]["iters"],
                        wl["cut"], fs)
    ref = oracle.find_tracks_event(model, ev.x, ev.y, ev.z, ev.plane, wl["radius2"], wl["k_max"],
                                   wl["cut"], feat_scale=fs)
    gk = {(int(s), int(d)) for s, d, k in zip(g["src"], g["dst"], g["kept"]) if k}
    ok = {(int(s), int(d)) for s, d, k in zip(ref.src, ref.dst, ref.keep) if k}
    G = gpu_triplets(tr, e)
    if gk != ok:
        return rep, None, None
    O, (ty, e1, e2, tl) = oracle_triplets(model, ev, ref, fs)
    assert set(G) == set(O), (len(set(G) - set(O)), len(set(O) - set(G)))
    tcut = math.log(wl.get("triplet_cut", 0.5) / (1 - wl.get("triplet_cut", 0.5)))
    err = max((abs(sigmoid(G[k][0]) - sigmoid(O[k])) for k in O), default=0.0)
    assert err <= SCORE_TOL, err
    clear = [k for k in O if abs(O[k] - tcut) > 4 * SCORE_TOL]
    assert all(G[k][1] == (O[k] >= tcut) for k in clear)
    same = all(G[k][1] == (O[k] >= tcut) for k in O)
    if not same:
        return rep, len(O), None
    tk = (tl >= tcut).astype(np.uint8)
    want = oracle.build_tracks(ev.n_hits, ref.src, ref.dst, ref.keep, ty, e1, e2, tk)
    assert canon(tracks) == canon(want)
    # hits of every track are in (plane, index) order
    for t in tracks:
        key = [(int(ev.plane[v]), int(v)) for v in t]
        assert key == sorted(key)
    return rep, len(O), len(want)


@pytest.fixture(scope="module")
def cfg6():
    wl = synth.workload("cfg6_triplets")
    return wl, model_of(wl)


def test_triplets_fp32_parity(cfg6):
    wl, model = cfg6
    b = synth.workload_batch(wl, 6)
    tr = pkg.tracker_for_workload(wl, precision="fp32", max_hits=b.n_hits, max_events=b.n_events)
    labels, tracks = pkg.run_batch_triplets(tr, b)
    fs = pkg.feat_scale_of(tr.cfg)
    n_trk = n_tri = 0
    for e in range(b.n_events):
        ev = b.event(e)
        a = int(b.offsets[e])
        _, nt, nk = compare_triplet_event(tr, e, ev, tr.get_graph(e), labels[a:a + ev.n_hits],
                                          tracks[e], model, wl, fs)
        n_tri += nt is not None
        n_trk += nk is not None
    assert n_tri >= 5 and n_trk >= 4, (n_tri, n_trk)
    st = tr.triplet_stats()
    assert st["tracks"] == sum(len(t) for t in tracks)
    assert st["track_hits"] == sum(len(x) for t in tracks for x in t)


def test_triplets_random_heads_stress():
    """Seeded random weights with random triplet classifiers: dense graphs,
    about half of the triplets kept, many forks and shared links; tracks
    element by element against the oracle."""
    wl = dict(synth.workload("cfg3_batched_bf16"))
    sh = synth.shape_of(wl)
    h = sh.hidden
    arrs = synth.weight_arrays(synth.workload_weights(wl))
    rng = np.random.default_rng(77)
    heads = []
    for _ in range(2):
        heads.append((rng.uniform(-0.2, 0.2, (h, 2 * h)).astype(np.float32),
                      rng.uniform(-0.1, 0.1, h).astype(np.float32)))
        heads.append((rng.uniform(-0.3, 0.3, (1, h)).astype(np.float32),
                      np.zeros(1, np.float32)))
    blob = synth.pack_weights(arrs + heads)
    model = model_of(wl, blob)
    b = synth.workload_batch(wl, 3)
    cfg = pkg.make_cfg(wl["model"], wl["radius2"], k_max=wl["k_max"], max_hits=b.n_hits,
                       max_events=b.n_events, triplets=True, triplets_per_hit=64)
    tr = pkg.Tracker(blob, cfg)
    labels, tracks = pkg.run_batch_triplets(tr, b, tracks_per_hit=8, hits_per_hit=64)
    fs = pkg.feat_scale_of(cfg)
    done = 0
    for e in range(b.n_events):
        ev = b.event(e)
        a = int(b.offsets[e])
        _, nt, nk = compare_triplet_event(tr, e, ev, tr.get_graph(e), labels[a:a + ev.n_hits],
                                          tracks[e], model, wl, fs)
        done += nk is not None
    assert done >= 2
    st = tr.triplet_stats()
    assert st["articulations"] > 10 * b.n_hits // 10 and 0 < st["kept"]


def test_triplets_bf16_metrics_match_oracle(cfg6):
    """BF16 + FP32 re-score: keep decisions of edges and triplets agree with
    the oracle, and the track metrics equal the oracle's within 0.5 pp."""
    from oracle import metrics
    wl, model = cfg6
    b = synth.workload_batch(wl, 12, first_event=30)
    tr = pkg.tracker_for_workload(wl, max_hits=b.n_hits, max_events=b.n_events)
    assert tr.cfg.precision == pkg.BF16 and tr.cfg.triplets == 1
    labels, tracks = pkg.run_batch_triplets(tr, b)
    fs = pkg.feat_scale_of(tr.cfg)
    ref_tracks = []
    agree = union = 0
    for e in range(b.n_events):
        ev = b.event(e)
        r = oracle.find_tracks_triplets_event(model, ev.x, ev.y, ev.z, ev.plane, wl["radius2"],
                                              wl["k_max"], wl["cut"], wl["triplet_cut"],
                                              feat_scale=fs)
        ref_tracks.append(r.tracks)
        G = gpu_triplets(tr, e)
        O = {}
        for t, a, c, l, k in zip(r.ttype, r.te1, r.te2, r.tlogit, r.tkeep):
            key = ((0, int(r.src[a]), int(r.dst[a]), int(r.dst[c])) if t == 0 else
                   (1, int(r.dst[a]), int(r.src[a]), int(r.dst[c])) if t == 1 else
                   (2, int(r.src[a]), int(r.dst[a]), int(r.src[c])))
            O[key] = int(k)
        for key in set(O) | set(G):
            agree += O.get(key, 0) == G.get(key, (0.0, 0))[1]
            union += 1
    # triplets: BF16 final edge encodings feed the FP32 triplet classifier
    # (the re-score band covers edge decisions only)
    assert agree / union >= 0.995, agree / union
    g = metrics.batch_track_counts(tracks, b.pid, b.offsets, pid2=b.pid2).summary()
    o = metrics.batch_track_counts(ref_tracks, b.pid, b.offsets, pid2=b.pid2).summary()
    for k in ("efficiency", "ghost_rate", "clone_rate"):
        assert abs(g[k] - o[k]) <= 0.005, (k, g, o)


def test_triplet_outputs_capacity_and_repeat(cfg6):
    wl, _ = cfg6
    b = synth.workload_batch(wl, 2)
    tr = pkg.tracker_for_workload(wl, precision="fp32", max_hits=b.n_hits, max_events=b.n_events)
    l1, t1 = pkg.run_batch_triplets(tr, b)
    l2, t2 = pkg.run_batch_triplets(tr, b)
    assert np.array_equal(l1, l2)
    assert [[x.tolist() for x in t] for t in t1] == [[x.tolist() for x in t] for t in t2]
    with pytest.raises(pkg.GnntrkError) as ei:
        pkg.run_batch_triplets(tr, b, tracks_per_hit=0, hits_per_hit=0)
    assert ei.value.status == 4
    l3, t3 = pkg.run_batch_triplets(tr, b)
    assert [[x.tolist() for x in t] for t in t3] == [[x.tolist() for x in t] for t in t1]


def test_triplets_need_heads_and_flag():
    wl = synth.workload("cfg3_trained_bf16")
    with pytest.raises(pkg.GnntrkError) as ei:
        pkg.tracker_for_workload(wl, max_hits=1024, max_events=2, triplets=True)
    assert ei.value.status == 6
    tr = pkg.tracker_for_workload(synth.workload("cfg6_triplets"), max_hits=1024, max_events=2,
                                  triplets=False)
    b = synth.gen_batch(1, 3, {"kind": "fixed", "n": 5}, 0.0)
    with pytest.raises(pkg.GnntrkError) as ei:
        pkg.run_batch_triplets(tr, b)
    assert ei.value.status == 1


def test_triplets_ragged_and_degenerate_events(cfg6):
    """Empty, single-hit, one-plane and last-plane-only events, a dense event
    and a small one in one batch: per event, triplets and tracks against the
    oracle; events without kept edges have no tracks."""
    from test_gpu_parity import special_events
    wl, model = cfg6
    evs = special_events()
    b = synth.concat(evs)
    tr = pkg.tracker_for_workload(wl, precision="fp32", max_hits=b.n_hits, max_events=b.n_events)
    labels, tracks = pkg.run_batch_triplets(tr, b)
    fs = pkg.feat_scale_of(tr.cfg)
    assert tracks[0] == [] and tracks[1] == [] and tracks[2] == [] and tracks[3] == []
    checked = 0
    for e in range(b.n_events):
        ev = b.event(e)
        a = int(b.offsets[e])
        _, nt, nk = compare_triplet_event(tr, e, ev, tr.get_graph(e), labels[a:a + ev.n_hits],
                                          tracks[e], model, wl, fs)
        checked += nk is not None
    assert checked >= 5


def test_triplet_workspace_capacity_latches_and_recovers(cfg6):
    wl, _ = cfg6
    b = synth.workload_batch(wl, 2)
    tr = pkg.tracker_for_workload(wl, precision="fp32", max_hits=b.n_hits, max_events=b.n_events,
                                  triplets_per_hit=1)
    with pytest.raises(pkg.GnntrkError) as ei:
        pkg.run_batch_triplets(tr, b)
    assert ei.value.status == 4 and "articulations" in str(ei.value)
    # a call that fits works afterwards
    small = synth.gen_batch(1, 5, {"kind": "fixed", "n": 3}, 0.0)
    pkg.run_batch_triplets(tr, small)
