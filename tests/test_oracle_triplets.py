"""Pins of the oracle's triplet stage (Secs. "Triplet Building" and "Track
Building"): brute-force triplet enumeration, classifier routing and operand
order tied to the (separately pinned) edge classifier, hand-worked track
building cases including the thesis's motivating shared-hit pair."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2508_07423_gb300 import synth


def brute_triplets(plane, src, dst, keep):
    """Every unordered pair of kept edges sharing one hit, classified by the
    role of the shared hit."""
    out = set()
    kept = [e for e in range(len(src)) if keep[e]]
    key = lambda h: (int(plane[h]), int(h))
    for a, b in itertools.combinations(kept, 2):
        if dst[a] == src[b]:
            out.add((0, a, b))
        elif dst[b] == src[a]:
            out.add((0, b, a))
        elif src[a] == src[b]:
            x, y = (a, b) if key(dst[a]) < key(dst[b]) else (b, a)
            out.add((1, x, y))
        elif dst[a] == dst[b]:
            x, y = (a, b) if key(src[a]) < key(src[b]) else (b, a)
            out.add((2, x, y))
    return out


def random_graph(rng, n=40, ne=150, planes=6):
    plane = rng.integers(0, planes, n).astype(np.uint8)
    pairs = set()
    while len(pairs) < ne:
        a, b = rng.integers(0, n, 2)
        if plane[a] < plane[b]:
            pairs.add((int(a), int(b)))
    pairs = sorted(pairs)
    src = np.array([p[0] for p in pairs], np.int32)
    dst = np.array([p[1] for p in pairs], np.int32)
    keep = (rng.uniform(size=ne) < 0.7).astype(np.uint8)
    return plane, src, dst, keep


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_triplets_match_brute_force(seed):
    rng = np.random.default_rng(seed)
    plane, src, dst, keep = random_graph(rng)
    ty, e1, e2 = oracle.triplets(plane, src, dst, keep)
    got = set(zip(ty.tolist(), e1.tolist(), e2.tolist()))
    assert len(got) == len(ty)
    assert got == brute_triplets(plane, src, dst, keep)
    # count identity: sum over hits of in*out + C(out, 2) + C(in, 2)
    k = keep.astype(bool)
    din = np.bincount(dst[k], minlength=len(plane))
    dout = np.bincount(src[k], minlength=len(plane))
    assert len(ty) == int(np.sum(din * dout + dout * (dout - 1) // 2 + din * (din - 1) // 2))
    # listed by shared hit ascending
    shared = np.where(ty == 0, dst[e1], np.where(ty == 1, src[e1], dst[e1]))
    assert np.all(np.diff(shared) >= 0)


def with_heads(wl, art, elb):
    """The workload's blob with triplet classifiers appended."""
    arrs = synth.weight_arrays(synth.workload_weights(wl))
    return synth.pack_weights(arrs + list(art) + list(elb))


def test_triplet_classifier_order_and_routing():
    """An articulation classifier made of the edge classifier applied to the
    first operand (zero weights on the second) scores a triplet with the edge
    logit of e1; the elbow classifier built on the second operand gives the
    edge logit of e2. A swapped operand order or classifier fails here."""
    wl = synth.workload("cfg1_plain_fp32")
    sh = synth.shape_of(wl)
    h = sh.hidden
    arrs = synth.weight_arrays(synth.workload_weights(wl))
    (c1w, c1b), (c2w, c2b) = arrs[-2], arrs[-1]
    z = np.zeros((h, h), np.float32)
    art = [(np.concatenate([c1w, z], 1), c1b), (c2w, c2b)]
    elb = [(np.concatenate([z, c1w], 1), c1b), (c2w, c2b)]
    m = oracle.Model(with_heads(wl, art, elb), sh.embed, sh.hidden, sh.iters)
    ev = synth.workload_batch(wl, 1)
    r = oracle.find_tracks_event(m, ev.x, ev.y, ev.z, ev.plane, wl["radius2"], wl["k_max"])
    E = oracle.edge_states(m, ev.x, ev.y, ev.z, r.src, r.dst)
    ty, e1, e2 = oracle.triplets(ev.plane, r.src, r.dst, r.keep)
    assert (ty == 0).any() and (ty > 0).any()
    tl = oracle.triplet_logits(m, ty, e1, e2, E)
    want = np.where(ty == 0, r.logit[e1], r.logit[e2])
    assert np.max(np.abs(tl - want)) < 1e-12


def test_triplet_classifier_types_and_degenerate_input():
    """Zero layer-2 weights: the output is the layer-2 bias of the classifier
    the type selects (articulation +5, elbows -5)."""
    wl = synth.workload("cfg1_plain_fp32")
    sh = synth.shape_of(wl)
    h = sh.hidden
    rng = np.random.default_rng(0)
    l1 = (rng.normal(size=(h, 2 * h)).astype(np.float32), np.zeros(h, np.float32))
    art = [l1, (np.zeros((1, h), np.float32), np.array([5.0], np.float32))]
    elb = [l1, (np.zeros((1, h), np.float32), np.array([-5.0], np.float32))]
    m = oracle.Model(with_heads(wl, art, elb), sh.embed, sh.hidden, sh.iters)
    E = rng.normal(size=(4, h))
    ty = np.array([0, 1, 2, 0], np.int32)
    tl = oracle.triplet_logits(m, ty, [0, 1, 2, 3], [1, 2, 3, 0], E)
    assert np.array_equal(tl, [5.0, -5.0, -5.0, 5.0])
    # e1 == e2 with W1 = [I, -I], b1 = 0: the hidden row is 0, LayerNorm of a
    # constant row is 0, the logit is the bias alone
    I = np.eye(h, dtype=np.float32)
    art = [(np.concatenate([I, -I], 1), np.zeros(h, np.float32)),
           (rng.normal(size=(1, h)).astype(np.float32), np.array([0.25], np.float32))]
    m = oracle.Model(with_heads(wl, art, art), sh.embed, sh.hidden, sh.iters)
    tl = oracle.triplet_logits(m, np.zeros(3, np.int32), [0, 1, 2], [0, 1, 2], E)
    assert np.allclose(tl, 0.25, atol=0, rtol=0)


def tracks_of(n, plane, edges, reject=()):
    """Track building with every triplet kept except those in `reject`
    (given as (type, (a, b), (c, d)) edge pairs)."""
    src = np.array([a for a, _ in edges], np.int32)
    dst = np.array([b for _, b in edges], np.int32)
    keep = np.ones(len(edges), np.uint8)
    ty, e1, e2 = oracle.triplets(np.asarray(plane, np.uint8), src, dst, keep)
    idx = {e: i for i, e in enumerate(edges)}
    rej = {(t, idx[a], idx[b]) for t, a, b in reject}
    tk = np.array([(int(t), int(a), int(b)) not in rej for t, a, b in zip(ty, e1, e2)], np.uint8)
    assert len(rej) == len(tk) - int(tk.sum())
    return [t.tolist() for t in oracle.build_tracks(n, src, dst, keep, ty, e1, e2, tk)]


def test_track_building_straight_track_with_skips():
    # hits 0..3 on planes 0..3, consecutive edges and the two skip edges; every
    # triplet kept: the elbows merge the skip edges into the chain, one track
    edges = [(0, 1), (1, 2), (2, 3), (0, 2), (1, 3)]
    assert tracks_of(4, [0, 1, 2, 3], edges) == [[0, 1, 2, 3]]


def test_track_building_splits_shared_hit_pair():
    """The thesis's motivating case: two tracks sharing their first two hits
    (S0, S1), then branching (A2, A3) and (B2, B3). The elbow S1->A2, S1->B2
    joins two different tracks and is rejected; the two articulations leaving
    the shared edge are then shared links and the shared segment is
    duplicated into each branch. Plain components would merge all six hits."""
    S0, S1, A2, A3, B2, B3 = range(6)
    plane = [0, 1, 2, 3, 2, 3]
    edges = [(S0, S1), (S1, A2), (A2, A3), (S1, B2), (B2, B3)]
    got = tracks_of(6, plane, edges, reject=[(1, (S1, A2), (S1, B2))])
    assert got == [[S0, S1, A2, A3], [S0, S1, B2, B3]]
    src = np.array([a for a, _ in edges], np.int32)
    dst = np.array([b for _, b in edges], np.int32)
    labels = oracle.components(6, src, dst, np.ones(5, np.uint8))
    assert len(set(labels.tolist())) == 1


def test_track_building_rejected_articulation_splits():
    edges = [(0, 1), (1, 2), (2, 3)]
    got = tracks_of(4, [0, 1, 2, 3], edges, reject=[(0, (1, 2), (2, 3))])
    assert got == [[0, 1, 2], [2, 3]]


def test_track_building_without_triplets_gives_edges():
    """No triplet kept: every kept edge is its own group and component, so
    the tracks are exactly the kept edges' hit pairs."""
    rng = np.random.default_rng(5)
    plane, src, dst, keep = random_graph(rng, n=30, ne=80)
    ty, e1, e2 = oracle.triplets(plane, src, dst, keep)
    tracks = oracle.build_tracks(30, src, dst, keep, ty, e1, e2, np.zeros(len(ty), np.uint8))
    want = sorted([sorted([int(a), int(b)]) for a, b, k in zip(src, dst, keep) if k])
    assert [t.tolist() for t in tracks] == want


def test_track_building_all_kept_no_forks_equals_components():
    """Every triplet kept on a graph where no group links to two groups (a
    set of disjoint chains): the tracks are the weakly connected components."""
    rng = np.random.default_rng(9)
    edges, plane = [], []
    n = 0
    for _ in range(6):
        L = int(rng.integers(2, 7))
        ids = list(range(n, n + L))
        plane += list(range(L))
        edges += [(ids[i], ids[i + 1]) for i in range(L - 1)]
        n += L
    got = tracks_of(n, plane, edges)
    src = np.array([a for a, _ in edges], np.int32)
    dst = np.array([b for _, b in edges], np.int32)
    lab = oracle.components(n, src, dst, np.ones(len(edges), np.uint8))
    comps = {}
    for i, l in enumerate(lab):
        comps.setdefault(int(l), []).append(i)
    assert got == sorted(v for v in comps.values() if len(v) > 1)


def test_empty_inputs():
    """No hits, no edges, no kept edges: no triplets and no tracks."""
    e = np.zeros(0, np.int32)
    ty, e1, e2 = oracle.triplets(np.zeros(0, np.uint8), e, e, np.zeros(0, np.uint8))
    assert len(ty) == 0
    assert oracle.build_tracks(0, e, e, np.zeros(0, np.uint8), ty, e1, e2,
                               np.zeros(0, np.uint8)) == []
    src, dst = np.array([0], np.int32), np.array([1], np.int32)
    ty, e1, e2 = oracle.triplets(np.array([0, 1], np.uint8), src, dst, np.zeros(1, np.uint8))
    assert len(ty) == 0
    assert oracle.build_tracks(2, src, dst, np.zeros(1, np.uint8), ty, e1, e2,
                               np.zeros(0, np.uint8)) == []


def test_whole_path_with_triplets_on_hand_built_event():
    """The hand-built event through the whole path and the triplet stage, for
    the four on/off settings of the two triplet heads; the triplet counts and
    the tracks are those worked out by hand in
    tests/golden/triplet_pipeline_hand.json."""
    import json
    import os
    from parity import hand_pipeline, hand_pipeline_blob
    gold = os.path.join(os.path.dirname(__file__), "golden", "triplet_pipeline_hand.json")
    with open(gold) as f:
        t = json.load(f)
    g, x, y, z, plane, idx = hand_pipeline()
    for case in t["cases"]:
        blob = hand_pipeline_blob(8, 2, g["classifier_bias"],
                                  triplet_bias=(case["articulation_bias"], case["elbow_bias"]))
        m = oracle.Model(blob, [3, 4, 4], 8, 2)
        r = oracle.find_tracks_triplets_event(m, x, y, z, plane, g["r2"], g["k_max"],
                                              cut=g["cut_keep_all"])
        assert np.all(r.keep == 1)
        counts = np.bincount(r.ttype, minlength=3)
        assert list(counts) == [t["triplets"]["articulation"], t["triplets"]["left_elbow"],
                                t["triplets"]["right_elbow"]]
        want = sorted(sorted(idx[n] for n in tr) for tr in case["tracks"])
        got = sorted(sorted(int(i) for i in tr) for tr in r.tracks)
        assert got == want, case
