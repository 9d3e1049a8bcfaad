"""Pins of the FP64 oracle against things other than itself: hand-worked
examples, closed forms of special weight choices, brute force on tiny inputs and
invariants. CPU only."""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import metrics
from paper_2508_07423_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
EPS_LN = 1e-5


def gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def zeros(o, i):
    return (np.zeros((o, i), np.float32), np.zeros(o, np.float32))


def gnn_layers(h, K, rng=None, zero_steps=False):
    """Weight list for the GNN part (after the embedding layers)."""
    def rnd(o, i):
        b = math.sqrt(6.0 / i)
        return (rng.uniform(-b, b, (o, i)).astype(np.float32),
                rng.uniform(-0.3, 0.3, o).astype(np.float32))
    L = [rnd(h, 3), rnd(h, h), rnd(h, 2 * h), rnd(h, h)]
    for _ in range(K):
        if zero_steps:
            L += [zeros(h, 3 * h), zeros(h, h), zeros(h, 3 * h), zeros(h, h)]
        else:
            L += [rnd(h, 3 * h), rnd(h, h), rnd(h, 3 * h), rnd(h, h)]
    L += [rnd(h, h), rnd(1, h)]
    return L


# ----------------------------------------------------------------------------
# embedding MLP
# ----------------------------------------------------------------------------
def test_embed_hand_worked():
    g = gold("embed_hand.json")
    x, y, z = ([v] for v in g["hit"])
    for case in g["cases"]:
        W = [(np.array(g["W1"], np.float32), np.array(g["b1"], np.float32)),
             (np.array(case["W2"], np.float32), np.array(case["b2"], np.float32))]
        blob = synth.pack_weights(W + gnn_layers(2, 0, np.random.default_rng(0)))
        m = oracle.Model(blob, [3, 2, 1], 2, 0)
        e = oracle.embed(m, x, y, z)
        assert e[0, 0] == pytest.approx(case["expected"], abs=1e-12)


def test_embed_identity_weights_give_features():
    # identity layers and zero biases: ReLU leaves the non-negative features
    # (r/45, phi/pi, z/750) unchanged. Hit (3, 4, 150): r = 5, phi = atan2(4, 3).
    I3 = (np.eye(3, dtype=np.float32), np.zeros(3, np.float32))
    blob = synth.pack_weights([I3, I3, I3] + gnn_layers(2, 0, np.random.default_rng(0)))
    m = oracle.Model(blob, [3, 3, 3, 3], 2, 0)
    e = oracle.embed(m, [3.0], [4.0], [150.0])
    assert e[0] == pytest.approx([5 / 45, 0.9272952180016122 / math.pi, 0.2], abs=1e-12)


# ----------------------------------------------------------------------------
# rough graph
# ----------------------------------------------------------------------------
def edge_set(src, dst):
    return {(int(a), int(b)) for a, b in zip(src, dst)}


def test_radius_graph_hand_worked():
    g = gold("radius_hand.json")
    emb = np.array(g["emb"], np.float64)[:, None]
    src, dst, d2 = oracle.radius_graph(g["plane"], emb, g["r2"], g["k_max"])
    assert edge_set(src, dst) == {tuple(e) for e in g["edges"]}
    assert np.allclose(d2, (emb[src, 0] - emb[dst, 0]) ** 2)


def test_radius_graph_is_strict():
    # d2 exactly equal to the squared radius does not pass
    plane = [0, 1]
    emb = np.array([[0.0], [0.5]])
    s, d, _ = oracle.radius_graph(plane, emb, 0.25, 64)
    assert len(s) == 0
    s, d, _ = oracle.radius_graph(plane, emb, np.nextafter(0.25, 1.0), 64)
    assert edge_set(s, d) == {(0, 1)}


def test_radius_graph_kmax_and_tiebreak():
    # hit 0 (plane 0) has six plane-1 candidates at 0.1 .. 0.6 and a plane-2
    # candidate at 0.05; with k_max = 3 the three nearest survive
    plane = [0, 1, 1, 1, 1, 1, 1, 2]
    emb = np.array([0.0, 0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.05])[:, None]
    s, d, _ = oracle.radius_graph(plane, emb, 1.0, 3)
    assert {e for e in edge_set(s, d) if e[0] == 0} == {(0, 7), (0, 1), (0, 2)}
    # equal distances: the key (d2, plane, index) prefers the lower plane,
    # then the lower index
    plane = [0, 2, 1, 1]
    emb = np.array([0.0, 0.25, 0.25, 0.25])[:, None]
    row0 = lambda s, d: {e for e in edge_set(s, d) if e[0] == 0}
    s, d, _ = oracle.radius_graph(plane, emb, 1.0, 1)
    assert row0(s, d) == {(0, 2)}
    s, d, _ = oracle.radius_graph(plane, emb, 1.0, 2)
    assert row0(s, d) == {(0, 2), (0, 3)}


def brute_force_graph(plane, emb, r2, k_max):
    out = set()
    n = len(plane)
    for i in range(n):
        c = []
        for j in range(n):
            if plane[j] - plane[i] in (1, 2):
                dd = float(np.sum((emb[i] - emb[j]) ** 2))
                if dd < r2:
                    c.append((dd, plane[j], j))
        for dd, _, j in sorted(c)[:k_max]:
            out.add((i, j))
    return out


@pytest.mark.parametrize("seed", range(6))
def test_radius_graph_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = 40
    plane = rng.integers(0, 6, n)
    emb = rng.normal(size=(n, 3))
    for k_max in (2, 64):
        s, d, _ = oracle.radius_graph(plane, emb, 1.5, k_max)
        assert edge_set(s, d) == brute_force_graph(plane, emb, 1.5, k_max)


@pytest.mark.parametrize("seed", range(4))
def test_candidate_d2_brute_force(seed):
    """The all-pairs list the radius calibration draws its quantiles from: every
    pair from plane p to plane p+1 or p+2 (below n_planes), squared distance,
    no radius and no cap, as a multiset; its size is sum_p n_p (n_p+1 + n_p+2)."""
    rng = np.random.default_rng(100 + seed)
    n, n_planes = 30, 5
    plane = rng.integers(0, n_planes + 2, n)  # some hits on planes past the last
    emb = rng.normal(size=(n, 4))
    got = np.sort(oracle.candidate_d2(plane, emb, n_planes=n_planes))
    ref = sorted(float(np.sum((emb[i] - emb[j]) ** 2)) for i in range(n) for j in range(n)
                 if plane[j] - plane[i] in (1, 2) and plane[j] < n_planes)
    assert got.size == len(ref)
    assert np.allclose(got, ref, rtol=0, atol=1e-12)
    cnt = np.bincount(plane, minlength=n_planes + 4)
    assert got.size == sum(int(cnt[p]) * (int(cnt[p + 1]) * (p + 1 < n_planes) +
                                          int(cnt[p + 2]) * (p + 2 < n_planes))
                           for p in range(n_planes))
    # with no radius and no cap the radius graph keeps exactly these pairs
    _, _, d2 = oracle.radius_graph(plane, emb, 1e30, n, n_planes=n_planes)
    assert np.allclose(np.sort(d2), got, rtol=0, atol=1e-12)


def test_radius_graph_invariants_on_event():
    wl = synth.workload("cfg1_plain_fp32")
    sh = synth.shape_of(wl)
    m = oracle.Model(synth.workload_weights(wl), sh.embed, sh.hidden, sh.iters)
    ev = synth.workload_batch(wl, 1).event(0)
    emb = oracle.embed(m, ev.x, ev.y, ev.z)
    s, d, d2 = oracle.radius_graph(ev.plane, emb, wl["radius2"], 4)
    dp = ev.plane[d].astype(int) - ev.plane[s].astype(int)
    assert set(np.unique(dp)) <= {1, 2}
    assert np.all(d2 < wl["radius2"])
    assert np.bincount(s, minlength=ev.n_hits).max() <= 4
    # symmetric metric: d2(i, j) = d2(j, i)
    assert np.allclose(d2, np.sum((emb[s] - emb[d]) ** 2, axis=1))


# ----------------------------------------------------------------------------
# interaction network
# ----------------------------------------------------------------------------
def switch(z, W2, b2):
    """Closed form of Linear -> LayerNorm -> ReLU -> Linear when the first
    layer is [u; -u] with bias [beta; -beta] (z = u.v + beta): the hidden pair
    [z, -z] normalises to [z, -z] / sqrt(z^2 + eps), the ReLU keeps one entry,
    so the output is g * W2[:, 0 if z > 0 else 1] + b2 with
    g = |z| / sqrt(z^2 + eps) (just b2 when z = 0)."""
    # the blob stores float32 weights: use the same rounded values
    W2 = np.asarray(W2, np.float32).astype(float)
    b2 = np.asarray(b2, np.float32).astype(float)
    if z == 0:
        return b2.copy()
    g = abs(z) / math.sqrt(z * z + EPS_LN)
    return g * W2[:, 0 if z > 0 else 1] + b2


def pm(u, beta):
    u = np.asarray(u, np.float32)
    return (np.stack([u, -u]), np.array([beta, -beta], np.float32))


def test_in_hand_worked_switch_network():
    """Three hits, edges 0->1, 1->2, 0->2, h = 2, one message-passing step.
    Every sub-network uses the switch form above, so each value is a column of
    its second layer; the composition below is written out by hand for this
    graph (which sums feed which node, which encodings feed which edge)."""
    NE2 = ([[1, 0], [0, 1]], [0, 0])
    EE2 = ([[2, 0], [0, 3]], [0.5, -0.5])
    N2 = ([[1, -1], [0.5, 2]], [0.25, 0])
    E2 = ([[1, 0], [0, 1]], [0, 0.1])
    C2 = ([[1, -2]], [0.1])
    arr = lambda t: (np.array(t[0], np.float32), np.array(t[1], np.float32))
    layers = [zeros(1, 3),                       # embedding (unused here)
              pm([1, 0, 0], 0), arr(NE2),        # node encoder: z = x/45
              pm([1, 0, -1, 0], 0), arr(EE2),    # edge encoder: z = h_src[0] - h_dst[0]
              pm([0, 0, 1, 0, -1, 0], 0), arr(N2),  # node net: z = out[0] - in[0]
              pm([1, 0, 0, 1, 0, -1], -1), arr(E2),  # edge net: z = e[0] + hs[1] - hd[1] - 1
              pm([1, -1], 0), arr(C2)]           # classifier: z = e[0] - e[1]
    m = oracle.Model(synth.pack_weights(layers), [3, 1], 2, 1)
    x, y, z = [45.0, -45.0, 45.0], [0.0] * 3, [0.0] * 3
    src, dst = [0, 1, 0], [1, 2, 2]
    got = oracle.in_logits(m, x, y, z, src, dst)

    # node encoder: x/45 = +1, -1, +1
    h = [switch(1.0, *NE2), switch(-1.0, *NE2), switch(1.0, *NE2)]
    # edge encoder on [h_src, h_dst]
    e = [switch(h[0][0] - h[1][0], *EE2),    # 0->1
         switch(h[1][0] - h[2][0], *EE2),    # 1->2
         switch(h[0][0] - h[2][0], *EE2)]    # 0->2 (z = 0)
    # messages: node 0 sends e0, e2; node 1 sends e1 and receives e0;
    # node 2 receives e1, e2
    out0, in0 = e[0] + e[2], np.zeros(2)
    out1, in1 = e[1], e[0]
    out2, in2 = np.zeros(2), e[1] + e[2]
    h = [h[0] + switch(out0[0] - in0[0], *N2),
         h[1] + switch(out1[0] - in1[0], *N2),
         h[2] + switch(out2[0] - in2[0], *N2)]
    # edge network on [e, h_src, h_dst] with the UPDATED node encodings
    e = [e[0] + switch(e[0][0] + h[0][1] - h[1][1] - 1, *E2),
         e[1] + switch(e[1][0] + h[1][1] - h[2][1] - 1, *E2),
         e[2] + switch(e[2][0] + h[0][1] - h[2][1] - 1, *E2)]
    want = [switch(v[0] - v[1], *C2)[0] for v in e]
    assert got == pytest.approx(want, abs=1e-12)


def test_in_zero_step_networks_are_identity():
    # zero node/edge networks: the residual steps change nothing, so K = 3
    # gives the same logits as K = 0 with the same encoders and classifier
    rng = np.random.default_rng(3)
    h = 8
    base = gnn_layers(h, 0, np.random.default_rng(7))
    with_steps = base[:4] + [l for _ in range(3) for l in
                             (zeros(h, 3 * h), zeros(h, h), zeros(h, 3 * h), zeros(h, h))] + base[4:]
    emb = [zeros(2, 3)]
    m0 = oracle.Model(synth.pack_weights(emb + base), [3, 2], h, 0)
    m3 = oracle.Model(synth.pack_weights(emb + with_steps), [3, 2], h, 3)
    n = 20
    x, y, z = rng.uniform(-40, 40, n), rng.uniform(-40, 40, n), rng.uniform(-300, 700, n)
    src, dst = rng.integers(0, n, 50), rng.integers(0, n, 50)
    a = oracle.in_logits(m0, x, y, z, src, dst)
    b = oracle.in_logits(m3, x, y, z, src, dst)
    assert np.array_equal(a, b)


def test_in_permutation_invariance():
    # relabelling hits and reordering edges permutes the logits (sum
    # aggregation is permutation invariant)
    rng = np.random.default_rng(11)
    h, K, n, ne = 8, 3, 30, 90
    m = oracle.Model(synth.pack_weights([zeros(2, 3)] + gnn_layers(h, K, rng)), [3, 2], h, K)
    x, y, z = rng.uniform(-40, 40, n), rng.uniform(-40, 40, n), rng.uniform(-300, 700, n)
    src, dst = rng.integers(0, n, ne), rng.integers(0, n, ne)
    base = oracle.in_logits(m, x, y, z, src, dst)
    pn, pe = rng.permutation(n), rng.permutation(ne)
    inv = np.argsort(pn)
    got = oracle.in_logits(m, x[pn], y[pn], z[pn], inv[src][pe], inv[dst][pe])
    assert np.allclose(got, base[pe], rtol=1e-11, atol=1e-11)
    # and the direction matters: reversing every edge changes the logits
    rev = oracle.in_logits(m, x, y, z, dst, src)
    assert not np.allclose(rev, base)


# ----------------------------------------------------------------------------
# connected components
# ----------------------------------------------------------------------------
def closure_labels(n, pairs):
    R = np.eye(n, dtype=bool)
    for a, b in pairs:
        R[a, b] = R[b, a] = True
    for k in range(n):
        R |= R[:, k:k + 1] & R[k:k + 1, :]
    return np.array([int(np.nonzero(R[i])[0].min()) for i in range(n)])


def test_components_exhaustive_small_graphs():
    n = 5
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        chosen = [p for b, p in enumerate(pairs) if mask >> b & 1]
        # alternate the direction: components are weak (undirected)
        src = [a if i % 2 else b for i, (a, b) in enumerate(chosen)]
        dst = [b if i % 2 else a for i, (a, b) in enumerate(chosen)]
        got = oracle.components(n, src, dst)
        assert np.array_equal(got, closure_labels(n, chosen)), chosen


def test_components_hand_built_tracks_and_keep_mask():
    # three tracks 0-3-6-9, 1-4-7, 2-5-8 plus singleton 10; the edge 9->10 is
    # not kept and the edge 6->7 is not kept
    src = [0, 3, 6, 1, 4, 2, 5, 9, 6]
    dst = [3, 6, 9, 4, 7, 5, 8, 10, 7]
    keep = [1, 1, 1, 1, 1, 1, 1, 0, 0]
    got = oracle.components(11, src, dst, keep)
    assert list(got) == [0, 1, 2, 0, 1, 2, 0, 1, 2, 0, 10]


def test_components_invariants_random():
    rng = np.random.default_rng(5)
    n = 200
    src, dst = rng.integers(0, n, 150), rng.integers(0, n, 150)
    keep = rng.integers(0, 2, 150)
    lab = oracle.components(n, src, dst, keep)
    assert np.all(lab <= np.arange(n))
    assert np.array_equal(lab[lab], lab)
    k = keep.astype(bool)
    assert np.array_equal(lab[src[k]], lab[dst[k]])


# ----------------------------------------------------------------------------
# whole pipeline glue and metrics
# ----------------------------------------------------------------------------
def test_pipeline_is_composition_of_steps():
    wl = synth.workload("cfg1_plain_fp32")
    sh = synth.shape_of(wl)
    m = oracle.Model(synth.workload_weights(wl), sh.embed, sh.hidden, sh.iters)
    ev = synth.workload_batch(wl, 1, first_event=3).event(0)
    r = oracle.find_tracks_event(m, ev.x, ev.y, ev.z, ev.plane, wl["radius2"], wl["k_max"])
    emb = oracle.embed(m, ev.x, ev.y, ev.z)
    s, d, d2 = oracle.radius_graph(ev.plane, emb, wl["radius2"], wl["k_max"])
    assert np.array_equal(s, r.src) and np.array_equal(d, r.dst)
    lg = oracle.in_logits(m, ev.x, ev.y, ev.z, s, d)
    assert np.array_equal(lg, r.logit)
    keep = (lg >= 0).astype(np.uint8)
    assert np.array_equal(keep, r.keep)
    assert np.array_equal(oracle.components(ev.n_hits, s, d, keep), r.labels)
    # the workload's calibrated radius gives about the stated mean degree
    deg = 2 * len(s) / ev.n_hits
    assert 6 < deg < 24


def test_pipeline_hand_built_event():
    """The whole pipeline on the hand-built event of
    tests/golden/pipeline_hand.json: identity embedding, rough graph over
    planes p+1 and p+2, constant logit 0.5, the score cut, components. Edge
    set, logits, decisions and candidates are those worked out by hand."""
    from parity import hand_pipeline, hand_pipeline_blob, hand_pipeline_labels
    g, x, y, z, plane, idx = hand_pipeline()
    m = oracle.Model(hand_pipeline_blob(8, 2, g["classifier_bias"]), [3, 4, 4], 8, 2)
    want_edges = {(idx[a], idx[b]) for a, b in g["edges"]}
    for cut, keep_all in ((g["cut_keep_all"], True), (g["cut_keep_none"], False)):
        r = oracle.find_tracks_event(m, x, y, z, plane, g["r2"], g["k_max"], cut=cut)
        assert edge_set(r.src, r.dst) == want_edges
        assert np.all(r.logit == g["classifier_bias"])
        assert np.all(r.keep == (1 if keep_all else 0))
        assert np.array_equal(r.labels, hand_pipeline_labels(g, idx, keep_all))


def test_batch_matches_events_and_threads():
    wl = synth.workload("cfg1_plain_fp32")
    sh = synth.shape_of(wl)
    m = oracle.Model(synth.workload_weights(wl), sh.embed, sh.hidden, sh.iters)
    b = synth.workload_batch(wl, 4)
    l1, ne1 = oracle.find_tracks_batch(m, b.x, b.y, b.z, b.plane, b.offsets,
                                       wl["radius2"], wl["k_max"], threads=1)
    l3, ne3 = oracle.find_tracks_batch(m, b.x, b.y, b.z, b.plane, b.offsets,
                                       wl["radius2"], wl["k_max"], threads=3)
    assert np.array_equal(l1, l3) and ne1 == ne3
    ev = b.event(2)
    r = oracle.find_tracks_event(m, ev.x, ev.y, ev.z, ev.plane, wl["radius2"], wl["k_max"])
    a = int(b.offsets[2])
    assert np.array_equal(l1[a:a + ev.n_hits], r.labels)


def test_metrics_hand_worked():
    g = gold("metrics_hand.json")
    c = metrics.event_counts(g["labels"], g["pid"])
    got = c.summary()
    for k, v in g["expected"].items():
        assert got[k] == pytest.approx(v), k


def test_metrics_shared_hits_and_overlapping_tracks():
    g = gold("metrics_shared_hand.json")
    got = metrics.track_counts(g["tracks"], g["pid"], g["pid2"]).summary()
    for k, v in g["expected"].items():
        assert got[k] == pytest.approx(v, abs=1e-12), k
    # the per-event wrapper over a batch of two copies gives the same ratios
    n = len(g["pid"])
    tot = metrics.batch_track_counts([g["tracks"], g["tracks"]], g["pid"] * 2, [0, n, 2 * n],
                                     pid2=g["pid2"] * 2).summary()
    for k in ("efficiency", "ghost_rate", "clone_rate", "hit_purity", "hit_efficiency"):
        assert tot[k] == pytest.approx(g["expected"][k], abs=1e-12), k


def test_metrics_perfect_tracks():
    # labels equal to the truth: efficiency 1, no ghosts, no clones
    pid = [0, 0, 0, 1, 1, 1, 1, 2, 2, -1]
    labels = [0, 0, 0, 3, 3, 3, 3, 7, 7, 9]
    s = metrics.event_counts(labels, pid).summary()
    assert s["efficiency"] == 1.0 and s["ghost_rate"] == 0.0 and s["clone_rate"] == 0.0
    assert s["reconstructible"] == 2 and s["tracks"] == 2


def test_weight_blob_rejects_wrong_architecture():
    wl = synth.workload("cfg1_plain_fp32")
    blob = synth.workload_weights(wl)
    with pytest.raises(ValueError):
        oracle.Model(blob, [3, 64, 64, 4], 32, 3)
    with pytest.raises(ValueError):
        oracle.Model(blob[:-4], [3, 64, 64, 4], 32, 4)


# ---------------------------------------------------------------------------
# quantisation (oracle/quant.py)
# ---------------------------------------------------------------------------
def test_symmetric_quantisation_worked_example():
    """The thesis's symmetric example: inputs within [-10.8, 10.8] onto INT8
    with the bound mapped to 127 give S = 10.8 / 127; the bound quantises to
    +-127, values beyond are clipped, and x = S x_q inverts the grid points."""
    from oracle import quant
    S = quant.symmetric_scale(10.8, 127)
    assert S == pytest.approx(10.8 / 127, rel=1e-15)
    aq = int(round(10.8 / S))
    assert aq == 127
    xq = quant.quantize([10.8, -10.8, 0.0, 20.0, -50.0, S * 3.4, S * 3.6], S, aq)
    assert list(xq) == [127, -127, 0, 127, -127, 3, 4]
    assert quant.dequantize(xq[:2], S) == pytest.approx([10.8, -10.8], rel=1e-12)


def test_e4m3_codes_closed_forms():
    """Landmark codes of E4M3: 0, the smallest subnormal 2^-9, the largest
    subnormal 7 * 2^-9, the smallest normal 2^-6, one, the largest finite 448,
    NaN at 0x7F / 0xFF, and sign symmetry for every code."""
    from oracle import quant
    d = quant.e4m3_decode
    assert d(0x00) == 0.0 and d(0x01) == 2.0 ** -9 and d(0x07) == 7 * 2.0 ** -9
    assert d(0x08) == 2.0 ** -6 and d(0x38) == 1.0 and d(0x7E) == 448.0
    assert math.isnan(d(0x7F)) and math.isnan(d(0xFF))
    for c in range(0x7F):
        assert d(c | 0x80) == -d(c)
    finite = sorted(d(c) for c in range(0x7F))
    assert len(set(finite)) == 127 and finite == sorted(set(finite))  # strictly increasing


def test_e4m3_round_trip_and_rounding():
    """encode(decode(c)) == c for all 254 finite codes (+-0 keep their sign);
    midpoints round to the even mantissa; beyond 448 saturates; NaN -> 0x7F."""
    from oracle import quant
    for c in range(256):
        v = quant.e4m3_decode(c)
        if math.isnan(v):
            continue
        assert quant.e4m3_encode(v) == c, hex(c)
    # 1.0 (m=0) and 1.125 (m=1): the midpoint goes to the even mantissa, 1.0
    assert quant.e4m3_encode(1.0625) == 0x38
    # 1.125 (m=1) and 1.25 (m=2): midpoint 1.1875 -> 1.25
    assert quant.e4m3_encode(1.1875) == 0x3A
    # largest subnormal / smallest normal midpoint -> the normal (even mantissa 0)
    assert quant.e4m3_encode(7.5 * 2.0 ** -9) == 0x08
    assert quant.e4m3_encode(1e6) == 0x7E and quant.e4m3_encode(-449.0) == 0xFE
    assert quant.e4m3_encode(float("nan")) == 0x7F
    # a planted mistake: round half away from zero would give 1.125 here
    assert quant.e4m3_decode(quant.e4m3_encode(1.0625)) == 1.0


# ---------------------------------------------------------------------------
# INT8 embedding (the thesis's post-training quantisation)
# ---------------------------------------------------------------------------
def test_int8_layer_exact_on_representable_values():
    """Inputs that are multiples of S_a and weights that are multiples of their
    row's S_w quantise without error, so the INT8 layer equals the float
    product: a dropped or swapped scale, or a transposed weight, fails."""
    from oracle import quant
    rng = np.random.default_rng(3)
    alpha = 2.54
    sa = np.float32(alpha) / np.float32(127)
    xq = rng.integers(-127, 128, (20, 12))
    W = np.zeros((5, 12), np.float32)
    sw = np.float32([0.01, 0.02, 0.05, 0.1, 0.5]) / np.float32(127)
    Wq = rng.integers(-126, 127, (5, 12))
    Wq[:, 0] = 127  # the row maximum fixes S_w exactly
    W[:] = (Wq * sw[:, None]).astype(np.float32)
    b = rng.normal(size=5).astype(np.float32)
    x = (xq * np.float64(sa)).astype(np.float32)
    codes = quant.int8_codes(x, np.float32(127) / np.float32(alpha))
    assert np.array_equal(codes, xq)
    y = quant.int8_layer(codes, alpha, W, b)
    want = x.astype(np.float64) @ W.T.astype(np.float64) + b
    assert np.allclose(y, want, rtol=1e-6, atol=1e-6)
    # saturation: inputs beyond alpha clip to +-127
    assert list(quant.int8_codes([10.0, -10.0], np.float32(127) / np.float32(alpha))) == [127, -127]
    # ties round half to even (reading Q1, the rounding of the device's
    # float-to-int conversion): 0.5, 1.5, 2.5, 3.5 -> 0, 2, 2, 4 and the negatives
    ties = [0.5, 1.5, 2.5, 3.5, -0.5, -1.5, -2.5, -3.5]
    assert list(quant.int8_codes(ties, 1.0)) == [0, 2, 2, 4, 0, -2, -2, -4]


def test_int8_embedding_converges_to_float_with_range():
    """With a calibrated range the INT8 embedding stays within a few code steps
    of the float64 one; with a range 100x too wide it is far coarser (the
    thesis's uncalibrated case)."""
    from oracle import quant
    wl = synth.workload("cfg3_trained_bf16")
    arrs = synth.weight_arrays(synth.workload_weights(wl))
    n_emb = len(wl["model"]["embed"]) - 1
    layers = arrs[:n_emb]
    ev = synth.workload_batch(wl, 1)
    r = np.hypot(ev.x.astype(np.float64), ev.y)
    feats = np.stack([r / 45.0, np.arctan2(ev.y.astype(np.float64), ev.x) / np.pi, ev.z / 750.0],
                     1).astype(np.float32)
    ref = feats.astype(np.float64)
    for l, (W, b) in enumerate(layers):
        ref = ref @ W.T.astype(np.float64) + b
        if l + 1 < n_emb:
            ref = np.maximum(ref, 0)
    amax = quant.embed_amax(layers, feats)
    cal = quant.int8_embed(layers, amax, feats)
    wide = quant.int8_embed(layers, [100 * a for a in amax], feats)
    e_cal = np.abs(cal - ref).max()
    e_wide = np.abs(wide - ref).max()
    assert e_cal < 0.05 * np.abs(ref).max(), e_cal
    assert e_wide > 5 * e_cal, (e_wide, e_cal)


@pytest.mark.parametrize("name", ["cfg1_plain_fp32", "cfg2_run3_single", "cfg3_batched_bf16",
                                  "cfg4_batched_fp8", "cfg5_serving"])
def test_stored_radii_come_from_the_calibration(name):
    """Every stored squared radius of a seeded-weight workload is what
    oracle/calibrate.py computes from the workload's calibration events (its
    own seed): exactly E = round(degree x N / 2) candidate pairs pass."""
    from oracle import calibrate
    wl = synth.workload(name)
    assert calibrate.calibrate(name, wl) == wl["radius2"]
