"""Comparison helpers for the GPU-vs-oracle parity tests (test support only)."""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

import oracle

# parity tolerances: scores within 1e-4 absolute; edge sets identical except
# pairs whose embedding distance lies within 1e-5 relative of the radius (or of
# the k_max-th distance of a capped row)
SCORE_TOL = 1e-4
DIST_REL = 1e-5


def sigmoid(v):
    return 1.0 / (1.0 + np.exp(-np.asarray(v, np.float64)))


def cc_labels(n, src, dst, keep):
    """Smallest member index of each hit's component (scipy, not the oracle)."""
    k = np.asarray(keep).astype(bool)
    A = sp.coo_matrix((np.ones(int(k.sum())), (np.asarray(src)[k], np.asarray(dst)[k])),
                      shape=(n, n))
    _, comp = connected_components(A, directed=True, connection="weak")
    mins = np.full(comp.max() + 1 if n else 0, n, dtype=np.int64)
    np.minimum.at(mins, comp, np.arange(n))
    return mins[comp].astype(np.int32)


def hops_from(n, src, dst, seeds, hops):
    adj = [[] for _ in range(n)]
    for a, b in zip(src, dst):
        adj[a].append(b)
        adj[b].append(a)
    seen = set(seeds)
    front = list(seeds)
    for _ in range(hops):
        nxt = []
        for v in front:
            for w in adj[v]:
                if w not in seen:
                    seen.add(w)
                    nxt.append(w)
        front = nxt
    return seen


class EventReport:
    def __init__(self):
        self.edges = 0
        self.exempt_pairs = 0
        self.bad_pairs = []
        self.max_score_err = 0.0
        self.scores_compared = 0
        self.decision_mismatch = 0
        self.labels_compared = False
        self.labels_equal = None


def compare_event(ev, g, labels, model, r2, k_max, iters, cut=0.5, feat_scale=None,
                  ref=None):
    """Compare one event's GPU graph/labels with the oracle; returns EventReport.

    Raises AssertionError on any violation of the parity bar.
    """
    kw = {} if feat_scale is None else {"feat_scale": feat_scale}
    if ref is None:
        ref = oracle.find_tracks_event(model, ev.x, ev.y, ev.z, ev.plane, r2, k_max, cut, **kw)
    emb = oracle.embed(model, ev.x, ev.y, ev.z, **kw)
    n = ev.n_hits
    rep = EventReport()
    gsrc, gdst = g["src"].astype(np.int64), g["dst"].astype(np.int64)
    rep.edges = len(gsrc)
    G = {(int(a), int(b)): i for i, (a, b) in enumerate(zip(gsrc, gdst))}
    O = {(int(a), int(b)): i for i, (a, b) in enumerate(zip(ref.src, ref.dst))}
    r = math.sqrt(r2)
    row_n = np.bincount(ref.src, minlength=n) if len(ref.src) else np.zeros(n, int)
    kth = np.zeros(n)
    if len(ref.src):
        np.maximum.at(kth, ref.src, np.sqrt(ref.d2))
    diff = set(G) ^ set(O)
    for (i, j) in diff:
        d = float(np.sqrt(np.sum((emb[i] - emb[j]) ** 2)))
        if abs(d - r) / r <= DIST_REL:
            rep.exempt_pairs += 1
            continue
        if row_n[i] == k_max and kth[i] > 0 and abs(d - kth[i]) / kth[i] <= DIST_REL:
            rep.exempt_pairs += 1
            continue
        rep.bad_pairs.append((i, j, d))
    assert not rep.bad_pairs, f"edge sets differ beyond the boundary rule: {rep.bad_pairs[:5]}"
    # edges away from any difference: the GNN sees identical neighbourhoods
    if diff:
        touched = {v for e in diff for v in e}
        aff = hops_from(n, np.concatenate([gsrc, ref.src]), np.concatenate([gdst, ref.dst]),
                        touched, iters + 1)
    else:
        aff = set()
    common = [e for e in G if e in O and e[0] not in aff and e[1] not in aff]
    if common:
        gi = np.array([G[e] for e in common])
        oi = np.array([O[e] for e in common])
        err = np.abs(sigmoid(g["logit"][gi]) - sigmoid(ref.logit[oi]))
        rep.max_score_err = float(err.max())
        rep.scores_compared = len(common)
        assert rep.max_score_err <= SCORE_TOL, f"score error {rep.max_score_err}"
        cutl = math.log(cut / (1 - cut))
        clear = np.abs(ref.logit[oi] - cutl) > 4 * SCORE_TOL
        mism = (g["kept"][gi].astype(bool) != ref.keep[oi].astype(bool)) & clear
        rep.decision_mismatch = int(mism.sum())
        assert rep.decision_mismatch == 0, "keep decisions differ away from the cut"
    # labels are exactly the components of the GPU's own kept edges
    own = cc_labels(n, gsrc, gdst, g["kept"])
    assert np.array_equal(labels, own), "labels are not the components of the kept edges"
    # and equal the oracle's when the kept edge sets agree
    gk = {e for e, i in G.items() if g["kept"][i]}
    ok = {e for e, i in O.items() if ref.keep[i]}
    if gk == ok:
        rep.labels_compared = True
        rep.labels_equal = bool(np.array_equal(labels, ref.labels))
        assert rep.labels_equal, "labels differ from the oracle for the same kept edges"
    return rep


# ----------------------------------------------------------------------------
# the hand-built whole-pipeline event (tests/golden/pipeline_hand.json)
# ----------------------------------------------------------------------------
def hand_pipeline():
    """(fixture, x, y, z, plane, index of each hit name) of the hand-built event."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "pipeline_hand.json")) as f:
        g = json.load(f)
    z0, dz = g["z_of_plane_mm"]
    phi = np.array([h[1] for h in g["hits"]])
    r = np.array([h[2] for h in g["hits"]])
    plane = np.array([h[3] for h in g["hits"]], np.uint8)
    x = (r * np.cos(phi)).astype(np.float32)
    y = (r * np.sin(phi)).astype(np.float32)
    z = (z0 + dz * plane.astype(np.float64)).astype(np.float32)
    idx = {h[0]: i for i, h in enumerate(g["hits"])}
    return g, x, y, z, plane, idx


def hand_pipeline_blob(h: int, K: int, bias: float, seed: int = 0,
                       triplet_bias=None) -> bytes:
    """Weights of the hand-built event: identity embedding 3 -> 4 -> 4 (the
    features and a zero coordinate), a random interaction network of width h
    and K steps, and a classifier whose last layer is zero with bias `bias`.
    triplet_bias = (articulation, elbow): the two triplet classifiers appended,
    random first layers and zero last layers with these biases."""
    from paper_2508_07423_gb300 import synth
    rng = np.random.default_rng(seed)

    def rnd(o, i):
        b = math.sqrt(6.0 / i)
        return (rng.uniform(-b, b, (o, i)).astype(np.float32),
                rng.uniform(-0.3, 0.3, o).astype(np.float32))
    W1 = np.zeros((4, 3), np.float32)
    W1[:3, :3] = np.eye(3)
    layers = [(W1, np.zeros(4, np.float32)), (np.eye(4, dtype=np.float32), np.zeros(4, np.float32))]
    layers += [rnd(h, 3), rnd(h, h), rnd(h, 2 * h), rnd(h, h)]
    for _ in range(K):
        layers += [rnd(h, 3 * h), rnd(h, h), rnd(h, 3 * h), rnd(h, h)]
    layers += [rnd(h, h), (np.zeros((1, h), np.float32), np.array([bias], np.float32))]
    if triplet_bias is not None:
        for tb in triplet_bias:
            layers += [rnd(h, 2 * h), (np.zeros((1, h), np.float32), np.array([tb], np.float32))]
    return synth.pack_weights(layers)


def hand_pipeline_labels(g, idx, keep_all: bool) -> np.ndarray:
    """Expected canonical labels: the smallest input index of each hand-listed
    candidate (every hit alone when no edge is kept)."""
    n = len(idx)
    lab = np.arange(n, dtype=np.int32)
    if keep_all:
        for group in g["candidates_keep_all"]:
            ids = [idx[nm] for nm in group]
            lab[ids] = min(ids)
    return lab
