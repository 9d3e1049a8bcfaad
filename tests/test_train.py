"""The offline training tool and the trained weights shipped with the package.

CPU only: a short training run must produce a model that finds tracks (the
oracle scores it on held-out events), and the shipped blob must be a
physics-meaningful config-1 model at the radius the workload states."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import metrics
from paper_2508_07423_gb300 import synth

torch = pytest.importorskip("torch")
train = pytest.importorskip("paper_2508_07423_gb300.train")


def efficiency(blob, shape, r2, batch, cut=0.5):
    m = oracle.Model(blob, shape.embed, shape.hidden, shape.iters)
    lab, _ = oracle.find_tracks_batch(m, batch.x, batch.y, batch.z, batch.plane, batch.offsets,
                                      r2, 64, cut, threads=4)
    return metrics.batch_counts(lab, batch.pid, batch.offsets).summary()


def test_focal_loss_closed_forms():
    """alpha-balanced focal loss (Lin et al.): gamma = 0 gives alpha-weighted
    cross entropy; a confident correct prediction costs ~0; p = 1/2 gives
    w (1/2)^gamma ln 2."""
    lg = torch.tensor([0.0, 0.0, 3.0, -2.0], dtype=torch.float64)
    y = torch.tensor([1.0, 0.0, 1.0, 0.0], dtype=torch.float64)
    ce = [math.log(2), math.log(2), math.log(1 + math.exp(-3)), math.log(1 + math.exp(-2))]
    w = [0.25, 0.75, 0.25, 0.75]
    g0 = train.focal_loss(lg, y, alpha=0.25, gamma=0.0).item()
    assert abs(g0 - np.mean([a * b for a, b in zip(w, ce)])) < 1e-12
    p = [0.5, 0.5, 1 / (1 + math.exp(-3)), 1 / (1 + math.exp(2))]
    pt = [p[0], 1 - p[1], p[2], 1 - p[3]]
    g2 = train.focal_loss(lg, y).item()
    ref = np.mean([wi * (1 - t) ** 2 * c for wi, t, c in zip(w, pt, ce)])
    assert abs(g2 - ref) < 1e-12
    assert train.focal_loss(torch.tensor([30.0]), torch.tensor([1.0])).item() < 1e-12


def test_gnn_forward_matches_oracle_logits():
    """The training model's forward pass is the library's architecture: its
    logits on a hand-made graph equal the oracle's FP64 logits for the same
    blob."""
    shape = synth.ModelShape([3, 16, 4], 8, 2)
    m = train.build(shape, 3, "cpu").double()
    blob = train.to_blob(m)
    ev = synth.gen_batch(1, 11, {"kind": "fixed", "n": 6}, 0.0)
    n = ev.n_hits
    rng = np.random.default_rng(0)
    src = rng.integers(0, n, 40).astype(np.int32)
    dst = rng.integers(0, n, 40).astype(np.int32)
    fs = oracle.DEFAULT_FEAT_SCALE
    om = oracle.Model(blob, shape.embed, shape.hidden, shape.iters)
    ref = oracle.in_logits(om, ev.x, ev.y, ev.z, src, dst, feat_scale=fs)
    xyz = [np.asarray(v, np.float64) for v in (ev.x, ev.y, ev.z)]
    node_in = np.stack([xyz[0] / fs[3], xyz[1] / fs[4], xyz[2] / fs[5]], 1)
    # the blob stores float32: compare against a float32-rounded copy
    m32 = train.build(shape, 3, "cpu").double()
    for (p32, p) in zip(m32.parameters(), m.parameters()):
        p32.data.copy_(p.data.float().double())
    got = train.gnn_forward(m32, torch.from_numpy(node_in),
                            torch.from_numpy(src.astype(np.int64)),
                            torch.from_numpy(dst.astype(np.int64))).detach().numpy()
    assert np.max(np.abs(got - ref)) < 1e-9 * max(1.0, np.max(np.abs(ref)))


def test_short_training_finds_tracks():
    shape = synth.ModelShape([3, 32, 32, 4], 16, 2)
    tracks = {"kind": "fixed", "n": 30}
    blob, r2 = train.train(shape, tracks, 0.05, 24, 77, device="cpu", emb_epochs=6, gnn_epochs=10)
    held = synth.gen_batch(4, 78, tracks, 0.05)
    s = efficiency(blob, shape, r2, held)
    rnd = efficiency(synth.make_weights(shape, 5), shape, r2, held)
    assert s["efficiency"] > 0.6 and s["efficiency"] > rnd["efficiency"] + 0.4, (s, rnd)


@pytest.mark.parametrize("name,min_eff,max_ghost", [("cfg3_trained_bf16", 0.95, 0.03),
                                                    ("cfg4_trained_fp8", 0.88, 0.06)])
def test_shipped_trained_model(name, min_eff, max_ghost):
    wl = synth.workload(name)
    sh = synth.shape_of(wl)
    blob = synth.workload_weights(wl)
    dims = [(W.shape[1], W.shape[0]) for W, _ in synth.weight_arrays(blob)]
    assert dims == [tuple(d) for d in sh.layers]
    meta_path = os.path.join(os.path.dirname(synth.__file__), wl["weights_file"][:-4] + ".json")
    with open(meta_path) as f:
        meta = json.load(f)
    assert meta["radius2"] == wl["radius2"]
    assert meta["train_seed"] != wl["seeds"]["events"]  # trained on other events
    b = synth.workload_batch(wl, 3)
    s = efficiency(blob, sh, wl["radius2"], b)
    assert s["efficiency"] >= min_eff and s["ghost_rate"] <= max_ghost, s


def test_triplet_heads_and_joint_training_produce_a_loadable_blob():
    """Triplet-head training and the joint edge + triplet fine-tuning run on a
    few events with close pairs, and the blob carries both classifiers the
    oracle's triplet stage reads."""
    shape = synth.ModelShape([3, 16, 4], 16, 1)
    tracks = {"kind": "fixed", "n": 20}
    blob, r2 = train.train(shape, tracks, 0.05, 6, 31, device="cpu", emb_epochs=2, gnn_epochs=2,
                           pair_frac=0.2, triplet_epochs=1, joint_epochs=1)
    assert len(synth.weight_arrays(blob)) == len(shape.layers) + 4
    m = oracle.Model(blob, shape.embed, shape.hidden, shape.iters)
    ev = synth.gen_batch(1, 32, tracks, 0.05, pair_frac=0.2)
    r = oracle.find_tracks_triplets_event(m, ev.x, ev.y, ev.z, ev.plane, r2, 64)
    assert len(r.tlogit) == len(r.ttype) and np.all(np.isfinite(r.tlogit))


def test_training_is_deterministic():
    """Same seed and settings: byte-identical weights and the same radius."""
    shape = synth.ModelShape([3, 16, 16, 4], 8, 1)
    tracks = {"kind": "fixed", "n": 20}
    runs = [train.train(shape, tracks, 0.05, 6, 41, device="cpu", emb_epochs=2, gnn_epochs=2)
            for _ in range(2)]
    assert runs[0][0] == runs[1][0]
    assert runs[0][1] == runs[1][1]


@pytest.mark.parametrize("name", ["cfg3_trained_bf16", "cfg4_trained_fp8"])
def test_shipped_radius_is_the_genuine_pair_quantile(name):
    """The trained blob's stored squared radius is the 99.5 % quantile of the
    squared embedding distances of genuine pairs (same particle, next two
    planes, particles of at least 3 hits) over its training events (reading
    R19), recomputed here with the FP64 oracle embedding."""
    wl = synth.workload(name)
    meta_path = os.path.join(os.path.dirname(synth.__file__), wl["weights_file"][:-4] + ".json")
    with open(meta_path) as f:
        meta = json.load(f)
    sh = synth.shape_of(wl)
    m = oracle.Model(synth.workload_weights(wl), sh.embed, sh.hidden, sh.iters)
    b = synth.gen_batch(meta["train_events"], meta["train_seed"], meta["tracks"], meta["noise"])
    ds = []
    for e in range(b.n_events):
        ev = b.event(e)
        keep = ev.pid >= 0
        keep &= np.bincount(ev.pid[keep])[np.maximum(ev.pid, 0)] >= 3
        idx = np.flatnonzero(keep)
        emb = oracle.embed(m, ev.x[idx], ev.y[idx], ev.z[idx])
        pl, pid = ev.plane[idx].astype(int), ev.pid[idx]
        dp = pl[None, :] - pl[:, None]
        q, a = np.nonzero(((dp == 1) | (dp == 2)) & (pid[:, None] == pid[None, :]))
        ds.append(((emb[q] - emb[a]) ** 2).sum(1))
    r2 = np.quantile(np.concatenate(ds), meta["radius_quantile_of_genuine_pairs"])
    assert r2 == pytest.approx(meta["radius2"], rel=1e-4)
    assert meta["radius2"] == wl["radius2"]
