"""Offline training of track-finding weights on synthetic events.

An offline tool, outside the hot path: it produces a weight blob (the format
`gnntrk_create` and the oracle read) whose scores mean something, so that
track efficiency and the near-cut band fraction can be measured on a trained
model instead of seeded random weights. It uses PyTorch autograd (CUDA when
available) and is imported neither by the CUDA library's binding nor by the
oracle.

Training follows the thesis's description (Sec. "Hit Embedding and Rough
Graph Construction", Sec. "Graph Neural Network and Classifiers"):

* embedding MLP: per event, noise hits removed, query hits are hits of
  particles with at least 3 hits; the training pairs q -> a (a on the next two
  planes) are all genuine pairs (same particle), hard negatives (fake pairs
  among the k nearest candidates within a training radius in the current
  embedding) and one random pair per query; the loss is
  L = L_fake + w_genuine * L_genuine with L_genuine the mean squared distance
  of genuine pairs and L_fake the mean of max(0, m - d^2) over fake pairs
  (margin m = 1);
* interaction network (the library's architecture: every sub-network is
  Linear -> LayerNorm without affine -> ReLU -> Linear, residual node and edge
  updates, distinct weights per step): the rough graph of the trained
  embedding at the inference radius, edges labelled genuine when both hits
  belong to the same particle, trained with the sigmoid focal loss
  (alpha = 0.25, gamma = 2).

    python -m paper_2508_07423_gb300.train --out paper_2508_07423_gb300/trained/velo_h32k4.bin

(the defaults train the config-1 model, embed 3-64-64-4 and h 32, K 4, on
120 events of Poisson(150) tracks with 5% noise, on the CPU).
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import synth


def _torch():
    import torch
    return torch


# ----------------------------------------------------------------------------
# model (same layer order as synth.ModelShape)
# ----------------------------------------------------------------------------
def build(shape: synth.ModelShape, seed: int, device, triplets: bool = False):
    torch = _torch()
    nn = torch.nn
    gen = torch.Generator().manual_seed(seed)

    def lin(fi, fo):
        m = nn.Linear(fi, fo)
        bw, bb = math.sqrt(6.0 / fi), 1.0 / math.sqrt(fi)
        with torch.no_grad():
            m.weight.uniform_(-bw, bw, generator=gen)
            m.bias.uniform_(-bb, bb, generator=gen)
        return m

    h, K = shape.hidden, shape.iters
    e = shape.embed
    mods = {
        "embed": nn.ModuleList([lin(e[i], e[i + 1]) for i in range(len(e) - 1)]),
        "node_enc": nn.ModuleList([lin(3, h), lin(h, h)]),
        "edge_enc": nn.ModuleList([lin(2 * h, h), lin(h, h)]),
        "node": nn.ModuleList([nn.ModuleList([lin(3 * h, h), lin(h, h)]) for _ in range(K)]),
        "edge": nn.ModuleList([nn.ModuleList([lin(3 * h, h), lin(h, h)]) for _ in range(K)]),
        "cls": nn.ModuleList([lin(h, h), lin(h, 1)]),
    }
    if triplets:  # articulation and elbow classifiers on [e_first, e_second]
        mods["art"] = nn.ModuleList([lin(2 * h, h), lin(h, 1)])
        mods["elb"] = nn.ModuleList([lin(2 * h, h), lin(h, 1)])
    return nn.ModuleDict(mods).to(device)


def embed_forward(m, f):
    torch = _torch()
    x = f
    for i, l in enumerate(m["embed"]):
        x = l(x)
        if i + 1 < len(m["embed"]):
            x = torch.relu(x)
    return x


def _sub(pair, x):
    torch = _torch()
    y = pair[0](x)
    y = torch.nn.functional.layer_norm(y, (y.shape[-1],), eps=1e-5)
    return pair[1](torch.relu(y))


def gnn_forward(m, nf, src, dst, with_states: bool = False):
    """Logits of the edges src -> dst for node features nf [N, 3] (and the
    final edge encodings e^K with `with_states`)."""
    torch = _torch()
    h = _sub(m["node_enc"], nf)
    e = _sub(m["edge_enc"], torch.cat([h[src], h[dst]], 1))
    n = nf.shape[0]
    for k in range(len(m["node"])):
        mo = e.new_zeros(n, e.shape[1]).index_add(0, src, e)
        mi = e.new_zeros(n, e.shape[1]).index_add(0, dst, e)
        h = h + _sub(m["node"][k], torch.cat([h, mo, mi], 1))
        e = e + _sub(m["edge"][k], torch.cat([e, h[src], h[dst]], 1))
    logit = _sub(m["cls"], e).squeeze(1)
    return (logit, e) if with_states else logit


def to_blob(m) -> bytes:
    arrays = []
    for group in ("embed", "node_enc", "edge_enc"):
        for l in m[group]:
            arrays.append((l.weight.detach().cpu().numpy(), l.bias.detach().cpu().numpy()))
    for k in range(len(m["node"])):
        for group in ("node", "edge"):
            for l in m[group][k]:
                arrays.append((l.weight.detach().cpu().numpy(), l.bias.detach().cpu().numpy()))
    for g in ("cls", "art", "elb"):
        if g in m:
            for l in m[g]:
                arrays.append((l.weight.detach().cpu().numpy(), l.bias.detach().cpu().numpy()))
    return synth.pack_weights(arrays)


# ----------------------------------------------------------------------------
# per-event training data
# ----------------------------------------------------------------------------
def _features(ev, fs):
    r = np.hypot(ev.x, ev.y)
    emb_in = np.stack([r / fs[0], np.arctan2(ev.y, ev.x) / fs[1], ev.z / fs[2]], 1)
    node_in = np.stack([ev.x / fs[3], ev.y / fs[4], ev.z / fs[5]], 1)
    return emb_in.astype(np.float32), node_in.astype(np.float32)


def _candidate_pairs(plane):
    """All (q, a) with plane[a] - plane[q] in {1, 2}."""
    order = np.argsort(plane, kind="stable")
    ps = plane[order]
    starts = np.searchsorted(ps, np.arange(int(ps.max()) + 3 if len(ps) else 3))
    qs, as_ = [], []
    for p in range(int(ps.max()) + 1 if len(ps) else 0):
        q = order[starts[p]:starts[p + 1]]
        a = order[starts[min(p + 1, len(starts) - 1)]:starts[min(p + 3, len(starts) - 1)]]
        if len(q) and len(a):
            qq, aa = np.meshgrid(q, a, indexing="ij")
            qs.append(qq.ravel())
            as_.append(aa.ravel())
    if not qs:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(qs), np.concatenate(as_)


def _signal_only(ev):
    keep = ev.pid >= 0
    counts = np.bincount(ev.pid[keep], minlength=1) if keep.any() else np.zeros(1, int)
    keep &= counts[np.maximum(ev.pid, 0)] >= 3
    idx = np.flatnonzero(keep)
    return idx


def _same_particle(ev, i, j):
    """Hits i and j (arrays) share a particle (a shared hit belongs to both
    of its particles); noise shares none."""
    p1, p2 = ev.pid, ev.pid2 if ev.pid2 is not None else np.full(len(ev.pid), -1)
    a1, a2, b1, b2 = p1[i], p2[i], p1[j], p2[j]
    return (((a1 == b1) & (a1 >= 0)) | ((a1 == b2) & (a1 >= 0)) |
            ((a2 == b1) & (a2 >= 0)) | ((a2 == b2) & (a2 >= 0)))


def triplets_of(plane, src, dst, kept):
    """Triplets of the kept edges (indices `kept`): (type, e1, e2) with type 0
    articulation (A->C, C->B), 1 left elbow (C->A, C->B), 2 right elbow
    (A->C, B->C); elbow edges ordered by the (plane, index) of the far hit."""
    n = len(plane)
    ins = [[] for _ in range(n)]
    outs = [[] for _ in range(n)]
    for e in kept:
        outs[src[e]].append(e)
        ins[dst[e]].append(e)
    key = lambda v: (int(plane[v]), int(v))
    T = []
    for c in range(n):
        I = sorted(ins[c], key=lambda e: key(src[e]))
        O = sorted(outs[c], key=lambda e: key(dst[e]))
        T += [(0, a, b) for a in I for b in O]
        T += [(1, O[i], O[j]) for i in range(len(O)) for j in range(i + 1, len(O))]
        T += [(2, I[i], I[j]) for i in range(len(I)) for j in range(i + 1, len(I))]
    return np.array(T, np.int64).reshape(-1, 3)


def triplet_labels(ev, src, dst, T):
    """A triplet is genuine when one particle left all three of its hits."""
    ty, a, b = T[:, 0], T[:, 1], T[:, 2]
    hits = np.where(ty[:, None] == 0, np.stack([src[a], dst[a], dst[b]], 1),
                    np.where(ty[:, None] == 1, np.stack([src[a], dst[a], dst[b]], 1),
                             np.stack([dst[a], src[a], src[b]], 1)))
    p1 = ev.pid
    p2 = ev.pid2 if ev.pid2 is not None else np.full(len(p1), -1)
    lab = np.zeros(len(T), bool)
    for cand in (p1[hits[:, 0]], p2[hits[:, 0]]):  # the first hit's particles
        ok = cand >= 0
        for k in (1, 2):
            ok &= (p1[hits[:, k]] == cand) | (p2[hits[:, k]] == cand)
        lab |= ok
    return lab


# ----------------------------------------------------------------------------
# training
# ----------------------------------------------------------------------------
def train_embedding(m, events, fs, device, epochs=6, lr=2e-3, w_genuine=3.0, margin=1.0,
                    hard_r2=1.5, hard_k=50, seed=0):
    torch = _torch()
    rng = np.random.default_rng(seed)
    params = [p for l in m["embed"] for p in l.parameters()]
    opt = torch.optim.Adam(params, lr=lr)
    data = []
    for ev in events:
        idx = _signal_only(ev)
        emb_in, _ = _features(ev, fs)
        q, a = _candidate_pairs(ev.plane[idx])
        q, a = idx[q], idx[a]
        genuine = _same_particle(ev, q, a)
        data.append((torch.from_numpy(emb_in).to(device), q, a, genuine))
    for ep in range(epochs):
        tot = 0.0
        for ei in rng.permutation(len(data)):
            f, q, a, gen = data[ei]
            with torch.no_grad():
                z = embed_forward(m, f)
                d2 = ((z[torch.from_numpy(q).to(device)] - z[torch.from_numpy(a).to(device)]) ** 2).sum(1)
                d2 = d2.cpu().numpy()
            # hard negatives: fake pairs within the training radius, the k
            # nearest per query; plus one random fake candidate per query
            fake = ~gen & (d2 < hard_r2)
            order = np.lexsort((d2, q))
            rank = np.zeros(len(q), np.int64)
            qs = q[order]
            first = np.r_[0, np.flatnonzero(np.diff(qs)) + 1]
            run = np.arange(len(qs)) - np.repeat(first, np.diff(np.r_[first, len(qs)]))
            rank[order] = run
            hard = fake & (rank < hard_k)
            rnd = np.zeros(len(q), bool)
            cand_fake = np.flatnonzero(~gen)
            if len(cand_fake):
                # one random fake pair per query among its fake candidates
                perm = rng.permutation(cand_fake)
                _, pick = np.unique(q[perm], return_index=True)
                rnd[perm[pick]] = True
            sel_g = np.flatnonzero(gen)
            sel_f = np.flatnonzero(hard | rnd)
            if len(sel_g) == 0 or len(sel_f) == 0:
                continue
            z = embed_forward(m, f)
            qg, ag = torch.from_numpy(q[sel_g]).to(device), torch.from_numpy(a[sel_g]).to(device)
            qf, af = torch.from_numpy(q[sel_f]).to(device), torch.from_numpy(a[sel_f]).to(device)
            lg = ((z[qg] - z[ag]) ** 2).sum(1).mean()
            lf = torch.relu(margin - ((z[qf] - z[af]) ** 2).sum(1)).mean()
            loss = lf + w_genuine * lg
            opt.zero_grad()
            loss.backward()
            opt.step()
            tot += float(loss.detach())
        print(json.dumps({"stage": "embedding", "epoch": ep, "loss": round(tot / max(len(data), 1), 5)}),
              flush=True)


def embedding_radius(m, events, fs, device, keep=0.995):
    """Inference radius: the squared distance below which `keep` of the
    genuine pairs (same particle, next two planes) fall."""
    torch = _torch()
    ds = []
    with torch.no_grad():
        for ev in events:
            idx = _signal_only(ev)
            emb_in, _ = _features(ev, fs)
            q, a = _candidate_pairs(ev.plane[idx])
            q, a = idx[q], idx[a]
            g = _same_particle(ev, q, a)
            z = embed_forward(m, torch.from_numpy(emb_in).to(device))
            d2 = ((z[torch.from_numpy(q[g]).to(device)] - z[torch.from_numpy(a[g]).to(device)]) ** 2).sum(1)
            ds.append(d2.cpu().numpy())
    return float(np.float32(np.quantile(np.concatenate(ds), keep)))


def graph(m, ev, fs, r2, k_max, device):
    """Rough graph of one event (all hits) with the embedding: i -> j on the
    next two planes with d^2 < r2, at most k_max nearest per i."""
    torch = _torch()
    emb_in, node_in = _features(ev, fs)
    with torch.no_grad():
        z = embed_forward(m, torch.from_numpy(emb_in).to(device)).cpu().numpy().astype(np.float64)
    q, a = _candidate_pairs(ev.plane)
    d2 = ((z[q] - z[a]) ** 2).sum(1)
    ok = d2 < r2
    q, a, d2 = q[ok], a[ok], d2[ok]
    order = np.lexsort((a, d2, q))
    q, a = q[order], a[order]
    first = np.r_[0, np.flatnonzero(np.diff(q)) + 1] if len(q) else np.zeros(0, int)
    run = np.arange(len(q)) - np.repeat(first, np.diff(np.r_[first, len(q)])) if len(q) else q
    keep = run < k_max
    return q[keep], a[keep], node_in


def focal_loss(logit, y, alpha=0.25, gamma=2.0):
    torch = _torch()
    p = torch.sigmoid(logit)
    ce = torch.nn.functional.binary_cross_entropy_with_logits(logit, y, reduction="none")
    pt = p * y + (1 - p) * (1 - y)
    w = alpha * y + (1 - alpha) * (1 - y)
    return (w * (1 - pt) ** gamma * ce).mean()


def train_gnn(m, events, fs, r2, k_max, device, epochs=8, lr=2e-3, seed=0):
    torch = _torch()
    rng = np.random.default_rng(seed)
    params = [p for g in ("node_enc", "edge_enc", "node", "edge", "cls") for p in m[g].parameters()]
    opt = torch.optim.Adam(params, lr=lr)
    data = []
    for ev in events:
        src, dst, node_in = graph(m, ev, fs, r2, k_max, device)
        y = _same_particle(ev, src, dst).astype(np.float32)
        data.append((torch.from_numpy(node_in).to(device), torch.from_numpy(src).to(device),
                     torch.from_numpy(dst).to(device), torch.from_numpy(y).to(device)))
    for ep in range(epochs):
        tot = 0.0
        for ei in rng.permutation(len(data)):
            nf, s, d, y = data[ei]
            if len(s) == 0:
                continue
            loss = focal_loss(gnn_forward(m, nf, s, d), y)
            opt.zero_grad()
            loss.backward()
            opt.step()
            tot += float(loss.detach())
        print(json.dumps({"stage": "gnn", "epoch": ep, "loss": round(tot / max(len(data), 1), 6)}),
              flush=True)


def train_triplets(m, events, fs, r2, k_max, device, epochs=10, lr=2e-3, seed=0):
    """The two triplet classifiers on the final edge encodings of the trained
    (frozen) GNN, over the triplets of the edges it keeps (score >= 0.5)."""
    torch = _torch()
    rng = np.random.default_rng(seed)
    opt = torch.optim.Adam([p for g in ("art", "elb") for p in m[g].parameters()], lr=lr)
    data = []
    for ev in events:
        src, dst, node_in = graph(m, ev, fs, r2, k_max, device)
        if len(src) == 0:
            continue
        with torch.no_grad():
            logit, e = gnn_forward(m, torch.from_numpy(node_in).to(device),
                                   torch.from_numpy(src).to(device),
                                   torch.from_numpy(dst).to(device), with_states=True)
        kept = np.flatnonzero(logit.cpu().numpy() >= 0.0)
        T = triplets_of(ev.plane, src, dst, kept)
        if len(T) == 0:
            continue
        y = triplet_labels(ev, src, dst, T).astype(np.float32)
        data.append((e, torch.from_numpy(T).to(device), torch.from_numpy(y).to(device)))
    for ep in range(epochs):
        tot = 0.0
        for ei in rng.permutation(len(data)):
            e, T, y = data[ei]
            x = torch.cat([e[T[:, 1]], e[T[:, 2]]], 1)
            art = T[:, 0] == 0
            lg = torch.where(art, _sub(m["art"], x).squeeze(1), _sub(m["elb"], x).squeeze(1))
            loss = focal_loss(lg, y)
            opt.zero_grad()
            loss.backward()
            opt.step()
            tot += float(loss.detach())
        print(json.dumps({"stage": "triplets", "epoch": ep,
                          "loss": round(tot / max(len(data), 1), 6)}), flush=True)


def train_joint(m, events, fs, r2, k_max, device, epochs=5, lr=5e-4, seed=0):
    """The GNN and both triplet classifiers together on L = L_edges +
    L_triplets (the thesis's joint objective), each step taking the triplets
    of the edges the current model keeps."""
    torch = _torch()
    rng = np.random.default_rng(seed)
    params = [p for g in ("node_enc", "edge_enc", "node", "edge", "cls", "art", "elb")
              for p in m[g].parameters()]
    opt = torch.optim.Adam(params, lr=lr)
    data = []
    for ev in events:
        src, dst, node_in = graph(m, ev, fs, r2, k_max, device)
        if len(src) == 0:
            continue
        y = _same_particle(ev, src, dst).astype(np.float32)
        data.append((ev, src, dst, torch.from_numpy(node_in).to(device),
                     torch.from_numpy(src).to(device), torch.from_numpy(dst).to(device),
                     torch.from_numpy(y).to(device)))
    for ep in range(epochs):
        tot = 0.0
        for ei in rng.permutation(len(data)):
            ev, src, dst, nf, s_, d_, y = data[ei]
            logit, e = gnn_forward(m, nf, s_, d_, with_states=True)
            loss = focal_loss(logit, y)
            kept = np.flatnonzero(logit.detach().cpu().numpy() >= 0.0)
            T = triplets_of(ev.plane, src, dst, kept)
            if len(T):
                ty = torch.from_numpy(triplet_labels(ev, src, dst, T).astype(np.float32)).to(device)
                Tt = torch.from_numpy(T).to(device)
                x = torch.cat([e[Tt[:, 1]], e[Tt[:, 2]]], 1)
                art = Tt[:, 0] == 0
                lg = torch.where(art, _sub(m["art"], x).squeeze(1), _sub(m["elb"], x).squeeze(1))
                loss = loss + focal_loss(lg, ty)
            opt.zero_grad()
            loss.backward()
            opt.step()
            tot += float(loss.detach())
        print(json.dumps({"stage": "joint", "epoch": ep, "loss": round(tot / max(len(data), 1), 6)}),
              flush=True)


def train(shape: synth.ModelShape, tracks: dict, noise: float, n_events: int, seed: int,
          k_max: int = 64, device=None, emb_epochs=6, gnn_epochs=8, pair_frac: float = 0.0,
          triplet_epochs: int = 0, joint_epochs: int = 0):
    """Train a model of `shape` (with triplet classifiers when
    `triplet_epochs` > 0); returns (blob, r2)."""
    torch = _torch()
    device = device or ("cuda" if torch.cuda.is_available() else "cpu")
    torch.manual_seed(seed)
    fs = (45.0, math.pi, 750.0, 45.0, 45.0, 750.0)
    events = [synth.gen_batch(1, seed, tracks, noise, first_event=e, pair_frac=pair_frac)
              for e in range(n_events)]
    m = build(shape, seed, device, triplets=triplet_epochs > 0)
    train_embedding(m, events, fs, device, epochs=emb_epochs, seed=seed)
    r2 = embedding_radius(m, events, fs, device)
    train_gnn(m, events, fs, r2, k_max, device, epochs=gnn_epochs, seed=seed)
    if triplet_epochs > 0:
        train_triplets(m, events, fs, r2, k_max, device, epochs=triplet_epochs, seed=seed)
        if joint_epochs > 0:
            train_joint(m, events, fs, r2, k_max, device, epochs=joint_epochs, seed=seed)
    return to_blob(m), r2


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--out", required=True, help="weight blob to write (a .json beside it "
                   "records the radius and the training settings)")
    p.add_argument("--events", type=int, default=120)
    p.add_argument("--seed", type=int, default=5003)
    p.add_argument("--tracks", default='{"kind": "poisson", "mean": 150, "min": 20, "max": 400}')
    p.add_argument("--noise", type=float, default=0.05)
    p.add_argument("--embed", default="3,64,64,4")
    p.add_argument("--hidden", type=int, default=32)
    p.add_argument("--iters", type=int, default=4)
    p.add_argument("--emb-epochs", type=int, default=8)
    p.add_argument("--gnn-epochs", type=int, default=15)
    p.add_argument("--device", default="cpu")
    p.add_argument("--pair-frac", type=float, default=0.0,
                   help="close track pairs with shared hits per track (generator option)")
    p.add_argument("--triplet-epochs", type=int, default=0,
                   help="> 0: also train the articulation and elbow classifiers")
    p.add_argument("--joint-epochs", type=int, default=0,
                   help="then fine-tune the GNN and the triplet classifiers together")
    a = p.parse_args()
    _torch().use_deterministic_algorithms(True)
    shape = synth.ModelShape([int(v) for v in a.embed.split(",")], a.hidden, a.iters)
    tracks = json.loads(a.tracks)
    blob, r2 = train(shape, tracks, a.noise, a.events, a.seed, device=a.device,
                     emb_epochs=a.emb_epochs, gnn_epochs=a.gnn_epochs, pair_frac=a.pair_frac,
                     triplet_epochs=a.triplet_epochs, joint_epochs=a.joint_epochs)
    with open(a.out, "wb") as f:
        f.write(blob)
    meta = {"radius2": r2, "embed": shape.embed, "hidden": a.hidden, "iters": a.iters,
            "train_events": a.events, "train_seed": a.seed, "tracks": tracks, "noise": a.noise,
            "emb_epochs": a.emb_epochs, "gnn_epochs": a.gnn_epochs, "device": a.device,
            "pair_frac": a.pair_frac, "triplet_epochs": a.triplet_epochs,
            "joint_epochs": a.joint_epochs,
            "radius_quantile_of_genuine_pairs": 0.995}
    with open(a.out.rsplit(".", 1)[0] + ".json", "w") as f:
        json.dump(meta, f, indent=2)
        f.write("\n")
    print(json.dumps({"out": a.out, "radius2": r2}))


if __name__ == "__main__":
    main()
