"""Seeded synthetic inputs: vertex-detector events and model weight blobs.

This module holds input generation only. It computes none of the track-finding
arithmetic (no embedding, no graph, no GNN, no components); both the CUDA
library and the FP64 oracle consume what it produces.

Event model (stands in for the LHCb minimum-bias samples of Sec. "Datasets",
which are not available): straight-line tracks from a beam-spot origin through
26 planes of a silicon-pixel vertex detector, as in the VELO geometry of
Sec. "The Vertex Locator" (26 modules spanning roughly -300..750 mm in z, an
active annulus of about 5-45 mm around the beam, straight tracks because the
VELO sits outside the magnet).

  * origin x, y ~ N(0, 0.05 mm), z ~ N(0, 50 mm)
  * pseudorapidity eta ~ U[2, 5], azimuth phi ~ U[0, 2 pi), polar angle
    theta = 2 atan(exp(-eta))
  * plane p at z_p = linspace(-300, 750, 26)[p]; a track leaves a hit on
    plane p when z_p > v_z, 5 <= r <= 45 mm at the plane, and a Bernoulli(0.98)
    draw succeeds
  * x, y smeared by N(0, 0.012 mm) each; z is the plane position
  * noise: round(f * n_signal) hits, uniform plane, r^2 ~ U[25, 2025] mm^2,
    phi ~ U[0, 2 pi), particle id -1
  * hits of an event are shuffled (the consumer must not assume plane order)

Weight blob format (little endian), read independently by the oracle and by
the CUDA library:

    uint32 magic = 0x57544E47 ("GNTW"), uint32 version = 1,
    uint32 n_layers, uint32 reserved = 0,
    n_layers x (uint32 fan_in, uint32 fan_out),
    then for each layer: float32 W[fan_out][fan_in], float32 b[fan_out]

Layer order: embedding MLP layers; node encoder (3->h, h->h); edge encoder
(2h->h, h->h); for k = 0..K-1: node network k (3h->h, h->h) then edge network
k (3h->h, h->h); edge classifier (h->h, h->1).

Weights are Kaiming-uniform, W ~ U(-sqrt(6/fan_in), +sqrt(6/fan_in)), and
biases follow the usual Linear default, b ~ U(-1/sqrt(fan_in), +1/sqrt(fan_in)),
drawn from numpy's PCG64 seeded with (seed, layer index).
"""
from __future__ import annotations

import json
import os
import struct
from dataclasses import dataclass, field

import numpy as np

N_PLANES = 26
PLANE_Z = np.linspace(-300.0, 750.0, N_PLANES)
R_MIN, R_MAX = 5.0, 45.0
HIT_EFF = 0.98
SMEAR_MM = 0.012
WEIGHTS_MAGIC = 0x57544E47
WEIGHTS_VERSION = 1

_HERE = os.path.dirname(os.path.abspath(__file__))
WORKLOADS_PATH = os.path.join(_HERE, "workloads.json")


# ----------------------------------------------------------------------------
# events
# ----------------------------------------------------------------------------
@dataclass
class Batch:
    """Events concatenated in structure-of-arrays form.

    x, y, z: float32 [n_hits]; plane: uint8 [n_hits]; pid: int32 [n_hits]
    (-1 for noise); offsets: int64 [n_events + 1]; pid2: int32 [n_hits], the
    second particle of a hit that two particles share (-1 otherwise), or None
    when no hit is shared.
    """
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    plane: np.ndarray
    pid: np.ndarray
    offsets: np.ndarray
    pid2: np.ndarray | None = None

    @property
    def n_events(self) -> int:
        return len(self.offsets) - 1

    @property
    def n_hits(self) -> int:
        return int(self.offsets[-1])

    def event(self, e: int) -> "Batch":
        a, b = int(self.offsets[e]), int(self.offsets[e + 1])
        return Batch(self.x[a:b], self.y[a:b], self.z[a:b], self.plane[a:b],
                     self.pid[a:b], np.array([0, b - a], dtype=np.int64),
                     None if self.pid2 is None else self.pid2[a:b])

    def xyz_soa(self) -> np.ndarray:
        """float32 [3][n_hits]: the layout the library takes."""
        return np.stack([self.x, self.y, self.z]).astype(np.float32)

    def subset(self, events) -> "Batch":
        parts = [self.event(int(e)) for e in events]
        return concat(parts)


def concat(parts) -> Batch:
    sizes = [p.n_hits for p in parts]
    offs = np.zeros(len(parts) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(sizes)
    cat = lambda k, dt: (np.concatenate([getattr(p, k) for p in parts]).astype(dt)
                         if parts else np.zeros(0, dt))
    pid2 = None
    if any(p.pid2 is not None for p in parts):
        pid2 = np.concatenate([p.pid2 if p.pid2 is not None else np.full(p.n_hits, -1)
                               for p in parts]).astype(np.int32)
    return Batch(cat("x", np.float32), cat("y", np.float32), cat("z", np.float32),
                 cat("plane", np.uint8), cat("pid", np.int32), offs, pid2)


def gen_event(rng: np.random.Generator, n_tracks: int, noise_frac: float,
              pair_frac: float = 0.0) -> Batch:
    """One event of `n_tracks` straight tracks plus uniform noise hits.

    pair_frac > 0 adds round(pair_frac * n_tracks) close pairs standing in for
    the electron-positron conversions of the thesis's triplet motivation: each
    pair is a new track from the vertex of a randomly chosen track, its slopes
    off by N(0, PAIR_OPENING) in x and y; where the two true positions on a
    plane lie within PAIR_MERGE_MM they leave one shared hit (at their mean,
    smeared; pid = the first track, pid2 = the partner). With pair_frac = 0
    the draws are exactly those of the plain generator.
    """
    if pair_frac > 0.0:
        return _gen_event_pairs(rng, n_tracks, noise_frac, pair_frac)
    vx = rng.normal(0.0, 0.05, n_tracks)
    vy = rng.normal(0.0, 0.05, n_tracks)
    vz = rng.normal(0.0, 50.0, n_tracks)
    eta = rng.uniform(2.0, 5.0, n_tracks)
    phi = rng.uniform(0.0, 2.0 * np.pi, n_tracks)
    theta = 2.0 * np.arctan(np.exp(-eta))
    tx = np.tan(theta) * np.cos(phi)
    ty = np.tan(theta) * np.sin(phi)

    dz = PLANE_Z[None, :] - vz[:, None]                      # [T, P]
    xs = vx[:, None] + tx[:, None] * dz
    ys = vy[:, None] + ty[:, None] * dz
    r = np.hypot(xs, ys)
    eff = rng.uniform(0.0, 1.0, dz.shape) < HIT_EFF
    hit = (dz > 0) & (r >= R_MIN) & (r <= R_MAX) & eff
    ti, pi = np.nonzero(hit)
    sx = xs[ti, pi] + rng.normal(0.0, SMEAR_MM, ti.size)
    sy = ys[ti, pi] + rng.normal(0.0, SMEAR_MM, ti.size)
    sz = PLANE_Z[pi]

    n_noise = int(round(noise_frac * ti.size))
    npl = rng.integers(0, N_PLANES, n_noise)
    nr = np.sqrt(rng.uniform(R_MIN ** 2, R_MAX ** 2, n_noise))
    nphi = rng.uniform(0.0, 2.0 * np.pi, n_noise)

    x = np.concatenate([sx, nr * np.cos(nphi)])
    y = np.concatenate([sy, nr * np.sin(nphi)])
    z = np.concatenate([sz, PLANE_Z[npl]])
    plane = np.concatenate([pi, npl]).astype(np.uint8)
    pid = np.concatenate([ti, np.full(n_noise, -1)]).astype(np.int32)
    order = rng.permutation(x.size)
    return Batch(x[order].astype(np.float32), y[order].astype(np.float32),
                 z[order].astype(np.float32), plane[order], pid[order],
                 np.array([0, x.size], dtype=np.int64))


PAIR_OPENING = 4e-4      # rad, per slope component
PAIR_MERGE_MM = 0.1      # two crossings closer than this make one hit


def _gen_event_pairs(rng, n_tracks, noise_frac, pair_frac):
    n_pairs = int(round(pair_frac * n_tracks))
    vx = rng.normal(0.0, 0.05, n_tracks)
    vy = rng.normal(0.0, 0.05, n_tracks)
    vz = rng.normal(0.0, 50.0, n_tracks)
    eta = rng.uniform(2.0, 5.0, n_tracks)
    phi = rng.uniform(0.0, 2.0 * np.pi, n_tracks)
    theta = 2.0 * np.arctan(np.exp(-eta))
    tx = np.tan(theta) * np.cos(phi)
    ty = np.tan(theta) * np.sin(phi)
    mother = rng.choice(n_tracks, n_pairs, replace=False) if n_pairs else np.zeros(0, np.int64)
    ptx = tx[mother] + rng.normal(0.0, PAIR_OPENING, n_pairs)
    pty = ty[mother] + rng.normal(0.0, PAIR_OPENING, n_pairs)
    T = n_tracks + n_pairs
    VX = np.concatenate([vx, vx[mother]])
    VY = np.concatenate([vy, vy[mother]])
    VZ = np.concatenate([vz, vz[mother]])
    TX = np.concatenate([tx, ptx])
    TY = np.concatenate([ty, pty])
    dz = PLANE_Z[None, :] - VZ[:, None]
    xs = VX[:, None] + TX[:, None] * dz
    ys = VY[:, None] + TY[:, None] * dz
    r = np.hypot(xs, ys)
    eff = rng.uniform(0.0, 1.0, dz.shape) < HIT_EFF
    hit = (dz > 0) & (r >= R_MIN) & (r <= R_MAX) & eff
    # a partner crossing within the merge distance of its mother's crossing on
    # the same plane (both detected) is absorbed into one shared hit
    shared = np.zeros((T, N_PLANES), bool)
    for k, mo in enumerate(mother):
        pk = n_tracks + k
        close = np.hypot(xs[pk] - xs[mo], ys[pk] - ys[mo]) < PAIR_MERGE_MM
        both = hit[pk] & hit[mo] & close
        shared[mo] = both
        hit[pk] &= ~both
        xs[mo, both] = 0.5 * (xs[mo, both] + xs[pk, both])
        ys[mo, both] = 0.5 * (ys[mo, both] + ys[pk, both])
    partner = np.full(T, -1)
    partner[mother] = n_tracks + np.arange(n_pairs)
    ti, pi = np.nonzero(hit)
    sx = xs[ti, pi] + rng.normal(0.0, SMEAR_MM, ti.size)
    sy = ys[ti, pi] + rng.normal(0.0, SMEAR_MM, ti.size)
    sz = PLANE_Z[pi]
    p2 = np.where(shared[ti, pi], partner[ti], -1)

    n_noise = int(round(noise_frac * ti.size))
    npl = rng.integers(0, N_PLANES, n_noise)
    nr = np.sqrt(rng.uniform(R_MIN ** 2, R_MAX ** 2, n_noise))
    nphi = rng.uniform(0.0, 2.0 * np.pi, n_noise)

    x = np.concatenate([sx, nr * np.cos(nphi)])
    y = np.concatenate([sy, nr * np.sin(nphi)])
    z = np.concatenate([sz, PLANE_Z[npl]])
    plane = np.concatenate([pi, npl]).astype(np.uint8)
    pid = np.concatenate([ti, np.full(n_noise, -1)]).astype(np.int32)
    pid2 = np.concatenate([p2, np.full(n_noise, -1)]).astype(np.int32)
    order = rng.permutation(x.size)
    return Batch(x[order].astype(np.float32), y[order].astype(np.float32),
                 z[order].astype(np.float32), plane[order], pid[order],
                 np.array([0, x.size], dtype=np.int64), pid2[order])


def track_count(rng: np.random.Generator, spec: dict) -> int:
    if spec["kind"] == "fixed":
        return int(spec["n"])
    if spec["kind"] == "poisson":
        return int(np.clip(rng.poisson(spec["mean"]), spec["min"], spec["max"]))
    raise ValueError(f"unknown track-count kind {spec['kind']!r}")


def gen_batch(n_events: int, seed: int, tracks: dict, noise_frac: float,
              first_event: int = 0, pair_frac: float = 0.0) -> Batch:
    """Events first_event .. first_event + n_events - 1 of the stream `seed`.

    Event e draws from its own PCG64 stream seeded with (seed, e), so any
    subset of a workload can be regenerated on its own.
    """
    parts = []
    for e in range(first_event, first_event + n_events):
        rng = np.random.default_rng([seed, e])
        parts.append(gen_event(rng, track_count(rng, tracks), noise_frac, pair_frac))
    return concat(parts)


# ----------------------------------------------------------------------------
# model shapes and weights
# ----------------------------------------------------------------------------
@dataclass
class ModelShape:
    embed: list            # e.g. [3, 64, 64, 4]
    hidden: int            # n_h = n_e
    iters: int             # message-passing steps K
    layers: list = field(default_factory=list)

    def __post_init__(self):
        h = self.hidden
        L = [(self.embed[i], self.embed[i + 1]) for i in range(len(self.embed) - 1)]
        L += [(3, h), (h, h)]                    # node encoder
        L += [(2 * h, h), (h, h)]                # edge encoder
        for _ in range(self.iters):
            L += [(3 * h, h), (h, h)]            # node network k
            L += [(3 * h, h), (h, h)]            # edge network k
        L += [(h, h), (h, 1)]                    # edge classifier
        self.layers = L


def make_weights(shape: ModelShape, seed: int) -> bytes:
    """Kaiming-uniform weights and Linear-default biases, packed as a blob."""
    head = struct.pack("<IIII", WEIGHTS_MAGIC, WEIGHTS_VERSION, len(shape.layers), 0)
    dims = b"".join(struct.pack("<II", i, o) for i, o in shape.layers)
    body = []
    for li, (fi, fo) in enumerate(shape.layers):
        rng = np.random.default_rng([seed, li])
        bw = np.sqrt(6.0 / fi)
        bb = 1.0 / np.sqrt(fi)
        body.append(rng.uniform(-bw, bw, (fo, fi)).astype("<f4").tobytes())
        body.append(rng.uniform(-bb, bb, fo).astype("<f4").tobytes())
    return head + dims + b"".join(body)


def weight_arrays(blob: bytes):
    """Split a blob into [(W[fo][fi], b[fo])] float32 arrays (for tests)."""
    magic, ver, n, _ = struct.unpack_from("<IIII", blob, 0)
    assert magic == WEIGHTS_MAGIC and ver == WEIGHTS_VERSION
    dims = [struct.unpack_from("<II", blob, 16 + 8 * i) for i in range(n)]
    off = 16 + 8 * n
    out = []
    for fi, fo in dims:
        W = np.frombuffer(blob, "<f4", fi * fo, off).reshape(fo, fi)
        off += 4 * fi * fo
        b = np.frombuffer(blob, "<f4", fo, off)
        off += 4 * fo
        out.append((W.copy(), b.copy()))
    return out


def pack_weights(arrays) -> bytes:
    """Inverse of weight_arrays: pack explicit (W, b) pairs (for hand-built tests)."""
    head = struct.pack("<IIII", WEIGHTS_MAGIC, WEIGHTS_VERSION, len(arrays), 0)
    dims = b"".join(struct.pack("<II", W.shape[1], W.shape[0]) for W, _ in arrays)
    body = b"".join(np.asarray(W, "<f4").tobytes() + np.asarray(b, "<f4").tobytes()
                    for W, b in arrays)
    return head + dims + body


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------
def workloads() -> dict:
    with open(WORKLOADS_PATH) as f:
        return json.load(f)


def workload(name: str) -> dict:
    return workloads()[name]


def shape_of(wl: dict) -> ModelShape:
    m = wl["model"]
    return ModelShape(list(m["embed"]), int(m["hidden"]), int(m["iters"]))


def workload_batch(wl: dict, n_events: int | None = None, first_event: int = 0,
                   seed_key: str = "events") -> Batch:
    n = wl["n_events"] if n_events is None else n_events
    return gen_batch(n, wl["seeds"][seed_key], wl["tracks"], wl["noise"], first_event,
                     wl.get("pair_frac", 0.0))


def workload_weights(wl: dict) -> bytes:
    """The workload's weight blob: a trained blob shipped with the package
    (`weights_file`, written by the training tool) or seeded random weights."""
    if wl.get("weights_file"):
        with open(os.path.join(_HERE, wl["weights_file"]), "rb") as f:
            return f.read()
    return make_weights(shape_of(wl), wl["seeds"]["weights"])
