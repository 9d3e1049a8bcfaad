"""FP64 CPU oracle for the track-finding hot path -- TEST INFRASTRUCTURE.

Only the test suite, the package smoke check and the benchmark's CPU-baseline
leg may import this package. The product path (the CUDA library and its Python
binding) never imports it.

The arithmetic lives in `oracle.cpp` (plain C++, double precision), compiled to
`liboracle.so` by `build()`; this module only marshals numpy arrays. `metrics`
holds the track-finding metrics of the thesis (efficiency, ghost rate, clone
rate, hit purity, hit efficiency).

Parity status: every step is pinned by tests against closed forms, hand-worked
examples and brute force (see tests/test_oracle_pins.py; the triplet stage in
tests/test_oracle_triplets.py: triplets against a brute-force pair
enumeration, the classifiers' operand order and routing tied to the edge
classifier, track building on hand-worked graphs including a shared-hit pair,
and the whole path with the triplet stage on a hand-built event for every
on/off setting of the two heads). The composition of
the steps into the whole pipeline is pinned by a hand-built event
(tests/golden/pipeline_hand.json: identity embedding, straight lines with
gaps of one and two planes, a constant classifier on either side of the cut)
whose edge set and candidates are worked out by hand.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
# a prebuilt variant of the library to load instead (the planted-mistake tests
# compile copies of oracle.cpp with one mistake each and point here)
_LIB_VARIANT = os.environ.get("GNNTRK_ORACLE_LIB")
_lib = None

DEFAULT_FEAT_SCALE = (45.0, math.pi, 750.0, 45.0, 45.0, 750.0)


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so (plain g++, no GPU code)."""
    if _LIB_VARIANT:
        return _LIB_VARIANT
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.orc_model_load.restype = vp
        L.orc_model_load.argtypes = [vp, ctypes.c_size_t, i32, vp, i32, i32, ctypes.c_char_p, i32]
        L.orc_model_free.argtypes = [vp]
        L.orc_embed.argtypes = [vp, i64, vp, vp, vp, vp, vp]
        L.orc_radius_graph.restype = i64
        L.orc_radius_graph.argtypes = [i64, vp, vp, i32, i32, dbl, i32, vp, vp, vp, i64]
        L.orc_in_logits.argtypes = [vp, i64, vp, vp, vp, vp, i64, vp, vp, vp]
        L.orc_components.argtypes = [i64, i64, vp, vp, vp, vp]
        L.orc_find_tracks_event.restype = i64
        L.orc_find_tracks_event.argtypes = [vp, i32, i32, dbl, dbl, vp, i64, vp, vp, vp, vp,
                                            vp, vp, vp, vp, vp, vp, i64]
        L.orc_find_tracks_batch.restype = i64
        L.orc_find_tracks_batch.argtypes = [vp, i32, i32, dbl, dbl, vp, i32, vp, vp, vp, vp,
                                            vp, vp, i32]
        L.orc_candidate_d2.restype = i64
        L.orc_candidate_d2.argtypes = [i64, vp, vp, i32, i32, vp, i64]
        L.orc_edge_states.argtypes = [vp, i64, vp, vp, vp, vp, i64, vp, vp, vp]
        L.orc_triplets.restype = i64
        L.orc_triplets.argtypes = [i64, vp, i64, vp, vp, vp, vp, vp, vp, i64]
        L.orc_triplet_logits.restype = i32
        L.orc_triplet_logits.argtypes = [vp, i64, vp, vp, vp, vp, vp]
        L.orc_build_tracks.restype = i64
        L.orc_build_tracks.argtypes = [i64, i64, vp, vp, vp, i64, vp, vp, vp, vp, vp, i64, vp,
                                       i64, vp]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def cut_logit(score_cut: float) -> float:
    """Score cut s on sigmoid(logit) as a cut on the logit: log(s / (1 - s))."""
    return math.log(score_cut / (1.0 - score_cut))


class Model:
    """FP64 copy of a weight blob, checked against the architecture."""

    def __init__(self, blob: bytes, embed_dims, hidden: int, iters: int):
        self._blob = np.frombuffer(blob, dtype=np.uint8).copy()
        dims = np.asarray(embed_dims, dtype=np.int32)
        err = ctypes.create_string_buffer(256)
        self.D = int(dims[-1])
        self.hidden, self.iters = hidden, iters
        self.ptr = lib().orc_model_load(_p(self._blob), self._blob.size, len(dims) - 1,
                                        _p(dims), hidden, iters, err, 256)
        self._dims = dims
        if not self.ptr:
            raise ValueError("oracle: " + err.value.decode())

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.orc_model_free(self.ptr)
            self.ptr = None


def embed(model: Model, x, y, z, feat_scale=DEFAULT_FEAT_SCALE) -> np.ndarray:
    x, y, z = _c(x, np.float32), _c(y, np.float32), _c(z, np.float32)
    out = np.zeros((x.size, model.D), dtype=np.float64)
    fs = _c(feat_scale, np.float64)
    lib().orc_embed(model.ptr, x.size, _p(x), _p(y), _p(z), _p(fs), _p(out))
    return out


def radius_graph(plane, emb, r2: float, k_max: int, n_planes: int = 26):
    """(src, dst, d2) of the rough graph of one event."""
    plane = _c(plane, np.uint8)
    emb = _c(emb, np.float64)
    n, D = emb.shape
    ne = lib().orc_radius_graph(n, _p(plane), _p(emb), D, n_planes, r2, k_max,
                                None, None, None, 0)
    src, dst = np.zeros(ne, np.int32), np.zeros(ne, np.int32)
    d2 = np.zeros(ne, np.float64)
    lib().orc_radius_graph(n, _p(plane), _p(emb), D, n_planes, r2, k_max,
                           _p(src), _p(dst), _p(d2), ne)
    return src, dst, d2


def in_logits(model: Model, x, y, z, src, dst, feat_scale=DEFAULT_FEAT_SCALE) -> np.ndarray:
    x, y, z = _c(x, np.float32), _c(y, np.float32), _c(z, np.float32)
    src, dst = _c(src, np.int32), _c(dst, np.int32)
    out = np.zeros(src.size, np.float64)
    fs = _c(feat_scale, np.float64)
    lib().orc_in_logits(model.ptr, x.size, _p(x), _p(y), _p(z), _p(fs), src.size,
                        _p(src), _p(dst), _p(out))
    return out


def components(n: int, src, dst, keep=None) -> np.ndarray:
    src, dst = _c(src, np.int32), _c(dst, np.int32)
    k = None if keep is None else _c(keep, np.uint8)
    out = np.zeros(n, np.int32)
    lib().orc_components(n, src.size, _p(src), _p(dst), _p(k), _p(out))
    return out


class EventResult:
    def __init__(self, labels, src, dst, d2, logit, keep):
        self.labels, self.src, self.dst = labels, src, dst
        self.d2, self.logit, self.keep = d2, logit, keep


def find_tracks_event(model: Model, x, y, z, plane, r2: float, k_max: int, cut: float = 0.5,
                      n_planes: int = 26, feat_scale=DEFAULT_FEAT_SCALE) -> EventResult:
    x, y, z = _c(x, np.float32), _c(y, np.float32), _c(z, np.float32)
    plane = _c(plane, np.uint8)
    fs = _c(feat_scale, np.float64)
    n = x.size
    labels = np.zeros(n, np.int32)
    cap = max(64, 40 * n)
    while True:
        src, dst = np.zeros(cap, np.int32), np.zeros(cap, np.int32)
        d2, lg = np.zeros(cap, np.float64), np.zeros(cap, np.float64)
        keep = np.zeros(cap, np.uint8)
        ne = lib().orc_find_tracks_event(model.ptr, n_planes, k_max, r2, cut_logit(cut), _p(fs),
                                         n, _p(x), _p(y), _p(z), _p(plane), _p(labels),
                                         _p(src), _p(dst), _p(d2), _p(lg), _p(keep), cap)
        if ne <= cap:
            return EventResult(labels, src[:ne], dst[:ne], d2[:ne], lg[:ne], keep[:ne])
        cap = ne


def find_tracks_batch(model: Model, x, y, z, plane, offsets, r2: float, k_max: int,
                      cut: float = 0.5, threads: int = 1, n_planes: int = 26,
                      feat_scale=DEFAULT_FEAT_SCALE):
    """Event-local labels for every hit of a batch; returns (labels, n_edges)."""
    x, y, z = _c(x, np.float32), _c(y, np.float32), _c(z, np.float32)
    plane, offsets = _c(plane, np.uint8), _c(offsets, np.int64)
    fs = _c(feat_scale, np.float64)
    labels = np.zeros(x.size, np.int32)
    ne = lib().orc_find_tracks_batch(model.ptr, n_planes, k_max, r2, cut_logit(cut), _p(fs),
                                     offsets.size - 1, _p(offsets), _p(x), _p(y), _p(z),
                                     _p(plane), _p(labels), threads)
    return labels, ne


def candidate_d2(plane, emb, n_planes: int = 26) -> np.ndarray:
    plane = _c(plane, np.uint8)
    emb = _c(emb, np.float64)
    n, D = emb.shape
    c = lib().orc_candidate_d2(n, _p(plane), _p(emb), D, n_planes, None, 0)
    out = np.zeros(c, np.float64)
    lib().orc_candidate_d2(n, _p(plane), _p(emb), D, n_planes, _p(out), c)
    return out


# ---------------------------------------------------------------------------
# Triplet stage (Secs. "Triplet Building" and "Track Building")
# ---------------------------------------------------------------------------
TRIPLET_TYPES = ("articulation", "left_elbow", "right_elbow")


def edge_states(model: Model, x, y, z, src, dst, feat_scale=DEFAULT_FEAT_SCALE) -> np.ndarray:
    """Final edge encodings e^K [ne][h] (FP64)."""
    x, y, z = _c(x, np.float32), _c(y, np.float32), _c(z, np.float32)
    src, dst = _c(src, np.int32), _c(dst, np.int32)
    out = np.zeros((src.size, model.hidden), np.float64)
    fs = _c(feat_scale, np.float64)
    lib().orc_edge_states(model.ptr, x.size, _p(x), _p(y), _p(z), _p(fs), src.size, _p(src),
                          _p(dst), _p(out))
    return out


def triplets(plane, src, dst, keep):
    """(type, e1, e2) of every triplet of the purified graph (kept edges)."""
    plane, src, dst = _c(plane, np.uint8), _c(src, np.int32), _c(dst, np.int32)
    keep = _c(keep, np.uint8)
    n = lib().orc_triplets(plane.size, _p(plane), src.size, _p(src), _p(dst), _p(keep),
                           None, None, None, 0)
    ty, a, b = np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n, np.int32)
    lib().orc_triplets(plane.size, _p(plane), src.size, _p(src), _p(dst), _p(keep),
                       _p(ty), _p(a), _p(b), n)
    return ty, a, b


def triplet_logits(model: Model, ty, e1, e2, e_final) -> np.ndarray:
    ty, e1, e2 = _c(ty, np.int32), _c(e1, np.int32), _c(e2, np.int32)
    E = _c(e_final, np.float64)
    out = np.zeros(ty.size, np.float64)
    if lib().orc_triplet_logits(model.ptr, ty.size, _p(ty), _p(e1), _p(e2), _p(E), _p(out)) != 0:
        raise ValueError("oracle: the model has no triplet classifiers")
    return out


def build_tracks(n_hits: int, src, dst, keep, ty, e1, e2, tkeep):
    """Tracks (list of ascending hit-index arrays, lexicographic order)."""
    src, dst, keep = _c(src, np.int32), _c(dst, np.int32), _c(keep, np.uint8)
    ty, e1, e2, tk = _c(ty, np.int32), _c(e1, np.int32), _c(e2, np.int32), _c(tkeep, np.uint8)
    th = np.zeros(1, np.int64)
    args = lambda off, co, hits, ch: (n_hits, src.size, _p(src), _p(dst), _p(keep), ty.size,
                                      _p(ty), _p(e1), _p(e2), _p(tk), _p(off), co, _p(hits), ch,
                                      _p(th))
    nk = lib().orc_build_tracks(*args(None, 0, None, 0))
    off = np.zeros(nk + 1, np.int32)
    hits = np.zeros(int(th[0]), np.int32)
    lib().orc_build_tracks(*args(off, nk, hits, hits.size))
    return [hits[off[k]:off[k + 1]].copy() for k in range(nk)]


class TripletResult(EventResult):
    def __init__(self, base: EventResult, ty, e1, e2, tlogit, tkeep, tracks):
        super().__init__(base.labels, base.src, base.dst, base.d2, base.logit, base.keep)
        self.ttype, self.te1, self.te2 = ty, e1, e2
        self.tlogit, self.tkeep, self.tracks = tlogit, tkeep, tracks


def find_tracks_triplets_event(model: Model, x, y, z, plane, r2: float, k_max: int,
                               cut: float = 0.5, triplet_cut: float = 0.5, n_planes: int = 26,
                               feat_scale=DEFAULT_FEAT_SCALE) -> TripletResult:
    """The whole path with the triplet stage for one event: graph, edge scores
    and cut, triplets of the kept edges scored by the triplet classifiers and
    cut at `triplet_cut`, then track building."""
    base = find_tracks_event(model, x, y, z, plane, r2, k_max, cut, n_planes, feat_scale)
    E = edge_states(model, x, y, z, base.src, base.dst, feat_scale)
    ty, e1, e2 = triplets(plane, base.src, base.dst, base.keep)
    tl = triplet_logits(model, ty, e1, e2, E)
    tk = (tl >= cut_logit(triplet_cut)).astype(np.uint8)
    tracks = build_tracks(len(x), base.src, base.dst, base.keep, ty, e1, e2, tk)
    return TripletResult(base, ty, e1, e2, tl, tk, tracks)
