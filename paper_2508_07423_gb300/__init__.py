"""gnntrk: GNN track finding for one GB300 -- Python binding of libgnntrk.

This module only marshals arguments to the C ABI of include/gnntrk.h (ctypes,
plain pointers); every step of the hot path runs in the library's CUDA
kernels. Importing works without a GPU; using a Tracker needs the built
library (`paper_2508_07423_gb300.build.build()`) and a CUDA device, and fails
loudly otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libgnntrk.so")

FP32, BF16, FP8_E4M3 = 0, 1, 2
PRECISIONS = {"fp32": FP32, "bf16": BF16, "fp8": FP8_E4M3}

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "CAPACITY", 5: "TIMEOUT",
          6: "WEIGHTS", 7: "UNSUPPORTED"}

EXPORTS = ["gnntrk_default_cfg", "gnntrk_create", "gnntrk_find_tracks", "gnntrk_sync_status",
           "gnntrk_get_graph", "gnntrk_stats", "gnntrk_set_profiling", "gnntrk_stage_times",
           "gnntrk_components_noalloc", "gnntrk_workspace_bytes", "gnntrk_serve_run",
           "gnntrk_autotune", "gnntrk_set_tuning", "gnntrk_selftest_wait", "gnntrk_rescore_rows", "gnntrk_e4m3_encode",
           "gnntrk_e4m3_decode", "gnntrk_tc_throughput",
           "gnntrk_find_tracks_triplets", "gnntrk_triplet_stats", "gnntrk_get_triplets",
           "gnntrk_embed_amax", "gnntrk_set_embed_scales",
           "gnntrk_last_error", "gnntrk_destroy"]

NOALLOC_MAX_HITS = 1 << 20


class GnntrkError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"gnntrk {STATUS.get(status, status)}: {msg}")
        self.status = status


# the entries of a launch configuration (gnntrk_autotune / gnntrk_set_tuning)
TUNING_KEYS = ("tc_node_prep", "tc_edge_encoder", "tc_node_update", "tc_edge_update",
               "f32_encoders", "f32_node_update", "f32_edge_update", "tc_edge_tma")


class ServeCfg(ctypes.Structure):
    """Mirror of gnntrk_serve_cfg."""
    _fields_ = [
        ("n_slots", ctypes.c_int32),
        ("max_events_per_batch", ctypes.c_int32),
        ("max_hits_per_batch", ctypes.c_int64),
        ("memory_budget_bytes", ctypes.c_int64),
        ("apply_tuning", ctypes.c_int32),
        ("tuning", ctypes.c_int32 * 8),
        ("reserved", ctypes.c_int32 * 7),
    ]


class Cfg(ctypes.Structure):
    """Mirror of gnntrk_cfg (include/gnntrk.h)."""
    _fields_ = [
        ("n_embed_layers", ctypes.c_int32),
        ("embed_dims", ctypes.c_int32 * 9),
        ("hidden", ctypes.c_int32),
        ("iters", ctypes.c_int32),
        ("n_planes", ctypes.c_int32),
        ("k_max", ctypes.c_int32),
        ("radius2", ctypes.c_float),
        ("score_cut", ctypes.c_float),
        ("feat_scale", ctypes.c_float * 6),
        ("precision", ctypes.c_int32),
        ("rescore_band", ctypes.c_float),
        ("max_hits", ctypes.c_int64),
        ("max_events", ctypes.c_int32),
        ("edges_per_hit", ctypes.c_int32),
        ("use_graph", ctypes.c_int32),
        ("triplets", ctypes.c_int32),
        ("triplet_cut", ctypes.c_float),
        ("triplets_per_hit", ctypes.c_int32),
        ("embed_int8", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 3),
    ]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libgnntrk.so and declare its exports (no GPU needed)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libgnntrk.so not built ({path}); run paper_2508_07423_gb300.build")
    L = ctypes.CDLL(path)
    vp, i32, i64, st = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int
    L.gnntrk_default_cfg.argtypes = [ctypes.POINTER(Cfg)]
    L.gnntrk_default_cfg.restype = None
    L.gnntrk_create.argtypes = [vp, ctypes.c_size_t, ctypes.POINTER(Cfg), ctypes.POINTER(vp)]
    L.gnntrk_create.restype = st
    L.gnntrk_find_tracks.argtypes = [vp, i32, i64, vp, vp, vp, vp, vp]
    L.gnntrk_find_tracks.restype = st
    L.gnntrk_sync_status.argtypes = [vp, vp]
    L.gnntrk_sync_status.restype = st
    L.gnntrk_get_graph.argtypes = [vp, i32, i64, vp, vp, vp, vp, vp, ctypes.POINTER(i64)]
    L.gnntrk_get_graph.restype = st
    L.gnntrk_stats.argtypes = [vp, vp]
    L.gnntrk_stats.restype = st
    L.gnntrk_rescore_rows.argtypes = [vp, i32, vp, vp]
    L.gnntrk_rescore_rows.restype = st
    L.gnntrk_e4m3_encode.argtypes = [vp, vp, i64, i32, vp]
    L.gnntrk_e4m3_encode.restype = st
    L.gnntrk_e4m3_decode.argtypes = [vp, vp, i64]
    L.gnntrk_e4m3_decode.restype = st
    L.gnntrk_tc_throughput.argtypes = [i32, i64, ctypes.POINTER(ctypes.c_double)]
    L.gnntrk_tc_throughput.restype = st
    L.gnntrk_set_profiling.argtypes = [vp, i32]
    L.gnntrk_set_profiling.restype = st
    L.gnntrk_stage_times.argtypes = [vp, i32, vp, vp, vp]
    L.gnntrk_stage_times.restype = i32
    L.gnntrk_components_noalloc.argtypes = [i64, i64, vp, vp, vp, vp, vp]
    L.gnntrk_components_noalloc.restype = st
    L.gnntrk_autotune.argtypes = [vp, i32, i64, vp, vp, vp, vp, vp, vp]
    L.gnntrk_autotune.restype = st
    L.gnntrk_set_tuning.argtypes = [vp, vp]
    L.gnntrk_set_tuning.restype = st
    L.gnntrk_selftest_wait.argtypes = [vp, i64, vp]
    L.gnntrk_selftest_wait.restype = st
    L.gnntrk_workspace_bytes.argtypes = [ctypes.POINTER(Cfg)]
    L.gnntrk_workspace_bytes.restype = i64
    L.gnntrk_serve_run.argtypes = [vp, ctypes.c_size_t, ctypes.POINTER(Cfg),
                                   ctypes.POINTER(ServeCfg), i32, vp, vp, vp, vp, vp, vp, vp]
    L.gnntrk_serve_run.restype = st
    L.gnntrk_find_tracks_triplets.argtypes = [vp, i32, i64, vp, vp, vp, vp, vp, vp, vp, i64, i64,
                                              vp]
    L.gnntrk_find_tracks_triplets.restype = st
    L.gnntrk_triplet_stats.argtypes = [vp, vp]
    L.gnntrk_triplet_stats.restype = st
    L.gnntrk_get_triplets.argtypes = [vp, i32, i64, vp, vp, vp, vp, ctypes.POINTER(i64)]
    L.gnntrk_get_triplets.restype = st
    L.gnntrk_embed_amax.argtypes = [vp, i64, vp, vp, vp]
    L.gnntrk_embed_amax.restype = st
    L.gnntrk_set_embed_scales.argtypes = [vp, vp, i32]
    L.gnntrk_set_embed_scales.restype = st
    L.gnntrk_last_error.argtypes = [vp]
    L.gnntrk_last_error.restype = ctypes.c_char_p
    L.gnntrk_destroy.argtypes = [vp]
    L.gnntrk_destroy.restype = None
    _lib = L
    return L


def default_cfg() -> Cfg:
    c = Cfg()
    load_library().gnntrk_default_cfg(ctypes.byref(c))
    return c


def make_cfg(model: dict, radius2: float, k_max: int = 64, score_cut: float = 0.5,
             precision="fp32", rescore_band: float = 0.0, max_hits: int = 1 << 20,
             max_events: int = 4096, edges_per_hit: int = 24, use_graph: bool = False,
             n_planes: int = 26, feat_scale=None, triplets: bool = False,
             triplet_cut: float = 0.5, triplets_per_hit: int = 16,
             embed_int8: bool = False) -> Cfg:
    """Build a cfg from a model description {"embed": [...], "hidden", "iters"}."""
    c = default_cfg()
    emb = list(model["embed"])
    c.n_embed_layers = len(emb) - 1
    for i in range(9):
        c.embed_dims[i] = emb[i] if i < len(emb) else 0
    c.hidden = int(model["hidden"])
    c.iters = int(model["iters"])
    c.n_planes = n_planes
    c.k_max = k_max
    c.radius2 = radius2
    c.score_cut = score_cut
    if feat_scale is not None:
        for i in range(6):
            c.feat_scale[i] = feat_scale[i]
    c.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    c.rescore_band = rescore_band
    c.max_hits = max_hits
    c.max_events = max_events
    c.edges_per_hit = edges_per_hit
    c.use_graph = int(bool(use_graph))
    c.triplets = int(bool(triplets))
    c.triplet_cut = triplet_cut
    c.triplets_per_hit = triplets_per_hit
    c.embed_int8 = int(bool(embed_int8))
    return c


def feat_scale_of(cfg: Cfg):
    """The float32 feature scales the library uses (for an identical oracle input)."""
    return tuple(float(np.float32(cfg.feat_scale[i])) for i in range(6))


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


class Tracker:
    """One library handle: resident weights and workspace on the current GPU."""

    def __init__(self, weights: bytes, cfg: Cfg):
        L = load_library()
        self._L = L
        self.cfg = cfg
        self._blob = ctypes.create_string_buffer(weights, len(weights))
        h = ctypes.c_void_p()
        st = L.gnntrk_create(self._blob, len(weights), ctypes.byref(cfg), ctypes.byref(h))
        if st != 0:
            raise GnntrkError(st, L.gnntrk_last_error(None).decode())
        self._h = h

    def _check(self, st):
        if st != 0:
            raise GnntrkError(st, self._L.gnntrk_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.gnntrk_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def find_tracks(self, n_events: int, n_hits: int, hits_xyz, plane, offsets, out_labels,
                    stream=None):
        """Enqueue the hot path on `stream` (torch.cuda.Stream or raw handle).

        hits_xyz: float32 CUDA tensor [3, n_hits]; plane: uint8 [n_hits];
        offsets: int64 [n_events + 1]; out_labels: int32 [n_hits].
        """
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
        self._check(self._L.gnntrk_find_tracks(self._h, n_events, n_hits, _ptr(hits_xyz),
                                               _ptr(plane), _ptr(offsets), _ptr(out_labels),
                                               ctypes.c_void_p(s)))

    def find_tracks_triplets(self, n_events: int, n_hits: int, hits_xyz, plane, offsets,
                             out_labels, out_event_tracks, out_track_off, out_track_hits,
                             stream=None):
        """The hot path plus the triplet stage (handle created with
        cfg.triplets). out_event_tracks: int32 [n_events + 1];
        out_track_off: int64 [max_tracks + 1]; out_track_hits: int32
        [max_track_hits] (CUDA tensors; capacities from their sizes)."""
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
        self._check(self._L.gnntrk_find_tracks_triplets(
            self._h, n_events, n_hits, _ptr(hits_xyz), _ptr(plane), _ptr(offsets),
            _ptr(out_labels), _ptr(out_event_tracks), _ptr(out_track_off), _ptr(out_track_hits),
            out_track_off.numel() - 1, out_track_hits.numel(), ctypes.c_void_p(s)))

    def embed_amax(self, hits_xyz, stream=None) -> np.ndarray:
        """Max calibration: the largest |input| of every embedding layer over
        the hits of hits_xyz (float32 CUDA tensor [3, n_hits])."""
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
        out = np.zeros(self.cfg.n_embed_layers, np.float32)
        self._check(self._L.gnntrk_embed_amax(self._h, hits_xyz.shape[1], _ptr(hits_xyz),
                                              out.ctypes.data_as(ctypes.c_void_p),
                                              ctypes.c_void_p(s)))
        return out

    def set_embed_scales(self, alpha):
        """Ranges alpha of the INT8 embedding's layer inputs (scale alpha / 127)."""
        a = np.ascontiguousarray(alpha, np.float32)
        self._check(self._L.gnntrk_set_embed_scales(self._h, a.ctypes.data_as(ctypes.c_void_p),
                                                    a.size))

    def triplet_stats(self) -> dict:
        out = np.zeros(6, np.int64)
        self._check(self._L.gnntrk_triplet_stats(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return {"articulations": int(out[0]), "elbows": int(out[1]), "kept": int(out[2]),
                "tracks": int(out[3]), "track_hits": int(out[4]), "capacity": int(out[5])}

    def get_triplets(self, event: int) -> dict:
        """Triplets of one event of the last triplet call: 'type' (0 articulation,
        1 left elbow, 2 right elbow), 'hits' [n, 3] = (A, C, B), 'logit', 'kept'."""
        n = ctypes.c_int64(0)
        st = self._L.gnntrk_get_triplets(self._h, event, 0, None, None, None, None,
                                         ctypes.byref(n))
        if st not in (0, 4):
            self._check(st)
        nt = n.value
        ty = np.zeros(nt, np.int32)
        h3 = np.zeros((nt, 3), np.int32)
        lg = np.zeros(nt, np.float32)
        kp = np.zeros(nt, np.uint8)
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        self._check(self._L.gnntrk_get_triplets(self._h, event, nt, p(ty), p(h3), p(lg), p(kp),
                                                ctypes.byref(n)))
        return {"type": ty, "hits": h3, "logit": lg, "kept": kp}

    def sync_status(self, stream=None):
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
        self._check(self._L.gnntrk_sync_status(self._h, ctypes.c_void_p(s)))

    def stats(self) -> dict:
        out = np.zeros(10, np.int64)
        self._check(self._L.gnntrk_stats(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return {"edges": int(out[0]), "kept": int(out[1]), "band": int(out[2]),
                "rerun_events": int(out[3]), "events": int(out[4]), "hits": int(out[5]),
                "edge_capacity": int(out[6]), "launches": int(out[7]),
                "rescore_edges": int(out[8]), "rescore_hits": int(out[9])}

    def rescore_rows(self) -> dict:
        """Rows the FP32 re-score recomputed, per step: 'edges'[0] / 'hits'[0]
        the encoders, [k + 1] message-passing step k."""
        n = 18
        e = np.zeros(n, np.int64)
        v = np.zeros(n, np.int64)
        self._check(self._L.gnntrk_rescore_rows(self._h, n, e.ctypes.data_as(ctypes.c_void_p),
                                                v.ctypes.data_as(ctypes.c_void_p)))
        k = self.cfg.iters
        return {"edges": e[:k + 1].tolist(), "hits": v[:k + 1].tolist()}

    def autotune(self, n_events: int, n_hits: int, hits_xyz, plane, offsets, out_labels,
                 stream=None) -> dict:
        """Tune the tensor-core launch configuration on this call's data."""
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
        ch = np.zeros(8, np.int32)
        self._check(self._L.gnntrk_autotune(self._h, n_events, n_hits, _ptr(hits_xyz),
                                            _ptr(plane), _ptr(offsets), _ptr(out_labels),
                                            ctypes.c_void_p(s),
                                            ch.ctypes.data_as(ctypes.c_void_p)))
        return dict(zip(TUNING_KEYS, (int(v) for v in ch)))

    def set_tuning(self, choice: dict):
        """Apply a launch configuration (the dict autotune returns) without timing."""
        ch = np.zeros(8, np.int32)
        for i, k in enumerate(TUNING_KEYS):
            ch[i] = int(choice.get(k, 0))
        self._check(self._L.gnntrk_set_tuning(self._h, ch.ctypes.data_as(ctypes.c_void_p)))

    def selftest_wait(self, max_cycles: int, stream=None):
        """Test hook: a bounded device wait that runs out and latches a timeout."""
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
        self._check(self._L.gnntrk_selftest_wait(self._h, int(max_cycles), ctypes.c_void_p(s)))

    def set_profiling(self, enable: bool):
        self._check(self._L.gnntrk_set_profiling(self._h, int(bool(enable))))

    def stage_times(self) -> dict:
        """{stage: (total device ms, runs)} accumulated since profiling was enabled."""
        n = self._L.gnntrk_stage_times(self._h, 0, None, None, None)
        if n < 0:
            raise GnntrkError(1, "stage_times failed")
        names = ctypes.create_string_buffer(32 * max(n, 1))
        ms = np.zeros(max(n, 1), np.float64)
        runs = np.zeros(max(n, 1), np.int64)
        self._L.gnntrk_stage_times(self._h, n, names, ms.ctypes.data_as(ctypes.c_void_p),
                                   runs.ctypes.data_as(ctypes.c_void_p))
        out = {}
        for i in range(n):
            nm = names.raw[32 * i:32 * i + 32].split(b"\0")[0].decode()
            out[nm] = (float(ms[i]), int(runs[i]))
        return out

    def get_graph(self, event: int) -> dict:
        """Rough graph of one event of the last call (host numpy arrays)."""
        n = ctypes.c_int64(0)
        st = self._L.gnntrk_get_graph(self._h, event, 0, None, None, None, None, None,
                                      ctypes.byref(n))
        if st not in (0, 4):
            self._check(st)
        ne = n.value
        src, dst = np.zeros(ne, np.int32), np.zeros(ne, np.int32)
        d2, lg = np.zeros(ne, np.float32), np.zeros(ne, np.float32)
        kept = np.zeros(ne, np.uint8)
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        self._check(self._L.gnntrk_get_graph(self._h, event, ne, p(src), p(dst), p(d2), p(lg),
                                             p(kept), ctypes.byref(n)))
        return {"src": src, "dst": dst, "d2": d2, "logit": lg, "kept": kept}


def run_batch(tracker: Tracker, batch, device="cuda", stream=None, check=True):
    """Copy a host `synth.Batch` to the device, find tracks, return labels (numpy)."""
    import torch
    xyz = torch.from_numpy(batch.xyz_soa()).to(device)
    plane = torch.from_numpy(batch.plane).to(device)
    offs = torch.from_numpy(batch.offsets).to(device)
    labels = torch.full((batch.n_hits,), -7, dtype=torch.int32, device=device)
    tracker.find_tracks(batch.n_events, batch.n_hits, xyz, plane, offs, labels, stream)
    if check:
        tracker.sync_status(stream)
    return labels.cpu().numpy()


def run_batch_triplets(tracker: Tracker, batch, device="cuda", stream=None, tracks_per_hit=2,
                       hits_per_hit=8):
    """As run_batch, with the triplet stage: returns (labels, tracks) where
    tracks[e] is the list of event e's tracks (numpy arrays of event-local
    input indices)."""
    import torch
    xyz = torch.from_numpy(batch.xyz_soa()).to(device)
    plane = torch.from_numpy(batch.plane).to(device)
    offs = torch.from_numpy(batch.offsets).to(device)
    labels = torch.full((batch.n_hits,), -7, dtype=torch.int32, device=device)
    ev_t = torch.zeros(batch.n_events + 1, dtype=torch.int32, device=device)
    t_off = torch.zeros(tracks_per_hit * batch.n_hits + 2, dtype=torch.int64, device=device)
    t_hits = torch.zeros(hits_per_hit * batch.n_hits + 16, dtype=torch.int32, device=device)
    tracker.find_tracks_triplets(batch.n_events, batch.n_hits, xyz, plane, offs, labels, ev_t,
                                 t_off, t_hits, stream)
    tracker.sync_status(stream)
    ev_t, t_off, t_hits = ev_t.cpu().numpy(), t_off.cpu().numpy(), t_hits.cpu().numpy()
    tracks = [[t_hits[t_off[t]:t_off[t + 1]] for t in range(ev_t[e], ev_t[e + 1])]
              for e in range(batch.n_events)]
    return labels.cpu().numpy(), tracks


def tracker_for_workload(wl: dict, precision=None, **kw) -> Tracker:
    """A Tracker for a workload of workloads.json (seeded random weights, or
    the trained blob the workload names)."""
    from . import synth
    prec = precision if precision is not None else wl.get("precision", "fp32")
    band = float(wl.get("rescore_band_score", 0.0)) if prec != "fp32" else 0.0
    args = dict(k_max=wl["k_max"], score_cut=wl["cut"], precision=prec, rescore_band=band)
    if wl.get("triplets"):
        args.update(triplets=True, triplet_cut=float(wl.get("triplet_cut", 0.5)))
    args.update(kw)
    cfg = make_cfg(wl["model"], wl["radius2"], **args)
    return Tracker(synth.workload_weights(wl), cfg)


def components_noalloc(n_hits: int, src, dst, kept, out_labels, stream=None):
    """Component labels of one graph with no allocation (CUDA tensors in/out);
    see gnntrk_components_noalloc in include/gnntrk.h."""
    L = load_library()
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
    st = L.gnntrk_components_noalloc(n_hits, 0 if src is None else src.numel(), _ptr(src),
                                     _ptr(dst), _ptr(kept), _ptr(out_labels), ctypes.c_void_p(s))
    if st != 0:
        raise GnntrkError(st, L.gnntrk_last_error(None).decode())


def tc_throughput(n: int, iters: int = 20000) -> float:
    """TFLOP/s the tensor cores sustain on back-to-back BF16 MMAs of M = 128,
    N = n, K = 16 (one issuing thread per SM); see gnntrk_tc_throughput."""
    L = load_library()
    ms = ctypes.c_double(0.0)
    st = L.gnntrk_tc_throughput(n, iters, ctypes.byref(ms))
    if st != 0:
        raise GnntrkError(st, L.gnntrk_last_error(None).decode())
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return sms * iters * 4 * 2.0 * 128 * n * 16 / (ms.value / 1e3) / 1e12


def workspace_bytes(cfg: Cfg) -> int:
    return int(load_library().gnntrk_workspace_bytes(ctypes.byref(cfg)))


def serve_run(weights: bytes, cfg: Cfg, batch, arrival_s, n_slots: int = 4,
              max_events_per_batch: int = 512, max_hits_per_batch: int = 1 << 20,
              memory_budget_bytes: int = 40_000_000_000, tuning: dict | None = None):
    """Run the continuous-batching server over a host `synth.Batch` whose events
    arrive at `arrival_s` (seconds); `tuning` is a dict `Tracker.autotune`
    returned, applied to every slot. Returns (labels, done_s, stats)."""
    L = load_library()
    sc = ServeCfg(n_slots, max_events_per_batch, max_hits_per_batch, memory_budget_bytes)
    if tuning is not None:
        sc.apply_tuning = 1
        for i, k in enumerate(TUNING_KEYS):
            sc.tuning[i] = int(tuning.get(k, 0))
    xyz = np.ascontiguousarray(batch.xyz_soa(), np.float32)
    plane = np.ascontiguousarray(batch.plane, np.uint8)
    offs = np.ascontiguousarray(batch.offsets, np.int64)
    arr = np.ascontiguousarray(arrival_s, np.float64)
    labels = np.full(batch.n_hits, -7, np.int32)
    done = np.zeros(batch.n_events, np.float64)
    stats = np.zeros(8, np.int64)
    blob = ctypes.create_string_buffer(weights, len(weights))
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    st = L.gnntrk_serve_run(blob, len(weights), ctypes.byref(cfg), ctypes.byref(sc),
                            batch.n_events, p(offs), p(xyz), p(plane), p(arr), p(labels),
                            p(done), p(stats))
    if st != 0:
        raise GnntrkError(st, L.gnntrk_last_error(None).decode())
    names = ["batches", "slots", "failed_batches", "max_in_flight", "slot_bytes",
             "largest_batch", "wall_us"]
    return labels, done, dict(zip(names, (int(v) for v in stats[:7])))


def poisson_arrivals(n: int, rate_hz: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process: exponential gaps, seeded."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_hz, n))


def cut_logit(score_cut: float) -> float:
    return math.log(score_cut / (1.0 - score_cut))


def _check_global(L, st):
    if st != 0:
        raise GnntrkError(st, L.gnntrk_last_error(None).decode())


def e4m3_encode(values, stream=None):
    """FP8-E4M3 codes of `values` through the library: a numpy array is
    converted on the host (the weight-packing routine), a CUDA tensor on the
    device (the activation conversion of the tensor-core kernels)."""
    L = load_library()
    if isinstance(values, np.ndarray):
        x = np.ascontiguousarray(values, np.float32).ravel()
        out = np.zeros(x.size, np.uint8)
        _check_global(L, L.gnntrk_e4m3_encode(x.ctypes.data_as(ctypes.c_void_p),
                                               out.ctypes.data_as(ctypes.c_void_p),
                                               x.size, 0, None))
        return out
    import torch
    x = values.contiguous().view(-1)
    out = torch.empty(x.numel(), dtype=torch.uint8, device=x.device)
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
    _check_global(L, L.gnntrk_e4m3_encode(ctypes.c_void_p(x.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr()), x.numel(), 1,
                                           ctypes.c_void_p(s)))
    return out


def e4m3_decode(codes) -> np.ndarray:
    """Values of FP8-E4M3 codes (host)."""
    L = load_library()
    c = np.ascontiguousarray(codes, np.uint8).ravel()
    out = np.zeros(c.size, np.float32)
    _check_global(L, L.gnntrk_e4m3_decode(c.ctypes.data_as(ctypes.c_void_p),
                                           out.ctypes.data_as(ctypes.c_void_p), c.size))
    return out
