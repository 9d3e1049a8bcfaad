"""gnntrk_components_noalloc: component labelling with no allocation.

Some callers cannot allocate device memory -- a host framework that owns all
device memory and forbids allocations inside its algorithms, or a real-time
path that may not pay for one. For them the library offers a component
labelling call whose scratch is a fixed array in device memory. This test
calls it through the C ABI on graphs that gnntrk_find_tracks built, twice in a
row (a large graph, then a smaller one, so stale scratch from the first call
would show), and checks that it reproduces gnntrk_find_tracks' labels exactly
(labels are integers: the tolerance is zero).

The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

import paper_2508_07423_gb300 as pkg
from paper_2508_07423_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def call_noalloc(L, n, src, dst, kept, out, stream=0):
    return L.gnntrk_components_noalloc(n, src.numel(), src.data_ptr(), dst.data_ptr(),
                                       None if kept is None else kept.data_ptr(),
                                       out.data_ptr(), ctypes.c_void_p(stream))


def test_noalloc_matches_find_tracks_on_two_calls():
    from paper_2508_07423_gb300 import build
    build.build()
    L = pkg.load_library()
    wl = synth.workload("cfg1_plain_fp32")
    big = synth.gen_batch(1, 4321, {"kind": "fixed", "n": 300}, 0.05)
    small = synth.workload_batch(wl, 1, first_event=7)
    batch = synth.concat([big, small])
    tr = pkg.tracker_for_workload(wl, max_hits=batch.n_hits, max_events=2, edges_per_hit=64)
    labels = pkg.run_batch(tr, batch)
    for e in (0, 1):
        g = tr.get_graph(e)
        a, z = int(batch.offsets[e]), int(batch.offsets[e + 1])
        n = z - a
        src = torch.from_numpy(g["src"]).cuda()
        dst = torch.from_numpy(g["dst"]).cuda()
        kept = torch.from_numpy(g["kept"]).cuda()
        out = torch.full((n,), -5, dtype=torch.int32, device="cuda")
        assert call_noalloc(L, n, src, dst, kept, out) == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.array_equal(got, labels[a:z]), f"event {e}"
        # the graph has real components, not only singletons
        assert len(np.unique(got)) < n
    tr.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L = pkg.load_library()
    z = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = call_noalloc(L, pkg.NOALLOC_MAX_HITS + 1, z, z, None, z)
    assert st == 1
    assert b"at most" in L.gnntrk_last_error(None)


def test_noalloc_rejects_edges_without_vertices():
    L = pkg.load_library()
    z = torch.zeros(4, dtype=torch.int32, device="cuda")
    st = L.gnntrk_components_noalloc(0, 4, z.data_ptr(), z.data_ptr(), None, z.data_ptr(),
                                     ctypes.c_void_p(0))
    assert st == 1
    assert b"n_hits == 0" in L.gnntrk_last_error(None)
