"""The C ABI library loads and exports every entry point its header declares
(CPU only: no compute call)."""
import os
import re

import numpy as np
import pytest

import paper_2508_07423_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(gnntrk_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2508_07423_gb300 import build
    build.build()
    return pkg.load_library()


def test_library_exports_every_declared_symbol(lib):
    declared = header_functions()
    assert declared, "no declarations found"
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(pkg.EXPORTS) == declared, sorted(declared ^ set(pkg.EXPORTS))


def test_default_cfg_layout(lib):
    c = pkg.default_cfg()
    assert c.n_embed_layers == 3 and list(c.embed_dims[:4]) == [3, 64, 64, 4]
    assert c.hidden == 32 and c.iters == 4 and c.n_planes == 26 and c.k_max == 64
    assert abs(c.feat_scale[1] - 3.14159265) < 1e-6
    assert c.max_hits == 1 << 20 and c.max_events == 4096 and c.edges_per_hit == 24
    assert c.triplets == 0 and abs(c.triplet_cut - 0.5) < 1e-7 and c.triplets_per_hit == 16
    assert c.embed_int8 == 0


def test_create_rejects_bad_blob_without_gpu_work(lib):
    # argument and blob checks run before any device call
    c = pkg.default_cfg()
    with pytest.raises(pkg.GnntrkError) as ei:
        pkg.Tracker(b"\x00" * 8, c)
    assert ei.value.status == 6
    c.hidden = 48
    with pytest.raises(pkg.GnntrkError) as ei:
        pkg.Tracker(b"\x00" * 64, c)
    assert ei.value.status == 7


def test_host_e4m3_encoder_matches_the_oracle_codec():
    """The library's host E4M3 encoder (FP8 weight packing) against the
    oracle's brute-force codec: every code's value, the midpoints between
    neighbouring codes (ties to even), values past 448 and seeded randoms."""
    from oracle import quant
    dec = np.array([quant.e4m3_decode(c) for c in range(256)])
    fin = np.sort(np.unique(dec[~np.isnan(dec)]))
    mids = (fin[:-1] + fin[1:]) / 2
    rng = np.random.default_rng(17)
    vals = np.concatenate([fin, mids, [447.9, 448.0, 460.0, 1e9, -1e9, 2.0 ** -12],
                           rng.normal(0, 30, 4000), rng.uniform(-1e-2, 1e-2, 2000)]).astype(np.float32)
    got = pkg.e4m3_encode(vals)
    want = quant.e4m3_encode_array(vals.astype(np.float64))
    assert np.array_equal(got, want), np.flatnonzero(got != want)[:10]
    codes = np.arange(256, dtype=np.uint8)
    back = pkg.e4m3_decode(codes)
    ok = ~np.isnan(dec)
    assert np.array_equal(back[ok], dec[ok].astype(np.float32)) and np.isnan(back[~ok]).all()


def test_triplet_and_int8_arguments_rejected_without_gpu_work(lib):
    """cfg checks of the triplet stage and the INT8 embedding run before any
    device call."""
    from paper_2508_07423_gb300 import synth
    wl = synth.workload("cfg6_triplets")
    blob = synth.workload_weights(wl)
    for field, value in (("triplets", 2), ("triplet_cut", 1.5), ("triplets_per_hit", 0),
                         ("embed_int8", 3)):
        c = pkg.make_cfg(wl["model"], wl["radius2"], triplets=True)
        setattr(c, field, value)
        with pytest.raises(pkg.GnntrkError) as ei:
            pkg.Tracker(blob, c)
        assert ei.value.status == 1, field


def test_set_tuning_null_arguments_rejected_without_gpu_work(lib):
    import ctypes
    ch = (ctypes.c_int32 * 8)()
    assert lib.gnntrk_set_tuning(None, ch) == 1
    assert lib.gnntrk_set_tuning(None, None) == 1


def test_handle_less_errors_are_per_thread(lib):
    """gnntrk_last_error(NULL) reports the calling thread's own failure while
    other threads fail differently at the same time (no GPU work: the blob and
    cfg checks come first)."""
    import ctypes
    import threading
    bad_blob = pkg.default_cfg()
    bad_width = pkg.default_cfg()
    bad_width.hidden = 48
    cases = [(b"\x00" * 8, bad_blob, 6), (b"\x00" * 64, bad_width, 7)]
    errors = []

    def worker(blob, cfg, want):
        buf = ctypes.create_string_buffer(blob, len(blob))
        h = ctypes.c_void_p()
        first = None
        for _ in range(25):
            st = lib.gnntrk_create(buf, len(blob), ctypes.byref(cfg), ctypes.byref(h))
            msg = lib.gnntrk_last_error(None).decode()
            first = first or msg
            if st != want or msg != first:
                errors.append((want, st, msg, first))
                return

    threads = [threading.Thread(target=worker, args=c) for c in cases for _ in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors[:3]


def test_selftest_wait_null_handle_rejected_without_gpu_work(lib):
    assert lib.gnntrk_selftest_wait(None, 1000, None) == 1


def test_header_is_plain_c_and_links(lib, tmp_path):
    """include/gnntrk.h compiles as pedantic C99, and a C program linked
    against the library gets the documented defaults (no GPU work)."""
    import subprocess
    from paper_2508_07423_gb300 import LIB_PATH
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "use.c"
    src.write_text('#include "gnntrk.h"\n'
                   "int main(void) {\n"
                   "  gnntrk_cfg c;\n"
                   "  gnntrk_default_cfg(&c);\n"
                   "  if (c.hidden != 32 || c.iters != 4 || c.embed_dims[3] != 4) return 1;\n"
                   "  if (sizeof(gnntrk_cfg) != SZ_CFG || sizeof(gnntrk_serve_cfg) != SZ_SERVE)"
                   " return 3;\n"
                   "  return gnntrk_set_tuning(0, 0) == GNNTRK_ERR_INVALID_ARG ? 0 : 2;\n"
                   "}\n")
    libdir = os.path.dirname(LIB_PATH)
    exe = tmp_path / "use"
    import ctypes
    import paper_2508_07423_gb300 as pkg
    # the binding's struct mirrors have the C layout's sizes
    sizes = [f"-DSZ_CFG={ctypes.sizeof(pkg.Cfg)}", f"-DSZ_SERVE={ctypes.sizeof(pkg.ServeCfg)}"]
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                           *sizes,
                           "-I", os.path.join(root, "include"), str(src), "-L", libdir,
                           "-lgnntrk", f"-Wl,-rpath,{libdir}", "-o", str(exe)])
    assert subprocess.run([str(exe)]).returncode == 0
