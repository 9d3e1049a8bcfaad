"""Planted mistakes in the oracle: each test compiles a copy of oracle.cpp with
one plausible mistake (a dropped term, a wrong sign, index or operand order)
and runs the oracle's pins against it in a child process; at least one pin
must fail. A control build of the unmodified source must pass them all, so a
failure means the pins caught the mistake, not that the harness broke.
CPU only; the shipped oracle is never modified."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.cpp")
# the pins (the slower stored-radius checks are left to the main run)
PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_triplets.py"]

# (name, [(text in oracle.cpp, planted replacement), ...]); every text must
# occur exactly once, so the list follows the source.
MUTANTS = [
    ("out_sum_by_dst", [("out_sum[size_t(src[e]) * h + c] += ",
                         "out_sum[size_t(dst[e]) * h + c] += ")]),
    ("message_slots_swapped", [("cat[h + c] = out_sum[size_t(l) * h + c];",
                                "cat[h + c] = in_sum[size_t(l) * h + c];"),
                               ("cat[2 * h + c] = in_sum[size_t(l) * h + c];",
                                "cat[2 * h + c] = out_sum[size_t(l) * h + c];")]),
    ("no_layer_norm", [("  linear(L1, in, t.data());\n  layer_norm(t);\n",
                        "  linear(L1, in, t.data());\n")]),
    ("unbiased_variance", [("var /= double(v.size());", "var /= double(v.size() - 1);")]),
    ("no_node_residual", [("for (int c = 0; c < h; ++c) H[size_t(l) * h + c] += delta[c];",
                           "for (int c = 0; c < h; ++c) H[size_t(l) * h + c] = delta[c];")]),
    ("no_edge_residual", [("for (int c = 0; c < h; ++c) E[size_t(e) * h + c] += delta[c];",
                           "for (int c = 0; c < h; ++c) E[size_t(e) * h + c] = delta[c];")]),
    ("dropped_bias", [("double acc = L.b[o];", "double acc = 0.0;")]),
    ("edge_net_dst_as_src", [("cat[2 * h + c] = H[size_t(dst[e]) * h + c];",
                              "cat[2 * h + c] = H[size_t(src[e]) * h + c];")]),
    ("radius_not_strict", [("if (d2 < r2) cand", "if (d2 <= r2) cand")]),
    ("next_plane_only", [("if (q != p + 1 && q != p + 2) continue;",
                          "if (q != p + 1) continue;")]),
    ("atan2_transposed", [("std::atan2(yd, xd)", "std::atan2(xd, yd)")]),
    ("components_directed", [("    adj[dst[e]].push_back(src[e]);\n", "")]),
    ("triplet_operands_swapped", [("cat[c] = e_final[size_t(e1[t]) * h + c];",
                                   "cat[c] = e_final[size_t(e2[t]) * h + c];"),
                                  ("cat[h + c] = e_final[size_t(e2[t]) * h + c];",
                                   "cat[h + c] = e_final[size_t(e1[t]) * h + c];")]),
    ("triplet_heads_swapped", [("const bool art = type[t] == 0;",
                                "const bool art = type[t] != 0;")]),
    ("shared_link_needs_both_forks", [("if (n_out[l.first] > 1 || n_in[l.second] > 1)",
                                       "if (n_out[l.first] > 1 && n_in[l.second] > 1)")]),
    ("articulations_join_groups", [("if (tkeep[t] && type[t] != 0) grp.unite(e1[t], e2[t]);",
                                    "if (tkeep[t]) grp.unite(e1[t], e2[t]);")]),
    ("embedding_relu_on_output", [("    if (l + 1 < m.embed.size())\n      for (double& v : o)",
                                   "    for (double& v : o)")]),
    ("kmax_keeps_farthest", [("    std::sort(cand.begin(), cand.end());\n    size_t keep",
                              "    std::sort(cand.rbegin(), cand.rend());\n    size_t keep")]),
    ("radius_feature_from_x_only", [("std::sqrt(xd * xd + yd * yd) / P.feat_scale[0]",
                                     "std::sqrt(xd * xd) / P.feat_scale[0]")]),
    ("elbow_order_ignores_plane", [("return std::make_pair(int(plane[far]), far);",
                                    "return std::make_pair(0, far);")]),
    ("triplets_from_cut_edges", [("    if (!keep[e]) continue;\n    out[src[e]].push_back",
                                  "    out[src[e]].push_back")]),
    ("elbows_counted_both_ways", [("for (size_t j = i + 1; j < O.size(); ++j) put(1, O[i], O[j]);",
                                   "for (size_t j = 0; j < O.size(); ++j) if (j != i) put(1, O[i], O[j]);")]),
]


def _build(tmp_path, edits):
    src = open(SRC).read()
    for old, new in edits:
        assert src.count(old) == 1, f"mutation site not found once: {old!r}"
        src = src.replace(old, new)
    cpp = tmp_path / "variant.cpp"
    cpp.write_text(src)
    so = tmp_path / "libvariant.so"
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-pthread", str(cpp),
                           "-o", str(so)])
    return so


def _run_pins(so):
    env = dict(os.environ, GNNTRK_ORACLE_LIB=str(so))
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           "-k", "not stored_radii", *PINS], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=900)


def test_unmodified_oracle_passes_the_pins(tmp_path):
    r = _run_pins(_build(tmp_path, []))
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("name,edits", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(name, edits, tmp_path):
    r = _run_pins(_build(tmp_path, edits))
    tail = r.stdout[-3000:]
    assert r.returncode == 1 and " failed" in tail, f"{name}: no pin failed\n{tail}"


# Planted mistakes in the oracle's Python parts (quantisers, track metrics):
# a copy of the oracle package with one edited file goes first on the path of
# the child process (the C++ library is the unmodified one).
PY_MUTANTS = [
    ("e4m3_ties_to_odd", "quant.py", [("if (pos[b] & 1) == 0]", "if (pos[b] & 1) == 1]")]),
    ("e4m3_subnormal_step", "quant.py", [("return sign * m * 2.0 ** -9",
                                          "return sign * m * 2.0 ** -10")]),
    ("int8_per_tensor_weight_scale", "quant.py", [("a = np.abs(W).max(axis=1)",
                                                   "a = np.full(W.shape[0], np.abs(W).max())")]),
    ("int8_round_half_up", "quant.py", [("q = np.rint(np.asarray(v, np.float32) * np.float32(inv_scale))",
                                         "q = np.floor(np.asarray(v, np.float32) * np.float32(inv_scale) + 0.5)")]),
    ("match_needs_more_than_70_percent", "metrics.py", [("if n_best < match_frac * len(hits):",
                                                         "if n_best <= match_frac * len(hits):")]),
    ("reconstructible_from_2_hits", "metrics.py", [("if n >= 3}", "if n >= 2}")]),
    ("shared_hit_votes_once", "metrics.py", [("            if p2[i] >= 0:\n                votes[p2[i]] += 1\n", "")]),
    ("clones_include_the_first", "metrics.py", [("c.clones = sum(n - 1 for n in matched_count.values())",
                                                 "c.clones = sum(n for n in matched_count.values())")]),
]


@pytest.mark.parametrize("name,fname,edits", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_planted_python_mistake_fails_a_pin(name, fname, edits, tmp_path):
    import oracle
    lib = oracle.build()
    pkg = tmp_path / "oracle"
    shutil.copytree(os.path.join(ROOT, "oracle"), pkg,
                    ignore=shutil.ignore_patterns("__pycache__", "*.so"))
    path = pkg / fname
    src = path.read_text()
    for old, new in edits:
        assert src.count(old) == 1, f"mutation site not found once: {old!r}"
        src = src.replace(old, new)
    path.write_text(src)
    env = dict(os.environ, GNNTRK_ORACLE_LIB=lib,
               PYTHONPATH=os.pathsep.join([str(tmp_path), ROOT]))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "-k", "not stored_radii", *[os.path.join(ROOT, p) for p in PINS]],
                       cwd=str(tmp_path), env=env,
                       capture_output=True, text=True, timeout=900)
    tail = r.stdout[-3000:]
    assert r.returncode == 1 and " failed" in tail, f"{name}: no pin failed\n{tail}"


def test_python_variant_harness_loads_the_copy(tmp_path):
    """Control of the harness: an unmodified copy passes, and a copy whose
    module raises on import is the one the child imports."""
    import oracle
    lib = oracle.build()
    pkg = tmp_path / "oracle"
    shutil.copytree(os.path.join(ROOT, "oracle"), pkg,
                    ignore=shutil.ignore_patterns("__pycache__", "*.so"))
    env = dict(os.environ, GNNTRK_ORACLE_LIB=lib,
               PYTHONPATH=os.pathsep.join([str(tmp_path), ROOT]))
    args = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
            "-k", "not stored_radii", *[os.path.join(ROOT, p) for p in PINS]]
    r = subprocess.run(args, cwd=str(tmp_path), env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-3000:]
    (pkg / "metrics.py").write_text("raise ImportError('variant copy imported')\n")
    r = subprocess.run(args, cwd=str(tmp_path), env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode != 0 and "variant copy imported" in r.stdout + r.stderr
