"""Planted mistakes in the oracle: each test compiles a copy of oracle.cpp with
one plausible mistake (a dropped term, a wrong sign, index or operand order)
and runs the oracle's pins against it in a child process; at least one pin
must fail. A control build of the unmodified source must pass them all, so a
failure means the pins caught the mistake, not that the harness broke.
CPU only; the shipped oracle is never modified."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.cpp")
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
                           *PINS], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=900)


def test_unmodified_oracle_passes_the_pins(tmp_path):
    r = _run_pins(_build(tmp_path, []))
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("name,edits", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(name, edits, tmp_path):
    r = _run_pins(_build(tmp_path, edits))
    tail = r.stdout[-3000:]
    assert r.returncode == 1 and " failed" in tail, f"{name}: no pin failed\n{tail}"
