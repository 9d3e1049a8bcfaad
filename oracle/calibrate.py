"""Pick the squared embedding radius of each workload and freeze it.

Each workload states a mean graph degree (2E/N over all hits) rather than a
radius. This script generates the workload's calibration events (their own
seed, distinct from the measured events), embeds them with the FP64 oracle,
collects the squared distances of every candidate pair (plane p to p+1 or p+2,
no k_max cap), and takes the squared radius halfway between the E-th and
(E+1)-th smallest value for E = round(degree * N / 2), rounded to float32. With
the strict comparison d^2 < r^2 exactly E candidate pairs of the calibration
set pass.

Run:  python -m oracle.calibrate            (rewrites the radius2 fields of
      paper_2508_07423_gb300/workloads.json; calls only the oracle and the
      seeded generators)
"""
from __future__ import annotations

import json
import sys

import numpy as np

import oracle
from paper_2508_07423_gb300 import synth


def calibrate(name: str, wl: dict) -> float:
    sh = synth.shape_of(wl)
    model = oracle.Model(synth.workload_weights(wl), sh.embed, sh.hidden, sh.iters)
    b = synth.workload_batch(wl, wl["calib_events"], seed_key="calib")
    d2 = []
    for e in range(b.n_events):
        ev = b.event(e)
        emb = oracle.embed(model, ev.x, ev.y, ev.z)
        d2.append(oracle.candidate_d2(ev.plane, emb))
    d2 = np.sort(np.concatenate(d2))
    target = int(round(wl["mean_degree"] * b.n_hits / 2))
    r2 = float(np.float32(0.5 * (d2[target - 1] + d2[target])))
    passed = int(np.count_nonzero(d2 < r2))
    print(f"{name}: N={b.n_hits} target E={target} r2={r2!r} passing={passed} "
          f"degree={2 * passed / b.n_hits:.3f}", file=sys.stderr)
    return r2


def main():
    with open(synth.WORKLOADS_PATH) as f:
        wls = json.load(f)
    for name, wl in wls.items():
        if wl.get("weights_file"):  # trained weights: the radius comes from training
            continue
        wl["radius2"] = calibrate(name, wl)
    with open(synth.WORKLOADS_PATH, "w") as f:
        json.dump(wls, f, indent=2)
        f.write("\n")


if __name__ == "__main__":
    main()
