"""The seeded synthetic-event generator against the recipe it implements
(straight tracks from a beam spot through 26 planes, acceptance 5-45 mm,
98 % hit efficiency, 12 um smearing, uniform noise, shuffled hits, close
pairs with shared hits) and its reproducibility contract. CPU only."""
import numpy as np

from paper_2508_07423_gb300 import synth


def test_event_subsets_regenerate_on_their_own():
    tracks = {"kind": "poisson", "mean": 150, "min": 20, "max": 400}
    whole = synth.gen_batch(6, 77, tracks, 0.05)
    part = synth.gen_batch(2, 77, tracks, 0.05, first_event=3)
    sub = whole.subset([3, 4])
    for f in ("x", "y", "z", "plane", "pid"):
        assert np.array_equal(getattr(part, f), getattr(sub, f)), f
    assert np.array_equal(part.offsets, sub.offsets)


def test_hits_follow_the_detector_recipe():
    rng = np.random.default_rng(5)
    ev = synth.gen_event(rng, 300, 0.05)
    sig = ev.pid >= 0
    r = np.hypot(ev.x, ev.y)
    # z is the plane's position; the smearing is 12 um, so r stays within
    # the acceptance up to a few sigma
    assert np.array_equal(ev.z, synth.PLANE_Z[ev.plane].astype(np.float32))
    assert r[sig].min() > synth.R_MIN - 0.1 and r[sig].max() < synth.R_MAX + 0.1
    assert r[~sig].min() >= synth.R_MIN - 1e-4 and r[~sig].max() <= synth.R_MAX + 1e-4
    # noise = round(5 % of the signal hits)
    assert (~sig).sum() == int(round(0.05 * sig.sum()))
    # a track leaves at most one hit per plane, and hits are shuffled
    key = ev.pid[sig].astype(np.int64) * 64 + ev.plane[sig]
    assert np.unique(key).size == key.size
    assert not np.all(np.diff(ev.plane.astype(int)) >= 0)
    # straight lines: the hits of one track lie on a line in (x, z) and (y, z)
    for p in np.unique(ev.pid[sig])[:40]:
        m = ev.pid == p
        if m.sum() < 4:
            continue
        for coord in (ev.x[m], ev.y[m]):
            fit = np.polyfit(ev.z[m].astype(float), coord.astype(float), 1)
            resid = coord - np.polyval(fit, ev.z[m].astype(float))
            assert np.abs(resid).max() < 0.1


def test_hit_efficiency_and_sizes():
    # mean hits per event of the Poisson(150) workload, about 1690
    tracks = {"kind": "poisson", "mean": 150, "min": 20, "max": 400}
    b = synth.gen_batch(40, 11, tracks, 0.05)
    mean_hits = b.n_hits / b.n_events
    assert 1450 < mean_hits < 1950
    # about 98 % of the plane crossings inside the acceptance leave a hit:
    # a track's hits span consecutive planes with few gaps
    gaps, spans = 0, 0
    for e in range(b.n_events):
        ev = b.event(e)
        for p in np.unique(ev.pid[ev.pid >= 0]):
            pl = np.sort(ev.plane[ev.pid == p].astype(int))
            spans += pl[-1] - pl[0] + 1
            gaps += pl[-1] - pl[0] + 1 - pl.size
    assert 0.005 < gaps / spans < 0.04


def test_pair_fraction_zero_is_the_plain_generator():
    a = synth.gen_event(np.random.default_rng(9), 120, 0.05)
    b = synth.gen_event(np.random.default_rng(9), 120, 0.05, pair_frac=0.0)
    for f in ("x", "y", "z", "plane", "pid"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    assert a.pid2 is None


def test_close_pairs_share_hits():
    ev = synth.gen_event(np.random.default_rng(3), 150, 0.05, pair_frac=0.1)
    assert ev.pid2 is not None
    shared = ev.pid2 >= 0
    assert shared.any()
    # a shared hit belongs to a mother track (pid) and its partner (pid2), on
    # a plane where the partner left no hit of its own
    assert np.all(ev.pid[shared] >= 0)
    for i in np.nonzero(shared)[0]:
        partner = ev.pid2[i]
        own = (ev.pid == partner) & (ev.plane == ev.plane[i])
        assert not own.any()
    # partner tracks are the last 15 ids (round(0.1 * 150)) and never mothers
    n_tracks = 150
    assert ev.pid2[shared].min() >= n_tracks and ev.pid2[shared].max() < n_tracks + 15
    assert ev.pid[shared].max() < n_tracks
