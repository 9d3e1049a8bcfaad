"""Track-finding metrics of the thesis (Sec. "Track Reconstruction Performance
Metrics"): efficiency, ghost rate, clone rate, hit purity and hit efficiency.

TEST INFRASTRUCTURE (part of the oracle package).

Definitions followed here:
  * a particle is reconstructible when it left at least 3 hits;
  * a track candidate is a component of the purified graph (or a track of the
    triplet track building) with at least `min_len` hits (3 by default);
  * a hit two particles share counts as a hit of both;
  * a track is matched to the particle that contributed most of its hits when
    that particle contributed at least 70 % of them (noise hits count against
    the match); otherwise the track is a ghost (fake);
  * efficiency = reconstructed particles / reconstructible particles, a particle
    being reconstructed when at least one track is matched to it;
  * ghost rate = fake tracks / all tracks;
  * clone rate = clone tracks / all tracks, a clone being every matched track
    beyond the first one matched to the same particle;
  * hit purity = hits from the matched particle / track hits, averaged over
    matched tracks;
  * hit efficiency = hits from the matched particle / hits of that particle,
    averaged over matched tracks.
"""
from __future__ import annotations

from collections import Counter
from dataclasses import dataclass


@dataclass
class Counts:
    reconstructible: int = 0
    reconstructed: int = 0
    tracks: int = 0
    ghosts: int = 0
    clones: int = 0
    matched_tracks: int = 0
    purity_sum: float = 0.0
    hit_eff_sum: float = 0.0

    def __iadd__(self, o: "Counts") -> "Counts":
        for k in self.__dataclass_fields__:
            setattr(self, k, getattr(self, k) + getattr(o, k))
        return self

    def summary(self) -> dict:
        def ratio(a, b):
            return a / b if b else 0.0
        return {
            "efficiency": ratio(self.reconstructed, self.reconstructible),
            "ghost_rate": ratio(self.ghosts, self.tracks),
            "clone_rate": ratio(self.clones, self.tracks),
            "hit_purity": ratio(self.purity_sum, self.matched_tracks),
            "hit_efficiency": ratio(self.hit_eff_sum, self.matched_tracks),
            "tracks": self.tracks,
            "reconstructible": self.reconstructible,
        }


def track_counts(tracks, pid, pid2=None, min_len: int = 3, match_frac: float = 0.7) -> Counts:
    """Metrics counts of one event from its track candidates.

    tracks: iterable of hit-index lists (a hit may belong to several tracks);
    pid: particle id per hit, -1 for noise; pid2: the second particle of a hit
    two particles share (-1 otherwise) or None. A shared hit counts as a hit of
    both particles, for their hit totals and for the match votes.
    """
    pid = [int(v) for v in pid]
    p2 = [-1] * len(pid) if pid2 is None else [int(v) for v in pid2]
    particle_hits: Counter = Counter()
    for a, b in zip(pid, p2):
        if a >= 0:
            particle_hits[a] += 1
        if b >= 0:
            particle_hits[b] += 1
    reconstructible = {p for p, n in particle_hits.items() if n >= 3}

    c = Counts(reconstructible=len(reconstructible))
    matched_count: Counter = Counter()
    for hits in tracks:
        if len(hits) < min_len:
            continue
        c.tracks += 1
        votes: Counter = Counter()
        for i in hits:
            votes[pid[i]] += 1
            if p2[i] >= 0:
                votes[p2[i]] += 1
        # the best real particle; noise (-1) never matches
        real = [(n, p) for p, n in votes.items() if p >= 0]
        if not real:
            c.ghosts += 1
            continue
        n_best, p_best = max(real, key=lambda t: (t[0], -t[1]))
        if n_best < match_frac * len(hits):
            c.ghosts += 1
            continue
        c.matched_tracks += 1
        matched_count[p_best] += 1
        c.purity_sum += n_best / len(hits)
        c.hit_eff_sum += n_best / particle_hits[p_best]
    c.reconstructed = sum(1 for p in matched_count if p in reconstructible)
    c.clones = sum(n - 1 for n in matched_count.values())
    return c


def event_counts(labels, pid, min_len: int = 3, match_frac: float = 0.7, pid2=None) -> Counts:
    """Metrics counts of one event from per-hit component labels and particle ids.

    labels: any per-hit component identifier; pid: particle id per hit, -1 for
    noise; each component is one track candidate.
    """
    members: dict[int, list[int]] = {}
    for i, lab in enumerate(labels):
        members.setdefault(int(lab), []).append(i)
    return track_counts(members.values(), pid, pid2, min_len, match_frac)


def batch_counts(labels, pid, offsets, min_len: int = 3, pid2=None) -> Counts:
    tot = Counts()
    for e in range(len(offsets) - 1):
        a, b = int(offsets[e]), int(offsets[e + 1])
        tot += event_counts(labels[a:b], pid[a:b], min_len,
                            pid2=None if pid2 is None else pid2[a:b])
    return tot


def batch_track_counts(tracks_per_event, pid, offsets, min_len: int = 3, pid2=None) -> Counts:
    """tracks_per_event[e]: event e's track candidates (event-local hit lists)."""
    tot = Counts()
    for e in range(len(offsets) - 1):
        a, b = int(offsets[e]), int(offsets[e + 1])
        tot += track_counts(tracks_per_event[e], pid[a:b],
                            None if pid2 is None else pid2[a:b], min_len)
    return tot
