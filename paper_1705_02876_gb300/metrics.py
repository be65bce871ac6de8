"""Track-finding efficiency and fake rate of built candidates (Section 3.2).

The paper counts efficiency and fake rate with the rule that candidates
matching fewer than 7 hits of a simulated track count as neither.  Reading
taken here: per seed the best candidate (rank 0) is taken; it *matches* the
simulated track that owns at least half of its hits (seed hits included); it
is *counted* if it has at least 7 hits.  Efficiency = fraction of simulated
tracks with at least 7 hits (and a seed) matched by a counted candidate; fake
rate = fraction of counted candidates that match no simulated track.  Host-side
evaluation only, not part of the hot path.  hit_purity = fraction of the
build hits of the best candidates that belong to their seed's own simulated
track.
"""
from __future__ import annotations

import numpy as np


def efficiency_fake_rate(best_hits, seed_track, hit_track, track_nhits, n_seed_hits=3, min_hits=7,
                         eligible_tracks=None):
    """best_hits [S, L]: global hit index per build layer (-1 = none) of each
    seed's best candidate; seed_track [S]: the simulated track each seed came
    from (-1: a seed whose hits are not all from one simulated track, whose
    seed hits then count for no track); hit_track [H]: owner of each hit (-1 =
    noise); track_nhits: hits of every simulated track over all layers;
    eligible_tracks: the simulated tracks efficiency is measured on (default:
    the seeds' tracks with at least min_hits hits)."""
    best_hits = np.asarray(best_hits)
    seed_track = np.asarray(seed_track)
    S = best_hits.shape[0]
    owner = np.where(best_hits >= 0, np.asarray(hit_track)[np.maximum(best_hits, 0)], -2)
    n_build = (best_hits >= 0).sum(1)
    n_total = n_build + n_seed_hits
    own = (owner == seed_track[:, None]).sum(1) + np.where(seed_track >= 0, n_seed_hits, 0)
    # the majority owner of a candidate's hits is its seed's track whenever it
    # has at least half; otherwise look for another owner with half
    matched_track = np.full(S, -1, dtype=np.int64)
    ok = 2 * own >= n_total
    matched_track[ok] = seed_track[ok]
    rest = np.nonzero(~ok)[0]
    if len(rest) and best_hits.shape[1]:
        # most frequent owner per row: sort each row, run lengths from the
        # start index of each run of equal values
        o = np.sort(owner[rest], axis=1)
        L = o.shape[1]
        j = np.broadcast_to(np.arange(L), o.shape)
        new_run = np.ones_like(o, dtype=bool)
        new_run[:, 1:] = o[:, 1:] != o[:, :-1]
        start = np.maximum.accumulate(np.where(new_run, j, 0), axis=1)
        run = np.where(o >= 0, j - start + 1, 0)
        arg = run.argmax(axis=1)
        cnt = run[np.arange(len(rest)), arg]
        hit = (cnt > 0) & (2 * cnt >= n_total[rest])
        matched_track[rest[hit]] = o[np.arange(len(rest)), arg][hit]
    counted = n_total >= min_hits
    fake = counted & (matched_track < 0)
    if eligible_tracks is None:
        st = seed_track[seed_track >= 0]
        eligible = np.unique(st[np.asarray(track_nhits)[st] >= min_hits])
    else:
        et = np.asarray(eligible_tracks)
        eligible = np.unique(et[np.asarray(track_nhits)[et] >= min_hits])
    found = np.unique(matched_track[counted & (matched_track >= 0)])
    eff = np.isin(eligible, found).mean() if len(eligible) else float("nan")
    fake_rate = fake.sum() / max(counted.sum(), 1)
    assigned = best_hits >= 0
    purity = (owner == np.asarray(seed_track)[:, None])[assigned].mean() if assigned.any() else float("nan")
    return dict(efficiency=float(eff), fake_rate=float(fake_rate), n_counted=int(counted.sum()),
                n_eligible=int(len(eligible)), mean_hits=float(n_total.mean()) if S else float("nan"),
                hit_purity=float(purity))
