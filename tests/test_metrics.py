"""The efficiency / fake-rate counting against a per-candidate loop written
from the definitions (majority owner with at least half of the hits, counted
at 7 hits or more)."""
import numpy as np

from paper_1705_02876_gb300 import metrics


def _loop(best, seed_track, hit_track, track_nhits, n_seed=3, min_hits=7):
    found, fakes, counted = set(), 0, 0
    for s in range(best.shape[0]):
        hits = [h for h in best[s] if h >= 0]
        owners = [int(hit_track[h]) for h in hits]
        if seed_track[s] >= 0:
            owners += [int(seed_track[s])] * n_seed
        n_total = len(hits) + n_seed
        if n_total < min_hits:
            continue
        counted += 1
        cand = [o for o in set(owners) if o >= 0 and 2 * owners.count(o) >= n_total]
        if cand:
            # several owners with half: the seed's own track, else the smallest
            found.add(int(seed_track[s]) if seed_track[s] in cand else min(cand))
        else:
            fakes += 1
    eligible = sorted({int(t) for t in seed_track if t >= 0 and track_nhits[t] >= min_hits})
    eff = np.mean([t in found for t in eligible])
    return eff, fakes / max(counted, 1), counted


def test_counting_matches_loop():
    rng = np.random.default_rng(7)
    n_tracks, H, S, L = 400, 3000, 500, 10
    hit_track = rng.integers(-1, n_tracks, H)
    track_nhits = rng.integers(3, 14, n_tracks)
    seed_track = rng.integers(-1, n_tracks, S)
    best = np.where(rng.random((S, L)) < 0.7, rng.integers(0, H, (S, L)), -1)
    # make some candidates follow their seed's track
    own = [np.nonzero(hit_track == t)[0] for t in range(n_tracks)]
    for s in range(0, S, 3):
        t = seed_track[s]
        if t >= 0 and len(own[t]):
            k = rng.integers(0, L + 1)
            best[s, :k] = rng.choice(own[t], k)
    m = metrics.efficiency_fake_rate(best, seed_track, hit_track, track_nhits)
    eff, fake, counted = _loop(best, seed_track, hit_track, track_nhits)
    assert m["n_counted"] == counted
    assert np.isclose(m["efficiency"], eff) and np.isclose(m["fake_rate"], fake)
    assert 0.0 < fake < 1.0 and 0.0 < eff < 1.0
