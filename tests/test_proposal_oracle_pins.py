"""Pins of the build oracle's training log and learned proposal (CPU).

The features are pinned by what the geometry and the build fix: the layer
fraction and hole count against the build's own output, q/pT at the first
build layer against the seed (a uniform solenoid conserves pT), the window
bound (|dz| <= 3 sqrt(C_zz + sigma_z^2) makes |f2| <= 3 when the hits carry
the nominal resolution, and likewise the tangential residual), and unit-width
pulls of the true hits.  The labels are pinned against the surviving
candidates.  The scoring is pinned against the numpy network and the bfloat16
rounding against hand-worked values.
"""
import numpy as np
import pytest

from oracle import mlp_oracle
from paper_1705_02876_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


@pytest.fixture(scope="module")
def events(oracle):
    ev = synth.make_build_events(41, 2, 600)
    f = oracle.fit_seeds(ev)
    seeds = dict(state=f["state"].astype(np.float32), cov=f["cov"].astype(np.float32))
    return ev, seeds


@pytest.fixture(scope="module")
def best_hit(oracle, events):
    ev, seeds = events
    return oracle.build_events(ev, seeds=seeds, max_cands=1, log=True)


def test_log_leaves_build_unchanged(oracle, events, best_hit):
    ev, seeds = events
    plain = oracle.build_events(ev, seeds=seeds, max_cands=1)
    for k in ("hit", "chi2", "nhits", "state", "cov"):
        assert np.array_equal(plain[k], best_hit[k]), k


def test_log_structure_best_hit(events, best_hit):
    """N = 1: layer fraction and holes from the output; label-1 rows are
    exactly the assigned hits."""
    ev, _ = events
    lg = best_hit["log"]
    L = ev.build_geom.n_layers
    ref, f, y = lg["ref"], lg["features"], lg["labels"]
    s, slot, l, h = ref.T
    assert (slot == 0).all()
    assert np.array_equal(f[:, 10], l / L)
    hits = best_hit["hit"][:, 0, :]  # [S][L]
    before = np.cumsum(hits >= 0, axis=1) - (hits >= 0)  # hits on layers < l
    assert np.array_equal(f[:, 11], l - before[s, l])
    assert int(y.sum()) == int(best_hit["nhits"].sum())
    kept = {(a, b, c) for a, b, c in zip(s[y == 1], l[y == 1], h[y == 1])}
    out = {(a, b, int(hits[a, b])) for a in range(hits.shape[0]) for b in range(L) if hits[a, b] >= 0}
    assert kept == out


def test_log_labels_cover_surviving_hits(oracle, events):
    ev, seeds = events
    res = oracle.build_events(ev, seeds=seeds, max_cands=6, log=True)
    ref, y = res["log"]["ref"], res["log"]["labels"]
    kept = {(a, c, d) for a, c, d in zip(ref[y == 1, 0], ref[y == 1, 2], ref[y == 1, 3])}
    hits = res["hit"]
    for a in range(hits.shape[0]):
        for j in range(hits.shape[1]):
            for l in np.nonzero(hits[a, j] >= 0)[0]:
                assert (a, l, hits[a, j, l]) in kept
    assert 0.5 < y.mean() < 1.0


def test_log_window_bound(events, best_hit):
    """Hits with the nominal resolution: |f2| <= nsigma exactly and the
    tangential pull within the window up to the chord; noise fills it."""
    f = best_hit["log"]["features"]
    assert np.abs(f[:, 2]).max() <= 3.0 * (1 + 1e-6)
    assert np.abs(f[:, 1]).max() <= 3.0 * (1 + 1e-4)
    assert np.abs(f[:, 2]).max() > 2.8


def test_log_curvature_first_layer(events, best_hit):
    ev, seeds = events
    lg = best_hit["log"]
    s, _, l, _ = lg["ref"].T
    first = l == 0
    st = seeds["state"].astype(np.float64)
    pt = np.hypot(st[3], st[4])
    q = ev.seed_fit.charge.astype(np.float64) * np.sign(ev.build_geom.bz)
    expect = q[s[first]] / pt[s[first]]
    assert np.allclose(lg["features"][first, 9], expect, rtol=1e-9, atol=0)


def test_true_hit_pulls(events, best_hit):
    ev, _ = events
    lg = best_hit["log"]
    s, _, _, h = lg["ref"].T
    true = ev.hit_track[h] == ev.seed_track[s]
    f = lg["features"][true]
    assert len(f) > 5000
    w = [np.std(f[:, i]) for i in range(3)]
    assert 0.9 < w[0] < 1.1, w  # radial: S_nn = V_nn, the prediction lies on the cylinder
    assert 0.8 < w[1] < 1.2 and 0.8 < w[2] < 1.2, w
    assert np.all(np.abs(f[:, :3].mean(0)) < 0.1)


def test_bf16_rounding():
    from oracle import kf_oracle as o
    assert o.bf16_round(1.0) == 1.0
    assert o.bf16_round(1 + 2 ** -8) == 1.0  # tie to even
    assert o.bf16_round(1 + 3 * 2 ** -8) == 1 + 2 ** -6  # tie to even, upwards
    assert o.bf16_round(1 + 2 ** -8 + 2 ** -20) == 1 + 2 ** -7
    assert o.bf16_round(-3.14159) == -3.140625
    assert o.bf16_round(0.0) == 0.0


def test_logit_matches_network_definition():
    from oracle import kf_oracle as o
    rng = np.random.default_rng(3)
    w = mlp_oracle.init_params(rng)
    w[12 * 64:12 * 64 + 64] = rng.normal(0, 0.1, 64)  # nonzero biases
    X = rng.normal(0, 1, (20, 12))
    z = mlp_oracle.forward(w, X)[0]
    for i in range(20):
        assert o.mlp_logit(w, X[i]) == pytest.approx(z[i], rel=1e-12, abs=1e-12)
        zb = o.mlp_logit(w, X[i], bf16=True)
        assert abs(zb - z[i]) <= 0.05 * (1 + abs(z[i]))


def test_proposal_wider_than_any_window_is_exhaustive(oracle, events):
    ev, seeds = events
    plain = oracle.build_events(ev, seeds=seeds, max_cands=6)
    w = mlp_oracle.init_params(np.random.default_rng(5))
    prop = oracle.build_events(ev, seeds=seeds, max_cands=6, mlp=w, topk=10 ** 6)
    for k in ("hit", "chi2", "nhits"):
        assert np.array_equal(plain[k], prop[k]), k


def test_constant_network_keeps_lowest_hit(oracle, events, best_hit):
    """All logits equal: top-1 is the in-window hit with the lowest index;
    at the first layer (candidate = seed) the build keeps it or a hole, and
    keeps it whenever the exhaustive build kept it."""
    ev, seeds = events
    prop = oracle.build_events(ev, seeds=seeds, max_cands=1, mlp=np.zeros(5057), topk=1)
    lg = best_hit["log"]
    s, _, l, h = lg["ref"].T
    y = lg["labels"]
    S = ev.n_seeds
    lowest = np.full(S, -1)
    kept_plain = np.full(S, -1)
    for a, b, c, d in zip(s, l, h, y):
        if b != 0:
            continue
        if lowest[a] < 0 or c < lowest[a]:
            lowest[a] = c
        if d == 1:
            kept_plain[a] = c
    got = prop["hit"][:, 0, 0]
    assert np.all((got == lowest) | (got == -1))
    m = kept_plain == lowest
    assert np.array_equal(got[m & (lowest >= 0)], lowest[m & (lowest >= 0)])
    multi = np.bincount(s[l == 0], minlength=S) > 1
    assert multi.any()
