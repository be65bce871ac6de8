"""Pins of the seeding oracle (triplets of hits on the first three layers):

* the triplet-circle function against an independent circumcentre
  computation, and closed forms (a circle through the origin has d0 = 0; a
  circle of radius R centred at distance R + d has d0 = d);
* the oracle's triplet set equals a vectorised brute force over every
  (h0, h1, h2) of a small event, written separately from the definitions;
* on events the generator made, every track with hits on the three seed
  layers is found, and the charge from the turning sense matches the
  generated charge wherever the circle's curvature is resolved (above the
  pT where both charges are seeded).
"""
import numpy as np
import pytest

from paper_1705_02876_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")
K = 0.00299792458


def _circumcentre(p0, p1, p2):
    ax, ay = p0
    bx, by = p1
    cx, cy = p2
    d = 2 * (ax * (by - cy) + bx * (cy - ay) + cx * (ay - by))
    ux = ((ax * ax + ay * ay) * (by - cy) + (bx * bx + by * by) * (cy - ay) + (cx * cx + cy * cy) * (ay - by)) / d
    uy = ((ax * ax + ay * ay) * (cx - bx) + (bx * bx + by * by) * (ax - cx) + (cx * cx + cy * cy) * (bx - ax)) / d
    return np.array([ux, uy]), np.hypot(ax - ux, ay - uy)


def test_triplet_circle(oracle):
    rng = np.random.default_rng(1)
    for _ in range(200):
        c = rng.normal(0, 50, 2)
        R = np.hypot(*c) + rng.uniform(-5, 5)
        ang = rng.uniform(0, 2 * np.pi) + np.sort(rng.uniform(0, 1.5, 3))
        pts = [c + R * np.array([np.cos(a), np.sin(a)]) for a in ang]
        k, d0, orient = oracle.triplet_circle(*pts)
        cc, rr = _circumcentre(*pts)
        assert abs(abs(k) - 1 / rr) <= 1e-9 / rr
        assert abs(d0 - abs(np.hypot(*cc) - rr)) <= 1e-8 * max(1.0, rr)
        assert np.sign(k) == np.sign(orient)
    for R, d in ((40.0, 0.0), (500.0, 0.05), (3000.0, 0.3), (1e6, 0.02)):
        c = np.array([R + d, 0.0])
        pts = [c + R * np.array([np.cos(np.pi - a), np.sin(np.pi - a)]) for a in (4 / R, 8 / R, 12 / R)]
        k, d0, _ = oracle.triplet_circle(*pts)
        assert abs(d0 - d) <= 1e-9 * max(R, 1.0) + 1e-12, (R, d, d0)
        assert abs(abs(k) - 1 / R) <= 1e-6 / R


def _brute(ev, opt):
    """Every (h0, h1, h2) of each event tested against the definitions,
    vectorised, with the circle from its circumcentre."""
    g = ev.geom
    hp = ev.seed_hit_pos.astype(np.float64)
    off = ev.seed_hit_offsets
    bz = float(np.float32(g.bz))
    Rl = np.asarray(g.radii[:3], dtype=np.float32).astype(np.float64)
    rmin = opt["pt_min"] / (K * abs(bz))
    win = lambda a, b: (np.arcsin(min(1, Rl[b] / (2 * rmin))) - np.arcsin(min(1, Rl[a] / (2 * rmin)))
                        + opt["d0_max"] * (1 / Rl[a] + 1 / Rl[b]))
    wrap = lambda d: np.remainder(d + np.pi, 2 * np.pi) - np.pi
    out = []
    for e in range(off.shape[0]):
        i0, i1, i2 = (np.arange(off[e, l], off[e, l + 1]) for l in range(3))
        h0, h1, h2 = np.meshgrid(i0, i1, i2, indexing="ij")
        h0, h1, h2 = h0.ravel(), h1.ravel(), h2.ravel()
        x = [hp[0, h] for h in (h0, h1, h2)]
        y = [hp[1, h] for h in (h0, h1, h2)]
        z = [hp[2, h] for h in (h0, h1, h2)]
        r = [np.hypot(a, b) for a, b in zip(x, y)]
        f = [np.arctan2(b, a) for a, b in zip(x, y)]
        ok = (np.abs(wrap(f[1] - f[0])) <= win(0, 1)) & (np.abs(wrap(f[2] - f[1])) <= win(1, 2))
        ok &= np.abs((z[0] * r[1] - z[1] * r[0]) / (r[1] - r[0])) <= opt["z0_max"]
        ok &= np.abs(z[2] - (z[1] + (z[1] - z[0]) * (r[2] - r[1]) / (r[1] - r[0]))) <= opt["dz_max"]
        ax, ay, bx, by = x[0][ok], y[0][ok], x[1][ok], y[1][ok]
        cx, cy = x[2][ok], y[2][ok]
        d = 2 * (ax * (by - cy) + bx * (cy - ay) + cx * (ay - by))
        ux = ((ax * ax + ay * ay) * (by - cy) + (bx * bx + by * by) * (cy - ay) + (cx * cx + cy * cy) * (ay - by)) / d
        uy = ((ax * ax + ay * ay) * (cx - bx) + (bx * bx + by * by) * (ax - cx) + (cx * cx + cy * cy) * (bx - ax)) / d
        rr = np.hypot(ax - ux, ay - uy)
        good = (K * abs(bz) * rr >= opt["pt_min"]) & (np.abs(np.hypot(ux, uy) - rr) <= opt["d0_max"])
        sel = np.nonzero(ok)[0][good]
        out.append(np.stack([np.full(len(sel), e), h0[sel], h1[sel], h2[sel]], axis=1))
    t = np.concatenate(out)
    return t[np.lexsort((t[:, 3], t[:, 1], t[:, 2], t[:, 0]))]


@pytest.mark.parametrize("loose", [False, True])
def test_oracle_equals_brute_force(oracle, loose):
    """With loose cuts many random triplets reach the azimuth windows' edges,
    so the windows themselves are compared too."""
    ev = synth.make_build_events(51, 2, 30, noise_factor=2, seed_layer_hits=True)
    opt = dict(oracle.SEED_DEFAULTS)
    if loose:
        opt.update(d0_max=2.0, z0_max=20.0, dz_max=5.0)
    a = oracle.seed_triplets(ev, **opt)
    b = _brute(ev, opt)
    assert len(a) > 40
    sa, sb = {tuple(r) for r in a}, {tuple(r) for r in b}
    assert sa == sb, (len(sa - sb), len(sb - sa))


def test_every_seedable_track_found_with_its_charge(oracle):
    ev = synth.make_build_events(52, 2, 300, seed_layer_hits=True)
    t = oracle.seed_triplets(ev)
    trk = ev.seed_hit_track
    true = (trk[t[:, 1]] >= 0) & (trk[t[:, 1]] == trk[t[:, 2]]) & (trk[t[:, 2]] == trk[t[:, 3]])
    found = set(trk[t[true, 1]].tolist())
    assert found <= set(ev.seed_track.tolist())
    assert len(found) >= 0.99 * ev.n_seeds, (len(found), ev.n_seeds)
    charge = dict(zip(ev.seed_track.tolist(), ev.seed_fit.charge.tolist()))
    hp = ev.seed_hit_pos.astype(np.float64)
    bz = float(ev.geom.bz)
    kamb = K * abs(bz) / oracle.SEED_DEFAULTS["pt_both_charges"]
    agree = both = 0
    for row in t[true]:
        k, d0, orient = oracle.triplet_circle(*(hp[:2, h] for h in row[1:]))
        q = 1 if orient * bz < 0 else -1
        if abs(k) <= kamb:  # straight within the hits' resolution: both charges are seeded
            both += 1
            agree += 1
        else:
            agree += q == charge[int(trk[row[1]])]
    assert agree >= 0.995 * true.sum(), (agree, true.sum(), both)
    assert both < 0.9 * true.sum()


def _exact_triplets(pt_lo, pt_hi, n=64, seed=3):
    """Noiseless helices (no smearing, no scattering) through the toy barrel's
    three seed layers, with the seed layers' hits as the seeding input."""
    from types import SimpleNamespace
    geom = synth.toy_geometry(3, bz=3.75)  # exact in FP32, the precision the library takes Bz in
    rng = np.random.default_rng(seed)
    vertex, q = synth.draw_vertex_tracks(rng, n, pt_lo, pt_hi, "uniform", 1.0, vtx_sigma_xy=0.0)
    sim = synth.simulate(rng, rng, rng, geom, vertex, q, smear=False, ms=False)
    assert (sim["hit_mask"] == 7).all()
    hp = np.concatenate([sim["hit_pos"][l] for l in range(3)], axis=1)
    hc = np.concatenate([sim["hit_cov"][l] for l in range(3)], axis=1)
    ev = SimpleNamespace(geom=geom, seed_hit_pos=hp, seed_hit_cov=hc)
    trip = np.stack([np.zeros(n, np.int64), np.arange(n), n + np.arange(n), 2 * n + np.arange(n)], axis=1)
    return ev, trip, q, sim["truth"][0]


def test_seed_start_on_exact_helices(oracle):
    """Three exact points of a helix fix its circle: the seed's pT is the
    generated pT, its transverse direction the helix's tangent at the first
    hit, its charge the generated one, and its tan(lambda) the helix's up to
    the chord-to-arc ratio; the start lies 1 cm before the first hit along
    that tangent and the covariance has the stated relative sigmas."""
    o = dict(pt_min=0.3, pt_both_charges=2.0, pt_unresolved=6.0, p_sigma_resolved=0.3, p_sigma_unresolved=1.0)
    ev, trip, q, t0 = _exact_triplets(0.5, 1.9)
    r = oracle.seed_fit_inputs(ev, trip, **o)
    assert len(r["key"]) == len(trip)  # resolved: one charge each
    idx = r["key"][:, 1]
    st = r["seed_state"]
    pt_true = np.hypot(t0[3, idx], t0[4, idx])
    pt = np.hypot(st[3], st[4])
    np.testing.assert_allclose(pt, pt_true, rtol=1e-9)
    np.testing.assert_array_equal(r["charge"], q[idx])
    np.testing.assert_allclose(st[3] / pt, t0[3, idx] / pt_true, atol=1e-9)
    np.testing.assert_allclose(st[4] / pt, t0[4, idx] / pt_true, atol=1e-9)
    hp0 = ev.seed_hit_pos[:, idx]
    np.testing.assert_allclose(st[0], hp0[0] - st[3] / pt, atol=1e-12)
    np.testing.assert_allclose(st[1], hp0[1] - st[4] / pt, atol=1e-12)
    tl_true = t0[5, idx] / pt_true
    np.testing.assert_allclose(st[5] / pt, tl_true, rtol=2e-3)
    assert (np.abs(st[5] / pt) >= np.abs(tl_true)).all()  # the chord is shorter than the arc
    np.testing.assert_allclose(st[2], hp0[2] - st[5] / pt, atol=1e-12)
    diag = r["seed_cov"][[0, 2, 5, 9, 14, 20]]
    np.testing.assert_allclose(diag[3:], (0.3 * st[3:]) ** 2 + 1e-6, rtol=1e-12)
    np.testing.assert_allclose(diag[:3], (0.1 * st[:3]) ** 2 + 1e-8, rtol=1e-12)
    assert np.count_nonzero(r["seed_cov"]) == 6 * len(trip)


def test_seed_start_of_straight_triplets(oracle):
    """Above pt_both_charges the three hits do not resolve the curvature:
    both charges are seeded, each starting at pt_unresolved with the
    unresolved momentum sigma, and each turning its own way over the first
    chord."""
    ev, trip, q, t0 = _exact_triplets(20.0, 50.0, n=32)
    r = oracle.seed_fit_inputs(ev, trip, pt_unresolved=5.0, p_sigma_unresolved=0.8)
    assert len(r["key"]) == 2 * len(trip)
    assert (r["key"][0::2, 1] == r["key"][1::2, 1]).all() and (r["key"][0::2, 4] == -1).all()
    st = r["seed_state"]
    pt = np.hypot(st[3], st[4])
    np.testing.assert_allclose(pt, 5.0, rtol=1e-12)
    np.testing.assert_allclose(r["seed_cov"][9], (0.8 * st[3]) ** 2 + 1e-6, rtol=1e-12)
    # the two starts differ by twice the half turning angle of a 5 GeV circle over the chord
    hp = ev.seed_hit_pos
    idx = r["key"][0::2, 1]
    chord = np.hypot(hp[0, trip[:, 2]] - hp[0, trip[:, 1]], hp[1, trip[:, 2]] - hp[1, trip[:, 1]])[idx]
    half = np.arcsin(0.5 * chord * K * float(ev.geom.bz) / 5.0)
    cosang = (st[3, 0::2] * st[3, 1::2] + st[4, 0::2] * st[4, 1::2]) / 25.0
    np.testing.assert_allclose(np.arccos(np.clip(cosang, -1, 1)), 2 * half, rtol=1e-6)
    # a negative charge turns counter-clockwise in Bz > 0: its start direction is clockwise of the chord's
    cross = st[3, 0::2] * st[4, 1::2] - st[4, 0::2] * st[3, 1::2]
    assert (cross > 0).all()
