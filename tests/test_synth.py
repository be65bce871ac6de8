"""The seeded input generator against the recipe it states (the toy detector of
Section 3.2 and the workloads' distributions), checked on the CPU from the
arrays alone: the geometry of the truth (crossings on the cylinders, and
without scattering on the helix of the vertex momentum), the smearing against
the stored hit covariance, the seed smear, momentum conservation through the
scattering kicks, hit efficiency, the ragged event sizes and the build events'
noise.  Both the oracle and the CUDA path consume these arrays, so a recipe
error here would be invisible to the parity tests."""
import math

import numpy as np
from scipy import stats

from paper_1705_02876_gb300 import synth


def test_deterministic_per_seed():
    a = synth.make_fit_batch(5, [300, 200])
    b = synth.make_fit_batch(5, [300, 200])
    c = synth.make_fit_batch(6, [300, 200])
    for k in ("seed_state", "seed_cov", "charge", "hit_pos", "hit_cov", "hit_mask"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k
    assert not np.array_equal(a.hit_pos, c.hit_pos)
    assert list(a.event_offsets) == [0, 300, 500]


def test_vertex_and_kinematics():
    b = synth.make_fit_batch(7, [20000])
    v = b.vertex
    assert abs(v[0].std() / 0.01 - 1) < 0.03 and abs(v[1].std() / 0.01 - 1) < 0.03
    assert abs(v[2].std() - 1) < 0.03
    pt = np.hypot(v[3], v[4])
    assert pt.min() >= 0.5 and pt.max() <= 10.0
    assert stats.kstest((pt - 0.5) / 9.5, "uniform").pvalue > 1e-3
    eta = np.arcsinh(v[5] / pt)
    assert np.abs(eta).max() <= 1.0
    assert stats.kstest((eta + 1) / 2, "uniform").pvalue > 1e-3
    phi = np.arctan2(v[4], v[3]) % (2 * math.pi)
    assert stats.kstest(phi / (2 * math.pi), "uniform").pvalue > 1e-3
    assert set(np.unique(b.charge)) == {-1, 1}
    assert abs((b.charge == 1).mean() - 0.5) < 0.02


def test_crossings_on_cylinders_and_helix_without_scattering():
    """With no material, every crossing lies on its cylinder and on the circle
    of radius pT / (k Bz) through the vertex, centred at
    (x0 + ty / omega, y0 - tx / omega) with omega = q k Bz / pT (a positive
    charge turns clockwise in Bz > 0), and z grows linearly with the turning
    angle: z - z0 = pz (phi / omega) / pT."""
    b = synth.make_fit_batch(8, [2000], ms=False)
    g, v, q = b.geom, b.vertex, b.charge.astype(np.float64)
    pt = np.hypot(v[3], v[4])
    tx, ty = v[3] / pt, v[4] / pt
    om = q * synth.K_FIELD * g.bz / pt
    cx, cy = v[0] + ty / om, v[1] - tx / om
    for l in range(g.n_layers):
        on = b.crossed[l]
        t = b.truth[l][:, on]
        assert np.allclose(np.hypot(t[0], t[1]), g.radii[l], rtol=0, atol=1e-9)
        R = 1 / np.abs(om[on])
        assert np.allclose(np.hypot(t[0] - cx[on], t[1] - cy[on]), R, rtol=1e-9)
        # momentum: transverse magnitude and pz unchanged, direction tangent
        assert np.allclose(np.hypot(t[3], t[4]), pt[on], rtol=1e-12)
        assert np.allclose(t[5], v[5][on], rtol=1e-12)
        # turning angle from the direction change, then z along the helix
        a0 = np.arctan2(ty[on], tx[on])
        a1 = np.arctan2(t[4], t[3])
        dphi = (a1 - a0 + math.pi) % (2 * math.pi) - math.pi  # |turn| < pi before the first crossing of r <= 40
        s = -dphi / om[on]
        assert (s > 0).all()
        assert np.allclose(t[2] - v[2][on], v[5][on] * s / pt[on], rtol=1e-8, atol=1e-8)


def test_scattering_keeps_momentum_magnitude():
    b = synth.make_fit_batch(9, [2000])
    p0 = np.sqrt((b.vertex[3:] ** 2).sum(0))
    for l in range(b.geom.n_layers):
        on = b.crossed[l]
        p = np.sqrt((b.truth[l][3:, on] ** 2).sum(0))
        assert np.allclose(p, p0[on], rtol=1e-12)
    # and the direction does change (scattering is on)
    on = b.crossed[-1]
    assert np.abs(b.truth[-1][5, on] - b.vertex[5, on]).max() > 1e-4


def test_hit_smearing_matches_stored_covariance():
    """Hit minus crossing, whitened by the stored V (radial 0.01, tangential
    0.01, z 0.1 cm), is a standard normal in each of its three components."""
    b = synth.make_fit_batch(10, [5000])
    for l in (0, 4, 9):
        on = b.crossed[l] & (((b.hit_mask >> np.uint32(l)) & np.uint32(1)) == 1)
        t = b.truth[l][:3, on]
        d = b.exact["hit_pos"][l][:, on] - t
        V = b.exact["hit_cov"][l][:, on]
        r = np.hypot(t[0], t[1])
        nx, ny = t[0] / r, t[1] / r
        # V's structure: n is an eigenvector with sigma_r^2, t with sigma_rphi^2
        vn_x = V[0] * nx + V[1] * ny
        vn_y = V[1] * nx + V[2] * ny
        assert np.allclose(vn_x, 1e-4 * nx, atol=1e-12) and np.allclose(vn_y, 1e-4 * ny, atol=1e-12)
        assert np.allclose(V[0] + V[2], 2e-4) and np.allclose(V[5], 1e-2)
        assert np.all(V[3] == 0) and np.all(V[4] == 0)
        wn = (d[0] * nx + d[1] * ny) / 0.01
        wt = (-d[0] * ny + d[1] * nx) / 0.01
        wz = d[2] / 0.1
        for w in (wn, wt, wz):
            assert abs(w.mean()) < 0.06 and abs(w.std() - 1) < 0.04


def test_seed_smear_and_covariance():
    b = synth.make_fit_batch(11, [20000])
    rel = b.exact["seed_state"] / b.vertex - 1
    assert np.all(np.abs(rel.std(1) - 0.1) < 0.004)
    floors = np.array([1e-4] * 3 + [1e-3] * 3)
    var = (0.1 * b.exact["seed_state"]) ** 2 + floors[:, None] ** 2
    for i, d in enumerate(synth.DIAG6):
        assert np.allclose(b.exact["seed_cov"][d], var[i], rtol=1e-12)
    off = [k for k in range(21) if k not in synth.DIAG6]
    assert np.all(b.exact["seed_cov"][off] == 0)


def test_hit_efficiency_and_mask():
    b = synth.make_fit_batch(12, [20000], geom=synth.toy_geometry(17), hit_eff=0.95)
    bits = ((b.hit_mask[None, :] >> np.arange(17, dtype=np.uint32)[:, None]) & np.uint32(1)).astype(bool)
    assert not (bits & ~b.crossed).any()  # no hit on a layer the track never reached
    share = bits[b.crossed].mean()
    assert abs(share - 0.95) < 0.005
    # a missing hit leaves zeros in its slots
    miss = b.crossed & ~bits
    assert np.all(b.hit_pos.transpose(1, 0, 2)[:, miss] == 0)


def test_ragged_event_sizes():
    s = synth.lognormal_event_sizes(3)
    assert len(s) == 256 and s.min() >= 500 and s.max() <= 50000
    assert 0.8 < np.median(s) / 5000 < 1.25
    ls = np.log(s[(s > 500) & (s < 50000)])
    assert abs(ls.std() - math.log(10) / 3) < 0.15


def test_build_events_noise_and_segments():
    ev = synth.make_build_events(13, 2, 400, noise_factor=10.0)
    Lb = ev.geom.n_layers - ev.n_seed_layers
    assert ev.hit_offsets.shape == (2, Lb + 1)
    assert ev.hit_offsets[0, 0] == 0 and ev.hit_offsets[-1, -1] == ev.hit_pos.shape[1]
    assert np.all(ev.hit_offsets[1:, 0] == ev.hit_offsets[:-1, -1])
    for e in range(2):
        for lb in range(Lb):
            lo, hi = ev.hit_offsets[e, lb], ev.hit_offsets[e, lb + 1]
            trk = ev.hit_track[lo:hi]
            noise = trk < 0
            assert noise.sum() == 4000
            # true hits of this event only, each track at most once per layer
            t = trk[~noise]
            assert np.all((t // 400) == e) and len(np.unique(t)) == len(t)
            p = ev.hit_pos[:, lo:hi][:, noise].astype(np.float64)
            r = ev.geom.radii[lb + ev.n_seed_layers]
            assert np.allclose(np.hypot(p[0], p[1]), r, rtol=1e-6)
            assert np.abs(p[2]).max() <= ev.geom.z_half
    # noise uniform in phi and z over one whole layer of both events
    sel = np.concatenate([np.arange(ev.hit_offsets[e, 5], ev.hit_offsets[e, 6]) for e in range(2)])
    sel = sel[ev.hit_track[sel] < 0]
    p = ev.hit_pos[:, sel].astype(np.float64)
    phi = np.arctan2(p[1], p[0]) % (2 * math.pi)
    assert stats.kstest(phi / (2 * math.pi), "uniform").pvalue > 1e-3
    assert stats.kstest((p[2] + ev.geom.z_half) / (2 * ev.geom.z_half), "uniform").pvalue > 1e-3
    # seeds: exactly the tracks with hits on all three seed layers
    bits = np.uint32(7)
    assert ev.n_seeds == len(ev.seed_track)
    assert np.all(ev.seed_fit.hit_mask == bits)
