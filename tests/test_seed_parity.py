"""Seeding from hits on the GPU (kf_seed_triplets + kf_seed_fetch) against the
oracle, and the whole chain seeding -> seed fit -> build against the oracle
doing the same.

Seeds are compared by key (event, h0, h1, h2, charge).  The cuts decide an
integer in floating point, FP32 on the GPU and FP64 in the oracle, so the two
sets may differ only by seeds that lie within 1e-4 (relative) of a cut or of
the two-charge curvature; everything else is identical.  The seed fit's inputs
of the common seeds (but those within 1e-4 of the two-charge curvature, where
the start switches from the circle's pT to a fixed one) match within 5e-4 of
each component (1e-3 for the covariance, quadratic in the state).  The builds
from the two chains assign at least 99.5% of the hits identically, with
efficiency and fake rate within 0.5%, and find at least 95% of the tracks the
truth-seeded build is measured on.
"""
import numpy as np
import pytest

from paper_1705_02876_gb300 import metrics, synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]
K = 0.00299792458


@pytest.fixture(scope="module")
def kf():
    from paper_1705_02876_gb300 import build, kf as kf_
    build.build()
    return kf_


@pytest.fixture(scope="module")
def ctx(kf):
    return kf.Context(0)


def _t(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype=dt)


def _margin(ev, h, opt):
    """Smallest relative distance of a triplet's FP64 cut variables to their cuts."""
    from oracle import kf_oracle as o
    g = ev.geom
    hp = ev.seed_hit_pos.astype(np.float64)
    R = np.asarray(g.radii[:3], dtype=np.float32).astype(np.float64)
    bz = float(np.float32(g.bz))
    rmin = opt["pt_min"] / (K * abs(bz))
    win = lambda a, b: (np.arcsin(min(1, R[b] / (2 * rmin))) - np.arcsin(min(1, R[a] / (2 * rmin)))
                        + opt["d0_max"] * (1 / R[a] + 1 / R[b]))
    wrap = lambda d: np.remainder(d + np.pi, 2 * np.pi) - np.pi
    x, y, z = hp[0, h], hp[1, h], hp[2, h]
    r, f = np.hypot(x, y), np.arctan2(y, x)
    zv = (z[0] * r[1] - z[1] * r[0]) / (r[1] - r[0])
    zp = z[1] + (z[1] - z[0]) * (r[2] - r[1]) / (r[1] - r[0])
    k, d0, _ = o.triplet_circle(*(hp[:2, i] for i in h))
    kmax, kamb = K * abs(bz) / opt["pt_min"], K * abs(bz) / opt["pt_both_charges"]
    m = [abs(abs(wrap(f[1] - f[0])) / win(0, 1) - 1), abs(abs(wrap(f[2] - f[1])) / win(1, 2) - 1),
         abs(abs(zv) / opt["z0_max"] - 1), abs(abs(z[2] - zp) / opt["dz_max"] - 1),
         abs(abs(k) / kmax - 1), abs(d0 / opt["d0_max"] - 1), abs(abs(k) / kamb - 1)]
    return min(m)


def gpu_seeds(kf, ctx, ev, opt=None):
    out = kf.seed_triplets(ctx, kf.GeometryArgs.of(ev.geom.sub(0, 3)), ev.seed_hit_offsets,
                           _t(ev.seed_hit_pos, torch.float32), _t(ev.seed_hit_cov, torch.float32), opt=opt)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in out.items()}
    key = np.stack([g["event"], g["hits"][0], g["hits"][1], g["hits"][2], g["charge"]], axis=1).astype(np.int64)
    order = np.lexsort((key[:, 4], key[:, 3], key[:, 1], key[:, 2], key[:, 0]))
    return key[order], {k: (v[..., order] if k != "event" else v[order]) for k, v in g.items()}, out, order


def seed_tracks(ev, key):
    """The simulated track of each seed whose three hits share one, else -1."""
    t = ev.seed_hit_track[key[:, 1:4]]
    return np.where((t[:, 0] >= 0) & (t[:, 0] == t[:, 1]) & (t[:, 1] == t[:, 2]), t[:, 0], -1)


def _match(a, b):
    """Indices of the common keys (rows of a, rows of b) and the two sets' differences."""
    ka = {tuple(r): i for i, r in enumerate(a)}
    kb = {tuple(r): i for i, r in enumerate(b)}
    common = sorted(set(ka) & set(kb))
    return (np.array([ka[c] for c in common], dtype=np.int64), np.array([kb[c] for c in common], dtype=np.int64),
            set(ka) - set(kb), set(kb) - set(ka))


@pytest.fixture(scope="module")
def events():
    return synth.make_build_events(55, 2, 400, seed_layer_hits=True)


def test_seed_triplets_and_inputs(kf, ctx, oracle, events):
    ev = events
    opt = dict(oracle.SEED_DEFAULTS)
    key, g, _, _ = gpu_seeds(kf, ctx, ev)
    ref = oracle.seed_fit_inputs(ev, oracle.seed_triplets(ev), opt["pt_min"], opt["pt_both_charges"])
    ig, io, only_g, only_o = _match(key, ref["key"])
    assert len(ig) > ev.n_seeds
    for k in list(only_g) + list(only_o):
        assert _margin(ev, np.array(k[1:4]), opt) < 1e-4, k
    assert len(only_g) + len(only_o) <= 1e-3 * len(ig)
    assert np.array_equal(g["hit_pos"][..., ig], ref["hit_pos"][..., io].astype(np.float32))
    # the seed fit's inputs of the common seeds away from the two-charge curvature
    hp = ev.seed_hit_pos.astype(np.float64)
    kamb = K * abs(float(np.float32(ev.geom.bz))) / opt["pt_both_charges"]
    kap = np.array([oracle.triplet_circle(*(hp[:2, h] for h in ref["key"][j, 1:4]))[0] for j in io])
    sel = np.abs(np.abs(kap) / kamb - 1) > 1e-4
    assert sel.mean() > 0.999
    ig, io = ig[sel], io[sel]
    st_g, st_o = g["seed_state"][:, ig].astype(np.float64), ref["seed_state"][:, io]
    scale = np.maximum(np.abs(st_o), np.array([1, 1, 1, 0.1, 0.1, 0.1])[:, None])
    assert (np.abs(st_g - st_o) / scale).max() <= 5e-4
    assert (np.abs(g["seed_cov"][:, ig] - ref["seed_cov"][:, io]) <= 1e-3 * np.abs(ref["seed_cov"][:, io]) + 1e-12).all()


def test_seeded_chain_against_oracle(kf, ctx, oracle, events):
    """Seeding, the 3-layer seed fit and the build on the GPU against the oracle
    doing all three, on the common seeds."""
    ev = events
    opt = dict(oracle.SEED_DEFAULTS)
    key, g, dev, order = gpu_seeds(kf, ctx, ev)
    sg = ev.geom.sub(0, 3)
    fit = kf.fit_tracks(ctx, kf.GeometryArgs.of(sg), dev["seed_state"], dev["seed_cov"], dev["charge"],
                        dev["hit_pos"], dev["hit_cov"], dev["hit_mask"])
    bg = ev.build_geom
    bo = kf.build_tracks(ctx, kf.GeometryArgs.of(bg), ev.hit_offsets, _t(ev.hit_pos, torch.float32),
                         _t(ev.hit_cov, torch.float32), dev["event"], fit["state"], fit["cov"], dev["charge"])
    torch.cuda.synchronize()
    gb = {k: v.cpu().numpy() for k, v in bo.items()}
    ref = oracle.seed_fit_inputs(ev, oracle.seed_triplets(ev), opt["pt_min"], opt["pt_both_charges"])
    f32 = lambda v: np.asarray(v, dtype=np.float32).astype(np.float64)
    rf = oracle.fit_arrays(f32(sg.radii), f32(sg.x_over_x0), float(np.float32(sg.z_half)), float(np.float32(sg.bz)),
                           ref["seed_state"].astype(np.float32), ref["seed_cov"].astype(np.float32), ref["charge"],
                           ref["hit_pos"].astype(np.float32), ref["hit_cov"].astype(np.float32), ref["hit_mask"])
    rb = oracle.build_arrays(f32(bg.radii), f32(bg.x_over_x0), float(np.float32(bg.z_half)), float(np.float32(bg.bz)),
                             ev.hit_offsets, ev.hit_pos, ev.hit_cov, ref["event"], rf["state"].astype(np.float32),
                             rf["cov"].astype(np.float32), ref["charge"], max_cands=6)
    ig, io, _, _ = _match(key, ref["key"])
    hit_g = gb["hit"][order][ig]
    hit_o = rb["hit"][io]
    assert (hit_g == hit_o).mean() >= 0.995, (hit_g == hit_o).mean()
    # track finding from the hits alone, against the truth-seeded build
    m_g = metrics.efficiency_fake_rate(gb["hit"][order][:, 0], seed_tracks(ev, key), ev.hit_track, ev.track_nhits,
                                       eligible_tracks=ev.seed_track)
    m_o = metrics.efficiency_fake_rate(rb["hit"][:, 0], seed_tracks(ev, ref["key"]), ev.hit_track, ev.track_nhits,
                                       eligible_tracks=ev.seed_track)
    assert abs(m_g["efficiency"] - m_o["efficiency"]) <= 0.005 and abs(m_g["fake_rate"] - m_o["fake_rate"]) <= 0.005
    assert m_g["efficiency"] > 0.95, m_g


def test_seeding_arguments(kf, ctx, events):
    ev = events
    with pytest.raises(kf.KFError, match="three seed layers"):
        kf.seed_triplets(ctx, kf.GeometryArgs.of(ev.geom.sub(0, 4)), ev.seed_hit_offsets,
                         _t(ev.seed_hit_pos, torch.float32), _t(ev.seed_hit_cov, torch.float32))
    with pytest.raises(kf.KFError, match="pt_min"):
        kf.seed_triplets(ctx, kf.GeometryArgs.of(ev.geom.sub(0, 3)), ev.seed_hit_offsets,
                         _t(ev.seed_hit_pos, torch.float32), _t(ev.seed_hit_cov, torch.float32),
                         opt=kf.seeding(pt_min=0.0))


def test_triplet_buffer_overflow_rerun(kf, ctx, oracle):
    """A dense event (3,000 tracks, no noise) makes more triplets than the
    first search's buffer holds (4 per hit): the search runs again with a
    buffer sized by the count, and the set still matches the oracle's."""
    ev = synth.make_build_events(61, 1, 3000, noise_per_layer=0, seed_layer_hits=True, seed_noise_per_layer=0)
    opt = dict(oracle.SEED_DEFAULTS)
    ctx2 = kf.Context(0)  # a fresh context: the first search starts from the smallest buffer
    key, _, _, _ = gpu_seeds(kf, ctx2, ev)
    assert len(key) > max(65536, 4 * ev.seed_hit_pos.shape[1])  # the first buffer's size
    ref = oracle.seed_fit_inputs(ev, oracle.seed_triplets(ev), opt["pt_min"], opt["pt_both_charges"])
    ig, io, only_g, only_o = _match(key, ref["key"])
    for k in list(only_g) + list(only_o):
        assert _margin(ev, np.array(k[1:4]), opt) < 1e-4, k
    assert len(only_g) + len(only_o) <= 1e-3 * len(ig)
    ctx2.close()


def test_seeding_degenerate_inputs(kf, ctx, events):
    """No events; events with an empty seed layer (no triplet can form); an
    event with an empty middle layer next to a full one."""
    ev = events
    g3 = kf.GeometryArgs.of(ev.geom.sub(0, 3))
    hp, hc = _t(ev.seed_hit_pos, torch.float32), _t(ev.seed_hit_cov, torch.float32)
    out = kf.seed_triplets(ctx, g3, np.zeros((0, 4), np.int64), hp, hc)
    assert out["charge"].shape == (0,)
    # event 0 with its layer-2 hits cut off, event 1 with an empty middle layer
    off = ev.seed_hit_offsets.copy()
    a = off[0].copy()
    b = off[1].copy()
    rows = np.array([[a[0], a[1], a[2], a[2]], [a[2], a[2] + (b[1] - b[0]), a[2] + (b[1] - b[0]),
                                                   a[2] + (b[1] - b[0])]], np.int64)
    out = kf.seed_triplets(ctx, g3, rows, hp, hc)
    torch.cuda.synchronize()
    assert out["charge"].shape == (0,)
    # only the first event, intact: the same seeds as that event alone in the full search
    key_all, _, _, _ = gpu_seeds(kf, ctx, ev)
    out = kf.seed_triplets(ctx, g3, off[:1], hp, hc)
    torch.cuda.synchronize()
    n0 = int(out["charge"].shape[0])
    assert n0 == int((key_all[:, 0] == 0).sum()) and n0 > 0


def test_full_size_seeding_sampled(kf, ctx, oracle):
    """One event of the build workload as the bench seeds it (5,000 tracks,
    every track's hit on the seed layers, no added noise; about 360,000
    seeds): the whole triplet set against the oracle's, the seed inputs on
    3,000 sampled seeds."""
    ev = synth.make_build_events(4, 1, 5000, seed_layer_hits=True, seed_noise_per_layer=0)
    opt = dict(oracle.SEED_DEFAULTS)
    key, g, _, _ = gpu_seeds(kf, ctx, ev)
    trip = oracle.seed_triplets(ev)
    tk = {tuple(r) for r in trip[:, :4]}
    gk = {tuple(r) for r in key[:, :4]}
    for k in (tk ^ gk):
        assert _margin(ev, np.array(k[1:4]), opt) < 1e-4, k
    assert len(tk ^ gk) <= 1e-3 * len(tk) and len(tk) > 300000 // 2
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(len(trip), 3000, replace=False))
    ref = oracle.seed_fit_inputs(ev, trip[pick], opt["pt_min"], opt["pt_both_charges"])
    ig, io, _, only_o = _match(key, ref["key"])
    assert len(only_o) <= 1e-3 * len(ref["key"]) + 2
    hp = ev.seed_hit_pos.astype(np.float64)
    kamb = K * abs(float(np.float32(ev.geom.bz))) / opt["pt_both_charges"]
    kap = np.array([oracle.triplet_circle(*(hp[:2, h] for h in ref["key"][j, 1:4]))[0] for j in io])
    sel = np.abs(np.abs(kap) / kamb - 1) > 1e-4
    ig, io = ig[sel], io[sel]
    st_g, st_o = g["seed_state"][:, ig].astype(np.float64), ref["seed_state"][:, io]
    scale = np.maximum(np.abs(st_o), np.array([1, 1, 1, 0.1, 0.1, 0.1])[:, None])
    assert (np.abs(st_g - st_o) / scale).max() <= 5e-4
    assert (np.abs(g["seed_cov"][:, ig] - ref["seed_cov"][:, io]) <= 1e-3 * np.abs(ref["seed_cov"][:, io]) + 1e-12).all()
