"""kf_smooth_tracks against the FP64 smoother oracle on the same FP32 inputs.

Bars, at every layer a track reached: smoothed positions |dx| / r <= 1e-4,
momenta |dp_i| / |p| <= 1e-4 (the fit's bars); local covariance entries within
5e-3 of sqrt(Cf_ii Cf_jj), the forward filter's covariance at that layer: the
bar the fit's own covariance meets (test_fit_parity), which is what the
smoothed covariance inherits (relative to the smaller smoothed entries it
reads up to 30 times larger); layers reached exact; NaN beyond them and for
non-finite inputs."""
import numpy as np
import pytest

from paper_1705_02876_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


@pytest.fixture(scope="module")
def kf():
    from paper_1705_02876_gb300 import build, kf as kf_
    build.build()
    return kf_


@pytest.fixture(scope="module")
def ctx(kf):
    return kf.Context(0)


def _local_cov(state, cov):
    """[5][5][n] local covariance at each state's radial direction."""
    r = np.hypot(state[0], state[1])
    nx, ny = state[0] / r, state[1] / r
    n = state.shape[1]
    C = np.zeros((6, 6, n))
    k = 0
    for i in range(6):
        for j in range(i + 1):
            C[i, j] = C[j, i] = cov[k]
            k += 1
    P = np.zeros((5, 6, n))
    P[0, 0], P[0, 1] = -ny, nx
    for i in range(1, 5):
        P[i, i + 1] = 1.0
    return np.einsum("ian,abn,jbn->ijn", P, C, P)


def _compare(kf, ctx, oracle, b, opt=None):
    d = kf.to_device(b)
    out = kf.smooth_tracks(ctx, kf.GeometryArgs.of(b.geom), **d, opt=opt)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in out.items()}
    ref = oracle.smooth_batch(b)
    filt = oracle.fit_batch(b, per_layer=True)
    assert np.array_equal(g["reached"].astype(np.int32), ref["reached"])
    worst = dict(pos=0.0, mom=0.0, cov=0.0)
    for l in range(b.geom.n_layers):
        ok = ref["reached"] > l
        assert np.isnan(g["state"][l][:, ~ok]).all() and np.isnan(g["cov"][l][:, ~ok]).all()
        if not ok.any():
            continue
        gs, rs = g["state"][l][:, ok].astype(np.float64), ref["state"][l][:, ok]
        r = np.maximum(np.hypot(rs[0], rs[1]), 1.0)
        p = np.linalg.norm(rs[3:], axis=0)
        worst["pos"] = max(worst["pos"], (np.abs(gs[:3] - rs[:3]) / r).max())
        worst["mom"] = max(worst["mom"], (np.abs(gs[3:] - rs[3:]) / p).max())
        Lg = _local_cov(rs, g["cov"][l][:, ok].astype(np.float64))
        Lr = _local_cov(rs, ref["cov"][l][:, ok])
        Lf = _local_cov(rs, filt["layer_cov"][l][:, ok])
        df = np.sqrt(np.abs(np.einsum("iin->in", Lf)))
        worst["cov"] = max(worst["cov"], (np.abs(Lg - Lr) / (df[:, None] * df[None, :])).max())
    assert worst["pos"] <= 1e-4 and worst["mom"] <= 1e-4 and worst["cov"] <= 5e-3, worst
    return g, ref, worst


def test_smoother_parity_workload(kf, ctx, oracle):
    _compare(kf, ctx, oracle, synth.workload("parity"))


def test_smoother_ragged_missing_hits(kf, ctx, oracle):
    _compare(kf, ctx, oracle, synth.workload("ragged", scale=0.02))


def test_smoother_fp32_only(kf, ctx, oracle):
    _compare(kf, ctx, oracle, synth.workload("parity"), opt=kf.options(precision_mode=kf.PRECISION_FP32))


def test_smoother_stops(kf, ctx, oracle):
    """Loopers and tracks leaving the barrel stop early (routed precision: the
    loopers below 0.25 GeV update in FP64, as the fit's parity bar needs)."""
    b = synth.make_fit_batch(40, [1500], pt_lo=0.2, pt_hi=2.0, eta_max=2.0)
    g, ref, _ = _compare(kf, ctx, oracle, b)
    assert (ref["reached"] < b.geom.n_layers).any()


def test_smoother_nonfinite_input(kf, ctx, oracle):
    b = synth.make_fit_batch(41, [64])
    b.seed_state[2, 3] = np.nan
    b.hit_pos[4, 0, 7] = np.inf
    d = kf.to_device(b)
    out = kf.smooth_tracks(ctx, kf.GeometryArgs.of(b.geom), **d)
    torch.cuda.synchronize()
    for t in (3, 7):
        assert int(out["reached"][t]) == 0 and torch.isnan(out["state"][:, :, t]).all()
        assert int(out["flags"][t]) & 8
    ref = oracle.smooth_batch(b)
    assert ref["reached"][3] == 0 and ref["reached"][7] == 0


def test_smoother_full_size_sampled(kf, ctx, oracle):
    """The fit workload (100 events x 20,000 tracks) smoothed in one launch, as
    the benchmark runs it; 2,000 sampled tracks against the oracle's smoother
    at every layer, with the bars above."""
    b = synth.workload("fit")
    out = kf.smooth_tracks(ctx, kf.GeometryArgs.of(b.geom), **kf.to_device(b))
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    sel = np.sort(rng.choice(b.n_tracks, 2000, replace=False))
    idx = torch.from_numpy(sel).cuda()
    g = dict(state=out["state"][:, :, idx].cpu().numpy(), cov=out["cov"][:, :, idx].cpu().numpy(),
             reached=out["reached"][idx].cpu().numpy())
    sub = synth.FitBatch(b.geom, b.seed_state[:, sel], b.seed_cov[:, sel], b.charge[sel],
                         b.hit_pos[:, :, sel], b.hit_cov[:, :, sel], b.hit_mask[sel],
                         np.array([0, len(sel)]), b.truth[:, :, sel], b.crossed[:, sel], b.vertex[:, sel])
    ref = oracle.smooth_batch(sub)
    filt = oracle.fit_batch(sub, per_layer=True)
    assert np.array_equal(g["reached"].astype(np.int32), ref["reached"])
    for l in range(b.geom.n_layers):
        ok = ref["reached"] > l
        if not ok.any():
            continue
        gs, rs = g["state"][l][:, ok].astype(np.float64), ref["state"][l][:, ok]
        r = np.maximum(np.hypot(rs[0], rs[1]), 1.0)
        p = np.linalg.norm(rs[3:], axis=0)
        assert (np.abs(gs[:3] - rs[:3]) / r).max() <= 1e-4
        assert (np.abs(gs[3:] - rs[3:]) / p).max() <= 1e-4
        Lg = _local_cov(rs, g["cov"][l][:, ok].astype(np.float64))
        Lr = _local_cov(rs, ref["cov"][l][:, ok])
        Lf = _local_cov(rs, filt["layer_cov"][l][:, ok])
        df = np.sqrt(np.abs(np.einsum("iin->in", Lf)))
        assert (np.abs(Lg - Lr) / (df[:, None] * df[None, :])).max() <= 5e-3
