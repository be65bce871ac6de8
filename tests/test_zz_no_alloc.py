"""kf_fit_tracks_noalloc, the fit for callers that cannot allocate device
memory, against kf_fit_tracks on the same inputs.

Such callers (code inside a device-memory pool it does not own, loops that must
not allocate after start-up) cannot create a kf_context, whose creation calls
cudaMalloc.  The entry point keeps its only scratch, the persistent kernel's
work counter, in a fixed array of the library's device memory and clears it
on every call; two calls in a row check that the second call starts from a
cleared counter.  This file is collected last so that a run stopping at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_1705_02876_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


def _close(a, b, ref_state):
    """Same tolerances as the fit parity tests: positions |d| / r <= 1e-4,
    momenta |d| / |p| <= 1e-4, chi2 |d| <= 1e-3 max(chi2, ndof); ndof and flags
    equal."""
    assert np.array_equal(a["flags"], b["flags"])
    assert np.array_equal(a["ndof"], b["ndof"])
    ok = (b["flags"].view(np.uint32) & 8) == 0
    r = np.maximum(np.hypot(ref_state[0], ref_state[1]), 1.0)
    p = np.linalg.norm(ref_state[3:], axis=0)
    assert ((np.abs(a["state"][:3] - b["state"][:3]) / r)[:, ok] <= 1e-4).all()
    assert ((np.abs(a["state"][3:] - b["state"][3:]) / p)[:, ok] <= 1e-4).all()
    nd = b["ndof"].astype(np.float64)
    assert (np.abs(a["chi2"] - b["chi2"]) <= 1e-3 * np.maximum(np.maximum(b["chi2"], nd), 1.0))[ok].all()


def test_noalloc_matches_context_fit_twice():
    from paper_1705_02876_gb300 import build, kf
    build.build()
    b = synth.make_fit_batch(41, [3000, 517, 20], geom=synth.toy_geometry(17), hit_eff=0.95)
    geom = kf.GeometryArgs.of(b.geom)
    dev = kf.to_device(b)
    opt = kf.options()
    ctx = kf.Context(0)
    ref = kf.fit_tracks(ctx, geom, **dev, opt=opt)
    torch.cuda.synchronize()
    ref = {k: v.cpu().numpy() for k, v in ref.items()}
    for call in range(2):
        out = kf.fit_outputs(b.n_tracks, dev["charge"].device)
        for v in out.values():
            v.fill_(-7)
        rc = kf.fit_tracks_noalloc(geom, **dev, out=out, opt=opt)
        assert rc == kf.KF_OK, (call, rc)
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy() for k, v in out.items()}
        _close(got, ref, ref["state"])
    ctx.close()


def test_noalloc_rejects_bad_arguments():
    from paper_1705_02876_gb300 import build, kf
    build.build()
    b = synth.make_fit_batch(42, [64])
    dev = kf.to_device(b)
    out = kf.fit_outputs(b.n_tracks, dev["charge"].device)
    bad = synth.Geometry(b.geom.radii[::-1].copy(), b.geom.x_over_x0, b.geom.z_half, b.geom.bz)
    assert kf.fit_tracks_noalloc(kf.GeometryArgs.of(bad), **dev, out=out) == -1
