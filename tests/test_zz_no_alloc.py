"""kf_fit_tracks_noalloc, the fit for callers that cannot allocate device
memory, against the FP64 oracle and against kf_fit_tracks on the same inputs.

Such callers (code inside a device-memory pool it does not own, loops that must
not allocate after start-up) cannot create a kf_context, whose creation calls
cudaMalloc.  The entry point keeps its only scratch, the persistent kernel's
work counter, in a fixed array of the library's device memory and clears it
on every call; two calls in a row check that the second call starts from a
cleared counter.  Two launch shapes: the default (64 tracks per block, no
register cap, hits prefetched into registers) and a shared-memory ring shape
(128 tracks per block, 128 registers, hits four layers ahead through
cp.async).  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

from paper_1705_02876_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

STOP = 1 | 2 | 8  # unreachable, left barrel, NaN input


def _close(a, b, ref_state, ref_flags=None):
    """The fit parity tolerances: positions |d| / r <= 1e-4, momenta |d| /
    |p| <= 1e-4, chi2 |d| <= 1e-3 max(chi2, ndof); ndof equal; flags equal
    (only the stop flags against the oracle, which has no routing flags)."""
    fa = a["flags"].view(np.uint32)
    if ref_flags is None:
        assert np.array_equal(fa, b["flags"].view(np.uint32))
        ok = (fa & 8) == 0
    else:
        assert np.array_equal(fa & STOP, ref_flags & STOP)
        ok = (ref_flags & 8) == 0
    assert np.array_equal(a["ndof"].astype(np.int32), b["ndof"].astype(np.int32))
    r = np.maximum(np.hypot(ref_state[0], ref_state[1]), 1.0)
    p = np.linalg.norm(ref_state[3:], axis=0)
    sa, sb = a["state"].astype(np.float64), b["state"].astype(np.float64)
    assert ((np.abs(sa[:3] - sb[:3]) / r)[:, ok] <= 1e-4).all()
    assert ((np.abs(sa[3:] - sb[3:]) / p)[:, ok] <= 1e-4).all()
    nd = b["ndof"].astype(np.float64)
    ca, cb = a["chi2"].astype(np.float64), b["chi2"].astype(np.float64)
    assert (np.abs(ca - cb) <= 1e-3 * np.maximum(np.maximum(cb, nd), 1.0))[ok].all()


@pytest.mark.parametrize("shape", [None, (128, 128, 4)])
def test_noalloc_matches_oracle_and_context_fit_twice(oracle, shape):
    from paper_1705_02876_gb300 import build, kf
    build.build()
    b = synth.make_fit_batch(41, [3000, 517, 20], geom=synth.toy_geometry(17), hit_eff=0.95)
    geom = kf.GeometryArgs.of(b.geom)
    dev = kf.to_device(b)
    opt = kf.options() if shape is None else kf.options(tracks_per_block=shape[0], reg_cap=shape[1],
                                                        hit_prefetch=shape[2])
    orc = oracle.fit_batch(b)
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
        _close(got, ref, orc["state"])
        _close(got, orc, orc["state"], ref_flags=orc["flags"])
    ctx.close()


def test_noalloc_rejects_bad_arguments():
    from paper_1705_02876_gb300 import build, kf
    build.build()
    b = synth.make_fit_batch(42, [64])
    dev = kf.to_device(b)
    out = kf.fit_outputs(b.n_tracks, dev["charge"].device)
    bad = synth.Geometry(b.geom.radii[::-1].copy(), b.geom.x_over_x0, b.geom.z_half, b.geom.bz)
    assert kf.fit_tracks_noalloc(kf.GeometryArgs.of(bad), **dev, out=out) == -1
    # a (block, cap, depth) combination that is not compiled in
    geom = kf.GeometryArgs.of(b.geom)
    assert kf.fit_tracks_noalloc(geom, **dev, out=out, opt=kf.options(reg_cap=168, tracks_per_block=256)) == -1
    assert kf.fit_tracks_noalloc(geom, **dev, out=out, opt=kf.options(hit_prefetch=2)) == -1
