"""kf_fit_tracks_host (host buffers: read and written in place when every
buffer is page-locked, else chunked copies overlapping the fit) against
kf_fit_tracks on the same inputs: the same kernel on the same tracks, so the
outputs agree bit for bit; and against the oracle."""
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


def _device_fit(kf, ctx, b, opt):
    r = kf.fit_tracks(ctx, kf.GeometryArgs.of(b.geom), **kf.to_device(b), opt=opt)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in r.items()}


@pytest.mark.parametrize("chunk,pin,pin_out", [(96, True, True), (0, True, True), (0, True, False),
                                               (0, False, False), (200, False, False)])
def test_host_fit_equals_device_fit(kf, ctx, chunk, pin, pin_out):
    """chunk 0 with every buffer pinned is the in-place path; a pageable
    buffer anywhere sends chunk 0 to the chunked copies."""
    b = synth.workload("ragged", scale=0.02)  # 17 layers, missing hits, uneven events
    opt = kf.options(tracks_per_block=64, reg_cap=128, hit_prefetch=1)
    ref = _device_fit(kf, ctx, b, opt)
    out = kf.fit_outputs_host(b.n_tracks, pin=pin_out)
    kf.fit_tracks_host(ctx, kf.GeometryArgs.of(b.geom), **kf.to_host(b, pin=pin), opt=opt, chunk_tracks=chunk,
                       out=out)
    for k in ref:
        assert np.array_equal(out[k].numpy(), ref[k], equal_nan=True), k


def test_host_fit_matches_oracle(kf, ctx, oracle):
    b = synth.workload("parity")
    out = kf.fit_tracks_host(ctx, kf.GeometryArgs.of(b.geom), **kf.to_host(b), chunk_tracks=128)
    ref = oracle.fit_batch(b)
    st = out["state"].numpy().astype(np.float64)
    r = np.maximum(np.hypot(ref["state"][0], ref["state"][1]), 1.0)
    p = np.linalg.norm(ref["state"][3:], axis=0)
    assert (np.abs(st[:3] - ref["state"][:3]) / r <= 1e-4).all()
    assert (np.abs(st[3:] - ref["state"][3:]) / p <= 1e-4).all()
    assert np.array_equal(out["ndof"].numpy(), ref["ndof"])


def test_host_fit_arguments(kf, ctx):
    b = synth.workload("parity", scale=0.05)
    with pytest.raises(kf.KFError, match="chunk_tracks"):
        kf.fit_tracks_host(ctx, kf.GeometryArgs.of(b.geom), **kf.to_host(b, pin=False), chunk_tracks=-1)
    empty = synth.make_fit_batch(0, [0])
    out = kf.fit_tracks_host(ctx, kf.GeometryArgs.of(empty.geom), **kf.to_host(empty, pin=False))
    assert out["state"].shape == (6, 0)
