"""kf_build_tracks_host, the build from and to host memory, against the
device build and the FP64 oracle, through the C interface.

The events are cut into batches whose uploads, builds and downloads overlap on
three streams; the build does not depend on the batching, so the outputs must
equal kf_build_tracks' bit for bit (same kernel, same bins), with page-locked
and with pageable buffers, for batches that divide the events and for a
ragged last batch, and match the oracle as the device build does (at least
99.9% identical hit assignments).
"""
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


@pytest.fixture(scope="module")
def events(oracle):
    ev = synth.make_build_events(81, 5, 600)
    f = oracle.fit_seeds(ev)
    assert (np.diff(ev.seed_event) >= 0).all()  # seeds grouped by event
    return ev, dict(state=f["state"].astype(np.float32), cov=f["cov"].astype(np.float32))


def host(a, dt, pin):
    t = torch.from_numpy(np.ascontiguousarray(a)).to(dt)
    return t.pin_memory() if pin else t


@pytest.mark.parametrize("pin", [True, False])
@pytest.mark.parametrize("batch", [0, 1, 2])
def test_host_build_equals_device_build(kf, ctx, events, pin, batch):
    ev, seeds = events
    opt = kf.options(n_phi_bins=256, n_z_bins=64)
    d = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype=dt)
    geom = kf.GeometryArgs.of(ev.build_geom)
    dev = kf.build_tracks(ctx, geom, ev.hit_offsets, d(ev.hit_pos, torch.float32), d(ev.hit_cov, torch.float32),
                          d(ev.seed_event, torch.int32), d(seeds["state"], torch.float32),
                          d(seeds["cov"], torch.float32), d(ev.seed_fit.charge, torch.int8), opt=opt)
    torch.cuda.synchronize()
    out = kf.build_outputs_host(ev.n_seeds, opt.max_cands, ev.build_geom.n_layers, pin=pin)
    for v in out.values():
        v.fill_(-3)
    got = kf.build_tracks_host(ctx, geom, ev.hit_offsets, host(ev.hit_pos, torch.float32, pin),
                               host(ev.hit_cov, torch.float32, pin), host(ev.seed_event, torch.int32, pin),
                               host(seeds["state"], torch.float32, pin), host(seeds["cov"], torch.float32, pin),
                               host(ev.seed_fit.charge, torch.int8, pin), opt=opt, out=out, events_per_batch=batch)
    for k in dev:
        assert np.array_equal(dev[k].cpu().numpy(), got[k].numpy()), k


def test_host_build_matches_oracle(kf, ctx, oracle, events):
    ev, seeds = events
    geom = kf.GeometryArgs.of(ev.build_geom)
    got = kf.build_tracks_host(ctx, geom, ev.hit_offsets, host(ev.hit_pos, torch.float32, True),
                               host(ev.hit_cov, torch.float32, True), host(ev.seed_event, torch.int32, True),
                               host(seeds["state"], torch.float32, True), host(seeds["cov"], torch.float32, True),
                               host(ev.seed_fit.charge, torch.int8, True), events_per_batch=2)
    ref = oracle.build_events(ev, seeds=seeds, max_cands=6)
    assert float((got["hit"].numpy() == ref["hit"]).mean()) >= 0.999


def test_host_build_argument_errors(kf, ctx, events):
    ev, seeds = events
    geom = kf.GeometryArgs.of(ev.build_geom)
    se = ev.seed_event.copy()[::-1].copy()  # not grouped by event
    with pytest.raises(kf.KFError, match="non-decreasing"):
        kf.build_tracks_host(ctx, geom, ev.hit_offsets, host(ev.hit_pos, torch.float32, False),
                             host(ev.hit_cov, torch.float32, False), host(se, torch.int32, False),
                             host(seeds["state"], torch.float32, False), host(seeds["cov"], torch.float32, False),
                             host(ev.seed_fit.charge, torch.int8, False))
