"""Benchmark: Kalman-filter track fit throughput on one GB300 (or N replicas).

One step is one pass of the fit hot path (propagate, transport, scatter,
update, precision routing, write) over the whole batch: 100 events x 20,000
tracks of the 10-layer toy barrel (r = 4..40 cm, Bz = 3.8 T), all events in one
persistent, graph-captured launch.  Inputs sit in HBM before the timed region
(1.18 GB per step, larger than the 129 MB L2, so L2 is not flushed).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank fits its own batch
(weak scaling, no collective on the data path); the time is the maximum over
ranks.  ``--impl reference`` times the FP64 CPU oracle on the host cores on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fitted tracks/s and built seeds/s on 1 GB300 (chosen vs plain form), % of FP32 roofline"
WORKLOAD = ("fit: 10-layer toy barrel r=4..40 cm, |z|<100 cm, Bz=3.8 T, x/X0=0.01; 100 events x 20,000 "
            "tracks, pT U(0.5,10) GeV, |eta|<1, seeds smeared 10%; FP32 with FP64 routing, one persistent "
            "graph-captured launch")
N_LAYERS = 10
# FP32 flops of one track-layer with a hit, counted on the kernel's formulation
# (add, multiply, reciprocal, square root, log = 1, FMA = 2): propagation 75,
# Jacobian 88, J C J^T 308, scattering 42, local-frame update 255.  The routed
# form also spends about 30 flops per update on its routing tests (not counted).
FLOPS_PER_TRACK_LAYER = 768
# the proposal network per scored row: 2 (12 x 64 + 64 x 64 + 64) multiply-adds
# (the split activations issue each layer-1 and layer-2 product twice; that
# doubling is not counted)
ROW_FLOPS = 2 * (12 * 64 + 64 * 64 + 64)
# algorithmic HBM bytes per track at 10 layers: seed 108 + charge 1 + mask 4 +
# hits 10 x 36 in, state/cov 108 + chi2 4 + ndof 2 + flags 4 out
BYTES_PER_TRACK = 108 + 1 + 4 + 36 * N_LAYERS + 108 + 4 + 2 + 4
# FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 flop/FMA x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--events", type=int, default=100)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--precision", default="routed", choices=["routed", "fp32"],
                   help="precision of the timed fit (the chosen form is routed)")
    p.add_argument("--shape", default=None,
                   help="fixed fit launch shape TRACKS_PER_BLOCK:REG_CAP[:HIT_PREFETCH] (no tuning; prefetch 1 if omitted)")
    p.add_argument("--build-events", type=int, default=64, help="events of the build workload (0: skip it)")
    p.add_argument("--build-steps", type=int, default=10)
    p.add_argument("--no-ragged", action="store_true", help="skip the ragged-batching comparison")
    p.add_argument("--no-transport", action="store_true", help="skip the batched 6x6 transport comparison")
    p.add_argument("--train-events", type=int, default=3, help="events logged to train the proposal")
    p.add_argument("--seed-events", type=int, default=4, help="build-workload events seeded from hits")
    p.add_argument("--train-epochs", type=int, default=4)
    p.add_argument("--dense-events", type=int, default=8, help="100x-noise events of the learned comparison (0: skip)")
    p.add_argument("--no-scoring", action="store_true", help="skip the scoring engines' comparison")
    return p.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The maximum of x over all ranks of the default process group (x itself
    on one rank): the timed region ends when the slowest rank ends."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(units_per_rank: int, world: int, ms_per_step: float) -> float:
    """Whole-job throughput of a weak-scaling step: every rank processes its
    own units_per_rank, and the step takes the slowest rank's time."""
    return world * units_per_rank / (ms_per_step * 1e-3)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def kernel_source_hash(unit: str = "kf_fit.cu") -> str:
    """Hash of a kernel's sources (its translation unit, by default the fit's,
    and every header it includes from the package's csrc/) and of the build
    script.  The public header include/kf.h (declarations and their
    documentation) is left out."""
    import re
    csrc = os.path.join(ROOT, "paper_1705_02876_gb300", "csrc")
    todo, seen = [os.path.join(csrc, unit)], []
    while todo:
        p = todo.pop()
        if p in seen:
            continue
        seen.append(p)
        for name in re.findall(r'#include\s+"([^"]+)"', open(p).read()):
            if os.path.exists(os.path.join(csrc, name)):
                todo.append(os.path.join(csrc, name))
    h = hashlib.sha256()
    for p in sorted(seen) + [os.path.join(ROOT, "paper_1705_02876_gb300", "build.py")]:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_build_traffic(src_hash: str):
    """DRAM bytes of one W4 build call (the build kernel and the binning) from
    the committed ncu summary, if it was taken on the current build sources."""
    path = os.path.join(ROOT, "profiles", "build_kernel_build_workload.txt")
    try:
        vals = {k.strip(): v.strip() for k, v in (line.split(":", 1) for line in open(path).read().splitlines()
                                                  if ":" in line and not line.startswith((" ", "#")))}
        if vals.get("source_hash") != src_hash:
            return None
        return (float(vals["dram_bytes_read_per_launch"]) + float(vals["dram_bytes_write_per_launch"])
                + float(vals["binning_dram_bytes_per_launch"]))
    except (OSError, KeyError, ValueError):
        return None


def recorded_traffic(src_hash: str):
    """DRAM bytes per launch of the fit kernel from the committed ncu summary,
    if it was taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "fit_kernel_fit_workload.txt")
    try:
        text = open(path).read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_hash") != src_hash:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.dev = device_index

    def _target(self):
        import torch
        try:
            uuid = str(torch.cuda.get_device_properties(self.dev).uuid)
            return uuid if uuid.startswith("GPU-") else "GPU-" + uuid
        except Exception:
            return None

    def start(self):
        target = self._target()
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "20"]
        if target:
            cmd += ["-i", target]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.05)

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.05)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(batch, n_sample: int):
    from oracle import kf_oracle
    sub = slice(0, n_sample)
    g = batch.geom
    f32 = lambda v: np.asarray(v, dtype=np.float32).astype(np.float64)
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    kf_oracle.fit_arrays(f32(g.radii), f32(g.x_over_x0), float(np.float32(g.z_half)), float(np.float32(g.bz)),
                         batch.seed_state[:, sub], batch.seed_cov[:, sub], batch.charge[sub],
                         batch.hit_pos[:, :, sub], batch.hit_cov[:, :, sub], batch.hit_mask[sub],
                         threads=threads)
    dt = time.perf_counter() - t0
    n1 = min(n_sample, 200_000)  # one core on a smaller sample
    sub1 = slice(0, n1)
    t1 = time.perf_counter()
    kf_oracle.fit_arrays(f32(g.radii), f32(g.x_over_x0), float(np.float32(g.z_half)), float(np.float32(g.bz)),
                         batch.seed_state[:, sub1], batch.seed_cov[:, sub1], batch.charge[sub1],
                         batch.hit_pos[:, :, sub1], batch.hit_cov[:, :, sub1], batch.hit_mask[sub1], threads=1)
    dt1 = time.perf_counter() - t1
    return {"value": n_sample / dt, "unit": "tracks/s", "cores": threads, "kind": "oracle",
            "sample": f"first {n_sample} tracks of the workload, FP64 C oracle split over {threads} threads "
                      f"({dt:.2f} s wall)",
            "single_core": {"value": n1 / dt1, "unit": "tracks/s", "sample": f"first {n1} tracks, 1 thread"},
            "cpu_model": cpu_model()}


def cpu_model() -> str | None:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores, one bounded sample per step."""
    if rank != 0:
        return
    from paper_1705_02876_gb300 import synth
    # ten of the workload's 20,000-track events (the same generator and
    # distributions), about 65 ms of oracle work per step on 16 cores
    batch = synth.make_fit_batch(1, [20000] * 10)
    n_sample = batch.seed_state.shape[1]
    from oracle import kf_oracle
    g = batch.geom
    f32 = lambda v: np.asarray(v, dtype=np.float32).astype(np.float64)
    threads = os.cpu_count() or 1

    def step():
        kf_oracle.fit_arrays(f32(g.radii), f32(g.x_over_x0), float(np.float32(g.z_half)),
                             float(np.float32(g.bz)), batch.seed_state, batch.seed_cov, batch.charge,
                             batch.hit_pos, batch.hit_cov, batch.hit_mask, threads=threads)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    v = n_sample / dt
    line = {"metric": METRIC, "value": v, "unit": "tracks/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "sample_tracks_per_step": n_sample},
            "cpu_baseline": {"value": v, "unit": "tracks/s", "cores": threads, "kind": "oracle",
                             "sample": f"{n_sample} tracks (ten 20,000-track events) per step"},
            "e2e": {"value": v, "unit": "tracks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


BUILD_WORKLOAD = ("build: 17-layer toy barrel r=4..68 cm, {E} events x 5,000 tracks, 10x uniform noise hits per "
                  "layer (55,000 hits per layer per event), seeds fitted from the first 3 layers, 14 layers built, "
                  "N=6 candidates, chi2 cut 30, 3-sigma window, 256 x 64 bins")


def bench_build(args, kf, ctx, dev, stream, rank, world):
    """Seed fit (3 layers) + binning + clone-engine build of the build workload."""
    import torch
    from paper_1705_02876_gb300 import metrics, synth
    E = args.build_events
    # the seed layers' hits (every track's hits, no added noise) feed the
    # seeding-from-hits section; they come from streams of their own and leave
    # the build's events unchanged
    ev = synth.make_build_events(4 + 1000 * rank, E, 5000, seed_layer_hits=True, seed_noise_per_layer=0)
    sf = ev.seed_fit
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dtype=dt)
    d_sf = kf.to_device(sf, dev)
    seed_geom = kf.GeometryArgs.of(sf.geom)
    build_geom = kf.GeometryArgs.of(ev.build_geom)
    hp, hc = t(ev.hit_pos, torch.float32), t(ev.hit_cov, torch.float32)
    se, sq = t(ev.seed_event, torch.int32), t(sf.charge, torch.int8)
    S = ev.n_seeds
    chosen = kf.options()
    plain = kf.options(precision_mode=kf.PRECISION_FP32, launch_mode=kf.LAUNCH_PER_EVENT)
    fit_out = kf.fit_outputs(S, dev)
    b_out = None

    def step_chosen():
        nonlocal b_out
        kf.fit_tracks(ctx, seed_geom, **d_sf, opt=chosen, out=fit_out, stream=stream)
        b_out = kf.build_tracks(ctx, build_geom, ev.hit_offsets, hp, hc, se, fit_out["state"], fit_out["cov"], sq,
                                opt=chosen, out=b_out, stream=stream)

    # plain: FP32, one fit launch and one build launch per event
    ev_seeds = [np.nonzero(ev.seed_event == e)[0] for e in range(E)]
    zeros = [torch.zeros(len(ix), dtype=torch.int32, device=dev) for ix in ev_seeds]
    plain_outs = [None] * E
    lo_hi = [(int(ix[0]), int(ix[-1]) + 1) if len(ix) else (0, 0) for ix in ev_seeds]
    sfo = kf.fit_outputs(S, dev)

    def step_plain():
        kf.fit_tracks(ctx, seed_geom, **d_sf, event_offsets=np.array([0] + [hi for _, hi in lo_hi]),
                      opt=plain, out=sfo, stream=stream)
        for e in range(E):
            lo, hi = lo_hi[e]
            if hi <= lo:
                continue
            plain_outs[e] = kf.build_tracks(ctx, build_geom, ev.hit_offsets[e:e + 1], hp, hc, zeros[e],
                                            sfo["state"][:, lo:hi].contiguous(), sfo["cov"][:, lo:hi].contiguous(),
                                            sq[lo:hi], opt=plain, out=plain_outs[e], stream=stream)

    def timed(fn, n):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n

    ms = timed(step_chosen, args.build_steps)
    best = b_out["hit"][:, 0].cpu().numpy()

    # the build call alone (binning + build kernel) for its roofline fractions
    def step_build_only():
        kf.build_tracks(ctx, build_geom, ev.hit_offsets, hp, hc, se, fit_out["state"], fit_out["cov"], sq,
                        opt=chosen, out=b_out, stream=stream)

    ms_call = timed(step_build_only, args.build_steps)
    peaks = measured_peaks()
    Lb = ev.build_geom.n_layers
    flops = S * Lb * chosen.max_cands * FLOPS_PER_TRACK_LAYER  # every candidate slot live: an upper bound
    build_hash = kernel_source_hash("kf_build.cu")
    dram = recorded_build_traffic(build_hash) if E == 64 else None
    hbm = peaks.get("hbm_gbs")
    build_roofline = {
        "bound": "latency", "call_ms": ms_call, "fp32_tflops": flops / (ms_call * 1e-3) / 1e12,
        "fp32_frac": flops / (ms_call * 1e-3) / 1e12 / FP32_PEAK_TFLOPS,
        "fp32_flops_per_call": flops,
        "fp32_flops_note": "seeds x build layers x N x 768: every candidate slot live at every layer (upper bound)",
        "dram_gbs": dram / (ms_call * 1e-3) / 1e9 if dram else None,
        "dram_frac": (dram / (ms_call * 1e-3) / 1e9 / hbm) if (dram and hbm) else None,
        "dram_bytes_per_call": dram,
        "dram_bytes_source": "ncu capture of the 64-event call (build kernel + binning), committed summary",
        "kernel_source_hash": build_hash}
    q = metrics.efficiency_fake_rate(best, ev.seed_track, ev.hit_track, ev.track_nhits)
    e2e = bench_build_e2e(args, kf, ctx, ev, fit_out, b_out, chosen)
    ms_plain = timed(step_plain, max(2, args.build_steps // 2))
    qp = metrics.efficiency_fake_rate(np.concatenate([o["hit"][:, 0].cpu().numpy() for o in plain_outs if o is not None]),
                                      ev.seed_track, ev.hit_track, ev.track_nhits)
    learned = bench_learned(args, kf, ctx, dev, stream, rank, ev, seed_geom, d_sf, fit_out, build_geom, hp, hc, se,
                            sq, timed)
    seeding = bench_seeding(args, kf, ctx, dev, stream, ev, build_geom, hp, hc, timed)
    out = {"value": S / (ms * 1e-3), "unit": "seeds/s", "ms_per_step": ms, "seeds": S,
           "workload": BUILD_WORKLOAD.format(E=E),
           "form": "seed fit + binning + build of all events in one launch each, routed precision, "
                   "exhaustive chi2 in every window",
           "efficiency": q["efficiency"], "fake_rate": q["fake_rate"], "mean_hits": q["mean_hits"],
           "hit_purity": q["hit_purity"], "roofline": build_roofline,
           "plain": {"value": S / (ms_plain * 1e-3), "unit": "seeds/s", "ms_per_step": ms_plain,
                     "form": "FP32 only, one launch per event", "efficiency": qp["efficiency"],
                     "fake_rate": qp["fake_rate"]},
           "learned": learned, "seeding": seeding, "e2e": e2e,
           "tuned_bins": ctx.build_tuned_shape(Lb, chosen.max_cands, 0, S, int(ev.hit_pos.shape[1]))}
    return out


def bench_build_e2e(args, kf, ctx, ev, fit_out, b_out, opt):
    """The build end to end through kf_build_tracks_host: hits, seeds and
    outputs in pinned host memory, every byte crossing the host link inside the
    timed region (batches of 16 events, uploads, builds and downloads
    overlapped on three streams); checked equal to the device build."""
    import torch
    pin = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dt).pin_memory()
    hin = dict(hit_pos=pin(ev.hit_pos, torch.float32), hit_cov=pin(ev.hit_cov, torch.float32),
               seed_event=pin(ev.seed_event, torch.int32), seed_state=fit_out["state"].cpu().pin_memory(),
               seed_cov=fit_out["cov"].cpu().pin_memory(), seed_charge=pin(ev.seed_fit.charge, torch.int8))
    geom = kf.GeometryArgs.of(ev.build_geom)
    hout = kf.build_outputs_host(ev.n_seeds, opt.max_cands, ev.build_geom.n_layers)

    def step():
        kf.build_tracks_host(ctx, geom, ev.hit_offsets, **hin, opt=opt, out=hout, events_per_batch=16)

    for _ in range(2):
        step()
    n = max(3, args.build_steps // 2)
    t0 = time.perf_counter()
    for _ in range(n):
        step()
    ms = (time.perf_counter() - t0) * 1e3 / n
    same = bool(np.array_equal(hout["hit"].numpy(), b_out["hit"].cpu().numpy()))
    h2d = sum(v.numel() * v.element_size() for v in hin.values())
    d2h = sum(v.numel() * v.element_size() for v in hout.values())
    return {"value": ev.n_seeds / (ms * 1e-3), "unit": "seeds/s", "ms_per_step": ms, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "link_gbs": (h2d + d2h) / (ms * 1e-3) / 1e9, "equals_device_build": same,
            "form": "kf_build_tracks_host: pinned host buffers, 16-event batches, copies overlapped with the builds"}


def bench_seeding(args, kf, ctx, dev, stream, ev, build_geom, hp, hc, timed):
    """Seeding from hits on the first --seed-events events of the build
    workload: the triplet search over the three seed layers' hits (every
    track's hit, no added noise) with the seed fit's inputs, alone and followed
    by the 3-layer seed fit and the build of every seed."""
    import torch
    from paper_1705_02876_gb300 import metrics
    E = min(args.seed_events, ev.n_events)
    g3 = kf.GeometryArgs.of(ev.geom.sub(0, 3))
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dtype=dt)
    soff = ev.seed_hit_offsets[:E]
    n_hits = int(soff[-1, -1] - soff[0, 0])
    shp, shc = t(ev.seed_hit_pos, torch.float32), t(ev.seed_hit_cov, torch.float32)
    seeds = None

    def step_seed():
        nonlocal seeds
        seeds = kf.seed_triplets(ctx, g3, soff, shp, shc, stream=stream)

    ms_seed = timed(step_seed, args.build_steps)
    n = int(seeds["charge"].shape[0])
    fit_out = kf.fit_outputs(n, dev)
    b_out = None

    def step_chain():
        nonlocal seeds, b_out
        seeds = kf.seed_triplets(ctx, g3, soff, shp, shc, stream=stream)
        kf.fit_tracks(ctx, g3, seeds["seed_state"], seeds["seed_cov"], seeds["charge"], seeds["hit_pos"],
                      seeds["hit_cov"], seeds["hit_mask"], out=fit_out, stream=stream)
        b_out = kf.build_tracks(ctx, build_geom, ev.hit_offsets[:E], hp, hc, seeds["event"], fit_out["state"],
                                fit_out["cov"], seeds["charge"], out=b_out, stream=stream)

    ms_chain = timed(step_chain, max(2, args.build_steps // 2))
    hits = seeds["hits"].cpu().numpy()
    trk = ev.seed_hit_track[hits]
    st = np.where((trk[0] >= 0) & (trk[0] == trk[1]) & (trk[1] == trk[2]), trk[0], -1)
    q = metrics.efficiency_fake_rate(b_out["hit"][:, 0].cpu().numpy(), st, ev.hit_track, ev.track_nhits,
                                     eligible_tracks=ev.seed_track[ev.seed_event < E])
    # efficiency against fakes at tighter seeding cuts (the same chain, once each)
    points = {}
    for name, cuts in (("d0_0.10_dz_0.5", dict(d0_max=0.10, dz_max=0.5)),
                       ("d0_0.05_dz_0.4", dict(d0_max=0.05, dz_max=0.4))):
        so = kf.seeding(**cuts)
        sd = kf.seed_triplets(ctx, g3, soff, shp, shc, opt=so, stream=stream)
        m = int(sd["charge"].shape[0])
        fo = kf.fit_outputs(m, dev)
        kf.fit_tracks(ctx, g3, sd["seed_state"], sd["seed_cov"], sd["charge"], sd["hit_pos"], sd["hit_cov"],
                      sd["hit_mask"], out=fo, stream=stream)
        bo = kf.build_tracks(ctx, build_geom, ev.hit_offsets[:E], hp, hc, sd["event"], fo["state"], fo["cov"],
                             sd["charge"], stream=stream)
        t2 = ev.seed_hit_track[sd["hits"].cpu().numpy()]
        s2 = np.where((t2[0] >= 0) & (t2[0] == t2[1]) & (t2[1] == t2[2]), t2[0], -1)
        q2 = metrics.efficiency_fake_rate(bo["hit"][:, 0].cpu().numpy(), s2, ev.hit_track, ev.track_nhits,
                                          eligible_tracks=ev.seed_track[ev.seed_event < E])
        points[name] = {"seeds": m, "efficiency": q2["efficiency"], "fake_rate": q2["fake_rate"],
                        "hit_purity": q2["hit_purity"]}
    return {"value": E / (ms_chain * 1e-3), "unit": "events/s", "ms_per_step": ms_chain, "events": E,
            "seeds": n, "seeds_per_event": n / E, "true_seed_share": float((st >= 0).mean()),
            "form": "triplet search + seed inputs + 3-layer seed fit + build of every seed, default cuts "
                    "(pT > 0.3 GeV, d0 < 0.15 cm, |z0| < 4 cm, dz < 0.8 cm; both charges above 2 GeV)",
            "efficiency": q["efficiency"], "fake_rate": q["fake_rate"], "hit_purity": q["hit_purity"],
            "operating_points": points,
            "search": {"value": n_hits / (ms_seed * 1e-3), "unit": "seed-layer hits/s", "ms_per_step": ms_seed,
                       "seed_layer_hits": n_hits, "events_per_s": E / (ms_seed * 1e-3),
                       "form": "binning + triplet search + count read-back + seed inputs"}}


def bench_learned(args, kf, ctx, dev, stream, rank, ev, seed_geom, d_sf, fit_out, build_geom, hp, hc, se, sq, timed):
    """The chosen build with the learned proposal (top-k = 4).  Its network is
    trained first, untimed, on up to 1M (candidate, hit) rows the plain build
    logs on separate events, by the library's own training kernels."""
    import torch
    from paper_1705_02876_gb300 import metrics, synth
    tr = synth.make_build_events(10 + 1000 * rank, args.train_events, 5000)
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dtype=dt)
    d_tr = kf.to_device(tr.seed_fit, dev)
    tf = kf.fit_tracks(ctx, kf.GeometryArgs.of(tr.seed_fit.geom), **d_tr, stream=stream)
    log = kf.new_build_log(1_000_000, dev)
    kf.build_tracks(ctx, build_geom, tr.hit_offsets, t(tr.hit_pos, torch.float32), t(tr.hit_cov, torch.float32),
                    t(tr.seed_event, torch.int32), tf["state"], tf["cov"], t(tr.seed_fit.charge, torch.int8),
                    stream=stream, log=log)
    torch.cuda.synchronize()
    n = kf.log_rows(log)
    ref = log["ref"][:n].cpu().numpy().astype(np.int64)
    win = np.unique((ref[:, 0] * 8 + ref[:, 1]) * 64 + ref[:, 2], return_counts=True)[1]
    w = torch.from_numpy(synth.proposal_init(np.random.default_rng(9 + rank))).to(dev, torch.float32)
    t0 = time.perf_counter()
    losses = kf.proposal_train(ctx, w, log["features"][:n].contiguous(), log["labels"][:n].contiguous(),
                               epochs=args.train_epochs, batch=4096, lr=2e-3, stream=stream)
    train_s = time.perf_counter() - t0
    kf.proposal_load(ctx, w, stream=stream)
    opt = kf.options(use_proposal=1, topk=4)
    b_out = None

    def step_learned():
        nonlocal b_out
        kf.fit_tracks(ctx, seed_geom, **d_sf, opt=opt, out=fit_out, stream=stream)
        b_out = kf.build_tracks(ctx, build_geom, ev.hit_offsets, hp, hc, se, fit_out["state"], fit_out["cov"], sq,
                                opt=opt, out=b_out, stream=stream)

    ms = timed(step_learned, args.build_steps)
    q = metrics.efficiency_fake_rate(b_out["hit"][:, 0].cpu().numpy(), ev.seed_track, ev.hit_track, ev.track_nhits)
    dense = bench_learned_dense(args, kf, ctx, dev, stream, rank, timed) if args.dense_events > 0 else None
    kf.proposal_load(ctx, w, stream=stream)
    return {"value": ev.n_seeds / (ms * 1e-3), "unit": "seeds/s", "ms_per_step": ms, "topk": 4, "dense": dense,
            "efficiency": q["efficiency"], "fake_rate": q["fake_rate"], "hit_purity": q["hit_purity"],
            "training": {"rows": n, "events": args.train_events, "epochs": args.train_epochs,
                         "loss_first_last": [losses[0], losses[-1]], "seconds": round(train_s, 3)},
            "windows_above_topk": float((win > 4).mean()), "mean_window_hits": float(win.mean())}


def bench_learned_dense(args, kf, ctx, dev, stream, rank, timed):
    """Where windows hold more hits than top-k: 100x noise (1,000 tracks per
    event, 100,000 noise hits per build layer).  A network trained (by the
    library's kernels) on the plain build's rows of separate 100x events
    ranks each window's hits; against the exhaustive chi2 search and the
    same top-k cut without a network (hit order).  Seeds fitted on the GPU."""
    import torch
    from paper_1705_02876_gb300 import metrics, synth
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dtype=dt)

    def load(ev):
        sf = ev.seed_fit
        fo = kf.fit_tracks(ctx, kf.GeometryArgs.of(sf.geom), **kf.to_device(sf, dev), stream=stream)
        return dict(geom=kf.GeometryArgs.of(ev.build_geom), hp=t(ev.hit_pos, torch.float32),
                    hc=t(ev.hit_cov, torch.float32), se=t(ev.seed_event, torch.int32), st=fo["state"],
                    cv=fo["cov"], sq=t(sf.charge, torch.int8))

    tr = synth.make_build_events(60 + 1000 * rank, 4, 1000, noise_factor=100)
    d = load(tr)
    log = kf.new_build_log(2_000_000, dev)
    kf.build_tracks(ctx, d["geom"], tr.hit_offsets, d["hp"], d["hc"], d["se"], d["st"], d["cv"], d["sq"],
                    stream=stream, log=log)
    torch.cuda.synchronize()
    n = kf.log_rows(log)
    w = torch.from_numpy(synth.proposal_init(np.random.default_rng(19 + rank))).to(dev, torch.float32)
    kf.proposal_train(ctx, w, log["features"][:n].contiguous(), log["labels"][:n].contiguous(), epochs=8,
                      batch=1024, lr=2e-3, stream=stream)
    ev = synth.make_build_events(61 + 1000 * rank, args.dense_events, 1000, noise_factor=100)
    d = load(ev)
    res = {"workload": f"build geometry, {args.dense_events} events x 1,000 tracks, 100x uniform noise hits "
                       "(100,000 per build layer per event), N = 6", "training_rows": n}
    for name, opt, weights in (("exhaustive", kf.options(), None),
                               ("learned_top1", kf.options(use_proposal=1, topk=1), w),
                               ("learned_top4", kf.options(use_proposal=1, topk=4), w),
                               ("blind_top1", kf.options(use_proposal=1, topk=1), torch.zeros_like(w))):
        if weights is not None:
            kf.proposal_load(ctx, weights, stream=stream)
        out = None

        def step():
            nonlocal out
            out = kf.build_tracks(ctx, d["geom"], ev.hit_offsets, d["hp"], d["hc"], d["se"], d["st"], d["cv"],
                                  d["sq"], opt=opt, out=out, stream=stream)

        ms = timed(step, max(3, args.build_steps // 2))
        q = metrics.efficiency_fake_rate(out["hit"][:, 0].cpu().numpy(), ev.seed_track, ev.hit_track,
                                         ev.track_nhits)
        res[name] = {"value": ev.n_seeds / (ms * 1e-3), "unit": "seeds/s", "ms_per_step": ms,
                     "efficiency": q["efficiency"], "fake_rate": q["fake_rate"], "hit_purity": q["hit_purity"]}
    return res


def bench_scoring(args, kf, ctx, dev):
    """The proposal's batched scoring on both tensor-core engines, on the same
    rows: mma.sync (warp-level, accumulators in registers) and tcgen05 (128-row
    CTA tiles, accumulators in tensor memory); kf_proposal_score's automatic
    choice per size."""
    import torch
    from paper_1705_02876_gb300 import synth
    w = torch.from_numpy(synth.proposal_init(np.random.default_rng(5))).to(dev, torch.float32)
    kf.proposal_load(ctx, w)
    res = {"form": "12 -> 64 -> 64 -> 1, BF16 weights, split BF16 activations (hi + lo), FP32 accumulation",
           "algorithmic_flops_per_row": ROW_FLOPS, "sizes": {}}
    for n in (1 << 16, 1 << 20, 1 << 24):
        X = torch.randn(n, 12, device=dev, dtype=torch.float32)
        row = {}
        for name, eng in (("mma_sync", kf.SCORE_MMA_SYNC), ("tcgen05", kf.SCORE_TCGEN05), ("auto", None)):
            for _ in range(3):
                kf.proposal_score(ctx, X, engine=eng)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(10):
                kf.proposal_score(ctx, X, engine=eng)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / 10
            row[name] = {"ms": ms, "rows_per_s": n / (ms * 1e-3), "tflops": n * ROW_FLOPS / (ms * 1e-3) / 1e12}
        res["sizes"][str(n)] = row
    return res


def bench_ragged(args, kf, ctx, dev, stream, rank):
    """Ragged batching: 256 events of lognormal sizes (median 5,000, clamped
    to 500..50,000), 17 layers, hit efficiency 0.95, fitted as one persistent
    graph-captured launch (autotuned shape), one plain launch over all tracks,
    and one plain launch per event."""
    import torch
    from paper_1705_02876_gb300 import synth
    b = synth.workload("ragged", seed=3 + 1000 * rank)
    T = b.n_tracks
    geom = kf.GeometryArgs.of(b.geom)
    d_in = kf.to_device(b, dev)
    out = kf.fit_outputs(T, dev)
    res = {"workload": "17-layer toy barrel r=4..68 cm, 256 events, lognormal sizes (median 5,000, "
                       "500..50,000), hit efficiency 0.95", "tracks": T}
    for name, mode in (("persistent", kf.LAUNCH_AUTO), ("flat", kf.LAUNCH_FLAT), ("per_event", kf.LAUNCH_PER_EVENT)):
        opt = kf.options(launch_mode=mode)

        def step():
            kf.fit_tracks(ctx, geom, **d_in, event_offsets=b.event_offsets, opt=opt, out=out, stream=stream)

        for _ in range(max(args.warmup, 3)):
            step()
        torch.cuda.synchronize()
        n = 20 if mode != kf.LAUNCH_PER_EVENT else 5
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / n
        res[name] = {"value": T / (ms * 1e-3), "unit": "tracks/s", "ms_per_step": ms,
                     "launches_per_step": 1 if mode != kf.LAUNCH_PER_EVENT else len(b.event_offsets) - 1}
    shape = ctx.tuned_shape(b.geom.n_layers, T)
    res["tuned_shape"] = ({"tracks_per_block": shape[0], "reg_cap": shape[1], "hit_prefetch": shape[2]}
                          if shape else None)
    return res


def bench_smoother(args, kf, ctx, dev, stream, batch, d_in):
    """The fit followed by the Rauch-Tung-Striebel smoother on the fit
    workload: smoothed state and covariance after every layer."""
    import torch
    geom = kf.GeometryArgs.of(batch.geom)
    out = None

    def step():
        nonlocal out
        out = kf.smooth_tracks(ctx, geom, **d_in, out=out, stream=stream)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    n = 10
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(n):
        step()
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / n
    T, L = batch.n_tracks, batch.geom.n_layers
    # bytes per track the kernel moves: fit inputs 473, per layer 108 B of
    # filtered estimates written and read back and 108 B of smoothed ones written
    per_track = 113 + 36 * L + L * 3 * 108 + 2 + 4
    # inputs and the smoothed outputs alone (the filtered estimates read back from L2)
    io_track = 113 + 36 * L + L * 108 + 2 + 4
    hbm = measured_peaks().get("hbm_gbs")
    io_gbs = io_track * T / (ms * 1e-3) / 1e9
    return {"value": T / (ms * 1e-3), "unit": "tracks/s", "ms_per_step": ms, "layers": L,
            "gbs_kernel_bytes": per_track * T / (ms * 1e-3) / 1e9, "hbm_gbs_inputs_outputs": io_gbs,
            "hbm_frac_inputs_outputs": io_gbs / hbm if hbm else None,
            "form": "one thread per track: routed forward fit keeping every layer's filtered estimate, then the "
                    "backward pass recomputing each prediction"}


def bench_transport(args, kf, ctx, dev, stream):
    """Batched 6x6 covariance transport C <- J C J^T (the paper's Section 4.1
    study of many small matrix products): the library's one-thread-per-matrix
    kernel on SoA data against two batched cuBLAS products (torch.bmm, FP32,
    TF32 off) on [n][6][6] data, at growing batch sizes."""
    import torch
    torch.backends.cuda.matmul.allow_tf32 = False
    rng = np.random.default_rng(11)
    res = {"form": "ours: kf_transport_batch, J [36][n] + packed C [21][n] in registers, 312 B per matrix; "
                   "cublas: bmm(bmm(J, C), J^T) on [n][6][6], 576 B per matrix", "sizes": {}}
    for n in (10_000, 100_000, 1_000_000, 10_000_000):
        J = torch.from_numpy((np.eye(6, dtype=np.float32).reshape(36, 1) +
                              0.1 * rng.standard_normal((36, n), dtype=np.float32))).to(dev)
        C0 = torch.from_numpy(rng.standard_normal((21, n), dtype=np.float32)).to(dev)
        C = C0.clone()
        Ja = J.T.reshape(n, 6, 6).contiguous()
        Ca = torch.randn(n, 6, 6, device=dev)
        Jt = Ja.transpose(1, 2)

        def timed(fn, reps):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b) / reps

        reps = max(5, int(2e8 // (n * 312)))
        ms = timed(lambda: kf.transport_batch(ctx, J, C, stream=stream), reps)
        ms_cb = timed(lambda: torch.bmm(torch.bmm(Ja, Ca), Jt), reps)
        res["sizes"][str(n)] = {
            "ours": {"matrices_per_s": n / (ms * 1e-3), "ms": ms, "hbm_gbs": 312 * n / (ms * 1e-3) / 1e9},
            "cublas": {"matrices_per_s": n / (ms_cb * 1e-3), "ms": ms_cb}}
        del J, C0, C, Ja, Ca, Jt
    return res


def main():
    args = parse()
    rank, world, local = dist_info()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    import torch.distributed as dist

    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_1705_02876_gb300 import build, kf, synth
    build.build()
    batch = synth.make_fit_batch(1 + 1000 * rank, [20000] * args.events)
    T = batch.n_tracks
    ctx = kf.Context(dev.index)
    geom = kf.GeometryArgs.of(batch.geom)
    d_in = kf.to_device(batch, dev)
    out = kf.fit_outputs(T, dev)
    stream = torch.cuda.current_stream(dev)
    chosen = kf.options(precision_mode=kf.PRECISION_ROUTED if args.precision == "routed" else kf.PRECISION_FP32)
    if args.shape:
        parts = [int(v) for v in args.shape.split(":")]
        chosen.tracks_per_block, chosen.reg_cap = parts[0], parts[1]
        chosen.hit_prefetch = parts[2] if len(parts) > 2 else 1

    def step(opt=chosen, o=out):
        kf.fit_tracks(ctx, geom, **d_in, event_offsets=batch.event_offsets, opt=opt, out=o, stream=stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(dev.index)
    barrier()
    sampler.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    t_wall = time.perf_counter()
    for i in range(args.steps):
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    barrier()
    t_wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = max_over_ranks(starts[0].elapsed_time(ends[-1]), world, dev)
    ms_per_step = total_ms / args.steps
    value = weak_value(T, world, ms_per_step)
    kern_ms = statistics.mean(step_ms)

    # plain form: one FP32 launch per event, same data (outside the timed region)
    plain_opt = kf.options(precision_mode=kf.PRECISION_FP32, launch_mode=kf.LAUNCH_PER_EVENT)
    plain_out = kf.fit_outputs(T, dev)
    for _ in range(3):
        step(plain_opt, plain_out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_plain = max(3, min(args.steps, 50))
    e0.record(stream)
    for _ in range(n_plain):
        step(plain_opt, plain_out)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1) / n_plain

    # end to end through the public host-buffer call: the fit reads the pinned
    # host inputs and writes the pinned host outputs in place (every byte
    # crosses the host link inside the timed region); the call returns with
    # every output in host memory
    host_in = kf.to_host(batch)
    host_out = kf.fit_outputs_host(T)
    h2d = sum(v.numel() * v.element_size() for v in host_in.values())
    d2h = sum(v.numel() * v.element_size() for v in host_out.values())
    host_opt = kf.options(precision_mode=chosen.precision_mode)

    def e2e_step():
        kf.fit_tracks_host(ctx, geom, **host_in, opt=host_opt, out=host_out)

    for _ in range(3):
        e2e_step()
    n_e2e = max(3, min(args.steps, 20))
    barrier()
    t_e = time.perf_counter()
    for _ in range(n_e2e):
        e2e_step()
    barrier()
    e2e_ms = max_over_ranks((time.perf_counter() - t_e) * 1e3 / n_e2e, world, dev)

    routed_share = float(((out["flags"] & 16) != 0).float().mean().item())
    flops = FLOPS_PER_TRACK_LAYER * N_LAYERS * T
    achieved_tflops = flops / (kern_ms * 1e-3) / 1e12
    src_hash = kernel_source_hash()
    traffic = recorded_traffic(src_hash)
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    tuned = (ctx.tuned_shape(N_LAYERS, T) if not args.shape
             else (chosen.tracks_per_block, chosen.reg_cap, chosen.hit_prefetch))
    line = {
        "metric": METRIC, "value": value, "unit": "tracks/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "tracks_per_gpu": T, "layers": N_LAYERS,
                   "l2": "inputs larger than L2 (1.18 GB per step), not flushed",
                   "tracks_per_block": tuned[0] if tuned else None, "reg_cap": tuned[1] if tuned else None,
                   "hit_prefetch": tuned[2] if tuned else None,
                   "parallelism": f"replicas{world}"},
        "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": FP32_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved_tflops / FP32_PEAK_TFLOPS, "traffic": traffic,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                     "algorithmic_flops_per_launch": flops,
                     "hbm_gbs": BYTES_PER_TRACK * T / (kern_ms * 1e-3) / 1e9,
                     "hbm_frac_of_measured": (BYTES_PER_TRACK * T / (kern_ms * 1e-3) / 1e9 / hbm) if hbm else None},
        # the build's headline fields, filled in below, near the front of the line
        "build_summary": None,
        "plain": {"value": T / (plain_ms * 1e-3), "unit": "tracks/s", "ms_per_step": plain_ms,
                  "form": "FP32 only, one plain launch per event (100 launches)"},
        "e2e": {"value": weak_value(T, world, e2e_ms), "unit": "tracks/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "form": "kf_fit_tracks_host on pinned host buffers: one persistent launch reads the inputs and "
                        "writes the outputs in host memory over the host link"},
        "fp64_routed_share": routed_share,
        "gpu_launches": args.steps,
        "clocks": clocks,
        "kernel_source_hash": src_hash,
        "wall_s_timed": t_wall,
    }
    if args.build_events > 0:
        b = line["build"] = bench_build(args, kf, ctx, dev, stream, rank, world)
        r = b["roofline"]
        line["build_summary"] = {
            "seeds_per_s": b["value"], "plain_seeds_per_s": b["plain"]["value"],
            "learned_seeds_per_s": b["learned"]["value"], "efficiency": b["efficiency"],
            "fake_rate": b["fake_rate"], "learned_efficiency": b["learned"]["efficiency"],
            "call_ms": r["call_ms"], "fp32_frac": r["fp32_frac"], "dram_frac": r["dram_frac"],
            "dram_bytes_per_call": r["dram_bytes_per_call"], "e2e_seeds_per_s": b["e2e"]["value"],
            "tuned_bins": b["tuned_bins"]}
        dn = b["learned"].get("dense")
        if dn:
            line["build_summary"]["dense_100x"] = {k: {"seeds_per_s": dn[k]["value"], "efficiency": dn[k]["efficiency"],
                                                       "hit_purity": dn[k]["hit_purity"]}
                                                   for k in ("exhaustive", "learned_top1", "learned_top4", "blind_top1")}
    else:
        del line["build_summary"]
    if not args.no_ragged:
        line["ragged"] = bench_ragged(args, kf, ctx, dev, stream, rank)
    if not args.no_transport:
        line["transport6x6"] = bench_transport(args, kf, ctx, dev, stream)
    line["smoother"] = bench_smoother(args, kf, ctx, dev, stream, batch, d_in)
    if not args.no_scoring:
        line["proposal_scoring"] = bench_scoring(args, kf, ctx, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(batch, T)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
