"""ctypes loader for the plain FP64 C oracle (``kf_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package smoke check and
by the CPU-baseline leg of the benchmark.  Nothing in the library imports it.

The C code processes a contiguous range of tracks; ``fit_tracks`` splits a
batch into ranges and runs them on a thread pool (ctypes releases the GIL
during the call), so the oracle uses the host's cores without any threading
inside the C source.
"""
from __future__ import annotations

import concurrent.futures as cf
import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libkf_oracle.so")
_lock = threading.Lock()
_lib = None

FLAG_UNREACHABLE = 1
FLAG_LEFT_BARREL = 2
FLAG_INVERSION_FAILED = 4
FLAG_NAN_INPUT = 8

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [_SRC] + [os.path.join(_HERE, f) for f in sorted(os.listdir(_HERE))
                     if f.endswith(".c") and f != "kf_oracle.c"]
    stale = force or not os.path.exists(_LIB) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB) for s in srcs)
    if stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp] + srcs + ["-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def build_op_count(force: bool = False) -> str:
    """Compile the operation-counting build of the oracle (kf_opcount.cpp,
    which includes kf_oracle.c) with g++."""
    src = os.path.join(_HERE, "kf_opcount.cpp")
    so = os.path.join(_BUILD, "libkf_opcount.so")
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(so) or any(os.path.getmtime(d) > os.path.getmtime(so) for d in (src, _SRC)):
        tmp = so + f".{os.getpid()}.tmp"
        subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                        "-o", tmp, src], check=True)
        os.replace(tmp, so)
    return so


def op_count_fit(batch) -> dict:
    """Operations the FP64 oracle performs to fit a ``synth.FitBatch``: its
    own source compiled with a counting scalar type (kf_opcount.cpp).  Returns
    the counts by kind and the layers processed."""
    cl = ctypes.CDLL(build_op_count())
    cl.orc_count_fit.restype = ctypes.c_int
    cl.orc_count_fit.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_int64] + \
        [ctypes.c_void_p] * 7
    g = batch.geom
    f32 = lambda v: np.ascontiguousarray(np.asarray(v, dtype=np.float32).astype(np.float64))
    r, xx0 = f32(g.radii), f32(g.x_over_x0)
    arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (batch.seed_state, batch.seed_cov)]
    q = np.ascontiguousarray(batch.charge, dtype=np.int8)
    hp = np.ascontiguousarray(batch.hit_pos, dtype=np.float32)
    hc = np.ascontiguousarray(batch.hit_cov, dtype=np.float32)
    mask = np.ascontiguousarray(batch.hit_mask, dtype=np.uint32)
    counts = np.zeros(7, dtype=np.uint64)
    rc = cl.orc_count_fit(len(r), _p(r), _p(xx0), float(np.float32(g.z_half)), float(np.float32(g.bz)),
                          int(batch.n_tracks), arrs[0].ctypes.data, arrs[1].ctypes.data, q.ctypes.data,
                          hp.ctypes.data, hc.ctypes.data, mask.ctypes.data, counts.ctypes.data)
    assert rc == 0
    names = ("add", "mul", "div", "sqrt", "call", "total", "layers")
    return {k: int(v) for k, v in zip(names, counts)}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _lib.orc_propagate.restype = ctypes.c_int
            _lib.orc_propagate.argtypes = [_dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           _dp, _dp, _dp]
            _lib.orc_ms_noise.argtypes = [_dp, ctypes.c_double, _dp]
            _lib.orc_inv3_cholesky.restype = ctypes.c_int
            _lib.orc_inv3_cholesky.argtypes = [_dp, _dp]
            _lib.orc_update.restype = ctypes.c_int
            _lib.orc_update.argtypes = [_dp, _dp, _dp, _dp, _dp]
            _lib.orc_transport.argtypes = [_dp, _dp, _dp]
            _lib.orc_build_prepare.restype = None
            _lib.orc_build_prepare.argtypes = [ctypes.c_int64] + [ctypes.c_void_p] * 2 + [ctypes.c_int64] + \
                [ctypes.c_void_p] * 2
            _lib.orc_build_tracks.restype = ctypes.c_int
            _lib.orc_build_tracks.argtypes = (
                [ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                 ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                 ctypes.c_int64, ctypes.c_int64] + [ctypes.c_void_p] * 4 +
                [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double] +
                [ctypes.c_void_p] * 6)
            _lib.orc_build_tracks_ex.restype = ctypes.c_int
            _lib.orc_build_tracks_ex.argtypes = _lib.orc_build_tracks.argtypes + \
                [ctypes.c_void_p] * 3 + [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_void_p]
            _lib.orc_smooth_tracks.restype = ctypes.c_int
            _lib.orc_smooth_tracks.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_int64, ctypes.c_int64, ctypes.c_int64] + \
                [ctypes.c_void_p] * 10
            _lib.orc_propagate_back.restype = ctypes.c_int
            _lib.orc_propagate_back.argtypes = [_dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp]
            _lib.orc_triplet_circle.restype = ctypes.c_int
            _lib.orc_triplet_circle.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp]
            _lib.orc_seed_triplets.restype = ctypes.c_int64
            _lib.orc_seed_triplets.argtypes = [_dp] + [ctypes.c_double] * 5 + \
                [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                 ctypes.c_void_p, ctypes.c_int64]
            _lib.orc_bf16_round.restype = ctypes.c_double
            _lib.orc_bf16_round.argtypes = [ctypes.c_double]
            _lib.orc_mlp_logit.restype = ctypes.c_double
            _lib.orc_mlp_logit.argtypes = [_dp, _dp, ctypes.c_int]
            for fn in (_lib.orc_fit_tracks, _lib.orc_fit_tracks_f64):
                fn.restype = ctypes.c_int
                fn.argtypes = ([ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]
                               + [ctypes.c_void_p] * 13)
        return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# single-state helpers (pins call these)


def propagate(state, q, bz, r, jacobian=True):
    """Returns (ok, new_state, J or None, s)."""
    st = _f64(state).copy()
    out = np.zeros(6)
    J = np.zeros(36) if jacobian else None
    s = ctypes.c_double(0.0)
    rc = lib().orc_propagate(_p(st), int(q), float(bz), float(r), _p(out),
                             _p(J) if jacobian else None, ctypes.byref(s))
    return rc == 0, out, (J.reshape(6, 6) if jacobian else None), s.value


def ms_noise(state, x_over_x0):
    Q = np.zeros(36)
    lib().orc_ms_noise(_p(_f64(state).copy()), float(x_over_x0), _p(Q))
    return Q.reshape(6, 6)


def inv3(S):
    out = np.zeros(9)
    rc = lib().orc_inv3_cholesky(_p(_f64(S).reshape(9).copy()), _p(out))
    return rc == 0, out.reshape(3, 3)


def update(x, C, m, V_packed):
    """Returns (ok, x', C', dchi2)."""
    x = _f64(x).copy()
    C = _f64(C).reshape(36).copy()
    d = ctypes.c_double(0.0)
    rc = lib().orc_update(_p(x), _p(C), _p(_f64(m).copy()), _p(_f64(V_packed).copy()),
                          ctypes.byref(d))
    return rc == 0, x, C.reshape(6, 6), d.value


def transport(J, C, Q):
    C = _f64(C).reshape(36).copy()
    lib().orc_transport(_p(_f64(J).reshape(36).copy()), _p(C), _p(_f64(Q).reshape(36).copy()))
    return C.reshape(6, 6)


# ---------------------------------------------------------------------------
# batch fit


def fit_arrays(radii, x_over_x0, z_half, bz, seed_state, seed_cov, charge, hit_pos, hit_cov,
               hit_mask, threads: int | None = None, per_layer: bool = False,
               track_range: tuple[int, int] | None = None, double_inputs: bool = False):
    """Fit a batch with the FP64 oracle.  Input arrays use the library layout
    (float32 SoA, or float64 with ``double_inputs``).  Returns a dict of
    float64 results; with ``track_range`` only that slice is fitted (other
    entries are left zero)."""
    T = int(charge.shape[0])
    L = int(len(radii))
    real = np.float64 if double_inputs else np.float32
    ss = np.ascontiguousarray(seed_state, dtype=real)
    sc = np.ascontiguousarray(seed_cov, dtype=real)
    ch = np.ascontiguousarray(charge, dtype=np.int8)
    hp = np.ascontiguousarray(hit_pos, dtype=real)
    hc = np.ascontiguousarray(hit_cov, dtype=real)
    hm = np.ascontiguousarray(hit_mask, dtype=np.uint32)
    rad = _f64(radii)
    xx0 = _f64(x_over_x0)
    out = dict(state=np.zeros((6, T)), cov=np.zeros((21, T)), chi2=np.zeros(T),
               ndof=np.zeros(T, dtype=np.int32), flags=np.zeros(T, dtype=np.uint32))
    if per_layer:
        out["layer_state"] = np.zeros((L, 6, T))
        out["layer_cov"] = np.zeros((L, 21, T))
    t0, t1 = track_range if track_range is not None else (0, T)
    if t1 <= t0:
        return out
    threads = threads or os.cpu_count() or 1
    chunk = max(1, -(-(t1 - t0) // (threads * 4)))
    ranges = [(a, min(a + chunk, t1)) for a in range(t0, t1, chunk)]
    L_ = lib()
    fn = L_.orc_fit_tracks_f64 if double_inputs else L_.orc_fit_tracks
    ptr = lambda a: a.ctypes.data if a is not None else None

    def run(rg):
        return fn(L, _p(rad), _p(xx0), float(z_half), float(bz), rg[0], rg[1], T,
                                 ptr(ss), ptr(sc), ptr(ch), ptr(hp), ptr(hc), ptr(hm),
                                 ptr(out["state"]), ptr(out["cov"]), ptr(out["chi2"]),
                                 ptr(out["ndof"]), ptr(out["flags"]),
                                 ptr(out.get("layer_state")), ptr(out.get("layer_cov")))

    if threads == 1 or len(ranges) == 1:
        for rg in ranges:
            run(rg)
    else:
        with cf.ThreadPoolExecutor(threads) as ex:
            list(ex.map(run, ranges))
    return out


def fit_batch(batch, threads=None, per_layer=False, track_range=None):
    """Fit a ``synth.FitBatch``."""
    g = batch.geom
    f32 = lambda v: np.asarray(v, dtype=np.float32).astype(np.float64)  # the library's inputs
    return fit_arrays(f32(g.radii), f32(g.x_over_x0), float(np.float32(g.z_half)),
                      float(np.float32(g.bz)), batch.seed_state, batch.seed_cov,
                      batch.charge, batch.hit_pos, batch.hit_cov, batch.hit_mask, threads,
                      per_layer, track_range)


def fit_batch_exact(batch, threads=None, per_layer=False):
    """Fit a ``synth.FitBatch`` from its float64 arrays (before the rounding to
    float32 that the library's inputs carry), in the batch's float64 geometry."""
    g, e = batch.geom, batch.exact
    return fit_arrays(g.radii, g.x_over_x0, g.z_half, g.bz, e["seed_state"], e["seed_cov"],
                      batch.charge, e["hit_pos"], e["hit_cov"], batch.hit_mask, threads,
                      per_layer, None, double_inputs=True)


def smooth_batch(batch, threads=None, track_range=None):
    """Forward fit + Rauch-Tung-Striebel smoother of a ``synth.FitBatch`` in
    FP64.  Returns state [L][6][T] and cov [L][21][T] (smoothed, NaN where the
    fit did not reach), filt_state [L][6][T] (forward filter) and reached [T]."""
    g = batch.geom
    T = batch.n_tracks
    L = g.n_layers
    f32 = lambda v: np.asarray(v, dtype=np.float32).astype(np.float64)
    arr = lambda a, dt: np.ascontiguousarray(a, dtype=dt)
    ss, sc = arr(batch.seed_state, np.float32), arr(batch.seed_cov, np.float32)
    ch, hm = arr(batch.charge, np.int8), arr(batch.hit_mask, np.uint32)
    hp, hc = arr(batch.hit_pos, np.float32), arr(batch.hit_cov, np.float32)
    out = dict(state=np.zeros((L, 6, T)), cov=np.zeros((L, 21, T)), filt_state=np.zeros((L, 6, T)),
               reached=np.zeros(T, dtype=np.int32))
    rad, xx0 = f32(g.radii), f32(g.x_over_x0)
    t0, t1 = track_range if track_range is not None else (0, T)
    threads = threads or os.cpu_count() or 1
    chunk = max(1, -(-(t1 - t0) // (threads * 4)))
    ranges = [(a, min(a + chunk, t1)) for a in range(t0, t1, chunk)]

    def run(rg):
        rc = lib().orc_smooth_tracks(L, _p(rad), _p(xx0), float(np.float32(g.z_half)), float(np.float32(g.bz)),
                                     rg[0], rg[1], T, ss.ctypes.data, sc.ctypes.data, ch.ctypes.data,
                                     hp.ctypes.data, hc.ctypes.data, hm.ctypes.data, out["state"].ctypes.data,
                                     out["cov"].ctypes.data, out["filt_state"].ctypes.data,
                                     out["reached"].ctypes.data)
        assert rc == 0

    if len(ranges) <= 1:
        for rg in ranges:
            run(rg)
    else:
        with cf.ThreadPoolExecutor(threads) as ex:
            list(ex.map(run, ranges))
    return out


SEED_DEFAULTS = dict(pt_min=0.3, d0_max=0.15, z0_max=4.0, dz_max=0.8, pt_both_charges=2.0)


def triplet_circle(p0, p1, p2):
    """(curvature, distance of the origin to the circle, orientation) of three
    (x, y) points, or None if collinear."""
    k, d0, o = (ctypes.c_double() for _ in range(3))
    rc = lib().orc_triplet_circle(_p(_f64(p0).copy()), _p(_f64(p1).copy()), _p(_f64(p2).copy()),
                                  ctypes.byref(k), ctypes.byref(d0), ctypes.byref(o))
    return (k.value, d0.value, o.value) if rc else None


def seed_triplets(events, **opt):
    """Seeding triplets of a ``synth.BuildEvents`` with seed-layer hits:
    int64 [n][4] (event, h0, h1, h2), sorted."""
    o_ = dict(SEED_DEFAULTS, **opt)  # pt_both_charges only decides which charges a triplet seeds
    g = events.geom
    r = np.asarray(g.radii[:3], dtype=np.float32).astype(np.float64)
    hp = np.ascontiguousarray(events.seed_hit_pos, dtype=np.float32)
    off = np.ascontiguousarray(events.seed_hit_offsets, dtype=np.int64)
    H = hp.shape[1]
    E = off.shape[0]
    bz = float(np.float32(g.bz))

    def run(e0, e1, cap):
        out = np.zeros((max(cap, 1), 4), dtype=np.int64)
        n = lib().orc_seed_triplets(_p(r), bz, o_["pt_min"], o_["d0_max"], o_["z0_max"], o_["dz_max"],
                                    hp.ctypes.data, H, off.ctypes.data, e0, e1, out.ctypes.data, cap)
        assert n >= 0
        return n, out

    parts = []
    for e in range(E):
        n, _ = run(e, e + 1, 0)
        n2, out = run(e, e + 1, n)
        assert n2 == n
        parts.append(out[:n])
    t = np.concatenate(parts) if parts else np.zeros((0, 4), dtype=np.int64)
    return t[np.lexsort((t[:, 3], t[:, 1], t[:, 2], t[:, 0]))]


def seed_fit_inputs(events, trip, pt_min=0.3, pt_both_charges=2.0, pt_unresolved=6.0, p_sigma_resolved=0.3,
                    p_sigma_unresolved=1.0):
    """The seed fit's inputs of seeding triplets [n][4] in FP64, from the
    recipe's definition: one seed per charge the triplet seeds (its turning
    sense's, and the other as well when the circle's pT is at least
    pt_both_charges); the state 1 cm before the first hit along the circle's
    tangent there, pT from the circle (pt_unresolved for a two-charge triplet,
    whose curvature the three hits do not measure), pz from the first chord's
    slope; a diagonal covariance with sigma 10% of each position component and
    p_sigma_resolved (p_sigma_unresolved for a two-charge triplet) of each
    momentum component, floors 1e-4 cm, 1e-3 GeV.  Returns arrays sorted by
    the key (event, h0, h1, h2, charge)."""
    hp = events.seed_hit_pos.astype(np.float64)
    hc = events.seed_hit_cov.astype(np.float64)
    bz = float(np.float32(events.geom.bz))
    k_field = 0.00299792458
    kamb = k_field * abs(bz) / pt_both_charges
    keys, states, covs = [], [], []
    for e, h0, h1, h2 in trip:
        P = [hp[:2, h] for h in (h0, h1, h2)]
        r = triplet_circle(*P)
        k, orient = (r[0], r[2]) if r is not None else (0.0, 0.0)
        both = abs(k) <= kamb
        q0 = 1 if orient * bz < 0 else -1
        for q in ((q0, -q0) if both else (q0,)):
            pt = pt_unresolved if both else k_field * abs(bz) / abs(k)
            ka = k_field * abs(bz) / pt
            a = P[1] - P[0]
            alen = np.hypot(*a)
            turn = 1.0 if q * bz < 0 else -1.0
            half = np.arcsin(min(1.0, 0.5 * alen * ka)) * turn
            c, s_ = np.cos(-half), np.sin(-half)
            cx, cy = a / alen
            tx, ty = c * cx - s_ * cy, s_ * cx + c * cy
            tanl = (hp[2, h1] - hp[2, h0]) / alen
            st = np.array([P[0][0] - tx, P[0][1] - ty, hp[2, h0] - tanl, pt * tx, pt * ty, pt * tanl])
            rel = np.array([0.1, 0.1, 0.1] + [p_sigma_unresolved if both else p_sigma_resolved] * 3)
            fl = np.array([1e-4] * 3 + [1e-3] * 3)
            cv = np.zeros(21)
            for i in range(6):
                cv[i * (i + 1) // 2 + i] = (rel[i] * st[i]) ** 2 + fl[i] ** 2
            keys.append((e, h0, h1, h2, q))
            states.append(st)
            covs.append(cv)
    key = np.array(keys, dtype=np.int64).reshape(-1, 5)
    order = np.lexsort((key[:, 4], key[:, 3], key[:, 1], key[:, 2], key[:, 0])) if len(key) else np.zeros(0, int)
    key = key[order]
    n = len(key)
    hits = key[:, 1:4].T
    return dict(key=key, seed_state=np.array(states).reshape(-1, 6)[order].T if n else np.zeros((6, 0)),
                seed_cov=np.array(covs).reshape(-1, 21)[order].T if n else np.zeros((21, 0)),
                charge=key[:, 4].astype(np.int8), event=key[:, 0].astype(np.int32),
                hit_pos=np.stack([hp[:, hits[l]] for l in range(3)]) if n else np.zeros((3, 3, 0)),
                hit_cov=np.stack([hc[:, hits[l]] for l in range(3)]) if n else np.zeros((3, 6, 0)),
                hit_mask=np.full(n, 7, dtype=np.uint32))


def propagate_back(state, q, bz, r):
    """The crossing of radius r backwards along the helix (None if unreachable)."""
    out = np.zeros(6)
    rc = lib().orc_propagate_back(_p(_f64(state).copy()), int(q), float(bz), float(r), _p(out))
    return None if rc else out


# ---------------------------------------------------------------------------
# combinatorial build


def build_arrays(radii, x_over_x0, z_half, bz, hit_offsets, hit_pos, hit_cov, seed_event, seed_state,
                 seed_cov, seed_charge, max_cands=6, chi2_cut=30.0, nsigma=3.0, sigma_rphi=0.01,
                 sigma_z=0.1, threads: int | None = None, seed_range=None, log=False, mlp=None, topk=4,
                 mlp_bf16=False, dphi_max=0.05, dz_max=5.0, margins=False):
    """Clone-engine build with the FP64 oracle over the given layers.  Arrays
    in the library's layout (float32 hits [3][H] / [6][H], offsets
    [E][L+1], seeds [6][S] / [21][S]).  Returns a dict of results.

    log=True adds the training log of the plain build: out["log"] = dict of
    features [n][12], labels [n], ref [n][4] (seed, candidate, layer, hit),
    rows in seed order.  mlp (5,057 float64 weights) turns on the learned
    proposal with the given topk; mlp_bf16 ranks with BF16 inputs, W1, W2 and
    first hidden layer (the tensor-core scoring's precision).  dphi_max (rad)
    and dz_max (cm) cap the window's half-widths (None: no cap).  margins=True
    adds out["margin"] [S][4]: per seed, how close its window tests, chi2 cuts,
    rankings and top-k choices came to going the other way (the C oracle's
    out_margin), for tracing a parity mismatch to a near-tie."""
    if log and mlp is not None:
        raise ValueError("the training log records the plain build")
    L = int(len(radii))
    hp = np.ascontiguousarray(hit_pos, dtype=np.float32)
    hc = np.ascontiguousarray(hit_cov, dtype=np.float32)
    off = np.ascontiguousarray(hit_offsets, dtype=np.int64)
    H = int(hp.shape[1])
    S = int(len(seed_event))
    N = int(max_cands)
    phi = np.zeros(H)
    order = np.zeros(H, dtype=np.int64)
    bounds = _segment_bounds(off, L)  # kept alive across the call
    lib().orc_build_prepare(off.shape[0] * L, bounds.ctypes.data, hp.ctypes.data, H,
                            phi.ctypes.data, order.ctypes.data)
    se = np.ascontiguousarray(seed_event, dtype=np.int32)
    ss = np.ascontiguousarray(seed_state, dtype=np.float32)
    sc = np.ascontiguousarray(seed_cov, dtype=np.float32)
    sq = np.ascontiguousarray(seed_charge, dtype=np.int8)
    out = dict(hit=np.zeros((S, N, L), dtype=np.int32), chi2=np.zeros((S, N)),
               nhits=np.zeros((S, N), dtype=np.int32), state=np.zeros((6, S * N)),
               cov=np.zeros((21, S * N)), ncand=np.zeros(S, dtype=np.int32))
    if margins:
        out["margin"] = np.full((S, 4), np.inf)
    rad, xx0 = _f64(radii), _f64(x_over_x0)
    s0, s1 = seed_range if seed_range is not None else (0, S)
    threads = threads or os.cpu_count() or 1
    chunk = max(1, -(-(s1 - s0) // (threads * 4)))
    ranges = [(a, min(a + chunk, s1)) for a in range(s0, s1, chunk)]

    w = None if mlp is None else np.ascontiguousarray(mlp, dtype=np.float64)
    if w is not None and w.shape != (5057,):
        raise ValueError("mlp must hold 5,057 weights")

    def call(rg, lg):
        n = np.zeros(1, dtype=np.int64)
        cap = 0 if lg is None else len(lg["labels"])
        rc = lib().orc_build_tracks_ex(
            L, _p(rad), _p(xx0), float(z_half), float(bz), off.ctypes.data, hp.ctypes.data, hc.ctypes.data, H,
            phi.ctypes.data, order.ctypes.data, rg[0], rg[1], S, se.ctypes.data, ss.ctypes.data, sc.ctypes.data,
            sq.ctypes.data, N, float(chi2_cut), float(nsigma), float(sigma_rphi), float(sigma_z),
            out["hit"].ctypes.data, out["chi2"].ctypes.data, out["nhits"].ctypes.data, out["state"].ctypes.data,
            out["cov"].ctypes.data, out["ncand"].ctypes.data,
            None if lg is None else lg["features"].ctypes.data, None if lg is None else lg["labels"].ctypes.data,
            None if lg is None else lg["ref"].ctypes.data, cap, n.ctypes.data if log else None,
            None if w is None else w.ctypes.data, int(topk), int(bool(mlp_bf16)),
            math.inf if dphi_max is None else float(dphi_max), math.inf if dz_max is None else float(dz_max),
            out["margin"].ctypes.data if margins else None)
        assert rc == 0, rc
        return int(n[0])

    def run(rg):
        if not log:
            call(rg, None)
            return None
        n = call(rg, None)  # count the rows, then fill them
        lg = dict(features=np.zeros((n, 12)), labels=np.zeros(n), ref=np.zeros((n, 4), dtype=np.int32))
        assert call(rg, lg) == n
        return lg

    if len(ranges) <= 1:
        logs = [run(rg) for rg in ranges]
    else:
        with cf.ThreadPoolExecutor(threads) as ex:
            logs = list(ex.map(run, ranges))
    if log:
        logs = [lg for lg in logs if lg is not None]
        out["log"] = {k: (np.concatenate([lg[k] for lg in logs]) if logs else
                          np.zeros((0,) + ((12,) if k == "features" else (4,) if k == "ref" else ()),
                                   dtype=np.int32 if k == "ref" else np.float64))
                      for k in ("features", "labels", "ref")}
    return out


def bf16_round(v: float) -> float:
    """v rounded to float32, then to bfloat16 (nearest, ties to even)."""
    return lib().orc_bf16_round(float(v))


def mlp_logit(weights, features, bf16=False) -> float:
    """The build oracle's scoring of one (candidate, hit) pair."""
    w = np.ascontiguousarray(weights, dtype=np.float64)
    f = np.ascontiguousarray(features, dtype=np.float64)
    assert w.shape == (5057,) and f.shape == (12,)
    return lib().orc_mlp_logit(_p(w), _p(f), int(bool(bf16)))


def _segment_bounds(off, L):
    """Flattened segment boundaries [E*L + 1] of the offsets table [E][L+1]
    (segments of one event are contiguous; events may follow one another or
    not, so each segment's end is taken from its own row)."""
    E = off.shape[0]
    b = np.zeros(E * L + 1, dtype=np.int64)
    if E == 0:
        return b
    b[:-1] = off[:, :L].reshape(-1)
    b[-1] = off[-1, L]
    # an event's last segment ends at off[e, L]; the next event's first
    # segment must start there for the flattening to hold
    assert np.all(off[1:, 0] == off[:-1, L]), "events must be stored back to back"
    return np.ascontiguousarray(b)


def fit_seeds(events, threads=None):
    """Seed states of a ``synth.BuildEvents``: the oracle fit of the seed hits."""
    return fit_batch(events.seed_fit, threads)


def build_events(events, seeds=None, threads=None, **opt):
    """Build a ``synth.BuildEvents`` with the oracle; ``seeds`` is a dict with
    float32 state [6][S] and cov [21][S] (default: the oracle's seed fit)."""
    if seeds is None:
        f = fit_seeds(events, threads)
        seeds = dict(state=f["state"].astype(np.float32), cov=f["cov"].astype(np.float32))
    g = events.build_geom
    f32 = lambda v: np.asarray(v, dtype=np.float32).astype(np.float64)
    return build_arrays(f32(g.radii), f32(g.x_over_x0), float(np.float32(g.z_half)), float(np.float32(g.bz)),
                        events.hit_offsets, events.hit_pos, events.hit_cov, events.seed_event, seeds["state"],
                        seeds["cov"], events.seed_fit.charge, threads=threads, **opt)
