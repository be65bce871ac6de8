"""Python binding of the C library (``include/kf.h``): argument marshalling only.

Every step of the fit and the build runs in the library's CUDA kernels; this
module turns torch CUDA tensors into the pointers, sizes and stream the C
entry points take, and allocates output tensors.  It has no fallback: if the
compiled library is missing or no sm_103a device is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import torch

from . import build as _build

HEADER = os.path.join(_build.INCLUDE, "kf.h")

KF_OK = 0
FLAG_UNREACHABLE = 1
FLAG_LEFT_BARREL = 2
FLAG_INVERSION_FAILED = 4
FLAG_NAN_INPUT = 8
FLAG_FP64_PATH = 16
FLAG_PSD_REPAIRED = 32
PRECISION_FP32 = 0
PRECISION_ROUTED = 1
LAUNCH_AUTO = 0
LAUNCH_PER_EVENT = 1
LAUNCH_FLAT = 2


class KFError(RuntimeError):
    pass


class Geometry(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int), ("r", ctypes.POINTER(ctypes.c_float)),
                ("x_over_x0", ctypes.POINTER(ctypes.c_float)), ("z_half", ctypes.c_float),
                ("bz_tesla", ctypes.c_float)]


class Options(ctypes.Structure):
    _fields_ = [("precision_mode", ctypes.c_int), ("cond_max", ctypes.c_float),
                ("pt_lo", ctypes.c_float), ("pt_hi", ctypes.c_float), ("gain_max", ctypes.c_float),
                ("launch_mode", ctypes.c_int), ("tracks_per_block", ctypes.c_int),
                ("reg_cap", ctypes.c_int), ("hit_prefetch", ctypes.c_int), ("max_cands", ctypes.c_int),
                ("chi2_cut", ctypes.c_float), ("window_nsigma", ctypes.c_float),
                ("hit_sigma_rphi", ctypes.c_float), ("hit_sigma_z", ctypes.c_float),
                ("window_max_dphi", ctypes.c_float), ("window_max_dz", ctypes.c_float),
                ("n_phi_bins", ctypes.c_int), ("n_z_bins", ctypes.c_int),
                ("use_proposal", ctypes.c_int), ("topk", ctypes.c_int), ("build_variant", ctypes.c_int)]


_lib = None
_vp = ctypes.c_void_p


def library_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Load the compiled library (``build()`` must have produced it)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise KFError(f"{path} is missing: run paper_1705_02876_gb300.build.build() first")
        L = ctypes.CDLL(path)
        L.kf_options_default.argtypes = [ctypes.POINTER(Options)]
        L.kf_options_default.restype = None
        L.kf_context_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int]
        L.kf_context_destroy.argtypes = [_vp]
        L.kf_context_destroy.restype = None
        L.kf_last_error.argtypes = [_vp]
        L.kf_last_error.restype = ctypes.c_char_p
        L.kf_fit_tracks.argtypes = [_vp, ctypes.POINTER(Geometry), ctypes.c_int64, _vp, ctypes.c_int] + \
            [_vp] * 11 + [ctypes.POINTER(Options), _vp]
        L.kf_fit_tracks_host.argtypes = [_vp, ctypes.POINTER(Geometry), ctypes.c_int64] + [_vp] * 11 + \
            [ctypes.c_int64, ctypes.POINTER(Options)]
        L.kf_seeding_default.argtypes = [ctypes.POINTER(Seeding)]
        L.kf_seeding_default.restype = None
        L.kf_seed_triplets.argtypes = [_vp, ctypes.POINTER(Geometry), ctypes.c_int, _vp, _vp, ctypes.c_int64,
                                       ctypes.POINTER(Seeding), ctypes.POINTER(ctypes.c_int64), _vp]
        L.kf_seed_fetch.argtypes = [_vp, ctypes.POINTER(Geometry), _vp, _vp, ctypes.POINTER(Seeding),
                                    ctypes.c_int64] + [_vp] * 8 + [_vp]
        L.kf_smooth_tracks.argtypes = [_vp, ctypes.POINTER(Geometry), ctypes.c_int64] + [_vp] * 10 + \
            [ctypes.POINTER(Options), _vp]
        L.kf_transport_batch.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp]
        L.kf_fit_tuned_shape.argtypes = [_vp, ctypes.c_int, ctypes.c_int64] + [ctypes.POINTER(ctypes.c_int)] * 3
        L.kf_build_tracks.argtypes = [_vp, ctypes.POINTER(Geometry), ctypes.c_int, _vp, _vp, _vp,
                                      ctypes.c_int64, ctypes.c_int64] + [_vp] * 10 + \
            [ctypes.POINTER(Options), _vp]
        L.kf_build_tracks_logged.argtypes = [_vp, ctypes.POINTER(Geometry), ctypes.c_int, _vp, _vp, _vp,
                                             ctypes.c_int64, ctypes.c_int64] + [_vp] * 10 + \
            [ctypes.POINTER(Options), _vp, _vp, _vp, ctypes.c_int64, _vp, _vp]
        L.kf_proposal_gradient.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int64, _vp, ctypes.POINTER(ctypes.c_float), _vp]
        L.kf_proposal_train.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                        ctypes.POINTER(ctypes.c_float), _vp]
        L.kf_proposal_load.argtypes = [_vp, _vp, _vp]
        L.kf_load_proposal.argtypes = [_vp, _vp, ctypes.c_size_t]
        L.kf_proposal_score.argtypes = [_vp, _vp, ctypes.c_int64, _vp, _vp]
        L.kf_build_tracks_host.argtypes = [_vp, ctypes.POINTER(Geometry), ctypes.c_int, _vp, _vp, _vp,
                                           ctypes.c_int64, ctypes.c_int64] + [_vp] * 10 + \
            [ctypes.c_int, ctypes.POINTER(Options)]
        L.kf_build_tuned_shape.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                           ctypes.c_int64] + [ctypes.POINTER(ctypes.c_int)] * 3
        L.kf_proposal_score_with.argtypes = [_vp, _vp, ctypes.c_int64, _vp, ctypes.c_int, _vp]
        L.kf_proposal_status.argtypes = [_vp, ctypes.POINTER(ctypes.c_int)]
        L.kf_fit_tracks_noalloc.argtypes = [ctypes.POINTER(Geometry), ctypes.c_int64] + [_vp] * 11 + \
            [ctypes.POINTER(Options), _vp]
        _lib = L
    return _lib


def header_functions() -> list[str]:
    """Names of the functions declared in include/kf.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kf_[a-z0-9_]+)\s*\(", text)))


class Seeding(ctypes.Structure):
    _fields_ = [("pt_min", ctypes.c_float), ("d0_max", ctypes.c_float), ("z0_max", ctypes.c_float),
                ("dz_max", ctypes.c_float), ("pt_both_charges", ctypes.c_float), ("pt_unresolved", ctypes.c_float),
                ("p_sigma_resolved", ctypes.c_float), ("p_sigma_unresolved", ctypes.c_float),
                ("n_phi_bins", ctypes.c_int), ("n_z_bins", ctypes.c_int)]


def seeding(**kw) -> Seeding:
    o = Seeding()
    load().kf_seeding_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def options(**kw) -> Options:
    o = Options()
    load().kf_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Context:
    """A library context on one CUDA device."""

    def __init__(self, device: int | None = None):
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        self._h = _vp()
        rc = load().kf_context_create(ctypes.byref(self._h), self.device)
        if rc != KF_OK:
            raise KFError(f"kf_context_create failed with {rc} (needs an sm_103 device)")

    @property
    def handle(self):
        return self._h

    def check(self, rc: int, what: str):
        if rc != KF_OK:
            msg = load().kf_last_error(self._h).decode()
            raise KFError(f"{what} failed ({rc}): {msg}")

    def close(self):
        if self._h:
            load().kf_context_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build_tuned_shape(self, n_layers: int, max_cands: int, mode: int, n_seeds: int, n_hits: int):
        """(n_phi_bins, n_z_bins, speculative) the build autotuner picked, or
        None before a build of that class."""
        p_, z, sp = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        rc = load().kf_build_tuned_shape(self._h, n_layers, max_cands, mode, n_seeds, n_hits, ctypes.byref(p_),
                                         ctypes.byref(z), ctypes.byref(sp))
        return (p_.value, z.value, sp.value) if rc == KF_OK else None

    def tuned_shape(self, n_layers: int, n_tracks: int):
        """(tracks per block, register cap, hit prefetch depth) the autotuner
        picked, or None before a fit of that size class."""
        b, t, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        rc = load().kf_fit_tuned_shape(self._h, n_layers, n_tracks, ctypes.byref(b), ctypes.byref(t), ctypes.byref(d))
        return (b.value, t.value, d.value) if rc == KF_OK else None


class GeometryArgs:
    """Host-side geometry struct with its arrays kept alive."""

    def __init__(self, radii, x_over_x0, z_half, bz):
        self.r = np.ascontiguousarray(radii, dtype=np.float32)
        self.x = np.ascontiguousarray(x_over_x0, dtype=np.float32)
        fp = ctypes.POINTER(ctypes.c_float)
        self.struct = Geometry(len(self.r), self.r.ctypes.data_as(fp), self.x.ctypes.data_as(fp),
                               float(z_half), float(bz))

    @classmethod
    def of(cls, geom):
        return cls(geom.radii, geom.x_over_x0, geom.z_half, geom.bz)


def _ptr(t: torch.Tensor, dtype, shape=None, name=""):
    if t.dtype != dtype or not t.is_cuda or not t.is_contiguous():
        raise KFError(f"{name}: expected a contiguous CUDA {dtype} tensor, got {t.dtype} "
                      f"{'cuda' if t.is_cuda else 'cpu'} contiguous={t.is_contiguous()}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise KFError(f"{name}: shape {tuple(t.shape)} != {tuple(shape)}")
    return t.data_ptr() if t.numel() else None


def fit_outputs(n_tracks: int, device) -> dict:
    return dict(state=torch.empty((6, n_tracks), dtype=torch.float32, device=device),
                cov=torch.empty((21, n_tracks), dtype=torch.float32, device=device),
                chi2=torch.empty(n_tracks, dtype=torch.float32, device=device),
                ndof=torch.empty(n_tracks, dtype=torch.int16, device=device),
                flags=torch.empty(n_tracks, dtype=torch.int32, device=device))


def fit_tracks(ctx: Context, geom: GeometryArgs, seed_state, seed_cov, charge, hit_pos, hit_cov,
               hit_mask, event_offsets=None, opt: Options | None = None, out: dict | None = None,
               stream: torch.cuda.Stream | None = None) -> dict:
    """kf_fit_tracks on CUDA tensors; returns (or fills) the output tensors."""
    T = int(charge.shape[0])
    L = geom.struct.n_layers
    if out is None:
        out = fit_outputs(T, charge.device)
    args = [
        _ptr(seed_state, torch.float32, (6, T), "seed_state"),
        _ptr(seed_cov, torch.float32, (21, T), "seed_cov"),
        _ptr(charge, torch.int8, (T,), "charge"),
        _ptr(hit_pos, torch.float32, (L, 3, T), "hit_pos"),
        _ptr(hit_cov, torch.float32, (L, 6, T), "hit_cov"),
        _ptr(hit_mask, torch.int32, (T,), "hit_mask"),
        _ptr(out["state"], torch.float32, (6, T), "out_state"),
        _ptr(out["cov"], torch.float32, (21, T), "out_cov"),
        _ptr(out["chi2"], torch.float32, (T,), "out_chi2"),
        _ptr(out["ndof"], torch.int16, (T,), "out_ndof"),
        _ptr(out["flags"], torch.int32, (T,), "out_flags"),
    ]
    n_ev = 0
    ev_ptr = None
    if event_offsets is not None:
        ev = np.ascontiguousarray(event_offsets, dtype=np.int64)
        n_ev = len(ev) - 1
        ev_ptr = ev.ctypes.data
    s = stream if stream is not None else torch.cuda.current_stream(charge.device)
    rc = load().kf_fit_tracks(ctx.handle, ctypes.byref(geom.struct), T, ev_ptr, n_ev, *args,
                              ctypes.byref(opt) if opt is not None else None, s.cuda_stream)
    ctx.check(rc, "kf_fit_tracks")
    return out


def _host_ptr(t: torch.Tensor, dtype, shape, name=""):
    if t.dtype != dtype or t.is_cuda or not t.is_contiguous():
        raise KFError(f"{name}: expected a contiguous host {dtype} tensor, got {t.dtype} "
                      f"{'cuda' if t.is_cuda else 'cpu'} contiguous={t.is_contiguous()}")
    if tuple(t.shape) != tuple(shape):
        raise KFError(f"{name}: shape {tuple(t.shape)} != {tuple(shape)}")
    return t.data_ptr() if t.numel() else None


def fit_outputs_host(n_tracks: int, pin: bool = True) -> dict:
    e = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=pin)
    return dict(state=e((6, n_tracks), torch.float32), cov=e((21, n_tracks), torch.float32),
                chi2=e((n_tracks,), torch.float32), ndof=e((n_tracks,), torch.int16),
                flags=e((n_tracks,), torch.int32))


def fit_tracks_host(ctx: Context, geom: GeometryArgs, seed_state, seed_cov, charge, hit_pos, hit_cov, hit_mask,
                    opt: Options | None = None, out: dict | None = None, chunk_tracks: int = 0) -> dict:
    """kf_fit_tracks_host on host (CPU, ideally pinned) tensors: copies in,
    fits and copies out in overlapping chunks; returns when the outputs are
    filled."""
    T = int(charge.shape[0])
    L = geom.struct.n_layers
    if out is None:
        out = fit_outputs_host(T)
    args = [
        _host_ptr(seed_state, torch.float32, (6, T), "seed_state"),
        _host_ptr(seed_cov, torch.float32, (21, T), "seed_cov"),
        _host_ptr(charge, torch.int8, (T,), "charge"),
        _host_ptr(hit_pos, torch.float32, (L, 3, T), "hit_pos"),
        _host_ptr(hit_cov, torch.float32, (L, 6, T), "hit_cov"),
        _host_ptr(hit_mask, torch.int32, (T,), "hit_mask"),
        _host_ptr(out["state"], torch.float32, (6, T), "out_state"),
        _host_ptr(out["cov"], torch.float32, (21, T), "out_cov"),
        _host_ptr(out["chi2"], torch.float32, (T,), "out_chi2"),
        _host_ptr(out["ndof"], torch.int16, (T,), "out_ndof"),
        _host_ptr(out["flags"], torch.int32, (T,), "out_flags"),
    ]
    rc = load().kf_fit_tracks_host(ctx.handle, ctypes.byref(geom.struct), T, *args, int(chunk_tracks),
                                   ctypes.byref(opt) if opt is not None else None)
    ctx.check(rc, "kf_fit_tracks_host")
    return out


def to_host(batch, pin: bool = True) -> dict:
    """A ``synth.FitBatch``'s input arrays as (pinned) host tensors."""
    t = lambda a, dt: (torch.from_numpy(np.ascontiguousarray(a)).to(dtype=dt)).pin_memory() if pin else \
        torch.from_numpy(np.ascontiguousarray(a)).to(dtype=dt)
    return dict(seed_state=t(batch.seed_state, torch.float32), seed_cov=t(batch.seed_cov, torch.float32),
                charge=t(batch.charge, torch.int8), hit_pos=t(batch.hit_pos, torch.float32),
                hit_cov=t(batch.hit_cov, torch.float32), hit_mask=t(batch.hit_mask.view(np.int32), torch.int32))


def build_tracks(ctx: Context, geom: GeometryArgs, hit_offsets, hit_pos, hit_cov, seed_event, seed_state,
                 seed_cov, seed_charge, opt: Options | None = None, out: dict | None = None,
                 stream: torch.cuda.Stream | None = None, log: dict | None = None) -> dict:
    """kf_build_tracks: hit_offsets is a host int64 array [E][L+1]; every other
    array a CUDA tensor.  Returns (or fills) the output tensors.

    With `log` (a dict from new_build_log) the call is kf_build_tracks_logged:
    the log's tensors receive the training rows and its "count" the number of
    in-window pairs met."""
    opt = opt if opt is not None else options()
    N = int(opt.max_cands)
    L = geom.struct.n_layers
    S = int(seed_event.shape[0])
    H = int(hit_pos.shape[1])
    off = np.ascontiguousarray(hit_offsets, dtype=np.int64)
    dev = seed_event.device
    if out is None:
        out = dict(hit=torch.empty((S, N, L), dtype=torch.int32, device=dev),
                   chi2=torch.empty((S, N), dtype=torch.float32, device=dev),
                   nhits=torch.empty((S, N), dtype=torch.int16, device=dev),
                   state=torch.empty((6, S * N), dtype=torch.float32, device=dev),
                   cov=torch.empty((21, S * N), dtype=torch.float32, device=dev),
                   flags=torch.empty((S, N), dtype=torch.int32, device=dev))
    args = [
        off.ctypes.data if off.size else None,
        _ptr(hit_pos, torch.float32, (3, H), "hit_pos"),
        _ptr(hit_cov, torch.float32, (6, H), "hit_cov"),
        H, S,
        _ptr(seed_event, torch.int32, (S,), "seed_event"),
        _ptr(seed_state, torch.float32, (6, S), "seed_state"),
        _ptr(seed_cov, torch.float32, (21, S), "seed_cov"),
        _ptr(seed_charge, torch.int8, (S,), "seed_charge"),
        _ptr(out["hit"], torch.int32, (S, N, L), "out_hit_idx"),
        _ptr(out["chi2"], torch.float32, (S, N), "out_chi2"),
        _ptr(out["nhits"], torch.int16, (S, N), "out_nhits"),
        _ptr(out["state"], torch.float32, (6, S * N), "out_state"),
        _ptr(out["cov"], torch.float32, (21, S * N), "out_cov"),
        _ptr(out["flags"], torch.int32, (S, N), "out_flags"),
    ]
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    if log is None:
        rc = load().kf_build_tracks(ctx.handle, ctypes.byref(geom.struct), int(off.shape[0]), *args,
                                    ctypes.byref(opt), s.cuda_stream)
        ctx.check(rc, "kf_build_tracks")
        return out
    cap = int(log["labels"].shape[0])
    rc = load().kf_build_tracks_logged(
        ctx.handle, ctypes.byref(geom.struct), int(off.shape[0]), *args, ctypes.byref(opt),
        _ptr(log["features"], torch.float32, (cap, 12), "log_features"),
        _ptr(log["labels"], torch.float32, (cap,), "log_labels"),
        _ptr(log["ref"], torch.int32, (cap, 4), "log_ref"), cap,
        _ptr(log["count"], torch.int64, (1,), "log_count"), s.cuda_stream)
    ctx.check(rc, "kf_build_tracks_logged")
    return out


def build_outputs_host(n_seeds: int, max_cands: int, n_layers: int, pin: bool = True) -> dict:
    """Host output tensors of kf_build_tracks_host (page-locked by default)."""
    S, N, L = int(n_seeds), int(max_cands), int(n_layers)
    z = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=pin)
    return dict(hit=z((S, N, L), torch.int32), chi2=z((S, N), torch.float32), nhits=z((S, N), torch.int16),
                state=z((6, S * N), torch.float32), cov=z((21, S * N), torch.float32), flags=z((S, N), torch.int32))


def build_tracks_host(ctx: Context, geom: GeometryArgs, hit_offsets, hit_pos, hit_cov, seed_event, seed_state,
                      seed_cov, seed_charge, opt: Options | None = None, out: dict | None = None,
                      events_per_batch: int = 0) -> dict:
    """kf_build_tracks_host: every array a CPU tensor (page-locked for the
    overlapped copies), hit_offsets a host int64 array [E][L+1]; seeds grouped
    by event.  Returns (or fills) host output tensors; the call returns with
    every output written."""
    opt = opt if opt is not None else options()
    N = int(opt.max_cands)
    L = geom.struct.n_layers
    S = int(seed_event.shape[0])
    H = int(hit_pos.shape[1])
    off = np.ascontiguousarray(hit_offsets, dtype=np.int64)
    if out is None:
        out = build_outputs_host(S, N, L)
    args = [
        off.ctypes.data if off.size else None,
        _host_ptr(hit_pos, torch.float32, (3, H), "hit_pos"),
        _host_ptr(hit_cov, torch.float32, (6, H), "hit_cov"),
        H, S,
        _host_ptr(seed_event, torch.int32, (S,), "seed_event"),
        _host_ptr(seed_state, torch.float32, (6, S), "seed_state"),
        _host_ptr(seed_cov, torch.float32, (21, S), "seed_cov"),
        _host_ptr(seed_charge, torch.int8, (S,), "seed_charge"),
        _host_ptr(out["hit"], torch.int32, (S, N, L), "out_hit_idx"),
        _host_ptr(out["chi2"], torch.float32, (S, N), "out_chi2"),
        _host_ptr(out["nhits"], torch.int16, (S, N), "out_nhits"),
        _host_ptr(out["state"], torch.float32, (6, S * N), "out_state"),
        _host_ptr(out["cov"], torch.float32, (21, S * N), "out_cov"),
        _host_ptr(out["flags"], torch.int32, (S, N), "out_flags"),
    ]
    rc = load().kf_build_tracks_host(ctx.handle, ctypes.byref(geom.struct), int(off.shape[0]), *args,
                                     int(events_per_batch), ctypes.byref(opt))
    ctx.check(rc, "kf_build_tracks_host")
    return out


def new_build_log(capacity: int, device="cuda") -> dict:
    """Device tensors for kf_build_tracks_logged with room for `capacity` rows."""
    return dict(features=torch.empty((capacity, 12), dtype=torch.float32, device=device),
                labels=torch.empty((capacity,), dtype=torch.float32, device=device),
                ref=torch.empty((capacity, 4), dtype=torch.int32, device=device),
                count=torch.zeros((1,), dtype=torch.int64, device=device))


def log_rows(log: dict) -> int:
    """Rows written into a build log (waits for the device)."""
    return min(int(log["count"].item()), int(log["labels"].shape[0]))


PROPOSAL_PARAMS = 5057


def _cur_stream(t, stream):
    return (stream if stream is not None else torch.cuda.current_stream(t.device)).cuda_stream


def proposal_gradient(ctx: Context, weights, features, labels, stream=None):
    """(grad tensor [5057], mean loss) of the proposal network on (features, labels)."""
    n = int(labels.shape[0])
    grad = torch.empty(PROPOSAL_PARAMS, dtype=torch.float32, device=weights.device)
    loss = ctypes.c_float()
    rc = load().kf_proposal_gradient(ctx.handle, _ptr(weights, torch.float32, (PROPOSAL_PARAMS,), "weights"),
                                     _ptr(features, torch.float32, (n, 12), "features"),
                                     _ptr(labels, torch.float32, (n,), "labels"), n, grad.data_ptr(),
                                     ctypes.byref(loss), _cur_stream(weights, stream))
    ctx.check(rc, "kf_proposal_gradient")
    return grad, loss.value


def proposal_train(ctx: Context, weights, features, labels, epochs=5, batch=4096, lr=1e-3, stream=None):
    """Train ``weights`` (CUDA float32 [5057]) in place; returns the per-epoch losses."""
    n = int(labels.shape[0])
    losses = (ctypes.c_float * max(epochs, 1))()
    rc = load().kf_proposal_train(ctx.handle, _ptr(weights, torch.float32, (PROPOSAL_PARAMS,), "weights"),
                                  _ptr(features, torch.float32, (n, 12), "features"),
                                  _ptr(labels, torch.float32, (n,), "labels"), n, epochs, batch, lr, losses,
                                  _cur_stream(weights, stream))
    ctx.check(rc, "kf_proposal_train")
    return [losses[i] for i in range(epochs)]


def proposal_load(ctx: Context, weights, stream=None):
    rc = load().kf_proposal_load(ctx.handle, _ptr(weights, torch.float32, (PROPOSAL_PARAMS,), "weights"),
                                 _cur_stream(weights, stream))
    ctx.check(rc, "kf_proposal_load")


def load_proposal(ctx: Context, weights):
    """kf_load_proposal: the weights as bytes (a CUDA tensor of any dtype whose
    storage holds the 5,057 FP32 parameters), on the default stream."""
    if not weights.is_cuda or not weights.is_contiguous():
        raise KFError("weights: expected a contiguous CUDA tensor")
    rc = load().kf_load_proposal(ctx.handle, weights.data_ptr(), weights.numel() * weights.element_size())
    ctx.check(rc, "kf_load_proposal")


SCORE_AUTO, SCORE_MMA_SYNC, SCORE_TCGEN05 = 0, 1, 2


def proposal_score(ctx: Context, features, stream=None, engine: int | None = None):
    """Logits of the loaded network; engine None is kf_proposal_score (the
    engine chosen by measurement), else kf_proposal_score_with(engine)."""
    n = int(features.shape[0])
    logits = torch.empty(n, dtype=torch.float32, device=features.device)
    args = (ctx.handle, _ptr(features, torch.float32, (n, 12), "features"), n, logits.data_ptr() if n else None)
    if engine is None:
        rc = load().kf_proposal_score(*args, _cur_stream(features, stream))
    else:
        rc = load().kf_proposal_score_with(*args, int(engine), _cur_stream(features, stream))
    ctx.check(rc, "kf_proposal_score")
    return logits


def proposal_status(ctx: Context) -> bool:
    """kf_proposal_status: True if a bounded scoring wait has expired."""
    v = ctypes.c_int(0)
    ctx.check(load().kf_proposal_status(ctx.handle, ctypes.byref(v)), "kf_proposal_status")
    return bool(v.value)


def seed_triplets(ctx: Context, geom: GeometryArgs, hit_offsets, hit_pos, hit_cov, opt: Seeding | None = None,
                  stream: torch.cuda.Stream | None = None) -> dict:
    """kf_seed_triplets + kf_seed_fetch: the seeds of the seed layers' hits
    (hit_offsets host int64 [E][4], hit_pos [3][H] and hit_cov [6][H] CUDA
    tensors) as the seed fit's inputs (state, cov, charge, hit_pos, hit_cov,
    hit_mask, laid out for fit_tracks) plus event [n] and hits [3][n]."""
    off = np.ascontiguousarray(hit_offsets, dtype=np.int64)
    H = int(hit_pos.shape[1])
    dev = hit_pos.device
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    n = ctypes.c_int64()
    optp = ctypes.byref(opt) if opt is not None else None
    rc = load().kf_seed_triplets(ctx.handle, ctypes.byref(geom.struct), int(off.shape[0]),
                                 off.ctypes.data if off.size else None, _ptr(hit_pos, torch.float32, (3, H), "hit_pos"),
                                 H, optp, ctypes.byref(n), s.cuda_stream)
    ctx.check(rc, "kf_seed_triplets")
    n = int(n.value)
    e = lambda shape, dt: torch.empty(shape, dtype=dt, device=dev)
    out = dict(event=e((n,), torch.int32), hits=e((3, n), torch.int32), seed_state=e((6, n), torch.float32),
               seed_cov=e((21, n), torch.float32), charge=e((n,), torch.int8), hit_pos=e((3, 3, n), torch.float32),
               hit_cov=e((3, 6, n), torch.float32), hit_mask=e((n,), torch.int32))
    rc = load().kf_seed_fetch(ctx.handle, ctypes.byref(geom.struct), _ptr(hit_pos, torch.float32, (3, H), "hit_pos"),
                              _ptr(hit_cov, torch.float32, (6, H), "hit_cov"), optp, n,
                              *[_ptr(out[k], out[k].dtype, tuple(out[k].shape), k) for k in
                                ("event", "hits", "seed_state", "seed_cov", "charge", "hit_pos", "hit_cov",
                                 "hit_mask")], s.cuda_stream)
    ctx.check(rc, "kf_seed_fetch")
    return out


def smooth_tracks(ctx: Context, geom: GeometryArgs, seed_state, seed_cov, charge, hit_pos, hit_cov, hit_mask,
                  opt: Options | None = None, out: dict | None = None,
                  stream: torch.cuda.Stream | None = None) -> dict:
    """kf_smooth_tracks on CUDA tensors: the smoothed state [L][6][T] and
    covariance [L][21][T] after every layer, layers reached [T], flags [T]."""
    T = int(charge.shape[0])
    L = geom.struct.n_layers
    dev = charge.device
    if out is None:
        out = dict(state=torch.empty((L, 6, T), dtype=torch.float32, device=dev),
                   cov=torch.empty((L, 21, T), dtype=torch.float32, device=dev),
                   reached=torch.empty(T, dtype=torch.int16, device=dev),
                   flags=torch.empty(T, dtype=torch.int32, device=dev))
    args = [
        _ptr(seed_state, torch.float32, (6, T), "seed_state"),
        _ptr(seed_cov, torch.float32, (21, T), "seed_cov"),
        _ptr(charge, torch.int8, (T,), "charge"),
        _ptr(hit_pos, torch.float32, (L, 3, T), "hit_pos"),
        _ptr(hit_cov, torch.float32, (L, 6, T), "hit_cov"),
        _ptr(hit_mask, torch.int32, (T,), "hit_mask"),
        _ptr(out["state"], torch.float32, (L, 6, T), "out_state"),
        _ptr(out["cov"], torch.float32, (L, 21, T), "out_cov"),
        _ptr(out["reached"], torch.int16, (T,), "out_reached"),
        _ptr(out["flags"], torch.int32, (T,), "out_flags"),
    ]
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    rc = load().kf_smooth_tracks(ctx.handle, ctypes.byref(geom.struct), T, *args,
                                 ctypes.byref(opt) if opt is not None else None, s.cuda_stream)
    ctx.check(rc, "kf_smooth_tracks")
    return out


def transport_batch(ctx: Context, J, C, stream=None):
    """kf_transport_batch: C [21][n] <- J C J^T in place, J [36][n] (CUDA tensors)."""
    n = int(C.shape[1])
    rc = load().kf_transport_batch(ctx.handle, n, _ptr(J, torch.float32, (36, n), "J"),
                                   _ptr(C, torch.float32, (21, n), "C"), _cur_stream(C, stream))
    ctx.check(rc, "kf_transport_batch")
    return C


def to_device(batch, device="cuda") -> dict:
    """Copy a ``synth.FitBatch``'s input arrays to the device."""
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(device=device, dtype=dt)
    return dict(seed_state=t(batch.seed_state, torch.float32), seed_cov=t(batch.seed_cov, torch.float32),
                charge=t(batch.charge, torch.int8), hit_pos=t(batch.hit_pos, torch.float32),
                hit_cov=t(batch.hit_cov, torch.float32),
                hit_mask=t(batch.hit_mask.view(np.int32), torch.int32))


def fit_tracks_noalloc(geom: GeometryArgs, seed_state, seed_cov, charge, hit_pos, hit_cov, hit_mask,
                       out: dict, opt: Options | None = None,
                       stream: torch.cuda.Stream | None = None) -> int:
    """kf_fit_tracks_noalloc on CUDA tensors: the fit without a context, for
    callers that cannot allocate device memory.  The caller provides the
    output tensors; returns the C status code (KF_OK is 0)."""
    T = int(charge.shape[0])
    L = geom.struct.n_layers
    args = [
        _ptr(seed_state, torch.float32, (6, T), "seed_state"),
        _ptr(seed_cov, torch.float32, (21, T), "seed_cov"),
        _ptr(charge, torch.int8, (T,), "charge"),
        _ptr(hit_pos, torch.float32, (L, 3, T), "hit_pos"),
        _ptr(hit_cov, torch.float32, (L, 6, T), "hit_cov"),
        _ptr(hit_mask, torch.int32, (T,), "hit_mask"),
        _ptr(out["state"], torch.float32, (6, T), "out_state"),
        _ptr(out["cov"], torch.float32, (21, T), "out_cov"),
        _ptr(out["chi2"], torch.float32, (T,), "out_chi2"),
        _ptr(out["ndof"], torch.int16, (T,), "out_ndof"),
        _ptr(out["flags"], torch.int32, (T,), "out_flags"),
    ]
    s = stream if stream is not None else torch.cuda.current_stream(charge.device)
    return load().kf_fit_tracks_noalloc(ctypes.byref(geom.struct), T, *args,
                                        ctypes.byref(opt) if opt is not None else None, s.cuda_stream)
