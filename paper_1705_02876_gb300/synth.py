"""Seeded synthetic toy-detector events (Section 3.2: concentric cylinders,
Gaussian hit smearing, in-house simulation).

This module is data only.  It draws random numbers and simulates the toy
detector's truth: helix crossings of the cylinders in a uniform solenoid field,
Gaussian smearing of the crossings into hits, and multiple-scattering kicks of
the momentum direction.  It holds none of the Kalman filter's arithmetic (no
covariance transport, no update) and shares no code with the CUDA library or
with the oracle; both consume the arrays returned here.

The truth crossing is found by a bracketed Newton iteration on the transverse
path length, written in displacement form.  That is a different formulation
from both the oracle (closed-form circle-circle intersection) and the CUDA
kernels (half-angle quadratic), so a formula error on either side cannot be
shared with the truth.

Every random stream is a child of one ``numpy.random.SeedSequence(seed)``; each
purpose draws from its own child and draws for every track at every layer, so a
stream never depends on which tracks are still alive.

Conventions (shared inputs, not arithmetic of the method):
  * state = (x, y, z, px, py, pz) in cm and GeV, global Cartesian (Section 2.1)
  * packed symmetric matrices store the lower triangle row by row:
    (0,0), (1,0), (1,1), (2,0), (2,1), (2,2), ...
  * K_FIELD = 0.00299792458 GeV / (cm T): pT = K_FIELD * Bz * R
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

K_FIELD = 0.00299792458
DIAG6 = (0, 2, 5, 9, 14, 20)  # packed indices of the diagonal of a 6x6


@dataclasses.dataclass
class Geometry:
    """Barrel of concentric cylinders (Section 3.2)."""
    radii: np.ndarray          # [L] cm, increasing
    x_over_x0: np.ndarray      # [L] radiation lengths at normal incidence
    z_half: float = 100.0      # cm
    bz: float = 3.8            # tesla

    @property
    def n_layers(self) -> int:
        return int(len(self.radii))

    def sub(self, first: int, last: int) -> "Geometry":
        return Geometry(self.radii[first:last].copy(), self.x_over_x0[first:last].copy(),
                        self.z_half, self.bz)


def toy_geometry(n_layers: int = 10, spacing: float = 4.0, z_half: float = 100.0,
                 bz: float = 3.8, x_over_x0: float = 0.01) -> Geometry:
    """Equally spaced fixed-length cylinders at r = spacing * (1..n_layers)."""
    radii = spacing * np.arange(1, n_layers + 1, dtype=np.float64)
    return Geometry(radii, np.full(n_layers, x_over_x0), float(z_half), float(bz))


# ----------------------------------------------------------------------------
# random draws


def _streams(seed: int, n: int = 8):
    return [np.random.default_rng(s) for s in np.random.SeedSequence(seed).spawn(n)]


def draw_vertex_tracks(rng, n, pt_lo=0.5, pt_hi=10.0, pt_dist="uniform", eta_max=1.0,
                       vtx_sigma_xy=0.01, vtx_sigma_z=1.0):
    """Truth at the vertex: state [6, n] float64 and charge [n] int8."""
    x = rng.normal(0.0, vtx_sigma_xy, n)
    y = rng.normal(0.0, vtx_sigma_xy, n)
    z = rng.normal(0.0, vtx_sigma_z, n)
    if pt_dist == "uniform":
        pt = rng.uniform(pt_lo, pt_hi, n)
    elif pt_dist == "loguniform":
        pt = np.exp(rng.uniform(math.log(pt_lo), math.log(pt_hi), n))
    else:
        raise ValueError(pt_dist)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    eta = rng.uniform(-eta_max, eta_max, n)
    q = np.where(rng.random(n) < 0.5, 1, -1).astype(np.int8)
    st = np.stack([x, y, z, pt * np.cos(phi), pt * np.sin(phi), pt * np.sinh(eta)])
    return st, q


# ----------------------------------------------------------------------------
# truth helix in displacement form


def _sinc(a):
    return np.sinc(a / math.pi)  # sin(a)/a


def _helix_point(st, tx, ty, pt, omega, s):
    """Position and transverse direction after transverse path length s."""
    phi = omega * s
    a = s * _sinc(phi)                           # sin(phi)/omega
    b = s * (0.5 * phi) * _sinc(0.5 * phi) ** 2  # (1 - cos(phi))/omega
    x = st[0] + tx * a + ty * b
    y = st[1] + ty * a - tx * b
    c, sn = np.cos(phi), np.sin(phi)
    return x, y, tx * c + ty * sn, ty * c - tx * sn, phi


def truth_crossing(st, q, bz, r):
    """Move each truth state to its first forward crossing of radius r.

    Returns (new_state [6, n], reached [n] bool).  Tracks that cannot reach r,
    or start moving inwards, are marked unreached (their state is returned
    unchanged)."""
    st = np.asarray(st, dtype=np.float64)
    n = st.shape[1]
    pt = np.hypot(st[3], st[4])
    tx, ty = st[3] / pt, st[4] / pt
    omega = q.astype(np.float64) * K_FIELD * bz / pt
    u = st[0] * tx + st[1] * ty
    r0sq = st[0] ** 2 + st[1] ** 2
    disc = u * u + r * r - r0sq
    # a start inside the cylinder has exactly one crossing before the point of
    # the circle farthest from the axis: |P|^2 is a sinusoid in the turning angle
    reached = (disc >= 0.0) & (r0sq < r * r)
    s_line = -u + np.sqrt(np.maximum(disc, 0.0))
    # bracket [0, s_far]: below the crossing |P| < r, above it |P| > r
    curved = omega != 0.0
    om = np.where(curved, omega, 1.0)
    cx = st[0] + ty / om
    cy = st[1] - tx / om
    rho = 1.0 / np.abs(om)
    dc = np.hypot(cx, cy)
    reached &= np.where(curved, dc + rho >= r, True)
    e0x, e0y = st[0] - cx, st[1] - cy
    efx, efy = rho * cx / np.maximum(dc, 1e-300), rho * cy / np.maximum(dc, 1e-300)
    alpha = np.arctan2(e0x * efy - e0y * efx, e0x * efx + e0y * efy)
    period = 2.0 * math.pi / np.abs(om)
    s_far = np.mod(-alpha / om, period)
    s_far = np.where(curved, s_far, np.inf)
    lo = np.zeros(n)
    hi = np.where(curved, s_far, s_line * 2.0 + 1.0)
    s = np.clip(s_line, lo, hi)
    for _ in range(100):
        x, y, dx, dy, _ = _helix_point(st, tx, ty, pt, omega, s)
        f = x * x + y * y - r * r
        fp = 2.0 * (x * dx + y * dy)
        lo = np.where(f < 0.0, s, lo)
        hi = np.where(f > 0.0, s, hi)
        step = np.where(fp != 0.0, -f / np.where(fp != 0.0, fp, 1.0), 0.0)
        s_new = s + step
        bad = ~np.isfinite(s_new) | (s_new <= lo) | (s_new >= hi)
        s_new = np.where(bad, 0.5 * (lo + np.where(np.isfinite(hi), hi, 2.0 * lo + 1.0)), s_new)
        done = np.abs(s_new - s) <= 1e-14 * (1.0 + np.abs(s))
        s = s_new
        if np.all(done | ~reached):
            break
    x, y, dx, dy, phi = _helix_point(st, tx, ty, pt, omega, s)
    ok = np.abs(np.hypot(x, y) - r) < 1e-9 * max(r, 1.0)
    reached &= ok
    out = st.copy()
    out[0], out[1] = x, y
    out[2] = st[2] + st[5] * s / pt
    out[3], out[4] = pt * dx, pt * dy
    out = np.where(reached[None, :], out, st)
    return out, reached


def highland_theta0(p, pdotn_over_p, x_over_x0):
    """Highland (PDG) scattering width for beta = 1 and unit charge.

    The effective thickness is x_over_x0 / |cos(incidence)| (Section 2: the
    filter folds multiple-scattering estimates into the trajectory)."""
    xx0 = x_over_x0 / np.maximum(np.abs(pdotn_over_p), 1e-12)
    with np.errstate(divide="ignore", invalid="ignore"):
        th = 0.0136 / p * np.sqrt(xx0) * (1.0 + 0.038 * np.log(xx0))
    return np.where(xx0 > 0.0, th, 0.0)


def _kick(st, theta0, g):
    """Rotate the momentum direction by two Gaussian angles (g * theta0)
    about two axes perpendicular to p; |p| is kept."""
    p = np.sqrt(st[3] ** 2 + st[4] ** 2 + st[5] ** 2)
    ux, uy, uz = st[3] / p, st[4] / p, st[5] / p
    nt = np.hypot(ux, uy)
    e1x, e1y, e1z = -uy / nt, ux / nt, np.zeros_like(ux)
    e2x, e2y, e2z = uy * e1z - uz * e1y, uz * e1x - ux * e1z, ux * e1y - uy * e1x
    t1, t2 = g[0] * theta0, g[1] * theta0
    th = np.hypot(t1, t2)
    sc = _sinc(th)
    c = np.cos(th)
    out = st.copy()
    out[3] = p * (ux * c + sc * (t1 * e1x + t2 * e2x))
    out[4] = p * (uy * c + sc * (t1 * e1y + t2 * e2y))
    out[5] = p * (uz * c + sc * (t1 * e1z + t2 * e2z))
    return out


def hit_covariance(x, y, sigma_r, sigma_rphi, sigma_z):
    """V = sr^2 n n^T + srphi^2 t t^T + sz^2 z z^T at (x, y), packed [6, n]."""
    r = np.hypot(x, y)
    nx, ny = x / r, y / r
    tx, ty = -ny, nx
    v = np.zeros((6,) + np.shape(x))
    v[0] = sigma_r ** 2 * nx * nx + sigma_rphi ** 2 * tx * tx
    v[1] = sigma_r ** 2 * nx * ny + sigma_rphi ** 2 * tx * ty
    v[2] = sigma_r ** 2 * ny * ny + sigma_rphi ** 2 * ty * ty
    v[5] = sigma_z ** 2 * np.ones_like(r)
    return v


def simulate(rng_hit, rng_ms, rng_eff, geom: Geometry, vertex, q, sigma_rphi=0.01,
             sigma_z=0.1, sigma_r=None, hit_eff=1.0, ms=True, smear=True):
    """Step truth tracks through the barrel.

    At each layer: cross the cylinder; stop if unreachable or |z| > z_half;
    record the hit (smeared unless ``smear`` is False) if the efficiency draw
    passes; then kick the direction (if ``ms``).
    """
    if sigma_r is None:
        sigma_r = sigma_rphi
    L, n = geom.n_layers, vertex.shape[1]
    hit_pos = np.zeros((L, 3, n))
    hit_cov = np.zeros((L, 6, n))
    mask = np.zeros(n, dtype=np.uint32)
    truth = np.full((L, 6, n), np.nan)
    crossed = np.zeros((L, n), dtype=bool)
    alive = np.ones(n, dtype=bool)
    st = vertex.astype(np.float64).copy()
    for l in range(L):
        g_hit = rng_hit.standard_normal((3, n))
        u_eff = rng_eff.random(n)
        g_ms = rng_ms.standard_normal((2, n))
        new, ok = truth_crossing(st, q, geom.bz, geom.radii[l])
        alive &= ok
        alive &= np.abs(new[2]) <= geom.z_half
        st = np.where(alive[None, :], new, st)
        crossed[l] = alive
        x, y, z = st[0], st[1], st[2]
        r = np.hypot(x, y)
        nx, ny = x / r, y / r
        v = hit_covariance(x, y, sigma_r, sigma_rphi, sigma_z)
        hx, hy, hz = x.copy(), y.copy(), z.copy()
        if smear:
            hx += sigma_r * nx * g_hit[0] - sigma_rphi * ny * g_hit[1]
            hy += sigma_r * ny * g_hit[0] + sigma_rphi * nx * g_hit[1]
            hz += sigma_z * g_hit[2]
        has = alive & (u_eff < hit_eff)
        hit_pos[l] = np.where(has[None, :], np.stack([hx, hy, hz]), 0.0)
        hit_cov[l] = np.where(has[None, :], v, 0.0)
        mask |= (has.astype(np.uint32) << np.uint32(l))
        if ms and geom.x_over_x0[l] > 0.0:
            p = np.sqrt(st[3] ** 2 + st[4] ** 2 + st[5] ** 2)
            pn = (st[3] * nx + st[4] * ny) / p
            th0 = highland_theta0(p, pn, geom.x_over_x0[l])
            st = np.where(alive[None, :], _kick(st, th0, g_ms), st)
        truth[l] = np.where(alive[None, :], st, np.nan)
    return dict(hit_pos=hit_pos, hit_cov=hit_cov, hit_mask=mask, truth=truth, crossed=crossed)


def smeared_seed(rng, vertex, smear=0.1, floor_pos=1e-4, floor_mom=1e-3, diffuse=1.0,
                 mode="scaled"):
    """Seed state and packed covariance [21, n] from the vertex truth.

    mode "scaled": seed_i = truth_i (1 + smear N(0,1)), covariance
        diag((smear seed_i)^2 + floor_i^2) (the recipe of the parity workload);
    mode "prior":  covariance diag((smear truth_i)^2 + floor_i^2) and the seed
        drawn from exactly that Gaussian around the truth, so that the prior is
        consistent with the seed's error.
    The covariance is multiplied by ``diffuse`` after the draw."""
    n = vertex.shape[1]
    g = rng.standard_normal((6, n))
    floors = np.array([floor_pos] * 3 + [floor_mom] * 3)[:, None]
    if mode == "scaled":
        seed = vertex * (1.0 + smear * g)
        var = (smear * seed) ** 2 + floors ** 2
    elif mode == "prior":
        var = (smear * vertex) ** 2 + floors ** 2
        seed = vertex + np.sqrt(var) * g
    else:
        raise ValueError(mode)
    cov = np.zeros((21, n))
    for i, d in enumerate(DIAG6):
        cov[d] = var[i] * diffuse
    return seed, cov


# ----------------------------------------------------------------------------
# fit workloads


@dataclasses.dataclass
class FitBatch:
    geom: Geometry
    seed_state: np.ndarray     # [6, T] float32
    seed_cov: np.ndarray       # [21, T] float32
    charge: np.ndarray         # [T] int8
    hit_pos: np.ndarray        # [L, 3, T] float32
    hit_cov: np.ndarray        # [L, 6, T] float32
    hit_mask: np.ndarray       # [T] uint32
    event_offsets: np.ndarray  # [E + 1] int64
    truth: np.ndarray          # [L, 6, T] float64, post-kick truth (nan when not crossed)
    crossed: np.ndarray        # [L, T] bool
    vertex: np.ndarray         # [6, T] float64
    exact: dict | None = None  # float64 seed/hit arrays before rounding to float32

    @property
    def n_tracks(self) -> int:
        return int(self.charge.shape[0])


def make_fit_batch(seed: int, event_sizes, geom: Geometry | None = None, pt_lo=0.5,
                   pt_hi=10.0, pt_dist="uniform", eta_max=1.0, sigma_rphi=0.01,
                   sigma_z=0.1, sigma_r=None, hit_eff=1.0, ms=True, smear=True,
                   seed_smear=0.1, diffuse=1.0, seed_mode="scaled", seed_floors=(1e-4, 1e-3),
                   vtx_sigma_xy=0.01, vtx_sigma_z=1.0) -> FitBatch:
    """Events of the given sizes, concatenated track-major into one SoA batch."""
    geom = geom or toy_geometry()
    if not ms:  # no scattering: the detector has no material
        geom = Geometry(geom.radii.copy(), np.zeros_like(geom.x_over_x0), geom.z_half, geom.bz)
    sizes = np.asarray(list(event_sizes), dtype=np.int64)
    n = int(sizes.sum())
    r_kin, r_hit, r_ms, r_eff, r_seed = _streams(seed, 5)
    vertex, q = draw_vertex_tracks(r_kin, n, pt_lo, pt_hi, pt_dist, eta_max,
                                   vtx_sigma_xy, vtx_sigma_z)
    sim = simulate(r_hit, r_ms, r_eff, geom, vertex, q, sigma_rphi, sigma_z, sigma_r,
                   hit_eff, ms, smear)
    s_state, s_cov = smeared_seed(r_seed, vertex, seed_smear, seed_floors[0], seed_floors[1],
                                  diffuse=diffuse, mode=seed_mode)
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    exact = dict(seed_state=s_state, seed_cov=s_cov, hit_pos=sim["hit_pos"],
                 hit_cov=sim["hit_cov"])
    return FitBatch(geom, f32(s_state), f32(s_cov), q, f32(sim["hit_pos"]),
                    f32(sim["hit_cov"]), sim["hit_mask"], off, sim["truth"],
                    sim["crossed"], vertex, exact)


def lognormal_event_sizes(seed: int, n_events=256, median=5000, sigma=math.log(10.0) / 3.0,
                          lo=500, hi=50000):
    """Ragged event sizes: lognormal around ``median``, clamped to [lo, hi]."""
    rng = _streams(seed, 8)[7]
    sizes = np.exp(rng.normal(math.log(median), sigma, n_events))
    return np.clip(np.rint(sizes), lo, hi).astype(np.int64)


def workload(name: str, seed: int | None = None, scale: float = 1.0) -> FitBatch:
    """Named fit workloads; ``scale`` shrinks the event count or size for tests.

    parity  : 10 layers r = 4..40 cm, 1 event x 1,000 tracks, pT U(0.5, 10), |eta| < 1
    fit     : same detector, 100 events x 20,000 tracks
    precision: 10 layers, pT log-uniform 0.2-500, |eta| < 2.5, sigma_rphi 0.001 cm
    ragged  : 17 layers r = 4..68 cm, hit efficiency 0.95, 256 lognormal events
    """
    if name == "parity":
        return make_fit_batch(0 if seed is None else seed, [max(1, int(1000 * scale))])
    if name == "fit":
        ev = max(1, int(round(100 * scale)))
        return make_fit_batch(1 if seed is None else seed, [20000] * ev)
    if name == "precision":
        n = max(1, int(1_000_000 * scale))
        return make_fit_batch(2 if seed is None else seed, [n], pt_lo=0.2, pt_hi=500.0,
                              pt_dist="loguniform", eta_max=2.5, sigma_rphi=0.001)
    if name == "ragged":
        s = 3 if seed is None else seed
        sizes = lognormal_event_sizes(s)
        if scale != 1.0:
            sizes = np.maximum(1, (sizes * scale).astype(np.int64))
        return make_fit_batch(s, sizes, geom=toy_geometry(17), hit_eff=0.95)
    raise KeyError(name)


# ----------------------------------------------------------------------------
# build workloads (Sections 3 and 4.3)


@dataclasses.dataclass
class BuildEvents:
    """Events for combinatorial building.

    Seeds (Section 3.2: seeds derived from the first three hits of each
    simulated track): for every simulated track with hits on the first
    ``n_seed_layers`` layers, a fit of those hits from the vertex truth smeared
    10% (the fit workload's seed recipe) gives the seed at the last seed
    layer; ``seed_fit`` holds that fit's inputs.  Building runs over the
    remaining layers, whose hits (true hits of every track plus uniform noise)
    are stored per (event, layer) segment in a shuffled order.
    """
    geom: Geometry                 # all layers
    n_seed_layers: int
    seed_fit: FitBatch             # geometry = the seed layers; one entry per seed
    seed_event: np.ndarray         # [S] int32 event of each seed
    seed_track: np.ndarray         # [S] int64 global sim-track id of each seed
    hit_pos: np.ndarray            # [3, H] float32, build layers only
    hit_cov: np.ndarray            # [6, H] float32
    hit_offsets: np.ndarray        # [E, Lb + 1] int64: segment (e, l) is hit_offsets[e, l] .. [e, l+1]
    hit_track: np.ndarray          # [H] int64 global sim-track id, -1 for noise
    track_nhits: np.ndarray        # [n_sim] hits of each sim track over all layers
    n_events: int
    # every hit of the seed layers (true hits and, for seeding from hits, noise),
    # per (event, seed layer) segment; None unless requested
    seed_hit_pos: np.ndarray | None = None      # [3, Hs] float32
    seed_hit_cov: np.ndarray | None = None      # [6, Hs] float32
    seed_hit_offsets: np.ndarray | None = None  # [E, n_seed_layers + 1] int64
    seed_hit_track: np.ndarray | None = None    # [Hs] int64, -1 for noise
    track_pt: np.ndarray | None = None          # [n_sim] generated pT

    @property
    def build_geom(self) -> Geometry:
        return self.geom.sub(self.n_seed_layers, self.geom.n_layers)

    @property
    def n_seeds(self) -> int:
        return int(self.seed_event.shape[0])


def make_build_events(seed: int, n_events: int, tracks_per_event: int, geom: Geometry | None = None,
                      noise_factor: float = 10.0, n_seed_layers: int = 3, sigma_rphi=0.01,
                      sigma_z=0.1, ms=True, pt_lo=0.5, pt_hi=10.0, eta_max=1.0,
                      noise_per_layer: int | None = None, seed_layer_hits: bool = False,
                      seed_noise_per_layer: int | None = None) -> BuildEvents:
    """``n_events`` events of ``tracks_per_event`` simulated tracks each, plus
    ``noise_factor`` x tracks_per_event uniform noise hits per layer (or
    ``noise_per_layer``), on the toy barrel (17 layers by default).  With
    ``seed_layer_hits`` the seed layers' hits (every track's true hits plus the
    same density of noise, or ``seed_noise_per_layer`` noise hits, from a
    stream of their own) are stored too, for seeding from hits."""
    geom = geom or toy_geometry(17)
    L = geom.n_layers
    r_kin, r_hit, r_ms, r_eff, r_seed, r_noise, r_perm = _streams(seed, 7)
    n = n_events * tracks_per_event
    vertex, q = draw_vertex_tracks(r_kin, n, pt_lo, pt_hi, "uniform", eta_max)
    sim = simulate(r_hit, r_ms, r_eff, geom, vertex, q, sigma_rphi, sigma_z, None, 1.0, ms, True)
    track_nhits = np.zeros(n, dtype=np.int64)
    for l in range(L):
        track_nhits += (sim["hit_mask"] >> np.uint32(l)) & np.uint32(1)
    event_of = np.repeat(np.arange(n_events), tracks_per_event)
    # seeds: tracks with hits on every seed layer
    seed_bits = np.uint32((1 << n_seed_layers) - 1)
    is_seed = (sim["hit_mask"] & seed_bits) == seed_bits
    sidx = np.nonzero(is_seed)[0]
    s_state, s_cov = smeared_seed(r_seed, vertex[:, sidx], 0.1)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    seed_fit = FitBatch(geom.sub(0, n_seed_layers), f32(s_state), f32(s_cov), q[sidx],
                        f32(sim["hit_pos"][:n_seed_layers][:, :, sidx]),
                        f32(sim["hit_cov"][:n_seed_layers][:, :, sidx]),
                        np.full(len(sidx), seed_bits, dtype=np.uint32), np.array([0, len(sidx)]),
                        sim["truth"][:n_seed_layers][:, :, sidx], sim["crossed"][:n_seed_layers][:, sidx],
                        vertex[:, sidx])
    # build-layer hits per (event, layer): true hits then noise, shuffled
    Lb = L - n_seed_layers
    n_noise = int(noise_per_layer if noise_per_layer is not None else round(noise_factor * tracks_per_event))
    pos_parts, cov_parts, trk_parts = [], [], []
    offsets = np.zeros((n_events, Lb + 1), dtype=np.int64)
    cursor = 0
    for e in range(n_events):
        lo, hi = e * tracks_per_event, (e + 1) * tracks_per_event
        for lb in range(Lb):
            l = lb + n_seed_layers
            has = ((sim["hit_mask"][lo:hi] >> np.uint32(l)) & np.uint32(1)).astype(bool)
            tp = sim["hit_pos"][l][:, lo:hi][:, has]
            tc = sim["hit_cov"][l][:, lo:hi][:, has]
            tt = np.arange(lo, hi)[has]
            phi = r_noise.uniform(0.0, 2.0 * math.pi, n_noise)
            zz = r_noise.uniform(-geom.z_half, geom.z_half, n_noise)
            nxp, nyp = geom.radii[l] * np.cos(phi), geom.radii[l] * np.sin(phi)
            npos = np.stack([nxp, nyp, zz])
            ncov = hit_covariance(nxp, nyp, sigma_rphi, sigma_rphi, sigma_z)
            pos = np.concatenate([tp, npos], axis=1)
            cov = np.concatenate([tc, ncov], axis=1)
            trk = np.concatenate([tt, np.full(n_noise, -1, dtype=np.int64)])
            perm = r_perm.permutation(pos.shape[1])
            pos_parts.append(pos[:, perm])
            cov_parts.append(cov[:, perm])
            trk_parts.append(trk[perm])
            offsets[e, lb] = cursor
            cursor += pos.shape[1]
            offsets[e, lb + 1] = cursor
    hit_pos = f32(np.concatenate(pos_parts, axis=1)) if pos_parts else np.zeros((3, 0), np.float32)
    hit_cov = f32(np.concatenate(cov_parts, axis=1)) if cov_parts else np.zeros((6, 0), np.float32)
    hit_track = np.concatenate(trk_parts) if trk_parts else np.zeros(0, np.int64)
    ev = BuildEvents(geom, n_seed_layers, seed_fit, event_of[sidx].astype(np.int32), sidx.astype(np.int64),
                     hit_pos, hit_cov, offsets, hit_track, track_nhits, n_events)
    ev.track_pt = np.hypot(vertex[3], vertex[4])
    if seed_layer_hits:
        r_snoise, r_sperm = _streams(seed, 10)[8:10]
        n_snoise = n_noise if seed_noise_per_layer is None else int(seed_noise_per_layer)
        sp, sc, st = [], [], []
        soff = np.zeros((n_events, n_seed_layers + 1), dtype=np.int64)
        cur = 0
        for e in range(n_events):
            lo, hi = e * tracks_per_event, (e + 1) * tracks_per_event
            for l in range(n_seed_layers):
                has = ((sim["hit_mask"][lo:hi] >> np.uint32(l)) & np.uint32(1)).astype(bool)
                phi = r_snoise.uniform(0.0, 2.0 * math.pi, n_snoise)
                zz = r_snoise.uniform(-geom.z_half, geom.z_half, n_snoise)
                nxp, nyp = geom.radii[l] * np.cos(phi), geom.radii[l] * np.sin(phi)
                pos = np.concatenate([sim["hit_pos"][l][:, lo:hi][:, has], np.stack([nxp, nyp, zz])], axis=1)
                cov = np.concatenate([sim["hit_cov"][l][:, lo:hi][:, has],
                                      hit_covariance(nxp, nyp, sigma_rphi, sigma_rphi, sigma_z)], axis=1)
                trk = np.concatenate([np.arange(lo, hi)[has], np.full(n_snoise, -1, dtype=np.int64)])
                perm = r_sperm.permutation(pos.shape[1])
                sp.append(pos[:, perm])
                sc.append(cov[:, perm])
                st.append(trk[perm])
                soff[e, l] = cur
                cur += pos.shape[1]
                soff[e, l + 1] = cur
        ev.seed_hit_pos = f32(np.concatenate(sp, axis=1))
        ev.seed_hit_cov = f32(np.concatenate(sc, axis=1))
        ev.seed_hit_offsets = soff
        ev.seed_hit_track = np.concatenate(st)
    return ev


def build_workload(scale_events: int | None = None, seed: int = 4, tracks_per_event: int = 5000):
    """The build workload: 17 layers, 5,000 tracks per event, 10x uniform noise
    per layer, seeds from the first three layers, 64 events per launch."""
    return make_build_events(seed, 64 if scale_events is None else scale_events, tracks_per_event)


def proposal_init(rng) -> np.ndarray:
    """Initial weights of the proposal network (12 -> 64 -> 64 -> 1) in its
    flat float32 layout W1 [12][64], b1, W2 [64][64], b2, W3 [64], b3:
    He-normal draws for W1 and W2, N(0, 1/64) for W3, zero biases."""
    parts = [rng.normal(0.0, np.sqrt(2.0 / 12), 12 * 64), np.zeros(64),
             rng.normal(0.0, np.sqrt(2.0 / 64), 64 * 64), np.zeros(64),
             rng.normal(0.0, np.sqrt(1.0 / 64), 64), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)
