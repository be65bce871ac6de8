"""Precision of the FP32 fit against the FP64 oracle on the precision workload
(pT log-uniform 0.2..500 GeV, |eta| < 2.5, hit resolution 0.01, 0.003 and
0.001 cm): per-parameter error of the GPU result in units of the oracle's
fitted sigma (median, 99th percentile, maximum; the position taken along
the layer's tangent, since the radial one is fixed by the cylinder and has
no sigma) for the FP32-only form and
the routed form (ill-conditioned updates redone in FP64), the share of
tracks routed, and the pull widths against the simulated truth for the
oracle and both forms.  With KF_REPORT_DIR set the numbers are written there
as precision_study.json.

Bars: the routed form's median error stays below 1e-3 sigma and its 99th
percentile below 0.05 sigma on every parameter; the routed form is never
worse than the FP32-only one at the 99th percentile beyond rounding; the
pull widths of both forms are within 5% of the oracle's.
"""
import json
import os

import numpy as np
import pytest

from paper_1705_02876_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

PARAMS = ("t", "z", "px", "py", "pz")  # t: tangential position at the last crossing
N_TRACKS = 1_000_000  # per resolution, the precision workload's size


@pytest.fixture(scope="module")
def kf():
    from paper_1705_02876_gb300 import build, kf as kf_
    build.build()
    return kf_


def _width(v):
    p16, p84 = np.percentile(v, [16, 84])
    return float((p84 - p16) / 2)


def test_precision_study(kf, oracle):
    ctx = kf.Context(0)
    report = {}
    for sig in (0.01, 0.003, 0.001):
        b = synth.make_fit_batch(2, [N_TRACKS], pt_lo=0.2, pt_hi=500.0, pt_dist="loguniform", eta_max=2.5,
                                 sigma_rphi=sig)
        ref = oracle.fit_batch(b)
        dev = kf.to_device(b)
        outs = {}
        for name, mode in (("fp32", kf.PRECISION_FP32), ("routed", kf.PRECISION_ROUTED)):
            r = kf.fit_tracks(ctx, kf.GeometryArgs.of(b.geom), **dev, opt=kf.options(precision_mode=mode))
            torch.cuda.synchronize()
            outs[name] = {k: v.cpu().numpy() for k, v in r.items()}
        bad = 4 | 8  # inversion failed, NaN input (tracks that stopped early keep their fit)
        ok = ((ref["flags"] & bad) == 0) & (ref["ndof"] > 0)
        for o in outs.values():
            ok &= ((o["flags"].astype(np.int64) & bad) == 0) & (o["ndof"] == ref["ndof"])
        # positions in the local frame of the last crossing: the tangential
        # component over its sigma (the radial one is fixed by the cylinder and
        # its sigma is zero), the rest as is
        st, cv = ref["state"][:, ok], ref["cov"][:, ok]
        r = np.hypot(st[0], st[1])
        nx, ny = st[0] / r, st[1] / r
        var_t = ny * ny * cv[0] - 2 * nx * ny * cv[1] + nx * nx * cv[2]
        var = np.stack([var_t] + [cv[i * (i + 1) // 2 + i] for i in range(2, 6)])
        # a track crossing its last layer almost tangentially (a looper at
        # 2R ~ r) can leave even the FP64 oracle, which has no PSD repair, with a
        # negative variance: such tracks have no sigma to measure errors in
        psd = (var > 0).all(0)
        keep = np.nonzero(ok)[0][psd]
        ok = np.zeros_like(ok)
        ok[keep] = True
        st, cv, var, nx, ny, r = st[:, psd], cv[:, psd], var[:, psd], nx[psd], ny[psd], r[psd]
        sig_ref = np.sqrt(var)

        def local(state):
            return np.stack([-ny * state[0] + nx * state[1], state[2], state[3], state[4], state[5]])

        # the layer after which the fit ended: every layer reached has a hit
        # (efficiency 1), so hits = ndof / 3 + 2 = layers reached
        reached = (ref["ndof"][ok] + 6) // 3
        truth = np.stack([b.truth[reached - 1, i, np.nonzero(ok)[0]] for i in range(6)])
        pt = np.hypot(truth[3], truth[4])
        bins = {"pt<0.5": pt < 0.5, "0.5<=pt<100": (pt >= 0.5) & (pt < 100), "pt>=100": pt >= 100}
        entry = {"tracks": int(ok.sum()), "oracle_not_psd": int((~psd).sum()), "oracle_pull_width": {}}
        lt, lr = local(truth), local(st)
        for i, p in enumerate(PARAMS):
            entry["oracle_pull_width"][p] = _width((lr[i] - lt[i]) / sig_ref[i])
        for name, o in outs.items():
            lo = local(o["state"][:, ok])
            err = np.abs(lo - lr) / sig_ref
            e = {p: {"median": float(np.median(err[i])), "p99": float(np.percentile(err[i], 99)),
                     "max": float(err[i].max())} for i, p in enumerate(PARAMS)}
            worst = err.max(0)
            by_pt = {k: {"tracks": int(m.sum()), "p99_worst_param": float(np.percentile(worst[m], 99)) if m.any() else None,
                         "max_worst_param": float(worst[m].max()) if m.any() else None} for k, m in bins.items()}
            # fits the oracle itself finds consistent with the hits (the worst
            # tracks overall have chi2/ndof of 100 and more: a seed far outside
            # what the hits allow, where the extended filter is nonlinear)
            sane = ref["chi2"][ok] <= 10.0 * ref["ndof"][ok]
            sane_worst = {"tracks": int(sane.sum()), "max_worst_param": float(worst[sane].max()) if sane.any() else None,
                          "p99_worst_param": float(np.percentile(worst[sane], 99)) if sane.any() else None}
            radial = np.abs(np.hypot(o["state"][0, ok], o["state"][1, ok]) - r) * 1e4
            pulls = {p: _width((lo[i] - lt[i]) / sig_ref[i]) for i, p in enumerate(PARAMS)}
            chi = np.abs(o["chi2"][ok] - ref["chi2"][ok]) / np.maximum(ref["chi2"][ok], 1.0)
            entry[name] = {"error_in_sigma": e, "by_pt": by_pt, "chi2_ndof_le_10": sane_worst, "pull_width": pulls,
                           "radial_position_error_um": {"median": float(np.median(radial)), "max": float(radial.max())},
                           "chi2_rel_error": {"median": float(np.median(chi)), "p99": float(np.percentile(chi, 99)),
                                              "max": float(chi.max())},
                           "fp64_routed_share": float(((o["flags"][ok].astype(np.int64) & 16) != 0).mean())}
        report[f"sigma_rphi={sig}"] = entry
    out_dir = os.environ.get("KF_REPORT_DIR")
    if out_dir:
        os.makedirs(out_dir, exist_ok=True)
        with open(os.path.join(out_dir, "precision_study.json"), "w") as f:
            json.dump(report, f, indent=1)
    for sig, entry in report.items():
        for p in PARAMS:
            r, f = entry["routed"]["error_in_sigma"][p], entry["fp32"]["error_in_sigma"][p]
            assert r["median"] < 1e-3, (sig, p, r)
            assert r["p99"] < 0.05, (sig, p, r)
            assert r["p99"] <= 1.1 * f["p99"] + 1e-4, (sig, p, r, f)
            w0 = entry["oracle_pull_width"][p]
            for name in ("fp32", "routed"):
                assert abs(entry[name]["pull_width"][p] / w0 - 1) < 0.05, (sig, p, name, entry[name]["pull_width"][p], w0)
    ctx.close()
