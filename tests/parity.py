"""Shared tolerance checks for GPU-vs-oracle parity (test-only).

APPs: FP32 path vs FP64 oracle.  The maximum relative error is taken over
entries whose reference is at least 1e-6 (FP32 underflows far below that, so a
relative error over every entry is ill-posed), together with the maximum
absolute error over all entries; both must be <= 1e-4.  log P: relative error
<= 1e-6.

Gradients are checked entry by entry:
  - channel gradients d logP / d(Pi, Pd, Ps): relative error <= 1e-4 for every
    entry with |ref| >= GRAD_FLOOR, absolute error <= 1e-4 * GRAD_FLOOR below
    it (every case in the suite has |ref| > 1);
  - prior gradients d logP / d Pr{D_i = D} = APP_i(D) / Pr{D_i = D}: weighted by
    the prior, each entry is the APP, so the APP criterion applies entry by
    entry -- relative error <= 1e-4 wherever prior * |ref| >= 1e-6, and
    prior * |g - ref| <= 1e-4 everywhere.
"""
import numpy as np

APP_TOL = 1e-4
LL_TOL = 1e-6
GRAD_TOL = 1e-4
GRAD_FLOOR = 1e-3
APP_FLOOR = 1e-6


def app_errors(app, ref):
    app = np.asarray(app, np.float64)
    ref = np.asarray(ref, np.float64)
    mask = ref >= APP_FLOOR
    rel = float(np.max(np.abs(app[mask] - ref[mask]) / ref[mask])) if mask.any() else 0.0
    ab = float(np.max(np.abs(app - ref))) if ref.size else 0.0
    return rel, ab


def check_app(app, ref, tol=APP_TOL, what=""):
    rel, ab = app_errors(app, ref)
    assert rel <= tol and ab <= tol, f"{what} APP rel {rel:.3e} abs {ab:.3e}"
    return rel, ab


def check_ll(ll, ref, tol=LL_TOL, what=""):
    r = abs(ll - ref) / max(abs(ref), 1e-300)
    assert r <= tol, f"{what} logP {ll!r} vs {ref!r} rel {r:.3e}"
    return r


def grad_errors(g, ref, floor=GRAD_FLOOR):
    """(max relative error over |ref| >= floor, max absolute error over the rest)."""
    g = np.asarray(g, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    big = np.abs(ref) >= floor
    rel = float(np.max(np.abs(g[big] - ref[big]) / np.abs(ref[big]))) if big.any() else 0.0
    ab = float(np.max(np.abs(g[~big] - ref[~big]))) if (~big).any() else 0.0
    return rel, ab


def check_grad(g, ref, tol=GRAD_TOL, floor=GRAD_FLOOR, what=""):
    """Channel-parameter (or any dense) gradient, entry by entry."""
    rel, ab = grad_errors(g, ref, floor)
    assert rel <= tol and ab <= tol * floor, (
        f"{what} grad rel {rel:.3e} (|ref| >= {floor:g}), abs {ab:.3e} below\n"
        f"{np.asarray(g)}\n{np.asarray(ref)}")
    return rel


def check_grad_priors(g, ref, priors, tol=GRAD_TOL, what=""):
    """d logP / d prior, entry by entry on the APP scale (prior * gradient)."""
    pri = np.asarray(priors, np.float64)
    rel, ab = app_errors(pri * np.asarray(g, np.float64), pri * np.asarray(ref, np.float64))
    assert rel <= tol and ab <= tol, f"{what} d/dprior rel {rel:.3e} abs {ab:.3e}"
    return rel
