"""Shared tolerance checks for GPU-vs-oracle parity (test-only).

APPs: FP32 path vs FP64 oracle.  The maximum relative error is taken over
entries whose reference is at least 1e-6 (FP32 underflows far below that, so a
relative error over every entry is ill-posed), together with the maximum
absolute error over all entries; both must be <= 1e-4.  log P: relative error
<= 1e-6.  Gradients: relative error <= 1e-4 against the reference, measured
against the reference's magnitude.
"""
import numpy as np

APP_TOL = 1e-4
LL_TOL = 1e-6
GRAD_TOL = 1e-4


def app_errors(app, ref):
    app = np.asarray(app, np.float64)
    ref = np.asarray(ref, np.float64)
    mask = ref >= 1e-6
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


def check_grad(g, ref, tol=GRAD_TOL, what=""):
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = max(float(np.max(np.abs(ref))), 1e-30)
    err = float(np.max(np.abs(g - ref))) / scale
    assert err <= tol, f"{what} grad rel-to-max {err:.3e}\n{g}\n{ref}"
    return err
