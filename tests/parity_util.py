"""Comparison helpers and tolerances for CUDA-vs-oracle parity.

Tolerances (floating point; the stated bar for each precision):
  * FP64 path: every output within 1e-10 relative, with the denominator
    max(|ref_i|, 1e-3 * max_j |ref_j|) for vector outputs (so entries near zero
    are compared on the scale of the vector).
  * FP32C path: log-likelihood within 1e-5 relative and the gradient within
    ||g - g_ref||_2 <= 1e-5 ||g_ref||_2.  Per-entry errors are reported and held
    to a looser guard that still catches a wrong formula: global gradient and
    Hessian entries within 1e-4 (scaled as above), log-rate entries within 2e-3,
    ||H - H_ref||_2 <= 1e-4 ||H_ref||_2.  The per-entry log-rate error is larger
    because each log-rate gradient is a short sum minus a subtraction of similar
    size, and FP32 event coordinates carry a relative error of ~6e-8 of the
    coordinate range (about 1e-5 of the excitation bandwidth at 2000 km / 5 km).
"""
import numpy as np

FP64_TOL = 1e-10
FP32C_LL_TOL = 1e-5
FP32C_GNORM_TOL = 1e-5
FP32C_GLOBAL_TOL = 1e-4
FP32C_RATE_TOL = 2e-3
FP32C_HNORM_TOL = 1e-4


def scaled_err(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    if b.size == 0:
        return 0.0
    den = np.maximum(np.abs(b), 1e-3 * np.abs(b).max())
    den = np.where(den > 0, den, 1.0)
    return float(np.max(np.abs(a - b) / den))


def rel(a, b):
    return abs(float(a) - float(b)) / max(abs(float(b)), 1e-300)


def norm_rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def check(prec, ll, g, h, ref, label=""):
    """Assert parity of (ll, g, h) against an oracle dict; returns the error report."""
    rep = {"ll": rel(ll, ref["loglik"])}
    if g is not None:
        rep.update(g_p=scaled_err(g[:6], ref["grad"][:6]), g_r=scaled_err(g[6:], ref["grad"][6:]),
                   g_norm=norm_rel(g, ref["grad"]))
    if h is not None:
        rep.update(h_p=scaled_err(h[:6], ref["hdiag"][:6]), h_r=scaled_err(h[6:], ref["hdiag"][6:]),
                   h_norm=norm_rel(h, ref["hdiag"]))
    msg = f"{label} {prec}: {rep}"
    if prec == "fp64":
        for k, v in rep.items():
            assert v <= FP64_TOL, msg
    else:
        assert rep["ll"] <= FP32C_LL_TOL, msg
        if g is not None:
            assert rep["g_norm"] <= FP32C_GNORM_TOL, msg
            assert rep["g_p"] <= FP32C_GLOBAL_TOL, msg
            assert rep["g_r"] <= FP32C_RATE_TOL, msg
        if h is not None:
            assert rep["h_norm"] <= FP32C_HNORM_TOL, msg
            assert rep["h_p"] <= FP32C_GLOBAL_TOL, msg
            assert rep["h_r"] <= FP32C_RATE_TOL, msg
    return rep
