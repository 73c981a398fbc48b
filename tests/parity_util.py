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
    Where that subtraction cancels by more than the guard allows (an entry
    dl/dr_m = C1_m - dLambda/dr_m of Eq. 4 that is 1/200 of its parts, seen at
    100,000 events), the entry is held instead to its condition scale: the
    error of a difference of two positive sums whose FP32 terms each carry a
    relative error of order 1e-5 is bounded by that error times the sum of the
    parts, so |dg_m| <= 1e-4 (C1_m + dLambda/dr_m) and |dh_m| <= 1e-4 (C1_m +
    C2_m + dLambda/dr_m), with C1_m = sum_n w_nm and C2_m = sum_n w_nm^2 from
    the oracle's own outputs (Eqs. 4-5).
"""
import hashlib
import os

import numpy as np

FP64_TOL = 1e-10
FP32C_LL_TOL = 1e-5
FP32C_GNORM_TOL = 1e-5
FP32C_GLOBAL_TOL = 1e-4
FP32C_RATE_TOL = 2e-3
FP32C_HNORM_TOL = 1e-4
FP32C_RATE_COND_TOL = 1e-4


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


def rate_condition_scales(t, r, params, ref):
    """The parts of each log-rate entry (Eqs. 4-5 times theta_m): with
    dLambda/dr_m = theta0 e^{r_m} (1 - e^{-omega (t_N - t_m)}) (Appendix A),
    C1_m = g_m + dLambda/dr_m and C2_m = g_m - h_m; returns the scales
    C1 + dLambda/dr (gradient) and C1 + C2 + dLambda/dr (Hessian)."""
    t, r, p = np.asarray(t, float), np.asarray(r, float), np.asarray(params, float)
    dlam = p[3] * np.exp(r) * (1.0 - np.exp(-p[4] * (t.max() - t)))
    c1 = ref["grad"][6:] + dlam
    c2 = ref["grad"][6:] - ref["hdiag"][6:]
    return {"g": np.abs(c1) + dlam, "h": np.abs(c1) + np.abs(c2) + dlam}


def rate_entry_err(a, b, cond):
    """max over m of |a_m - b_m| / max(2e-3-guard denominator scaled to the
    rate guard, condition scale scaled to its bar): <= 1 passes."""
    a, b = np.asarray(a, float), np.asarray(b, float)
    den = np.maximum(np.abs(b), 1e-3 * np.abs(b).max())
    allowed = np.maximum(FP32C_RATE_TOL * den, FP32C_RATE_COND_TOL * cond)
    allowed = np.where(allowed > 0, allowed, 1e-300)
    return float(np.max(np.abs(a - b) / allowed))


def check(prec, ll, g, h, ref, label="", cond=None):
    """Assert parity of (ll, g, h) against an oracle dict; returns the error report.
    cond: optional rate_condition_scales(...) for the FP32C per-entry log-rate guard."""
    rep = {"ll": rel(ll, ref["loglik"])}
    if g is not None:
        rep.update(g_p=scaled_err(g[:6], ref["grad"][:6]), g_r=scaled_err(g[6:], ref["grad"][6:]),
                   g_norm=norm_rel(g, ref["grad"]))
        if cond is not None:
            rep["g_r_guard"] = rate_entry_err(g[6:], ref["grad"][6:], cond["g"])
    if h is not None:
        rep.update(h_p=scaled_err(h[:6], ref["hdiag"][:6]), h_r=scaled_err(h[6:], ref["hdiag"][6:]),
                   h_norm=norm_rel(h, ref["hdiag"]))
        if cond is not None:
            rep["h_r_guard"] = rate_entry_err(h[6:], ref["hdiag"][6:], cond["h"])
    msg = f"{label} {prec}: {rep}"
    if prec == "fp64":
        for k, v in rep.items():
            if not k.endswith("_guard"):
                assert v <= FP64_TOL, msg
    else:
        assert rep["ll"] <= FP32C_LL_TOL, msg
        if g is not None:
            assert rep["g_norm"] <= FP32C_GNORM_TOL, msg
            assert rep["g_p"] <= FP32C_GLOBAL_TOL, msg
            assert (rep["g_r_guard"] <= 1.0) if cond is not None else (rep["g_r"] <= FP32C_RATE_TOL), msg
        if h is not None:
            assert rep["h_norm"] <= FP32C_HNORM_TOL, msg
            assert rep["h_p"] <= FP32C_GLOBAL_TOL, msg
            assert (rep["h_r_guard"] <= 1.0) if cond is not None else (rep["h_r"] <= FP32C_RATE_TOL), msg
    return rep


def error_report(ll, g, h, ref):
    """Per-output relative errors against an oracle dict: max and median of the
    scaled entry errors (denominator max(|ref_i|, 1e-3 max|ref|)) for the six
    global and the N log-rate entries of the gradient and Hessian diagonal."""
    def vec(a, b):
        a, b = np.asarray(a, float), np.asarray(b, float)
        den = np.maximum(np.abs(b), 1e-3 * np.abs(b).max())
        e = np.abs(a - b) / np.where(den > 0, den, 1.0)
        return {"max": float(e.max()), "median": float(np.median(e))}
    return {"loglik": rel(ll, ref["loglik"]),
            "grad_globals": vec(g[:6], ref["grad"][:6]), "grad_rates": vec(g[6:], ref["grad"][6:]),
            "grad_norm": norm_rel(g, ref["grad"]),
            "hdiag_globals": vec(h[:6], ref["hdiag"][:6]), "hdiag_rates": vec(h[6:], ref["hdiag"][6:]),
            "hdiag_norm": norm_rel(h, ref["hdiag"])}


LARGE_FIXTURE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "large_N100000.npz")


def input_digest(w) -> str:
    """SHA-256 of a workload's inputs (x, y, t, r, params as FP64 bytes)."""
    d = hashlib.sha256()
    for a in (w.x, w.y, w.t, w.r, np.asarray(w.params, float)):
        d.update(np.ascontiguousarray(a, dtype=np.float64).tobytes())
    return d.hexdigest()


def large_reference(w):
    """The stored full FP64 oracle evaluation of the 100,000-event workload,
    after checking that the seeded generator reproduced its inputs."""
    z = np.load(LARGE_FIXTURE)
    assert str(z["input_sha256"]) == input_digest(w), "the generator no longer reproduces the fixture's inputs"
    return {"loglik": float(z["loglik"]), "grad": z["grad"], "hdiag": z["hdiag"], "lam": z["lam"],
            "Lambda": float(z["Lambda"])}
