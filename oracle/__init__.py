"""FP64 CPU oracle for the spatiotemporal Hawkes log-likelihood, gradient and
Hessian diagonal (arXiv 2103.03348, Section 2.1 Eq. 1, Eqs. 4-5, Appendix A).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The product path (the
CUDA library and its Python binding) never touches it.

The arithmetic lives in ``hawkes_oracle.c`` (plain double loops, libm exp, log
and erfc); this module compiles it with gcc (``-O2``, no fast-math, OpenMP over
independent rows only) and calls it through ctypes.  ``hmc_oracle.py`` and
``mlp_oracle.py`` hold the NumPy FP64 oracles of the sampler step and the
surrogate network.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hawkes_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

NPAR = 6


def build_all(force: bool = False):
    """Compile every C part of the oracle (the likelihood and the tree prior)."""
    from . import tree_oracle
    build(force)
    tree_oracle.build(force)


def build(force: bool = False, src: str = _SRC, so: str = _SO) -> str:
    """Compile the C oracle (default: oracle/_build/liboracle.so; idempotent)."""
    os.makedirs(os.path.dirname(so), exist_ok=True)
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        tmp = so + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               "-std=c99", "-Wall", "-o", tmp, src, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, so)
    return so


def _typed(lib):
    d = ctypes.POINTER(ctypes.c_double)
    i64 = ctypes.c_int64
    l64 = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_eval.argtypes = [i64, d, d, d, d, d, ctypes.c_int, d, d, d, d, d, ctypes.c_int]
    lib.oracle_eval.restype = ctypes.c_int
    lib.oracle_intensity.argtypes = [i64, d, d, d, d, d, i64, d, d, d, d, ctypes.c_int]
    lib.oracle_intensity.restype = ctypes.c_int
    lib.oracle_integral.argtypes = [i64, d, d, d]
    lib.oracle_integral.restype = ctypes.c_double
    lib.oracle_rows.argtypes = [i64, d, d, d, d, d, i64, l64, d, d, d, ctypes.c_int]
    lib.oracle_rows.restype = ctypes.c_int
    lib.oracle_rate_terms.argtypes = [i64, d, d, d, d, d, d, i64, l64, d, d, ctypes.c_int]
    lib.oracle_rate_terms.restype = ctypes.c_int
    lib.oracle_max_threads.argtypes = []
    lib.oracle_max_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _typed(ctypes.CDLL(build()))
    return _lib


def load_variant(src_text: str, workdir: str):
    """Compile a modified copy of the oracle's C source (for tests that plant a
    mistake in the oracle) and return its library handle, to pass as lib=."""
    src = os.path.join(workdir, "variant.c")
    with open(src, "w") as f:
        f.write(src_text)
    return _typed(ctypes.CDLL(build(force=True, src=src, so=os.path.join(workdir, "libvariant.so"))))


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _arr(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def evaluate(x, y, t, r, params, want: int = 2, threads: int = 0, lib=None):
    """Log-likelihood (want=0), + gradient (1), + Hessian diagonal (2).

    Returns a dict with ``loglik`` (float), ``grad`` and ``hdiag`` ([6+N] or
    None), ``lam`` ([N], lambda_n) and ``Lambda`` (the integral term), and
    ``status`` (0 ok, 1 when some lambda_n == 0).  ``threads=0`` uses OpenMP's
    default.  The result does not depend on the thread count.
    """
    lib = lib or _load()
    x, y, t, r, p = _arr(x), _arr(y), _arr(t), _arr(r), _arr(params)
    n = t.shape[0]
    ll = np.zeros(1)
    lam = np.zeros(n)
    Lam = np.zeros(1)
    grad = np.zeros(NPAR + n) if want >= 1 else None
    hd = np.zeros(NPAR + n) if want >= 2 else None
    null = ctypes.POINTER(ctypes.c_double)()
    st = lib.oracle_eval(n, _p(x), _p(y), _p(t), _p(r), _p(p), int(want), _p(ll),
                         _p(grad) if grad is not None else null, _p(hd) if hd is not None else null,
                         _p(lam), _p(Lam), int(threads))
    if st < 0:
        raise ValueError("oracle_eval: invalid arguments")
    return {"loglik": float(ll[0]), "grad": grad, "hdiag": hd, "lam": lam, "Lambda": float(Lam[0]),
            "status": int(st)}


def intensity(x, y, t, r, params, xq, yq, tq, threads: int = 0):
    """lambda(x_q, t_q) at arbitrary query points given the events."""
    lib = _load()
    x, y, t, r, p = _arr(x), _arr(y), _arr(t), _arr(r), _arr(params)
    xq, yq, tq = _arr(xq), _arr(yq), _arr(tq)
    out = np.zeros(tq.shape[0])
    st = lib.oracle_intensity(t.shape[0], _p(x), _p(y), _p(t), _p(r), _p(p), tq.shape[0], _p(xq), _p(yq),
                              _p(tq), _p(out), int(threads))
    if st < 0:
        raise ValueError("oracle_intensity: invalid arguments")
    return out


def integral(t, r, params, lib=None) -> float:
    """The integral term Lambda alone (Appendix A Claim, background integrated exactly)."""
    lib = lib or _load()
    t, r, p = _arr(t), _arr(r), _arr(params)
    return float(lib.oracle_integral(t.shape[0], _p(t), _p(r), _p(p)))


def _pi(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def rows(x, y, t, r, params, idx, threads: int = 0, lib=None):
    """lambda_n and per-row derivative sums (d lambda_n/dp, d2 lambda_n/dp2) for the rows in idx."""
    lib = lib or _load()
    x, y, t, r, p = _arr(x), _arr(y), _arr(t), _arr(r), _arr(params)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    k = idx.shape[0]
    lam, d1, d2 = np.zeros(k), np.zeros(k * NPAR), np.zeros(k * NPAR)
    st = lib.oracle_rows(t.shape[0], _p(x), _p(y), _p(t), _p(r), _p(p), k, _pi(idx), _p(lam), _p(d1), _p(d2),
                         int(threads))
    if st < 0:
        raise ValueError("oracle_rows: invalid arguments")
    return lam, d1.reshape(k, NPAR), d2.reshape(k, NPAR)


def rate_terms(x, y, t, r, params, lam, idx, threads: int = 0, lib=None):
    """Gradient and Hessian diagonal w.r.t. r_m for the sources in idx, given lambda for later targets."""
    lib = lib or _load()
    x, y, t, r, p, lam = _arr(x), _arr(y), _arr(t), _arr(r), _arr(params), _arr(lam)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    k = idx.shape[0]
    g, h = np.zeros(k), np.zeros(k)
    st = lib.oracle_rate_terms(t.shape[0], _p(x), _p(y), _p(t), _p(r), _p(p), _p(lam), k, _pi(idx), _p(g), _p(h),
                                int(threads))
    if st < 0:
        raise ValueError("oracle_rate_terms: invalid arguments")
    return g, h
