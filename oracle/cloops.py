"""ctypes binding of oracle/loops.c (TEST INFRASTRUCTURE ONLY; see oracle/nlpr.py).

build() compiles loops.c with gcc into oracle/_build/liboracle_loops.so; the library
is plain C with OpenMP, no CUDA, and shares nothing with the CUDA path."""
from __future__ import annotations

import ctypes
import os
import pathlib
import subprocess

import numpy as np

_HERE = pathlib.Path(__file__).resolve().parent
_SRC = _HERE / "loops.c"
_OUT = _HERE / "_build" / "liboracle_loops.so"
_lib = None


def build(force: bool = False) -> pathlib.Path:
    if _OUT.exists() and not force and _OUT.stat().st_mtime >= _SRC.stat().st_mtime:
        return _OUT
    _OUT.parent.mkdir(exist_ok=True)
    tmp = _OUT.with_suffix(f".{os.getpid()}.tmp")
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
                    str(_SRC), "-o", str(tmp), "-lm"], check=True)
    os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(str(build()))
        D = ctypes.POINTER(ctypes.c_double)
        i, d = ctypes.c_int, ctypes.c_double
        _lib.oracle_weights.argtypes = [D, i, i, i, i, i, d, D]
        _lib.oracle_latent.argtypes = [D, D, D, D, i, i, i, i, i, d, d]
        _lib.oracle_dt_sum.argtypes = [D, D, i, i, i, i, i, D]
        for f in (_lib.oracle_weights, _lib.oracle_latent, _lib.oracle_dt_sum):
            f.restype = None
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def weights(G: np.ndarray, K: int, S: int, h: float) -> np.ndarray:
    G = np.ascontiguousarray(G, dtype=np.float64)
    H, W, L = G.shape
    nW = (2 * S + 1) ** 2 - 1
    out = np.empty((nW, H, W))
    lib().oracle_weights(_p(G), H, W, L, K, S, float(h), _p(out))
    return out


def latent_update(X, st, su):
    """(Q, Sigma) of eqs. Qj_main and dualvar3_main with explicit loops."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    H, W, L = X.shape
    Q = np.empty_like(st.Sig)
    Sig = st.Sig.copy()
    om = np.ascontiguousarray(su.omega, dtype=np.float64)
    lib().oracle_latent(_p(X), _p(om), _p(Q), _p(Sig), H, W, L, su.K, su.S,
                        float(su.lam2), float(su.rho))
    return Q, Sig


def latent_update_inplace(X, st, su):
    """As latent_update, overwriting st.Q and st.Sig (eqs. Qj_main, dualvar3_main)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    H, W, L = X.shape
    om = np.ascontiguousarray(su.omega, dtype=np.float64)
    lib().oracle_latent(_p(X), _p(om), _p(st.Q), _p(st.Sig), H, W, L, su.K, su.S,
                        float(su.lam2), float(su.rho))
    return st.Q, st.Sig


def dt_sum(Q: np.ndarray, Sig: np.ndarray, K: int, S: int) -> np.ndarray:
    H, W, L = Q.shape[2:]
    out = np.empty((H, W, L))
    lib().oracle_dt_sum(_p(np.ascontiguousarray(Q)), _p(np.ascontiguousarray(Sig)),
                        H, W, L, K, S, _p(out))
    return out
