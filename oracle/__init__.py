"""FP64 CPU oracle for the BSID MAP decoder -- test infrastructure only.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The decoder library never loads it, and
it shares no code with the CUDA path.  The arithmetic lives in
``mapdec_oracle.c`` (plain C, double precision, following the paper's Sec. II
step by step); this module compiles it with gcc and marshals numpy arrays.

Every function here is pinned by the ``-m "not gpu"`` tests against brute-force
enumeration of channel events, closed forms and invariants (see
``tests/test_oracle_*.py``).  No function is left "parity unpinned".

``decode_ext`` and ``loglik_grad`` also take per-symbol codebooks (the
constituent encodings C_i of Sec. II-A) and ``decode_ext`` returns the
extrinsic outputs used in iterative decoding.  The CUDA decoder produces the
extrinsic outputs too (checked against ``decode_ext``); per-symbol codebooks
exist only here so far, as the reference for that next step.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mapdec_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

ORC_OK = 0
ORC_ERR_ARG = 1
ORC_ERR_DRIFT_RANGE = 2
ORC_ERR_ZERO_PROB = 3
ORC_ERR_NOMEM = 4

_lib = None
_lock = threading.Lock()


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_receiver_metric.argtypes = [ctypes.c_int, ctypes.c_int, u8p, u8p, ctypes.c_int,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                            dp]
        lib.orc_receiver_metric.restype = ctypes.c_int
        common = [ctypes.c_int, ctypes.c_int, u8p, ctypes.c_int, ctypes.c_double,
                  ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int, u8p,
                  ctypes.c_int64, dp]
        lib.orc_decode.argtypes = common + [ctypes.c_int, dp, dp]
        lib.orc_decode.restype = ctypes.c_int
        lib.orc_forward_backward.argtypes = common + [dp, dp, dp]
        lib.orc_forward_backward.restype = ctypes.c_int
        lib.orc_loglik_grad.argtypes = common + [ctypes.c_int, dp, dp, dp]
        lib.orc_loglik_grad.restype = ctypes.c_int
        general = common[:3] + [ctypes.c_int] + common[3:]
        lib.orc_decode_general.argtypes = general + [ctypes.c_int, dp, dp, dp, dp, dp]
        lib.orc_decode_general.restype = ctypes.c_int
        lib.orc_loglik_grad_general.argtypes = general + [ctypes.c_int, dp, dp, dp, dp, dp]
        lib.orc_loglik_grad_general.restype = ctypes.c_int
        lib.orc_set_received_bit_weight.argtypes = [ctypes.c_double]
        lib.orc_set_received_bit_weight.restype = None
        _lib = lib
        return lib


def _u8(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


_NULL_D = ctypes.POINTER(ctypes.c_double)()


def receiver_metric(x, y, I: int, Pi: float, Pd: float, Ps: float) -> np.ndarray:
    """R(y[0:j] | x) for j = 0..len(y): last lattice row, eqs. (F), (F_lastrow)."""
    lib = _load()
    x, xp = _u8(x)
    y = np.ascontiguousarray(y, dtype=np.uint8)
    ybuf = y if y.size else np.zeros(1, np.uint8)
    yp = ybuf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    out = np.zeros(y.size + 1, np.float64)
    st = lib.orc_receiver_metric(int(x.size), int(I), xp, yp, int(y.size), float(Pi), float(Pd),
                                 float(Ps), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if st:
        raise OracleError(st, "receiver_metric")
    return out


def _frame_args(codebook, N, Pi, Pd, Ps, I, xmax, rx, priors):
    cb, cbp = _u8(codebook)
    if cb.ndim == 3:
        raise ValueError("per-symbol codebooks go through decode_ext / loglik_grad")
    q, n = cb.shape
    rxa = np.ascontiguousarray(rx, dtype=np.uint8)
    rbuf = rxa if rxa.size else np.zeros(1, np.uint8)
    rxp = rbuf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    keep = [cb, rbuf]
    if priors is None:
        prp = _NULL_D
    else:
        pr, prp = _f64(np.asarray(priors, dtype=np.float64).reshape(N, q))
        keep.append(pr)
    args = [int(q), int(n), cbp, int(N), float(Pi), float(Pd), float(Ps), int(I), int(xmax),
            rxp, int(rxa.size), prp]
    return q, n, args, keep


def decode(codebook, N, Pi, Pd, Ps, I, xmax, rx, priors=None, memo=True, kappa=1.0):
    """APPs (N, q) and log P(Y) of one frame (FP64).  kappa != 1 applies the
    exact received-bit reweighting (for frames whose literal recursion
    underflows FP64)."""
    lib = _load()
    lib.orc_set_received_bit_weight(float(kappa))
    q, n, args, keep = _frame_args(codebook, N, Pi, Pd, Ps, I, xmax, rx, priors)
    app = np.zeros((N, q), np.float64)
    ll = ctypes.c_double(0.0)
    st = lib.orc_decode(*args, int(bool(memo)),
                        app.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(ll))
    if st:
        raise OracleError(st, "decode")
    return app, ll.value


def loglik(codebook, N, Pi, Pd, Ps, I, xmax, rx, priors=None, memo=True, kappa=1.0) -> float:
    """log P(Y) only (forward pass)."""
    lib = _load()
    lib.orc_set_received_bit_weight(float(kappa))
    q, n, args, keep = _frame_args(codebook, N, Pi, Pd, Ps, I, xmax, rx, priors)
    ll = ctypes.c_double(0.0)
    st = lib.orc_decode(*args, int(bool(memo)), _NULL_D, ctypes.byref(ll))
    if st:
        raise OracleError(st, "loglik")
    return ll.value


def forward_backward(codebook, N, Pi, Pd, Ps, I, xmax, rx, priors=None):
    """Normalised alpha, beta ((N+1, M) each) and log c_1..log c_N (literal)."""
    lib = _load()
    lib.orc_set_received_bit_weight(1.0)
    q, n, args, keep = _frame_args(codebook, N, Pi, Pd, Ps, I, xmax, rx, priors)
    M = 2 * xmax + 1
    A = np.zeros((N + 1, M), np.float64)
    B = np.zeros((N + 1, M), np.float64)
    lc = np.zeros(N, np.float64)
    dpp = ctypes.POINTER(ctypes.c_double)
    st = lib.orc_forward_backward(*args, A.ctypes.data_as(dpp), B.ctypes.data_as(dpp),
                                  lc.ctypes.data_as(dpp))
    if st:
        raise OracleError(st, "forward_backward")
    return A, B, lc


def _general_args(codebook, N, Pi, Pd, Ps, I, xmax, rx, priors):
    """Arguments of the general entry points: codebook (q, n) is one codebook
    for every symbol, (N, q, n) the per-symbol codebooks C_0..C_{N-1}."""
    cb = np.ascontiguousarray(codebook, dtype=np.uint8)
    if cb.ndim == 3:
        if cb.shape[0] != N:
            raise ValueError(f"per-symbol codebooks: {cb.shape[0]} codebooks for N = {N}")
        per_symbol = 1
        flat = cb[0]
    elif cb.ndim == 2:
        per_symbol = 0
        flat = cb
    else:
        raise ValueError("codebook must be (q, n) or (N, q, n)")
    q, n, args, keep = _frame_args(flat, N, Pi, Pd, Ps, I, xmax, rx, priors)
    args[2] = cb.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    keep.append(cb)
    return q, n, args[:3] + [per_symbol] + args[3:], keep


def _boundary(phi, xmax, keep):
    """Drift prior over the 2 xmax + 1 boundary states (index m + xmax), or NULL."""
    if phi is None:
        return _NULL_D
    a = np.ascontiguousarray(phi, np.float64).reshape(-1)
    if a.size != 2 * xmax + 1:
        raise ValueError(f"a boundary drift prior has 2 xmax + 1 = {2 * xmax + 1} entries")
    keep.append(a)
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def decode_ext(codebook, N, Pi, Pd, Ps, I, xmax, rx, priors=None, memo=True, kappa=1.0,
               drift_start=None, drift_end=None):
    """(APPs (N, q), extrinsic outputs (N, q), log P(Y)) of one frame (FP64).

    codebook is (q, n), one codebook for every symbol, or (N, q, n), the
    constituent encodings C_i of Sec. II-A.  The extrinsic output of symbol i
    is eq. (L) without the symbol's own prior, normalised over D.
    drift_start / drift_end: priors of the drift at the frame's start and end
    (2 xmax + 1 values, index m + xmax; the boundaries alpha_0, beta_N of
    Sec. II-C in stream decoding), None for an isolated frame
    (alpha_0 = [m = 0], beta_N = [m = rho - tau])."""
    lib = _load()
    lib.orc_set_received_bit_weight(float(kappa))
    q, n, args, keep = _general_args(codebook, N, Pi, Pd, Ps, I, xmax, rx, priors)
    dpp = ctypes.POINTER(ctypes.c_double)
    app = np.zeros((N, q), np.float64)
    ext = np.zeros((N, q), np.float64)
    ll = ctypes.c_double(0.0)
    st = lib.orc_decode_general(*args, int(bool(memo)), app.ctypes.data_as(dpp),
                                ext.ctypes.data_as(dpp), ctypes.byref(ll),
                                _boundary(drift_start, xmax, keep), _boundary(drift_end, xmax, keep))
    if st:
        raise OracleError(st, "decode_ext")
    return app, ext, ll.value


def loglik_grad(codebook, N, Pi, Pd, Ps, I, xmax, rx, priors=None, memo=True,
                want_chan=True, want_priors=True, kappa=1.0, drift_start=None, drift_end=None):
    """(logP, d logP/d(Pi,Pd,Ps) or None, d logP/d priors (N,q) or None).
    codebook is (q, n) or per-symbol (N, q, n), and the boundary drift priors,
    as for decode_ext."""
    lib = _load()
    lib.orc_set_received_bit_weight(float(kappa))
    q, n, args, keep = _general_args(codebook, N, Pi, Pd, Ps, I, xmax, rx, priors)
    dpp = ctypes.POINTER(ctypes.c_double)
    dchan = np.zeros(3, np.float64) if want_chan else None
    dpri = np.zeros((N, q), np.float64) if want_priors else None
    ll = ctypes.c_double(0.0)
    st = lib.orc_loglik_grad_general(*args, int(bool(memo)),
                                     dchan.ctypes.data_as(dpp) if want_chan else _NULL_D,
                                     dpri.ctypes.data_as(dpp) if want_priors else _NULL_D,
                                     ctypes.byref(ll), _boundary(drift_start, xmax, keep),
                                     _boundary(drift_end, xmax, keep))
    if st:
        raise OracleError(st, "loglik_grad")
    return ll.value, dchan, dpri


def decode_frame(fr, memo=True, kappa=1.0):
    """Convenience: decode a synthetic frame object (fields as in the input generator)."""
    return decode(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                  priors=fr.priors, memo=memo, kappa=kappa)
