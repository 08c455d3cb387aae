"""ctypes binding of libmapdec.so (include/mapdec.h), argument marshalling only.

Every function named ``mapdec_*`` here calls the C entry point of the same
name.  Array arguments may be numpy arrays (host memory), torch tensors (host
or CUDA; must be contiguous), raw integer addresses, or None for NULL.  Every
step of the decoder runs in the library's CUDA kernels; there is no CPU path.
A missing library raises immediately.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmapdec.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "mapdec.h")

MAPDEC_OK = 0
MAPDEC_ERR_ARG = 1
MAPDEC_ERR_DRIFT_RANGE = 2
MAPDEC_ERR_ZERO_PROB = 3
MAPDEC_ERR_NOMEM = 4
MAPDEC_ERR_CUDA = 5
MAPDEC_ERR_TIMEOUT = 6
MAPDEC_ERR_UNSUPPORTED = 7
MAPDEC_ERR_TOO_LARGE = 8

MAPDEC_BATCH_GRAPH = 1
MAPDEC_BATCH_PLAIN = 2
MAPDEC_BATCH_GRAD = 4
MAPDEC_BATCH_TIMING = 8
MAPDEC_BATCH_SEGMENTED = 16
MAPDEC_BATCH_EXTRINSIC = 32
PHASES = ("pack", "forward", "chains", "backward", "finalize")


class MapDecError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.mapdec_strerror(status).decode() if _lib is not None else str(status)
        super().__init__(f"{where}: {msg} (status {status})")


class FrameDesc(ctypes.Structure):
    _fields_ = [("q", ctypes.c_int), ("n", ctypes.c_int), ("N", ctypes.c_int),
                ("I", ctypes.c_int), ("xmax", ctypes.c_int), ("Pi", ctypes.c_double),
                ("Pd", ctypes.c_double), ("Ps", ctypes.c_double),
                ("codebook", ctypes.c_void_p), ("rx_len", ctypes.c_int64),
                ("codebook_per_symbol", ctypes.c_int), ("drift_start", ctypes.c_void_p),
                ("drift_end", ctypes.c_void_p)]


_lib = None

_VP = ctypes.c_void_p
_SIGS = {
    "mapdec_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, ctypes.c_int, _VP,
                                     ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_int]),
    "mapdec_set_stream": (ctypes.c_int, [_VP, _VP]),
    "mapdec_decode": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP, _VP, _VP]),
    "mapdec_decode_ext": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP, _VP, _VP, _VP]),
    "mapdec_loglik_grad": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP, _VP, _VP, _VP]),
    "mapdec_receiver_metric": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP]),
    "mapdec_destroy": (None, [_VP]),
    "mapdec_decode_noalloc": (ctypes.c_int, [ctypes.POINTER(FrameDesc), _VP, _VP, _VP, _VP, _VP]),
    "mapdec_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "mapdec_batch_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.POINTER(FrameDesc),
                                           ctypes.c_int, ctypes.c_int, ctypes.c_int64]),
    "mapdec_batch_layout": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "mapdec_batch_buffers": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "mapdec_batch_rx_offset": (ctypes.c_int64, [_VP, ctypes.c_int]),
    "mapdec_batch_run": (ctypes.c_int, [_VP]),
    "mapdec_batch_sync": (ctypes.c_int, [_VP]),
    "mapdec_batch_status": (ctypes.c_int, [_VP, _VP]),
    "mapdec_batch_decode": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "mapdec_batch_decode_ext": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "mapdec_batch_loglik_grad": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "mapdec_batch_set_stream": (ctypes.c_int, [_VP, _VP]),
    "mapdec_batch_destroy": (None, [_VP]),
    "mapdec_batch_last_launches": (ctypes.c_int64, [_VP]),
    "mapdec_batch_phase_ms": (ctypes.c_int, [_VP, _VP]),
    "mapdec_batch_num_waves": (ctypes.c_int, [_VP]),
    "mapdec_batch_tc_frames": (ctypes.c_int, [_VP, _VP]),
    "mapdec_set_drift_priors": (ctypes.c_int, [_VP, _VP, _VP]),
    "mapdec_fp32_fma_peak": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), _VP]),
    "mapdec_tune_set": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP]),
    "mapdec_tune_get": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP]),
    "mapdec_tune_clear": (ctypes.c_int, []),
}


class Tune(ctypes.Structure):
    """mapdec_tune_t: launch parameters of one (q, n, I) class (0 = planner's choice)."""
    _fields_ = [("P", ctypes.c_int), ("nsub", ctypes.c_int), ("chain_budget_kb", ctypes.c_int),
                ("chain_stages", ctypes.c_int), ("store_metric", ctypes.c_int),
                ("tensor_cores", ctypes.c_int), ("chain_threads", ctypes.c_int)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


def header_symbols() -> list:
    """Every function declared in include/mapdec.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mapdec_[a-z_0-9]+)\s*\(", txt)))


def load(path: Optional[str] = None):
    """Load libmapdec.so (raises if it has not been built).  The environment
    variable MAPDEC_LIB names an alternative build of the same library (for
    comparing kernel variants); by default the in-tree build is loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("MAPDEC_LIB") or LIB_PATH  # MAPDEC_LIB: an alternative build
    if not os.path.exists(path):
        raise RuntimeError(f"libmapdec.so not found at {path}; run __graft_entry__.build() "
                           "(the decoder has no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(x):
    """Address of an array argument (numpy, torch, int) or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported buffer type {type(x)}")


def _check(st: int, where: str):
    if st != MAPDEC_OK:
        raise MapDecError(st, where)


# --------------------------------------------------------------------------
# same-name wrappers of the C entry points
# --------------------------------------------------------------------------
def mapdec_strerror(status: int) -> str:
    return load().mapdec_strerror(int(status)).decode()


def mapdec_create(q, n, codebook, N, Pi, Pd, Ps, I, xmax):
    lib = load()
    h = _VP()
    cb = np.ascontiguousarray(codebook, dtype=np.uint8) if isinstance(codebook, np.ndarray) \
        else codebook
    _check(lib.mapdec_create(ctypes.byref(h), int(q), int(n), _ptr(cb), int(N), float(Pi),
                             float(Pd), float(Ps), int(I), int(xmax)), "mapdec_create")
    return h


def mapdec_set_stream(h, stream):
    _check(load().mapdec_set_stream(h, stream), "mapdec_set_stream")


def mapdec_decode(h, rx, rx_len, priors, app_out, loglik_out):
    return load().mapdec_decode(h, _ptr(rx), int(rx_len), _ptr(priors), _ptr(app_out),
                                _ptr(loglik_out))


def mapdec_decode_ext(h, rx, rx_len, priors, app_out, ext_out, loglik_out):
    return load().mapdec_decode_ext(h, _ptr(rx), int(rx_len), _ptr(priors), _ptr(app_out),
                                    _ptr(ext_out), _ptr(loglik_out))


def mapdec_loglik_grad(h, rx, rx_len, priors, dlogp_dchan, dlogp_dpriors, loglik_out):
    return load().mapdec_loglik_grad(h, _ptr(rx), int(rx_len), _ptr(priors), _ptr(dlogp_dchan),
                                     _ptr(dlogp_dpriors), _ptr(loglik_out))


def mapdec_receiver_metric(h, rx, rx_len, R_out):
    return load().mapdec_receiver_metric(h, _ptr(rx), int(rx_len), _ptr(R_out))


def mapdec_set_drift_priors(h, drift_start, drift_end):
    _check(load().mapdec_set_drift_priors(h, _ptr(drift_start), _ptr(drift_end)),
           "mapdec_set_drift_priors")


def mapdec_destroy(h):
    load().mapdec_destroy(h)


def mapdec_decode_noalloc(frame, rx_dev, priors_dev, app_dev, loglik_dev, stream=None):
    """frame: object with q, n, N, I, xmax, Pi, Pd, Ps, codebook and rho (or rx_len)."""
    cb = np.ascontiguousarray(frame.codebook, dtype=np.uint8)
    rho = frame.rho if hasattr(frame, "rho") else int(frame.rx_len)
    desc = FrameDesc(int(frame.q), int(frame.n), int(frame.N), int(frame.I), int(frame.xmax),
                     float(frame.Pi), float(frame.Pd), float(frame.Ps), cb.ctypes.data, int(rho))
    return load().mapdec_decode_noalloc(ctypes.byref(desc), _ptr(rx_dev), _ptr(priors_dev),
                                        _ptr(app_dev), _ptr(loglik_dev), stream)


def mapdec_batch_create(frames, flags=0, mem_budget_bytes=0):
    """frames: sequence of objects with q, n, N, I, xmax, Pi, Pd, Ps, codebook, rx (or rho)."""
    lib = load()
    arr = (FrameDesc * len(frames))()
    keep = []
    for k, fr in enumerate(frames):
        cb = np.ascontiguousarray(fr.codebook, dtype=np.uint8)
        keep.append(cb)
        rho = fr.rho if hasattr(fr, "rho") else int(fr.rx_len)
        # a (q, n) codebook serves every symbol; (N, q, n) gives one per symbol;
        # optional boundary drift priors (stream decoding): fr.drift_start / drift_end
        bounds = []
        for name in ("drift_start", "drift_end"):
            v = getattr(fr, name, None)
            if v is None:
                bounds.append(None)
            else:
                a = np.ascontiguousarray(v, dtype=np.float32)
                keep.append(a)
                bounds.append(a.ctypes.data)
        arr[k] = FrameDesc(int(fr.q), int(fr.n), int(fr.N), int(fr.I), int(fr.xmax),
                           float(fr.Pi), float(fr.Pd), float(fr.Ps), cb.ctypes.data, int(rho),
                           1 if cb.ndim == 3 else 0, bounds[0], bounds[1])
    b = _VP()
    _check(lib.mapdec_batch_create(ctypes.byref(b), arr, len(frames), int(flags),
                                   int(mem_budget_bytes)), "mapdec_batch_create")
    return b


def mapdec_batch_layout(b, nframes):
    rx_off = np.zeros(nframes, np.int64)
    sym_off = np.zeros(nframes, np.int64)
    rx_total = ctypes.c_int64()
    pr_total = ctypes.c_int64()
    _check(load().mapdec_batch_layout(b, _ptr(rx_off), _ptr(sym_off), ctypes.addressof(rx_total),
                                      ctypes.addressof(pr_total)), "mapdec_batch_layout")
    return rx_off, sym_off, rx_total.value, pr_total.value


def mapdec_batch_buffers(b):
    ptrs = [_VP() for _ in range(4)]
    _check(load().mapdec_batch_buffers(b, *[ctypes.addressof(p) for p in ptrs]),
           "mapdec_batch_buffers")
    return tuple(p.value for p in ptrs)


def mapdec_batch_rx_offset(b, frame):
    return int(load().mapdec_batch_rx_offset(b, int(frame)))


def mapdec_batch_run(b):
    return load().mapdec_batch_run(b)


def mapdec_batch_sync(b):
    return load().mapdec_batch_sync(b)


def mapdec_batch_status(b, nframes):
    st = np.zeros(nframes, np.int32)
    _check(load().mapdec_batch_status(b, _ptr(st)), "mapdec_batch_status")
    return st


def mapdec_batch_decode(b, rx_all, priors_all, app_all, loglik_all):
    return load().mapdec_batch_decode(b, _ptr(rx_all), _ptr(priors_all), _ptr(app_all),
                                      _ptr(loglik_all))


def mapdec_batch_decode_ext(b, rx_all, priors_all, app_all, ext_all, loglik_all):
    return load().mapdec_batch_decode_ext(b, _ptr(rx_all), _ptr(priors_all), _ptr(app_all),
                                          _ptr(ext_all), _ptr(loglik_all))


def mapdec_batch_loglik_grad(b, rx_all, priors_all, dchan_all, dpriors_all, loglik_all):
    return load().mapdec_batch_loglik_grad(b, _ptr(rx_all), _ptr(priors_all), _ptr(dchan_all),
                                           _ptr(dpriors_all), _ptr(loglik_all))


def mapdec_batch_set_stream(b, stream):
    _check(load().mapdec_batch_set_stream(b, stream), "mapdec_batch_set_stream")


def mapdec_batch_destroy(b):
    load().mapdec_batch_destroy(b)


def mapdec_batch_last_launches(b):
    return int(load().mapdec_batch_last_launches(b))


def mapdec_batch_phase_ms(b):
    ms = np.zeros(5, np.float64)
    _check(load().mapdec_batch_phase_ms(b, _ptr(ms)), "mapdec_batch_phase_ms")
    return ms


def mapdec_batch_num_waves(b):
    return int(load().mapdec_batch_num_waves(b))


def mapdec_batch_tc_frames(b, nframes=None):
    """Frames whose forward producer runs on the tensor cores; with nframes,
    (count, per-frame flags: bit 0 forward producer, bit 1 APP producer)."""
    if nframes is None:
        return int(load().mapdec_batch_tc_frames(b, None))
    fl = np.zeros(int(nframes), np.int32)
    c = int(load().mapdec_batch_tc_frames(b, _ptr(fl)))
    return c, fl


def mapdec_tune_set(q, n, I, tune=None):
    """Set (tune: Tune or dict) or remove (None) the tuning entry of class (q, n, I)."""
    if isinstance(tune, dict):
        tune = Tune(**{k: int(v) for k, v in tune.items() if k in dict(Tune._fields_)})
    _check(load().mapdec_tune_set(int(q), int(n), int(I),
                                  ctypes.byref(tune) if tune is not None else None),
           "mapdec_tune_set")


def mapdec_tune_get(q, n, I):
    """The tuning entry of class (q, n, I) as a dict, or None."""
    t = Tune()
    st = load().mapdec_tune_get(int(q), int(n), int(I), ctypes.byref(t))
    return t.as_dict() if st == MAPDEC_OK else None


def mapdec_tune_clear():
    _check(load().mapdec_tune_clear(), "mapdec_tune_clear")


def mapdec_fp32_fma_peak(stream=None) -> float:
    """Measured FP32 FMA throughput of the current device, TFLOP/s."""
    v = ctypes.c_double(0.0)
    _check(load().mapdec_fp32_fma_peak(ctypes.byref(v), _ptr(stream)), "mapdec_fp32_fma_peak")
    return v.value


# --------------------------------------------------------------------------
# small conveniences over the same calls
# --------------------------------------------------------------------------
class Decoder:
    """One code and channel; decode(rx, priors) -> (app, loglik) as numpy arrays."""

    def __init__(self, q, n, codebook, N, Pi, Pd, Ps, I, xmax):
        self.q, self.n, self.N, self.I, self.xmax = int(q), int(n), int(N), int(I), int(xmax)
        self.Pi, self.Pd, self.Ps = float(Pi), float(Pd), float(Ps)
        self.h = None
        self.h = mapdec_create(q, n, codebook, N, Pi, Pd, Ps, I, xmax)

    @classmethod
    def for_frame(cls, fr):
        return cls(fr.q, fr.n, fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax)

    def decode(self, rx, priors=None):
        rx = np.ascontiguousarray(rx, dtype=np.uint8)
        pr = None if priors is None else np.ascontiguousarray(priors, dtype=np.float32)
        app = np.zeros((self.N, self.q), np.float32)
        ll = np.zeros(1, np.float64)
        _check(mapdec_decode(self.h, rx, rx.size, pr, app, ll), "mapdec_decode")
        return app, float(ll[0])

    def decode_ext(self, rx, priors=None):
        """(APPs, extrinsic outputs, log P): eq. (L) with and without each
        symbol's own prior, both normalised over D."""
        rx = np.ascontiguousarray(rx, dtype=np.uint8)
        pr = None if priors is None else np.ascontiguousarray(priors, dtype=np.float32)
        app = np.zeros((self.N, self.q), np.float32)
        ext = np.zeros((self.N, self.q), np.float32)
        ll = np.zeros(1, np.float64)
        _check(mapdec_decode_ext(self.h, rx, rx.size, pr, app, ext, ll), "mapdec_decode_ext")
        return app, ext, float(ll[0])

    def loglik_grad(self, rx, priors=None):
        rx = np.ascontiguousarray(rx, dtype=np.uint8)
        pr = None if priors is None else np.ascontiguousarray(priors, dtype=np.float32)
        dchan = np.zeros(3, np.float64)
        dpri = np.zeros((self.N, self.q), np.float32)
        ll = np.zeros(1, np.float64)
        _check(mapdec_loglik_grad(self.h, rx, rx.size, pr, dchan, dpri, ll), "mapdec_loglik_grad")
        return float(ll[0]), dchan, dpri

    def loglik_into(self, rx, priors, ll_out):
        """log P(Y) alone (no APPs copied out) into ll_out: 1 double, host or
        device.  priors: a contiguous float32 array or tensor (host or device)
        or None."""
        rx = np.ascontiguousarray(rx, dtype=np.uint8)
        _check(mapdec_decode(self.h, rx, rx.size, priors, None, ll_out), "mapdec_decode")

    def loglik_grad_into(self, rx, priors, dchan_out, dpri_out, ll_out):
        """The adjoint path into caller-owned buffers (host or device)."""
        rx = np.ascontiguousarray(rx, dtype=np.uint8)
        _check(mapdec_loglik_grad(self.h, rx, rx.size, priors, dchan_out, dpri_out, ll_out),
               "mapdec_loglik_grad")

    def set_stream(self, stream):
        mapdec_set_stream(self.h, stream)

    def set_drift_priors(self, drift_start=None, drift_end=None):
        """Stream decoding: priors (2 xmax + 1 each, index m + xmax) of the drift
        at the frame's start and end for the following calls; None = the
        isolated frame's boundary."""
        a = None if drift_start is None else np.ascontiguousarray(drift_start, np.float32)
        b = None if drift_end is None else np.ascontiguousarray(drift_end, np.float32)
        mapdec_set_drift_priors(self.h, a, b)

    def receiver_metric(self, rx, MN):
        rx = np.ascontiguousarray(rx, dtype=np.uint8)
        R = np.zeros((rx.size + 1, self.q, MN), np.float32)
        _check(mapdec_receiver_metric(self.h, rx, rx.size, R), "mapdec_receiver_metric")
        return R

    def close(self):
        if self.h is not None:
            mapdec_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many frames decoded together; inputs concatenated in frame order."""

    def __init__(self, frames, flags=MAPDEC_BATCH_GRAPH, mem_budget_bytes=0):
        self.frames = list(frames)
        self.nf = len(self.frames)
        self.b = mapdec_batch_create(self.frames, flags, mem_budget_bytes)
        self.rx_off, self.sym_off, self.rx_total, self.prior_total = \
            mapdec_batch_layout(self.b, self.nf)

    def concat_inputs(self):
        rx = np.concatenate([f.rx for f in self.frames]).astype(np.uint8)
        pr = np.concatenate([f.priors_or_uniform().reshape(-1) for f in self.frames])
        return rx, pr.astype(np.float32)

    def split(self, flat):
        out = []
        for k, f in enumerate(self.frames):
            o = int(self.sym_off[k])
            out.append(flat[o:o + f.N * f.q].reshape(f.N, f.q))
        return out

    def decode(self, rx_all, priors_all):
        app = np.zeros(self.prior_total, np.float32)
        ll = np.zeros(self.nf, np.float64)
        st = mapdec_batch_decode(self.b, rx_all, priors_all, app, ll)
        return st, app, ll

    def decode_ext(self, rx_all, priors_all):
        """Batch created with MAPDEC_BATCH_EXTRINSIC: (status, APPs, extrinsic
        outputs, log-likelihoods), APPs and extrinsic outputs concatenated."""
        app = np.zeros(self.prior_total, np.float32)
        ext = np.zeros(self.prior_total, np.float32)
        ll = np.zeros(self.nf, np.float64)
        st = mapdec_batch_decode_ext(self.b, rx_all, priors_all, app, ext, ll)
        return st, app, ext, ll

    def loglik_into(self, rx_all, priors_all, ll_out):
        """Per-frame log P(Y) alone (no APPs copied out) into ll_out (host or
        device); returns the worst frame status."""
        return mapdec_batch_decode(self.b, rx_all, priors_all, None, ll_out)

    def loglik_grad_into(self, rx_all, priors_all, dchan_out, dpri_out, ll_out):
        """The adjoint path into caller-owned buffers (host or device)."""
        return mapdec_batch_loglik_grad(self.b, rx_all, priors_all, dchan_out, dpri_out, ll_out)

    def set_stream(self, stream):
        mapdec_batch_set_stream(self.b, stream)

    def loglik_grad(self, rx_all, priors_all):
        dchan = np.zeros(3 * self.nf, np.float64)
        dpri = np.zeros(self.prior_total, np.float32)
        ll = np.zeros(self.nf, np.float64)
        st = mapdec_batch_loglik_grad(self.b, rx_all, priors_all, dchan, dpri, ll)
        return st, dchan.reshape(self.nf, 3), dpri, ll

    def close(self):
        if self.b is not None:
            mapdec_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
