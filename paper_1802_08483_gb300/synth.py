"""Seeded synthetic inputs for the BSID MAP decoder.

This module generates codebooks, messages, symbol priors and BSID channel
realisations.  It holds none of the decoder's arithmetic: it only *draws*
inputs, so both the FP64 oracle and the CUDA path may use it.

Channel (Sec. II-B): at each time one bit waits to enter; with probability Pi
a uniformly random bit is inserted and the channel stays at the same time;
otherwise the bit is deleted (Pd) or transmitted (Pt = 1 - Pi - Pd), and a
transmitted bit is flipped with probability Ps.  The decoder caps insertions
at I per transmitted bit, so the simulator draws at most I insertions before
each bit: the count is a geometric run truncated at I, after which the bit is
deleted with probability Pd / (Pd + Pt) or transmitted.  A realisation whose
final drift exceeds the frame's drift limit is redrawn from the same stream.

Workloads (all seeded, seed = 180208483 + 1e6 * config + frame):
  1: one frame, N=50, q=16, n=10, uniform priors, Pi=Pd=0.01, Ps=0, I=2, xmax=20
  2: one frame, N=1000, q=16, n=10, uniform priors, Pi=Pd=0.05, Ps=0.001, I=2, xmax=200
  3: 4096 mixed frames: N ~ U[100,4000], (q,n) uniform over
     {(2,4),(8,6),(16,10),(32,8),(64,12)}, Pi=Pd log-uniform in [1e-3,0.1],
     Ps ~ U[0,0.01], I=2, xmax = ceil(6 sqrt(N n (Pi+Pd))), Dirichlet(1) priors
  4: 256 frames, N=2000, q=32, n=8, Pi=Pd=0.03, Ps=0.005, I=2, xmax=120, Dirichlet(1)
  5: 64 frames, N=8000, q=64, n=12, Pi=Pd=0.1, Ps=0.01, I=3, xmax=830, Dirichlet(1)
Configs 4 and 5 share one codebook per config (drawn from frame 0's stream);
config 3 draws a codebook per frame.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

SEED_BASE = 180208483
QN_CHOICES = [(2, 4), (8, 6), (16, 10), (32, 8), (64, 12)]


def frame_seed(config: int, frame: int) -> int:
    return SEED_BASE + 1_000_000 * int(config) + int(frame)


@dataclass
class Frame:
    q: int
    n: int
    N: int
    I: int
    xmax: int
    Pi: float
    Pd: float
    Ps: float
    codebook: np.ndarray          # (q, n) uint8 0/1, distinct rows; or (N, q, n): one per symbol
    message: np.ndarray           # (N,) int64
    priors: Optional[np.ndarray]  # (N, q) float32, or None for uniform
    rx: np.ndarray                # (rho,) uint8 0/1
    tag: str = ""
    # stream decoding: priors of the drift at the frame's start and end
    # (2 xmax + 1 each, index m + xmax), or None for an isolated frame
    drift_start: Optional[np.ndarray] = None
    drift_end: Optional[np.ndarray] = None

    @property
    def rho(self) -> int:
        return int(self.rx.size)

    @property
    def tau(self) -> int:
        return self.n * self.N

    @property
    def info_bits(self) -> float:
        return self.N * math.log2(self.q)

    def priors_or_uniform(self) -> np.ndarray:
        if self.priors is not None:
            return self.priors
        return np.full((self.N, self.q), 1.0 / self.q, np.float32)


def random_codebook(rng: np.random.Generator, q: int, n: int) -> np.ndarray:
    """q distinct uniformly random n-bit words, as a (q, n) 0/1 array."""
    if q > (1 << n):
        raise ValueError("q > 2^n")
    words = rng.choice(1 << n, size=q, replace=False)
    return ((words[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)


def dirichlet_priors(rng: np.random.Generator, N: int, q: int) -> np.ndarray:
    p = rng.dirichlet(np.ones(q), size=N).astype(np.float32)
    return p


def draw_message(rng: np.random.Generator, priors: Optional[np.ndarray], N: int, q: int):
    if priors is None:
        return rng.integers(0, q, size=N)
    cdf = np.cumsum(priors.astype(np.float64), axis=1)
    u = rng.random(N) * cdf[:, -1]
    msg = (u[:, None] > cdf).sum(axis=1)
    return np.minimum(msg, q - 1)


def bsid_channel(rng: np.random.Generator, x: np.ndarray, Pi: float, Pd: float, Ps: float,
                 I: int) -> np.ndarray:
    """One BSID realisation of the 0/1 array x with at most I insertions per bit."""
    tau = x.size
    if Pi > 0:
        g = rng.geometric(1.0 - Pi, size=tau) - 1
        ins = np.minimum(g, I)
    else:
        ins = np.zeros(tau, np.int64)
    Pt = 1.0 - Pi - Pd
    keep = rng.random(tau) >= (Pd / (Pd + Pt) if (Pd + Pt) > 0 else 0.0)
    flip = rng.random(tau) < Ps
    per_bit = ins + keep.astype(np.int64)
    rho = int(per_bit.sum())
    out = rng.integers(0, 2, size=rho).astype(np.uint8)   # inserted bits (overwritten below)
    start = np.concatenate([[0], np.cumsum(per_bit)[:-1]])
    pos = start + ins
    tx = keep
    out[pos[tx]] = (x[tx] ^ flip[tx]).astype(np.uint8)
    return out


def make_frame(rng: np.random.Generator, q: int, n: int, N: int, I: int, xmax: int,
               Pi: float, Pd: float, Ps: float, codebook: Optional[np.ndarray] = None,
               dirichlet: bool = False, tag: str = "") -> Frame:
    if codebook is None:
        codebook = random_codebook(rng, q, n)
    priors = dirichlet_priors(rng, N, q) if dirichlet else None
    msg = draw_message(rng, priors, N, q)
    x = codebook[msg].reshape(-1)
    for _ in range(10000):
        rx = bsid_channel(rng, x, Pi, Pd, Ps, I)
        if abs(rx.size - x.size) <= xmax:
            break
    else:
        raise RuntimeError("could not draw a realisation within the drift limit")
    return Frame(q=q, n=n, N=N, I=I, xmax=xmax, Pi=float(Pi), Pd=float(Pd), Ps=float(Ps),
                 codebook=codebook, message=msg.astype(np.int64), priors=priors, rx=rx, tag=tag)


def per_symbol_frame(rng: np.random.Generator, q: int, n: int, N: int, I: int, xmax: int,
                     Pi: float, Pd: float, Ps: float, tag: str = "") -> Frame:
    """Frame whose symbol i is sent with its own random codebook C_i (an (N, q, n)
    codebook array), Dirichlet(1) priors, message drawn from the priors."""
    books = np.stack([random_codebook(rng, q, n) for _ in range(N)])
    priors = dirichlet_priors(rng, N, q)
    msg = draw_message(rng, priors, N, q)
    x = books[np.arange(N), msg].reshape(-1)
    for _ in range(10000):
        rx = bsid_channel(rng, x, Pi, Pd, Ps, I)
        if abs(rx.size - x.size) <= xmax:
            break
    else:
        raise RuntimeError("could not draw a realisation within the drift limit")
    return Frame(q=q, n=n, N=N, I=I, xmax=xmax, Pi=float(Pi), Pd=float(Pd), Ps=float(Ps),
                 codebook=books, message=msg.astype(np.int64), priors=priors, rx=rx, tag=tag)


def _gauss_window(xmax: int, centre: float, sd: float, lo: int, hi: int) -> np.ndarray:
    """Discretised Gaussian over drift states m in [lo, hi] (index m + xmax)."""
    m = np.arange(-xmax, xmax + 1)
    w = np.exp(-0.5 * ((m - centre) / sd) ** 2)
    w[(m < lo) | (m > hi)] = 0.0
    return (w / w.sum()).astype(np.float32)


def stream_frame(rng: np.random.Generator, q: int, n: int, N: int, I: int, xmax: int,
                 Pi: float, Pd: float, Ps: float, pre: int, post: int, sd: float,
                 tag: str = "") -> Frame:
    """A frame cut from a stream: `pre` bits of the previous frame before it and
    `post` bits of the next one after it.  The boundary drift priors are
    discretised Gaussians of width sd around the true start (drift pre) and the
    true end, over the states the received bits allow."""
    fr = make_frame(rng, q, n, N, I, max(1, xmax - pre - post), Pi, Pd, Ps, dirichlet=True,
                    tag=tag)
    body = fr.rx
    rx = np.concatenate([rng.integers(0, 2, pre), body, rng.integers(0, 2, post)]).astype(np.uint8)
    tau = n * N
    end = pre + body.size - tau  # true end drift
    fr.rx = rx
    fr.xmax = xmax
    fr.drift_start = _gauss_window(xmax, pre, sd, 0, xmax)
    fr.drift_end = _gauss_window(xmax, end, sd, -xmax, rx.size - tau)
    return fr


def c3_params(rng: np.random.Generator):
    N = int(rng.integers(100, 4001))
    q, n = QN_CHOICES[int(rng.integers(0, len(QN_CHOICES)))]
    p = float(math.exp(rng.uniform(math.log(1e-3), math.log(0.1))))
    Ps = float(rng.uniform(0.0, 0.01))
    xmax = int(math.ceil(6.0 * math.sqrt(N * n * (p + p))))
    return q, n, N, p, Ps, xmax


def config_frame(config: int, frame: int) -> Frame:
    """Frame `frame` of workload `config` (1..7), fully determined by its seed."""
    rng = np.random.default_rng(frame_seed(config, frame))
    if config == 1:
        return make_frame(rng, 16, 10, 50, 2, 20, 0.01, 0.01, 0.0, tag="c1")
    if config == 2:
        return make_frame(rng, 16, 10, 1000, 2, 200, 0.05, 0.05, 0.001, tag="c2")
    if config == 3:
        q, n, N, p, Ps, xmax = c3_params(rng)
        return make_frame(rng, q, n, N, 2, xmax, p, p, Ps, dirichlet=True, tag=f"c3/{frame}")
    if config in (4, 5):
        cb_rng = np.random.default_rng(frame_seed(config, 0) ^ 0x5EED)
        if config == 4:
            cb = random_codebook(cb_rng, 32, 8)
            return make_frame(rng, 32, 8, 2000, 2, 120, 0.03, 0.03, 0.005, codebook=cb,
                              dirichlet=True, tag=f"c4/{frame}")
        cb = random_codebook(cb_rng, 64, 12)
        return make_frame(rng, 64, 12, 8000, 3, 830, 0.1, 0.1, 0.01, codebook=cb,
                          dirichlet=True, tag=f"c5/{frame}")
    if config == 6:
        # one codebook per symbol (Sec. II-A), N=1000, q=16, n=10, xmax by the
        # mixed workload's rule: ceil(6 sqrt(N n (Pi + Pd))) = 85
        return per_symbol_frame(rng, 16, 10, 1000, 2, 85, 0.01, 0.01, 0.001, tag=f"c6/{frame}")
    if config == 7:
        # frames cut from a stream: up to 8 bits of each neighbour inside the
        # received window, Gaussian drift priors (sd 3 bits) on both boundaries
        pre, post = int(rng.integers(0, 9)), int(rng.integers(0, 9))
        return stream_frame(rng, 16, 10, 1000, 2, 85, 0.01, 0.01, 0.001, pre, post, 3.0,
                            tag=f"c7/{frame}")
    raise ValueError(f"unknown workload {config}")


CONFIG_FRAMES = {1: 1, 2: 1, 3: 4096, 4: 256, 5: 64, 6: 64, 7: 256}


def config_frames(config: int, frames: Optional[List[int]] = None) -> List[Frame]:
    if frames is None:
        frames = list(range(CONFIG_FRAMES[config]))
    return [config_frame(config, f) for f in frames]


def c3_frame_shape(frame: int):
    """(q, n, N, xmax) of workload-3 frame `frame` without simulating it."""
    rng = np.random.default_rng(frame_seed(3, frame))
    q, n, N, p, Ps, xmax = c3_params(rng)
    return q, n, N, xmax


def tiny_frame(seed: int, q: int = 4, n: int = 3, N: int = 3, I: int = 1, xmax: int = 9,
               Pi: float = 0.1, Pd: float = 0.1, Ps: float = 0.05, dirichlet: bool = True) -> Frame:
    """Small random frame for brute-force and parity tests."""
    rng = np.random.default_rng(seed)
    return make_frame(rng, q, n, N, I, xmax, Pi, Pd, Ps, dirichlet=dirichlet, tag=f"tiny/{seed}")
