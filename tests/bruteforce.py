"""Brute-force references that pin the FP64 oracle (test-only, pure Python).

None of this reuses the oracle's lattice.  The per-codeword reference
enumerates every channel event pattern bit by bit, as the BSID channel is
described in Sec. II-B: before each transmitted bit, 0..I inserted bits of
either value (weight Pi/2 each), then the bit is deleted (Pd) or transmitted
(Pt), a transmitted bit being flipped with probability Ps.  The frame-level
reference enumerates every message and every split of the received sequence
into per-symbol pieces, and a separate whole-frame recursion over the
transmitted bits cross-checks the split sum.
"""
from __future__ import annotations

import itertools
import math
from collections import defaultdict

import numpy as np


def enumerate_channel(x, I, Pi, Pd, Ps):
    """dict: received tuple -> probability, over all event patterns for bits x."""
    Pt = 1.0 - Pi - Pd
    dist = {(): 1.0}
    for bit in x:
        # all outputs this single bit can produce, with probabilities
        local = defaultdict(float)
        for a in range(I + 1):
            for ins in itertools.product((0, 1), repeat=a):
                w = (Pi / 2.0) ** a
                local[ins] += w * Pd                          # deleted
                local[ins + (int(bit),)] += w * Pt * (1 - Ps)  # transmitted as is
                local[ins + (1 - int(bit),)] += w * Pt * Ps   # transmitted, flipped
        nxt = defaultdict(float)
        for y, p in dist.items():
            for z, pz in local.items():
                if pz != 0.0:
                    nxt[y + z] += p * pz
        dist = dict(nxt)
    return dist


def all_strings(max_len):
    for L in range(max_len + 1):
        for s in itertools.product((0, 1), repeat=L):
            yield s


def length_sum_closed_form(n, I, Pi, Pd, mu):
    """[z^mu] (sum_{a=0}^{I} (Pi z)^a (Pd + Pt z))^n : total probability of
    receiving exactly mu bits (independent of x and Ps)."""
    Pt = 1.0 - Pi - Pd
    per_bit = np.zeros(I + 2)
    for a in range(I + 1):
        per_bit[a] += Pi ** a * Pd
        per_bit[a + 1] += Pi ** a * Pt
    poly = np.array([1.0])
    for _ in range(n):
        poly = np.convolve(poly, per_bit)
    return float(poly[mu]) if mu < poly.size else 0.0


def frame_bruteforce(codebook, priors, rx, I, Pi, Pd, Ps, xmax):
    """Exhaustive P(Y), APPs and d logP/d priors for a tiny frame.

    Sums over every message (q^N) and every split of rx into N consecutive
    pieces of length 0..n(I+1) whose boundary drifts stay within [-xmax, xmax],
    with per-piece probabilities from `enumerate_channel`.  codebook is (q, n),
    one codebook for every symbol, or (N, q, n), a codebook C_k per symbol
    (the constituent encodings of Sec. II-A).
    """
    codebook = np.asarray(codebook)
    N = priors.shape[0]
    books = codebook if codebook.ndim == 3 else np.broadcast_to(codebook, (N,) + codebook.shape)
    q, n = books.shape[1:]
    rho = len(rx)
    ry = tuple(int(b) for b in rx)
    cache = {}

    def table(k, d):
        key = tuple(int(b) for b in books[k][d])
        if key not in cache:
            cache[key] = enumerate_channel(books[k][d], I, Pi, Pd, Ps)
        return cache[key]

    tables = [[table(k, d) for d in range(q)] for k in range(N)]
    maxlen = n * (I + 1)

    def p_given_msg(msg):
        # dynamic program over split points would reuse structure; keep it
        # literal: enumerate every split.
        total = 0.0

        def rec(k, pos, acc):
            nonlocal total
            if k == N:
                if pos == rho:
                    total += acc
                return
            for L in range(0, maxlen + 1):
                end = pos + L
                if end > rho:
                    break
                drift = end - n * (k + 1)
                if abs(drift) > xmax:
                    continue
                pr = tables[k][msg[k]].get(ry[pos:end], 0.0)
                if pr != 0.0:
                    rec(k + 1, end, acc * pr)

        rec(0, 0, 1.0)
        return total

    PY = 0.0
    marg = np.zeros((N, q))
    dpri = np.zeros((N, q))
    for msg in itertools.product(range(q), repeat=N):
        pyx = p_given_msg(msg)
        if pyx == 0.0:
            continue
        w = 1.0
        for k in range(N):
            w *= float(priors[k, msg[k]])
        PY += w * pyx
        for k in range(N):
            marg[k, msg[k]] += w * pyx
            # derivative of w*pyx w.r.t. priors[k, msg[k]]
            rest = 1.0
            for kk in range(N):
                if kk != k:
                    rest *= float(priors[kk, msg[kk]])
            dpri[k, msg[k]] += rest * pyx
    return PY, marg / PY, dpri / PY


def whole_frame_lattice(x, rx, I, Pi, Pd, Ps):
    """P(Y | X) by one recursion over all transmitted bits of the frame, with
    no symbol boundaries and no drift limit (independent cross-check)."""
    Pt = 1.0 - Pi - Pd
    rho = len(rx)
    H = [0.0] * (rho + 1)
    H[0] = 1.0
    for t in range(len(x)):
        K = [0.0] * (rho + 1)
        for j in range(rho + 1):
            s = 0.0
            for a in range(0, min(I, j) + 1):
                s += (Pi / 2.0) ** a * H[j - a]
            K[j] = s
        Hn = [0.0] * (rho + 1)
        for j in range(rho + 1):
            v = Pd * K[j]
            if j >= 1:
                v += (Pt * Ps if rx[j - 1] != x[t] else Pt * (1 - Ps)) * K[j - 1]
            Hn[j] = v
        H = Hn
    return H[rho]


def bsc_symbolwise(codebook, priors, rx, Ps):
    """Pi = Pd = 0: the decoder reduces to symbol-wise MAP on a BSC.
    codebook is (q, n) or per-symbol (N, q, n)."""
    codebook = np.asarray(codebook)
    N = priors.shape[0]
    books = codebook if codebook.ndim == 3 else np.broadcast_to(codebook, (N,) + codebook.shape)
    q, n = books.shape[1:]
    app = np.zeros((N, q))
    logp = 0.0
    for i in range(N):
        y = np.asarray(rx[n * i:n * (i + 1)])
        for d in range(q):
            dh = int(np.sum(y != books[i][d]))
            app[i, d] = float(priors[i, d]) * Ps ** dh * (1 - Ps) ** (n - dh)
        s = app[i].sum()
        logp += math.log(s)
        app[i] /= s
    return app, logp
