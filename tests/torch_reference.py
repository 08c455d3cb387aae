"""FP64 torch-autograd restatement of the decoder's forward pass (test-only).

A third, independently written reference for the gradients: the receiver
metric lattice (eqs. F, F_lastrow with an insertion cap), gamma (eq. gamma)
and the normalised forward recursion (eqs. alpha_prenorm, alpha_norm) are
written with torch tensor ops, and torch's reverse-mode autograd supplies
d logP / d(Pi, Pd, Ps, priors).  Meant for small frames only.
"""
from __future__ import annotations

import torch


def _lattice(x, y, I, Pi, Pd, Ps):
    """Last lattice row F_{n, j}, j = 0..len(y), as a list of 0-d tensors."""
    n = len(x)
    mu = len(y)
    Pt = 1.0 - Pi - Pd
    w = Pi / 2.0
    zero = Pi * 0.0
    F = [zero + 1.0] + [zero] * mu
    for r in range(n):
        G = []
        for j in range(mu + 1):
            g = zero
            wa = zero + 1.0
            for a in range(0, min(I, j) + 1):
                g = g + wa * F[j - a]
                wa = wa * w
            G.append(g)
        Fn = []
        for j in range(mu + 1):
            v = Pd * G[j]
            if j >= 1:
                Q = Pt * Ps if int(y[j - 1]) != int(x[r]) else Pt * (1.0 - Ps)
                v = v + Q * G[j - 1]
            Fn.append(v)
        F = Fn
    return F


def loglik(codebook, priors, rx, I, xmax, Pi, Pd, Ps):
    """log P(Y) as a differentiable function of Pi, Pd, Ps (0-d tensors) and
    priors ((N, q) tensor)."""
    q, n = codebook.shape
    N = priors.shape[0]
    rho = len(rx)
    M = 2 * xmax + 1
    Mn = n * (I + 1) + 1
    # receiver metric per (p, D): list of Mn tensors (zero past rho)
    cache = {}

    def R(p, d):
        key = (p, d)
        if key not in cache:
            mu = min(Mn - 1, rho - p)
            F = _lattice(codebook[d], rx[p:p + mu], I, Pi, Pd, Ps)
            cache[key] = F + [Pi * 0.0] * (Mn - 1 - mu)
        return cache[key]

    alpha = [Pi * 0.0] * M
    alpha[xmax] = Pi * 0.0 + 1.0
    logsum = Pi * 0.0
    for i in range(N):
        an = [Pi * 0.0] * M
        for mp in range(M):
            p = n * i + mp - xmax
            if p < 0 or p > rho:
                continue
            for d in range(q):
                Rv = R(p, d)
                for j in range(Mn):
                    m = mp + j - n
                    if 0 <= m < M:
                        an[m] = an[m] + alpha[mp] * priors[i, d] * Rv[j]
        c = sum(an)
        alpha = [a / c for a in an]
        logsum = logsum + torch.log(c)
    end = rho - n * N + xmax
    return logsum + torch.log(alpha[end])


def grads(codebook, priors_np, rx, I, xmax, Pi, Pd, Ps):
    """(logP, [dPi, dPd, dPs], dpriors (N, q)) via torch autograd in FP64."""
    tPi = torch.tensor(float(Pi), dtype=torch.float64, requires_grad=True)
    tPd = torch.tensor(float(Pd), dtype=torch.float64, requires_grad=True)
    tPs = torch.tensor(float(Ps), dtype=torch.float64, requires_grad=True)
    pr = torch.tensor(priors_np, dtype=torch.float64, requires_grad=True)
    lp = loglik(codebook, pr, rx, I, xmax, tPi, tPd, tPs)
    lp.backward()
    return (lp.item(), [float(tPi.grad), float(tPd.grad), float(tPs.grad)],
            pr.grad.numpy().copy())
