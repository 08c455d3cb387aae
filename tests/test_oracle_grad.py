"""Pins for the oracle's gradients d logP / d(Pi, Pd, Ps, priors).

(i) central finite differences of the brute-force P(Y) on tiny frames (fully
    independent of the oracle), and of the oracle's own log P(Y) (h = 1e-6);
(ii) the path-count identities: every path has #ins - #del = rho - tau and
     #del + #trans = tau, which tie d/dPi to d/dPd;
(iii) sum_D Pr{D_i = D} d logP / d Pr{D_i = D} = 1 for every i;
(iv) an FP64 torch-autograd restatement of the forward pass.
"""
import math

import numpy as np
import pytest

import oracle
import torch_reference
from bruteforce import frame_bruteforce
from paper_1802_08483_gb300 import synth


def _grad(fr, priors=None, memo=True):
    pr = fr.priors_or_uniform().astype(np.float64) if priors is None else priors
    return oracle.loglik_grad(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                              priors=pr, memo=memo)


def _ll(fr, Pi, Pd, Ps, priors=None):
    pr = fr.priors_or_uniform().astype(np.float64) if priors is None else priors
    return oracle.loglik(fr.codebook, fr.N, Pi, Pd, Ps, fr.I, fr.xmax, fr.rx, priors=pr)


@pytest.mark.parametrize("seed", [101, 102, 103])
def test_channel_grad_vs_bruteforce_fd(seed):
    fr = synth.tiny_frame(seed, q=3, n=3, N=3, I=1, xmax=3, Pi=0.12, Pd=0.08, Ps=0.06)
    pr = fr.priors.astype(np.float64)
    ll, dchan, _ = _grad(fr)
    h = 1e-6
    base = [fr.Pi, fr.Pd, fr.Ps]
    for k in range(3):
        up = list(base); up[k] += h
        dn = list(base); dn[k] -= h
        pu, _, _ = frame_bruteforce(fr.codebook, pr, fr.rx, fr.I, *up, fr.xmax)
        pd, _, _ = frame_bruteforce(fr.codebook, pr, fr.rx, fr.I, *dn, fr.xmax)
        fd = (math.log(pu) - math.log(pd)) / (2 * h)
        assert dchan[k] == pytest.approx(fd, rel=1e-6, abs=1e-6), k


@pytest.mark.parametrize("seed", [111, 112])
def test_prior_grad_vs_bruteforce(seed):
    fr = synth.tiny_frame(seed, q=3, n=3, N=3, I=1, xmax=4, Pi=0.1, Pd=0.1, Ps=0.05)
    pr = fr.priors.astype(np.float64)
    _, _, dpri = _grad(fr)
    _, _, dpri_ref = frame_bruteforce(fr.codebook, pr, fr.rx, fr.I, fr.Pi, fr.Pd, fr.Ps, fr.xmax)
    np.testing.assert_allclose(dpri, dpri_ref, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("seed", [121, 122])
def test_channel_grad_vs_oracle_fd(seed):
    rng = np.random.default_rng(seed)
    fr = synth.make_frame(rng, 8, 6, 40, 2, 14, 0.04, 0.03, 0.01, dirichlet=True)
    ll, dchan, _ = _grad(fr)
    h = 1e-6
    base = [fr.Pi, fr.Pd, fr.Ps]
    for k in range(3):
        up = list(base); up[k] += h
        dn = list(base); dn[k] -= h
        fd = (_ll(fr, *up) - _ll(fr, *dn)) / (2 * h)
        assert dchan[k] == pytest.approx(fd, rel=1e-6, abs=1e-5), k


def test_prior_grad_vs_oracle_fd():
    rng = np.random.default_rng(131)
    fr = synth.make_frame(rng, 4, 4, 12, 2, 8, 0.05, 0.05, 0.02, dirichlet=True)
    pr = fr.priors.astype(np.float64)
    _, _, dpri = _grad(fr)
    h = 1e-6
    ll0 = _ll(fr, fr.Pi, fr.Pd, fr.Ps)
    # central-difference rounding noise is about eps * |logP| / h
    noise = 4 * np.finfo(np.float64).eps * abs(ll0) / h
    for (i, d) in [(0, 0), (3, 2), (11, 3), (6, 1), (5, int(np.argmax(dpri[5])))]:
        up = pr.copy(); up[i, d] += h
        dn = pr.copy(); dn[i, d] -= h
        fd = (_ll(fr, fr.Pi, fr.Pd, fr.Ps, up) - _ll(fr, fr.Pi, fr.Pd, fr.Ps, dn)) / (2 * h)
        assert dpri[i, d] == pytest.approx(fd, rel=1e-6, abs=noise)


@pytest.mark.parametrize("seed", [141, 142, 143])
def test_path_count_identity(seed):
    """With independent partials (Pi, Pd, Pt free): Pi d_i - Pd d_d = rho - tau and
    Pd d_d + Pt d_t = tau.  The totals are g_i = d_i - d_t, g_d = d_d - d_t; solving the
    second identity for d_d and substituting leaves one constraint on (g_i, g_d)."""
    rng = np.random.default_rng(seed)
    fr = synth.make_frame(rng, 8, 5, 30, 2, 12, 0.06, 0.04, 0.02, dirichlet=True)
    _, g, _ = _grad(fr)
    Pi, Pd = fr.Pi, fr.Pd
    Pt = 1 - Pi - Pd
    tau, rho = fr.tau, fr.rho
    dd = (g[1] * Pt + tau) / (Pt + Pd)
    dt = (tau - Pd * dd) / Pt
    di = (rho - tau + Pd * dd) / Pi
    assert g[0] == pytest.approx(di - dt, rel=1e-9, abs=1e-7)


def test_prior_grad_weighted_sum_is_one():
    fr = synth.config_frame(1, 0)
    pr = fr.priors_or_uniform().astype(np.float64)
    _, _, dpri = _grad(fr)
    np.testing.assert_allclose((pr * dpri).sum(axis=1), 1.0, rtol=1e-12)


@pytest.mark.parametrize("seed", [151, 152])
def test_grad_vs_torch_fp64_autograd(seed):
    fr = synth.tiny_frame(seed, q=4, n=3, N=5, I=2, xmax=5, Pi=0.1, Pd=0.07, Ps=0.04)
    pr = fr.priors.astype(np.float64)
    ll, dchan, dpri = _grad(fr)
    ll_t, dchan_t, dpri_t = torch_reference.grads(fr.codebook, pr, fr.rx, fr.I, fr.xmax,
                                                  fr.Pi, fr.Pd, fr.Ps)
    assert ll == pytest.approx(ll_t, rel=1e-12)
    np.testing.assert_allclose(dchan, dchan_t, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(dpri, dpri_t, rtol=1e-10, atol=1e-12)


def test_grad_memo_matches_plain():
    fr = synth.tiny_frame(161, q=4, n=3, N=6, I=2, xmax=6, Pi=0.1, Pd=0.1, Ps=0.05)
    a = _grad(fr, memo=True)
    b = _grad(fr, memo=False)
    assert a[0] == b[0]
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_channel_grad_vs_oracle_fd_on_gradient_workload_frame():
    """Frame 0 of the 256-frame gradient workload (N = 2000, q = 32, n = 8,
    xmax = 120): the dual-number channel gradient against central differences
    of the oracle's log P (h = 1e-6), and the path-count identity, at full size."""
    fr = synth.config_frame(4, 0)
    pr = fr.priors.astype(np.float64)
    ll, g, _ = oracle.loglik_grad(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                                  priors=pr, want_priors=False)
    h = 1e-6
    noise = 8 * np.finfo(np.float64).eps * abs(ll) / h
    base = [fr.Pi, fr.Pd, fr.Ps]
    for k in range(3):
        up = list(base); up[k] += h
        dn = list(base); dn[k] -= h
        fd = (_ll(fr, *up, priors=pr) - _ll(fr, *dn, priors=pr)) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-6, abs=noise), k
    Pi, Pd = fr.Pi, fr.Pd
    Pt = 1 - Pi - Pd
    dd = (g[1] * Pt + fr.tau) / (Pt + Pd)
    dt = (fr.tau - Pd * dd) / Pt
    di = (fr.rho - fr.tau + Pd * dd) / Pi
    assert g[0] == pytest.approx(di - dt, rel=1e-9, abs=1e-7)
