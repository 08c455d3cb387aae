"""Pins for the oracle's frame-boundary priors (stream decoding).

Sec. II-C defines alpha_0 and beta_N as the prior probabilities of the frame
boundaries.  An isolated frame has alpha_0 = [m = 0] and beta_N = [m = rho -
tau].  When the frame is cut from a stream, its boundaries are uncertain: it
starts at received position m0 with probability phi0(m0) (earlier bits belong
to the previous frame) and ends at tau + mN with probability phiN(mN) (later
bits belong to the next frame), so
    P(Y) = sum_{m0, mN} phi0(m0) phiN(mN) P(Y[m0 .. tau + mN) | frame),
and each symbol's APP is the same mixture of the isolated frames' APPs,
weighted by phi0 phiN P(piece).  The pins, each against the brute-force
enumeration of messages and splits (tests/bruteforce.py, independent of the
oracle):
  (i)   log P, APPs and prior gradients with boundary priors equal that
        mixture over the pieces of a received sequence padded with bits of
        the neighbouring frames (drift limits wide enough never to bind);
  (ii)  point-mass boundary priors give the isolated frame's results;
  (iii) the received-bit weight kappa cancels with boundary priors;
  (iv)  channel gradients match central finite differences of the mixture.
"""
import math

import numpy as np
import pytest

import oracle
from bruteforce import frame_bruteforce
from paper_1802_08483_gb300 import synth


def _stream_frame(seed, q=3, n=3, N=3, I=1, Pi=0.1, Pd=0.1, Ps=0.05, pre=2, post=2):
    """Tiny frame received inside a stream: `pre` bits of the previous frame
    before it and `post` bits of the next one after it."""
    rng = np.random.default_rng(seed)
    cb = synth.random_codebook(rng, q, n)
    priors = synth.dirichlet_priors(rng, N, q).astype(np.float64)
    msg = synth.draw_message(rng, priors, N, q)
    x = cb[msg].reshape(-1)
    body = synth.bsid_channel(rng, x, Pi, Pd, Ps, I)
    rx = np.concatenate([rng.integers(0, 2, pre), body, rng.integers(0, 2, post)]).astype(np.uint8)
    return cb, priors, rx


def _mixture(cb, priors, rx, I, Pi, Pd, Ps, xmax, phi0, phiN):
    """P(Y), APPs and d/dprior of the boundary mixture by brute force."""
    N, q = priors.shape
    n = cb.shape[1]
    tau = n * N
    rho = len(rx)
    PY, marg, dpri = 0.0, np.zeros((N, q)), np.zeros((N, q))
    for i0, w0 in enumerate(phi0):
        m0 = i0 - xmax
        if w0 == 0.0 or m0 < 0:
            continue  # a frame cannot start before the received bits
        for iN, wN in enumerate(phiN):
            mN = iN - xmax
            if wN == 0.0 or tau + mN > rho or tau + mN < m0:
                continue
            piece = rx[m0:tau + mN]
            p, app, dp = frame_bruteforce(cb, priors, piece, I, Pi, Pd, Ps, 4 * tau)
            w = w0 * wN * p
            PY += w
            marg += w * app
            dpri += w * dp
    return PY, marg / PY, dpri / PY


def _priors_over(xmax, support, rng):
    phi = np.zeros(2 * xmax + 1)
    for m in support:
        phi[m + xmax] = rng.uniform(0.2, 1.0)
    return phi / phi.sum()


CASES = [  # seed, pre, post, start drift support, end drift support
    (701, 2, 2, (0, 1, 2), (-1, 0, 1, 2, 3, 4)),
    (702, 1, 3, (0, 1), (0, 2, 4)),
    (703, 0, 2, (0,), (-2, -1, 0, 1, 2)),     # known start, uncertain end
    (704, 2, 0, (0, 1, 2), (2,)),             # uncertain start, end at the last bit
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("kappa", [1.0, 2.0])
def test_boundary_priors_match_mixture_of_pieces(case, kappa):
    seed, pre, post, s0, sN = case
    cb, priors, rx = _stream_frame(seed, pre=pre, post=post)
    I, Pi, Pd, Ps = 1, 0.1, 0.1, 0.05
    N, q = priors.shape
    tau = cb.shape[1] * N
    xmax = 12  # wider than any drift a 3-symbol frame plus the padding reaches
    rng = np.random.default_rng(seed + 1)
    phi0 = _priors_over(xmax, s0, rng)
    phiN = _priors_over(xmax, [m for m in sN if 0 <= tau + m <= len(rx)], rng)
    PY, app_bf, dpri_bf = _mixture(cb, priors, rx, I, Pi, Pd, Ps, xmax, phi0, phiN)
    app, ext, ll = oracle.decode_ext(cb, N, Pi, Pd, Ps, I, xmax, rx, priors=priors,
                                     kappa=kappa, drift_start=phi0, drift_end=phiN)
    assert abs(ll - math.log(PY)) <= 1e-12 * abs(math.log(PY)) + 1e-13, (ll, math.log(PY))
    np.testing.assert_allclose(app, app_bf, rtol=1e-10, atol=1e-14)
    ll2, _, dpri = oracle.loglik_grad(cb, N, Pi, Pd, Ps, I, xmax, rx, priors=priors,
                                      kappa=kappa, drift_start=phi0, drift_end=phiN,
                                      want_chan=False)
    assert abs(ll2 - ll) <= 1e-12 * abs(ll)
    np.testing.assert_allclose(dpri, dpri_bf, rtol=1e-10, atol=1e-12)


def test_start_mass_before_the_received_bits_is_dropped():
    """Drift-prior mass at m0 < 0 (a start before the received bits) carries
    no path: the result equals the prior restricted to m0 >= 0 (renormalising
    it only shifts log P by the log of the kept mass)."""
    cb, priors, rx = _stream_frame(705, pre=1, post=1)
    N, q = priors.shape
    xmax = 12
    phi0 = np.zeros(2 * xmax + 1)
    phi0[xmax - 2], phi0[xmax], phi0[xmax + 1] = 0.3, 0.4, 0.3
    kept = phi0.copy()
    kept[:xmax] = 0.0
    phiN = np.zeros(2 * xmax + 1)
    phiN[xmax + 1] = 1.0
    a1, _, l1 = oracle.decode_ext(cb, N, 0.1, 0.1, 0.05, 1, xmax, rx, priors=priors,
                                  drift_start=phi0, drift_end=phiN)
    a2, _, l2 = oracle.decode_ext(cb, N, 0.1, 0.1, 0.05, 1, xmax, rx, priors=priors,
                                  drift_start=kept, drift_end=phiN)
    np.testing.assert_allclose(a1, a2, rtol=1e-12, atol=1e-15)
    assert abs(l1 - l2) <= 1e-12 * abs(l2)


@pytest.mark.parametrize("seed", [711, 712])
def test_point_mass_boundaries_give_the_isolated_frame(seed):
    fr = synth.tiny_frame(seed, q=4, n=4, N=5, I=2, xmax=6, Pi=0.08, Pd=0.06, Ps=0.03)
    M = 2 * fr.xmax + 1
    phi0 = np.zeros(M)
    phi0[fr.xmax] = 1.0
    phiN = np.zeros(M)
    phiN[fr.rho - fr.tau + fr.xmax] = 1.0
    pri = fr.priors.astype(np.float64)
    for kappa in (1.0, 2.0):
        a1, e1, l1 = oracle.decode_ext(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax,
                                       fr.rx, priors=pri, kappa=kappa)
        a2, e2, l2 = oracle.decode_ext(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax,
                                       fr.rx, priors=pri, kappa=kappa, drift_start=phi0,
                                       drift_end=phiN)
        np.testing.assert_allclose(a2, a1, rtol=1e-13, atol=1e-16)
        np.testing.assert_allclose(e2, e1, rtol=1e-13, atol=1e-16)
        assert abs(l2 - l1) <= 1e-13 * abs(l1)
        g1 = oracle.loglik_grad(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                                priors=pri, kappa=kappa)
        g2 = oracle.loglik_grad(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                                priors=pri, kappa=kappa, drift_start=phi0, drift_end=phiN)
        np.testing.assert_allclose(g2[1], g1[1], rtol=1e-12)
        np.testing.assert_allclose(g2[2], g1[2], rtol=1e-12, atol=1e-15)


def test_channel_gradient_with_boundaries_matches_mixture_differences():
    seed, pre, post, s0, sN = CASES[0]
    cb, priors, rx = _stream_frame(seed, pre=pre, post=post)
    I, Pi, Pd, Ps = 1, 0.1, 0.1, 0.05
    N, q = priors.shape
    tau = cb.shape[1] * N
    xmax = 12
    rng = np.random.default_rng(seed + 1)
    phi0 = _priors_over(xmax, s0, rng)
    phiN = _priors_over(xmax, [m for m in sN if 0 <= tau + m <= len(rx)], rng)
    _, dchan, _ = oracle.loglik_grad(cb, N, Pi, Pd, Ps, I, xmax, rx, priors=priors,
                                     drift_start=phi0, drift_end=phiN, want_priors=False)
    h = 1e-6
    base = [Pi, Pd, Ps]
    for k in range(3):
        up, dn = list(base), list(base)
        up[k] += h
        dn[k] -= h
        lu = math.log(_mixture(cb, priors, rx, I, *up, xmax, phi0, phiN)[0])
        ld = math.log(_mixture(cb, priors, rx, I, *dn, xmax, phi0, phiN)[0])
        fd = (lu - ld) / (2 * h)
        assert abs(dchan[k] - fd) <= 1e-6 * max(1.0, abs(fd)), (k, dchan[k], fd)
