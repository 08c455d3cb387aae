"""Pins for the oracle's general constituent encodings and extrinsic outputs.

Per-symbol codebooks: the encoding of Sec. II-A uses one injective map C_i
per symbol, and eq. (gamma) takes the codeword of symbol i from C_i.  The
extrinsic output of symbol i is eq. (L) without the symbol's own prior,
normalised over D: in iterative decoding (Sec. II-A) this is what the inner
decoder hands to the outer decoder, whose own extrinsic information comes
back as the next pass's priors.

(i)   exhaustive enumeration of messages and splits with a codebook per
      symbol: APPs, log P(Y), prior gradients, extrinsic outputs;
(ii)  per-symbol codebooks that are all equal give bitwise the results of the
      one-codebook decoder;
(iii) Pi = Pd = 0 reduces to symbol-wise MAP on a BSC with codebook C_i;
(iv)  the extrinsic output of symbol i does not depend on symbol i's prior,
      is exactly proportional to R(Y | C(D)) for one symbol, and the APP is
      the prior times the extrinsic output, renormalised;
(v)   channel gradients with per-symbol codebooks: brute-force finite
      differences and the path-count identity.
"""
import math

import numpy as np
import pytest

import oracle
from bruteforce import bsc_symbolwise, enumerate_channel, frame_bruteforce
from paper_1802_08483_gb300 import synth


def _frame(seed, q, n, N, I, xmax, Pi, Pd, Ps, same_books=False):
    """Seeded tiny frame with a random codebook per symbol and Dirichlet priors."""
    rng = np.random.default_rng(seed)
    if same_books:
        one = synth.random_codebook(rng, q, n)
        books = np.stack([one] * N)
    else:
        books = np.stack([synth.random_codebook(rng, q, n) for _ in range(N)])
    priors = synth.dirichlet_priors(rng, N, q).astype(np.float64)
    msg = synth.draw_message(rng, priors, N, q)
    x = books[np.arange(N), msg].reshape(-1)
    for _ in range(10000):
        rx = synth.bsid_channel(rng, x, Pi, Pd, Ps, I)
        if abs(rx.size - x.size) <= xmax:
            break
    return books, priors, rx


PER_SYMBOL = [
    # seed, q, n, N, I, xmax, Pi, Pd, Ps
    (301, 4, 3, 3, 1, 9, 0.1, 0.1, 0.05),
    (302, 3, 4, 2, 1, 8, 0.15, 0.1, 0.02),
    (303, 4, 3, 3, 1, 1, 0.1, 0.1, 0.05),   # narrow drift limit: truncation active
    (304, 2, 3, 3, 2, 18, 0.1, 0.1, 0.05),  # I = 2
]


@pytest.mark.parametrize("case", PER_SYMBOL)
def test_per_symbol_codebooks_match_exhaustive_enumeration(case):
    seed, q, n, N, I, xmax, Pi, Pd, Ps = case
    books, pr, rx = _frame(seed, q, n, N, I, xmax, Pi, Pd, Ps)
    assert not all(np.array_equal(books[0], b) for b in books[1:])
    PY, app_ref, dpri_ref = frame_bruteforce(books, pr, rx, I, Pi, Pd, Ps, xmax)
    app, ext, ll = oracle.decode_ext(books, N, Pi, Pd, Ps, I, xmax, rx, priors=pr)
    assert ll == pytest.approx(math.log(PY), rel=1e-12, abs=1e-12)
    np.testing.assert_allclose(app, app_ref, rtol=1e-11, atol=1e-14)
    # d P(Y)/d prior_k(d) sums the other symbols' priors over messages with
    # D_k = d: the extrinsic output, up to its normalisation
    ext_ref = dpri_ref / dpri_ref.sum(axis=1, keepdims=True)
    np.testing.assert_allclose(ext, ext_ref, rtol=1e-11, atol=1e-14)
    ll2, _, dpri = oracle.loglik_grad(books, N, Pi, Pd, Ps, I, xmax, rx, priors=pr,
                                      want_chan=False)
    assert ll2 == pytest.approx(math.log(PY), rel=1e-12, abs=1e-12)
    np.testing.assert_allclose(dpri, dpri_ref, rtol=1e-11, atol=1e-13)


def test_per_symbol_codebooks_differ_from_first_codebook():
    """A per-symbol decode is not the one-codebook decode of C_0 (the codebook
    index i reaches the lattice)."""
    books, pr, rx = _frame(305, 4, 3, 3, 1, 9, 0.1, 0.1, 0.05)
    app, _, ll = oracle.decode_ext(books, 3, 0.1, 0.1, 0.05, 1, 9, rx, priors=pr)
    app0, ll0 = oracle.decode(books[0], 3, 0.1, 0.1, 0.05, 1, 9, rx, priors=pr)
    assert abs(ll - ll0) > 1e-6 or np.max(np.abs(app - app0)) > 1e-6


@pytest.mark.parametrize("memo", [True, False])
def test_equal_per_symbol_codebooks_are_bitwise_the_one_codebook_decoder(memo):
    rng = np.random.default_rng(311)
    fr = synth.make_frame(rng, 8, 5, 20, 2, 10, 0.05, 0.04, 0.02, dirichlet=True)
    pr = fr.priors.astype(np.float64)
    books = np.stack([fr.codebook] * fr.N)
    app1, ll1 = oracle.decode(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                              priors=pr, memo=memo)
    app2, ext2, ll2 = oracle.decode_ext(books, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                                        priors=pr)
    assert ll1 == ll2
    assert np.array_equal(app1, app2)
    g1 = oracle.loglik_grad(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                            priors=pr, memo=memo)
    g2 = oracle.loglik_grad(books, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx, priors=pr)
    assert g1[0] == g2[0]
    assert np.array_equal(g1[1], g2[1]) and np.array_equal(g1[2], g2[2])


@pytest.mark.parametrize("Ps", [0.0, 0.03, 0.2])
def test_per_symbol_no_sync_errors_reduce_to_bsc_map(Ps):
    q, n, N, I, xmax = 8, 6, 12, 2, 5
    books, pr, rx = _frame(int(Ps * 1000) + 321, q, n, N, I, xmax, 0.0, 0.0, Ps)
    assert rx.size == n * N
    app, ext, ll = oracle.decode_ext(books, N, 0.0, 0.0, Ps, I, xmax, rx, priors=pr)
    app_ref, ll_ref = bsc_symbolwise(books, pr, rx, Ps)
    np.testing.assert_allclose(app, app_ref, rtol=1e-11, atol=1e-300)
    assert ll == pytest.approx(ll_ref, rel=1e-12)
    # without synchronisation errors the symbols decouple: the extrinsic output
    # is the BSC likelihood of C_i(D) alone
    ext_ref, _ = bsc_symbolwise(books, np.ones_like(pr), rx, Ps)
    np.testing.assert_allclose(ext, ext_ref, rtol=1e-11, atol=1e-300)


@pytest.mark.parametrize("per_symbol", [False, True])
def test_extrinsic_output_ignores_own_prior(per_symbol):
    q, n, N, I, xmax = 4, 4, 10, 2, 8
    books, pr, rx = _frame(331 + per_symbol, q, n, N, I, xmax, 0.08, 0.06, 0.03,
                           same_books=not per_symbol)
    cb = books if per_symbol else books[0]
    app, ext, _ = oracle.decode_ext(cb, N, 0.08, 0.06, 0.03, I, xmax, rx, priors=pr)
    i = 4
    pr2 = pr.copy()
    pr2[i] = np.array([0.7, 0.1, 0.15, 0.05])
    app2, ext2, _ = oracle.decode_ext(cb, N, 0.08, 0.06, 0.03, I, xmax, rx, priors=pr2)
    np.testing.assert_allclose(ext2[i], ext[i], rtol=1e-12, atol=1e-300)
    assert np.max(np.abs(app2[i] - app[i])) > 1e-3
    # the APP is the prior times the extrinsic output, renormalised over D
    for p, a, e in ((pr, app, ext), (pr2, app2, ext2)):
        un = p * e
        np.testing.assert_allclose(a, un / un.sum(axis=1, keepdims=True), rtol=1e-11,
                                   atol=1e-300)


def test_extrinsic_output_with_zero_prior():
    """A symbol value with prior 0 has APP 0 but a defined extrinsic output."""
    books, pr, rx = _frame(341, 4, 3, 3, 1, 9, 0.1, 0.1, 0.05)
    pr[1] = np.array([0.5, 0.0, 0.5, 0.0])
    PY, app_ref, dpri_ref = frame_bruteforce(books, pr, rx, 1, 0.1, 0.1, 0.05, 9)
    app, ext, ll = oracle.decode_ext(books, 3, 0.1, 0.1, 0.05, 1, 9, rx, priors=pr)
    assert app[1, 1] == 0.0 and app[1, 3] == 0.0
    assert ext[1, 1] > 0.0 and ext[1, 3] > 0.0
    np.testing.assert_allclose(ext, dpri_ref / dpri_ref.sum(axis=1, keepdims=True),
                               rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("seed", [351, 352])
def test_single_symbol_extrinsic_is_channel_likelihood(seed):
    """N = 1: the extrinsic output is R(Y | C(D)) normalised over D, whatever the
    prior; R from the brute-force channel enumeration."""
    q, n, I = 4, 4, 1
    rng = np.random.default_rng(seed)
    cb = synth.random_codebook(rng, q, n)
    rx = synth.bsid_channel(rng, cb[1], 0.1, 0.1, 0.05, I)
    pr = synth.dirichlet_priors(rng, 1, q).astype(np.float64)
    app, ext, ll = oracle.decode_ext(cb, 1, 0.1, 0.1, 0.05, I, n * I, rx, priors=pr)
    y = tuple(int(b) for b in rx)
    R = np.array([enumerate_channel(cb[d], I, 0.1, 0.1, 0.05).get(y, 0.0) for d in range(q)])
    np.testing.assert_allclose(ext[0], R / R.sum(), rtol=1e-12, atol=1e-300)
    assert ll == pytest.approx(math.log(float(pr[0] @ R)), rel=1e-12)


@pytest.mark.parametrize("seed", [361, 362])
def test_per_symbol_channel_grad_vs_bruteforce_fd(seed):
    Pi, Pd, Ps = 0.12, 0.08, 0.06
    books, pr, rx = _frame(seed, 3, 3, 3, 1, 3, Pi, Pd, Ps)
    _, dchan, _ = oracle.loglik_grad(books, 3, Pi, Pd, Ps, 1, 3, rx, priors=pr)
    h = 1e-6
    base = [Pi, Pd, Ps]
    for k in range(3):
        up = list(base); up[k] += h
        dn = list(base); dn[k] -= h
        pu, _, _ = frame_bruteforce(books, pr, rx, 1, *up, 3)
        pd, _, _ = frame_bruteforce(books, pr, rx, 1, *dn, 3)
        fd = (math.log(pu) - math.log(pd)) / (2 * h)
        assert dchan[k] == pytest.approx(fd, rel=1e-6, abs=1e-6), k


def test_per_symbol_path_count_identity():
    """Every path has #ins - #del = rho - tau and #del + #trans = tau whatever the
    codewords, so the identity that ties d/dPi to d/dPd holds unchanged."""
    q, n, N, I, xmax = 8, 5, 24, 2, 12
    Pi, Pd, Ps = 0.06, 0.04, 0.02
    books, pr, rx = _frame(371, q, n, N, I, xmax, Pi, Pd, Ps)
    _, g, _ = oracle.loglik_grad(books, N, Pi, Pd, Ps, I, xmax, rx, priors=pr)
    Pt = 1 - Pi - Pd
    tau, rho = n * N, rx.size
    dd = (g[1] * Pt + tau) / (Pt + Pd)
    dt = (tau - Pd * dd) / Pt
    di = (rho - tau + Pd * dd) / Pi
    assert g[0] == pytest.approx(di - dt, rel=1e-9, abs=1e-7)


def test_per_symbol_codebook_count_is_checked():
    books, pr, rx = _frame(381, 4, 3, 3, 1, 9, 0.1, 0.1, 0.05)
    with pytest.raises(ValueError):
        oracle.decode_ext(books[:2], 3, 0.1, 0.1, 0.05, 1, 9, rx, priors=pr)
    with pytest.raises(ValueError):
        oracle.decode(books, 3, 0.1, 0.1, 0.05, 1, 9, rx, priors=pr)
