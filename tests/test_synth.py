"""Host-side checks of the seeded input generator (no decoder arithmetic)."""
import math

import numpy as np

from paper_1802_08483_gb300 import synth


def test_seeded_frames_are_reproducible():
    a = synth.config_frame(3, 17)
    b = synth.config_frame(3, 17)
    assert np.array_equal(a.rx, b.rx) and np.array_equal(a.codebook, b.codebook)
    assert np.array_equal(a.priors, b.priors)


def test_codebooks_distinct_and_shapes():
    for f in range(20):
        fr = synth.config_frame(3, f)
        words = {tuple(r) for r in fr.codebook}
        assert len(words) == fr.q
        assert (fr.q, fr.n) in synth.QN_CHOICES
        assert 100 <= fr.N <= 4000
        assert fr.xmax == math.ceil(6 * math.sqrt(fr.N * fr.n * (fr.Pi + fr.Pd)))
        assert abs(fr.rho - fr.tau) <= fr.xmax
        np.testing.assert_allclose(fr.priors.sum(axis=1), 1.0, rtol=1e-5)


def test_channel_event_rates():
    """Insertion count per bit is a geometric run capped at I; deletions and
    flips occur at Pd/(Pd+Pt) and Ps (Sec. II-B, with the insertion cap)."""
    rng = np.random.default_rng(5)
    tau, Pi, Pd, Ps, I = 400000, 0.1, 0.05, 0.02, 2
    x = np.zeros(tau, np.uint8)
    y = synth.bsid_channel(rng, x, Pi, Pd, Ps, I)
    # expected output length per input bit: E[ins] + P(keep)
    e_ins = sum(Pi ** k for k in range(1, I + 1))
    p_keep = (1 - Pi - Pd) / (1 - Pi)
    assert abs(y.size / tau - (e_ins + p_keep)) < 5e-3
    # ones come only from inserted bits (value 1 w.p. 1/2) and flips
    ones = y.sum() / tau
    assert abs(ones - (0.5 * e_ins + p_keep * Ps)) < 5e-3


def test_config_shapes():
    fr = synth.config_frame(1, 0)
    assert (fr.q, fr.n, fr.N, fr.I, fr.xmax) == (16, 10, 50, 2, 20)
    fr = synth.config_frame(2, 0)
    assert (fr.q, fr.n, fr.N, fr.xmax) == (16, 10, 1000, 200)
    fr = synth.config_frame(4, 1)
    assert (fr.q, fr.n, fr.N, fr.xmax) == (32, 8, 2000, 120)
    assert np.array_equal(fr.codebook, synth.config_frame(4, 2).codebook)
