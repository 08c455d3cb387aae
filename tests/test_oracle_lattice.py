"""Pins for the oracle's receiver-metric lattice (Sec. II-C, eqs. F, F_lastrow).

The lattice is checked against (i) exhaustive enumeration of channel event
patterns, (ii) hand-derived closed forms (tests/golden), (iii) the
length-distribution generating function, (iv) the substitution-only limit.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from bruteforce import all_strings, enumerate_channel, length_sum_closed_form

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lattice_handworked.json")

PARAMS = [(0.1, 0.1, 0.05), (0.2, 0.05, 0.0), (0.03, 0.3, 0.2), (0.0, 0.2, 0.1),
          (0.25, 0.0, 0.3)]


def oracle_R(x, y, I, Pi, Pd, Ps):
    return oracle.receiver_metric(np.array(x, np.uint8), np.array(y, np.uint8), I, Pi, Pd, Ps)


@pytest.mark.parametrize("n,I", [(1, 1), (2, 1), (3, 1), (4, 1), (2, 2), (3, 2), (1, 3)])
@pytest.mark.parametrize("params", PARAMS)
def test_lattice_matches_event_enumeration(n, I, params):
    Pi, Pd, Ps = params
    rng = np.random.default_rng(1000 * n + 10 * I)
    for _ in range(2):
        x = tuple(int(b) for b in rng.integers(0, 2, n))
        bf = enumerate_channel(x, I, Pi, Pd, Ps)
        maxlen = n * (I + 1)
        for y in all_strings(maxlen):
            r = oracle_R(x, y, I, Pi, Pd, Ps)
            # out[j] is R of the prefix y[:j]; check the full string and all prefixes
            for j in range(len(y) + 1):
                ref = bf.get(tuple(y[:j]), 0.0)
                assert abs(r[j] - ref) <= 1e-15 * max(1.0, abs(ref)), (x, y, j, r[j], ref)
        # strings longer than n(I+1) are impossible
        for y in itertools.product((0, 1), repeat=maxlen + 1):
            assert oracle_R(x, y, I, Pi, Pd, Ps)[-1] == 0.0
            break


def test_lattice_handworked_golden():
    g = json.load(open(GOLDEN))
    for prm in g["params"]:
        Pi, Pd, Ps = prm["Pi"], prm["Pd"], prm["Ps"]
        env = {"Pi": Pi, "Pd": Pd, "Ps": Ps, "Pt": 1 - Pi - Pd, "w": Pi / 2}
        for case in g["cases"]:
            ref = eval(case["R"], {}, env)
            got = oracle_R(case["x"], case["y"], case["I"], Pi, Pd, Ps)[len(case["y"])]
            assert got == pytest.approx(ref, rel=1e-14, abs=1e-300), case


@pytest.mark.parametrize("n,I", [(5, 2), (4, 3), (7, 1)])
@pytest.mark.parametrize("params", [(0.1, 0.1, 0.05), (0.3, 0.2, 0.4)])
def test_lattice_length_generating_function(n, I, params):
    """sum over all y of length mu of R(y|x) = [z^mu](sum_a (Pi z)^a (Pd + Pt z))^n,
    and the total over mu is (1 - Pi^(I+1))^n, for any x and Ps."""
    Pi, Pd, Ps = params
    rng = np.random.default_rng(7 + n + I)
    x = rng.integers(0, 2, n).astype(np.uint8)
    maxlen = n * (I + 1)
    sums = np.zeros(maxlen + 1)
    # every string of length mu is a prefix-closed family: evaluate each full
    # string once and read only its own length
    for mu in range(maxlen + 1):
        if mu > 18:
            break
        tot = 0.0
        for y in itertools.product((0, 1), repeat=mu):
            tot += oracle_R(x, y, I, Pi, Pd, Ps)[mu]
        sums[mu] = tot
        ref = length_sum_closed_form(n, I, Pi, Pd, mu)
        assert tot == pytest.approx(ref, rel=1e-12, abs=1e-300)
    if maxlen <= 18:
        assert sums.sum() == pytest.approx((1 - Pi ** (I + 1)) ** n, rel=1e-12)


def test_lattice_total_mass_large_cap():
    """With a large insertion cap the receiver metric sums to ~1 over all
    received strings (the cap only removes mass Pi^(I+1) per bit)."""
    Pi, Pd, Ps = 0.1, 0.15, 0.2
    n, I = 1, 12
    x = np.array([1], np.uint8)
    tot = 0.0
    for mu in range(n * (I + 1) + 1):
        for y in itertools.product((0, 1), repeat=mu):
            tot += oracle_R(x, y, I, Pi, Pd, Ps)[mu]
    assert tot == pytest.approx(1.0 - Pi ** (I + 1), rel=1e-12)
    assert abs(tot - 1.0) < 1e-11


@pytest.mark.parametrize("Ps", [0.0, 0.01, 0.3])
def test_lattice_substitution_only(Ps):
    """Pi = Pd = 0: R(y|x) = Ps^dH (1-Ps)^(n-dH) for |y| = n, 0 otherwise."""
    rng = np.random.default_rng(3)
    n, I = 7, 2
    for _ in range(20):
        x = rng.integers(0, 2, n).astype(np.uint8)
        y = rng.integers(0, 2, n * (I + 1)).astype(np.uint8)
        r = oracle_R(x, y, I, 0.0, 0.0, Ps)
        dh = int(np.sum(x != y[:n]))
        for j in range(r.size):
            ref = Ps ** dh * (1 - Ps) ** (n - dh) if j == n else 0.0
            assert r[j] == pytest.approx(ref, rel=1e-14, abs=0.0)
