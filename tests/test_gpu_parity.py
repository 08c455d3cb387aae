"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Sizes span several producer tiles and a ragged tail; shapes cover every
compiled (n, I) family and the run-time lattice, q not a power of two, tight
and wide drift limits, N = 1 and an empty received sequence.
"""
import os

import numpy as np
import pytest

import oracle
from parity import check_app, check_grad, check_grad_priors, check_ll
from paper_1802_08483_gb300 import mapdec, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_08483_gb300 import build
    build.build()
    mapdec.load()


def _oracle(fr, memo=True):
    return oracle.decode(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                         priors=fr.priors_or_uniform(), memo=memo)


# ---------------------------------------------------------------------------
# step (1): receiver metric, element by element
# ---------------------------------------------------------------------------
RM_CASES = [  # n, I, q, Pi, Pd, Ps
    (10, 2, 16, 0.05, 0.05, 0.01), (4, 2, 2, 0.1, 0.1, 0.0), (3, 1, 8, 0.2, 0.1, 0.05),
    (12, 3, 64, 0.1, 0.1, 0.01), (8, 2, 32, 0.03, 0.03, 0.005), (6, 2, 8, 0.01, 0.3, 0.2),
    (1, 1, 2, 0.3, 0.2, 0.1), (13, 2, 8, 0.05, 0.05, 0.01), (5, 4, 4, 0.2, 0.1, 0.05),
    (12, 1, 3, 0.1, 0.1, 0.1),
]


@pytest.mark.parametrize("case", RM_CASES)
def test_receiver_metric_parity(case):
    n, I, q, Pi, Pd, Ps = case
    rng = np.random.default_rng(1000 + n * 10 + I)
    cb = synth.random_codebook(rng, q, n)
    N = max(1, 240 // n)
    rx = rng.integers(0, 2, n * N + 3).astype(np.uint8)
    dec = mapdec.Decoder(q, n, cb, N, Pi, Pd, Ps, I, xmax=8)
    MN = n * (I + 1) + 1
    R = dec.receiver_metric(rx, MN).astype(np.float64)
    rho = rx.size
    worst = 0.0
    for p in range(rho + 1):
        mu = min(MN - 1, rho - p)
        for d in range(q):
            ref = oracle.receiver_metric(cb[d], rx[p:p + mu], I, Pi, Pd, Ps)
            got = R[p, d, :mu + 1]
            err = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-30)
            worst = max(worst, float(err.max()))
            assert np.all(R[p, d, mu + 1:] == 0.0)
    assert worst <= 3e-5, worst
    dec.close()


# ---------------------------------------------------------------------------
# full decode, small frames of many shapes
# ---------------------------------------------------------------------------
DEC_CASES = [  # seed, q, n, N, I, xmax, Pi, Pd, Ps
    (1, 16, 10, 50, 2, 20, 0.01, 0.01, 0.0),
    (2, 2, 4, 300, 2, 30, 0.05, 0.05, 0.005),
    (3, 3, 2, 200, 1, 25, 0.1, 0.05, 0.05),
    (4, 8, 5, 120, 3, 40, 0.08, 0.08, 0.02),
    (5, 8, 13, 40, 2, 30, 0.05, 0.05, 0.01),       # run-time lattice (n > 12)
    (6, 4, 6, 1, 2, 8, 0.1, 0.1, 0.05),            # N = 1
    (7, 64, 12, 60, 3, 90, 0.1, 0.1, 0.01),
    (8, 32, 8, 150, 2, 50, 0.03, 0.03, 0.005),
    (9, 16, 7, 90, 1, 15, 0.02, 0.06, 0.03),
    (10, 5, 3, 77, 2, 0, 0.0, 0.0, 0.1),           # xmax = 0, substitution only
]


@pytest.mark.parametrize("case", DEC_CASES)
def test_decode_parity(case):
    seed, q, n, N, I, xmax, Pi, Pd, Ps = case
    rng = np.random.default_rng(seed)
    fr = synth.make_frame(rng, q, n, N, I, xmax, Pi, Pd, Ps, dirichlet=(seed % 2 == 0))
    app_ref, ll_ref = _oracle(fr)
    dec = mapdec.Decoder.for_frame(fr)
    app, ll = dec.decode(fr.rx, fr.priors)
    check_app(app, app_ref, what=str(case))
    check_ll(ll, ll_ref, what=str(case))
    np.testing.assert_allclose(app.sum(axis=1), 1.0, rtol=1e-5)
    dec.close()


def test_decode_empty_received_sequence():
    """N = 1, n = 2, every bit deleted: rho = 0."""
    cb = np.array([[0, 1], [1, 1], [0, 0]], np.uint8)
    rx = np.zeros(0, np.uint8)
    pr = np.array([[0.2, 0.5, 0.3]], np.float32)
    app_ref, ll_ref = oracle.decode(cb, 1, 0.1, 0.2, 0.05, 1, 2, rx, priors=pr)
    dec = mapdec.Decoder(3, 2, cb, 1, 0.1, 0.2, 0.05, 1, 2)
    app, ll = dec.decode(rx, pr)
    check_app(app, app_ref)
    check_ll(ll, ll_ref)


def test_decode_c2_full():
    fr = synth.config_frame(2, 0)
    app_ref, ll_ref = _oracle(fr)
    dec = mapdec.Decoder.for_frame(fr)
    app, ll = dec.decode(fr.rx, None)
    rel, ab = check_app(app, app_ref, what="c2")
    check_ll(ll, ll_ref, what="c2")
    print(f"c2: APP rel {rel:.2e} abs {ab:.2e}")


def test_decode_device_pointers():
    import torch
    fr = synth.config_frame(1, 0)
    dec = mapdec.Decoder.for_frame(fr)
    rx = torch.from_numpy(fr.rx).cuda()
    app = torch.zeros((fr.N, fr.q), dtype=torch.float32, device="cuda")
    ll = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert mapdec.mapdec_decode(dec.h, rx, fr.rho, None, app, ll) == 0
    app_h, ll_h = dec.decode(fr.rx, None)
    assert np.array_equal(app.cpu().numpy(), app_h)
    assert float(ll.cpu()[0]) == ll_h


# ---------------------------------------------------------------------------
# batches: heterogeneous frames, forced small tiles, several waves, graph
# ---------------------------------------------------------------------------
def _mixed_frames(k, seed=77, Nmax=160):
    rng = np.random.default_rng(seed)
    out = []
    for f in range(k):
        q, n = synth.QN_CHOICES[f % len(synth.QN_CHOICES)]
        N = int(rng.integers(20, Nmax))
        p = float(np.exp(rng.uniform(np.log(1e-3), np.log(0.1))))
        Ps = float(rng.uniform(0, 0.01))
        xmax = int(np.ceil(6 * np.sqrt(N * n * 2 * p)))
        out.append(synth.make_frame(rng, q, n, N, 2, xmax, p, p, Ps, dirichlet=True))
    return out


@pytest.mark.parametrize("forceP", [0, 4])
def test_batch_heterogeneous_parity(forceP, monkeypatch):
    if forceP:
        monkeypatch.setenv("MAPDEC_FORCE_P", str(forceP))
    frames = _mixed_frames(10)
    b = mapdec.Batch(frames, flags=mapdec.MAPDEC_BATCH_GRAPH)
    rx, pr = b.concat_inputs()
    for rep in range(2):  # second call replays the captured graph
        st, app, ll = b.decode(rx, pr)
        assert st == 0, mapdec.mapdec_strerror(st)
        apps = b.split(app)
        for k, fr in enumerate(frames):
            app_ref, ll_ref = _oracle(fr)
            check_app(apps[k], app_ref, what=f"frame {k} rep {rep}")
            check_ll(ll[k], ll_ref, what=f"frame {k} rep {rep}")
    b.close()


def test_batch_many_supertiles_per_symbol(monkeypatch):
    """Tiny tiles (P = 1, one sub-tile per super-tile): every symbol's APP sums
    come from more than 32 partial rows."""
    monkeypatch.setenv("MAPDEC_FORCE_P", "1")
    monkeypatch.setenv("MAPDEC_FORCE_NSUB", "1")
    rng = np.random.default_rng(91)
    frames = [synth.make_frame(rng, 8, 6, 60, 2, 40, 0.05, 0.05, 0.01, dirichlet=True),
              synth.make_frame(rng, 4, 4, 90, 2, 36, 0.08, 0.06, 0.01, dirichlet=True)]
    b = mapdec.Batch(frames, flags=mapdec.MAPDEC_BATCH_GRAD)
    rx, pr = b.concat_inputs()
    st, app, ll = b.decode(rx, pr)
    assert st == 0, mapdec.mapdec_strerror(st)
    st, dchan, dpri, ll2 = b.loglik_grad(rx, pr)
    assert st == 0
    for k, (fr, a) in enumerate(zip(frames, b.split(app))):
        app_ref, ll_ref = _oracle(fr)
        check_app(a, app_ref, what=f"frame {k}")
        check_ll(ll[k], ll_ref)
        _, g_ref, _ = oracle.loglik_grad(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax,
                                         fr.rx, priors=fr.priors, want_priors=False)
        check_grad(dchan[k], g_ref, what=f"frame {k}")
    b.close()


def test_batch_waves_match_single_wave():
    frames = _mixed_frames(8, seed=78)
    b1 = mapdec.Batch(frames, flags=0)
    rx, pr = b1.concat_inputs()
    st, app1, ll1 = b1.decode(rx, pr)
    assert st == 0
    b2 = mapdec.Batch(frames, flags=mapdec.MAPDEC_BATCH_GRAPH, mem_budget_bytes=1 << 20)
    st, app2, ll2 = b2.decode(rx, pr)
    assert st == 0
    assert np.array_equal(app1, app2) and np.array_equal(ll1, ll2)
    b1.close()
    b2.close()


def test_batch_resident_buffers_run():
    frames = _mixed_frames(4, seed=79)
    b = mapdec.Batch(frames, flags=mapdec.MAPDEC_BATCH_GRAPH)
    rx, pr = b.concat_inputs()
    st, app_ref, ll_ref = b.decode(rx, pr)
    assert st == 0
    ptrs = mapdec.mapdec_batch_buffers(b.b)
    assert all(p for p in ptrs)
    assert mapdec.mapdec_batch_rx_offset(b.b, 1) >= frames[0].rho
    assert mapdec.mapdec_batch_rx_offset(b.b, len(frames)) == -1
    # rerun on the resident inputs, then read the outputs through a decode call
    assert mapdec.mapdec_batch_run(b.b) == 0
    assert mapdec.mapdec_batch_sync(b.b) == 0
    assert (mapdec.mapdec_batch_status(b.b, len(frames)) == 0).all()
    assert mapdec.mapdec_batch_last_launches(b.b) > 0
    st, app2, ll2 = b.decode(rx, pr)
    assert st == 0 and np.array_equal(app2, app_ref) and np.array_equal(ll2, ll_ref)
    b.close()


# ---------------------------------------------------------------------------
# gradients
# ---------------------------------------------------------------------------
GRAD_CASES = [  # seed, q, n, N, I, xmax, Pi, Pd, Ps
    (21, 8, 6, 40, 2, 14, 0.04, 0.03, 0.01),
    (22, 4, 4, 60, 1, 16, 0.08, 0.05, 0.02),
    (23, 16, 10, 30, 2, 20, 0.05, 0.05, 0.005),
    (24, 32, 8, 50, 2, 24, 0.03, 0.03, 0.005),
    (25, 8, 12, 20, 3, 30, 0.1, 0.1, 0.01),
]


@pytest.mark.parametrize("case", GRAD_CASES)
def test_grad_parity(case):
    seed, q, n, N, I, xmax, Pi, Pd, Ps = case
    rng = np.random.default_rng(seed)
    fr = synth.make_frame(rng, q, n, N, I, xmax, Pi, Pd, Ps, dirichlet=True)
    ll_ref, dchan_ref, dpri_ref = oracle.loglik_grad(fr.codebook, fr.N, Pi, Pd, Ps, I, xmax,
                                                     fr.rx, priors=fr.priors)
    dec = mapdec.Decoder.for_frame(fr)
    ll, dchan, dpri = dec.loglik_grad(fr.rx, fr.priors)
    check_ll(ll, ll_ref, what=str(case))
    check_grad(dchan, dchan_ref, what=f"{case} channel")
    check_grad_priors(dpri, dpri_ref, fr.priors, what=f"{case} priors")
    dec.close()


# ---------------------------------------------------------------------------
# statuses
# ---------------------------------------------------------------------------
def test_error_statuses():
    fr = synth.config_frame(1, 0)
    dec = mapdec.Decoder.for_frame(fr)
    with pytest.raises(mapdec.MapDecError) as e:
        dec.decode(fr.rx[: fr.tau - fr.xmax - 1])
    assert e.value.status == mapdec.MAPDEC_ERR_DRIFT_RANGE
    cb = fr.codebook.copy()
    cb[1] = cb[0]
    with pytest.raises(mapdec.MapDecError) as e:
        mapdec.Decoder(fr.q, fr.n, cb, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax)
    assert e.value.status == mapdec.MAPDEC_ERR_ARG
    with pytest.raises(mapdec.MapDecError) as e:
        mapdec.Decoder(2, 1, np.array([[0], [1]], np.uint8), 3, 0.6, 0.5, 0.0, 1, 2)
    assert e.value.status == mapdec.MAPDEC_ERR_ARG
    with pytest.raises(mapdec.MapDecError) as e:
        mapdec.Decoder(5, 2, np.zeros((5, 2), np.uint8), 3, 0.1, 0.1, 0.0, 1, 2)
    assert e.value.status == mapdec.MAPDEC_ERR_ARG
    # no channel path: no synchronisation errors, no substitutions, rx matches no codeword
    cb = np.array([[0, 0, 0], [1, 1, 1]], np.uint8)
    d2 = mapdec.Decoder(2, 3, cb, 2, 0.0, 0.0, 0.0, 1, 2)
    with pytest.raises(mapdec.MapDecError) as e:
        d2.decode(np.array([0, 1, 0, 0, 0, 0], np.uint8))
    assert e.value.status == mapdec.MAPDEC_ERR_ZERO_PROB
    # the handle stays usable after an error
    app, ll = d2.decode(np.array([0, 0, 0, 1, 1, 1], np.uint8))
    assert app[0, 0] == pytest.approx(1.0) and app[1, 1] == pytest.approx(1.0)


def test_fp32_fma_peak_probe():
    """The FMA probe reports a throughput between half and 105% of the
    SM-count x 128 lanes x 2 x maximum-clock figure."""
    import torch
    v = mapdec.mapdec_fp32_fma_peak()
    props = torch.cuda.get_device_properties(0)
    nominal = props.multi_processor_count * 128 * 2 * 2.07e9 / 1e12
    assert 0.5 * nominal <= v <= 1.05 * nominal, (v, nominal)


def test_recursion_wait_timeout_reports_status(monkeypatch):
    """A recursion whose first copy is never issued (test hook) gives up after
    its bounded wait and reports MAPDEC_ERR_TIMEOUT; the device stays usable and
    the next decode is correct."""
    fr = synth.config_frame(1, 0)
    monkeypatch.setenv("MAPDEC_TEST_STALL_CHAIN", "1")
    dec = mapdec.Decoder.for_frame(fr)
    with pytest.raises(mapdec.MapDecError) as e:
        dec.decode(fr.rx, fr.priors_or_uniform())
    assert e.value.status == mapdec.MAPDEC_ERR_TIMEOUT
    dec.close()
    b = mapdec.Batch([fr, synth.config_frame(3, 1)], flags=mapdec.MAPDEC_BATCH_GRAPH)
    rx, pr = b.concat_inputs()
    st, _, _ = b.decode(rx, pr)
    assert st == mapdec.MAPDEC_ERR_TIMEOUT
    b.close()
    monkeypatch.delenv("MAPDEC_TEST_STALL_CHAIN")
    dec = mapdec.Decoder.for_frame(fr)
    app, ll = dec.decode(fr.rx, fr.priors_or_uniform())
    dec.close()
    app_ref, ll_ref = oracle.decode(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                                    priors=fr.priors_or_uniform())
    check_app(app, app_ref)
    check_ll(ll, ll_ref)


def test_nan_priors_rejected_by_the_recursion():
    """Host-injected fault: NaN priors poison the transition sums; the forward
    recursion's normaliser check reports MAPDEC_ERR_ZERO_PROB instead of
    returning NaNs, and the handle decodes valid priors afterwards."""
    fr = synth.config_frame(1, 0)
    dec = mapdec.Decoder.for_frame(fr)
    pri = fr.priors_or_uniform().astype(np.float32).copy()
    pri[fr.N // 2, :] = np.nan
    with pytest.raises(mapdec.MapDecError) as e:
        dec.decode(fr.rx, pri)
    assert e.value.status == mapdec.MAPDEC_ERR_ZERO_PROB
    app, ll = dec.decode(fr.rx, fr.priors_or_uniform())
    assert np.isfinite(ll) and np.all(np.isfinite(app))
    dec.close()
