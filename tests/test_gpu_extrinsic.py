"""GPU parity of the extrinsic outputs (eq. L without each symbol's own prior,
the quantity iterative decoding with an outer code exchanges, Sec. II-A)
against the FP64 oracle, through the C ABI: one frame, a heterogeneous graph
batch, a checkpointed batch, a zero prior, and the flag check."""
import numpy as np
import pytest

import oracle
from parity import check_app, check_ll
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


def _oracle_ext(fr, priors=None):
    pr = fr.priors_or_uniform() if priors is None else priors
    return oracle.decode_ext(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                             priors=pr, kappa=2.0)


CASES = [  # seed, q, n, N, I, xmax, Pi, Pd, Ps
    (1, 16, 10, 120, 2, 20, 0.02, 0.02, 0.005),
    (2, 8, 6, 200, 2, 30, 0.05, 0.04, 0.01),
    (3, 32, 8, 90, 2, 25, 0.03, 0.03, 0.005),
    (4, 4, 3, 150, 1, 12, 0.08, 0.06, 0.03),
]


@pytest.mark.parametrize("case", CASES)
def test_single_frame_extrinsic(case):
    seed, q, n, N, I, xmax, Pi, Pd, Ps = case
    rng = np.random.default_rng(seed + 700)
    fr = synth.make_frame(rng, q, n, N, I, xmax, Pi, Pd, Ps, dirichlet=True)
    app_ref, ext_ref, ll_ref = _oracle_ext(fr)
    dec = mapdec.Decoder.for_frame(fr)
    app, ext, ll = dec.decode_ext(fr.rx, fr.priors)
    check_app(app, app_ref, what=f"{case} app")
    check_app(ext, ext_ref, what=f"{case} ext")
    check_ll(ll, ll_ref, what=str(case))
    np.testing.assert_allclose(ext.sum(axis=1), 1.0, rtol=1e-5)
    # the plain decode of the same handle is unchanged by the extra output
    app2, ll2 = dec.decode(fr.rx, fr.priors)
    check_app(app2, app_ref, what=f"{case} plain")
    dec.close()


def _mixed(k, seed):
    rng = np.random.default_rng(seed)
    out = []
    for f in range(k):
        q, n = synth.QN_CHOICES[f % len(synth.QN_CHOICES)]
        N = int(rng.integers(20, 160))
        p = float(np.exp(rng.uniform(np.log(1e-3), np.log(0.1))))
        xmax = int(np.ceil(6 * np.sqrt(N * n * 2 * p)))
        out.append(synth.make_frame(rng, q, n, N, 2, xmax, p, p, float(rng.uniform(0, 0.01)),
                                    dirichlet=True))
    return out


@pytest.mark.parametrize("segmented", [False, True])
def test_batch_extrinsic(segmented, monkeypatch):
    flags = mapdec.MAPDEC_BATCH_GRAPH | mapdec.MAPDEC_BATCH_EXTRINSIC
    if segmented:
        monkeypatch.setenv("MAPDEC_SEG_K", "13")
        flags |= mapdec.MAPDEC_BATCH_SEGMENTED
    frames = _mixed(10, 881 + segmented)
    b = mapdec.Batch(frames, flags=flags)
    rx, pr = b.concat_inputs()
    for rep in range(2):  # the second call replays the captured graph
        st, app, ext, ll = b.decode_ext(rx, pr)
        assert st == 0, mapdec.mapdec_strerror(st)
        apps, exts = b.split(app), b.split(ext)
        for k, fr in enumerate(frames):
            app_ref, ext_ref, ll_ref = _oracle_ext(fr)
            check_app(apps[k], app_ref, what=f"frame {k} rep {rep} app")
            check_app(exts[k], ext_ref, what=f"frame {k} rep {rep} ext")
            check_ll(ll[k], ll_ref, what=f"frame {k} rep {rep}")
    b.close()


def test_extrinsic_with_zero_prior():
    rng = np.random.default_rng(891)
    fr = synth.make_frame(rng, 8, 6, 60, 2, 15, 0.04, 0.04, 0.01, dirichlet=True)
    pr = fr.priors.astype(np.float32).copy()
    pr[7] = 0.0
    pr[7, fr.message[7]] = 1.0  # a symbol known to the outer code
    app_ref, ext_ref, ll_ref = _oracle_ext(fr, priors=pr.astype(np.float64))
    dec = mapdec.Decoder.for_frame(fr)
    app, ext, ll = dec.decode_ext(fr.rx, pr)
    assert np.count_nonzero(app[7]) == 1
    assert np.count_nonzero(ext[7]) > 1
    check_app(ext, ext_ref, what="ext")
    check_app(app, app_ref, what="app")
    check_ll(ll, ll_ref)
    dec.close()


def test_extrinsic_needs_the_flag():
    frames = _mixed(2, 893)
    b = mapdec.Batch(frames, flags=mapdec.MAPDEC_BATCH_GRAPH)
    rx, pr = b.concat_inputs()
    st, _, _, _ = b.decode_ext(rx, pr)
    assert st == mapdec.MAPDEC_ERR_ARG
    b.close()
