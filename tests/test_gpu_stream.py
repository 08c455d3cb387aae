"""Stream decoding on the GPU: frames cut from a stream (bits of the
neighbouring frames before and after them) with drift priors on both
boundaries (Sec. II-C: alpha_0 and beta_N are the priors of the frame
boundaries) -- APPs, extrinsic outputs, log P(Y) and gradients of the
batched decoder and of a single-frame handle against the FP64 oracle with the
same boundary priors, including the checkpointed mode and isolated frames in
the same batch."""
import copy

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
    oracle.build()


STREAM_CASES = [  # seed, q, n, N, I, xmax, Pi, Pd, Ps, pre, post, sd
    (801, 16, 10, 80, 2, 40, 0.03, 0.03, 0.005, 6, 7, 3.0),
    (802, 64, 12, 40, 2, 50, 0.05, 0.05, 0.01, 10, 5, 4.0),
    (803, 4, 4, 120, 1, 30, 0.04, 0.02, 0.01, 3, 9, 2.0),
    (804, 32, 8, 200, 2, 60, 0.02, 0.04, 0.005, 15, 15, 6.0),
]


def _frames():
    out = []
    for seed, q, n, N, I, xmax, Pi, Pd, Ps, pre, post, sd in STREAM_CASES:
        out.append(synth.stream_frame(np.random.default_rng(seed), q, n, N, I, xmax, Pi, Pd,
                                      Ps, pre, post, sd))
    out.append(synth.make_frame(np.random.default_rng(899), 16, 10, 50, 2, 20, 0.04, 0.04,
                                0.01, dirichlet=True))  # an isolated frame in the same batch
    return out


def _ref(fr):
    return oracle.decode_ext(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                             priors=fr.priors_or_uniform(), kappa=2.0,
                             drift_start=fr.drift_start, drift_end=fr.drift_end)


@pytest.mark.parametrize("segmented", [False, True])
def test_stream_batch_decode_against_oracle(segmented, monkeypatch):
    frames = _frames()
    flags = mapdec.MAPDEC_BATCH_GRAPH | mapdec.MAPDEC_BATCH_EXTRINSIC
    if segmented:
        flags |= mapdec.MAPDEC_BATCH_SEGMENTED
        monkeypatch.setenv("MAPDEC_SEG_K", "7")
    b = mapdec.Batch(frames, flags=flags)
    rx, pr = b.concat_inputs()
    st, app, ext, ll = b.decode_ext(rx, pr)
    assert st == 0, mapdec.mapdec_strerror(st)
    apps, exts = b.split(app), b.split(ext)
    for k, fr in enumerate(frames):
        app_ref, ext_ref, ll_ref = _ref(fr)
        what = f"frame {k} (q={fr.q}, stream={fr.drift_start is not None})"
        check_app(apps[k], app_ref, what=what)
        check_app(exts[k], ext_ref, what=what + " extrinsic")
        check_ll(ll[k], ll_ref, what=what)
    b.close()


def test_stream_gradients_against_oracle():
    frames = _frames()
    b = mapdec.Batch(frames, flags=mapdec.MAPDEC_BATCH_GRAPH | mapdec.MAPDEC_BATCH_GRAD)
    rx, pr = b.concat_inputs()
    st, dchan, dpri, ll = b.loglik_grad(rx, pr)
    assert st == 0, mapdec.mapdec_strerror(st)
    dpris = b.split(dpri)
    for k, fr in enumerate(frames):
        pri = fr.priors_or_uniform().astype(np.float64)
        ll_ref, dchan_ref, dpri_ref = oracle.loglik_grad(
            fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx, priors=pri,
            kappa=2.0, drift_start=fr.drift_start, drift_end=fr.drift_end)
        check_ll(ll[k], ll_ref, what=f"frame {k}")
        check_grad(dchan[k], dchan_ref, what=f"frame {k} channel")
        check_grad_priors(dpris[k], dpri_ref, pri, what=f"frame {k} priors")
    b.close()


def test_stream_single_handle_priors_set_and_cleared():
    fr = _frames()[0]
    dec = mapdec.Decoder.for_frame(fr)
    dec.set_drift_priors(fr.drift_start, fr.drift_end)
    app, ext, ll = dec.decode_ext(fr.rx, fr.priors)
    app_ref, ext_ref, ll_ref = _ref(fr)
    check_app(app, app_ref)
    check_app(ext, ext_ref)
    check_ll(ll, ll_ref)
    llg, dchan, dpri = dec.loglik_grad(fr.rx, fr.priors)
    check_ll(llg, ll_ref)
    # cleared: the isolated frame's boundaries (the whole received sequence)
    dec.set_drift_priors(None, None)
    iso = copy.copy(fr)
    iso.drift_start = iso.drift_end = None
    app2, ll2 = dec.decode(fr.rx, fr.priors)
    a_iso, _, l_iso = _ref(iso)
    check_app(app2, a_iso)
    check_ll(ll2, l_iso)
    with pytest.raises(mapdec.MapDecError):
        dec.set_drift_priors(np.zeros(2 * fr.xmax + 1, np.float32), None)
    dec.close()


def _per_symbol_stream_frame(seed, q, n, N, I, xmax, p, pre, post, sd):
    """A frame with one codebook per symbol, cut from a stream (both widenings
    at once)."""
    rng = np.random.default_rng(seed)
    fr = synth.per_symbol_frame(rng, q, n, N, I, max(1, xmax - pre - post), p, p, 0.005)
    body = fr.rx
    fr.rx = np.concatenate([rng.integers(0, 2, pre), body,
                            rng.integers(0, 2, post)]).astype(np.uint8)
    tau = n * N
    fr.xmax = xmax
    fr.drift_start = synth._gauss_window(xmax, pre, sd, 0, xmax)
    fr.drift_end = synth._gauss_window(xmax, pre + body.size - tau, sd, -xmax, fr.rx.size - tau)
    return fr


def test_per_symbol_codebooks_with_boundary_priors_against_oracle():
    frames = [_per_symbol_stream_frame(861, 16, 10, 30, 2, 30, 0.03, 4, 6, 2.0),
              _per_symbol_stream_frame(862, 5, 5, 50, 1, 20, 0.04, 3, 2, 1.5),
              _per_symbol_stream_frame(863, 64, 12, 12, 2, 40, 0.05, 7, 5, 3.0)]
    b = mapdec.Batch(frames, flags=mapdec.MAPDEC_BATCH_GRAPH | mapdec.MAPDEC_BATCH_EXTRINSIC)
    rx, pr = b.concat_inputs()
    st, app, ext, ll = b.decode_ext(rx, pr)
    assert st == 0, mapdec.mapdec_strerror(st)
    apps, exts = b.split(app), b.split(ext)
    for k, fr in enumerate(frames):
        app_ref, ext_ref, ll_ref = _ref(fr)
        what = f"per-symbol stream frame {k} (q={fr.q})"
        check_app(apps[k], app_ref, what=what)
        check_app(exts[k], ext_ref, what=what + " extrinsic")
        check_ll(ll[k], ll_ref, what=what)
    b.close()
