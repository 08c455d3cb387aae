"""Allocation-free decode checked against the allocating entry point.

Some callers cannot allocate device memory once they are running -- a receive
pipeline whose memory is fixed at start-up, a host framework that owns every
device allocation, real-time code that must not risk a cudaMalloc blocking or
failing mid-stream.  mapdec_decode_noalloc serves them from a static device
array.  These tests call it through the C ABI and compare its APPs and
log-likelihood with mapdec_decode's, within the parity tolerances used
everywhere else, on calls in a row with different frames (the shared array
keeps the previous call's contents).
"""
import numpy as np
import pytest

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


def _noalloc(fr, priors):
    import torch
    rx = torch.from_numpy(np.ascontiguousarray(fr.rx)).cuda()
    pr = None if priors is None else torch.from_numpy(np.ascontiguousarray(priors)).cuda()
    app = torch.full((fr.N, fr.q), float("nan"), dtype=torch.float32, device="cuda")
    ll = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    st = mapdec.mapdec_decode_noalloc(fr, rx, pr, app, ll)
    return st, app.cpu().numpy(), float(ll.cpu()[0])


def _frames():
    a = synth.config_frame(1, 0)  # uniform priors
    rng = np.random.default_rng(4242)
    b = synth.make_frame(rng, 32, 8, 300, 2, 40, 0.03, 0.03, 0.005, dirichlet=True)
    return a, b


def test_noalloc_matches_decode_on_consecutive_calls():
    a, b = _frames()
    for fr, pri in [(a, None), (b, b.priors), (a, None)]:
        dec = mapdec.Decoder.for_frame(fr)
        app_ref, ll_ref = dec.decode(fr.rx, pri)
        dec.close()
        st, app, ll = _noalloc(fr, pri)
        assert st == mapdec.MAPDEC_OK, mapdec.mapdec_strerror(st)
        check_app(app, app_ref, what=fr.tag)
        check_ll(ll, ll_ref, what=fr.tag)


def test_noalloc_rejects_frame_larger_than_arena():
    fr = synth.config_frame(2, 0)  # N=1000, 401 drift states: transition sums alone ~50 MB
    st, _, _ = _noalloc(fr, None)
    assert st == mapdec.MAPDEC_ERR_TOO_LARGE
    assert "static arena" in mapdec.mapdec_strerror(st)
