"""Inputs and outputs of a batch in pinned host memory.

Pinned host buffers of 1 MiB or more are moved by the SMs through their
device mapping when both sides are 16-byte aligned (the tail under 16 bytes by
the copy engine), and by the copy engine otherwise; pageable buffers always by
the copy engine.
Every route must give the same bits as resident device buffers.
"""
import numpy as np
import pytest

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


def _frames():
    out = []
    # priors and APPs above 1 MiB (the SM route), received bits below it
    for seed, q, n, N, xmax, p in [(951, 16, 10, 37, 12, 0.02), (952, 4, 4, 101, 20, 0.03),
                                   (953, 64, 12, 23, 30, 0.05), (954, 64, 12, 4500, 60, 0.004)]:
        out.append(synth.make_frame(np.random.default_rng(seed), q, n, N, 2, xmax, p, p, 0.004,
                                    dirichlet=True))
    return out


def _pinned(arr, offset):
    """A pinned host copy of arr starting `offset` bytes into a pinned buffer."""
    import torch
    raw = torch.empty(arr.nbytes + 64, dtype=torch.uint8).pin_memory()
    view = raw[offset:offset + arr.nbytes]
    view.copy_(torch.from_numpy(arr.view(np.uint8).reshape(-1)))
    return raw, view


@pytest.mark.parametrize("offset", [0, 4, 16])
def test_pinned_host_buffers_match_device_buffers(offset):
    import torch
    frames = _frames()
    b = mapdec.Batch(frames, flags=mapdec.MAPDEC_BATCH_GRAPH)
    rx, pr = b.concat_inputs()
    st, app_ref, ll_ref = b.decode(rx, pr)  # pageable host buffers
    assert st == 0, mapdec.mapdec_strerror(st)
    rx_raw, rx_h = _pinned(rx, offset)
    pr_raw, pr_h = _pinned(pr, offset)
    app_raw = torch.zeros(app_ref.nbytes + 64, dtype=torch.uint8).pin_memory()
    ll_raw = torch.zeros(ll_ref.nbytes + 64, dtype=torch.uint8).pin_memory()
    app_h = app_raw[offset:offset + app_ref.nbytes]
    ll_h = ll_raw[offset:offset + ll_ref.nbytes]
    st = mapdec.mapdec_batch_decode(b.b, rx_h, pr_h, app_h, ll_h)
    assert st == 0, mapdec.mapdec_strerror(st)
    torch.cuda.synchronize()
    app = app_h.numpy().view(np.float32)
    ll = ll_h.numpy().view(np.float64)
    assert np.array_equal(app, app_ref)
    assert np.array_equal(ll, ll_ref)
    # resident device buffers, then pinned inputs with a pageable output
    rx_d, pr_d, app_d, ll_d = mapdec.mapdec_batch_buffers(b.b)
    assert mapdec.mapdec_batch_decode(b.b, rx_d, pr_d, app_d, ll_d) == 0
    out = np.empty_like(app_ref)
    assert mapdec.mapdec_batch_decode(b.b, rx_h, pr_h, out, ll_h) == 0
    assert np.array_equal(out, app_ref)
    b.close()
