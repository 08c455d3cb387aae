"""Per-symbol codebooks on the GPU (the constituent encodings C_i of Sec. II-A;
eq. (gamma) takes C_i(D)): APPs, extrinsic outputs, log P(Y) and the
gradients of the batched decoder against the FP64 oracle's general decoder,
frame by frame, element by element, on shapes that reach every lane layout of
the per-symbol producers (q below and above one warp, q not a power of two,
several chunks of start states per symbol) and with one-codebook frames in the
same batch."""
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


PS_CASES = [  # seed, q, n, N, I, xmax, Pi, Pd, Ps
    (401, 2, 4, 60, 2, 12, 0.05, 0.05, 0.01),
    (402, 8, 6, 40, 2, 20, 0.04, 0.03, 0.01),
    (403, 16, 10, 30, 2, 25, 0.05, 0.05, 0.005),
    (404, 64, 12, 12, 2, 40, 0.08, 0.08, 0.01),   # two warps of codewords, 3 chunks of states
    (405, 5, 5, 50, 1, 15, 0.06, 0.04, 0.02),     # q not a power of two
    (406, 48, 8, 20, 3, 30, 0.05, 0.05, 0.01),    # I = 3, q = 48
]


def _frames():
    out = []
    for seed, q, n, N, I, xmax, Pi, Pd, Ps in PS_CASES:
        out.append(synth.per_symbol_frame(np.random.default_rng(seed), q, n, N, I, xmax,
                                          Pi, Pd, Ps))
    # one-codebook frames in the same batch
    rng = np.random.default_rng(499)
    out.append(synth.make_frame(rng, 16, 10, 40, 2, 20, 0.04, 0.04, 0.01, dirichlet=True))
    out.append(synth.make_frame(rng, 64, 12, 30, 2, 30, 0.05, 0.05, 0.01, dirichlet=True))
    return out


def _oracle_ext(fr):
    return oracle.decode_ext(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                             priors=fr.priors_or_uniform())


def test_per_symbol_decode_ext_against_oracle():
    frames = _frames()
    b = mapdec.Batch(frames, flags=mapdec.MAPDEC_BATCH_GRAPH | mapdec.MAPDEC_BATCH_EXTRINSIC)
    rx, pr = b.concat_inputs()
    for rep in range(2):  # the second call replays the captured graph
        st, app, ext, ll = b.decode_ext(rx, pr)
        assert st == 0, mapdec.mapdec_strerror(st)
        apps, exts = b.split(app), b.split(ext)
        for k, fr in enumerate(frames):
            app_ref, ext_ref, ll_ref = _oracle_ext(fr)
            what = f"frame {k} (q={fr.q} n={fr.n} per-symbol={fr.codebook.ndim == 3}) rep {rep}"
            check_app(apps[k], app_ref, what=what)
            check_app(exts[k], ext_ref, what=what + " extrinsic")
            check_ll(ll[k], ll_ref, what=what)
    b.close()


def test_per_symbol_gradients_against_oracle():
    frames = _frames()
    b = mapdec.Batch(frames, flags=mapdec.MAPDEC_BATCH_GRAPH | mapdec.MAPDEC_BATCH_GRAD)
    rx, pr = b.concat_inputs()
    st, dchan, dpri, ll = b.loglik_grad(rx, pr)
    assert st == 0, mapdec.mapdec_strerror(st)
    dpris = b.split(dpri)
    for k, fr in enumerate(frames):
        pri = fr.priors_or_uniform().astype(np.float64)
        ll_ref, dchan_ref, dpri_ref = oracle.loglik_grad(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps,
                                                         fr.I, fr.xmax, fr.rx, priors=pri)
        check_ll(ll[k], ll_ref, what=f"frame {k}")
        check_grad(dchan[k], dchan_ref, what=f"frame {k} channel")
        check_grad_priors(dpris[k], dpri_ref, pri, what=f"frame {k} priors")
    b.close()


def test_equal_per_symbol_codebooks_match_one_codebook():
    """N copies of one codebook through the per-symbol producers give the
    one-codebook decoder's results to FP32 rounding."""
    fr = synth.make_frame(np.random.default_rng(498), 16, 8, 50, 2, 20, 0.04, 0.03, 0.01,
                          dirichlet=True)
    import copy
    fr2 = copy.copy(fr)
    fr2.codebook = np.stack([fr.codebook] * fr.N)
    outs = []
    for f in (fr, fr2):
        b = mapdec.Batch([f], flags=mapdec.MAPDEC_BATCH_GRAPH)
        rx, pr = b.concat_inputs()
        st, app, ll = b.decode(rx, pr)
        assert st == 0
        outs.append((app.copy(), ll.copy()))
        b.close()
    check_app(outs[1][0], outs[0][0])
    check_ll(outs[1][1][0], outs[0][1][0])


def test_per_symbol_unsupported_modes():
    fr = synth.per_symbol_frame(np.random.default_rng(497), 4, 4, 10, 1, 8, 0.05, 0.05, 0.01)
    with pytest.raises(mapdec.MapDecError) as e:
        mapdec.Batch([fr], flags=mapdec.MAPDEC_BATCH_SEGMENTED)
    assert e.value.status == mapdec.MAPDEC_ERR_UNSUPPORTED
