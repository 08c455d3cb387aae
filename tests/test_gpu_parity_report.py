"""Parity of every synthetic configuration against the FP64 oracle, in the
launch shape the configuration calls for, with the errors printed as one
`PARITY {...}` line per configuration (run with -s to see them):

  config 1, 2 : one frame, plain decode call, every APP and log P;
  config 3    : the 4096-frame batch (one graph), 12 frames across the classes;
  config 4    : 256 frames, checkpoint every 45 symbols, log P and gradients
                of frames 0-3 (dual-number oracle gradient);
  config 5    : 64 frames, checkpointed, frames 0 and 1 against the stored
                oracle references (every 16th symbol).

The single-frame oracle timings (one host thread) are printed beside them.
"""
import json
import os
import time

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


def _report(cfg, **kw):
    print("PARITY " + json.dumps(dict({"config": cfg}, **kw)), flush=True)


def _oracle(fr, kappa=2.0):
    t = time.time()
    app, ll = oracle.decode(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                            priors=fr.priors_or_uniform(), kappa=kappa)
    return app, ll, time.time() - t


@pytest.mark.parametrize("cfg", [1, 2])
def test_single_frame_configs(cfg):
    fr = synth.config_frame(cfg, 0)
    dec = mapdec.Decoder.for_frame(fr)
    app, ll = dec.decode(fr.rx, fr.priors_or_uniform())
    dec.close()
    app_ref, ll_ref, secs = _oracle(fr)
    rel, ab = check_app(app, app_ref)
    lr = check_ll(ll, ll_ref)
    _report(cfg, frames=1, max_app_rel=rel, max_app_abs=ab, logp_rel=lr,
            oracle_bits_per_s_1thread=fr.info_bits / secs)


def test_mixed_batch_sample():
    frames = [synth.config_frame(3, f) for f in range(4096)]
    b = mapdec.Batch(frames, flags=mapdec.MAPDEC_BATCH_GRAPH)
    rx, pr = b.concat_inputs()
    st, app, ll = b.decode(rx, pr)
    assert st == 0
    apps = b.split(app)
    b.close()
    # two cheapest frames of each (q, n) class, plus the cheapest of the last 96
    cost = {k: fr.N * (2 * fr.xmax + 1) * fr.q for k, fr in enumerate(frames)}
    pick = []
    for qn in synth.QN_CHOICES:
        ks = sorted((k for k, fr in enumerate(frames) if (fr.q, fr.n) == qn), key=cost.get)
        pick += ks[:2]
    pick += sorted(range(4000, 4096), key=cost.get)[:2]
    worst_rel = worst_ab = worst_ll = 0.0
    secs = bits = 0.0
    for k in pick:
        app_ref, ll_ref, s = _oracle(frames[k])
        rel, ab = check_app(apps[k], app_ref, what=f"frame {k}")
        lr = check_ll(ll[k], ll_ref, what=f"frame {k}")
        worst_rel, worst_ab, worst_ll = max(worst_rel, rel), max(worst_ab, ab), max(worst_ll, lr)
        secs += s
        bits += frames[k].info_bits
    _report(3, frames=len(pick), max_app_rel=worst_rel, max_app_abs=worst_ab, logp_rel=worst_ll,
            oracle_bits_per_s_1thread=bits / secs)


def test_gradient_config_checkpointed(monkeypatch):
    monkeypatch.setenv("MAPDEC_SEG_K", "45")
    frames = [synth.config_frame(4, f) for f in range(256)]
    b = mapdec.Batch(frames, flags=mapdec.MAPDEC_BATCH_GRAPH | mapdec.MAPDEC_BATCH_GRAD |
                     mapdec.MAPDEC_BATCH_SEGMENTED)
    rx, pr = b.concat_inputs()
    st, dchan, dpri, ll = b.loglik_grad(rx, pr)
    assert st == 0
    dpris = b.split(dpri)
    b.close()
    worst_ll = worst_dchan = worst_dpri = 0.0
    secs = 0.0
    for k in range(4):
        fr = frames[k]
        t = time.time()
        ll_ref, dchan_ref, dpri_ref = oracle.loglik_grad(
            fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
            priors=fr.priors.astype(np.float64))
        secs += time.time() - t
        worst_ll = max(worst_ll, check_ll(ll[k], ll_ref))
        worst_dchan = max(worst_dchan, check_grad(dchan[k], dchan_ref, what=f"frame {k}"))
        worst_dpri = max(worst_dpri, check_grad_priors(dpris[k], dpri_ref, fr.priors,
                                                       what=f"frame {k}"))
    _report(4, frames=4, logp_rel=worst_ll, dchan_rel=worst_dchan, dpriors_rel=worst_dpri,
            oracle_grad_bits_per_s_1thread=4 * frames[0].info_bits / secs)


def test_large_code_checkpointed():
    gold = np.load(os.path.join(os.path.dirname(__file__), "golden", "large64_frames.npz"))
    stride = int(gold["stride"])
    frames = [synth.config_frame(5, f) for f in range(64)]
    b = mapdec.Batch(frames, flags=mapdec.MAPDEC_BATCH_GRAPH | mapdec.MAPDEC_BATCH_SEGMENTED)
    rx, pr = b.concat_inputs()
    st, app, ll = b.decode(rx, pr)
    assert st == 0
    apps = b.split(app)
    b.close()
    worst_rel = worst_ab = worst_ll = 0.0
    for k in [int(x) for x in gold["frames"]]:
        rel, ab = check_app(apps[k][::stride], gold[f"app{k}"])
        lr = check_ll(ll[k], float(gold[f"ll{k}"]))
        worst_rel, worst_ab, worst_ll = max(worst_rel, rel), max(worst_ab, ab), max(worst_ll, lr)
    _report(5, frames=len(gold["frames"]), max_app_rel=worst_rel, max_app_abs=worst_ab,
            logp_rel=worst_ll, note="every 16th symbol against the stored oracle references")
