"""GPU parity at the workloads' full sizes, in the launch configuration the
benchmark times (one batch, CUDA graph), on outputs the oracle can compute
one frame at a time.

  mixed-4096 : all 4096 frames decoded; every frame's status checked; a
               sample of frames across the (q, n) classes compared with the
               oracle element by element, and the costliest frames of every
               class against committed oracle references.
  grad-256   : 256 frames N=2000, q=32, n=8 in gradient mode; frames 0-3
               against central finite differences (h = 1e-6) of the FP64
               oracle and against its dual-number gradient.
  large-64   : 64 frames N=8000, q=64, n=12, I=3; APPs (every 16th symbol)
               and log P of frames 0 and 1 against committed oracle references.
"""
import math
import multiprocessing as mp

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


def _oracle_decode(args):
    # Long frames with wide drift limits underflow the literal FP64 recursion;
    # the oracle's exact received-bit reweighting (kappa = 2) keeps them in range.
    cfg, idx = args
    fr = synth.config_frame(cfg, idx)
    return oracle.decode(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                         priors=fr.priors_or_uniform(), kappa=2.0)


def _pool_decode(items, procs):
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        return pool.map(_oracle_decode, items, chunksize=1)


def _decode_mixed(frames):
    b = mapdec.Batch(frames, flags=mapdec.MAPDEC_BATCH_GRAPH | mapdec.MAPDEC_BATCH_TIMING)
    rx, pr = b.concat_inputs()
    st, app, ll = b.decode(rx, pr)
    assert st == 0, mapdec.mapdec_strerror(st)
    stat = mapdec.mapdec_batch_status(b.b, b.nf)
    assert (stat == 0).all(), np.unique(stat, return_counts=True)
    assert np.all(np.isfinite(ll))
    apps = b.split(app)
    for k, fr in enumerate(frames):
        s = apps[k].sum(axis=1)
        assert np.all(np.abs(s - 1) < 1e-4), k
    b.close()
    return apps, ll


def test_mixed_4096_full_batch():
    """The whole workload in one batch with the planner's launch parameters
    and with the committed tuning table (the benchmark's: tuned tiles and the
    128-thread, 52 KB recursions), both against the FP64 oracle."""
    from paper_1802_08483_gb300 import tune
    frames = [synth.config_frame(3, f) for f in range(4096)]
    runs = [("planner", _decode_mixed(frames))]
    import os
    table = os.path.join(os.path.dirname(__file__), "..", "paper_1802_08483_gb300", "tuning",
                         "gb300_mixed4096.json")
    tune.load(table)
    try:
        runs.append(("tuned", _decode_mixed(frames)))
    finally:
        mapdec.mapdec_tune_clear()
    # sample: per (q, n) class the two cheapest frames for the oracle, plus a few
    # from each end of the batch, so every wave and every class is covered
    cost = {k: fr.N * (2 * fr.xmax + 1) * fr.q * (fr.n * 3 + 1) for k, fr in enumerate(frames)}
    sample = set()
    for qn in synth.QN_CHOICES:
        ks = sorted((k for k, fr in enumerate(frames) if (fr.q, fr.n) == qn), key=cost.get)
        sample.update(ks[:2])
    tail = sorted(range(4000, 4096), key=cost.get)[:2]
    head = sorted(range(0, 96), key=cost.get)[:2]
    sample.update(tail + head)
    sample = sorted(sample)
    refs = _pool_decode([(3, k) for k in sample], 8)
    for name, (apps, ll) in runs:
        worst = 0.0
        for k, (app_ref, ll_ref) in zip(sample, refs):
            rel, ab = check_app(apps[k], app_ref, what=f"{name}: frame {k}")
            check_ll(ll[k], ll_ref, what=f"{name}: frame {k}")
            worst = max(worst, rel)
        print(f"mixed-4096 ({name}): {len(sample)} frames checked, worst APP rel {worst:.2e}")
    # the costliest frames of every (q, n) class (N near 4000, the widest drift
    # limits), which dominate the timed step, against committed FP64 oracle
    # references (tests/golden/make_mixed_golden.py: every 16th symbol's APPs
    # and log P; kappa = 1.5 for two of them)
    gold = np.load(os.path.join(os.path.dirname(__file__), "golden", "mixed4096_heavy.npz"))
    stride = int(gold["stride"])
    assert {(frames[int(k)].q, frames[int(k)].n) for k in gold["frames"]} == set(synth.QN_CHOICES)
    for name, (apps, ll) in runs:
        for k in [int(x) for x in gold["frames"]]:
            rel, ab = check_app(apps[k][::stride], gold[f"app{k}"], what=f"{name}: heavy frame {k}")
            llr = check_ll(ll[k], float(gold[f"ll{k}"]), what=f"{name}: heavy frame {k}")
            fr = frames[k]
            print(f"mixed-4096 ({name}) heavy frame {k} (q={fr.q} n={fr.n} N={fr.N} "
                  f"xmax={fr.xmax}): APP rel {rel:.2e} abs {ab:.2e}, log P rel {llr:.2e}")


def test_grad_256_fd_on_first_frames():
    frames = [synth.config_frame(4, f) for f in range(256)]
    b = mapdec.Batch(frames, flags=mapdec.MAPDEC_BATCH_GRAPH | mapdec.MAPDEC_BATCH_GRAD)
    rx, pr = b.concat_inputs()
    st, dchan, dpri, ll = b.loglik_grad(rx, pr)
    assert st == 0, mapdec.mapdec_strerror(st)
    dpris = b.split(dpri)
    h = 1e-6
    for k in range(4):
        fr = frames[k]
        pri = fr.priors.astype(np.float64)
        ll_ref, dchan_ref, dpri_ref = oracle.loglik_grad(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps,
                                                         fr.I, fr.xmax, fr.rx, priors=pri)
        check_ll(ll[k], ll_ref, what=f"frame {k}")
        base = [fr.Pi, fr.Pd, fr.Ps]
        for c in range(3):
            up = list(base); up[c] += h
            dn = list(base); dn[c] -= h
            lu = oracle.loglik(fr.codebook, fr.N, *up, fr.I, fr.xmax, fr.rx, priors=pri)
            ld = oracle.loglik(fr.codebook, fr.N, *dn, fr.I, fr.xmax, fr.rx, priors=pri)
            fd = (lu - ld) / (2 * h)
            # central-difference rounding noise ~ N eps |log c| / h (a few 1e-6 here)
            check_grad([dchan_ref[c]], [fd], what=f"oracle frame {k} d/dchan[{c}] vs FD")
            check_grad([dchan[k, c]], [fd], what=f"frame {k} d/dchan[{c}] vs FD")
        check_grad(dchan[k], dchan_ref, what=f"frame {k} channel")
        check_grad_priors(dpris[k], dpri_ref, pri, what=f"frame {k} priors")
    b.close()


def test_large_64_two_frames():
    """Frames 0 and 1 against the committed FP64 oracle references
    (tests/golden/large64_frames.npz, written by make_large_golden.py: every
    16th symbol's APPs and log P), decoded inside the full 64-frame batch."""
    import os
    gold = np.load(os.path.join(os.path.dirname(__file__), "golden", "large64_frames.npz"))
    stride = int(gold["stride"])
    frames = [synth.config_frame(5, f) for f in range(64)]
    b = mapdec.Batch(frames, flags=mapdec.MAPDEC_BATCH_GRAPH)
    rx, pr = b.concat_inputs()
    st, app, ll = b.decode(rx, pr)
    assert st == 0, mapdec.mapdec_strerror(st)
    apps = b.split(app)
    for k in [int(x) for x in gold["frames"]]:
        rel, ab = check_app(apps[k][::stride], gold[f"app{k}"], what=f"frame {k}")
        check_ll(ll[k], float(gold[f"ll{k}"]), what=f"frame {k}")
        print(f"large-64 frame {k}: APP rel {rel:.2e} abs {ab:.2e}")
    b.close()
