"""Checkpoint-and-recompute batches (MAPDEC_BATCH_SEGMENTED).

The forward rows are kept only at every K-th symbol; the second sweep
recomputes a segment's transition weights and forward rows from its
checkpoint with the recorded tilts.  These tests check that the segmented
run gives the unsegmented run's results (same kernels, same tilt sequence),
that it matches the FP64 oracle at the two workloads that call for it (the
gradient batch with a checkpoint every 45 symbols, the large-code batch),
the segment-length edge cases (one symbol per segment, a one-symbol last
segment, one segment), and that it bounds the scratch memory.
"""
import os

import numpy as np
import pytest

import oracle
from parity import check_app, check_grad, check_grad_priors, check_ll
from paper_1802_08483_gb300 import mapdec, synth

pytestmark = pytest.mark.gpu

SEG = mapdec.MAPDEC_BATCH_SEGMENTED
GRAPH = mapdec.MAPDEC_BATCH_GRAPH
GRAD = mapdec.MAPDEC_BATCH_GRAD


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_08483_gb300 import build
    build.build()
    mapdec.load()
    oracle.build()


def _decode(frames, flags, monkeypatch=None, K=None):
    if monkeypatch is not None:
        if K is None:
            monkeypatch.delenv("MAPDEC_SEG_K", raising=False)
        else:
            monkeypatch.setenv("MAPDEC_SEG_K", str(K))
    b = mapdec.Batch(frames, flags=flags)
    rx, pr = b.concat_inputs()
    if flags & GRAD:
        st, dchan, dpri, ll = b.loglik_grad(rx, pr)
        out = (st, dchan.copy(), [a.copy() for a in b.split(dpri)], ll.copy())
    else:
        st, app, ll = b.decode(rx, pr)
        out = (st, [a.copy() for a in b.split(app)], ll.copy())
    b.close()
    return out


def _small_mixed(count=24, maxN=600):
    """Frames of the mixed workload (every (q, n) class) short enough for the oracle."""
    out, k = [], 0
    while len(out) < count:
        fr = synth.config_frame(3, k)
        if fr.N <= maxN:
            out.append(fr)
        k += 1
    return out


@pytest.mark.parametrize("K", [7, 45])
def test_segmented_equals_unsegmented_mixed(monkeypatch, K):
    frames = _small_mixed()
    st0, app0, ll0 = _decode(frames, GRAPH)
    st1, app1, ll1 = _decode(frames, GRAPH | SEG, monkeypatch, K)
    assert st0 == 0 and st1 == 0, (st0, st1)
    worst = 0.0
    for k in range(len(frames)):
        assert abs(ll1[k] - ll0[k]) <= 1e-9 * abs(ll0[k]), (k, ll0[k], ll1[k])
        d = np.abs(app1[k] - app0[k]).max()
        worst = max(worst, d)
        assert d <= 1e-6, (k, d)
    print(f"K={K}: worst |APP seg - APP unseg| {worst:.2e}")
    # and the oracle, for the cheapest frames of each class
    for fr, app, ll in list(zip(frames, app1, ll1))[:6]:
        app_ref, ll_ref = oracle.decode(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax,
                                        fr.rx, priors=fr.priors_or_uniform(), kappa=2.0)
        check_app(app, app_ref)
        check_ll(ll, ll_ref)


@pytest.mark.parametrize("K", [1, 2, 39, 40, 1000])
def test_segment_length_edges(monkeypatch, K):
    """K = 1 (a checkpoint at every symbol), N = 40 with K = 39 (last segment
    one symbol long), K = N and K > N (one segment), with gradients."""
    frames = [synth.tiny_frame(seed=11 + s, N=40, q=8, n=6, I=2, Pi=0.03, Pd=0.02, Ps=0.01,
                               xmax=12) for s in range(3)]
    st0, dchan0, dpri0, ll0 = _decode(frames, GRAPH | GRAD)
    st1, dchan1, dpri1, ll1 = _decode(frames, GRAPH | GRAD | SEG, monkeypatch, K)
    assert st0 == 0 and st1 == 0, (st0, st1)
    for k, fr in enumerate(frames):
        assert abs(ll1[k] - ll0[k]) <= 1e-9 * abs(ll0[k]), (k, ll0[k], ll1[k])
        np.testing.assert_allclose(dchan1[k], dchan0[k], rtol=1e-6, atol=1e-9)
        np.testing.assert_allclose(dpri1[k], dpri0[k], rtol=1e-5, atol=1e-7)
        ll_ref, dchan_ref, dpri_ref = oracle.loglik_grad(
            fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
            priors=fr.priors_or_uniform())
        check_ll(ll1[k], ll_ref)
        check_grad(dchan1[k], dchan_ref, what=f"frame {k} channel")
        check_grad_priors(dpri1[k], dpri_ref, fr.priors_or_uniform(), what=f"frame {k} priors")


def test_grad_256_checkpoint_every_45(monkeypatch):
    """The gradient workload as specified: 256 frames N=2000, q=32, n=8, the
    forward rows checkpointed every 45 symbols; frames 0-3 against the FP64
    oracle's dual-number gradient and central finite differences (h=1e-6)."""
    frames = [synth.config_frame(4, f) for f in range(256)]
    st, dchan, dpris, ll = _decode(frames, GRAPH | GRAD | SEG, monkeypatch, 45)
    assert st == 0, mapdec.mapdec_strerror(st)
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
            check_grad([dchan[k, c]], [fd], what=f"frame {k} d/dchan[{c}] vs FD")
        check_grad(dchan[k], dchan_ref, what=f"frame {k} channel")
        check_grad_priors(dpris[k], dpri_ref, pri, what=f"frame {k} priors")


def test_large_64_segmented_against_golden(monkeypatch):
    """The large-code workload with checkpointing (K = ceil(sqrt(8000)) = 90):
    frames 0 and 1 against the committed FP64 oracle references."""
    gold = np.load(os.path.join(os.path.dirname(__file__), "golden", "large64_frames.npz"))
    stride = int(gold["stride"])
    frames = [synth.config_frame(5, f) for f in range(64)]
    st, apps, ll = _decode(frames, GRAPH | SEG, monkeypatch, None)
    assert st == 0, mapdec.mapdec_strerror(st)
    for k in [int(x) for x in gold["frames"]]:
        rel, ab = check_app(apps[k][::stride], gold[f"app{k}"], what=f"frame {k}")
        check_ll(ll[k], float(gold[f"ll{k}"]), what=f"frame {k}")
        print(f"large-64 segmented frame {k}: APP rel {rel:.2e} abs {ab:.2e}")


def test_segmented_bounds_scratch(monkeypatch):
    """At a 4 GiB scratch budget the 64 large frames need one wave when
    segmented (about 40 MB each) and many waves otherwise (about 2.7 GB each,
    so one frame per wave)."""
    monkeypatch.delenv("MAPDEC_SEG_K", raising=False)
    frames = [synth.config_frame(5, f) for f in range(64)]
    bud = 4 << 30
    bs = mapdec.Batch(frames, flags=GRAPH | SEG, mem_budget_bytes=bud)
    assert mapdec.mapdec_batch_num_waves(bs.b) == 1
    bs.close()
    bu = mapdec.Batch(frames[:4], flags=GRAPH, mem_budget_bytes=bud)
    assert mapdec.mapdec_batch_num_waves(bu.b) == 4
    bu.close()
