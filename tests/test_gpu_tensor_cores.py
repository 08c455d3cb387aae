"""Tensor-core producers (tcgen05, split bf16 operands, FP32 accumulation)
against the FP64 oracle, on shapes that reach every branch of their tiling:
one or two 128-row MMA tiles, one or two tensor-memory accumulators (more or
fewer than 128 symbols per tile), q = 16, 32, 48 and 64, insertion caps 1-3,
positions past the end of the received bits, and frames the planner keeps on
the CUDA-core producers (more than 256 symbols per tile) in the same batch.
Also: the same batch with MAPDEC_TC=0 (CUDA-core producers only) agrees with
the default to within the FP32 tolerance."""
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
    oracle.build()


# seed, q, n, N, I, xmax, Pi, Pd, Ps: what the shape exercises
TC_CASES = [
    (301, 16, 4, 300, 2, 300, 0.05, 0.05, 0.01),   # > 128 symbols per tile: one accumulator
    (302, 16, 10, 200, 2, 60, 0.04, 0.04, 0.005),  # two M tiles, two accumulators
    (303, 32, 8, 250, 2, 80, 0.03, 0.03, 0.005),
    (304, 64, 12, 120, 2, 90, 0.08, 0.08, 0.01),   # the mixed workload's costliest class
    (305, 64, 12, 60, 3, 70, 0.1, 0.1, 0.01),      # I = 3 (MN = 49)
    (306, 48, 6, 150, 1, 40, 0.05, 0.03, 0.01),    # q = 48, I = 1
    (307, 32, 5, 400, 1, 20, 0.01, 0.01, 0.0),     # few symbols per tile (N = 16)
    (308, 16, 4, 320, 2, 600, 0.1, 0.1, 0.01),     # > 256 symbols per tile: CUDA cores
    (309, 16, 4, 40, 2, 600, 0.1, 0.1, 0.01),      # limits wider than the frame (40 symbols)
]


def _frames():
    out = []
    for seed, q, n, N, I, xmax, Pi, Pd, Ps in TC_CASES:
        rng = np.random.default_rng(seed)
        out.append(synth.make_frame(rng, q, n, N, I, xmax, Pi, Pd, Ps, dirichlet=True))
    return out


def _decode(frames, monkeypatch=None, tc="1", tc_bwd=None):
    if monkeypatch is not None and tc is not None:
        monkeypatch.setenv("MAPDEC_TC", tc)
    if monkeypatch is not None and tc_bwd is not None:
        monkeypatch.setenv("MAPDEC_TC_BWD", tc_bwd)
    b = mapdec.Batch(frames, flags=mapdec.MAPDEC_BATCH_GRAPH)
    ntc = mapdec.mapdec_batch_tc_frames(b.b)
    rx, pr = b.concat_inputs()
    st, app, ll = b.decode(rx, pr)
    assert st == 0, mapdec.mapdec_strerror(st)
    apps = [a.copy() for a in b.split(app)]
    b.close()
    return ntc, apps, ll


@pytest.mark.parametrize("tc_bwd", ["0", "1"])
def test_tensor_core_batch_against_oracle(monkeypatch, tc_bwd):
    """tc_bwd = 0: tensor cores in the forward producer only; 1: both producers."""
    frames = _frames()
    ntc, apps, ll = _decode(frames, monkeypatch, "1", tc_bwd)
    assert ntc == len(frames) - 1, ntc  # all but case 308 (> 256 symbols per tile)
    for k, fr in enumerate(frames):
        app_ref, ll_ref = oracle.decode(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax,
                                        fr.rx, priors=fr.priors, kappa=2.0)
        rel, ab = check_app(apps[k], app_ref, what=f"case {TC_CASES[k][0]}")
        llr = check_ll(ll[k], ll_ref, what=f"case {TC_CASES[k][0]}")
        print(f"case {TC_CASES[k][0]}: APP rel {rel:.2e} abs {ab:.2e} logP rel {llr:.2e}")


def test_tensor_cores_off_agrees(monkeypatch):
    frames = _frames()
    ntc0, apps0, ll0 = _decode(frames, monkeypatch, "0")
    assert ntc0 == 0
    ntc1, apps1, ll1 = _decode(frames, monkeypatch, "1")
    assert ntc1 > 0
    for k in range(len(frames)):
        check_app(apps1[k], apps0[k], what=f"case {TC_CASES[k][0]}")
        check_ll(ll1[k], ll0[k], what=f"case {TC_CASES[k][0]}")


def test_single_frame_handle_uses_tensor_cores(monkeypatch):
    """The single-frame path (one frame per call) runs the same producers."""
    monkeypatch.setenv("MAPDEC_TC", "1")
    fr = _frames()[3]
    dec = mapdec.Decoder.for_frame(fr)
    app, ll = dec.decode(fr.rx, fr.priors)
    app_ref, ll_ref = oracle.decode(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax,
                                    fr.rx, priors=fr.priors, kappa=2.0)
    check_app(app, app_ref)
    check_ll(ll, ll_ref)
    dec.close()


def test_tensor_cores_across_waves(monkeypatch):
    """A scratch budget of one frame per wave: the waves rotate over three
    scratch regions, and every wave's priors are split for the tensor cores in
    its own region before its forward producers run."""
    monkeypatch.setenv("MAPDEC_TC", "1")
    frames = _frames()
    b = mapdec.Batch(frames, flags=mapdec.MAPDEC_BATCH_GRAPH, mem_budget_bytes=1 << 20)
    assert mapdec.mapdec_batch_num_waves(b.b) >= 4
    rx, pr = b.concat_inputs()
    for rep in range(2):
        st, app, ll = b.decode(rx, pr)
        assert st == 0, mapdec.mapdec_strerror(st)
        apps = b.split(app)
        for k, fr in enumerate(frames):
            app_ref, ll_ref = oracle.decode(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I,
                                            fr.xmax, fr.rx, priors=fr.priors, kappa=2.0)
            check_app(apps[k], app_ref, what=f"case {TC_CASES[k][0]} rep {rep}")
            check_ll(ll[k], ll_ref, what=f"case {TC_CASES[k][0]} rep {rep}")
    b.close()
