"""One single-frame handle serves every received length in [tau - xmax, tau + xmax]
(the state-space limits of Sec. II-C): mapdec_create plans and allocates the
decode scratch once for the largest, mapdec_loglik_grad its own once, and
later calls with other lengths neither re-plan nor allocate device memory.
Every call is checked against the FP64 oracle."""
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


def _frames(count=20):
    rng = np.random.default_rng(4242)
    q, n, N, I, xmax, Pi, Pd, Ps = 16, 10, 150, 2, 40, 0.05, 0.04, 0.005
    cb = synth.random_codebook(rng, q, n)
    return [synth.make_frame(rng, q, n, N, I, xmax, Pi, Pd, Ps, codebook=cb, dirichlet=True)
            for _ in range(count)]


def test_one_handle_many_lengths_without_allocation():
    import torch
    frames = _frames()
    rhos = [f.rho for f in frames]
    assert len(set(rhos)) >= 8, rhos
    torch.cuda.init()
    dec = mapdec.Decoder.for_frame(frames[0])
    free = []
    for k, fr in enumerate(frames):
        app, ll = dec.decode(fr.rx, fr.priors)
        app2, ext, ll2 = dec.decode_ext(fr.rx, fr.priors)
        ll_ref, dchan_ref, dpri_ref = oracle.loglik_grad(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps,
                                                         fr.I, fr.xmax, fr.rx, priors=fr.priors)
        if k % 4 == 0:
            llg, dchan, dpri = dec.loglik_grad(fr.rx, fr.priors)
            check_ll(llg, ll_ref, what=f"frame {k} (rho {fr.rho}) grad")
            check_grad(dchan, dchan_ref, what=f"frame {k} channel")
            check_grad_priors(dpri, dpri_ref, fr.priors, what=f"frame {k} priors")
        app_ref, ext_ref, ll_ref2 = oracle.decode_ext(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps,
                                                      fr.I, fr.xmax, fr.rx, priors=fr.priors)
        check_app(app, app_ref, what=f"frame {k} (rho {fr.rho})")
        check_ll(ll, ll_ref2, what=f"frame {k} (rho {fr.rho})")
        check_app(app2, app_ref, what=f"frame {k} ext call")
        check_app(ext, ext_ref, what=f"frame {k} extrinsic")
        assert ll2 == ll
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
    # the first iteration made the gradient scratch and loaded the kernels;
    # nothing after it allocates device memory
    assert len(set(free[1:])) == 1, free
    dec.close()


def test_out_of_range_length_then_decode():
    frames = _frames(3)
    fr = frames[0]
    dec = mapdec.Decoder.for_frame(fr)
    too_long = np.zeros(fr.n * fr.N + fr.xmax + 1, np.uint8)
    with pytest.raises(mapdec.MapDecError) as e:
        dec.decode(too_long, fr.priors)
    assert e.value.status == mapdec.MAPDEC_ERR_DRIFT_RANGE
    for f in frames:
        app, ll = dec.decode(f.rx, f.priors)
        app_ref, ll_ref = oracle.decode(f.codebook, f.N, f.Pi, f.Pd, f.Ps, f.I, f.xmax, f.rx,
                                        priors=f.priors)
        check_app(app, app_ref)
        check_ll(ll, ll_ref)
    dec.close()
