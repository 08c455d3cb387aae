"""torch.autograd.Function wrappers: gradients through backward() against the
FP64 oracle and the FP64 torch-autograd restatement."""
import numpy as np
import pytest

import oracle
import torch_reference
from parity import check_grad, check_grad_priors, check_ll
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


def test_frame_loglik_backward_matches_oracle():
    import torch
    from paper_1802_08483_gb300.autograd import frame_loglik
    rng = np.random.default_rng(501)
    fr = synth.make_frame(rng, 16, 8, 60, 2, 20, 0.04, 0.03, 0.01, dirichlet=True)
    dec = mapdec.Decoder.for_frame(fr)
    pri = torch.tensor(fr.priors, device="cuda", requires_grad=True)
    chan = torch.tensor([fr.Pi, fr.Pd, fr.Ps], dtype=torch.float64, requires_grad=True)
    ll = frame_loglik(pri, chan, dec, fr.rx)
    (2.5 * ll).backward()
    ll_ref, dchan_ref, dpri_ref = oracle.loglik_grad(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps,
                                                     fr.I, fr.xmax, fr.rx, priors=fr.priors)
    check_ll(float(ll.detach()), ll_ref)
    check_grad_priors(pri.grad.cpu().numpy(), 2.5 * dpri_ref, fr.priors, what="priors")
    check_grad(chan.grad.numpy(), 2.5 * dchan_ref, what="channel")


def test_frame_loglik_vs_torch_fp64_autograd():
    import torch
    from paper_1802_08483_gb300.autograd import frame_loglik
    fr = synth.tiny_frame(502, q=4, n=3, N=6, I=2, xmax=6, Pi=0.1, Pd=0.08, Ps=0.05)
    dec = mapdec.Decoder.for_frame(fr)
    pri = torch.tensor(fr.priors, requires_grad=True)
    chan = torch.tensor([fr.Pi, fr.Pd, fr.Ps], dtype=torch.float64, requires_grad=True)
    ll = frame_loglik(pri, chan, dec, fr.rx)
    ll.backward()
    ll_t, dchan_t, dpri_t = torch_reference.grads(fr.codebook, fr.priors.astype(np.float64),
                                                  fr.rx, fr.I, fr.xmax, fr.Pi, fr.Pd, fr.Ps)
    check_ll(float(ll), ll_t)
    check_grad_priors(pri.grad.numpy(), dpri_t, fr.priors)
    check_grad(chan.grad.numpy(), np.array(dchan_t))


def test_batch_loglik_backward():
    import torch
    from paper_1802_08483_gb300.autograd import batch_loglik
    rng = np.random.default_rng(503)
    frames = []
    for k in range(6):
        q, n = synth.QN_CHOICES[k % 5]
        frames.append(synth.make_frame(rng, q, n, 40 + 10 * k, 2, 18, 0.03, 0.03, 0.005,
                                       dirichlet=True))
    b = mapdec.Batch(frames, flags=mapdec.MAPDEC_BATCH_GRAPH | mapdec.MAPDEC_BATCH_GRAD)
    rx, pr = b.concat_inputs()
    pri = torch.tensor(pr, device="cuda", requires_grad=True)
    chan = torch.tensor([[f.Pi, f.Pd, f.Ps] for f in frames], dtype=torch.float64,
                        requires_grad=True)
    ll = batch_loglik(pri, chan, b, rx)
    w = torch.arange(1, len(frames) + 1, dtype=torch.float64, device=ll.device)
    (w * ll).sum().backward()
    gp = b.split(pri.grad.cpu().numpy())
    for k, fr in enumerate(frames):
        ll_ref, dchan_ref, dpri_ref = oracle.loglik_grad(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps,
                                                         fr.I, fr.xmax, fr.rx, priors=fr.priors)
        check_ll(float(ll[k]), ll_ref)
        check_grad_priors(gp[k], (k + 1) * dpri_ref, fr.priors, what=f"frame {k}")
        check_grad(chan.grad[k].detach().cpu().numpy(), (k + 1) * dchan_ref, what=f"frame {k}")
    b.close()


def test_forward_without_grad_skips_the_adjoint():
    """With no input needing a gradient, forward runs the decode path alone:
    log P matches the oracle, and the gradient path's scratch (allocated by the
    first adjoint call) is never allocated.  CUDA priors are passed to the
    library in place."""
    import torch
    from paper_1802_08483_gb300.autograd import frame_loglik
    rng = np.random.default_rng(504)
    # large enough that the gradient scratch (about 12 MB) shows in the free memory
    fr = synth.make_frame(rng, 16, 8, 1000, 2, 60, 0.01, 0.01, 0.005, dirichlet=True)
    dec = mapdec.Decoder.for_frame(fr)
    dec.decode(fr.rx, fr.priors)  # loads the decode kernels
    pri = torch.tensor(fr.priors, device="cuda")
    chan = torch.tensor([fr.Pi, fr.Pd, fr.Ps], dtype=torch.float64)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    with torch.no_grad():
        ll = frame_loglik(pri, chan, dec, fr.rx)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    _, ll_ref = oracle.decode(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                              priors=fr.priors)
    check_ll(float(ll), ll_ref)
    assert ll.device.type == "cuda"
    assert free1 == free0, (free0, free1)
    pri.requires_grad_(True)
    ll2 = frame_loglik(pri, chan, dec, fr.rx)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] < free1  # the adjoint's scratch now exists
    ll2.backward()
    ll_ref2, _, dpri_ref = oracle.loglik_grad(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I,
                                              fr.xmax, fr.rx, priors=fr.priors)
    check_ll(float(ll2.detach()), ll_ref2)
    check_grad_priors(pri.grad.cpu().numpy(), dpri_ref, fr.priors)
    dec.close()
