"""Host-side checks of the autograd wrappers (CPU): the channel values passed
in must be the ones the decoder or batch was planned for, since the
derivative is taken there; a mismatch is refused before any device work."""
from types import SimpleNamespace

import pytest
import torch

from paper_1802_08483_gb300.autograd import BatchLogLik, FrameLogLik


class _NoDevice:
    """Stands in for a decoder or batch; any decode call (any method other than
    the channel attributes the test sets) is a test failure."""

    def __getattr__(self, name):
        raise AssertionError("reached the device path")


def test_frame_loglik_refuses_other_channel():
    dec = _NoDevice()
    dec.Pi, dec.Pd, dec.Ps = 0.01, 0.02, 0.001
    pri = torch.full((3, 4), 0.25)
    chan = torch.tensor([0.01, 0.03, 0.001], dtype=torch.float64)
    with pytest.raises(ValueError):
        FrameLogLik.apply(pri, chan, dec, [0, 1])


def test_batch_loglik_refuses_other_channel_or_shape():
    b = _NoDevice()
    b.frames = [SimpleNamespace(Pi=0.01, Pd=0.02, Ps=0.0, N=2, q=2),
                SimpleNamespace(Pi=0.05, Pd=0.05, Ps=0.01, N=2, q=2)]
    pri = torch.full((8,), 0.5)
    with pytest.raises(ValueError):  # one frame's channel is off
        BatchLogLik.apply(pri, torch.tensor([[0.01, 0.02, 0.0], [0.05, 0.04, 0.01]],
                                            dtype=torch.float64), b, [0, 1])
    with pytest.raises(ValueError):  # wrong number of values
        BatchLogLik.apply(pri, torch.tensor([0.01, 0.02, 0.0], dtype=torch.float64), b, [0, 1])


def test_float32_channel_values_are_accepted_up_to_rounding():
    """The first check passes for float32 copies of the channel (the device
    path is then reached, which the stand-in reports)."""
    dec = _NoDevice()
    dec.Pi, dec.Pd, dec.Ps = 0.013, 0.027, 0.0013
    chan = torch.tensor([0.013, 0.027, 0.0013], dtype=torch.float32)
    with pytest.raises(AssertionError, match="device path"):
        FrameLogLik.apply(torch.full((3, 4), 0.25), chan, dec, [0, 1])
