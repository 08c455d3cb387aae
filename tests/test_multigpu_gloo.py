"""The N>1 path on CPU: two gloo ranks shard the frames and combine timing and
bits exactly as the benchmark does on GPUs (no data-path collective)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1802_08483_gb300 import multigpu, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    idx = multigpu.frame_indices(rank, world, 3)
    bits = sum(synth.config_frame(3, f).info_bits for f in idx)
    ms = 100.0 + 50.0 * rank
    tmax, btot = multigpu.combine(ms, bits, dist)
    out[rank] = (idx, bits, tmax, btot)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_combine():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    i0, b0, t0, s0 = out[0]
    i1, b1, t1, s1 = out[1]
    assert set(i0).isdisjoint(i1) and i0 == [0, 1, 2] and i1 == [3, 4, 5]
    assert t0 == t1 == 150.0
    assert s0 == s1 == pytest.approx(b0 + b1)


def test_single_process_combine_is_identity():
    assert multigpu.combine(12.5, 1000.0) == (12.5, 1000.0)
    with pytest.raises(ValueError):
        multigpu.frame_indices(2, 2, 4)
