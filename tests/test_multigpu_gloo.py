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


def _worker_strong(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    frames = [synth.config_frame(3, f) for f in range(10)]
    parts = multigpu.lpt_partition([multigpu.frame_cost(fr) for fr in frames], world)
    mine = parts[rank]
    # stand-ins for the decoder's per-frame results, computed from the frame alone
    apps = [float(frames[f].N * 10 + f) for f in mine]
    lls = [-float(frames[f].rho) for f in mine]
    res = multigpu.gather_results(parts, apps, lls, dist, world)
    g = multigpu.allreduce_channel_grad([1.0 + rank, 2.0 * rank, -rank], dist)
    out[rank] = (parts, res, g.tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_lpt_gather_and_gradient_allreduce():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker_strong, args=(world, port, out), nprocs=world, join=True)
    parts, res0, g0 = out[0]
    _, res1, g1 = out[1]
    frames = [synth.config_frame(3, f) for f in range(10)]
    assert sorted(parts[0] + parts[1]) == list(range(10))
    assert res1 is None
    apps, lls = res0
    assert apps == [float(fr.N * 10 + f) for f, fr in enumerate(frames)]
    assert lls == [-float(fr.rho) for fr in frames]
    assert g0 == g1 == [3.0, 2.0, -1.0]


def test_lpt_partition_balances_and_is_deterministic():
    costs = [7, 5, 4, 3, 3, 2, 2, 1]
    parts = multigpu.lpt_partition(costs, 3)
    loads = [sum(costs[k] for k in p) for p in parts]
    assert sorted(k for p in parts for k in p) == list(range(8))
    assert max(loads) - min(loads) <= max(costs)
    assert parts == multigpu.lpt_partition(costs, 3)
    # the LPT bound: makespan <= 4/3 of the optimum (here the optimum is 9)
    assert max(loads) <= 12
    with pytest.raises(ValueError):
        multigpu.lpt_partition(costs, 0)
    assert multigpu.lpt_partition([], 2) == [[], []]
