#!/usr/bin/env python
"""Throughput benchmark of the batched BSID MAP decoder on one or more GPUs.

Workload (default): 4096 mixed frames per GPU -- N ~ U[100, 4000], (q, n) in
{(2,4),(8,6),(16,10),(32,8),(64,12)}, Pi = Pd log-uniform in [1e-3, 0.1],
Ps ~ U[0, 0.01], I = 2, xmax = ceil(6 sqrt(N n (Pi + Pd))), Dirichlet(1)
priors -- decoded in one batch replayed as a CUDA graph.  One step = the whole
decode (receiver metric, forward/backward recursions, APPs, log-likelihoods)
of every frame.  Metric: decoded information bits per second (sum over frames
of N log2 q, divided by the step time).

Multi-GPU (torchrun): every rank decodes its own 4096 frames (weak scaling);
no collective touches the data path.  `--impl reference` times the FP64 CPU
oracle on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time
from typing import Optional

ROOT = os.path.dirname(os.path.abspath(__file__))
DEFAULT_TUNING = os.path.join(ROOT, "paper_1802_08483_gb300", "tuning", "gb300_mixed4096.json")
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1802_08483_gb300 import synth  # noqa: E402

METRIC = "decoded info bits/s on 1 GB300, batched FP32 vs plain FP32, APP err<=1e-4 vs FP64"
UNIT = "bits/s"
FRAMES_PER_GPU = 4096
PLAIN_STRIDE = 8  # the plain comparator decodes every 8th frame of the workload


def workload_name(frames: int) -> str:
    """The timed workload, named the same way by both arms of the benchmark."""
    return (f"mixed-{frames}: N~U[100,4000], (q,n) in "
            "{(2,4),(8,6),(16,10),(32,8),(64,12)}, Pi=Pd log-U[1e-3,0.1], "
            "Ps~U[0,0.01], I=2, xmax=ceil(6 sqrt(N n (Pi+Pd))), "
            "Dirichlet(1) priors")


# ---------------------------------------------------------------------------
# work accounting
# ---------------------------------------------------------------------------
def lattice_cells(n, I):
    return (I + 1) * n * (n + 1) // 2 + n


def producer_settings(table: dict) -> dict:
    """A tuning table with its recursion setting reset to the planner's (the
    per-class producer parameters kept)."""
    out = json.loads(json.dumps(table))
    for e in out.get("entries", []):
        for k in ("chain_budget_kb", "chain_stages", "chain_threads"):
            e["tune"][k] = 0
    return out


def lattices(fr) -> int:
    """Receiver-metric lattices a frame needs: one per (rx start p, codeword D)
    with one codebook; with one codebook per symbol the metric also depends on
    i, so one per (i, s', D) with start position n i + s' - xmax in [0, rho]."""
    if np.ndim(fr.codebook) == 3:
        i = np.arange(fr.N, dtype=np.int64)
        lo = np.maximum(0, fr.xmax - fr.n * i)
        hi = np.minimum(2 * fr.xmax, fr.rho - fr.n * i + fr.xmax)
        return int(np.maximum(hi - lo + 1, 0).sum()) * fr.q
    return (fr.rho + 1) * fr.q


def valid_transitions(fr) -> int:
    """Number of (i, s', j) with start position in [0, rho], end drift inside the
    limits and window inside the received sequence."""
    n, N, M, x, rho = fr.n, fr.N, 2 * fr.xmax + 1, fr.xmax, fr.rho
    MN = n * (fr.I + 1) + 1
    i = np.arange(N, dtype=np.int64)
    tot = 0
    for j in range(MN):
        lo = np.maximum.reduce([np.zeros_like(i), x - n * i, np.full_like(i, n - j)])
        hi = np.minimum.reduce([np.full_like(i, M - 1), rho - n * i + x - j,
                                np.full_like(i, M - 1 - j + n)])
        tot += int(np.maximum(hi - lo + 1, 0).sum())
    return tot


def write_jsonl(path: str, frames, frame_offset: int, loglik, status, summary: dict) -> None:
    """Per-frame results of a run, one JSON object per line (frame index in the
    workload, shape, channel, log P(Y), status), then one summary object."""
    with open(path, "w") as fh:
        for k, f in enumerate(frames):
            fh.write(json.dumps({"frame": frame_offset + k, "q": int(f.q), "n": int(f.n),
                                 "N": int(f.N), "I": int(f.I), "xmax": int(f.xmax),
                                 "rho": int(f.rho), "Pi": float(f.Pi), "Pd": float(f.Pd),
                                 "Ps": float(f.Ps), "loglik": float(loglik[k]),
                                 "status": int(status[k])}) + "\n")
        fh.write(json.dumps(dict({"summary": True}, **summary)) + "\n")


def lattice_counts(frames) -> dict:
    """Lattices per step: evaluated here, one per (rx start p, D), against the
    paper's gamma grid of one per (i, m', D)."""
    ev = sum((f.rho + 1) * f.q for f in frames)
    grid = sum(f.N * (2 * f.xmax + 1) * f.q for f in frames)
    return {"evaluated": ev, "paper_grid": grid, "ratio": grid / ev if ev else None}


def pipe_flops(fr, tc_bits: int = 0) -> dict:
    """Algorithmic flops of one frame by phase and by the pipe that runs them:
    the contractions of a frame whose producers run on the tensor cores
    (tc_bits: bit 0 forward producer, bit 1 APP producer) count on the tensor
    pipe, everything else on the FP32 pipe.  "executed_fp32" adds the lattices
    the APP producer recomputes."""
    ff = frame_flops(fr)
    w = 2 * fr.q * ff["V"]
    out = {"forward": {"fp32": ff["lattice"] + (0 if tc_bits & 1 else w),
                       "tensor": w if tc_bits & 1 else 0},
           "chains": {"fp32": ff["chains"], "tensor": 0},
           "backward": {"fp32": 0 if tc_bits & 2 else w, "tensor": w if tc_bits & 2 else 0}}
    out["backward"]["executed_fp32"] = out["backward"]["fp32"] + ff["backward_recompute"]
    return out


def frame_flops(fr) -> dict:
    """FP32 flops per phase for one frame (one FMA = 2 flops).

    Algorithmic (the method's own work, counted once): the lattices, one per
    (rx start p, codeword D), in the forward phase with the W contraction
    (2q per valid transition); the two recursions (2 per valid transition
    each); the APP contraction of eq. (L) (2q per valid transition) in the
    backward phase.  The backward phase also re-evaluates every lattice (it
    recomputes R instead of storing it): executed work, reported apart as
    "backward_recompute", never as algorithmic."""
    lat = lattices(fr) * lattice_cells(fr.n, fr.I) * (2 * fr.I + 3)
    V = valid_transitions(fr)
    return {"forward": lat + 2 * fr.q * V, "chains": 4 * V, "backward": 2 * fr.q * V,
            "backward_recompute": lat, "lattice": lat, "V": V}


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle (reported baseline / reference arm)
# ---------------------------------------------------------------------------
def _oracle_frame(args):
    cfg, idx = args
    import oracle
    fr = synth.config_frame(cfg, idx)
    t = time.time()
    # kappa = 2: the oracle's exact received-bit reweighting (the literal FP64
    # recursion underflows on the longest, noisiest frames of the workload)
    oracle.decode(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                  priors=fr.priors_or_uniform(), kappa=2.0)
    return idx, fr.info_bits, time.time() - t


# oracle cost units (3 N M q MN) one host core gets through per second, as
# measured on the Arm host of the GPU machines; sizes the bounded samples
ORACLE_UNITS_PER_CORE_S = 3.6e8


def oracle_cost(q, n, N, xmax, I=2):
    M = 2 * xmax + 1
    MN = n * (I + 1) + 1
    return 3.0 * N * M * q * MN


def oracle_sample(frame_offset: int, budget_units: float, max_frame_units: float):
    """Frames of the workload in index order, skipping any whose oracle cost exceeds
    max_frame_units, until budget_units is used."""
    picked, used, f = [], 0.0, frame_offset
    while used < budget_units and f < frame_offset + FRAMES_PER_GPU:
        q, n, N, xmax = synth.c3_frame_shape(f)
        c = oracle_cost(q, n, N, xmax)
        if c <= max_frame_units:
            picked.append(f)
            used += c
        f += 1
    return picked


def run_oracle(frames_idx, cores):
    import multiprocessing as mp
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    t0 = time.time()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_frame, [(3, f) for f in frames_idx], chunksize=1)
    wall = time.time() - t0
    bits = sum(r[1] for r in res)
    return bits, wall


PHASE_KERNELS = {"pack": "k_pack", "forward": "k_fwd, all (n, I) classes",
                 "chains": "k_chain", "backward": "k_bwd, all (n, I) classes",
                 "finalize": "k_finalize"}


def kernel_sources_sha1() -> str:
    import hashlib
    h = hashlib.sha1()
    d = os.path.join(ROOT, "paper_1802_08483_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        h.update(f.encode())
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def phase_traffic(phase: str, path: str = "") -> Optional[int]:
    """DRAM bytes per step of one phase from the committed launch-list capture,
    or None when the kernel sources changed since the counters were taken (or
    the capture is missing)."""
    try:
        with open(path or os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            prof = json.load(fh)
    except (OSError, ValueError):
        return None
    if prof.get("csrc_sha1") != kernel_sources_sha1():
        return None
    return prof.get(phase)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def host_cpu() -> str:
    """Architecture and CPU model of the host (model name, else the Arm part
    number from /proc/cpuinfo)."""
    import platform
    model = ""
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key, _, val = line.partition(":")
                key = key.strip().lower()
                if key == "model name":
                    model = val.strip()
                    break
                if key == "cpu part" and not model:
                    model = "CPU part " + val.strip()
    except OSError:
        pass
    return f"{platform.machine()}, {model}" if model else platform.machine()


# ---------------------------------------------------------------------------
# per-configuration report (--configs): every synthetic configuration in the
# launch shape it calls for, device-timed, with algorithmic FP32 rates
# ---------------------------------------------------------------------------
def _time_ms(fn, reps=5, warm=2):
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def run_configs(fp32_peak, which=(1, 2, 4, 5, 6, 7)):
    import torch
    from paper_1802_08483_gb300 import mapdec
    out = []

    def report(name, frames, ms, flops, extra=None):
        bits = sum(f.info_bits for f in frames)
        line = {"report": name, "frames": len(frames), "ms": round(ms, 4),
                "bits_per_s": bits / (ms / 1e3), "algorithmic_tflops": flops / (ms / 1e3) / 1e12,
                "frac_fp32_peak": flops / (ms / 1e3) / 1e12 / fp32_peak}
        line.update(extra or {})
        print(json.dumps(line), flush=True)
        out.append(line)

    def flops_of(frames, grad=False):
        tot = 0
        for f in frames:
            ff = frame_flops(f)  # algorithmic: the lattice once, both contractions, chains
            tot += ff["forward"] + ff["chains"] + ff["backward"]
            if grad:
                # the three tangent lattices and their contractions in the APP producer
                tot += 3 * ff["lattice"] + 3 * 2 * f.q * ff["V"]
        return tot

    def batch_run(frames, flags, grad=False):
        b = mapdec.Batch(frames, flags=flags)
        rx, pr = b.concat_inputs()
        if grad:
            st = b.loglik_grad(rx, pr)[0]  # stages the inputs in the resident buffers
            rx_d, pr_d, _, _ = mapdec.mapdec_batch_buffers(b.b)
            dchan = torch.empty(3 * b.nf, dtype=torch.float64, device="cuda")
            dpri = torch.empty(b.prior_total, dtype=torch.float32, device="cuda")
            ll = torch.empty(b.nf, dtype=torch.float64, device="cuda")
            fn = lambda: mapdec.mapdec_batch_loglik_grad(b.b, rx_d, pr_d, dchan, dpri, ll)  # noqa: E731
        else:
            st = b.decode(rx, pr)[0]
            fn = lambda: mapdec.mapdec_batch_run(b.b)  # noqa: E731
        if st != 0:
            raise RuntimeError(mapdec.mapdec_strerror(st))
        return b, fn

    # config 1 and 2: one frame, plain path (one frame per call, default tiles)
    for cfg in [c for c in (1, 2) if c in which]:
        fr = synth.config_frame(cfg, 0)
        dec = mapdec.Decoder.for_frame(fr)
        ms = _time_ms(lambda: dec.decode(fr.rx, fr.priors_or_uniform()))
        report(f"config {cfg}: one frame, plain decode call (host buffers)", [fr], ms,
               flops_of([fr]))
        dec.close()
    # config 2: receiver metrics stored in HBM versus recomputed (batch of one, graph)
    fr = synth.config_frame(2, 0)
    if 2 not in which:
        fr = None
    key = (fr.q, fr.n, fr.I) if fr is not None else None
    for store in ((0, 1) if fr is not None else ()):
        mapdec.mapdec_tune_set(*key, {"store_metric": store})
        b, fn = batch_run([fr], mapdec.MAPDEC_BATCH_GRAPH)
        ms = _time_ms(fn)
        T = (fr.rho + 1)
        rbytes = 2 * T * ((fr.q + 3) // 4 * 4) * (fr.n * (fr.I + 1) + 1) * 4 if store else 0
        report(f"config 2: one frame, graph, R {'stored in HBM' if store else 'recomputed'}",
               [fr], ms, flops_of([fr]),
               {"executed_tflops": (flops_of([fr]) + (0 if store else frame_flops(fr)["lattice"]))
                / (ms / 1e3) / 1e12,
                "R_bytes_written_and_read": rbytes,
                "R_traffic_GBps": rbytes / (ms / 1e3) / 1e9})
        b.close()
    if key is not None:
        mapdec.mapdec_tune_set(*key, None)
    if 6 in which:
        # one codebook per symbol: lattices on the (i, s', D) grid, no position dedupe
        frames = synth.config_frames(6)
        b, fn = batch_run(frames, mapdec.MAPDEC_BATCH_GRAPH)
        ms = _time_ms(fn, reps=3, warm=1)
        report("config 6: 64 frames N=1000, q=16, n=10, one codebook per symbol, decode",
               frames, ms, flops_of(frames),
               {"executed_tflops": (flops_of(frames) + sum(frame_flops(f)["lattice"]
                                                          for f in frames)) / (ms / 1e3) / 1e12,
                "lattices_per_frame": lattices(frames[0])})
        b.close()
    if 7 in which:
        # frames cut from a stream, drift priors on both boundaries, extrinsic outputs
        frames = synth.config_frames(7)
        b, fn = batch_run(frames, mapdec.MAPDEC_BATCH_GRAPH | mapdec.MAPDEC_BATCH_EXTRINSIC)
        ms = _time_ms(fn, reps=3, warm=1)
        report("config 7: 256 frames N=1000, q=16, n=10 cut from a stream, boundary drift "
               "priors, APPs + extrinsic outputs", frames, ms, flops_of(frames))
        b.close()
    if 4 not in which and 5 not in which:
        return out
    # config 4: 256 frames, log-likelihood and gradients, alpha checkpoint every 45 symbols
    if 4 not in which:
        return _config5(out, report, flops_of, batch_run) if 5 in which else out
    os.environ["MAPDEC_SEG_K"] = "45"
    frames = synth.config_frames(4)
    b, fn = batch_run(frames, mapdec.MAPDEC_BATCH_GRAPH | mapdec.MAPDEC_BATCH_GRAD |
                      mapdec.MAPDEC_BATCH_SEGMENTED, grad=True)
    ms = _time_ms(fn, reps=3, warm=1)
    report("config 4: 256 frames N=2000, log P + gradients, checkpoint every 45 symbols",
           frames, ms, flops_of(frames, grad=True))
    b.close()
    os.environ.pop("MAPDEC_SEG_K", None)
    return _config5(out, report, flops_of, batch_run) if 5 in which else out


def _config5(out, report, flops_of, batch_run):
    from paper_1802_08483_gb300 import mapdec
    # config 5: 64 frames N=8000, q=64, n=12, I=3, checkpointed (K = ceil(sqrt(N)))
    frames = synth.config_frames(5)
    b, fn = batch_run(frames, mapdec.MAPDEC_BATCH_GRAPH | mapdec.MAPDEC_BATCH_SEGMENTED)
    ms = _time_ms(fn, reps=3, warm=1)
    report("config 5: 64 frames N=8000, decode, checkpoint every ceil(sqrt(N)) symbols",
           frames, ms, flops_of(frames),
           {"executed_tflops": (flops_of(frames) + sum(2 * frame_flops(f)["lattice"] +
                                                      2 * f.q * frame_flops(f)["V"]
                                                      for f in frames)) / (ms / 1e3) / 1e12,
            "note": "executed work adds the APP producer's lattice recompute and the forward "
                    "producers' second sweep (recording and recompute sweeps)"})
    b.close()
    return out


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames", type=int, default=FRAMES_PER_GPU,
                    help="frames per GPU (the workload is 4096; smaller only for profiling)")
    ap.add_argument("--frame-stride", type=int, default=1,
                    help="take every k-th frame of the workload (profiling a small case that "
                         "samples the whole mix)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--oracle-seconds", type=float, default=20.0)
    ap.add_argument("--configs", nargs="?", const="1,2,4,5,6,7", default=None,
                    help="instead of the benchmark line, report synthetic configurations "
                         "(comma list; default 1,2,4,5,6,7)")
    ap.add_argument("--tuning", default=DEFAULT_TUNING,
                    help="tuning table (JSON written by paper_1802_08483_gb300.tune); '' = none")
    ap.add_argument("--log-jsonl", default="",
                    help="write per-frame log P(Y) and status plus a summary to this JSONL file "
                         "(rank r > 0 appends .rank<r>)")
    ap.add_argument("--mem-budget-gb", type=float, default=0.0,
                    help="device scratch budget (0 = 60%% of free memory); frames beyond it "
                         "are decoded in further waves")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    n_gpus = max(args.gpus, world)
    from paper_1802_08483_gb300 import multigpu
    frame_offset = multigpu.frame_indices(rank, max(world, 1), FRAMES_PER_GPU)[0]
    steps, warmup = max(1, args.steps), max(3, args.warmup)

    if args.impl == "reference":
        if rank != 0:
            return 0
        cores = host_cores()
        per_step = []
        bits_tot = 0.0
        budget = (ORACLE_UNITS_PER_CORE_S * cores * min(args.oracle_seconds, 60.0)
                  / max(1, steps + warmup) * 2)
        sample = oracle_sample(0, budget, ORACLE_UNITS_PER_CORE_S * 20)
        for s in range(warmup + steps):
            bits, wall = run_oracle(sample, cores)
            if s >= warmup:
                per_step.append(wall)
                bits_tot = bits
        t = statistics.mean(per_step)
        val = bits_tot / t
        line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": n_gpus, "steps": steps,
                "warmup": warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "impl": "reference",
                "config": {"workload": workload_name(FRAMES_PER_GPU),
                           "frames_per_gpu": FRAMES_PER_GPU,
                           "reference": f"FP64 CPU oracle on {cores} host threads, a sample of "
                                        f"{len(sample)} frames per step"},
                "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "cpu": host_cpu(),
                                 "kind": "oracle",
                                 "sample": f"workload frames {sample[:8]}{'...' if len(sample) > 8 else ''} "
                                           f"({len(sample)} frames, {bits_tot:.0f} info bits)"},
                "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    # ---- CPU baseline first (spawned pool, before any GPU work) ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        sample = oracle_sample(0, ORACLE_UNITS_PER_CORE_S * cores * args.oracle_seconds / 2,
                               ORACLE_UNITS_PER_CORE_S * 25)
        bits, wall = run_oracle(sample, cores)
        cpu = {"value": bits / wall, "unit": UNIT, "cores": cores, "cpu": host_cpu(),
               "kind": "oracle",
               "sample": f"{len(sample)} frames of the mixed workload in index order "
                         f"(frames whose oracle cost exceeds ~25 core-s skipped), "
                         f"{bits:.0f} info bits in {wall:.1f} s"}

    import torch
    from paper_1802_08483_gb300 import build as libbuild
    from paper_1802_08483_gb300 import mapdec

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local_rank)
    libbuild.build()
    mapdec.load()
    tuning = None
    if args.tuning and os.path.exists(args.tuning):
        from paper_1802_08483_gb300 import tune as libtune
        libtune.load(args.tuning)
        tuning = os.path.relpath(args.tuning, ROOT)

    if args.configs:
        # the other workloads keep the table's producer parameters (per class)
        # and use the planner's recursion setting: the table's is chosen for
        # a batch whose recursions share the SMs with producers
        if tuning:
            libtune.apply(producer_settings(json.load(open(args.tuning))))
        props = torch.cuda.get_device_properties(local_rank)
        run_configs(props.multi_processor_count * 128 * 2 * 2070.0e6 / 1e12,
                    {int(c) for c in args.configs.split(",")})
        return 0

    # ---- workload ----
    t0 = time.time()
    stride = max(1, args.frame_stride)
    frames = [synth.config_frame(3, frame_offset + f * stride) for f in range(args.frames)]
    gen_s = time.time() - t0
    bits_per_step = sum(f.info_bits for f in frames)
    flops = {"forward": 0, "chains": 0, "backward": 0, "backward_recompute": 0, "lattice": 0,
             "V": 0}
    for f in frames:
        for k, v in frame_flops(f).items():
            flops[k] += v

    b = mapdec.Batch(frames, flags=mapdec.MAPDEC_BATCH_GRAPH | mapdec.MAPDEC_BATCH_TIMING,
                     mem_budget_bytes=int(args.mem_budget_gb * (1 << 30)))
    tc_count, tc_bits = mapdec.mapdec_batch_tc_frames(b.b, b.nf)
    pipes = {k: {"fp32": 0, "tensor": 0} for k in ("forward", "chains", "backward")}
    pipes["backward"]["executed_fp32"] = 0
    for f, bits in zip(frames, tc_bits):
        for k, v in pipe_flops(f, int(bits)).items():
            for kk, vv in v.items():
                pipes[k][kk] += vv
    rx_all, pr_all = b.concat_inputs()
    # stage inputs into the batch's resident device buffers (one decode call)
    st, app0, ll0 = b.decode(rx_all, pr_all)
    if st != 0:
        raise RuntimeError(f"decode failed: {mapdec.mapdec_strerror(st)}")
    stream = torch.cuda.current_stream()
    mapdec.mapdec_batch_set_stream(b.b, stream.cuda_stream)

    def one_step():
        rc = mapdec.mapdec_batch_run(b.b)
        if rc != 0:
            raise RuntimeError(mapdec.mapdec_strerror(rc))

    for _ in range(warmup):
        one_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    phase_tot = np.zeros(5)
    launches = 0
    ev0.record(stream)
    for _ in range(steps):
        one_step()
        launches += mapdec.mapdec_batch_last_launches(b.b)
        phase_tot += mapdec.mapdec_batch_phase_ms(b.b)  # events recorded inside the graph
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / steps
    status = mapdec.mapdec_batch_sync(b.b)
    if status != 0:
        raise RuntimeError(f"decode status {mapdec.mapdec_strerror(status)}")
    if world > 1:
        dist.barrier()
        ms, total_bits = multigpu.combine(ms, bits_per_step, dist, device="cuda")
    else:
        total_bits = bits_per_step
    value = total_bits / (ms / 1e3)
    phase_ms = phase_tot / steps

    # ---- roofline of the dominant phase, per pipe (FP32 CUDA cores, tensor cores) ----
    props = torch.cuda.get_device_properties(local_rank)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s
    names = list(mapdec.PHASES)
    dom = int(np.argmax(phase_ms))
    dom_name = names[dom]
    sec = phase_ms[dom] / 1e3
    # the dominant phase's algorithmic work on each pipe; the bound is the pipe
    # it uses the larger fraction of
    tensor_peak = float(peaks.get("bf16_tflops_sustained", 1709.5))  # timed inside a long step
    pf = pipes.get(dom_name, {"fp32": 0, "tensor": 0})
    fp32_t = pf["fp32"] / sec / 1e12 if sec > 0 else 0.0
    tens_t = pf["tensor"] / sec / 1e12 if sec > 0 else 0.0
    fp32_frac = fp32_t / fp32_peak if fp32_peak else 0.0
    tens_frac = tens_t / tensor_peak if tensor_peak else 0.0
    tensor_bound = tens_frac > fp32_frac
    achieved = tens_t if tensor_bound else fp32_t
    peak = tensor_peak if tensor_bound else fp32_peak
    traffic = phase_traffic(dom_name)
    try:
        probe = mapdec.mapdec_fp32_fma_peak(stream.cuda_stream)
    except mapdec.MapDecError:
        probe = None
    total_alg = flops["forward"] + flops["chains"] + flops["backward"]
    step_tflops = total_alg / (ms / 1e3) / 1e12
    step_fp32 = sum(pipes[k]["fp32"] for k in ("forward", "chains", "backward"))
    step_tens = sum(pipes[k]["tensor"] for k in ("forward", "chains", "backward"))
    roofline = {"bound": "tensor" if tensor_bound else "alu", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak if peak else None,
                "traffic": traffic,
                "kernel": f"{dom_name} phase ({PHASE_KERNELS.get(dom_name, '')})",
                "flops": "algorithmic: each lattice once, the W and APP contractions (2q per "
                         "valid transition each), the recursions (2 per transition each); the "
                         "backward phase's own work is the APP contraction",
                "pipes": {"fp32": {"achieved": fp32_t, "peak": fp32_peak, "frac": fp32_frac,
                                   "peak_source": f"{props.multi_processor_count} SMs x 128 "
                                                  f"FP32 lanes x 2 x {sm_max:.0f} MHz",
                                   "peak_probe": probe,
                                   "frac_of_probe": fp32_t / probe if probe else None},
                          "tensor": {"achieved": tens_t, "peak": tensor_peak, "frac": tens_frac,
                                     "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained "
                                                    "(cuBLAS bf16, of measured)",
                                     "executed_products": {"forward": 6, "backward": 3},
                                     "note": "split bf16: six (W) or three (APP) bf16 MMAs "
                                             "per algorithmic product, counted once"}},
                "executed_fp32": {"tflops": (pf.get("executed_fp32", pf["fp32"]) / sec / 1e12)
                                  if sec > 0 else 0.0,
                                  "note": "adds the lattices the APP producer recomputes "
                                          "(executed, not algorithmic)"},
                "step": {"algorithmic_tflops": step_tflops,
                         "fp32_frac": step_fp32 / (ms / 1e3) / 1e12 / fp32_peak,
                         "tensor_frac": step_tens / (ms / 1e3) / 1e12 / tensor_peak},
                "phase_ms": {names[k]: round(float(phase_ms[k]), 3) for k in range(5)}}

    # ---- end to end through the public API with host buffers ----
    e2e = None
    if not args.no_e2e:
        rx_h = torch.from_numpy(rx_all).pin_memory()
        pr_h = torch.from_numpy(pr_all).pin_memory()
        app_h = torch.empty(b.prior_total, dtype=torch.float32).pin_memory()
        ll_h = torch.empty(b.nf, dtype=torch.float64).pin_memory()
        e_steps = max(1, min(steps, 3))
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(e_steps):
            rc = mapdec.mapdec_batch_decode(b.b, rx_h, pr_h, app_h, ll_h)
            if rc != 0:
                raise RuntimeError(mapdec.mapdec_strerror(rc))
        e_s = (time.perf_counter() - t1) / e_steps
        e2e = {"value": bits_per_step / e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(rx_all.nbytes + pr_all.nbytes),
               "d2h_bytes_per_step": int(b.prior_total * 4 + b.nf * 8)}

    # ---- plain comparator: one frame per call, default tiles, no graph, host
    # buffers (compare with e2e); a systematic sample of the same frames ----
    plain = None
    if not args.no_plain and rank == 0:
        sub = frames[::PLAIN_STRIDE]
        p_s = 0.0
        for f in sub:
            d = mapdec.Decoder.for_frame(f)  # plans and allocates: not timed
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            d.decode(f.rx, f.priors)
            p_s += time.perf_counter() - t1
            d.close()
        plain = {"value": sum(f.info_bits for f in sub) / p_s, "unit": UNIT,
                 "frames": len(sub),
                 "note": f"every {PLAIN_STRIDE}th frame of the workload, one mapdec_decode call "
                         "each with host buffers (the same metric as e2e)"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": n_gpus, "steps": steps,
            "warmup": warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(args.frames) + (
                           f", every {stride}th frame of mixed-{FRAMES_PER_GPU}" if stride > 1 else ""),
                       "launch": "one CUDA-graph batch per GPU",
                       "frames_per_gpu": args.frames, "info_bits_per_gpu_step": bits_per_step,
                       "l2": "inputs and scratch larger than L2 (no flush needed)",
                       "waves": mapdec.mapdec_batch_num_waves(b.b),
                       "tensor_core_frames": {"forward": int(tc_count),
                                              "app": int(sum(1 for x in tc_bits if x & 2))},
                       "tuning": tuning,
                       "parallelism": f"frames sharded, {n_gpus} GPU(s), no collective",
                       "gen_seconds": round(gen_s, 1)},
            "roofline": roofline,
            "algorithmic_tflops": total_alg / (ms / 1e3) / 1e12,
            "lattices_per_step": lattice_counts(frames),
            "cpu_baseline": cpu, "e2e": e2e, "plain": plain,
            "gpu_launches": launches, "clocks": clk}
    if rank == 0:
        print(json.dumps(line))
    if args.log_jsonl:
        path = args.log_jsonl if rank == 0 else f"{args.log_jsonl}.rank{rank}"
        write_jsonl(path, frames, frame_offset, ll0, mapdec.mapdec_batch_status(b.b, b.nf),
                    {"rank": rank, "ms_per_step": ms, "job_bits_per_s": value,
                     "phase_ms": line["roofline"]["phase_ms"], "steps": steps})
    b.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
