"""Autotuner for the batched decoder's launch parameters.

For each (q, n, I) class of a workload it times candidate settings on a
sample of that class's frames and keeps the fastest:

  * P, the received positions per producer tile, and nsub, the tiles per
    APP super-tile (both bound by shared memory; the planner rejects what
    does not fit and falls back to its own choice);
  * store_metric: keep the receiver metrics R in device memory between the
    forward and the APP producer, or recompute them (decode only);
  * tensor_cores: the producers' contractions on the tensor cores (split
    bf16, FP32 accumulation) or on the FP32 CUDA cores;
  * the recursion CTA's shared-memory budget, bulk-copy stages and block size
    (128, 256 or 512 threads).

The producers' block size is fixed at 256 threads: the tensor-core producers
split their epilogue over two warpgroups and the CUDA-core producers' register
tiles are laid out for it; their work per block is tuned through P and nsub.

The producer parameters are searched per class, coordinate by coordinate
(tile size, super-tile depth, store-or-recompute), each candidate scored by
the producer phases' device time (events the library records at phase
boundaries) on a sample of the class's frames.  The recursion parameters
trade per-chain latency against chains resident per SM beside the producers,
which only the full mix of frames shows, so they are chosen once for all
classes by the wall time of a large sample of the whole workload (the
--chain-sample frames; 0 = all of them, which is what the co-residence of
recursions and producers needs to show in full).  Choices go to the
process-wide tuning table (mapdec_tune_set) and can be saved as JSON and
loaded again.  Only measurement and bookkeeping live here: every timed run
executes the library's kernels.
"""
from __future__ import annotations

import argparse
import json
import os
from typing import Dict, Iterable, List, Optional, Tuple

import numpy as np

from . import mapdec

FIELDS = ("P", "nsub", "chain_budget_kb", "chain_stages", "store_metric", "tensor_cores",
          "chain_threads")
DEFAULT = {k: 0 for k in FIELDS}
P_CANDIDATES = (0, 1, 2, 4, 8, 16, 32)
NSUB_CANDIDATES = (0, 2, 4, 8, 16, 32)
TC_CANDIDATES = (0, 2)  # planner's choice (tensor cores where supported), CUDA cores
# recursion settings: (shared-memory budget KB, stages, threads); 0 = planner's
CHAIN_CANDIDATES = ((0, 0, 0), (72, 2, 0), (150, 2, 0), (100, 3, 0), (0, 0, 128), (0, 0, 512),
                    (48, 2, 128), (52, 2, 128))


def class_of(fr) -> Tuple[int, int, int]:
    return (int(fr.q), int(fr.n), int(fr.I))


def classes(frames) -> Dict[Tuple[int, int, int], List[int]]:
    out: Dict[Tuple[int, int, int], List[int]] = {}
    for k, fr in enumerate(frames):
        out.setdefault(class_of(fr), []).append(k)
    return out


def sample_indices(idx: List[int], count: int) -> List[int]:
    """`count` indices spread evenly over idx (all of them if there are fewer,
    or if count <= 0)."""
    if count <= 0 or len(idx) <= count:
        return list(idx)
    pos = np.linspace(0, len(idx) - 1, count).round().astype(int)
    return [idx[p] for p in pos]


def time_frames(frames, reps: int = 3, mem_budget_bytes: int = 0, wall: bool = False) -> float:
    """Time (ms) of one decode of `frames` as one graph-captured batch, best of
    `reps` runs: the producer phases' device time (pack, forward, backward,
    finalize) or, with wall=True, the whole run's wall time."""
    import time
    b = mapdec.Batch(frames, flags=mapdec.MAPDEC_BATCH_GRAPH | mapdec.MAPDEC_BATCH_TIMING,
                     mem_budget_bytes=mem_budget_bytes)
    try:
        rx, pr = b.concat_inputs()
        st, _, _ = b.decode(rx, pr)
        if st != mapdec.MAPDEC_OK:
            raise mapdec.MapDecError(st, "tune: decode")
        best = float("inf")
        for _ in range(reps):
            t0 = time.perf_counter()
            st = mapdec.mapdec_batch_run(b.b)
            if st != mapdec.MAPDEC_OK:
                raise mapdec.MapDecError(st, "tune: run")
            ph = mapdec.mapdec_batch_phase_ms(b.b)  # waits for the run
            t1 = time.perf_counter()
            ms = (t1 - t0) * 1e3 if wall else float(ph[0] + ph[1] + ph[3] + ph[4])
            best = min(best, ms)
        st = mapdec.mapdec_batch_sync(b.b)
        if st != mapdec.MAPDEC_OK:
            raise mapdec.MapDecError(st, "tune: status")
        return best
    finally:
        b.close()


def tune_class(key, frames, reps: int = 3, log=None,
               p_candidates: Iterable[int] = P_CANDIDATES,
               nsub_candidates: Iterable[int] = NSUB_CANDIDATES,
               store_candidates: Iterable[int] = (0, 1),
               tc_candidates: Iterable[int] = TC_CANDIDATES) -> dict:
    """Coordinate search of the producer parameters of one class; leaves the
    winner in the table.  The kind of producer (tensor or CUDA cores) is chosen
    first, since the tile sizes that suit it differ."""
    q, n, I = key
    cur = dict(DEFAULT)
    mapdec.mapdec_tune_set(q, n, I, cur)
    base = time_frames(frames, reps)
    best_ms = base
    for field, values in (("tensor_cores", tc_candidates), ("P", p_candidates),
                          ("nsub", nsub_candidates), ("store_metric", store_candidates)):
        for v in values:
            if v == cur[field]:
                continue
            cand = dict(cur, **{field: int(v)})
            mapdec.mapdec_tune_set(q, n, I, cand)
            ms = time_frames(frames, reps)
            if log:
                log(f"  {key} {cand} producers {ms:.3f} ms")
            if ms < best_ms:
                best_ms, cur = ms, cand
    mapdec.mapdec_tune_set(q, n, I, cur)
    return {"q": q, "n": n, "I": I, "tune": cur, "producer_ms": best_ms,
            "untuned_producer_ms": base, "sample_frames": len(frames)}


def tune_chains(entries, frames, reps: int = 2, log=None,
                chain_candidates: Iterable[Tuple[int, int, int]] = CHAIN_CANDIDATES) -> dict:
    """One recursion setting (shared-memory budget, stages, block size) for
    every class, by the wall time of `frames`."""
    def set_all(kb, stg, thr):
        for e in entries:
            e["tune"]["chain_budget_kb"], e["tune"]["chain_stages"] = int(kb), int(stg)
            e["tune"]["chain_threads"] = int(thr)
            mapdec.mapdec_tune_set(e["q"], e["n"], e["I"], e["tune"])
    best = None
    for cand in chain_candidates:
        kb, stg, thr = (tuple(cand) + (0,))[:3]
        set_all(kb, stg, thr)
        ms = time_frames(frames, reps, wall=True)
        if log:
            log(f"  recursions {kb} KB / {stg} stages / {thr or 256} threads: {ms:.1f} ms wall")
        if best is None or ms < best[0]:
            best = (ms, kb, stg, thr)
    set_all(best[1], best[2], best[3])
    return {"chain_budget_kb": best[1], "chain_stages": best[2], "chain_threads": best[3],
            "wall_ms": best[0], "sample_frames": len(frames)}


def tune(frames, sample: int = 48, chain_sample: int = 0, reps: int = 3, log=None,
         chain_candidates: Iterable[Tuple[int, int]] = CHAIN_CANDIDATES, **kw) -> dict:
    """Tune every (q, n, I) class of `frames`; returns the JSON-ready table."""
    mapdec.load()
    entries = []
    for key, idx in sorted(classes(frames).items()):
        sub = [frames[k] for k in sample_indices(idx, sample)]
        if log:
            log(f"class {key}: {len(idx)} frames, sample {len(sub)}")
        entries.append(tune_class(key, sub, reps=reps, log=log, **kw))
    mix = [frames[k] for k in sample_indices(list(range(len(frames))), chain_sample)]
    chains = tune_chains(entries, mix, reps=max(1, reps - 1), log=log,
                         chain_candidates=chain_candidates)
    return {"entries": entries, "recursions": chains}


def apply(table: dict) -> None:
    """Load a table (as returned by tune() or read from JSON) into the library."""
    for e in table.get("entries", []):
        t = {k: int(e["tune"].get(k, 0)) for k in FIELDS}
        mapdec.mapdec_tune_set(e["q"], e["n"], e["I"], t)


def save(table: dict, path: str) -> None:
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    with open(path, "w") as fh:
        json.dump(table, fh, indent=1)


def load(path: str) -> dict:
    with open(path) as fh:
        table = json.load(fh)
    apply(table)
    return table


def main(argv: Optional[List[str]] = None) -> int:
    from . import synth
    ap = argparse.ArgumentParser(description="tune the batched decoder on a synthetic workload")
    ap.add_argument("--config", type=int, default=3, help="workload: synthetic config 1..5")
    ap.add_argument("--frames", type=int, default=0, help="frames of the workload (0 = all)")
    ap.add_argument("--sample", type=int, default=48, help="frames timed per class")
    ap.add_argument("--chain-sample", type=int, default=0,
                    help="frames of the whole workload timed for the recursion setting (0 = all)")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--out", required=True)
    a = ap.parse_args(argv)
    idx = None if a.frames <= 0 else list(range(a.frames))
    frames = synth.config_frames(a.config, idx)
    table = tune(frames, sample=a.sample, chain_sample=a.chain_sample, reps=a.reps, log=print)
    try:
        import torch
        table["device"] = torch.cuda.get_device_name(0)
    except Exception:  # noqa: BLE001 - the device name is informational
        table["device"] = "unknown"
    table["workload"] = f"synthetic config {a.config}, {len(frames)} frames"
    save(table, a.out)
    for e in table["entries"]:
        print(json.dumps(e))
    print(json.dumps(table["recursions"]))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
