"""Writes tests/golden/large64_frames.npz: FP64 oracle references for frames 0
and 1 of the 64-frame N=8000, q=64, n=12, I=3 workload (every 16th symbol's
APPs and log P(Y)).  Calls only the oracle and the seeded input generator.

The literal FP64 recursion underflows on frames this long (its forward rows
span beyond 2^-1074); the oracle's exact received-bit reweighting (kappa = 2)
is used.  Run:  python tests/golden/make_large_golden.py   (about 15 min/frame)
"""
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

STRIDE = 16
FRAMES = (0, 1)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "large64_frames.npz")


def _one(k):
    import oracle
    from paper_1802_08483_gb300 import synth
    fr = synth.config_frame(5, k)
    app, ll = oracle.decode(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                            priors=fr.priors_or_uniform(), kappa=2.0)
    return k, app[::STRIDE].copy(), ll


def main():
    with mp.get_context("spawn").Pool(len(FRAMES)) as pool:
        res = pool.map(_one, FRAMES)
    out = {"stride": np.array(STRIDE), "frames": np.array(FRAMES)}
    for k, app, ll in res:
        out[f"app{k}"] = app
        out[f"ll{k}"] = np.array(ll)
    np.savez_compressed(OUT, **out)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
