"""Writes tests/golden/mixed4096_heavy.npz: FP64 oracle references for the
costliest frames of the 4096-frame mixed workload, one or two per (q, n) class
(N near 4000, the widest drift limits of the class), which dominate the
decoder's time in that workload.  Stored per frame: the APPs of every 16th
symbol and log P(Y).  Calls only the oracle and the seeded input generator.

Cost of a frame = N * M * q * MN (M = 2 xmax + 1 drift states, MN = 3n + 1
received lengths): the oracle's work and the decoder's band work alike.

The received-bit weight kappa (an exact reweighting of every path by
kappa^{received length}, undone in log P) keeps the literal FP64 recursion in
range on these long frames.  Frames listed in KAPPA_15 use kappa = 1.5, so
that their references do not share the decoder's power-of-two weight; each of
them is also decoded with kappa = 2, and the script stops unless the two agree
to 1e-9 (APPs) and 1e-12 (log P, relative).

Run:  python tests/golden/make_mixed_golden.py   (a few minutes on 8 cores)
"""
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

STRIDE = 16
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mixed4096_heavy.npz")
FRAMES_TOTAL = 4096
QN = ((2, 4), (8, 6), (16, 10), (32, 8), (64, 12))


def heavy_frames():
    """Per (q, n) class: the frame of largest cost and the frame of largest
    xmax (often the same one)."""
    from paper_1802_08483_gb300 import synth
    by_cost, by_x = {}, {}
    for f in range(FRAMES_TOTAL):
        q, n, N, xmax = synth.c3_frame_shape(f)
        c = N * (2 * xmax + 1) * q * (3 * n + 1)
        if (q, n) not in by_cost or c > by_cost[(q, n)][0]:
            by_cost[(q, n)] = (c, f)
        if (q, n) not in by_x or xmax > by_x[(q, n)][0]:
            by_x[(q, n)] = (xmax, f)
    picked = set()
    for qn in QN:
        picked.add(by_cost[qn][1])
        picked.add(by_x[qn][1])
    return sorted(picked)


def _one(args):
    k, kappa = args
    import oracle
    from paper_1802_08483_gb300 import synth
    fr = synth.config_frame(3, k)
    app, ll = oracle.decode(fr.codebook, fr.N, fr.Pi, fr.Pd, fr.Ps, fr.I, fr.xmax, fr.rx,
                            priors=fr.priors_or_uniform(), kappa=kappa)
    return k, kappa, app[::STRIDE].copy(), ll


def main():
    frames = heavy_frames()
    from paper_1802_08483_gb300 import synth
    # kappa = 1.5 for the costliest frame of the q=64 and q=16 classes
    kappa15 = []
    for qn in ((64, 12), (16, 10)):
        best = max((f for f in frames if synth.c3_frame_shape(f)[:2] == qn),
                   key=lambda f: np.prod(synth.c3_frame_shape(f)[2:]))
        kappa15.append(best)
    jobs = [(k, 1.5 if k in kappa15 else 2.0) for k in frames] + [(k, 2.0) for k in kappa15]
    jobs.sort(key=lambda j: -np.prod(synth.c3_frame_shape(j[0])))
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 4)) as pool:
        res = pool.map(_one, jobs, chunksize=1)
    got = {(k, kap): (app, ll) for k, kap, app, ll in res}
    for k in kappa15:
        a15, l15 = got[(k, 1.5)]
        a2, l2 = got[(k, 2.0)]
        da = float(np.max(np.abs(a15 - a2)))
        dl = abs(l15 - l2) / abs(l2)
        print(f"frame {k}: kappa 1.5 vs 2: APP {da:.2e}, log P rel {dl:.2e}")
        if not (da <= 1e-9 and dl <= 1e-12):
            raise SystemExit(f"frame {k}: kappa 1.5 and 2 disagree")
    out = {"stride": np.array(STRIDE), "frames": np.array(frames),
           "kappa": np.array([1.5 if k in kappa15 else 2.0 for k in frames])}
    for k in frames:
        kap = 1.5 if k in kappa15 else 2.0
        app, ll = got[(k, kap)]
        if not (np.all(np.isfinite(app)) and np.isfinite(ll)):
            raise SystemExit(f"frame {k}: oracle result not finite")
        out[f"app{k}"] = app
        out[f"ll{k}"] = np.array(ll)
        q, n, N, xmax = synth.c3_frame_shape(k)
        print(f"frame {k}: q={q} n={n} N={N} xmax={xmax} kappa={kap} log P={ll:.6f}")
    np.savez_compressed(OUT, **out)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
