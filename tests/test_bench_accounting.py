"""Host-side work accounting of the benchmark (CPU): the count of valid
(i, m', j) transitions behind the algorithmic flop figures, checked against a
plain loop over the paper's state grid (Sec. II-C: drift m' in [-xmax, xmax]
at symbol i, received length n + delta with delta in [-n, nI], window inside
[0, rho]), and the lattice counts with and without the position dedupe."""
import numpy as np
import pytest

import bench
from paper_1802_08483_gb300 import synth


def _transitions_by_loop(fr):
    n, x, rho = fr.n, fr.xmax, fr.rho
    MN = n * (fr.I + 1) + 1
    count = 0
    for i in range(fr.N):
        for m1 in range(-x, x + 1):
            p = n * i + m1
            if p < 0 or p > rho:
                continue
            for j in range(MN):
                m2 = m1 + j - n
                if -x <= m2 <= x and p + j <= rho:
                    count += 1
    return count


@pytest.mark.parametrize("seed,q,n,N,I,xmax", [
    (1, 4, 3, 7, 1, 2),      # narrow limits
    (2, 8, 5, 20, 2, 9),
    (3, 2, 4, 30, 2, 40),    # limits wider than the frame
    (4, 16, 6, 12, 3, 5),
])
def test_valid_transitions_match_state_grid_loop(seed, q, n, N, I, xmax):
    rng = np.random.default_rng(seed)
    fr = synth.make_frame(rng, q, n, N, I, xmax, 0.08, 0.08, 0.01)
    assert bench.valid_transitions(fr) == _transitions_by_loop(fr)


def test_lattice_counts():
    frames = [synth.config_frame(3, f) for f in range(4)]
    c = bench.lattice_counts(frames)
    assert c["evaluated"] == sum((f.rho + 1) * f.q for f in frames)
    assert c["paper_grid"] == sum(f.N * (2 * f.xmax + 1) * f.q for f in frames)
    assert c["ratio"] > 1.0


def test_write_jsonl(tmp_path):
    import json
    frames = [synth.config_frame(3, f) for f in range(3)]
    path = tmp_path / "run.jsonl"
    bench.write_jsonl(str(path), frames, 10, [-1.5, -2.5, -3.5], [0, 0, 3],
                      {"ms_per_step": 1.0})
    rows = [json.loads(x) for x in path.read_text().splitlines()]
    assert len(rows) == 4 and rows[-1]["summary"] is True
    assert [r["frame"] for r in rows[:3]] == [10, 11, 12]
    assert rows[2]["status"] == 3 and rows[1]["loglik"] == -2.5
    assert rows[0]["rho"] == frames[0].rho and rows[0]["q"] == frames[0].q


def test_phase_traffic_follows_the_source_hash(tmp_path):
    """The committed DRAM bytes are reported only for the kernel sources they
    were taken on."""
    import json
    good = tmp_path / "good.json"
    good.write_text(json.dumps({"csrc_sha1": bench.kernel_sources_sha1(), "backward": 123}))
    stale = tmp_path / "stale.json"
    stale.write_text(json.dumps({"csrc_sha1": "0" * 40, "backward": 123}))
    assert bench.phase_traffic("backward", str(good)) == 123
    assert bench.phase_traffic("backward", str(stale)) is None
    assert bench.phase_traffic("backward", str(tmp_path / "missing.json")) is None


def test_pipe_flops_split():
    """The per-pipe split moves exactly the contractions of tensor-core frames
    to the tensor pipe; the sum over pipes is the algorithmic total."""
    fr = synth.config_frame(3, 5)
    ff = bench.frame_flops(fr)
    total = ff["forward"] + ff["chains"] + ff["backward"]
    w = 2 * fr.q * ff["V"]
    for bits in (0, 1, 3):
        pf = bench.pipe_flops(fr, bits)
        assert sum(pf[k]["fp32"] + pf[k]["tensor"] for k in pf) == total
        assert pf["forward"]["tensor"] == (w if bits & 1 else 0)
        assert pf["backward"]["tensor"] == (w if bits & 2 else 0)
        assert pf["backward"]["executed_fp32"] == pf["backward"]["fp32"] + ff["lattice"]


@pytest.mark.parametrize("seed,N,xmax", [(61, 7, 5), (62, 30, 12), (63, 3, 9)])
def test_per_symbol_lattice_count_matches_state_grid_loop(seed, N, xmax):
    """One codebook per symbol: one lattice per (i, s', D) whose start position
    n i + s' - xmax lies in [0, rho], counted by a plain loop."""
    fr = synth.per_symbol_frame(np.random.default_rng(seed), 4, 3, N, 1, xmax, 0.1, 0.1, 0.02)
    count = 0
    for i in range(fr.N):
        for s in range(2 * fr.xmax + 1):
            if 0 <= fr.n * i + s - fr.xmax <= fr.rho:
                count += fr.q
    assert bench.lattices(fr) == count
    one = synth.tiny_frame(seed, q=4, n=3, N=N, xmax=xmax)
    assert bench.lattices(one) == (one.rho + 1) * one.q


def test_producer_settings_keep_tiles_and_reset_recursions():
    import json
    import os
    table = json.load(open(os.path.join(os.path.dirname(__file__), "..", "paper_1802_08483_gb300",
                                        "tuning", "gb300_mixed4096.json")))
    out = bench.producer_settings(table)
    for a, b in zip(table["entries"], out["entries"]):
        assert (a["q"], a["n"], a["I"]) == (b["q"], b["n"], b["I"])
        for k in ("P", "nsub", "store_metric"):
            assert b["tune"][k] == a["tune"][k]
        assert b["tune"]["chain_budget_kb"] == b["tune"]["chain_stages"] == 0
        assert b["tune"]["chain_threads"] == 0
    assert table["entries"][0]["tune"]["chain_threads"] == 128  # the input is not modified
