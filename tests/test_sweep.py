"""Checkpoint/resume of the threshold sweeps (paper_2603_05381_gb300.sweep) on the CPU.

The per-range decoder here is the oracle (code capacity d = 3), standing in for the
library's sample_and_decode_range: both decode a global shot range whose errors depend only
on the shot indices and the seed.  A sweep stopped part-way (the range decoder raises, as a
killed process would stop) and started again from its state file must end with counts
bit-identical to an uninterrupted sweep, and with the same JSON-lines records apart from the
timing field."""
import json

import numpy as np
import pytest

from paper_2603_05381_gb300 import sweep as sw

SEED = 4


def _oracle_range(pt, first, n):
    from oracle.decoders import decode_shot
    from oracle.graph import code_capacity_tables
    from oracle.sampler import code_capacity_sample
    from oracle.surface import code_capacity_graph, rotated_code
    code = rotated_code(pt["d"])
    samp = code_capacity_sample(code, pt["p"], np.arange(first, first + n, dtype=np.uint64), seed=SEED)
    c = {"shots": n, "fail": [0, 0, 0], "unconverged": [0, 0], "forced_output": [0, 0], "conv_fail": [0, 0],
         "iterations": 0, "msg_updates": 0, "defects": 0, "forced_runs": 0, "forced_rounds": 0,
         "unconverged_any": 0, "conv_fail_any": 0}
    anyf = np.zeros(n, dtype=bool)
    allconv = np.ones(n, dtype=bool)
    for ty, kind in ((0, "X"), (1, "Z")):
        tb = code_capacity_tables(code_capacity_graph(code, kind), pt["p"])
        synd, obs = samp[kind]
        for k in range(n):
            r = decode_shot(tb, np.flatnonzero(synd[k]), pt["T"])
            f = r.obs_pred != obs[k]
            anyf[k] |= f
            allconv[k] &= bool(r.converged)
            c["fail"][ty] += int(f)
            c["unconverged"][ty] += int(not r.converged)
            c["conv_fail"][ty] += int(f and r.converged)
            c["forced_output"][ty] += int(r.from_forced)
            c["iterations"] += r.iters
            c["msg_updates"] += r.msg_updates
            c["defects"] += int(synd[k].sum())
    c["fail"][2] = int(anyf.sum())
    c["unconverged_any"] = int((~allconv).sum())
    c["conv_fail_any"] = int((allconv & anyf).sum())
    return c


class _Stop(Exception):
    pass


def _points():
    return sw.config_points("code_capacity", ds=(3,), ps=(0.09, 0.15))


def _records(path):
    recs = []
    with open(path) as f:
        for x in f:
            try:
                recs.append(json.loads(x))
            except json.JSONDecodeError:
                pass
    for r in recs:
        r.pop("seconds")
    return recs


def test_resumed_sweep_is_bit_identical(tmp_path):
    shots, chunk = 96, 32
    full = tmp_path / "full.jsonl"
    ref = sw.sweep(_points(), shots, state_path=str(full), chunk=chunk, seed=SEED, run_range=_oracle_range)

    part = tmp_path / "part.jsonl"
    calls = {"n": 0}

    def dying(pt, first, n):
        if calls["n"] == 4:      # dies in the middle of the second point
            raise _Stop()
        calls["n"] += 1
        return _oracle_range(pt, first, n)

    with pytest.raises(_Stop):
        sw.sweep(_points(), shots, state_path=str(part), chunk=chunk, seed=SEED, run_range=dying)
    state = sw.load_state(str(part))
    assert state[_points()[0]["key"]]["shots_done"] == 96
    assert state[_points()[1]["key"]]["shots_done"] == 32
    # a torn line from the killed writer is ignored on resume
    with open(part, "a") as f:
        f.write('{"key": "code_capacity:d=3')
    resumed_ranges = []

    def recording(pt, first, n):
        resumed_ranges.append((pt["key"], first, n))
        return _oracle_range(pt, first, n)

    got = sw.sweep(_points(), shots, state_path=str(part), chunk=chunk, seed=SEED, run_range=recording)
    # only the missing ranges of the second point were decoded again
    assert resumed_ranges == [(_points()[1]["key"], 32, 32), (_points()[1]["key"], 64, 32)]
    strip = lambda rs: [{k: v for k, v in r.items() if k not in ("shots_per_s", "msg_updates_per_s")} for r in rs]
    assert strip(got) == strip(ref)
    full_recs = _records(full)
    part_recs = _records(str(part))
    assert [r for r in part_recs if r["shots_done"] == shots] == [r for r in full_recs if r["shots_done"] == shots]
    # and the whole-run counts equal one range over all shots
    for pt, r in zip(_points(), ref):
        c = _oracle_range(pt, 0, shots)
        assert r["ler"] == c["fail"][2] / shots and r["r_nc"] == c["unconverged_any"] / shots


def test_summary_statistics():
    pt = {"key": "k", "model": "circuit", "d": 5, "p": 0.005, "T": 50}
    counts = {"shots": 1000, "fail": [50, 0, 50], "unconverged": [200, 0], "forced_output": [190, 0],
              "conv_fail": [10, 0], "iterations": 9000, "msg_updates": 10**6, "defects": 15000, "forced_runs": 200,
              "forced_rounds": 600, "unconverged_any": 200, "conv_fail_any": 10}
    r = sw.summarize(pt, counts, 2.0)
    assert r["ler"] == 0.05 and abs(r["ler_sigma"] - (0.05 * 0.95 / 1000) ** 0.5) < 1e-15
    assert r["r_nc"] == 0.2 and r["converged_ler"] == 10 / 800 and r["shots_per_s"] == 500.0
    assert len(sw.config_points("code_capacity")) == 128 and len(sw.config_points("circuit")) == 70
