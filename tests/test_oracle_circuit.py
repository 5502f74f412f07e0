"""Pins for the oracle's memory-Z circuit and its detector error model."""
import numpy as np
import pytest

from oracle.circuit import (Noise, backward_frames, circuit_graph, memory_z_circuit,
                            merge_probabilities)
from oracle.surface import code_capacity_graph, rotated_code
from statevector import detector_values, run_circuit
from test_oracle_surface import _odd_cycle_through_boundary


def test_noiseless_state_vector_d3_all_detectors_zero():
    circ = memory_z_circuit(3, Noise(0.0))
    assert circ.n_qubits == 17
    for seed in range(4):
        rec = run_circuit(circ, np.random.default_rng(seed))
        z, x, obs = detector_values(circ, rec)
        assert not any(z) and not any(x) and obs == 0


def _locations(circ):
    """(op index, target index, pauli) for every mechanism, in the order of backward_frames."""
    locs = []
    two = [(a, b) for a in "IXYZ" for b in "IXYZ" if (a, b) != ("I", "I")]
    for k, (name, tg, _) in enumerate(circ.ops):
        if name == "DEP1":
            locs += [(k, t, pa) for t in range(len(tg)) for pa in "XYZ"]
        elif name == "DEP2":
            locs += [(k, t, pp) for t in range(len(tg)) for pp in two]
        elif name == "XERR":
            locs += [(k, t, "X") for t in range(len(tg))]
    return locs


def test_injected_paulis_match_state_vector_d3():
    circ = memory_z_circuit(3, Noise(0.01))
    fr = backward_frames(circ, include_x_detectors=False)
    locs = _locations(circ)
    assert len(locs) == len(fr.mechanisms)
    rng = np.random.default_rng(5)
    picks = rng.choice(len(locs), size=60, replace=False)
    for m in picks:
        rec = run_circuit(circ, np.random.default_rng(int(m)), inject=locs[m])
        z, _, obs = detector_values(circ, rec)
        zs, ob, _ = fr.mechanisms[m]
        assert tuple(np.flatnonzero(z)) == zs, locs[m]
        assert obs == ob


@pytest.mark.parametrize("d", [3, 5, 7])
def test_dem_structure(d):
    g, circ, st = circuit_graph(d, Noise(0.004))
    assert g.n_det == (d * d - 1) // 2 * (d + 1)
    assert st["nondeterministic"] == []
    fr = backward_frames(circ, include_x_detectors=True)
    assert fr.nondeterministic == set()
    for zs, ob, _ in fr.mechanisms:
        assert len(zs) <= 2
        assert not (len(zs) == 0 and ob == 1)
    assert st["hyperedges"] == 0
    keys = [(u, v, o) for (u, v, o, _) in g.edges]
    assert keys == sorted(set(keys))


@pytest.mark.parametrize("d", [3, 5])
def test_circuit_distance_equals_d(d):
    g, _, _ = circuit_graph(d, Noise(0.004))
    assert _odd_cycle_through_boundary(g) == d


@pytest.mark.parametrize("d", [3, 5])
def test_reduces_to_code_capacity_graph(d):
    # Only before-round data depolarization, perfect everything else: every round layer is
    # the code-capacity X graph with q = p/3 merged with p/3, and nothing else fires.
    p = 0.01
    noise = Noise(p, data_round=True, gates=False, idle=False, reset_flip=False, meas_flip=False)
    g, _, _ = circuit_graph(d, noise)
    cc = code_capacity_graph(rotated_code(d), "X")
    nper = cc.n_det
    q = merge_probabilities([p / 3, p / 3])
    want = set()
    for rnd in range(d):
        for (u, v, ob, _) in cc.edges:
            uu = u + rnd * nper
            vv = g.n_det if v == cc.n_det else v + rnd * nper
            want.add((uu, vv, ob))
    got = {(u, v, ob) for (u, v, ob, _) in g.edges}
    assert got == want
    # parallel boundary qubits on the same check merge to the odd-parity probability
    for (u, v, ob, qq) in g.edges:
        mult = sum(1 for (a, b, o, _) in cc.edges
                   if (a, b if b < cc.n_det else g.n_det, o) == (u % nper, v if v == g.n_det else v % nper, ob))
        expect = merge_probabilities([p / 3] * (2 * mult))
        assert qq == pytest.approx(expect, rel=1e-12)
    assert q == pytest.approx(2 * p / 3 - 2 * (p / 3) ** 2, rel=1e-12)


def test_merge_is_odd_parity_probability():
    qs = [0.1, 0.02, 0.3]
    brute = 0.0
    for mask in range(8):
        pr = 1.0
        for k in range(3):
            pr *= qs[k] if (mask >> k) & 1 else 1 - qs[k]
        if bin(mask).count("1") % 2:
            brute += pr
    assert merge_probabilities(qs) == pytest.approx(brute, rel=1e-14)
    assert merge_probabilities([0.25]) == 0.25


def test_unrotated_state_vector_d2():
    # the unrotated schedule (X: N, W, E, S; Z: N, E, W, S) on the d = 2 code (9 qubits):
    # noiseless detectors are 0 and injected Paulis flip what the error model says
    circ = memory_z_circuit(2, Noise(0.0), "unrotated")
    for seed in range(4):
        z, x, obs = detector_values(circ, run_circuit(circ, np.random.default_rng(seed)))
        assert not any(z) and not any(x) and obs == 0
    circ = memory_z_circuit(2, Noise(0.01), "unrotated")
    fr = backward_frames(circ)
    locs = _locations(circ)
    assert len(locs) == len(fr.mechanisms)
    rng = np.random.default_rng(8)
    for m in rng.choice(len(locs), size=80, replace=False):
        z, _, obs = detector_values(circ, run_circuit(circ, np.random.default_rng(int(m)), inject=locs[m]))
        zs, ob, _ = fr.mechanisms[m]
        assert tuple(np.flatnonzero(z)) == zs and obs == ob


@pytest.mark.parametrize("d", [3, 5, 7])
def test_unrotated_dem_structure_and_distance(d):
    g, circ, st = circuit_graph(d, Noise(0.004), "unrotated")
    assert g.n_det == d * (d - 1) * (d + 1)
    assert st["nondeterministic"] == [] and st["hyperedges"] == 0
    fr = backward_frames(circ, include_x_detectors=True)
    assert fr.nondeterministic == set()
    if d <= 5:
        assert _odd_cycle_through_boundary(g) == d


def test_unrotated_reduces_to_code_capacity_graph():
    from oracle.surface import code_capacity_graph, unrotated_code
    d, p = 3, 0.01
    noise = Noise(p, data_round=True, gates=False, idle=False, reset_flip=False, meas_flip=False)
    g, _, _ = circuit_graph(d, noise, "unrotated")
    cc = code_capacity_graph(unrotated_code(d), "X")
    want = set()
    for rnd in range(d):
        for (u, v, ob, _) in cc.edges:
            want.add((u + rnd * cc.n_det, g.n_det if v == cc.n_det else v + rnd * cc.n_det, ob))
    assert {(u, v, ob) for (u, v, ob, _) in g.edges} == want
