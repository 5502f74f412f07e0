"""Pins for the oracle's decoders: exhaustive weight-1 decoding at d=3, syndrome
consistency of every output, and the orderings the paper states between decoders."""
import numpy as np
import pytest

from oracle import brute
from oracle.circuit import Noise, circuit_graph
from oracle.decoders import decode_shot
from oracle.graph import adjacency, circuit_tables, code_capacity_tables, edge_weights_circuit
from oracle.sampler import code_capacity_sample, graph_sample
from oracle.surface import code_capacity_graph, parity_check_matrices, rotated_code
from test_oracle_graph import _explicit_path


@pytest.mark.parametrize("decoder,early", [("bp4m", True), ("bp4m", False), ("bp4mf", False)])
def test_d3_all_weight_one_paulis_decode_without_failure(decoder, early):
    d, p = 3, 0.05
    code = rotated_code(d)
    hz, hx = parity_check_matrices(code)
    tables = {k: code_capacity_tables(code_capacity_graph(code, k), p) for k in ("X", "Z")}
    fails = 0
    for q in range(d * d):
        for pauli in "XYZ":
            e = np.zeros(d * d, dtype=int)
            e[q] = 1
            for kind, h, logical, on in (("X", hz, code.zl, pauli in "XY"),
                                         ("Z", hx, code.xl, pauli in "YZ")):
                comp = e if on else np.zeros_like(e)
                synd = (h @ comp) % 2
                obs = int(comp[logical].sum() % 2)
                r = decode_shot(tables[kind], np.flatnonzero(synd), 50, decoder=decoder,
                                early_exit=early)
                assert len(np.flatnonzero(synd)) <= 2
                fails += int(r.obs_pred != obs)
    assert fails == 0


def _check_consistency(tables, w, synd_row, r):
    g = tables.g
    n = g.n_det
    dets = np.flatnonzero(synd_row)
    seen = np.zeros(len(dets), dtype=int)
    for i, j in r.matching:
        seen[i] += 1
        if j != i:
            seen[j] += 1
    assert (seen == 1).all()  # a perfect matching with boundary
    adj = adjacency(g, w)
    ends = np.zeros(n + 1, dtype=int)
    par = 0
    for i, j in r.matching:
        a = int(dets[i])
        b = n if i == j else int(dets[j])
        for (u, v, ob) in _explicit_path(adj, min(a, b) if b < n else a, max(a, b) if b < n else n, n):
            ends[u] ^= 1
            ends[v] ^= 1
            par ^= ob
    want = np.zeros(n + 1, dtype=int)
    want[dets] = 1
    assert (ends[:n] == want[:n]).all()
    assert par == r.obs_pred


def test_syndrome_consistency_code_capacity():
    code = rotated_code(5)
    g = code_capacity_graph(code, "X")
    tb = code_capacity_tables(g, 0.1)
    synd, obs = code_capacity_sample(code, 0.1, np.arange(60), seed=3)["X"]
    for k in range(60):
        for dec, early in (("bp4m", True), ("bp4m", False), ("bp4mf", False)):
            r = decode_shot(tb, np.flatnonzero(synd[k]), 10, decoder=dec, early_exit=early)
            _check_consistency(tb, [1.0] * len(g.edges), synd[k], r)


def test_syndrome_consistency_circuit():
    g, _, _ = circuit_graph(3, Noise(0.01))
    tb = circuit_tables(g)
    synd, obs = graph_sample(g, np.arange(40), seed=5)
    for k in range(40):
        r = decode_shot(tb, np.flatnonzero(synd[k]), 20)
        _check_consistency(tb, edge_weights_circuit(g), synd[k], r)


def test_bp4mf_never_heavier_than_bp4m_and_map_is_lower_bound():
    code = rotated_code(5)
    g = code_capacity_graph(code, "X")
    tb = code_capacity_tables(g, 0.12)
    synd, _ = code_capacity_sample(code, 0.12, np.arange(80), seed=9)["X"]
    n_small = 0
    for k in range(80):
        dets = np.flatnonzero(synd[k])
        a = decode_shot(tb, dets, 10, decoder="bp4m", early_exit=False)
        b = decode_shot(tb, dets, 10, decoder="bp4mf")
        assert b.weight <= a.weight
        if len(dets) <= 8:
            n_small += 1
            Wsub = tb.W[np.ix_(dets, dets)]
            assert brute.min_weight(Wsub) <= b.weight + 1e-12
    assert n_small > 20


def test_full_t_keeps_lightest_converged():
    # full-T output is never heavier than the early-exit output when the latter converged
    code = rotated_code(5)
    g = code_capacity_graph(code, "X")
    tb = code_capacity_tables(g, 0.1)
    synd, _ = code_capacity_sample(code, 0.1, np.arange(80), seed=13)["X"]
    for k in range(80):
        dets = np.flatnonzero(synd[k])
        e = decode_shot(tb, dets, 12, early_exit=True)
        f = decode_shot(tb, dets, 12, early_exit=False)
        if e.converged:
            assert f.converged and f.weight <= e.weight


def test_circuit_single_mechanisms_d3_report():
    # Every single graphlike mechanism decoded alone: failures are reported, and with
    # priors from shortest paths there are none at d = 3.
    g, _, _ = circuit_graph(3, Noise(0.003))
    tb = circuit_tables(g)
    fails = []
    for e, (u, v, ob, q) in enumerate(g.edges):
        dets = [u] if v == g.n_det else [u, v]
        r = decode_shot(tb, np.array(sorted(dets)), 50)
        if r.obs_pred != ob:
            fails.append(e)
    assert fails == []
