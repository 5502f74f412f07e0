"""Pins for the oracle's error samplers (oracle/sampler.py) against what probability fixes.

Each mechanism fires independently, so a detector is unsatisfied with probability
(1 - prod_e (1 - 2 q_e)) / 2 over the edges that touch it (the probability that an odd
number of independent events occur), and the observable flips with the same expression
over the edges that carry the observable.  Per-detector and observable rates are compared
with these closed forms within 5 standard deviations; the strict threshold and the
edge-to-unit layout are pinned exactly on single draws.  A dropped or extra endpoint, a
dropped observable XOR, a wrong edge probability or a mis-assigned unit shifts one of these
rates by far more than 5 sigma at 2*10^4 shots.
"""
import numpy as np
import pytest

from oracle.circuit import Noise, circuit_graph
from oracle.philox import unit_words
from oracle.sampler import code_capacity_sample, graph_sample, pauli_thresholds
from oracle.surface import DetGraph, code_capacity_graph, rotated_code


def _odd_parity_rate(qs):
    return (1.0 - np.prod(1.0 - 2.0 * np.asarray(qs, dtype=np.float64))) / 2.0


def _within_5_sigma(freq, prob, n):
    sd = np.sqrt(prob * (1.0 - prob) / n)
    # a rate that is exactly 0 or 1 must be met exactly
    return np.abs(freq - prob) <= 5.0 * sd + 1e-12


@pytest.mark.parametrize("d,p", [(5, 0.01), (7, 0.008)])
def test_circuit_detector_and_observable_rates(d, p):
    og, _, _ = circuit_graph(d, Noise(p))
    n = 20000
    synd, obs = graph_sample(og, np.arange(n, dtype=np.uint64), seed=0x5EED + d)
    touching = [[] for _ in range(og.n_det)]
    obs_q = []
    for (u, v, ob, q) in og.edges:
        touching[u].append(q)
        if v < og.n_det:
            touching[v].append(q)
        if ob:
            obs_q.append(q)
    want = np.array([_odd_parity_rate(t) for t in touching])
    got = synd.mean(axis=0)
    bad = np.flatnonzero(~_within_5_sigma(got, want, n))
    assert bad.size == 0, [(int(j), float(got[j]), float(want[j])) for j in bad[:5]]
    pobs = _odd_parity_rate(obs_q)
    assert 0.01 < pobs < 0.5
    assert _within_5_sigma(obs.mean(), pobs, n)
    # the mean defect count follows from the same closed form (a plain sum of the rates)
    assert abs(synd.sum(axis=1).mean() - want.sum()) < 5 * np.sqrt((want * (1 - want)).sum() / n)


def test_circuit_rates_detect_a_planted_extra_endpoint():
    # the same statistic on a sampler that XORs the boundary side of each boundary edge
    # into its detector twice (a plausible slip) must fail: the check has power
    og, _, _ = circuit_graph(5, Noise(0.01))
    n = 20000
    synd, _ = graph_sample(og, np.arange(n, dtype=np.uint64), seed=3)
    u = unit_words(np.arange(n, dtype=np.uint64), len(og.edges), seed=3)
    planted = synd.copy()
    for e, (a, b, _, q) in enumerate(og.edges):
        if b == og.n_det:
            fired = u[:, e] < np.uint64(int(q * 4294967296.0))
            planted[:, a] ^= fired   # cancels the boundary edge's contribution
    touching = [[] for _ in range(og.n_det)]
    for (a, b, _, q) in og.edges:
        touching[a].append(q)
        if b < og.n_det:
            touching[b].append(q)
    want = np.array([_odd_parity_rate(t) for t in touching])
    assert not np.all(_within_5_sigma(planted.mean(axis=0), want, n))


def test_edge_threshold_is_strict_and_unit_is_edge_index():
    # a draw equal to the threshold does not fire (u < floor(q 2^32)); one above it does.
    # Single-edge graphs built around the actual draw of shot 0, unit e.
    n_det = 4
    words = unit_words(np.array([0], dtype=np.uint64), 8, seed=99, stream=2)[0]
    for e in (0, 3, 5):
        w = int(words[e])
        edges = []
        for k in range(8):
            q = 0.0
            if k == e:
                q = w / 4294967296.0          # floor(q 2^32) == w exactly
            edges.append((k % n_det, n_det if k % 2 else (k + 1) % n_det, k % 2, q))
        g = DetGraph(n_det=n_det, edges=edges)
        synd, obs = graph_sample(g, np.array([0], dtype=np.uint64), seed=99, stream=2)
        assert not synd.any() and obs[0] == 0
        edges[e] = edges[e][:3] + ((w + 1) / 4294967296.0,)
        g = DetGraph(n_det=n_det, edges=edges)
        synd, obs = graph_sample(g, np.array([0], dtype=np.uint64), seed=99, stream=2)
        a, b, ob, _ = edges[e]
        expect = np.zeros(n_det, dtype=bool)
        expect[a] ^= True
        if b < n_det:
            expect[b] ^= True
        assert np.array_equal(synd[0], expect) and obs[0] == ob


@pytest.mark.parametrize("d,p", [(5, 0.12), (7, 0.06)])
def test_code_capacity_check_and_observable_rates(d, p):
    # an X (Z) component occurs with probability 2p/3 per qubit (X or Y; Y or Z)
    code = rotated_code(d)
    n = 20000
    out = code_capacity_sample(code, p, np.arange(n, dtype=np.uint64), seed=21)
    qx = 2.0 * p / 3.0
    for kind in ("X", "Z"):
        g = code_capacity_graph(code, kind)
        touching = [0] * g.n_det
        n_obs = 0
        for (u, v, ob, _) in g.edges:
            touching[u] += 1
            if v < g.n_det:
                touching[v] += 1
            n_obs += ob
        want = np.array([_odd_parity_rate([qx] * t) for t in touching])
        synd, obs = out[kind]
        assert np.all(_within_5_sigma(synd.mean(axis=0), want, n)), kind
        assert n_obs == d
        assert _within_5_sigma(obs.mean(), _odd_parity_rate([qx] * d), n), kind
    # X and Z components are correlated through Y: P(both) = p/3 per qubit
    u = unit_words(np.arange(n, dtype=np.uint64), code.n, seed=21)
    t1, t2, _ = pauli_thresholds(p)
    y = (u >= t1) & (u < t2)
    assert _within_5_sigma(y.mean(), p / 3.0, y.size)
