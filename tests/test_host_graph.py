"""CPU tests of the library's host side: the C ABI loads and exports every declared
symbol, and the host graph builder reproduces the oracle's tables exactly.  Building a
graph touches no device, so these run without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle.circuit import Noise, circuit_graph
from oracle.graph import circuit_tables, code_capacity_tables
from oracle.sampler import edge_threshold, pauli_thresholds
from oracle.surface import code_capacity_graph, rotated_code

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_05381_gb300 import _capi
    return _capi.load()


def test_library_exports_every_declared_symbol(lib):
    header = open(os.path.join(ROOT, "include", "bp4m.h")).read()
    names = set(re.findall(r"\b(bp4m_[a-z_]+)\s*\(", header))
    assert len(names) >= 10
    so = ctypes.CDLL(os.path.join(ROOT, "paper_2603_05381_gb300", "libbp4m.so"))
    for name in sorted(names):
        assert hasattr(so, name), name


def test_bad_arguments_are_rejected(lib):
    from paper_2603_05381_gb300 import Bp4mError, Graph
    with pytest.raises(Bp4mError):
        Graph(4, "circuit", 0.005)
    with pytest.raises(Bp4mError):
        Graph(5, "circuit", 0.7)
    with pytest.raises(Bp4mError):
        Graph(5, "circuit", 0.005, rounds=3)


def test_decoder_options_are_checked_before_the_device(lib):
    # every decoder option is validated on the host before any device work: an empty shot range
    # with valid options returns zero counts, invalid options are rejected (no GPU needed)
    import paper_2603_05381_gb300 as pkg
    g = pkg.Graph(5, "circuit", 0.005)
    for form in (0, 1, 2):
        c = g.sample_and_decode(0, seed=1, iters=10, opts=pkg.make_opts(precision="fp32", tile_form=form))
        assert c["shots"] == 0 and c["msg_updates"] == 0
    bad = [dict(tile_form=3), dict(tile_form=-1), dict(stream_cluster=3), dict(forced=2), dict(alpha=0.0)]
    for kw in bad:
        with pytest.raises(pkg.Bp4mError):
            g.sample_and_decode(0, seed=1, iters=10, opts=pkg.make_opts(precision="fp32", **kw))
    with pytest.raises(pkg.Bp4mError):
        g.sample_and_decode(0, seed=1, iters=0, opts=pkg.make_opts(precision="fp32"))


@pytest.mark.parametrize("d", [3, 5, 7, 9])
def test_code_capacity_tables_match_oracle(lib, d):
    from paper_2603_05381_gb300 import Graph
    p = 0.09
    for prior, pp in (("p", p), ("2p/3", 2 * p / 3)):
        g = Graph(d, "code_capacity", p, prior=prior)
        info = g.info()
        assert info["n_types"] == 2 and info["n_units"] == d * d
        for ty, kind in ((0, "X"), (1, "Z")):
            og = code_capacity_graph(rotated_code(d), kind)
            ot = code_capacity_tables(og, pp)
            assert info["n_det"][ty] == og.n_det
            assert [(u, v, o) for (u, v, o, _) in g.export("edges", ty)] == [(u, v, o) for (u, v, o, _) in og.edges]
            assert np.array_equal(g.export("W", ty), ot.W)
            assert np.array_equal(g.export("parity", ty), ot.P)
            np.testing.assert_allclose(g.export("L", ty), ot.L, rtol=1e-15, atol=0)
        assert list(g.export("thresholds")) == pauli_thresholds(p)
        g.close()


@pytest.mark.parametrize("d,p", [(3, 0.001), (3, 0.01), (5, 0.005), (7, 0.004)])
def test_circuit_graph_matches_oracle(lib, d, p):
    from paper_2603_05381_gb300 import Graph
    g = Graph(d, "circuit", p)
    og, _, _ = circuit_graph(d, Noise(p))
    ot = circuit_tables(og)
    info = g.info()
    assert info["n_det"] == [og.n_det] and info["n_edges"] == [len(og.edges)]
    edges = g.export("edges")
    assert [(u, v, o) for (u, v, o, _) in edges] == [(u, v, o) for (u, v, o, _) in og.edges]
    assert all(a[3] == b[3] for a, b in zip(edges, og.edges))  # bit-identical merged q
    assert np.array_equal(g.export("thresholds"), np.array([edge_threshold(q) for (*_, q) in og.edges]))
    assert np.array_equal(g.export("W"), ot.W)
    assert np.array_equal(g.export("parity"), ot.P)
    np.testing.assert_allclose(g.export("L"), ot.L, rtol=1e-15, atol=0)


def test_circuit_graph_d13_matches_oracle(lib):
    # the benchmark's graph: rotated memory-Z, d = 13, p = 0.005
    from paper_2603_05381_gb300 import Graph
    g = Graph(13, "circuit", 0.005)
    og, _, _ = circuit_graph(13, Noise(0.005))
    assert g.info()["n_det"] == [1176]
    edges = g.export("edges")
    assert [(u, v, o, q) for (u, v, o, q) in edges] == list(og.edges)
    rng = np.random.default_rng(0)
    srcs = sorted(rng.choice(og.n_det, size=12, replace=False).tolist())
    from oracle.graph import all_pairs, edge_weights_circuit
    W, P = all_pairs(og, edge_weights_circuit(og), sources=srcs)
    Wg, Pg = g.export("W"), g.export("parity")
    for i in srcs:
        assert np.array_equal(Wg[i, i:], W[i, i:])
        assert np.array_equal(Pg[i, i:], P[i, i:])


@pytest.mark.parametrize("d", [3, 5, 7])
def test_unrotated_tables_match_oracle(lib, d):
    from paper_2603_05381_gb300 import Graph
    from oracle.surface import unrotated_code
    g = Graph(d, "circuit", 0.006, family="unrotated")
    og, _, _ = circuit_graph(d, Noise(0.006), "unrotated")
    ot = circuit_tables(og)
    assert g.export("edges") == list(og.edges)
    assert np.array_equal(g.export("W"), ot.W) and np.array_equal(g.export("parity"), ot.P)
    np.testing.assert_allclose(g.export("L"), ot.L, rtol=1e-15, atol=0)
    g2 = Graph(d, "code_capacity", 0.07, family="unrotated")
    assert g2.info()["n_units"] == d * d + (d - 1) ** 2
    for ty, kind in ((0, "X"), (1, "Z")):
        cg = code_capacity_graph(unrotated_code(d), kind)
        ct = code_capacity_tables(cg, 0.07)
        assert [(u, v, o) for (u, v, o, _) in g2.export("edges", ty)] == [(u, v, o) for (u, v, o, _) in cg.edges]
        assert np.array_equal(g2.export("W", ty), ct.W) and np.array_equal(g2.export("parity", ty), ct.P)


def test_mean_defects_closed_form_and_oracle_edges(lib):
    from paper_2603_05381_gb300 import Graph
    # rotated code capacity: per type (d-1)^2/2 checks of weight 4 and d-1 of weight 2; a data
    # qubit flips a check type with probability 2p/3, so a weight-w check is unsatisfied with
    # probability (1 - (1 - 4p/3)^w) / 2
    for d, p in ((5, 0.05), (9, 0.10), (21, 0.20)):
        g = Graph(d, "code_capacity", p)
        r = 1.0 - 4.0 * p / 3.0
        want = ((d - 1) ** 2 / 2 * (1 - r ** 4) + (d - 1) * (1 - r ** 2)) / 2
        got = g.info()["mean_defects"]
        assert len(got) == 2
        for x in got:
            assert abs(x - want) <= 1e-12 * want
        g.close()
    # circuits: the same sum over the oracle's merged edges
    for d, p in ((5, 0.008), (13, 0.005)):
        g = Graph(d, "circuit", p)
        og, _, _ = circuit_graph(d, Noise(p))
        prod = np.ones(og.n_det)
        for (u, v, _, q) in og.edges:
            prod[u] *= 1 - 2 * q
            if v < og.n_det:
                prod[v] *= 1 - 2 * q
        want = float(((1 - prod) / 2).sum())
        got = g.info()["mean_defects"][0]
        assert abs(got - want) <= 1e-9 * want
        g.close()
