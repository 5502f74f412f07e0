"""Pins for the oracle's B-BP4MF pieces: quaternary BP is exact on tree-shaped Tanner graphs,
the reweighting reduces to the ordinary priors under uniform posteriors, and the whole
decoder corrects every weight-1 error at d = 3."""
import numpy as np
import pytest

from oracle.bbp4mf import bbp4mf_shot, brute_posteriors, qbp, reweighted_tables, tanner
from oracle.graph import code_capacity_tables
from oracle.surface import code_capacity_graph, make_code, parity_check_matrices

TREES = [
    ([("Z", [0, 1]), ("Z", [1, 2]), ("X", [2, 3])], 4),
    ([("Z", [0, 1, 2]), ("X", [2, 3]), ("X", [0, 4])], 5),
    ([("X", [0, 1]), ("Z", [1, 2]), ("X", [1, 3]), ("Z", [3, 4])], 5),
]


@pytest.mark.parametrize("tree", range(len(TREES)))
def test_quaternary_bp_is_exact_on_trees(tree):
    checks, n = TREES[tree]
    rng = np.random.default_rng(tree)
    for _ in range(4):
        syn = [int(x) for x in rng.integers(0, 2, size=len(checks))]
        p = float(rng.uniform(0.02, 0.25))
        post, _, _, _ = qbp(checks, n, syn, p, 2 * n + 2, stop=False)
        assert np.allclose(post, brute_posteriors(checks, n, syn, p), atol=1e-12)


def test_quaternary_bp_with_no_syndrome_keeps_the_prior_decision():
    code = make_code(3)
    checks = tanner(code)
    post, dec, conv, it = qbp(checks, code.n, [0] * len(checks), 0.05, 10)
    assert conv and it == 1 and (dec == 0).all()


def test_reweighting_with_uniform_posteriors_is_the_ordinary_prior():
    code = make_code(5)
    g = code_capacity_graph(code, "X")
    q = 0.07
    tb = code_capacity_tables(g, q)
    dets = np.array([0, 3, 4, 9, 11])
    W, P, L = reweighted_tables(g, [q] * len(g.edges), dets)
    assert np.allclose(W, tb.W[np.ix_(dets, dets)], rtol=1e-12)
    assert np.array_equal(P, tb.P[np.ix_(dets, dets)])


@pytest.mark.parametrize("family", ["rotated", "unrotated"])
def test_bbp4mf_corrects_every_weight_one_error_d3(family):
    code = make_code(3, family)
    graphs = {k: code_capacity_graph(code, k) for k in ("X", "Z")}
    hz, hx = parity_check_matrices(code)
    for q in range(code.n):
        for pauli in "XYZ":
            ex = np.zeros(code.n, dtype=int)
            ez = np.zeros(code.n, dtype=int)
            if pauli in "XY":
                ex[q] = 1
            if pauli in "YZ":
                ez[q] = 1
            sx = (hx @ ez) % 2   # X-checks see Z components
            sz = (hz @ ex) % 2
            out = bbp4mf_shot(code, graphs, sx, sz, 0.05, 25, 25)
            assert out["X"] == int(ex[code.zl].sum() % 2)
            assert out["Z"] == int(ez[code.xl].sum() % 2)


def test_reweighting_floors_weights_of_likely_errors():
    # posteriors at or above one half would make edges free or negative; the floor keeps
    # every shortest path well defined and every prior finite, and a path over k floored
    # edges weighs exactly k * 2^-20
    from oracle.bbp4mf import MIN_WEIGHT
    code = make_code(5)
    g = code_capacity_graph(code, "X")
    probs = [0.9 if e % 3 == 0 else 0.5 for e in range(len(g.edges))]
    dets = np.arange(g.n_det)
    W, P, L = reweighted_tables(g, probs, dets)
    assert np.isfinite(L).all() and (W > 0).all()
    # every edge floored: W counts hops of the shortest path
    W1, _, _ = reweighted_tables(g, [0.75] * len(g.edges), dets)
    hops = np.rint(W1 / MIN_WEIGHT)
    assert np.allclose(W1, hops * MIN_WEIGHT, rtol=1e-12) and (hops >= 1).all()
    # neighbouring checks of one qubit are one hop apart
    u, v = g.edges[0][0], g.edges[0][1]
    if v < g.n_det:
        assert hops[u, v] == 1
