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


def _brute_map(g, probs, synd):
    """Most likely edge subset with syndrome `synd` under independent edge probabilities
    (enumeration of all 2^edges subsets) and the posterior probability that its observable
    parity is 1."""
    m = len(g.edges)
    best, best_p, p_obs1, p_tot = None, -1.0, 0.0, 0.0
    for mask in range(1 << m):
        sy = np.zeros(g.n_det, dtype=bool)
        ob = 0
        pr = 1.0
        for e, (u, v, o, _) in enumerate(g.edges):
            if (mask >> e) & 1:
                sy[u] ^= True
                if v < g.n_det:
                    sy[v] ^= True
                ob ^= o
                pr *= probs[e]
            else:
                pr *= 1.0 - probs[e]
        if not np.array_equal(sy, synd):
            continue
        p_tot += pr
        p_obs1 += pr * ob
        if pr > best_p:
            best, best_p = mask, pr
    return best, p_obs1 / p_tot


def test_flipping_likely_edges_is_an_exact_change_of_variables():
    # Taking every edge with P > 1/2 as present (flip its endpoints, add its observable bit
    # to a base parity) and giving it probability 1 - P leaves the distribution of
    # corrections unchanged: the most likely correction and the posterior of the observable
    # parity are the same for every syndrome (brute force over all edge subsets, d = 3)
    from oracle.bbp4mf import flip_likely_edges
    code = make_code(3)
    g = code_capacity_graph(code, "X")
    rng = np.random.default_rng(5)
    probs = rng.uniform(0.05, 0.95, size=len(g.edges))
    assert (probs > 0.5).sum() >= 2
    comp = np.where(probs > 0.5, 1.0 - probs, probs)
    fmask = sum(1 << e for e in range(len(g.edges)) if probs[e] > 0.5)
    for syn_bits in range(1 << g.n_det):
        synd = np.array([(syn_bits >> j) & 1 for j in range(g.n_det)], dtype=bool)
        b1, po1 = _brute_map(g, probs, synd)
        flipped, base, n = flip_likely_edges(g, probs, synd)
        assert n == bin(fmask).count("1")
        b2, po2 = _brute_map(g, comp, flipped)
        assert b1 == b2 ^ fmask
        assert abs(po1 - (po2 if base == 0 else 1.0 - po2)) < 1e-12


def test_edge_weight_is_symmetric_about_one_half():
    from oracle.bbp4mf import MIN_WEIGHT, edge_weight
    for p in (1e-9, 0.01, 0.3, 0.499):
        # 1 - (1 - p) carries the rounding of 1 - p: relative 1e-16 / p
        assert abs(edge_weight(p) - edge_weight(1.0 - p)) <= 1e-15 / p * edge_weight(p)
        assert abs(edge_weight(p) - np.log((1 - p) / p)) < 1e-12 * max(1.0, np.log((1 - p) / p))
    assert edge_weight(0.5) == MIN_WEIGHT
    # reweighted priors stay finite with edges at one half
    code = make_code(5)
    g = code_capacity_graph(code, "X")
    probs = [0.5 if e % 3 == 0 else 0.2 for e in range(len(g.edges))]
    W, P, L = reweighted_tables(g, probs, np.arange(g.n_det))
    assert np.isfinite(L).all() and (W > 0).all()
