"""Pins for the oracle's BP rules: closed forms, exactness on trees, the single-loop
theorem, and the paper's worked inference example."""
import json
import math
import os

import numpy as np
import pytest
from scipy.special import logsumexp

from oracle import bp, brute
from oracle.decoders import bp4m

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_example.json")


def _sym(rng, s, lo=-6.0, hi=-0.5):
    A = rng.uniform(lo, hi, size=(s, s))
    return np.triu(A) + np.triu(A, 1).T


def test_leave_one_out_matches_library_logsumexp():
    rng = np.random.default_rng(0)
    for s in (2, 3, 7):
        row = rng.normal(size=s) * 5
        valid = np.ones(s, dtype=bool)
        got = bp.loo_lse(row, valid)
        for j in range(s):
            assert got[j] == pytest.approx(logsumexp(np.delete(row, j)), rel=1e-13)
        Q = rng.normal(size=(s, s))
        rows = bp.loo_lse_rows(Q, np.ones((s, s), dtype=bool))
        for i in range(s):
            assert np.allclose(rows[i], bp.loo_lse(Q[i], valid), rtol=1e-13)


def test_single_detector_goes_to_boundary():
    L = np.array([[-4.0]])
    r = bp4m(L, np.array([[4.0]]), T=5)
    assert r.converged and r.iters == 1 and r.matching == [(0, 0)]
    assert r.lam[0, 0] == math.inf


def test_two_detectors_closed_form():
    # s = 2 is a tree: after iteration 1, lambda_01 = l01 - l00 - l11 and
    # lambda_00 = l00 - l01; from iteration 2 on lambda_00 = l00 - l01 + l11.
    l00, l01, l11 = -3.0, -2.2, -4.5
    L = np.array([[l00, l01], [l01, l11]])
    hist = bp.run_bp(L, 3)
    lam1 = hist[0][1]
    assert lam1[0, 1] == pytest.approx(l01 - l00 - l11, abs=1e-14)
    assert lam1[0, 0] == pytest.approx(l00 - l01, abs=1e-14)
    lam2 = hist[1][1]
    assert lam2[0, 0] == pytest.approx(l00 - l01 + l11, abs=1e-14)
    exact = brute.exact_marginal_llrs(L)
    assert np.allclose(lam2, exact, atol=1e-12)
    assert np.allclose(hist[2][1], exact, atol=1e-12)


def test_equal_weights_tie_is_not_kept():
    # lambda_00 is exactly 0 at iteration 1 when l00 == l01; a strict > keeps neither
    L = np.array([[-2.0, -2.0], [-2.0, -3.0]])
    lam = bp.run_bp(L, 1)[0][1]
    assert lam[0, 0] == 0.0
    V, conv = bp.decide(lam)
    assert not V[0, 0]


@pytest.mark.parametrize("s", [3, 4, 5, 6, 7, 8])
def test_trees_are_exact(s):
    # chain v_{i,i+1} plus all boundary variables: the factor graph is a tree
    rng = np.random.default_rng(s)
    L = _sym(rng, s)
    valid = np.zeros((s, s), dtype=bool)
    for i in range(s):
        valid[i, i] = True
        if i + 1 < s:
            valid[i, i + 1] = valid[i + 1, i] = True
    hist = bp.run_bp(L, 2 * s + 2, valid=valid)
    lam = hist[-1][1]
    exact = brute.exact_marginal_llrs(L, valid)
    assert np.allclose(lam[valid], exact[valid], rtol=1e-10, atol=1e-10)


def test_star_tree_is_exact():
    # one hub detector paired with every other one, no other pair variables
    s = 6
    rng = np.random.default_rng(42)
    L = _sym(rng, s)
    valid = np.eye(s, dtype=bool)
    valid[0, :] = valid[:, 0] = True
    lam = bp.run_bp(L, 8, valid=valid)[-1][1]
    exact = brute.exact_marginal_llrs(L, valid)
    assert np.allclose(lam[valid], exact[valid], rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("seed", range(6))
def test_single_loop_signs_match_exact_marginals(seed):
    # K_3 with its boundary variables is one loop c1-v12-c2-v23-c3-v13 with pendant
    # leaves v_ii; for binary variables on a single loop the BP belief and the true
    # marginal favour the same state (Weiss 2000).  The theorem covers the variables on
    # the loop; the pendant boundary variables can differ when their LLR is near 0.
    rng = np.random.default_rng(100 + seed)
    L = _sym(rng, 3, -5.0, -0.2)
    hist = bp.run_bp(L, 200)
    lam = hist[-1][1]
    assert np.allclose(hist[-1][0], hist[-2][0], atol=1e-9)  # reached a fixed point
    exact = brute.exact_marginal_llrs(L)
    for i, j in ((0, 1), (0, 2), (1, 2)):
        assert (lam[i, j] > 0) == (exact[i, j] > 0)


def test_ring_with_masked_chords_signs():
    s = 5
    valid = np.eye(s, dtype=bool)
    for i in range(s):
        j = (i + 1) % s
        valid[i, j] = valid[j, i] = True
    for seed in range(4):
        rng = np.random.default_rng(7 + seed)
        L = _sym(rng, s, -4.0, -0.3)
        hist = bp.run_bp(L, 300, valid=valid)
        assert np.allclose(hist[-1][0][valid], hist[-2][0][valid], atol=1e-8)
        exact = brute.exact_marginal_llrs(L, valid)
        lam = hist[-1][1]
        for i in range(s):
            j = (i + 1) % s
            assert (lam[i, j] > 0) == (exact[i, j] > 0)


def test_matching_counts():
    # involutions of s points (matchings with a boundary): 1, 2, 4, 10, 26, 76, 232, 764
    assert [len(brute.matchings(s)) for s in range(1, 9)] == [1, 2, 4, 10, 26, 76, 232, 764]


def test_worked_example_inference():
    ex = json.load(open(GOLDEN))
    s = ex["s"]
    lam = np.full((s, s), -np.inf)
    for key, pv in ex["prob_v1"].items():
        i, j = (int(x) - 1 for x in key.split(","))
        lam[i, j] = lam[j, i] = math.log(pv / (1 - pv))
    V, conv = bp.decide(lam)
    assert conv == ex["marginalization_converged"]
    assert [(i + 1, j + 1) for (i, j) in bp.matching_from(V)] == [tuple(x) for x in ex["marginalization"]]
    picks = bp.forced_convergence(lam)
    assert [(i + 1, j + 1) for (i, j) in picks] == [tuple(x) for x in ex["forced_pick_order"]]
