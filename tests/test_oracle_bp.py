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


# ------------------------------------------------------------------ decision margins
#
# The GPU/oracle comparison exempts a shot only where the oracle's margin says a rounding
# could change the outcome, so the margins must be sound (no perturbation below them
# changes the outcome) and tight (some perturbation slightly above changes it).


def _random_lambda(s, rng, ties):
    lam = rng.normal(0.0, 2.0, size=(s, s))
    lam = np.triu(lam) + np.triu(lam, 1).T
    if ties:
        # exact ties between variables that share an endpoint
        lam[0, 1] = lam[1, 0] = lam[0, 2] = lam[2, 0]
    return lam


def _perturb(lam, delta):
    out = lam + np.triu(delta) + np.triu(delta, 1).T
    return out


@pytest.mark.parametrize("seed", range(6))
def test_greedy_margin_is_sound_and_tight(seed):
    rng = np.random.default_rng(seed)
    s = 6 + seed % 3
    lam = _random_lambda(s, rng, ties=seed % 2 == 1)
    m = bp.greedy_margin(lam)
    ref = bp.forced_convergence(lam)
    if seed % 2 == 1:
        assert m == 0.0 or m > 0.0   # the tie may or may not decide; soundness below holds
    for _ in range(300):
        d = rng.uniform(-1, 1, size=(s, s)) * (0.49 * m if np.isfinite(m) else 1.0)
        assert sorted(bp.forced_convergence(_perturb(lam, d))) == sorted(ref)
    # never looser than the gap between any two posteriors
    assert m >= bp.order_margin(lam)


def test_greedy_margin_is_tight_on_a_decisive_pair():
    # (0, 1) and (0, 2) compete for factor 0 at the top of the order: their gap decides
    s = 5
    lam = np.full((s, s), -6.0)
    lam[0, 1] = lam[1, 0] = 5.0
    lam[0, 2] = lam[2, 0] = 4.9
    lam[3, 4] = lam[4, 3] = 2.0
    for i in range(s):
        lam[i, i] = -3.0 - i
    m = bp.greedy_margin(lam)
    assert abs(m - 0.1) < 1e-12
    ref = sorted(bp.forced_convergence(lam))
    d = np.zeros((s, s))
    d[0, 1], d[0, 2] = -0.051, 0.051
    assert sorted(bp.forced_convergence(_perturb(lam, d))) != ref


@pytest.mark.parametrize("seed", range(6))
def test_decision_margin_is_sound(seed):
    rng = np.random.default_rng(100 + seed)
    s = 5 + seed % 3
    if seed < 3:
        lam = _random_lambda(s, rng, ties=False)
    else:
        # a converged pattern (a perfect matching of positive posteriors) plus noise
        lam = -np.abs(rng.normal(3.0, 1.0, size=(s, s)))
        lam = np.triu(lam) + np.triu(lam, 1).T
        for i in range(0, s - 1, 2):
            lam[i, i + 1] = lam[i + 1, i] = abs(rng.normal(0.5, 0.3))
        if s % 2:
            lam[s - 1, s - 1] = 0.7
    m = bp.decision_margin(lam)
    V0, c0 = bp.decide(lam)
    assert m > 0
    for _ in range(300):
        d = rng.uniform(-1, 1, size=(s, s)) * 0.99 * min(m, 10.0)
        V, c = bp.decide(_perturb(lam, d))
        assert c == c0
        if c0:
            assert np.array_equal(V, V0)


def test_worked_example_static_partition():
    # the paper's static partition (each pair in the block of its smaller factor) reproduces
    # the worked example's pick order too: block maxima v14 (c1), v22 (c2), v33 (c3), v44
    # (c4); c1 takes c4 along v14, then c3 and c2 go to the boundary
    ex = json.load(open(GOLDEN))
    s = ex["s"]
    lam = np.full((s, s), -np.inf)
    for key, pv in ex["prob_v1"].items():
        i, j = (int(x) - 1 for x in key.split(","))
        lam[i, j] = lam[j, i] = math.log(pv / (1 - pv))
    picks = bp.forced_convergence_static(lam)
    assert [(i + 1, j + 1) for (i, j) in picks] == [tuple(x) for x in ex["forced_pick_order"]]


@pytest.mark.parametrize("seed", range(8))
def test_static_partition_gives_a_valid_matching_and_sound_margin(seed):
    rng = np.random.default_rng(300 + seed)
    s = 3 + seed
    lam = _random_lambda(s, rng, ties=False)
    picks = bp.forced_convergence_static(lam)
    covered = sorted(x for i, j in picks for x in ({i, j}))
    assert covered == list(range(s))           # every factor matched exactly once
    # each pick is its factor's block maximum, or the boundary when that partner was taken
    for i, j in picks:
        blk = [lam[i, k] for k in range(i, s)]
        assert j == i or lam[i, j] == max(blk)
    m = bp.static_margin(lam)
    for _ in range(200):
        d = rng.uniform(-1, 1, size=(s, s)) * 0.49 * m
        assert sorted(bp.forced_convergence_static(_perturb(lam, d))) == sorted(picks)


def test_static_partition_equals_greedy_without_conflicts():
    # when every factor's block maximum leads to an unmatched partner in processing order,
    # both readings pick the same variables (a diagonal-dominant case)
    s = 5
    lam = np.full((s, s), -5.0)
    for i in range(s):
        lam[i, i] = 1.0 + i
    assert sorted(bp.forced_convergence_static(lam)) == sorted(bp.forced_convergence(lam))
