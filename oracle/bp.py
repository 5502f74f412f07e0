"""Sum-product belief propagation on the per-shot matching factor graph (oracle side).

Test infrastructure only: nothing in the product path imports this module.

For a shot with s unsatisfied detectors the factor graph F = (V, C, A) of Sec.
"Bipartite Graph Representation" has one factor c_i per unsatisfied detector and one
binary variable v_ij (i <= j) per decoding-graph edge; v_ij (i != j) touches c_i and c_j,
v_ii (the edge to the boundary) touches c_i only.  Factor c_i is 1 iff exactly one of
its variables is 1 (Eq. syndrome factors).  The prior LLR of v_ij is l_ij (Eq. priorllr).

Log-domain sum-product (Sec. "Belief Propagation"), flooding schedule, all in FP64:
  M[i, j]  = message from factor c_i to variable v_ij, M = 0 before iteration 1;
  Q[i, k]  = l_ik + M[k, i] / alpha   (k != i), Q[i, i] = l_ii   (variable -> factor c_i);
  M'[i, j] = -max*_{k != j} Q[i, k]  with max*(x_1..x_n) = ln sum exp(x_k), evaluated
             directly on each leave-one-out set with a max shift; an empty set gives
             max* = -inf and so M' = +inf;
  lambda_ij = l_ij + (M'[i, j] + M'[j, i]) (i != j), lambda_ii = l_ii + M'[i, i]
             (Eq. marginalization).
One iteration = one factor update of every message from the previous ones, followed by
the posterior; "T iterations" means T such updates.  alpha = 1 is plain BP; alpha != 1
is the memory variant of Sec. "BP Improvements".

Inference (Sec. "Forced convergence"):
  * marginalization keeps v iff lambda_v > 0 (strict);
  * convergence: every factor has exactly one kept variable (Sec. "Checking convergence");
  * forced convergence, read as a global greedy: all variables sorted by lambda
    descending (ties: smaller i, then smaller j), each accepted iff all its endpoints
    are still unmatched.  v_ii matches i to the boundary.

A `valid` mask (s x s, symmetric) removes variables from the factor graph; it only serves
the exactness checks on tree- and cycle-shaped graphs.  Decoding always uses the full
graph.
"""
import math

import numpy as np


def loo_lse(row, valid_row):
    """out[j] = ln sum_{k != j, valid} exp(row[k]), computed per set with a max shift."""
    s = row.shape[0]
    out = np.full(s, -np.inf)
    for j in range(s):
        keep = valid_row.copy()
        keep[j] = False
        vals = row[keep]
        if vals.size == 0:
            continue
        m = vals.max()
        if m == -np.inf:
            continue
        out[j] = m + math.log(float(np.sum(np.exp(vals - m))))
    return out


def loo_lse_rows(Q, valid):
    """Row-wise leave-one-out max* of a whole matrix (same definition as `loo_lse`)."""
    s = Q.shape[0]
    out = np.full((s, s), -np.inf)
    eye = np.eye(s, dtype=bool)
    for i in range(s):
        sets = np.where(valid[i][None, :] & ~eye, Q[i][None, :], -np.inf)  # sets[j, k]
        m = sets.max(axis=1)
        ok = m > -np.inf
        if not ok.any():
            continue
        with np.errstate(invalid="ignore", over="ignore"):
            sh = np.exp(sets[ok] - m[ok, None])
        out[i, ok] = m[ok] + np.log(sh.sum(axis=1))
    return out


def full_valid(s):
    return np.ones((s, s), dtype=bool)


def var_to_factor(L, M, alpha=1.0, valid=None):
    s = L.shape[0]
    if valid is None:
        valid = full_valid(s)
    with np.errstate(invalid="ignore"):
        Q = L + M.T / alpha
    np.fill_diagonal(Q, np.diag(L))
    Q[~valid] = -np.inf
    return Q


def factor_update(L, M, alpha=1.0, valid=None):
    s = L.shape[0]
    if valid is None:
        valid = full_valid(s)
    Q = var_to_factor(L, M, alpha, valid)
    return -loo_lse_rows(Q, valid)


def posterior(L, M, valid=None):
    s = L.shape[0]
    if valid is None:
        valid = full_valid(s)
    with np.errstate(invalid="ignore"):
        lam = L + (M + M.T)
    np.fill_diagonal(lam, np.diag(L) + np.diag(M))
    lam[~valid] = -np.inf
    return lam


def decide(lam):
    """Marginalization: (kept-variable matrix, converged flag)."""
    V = lam > 0
    counts = V.sum(axis=1)
    return V, bool(np.all(counts == 1))


def matching_from(V):
    s = V.shape[0]
    return [(i, j) for i in range(s) for j in range(i, s) if V[i, j]]


def forced_convergence(lam, valid=None):
    """Global greedy matching on the posteriors; returns pairs in pick order."""
    s = lam.shape[0]
    if valid is None:
        valid = full_valid(s)
    cand = [(-float(lam[i, j]), i, j) for i in range(s) for j in range(i, s) if valid[i, j]]
    cand.sort()
    matched = [False] * s
    picks = []
    for _, i, j in cand:
        if matched[i] or matched[j]:
            continue
        matched[i] = True
        matched[j] = True
        picks.append((i, j))
    return picks


def forced_convergence_static(lam, valid=None):
    """Forced convergence with the paper's static partition (Sec. "Forced convergence"):
    the variables are partitioned into one block per factor, v_ij (i <= j) belonging to the
    block of c_i (the partition of the full detector set, each pair owned by its smaller
    detector, restricted to the shot); each block's maximum (ties: smaller j) represents its
    factor; the representatives are ordered by posterior, descending (ties: smaller i), and
    processed in that order: a factor not yet matched is matched along its representative
    v_ik, to the boundary if k = i, else together with c_k.  The paper does not say what
    happens when c_k has already been matched; then c_i is matched to the boundary (always
    available, so the result is a valid matching).  Returns pairs in pick order."""
    s = lam.shape[0]
    if valid is None:
        valid = full_valid(s)
    rep = []
    for i in range(s):
        best, bj = -math.inf, i
        for j in range(i, s):
            if valid[i, j] and (lam[i, j] > best or (bj == i and best == -math.inf)):
                best, bj = float(lam[i, j]), j
        rep.append((best, bj))
    order = sorted(range(s), key=lambda i: (-rep[i][0], i))
    matched = [False] * s
    picks = []
    for i in order:
        if matched[i]:
            continue
        k = rep[i][1]
        if k == i or matched[k]:
            picks.append((i, i))
            matched[i] = True
        else:
            picks.append((i, k))
            matched[i] = matched[k] = True
    return picks


def static_margin(lam, valid=None):
    """Smallest posterior gap that decides forced_convergence_static: within a block, its
    maximum against the block's next largest; across blocks, adjacent representatives in
    the processing order (inf if there are none)."""
    s = lam.shape[0]
    if valid is None:
        valid = full_valid(s)
    margin = math.inf
    reps = []
    for i in range(s):
        vals = sorted((float(lam[i, j]) for j in range(i, s) if valid[i, j]), reverse=True)
        if len(vals) >= 2:
            margin = min(margin, vals[0] - vals[1])
        if vals:
            reps.append(vals[0])
    reps.sort(reverse=True)
    for a, b in zip(reps, reps[1:]):
        margin = min(margin, a - b)
    return margin


# Perturbation size up to which decision_margin and the first-stage margin of B-BP4MF check
# that a decision cannot change: at least the largest tolerance the tests use (1e-2).
ROBUST_AT = 0.05


def greedy_margin(lam, valid=None):
    """Smallest posterior gap that decides forced_convergence's greedy matching.

    Processing two variables that share no endpoint in the other order gives the same
    matching, so the result can change under a perturbation of the posteriors only through
    an accepted variable v and a variable w that shares an endpoint with v and is still
    available (both endpoints unmatched) when v is accepted: the margin is the smallest
    lambda_v - lambda_w over such pairs (inf if there are none)."""
    s = lam.shape[0]
    if valid is None:
        valid = full_valid(s)
    cand = [(-float(lam[i, j]), i, j) for i in range(s) for j in range(i, s) if valid[i, j]]
    cand.sort()
    matched = [False] * s
    margin = math.inf
    for negl, i, j in cand:
        if matched[i] or matched[j]:
            continue
        best = -math.inf
        for a in {i, j}:
            for k in range(s):
                if matched[k] or not valid[min(a, k), max(a, k)]:
                    continue
                if (min(a, k), max(a, k)) == (i, j):
                    continue
                best = max(best, float(lam[min(a, k), max(a, k)]))
        if best > -math.inf:
            margin = min(margin, -negl - best)
        matched[i] = True
        matched[j] = True
    return margin


def decision_margin(lam, valid=None):
    """Smallest |lambda| that can decide one iteration's marginalization outcome.

    A converged iteration outputs its kept set, so every sign counts: min |lambda|.  An
    unconverged one only contributes its convergence status, which a sign change moves by
    at most two rows; if more rows violate the exactly-one rule than twice the number of
    posteriors within ROBUST_AT of zero, no perturbation below ROBUST_AT can make it
    converge, and the margin is at least ROBUST_AT."""
    s = lam.shape[0]
    if valid is None:
        valid = full_valid(s)
    iu = np.triu_indices(s)
    vals = np.abs(lam[iu])[valid[iu]]
    m = float(np.min(vals)) if vals.size else math.inf
    V, conv = decide(lam)
    if conv:
        return m
    viol = int(np.sum(V.sum(axis=1) != 1))
    near = int(np.sum(vals < ROBUST_AT))
    return max(m, ROBUST_AT) if viol > 2 * near else m


def order_margin(lam):
    """Smallest gap between two different posteriors of the upper triangle (inf if < 2)."""
    s = lam.shape[0]
    vals = np.sort(lam[np.triu_indices(s)])
    vals = vals[np.isfinite(vals)]
    if vals.size < 2:
        return math.inf
    return float(np.min(np.diff(vals)))


def run_bp(L, T, alpha=1.0, valid=None):
    """Plain T-iteration BP; returns the list of (M, lambda) after every iteration."""
    s = L.shape[0]
    M = np.zeros((s, s))
    out = []
    for _ in range(T):
        M = factor_update(L, M, alpha, valid)
        out.append((M, posterior(L, M, valid)))
    return out
