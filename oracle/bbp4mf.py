"""B-BP4MF under code-capacity noise (oracle side).

Test infrastructure only: nothing in the product path imports this module.

Sec. "Correlated decoding" and Sec. "Belief-BP4MF (B-BP4MF)": a first stage runs
quaternary BP on the code's Tanner graph; if its hard decision reproduces the syndrome,
that decision is the output.  Otherwise the qubit posteriors reweight the decoding graph:
every data qubit is an edge of G_D between its one or two checks (one check: to the
boundary), with weight ln((1 - P_e)/P_e) where P_e is the posterior probability that the
qubit carries an error component detected by that check type; Dijkstra from every
unsatisfied check gives the shot's pair and boundary weights, hence its priors
(Eq. two-syn var factors with the reweighted w), and BP4MF runs on them.

Posteriors above one half.  The paper does not say how an edge whose posterior P exceeds
1/2 enters Dijkstra's algorithm (its weight ln((1-P)/P) would be negative, and an undirected
graph with a negative edge has no shortest paths).  The reading here is the one of
matching decoders with negative weights (Belief-matching, which Sec. "Correlated decoding"
emulates): such an edge is taken as present.  Its endpoints' syndrome bits are flipped, its
observable bit goes into a base parity that is added to the decoded parity, and it enters
the graph with the complementary probability 1 - P, i.e. weight |ln((1-P)/P)|.  This is an
exact change of variables of the edge error model (the error E has the probability of
E + {e} under P_e -> 1 - P_e, and the syndrome of E is that of E + {e} plus the edge's
endpoints), so it moves no probability mass.  Weights are still floored at MIN_WEIGHT,
which now only acts at P = 1/2 exactly.

Quaternary BP (the paper cites it without restating it; this is the standard form with
one scalar message per Tanner edge):
  * qubit v has prior p_v(I) = 1 - p, p_v(X) = p_v(Y) = p_v(Z) = p / 3;
  * <E, c> = 1 iff Pauli E anticommutes with check c (X-checks see Z and Y, Z-checks see
    X and Y); z_c is the check's syndrome bit;
  * qubit -> check:  mu_vc = ln( sum_{<E,c>=0} q_vc(E) / sum_{<E,c>=1} q_vc(E) ) with
    q_vc(E) = p_v(E) prod_{c' != c} exp(-<E,c'> Delta_c'v);
  * check -> qubit:  Delta_cv = (-1)^z_c 2 atanh( prod_{v' != v} tanh(mu_v'c / 2) );
  * posterior q_v(E) = p_v(E) prod_c exp(-<E,c> Delta_cv), decision argmax_E q_v(E) (ties:
    I, X, Y, Z order); flooding schedule, Delta = 0 before iteration 1; converged when the
    decision's syndrome equals the observed one (checked after every iteration, first
    converged iteration kept).
"""
import math

import numpy as np

from . import bp
from .decoders import bp4mf
from .graph import adjacency, dijkstra, prior_llr
from .surface import parity_check_matrices

PAULIS = ("I", "X", "Y", "Z")
# anticommutation of E with an X-type / Z-type check
ANTI_X = np.array([0, 0, 1, 1])  # I, X, Y, Z vs X-check: Y, Z anticommute
ANTI_Z = np.array([0, 1, 1, 0])  # vs Z-check: X, Y anticommute
# Smallest reweighted edge weight: a posterior of exactly one half gives weight 0, which
# would make the pair prior infinite; the floor keeps it large but finite.
MIN_WEIGHT = 2.0 ** -20


def tanner(code):
    """Checks as (type, qubits) with X-checks first, then Z-checks (each in check order)."""
    out = [("X", list(qs)) for (_, _, qs) in code.x_checks]
    out += [("Z", list(qs)) for (_, _, qs) in code.z_checks]
    return out


def qbp(checks, n, syndrome, p, T, stop=True, margin=None):
    """Quaternary BP.  `checks` = [(type, qubits)], `syndrome` = bits per check.
    Returns (posterior [n, 4], decision [n] of Pauli indices, converged, iterations); with
    stop=False all T iterations run (used by the exactness checks).  `margin`, a list,
    receives per executed iteration the smallest relative gap (q1 - q2) / q1 between a
    qubit's two largest posteriors that can decide the outcome: any gap of an iteration
    whose decision reproduces the syndrome; for an unconverged iteration, whose only
    outcome is its convergence status, at least bp.ROBUST_AT when its mismatched checks
    outnumber 4 per qubit with a gap below bp.ROBUST_AT (one qubit's decision changes at
    most 4 checks)."""
    prior = np.array([1.0 - p, p / 3.0, p / 3.0, p / 3.0])
    anti = [ANTI_X if ty == "X" else ANTI_Z for ty, _ in checks]
    edges = [(c, v) for c, (_, qs) in enumerate(checks) for v in qs]
    delta = {e: 0.0 for e in edges}
    by_qubit = [[] for _ in range(n)]
    for c, v in edges:
        by_qubit[v].append(c)
    post = np.tile(prior, (n, 1))
    dec = np.zeros(n, dtype=int)
    gaps = np.zeros(n)
    conv = False
    it = 0
    for it in range(1, T + 1):
        mu = {}
        for c, v in edges:
            q = prior.copy()
            for c2 in by_qubit[v]:
                if c2 != c:
                    q = q * np.exp(-anti[c2] * delta[(c2, v)])
            mu[(c, v)] = math.log(q[anti[c] == 0].sum() / q[anti[c] == 1].sum())
        new = {}
        for c, v in edges:
            prod = 1.0
            for v2 in checks[c][1]:
                if v2 != v:
                    prod *= math.tanh(mu[(c, v2)] / 2.0)
            prod = min(max(prod, -1.0 + 1e-15), 1.0 - 1e-15)
            new[(c, v)] = (-1.0 if syndrome[c] else 1.0) * 2.0 * math.atanh(prod)
        delta = new
        for v in range(n):
            q = prior.copy()
            for c in by_qubit[v]:
                q = q * np.exp(-anti[c] * delta[(c, v)])
            post[v] = q / q.sum()
            dec[v] = int(np.argmax(q))
            if margin is not None:
                top = np.sort(q)[::-1]
                gaps[v] = (top[0] - top[1]) / top[0]
        synd = np.array([int(anti[c][dec[qs]].sum() % 2) for c, (_, qs) in enumerate(checks)])
        if margin is not None:
            mismatched = int((synd != np.asarray(syndrome, dtype=int)).sum())
            near = int((gaps < bp.ROBUST_AT).sum())
            g = float(gaps.min())
            margin.append(g if (mismatched == 0 or mismatched <= 4 * near) else max(g, bp.ROBUST_AT))
        if np.array_equal(synd, np.asarray(syndrome, dtype=int)):
            conv = True
            if stop:
                break
    return post, dec, conv, it


def flip_likely_edges(g, edge_prob, synd):
    """Takes every edge with probability above one half as present: returns the syndrome
    with their endpoints flipped (bool [n_det]), the XOR of their observable bits, and
    the number of flipped edges."""
    out = np.array(synd, dtype=bool).copy()
    base = 0
    n = 0
    for e, (u, v, ob, _) in enumerate(g.edges):
        if float(edge_prob[e]) > 0.5:
            out[u] ^= True
            if v < g.n_det:
                out[v] ^= True
            base ^= int(ob)
            n += 1
    return out, base, n


def edge_weight(prob):
    """|ln((1-P)/P)| of an edge (its complement when P > 1/2), floored at MIN_WEIGHT."""
    pe = min(max(float(prob), 1e-300), 1.0 - 1e-16)
    if pe > 0.5:
        pe = 1.0 - pe
    return max(math.log((1.0 - pe) / pe), MIN_WEIGHT)


def reweighted_tables(g, edge_prob, dets, through_boundary=False):
    """Shot priors from per-edge error probabilities: W, parity and l over the shot's
    unsatisfied detectors `dets` (W_ij for i < j from the search rooted at the smaller
    index, diagonal = boundary), same Dijkstra conventions as graph.py.  Edge weights are
    edge_weight(P) (edges above one half must already have been flipped out of the
    syndrome by flip_likely_edges)."""
    weights = [edge_weight(edge_prob[e]) for e in range(len(g.edges))]
    adj = adjacency(g, weights)
    s = len(dets)
    W = np.full((s, s), np.inf)
    P = np.zeros((s, s), dtype=np.uint8)
    for a, i in enumerate(dets):
        dist, par = dijkstra(adj, int(i), g.n_det, through_boundary)
        W[a, a] = dist[g.n_det]
        P[a, a] = par[g.n_det]
        for b in range(a + 1, s):
            W[a, b] = W[b, a] = dist[int(dets[b])]
            P[a, b] = P[b, a] = par[int(dets[b])]
    return W, P, prior_llr(W)


def bbp4mf_shot(code, graphs, synd_x_checks, synd_z_checks, p, T_q, T_bp, alpha=1.0):
    """One shot.  `graphs` = {"X": Z-check graph, "Z": X-check graph} (code_capacity_graph);
    synd_*: syndrome bits of the X-checks and of the Z-checks.  Returns dict with per-type
    predicted observable flips and whether the first stage converged."""
    checks = tanner(code)
    syndrome = list(synd_x_checks) + list(synd_z_checks)
    gaps = []
    post, dec, conv, it_q = qbp(checks, code.n, syndrome, p, T_q, margin=gaps)
    # decision margin: first-stage argmax gaps, the distance of every edge's posterior from
    # the flip threshold 1/2, and the second stage's BP4MF margin
    out = {"qbp_converged": conv, "qbp_iters": it_q, "margin_qbp": min(gaps) if gaps else math.inf,
           "margin_flip": math.inf, "margin_bp": math.inf}
    out["margin"] = out["margin_qbp"]
    if conv:
        ex = (dec == 1) | (dec == 2)   # X component
        ez = (dec == 2) | (dec == 3)   # Z component
        out["X"] = int(ex[code.zl].sum() % 2)
        out["Z"] = int(ez[code.xl].sum() % 2)
        return out
    for kind, synd in (("X", synd_z_checks), ("Z", synd_x_checks)):
        g = graphs[kind]
        comp = post[:, 1] + post[:, 2] if kind == "X" else post[:, 2] + post[:, 3]
        edge_prob = [comp[q] for q in g.unit_of_edge]
        out["margin_flip"] = min(out["margin_flip"], min(abs(float(x) - 0.5) for x in edge_prob))
        out["margin"] = min(out["margin"], out["margin_flip"])
        flipped, base, n_flip = flip_likely_edges(g, edge_prob, synd)
        out[kind + "_flipped"] = n_flip
        dets = np.flatnonzero(flipped)
        if len(dets) == 0:
            out[kind] = base
            continue
        W, P, L = reweighted_tables(g, edge_prob, dets)
        r = bp4mf(L, W, T_bp, alpha=alpha)
        par = base
        for i, j in r.matching:
            par ^= int(P[i, j])
        out[kind] = par
        out[kind + "_result"] = r
        out["margin_bp"] = min(out["margin_bp"], r.margin)
        out["margin"] = min(out["margin"], r.margin)
    return out


def brute_posteriors(checks, n, syndrome, p):
    """Exact qubit posteriors P(E_v | syndrome) by enumerating all 4^n errors (n <= 6)."""
    prior = np.array([1.0 - p, p / 3.0, p / 3.0, p / 3.0])
    anti = [ANTI_X if ty == "X" else ANTI_Z for ty, _ in checks]
    post = np.zeros((n, 4))
    for code_word in range(4 ** n):
        E = [(code_word >> (2 * v)) & 3 for v in range(n)]
        ok = all(int(sum(anti[c][E[v]] for v in qs) % 2) == syndrome[c] for c, (_, qs) in enumerate(checks))
        if not ok:
            continue
        w = 1.0
        for v in range(n):
            w *= prior[E[v]]
        for v in range(n):
            post[v, E[v]] += w
    return post / post.sum(axis=1, keepdims=True)
