"""Shortest-path priors on a detector graph (oracle side).

Test infrastructure only: nothing in the product path imports this module.

Eq. (two-syn var factors) gives each decoding-graph edge (i, j) the prior
rho_ij(1) = (p/(1-p))^{w_ij}, w_ij the weight of the lowest-weight error matching the
two unsatisfied checks (i == j: to the boundary).  For a general detector graph the
same quantity is omega_ij = exp(-W_ij), W_ij the shortest path under edge weights
W_e = ln((1-q_e)/q_e); under code-capacity noise W_e is one hop times ln((1-p)/p),
which reproduces the printed formula exactly.  The prior LLR of Eq. (priorllr) is
l_ij = ln(omega/(1-omega)) = -W - log1p(-exp(-W)).

Conventions shared with the product (an interface, stated once here):
  * parallel edges: the smaller W is kept, ties go to the edge with observable bit 0;
  * pair paths may not pass through the boundary node (Sec. "Correlated decoding" prefers
    the non-quotient graph); the boundary is a sink;
  * Dijkstra finalises nodes in (distance, node index) order and changes a predecessor
    only on a strict improvement; the observable parity of a path is accumulated along
    the predecessor tree; W_ij for i < j and its parity come from the search rooted at i.
"""
import heapq
import math

import numpy as np


def edge_weights_circuit(g):
    return [math.log((1.0 - q) / q) for (_, _, _, q) in g.edges]


def edge_weights_hops(g):
    return [1.0 for _ in g.edges]


def adjacency(g, weights):
    best = {}
    for (u, v, ob, _), w in zip(g.edges, weights):
        cur = best.get((u, v))
        if cur is None or (w, ob) < cur:
            best[(u, v)] = (w, ob)
    adj = [[] for _ in range(g.n_det + 1)]
    for (u, v), (w, ob) in sorted(best.items()):
        adj[u].append((v, w, ob))
        adj[v].append((u, w, ob))
    return adj


def dijkstra(adj, src, n_det, through_boundary=False):
    n = len(adj)
    dist = [math.inf] * n
    par = [0] * n
    done = [False] * n
    dist[src] = 0.0
    heap = [(0.0, src)]
    while heap:
        du, u = heapq.heappop(heap)
        if done[u]:
            continue
        done[u] = True
        if u == n_det and not through_boundary:
            continue
        for v, w, ob in adj[u]:
            nd = du + w
            if nd < dist[v]:
                dist[v] = nd
                par[v] = par[u] ^ ob
                heapq.heappush(heap, (nd, v))
    return dist, par


def all_pairs(g, weights, through_boundary=False, sources=None):
    """W (n x n, diagonal = boundary distance) and observable parity tables."""
    n = g.n_det
    adj = adjacency(g, weights)
    W = np.full((n, n), np.inf)
    P = np.zeros((n, n), dtype=np.uint8)
    srcs = range(n) if sources is None else sources
    for i in srcs:
        dist, par = dijkstra(adj, i, n, through_boundary)
        W[i, i] = dist[n]
        P[i, i] = par[n]
        for j in range(i + 1, n):
            W[i, j] = dist[j]
            P[i, j] = par[j]
    iu = np.triu_indices(n, 1)
    W[(iu[1], iu[0])] = W[iu]
    P[(iu[1], iu[0])] = P[iu]
    return W, P


def prior_llr(W):
    """l = ln(omega/(1-omega)) with omega = exp(-W), elementwise (Eq. priorllr)."""
    W = np.asarray(W, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        out = -W - np.log1p(-np.exp(-W))
    out[np.isinf(W)] = -np.inf
    return out


class Tables:
    """Per-graph tables: W, l, parity (n x n), the graph and its edge list."""

    def __init__(self, g, W, P):
        self.g = g
        self.n_det = g.n_det
        self.W = W
        self.P = P
        self.L = prior_llr(W)


def code_capacity_tables(g, p_prior, through_boundary=False):
    hops, P = all_pairs(g, edge_weights_hops(g), through_boundary)
    c = math.log((1.0 - p_prior) / p_prior)
    return Tables(g, hops * c, P)


def circuit_tables(g, through_boundary=False):
    W, P = all_pairs(g, edge_weights_circuit(g), through_boundary)
    return Tables(g, W, P)
