"""Pins for shortest-path weights, parities and prior LLRs of the oracle."""
import math

import networkx as nx
import numpy as np
import pytest
from scipy.sparse.csgraph import floyd_warshall

from oracle.circuit import Noise, circuit_graph
from oracle.graph import (adjacency, all_pairs, circuit_tables, code_capacity_tables,
                          edge_weights_circuit, prior_llr)
from oracle.surface import DetGraph, code_capacity_graph, rotated_code


def _fw_reference(g, weights):
    """Floyd-Warshall on detectors only (so no pair path uses the boundary), then the
    boundary distance as min over boundary edges."""
    n = g.n_det
    D = np.full((n, n), np.inf)
    np.fill_diagonal(D, 0.0)
    bnd = np.full(n, np.inf)
    for (u, v, _, _), w in zip(g.edges, weights):
        if v == n:
            bnd[u] = min(bnd[u], w)
        else:
            D[u, v] = min(D[u, v], w)
            D[v, u] = min(D[v, u], w)
    F = floyd_warshall(D)
    out = F.copy()
    for i in range(n):
        out[i, i] = np.min(F[i] + bnd)
    return out


@pytest.mark.parametrize("d", [3, 5])
def test_dijkstra_matches_floyd_warshall_circuit(d):
    g, _, _ = circuit_graph(d, Noise(0.006))
    w = edge_weights_circuit(g)
    W, _ = all_pairs(g, w)
    ref = _fw_reference(g, w)
    assert np.allclose(W, ref, rtol=1e-12, atol=0)


def test_dijkstra_matches_floyd_warshall_random_graphs():
    rng = np.random.default_rng(3)
    for _ in range(20):
        n = int(rng.integers(2, 12))
        edges = []
        for u in range(n):
            for v in range(u + 1, n + 1):
                if rng.random() < 0.35:
                    edges.append((u, v, int(rng.integers(0, 2)), float(rng.uniform(0.01, 0.3))))
        g = DetGraph(n, edges)
        w = [math.log((1 - q) / q) for (_, _, _, q) in edges]
        W, _ = all_pairs(g, w)
        assert np.allclose(np.where(np.isinf(W), -1, W),
                           np.where(np.isinf(_fw_reference(g, w)), -1, _fw_reference(g, w)), rtol=1e-12)


@pytest.mark.parametrize("d", [3, 5, 7])
def test_code_capacity_weights_are_hops_times_constant(d):
    p = 0.07
    for kind in ("X", "Z"):
        g = code_capacity_graph(rotated_code(d), kind)
        tb = code_capacity_tables(g, p)
        G = nx.Graph()
        G.add_nodes_from(range(g.n_det))
        for (u, v, _, _) in g.edges:
            if v < g.n_det:
                G.add_edge(u, v)
        hops = dict(nx.all_pairs_shortest_path_length(G))
        bnd = {u for (u, v, _, _) in g.edges if v == g.n_det}
        c = math.log((1 - p) / p)
        for i in range(g.n_det):
            for j in range(g.n_det):
                if i == j:
                    h = min(hops[i][k] for k in bnd) + 1
                else:
                    h = hops[i][j]
                assert tb.W[i, j] == pytest.approx(h * c, rel=1e-14)
                # Eq. (two-syn var factors): rho(1) = (p/(1-p))^w, l = ln(rho(1)/rho(0))
                rho1 = (p / (1 - p)) ** h
                assert tb.L[i, j] == pytest.approx(math.log(rho1 / (1 - rho1)), rel=1e-12)


def _explicit_path(adj, src, dst, n_det):
    """Re-run the tie-ruled Dijkstra with predecessors and return the path's edges."""
    import heapq
    n = len(adj)
    dist = [math.inf] * n
    pred = [None] * n
    done = [False] * n
    dist[src] = 0.0
    heap = [(0.0, src)]
    while heap:
        du, u = heapq.heappop(heap)
        if done[u]:
            continue
        done[u] = True
        if u == n_det:
            continue
        for v, w, ob in adj[u]:
            if du + w < dist[v]:
                dist[v] = du + w
                pred[v] = (u, ob)
                heapq.heappush(heap, (du + w, v))
    path = []
    v = dst
    while v != src:
        u, ob = pred[v]
        path.append((u, v, ob))
        v = u
    return path


@pytest.mark.parametrize("which", ["cc", "circuit"])
def test_parity_table_matches_explicit_paths(which):
    if which == "cc":
        g = code_capacity_graph(rotated_code(5), "X")
        tb = code_capacity_tables(g, 0.05)
        w = [1.0] * len(g.edges)
    else:
        g, _, _ = circuit_graph(3, Noise(0.005))
        tb = circuit_tables(g)
        w = edge_weights_circuit(g)
    adj = adjacency(g, w)
    n = g.n_det
    for i in range(n):
        for j in range(i, n):
            dst = n if i == j else j
            path = _explicit_path(adj, i, dst, n)
            ends = np.zeros(n + 1, dtype=int)
            par = 0
            for (u, v, ob) in path:
                ends[u] ^= 1
                ends[v] ^= 1
                par ^= ob
            want = np.zeros(n + 1, dtype=int)
            want[i] ^= 1
            want[dst] ^= 1
            assert (ends == want).all()
            assert par == tb.P[i, j]


def test_pair_parity_is_path_independent_code_capacity():
    # A cycle that avoids the boundary crosses supp(Z_L) an even number of times, so the
    # parity of a pair path does not depend on which shortest path is taken.
    g = code_capacity_graph(rotated_code(5), "X")
    n = g.n_det
    G = nx.MultiGraph()
    for (u, v, ob, _) in g.edges:
        if v < n:
            G.add_edge(u, v, ob=ob)
    for cyc in nx.cycle_basis(nx.Graph(G)):
        par = 0
        for a, b in zip(cyc, cyc[1:] + cyc[:1]):
            par ^= min(d["ob"] for d in G.get_edge_data(a, b).values())
        assert par == 0


def test_prior_llr_closed_form():
    W = np.array([0.5, 1.0, 3.0, 30.0, np.inf])
    got = prior_llr(W)
    om = np.exp(-W[:4])
    assert np.allclose(got[:4], np.log(om / (1 - om)), rtol=1e-12)
    assert got[4] == -np.inf
