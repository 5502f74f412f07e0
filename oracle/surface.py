"""Surface code geometry (rotated and unrotated) and code-capacity decoding graphs
(oracle side).

Test infrastructure only: nothing in the product path imports this module.

Rotated layout (one fixed convention, shared as an interface with the product):
  * data qubit (r, c), r, c in [0, d), index r*d + c;
  * a plaquette is named by its north-west corner (pr, pc), pr, pc in [-1, d-1], and
    covers the data qubits (pr, pc), (pr, pc+1), (pr+1, pc), (pr+1, pc+1) that exist;
  * plaquette type is X when (pr + pc) is even, Z when odd (checkerboard);
  * all four-qubit plaquettes are kept; two-qubit plaquettes are kept on the top and
    bottom edges when they are Z-type and on the left and right edges when X-type;
  * Z_L is Z on column c = 0 and X_L is X on row r = 0.

Unrotated layout: a (2d-1) x (2d-1) grid; data qubits at (r, c) with r + c even, numbered
row-major; Z-checks at (r odd, c even) and X-checks at (r even, c odd), each acting on its
N, S, W, E neighbours inside the grid; Z_L is Z on row 0 of the data, X_L is X on column 0.

CNOT schedules (the order in which a check's ancilla meets its data qubits; None = no
qubit in that step):
  rotated:   X-checks NW, SW, NE, SE; Z-checks NW, NE, SW, SE;
  unrotated: X-checks N, W, E, S;     Z-checks N, E, W, S.

The paper (Sec. "MWPM on the surface code") decodes X and Z errors separately on the
decoding graph of the matching checks.  "Type X" below means X errors detected by the
Z-checks, with the observable flipped by qubits in supp(Z_L); "type Z" is the mirror.
Checks of each type are numbered by (pr, pc) ascending.
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class SurfaceCode:
    d: int
    z_checks: list  # [(row, col, [qubits])] sorted by (row, col)
    x_checks: list
    zl: list        # qubits in supp(Z_L)
    xl: list        # qubits in supp(X_L)
    n: int = 0
    z_sched: list = None  # per Z-check: 4 qubits (or None) in CNOT order
    x_sched: list = None
    family: str = "rotated"


RotatedCode = SurfaceCode


def rotated_code(d):
    if d < 2:
        raise ValueError("distance must be at least 2")
    z_checks, x_checks = [], []
    for pr in range(-1, d):
        for pc in range(-1, d):
            corners = [(pr, pc), (pr, pc + 1), (pr + 1, pc), (pr + 1, pc + 1)]
            qs = [r * d + c for (r, c) in corners if 0 <= r < d and 0 <= c < d]
            kind = "X" if (pr + pc) % 2 == 0 else "Z"
            if len(qs) == 4:
                keep = True
            elif len(qs) == 2:
                top_bottom = pr in (-1, d - 1)
                keep = (kind == "Z") if top_bottom else (kind == "X")
            else:
                keep = False
            if keep:
                (z_checks if kind == "Z" else x_checks).append((pr, pc, qs))
    zl = [r * d + 0 for r in range(d)]
    xl = [0 * d + c for c in range(d)]

    def sched(checks, order):
        out = []
        for pr, pc, _ in checks:
            row = []
            for dr, dc in order:
                r, c = pr + dr, pc + dc
                row.append(r * d + c if 0 <= r < d and 0 <= c < d else None)
            out.append(row)
        return out

    nw, sw, ne, se = (0, 0), (1, 0), (0, 1), (1, 1)
    return SurfaceCode(d, z_checks, x_checks, zl, xl, d * d,
                       sched(z_checks, [nw, ne, sw, se]), sched(x_checks, [nw, sw, ne, se]), "rotated")


def unrotated_code(d):
    if d < 2:
        raise ValueError("distance must be at least 2")
    L = 2 * d - 1
    index = {}
    for r in range(L):
        for c in range(L):
            if (r + c) % 2 == 0:
                index[(r, c)] = len(index)
    z_checks, x_checks = [], []
    for r in range(L):
        for c in range(L):
            if (r + c) % 2 == 1:
                qs = [index[(r + dr, c + dc)] for dr, dc in ((-1, 0), (0, -1), (0, 1), (1, 0))
                      if (r + dr, c + dc) in index]
                (z_checks if r % 2 == 1 else x_checks).append((r, c, sorted(qs)))
    zl = [index[(0, c)] for c in range(0, L, 2)]
    xl = [index[(r, 0)] for r in range(0, L, 2)]
    N, S, W, E = (-1, 0), (1, 0), (0, -1), (0, 1)

    def sched(checks, order):
        return [[index.get((r + dr, c + dc)) for dr, dc in order] for r, c, _ in checks]

    return SurfaceCode(d, z_checks, x_checks, zl, xl, len(index),
                       sched(z_checks, [N, E, W, S]), sched(x_checks, [N, W, E, S]), "unrotated")


def make_code(d, family="rotated"):
    return rotated_code(d) if family == "rotated" else unrotated_code(d)


def parity_check_matrices(code):
    """H_Z (rows = Z-checks) and H_X (rows = X-checks) over GF(2), shape (checks, n)."""
    hz = np.zeros((len(code.z_checks), code.n), dtype=np.uint8)
    hx = np.zeros((len(code.x_checks), code.n), dtype=np.uint8)
    for a, (_, _, qs) in enumerate(code.z_checks):
        hz[a, qs] = 1
    for a, (_, _, qs) in enumerate(code.x_checks):
        hx[a, qs] = 1
    return hz, hx


@dataclass
class DetGraph:
    """A detector graph: detectors 0..n_det-1 plus the boundary node n_det.

    `edges` is a list of (u, v, obs, q) with u < v and v == n_det for a boundary
    edge; `unit_of_edge` (code capacity only) names the data qubit behind each edge.
    """
    n_det: int
    edges: list
    unit_of_edge: list = None


def code_capacity_graph(code, kind):
    """Decoding graph of one Pauli type under code-capacity noise (Sec. "MWPM on the
    surface code"): one node per check of the matching type, one edge per data qubit
    between its one or two checks (one check = edge to the boundary).

    kind "X": X errors on the Z-check graph, obs = qubit in supp(Z_L).
    kind "Z": Z errors on the X-check graph, obs = qubit in supp(X_L).
    q of every edge is left as None: the code-capacity sampler draws Paulis per qubit.
    """
    checks = code.z_checks if kind == "X" else code.x_checks
    logical = set(code.zl if kind == "X" else code.xl)
    n_det = len(checks)
    touching = [[] for _ in range(code.n)]
    for a, (_, _, qs) in enumerate(checks):
        for q in qs:
            touching[q].append(a)
    edges, units = [], []
    for q in range(code.n):
        ts = sorted(touching[q])
        if len(ts) == 1:
            u, v = ts[0], n_det
        elif len(ts) == 2:
            u, v = ts
        else:
            raise AssertionError("qubit %d touches %d checks of one type" % (q, len(ts)))
        edges.append((u, v, 1 if q in logical else 0, None))
        units.append(q)
    return DetGraph(n_det, edges, units)
