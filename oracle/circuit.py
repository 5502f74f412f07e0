"""Memory-Z circuits (rotated and unrotated surface code) and their detector error model by
backward Pauli-frame propagation (oracle side).

Test infrastructure only: nothing in the product path imports this module.

The paper generates its circuit-level experiments with Stim's rotated memory-Z
construction (Sec. "Numerical Results"): R = d rounds of syndrome extraction and a final
transversal Z measurement of the data, with a depolarizing error after every Clifford
gate and on the data before every round, and flips of probability p after resets and
before measurements.  Idle qubits in every gate layer also get a single-qubit
depolarizing error of probability p.

Circuit (qubits: data r*d+c, then X-ancillas, then Z-ancillas in check order):
  reset all; X-flip(p) on all
  round 1..d:
    DEP1(p) on data
    H on X-ancillas; DEP1(p) on X-ancillas; DEP1(p) on idle qubits
    four CNOT layers in the code's schedule (see surface.py), ancilla controls for
      X-checks and data controls for Z-checks;
      after each layer DEP2(p) on every CNOT pair and DEP1(p) on the idle qubits
    H on X-ancillas; DEP1(p) on X-ancillas; DEP1(p) on idle qubits
    X-flip(p) on ancillas; measure-and-reset ancillas; X-flip(p) on ancillas
  X-flip(p) on data; measure data
Z-detectors: round 1 outcome; rounds 2..d outcome XOR previous outcome; a final layer
comparing each Z-check's data parity with its last outcome.  Numbered by
(round, check row, check column) ascending, the final layer being round d+1.  Observable: parity of the
data outcomes on supp(Z_L).  X-detectors (rounds 2..d) exist only for the determinism
check: the Z-part of the model never needs them.

The error model treats every non-identity Pauli of every channel as an independent
mechanism: p/3 each for DEP1, p/15 each for DEP2, p for a flip.
"""
from dataclasses import dataclass, field

import numpy as np

from .surface import make_code


@dataclass
class Noise:
    p: float
    data_round: bool = True     # DEP1 on data before every round
    gates: bool = True          # DEP1 after H, DEP2 after CNOT
    idle: bool = True           # DEP1 on idle qubits of gate layers
    reset_flip: bool = True     # X-flip after resets
    meas_flip: bool = True      # X-flip before measurements


@dataclass
class Circuit:
    d: int
    n_qubits: int
    ops: list                   # (name, targets, prob)
    n_records: int
    z_detectors: list           # list of lists of record indices, canonical order
    x_detectors: list
    observable: list            # record indices
    zdet_coords: list = field(default_factory=list)  # (round, pr, pc)


def memory_z_circuit(d, noise, family="rotated"):
    code = make_code(d, family)
    n = code.n
    nx, nz = len(code.x_checks), len(code.z_checks)
    xanc = [n + a for a in range(nx)]
    zanc = [n + nx + a for a in range(nz)]
    anc = xanc + zanc
    allq = list(range(n + nx + nz))
    p = noise.p
    ops = []

    def add_noise(name, targets, prob, on):
        if on and prob > 0 and len(targets):
            ops.append((name, list(targets), prob))

    # CNOT layers
    layers = []
    for k in range(4):
        pairs = []
        for a in range(nx):
            q = code.x_sched[a][k]
            if q is not None:
                pairs.append((xanc[a], q))
        for a in range(nz):
            q = code.z_sched[a][k]
            if q is not None:
                pairs.append((q, zanc[a]))
        layers.append(pairs)

    ops.append(("R", allq, 0.0))
    add_noise("XERR", allq, p, noise.reset_flip)
    rec = 0
    zrec = []  # zrec[round][a]
    xrec = []
    h_idle = list(range(n)) + zanc
    for rnd in range(d):
        add_noise("DEP1", range(n), p, noise.data_round)
        ops.append(("H", xanc, 0.0))
        add_noise("DEP1", xanc, p, noise.gates)
        add_noise("DEP1", h_idle, p, noise.idle)
        for pairs in layers:
            ops.append(("CX", pairs, 0.0))
            add_noise("DEP2", pairs, p, noise.gates)
            busy = set(q for pr_ in pairs for q in pr_)
            add_noise("DEP1", [q for q in allq if q not in busy], p, noise.idle)
        ops.append(("H", xanc, 0.0))
        add_noise("DEP1", xanc, p, noise.gates)
        add_noise("DEP1", h_idle, p, noise.idle)
        add_noise("XERR", anc, p, noise.meas_flip)
        ops.append(("MR", anc, 0.0))
        xrec.append([rec + a for a in range(nx)])
        zrec.append([rec + nx + a for a in range(nz)])
        rec += nx + nz
        add_noise("XERR", anc, p, noise.reset_flip)
    add_noise("XERR", range(n), p, noise.meas_flip)
    ops.append(("M", list(range(n)), 0.0))
    drec = list(range(rec, rec + n))
    rec += n

    zdets, coords = [], []
    for rnd in range(d):
        for a, (pr, pc, _) in enumerate(code.z_checks):
            zdets.append([zrec[rnd][a]] if rnd == 0 else [zrec[rnd][a], zrec[rnd - 1][a]])
            coords.append((rnd + 1, pr, pc))
    for a, (pr, pc, qs) in enumerate(code.z_checks):
        zdets.append([zrec[d - 1][a]] + [drec[q] for q in qs])
        coords.append((d + 1, pr, pc))
    xdets = []
    for rnd in range(1, d):
        for a in range(nx):
            xdets.append([xrec[rnd][a], xrec[rnd - 1][a]])
    obs = [drec[q] for q in code.zl]
    return Circuit(d, n + nx + nz, ops, rec, zdets, xdets, obs, coords)


def _one_qubit_paulis():
    return ["X", "Y", "Z"]


def _two_qubit_paulis():
    ps = ["I", "X", "Y", "Z"]
    return [(a, b) for a in ps for b in ps if (a, b) != ("I", "I")]


@dataclass
class FrameResult:
    mechanisms: list      # (zdet tuple, obs, prob) in circuit order
    nondeterministic: set  # target columns found non-deterministic
    n_zdet: int


def backward_frames(circ, include_x_detectors=False):
    """Heisenberg (backward) propagation of every detector and the observable.

    Each target (Z-detector, observable, optionally X-detector) is a product of Z
    measurement outcomes.  Walking the circuit backwards, its operator picks up Z_q at
    each measurement it includes, is conjugated by every Clifford, and is cleared at a
    reset.  A single Pauli P on qubit q at some point flips the target iff P anticommutes
    with the target's operator there.  The target is deterministic iff its operator has
    no X component on a qubit where it meets a reset or a Z measurement.
    """
    nz = len(circ.z_detectors)
    targets = list(circ.z_detectors) + [circ.observable]
    if include_x_detectors:
        targets += list(circ.x_detectors)
    nt = len(targets)
    rec_targets = [[] for _ in range(circ.n_records)]
    for t, recs in enumerate(targets):
        for m in recs:
            rec_targets[m].append(t)
    X = np.zeros((circ.n_qubits, nt), dtype=bool)
    Z = np.zeros((circ.n_qubits, nt), dtype=bool)
    nondet = set()
    mech = []  # collected backwards, reversed at the end
    rec = circ.n_records

    def symptom(vec):
        idx = np.flatnonzero(vec)
        zs = tuple(int(i) for i in idx if i < nz)
        ob = int(vec[nz]) if nt > nz else 0
        return zs, ob

    def sens(q, pauli):
        if pauli == "X":
            return Z[q].copy()
        if pauli == "Z":
            return X[q].copy()
        if pauli == "Y":
            return X[q] ^ Z[q]
        return np.zeros(nt, dtype=bool)

    for name, tg, prob in reversed(circ.ops):
        if name in ("M", "MR"):
            for q in reversed(tg):
                rec -= 1
                if name == "MR":
                    nondet.update(int(i) for i in np.flatnonzero(X[q]))
                    X[q] = False
                    Z[q] = False
                for t in rec_targets[rec]:
                    Z[q, t] ^= True
                nondet.update(int(i) for i in np.flatnonzero(X[q]))
        elif name == "R":
            for q in tg:
                nondet.update(int(i) for i in np.flatnonzero(X[q]))
                X[q] = False
                Z[q] = False
        elif name == "H":
            for q in tg:
                X[q], Z[q] = Z[q].copy(), X[q].copy()
        elif name == "CX":
            for c, t in tg:
                X[t] ^= X[c]
                Z[c] ^= Z[t]
        elif name == "DEP1":
            for q in reversed(tg):
                for pa in reversed(_one_qubit_paulis()):
                    mech.append(symptom(sens(q, pa)) + (prob / 3.0,))
        elif name == "DEP2":
            for a, b in reversed(tg):
                for pa, pb in reversed(_two_qubit_paulis()):
                    mech.append(symptom(sens(a, pa) ^ sens(b, pb)) + (prob / 15.0,))
        elif name == "XERR":
            for q in reversed(tg):
                mech.append(symptom(sens(q, "X")) + (prob,))
        else:
            raise ValueError(name)
    assert rec == 0
    mech.reverse()
    return FrameResult(mech, nondet, nz)


def merge_probabilities(qs):
    """Probability that an odd number of independent mechanisms fire, folded as
    q <- q(1-q') + q'(1-q) over the contributing probabilities sorted ascending."""
    acc = 0.0
    for q2 in sorted(qs):
        acc = acc * (1.0 - q2) + q2 * (1.0 - acc)
    return acc


def circuit_graph(d, noise, family="rotated"):
    """Z-part detector graph of the rotated memory-Z experiment.

    Every mechanism is reduced to its Z-detector set and observable bit; mechanisms with
    the same (set, bit) are merged; sets of size 1 become boundary edges and size 2
    pair edges.  Larger sets are decomposed into existing edges (see
    `decompose_hyperedge`).  Returns (DetGraph-like dict, stats).
    """
    from .surface import DetGraph
    circ = memory_z_circuit(d, noise, family)
    fr = backward_frames(circ)
    nz = fr.n_zdet
    groups = {}
    hyper = []
    for zs, ob, prob in fr.mechanisms:
        if len(zs) == 0:
            if ob:
                raise AssertionError("undetectable logical mechanism")
            continue
        if len(zs) > 2:
            hyper.append((zs, ob, prob))
            continue
        groups.setdefault((zs, ob), []).append(prob)
    edge_keys = set(groups)
    for zs, ob, prob in hyper:
        parts = decompose_hyperedge(zs, ob, edge_keys)
        if parts is None:
            raise AssertionError("non-graphlike Z-part %r" % (zs,))
        for part in parts:
            groups[part].append(prob)
    edges = []
    for (zs, ob), probs in groups.items():
        u = zs[0]
        v = zs[1] if len(zs) == 2 else nz
        edges.append((u, v, ob, merge_probabilities(probs)))
    edges.sort(key=lambda e: (e[0], e[1], e[2]))
    stats = {"mechanisms": len(fr.mechanisms), "hyperedges": len(hyper),
             "nondeterministic": sorted(fr.nondeterministic)}
    return DetGraph(nz, edges), circ, stats


def decompose_hyperedge(zs, ob, edge_keys):
    """Split a Z-part with more than two detectors into single-fault edges.

    Tries every way of pairing the detectors (or sending one to the boundary) and
    returns the first, in lexicographic order of the parts, whose parts all exist as
    edges and whose observable bits XOR to `ob`.  None if there is none.
    """
    zs = tuple(sorted(zs))

    def rec(rem):
        if not rem:
            yield []
            return
        a = rem[0]
        rest = rem[1:]
        options = [((a,), rest)] + [((a, b), rest[:i] + rest[i + 1:]) for i, b in enumerate(rest)]
        for part, left in options:
            for tail in rec(left):
                yield [part] + tail

    for split in rec(zs):
        for bits in range(1 << len(split)):
            parts = [(split[i], (bits >> i) & 1) for i in range(len(split))]
            if all(pk in edge_keys for pk in parts) and sum(b for _, b in parts) % 2 == ob:
                return parts
    return None
