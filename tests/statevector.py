"""A tiny real-amplitude state-vector simulator for checking the d=3 circuit.

Test helper only.  It runs the noiseless Clifford circuit (R, H, CX, M, MR) exactly, and
can apply one Pauli at a chosen noise location, so that the detector error model of the
oracle can be checked against the physics rather than against itself.  H and CNOT have
real matrices and the initial state is |0...0>, so real amplitudes suffice; a Y error is
applied as X*Z (a global phase does not change any outcome).
"""
import numpy as np


class StateVector:
    def __init__(self, n, rng):
        self.n = n
        self.psi = np.zeros((2,) * n)
        self.psi[(0,) * n] = 1.0
        self.rng = rng

    def _ax(self, q):
        return q

    def h(self, q):
        a = np.take(self.psi, 0, axis=q)
        b = np.take(self.psi, 1, axis=q)
        self.psi = np.stack([(a + b) / np.sqrt(2.0), (a - b) / np.sqrt(2.0)], axis=q)

    def x(self, q):
        self.psi = np.flip(self.psi, axis=q).copy()

    def z(self, q):
        idx = [slice(None)] * self.n
        idx[q] = 1
        self.psi[tuple(idx)] *= -1.0

    def cx(self, c, t):
        idx = [slice(None)] * self.n
        idx[c] = 1
        sub = self.psi[tuple(idx)]
        tt = t if t < c else t - 1
        self.psi[tuple(idx)] = np.flip(sub, axis=tt)

    def measure(self, q):
        idx1 = [slice(None)] * self.n
        idx1[q] = 1
        p1 = float(np.sum(self.psi[tuple(idx1)] ** 2))
        if p1 < 1e-12:
            out = 0
        elif p1 > 1 - 1e-12:
            out = 1
        else:
            out = int(self.rng.random() < p1)
        idx0 = [slice(None)] * self.n
        idx0[q] = 1 - out
        self.psi[tuple(idx0)] = 0.0
        self.psi /= np.sqrt(np.sum(self.psi ** 2))
        return out

    def reset(self, q):
        if self.measure(q):
            self.x(q)

    def pauli(self, q, p):
        if p in ("X", "Y"):
            self.x(q)
        if p in ("Z", "Y"):
            self.z(q)


def run_circuit(circ, rng, inject=None):
    """Run the ops of an oracle Circuit; noise ops are skipped except `inject`, a tuple
    (op_index, target_index, pauli or pair of paulis).  Returns the measurement record."""
    sv = StateVector(circ.n_qubits, rng)
    rec = []
    for k, (name, tg, _) in enumerate(circ.ops):
        if name == "R":
            for q in tg:
                sv.reset(q)
        elif name == "H":
            for q in tg:
                sv.h(q)
        elif name == "CX":
            for c, t in tg:
                sv.cx(c, t)
        elif name == "M":
            for q in tg:
                rec.append(sv.measure(q))
        elif name == "MR":
            for q in tg:
                rec.append(sv.measure(q))
                sv.reset(q)
        if inject is not None and inject[0] == k:
            target = tg[inject[1]]
            if name == "DEP2":
                a, b = target
                pa, pb = inject[2]
                if pa != "I":
                    sv.pauli(a, pa)
                if pb != "I":
                    sv.pauli(b, pb)
            else:
                sv.pauli(target, inject[2])
    return rec


def detector_values(circ, rec):
    z = [sum(rec[m] for m in det) % 2 for det in circ.z_detectors]
    x = [sum(rec[m] for m in det) % 2 for det in circ.x_detectors]
    obs = sum(rec[m] for m in circ.observable) % 2
    return z, x, obs
