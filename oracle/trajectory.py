"""Standard quantum trajectories (test infrastructure only; FP64).

A second, differently derived check of noisy output distributions, written
from the textbook unravelling of a quantum operation rather than from Alg. 2:
the state vector is carried through the circuit; at a channel {E_i} operator
i is drawn with probability ||E_i psi||^2 and psi becomes E_i psi / ||E_i psi||
(Nielsen & Chuang 8.3; Sec. 3.1 uses the same Kraus form). The final bits are
drawn from |psi|^2. Averaged over trajectories this reproduces the diagonal of
the density matrix sum_i E_i rho E_i^dag.

Only the tests may use this module.
"""
from __future__ import annotations

import numpy as np

from . import statevector as SV


def sample(n: int, ops, rng: np.random.Generator) -> np.ndarray:
    """One trajectory; returns the measured bits as uint8 [n] (qubit q = bit q)."""
    psi = SV.zero_state(n)
    for op in ops:
        if op.kind == "gate":
            psi = SV.apply(psi, n, op.qubits, op.mat)
            continue
        branches = [SV.apply(psi, n, op.qubits, E) for E in op.mats]
        w = np.array([np.vdot(b, b).real for b in branches])
        i = int(rng.choice(len(branches), p=w / w.sum()))
        psi = branches[i] / np.sqrt(w[i])
    p = np.abs(psi) ** 2
    x = int(rng.choice(len(p), p=p / p.sum()))
    return np.array([(x >> q) & 1 for q in range(n)], dtype=np.uint8)


def exact_distribution(n: int, ops) -> np.ndarray:
    """The trajectory average without sampling: every Kraus branch is followed
    with its probability (exponential in the number of channels; tiny circuits
    only). Returns p(x) over the 2^n basis states."""
    out = np.zeros(1 << n)

    def walk(k, psi, weight):
        while k < len(ops) and ops[k].kind == "gate":
            psi = SV.apply(psi, n, ops[k].qubits, ops[k].mat)
            k += 1
        if k == len(ops):
            out[:] += weight * np.abs(psi) ** 2
            return
        for E in ops[k].mats:
            b = SV.apply(psi, n, ops[k].qubits, E)
            w = np.vdot(b, b).real
            if w > 0:
                walk(k + 1, b / np.sqrt(w), weight * w)

    walk(0, SV.zero_state(n), 1.0)
    return out
