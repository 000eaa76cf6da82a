"""Dense state-vector and density-matrix simulation in FP64 (oracle).

psi_0 = |0^n>, psi_t = U_t psi_{t-1} (Sec. 2); amp(C_t, i) = <i|psi_t>.
Noisy circuits: rho -> sum_i E_i rho E_i^dag (Sec. 3.1, Nielsen & Chuang 8.2.3).
Qubit q is bit q of the basis index; an operation's local index follows the
convention of ``oracle.circuit``.
"""
from __future__ import annotations

import numpy as np


def apply(psi: np.ndarray, n: int, qubits, U: np.ndarray) -> np.ndarray:
    """Return (U on ``qubits``) psi for a state of n qubits (tensordot form)."""
    m = len(qubits)
    t = psi.reshape([2] * n)                 # axis k <-> bit n-1-k
    axes = [n - 1 - q for q in qubits]
    Ut = U.reshape([2] * (2 * m))            # out bits (q_{m-1}..q_0), in bits (q_{m-1}..q_0)
    in_axes = [m + (m - 1 - i) for i in range(m)]
    res = np.tensordot(Ut, t, axes=(in_axes, axes))
    res = np.moveaxis(res, [m - 1 - i for i in range(m)], axes)
    return res.reshape(-1)


def embed(n: int, qubits, U: np.ndarray) -> np.ndarray:
    """The full 2^n x 2^n matrix of U on ``qubits``, entry by entry from the
    definition <y|U (x) I|x> = U[y_q, x_q] * [y_rest == x_rest]."""
    dim = 1 << n
    m = len(qubits)
    mask = sum(1 << q for q in qubits)
    F = np.zeros((dim, dim), dtype=complex)
    for x in range(dim):
        xl = sum(((x >> q) & 1) << i for i, q in enumerate(qubits))
        for yl in range(1 << m):
            y = x & ~mask
            for i, q in enumerate(qubits):
                y |= ((yl >> i) & 1) << q
            F[y, x] += U[yl, xl]
    return F


def zero_state(n: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=complex)
    psi[0] = 1.0
    return psi


def run(n: int, ops) -> np.ndarray:
    """psi_T for a list of unitary gate ops."""
    psi = zero_state(n)
    for op in ops:
        assert op.kind == "gate"
        psi = apply(psi, n, op.qubits, op.mat)
    return psi


def prefix_states(n: int, ops):
    """Yield psi_t after each gate t = 1..T (the amplitudes of every prefix C_t)."""
    psi = zero_state(n)
    for op in ops:
        psi = apply(psi, n, op.qubits, op.mat)
        yield psi


def density_run(n: int, ops) -> np.ndarray:
    """rho_T for a list of gates and Kraus channels (full matrices, small n)."""
    dim = 1 << n
    rho = np.zeros((dim, dim), dtype=complex)
    rho[0, 0] = 1.0
    for op in ops:
        if op.kind == "gate":
            U = embed(n, op.qubits, op.mat)
            rho = U @ rho @ U.conj().T
        else:
            acc = np.zeros_like(rho)
            for E in op.mats:
                F = embed(n, op.qubits, E)
                acc += F @ rho @ F.conj().T
            rho = acc
    return rho
