"""Circuit semantics in FP64 (oracle).

A circuit is a list of operations (paper App. A: a gate is a pair (A, q) with A
a 2^m x 2^m matrix and q a tuple of m qubits). Noise operations are quantum
operations given by Kraus lists {E_i} with sum_i E_i^dag E_i = I (Sec. 3.1).

Local index convention: for an operation on qubits (q_0, ..., q_{m-1}) the row
and column index of its matrix is sum_i b(q_i) 2^i, i.e. q_0 is the least
significant bit. Global basis index: qubit q is bit q.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SQ2 = 1.0 / math.sqrt(2.0)
PAULI = [np.eye(2, dtype=complex),
         np.array([[0, 1], [1, 0]], dtype=complex),
         np.array([[0, -1j], [1j, 0]], dtype=complex),
         np.array([[1, 0], [0, -1]], dtype=complex)]
SIGMA_X = PAULI[1]


@dataclass
class Op:
    """One circuit operation: a gate (one matrix) or a Kraus channel."""
    kind: str                 # "gate" or "kraus"
    qubits: tuple
    mats: list                # [A] for a gate, [E_0, ..., E_{k-1}] for a channel

    @property
    def mat(self) -> np.ndarray:
        return self.mats[0]


def gate(qubits, A) -> Op:
    return Op("gate", tuple(int(q) for q in qubits), [np.asarray(A, dtype=complex)])


def kraus(qubits, Es) -> Op:
    return Op("kraus", tuple(int(q) for q in qubits), [np.asarray(E, dtype=complex) for E in Es])


# ---------------------------------------------------------------------------
# Standard gates (App. D: R_P(theta) = exp(-i theta P / 2))
# ---------------------------------------------------------------------------

def h_mat() -> np.ndarray:
    return SQ2 * np.array([[1, 1], [1, -1]], dtype=complex)


def rx_mat(theta: float) -> np.ndarray:
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=complex)


def rz_mat(theta: float) -> np.ndarray:
    return np.diag([np.exp(-0.5j * theta), np.exp(0.5j * theta)])


def rzz_mat(theta: float) -> np.ndarray:
    """exp(-i theta Z(x)Z / 2) on local index b0 + 2 b1: the phase depends on parity."""
    d = [np.exp(-0.5j * theta * (1 - 2 * ((b & 1) ^ (b >> 1)))) for b in range(4)]
    return np.diag(d)


def cnot_mat() -> np.ndarray:
    """Control q_0, target q_1 (Fig. 1b, in the local-index convention)."""
    M = np.zeros((4, 4), dtype=complex)
    for b0 in range(2):
        for b1 in range(2):
            M[b0 + 2 * (b1 ^ b0), b0 + 2 * b1] = 1
    return M


def iswap_mat() -> np.ndarray:
    """iSWAP (Fig. 1b): |01> <-> i|10>, |00> and |11> fixed."""
    M = np.zeros((4, 4), dtype=complex)
    M[0, 0] = 1
    M[3, 3] = 1
    M[1, 2] = 1j
    M[2, 1] = 1j
    return M


def crx_mat(theta: float) -> np.ndarray:
    """Controlled RX (Fig. 1c): control q_0, RX(theta) on q_1 when the control is 1."""
    M = np.zeros((4, 4), dtype=complex)
    R = rx_mat(theta)
    M[0, 0] = 1
    M[2, 2] = 1
    for a in range(2):
        for b in range(2):
            M[1 + 2 * a, 1 + 2 * b] = R[a, b]
    return M


def fsim_mat(theta: float, phi: float) -> np.ndarray:
    """fSim(theta, phi) (Fig. 1c): mixes |01>,|10>, phase on |11>."""
    M = np.zeros((4, 4), dtype=complex)
    M[0, 0] = 1
    M[1, 1] = math.cos(theta)
    M[2, 2] = math.cos(theta)
    M[1, 2] = -1j * math.sin(theta)
    M[2, 1] = -1j * math.sin(theta)
    M[3, 3] = np.exp(1j * phi)
    return M


# ---------------------------------------------------------------------------
# Noise channels (Sec. 3; the chosen channel forms are readings of the paper)
# ---------------------------------------------------------------------------

def depolarizing2_kraus(p: float) -> list:
    """Two-qubit depolarizing (1-p) rho + p/15 sum_{P != II} P rho P.

    Kraus order: index k = a + 4 b for a, b in 0..3 (I, X, Y, Z), Pauli a on
    q_0 and Pauli b on q_1; k = 0 is the identity term.
    """
    out = []
    for k in range(16):
        a, b = k % 4, k // 4
        scale = math.sqrt(1.0 - p) if k == 0 else math.sqrt(p / 15.0)
        out.append(scale * np.kron(PAULI[b], PAULI[a]))
    return out


def depolarizing1_kraus(p: float) -> list:
    """One-qubit depolarizing (1-p) rho + p/3 (X rho X + Y rho Y + Z rho Z)."""
    return [math.sqrt(1 - p) * PAULI[0]] + [math.sqrt(p / 3.0) * PAULI[k] for k in (1, 2, 3)]


def amplitude_damping_kraus(gamma: float) -> list:
    """E0 = diag(1, sqrt(1-gamma)), E1 = sqrt(gamma) |0><1|."""
    return [np.array([[1, 0], [0, math.sqrt(1 - gamma)]], dtype=complex),
            np.array([[0, math.sqrt(gamma)], [0, 0]], dtype=complex)]


def phase_damping_kraus(lam: float) -> list:
    return [np.array([[1, 0], [0, math.sqrt(1 - lam)]], dtype=complex),
            np.array([[0, 0], [0, math.sqrt(lam)]], dtype=complex)]


# ---------------------------------------------------------------------------
# QAOA circuit (App. D)
# ---------------------------------------------------------------------------

def qaoa_circuit(spec) -> list:
    """The QAOA circuit of App. D for a ``workloads.QaoaSpec``.

    |+>^n by H on every qubit; for each layer l: exp(-i gamma_l w_e Z_u Z_v)
    = RZZ(2 gamma_l w_e) once per edge, exp(-i gamma_l h_j Z_j) = RZ(2 gamma_l h_j),
    exp(-i beta_l X_j) = RX(2 beta_l). Optional noise: a two-qubit depolarizing
    channel after every RZZ and amplitude damping on every qubit after each
    mixer layer.
    """
    n = spec.n
    ops = [gate((q,), h_mat()) for q in range(n)]
    dep = depolarizing2_kraus(spec.depol2) if spec.depol2 > 0 else None
    ad = amplitude_damping_kraus(spec.ad_gamma) if spec.ad_gamma > 0 else None
    for l in range(spec.p):
        g, b = float(spec.gammas[l]), float(spec.betas[l])
        for (u, v), w in zip(spec.edges, spec.weights):
            ops.append(gate((int(u), int(v)), rzz_mat(2 * g * float(w))))
            if dep is not None:
                ops.append(kraus((int(u), int(v)), dep))
        if spec.h is not None:
            for j in range(n):
                ops.append(gate((j,), rz_mat(2 * g * float(spec.h[j]))))
        for j in range(n):
            ops.append(gate((j,), rx_mat(2 * b)))
        if ad is not None:
            for j in range(n):
                ops.append(kraus((j,), ad))
    return ops


# ---------------------------------------------------------------------------
# Classification (Sec. 2, Alg. 1)
# ---------------------------------------------------------------------------

def is_diagonal(A: np.ndarray) -> bool:
    return bool(np.all(A[~np.eye(A.shape[0], dtype=bool)] == 0))


def is_monomial(A: np.ndarray) -> bool:
    """Exactly one nonzero entry in every row and every column (Prop. 1 definition)."""
    nz = A != 0
    return bool(np.all(nz.sum(axis=0) == 1) and np.all(nz.sum(axis=1) == 1))


def monomial_image(A: np.ndarray, x: int) -> int:
    """For a monomial A = M_sigma D, sigma(x): the row of the nonzero in column x."""
    rows = np.nonzero(A[:, x])[0]
    assert len(rows) == 1
    return int(rows[0])


def block_decompose_local(A: np.ndarray, x: int) -> list:
    """BlockDecompose of Alg. 1 on local indices: the connected component of x in
    the graph on {0,1}^m with an edge {u,v} whenever A[u,v] != 0, sorted."""
    dim = A.shape[0]
    seen = {x}
    stack = [x]
    while stack:
        u = stack.pop()
        for v in range(dim):
            if v not in seen and (A[u, v] != 0 or A[v, u] != 0):
                seen.add(v)
                stack.append(v)
    return sorted(seen)


def local_index(bits, qubits) -> int:
    return sum(int(bits[q]) << i for i, q in enumerate(qubits))


def set_local(bits, qubits, idx: int):
    out = np.array(bits, copy=True)
    for i, q in enumerate(qubits):
        out[q] = (idx >> i) & 1
    return out


# ---------------------------------------------------------------------------
# Local-submonomial factorisation (App. A)
# ---------------------------------------------------------------------------

def is_submonomial(M: np.ndarray) -> bool:
    nz = M != 0
    return bool(np.all(nz.sum(axis=0) <= 1) and np.all(nz.sum(axis=1) <= 1))


def lsm_factorize(E: np.ndarray, qubits) -> list:
    """Write an LSM Kraus operator as a tensor product of 2x2 submonomial factors.

    Returns [(M_i, q_i)] with E = M_{m-1} (x) ... (x) M_0 in the local-index
    convention; raises ValueError if E is not local-submonomial (App. A).
    """
    m = len(qubits)
    if m == 1:
        if not is_submonomial(E):
            raise ValueError("not submonomial")
        return [(np.array(E, dtype=complex), qubits[0])]
    if m != 2:
        raise ValueError("only 1- and 2-qubit channels")
    r, c = np.unravel_index(int(np.argmax(np.abs(E))), E.shape)
    r0, r1, c0, c1 = r & 1, r >> 1, c & 1, c >> 1
    piv = E[r, c]
    if piv == 0:
        raise ValueError("zero Kraus operator")
    M0 = np.array([[E[a + 2 * r1, b + 2 * c1] for b in range(2)] for a in range(2)], dtype=complex)
    M1 = np.array([[E[r0 + 2 * a, c0 + 2 * b] for b in range(2)] for a in range(2)], dtype=complex) / piv
    if not np.allclose(np.kron(M1, M0), E, atol=1e-14, rtol=0):
        raise ValueError("not a tensor product")
    if not (is_submonomial(M0) and is_submonomial(M1)):
        raise ValueError("factor not submonomial")
    return [(M0, qubits[0]), (M1, qubits[1])]
