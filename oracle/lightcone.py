"""Exact noisy correlators <Z_u Z_v> of large QAOA circuits by light cones (oracle).

Test infrastructure only: the tests, the smoke check and the bench's CPU legs
use it; the library never does.

For the circuits of App. D with the noise of Sec. 3 placed as in the noisy
workloads (a two-qubit Pauli channel after each RZZ, any one-qubit channels),
the expectation of an observable O supported on a few qubits is
Tr(O rho_T) = Tr(E_1^dag(...E_T^dag(O)) rho_0), with E_t^dag the adjoint of
operation t (Heisenberg picture). Every adjoint of a trace-preserving
operation maps the identity to the identity, so operations acting only where
the evolved observable is the identity drop out. Walking back through layer
l of p, the mixers keep the support and the cost gates extend it by one graph
step: after all p layers it lies within graph distance p of O's qubits, and on
the qubits first reached in a layer it holds only Z and I, which commute with
the diagonal two-qubit gates. So, with R the qubits within distance ``radius``
>= p of the targets:

* operations on qubits of R only are kept;
* a diagonal two-qubit gate with one qubit outside R is dropped (it meets Z or
  I on its inside qubit, I outside);
* a two-qubit Pauli channel sum_ab p_ab (P_a x P_b) rho (P_a x P_b) with one
  qubit outside R meets the identity there, and its adjoint then acts on the
  inside qubit as the one-qubit Pauli channel with the marginal rates
  sum_b p_ab: it becomes that channel;
* operations outside R are dropped.

The reduced circuit is simulated exactly as a density matrix (Sec. 3.1,
rho -> sum_i E_i rho E_i^dag) on |R| qubits, using the vectorised form
vec(A rho B^T) = (A x B) vec(rho): U rho U^dag applies U to the row bits and
conj(U) to the column bits of vec(rho), a state of 2|R| qubits.

Pinned by the full density matrix of small noisy circuits (path and grid
graphs, where the light cone cuts channels and gates) and by the p = 1 closed
form on large noiseless graphs.
"""
from __future__ import annotations

from collections import deque

import numpy as np

from oracle import circuit as OC
from oracle import statevector as SV


def density_diag(n: int, ops) -> np.ndarray:
    """The diagonal of rho_T (probabilities of the 2^n basis states) for gates
    and Kraus channels, through the vectorised density matrix: basis index
    r 2^n + c of vec(rho) is rho[r, c], so bit q is column bit q and bit n+q
    row bit q."""
    vec = np.zeros(1 << (2 * n), dtype=complex)
    vec[0] = 1.0
    for op in ops:
        rows = [q + n for q in op.qubits]
        cols = list(op.qubits)
        if op.kind == "gate":
            vec = SV.apply(SV.apply(vec, 2 * n, rows, op.mat), 2 * n, cols, op.mat.conj())
        else:
            acc = np.zeros_like(vec)
            for E in op.mats:
                acc += SV.apply(SV.apply(vec, 2 * n, rows, E), 2 * n, cols, E.conj())
            vec = acc
    rho = vec.reshape(1 << n, 1 << n)
    return np.real(np.diag(rho)).copy()


def _pauli_rates(Es):
    """The rates p_ab of a two-qubit Pauli channel given by Kraus operators
    that are each a multiple of one Pauli product (P_a on q_0, P_b on q_1);
    None when an operator is not."""
    rates = np.zeros((4, 4))
    if any(np.shape(E) != (4, 4) for E in Es):
        return None
    for E in Es:
        found = False
        for a in range(4):
            for b in range(4):
                P = np.kron(OC.PAULI[b], OC.PAULI[a])
                c = np.trace(P.conj().T @ E) / 4.0
                if abs(c) > 1e-15:
                    if found or not np.allclose(E, c * P, atol=1e-14):
                        return None
                    rates[a, b] += abs(c) ** 2
                    found = True
        if not found and np.abs(E).max() > 0:
            return None
    return rates


def region(n: int, edges, targets, radius: int) -> list:
    """The qubits within graph distance ``radius`` of ``targets`` (sorted)."""
    nbr = [[] for _ in range(n)]
    for u, v in edges:
        nbr[int(u)].append(int(v))
        nbr[int(v)].append(int(u))
    dist = {int(t): 0 for t in targets}
    todo = deque(dist)
    while todo:
        x = todo.popleft()
        if dist[x] == radius:
            continue
        for y in nbr[x]:
            if y not in dist:
                dist[y] = dist[x] + 1
                todo.append(y)
    return sorted(dist)


def reduced_ops(ops, keep) -> list:
    """The operations of a light cone over the qubits ``keep`` (renumbered
    0..len(keep)-1 in that order), by the rules of the module docstring.
    Raises ValueError for an operation the rules do not cover."""
    idx = {q: i for i, q in enumerate(keep)}
    out = []
    for op in ops:
        inside = [q in idx for q in op.qubits]
        if all(inside):
            out.append(OC.Op(op.kind, tuple(idx[q] for q in op.qubits), list(op.mats)))
            continue
        if not any(inside):
            continue
        if len(op.qubits) != 2:
            raise ValueError("operation on more than two qubits crosses the light cone")
        if op.kind == "gate":
            if not OC.is_diagonal(op.mat):
                raise ValueError("non-diagonal two-qubit gate crosses the light cone")
            continue
        rates = _pauli_rates(op.mats)
        if rates is None:
            raise ValueError("non-Pauli two-qubit channel crosses the light cone")
        pos = 0 if inside[0] else 1
        marg = rates.sum(axis=1) if pos == 0 else rates.sum(axis=0)
        Es = [np.sqrt(marg[a]) * OC.PAULI[a] for a in range(4) if marg[a] > 0]
        out.append(OC.kraus((idx[op.qubits[pos]],), Es))
    return out


def zz(spec, u: int, v: int, radius: int | None = None) -> float:
    """Exact <Z_u Z_v> of the (noisy) QAOA circuit of ``spec`` (App. D with
    the channels of Sec. 3 as ``oracle.circuit.qaoa_circuit`` places them),
    from the density matrix of its light cone (radius p by default)."""
    r = spec.p if radius is None else radius
    if r < spec.p:
        raise ValueError("the light cone of p layers needs radius >= p")
    keep = region(spec.n, spec.edges, (u, v), r)
    ops = reduced_ops(OC.qaoa_circuit(spec), keep)
    m = len(keep)
    prob = density_diag(m, ops)
    x = np.arange(1 << m)
    iu, iv = keep.index(int(u)), keep.index(int(v))
    z = (1 - 2 * ((x >> iu) & 1)) * (1 - 2 * ((x >> iv) & 1))
    return float(np.dot(prob, z))
