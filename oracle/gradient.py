"""Exact amplitude gradients of ideal QAOA circuits (test infrastructure only).

Only the tests and bench.py's oracle legs may use this package.

For the QAOA circuit of App. D, layer l applies exp(-i gamma_l H_C) with
H_C = sum_e w_e Z_u Z_v + sum_j h_j Z_j (all terms commute), then
exp(-i beta_l H_M) with H_M = sum_j X_j. Hence

  d amp(x) / d gamma_l = <x| U_after (-i H_C) exp(-i gamma_l H_C) |psi_l>,
  d amp(x) / d beta_l  = <x| U_after (-i H_M) exp(-i beta_l H_M) |phi_l>,

the generator inserted right after the layer's part (state vector, FP64).
Pinned by a closed form for one qubit with a field and by central finite
differences of the state-vector amplitude.
"""
import numpy as np

from . import circuit as C
from . import statevector as SV

PAULI_Z = np.diag([1.0, -1.0]).astype(complex)
PAULI_X = np.array([[0, 1], [1, 0]], dtype=complex)


def _apply_hc(psi, n, spec):
    """(-i H_C) psi."""
    out = np.zeros_like(psi)
    for (u, v), w in zip(spec.edges, spec.weights):
        out += float(w) * SV.apply(psi, n, (int(u), int(v)), np.kron(PAULI_Z, PAULI_Z))
    if spec.h is not None:
        for j in range(n):
            out += float(spec.h[j]) * SV.apply(psi, n, (j,), PAULI_Z)
    return -1j * out


def _apply_hm(psi, n):
    """(-i H_M) psi."""
    out = np.zeros_like(psi)
    for j in range(n):
        out += SV.apply(psi, n, (j,), PAULI_X)
    return -1j * out


def amp_and_grad(spec, bitstrings):
    """Amplitudes <x|C|0^n> of the ideal circuit and their derivatives.

    Returns (amp [K] complex, grad [K, 2p] complex) with grad[:, l] =
    d amp / d gamma_l and grad[:, p + l] = d amp / d beta_l. bitstrings: uint8
    [K, n], qubit q = bit q of the basis index.
    """
    n, p = spec.n, spec.p
    ops = C.qaoa_circuit(spec)
    # split the op list into: H layer, then per layer (cost ops, mixer ops)
    pos = n
    layers = []
    for l in range(p):
        m = len(spec.edges) + (n if spec.h is not None else 0)
        layers.append((ops[pos:pos + m], ops[pos + m:pos + m + n]))
        pos += m + n
    idx = np.asarray([int(sum(int(b) << q for q, b in enumerate(x))) for x in bitstrings])

    def run_from(psi, start_layer, start_part):
        for l in range(start_layer, p):
            parts = layers[l] if l > start_layer else layers[l][start_part:]
            for part in parts:
                for o in part:
                    psi = SV.apply(psi, n, o.qubits, o.mat)
        return psi

    psi = SV.zero_state(n)
    for o in ops[:n]:
        psi = SV.apply(psi, n, o.qubits, o.mat)
    grads = np.zeros((len(idx), 2 * p), dtype=complex)
    for l in range(p):
        for o in layers[l][0]:
            psi = SV.apply(psi, n, o.qubits, o.mat)
        grads[:, l] = run_from(_apply_hc(psi, n, spec), l, 1)[idx]     # rest of layer l: its mixers
        for o in layers[l][1]:
            psi = SV.apply(psi, n, o.qubits, o.mat)
        grads[:, p + l] = run_from(_apply_hm(psi, n), l + 1, 0)[idx] if l + 1 < p else _apply_hm(psi, n)[idx]
    return psi[idx], grads


def amp_and_grad_tn(spec, bitstrings, columns=None):
    """The same derivatives for circuits too wide for a state vector.

    Each derivative is the sum over the layer's terms c G (c = w_e for
    G = Z_u Z_v, h_j for Z_j, 1 for X_j) of c times the amplitude of the
    circuit with the gate -i G inserted right after the term's gate, evaluated
    by the variable-elimination oracle. columns: the derivative indices to
    compute (gammas 0..p-1, then betas p..2p-1); the others stay zero.
    """
    from . import tn as TN
    n, p = spec.n, spec.p
    ops = C.qaoa_circuit(spec)
    assert spec.depol2 == 0 and spec.ad_gamma == 0, "gradients of the noiseless circuit"
    cols = range(2 * p) if columns is None else columns
    per_layer = len(spec.edges) + (n if spec.h is not None else 0) + n
    grads = np.zeros((len(bitstrings), 2 * p), dtype=complex)
    for col in cols:
        l, is_beta = col % p, col >= p
        first = n + l * per_layer
        for t in range(per_layer):
            i = first + t
            mixer = t >= per_layer - n
            if mixer != is_beta:
                continue
            if mixer:
                coef, G = 1.0, PAULI_X
            elif t < len(spec.edges):
                coef, G = float(spec.weights[t]), np.kron(PAULI_Z, PAULI_Z)
            else:
                coef, G = float(spec.h[t - len(spec.edges)]), PAULI_Z
            ins = ops[:i + 1] + [C.gate(ops[i].qubits, -1j * G)] + ops[i + 1:]
            for k, x in enumerate(bitstrings):
                grads[k, col] += coef * TN.amplitudes(n, ins, x)
    return grads


def amp_grad_product_rule(n, ops, param_of_op, dmats, n_params, bitstrings):
    """d amp / d theta_k of a parameterised gate list by the product rule.

    Operation i depends on parameter param_of_op[i] (or -1); dmats lists the
    derivative matrices of the parameterised operations in operation order.
    d amp / d theta_k = sum over i with param_of_op[i] = k of the amplitude of
    the list with operation i's matrix replaced by its derivative (state
    vector, FP64). Returns grad [K, n_params] complex.
    """
    idx = np.asarray([int(sum(int(b) << q for q, b in enumerate(x))) for x in bitstrings])
    grads = np.zeros((len(idx), n_params), dtype=complex)
    j = 0
    for i, k in enumerate(param_of_op):
        if k < 0:
            continue
        repl = list(ops)
        repl[i] = C.gate(ops[i].qubits, dmats[j])
        j += 1
        grads[:, k] += SV.run(n, repl)[idx]
    return grads
