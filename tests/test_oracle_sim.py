"""Pins for the state-vector, density-matrix, elimination and closed-form oracles."""
import math
from functools import reduce

import numpy as np
from scipy.linalg import expm

import workloads as W
from oracle import circuit as C
from oracle import closed_form as CF
from oracle import statevector as SV
from oracle import tn as TN

X = np.array([[0, 1], [1, 0]], dtype=complex)
Z = np.array([[1, 0], [0, -1]], dtype=complex)
I2 = np.eye(2, dtype=complex)


def _kron_on(n, ops_by_qubit):
    """Full operator from single-qubit factors, qubit q = bit q (kron, MSB first)."""
    return reduce(np.kron, [ops_by_qubit.get(q, I2) for q in reversed(range(n))])


def _rand_unitary(rng, d):
    q, r = np.linalg.qr(rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d)))
    return q * (np.diag(r) / np.abs(np.diag(r)))


def test_apply_matches_full_matrix():
    rng = np.random.default_rng(3)
    n = 5
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    for qs in ((2,), (4, 1), (0, 3, 2)):
        U = _rand_unitary(rng, 1 << len(qs))
        assert np.allclose(SV.apply(psi, n, qs, U), SV.embed(n, qs, U) @ psi, atol=1e-12)
    # embed of single-qubit gates equals the plain Kronecker product
    U = _rand_unitary(rng, 2)
    assert np.allclose(SV.embed(n, (3,), U), _kron_on(n, {3: U}))


def test_qaoa_state_matches_matrix_exponentials():
    # App. D: |Psi> = U_M(beta_p) U_C(gamma_p) ... U_M(beta_1) U_C(gamma_1) |+>^n,
    # U_C = exp(-i gamma H_C), U_M = exp(-i beta H_M), H_C = sum_e w_e Z_u Z_v + sum_j h_j Z_j
    for seed, n, p in ((11, 6, 1), (12, 7, 2), (13, 8, 3)):
        spec = W.random_qaoa(n, p, seed=seed, with_h=True)
        HC = np.zeros((1 << n, 1 << n), dtype=complex)
        for (u, v), w in zip(spec.edges, spec.weights):
            HC += w * _kron_on(n, {int(u): Z, int(v): Z})
        for j in range(n):
            HC += spec.h[j] * _kron_on(n, {j: Z})
        HM = sum(_kron_on(n, {j: X}) for j in range(n))
        psi = np.full(1 << n, 2 ** (-n / 2), dtype=complex)
        for l in range(p):
            psi = expm(-1j * spec.gammas[l] * HC) @ psi
            psi = expm(-1j * spec.betas[l] * HM) @ psi
        got = SV.run(n, C.qaoa_circuit(spec))
        assert np.allclose(got, psi, atol=1e-11)


def test_density_matrix_of_unitary_circuit_is_pure_state():
    spec = W.random_qaoa(5, 2, seed=21, with_h=True)
    ops = C.qaoa_circuit(spec)
    psi = SV.run(spec.n, ops)
    rho = SV.density_run(spec.n, ops)
    assert np.allclose(rho, np.outer(psi, psi.conj()), atol=1e-12)


def test_density_matrix_is_a_state_under_noise():
    spec = W.random_qaoa(4, 2, seed=22, depol2=0.3, ad_gamma=0.4)
    rho = SV.density_run(spec.n, C.qaoa_circuit(spec))
    assert abs(np.trace(rho) - 1) < 1e-12
    assert np.allclose(rho, rho.conj().T, atol=1e-13)
    assert np.min(np.linalg.eigvalsh(rho)) > -1e-12


def test_full_depolarizing_gives_maximally_mixed_pair():
    # p = 15/16 two-qubit depolarizing maps every 2-qubit state to I/4
    ops = [C.gate((0,), C.h_mat()), C.gate((1,), C.rx_mat(0.8)),
           C.kraus((0, 1), C.depolarizing2_kraus(15 / 16))]
    rho = SV.density_run(2, ops)
    assert np.allclose(rho, np.eye(4) / 4, atol=1e-13)


def test_amplitude_damping_closed_form():
    # |1> decays to |0> with probability gamma per channel: P(1) = (1-g)^k
    g = 0.3
    ops = [C.gate((0,), C.rx_mat(math.pi))] + [C.kraus((0,), C.amplitude_damping_kraus(g))] * 3
    rho = SV.density_run(1, ops)
    assert abs(rho[1, 1].real - (1 - g) ** 3) < 1e-14


def _random_general_circuit(rng, n, T):
    ops = []
    for q in range(n):
        ops.append(C.gate((q,), C.h_mat()))
    for _ in range(T):
        k = rng.integers(0, 7)
        a, b = (int(v) for v in rng.choice(n, 2, replace=False))
        if k == 0:
            ops.append(C.gate((a,), C.rx_mat(rng.uniform(0, 3))))
        elif k == 1:
            ops.append(C.gate((a, b), C.rzz_mat(rng.uniform(-3, 3))))
        elif k == 2:
            ops.append(C.gate((a, b), C.cnot_mat()))
        elif k == 3:
            ops.append(C.gate((a, b), C.fsim_mat(rng.uniform(0, 3), rng.uniform(0, 3))))
        elif k == 4:
            ops.append(C.gate((a, b), C.crx_mat(rng.uniform(0, 3))))
        elif k == 5:
            ops.append(C.gate((a,), _rand_unitary(rng, 2)))
        else:
            ops.append(C.gate((a, b), _rand_unitary(rng, 4)))
    return ops


def test_elimination_matches_state_vector():
    rng = np.random.default_rng(5)
    for trial in range(6):
        n = int(rng.integers(3, 8))
        ops = _random_general_circuit(rng, n, int(rng.integers(5, 25)))
        for t in (len(ops) // 2, len(ops)):
            psi = SV.run(n, ops[:t])
            for _ in range(3):
                x = rng.integers(0, 2, n)
                idx = sum(int(b) << q for q, b in enumerate(x))
                a = TN.amplitudes(n, ops[:t], x)
                assert abs(a - psi[idx]) < 1e-12
            # one open qubit: both candidates from one contraction
            last = ops[t - 1]
            q = last.qubits[0]
            x = rng.integers(0, 2, n)
            if not C.is_diagonal(last.mat) or q >= 0:
                try:
                    tab = TN.amplitudes(n, ops[:t], x, open_qubits=(q,))
                except ValueError:
                    continue
                for y in range(2):
                    xx = x.copy()
                    xx[q] = y
                    idx = sum(int(b) << qq for qq, b in enumerate(xx))
                    assert abs(tab[y] - psi[idx]) < 1e-12


def test_elimination_on_qaoa_prefixes():
    spec = W.random_qaoa(10, 2, seed=31, with_h=True)
    ops = C.qaoa_circuit(spec)
    rng = np.random.default_rng(6)
    for t in (10, 40, 62, len(ops)):
        psi = SV.run(spec.n, ops[:t])
        x = rng.integers(0, 2, spec.n)
        idx = sum(int(b) << q for q, b in enumerate(x))
        assert abs(TN.amplitudes(spec.n, ops[:t], x) - psi[idx]) < 1e-12


def test_closed_form_single_edge():
    g, b = 0.41, 0.93
    v = CF.zz_p1(2, np.array([[0, 1]]), np.array([1.0]), g, b)[0]
    assert abs(v - math.sin(4 * b) * math.sin(2 * g)) < 1e-15


def test_closed_form_matches_state_vector():
    for seed, n in ((41, 8), (42, 10), (43, 12)):
        spec = W.random_qaoa(n, 1, seed=seed)
        psi = SV.run(n, C.qaoa_circuit(spec))
        pr = np.abs(psi) ** 2
        idx = np.arange(1 << n)
        pairs = [(int(u), int(v)) for u, v in spec.edges] + [(0, n - 1), (1, n // 2)]
        cf = CF.zz_p1(n, spec.edges, spec.weights, spec.gammas[0], spec.betas[0], pairs=pairs)
        for (u, v), val in zip(pairs, cf):
            z = (1 - 2 * ((idx >> u) & 1)) * (1 - 2 * ((idx >> v) & 1))
            assert abs(float((pr * z).sum()) - val) < 1e-12
