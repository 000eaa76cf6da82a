"""Pins for gate semantics, classification, BlockDecompose and the noise algebra."""
import math

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import circuit as C

X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z = np.array([[1, 0], [0, -1]], dtype=complex)


def test_rotations_match_exponentials():
    # App. D: R_P(theta) = exp(-i theta P / 2)
    for th in (0.0, 0.37, 1.9, -2.4):
        assert np.allclose(C.rx_mat(th), expm(-0.5j * th * X), atol=1e-14)
        assert np.allclose(C.rz_mat(th), expm(-0.5j * th * Z), atol=1e-14)
        assert np.allclose(C.rzz_mat(th), expm(-0.5j * th * np.kron(Z, Z)), atol=1e-14)
    Hm = (X + Z) / math.sqrt(2)
    assert np.allclose(C.h_mat(), Hm)


def test_figure1_monomial_gates():
    # Fig. 1b: CNOT and iSWAP are monomial
    assert C.is_monomial(C.cnot_mat())
    assert C.is_monomial(C.iswap_mat())
    assert not C.is_monomial(C.h_mat())
    assert C.is_monomial(C.rzz_mat(0.3)) and C.is_diagonal(C.rzz_mat(0.3))
    # CNOT moves |b0=1,b1=0> to |1,1>
    assert C.monomial_image(C.cnot_mat(), 1) == 3
    assert C.monomial_image(C.cnot_mat(), 3) == 1
    assert C.monomial_image(C.iswap_mat(), 1) == 2


def test_figure1_block_structure():
    # Fig. 1c: controlled RX has blocks {00}, {10 in q1}, and the 2-block on the
    # control=1 subspace; fSim has blocks {00}, {01,10}, {11}
    A = C.crx_mat(0.7)
    assert C.block_decompose_local(A, 0) == [0]
    assert C.block_decompose_local(A, 2) == [2]
    assert C.block_decompose_local(A, 1) == [1, 3]
    assert C.block_decompose_local(A, 3) == [1, 3]
    F = C.fsim_mat(0.4, 0.9)
    assert C.block_decompose_local(F, 0) == [0]
    assert C.block_decompose_local(F, 1) == [1, 2]
    assert C.block_decompose_local(F, 3) == [3]
    # RX / H: one block of size 2
    assert C.block_decompose_local(C.rx_mat(0.3), 0) == [0, 1]
    assert C.block_decompose_local(C.h_mat(), 1) == [0, 1]


def test_controlled_one_qubit_gate_max_block_two():
    # Sec. 2: a one-qubit gate with any number of controls has blocks of size <= 2
    rng = np.random.default_rng(0)
    G = np.linalg.qr(rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2)))[0]
    for nctrl in (1, 2, 3):
        dim = 1 << (nctrl + 1)
        A = np.eye(dim, dtype=complex)
        allc = (1 << nctrl) - 1
        for a in range(2):
            for b in range(2):
                A[allc + (a << nctrl), allc + (b << nctrl)] = G[a, b]
        sizes = [len(C.block_decompose_local(A, x)) for x in range(dim)]
        assert max(sizes) == 2


def test_blocks_are_invariant_subspaces():
    # Sec. 2 justification: no nonzero entry connects a component to its complement
    rng = np.random.default_rng(1)
    for A in (C.crx_mat(1.1), C.fsim_mat(0.2, 0.5), C.cnot_mat()):
        for x in range(4):
            b = set(C.block_decompose_local(A, x))
            rest = [y for y in range(4) if y not in b]
            for u in b:
                for v in rest:
                    assert A[u, v] == 0 and A[v, u] == 0
        _ = rng


def test_kraus_completeness():
    for Es in (C.depolarizing2_kraus(0.03), C.depolarizing1_kraus(0.2),
               C.amplitude_damping_kraus(0.3), C.phase_damping_kraus(0.4)):
        d = Es[0].shape[0]
        S = sum(E.conj().T @ E for E in Es)
        assert np.allclose(S, np.eye(d), atol=1e-14)


def test_antidiagonal_factorisation():
    # Sec. 3.2: A = [[0,a],[b,0]] = sigma_X diag(b, a); Alg. 2 uses M sigma_X = diag(a, b)
    a, b = 0.3 + 0.1j, -0.7j
    A = np.array([[0, a], [b, 0]])
    assert np.allclose(A, X @ np.diag([b, a]))
    assert np.allclose(A @ X, np.diag([a, b]))
    assert C.is_diagonal(A @ X)


def test_permutation_conjugates_diagonal_to_diagonal():
    # Sec. 3.2: P D P^dag is diagonal with permuted entries
    rng = np.random.default_rng(2)
    d = rng.normal(size=8) + 1j * rng.normal(size=8)
    perm = rng.permutation(8)
    P = np.zeros((8, 8))
    P[perm, np.arange(8)] = 1
    M = P @ np.diag(d) @ P.T
    assert C.is_diagonal(M)
    assert np.allclose(np.diag(M)[perm], d)


def test_lsm_factorisation():
    for Es, qs in ((C.depolarizing2_kraus(0.1), (3, 5)), (C.amplitude_damping_kraus(0.2), (4,))):
        for E in Es:
            fac = C.lsm_factorize(E, qs)
            if len(qs) == 2:
                assert np.allclose(np.kron(fac[1][0], fac[0][0]), E)
            for M, _ in fac:
                assert C.is_submonomial(M)
    with pytest.raises(ValueError):
        C.lsm_factorize(C.h_mat(), (0,))
    with pytest.raises(ValueError):
        C.lsm_factorize(C.cnot_mat() * 0.5 + C.iswap_mat() * 0.5, (0, 1))


def test_depolarizing_pauli_order():
    Es = C.depolarizing2_kraus(0.15)
    # k = a + 4 b: Pauli a on q_0 (least significant), Pauli b on q_1
    k = 1 + 4 * 3   # X on q_0, Z on q_1
    assert np.allclose(Es[k], math.sqrt(0.01) * np.kron(Z, X))
    assert np.allclose(Es[0], math.sqrt(0.85) * np.eye(4))


def test_qaoa_circuit_structure():
    import workloads as W
    spec = W.grid_6x6_p2()
    ops = C.qaoa_circuit(spec)
    n, E, p = spec.n, len(spec.edges), spec.p
    assert len(ops) == n + p * (E + n)
    nonmono = [o for o in ops if o.kind == "gate" and not C.is_monomial(o.mat)]
    assert len(nonmono) == n + p * n
    noisy = W.grid_8x8_p2_noisy()
    ops3 = C.qaoa_circuit(noisy)
    nk = sum(o.kind == "kraus" for o in ops3)
    assert nk == noisy.p * (len(noisy.edges) + noisy.n)
