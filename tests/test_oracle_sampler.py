"""Pins for the oracle's Alg. 1 / Alg. 2 samplers."""
import math

import numpy as np

import workloads as W
from oracle import circuit as C
from oracle import sampler as S
from oracle import statevector as SV
from tests.test_oracle_sim import _random_general_circuit


def test_markov_condition_eq1_every_gate():
    # Eq. (1): applying the UpdateState kernel to p_{t-1} gives p_t, for every t
    rng = np.random.default_rng(7)
    for _ in range(4):
        n = int(rng.integers(2, 5))
        ops = _random_general_circuit(rng, n, 14)
        chain, exact = S.exact_chain_distributions(n, ops)
        for a, b in zip(chain, exact):
            assert np.max(np.abs(a - b)) < 1e-12


def test_kernel_rows_stochastic_and_block_norm_preserved():
    # Sec. 2 proof: sum_y p(x->y) = 1 and sum_{block} p_{t-1} = sum_{block} p_t
    rng = np.random.default_rng(8)
    n = 4
    ops = _random_general_circuit(rng, n, 10)
    psi = SV.zero_state(n)
    for op in ops:
        prev = psi
        psi = SV.apply(psi, n, op.qubits, op.mat)
        P = S.transition_kernel(n, op.mat, op.qubits, psi)
        assert np.allclose(P.sum(axis=1), 1.0)
        if C.is_monomial(op.mat):
            continue
        for xg in range(1 << n):
            bits = [(xg >> q) & 1 for q in range(n)]
            xl = C.local_index(bits, op.qubits)
            ys = [sum(int(b) << q for q, b in enumerate(C.set_local(bits, op.qubits, y)))
                  for y in C.block_decompose_local(op.mat, xl)]
            assert abs(sum(abs(prev[y]) ** 2 for y in ys) - sum(abs(psi[y]) ** 2 for y in ys)) < 1e-12


def test_qaoa_markov_condition():
    spec = W.random_qaoa(5, 2, seed=51, with_h=True)
    chain, exact = S.exact_chain_distributions(spec.n, C.qaoa_circuit(spec))
    assert max(np.max(np.abs(a - b)) for a, b in zip(chain, exact)) < 1e-12


def _tvd_threshold(p, N, reps, rng):
    tv = []
    for _ in range(reps):
        c = rng.multinomial(N, p)
        tv.append(0.5 * np.abs(c / N - p).sum())
    return float(np.quantile(tv, 0.99))


def test_sampler_distribution_config1_tvd():
    # Alg. 1 with Philox draws: TVD to |psi_T|^2 within the 99th percentile of
    # i.i.d. multinomial draws of the same size
    spec = W.maxcut_3reg_n12()
    ops = C.qaoa_circuit(spec)
    p = np.abs(SV.run(spec.n, ops)) ** 2
    N = 4000
    samples, stats = S.sample_sv(spec.n, ops, seed=2024, sample_ids=range(N))
    idx = (samples.astype(np.int64) << np.arange(spec.n)).sum(axis=1)
    emp = np.bincount(idx, minlength=1 << spec.n) / N
    tvd = 0.5 * np.abs(emp - p).sum()
    thr = _tvd_threshold(p, N, 200, np.random.default_rng(1))
    assert tvd < thr
    # Sec. 2: at most 2T amplitude calls per sample (two candidates per gate)
    assert stats.amp_calls <= 2 * len(ops) * N
    assert stats.zero_mass == 0


def test_global_flip_symmetry_of_samples():
    # MaxCut with h = 0: p(x) = p(not x), so every bit has mean 1/2
    spec = W.maxcut_3reg_n12()
    ops = C.qaoa_circuit(spec)
    samples, _ = S.sample_sv(spec.n, ops, seed=99, sample_ids=range(3000))
    m = samples.mean(axis=0)
    assert np.all(np.abs(m - 0.5) < 4.5 * 0.5 / math.sqrt(3000))


def test_tn_and_sv_samplers_agree_bit_for_bit():
    spec = W.random_qaoa(8, 2, seed=61, with_h=True)
    ops = C.qaoa_circuit(spec)
    ids = list(range(6))
    sv, st = S.sample_sv(spec.n, ops, seed=5, sample_ids=ids)
    for k, sid in enumerate(ids):
        s, st2 = S.sample_tn(spec.n, ops, seed=5, sample_id=sid)
        if st2.near_boundary == 0:
            assert np.array_equal(s, sv[k])


def test_permuted_mixer_order_gives_same_distribution():
    # RX gates of one layer commute: a permuted execution order samples the same law
    spec = W.random_qaoa(4, 2, seed=62)
    ops = C.qaoa_circuit(spec)
    n = spec.n
    order = list(range(len(ops)))
    # reverse the RX block of the last layer
    rx = [i for i, o in enumerate(ops) if o.kind == "gate" and len(o.qubits) == 1][-n:]
    for a, b in zip(rx, reversed(rx)):
        order[a] = b
    perm = [ops[i] for i in order]
    chain, exact = S.exact_chain_distributions(n, perm)
    p_final = np.abs(SV.run(n, ops)) ** 2
    assert np.allclose(chain[-1], p_final, atol=1e-12)


def _small_noisy_circuits():
    out = []
    ops = [C.gate((0,), C.h_mat()), C.gate((1,), C.h_mat()),
           C.gate((0, 1), C.rzz_mat(1.3)),
           C.kraus((0, 1), C.depolarizing2_kraus(0.3)),
           C.gate((0,), C.rx_mat(0.9)), C.gate((1,), C.rx_mat(0.9)),
           C.kraus((0,), C.amplitude_damping_kraus(0.5)),
           C.gate((0, 1), C.rzz_mat(-0.7)),
           C.gate((1,), C.rx_mat(2.1)),
           C.kraus((1,), C.amplitude_damping_kraus(0.35))]
    out.append((2, ops))
    ops = [C.gate((q,), C.h_mat()) for q in range(3)]
    ops += [C.gate((0, 1), C.rzz_mat(0.8)), C.kraus((1,), C.depolarizing1_kraus(0.4)),
            C.gate((1, 2), C.rzz_mat(1.7)), C.kraus((2,), C.phase_damping_kraus(0.5)),
            C.gate((0,), C.rx_mat(1.2)), C.gate((1,), C.rx_mat(0.4)), C.gate((2,), C.rx_mat(2.6)),
            C.kraus((0,), C.amplitude_damping_kraus(0.6)),
            C.gate((0, 2), C.rzz_mat(2.2)),
            C.gate((2,), C.rx_mat(0.5)), C.gate((0,), C.rx_mat(1.5))]
    out.append((3, ops))
    return out


def test_noisy_exact_distribution_matches_density_matrix():
    # Alg. 2 with Eq. (5) at the true bit reproduces diag(rho) exactly
    for n, ops in _small_noisy_circuits():
        d = S.exact_noisy_distribution(n, ops)
        rho = SV.density_run(n, ops)
        assert np.max(np.abs(d - np.real(np.diag(rho)))) < 1e-12
        assert abs(d.sum() - 1) < 1e-12


def test_noise_draw_at_s_only_is_wrong_for_amplitude_damping():
    # the other reading of Eq. (5) (bit s instead of s XOR x) disagrees with the
    # density matrix once a frame flip precedes an amplitude-damping channel
    n, ops = _small_noisy_circuits()[0]
    d = S.exact_noisy_distribution(n, ops, kraus_rule="s_only")
    rho = SV.density_run(n, ops)
    assert np.max(np.abs(d - np.real(np.diag(rho)))) > 1e-3


def test_noisy_sampler_statistics_and_backends():
    n, ops = _small_noisy_circuits()[1]
    rho = SV.density_run(n, ops)
    p = np.real(np.diag(rho))
    N = 3000
    cnt = np.zeros(1 << n)
    for sid in range(N):
        s, _ = S.noisy_sample(n, ops, seed=17, sample_id=sid)
        cnt[sum(int(b) << q for q, b in enumerate(s))] += 1
    tvd = 0.5 * np.abs(cnt / N - p).sum()
    assert tvd < _tvd_threshold(p, N, 200, np.random.default_rng(2))
    for sid in range(20):
        a, _ = S.noisy_sample(n, ops, seed=17, sample_id=sid, backend="sv")
        b, st = S.noisy_sample(n, ops, seed=17, sample_id=sid, backend="tn")
        if st.near_boundary == 0:
            assert np.array_equal(a, b)


def test_lsm_noise_leaves_network_shape_unchanged():
    # Prop. 2: every gate Alg. 2 adds for LSM noise is a one-qubit diagonal, so
    # the simulated circuit differs from the noiseless prefix only by those
    n, ops = _small_noisy_circuits()[0]
    added = []
    for op in ops:
        if op.kind != "kraus":
            continue
        for E in op.mats:
            for M, q in C.lsm_factorize(E, op.qubits):
                MX = M @ C.SIGMA_X
                D = MX if (C.is_diagonal(MX) and not C.is_diagonal(M)) else M
                added.append(C.is_diagonal(D))
    assert all(added)


def _with_swaps(rng, n):
    spec = W.random_qaoa(n, 2, seed=int(rng.integers(1000)), with_h=True)
    ops = C.qaoa_circuit(spec)
    S_ = np.eye(4)[[0, 2, 1, 3]].astype(complex)
    pos = n + len(spec.edges) + n       # end of layer 1's diagonal section
    return ops[:n] + [C.gate((0, n - 1), C.iswap_mat())] + ops[n:pos] + \
        [C.gate((1, 2), S_ @ np.diag(np.exp(1j * rng.uniform(0, 6.3, 4))))] + ops[pos:]


def test_markov_condition_with_swap_class_gates():
    # Eq. (1) at every gate also across SWAP-class (monomial two-qubit) gates
    rng = np.random.default_rng(17)
    ops = _with_swaps(rng, 4)
    chain, exact = S.exact_chain_distributions(4, ops)
    for a, b in zip(chain, exact):
        assert np.max(np.abs(a - b)) < 1e-12


def test_wire_relabelling_identity():
    """The identity the planner uses for SWAP-class gates A = SWAP D: replacing
    each by its phase D on the current wires of its qubits, moving the qubits'
    contents between wires and acting with every later operation on the wires
    its qubits' contents are on gives the original state with qubit q read
    from wire wire_of[q]."""
    rng = np.random.default_rng(18)
    n = 5
    ops = _with_swaps(rng, n)
    wire_of = list(range(n))
    relabelled = []
    for op in ops:
        A = op.mat
        qs = tuple(wire_of[q] for q in op.qubits)
        if len(op.qubits) == 2 and C.is_monomial(A) and not C.is_diagonal(A) and \
                all(A[((x & 1) << 1) | (x >> 1), x] != 0 for x in range(4)):
            D = np.diag([A[((x & 1) << 1) | (x >> 1), x] for x in range(4)])
            relabelled.append(C.gate(qs, D))
            a, b = op.qubits
            wire_of[a], wire_of[b] = wire_of[b], wire_of[a]
        else:
            relabelled.append(C.gate(qs, A))
    psi = SV.run(n, ops)
    phi = SV.run(n, relabelled)
    for x in range(1 << n):
        w = sum(((x >> q) & 1) << wire_of[q] for q in range(n))
        assert abs(psi[x] - phi[w]) < 1e-13
