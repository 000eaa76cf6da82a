"""Pins for the light-cone correlator oracle (oracle/lightcone.py): the
vectorised density matrix against the full-matrix one, light-cone correlators
of noisy circuits against the whole circuit's density matrix (graphs where
the cone cuts gates and channels), and noiseless correlators of a 64-qubit
grid against the p = 1 closed form."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import circuit as C
from oracle import closed_form as CF
from oracle import lightcone as LC
from oracle import statevector as SV


def _rand_unitary(rng, d):
    q, r = np.linalg.qr(rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d)))
    return q * (np.diag(r) / np.abs(np.diag(r)))


def _full_zz(spec, u, v):
    prob = np.real(np.diag(SV.density_run(spec.n, C.qaoa_circuit(spec))))
    x = np.arange(1 << spec.n)
    z = (1 - 2 * ((x >> u) & 1)) * (1 - 2 * ((x >> v) & 1))
    return float(np.dot(prob, z))


def test_vectorised_density_matches_full_matrices():
    rng = np.random.default_rng(11)
    n = 4
    ops = []
    for _ in range(14):
        k = rng.integers(0, 5)
        if k == 0:
            ops.append(C.gate((int(rng.integers(n)),), _rand_unitary(rng, 2)))
        elif k == 1:
            a, b = rng.choice(n, 2, replace=False)
            ops.append(C.gate((int(a), int(b)), _rand_unitary(rng, 4)))
        elif k == 2:
            a, b = rng.choice(n, 2, replace=False)
            ops.append(C.kraus((int(a), int(b)), C.depolarizing2_kraus(0.3)))
        elif k == 3:
            ops.append(C.kraus((int(rng.integers(n)),), C.amplitude_damping_kraus(0.4)))
        else:
            ops.append(C.kraus((int(rng.integers(n)),), C.phase_damping_kraus(0.5)))
    want = np.real(np.diag(SV.density_run(n, ops)))
    got = LC.density_diag(n, ops)
    assert np.abs(got - want).max() < 1e-13
    assert abs(got.sum() - 1.0) < 1e-13


def test_pauli_rates_of_the_depolarizing_channel():
    r = LC._pauli_rates(C.depolarizing2_kraus(0.15))
    assert abs(r[0, 0] - 0.85) < 1e-15
    assert np.allclose(r.sum(), 1.0) and np.allclose(r[1:, :], 0.01) and np.allclose(r[0, 1:], 0.01)
    assert LC._pauli_rates(C.amplitude_damping_kraus(0.3)) is None
    assert LC._pauli_rates([np.kron(C.PAULI[1], C.PAULI[0]) + np.kron(C.PAULI[3], C.PAULI[3])]) is None


def _path(n, p, depol, ad, seed):
    e = np.array([(i, i + 1) for i in range(n - 1)], dtype=np.int64)
    rng = np.random.default_rng(seed)
    return W.QaoaSpec(n=n, edges=e, weights=rng.uniform(0.5, 1.5, len(e)),
                      gammas=rng.uniform(0, math.pi, p), betas=rng.uniform(0, math.pi, p),
                      depol2=depol, ad_gamma=ad)


@pytest.mark.parametrize("edge", [(0, 1), (3, 4)])
def test_light_cone_of_a_noisy_path_matches_the_whole_circuit(edge):
    """An 8-qubit path, p = 2, depolarizing 0.1 after each RZZ and damping
    0.2 per layer: the cone of radius 2 cuts RZZ gates and channels at its
    ends (the channels become their marginals); the correlator equals the
    whole circuit's density matrix. A cone of radius p - 1 would miss it."""
    spec = _path(8, 2, 0.1, 0.2, seed=4)
    u, v = edge
    keep = LC.region(spec.n, spec.edges, edge, 2)
    assert len(keep) < spec.n
    want = _full_zz(spec, u, v)
    got = LC.zz(spec, u, v)
    assert abs(got - want) < 1e-12, (got, want)
    small = LC.region(spec.n, spec.edges, edge, 1)
    prob = LC.density_diag(len(small), LC.reduced_ops(C.qaoa_circuit(spec), small))
    x = np.arange(1 << len(small))
    z = (1 - 2 * ((x >> small.index(u)) & 1)) * (1 - 2 * ((x >> small.index(v)) & 1))
    assert abs(float(np.dot(prob, z)) - want) > 1e-5   # (1.3e-4 and 6.9e-3 here)


def test_noise_changes_the_correlator():
    """The same path without its channels: a different correlator (the
    channels inside the cone are applied, not dropped)."""
    noisy = _path(8, 2, 0.1, 0.2, seed=4)
    clean = _path(8, 2, 0.0, 0.0, seed=4)
    assert abs(LC.zz(noisy, 3, 4) - LC.zz(clean, 3, 4)) > 1e-2
    assert abs(LC.zz(clean, 3, 4) - _full_zz(clean, 3, 4)) < 1e-12


def test_light_cone_of_a_noisy_grid_corner():
    """A 3x3 grid, p = 2, with noise: the corner edge's cone (radius 2) leaves
    out the far corner; a larger radius gives the same value."""
    e = W.grid_edges(3, 3)
    rng = np.random.default_rng(8)
    spec = W.QaoaSpec(n=9, edges=e, weights=np.ones(len(e)), gammas=rng.uniform(0, math.pi, 2),
                      betas=rng.uniform(0, math.pi, 2), depol2=0.08, ad_gamma=0.15)
    assert len(LC.region(9, e, (0, 1), 2)) == 8
    want = _full_zz(spec, 0, 1)
    assert abs(LC.zz(spec, 0, 1) - want) < 1e-12
    assert abs(LC.zz(spec, 0, 1, radius=3) - want) < 1e-12


def test_noiseless_grid_correlators_against_the_closed_form():
    """The 8x8 grid (64 qubits) at p = 1 with random weights: every cone
    correlator equals the p = 1 closed form."""
    e = W.grid_edges(8, 8)
    rng = np.random.default_rng(2)
    spec = W.QaoaSpec(n=64, edges=e, weights=rng.normal(size=len(e)), gammas=np.array([0.37]),
                      betas=np.array([1.13]))
    pairs = [tuple(int(x) for x in e[i]) for i in (0, 17, 60, len(e) - 1)]
    want = CF.zz_p1(64, e, spec.weights, 0.37, 1.13, pairs)
    for (u, v), w in zip(pairs, want):
        assert abs(LC.zz(spec, u, v) - w) < 1e-12


def test_cone_radius_below_p_is_refused():
    spec = _path(6, 2, 0.0, 0.0, seed=1)
    with pytest.raises(ValueError):
        LC.zz(spec, 0, 1, radius=1)
