"""Pins of the trajectory oracle: the branch-weighted average equals the
density-matrix diagonal, sampled trajectories match it within shot noise, and
a noiseless circuit reduces to |psi|^2."""
import numpy as np

import workloads as W
from oracle import circuit as OC
from oracle import sampler as OS
from oracle import statevector as SV
from oracle import trajectory as TR


def _noisy_spec():
    spec = W.random_qaoa(4, 1, seed=51, with_h=True, depol2=0.2, ad_gamma=0.3)
    spec.edges = spec.edges[:2]
    spec.weights = spec.weights[:2]
    return spec


def test_branch_average_equals_density_matrix():
    ops = OC.qaoa_circuit(_noisy_spec())
    want = np.real(np.diag(SV.density_run(4, ops)))
    assert np.abs(TR.exact_distribution(4, ops) - want).max() < 1e-12


def test_branch_average_equals_alg2_enumeration():
    spec = W.random_qaoa(3, 1, seed=54, with_h=True, depol2=0.2, ad_gamma=0.3)
    spec.edges = spec.edges[:1]
    spec.weights = spec.weights[:1]
    ops = OC.qaoa_circuit(spec)
    got = TR.exact_distribution(3, ops)
    want = OS.exact_noisy_distribution(3, ops)
    assert np.abs(got - np.asarray(want)).max() < 1e-12


def test_noiseless_reduces_to_state_vector():
    spec = W.random_qaoa(5, 2, seed=52, with_h=True)
    ops = OC.qaoa_circuit(spec)
    assert np.abs(TR.exact_distribution(5, ops) - np.abs(SV.run(5, ops)) ** 2).max() < 1e-14


def test_sampled_trajectories_within_shot_noise():
    ops = OC.qaoa_circuit(_noisy_spec())
    rng = np.random.default_rng(53)
    N = 4000
    counts = np.zeros(16)
    for _ in range(N):
        x = TR.sample(4, ops, rng)
        counts[int(sum(int(b) << q for q, b in enumerate(x)))] += 1
    p = TR.exact_distribution(4, ops)
    tvd = 0.5 * np.abs(counts / N - p).sum()
    # E[TVD] <= 0.5 sum sqrt(p (1 - p) / N); allow three times that
    assert tvd < 1.5 * np.sqrt(p * (1 - p) / N).sum()
