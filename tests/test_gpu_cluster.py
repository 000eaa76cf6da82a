"""GPU parity of the thread-block-cluster path (frontier split over CTAs).

A frontier too large for one CTA's shared memory is spread over a cluster;
the same split can be forced on small circuits so that the state-vector and
Alg. 2 oracles check it bit for bit.
"""
import numpy as np
import pytest

import workloads as W
from oracle import circuit as OC
from oracle import sampler as OS

from tests.test_gpu_parity import _circ, pair_err, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_24218_gb300 as mod
    mod.load_library()
    return mod


def _grid_spec(rows, cols, p, seed, **noise):
    spec = W.random_qaoa(rows * cols, p, seed=seed, with_h=True, **noise)
    e = W.grid_edges(rows, cols)
    spec.edges = e
    spec.weights = np.random.default_rng(seed).normal(size=len(e))
    return spec


@pytest.mark.parametrize("cr", [2, 4, 8])
def test_forced_cluster_split_bitwise(pw, cr):
    spec = _grid_spec(4, 4, 2, seed=90 + cr)
    g = run_gpu(pw, spec, 64, seed=cr, ctas_per_chain=cr, order=pw.PW_ORDER_NATURAL)
    assert g["plan_stats"]["ctas_per_chain"] == cr
    ops = OC.qaoa_circuit(spec)
    traces = [[] for _ in range(64)]
    want, ost = OS.sample_sv(spec.n, ops, cr, list(range(64)), order=g["order"], traces=traces)
    mism = int((~(want == g["bits"]).all(axis=1)).sum())
    assert mism <= max(ost.near_boundary, g["stats"]["near_boundary"])
    worst = max(pair_err(traces[k][spec.n + r][1], g["trace"][k, r])
                for k in range(64) if (want[k] == g["bits"][k]).all() for r in range(g["plan_stats"]["sampled_gates"]))
    assert worst < 1e-5


@pytest.mark.parametrize("cr", [2, 8])
def test_forced_cluster_split_noisy(pw, cr):
    spec = _grid_spec(4, 4, 2, seed=70 + cr, depol2=0.2, ad_gamma=0.3)
    g = run_gpu(pw, spec, 40, seed=cr, trace=False, ctas_per_chain=cr, order=pw.PW_ORDER_NATURAL)
    ops = OC.qaoa_circuit(spec)
    mism, near = 0, 0
    for k in range(40):
        s, st = OS.noisy_sample(spec.n, ops, cr, k, order=g["order"])
        near += st.near_boundary
        mism += int(not np.array_equal(s, g["bits"][k]))
    assert mism <= max(near, g["stats"]["near_boundary"])


def test_cluster_matches_single_cta(pw):
    """7x7 grid, p = 2 (2^14-entry frontier): one CTA per chain and a forced
    4-CTA cluster give the same samples and amplitudes."""
    spec = _grid_spec(7, 7, 2, seed=5)
    a = run_gpu(pw, spec, 512, seed=3)
    b = run_gpu(pw, spec, 512, seed=3, ctas_per_chain=4)
    assert a["plan_stats"]["ctas_per_chain"] == 1 and b["plan_stats"]["ctas_per_chain"] == 4
    same = (a["bits"] == b["bits"]).all(axis=1)
    assert (~same).sum() <= max(a["stats"]["near_boundary"], b["stats"]["near_boundary"])
    k = int(np.nonzero(same)[0][0])
    rows = a["plan_stats"]["sampled_gates"]
    worst = max(pair_err(a["trace"][k, r][0::2] + 1j * a["trace"][k, r][1::2], b["trace"][k, r]) for r in range(rows))
    assert worst < 1e-5


def test_grid8x8_noisy_chain_against_alg2(pw):
    """The 64-qubit noisy workload (8x8 grid, p = 2, depolarizing 1e-3 after
    every RZZ, amplitude damping 1e-3 per qubit per layer) on its cluster
    path: one chain against Alg. 2 with elimination amplitudes, bit for bit and
    amplitude pair by amplitude pair along the same trajectory."""
    spec = W.grid_8x8_p2_noisy()
    g = run_gpu(pw, spec, 4, seed=2027)
    assert g["plan_stats"]["ctas_per_chain"] > 1
    ops = OC.qaoa_circuit(spec)
    trace = []
    s, st = OS.noisy_sample(spec.n, ops, 2027, 3, order=g["order"], backend="tn", trace=trace)
    if st.near_boundary == 0:
        assert np.array_equal(s, g["bits"][3])
    rows = [t for t in trace if len(t[0]) == 2][spec.n:]
    assert len(rows) == g["plan_stats"]["sampled_gates"]
    worst = max(pair_err(rows[r][1], g["trace"][3, r]) for r in range(len(rows)))
    assert worst < 1e-5


def test_grid8x8_noisy_dirty_chains_against_alg2(pw):
    """The 8x8 p=2 cluster plan with noise rates raised to 4e-3: chains that
    draw a Kraus operator other than 0 midway leave the clean state (from then
    on tables built per chain and draws in dependency waves), the others keep
    the host-evaluated tables. Every chain must follow Alg. 2 bit for bit and
    amplitude pair by amplitude pair."""
    spec = W.grid_8x8_p2_noisy()
    spec.depol2 = 0.004
    spec.ad_gamma = 0.004
    g = run_gpu(pw, spec, 3, seed=77)
    assert g["plan_stats"]["ctas_per_chain"] > 1
    ops = OC.qaoa_circuit(spec)
    dirty = 0
    for k in range(3):
        trace, events = [], []
        s, st = OS.noisy_sample(spec.n, ops, 77, k, order=g["order"], backend="tn", trace=trace, events=events)
        dirty += int(any(i != 0 for _, i in events))
        if st.near_boundary == 0:
            assert np.array_equal(s, g["bits"][k])
        rows = [t for t in trace if len(t[0]) == 2][spec.n:]
        worst = max(pair_err(rows[r][1], g["trace"][k, r]) for r in range(len(rows)))
        assert worst < 1e-5
    assert dirty >= 1


@pytest.mark.parametrize("cr", [2, 8])
def test_forced_cluster_split_fp64(pw, cr):
    """The FP64 build on the cluster path (the 64-qubit grid's FP64 plan uses
    it by itself): bits equal to Alg. 1 and candidate pairs to 1e-12."""
    spec = _grid_spec(4, 4, 2, seed=110 + cr)
    g = run_gpu(pw, spec, 48, seed=cr, precision=pw.PW_PREC_FP64, ctas_per_chain=cr, order=pw.PW_ORDER_NATURAL)
    assert g["plan_stats"]["ctas_per_chain"] == cr
    ops = OC.qaoa_circuit(spec)
    traces = [[] for _ in range(48)]
    want, ost = OS.sample_sv(spec.n, ops, cr, list(range(48)), order=g["order"], traces=traces)
    mism = int((~(want == g["bits"]).all(axis=1)).sum())
    assert mism <= max(ost.near_boundary, g["stats"]["near_boundary"])
    worst = max(pair_err(traces[k][spec.n + r][1], g["trace"][k, r])
                for k in range(48) if (want[k] == g["bits"][k]).all() for r in range(g["plan_stats"]["sampled_gates"]))
    assert worst < 1e-12


def test_grid8x8_noisy_fp64_plan_runs_on_eight_ctas(pw):
    """The 64-qubit noisy workload in FP64 needs 8 CTAs per chain (2^13 of the
    2^16 entries each): one chain against Alg. 2 bit for bit and its candidate
    pairs to 1e-10 along the trajectory."""
    spec = W.grid_8x8_p2_noisy()
    g = run_gpu(pw, spec, 2, seed=2031, precision=pw.PW_PREC_FP64)
    assert g["plan_stats"]["ctas_per_chain"] == 8
    ops = OC.qaoa_circuit(spec)
    trace = []
    s, st = OS.noisy_sample(spec.n, ops, 2031, 1, order=g["order"], backend="tn", trace=trace)
    if st.near_boundary == 0:
        assert np.array_equal(s, g["bits"][1])
    rows = [t for t in trace if len(t[0]) == 2][spec.n:]
    worst = max(pair_err(rows[r][1], g["trace"][1, r]) for r in range(len(rows)))
    assert worst < 1e-10
