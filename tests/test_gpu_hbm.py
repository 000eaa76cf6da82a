"""GPU parity of the HBM engine: the frontier of every chain in HBM and the
forward passes of the wide layers run as dense GEMMs (tensor cores with
three-term split BF16 operands, or the FP32 SIMT arm), against the FP64
oracle: Alg. 1 and Alg. 2 bit for bit (draws within 1e-6 of a CDF boundary
excepted), candidate pairs to 1e-5, whole-circuit amplitudes of frontiers
beyond on-chip memory (2^18 and 2^21 entries per chain) against variable
elimination. The two- and one-term BF16 arms are checked against their own
precision: 16 and 8 significant bits per operand."""
import numpy as np
import pytest

import workloads as W
from oracle import circuit as OC
from oracle import sampler as OS
from oracle import tn as TN

from tests.test_gpu_cluster import _grid_spec
from tests.test_gpu_parity import check_against_sv, pair_err, run_gpu

pytestmark = pytest.mark.gpu

SPLIT3, SPLIT2, BF16, FP32 = 0, 1, 2, 3   # PW_GEMM_* of include/pw.h
HBM = 2                                    # PW_ENGINE_HBM


@pytest.fixture(scope="module")
def pw():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_24218_gb300 as mod
    mod.load_library()
    return mod


@pytest.mark.parametrize("gemm", [SPLIT3, FP32])
@pytest.mark.parametrize("n,p,seed,with_h", [(14, 3, 6, True), (16, 2, 8, False), (13, 3, 9, False)])
def test_hbm_engine_bitwise_against_alg1(pw, gemm, n, p, seed, with_h):
    spec = W.random_qaoa(n, p, seed=seed, with_h=with_h)
    g, worst = check_against_sv(pw, spec, 48, seed=seed, engine=HBM, gemm=gemm)
    st = g["plan_stats"]
    assert st["engine"] == HBM and st["gemm"] == gemm
    if st["width_bits"] >= 12:
        assert st["dense_passes_per_sample"] > 0   # the dense path ran


@pytest.mark.parametrize("gemm", [SPLIT3, FP32])
def test_hbm_engine_noisy_against_alg2(pw, gemm):
    """A 4x4 grid at p = 3 (2^12-entry frontier at the last layer: dense
    passes) with depolarizing and damping raised to 0.2 and 0.3 (most chains
    leave the clean state): Alg. 2 bit for bit."""
    spec = _grid_spec(4, 4, 3, seed=71, depol2=0.2, ad_gamma=0.3)
    g = run_gpu(pw, spec, 40, seed=7, trace=False, engine=HBM, gemm=gemm)
    assert g["plan_stats"]["dense_passes_per_sample"] > 0
    ops = OC.qaoa_circuit(spec)
    mism, near = 0, 0
    for k in range(40):
        s, st = OS.noisy_sample(spec.n, ops, 7, k, order=g["order"])
        near += st.near_boundary
        mism += int(not np.array_equal(s, g["bits"][k]))
    assert mism <= max(near, g["stats"]["near_boundary"])


def test_hbm_grid8x8_noisy_chain_against_alg2(pw):
    """The 64-qubit noisy workload (8x8 grid, p = 2) on the HBM engine with
    tensor-core passes: a chain against Alg. 2 with elimination amplitudes,
    bit for bit and pair by pair along its trajectory."""
    spec = W.grid_8x8_p2_noisy()
    g = run_gpu(pw, spec, 4, seed=2027, engine=HBM, gemm=SPLIT3)
    assert g["plan_stats"]["dense_tile_bits"] == 6
    ops = OC.qaoa_circuit(spec)
    trace = []
    s, st = OS.noisy_sample(spec.n, ops, 2027, 3, order=g["order"], backend="tn", trace=trace)
    if st.near_boundary == 0:
        assert np.array_equal(s, g["bits"][3])
    rows = [t for t in trace if len(t[0]) == 2][spec.n:]
    assert len(rows) == g["plan_stats"]["sampled_gates"]
    worst = max(pair_err(rows[r][1], g["trace"][3, r]) for r in range(len(rows)))
    assert worst < 1e-5


def test_hbm_matches_on_chip_engine(pw):
    """The 64-qubit noisy workload, 256 chains: the HBM engine (tensor cores)
    and the on-chip engine draw the same samples, with candidate pairs equal
    to FP32 rounding."""
    spec = W.grid_8x8_p2_noisy()
    a = run_gpu(pw, spec, 256, seed=11)
    b = run_gpu(pw, spec, 256, seed=11, engine=HBM, gemm=SPLIT3)
    same = (a["bits"] == b["bits"]).all(axis=1)
    assert (~same).sum() <= max(a["stats"]["near_boundary"], b["stats"]["near_boundary"])
    rows = a["plan_stats"]["sampled_gates"]
    worst = max(pair_err(a["trace"][k, r][0::2] + 1j * a["trace"][k, r][1::2], b["trace"][k, r])
                for k in np.nonzero(same)[0][:32] for r in range(rows))
    assert worst < 1e-5


@pytest.mark.parametrize("gemm,tol", [(SPLIT2, 5e-4), (BF16, 0.15)])
def test_hbm_reduced_precision_arms(pw, gemm, tol):
    """Two BF16 terms per operand (16 bits, three products) and one (8
    bits): candidate pairs of the chains that follow Alg. 1 within the
    accuracy of their operands (about 2^-17 and 2^-9 per pass, over the
    plan's passes); the decisions they flip are counted, not failed."""
    spec = W.random_qaoa(14, 3, seed=6, with_h=True)
    g = run_gpu(pw, spec, 48, 6, engine=HBM, gemm=gemm)
    ops = OC.qaoa_circuit(spec)
    traces = [[] for _ in range(48)]
    want, _ = OS.sample_sv(spec.n, ops, 6, list(range(48)), order=g["order"], traces=traces)
    same = (want == g["bits"]).all(axis=1)
    assert same.sum() >= 24
    worst = max(pair_err(traces[k][spec.n + r][1], g["trace"][k, r])
                for k in np.nonzero(same)[0] for r in range(g["plan_stats"]["sampled_gates"]))
    assert worst < tol


def _wide_instance(pw, name):
    spec = [s for s in W.gradient_instances() if s.name == name][0]
    return spec


@pytest.mark.parametrize("name,width", [("qaoa_p3_3reg_n24_i7", 18), ("qaoa_p3_3reg_n28_i17", 21)])
def test_hbm_wide_amplitudes_against_elimination(pw, name, width):
    """Whole-circuit amplitudes <x|C|0> of p = 3 random 3-regular instances
    whose frontier (2^18, 2^21 entries per chain) exceeds the on-chip
    engine: pw_amplitudes on the HBM engine against the oracle's variable
    elimination, 1e-5 relative."""
    import torch
    spec = _wide_instance(pw, name)
    c = pw.pw_circuit_qaoa(spec.n, spec.edges, spec.weights, None, spec.p, spec.gammas, spec.betas)
    plan = pw.pw_plan_build(c)
    st = pw.pw_plan_stats(plan)
    assert st["engine"] == HBM and st["width_bits"] == width
    rng = np.random.default_rng(5)
    bits = rng.integers(0, 2, (6, spec.n)).astype(np.uint8)
    d_bits = torch.from_numpy(pw.pack_bits(bits).view(np.int64)).cuda()
    amp = torch.zeros((6, 2), dtype=torch.float64, device="cuda")
    pw.pw_amplitudes(plan, st["n_ops"], d_bits, amp)
    got = amp.cpu().numpy()
    got = got[:, 0] + 1j * got[:, 1]
    pw.pw_plan_destroy(plan)
    pw.pw_circuit_destroy(c)
    ops = OC.qaoa_circuit(spec)
    want = np.array([TN.amplitudes(spec.n, ops, b) for b in bits])
    err = np.abs(got - want) / np.abs(want)
    assert err.max() < 1e-5, err


def test_hbm_wide_chain_against_alg1(pw):
    """Sampling a p = 3 instance with a 2^18-entry frontier (beyond the
    on-chip engine): one chain against Alg. 1 with elimination amplitudes,
    bit for bit and candidate pair by pair."""
    spec = _wide_instance(pw, "qaoa_p3_3reg_n24_i7")
    g = run_gpu(pw, spec, 3, seed=99)
    assert g["plan_stats"]["engine"] == HBM
    ops = OC.qaoa_circuit(spec)
    trace = []
    s, st = OS.sample_tn(spec.n, ops, 99, 1, order=g["order"], trace=trace)
    if st.near_boundary == 0 and g["stats"]["near_boundary"] == 0:
        assert np.array_equal(s, g["bits"][1])
    rows = trace[spec.n:]
    assert len(rows) == g["plan_stats"]["sampled_gates"]
    worst = max(pair_err(rows[r][1], g["trace"][1, r]) for r in range(len(rows)))
    assert worst < 1e-5


def test_hbm_without_trace_matches_on_chip(pw):
    """Without an amplitude trace (the sampling configuration of the bench),
    512 chains of the 64-qubit noisy workload on the HBM engine and on the
    on-chip engine: the same samples, and no block of zero mass. (Chains at
    different layers run at the same time: each keeps its frontier at one
    place for all layers, so a chain's layer-1 frontier can never sit inside
    another chain's layer-2 frontier.)"""
    spec = W.grid_8x8_p2_noisy()
    a = run_gpu(pw, spec, 512, seed=7, trace=False, chains_per_launch=512)
    b = run_gpu(pw, spec, 512, seed=7, trace=False, engine=HBM, gemm=SPLIT3, chains_per_launch=512)
    assert b["stats"]["zero_mass"] == 0 and a["stats"]["zero_mass"] == 0
    differ = int((~(a["bits"] == b["bits"]).all(axis=1)).sum())
    assert differ <= max(a["stats"]["near_boundary"], b["stats"]["near_boundary"])
