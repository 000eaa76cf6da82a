"""GPU parity tests: the CUDA path through the C-ABI against the FP64 oracle.

Bitstrings must be identical to the oracle's on the same Philox streams,
except for chains in which a draw fell within 1e-6 of a CDF boundary (counted
by both sides); amplitudes are compared per candidate pair with the relative
error ||a_gpu - a_ref||_2 / ||a_ref||_2, bound 1e-5 for the FP32 contraction
and 1e-12 for the FP64 one.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import circuit as OC
from oracle import closed_form as CF
from oracle import sampler as OS
from oracle import statevector as SV
from oracle import tn as TN

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-12}


@pytest.fixture(scope="module")
def pw():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_24218_gb300 as mod
    mod.load_library()
    return mod


def _circ(pw, spec):
    return pw.pw_circuit_qaoa(spec.n, spec.edges, spec.weights, spec.h, spec.p, spec.gammas, spec.betas,
                              spec.depol2, spec.ad_gamma)


def run_gpu(pw, spec, N, seed, precision=0, trace=True, first=0, **opts):
    import torch
    circ = _circ(pw, spec)
    plan = pw.pw_plan_build(circ, precision=precision, **opts)
    st = pw.pw_plan_stats(plan)
    words = (spec.n + 63) // 64
    bits = torch.zeros((N, words), dtype=torch.int64, device="cuda")
    tr = torch.zeros((N, st["sampled_gates"], 4), dtype=torch.float64, device="cuda") if trace else None
    stats = pw.pw_sample(plan, seed, first, N, bits, tr)
    torch.cuda.synchronize()
    order = pw.pw_plan_exec_order(plan)
    out = dict(bits=pw.unpack_bits(bits.cpu().numpy(), spec.n), trace=tr.cpu().numpy() if trace else None,
               stats=stats, order=order, plan_stats=st)
    pw.pw_plan_destroy(plan)
    pw.pw_circuit_destroy(circ)
    return out


def pair_err(o_amps, g_row):
    a = np.array(o_amps)
    b = g_row[0::2] + 1j * g_row[1::2]
    return float(np.linalg.norm(a - b) / np.linalg.norm(a))


def check_against_sv(pw, spec, N, seed, precision=0, trace_chains=64, **opts):
    g = run_gpu(pw, spec, N, seed, precision=precision, **opts)
    ops = OC.qaoa_circuit(spec)
    traces = [[] for _ in range(min(N, trace_chains))]
    ids = list(range(N))
    want, ost = OS.sample_sv(spec.n, ops, seed, ids[:len(traces)], order=g["order"], traces=traces)
    if N > len(traces):
        rest, ost2 = OS.sample_sv(spec.n, ops, seed, ids[len(traces):], order=g["order"])
        want = np.concatenate([want, rest])
        ost.near_boundary += ost2.near_boundary
    mism = int((~(want == g["bits"]).all(axis=1)).sum())
    allowed = max(g["stats"]["near_boundary"], ost.near_boundary)
    assert mism <= allowed, f"{mism} chains differ, {allowed} near-boundary draws"
    worst = 0.0
    for k in range(len(traces)):
        if not (want[k] == g["bits"][k]).all():
            continue
        o = traces[k][spec.n:]
        assert len(o) == g["plan_stats"]["sampled_gates"]
        for r in range(len(o)):
            worst = max(worst, pair_err(o[r][1], g["trace"][k, r]))
    assert worst < TOL[precision], worst
    return g, worst


# ---------------------------------------------------------------- config 1

@pytest.mark.parametrize("precision", [1, 0])
def test_config1_bitwise_against_oracle(pw, precision):
    """n=12 3-regular p=1 (gamma=0.4, beta=0.3), 10^4 samples, identical bits."""
    spec = W.maxcut_3reg_n12()
    g, worst = check_against_sv(pw, spec, 10000, seed=20251, precision=precision, trace_chains=256,
                                chains_per_launch=256)
    # TVD against the exact distribution within the multinomial 99th percentile
    p = np.abs(SV.run(spec.n, OC.qaoa_circuit(spec))) ** 2
    idx = (g["bits"].astype(np.int64) << np.arange(spec.n)).sum(axis=1)
    emp = np.bincount(idx, minlength=1 << spec.n) / len(idx)
    rng = np.random.default_rng(0)
    thr = np.quantile([0.5 * np.abs(rng.multinomial(len(idx), p) / len(idx) - p).sum() for _ in range(200)], 0.99)
    assert 0.5 * np.abs(emp - p).sum() < thr


@pytest.mark.parametrize("seed,n,p,with_h,tpc", [(31, 8, 1, False, 32), (32, 10, 2, True, 64), (33, 9, 3, False, 128),
                                                 (34, 12, 2, True, 256), (35, 6, 2, False, 32)])
def test_random_circuits_bitwise(pw, seed, n, p, with_h, tpc):
    spec = W.random_qaoa(n, p, seed=seed, with_h=with_h)
    check_against_sv(pw, spec, 97, seed=seed, threads_per_chain=tpc)


def test_natural_order_and_small_blocks(pw):
    spec = W.random_qaoa(10, 2, seed=41, with_h=True)
    check_against_sv(pw, spec, 50, seed=4, order=pw.PW_ORDER_NATURAL, max_block=2)
    check_against_sv(pw, spec, 50, seed=4, order=pw.PW_ORDER_AUTO, max_block=1)


def test_first_sample_offset_and_launch_split(pw):
    """Sample k depends only on (seed, k): any split of the range gives the same bits."""
    spec = W.random_qaoa(10, 2, seed=42)
    full = run_gpu(pw, spec, 300, seed=9, trace=False)["bits"]
    part = run_gpu(pw, spec, 120, seed=9, trace=False, first=150)["bits"]
    assert np.array_equal(full[150:270], part)
    split = run_gpu(pw, spec, 300, seed=9, trace=False, chains_per_launch=37)["bits"]
    assert np.array_equal(full, split)


def test_zero_samples_and_host_variant(pw):
    import torch
    spec = W.random_qaoa(8, 2, seed=43)
    circ = _circ(pw, spec)
    plan = pw.pw_plan_build(circ)
    bits = torch.zeros((1, 1), dtype=torch.int64, device="cuda")
    assert pw.pw_sample(plan, 1, 0, 0, bits)["launches"] == 0
    host = np.zeros((77, 1), dtype=np.uint64)
    pw.pw_sample_host(plan, 5, 3, 77, host)
    dev = torch.zeros((77, 1), dtype=torch.int64, device="cuda")
    pw.pw_sample(plan, 5, 3, 77, dev)
    assert np.array_equal(host.view(np.int64), dev.cpu().numpy())
    pw.pw_plan_destroy(plan)
    pw.pw_circuit_destroy(circ)


# ---------------------------------------------------------------- config 2

def test_grid6x6_chains_against_elimination_oracle(pw):
    """6x6 grid p=2 in the benchmark's launch shape: chains spread over the
    batch checked one by one against the variable-elimination oracle."""
    spec = W.grid_6x6_p2()
    N = 4096
    g = run_gpu(pw, spec, N, seed=777, chains_per_launch=4096)
    ops = OC.qaoa_circuit(spec)
    for k in (0, 1777, 4095):
        trace = []
        s, ost = OS.sample_tn(spec.n, ops, 777, k, order=g["order"], trace=trace)
        if ost.near_boundary == 0:
            assert np.array_equal(s, g["bits"][k])
        o = trace[spec.n:]
        worst = max(pair_err(o[r][1], g["trace"][k, r]) for r in range(len(o)))
        assert worst < 1e-5, (k, worst)


def test_grid6x6_symmetry_at_scale(pw):
    """MaxCut with h = 0: p(x) = p(not x), every bit has mean 1/2 (10^5 samples)."""
    spec = W.grid_6x6_p2()
    g = run_gpu(pw, spec, 100000, seed=99, trace=False)
    m = g["bits"].mean(axis=0)
    assert np.all(np.abs(m - 0.5) < 5 * 0.5 / math.sqrt(100000))


# ------------------------------------------------------------------- noise

@pytest.mark.parametrize("spec", [W.random_qaoa(6, 2, seed=51, depol2=0.3, ad_gamma=0.4),
                                  W.random_qaoa(8, 2, seed=52, depol2=0.1, ad_gamma=0.6, with_h=True),
                                  W.random_qaoa(10, 1, seed=53, depol2=0.5, ad_gamma=0.2)])
def test_noisy_bitwise_against_alg2(pw, spec):
    g = run_gpu(pw, spec, 120, seed=61, trace=False)
    ops = OC.qaoa_circuit(spec)
    mism = 0
    near = 0
    for k in range(120):
        s, st = OS.noisy_sample(spec.n, ops, 61, k, order=g["order"])
        near += st.near_boundary
        mism += int(not np.array_equal(s, g["bits"][k]))
    assert mism <= max(near, g["stats"]["near_boundary"])


@pytest.mark.parametrize("spec", [W.random_qaoa(10, 2, seed=55, depol2=0.01, ad_gamma=0.03),
                                  W.random_qaoa(8, 3, seed=56, depol2=0.02, ad_gamma=0.05)])
def test_noisy_clean_and_dirty_chains_against_alg2(pw, spec):
    """Low noise rates: most chains draw only Kraus operator 0 (clean: the
    kernel uses host-evaluated tables and one parallel draw per layer), the
    others leave that state midway (tables built per chain, draws in dependency
    waves). Both kinds must give Alg. 2's bits and amplitudes."""
    N = 64
    g = run_gpu(pw, spec, N, seed=63, trace=True)
    ops = OC.qaoa_circuit(spec)
    clean = dirty = mism = near = 0
    worst = 0.0
    for k in range(N):
        trace, events = [], []
        s, st = OS.noisy_sample(spec.n, ops, 63, k, order=g["order"], trace=trace, events=events)
        near += st.near_boundary
        mism += int(not np.array_equal(s, g["bits"][k]))
        if all(i == 0 for _, i in events):
            clean += 1
        else:
            dirty += 1
        rows = [t for t in trace if len(t[0]) == 2][spec.n:]
        if np.array_equal(s, g["bits"][k]):
            worst = max(worst, max(pair_err(rows[r][1], g["trace"][k, r]) for r in range(len(rows))))
    assert clean >= 8 and dirty >= 8
    assert mism <= max(near, g["stats"]["near_boundary"])
    assert worst < 1e-5


def test_noisy_distribution_against_density_matrix(pw):
    spec = W.random_qaoa(4, 2, seed=54, depol2=0.2, ad_gamma=0.5)
    N = 40000
    g = run_gpu(pw, spec, N, seed=62, trace=False)
    p = np.real(np.diag(SV.density_run(spec.n, OC.qaoa_circuit(spec))))
    idx = (g["bits"].astype(np.int64) << np.arange(spec.n)).sum(axis=1)
    emp = np.bincount(idx, minlength=1 << spec.n) / N
    rng = np.random.default_rng(1)
    thr = np.quantile([0.5 * np.abs(rng.multinomial(N, p) / N - p).sum() for _ in range(200)], 0.99)
    assert 0.5 * np.abs(emp - p).sum() < thr


def test_first_upload_then_non_blocking_stream(pw):
    """A fresh plan's first call on a non-blocking stream reads complete
    tables: the samples equal those of the same plan drawn on the default
    stream afterwards."""
    import torch
    spec = W.grid_6x6_p2()
    circ = _circ(pw, spec)
    words = 1
    for rep in range(3):
        plan = pw.pw_plan_build(circ, chains_per_launch=4096)
        side = torch.cuda.Stream()   # torch creates its streams non-blocking
        a = torch.empty((4096, words), dtype=torch.int64, device="cuda")
        b = torch.empty((4096, words), dtype=torch.int64, device="cuda")
        pw.pw_sample(plan, 5 + rep, 0, 4096, a, None, side, want_stats=False)
        side.synchronize()
        pw.pw_sample(plan, 5 + rep, 0, 4096, b, None, None, want_stats=False)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
        pw.pw_plan_destroy(plan)
    pw.pw_circuit_destroy(circ)


def test_noisy_distribution_against_trajectories(pw):
    """The same check against the second, differently derived noisy oracle:
    the branch-weighted average of standard quantum trajectories."""
    from oracle import trajectory as TR
    spec = W.random_qaoa(3, 2, seed=55, with_h=True, depol2=0.3, ad_gamma=0.4)
    spec.edges = spec.edges[:1]
    spec.weights = spec.weights[:1]
    N = 40000
    g = run_gpu(pw, spec, N, seed=63, trace=False)
    p = TR.exact_distribution(spec.n, OC.qaoa_circuit(spec))
    idx = (g["bits"].astype(np.int64) << np.arange(spec.n)).sum(axis=1)
    emp = np.bincount(idx, minlength=1 << spec.n) / N
    rng = np.random.default_rng(2)
    thr = np.quantile([0.5 * np.abs(rng.multinomial(N, p) / N - p).sum() for _ in range(200)], 0.99)
    assert 0.5 * np.abs(emp - p).sum() < thr


# -------------------------------------------------------------- amplitudes

def test_amplitudes_api_against_state_vector(pw):
    import torch
    spec = W.random_qaoa(10, 2, seed=71, with_h=True)
    circ = _circ(pw, spec)
    plan = pw.pw_plan_build(circ)
    order = pw.pw_plan_exec_order(plan)
    ops = OC.qaoa_circuit(spec)
    xs = W.random_bitstrings(32, spec.n, seed=72)
    d_bits = torch.from_numpy(pw.pack_bits(xs).view(np.int64)).cuda()
    amp = torch.zeros((32, 2), dtype=torch.float64, device="cuda")
    psi = SV.zero_state(spec.n)
    checked = 0
    for t, oi in enumerate(order, start=1):
        op = ops[oi]
        psi = SV.apply(psi, spec.n, op.qubits, op.mat) if op.kind == "gate" else psi
        if op.kind != "gate" or len(op.qubits) != 1 or OC.is_diagonal(op.mat) or t <= spec.n:
            continue
        pw.pw_amplitudes(plan, t, d_bits, amp)
        got = amp.cpu().numpy()
        for k in range(32):
            a = psi[sum(int(b) << q for q, b in enumerate(xs[k]))]
            assert abs(got[k, 0] + 1j * got[k, 1] - a) <= 1e-5 * max(abs(a), 1e-3 * np.abs(psi).max())
        checked += 1
    assert checked == spec.n * spec.p
    with pytest.raises(pw.PwError):
        pw.pw_amplitudes(plan, spec.n + 1, d_bits, amp)    # ends on a diagonal gate
    pw.pw_plan_destroy(plan)
    pw.pw_circuit_destroy(circ)


# ---------------------------------------------------------------- config 5

def test_heavy_hex_400_zz_closed_form(pw):
    """400 qubits, p=1: sample means of z_u z_v against the closed form."""
    spec = W.heavy_hex_400_p1()
    N = 20000
    g = run_gpu(pw, spec, N, seed=5, trace=False)
    z = 1 - 2 * g["bits"].astype(np.int64)
    cf = CF.zz_p1(spec.n, spec.edges, spec.weights, spec.gammas[0], spec.betas[0])
    zs = []
    for (u, v), want in zip(spec.edges, cf):
        zz = z[:, u] * z[:, v]
        se = math.sqrt(max(1e-12, (1 - want ** 2) / N))
        zs.append((zz.mean() - want) / se)
    assert np.max(np.abs(zs)) < 5.0, np.max(np.abs(zs))


def test_max_qubits_4096_path_zz_closed_form(pw):
    """The largest circuit a plan takes: 4096 qubits (64 words per sample), a
    weighted path at p = 1. Each of the 4095 edge means of z_u z_v is within
    five standard errors of the closed form, and their squared z-scores
    average about one (no systematic bias)."""
    n = 4096
    rng = np.random.default_rng(91)
    e = np.array([(i, i + 1) for i in range(n - 1)], dtype=np.int64)
    spec = W.QaoaSpec(n=n, edges=e, weights=rng.normal(size=n - 1), gammas=np.array([0.45]),
                      betas=np.array([0.35]), h=None, depol2=0.0, ad_gamma=0.0, name="path4096", extra={})
    N = 8192
    g = run_gpu(pw, spec, N, seed=92, trace=False)
    assert g["bits"].shape == (N, n)
    z = 1 - 2 * g["bits"].astype(np.int64)
    cf = CF.zz_p1(spec.n, spec.edges, spec.weights, spec.gammas[0], spec.betas[0])
    zz = (z[:, e[:, 0]] * z[:, e[:, 1]]).mean(axis=0)
    zs = (zz - cf) / np.sqrt(np.maximum(1e-12, (1 - cf ** 2) / N))
    assert np.max(np.abs(zs)) < 5.0, np.max(np.abs(zs))
    assert np.mean(zs ** 2) < 1.2, np.mean(zs ** 2)


def test_heavy_hex_400_amplitudes_against_elimination(pw):
    """400 qubits: FP64 amplitudes of random strings (full circuit) against the
    elimination oracle, and the FP64 sampler's candidate pairs along one
    sampled chain (rows spread over the sweep)."""
    import torch
    from oracle.philox import draw
    spec = W.heavy_hex_400_p1()
    circ = _circ(pw, spec)
    plan = pw.pw_plan_build(circ, precision=pw.PW_PREC_FP64)
    order = pw.pw_plan_exec_order(plan)
    ops = OC.qaoa_circuit(spec)
    xs = W.random_bitstrings(3, spec.n, seed=73)
    d_bits = torch.from_numpy(pw.pack_bits(xs).view(np.int64)).cuda()
    amp = torch.zeros((3, 2), dtype=torch.float64, device="cuda")
    pw.pw_amplitudes(plan, len(order), d_bits, amp)
    got = amp.cpu().numpy()
    pre = [ops[i] for i in order]
    for k in range(3):
        a = TN.amplitudes(spec.n, pre, xs[k])
        assert abs(got[k, 0] + 1j * got[k, 1] - a) <= 1e-10 * abs(a)
    pw.pw_plan_destroy(plan)
    pw.pw_circuit_destroy(circ)
    # FP32 trace of one chain: the state before the r-th mixer gate is the
    # final bit for qubits already resampled and the H-layer bit for the rest
    g = run_gpu(pw, spec, 1, seed=8, precision=pw.PW_PREC_FP64)
    final = g["bits"][0]
    h_bits = np.array([0 if draw(8, 0, q, 0) < 0.5 else 1 for q in range(spec.n)], dtype=np.uint8)
    mix_pos = [t for t, oi in enumerate(order) if t >= spec.n and ops[oi].kind == "gate" and len(ops[oi].qubits) == 1]
    for r in (0, 133, 266, 399):
        t = mix_pos[r]
        q = ops[order[t]].qubits[0]
        done = {ops[order[u]].qubits[0] for u in mix_pos[:r]}
        state = np.array([final[j] if j in done else h_bits[j] for j in range(spec.n)], dtype=np.uint8)
        tab = TN.amplitudes(spec.n, [ops[i] for i in order[:t + 1]], state, open_qubits=(q,))
        assert pair_err([tab[0], tab[1]], g["trace"][0, r]) < TOL[1], r


def test_heavy_hex_400_fp32_amplitudes_within_1e5(pw):
    """400 qubits on the FP32 path: full-string amplitudes and the candidate
    pairs of one sampled chain, spread over the sweep, against the elimination
    oracle within 1e-5. The FP32 error there is almost entirely a common
    magnitude drift (the same rounded constants act at every site); it grows
    with the number of sites and is the reason the FP64 path exists."""
    import torch
    from oracle.philox import draw
    spec = W.heavy_hex_400_p1()
    circ = _circ(pw, spec)
    plan = pw.pw_plan_build(circ, precision=pw.PW_PREC_FP32)
    order = pw.pw_plan_exec_order(plan)
    ops = OC.qaoa_circuit(spec)
    pre = [ops[i] for i in order]
    xs = W.random_bitstrings(2, spec.n, seed=74)
    d_bits = torch.from_numpy(pw.pack_bits(xs).view(np.int64)).cuda()
    amp = torch.zeros((2, 2), dtype=torch.float64, device="cuda")
    pw.pw_amplitudes(plan, len(order), d_bits, amp)
    got = amp.cpu().numpy()
    for k in range(2):
        a = TN.amplitudes(spec.n, pre, xs[k])
        assert abs(got[k, 0] + 1j * got[k, 1] - a) <= 1e-5 * abs(a)
    pw.pw_plan_destroy(plan)
    pw.pw_circuit_destroy(circ)
    g = run_gpu(pw, spec, 1, seed=8)
    final = g["bits"][0]
    h_bits = np.array([0 if draw(8, 0, q, 0) < 0.5 else 1 for q in range(spec.n)], dtype=np.uint8)
    mix_pos = [t for t, oi in enumerate(order) if t >= spec.n and ops[oi].kind == "gate" and len(ops[oi].qubits) == 1]
    for r in (0, 114, 285, 399):
        t = mix_pos[r]
        q = ops[order[t]].qubits[0]
        done = {ops[order[u]].qubits[0] for u in mix_pos[:r]}
        state = np.array([final[j] if j in done else h_bits[j] for j in range(spec.n)], dtype=np.uint8)
        tab = TN.amplitudes(spec.n, [ops[i] for i in order[:t + 1]], state, open_qubits=(q,))
        assert pair_err([tab[0], tab[1]], g["trace"][0, r]) < 1e-5, r


def _degenerate():
    from tests import test_native_host as H
    return H._degenerate_specs()


@pytest.mark.parametrize("spec", _degenerate(), ids=lambda s: s.name)
def test_degenerate_circuits_against_alg1(pw, spec):
    """No edges, isolated qubits (qubit 0 among them), gamma = 0, beta = 0 and a
    monomial mixer (a deterministic move, Sec. 2): bits equal to Alg. 1 on
    the same draws; candidate pairs too where every mixer is sampled."""
    if spec.name == "monomial_mixer":
        g = run_gpu(pw, spec, 64, seed=12, trace=False)
        want, ost = OS.sample_sv(spec.n, OC.qaoa_circuit(spec), 12, list(range(64)), order=g["order"])
        mism = int((~(want == g["bits"]).all(axis=1)).sum())
        assert mism <= max(g["stats"]["near_boundary"], ost.near_boundary)
    else:
        check_against_sv(pw, spec, 64, seed=12)


def _general_circuit(n, edges, p, seed, monomial_at=None):
    """Layers of random one-qubit unitaries separated by random diagonal
    two-qubit gates on the edges and random one-qubit diagonal gates; the
    first layer acts on |0^n>. monomial_at = (layer, qubit) puts a Pauli X
    there (a deterministic move)."""
    rng = np.random.default_rng(seed)

    def su2():
        z = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
        q, r = np.linalg.qr(z)
        return q * (np.diag(r) / np.abs(np.diag(r)))

    ops = []
    for m in range(p + 1):
        if m > 0:
            for (a, b) in edges:
                ops.append(OC.gate((a, b), np.diag(np.exp(1j * rng.uniform(0, 2 * np.pi, 4)))))
            for q in range(0, n, 3):
                ops.append(OC.gate((q,), np.diag(np.exp(1j * rng.uniform(0, 2 * np.pi, 2)))))
        for q in range(n):
            A = np.array([[0, 1], [1, 0]], dtype=complex) if monomial_at == (m, q) else su2()
            ops.append(OC.gate((q,), A))
    return ops


@pytest.mark.parametrize("n,rows,p,seed,mono", [(8, 2, 2, 5, None), (9, 3, 2, 6, (1, 4)), (6, 2, 3, 7, None)])
def test_general_circuits_through_the_c_abi(pw, n, rows, p, seed, mono):
    """Circuits built gate by gate (pw_circuit_add_gate), not QAOA: random
    one-qubit unitaries between random diagonal gates, on a grid. Bits equal
    to Alg. 1 on the same draws; candidate pairs within 1e-5 (FP32)."""
    import torch
    edges = [(a, b) for a, b in W.grid_edges(rows, n // rows)]
    ops = _general_circuit(n, edges, p, seed, monomial_at=mono)
    circ = pw.pw_circuit_create(n)
    for o in ops:
        pw.pw_circuit_add_gate(circ, list(o.qubits), o.mat)
    plan = pw.pw_plan_build(circ)
    st = pw.pw_plan_stats(plan)
    N = 64
    bits = torch.zeros((N, 1), dtype=torch.int64, device="cuda")
    tr = torch.zeros((N, st["sampled_gates"], 4), dtype=torch.float64, device="cuda")
    stats = pw.pw_sample(plan, 21, 0, N, bits, tr)
    torch.cuda.synchronize()
    order = pw.pw_plan_exec_order(plan)
    got = pw.unpack_bits(bits.cpu().numpy(), n)
    trace = tr.cpu().numpy()
    traces = [[] for _ in range(N)]
    want, ost = OS.sample_sv(n, ops, 21, list(range(N)), order=order, traces=traces)
    mism = int((~(want == got).all(axis=1)).sum())
    assert mism <= max(stats["near_boundary"], ost.near_boundary)
    if mono is None:
        worst = max(pair_err(traces[k][n + r][1], trace[k, r])
                    for k in range(N) if (want[k] == got[k]).all() for r in range(st["sampled_gates"]))
        assert worst < 1e-5
    pw.pw_plan_destroy(plan)
    pw.pw_circuit_destroy(circ)


def _general_noisy(n, edges, p, seed):
    """A general circuit with channels: a bit flip listed with its X operator
    first (so no chain state has fixed tables: every chain builds its tables)
    after every two-qubit diagonal gate's first qubit, phase damping on every
    qubit after each one-qubit layer."""
    ops = _general_circuit(n, edges, p, seed)
    out = []
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    for o in ops:
        out.append(o)
        if o.kind == "gate" and len(o.qubits) == 2:
            out.append(OC.kraus((o.qubits[0],), [np.sqrt(0.15) * X, np.sqrt(0.85) * np.eye(2)]))
    res = []
    layer_end = {i for i, o in enumerate(out) if o.kind == "gate" and len(o.qubits) == 1
                 and not OC.is_diagonal(o.mat) and o.qubits[0] == n - 1}
    for i, o in enumerate(out):
        res.append(o)
        if i in layer_end:
            for q in range(n):
                res.append(OC.kraus((q,), OC.phase_damping_kraus(0.3)))
    return res


def test_general_noisy_circuit_without_fixed_tables(pw):
    """Channels whose operator 0 flips the frame, and phase damping: bits
    equal to Alg. 2 on the same draws, and the distribution of 30000 samples
    against the density-matrix diagonal (TVD within the 99th percentile of
    multinomial noise)."""
    import torch
    n = 4
    ops = _general_noisy(n, [(0, 1), (1, 2), (2, 3)], 2, seed=9)
    circ = pw.pw_circuit_create(n)
    for o in ops:
        if o.kind == "gate":
            pw.pw_circuit_add_gate(circ, list(o.qubits), o.mat)
        else:
            pw.pw_circuit_add_kraus(circ, list(o.qubits), o.mats)
    plan = pw.pw_plan_build(circ)
    order = pw.pw_plan_exec_order(plan)
    N = 30000
    bits = torch.zeros((N, 1), dtype=torch.int64, device="cuda")
    stats = pw.pw_sample(plan, 31, 0, N, bits)
    torch.cuda.synchronize()
    got = pw.unpack_bits(bits.cpu().numpy(), n)
    mism = near = 0
    for k in range(60):
        s, st = OS.noisy_sample(n, ops, 31, k, order=order)
        near += st.near_boundary
        mism += int(not np.array_equal(s, got[k]))
    assert mism <= max(near, stats["near_boundary"])
    pdm = np.real(np.diag(SV.density_run(n, ops)))
    idx = (got.astype(np.int64) << np.arange(n)).sum(axis=1)
    emp = np.bincount(idx, minlength=1 << n) / N
    rng = np.random.default_rng(2)
    thr = np.quantile([0.5 * np.abs(rng.multinomial(N, pdm) / N - pdm).sum() for _ in range(200)], 0.99)
    assert 0.5 * np.abs(emp - pdm).sum() < thr
    pw.pw_plan_destroy(plan)
    pw.pw_circuit_destroy(circ)


def _chip_noise_qaoa(spec, rates):
    """A QAOA circuit under a device noise model built from LSM channels only:
    a two-qubit Pauli channel with unequal rates after every RZZ, a one-qubit
    Pauli channel with unequal X/Y/Z rates after every RX, amplitude plus phase
    damping (T1/T2) on every qubit after each mixer layer, and a readout flip
    (bit-flip channel) on every qubit at the end."""
    from oracle.circuit import PAULI
    p2, (px, py, pz), g1, lam, ro = rates
    w2 = [1.0 - p2] + [p2 * (1 + (k % 3)) / 30.0 for k in range(1, 16)]   # unequal, sum p2
    w2 = np.array(w2) / sum(w2) * 1.0
    k2 = [np.sqrt(w2[k]) * np.kron(PAULI[k // 4], PAULI[k % 4]) for k in range(16)]
    k1 = [np.sqrt(1 - px - py - pz) * PAULI[0], np.sqrt(px) * PAULI[1], np.sqrt(py) * PAULI[2], np.sqrt(pz) * PAULI[3]]
    out = []
    base = OC.qaoa_circuit(spec)
    n = spec.n
    for i, o in enumerate(base):
        out.append(o)
        if i < n:
            continue   # the first (Hadamard) layer
        if o.kind == "gate" and len(o.qubits) == 2:
            out.append(OC.kraus(o.qubits, k2))
        elif o.kind == "gate" and len(o.qubits) == 1 and not OC.is_diagonal(o.mat):
            out.append(OC.kraus(o.qubits, k1))
            if o.qubits[0] == n - 1:
                for q in range(n):
                    out.append(OC.kraus((q,), OC.amplitude_damping_kraus(g1)))
                    out.append(OC.kraus((q,), OC.phase_damping_kraus(lam)))
    for q in range(n):
        out.append(OC.kraus((q,), [np.sqrt(1 - ro) * PAULI[0], np.sqrt(ro) * PAULI[1]]))
    return out


def test_chip_noise_model_qaoa(pw):
    """The device noise model of the paper's hardware discussion, as channels
    through pw_circuit_add_kraus (rates raised to make every event common):
    bits equal to Alg. 2 on the same draws, and 30000 samples against the
    density-matrix diagonal."""
    import torch
    spec = W.random_qaoa(4, 2, seed=57)
    ops = _chip_noise_qaoa(spec, (0.06, (0.02, 0.03, 0.05), 0.1, 0.2, 0.04))
    n = spec.n
    circ = pw.pw_circuit_create(n)
    for o in ops:
        if o.kind == "gate":
            pw.pw_circuit_add_gate(circ, list(o.qubits), o.mat)
        else:
            pw.pw_circuit_add_kraus(circ, list(o.qubits), o.mats)
    plan = pw.pw_plan_build(circ)
    order = pw.pw_plan_exec_order(plan)
    N = 30000
    bits = torch.zeros((N, 1), dtype=torch.int64, device="cuda")
    stats = pw.pw_sample(plan, 41, 0, N, bits)
    torch.cuda.synchronize()
    got = pw.unpack_bits(bits.cpu().numpy(), n)
    mism = near = 0
    for k in range(60):
        s, st = OS.noisy_sample(n, ops, 41, k, order=order)
        near += st.near_boundary
        mism += int(not np.array_equal(s, got[k]))
    assert mism <= max(near, stats["near_boundary"])
    pdm = np.real(np.diag(SV.density_run(n, ops)))
    idx = (got.astype(np.int64) << np.arange(n)).sum(axis=1)
    emp = np.bincount(idx, minlength=1 << n) / N
    rng = np.random.default_rng(3)
    thr = np.quantile([0.5 * np.abs(rng.multinomial(N, pdm) / N - pdm).sum() for _ in range(200)], 0.99)
    assert 0.5 * np.abs(emp - pdm).sum() < thr
    pw.pw_plan_destroy(plan)
    pw.pw_circuit_destroy(circ)


def test_autotune_keeps_the_samples(pw):
    """pw_plan_autotune picks a threads-per-chain value in 32..256 and stores it
    in the plan; sampling afterwards still follows Alg. 1 on the same draws."""
    import torch
    spec = W.random_qaoa(12, 2, seed=77, with_h=True)
    circ = _circ(pw, spec)
    plan = pw.pw_plan_build(circ, chains_per_launch=1024)
    chosen = pw.pw_plan_autotune(plan, 2048)
    st = pw.pw_plan_stats(plan)
    assert chosen in (32, 64, 128, 256) and st["threads_per_chain"] == chosen
    N = 128
    bits = torch.zeros((N, 1), dtype=torch.int64, device="cuda")
    tr = torch.zeros((N, st["sampled_gates"], 4), dtype=torch.float64, device="cuda")
    stats = pw.pw_sample(plan, 5, 0, N, bits, tr)
    torch.cuda.synchronize()
    got = pw.unpack_bits(bits.cpu().numpy(), spec.n)
    ops = OC.qaoa_circuit(spec)
    traces = [[] for _ in range(N)]
    want, ost = OS.sample_sv(spec.n, ops, 5, list(range(N)), order=pw.pw_plan_exec_order(plan), traces=traces)
    mism = int((~(want == got).all(axis=1)).sum())
    assert mism <= max(stats["near_boundary"], ost.near_boundary)
    trace = tr.cpu().numpy()
    worst = max(pair_err(traces[k][spec.n + r][1], trace[k, r])
                for k in range(N) if (want[k] == got[k]).all() for r in range(st["sampled_gates"]))
    assert worst < 1e-5
    pw.pw_plan_destroy(plan)
    pw.pw_circuit_destroy(circ)


def _swap_class(rng):
    """SWAP times a random diagonal of phases (SWAP, iSWAP and fSim(pi/2, phi)
    are of this form)."""
    S = np.eye(4)[[0, 2, 1, 3]].astype(complex)
    return S @ np.diag(np.exp(1j * rng.uniform(0, 2 * np.pi, 4)))


@pytest.mark.parametrize("n,rows,p,seed", [(8, 2, 2, 15), (9, 3, 2, 16)])
def test_swap_class_gates_against_alg1(pw, n, rows, p, seed):
    """Two-qubit SWAP-class gates (a swap of two qubits' contents times
    phases) between the sections, planned as relabellings of the wires: bits
    equal to Alg. 1 on the original gate list (the swaps as deterministic
    moves) and candidate pairs within 1e-5."""
    import torch
    rng = np.random.default_rng(seed + 100)
    edges = [(a, b) for a, b in W.grid_edges(rows, n // rows)]
    ops = _general_circuit(n, edges, p, seed)
    sec = len(edges) + len(range(0, n, 3))
    pos1 = n + sec                      # end of layer 1's diagonal section
    pos2 = n + (sec + n) + sec          # end of layer 2's diagonal section
    ops = (ops[:n] + [OC.gate((0, n - 1), _swap_class(rng))] + ops[n:pos1] +
           [OC.gate((1, 2), OC.iswap_mat()), OC.gate((5, 3), _swap_class(rng))] + ops[pos1:pos2] +
           [OC.gate((2, n - 2), _swap_class(rng))] + ops[pos2:])
    circ = pw.pw_circuit_create(n)
    for o in ops:
        pw.pw_circuit_add_gate(circ, list(o.qubits), o.mat)
    plan = pw.pw_plan_build(circ)
    st = pw.pw_plan_stats(plan)
    N = 64
    bits = torch.zeros((N, 1), dtype=torch.int64, device="cuda")
    tr = torch.zeros((N, st["sampled_gates"], 4), dtype=torch.float64, device="cuda")
    stats = pw.pw_sample(plan, 23, 0, N, bits, tr)
    torch.cuda.synchronize()
    order = pw.pw_plan_exec_order(plan)
    assert sorted(order) == list(range(len(ops)))
    # whole-circuit amplitudes of random strings (FP32 plan) against the state
    # vector; a shorter prefix is refused
    xs = W.random_bitstrings(32, n, seed=seed + 200)
    d_x = torch.from_numpy(pw.pack_bits(xs).view(np.int64)).cuda()
    amp = torch.zeros((32, 2), dtype=torch.float64, device="cuda")
    pw.pw_amplitudes(plan, len(ops), d_x, amp)
    psi = SV.run(n, ops)
    want_a = psi[[int(sum(int(b) << q for q, b in enumerate(x))) for x in xs]]
    got_a = amp.cpu().numpy()
    assert np.abs(got_a[:, 0] + 1j * got_a[:, 1] - want_a).max() <= 1e-5 * np.abs(psi).max()
    with pytest.raises(pw.PwError):
        pw.pw_amplitudes(plan, len(ops) - n, d_x, amp)
    pw.pw_plan_destroy(plan)
    pw.pw_circuit_destroy(circ)
    got = pw.unpack_bits(bits.cpu().numpy(), n)
    trace = tr.cpu().numpy()
    traces = [[] for _ in range(N)]
    want, ost = OS.sample_sv(n, ops, 23, list(range(N)), order=order, traces=traces)
    mism = int((~(want == got).all(axis=1)).sum())
    assert mism <= max(stats["near_boundary"], ost.near_boundary)
    worst = max(pair_err(traces[k][n + r][1], trace[k, r])
                for k in range(N) if (want[k] == got[k]).all() for r in range(st["sampled_gates"]))
    assert worst < 1e-5


def test_sampling_step_replays_as_a_cuda_graph(pw):
    """A step of pw_sample (several launches of a 4096-chain plan and the
    counter reset) captured once into a CUDA graph and replayed gives the
    samples of a direct call (after the plan's first, uploading call)."""
    import torch
    spec = W.grid_6x6_p2()
    circ = _circ(pw, spec)
    plan = pw.pw_plan_build(circ, chains_per_launch=4096)
    N = 10000
    s = torch.cuda.Stream()
    direct = torch.empty((N, 1), dtype=torch.int64, device="cuda")
    replay = torch.zeros((N, 1), dtype=torch.int64, device="cuda")
    with torch.cuda.stream(s):
        pw.pw_sample(plan, 31, 0, N, direct, None, s, want_stats=False)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        pw.pw_sample(plan, 31, 0, N, replay, None, s, want_stats=False)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(direct, replay)
    pw.pw_plan_destroy(plan)
    pw.pw_circuit_destroy(circ)
