"""CPU-only checks of the C-ABI library: symbols, circuit validation, planner.

No compute call is made here (there is no GPU on this host); plan building is
pure host code.
"""
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pw():
    import paper_2510_24218_gb300 as mod
    from paper_2510_24218_gb300 import build as B
    if not os.path.exists(mod.library_path()):
        B.build()
    mod.load_library()
    return mod


def _declared_functions():
    txt = open(os.path.join(ROOT, "include", "pw.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(pw_\w+)\s*\(", txt, flags=re.M)))


def test_library_exports_every_declared_symbol(pw):
    import ctypes
    lib = ctypes.CDLL(pw.library_path())
    names = _declared_functions()
    assert len(names) >= 13
    for name in names:
        assert hasattr(lib, name), name


def _circ(pw, spec):
    return pw.pw_circuit_qaoa(spec.n, spec.edges, spec.weights, spec.h, spec.p, spec.gammas, spec.betas,
                              spec.depol2, spec.ad_gamma)


def test_circuit_validation_errors(pw):
    c = pw.pw_circuit_create(3)
    with pytest.raises(pw.PwError) as e:
        pw.pw_circuit_add_gate(c, [0, 5], np.eye(4))
    assert e.value.code == -1
    with pytest.raises(pw.PwError) as e:
        pw.pw_circuit_add_gate(c, [1, 1], np.eye(4))
    assert e.value.code == -1
    with pytest.raises(pw.PwError) as e:
        pw.pw_circuit_add_gate(c, [0], np.array([[np.nan, 0], [0, 1]]))
    assert e.value.code == -6
    H = np.array([[1, 1], [1, -1]]) / np.sqrt(2)
    with pytest.raises(pw.PwError) as e:     # Hadamard is not submonomial (App. A)
        pw.pw_circuit_add_kraus(c, [0], [H])
    assert e.value.code == -2
    with pytest.raises(pw.PwError) as e:     # CNOT-like 2-qubit Kraus is not a tensor product
        cn = np.eye(4)[[0, 3, 2, 1]]
        pw.pw_circuit_add_kraus(c, [0, 1], [0.5 * cn + 0.5 * np.eye(4)])
    assert e.value.code == -2
    pw.pw_circuit_destroy(c)


def test_dense_pass_descriptor_validation(pw):
    """pw_dense_apply checks its descriptor before any device work (zero
    tensors: nothing runs): distinct tile and row bits, widths, gemm kinds."""
    SPLIT3 = 0
    desc = pw.make_dense_desc(14, [7, 8, 9, 10, 11, 12], [0, 1, 2, 3, 4, 5, 6])
    pw.pw_dense_apply(SPLIT3, desc, 0, None, None)
    with pytest.raises(pw.PwError) as e:
        pw.pw_dense_apply(9, desc, 0, None, None)     # not a PW_GEMM_* kind
    assert e.value.code == -1
    with pytest.raises(pw.PwError) as e:             # width below tile_bits + 7
        pw.pw_dense_apply(SPLIT3, pw.make_dense_desc(12, [7, 8, 9, 10, 11, 5], [0, 1, 2, 3, 4, 6, 12]), 0, None, None)
    assert e.value.code == -1
    bad = pw.make_dense_desc(14, [7, 8, 9, 10, 11, 12], [0, 1, 2, 3, 4, 5, 7])   # row bit 7 is a tile bit
    with pytest.raises(pw.PwError) as e:
        pw.pw_dense_apply(SPLIT3, bad, 0, None, None)
    assert e.value.code == -1


def test_unsupported_structures_are_rejected(pw):
    H = np.array([[1, 1], [1, -1]]) / np.sqrt(2)
    cnot = np.eye(4)[[0, 3, 2, 1]]
    c = pw.pw_circuit_create(2)
    pw.pw_circuit_add_gate(c, [0], H)
    pw.pw_circuit_add_gate(c, [1], H)
    pw.pw_circuit_add_gate(c, [0, 1], cnot)
    with pytest.raises(pw.PwError) as e:
        pw.pw_plan_build(c)
    assert e.value.code == -7
    pw.pw_circuit_destroy(c)
    c = pw.pw_circuit_create(2)
    pw.pw_circuit_add_gate(c, [0], H)       # layer incomplete, then a diagonal gate
    pw.pw_circuit_add_gate(c, [0, 1], np.diag([1, -1, -1, 1]))
    with pytest.raises(pw.PwError):
        pw.pw_plan_build(c)
    pw.pw_circuit_destroy(c)


@pytest.mark.parametrize("spec,S,K", [(W.grid_6x6_p2(), 6, 6), (W.grid_8x8_p2_noisy(), 8, 8)])
def test_grid_plans_sweep_rows(pw, spec, S, K):
    c = _circ(pw, spec)
    plan = pw.pw_plan_build(c)
    st = pw.pw_plan_stats(plan)
    assert st["n_slots"] == S and st["n_blocks"] == K
    assert st["width_bits"] == S * spec.p and st["width_low_bits"] == S * (spec.p - 1)
    assert st["sampled_gates"] == spec.n * spec.p
    assert st["amps_per_sample"] == 2 * spec.n * spec.p
    pw.pw_plan_destroy(plan)
    pw.pw_circuit_destroy(c)


def test_hbm_plan_of_the_64_qubit_grid(pw):
    """The HBM engine's plan of the 8x8 noisy grid (p = 2): 2^16-entry
    frontiers, 6-bit GEMM tiles, split-3 passes by default. Readout blocks of
    6 sites give 11 blocks and 28 dense passes per chain, blocks of 8 give 8
    and 35. Tiles over dead legs are skipped, so the passes' flops stay well
    below those of full-width passes (2^16 x 2^6 complex multiply-adds each)."""
    spec = W.grid_8x8_p2_noisy()
    c = _circ(pw, spec)
    auto = pw.pw_plan_build(c)
    assert pw.pw_plan_stats(auto)["engine"] == pw.PW_ENGINE_ONCHIP   # 2^16 entries fit a cluster
    pw.pw_plan_destroy(auto)
    for max_block, blocks, passes in ((6, 11, 28), (8, 8, 35)):
        plan = pw.pw_plan_build(c, max_block=max_block, engine=pw.PW_ENGINE_HBM)
        st = pw.pw_plan_stats(plan)
        assert st["engine"] == pw.PW_ENGINE_HBM and st["gemm"] == pw.PW_GEMM_SPLIT3
        assert st["width_bits"] == 16 and st["dense_tile_bits"] == 6 and st["noisy"] == 1
        assert st["n_blocks"] == blocks and st["dense_passes_per_sample"] == passes
        full = passes * (1 << 16) * (1 << 6) * 8
        assert 0.2 * full < st["dense_flops_per_sample"] < 0.8 * full
        pw.pw_plan_destroy(plan)
    pw.pw_circuit_destroy(c)


def test_exec_order_is_a_valid_reordering(pw):
    spec = W.random_qaoa(14, 2, seed=8, with_h=True, depol2=0.01, ad_gamma=0.01)
    c = _circ(pw, spec)
    plan = pw.pw_plan_build(c)
    order = pw.pw_plan_exec_order(plan)
    nops = pw.pw_circuit_num_ops(c)
    assert sorted(order.tolist()) == list(range(nops))
    # only one-qubit gates of one layer move, and only among themselves
    from oracle import circuit as OC
    ops = OC.qaoa_circuit(spec)
    kinds = [(o.kind, len(o.qubits)) for o in ops]
    assert [kinds[i] for i in order] == kinds
    pw.pw_plan_destroy(plan)
    pw.pw_circuit_destroy(c)


def test_lsm_noise_keeps_the_plan_shape(pw):
    # Prop. 2: with LSM noise the network, the contraction order and its cost
    # are those of the noiseless circuit
    base = W.grid_6x6_p2()
    noisy = W.grid_6x6_p2()
    noisy.depol2, noisy.ad_gamma = 1e-3, 1e-3
    s = []
    for spec in (base, noisy):
        c = _circ(pw, spec)
        plan = pw.pw_plan_build(c)
        s.append(pw.pw_plan_stats(plan))
        pw.pw_plan_destroy(plan)
        pw.pw_circuit_destroy(c)
    for key in ("n_slots", "width_bits", "width_low_bits", "n_blocks", "sampled_gates", "flops_per_sample"):
        assert s[0][key] == s[1][key], key
    assert s[1]["noisy"] == 1 and s[0]["noisy"] == 0


def test_orders_and_widths(pw):
    # 3-regular and heavy-hex graphs: the automatic order keeps the frontier small
    for spec, smax in ((W.maxcut_3reg_n12(), 6), (W.heavy_hex_400_p1(), 14)):
        c = _circ(pw, spec)
        plan = pw.pw_plan_build(c)
        st = pw.pw_plan_stats(plan)
        assert st["n_slots"] <= smax
        natural = pw.pw_plan_build(c, order=pw.PW_ORDER_NATURAL)
        assert pw.pw_plan_stats(natural)["n_slots"] >= st["n_slots"]
        pw.pw_plan_destroy(natural)
        pw.pw_plan_destroy(plan)
        pw.pw_circuit_destroy(c)


def test_bad_options(pw):
    spec = W.maxcut_3reg_n12()
    c = _circ(pw, spec)
    with pytest.raises(pw.PwError):
        pw.pw_plan_build(c, precision=7)
    with pytest.raises(pw.PwError):
        pw.pw_plan_build(c, threads_per_chain=48)
    pw.pw_circuit_destroy(c)


def test_pack_roundtrip(pw):
    x = W.random_bitstrings(9, 130, seed=3)
    assert np.array_equal(pw.unpack_bits(pw.pack_bits(x), 130), x)


def _degenerate_specs():
    """Degenerate QAOA circuits: no edges at all, isolated qubits (qubit 0
    among them), a monomial mixer (beta = pi/2: RX(pi) = -iX), gamma = 0 and
    beta = 0 (identity mixers, nothing to sample)."""
    def spec(n, edges, p, gammas, betas, name):
        e = np.array(edges, dtype=np.int64).reshape(-1, 2)
        return W.QaoaSpec(n=n, edges=e, weights=np.ones(len(e)), gammas=np.array(gammas, dtype=float),
                          betas=np.array(betas, dtype=float), h=None, depol2=0.0, ad_gamma=0.0, name=name, extra={})
    return [spec(1, [], 1, [0.3], [0.2], "n1_no_edges"),
            spec(2, [], 2, [0.3, 0.1], [0.2, 0.5], "n2_no_edges_p2"),
            spec(3, [(1, 2)], 2, [0.4, 0.2], [0.3, 0.6], "qubit0_isolated"),
            spec(5, [(1, 2), (3, 4)], 3, [0.4, 0.2, 0.7], [0.3, 0.6, 0.1], "qubits_0_isolated_pairs"),
            spec(4, [(0, 1), (1, 2), (2, 3)], 2, [0.4, 0.3], [np.pi / 2, 0.5], "monomial_mixer"),
            spec(4, [(0, 1), (1, 2), (2, 3)], 2, [0.0, 0.0], [0.3, 0.7], "gamma0"),
            spec(5, [(0, 1), (1, 2), (2, 3), (3, 4)], 1, [0.5], [0.0], "beta0")]


@pytest.mark.parametrize("spec", _degenerate_specs(), ids=lambda s: s.name)
def test_degenerate_circuits_plan_every_gate(pw, spec):
    """Every op appears once in the execution order (an isolated qubit 0 was
    once left out of the sweep order), and every non-diagonal mixer is a
    sampled gate."""
    from oracle import circuit as OC
    c = _circ(pw, spec)
    plan = pw.pw_plan_build(c)
    order = pw.pw_plan_exec_order(plan)
    assert sorted(order.tolist()) == list(range(pw.pw_circuit_num_ops(c)))
    ops = OC.qaoa_circuit(spec)
    mixers = sum(1 for o in ops[spec.n:] if o.kind == "gate" and len(o.qubits) == 1 and not OC.is_diagonal(o.mat))
    assert pw.pw_plan_stats(plan)["sampled_gates"] == mixers
    pw.pw_plan_destroy(plan)
    pw.pw_circuit_destroy(c)


def test_ops_inside_a_layer_move_out_exactly(pw):
    """Channels right after each one-qubit gate of a layer (a device noise
    model) are moved past the layer by the planner; the exported order must
    give the same density matrix as circuit order (the moves commute)."""
    from oracle import circuit as OC
    from oracle import statevector as SV
    from tests.test_gpu_parity import _chip_noise_qaoa
    spec = W.random_qaoa(4, 2, seed=57)
    ops = _chip_noise_qaoa(spec, (0.06, (0.02, 0.03, 0.05), 0.1, 0.2, 0.04))
    c = pw.pw_circuit_create(spec.n)
    for o in ops:
        if o.kind == "gate":
            pw.pw_circuit_add_gate(c, list(o.qubits), o.mat)
        else:
            pw.pw_circuit_add_kraus(c, list(o.qubits), o.mats)
    plan = pw.pw_plan_build(c)
    order = pw.pw_plan_exec_order(plan)
    assert sorted(order.tolist()) == list(range(len(ops)))
    assert order.tolist() != list(range(len(ops)))   # something did move
    r1 = SV.density_run(spec.n, ops)
    r2 = SV.density_run(spec.n, [ops[i] for i in order])
    assert np.abs(r1 - r2).max() < 1e-14
    # an op on one qubit that had its gate and one that had not cannot move
    c2 = pw.pw_circuit_create(2)
    H = OC.h_mat()
    pw.pw_circuit_add_gate(c2, [0], H)
    pw.pw_circuit_add_gate(c2, [1], H)
    pw.pw_circuit_add_gate(c2, [0], OC.rx_mat(0.3))
    pw.pw_circuit_add_gate(c2, [0, 1], OC.rzz_mat(0.4))
    pw.pw_circuit_add_gate(c2, [1], OC.rx_mat(0.3))
    with pytest.raises(pw.PwError):
        pw.pw_plan_build(c2)
    pw.pw_plan_destroy(plan)
    pw.pw_circuit_destroy(c)
    pw.pw_circuit_destroy(c2)


def test_gradient_calls_validate_before_device_work(pw):
    """The gradient entry points check their arguments and plan the circuit
    before any CUDA call: no strings is a no-op, p < 1, missing buffers and
    an empty sample are errors (host-only paths)."""
    import ctypes as C
    from paper_2510_24218_gb300 import native as N
    lib = pw.load_library()
    spec = W.random_qaoa(6, 2, seed=81)
    e = np.ascontiguousarray(spec.edges.astype(np.int32).ravel())
    w = np.ascontiguousarray(spec.weights)
    g = np.ascontiguousarray(spec.gammas)
    b = np.ascontiguousarray(spec.betas)
    ip, dp = C.POINTER(C.c_int), C.POINTER(C.c_double)
    args = (spec.n, len(spec.edges), e.ctypes.data_as(ip), w.ctypes.data_as(dp), None)
    o = N.PlanOpts()
    assert lib.pw_qaoa_amp_grad(*args, 2, g.ctypes.data_as(dp), b.ctypes.data_as(dp), C.byref(o), 0, None, None,
                                None, None) == 0
    assert lib.pw_qaoa_amp_grad(*args, 0, g.ctypes.data_as(dp), b.ctypes.data_as(dp), C.byref(o), 0, None, None,
                                None, None) == -1
    assert lib.pw_qaoa_amp_grad(*args, 2, g.ctypes.data_as(dp), b.ctypes.data_as(dp), C.byref(o), 4, None, None,
                                None, None) == -1
    assert lib.pw_qaoa_cost_grad(*args, 2, g.ctypes.data_as(dp), b.ctypes.data_as(dp), C.byref(o), 0, None, None,
                                 None) == -1
    assert "n_samples" in pw.pw_last_error()
    # a structure the planner rejects is reported before any device work
    bad = np.ascontiguousarray(np.array([0, 0], dtype=np.int32))
    assert lib.pw_qaoa_amp_grad(spec.n, 1, bad.ctypes.data_as(ip), w.ctypes.data_as(dp), None, 2,
                                g.ctypes.data_as(dp), b.ctypes.data_as(dp), C.byref(o), 0, None, None, None,
                                None) < 0


def test_general_gradient_validates_its_arguments(pw):
    """pw_amp_grad rejects bad parameter maps and parameterised channels on
    the host, before any device work."""
    import ctypes as C
    from paper_2510_24218_gb300 import native as N
    from oracle import circuit as OC
    lib = pw.load_library()
    spec = W.random_qaoa(4, 1, seed=82, depol2=0.1)
    ops = OC.qaoa_circuit(spec)
    circ = pw.pw_circuit_qaoa(spec.n, spec.edges, spec.weights, None, 1, spec.gammas, spec.betas, spec.depol2)
    n_ops = pw.pw_circuit_num_ops(circ)
    o = N.PlanOpts()
    ip, dp = C.POINTER(C.c_int), C.POINTER(C.c_double)
    d = np.zeros(2 * 16 * n_ops)
    def call(param, n_params=2):
        q = np.ascontiguousarray(np.asarray(param, dtype=np.int32))
        return lib.pw_amp_grad(circ, n_params, q.ctypes.data_as(ip), d.ctypes.data_as(dp), C.byref(o), 0, None,
                               None, None, None)
    assert call([-1] * n_ops) == 0
    assert call([-1] * n_ops, n_params=0) == -1
    assert call([5] + [-1] * (n_ops - 1)) == -1
    kraus_at = next(i for i, op in enumerate(ops) if op.kind == "kraus")
    bad = [-1] * n_ops
    bad[kraus_at] = 0
    assert call(bad) == -1 and "must be a gate" in pw.pw_last_error()
    pw.pw_circuit_destroy(circ)


def test_swap_class_gates_plan_or_fail_cleanly(pw):
    """SWAP-class two-qubit gates between sections plan (the exported order is
    a permutation of every operation); in a noisy circuit, or placed where a
    wire would get two gates of one layer, they are refused."""
    from oracle import circuit as OC
    S = np.eye(4)[[0, 2, 1, 3]].astype(complex)
    spec = W.random_qaoa(6, 2, seed=83)
    ops = OC.qaoa_circuit(spec)
    n = spec.n
    pos = n + len(spec.edges)          # after layer 1's cost gates, before its mixers

    def plan_of(oplist):
        c = pw.pw_circuit_create(n)
        for o in oplist:
            if o.kind == "gate":
                pw.pw_circuit_add_gate(c, list(o.qubits), o.mat)
            else:
                pw.pw_circuit_add_kraus(c, list(o.qubits), o.mats)
        try:
            p = pw.pw_plan_build(c)
            order = pw.pw_plan_exec_order(p)
            pw.pw_plan_destroy(p)
            return order
        finally:
            pw.pw_circuit_destroy(c)

    good = ops[:pos] + [OC.gate((0, 3), S)] + ops[pos:]
    assert sorted(plan_of(good)) == list(range(len(good)))
    # inside layer 1's mixers, after qubit 0's mixer and before qubit 3's
    bad = ops[:pos + 1] + [OC.gate((0, 3), S)] + ops[pos + 1:]
    with pytest.raises(pw.PwError):
        plan_of(bad)
    noisy = W.random_qaoa(6, 2, seed=83, depol2=0.1)
    nops = OC.qaoa_circuit(noisy)
    with pytest.raises(pw.PwError, match="SWAP-class"):
        plan_of(nops[:n] + [OC.gate((0, 3), S)] + nops[n:])


def test_binding_has_every_declared_call(pw):
    """The Python binding offers every call of the C ABI under its own name."""
    missing = [name for name in _declared_functions() if not hasattr(pw, name)]
    assert not missing, missing
