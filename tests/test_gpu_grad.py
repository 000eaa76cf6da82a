"""GPU parity of pw_qaoa_amp_grad: exact derivatives of QAOA amplitudes
against the oracle's generator-insertion gradients (state vector on small
circuits, variable elimination on the 36-qubit grid)."""
import numpy as np
import pytest

import workloads as W
from oracle import gradient as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_24218_gb300 as mod
    mod.load_library()
    return mod


def _grad(pw, spec, xs, precision):
    import torch
    bits = torch.from_numpy(pw.pack_bits(xs).view(np.int64)).cuda()
    grad = torch.full((len(xs), 2 * spec.p, 2), np.nan, dtype=torch.float64, device="cuda")
    amp = torch.zeros((len(xs), 2), dtype=torch.float64, device="cuda")
    pw.pw_qaoa_amp_grad(spec.n, spec.edges, spec.weights, spec.h, spec.p, spec.gammas, spec.betas, bits, grad,
                        amp_out=amp, precision=precision)
    g = grad.cpu().numpy()
    a = amp.cpu().numpy()
    return a[:, 0] + 1j * a[:, 1], g[..., 0] + 1j * g[..., 1]


@pytest.mark.parametrize("with_h", [False, True])
@pytest.mark.parametrize("prec,tol", [(1, 1e-11), (0, 2e-5)])
def test_gradient_against_state_vector(pw, with_h, prec, tol):
    """12 qubits, p = 3: every derivative of 24 amplitudes; FP64 to 1e-11 and
    FP32 to 2e-5 of the largest derivative."""
    spec = W.random_qaoa(12, 3, seed=31 + with_h, with_h=with_h)
    xs = W.random_bitstrings(24, spec.n, seed=32)
    amp, grad = _grad(pw, spec, xs, prec)
    want_amp, want = G.amp_and_grad(spec, xs)
    scale = np.abs(want).max()
    assert np.abs(grad - want).max() <= tol * scale
    assert np.abs(amp - want_amp).max() <= tol * np.abs(want_amp).max()


def test_gradient_grid6x6_against_elimination(pw):
    """The 36-qubit 6x6 grid at p = 2 (FP64): d amp / d gamma_1 and
    d amp / d beta_0 of two bitstrings against the elimination oracle."""
    spec = W.grid_6x6_p2()
    xs = W.random_bitstrings(2, spec.n, seed=33)
    _, grad = _grad(pw, spec, xs, 1)
    cols = [1, spec.p]
    want = G.amp_and_grad_tn(spec, xs, columns=cols)
    for c in cols:
        assert np.abs(grad[:, c] - want[:, c]).max() <= 1e-10 * np.abs(want[:, c]).max()


def test_gradient_edge_cases(pw):
    import torch
    spec = W.random_qaoa(6, 1, seed=34)
    empty = torch.zeros((0, 1), dtype=torch.int64, device="cuda")
    grad = torch.zeros((0, 2, 2), dtype=torch.float64, device="cuda")
    pw.pw_qaoa_amp_grad(spec.n, spec.edges, spec.weights, None, 1, spec.gammas, spec.betas, empty, grad)
    with pytest.raises(pw.PwError):
        pw.pw_qaoa_amp_grad(spec.n, spec.edges, spec.weights, None, 0, spec.gammas, spec.betas, empty, grad)
    # a zero weight drops its term; the result still matches the oracle
    spec.weights[0] = 0.0
    xs = W.random_bitstrings(4, spec.n, seed=35)
    _, got = _grad(pw, spec, xs, 1)
    _, want = G.amp_and_grad(spec, xs)
    assert np.abs(got - want).max() <= 1e-11 * np.abs(want).max()


def test_autograd_function_matches_oracle_gradient(pw):
    """The torch.autograd binding: a real loss of the amplitudes back-propagates
    the oracle's derivatives, and gradcheck's finite differences agree."""
    import torch
    from paper_2510_24218_gb300.autograd import qaoa_amplitudes
    spec = W.random_qaoa(10, 2, seed=36, with_h=True)
    xs = W.random_bitstrings(6, spec.n, seed=37)
    bits = torch.from_numpy(pw.pack_bits(xs).view(np.int64)).cuda()
    gam = torch.tensor(spec.gammas, dtype=torch.float64, requires_grad=True)
    bet = torch.tensor(spec.betas, dtype=torch.float64, requires_grad=True)
    c = torch.from_numpy(np.random.default_rng(38).normal(size=(6, 2))).cuda()
    loss = (qaoa_amplitudes(gam, bet, spec.n, spec.edges, spec.weights, spec.h, bits) * c).sum()
    loss.backward()
    _, want = G.amp_and_grad(spec, xs)
    cc = c.cpu().numpy()
    want_d = (cc[:, :1] * want.real + cc[:, 1:] * want.imag).sum(axis=0)
    got = np.concatenate([gam.grad.numpy(), bet.grad.numpy()])
    assert np.abs(got - want_d).max() <= 1e-11 * np.abs(want_d).max()
    f = lambda g_, b_: qaoa_amplitudes(g_, b_, spec.n, spec.edges, spec.weights, spec.h, bits)  # noqa: E731
    assert torch.autograd.gradcheck(f, (gam.detach().requires_grad_(), bet.detach().requires_grad_()),
                                    eps=1e-6, atol=1e-7, rtol=1e-5)


def _closed_form_cost(spec, g, b):
    from oracle import closed_form as CF
    return float(np.dot(spec.weights, CF.zz_p1(spec.n, spec.edges, spec.weights, g, b)))


def test_score_function_cost_gradient_against_p1_closed_form(pw):
    """Samples of a 20-qubit 3-regular p = 1 circuit from the GPU sampler feed
    pw_qaoa_cost_grad; its mean cost and its gradient estimate agree with the
    closed-form p = 1 expectation (and its central differences) within five
    standard errors, and with the same estimator formed on the host from
    pw_qaoa_amp_grad to 1e-10."""
    import torch
    from tests.test_gpu_parity import run_gpu
    spec = W.random_qaoa(20, 1, seed=39)
    N = 20000
    g = run_gpu(pw, spec, N, seed=40, precision=1, trace=False)
    xs = g["bits"]
    bits = torch.from_numpy(pw.pack_bits(xs).view(np.int64)).cuda()
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    pw.pw_qaoa_cost_grad(spec.n, spec.edges, spec.weights, None, 1, spec.gammas, spec.betas, bits, out,
                         precision=pw.PW_PREC_FP64)
    got = out.cpu().numpy()
    # host formation of the same estimator from the amplitude derivatives
    amp, grad = _grad(pw, spec, xs, 1)
    z = 1.0 - 2.0 * xs.astype(np.float64)
    cost = (spec.weights * z[:, spec.edges[:, 0]] * z[:, spec.edges[:, 1]]).sum(axis=1)
    score = 2.0 * (np.conj(amp)[:, None] * grad).real / (np.abs(amp) ** 2)[:, None]
    est = N / (N - 1) * ((cost[:, None] * score).mean(axis=0) - cost.mean() * score.mean(axis=0))
    assert abs(got[0] - cost.mean()) <= 1e-10 * np.abs(cost).max()
    assert np.abs(got[1:] - est).max() <= 1e-9 * np.abs(est).max()
    # statistics against the closed form
    ga, be = float(spec.gammas[0]), float(spec.betas[0])
    exact_c = _closed_form_cost(spec, ga, be)
    assert abs(cost.mean() - exact_c) <= 5 * cost.std() / np.sqrt(N)
    hstep = 1e-6
    d_exact = [(_closed_form_cost(spec, ga + hstep, be) - _closed_form_cost(spec, ga - hstep, be)) / (2 * hstep),
               (_closed_form_cost(spec, ga, be + hstep) - _closed_form_cost(spec, ga, be - hstep)) / (2 * hstep)]
    for j in range(2):
        se = ((cost - cost.mean()) * score[:, j]).std() / np.sqrt(N)
        assert abs(got[1 + j] - d_exact[j]) <= 5 * se, (j, got[1 + j], d_exact[j], se)


def test_gradient_cluster_instance_in_bench_configuration(pw):
    """The gradient workload's launch configuration: the first seeded p = 3
    3-regular instance whose FP32 plan runs on a 2-CTA cluster, 64 bitstrings
    drawn by its own sampler; two of them checked against the elimination
    oracle on every derivative, to 1e-4 of the largest (FP32 amplitudes summed
    over 3(|E| + n) terms), and every row finite."""
    import torch
    spec = None
    for s in W.gradient_instances():
        c = pw.pw_circuit_qaoa(s.n, s.edges, s.weights, None, s.p, s.gammas, s.betas)
        try:
            pl = pw.pw_plan_build(c)
        except pw.PwError:
            pw.pw_circuit_destroy(c)
            continue
        st = pw.pw_plan_stats(pl)
        if st["ctas_per_chain"] == 2 and s.n <= 22:
            spec = s
            bits = torch.empty((64, 1), dtype=torch.int64, device="cuda")
            pw.pw_sample(pl, 11, 0, 64, bits, None)
        pw.pw_plan_destroy(pl)
        pw.pw_circuit_destroy(c)
        if spec is not None:
            break
    assert spec is not None
    xs = pw.unpack_bits(bits.cpu().numpy(), spec.n)
    _, grad = _grad(pw, spec, xs, 0)
    assert np.isfinite(grad).all()
    want = G.amp_and_grad_tn(spec, xs[[0, 37]])
    assert np.abs(grad[[0, 37]] - want).max() <= 1e-4 * np.abs(want).max()


def test_cost_gradient_with_fields_against_exact_expectation(pw):
    """With fields h the cost gains sum_j h_j z_j: the kernel's estimate equals
    the host-formed one, and it is within five standard errors of the exact
    d E[C] from the state-vector oracle (sum over all 2^n strings)."""
    import torch
    from tests.test_gpu_parity import run_gpu
    spec = W.random_qaoa(10, 2, seed=41, with_h=True)
    N = 8000
    xs = run_gpu(pw, spec, N, seed=42, precision=1, trace=False)["bits"]
    bits = torch.from_numpy(pw.pack_bits(xs).view(np.int64)).cuda()
    out = torch.zeros(1 + 2 * spec.p, dtype=torch.float64, device="cuda")
    pw.pw_qaoa_cost_grad(spec.n, spec.edges, spec.weights, spec.h, spec.p, spec.gammas, spec.betas, bits, out,
                         precision=pw.PW_PREC_FP64)
    got = out.cpu().numpy()

    def cost_of(x):
        z = 1.0 - 2.0 * x.astype(np.float64)
        return (spec.weights * z[:, spec.edges[:, 0]] * z[:, spec.edges[:, 1]]).sum(axis=1) + z @ spec.h

    amp, grad = _grad(pw, spec, xs, 1)
    cost = cost_of(xs)
    score = 2.0 * (np.conj(amp)[:, None] * grad).real / (np.abs(amp) ** 2)[:, None]
    est = N / (N - 1) * ((cost[:, None] * score).mean(axis=0) - cost.mean() * score.mean(axis=0))
    assert abs(got[0] - cost.mean()) <= 1e-10 * np.abs(cost).max()
    assert np.abs(got[1:] - est).max() <= 1e-9 * np.abs(est).max()
    allx = np.array([[(i >> q) & 1 for q in range(spec.n)] for i in range(1 << spec.n)], dtype=np.uint8)
    a_all, g_all = G.amp_and_grad(spec, allx)
    c_all = cost_of(allx)
    exact = (c_all[:, None] * 2.0 * (np.conj(a_all)[:, None] * g_all).real).sum(axis=0)
    for j in range(2 * spec.p):
        se = ((cost - cost.mean()) * score[:, j]).std() / np.sqrt(N)
        assert abs(got[1 + j] - exact[j]) <= 5 * se, (j, got[1 + j], exact[j], se)


def test_gradient_is_deterministic_across_calls(pw):
    """The derivative terms run on concurrent streams with fresh plans each
    call; four calls give bit-identical FP64 rows (each plan's tables are
    complete before any stream reads them, and the lanes are summed in a fixed
    order), equal to the oracle."""
    import torch
    spec = W.random_qaoa(16, 1, seed=43)
    N = 20000
    xs = W.random_bitstrings(N, spec.n, seed=44)
    bits = torch.from_numpy(pw.pack_bits(xs).view(np.int64)).cuda()
    runs = []
    for _ in range(4):
        g = torch.full((N, 2, 2), np.nan, dtype=torch.float64, device="cuda")
        pw.pw_qaoa_amp_grad(spec.n, spec.edges, spec.weights, None, 1, spec.gammas, spec.betas, bits, g,
                            precision=pw.PW_PREC_FP64)
        runs.append(g.cpu().numpy())
    assert all(np.array_equal(runs[0], r) for r in runs[1:])
    _, want = G.amp_and_grad(spec, xs[:500])
    got = runs[0][:500, :, 0] + 1j * runs[0][:500, :, 1]
    assert np.abs(got - want).max() <= 1e-11 * np.abs(want).max()


def _build_param_circuit(pw, n, ops):
    circ = pw.pw_circuit_create(n)
    for o in ops:
        pw.pw_circuit_add_gate(circ, o.qubits, o.mat)
    return circ


@pytest.mark.parametrize("prec,tol", [(1, 1e-11), (0, 2e-5)])
def test_general_parameterised_gradient_against_product_rule_oracle(pw, prec, tol):
    """pw_amp_grad on a circuit with one parameter per layer on its RZZ gates
    and one per RY mixer (26 parameters, 12 qubits, p = 2) against the oracle's
    product rule on the state vector; a parameter nothing depends on is zero."""
    import torch
    from tests.test_oracle_gradient import parameterised_circuit
    rng = np.random.default_rng(45)
    n, p = 12, 2
    spec = W.random_qaoa(n, 1, seed=46)
    theta = rng.uniform(0, np.pi, size=p + p * n)
    ops, param, dm = parameterised_circuit(n, spec.edges, spec.weights, theta, p)
    circ = _build_param_circuit(pw, n, ops)
    xs = W.random_bitstrings(24, n, seed=47)
    bits = torch.from_numpy(pw.pack_bits(xs).view(np.int64)).cuda()
    n_params = len(theta) + 1
    grad = torch.full((24, n_params, 2), np.nan, dtype=torch.float64, device="cuda")
    amp = torch.zeros((24, 2), dtype=torch.float64, device="cuda")
    pw.pw_amp_grad(circ, n_params, param, dm, bits, grad, amp_out=amp, precision=prec)
    pw.pw_circuit_destroy(circ)
    g = grad.cpu().numpy()
    g = g[..., 0] + 1j * g[..., 1]
    want = G.amp_grad_product_rule(n, ops, param, dm, n_params, xs)
    assert np.abs(g - want).max() <= tol * np.abs(want).max()
    assert not g[:, -1].any()
    a = amp.cpu().numpy()
    from oracle import statevector as SV
    psi = SV.run(n, ops)
    idx = [int(sum(int(b) << q for q, b in enumerate(x))) for x in xs]
    assert np.abs(a[:, 0] + 1j * a[:, 1] - psi[idx]).max() <= tol * np.abs(psi[idx]).max()


def test_general_gradient_equals_qaoa_gradient(pw):
    """The QAOA circuit written as a parameterised circuit (the gammas on the
    RZZ and RZ gates, the betas on the RX gates, derivatives -i coef G A) gives
    the rows of pw_qaoa_amp_grad."""
    import torch
    from oracle import circuit as OC
    spec = W.random_qaoa(10, 2, seed=48, with_h=True)
    ops = OC.qaoa_circuit(spec)
    n, p = spec.n, spec.p
    Z2 = np.diag([1.0, -1.0, -1.0, 1.0]).astype(complex)
    Z1 = np.diag([1.0, -1.0]).astype(complex)
    X1 = np.array([[0, 1], [1, 0]], dtype=complex)
    param, dm = [-1] * n, []
    pos = n
    for l in range(p):
        for w in spec.weights:
            param.append(l)
            dm.append(-1j * w * Z2 @ ops[pos].mat)
            pos += 1
        for j in range(n):
            param.append(l)
            dm.append(-1j * spec.h[j] * Z1 @ ops[pos].mat)
            pos += 1
        for j in range(n):
            param.append(p + l)
            dm.append(-1j * X1 @ ops[pos].mat)
            pos += 1
    circ = _build_param_circuit(pw, n, ops)
    xs = W.random_bitstrings(16, n, seed=49)
    bits = torch.from_numpy(pw.pack_bits(xs).view(np.int64)).cuda()
    g1 = torch.zeros((16, 2 * p, 2), dtype=torch.float64, device="cuda")
    pw.pw_amp_grad(circ, 2 * p, param, dm, bits, g1, precision=pw.PW_PREC_FP64)
    pw.pw_circuit_destroy(circ)
    _, g2 = _grad(pw, spec, xs, 1)
    a = g1.cpu().numpy()
    assert np.abs(a[..., 0] + 1j * a[..., 1] - g2).max() <= 1e-12 * np.abs(g2).max()


def test_general_gradient_with_swap_class_gates(pw):
    """pw_amp_grad on a parameterised circuit with SWAP-class gates between
    its sections (planned as wire relabellings) against the product rule on
    the state vector, FP64."""
    import torch
    from oracle import circuit as OC
    from tests.test_oracle_gradient import parameterised_circuit
    rng = np.random.default_rng(50)
    n, p = 8, 2
    spec = W.random_qaoa(n, 1, seed=51)
    theta = rng.uniform(0, np.pi, size=p + p * n)
    ops, param, dm = parameterised_circuit(n, spec.edges, spec.weights, theta, p)
    pos = n + len(spec.edges)          # after layer 1's RZZ gates, before its RY gates
    S = np.eye(4)[[0, 2, 1, 3]].astype(complex)
    ops = ops[:pos] + [OC.gate((0, 5), S), OC.gate((2, 3), OC.iswap_mat())] + ops[pos:]
    param = param[:pos] + [-1, -1] + param[pos:]
    circ = _build_param_circuit(pw, n, ops)
    xs = W.random_bitstrings(12, n, seed=52)
    bits = torch.from_numpy(pw.pack_bits(xs).view(np.int64)).cuda()
    grad = torch.zeros((12, len(theta), 2), dtype=torch.float64, device="cuda")
    pw.pw_amp_grad(circ, len(theta), param, dm, bits, grad, precision=pw.PW_PREC_FP64)
    pw.pw_circuit_destroy(circ)
    g = grad.cpu().numpy()
    want = G.amp_grad_product_rule(n, ops, param, dm, len(theta), xs)
    assert np.abs(g[..., 0] + 1j * g[..., 1] - want).max() <= 1e-11 * np.abs(want).max()


def test_autograd_general_circuit(pw):
    """The autograd binding of pw_amp_grad: a real loss of the amplitudes of a
    parameterised circuit back-propagates the product-rule derivatives, and
    gradcheck's finite differences agree."""
    import torch
    from paper_2510_24218_gb300.autograd import circuit_amplitudes
    from tests.test_oracle_gradient import parameterised_circuit
    rng = np.random.default_rng(53)
    n, p = 8, 2
    spec = W.random_qaoa(n, 1, seed=54)

    def build(th):
        ops, param, dm = parameterised_circuit(n, spec.edges, spec.weights, th, p)
        return [(list(o.qubits), o.mat) for o in ops], param, dm

    theta = torch.tensor(rng.uniform(0, np.pi, size=p + p * n), dtype=torch.float64, requires_grad=True)
    xs = W.random_bitstrings(5, n, seed=55)
    bits = torch.from_numpy(pw.pack_bits(xs).view(np.int64)).cuda()
    c = torch.from_numpy(rng.normal(size=(5, 2))).cuda()
    (circuit_amplitudes(theta, build, n, bits) * c).sum().backward()
    ops, param, dm = parameterised_circuit(n, spec.edges, spec.weights, theta.detach().numpy(), p)
    want = G.amp_grad_product_rule(n, ops, param, dm, theta.numel(), xs)
    cc = c.cpu().numpy()
    want_d = (cc[:, :1] * want.real + cc[:, 1:] * want.imag).sum(axis=0)
    assert np.abs(theta.grad.numpy() - want_d).max() <= 1e-11 * np.abs(want_d).max()
    f = lambda t: circuit_amplitudes(t, build, n, bits)  # noqa: E731
    assert torch.autograd.gradcheck(f, (theta.detach().requires_grad_(),), eps=1e-6, atol=1e-7, rtol=1e-5)


def test_gradient_wide_instances_against_elimination_differences(pw):
    """Four of the seeded p = 3 instances with n > 26 (beyond a state vector),
    FP32 plans as in the gradient workload: every derivative of two strings
    drawn by each instance's sampler against central differences (h = 1e-4) of
    the FP64 elimination oracle's amplitude, to 2e-4 of the largest."""
    import copy
    import torch
    from oracle import circuit as OC
    from oracle import tn as TN
    picked = []
    for s in W.gradient_instances():
        if s.n <= 26:
            continue
        c = pw.pw_circuit_qaoa(s.n, s.edges, s.weights, None, s.p, s.gammas, s.betas)
        try:
            # (the gradient workload's instances: frontiers that fit on chip)
            pl = pw.pw_plan_build(c, engine=pw.PW_ENGINE_ONCHIP)
        except pw.PwError:
            pw.pw_circuit_destroy(c)
            continue
        bits = torch.empty((2, 1), dtype=torch.int64, device="cuda")
        pw.pw_sample(pl, 13, 0, 2, bits, None)
        pw.pw_plan_destroy(pl)
        pw.pw_circuit_destroy(c)
        picked.append((s, pw.unpack_bits(bits.cpu().numpy(), s.n)))
        if len(picked) == 4:
            break
    assert len(picked) == 4
    h = 1e-4
    for spec, xs in picked:
        _, grad = _grad(pw, spec, xs, 0)
        fd = np.zeros_like(grad)
        for j in range(2 * spec.p):
            sp, sm = copy.deepcopy(spec), copy.deepcopy(spec)
            arr = "gammas" if j < spec.p else "betas"
            getattr(sp, arr)[j % spec.p] += h
            getattr(sm, arr)[j % spec.p] -= h
            ops_p, ops_m = OC.qaoa_circuit(sp), OC.qaoa_circuit(sm)
            for k, x in enumerate(xs):
                fd[k, j] = (TN.amplitudes(spec.n, ops_p, x) - TN.amplitudes(spec.n, ops_m, x)) / (2 * h)
        assert np.abs(grad - fd).max() <= 2e-4 * np.abs(fd).max(), spec.name


def test_gradient_on_the_hbm_engine(pw):
    """A p = 3 instance whose frontier (2^18 entries) exceeds the on-chip
    engine: every shifted-circuit amplitude runs on the HBM engine with
    tensor-core passes; the derivatives of one string against central
    differences (h = 1e-4) of the FP64 elimination oracle, 2e-4 of the
    largest."""
    import copy
    import torch
    from oracle import circuit as OC
    from oracle import tn as TN
    spec = [s for s in W.gradient_instances() if s.name == "qaoa_p3_3reg_n24_i7"][0]
    c = pw.pw_circuit_qaoa(spec.n, spec.edges, spec.weights, None, spec.p, spec.gammas, spec.betas)
    pl = pw.pw_plan_build(c)
    assert pw.pw_plan_stats(pl)["engine"] == pw.PW_ENGINE_HBM
    bits = torch.empty((1, 1), dtype=torch.int64, device="cuda")
    pw.pw_sample(pl, 17, 0, 1, bits, None)
    pw.pw_plan_destroy(pl)
    pw.pw_circuit_destroy(c)
    xs = pw.unpack_bits(bits.cpu().numpy(), spec.n)
    _, grad = _grad(pw, spec, xs, 0)
    h = 1e-4
    fd = np.zeros_like(grad)
    for j in range(2 * spec.p):
        sp, sm = copy.deepcopy(spec), copy.deepcopy(spec)
        arr = "gammas" if j < spec.p else "betas"
        getattr(sp, arr)[j % spec.p] += h
        getattr(sm, arr)[j % spec.p] -= h
        fd[0, j] = (TN.amplitudes(spec.n, OC.qaoa_circuit(sp), xs[0]) -
                    TN.amplitudes(spec.n, OC.qaoa_circuit(sm), xs[0])) / (2 * h)
    assert np.abs(grad - fd).max() <= 2e-4 * np.abs(fd).max()
