"""Pins of the gradient oracle: a one-qubit closed form and central finite
differences of the state-vector amplitude."""
import copy

import numpy as np

import workloads as W
from oracle import circuit as OC
from oracle import gradient as G
from oracle import statevector as SV


def _amp(spec, x):
    psi = SV.run(spec.n, OC.qaoa_circuit(spec))
    return psi[int(sum(int(b) << q for q, b in enumerate(x)))]


def test_one_qubit_closed_form():
    # |+>, exp(-i g h Z), exp(-i b X):  amp0 = (cos b e^{-igh} - i sin b e^{igh}) / sqrt 2
    g, b, h = 0.37, 0.81, 1.3
    spec = W.QaoaSpec(n=1, edges=np.zeros((0, 2), dtype=np.int64), weights=np.zeros(0), gammas=np.array([g]),
                      betas=np.array([b]), h=np.array([h]), depol2=0.0, ad_gamma=0.0, name="one", extra={})
    amp, grad = G.amp_and_grad(spec, np.array([[0], [1]], dtype=np.uint8))
    e = np.exp(-1j * g * h)
    want0 = (np.cos(b) * e - 1j * np.sin(b) / e) / np.sqrt(2)
    want1 = (-1j * np.sin(b) * e + np.cos(b) / e) / np.sqrt(2)
    assert np.allclose(amp, [want0, want1], atol=1e-14)
    d_b0 = (-np.sin(b) * e - 1j * np.cos(b) / e) / np.sqrt(2)
    d_g0 = (-1j * h * np.cos(b) * e + h * np.sin(b) / e) / np.sqrt(2)
    assert abs(grad[0, 1] - d_b0) < 1e-14 and abs(grad[0, 0] - d_g0) < 1e-14


def test_gradient_matches_central_differences():
    spec = W.random_qaoa(7, 3, seed=21, with_h=True)
    xs = W.random_bitstrings(5, spec.n, seed=22)
    amp, grad = G.amp_and_grad(spec, xs)
    for k, x in enumerate(xs):
        assert abs(amp[k] - _amp(spec, x)) < 1e-13
        for j in range(2 * spec.p):
            hstep = 1e-5
            sp, sm = copy.deepcopy(spec), copy.deepcopy(spec)
            arr = "gammas" if j < spec.p else "betas"
            l = j % spec.p
            getattr(sp, arr)[l] += hstep
            getattr(sm, arr)[l] -= hstep
            fd = (_amp(sp, x) - _amp(sm, x)) / (2 * hstep)
            assert abs(fd - grad[k, j]) < 1e-8 * max(1.0, abs(grad[k, j])), (k, j)


def test_elimination_gradient_matches_state_vector_gradient():
    spec = W.random_qaoa(8, 2, seed=23, with_h=True)
    xs = W.random_bitstrings(3, spec.n, seed=24)
    _, want = G.amp_and_grad(spec, xs)
    got = G.amp_and_grad_tn(spec, xs)
    assert np.abs(got - want).max() < 1e-13
    part = G.amp_and_grad_tn(spec, xs, columns=[3])
    assert np.abs(part[:, 3] - want[:, 3]).max() < 1e-13 and not part[:, :3].any()


def test_expected_cost_gradient_matches_p1_closed_form():
    """sum_x C(x) 2 Re(conj(amp) d amp) over all 2^n strings is d E[C]; at
    p = 1 it must equal central differences of the closed-form correlators."""
    from oracle import closed_form as CF
    spec = W.random_qaoa(10, 1, seed=39)
    xs = np.array([[(i >> q) & 1 for q in range(spec.n)] for i in range(1 << spec.n)], dtype=np.uint8)
    amp, grad = G.amp_and_grad(spec, xs)
    z = 1.0 - 2.0 * xs
    cost = (spec.weights * z[:, spec.edges[:, 0]] * z[:, spec.edges[:, 1]]).sum(axis=1)
    d = (cost[:, None] * 2.0 * (np.conj(amp)[:, None] * grad).real).sum(axis=0)
    f = lambda g, b: float(np.dot(spec.weights, CF.zz_p1(spec.n, spec.edges, spec.weights, g, b)))  # noqa: E731
    g0, b0, h = float(spec.gammas[0]), float(spec.betas[0]), 1e-6
    want = [(f(g0 + h, b0) - f(g0 - h, b0)) / (2 * h), (f(g0, b0 + h) - f(g0, b0 - h)) / (2 * h)]
    assert np.allclose(d, want, atol=1e-7, rtol=0)


def ry_mat(phi):
    c, s = np.cos(phi / 2), np.sin(phi / 2)
    return np.array([[c, -s], [s, c]], dtype=complex)


def d_ry_mat(phi):
    c, s = np.cos(phi / 2), np.sin(phi / 2)
    return 0.5 * np.array([[-s, -c], [c, -s]], dtype=complex)


def parameterised_circuit(n, edges, weights, theta, p):
    """H layer, then per layer l: RZZ(theta[l] w_e) on every edge and
    RY(theta[p + l n + j]) on every qubit j. Returns (ops, param_of_op, dmats)."""
    Z2 = np.diag([1.0, -1.0, -1.0, 1.0]).astype(complex)
    ops = [OC.gate((q,), OC.h_mat()) for q in range(n)]
    param, dm = [-1] * n, []
    for l in range(p):
        for (u, v), w in zip(edges, weights):
            A = OC.rzz_mat(theta[l] * w)
            ops.append(OC.gate((int(u), int(v)), A))
            param.append(l)
            dm.append(w * (-0.5j) * Z2 @ A)
        for j in range(n):
            k = p + l * n + j
            ops.append(OC.gate((j,), ry_mat(theta[k])))
            param.append(k)
            dm.append(d_ry_mat(theta[k]))
    return ops, param, dm


def test_product_rule_gradient_matches_central_differences():
    rng = np.random.default_rng(25)
    n, p = 6, 2
    edges = np.array([(i, (i + 1) % n) for i in range(n)])
    weights = rng.normal(size=n)
    theta = rng.uniform(0, np.pi, size=p + p * n)
    xs = W.random_bitstrings(4, n, seed=26)
    ops, param, dm = parameterised_circuit(n, edges, weights, theta, p)
    got = G.amp_grad_product_rule(n, ops, param, dm, len(theta), xs)
    idx = [int(sum(int(b) << q for q, b in enumerate(x))) for x in xs]
    h = 1e-5
    for k in range(len(theta)):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fp = SV.run(n, parameterised_circuit(n, edges, weights, tp, p)[0])[idx]
        fm = SV.run(n, parameterised_circuit(n, edges, weights, tm, p)[0])[idx]
        assert np.abs((fp - fm) / (2 * h) - got[:, k]).max() < 1e-8, k
