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
