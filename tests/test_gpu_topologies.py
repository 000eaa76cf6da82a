"""GPU: the other topologies of the paper's timing study (King's graph,
Chimera) at p = 1 with Gaussian couplings: the per-edge correlators
<Z_u Z_v> of the sampled bitstrings against the closed form of p = 1 QAOA
(the oracle's closed_form, pinned against the state vector), within shot
noise. The 100-qubit King's graph runs on the on-chip engine, the 128-qubit
Chimera graph (a 2^20-entry frontier) on the HBM engine with tensor-core
passes."""
import numpy as np
import pytest

import workloads as W
from oracle import closed_form as CF

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_24218_gb300 as mod
    mod.load_library()
    return mod


@pytest.mark.parametrize("make,engine,N", [(W.kings_10x10_p1, 1, 40000), (W.chimera_c444_p1, 2, 16384)])
def test_p1_correlators_on_other_topologies(pw, make, engine, N):
    import torch
    spec = make()
    c = pw.pw_circuit_qaoa(spec.n, spec.edges, spec.weights, spec.h, spec.p, spec.gammas, spec.betas)
    plan = pw.pw_plan_build(c)
    st = pw.pw_plan_stats(plan)
    assert st["engine"] == engine
    bits = torch.zeros((N, (spec.n + 63) // 64), dtype=torch.int64, device="cuda")
    pw.pw_sample(plan, 4242, 0, N, bits)
    x = pw.unpack_bits(bits.cpu().numpy(), spec.n).astype(np.int8)
    pw.pw_plan_destroy(plan)
    pw.pw_circuit_destroy(c)
    z = 1 - 2 * x
    u, v = spec.edges[:, 0], spec.edges[:, 1]
    emp = (z[:, u] * z[:, v]).mean(axis=0)
    want = CF.zz_p1(spec.n, spec.edges, spec.weights, spec.gammas[0], spec.betas[0])
    se = np.sqrt(np.maximum(1 - want ** 2, 1e-12) / N)
    zs = (emp - want) / se
    assert np.abs(zs).max() < 5.0, (np.abs(zs).max(), int(np.argmax(np.abs(zs))))
    # the global spin flip is a symmetry without fields: every <Z_j> is 0
    zj = z.mean(axis=0)
    assert np.abs(zj).max() < 5.0 / np.sqrt(N)
