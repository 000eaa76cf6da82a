"""GPU: the caller's allocator owns the library's device memory.

With torch's caching allocator registered (pw_set_allocator), the buffers the
library keeps (a plan's tables and counters, the HBM engine's frontiers,
environments, saved chain states and operators) and its scratch (the
gradient lanes) are torch allocations: torch.cuda.memory_allocated() counts
them while they live and drops back when they are released, and the samples
and derivatives are those of the default allocator."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_24218_gb300 as mod
    mod.load_library()
    return mod


def _sample(pw, spec, N, **opts):
    import torch
    c = pw.pw_circuit_qaoa(spec.n, spec.edges, spec.weights, spec.h, spec.p, spec.gammas, spec.betas,
                           spec.depol2, spec.ad_gamma)
    plan = pw.pw_plan_build(c, **opts)
    bits = torch.zeros((N, (spec.n + 63) // 64), dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    st = pw.pw_sample(plan, 7, 0, N, bits)
    torch.cuda.synchronize()
    held = torch.cuda.memory_allocated() - before
    pw.pw_plan_destroy(plan)
    pw.pw_circuit_destroy(c)
    torch.cuda.synchronize()
    released = torch.cuda.memory_allocated() - before
    return bits.cpu().numpy(), held, released, st


def test_torch_allocator_owns_the_hbm_engine_buffers(pw):
    spec = W.grid_8x8_p2_noisy()
    N = 512
    want, held0, _, st0 = _sample(pw, spec, N, engine=pw.PW_ENGINE_HBM, chains_per_launch=N)
    assert held0 == 0   # cudaMalloc: torch sees nothing
    pw.use_torch_allocator()
    try:
        got, held, released, st1 = _sample(pw, spec, N, engine=pw.PW_ENGINE_HBM, chains_per_launch=N)
    finally:
        pw.pw_set_allocator()
    assert held >= N * (1 << 16) * 8   # at least the chains' 2^16-entry frontiers
    assert released == 0
    differ = np.nonzero((got != want).any(axis=1))[0]
    assert len(differ) == 0, (differ[:10], st0, st1)


def test_torch_allocator_owns_the_gradient_scratch(pw):
    import torch
    spec = W.random_qaoa(12, 2, seed=3, with_h=True)
    bits = torch.from_numpy(pw.pack_bits(np.random.default_rng(1).integers(0, 2, (16, spec.n)).astype(np.uint8))
                            .view(np.int64)).cuda()

    def grad():
        g = torch.zeros((16, 2 * spec.p, 2), dtype=torch.float64, device="cuda")
        pw.pw_qaoa_amp_grad(spec.n, spec.edges, spec.weights, spec.h, spec.p, spec.gammas, spec.betas, bits, g,
                            precision=pw.PW_PREC_FP64)
        return g.cpu().numpy()

    want = grad()
    pw.use_torch_allocator()
    try:
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        m0 = torch.cuda.memory_allocated()
        got = grad()
        torch.cuda.synchronize()
        peak = torch.cuda.max_memory_allocated()
        m1 = torch.cuda.memory_allocated()
    finally:
        pw.pw_set_allocator()
    g_bytes = 16 * 2 * spec.p * 2 * 8
    assert peak - m0 > g_bytes   # the lanes' accumulators and the plans' tables were torch's
    assert m1 - m0 == 0          # and were all returned
    assert np.array_equal(got, want)
