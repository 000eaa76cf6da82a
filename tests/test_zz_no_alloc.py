"""pw_sample_static: sampling without any device allocation by the library.

Some callers cannot allocate device memory (their framework has reserved it
all for its own pool, or their sampling loop must not allocate); for them the
library keeps the kernel's scratch in one fixed device array. This checks,
through the C ABI, that two consecutive calls give exactly the bits and the
counters of pw_sample for the same plan and arguments (bit-exact, like the
other parity tests of integer outputs), and that an oversized plan is refused.
"""
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


def test_static_matches_pw_sample_on_two_calls(pw):
    import torch
    for spec, precision in ((W.grid_6x6_p2(), pw.PW_PREC_FP32), (W.random_qaoa(10, 2, seed=88, depol2=0.1,
                                                                                   ad_gamma=0.3), pw.PW_PREC_FP32),
                            (W.maxcut_3reg_n12(), pw.PW_PREC_FP64)):
        circ = pw.pw_circuit_qaoa(spec.n, spec.edges, spec.weights, spec.h, spec.p, spec.gammas, spec.betas,
                                  spec.depol2, spec.ad_gamma)
        plan = pw.pw_plan_build(circ, precision=precision)
        words = (spec.n + 63) // 64
        for seed, first, n in ((11, 0, 1000), (12, 777, 513)):
            ref = torch.zeros((n, words), dtype=torch.int64, device="cuda")
            got = torch.full((n, words), -1, dtype=torch.int64, device="cuda")
            st_ref = pw.pw_sample(plan, seed, first, n, ref)
            st_got = pw.pw_sample_static(plan, seed, first, n, got)
            torch.cuda.synchronize()
            assert torch.equal(ref, got)
            assert st_ref["near_boundary"] == st_got["near_boundary"]
            assert st_ref["zero_mass"] == st_got["zero_mass"]
        pw.pw_plan_destroy(plan)
        pw.pw_circuit_destroy(circ)


def test_static_rejects_plans_beyond_its_array(pw):
    import torch
    # a 2000-qubit chain plan: its tables exceed the 2 MiB array
    n = 2000
    edges = np.array([(i, i + 1) for i in range(n - 1)])
    circ = pw.pw_circuit_qaoa(n, edges, np.ones(n - 1), None, 2, [0.3, 0.5], [0.2, 0.4])
    plan = pw.pw_plan_build(circ)
    assert pw.pw_plan_stats(plan)["device_bytes"] > (2 << 20) - 256
    out = torch.zeros((4, (n + 63) // 64), dtype=torch.int64, device="cuda")
    with pytest.raises(pw.PwError) as e:
        pw.pw_sample_static(plan, 1, 0, 4, out)
    assert e.value.code == -8
    pw.pw_plan_destroy(plan)
    pw.pw_circuit_destroy(circ)
