"""The plan-shape search (pw_autotune): the tuned plan samples bit for bit
like Alg. 1 in its own sweep order, the result persists in the JSON-lines
cache and is returned from it without timing, pinned options stay fixed."""
import json

import numpy as np
import pytest

import workloads as W
from oracle import circuit as OC
from oracle import sampler as OS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_24218_gb300 as mod
    mod.load_library()
    return mod


def test_tuned_plan_samples_like_alg1_and_is_cached(pw, tmp_path):
    import torch
    spec = W.random_qaoa(12, 2, seed=21, with_h=True)
    circ = pw.pw_circuit_qaoa(spec.n, spec.edges, spec.weights, spec.h, spec.p, spec.gammas, spec.betas)
    cache = str(tmp_path / "tune.jsonl")
    opts, rate, hit = pw.pw_autotune(circ, 2048, cache)
    assert not hit and rate > 0
    lines = open(cache).read().splitlines()
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["max_block"] == opts["max_block"] and rec["threads_per_chain"] == opts["threads_per_chain"]
    assert rec["order"] == opts["order"] and rec["engine"] == opts["engine"]
    # from the cache: the same shape, no new line
    opts2, rate2, hit2 = pw.pw_autotune(circ, 2048, cache)
    assert hit2 and opts2 == opts and abs(rate2 - rate) <= 1e-5 * rate
    assert len(open(cache).read().splitlines()) == 1
    # the tuned plan against Alg. 1 in its own order
    plan = pw.pw_plan_build(circ, **opts)
    N = 48
    bits = torch.zeros((N, 1), dtype=torch.int64, device="cuda")
    st = pw.pw_sample(plan, 404, 0, N, bits)
    torch.cuda.synchronize()
    got = pw.unpack_bits(bits.cpu().numpy(), spec.n)
    order = pw.pw_plan_exec_order(plan)
    pw.pw_plan_destroy(plan)
    want, ost = OS.sample_sv(spec.n, OC.qaoa_circuit(spec), 404, list(range(N)), order=order)
    differ = int((~(want == got).all(axis=1)).sum())
    assert differ <= max(st["near_boundary"], ost.near_boundary)
    pw.pw_circuit_destroy(circ)


def test_pinned_options_stay(pw):
    spec = W.random_qaoa(12, 2, seed=22)
    circ = pw.pw_circuit_qaoa(spec.n, spec.edges, spec.weights, None, spec.p, spec.gammas, spec.betas)
    opts, rate, hit = pw.pw_autotune(circ, 1024, None, threads_per_chain=64, max_block=6,
                                     precision=pw.PW_PREC_FP64)
    assert not hit and rate > 0
    assert opts["threads_per_chain"] == 64 and opts["max_block"] == 6 and opts["precision"] == pw.PW_PREC_FP64
    assert opts["engine"] == pw.PW_ENGINE_AUTO   # (FP64 plans: no engine choice)
    pw.pw_circuit_destroy(circ)


def test_cache_keys_on_the_circuit(pw, tmp_path):
    """Two circuits that differ in one angle get two cache lines."""
    cache = str(tmp_path / "tune.jsonl")
    for gamma0 in (0.4, 0.41):
        spec = W.maxcut_3reg_n12()
        g = np.array(spec.gammas, dtype=float)
        g[0] = gamma0
        circ = pw.pw_circuit_qaoa(spec.n, spec.edges, spec.weights, None, spec.p, g, spec.betas)
        pw.pw_autotune(circ, 1024, cache, max_block=8, order=pw.PW_ORDER_NATURAL, threads_per_chain=32)
        pw.pw_circuit_destroy(circ)
    assert len(open(cache).read().splitlines()) == 2
