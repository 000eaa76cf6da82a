"""GPU: one dense pass of the sweep contraction (pw_dense_apply) against the
oracle. The pass applies a 2^k x 2^k operator to the k tile bits of every
tensor and then diagonal factors over other bit sets: on a tensor of 2^W
entries that is a k-qubit gate followed by diagonal gates in the oracle's
state-vector simulator (Sec. 2's gate application, ``oracle.statevector``).
Every arithmetic kind, both tile sizes, swizzled and plain storage, a ragged
number of 128-row tiles."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# relative error of every tensor, ||y - y_ref|| / ||y_ref||: FP32-level for the
# FP32 arm and the three-term split (24-bit inputs, products to 2^-24), about
# 2^-17 per input term for the two-term split, 2^-9 for plain BF16
FP32, BF16, SPLIT2, SPLIT3 = 3, 2, 1, 0   # PW_GEMM_* of include/pw.h
TOL = {FP32: 2e-6, SPLIT3: 2e-6, SPLIT2: 4e-5, BF16: 1.5e-2}


def _swz(i):
    return i ^ ((i >> 4) & 15)


def _case(k, swizzled, seed, n_t=5, extra=1):
    rng = np.random.default_rng(seed)
    W = k + 7 + extra
    tile = [int(b) for b in rng.permutation(W)[:k]]
    rest = [b for b in range(W) if b not in tile]
    row = rest[:7]
    diag_pos = [sorted(int(b) for b in rng.permutation(W)[:3]), [int(b) for b in rng.permutation(W)[:5]]]
    x = (rng.standard_normal((n_t, 1 << W)) + 1j * rng.standard_normal((n_t, 1 << W))) / np.sqrt(2)
    ops = (rng.standard_normal((n_t, 1 << k, 1 << k)) + 1j * rng.standard_normal((n_t, 1 << k, 1 << k))) / np.sqrt(2 << k)
    diag = np.exp(1j * rng.uniform(0, 2 * np.pi, (n_t, 2, 32))) * rng.uniform(0.5, 1.5, (n_t, 2, 32))
    return W, tile, row, diag_pos, x, ops, diag


def _reference(W, tile, diag_pos, x, op, diag):
    from oracle import statevector as SV
    y = SV.apply(x, W, tile, op)
    for d, bits in enumerate(diag_pos):
        y = SV.apply(y, W, bits, np.diag(diag[d][: 1 << len(bits)]))
    return y


@pytest.mark.parametrize("gemm", [FP32, SPLIT3, SPLIT2, BF16])
@pytest.mark.parametrize("k", [5, 6])
@pytest.mark.parametrize("swizzled", [0, 1])
def test_dense_pass_matches_the_oracle(gemm, k, swizzled):
    import torch
    import paper_2510_24218_gb300 as pw
    W, tile, row, diag_pos, x, ops, diag = _case(k, swizzled, seed=1000 * gemm + 10 * k + swizzled)
    n_t = x.shape[0]
    idx = np.arange(1 << W)
    phys = _swz(idx) if swizzled else idx
    stored = np.empty_like(x)
    stored[:, phys] = x
    d_x = torch.from_numpy(stored.astype(np.complex64)).cuda()
    d_op = torch.from_numpy(ops.astype(np.complex64)).cuda()
    d_dg = torch.from_numpy(diag.astype(np.complex64)).cuda()
    desc = pw.make_dense_desc(W, tile, row, swizzled, diag_pos)
    pw.pw_dense_apply(gemm, desc, n_t, d_x, d_op, d_dg)
    got = d_x.cpu().numpy().astype(np.complex128)[:, phys]
    # the oracle sees the FP32-rounded inputs (the rounding of the inputs is not the pass's error)
    x32 = x.astype(np.complex64).astype(np.complex128)
    o32 = ops.astype(np.complex64).astype(np.complex128)
    d32 = diag.astype(np.complex64).astype(np.complex128)
    for b in range(n_t):
        want = _reference(W, tile, diag_pos, x32[b], o32[b], d32[b])
        err = np.linalg.norm(got[b] - want) / np.linalg.norm(want)
        assert err < TOL[gemm], (gemm, k, swizzled, b, err)


@pytest.mark.parametrize("gemm", [FP32, SPLIT3])
def test_dense_pass_many_tiles_and_identity(gemm):
    """An identity operator with no diagonal leaves 131 tensors of 2^14
    entries as they are (to FP32 rounding of the split), over many tiles per
    CTA, so the operator changes between consecutive tiles of a CTA."""
    import torch
    import paper_2510_24218_gb300 as pw
    rng = np.random.default_rng(7)
    k, W, n_t = 6, 14, 131
    x = (rng.standard_normal((n_t, 1 << W)) + 1j * rng.standard_normal((n_t, 1 << W))).astype(np.complex64)
    ops = np.broadcast_to(np.eye(1 << k, dtype=np.complex64), (n_t, 1 << k, 1 << k)).copy()
    d_x = torch.from_numpy(x.copy()).cuda()
    d_op = torch.from_numpy(ops).cuda()
    desc = pw.make_dense_desc(W, [7, 8, 9, 10, 11, 12], [0, 1, 2, 3, 4, 5, 6], 0, [])
    pw.pw_dense_apply(gemm, desc, n_t, d_x, d_op, None)
    got = d_x.cpu().numpy()
    assert np.abs(got - x).max() <= 1e-7 * np.abs(x).max()


@pytest.mark.parametrize("gemm", [FP32, SPLIT3, BF16])
def test_dense_pass_any_bit_roles(gemm):
    """Row bits above the outer bits and tile bits among the swizzled low
    bits: positions combine the three parts by XOR, whatever bits they hold."""
    import torch
    import paper_2510_24218_gb300 as pw
    rng = np.random.default_rng(31 + gemm)
    k, W, n_t = 6, 17, 3
    tile = [3, 0, 9, 1, 8, 2]
    row = [10, 11, 12, 13, 14, 15, 16]
    diag_pos = [[4, 5, 0], [6, 7, 13, 9]]
    x = (rng.standard_normal((n_t, 1 << W)) + 1j * rng.standard_normal((n_t, 1 << W))) / np.sqrt(2)
    ops = (rng.standard_normal((n_t, 1 << k, 1 << k)) + 1j * rng.standard_normal((n_t, 1 << k, 1 << k))) / np.sqrt(2 << k)
    diag = np.exp(1j * rng.uniform(0, 2 * np.pi, (n_t, 2, 32)))
    phys = _swz(np.arange(1 << W))
    stored = np.empty_like(x)
    stored[:, phys] = x
    d_x = torch.from_numpy(stored.astype(np.complex64)).cuda()
    pw.pw_dense_apply(gemm, pw.make_dense_desc(W, tile, row, 1, diag_pos), n_t, d_x,
                      torch.from_numpy(ops.astype(np.complex64)).cuda(), torch.from_numpy(diag.astype(np.complex64)).cuda())
    got = d_x.cpu().numpy().astype(np.complex128)[:, phys]
    for b in range(n_t):
        want = _reference(W, tile, diag_pos, x[b].astype(np.complex64).astype(complex),
                          ops[b].astype(np.complex64).astype(complex), diag[b].astype(np.complex64).astype(complex))
        assert np.linalg.norm(got[b] - want) / np.linalg.norm(want) < TOL[gemm]
