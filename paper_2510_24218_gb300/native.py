"""ctypes binding of ``include/pw.h`` (argument marshalling only).

Every function keeps the C name. Device buffers are torch CUDA tensors passed
by ``data_ptr()``; streams are torch streams (or None for the legacy default
stream). Errors raise ``PwError`` with the library's message.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

PW_PREC_FP32 = 0
PW_PREC_FP64 = 1
PW_ORDER_AUTO = 0
PW_ORDER_NATURAL = 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def library_path() -> str:
    return os.path.join(_HERE, "libpw.so")


class PwError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pw error {code}: {msg}")
        self.code = code


class PlanOpts(C.Structure):
    _fields_ = [("precision", C.c_int), ("order", C.c_int), ("max_block", C.c_int),
                ("threads_per_chain", C.c_int), ("chains_per_launch", C.c_int),
                ("ctas_per_chain", C.c_int), ("engine", C.c_int), ("gemm", C.c_int), ("reserved", C.c_int * 4)]


class PlanStats(C.Structure):
    _fields_ = [("n_qubits", C.c_int), ("n_ops", C.c_int), ("n_layers", C.c_int), ("n_slots", C.c_int),
                ("width_bits", C.c_int), ("width_low_bits", C.c_int), ("n_blocks", C.c_int),
                ("sampled_gates", C.c_int), ("threads_per_chain", C.c_int), ("chains_per_cta", C.c_int),
                ("smem_bytes_per_cta", C.c_int), ("noisy", C.c_int), ("flops_per_sample", C.c_double),
                ("amps_per_sample", C.c_double),
                ("device_bytes", C.c_double), ("ctas_per_chain", C.c_int), ("flops_per_amplitude", C.c_double),
                ("engine", C.c_int), ("gemm", C.c_int), ("dense_tile_bits", C.c_int),
                ("dense_passes_per_sample", C.c_double), ("dense_flops_per_sample", C.c_double)]


PW_GEMM_SPLIT3 = 0
PW_GEMM_SPLIT2 = 1
PW_GEMM_BF16 = 2
PW_GEMM_FP32 = 3
PW_ENGINE_AUTO = 0
PW_ENGINE_ONCHIP = 1
PW_ENGINE_HBM = 2


class DenseDesc(C.Structure):
    _fields_ = [("width_bits", C.c_int), ("tile_bits", C.c_int), ("tile_pos", C.c_int * 8), ("row_pos", C.c_int * 7),
                ("swizzled", C.c_int), ("n_diag", C.c_int), ("diag_bits", C.c_int * 4),
                ("diag_pos", (C.c_int * 5) * 4), ("reserved", C.c_int * 8)]


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_uint64, C.c_int, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p)
_ALLOCATOR_REFS = []   # the registered callbacks stay alive while registered


class RunStats(C.Structure):
    _fields_ = [("near_boundary", C.c_uint64), ("zero_mass", C.c_uint64), ("launches", C.c_uint64),
                ("dense_passes", C.c_uint64), ("dense_ms", C.c_double), ("dense_bytes", C.c_double),
                ("dense_flops", C.c_double)]


def load_library():
    """Load libpw.so (raises if it has not been built; there is no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    vp, ip, dp = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)
    sig = {
        "pw_circuit_create": (C.c_int, [C.c_int, C.POINTER(vp)]),
        "pw_circuit_add_gate": (C.c_int, [vp, C.c_int, ip, dp]),
        "pw_circuit_add_kraus": (C.c_int, [vp, C.c_int, ip, C.c_int, dp]),
        "pw_circuit_qaoa": (C.c_int, [C.c_int, C.c_int, ip, dp, dp, C.c_int, dp, dp, C.c_double, C.c_double,
                                      C.POINTER(vp)]),
        "pw_circuit_num_ops": (C.c_int, [vp, ip]),
        "pw_circuit_destroy": (None, [vp]),
        "pw_plan_build": (C.c_int, [vp, C.POINTER(PlanOpts), C.POINTER(vp)]),
        "pw_plan_stats": (C.c_int, [vp, C.POINTER(PlanStats)]),
        "pw_plan_exec_order": (C.c_int, [vp, ip]),
        "pw_plan_destroy": (None, [vp]),
        "pw_sample": (C.c_int, [vp, C.c_uint64, C.c_uint64, C.c_uint64, vp, vp, vp, C.POINTER(RunStats)]),
        "pw_plan_autotune": (C.c_int, [vp, C.c_uint64, vp, C.POINTER(C.c_int)]),
        "pw_autotune": (C.c_int, [vp, C.POINTER(PlanOpts), C.c_uint64, C.c_char_p, vp, C.POINTER(PlanOpts),
                                  dp, ip]),
        "pw_sample_host": (C.c_int, [vp, C.c_uint64, C.c_uint64, C.c_uint64, vp, vp, C.POINTER(RunStats)]),
        "pw_amplitudes": (C.c_int, [vp, C.c_int, C.c_uint64, vp, vp, vp]),
        "pw_qaoa_amp_grad": (C.c_int, [C.c_int, C.c_int, ip, dp, dp, C.c_int, dp, dp, C.POINTER(PlanOpts),
                                       C.c_uint64, vp, vp, vp, vp]),
        "pw_amp_grad": (C.c_int, [vp, C.c_int, ip, dp, C.POINTER(PlanOpts), C.c_uint64, vp, vp, vp, vp]),
        "pw_qaoa_cost_grad": (C.c_int, [C.c_int, C.c_int, ip, dp, dp, C.c_int, dp, dp, C.POINTER(PlanOpts),
                                        C.c_uint64, vp, vp, vp]),
        "pw_sample_static": (C.c_int, [vp, C.c_uint64, C.c_uint64, C.c_uint64, vp, vp, C.POINTER(RunStats)]),
        "pw_device_fma_rate": (C.c_int, [C.c_int, vp, dp]),
        "pw_set_allocator": (C.c_int, [_ALLOC_FN, _FREE_FN, vp]),
        "pw_dense_apply": (C.c_int, [C.c_int, C.POINTER(DenseDesc), C.c_uint64, vp, vp, vp, vp]),
        "pw_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def pw_last_error() -> str:
    return load_library().pw_last_error().decode()


def _check(rc: int):
    if rc != 0:
        raise PwError(rc, pw_last_error())


def _iarr(v):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.int32).ravel())
    return a, a.ctypes.data_as(C.POINTER(C.c_int))


def _darr(v):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.float64).ravel())
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _cplx(M):
    a = np.ascontiguousarray(np.asarray(M, dtype=np.complex128))
    return _darr(a.view(np.float64))


def _stream_ptr(stream):
    if stream is None:
        return None
    return C.c_void_p(int(getattr(stream, "cuda_stream", stream)))


# ------------------------------------------------------------------ circuit

def pw_circuit_create(n_qubits: int):
    h = C.c_void_p()
    _check(load_library().pw_circuit_create(int(n_qubits), C.byref(h)))
    return h


def pw_circuit_add_gate(circ, qubits, A):
    q, qp = _iarr(qubits)
    a, ap = _cplx(A)
    _check(load_library().pw_circuit_add_gate(circ, len(q), qp, ap))


def pw_circuit_add_kraus(circ, qubits, kraus_ops):
    q, qp = _iarr(qubits)
    a, ap = _cplx(np.stack([np.asarray(E, dtype=np.complex128) for E in kraus_ops]))
    _check(load_library().pw_circuit_add_kraus(circ, len(q), qp, len(kraus_ops), ap))


def pw_circuit_qaoa(n, edges, weights, h, p, gammas, betas, depol2=0.0, ad_gamma=0.0):
    e, ep = _iarr(edges)
    w, wp = _darr(weights)
    g, gp = _darr(gammas)
    b, bp = _darr(betas)
    if h is not None:
        hh, hp = _darr(h)
    else:
        hh, hp = None, None
    out = C.c_void_p()
    _check(load_library().pw_circuit_qaoa(int(n), len(e) // 2, ep, wp, hp, int(p), gp, bp, float(depol2),
                                          float(ad_gamma), C.byref(out)))
    return out


def pw_circuit_num_ops(circ) -> int:
    v = C.c_int()
    _check(load_library().pw_circuit_num_ops(circ, C.byref(v)))
    return v.value


def pw_circuit_destroy(circ):
    if circ:
        load_library().pw_circuit_destroy(circ)


# --------------------------------------------------------------------- plan

def pw_plan_build(circ, precision=PW_PREC_FP32, order=PW_ORDER_AUTO, max_block=0, threads_per_chain=0,
                  chains_per_launch=0, ctas_per_chain=0, engine=PW_ENGINE_AUTO, gemm=PW_GEMM_SPLIT3):
    o = PlanOpts()
    o.precision, o.order, o.max_block = precision, order, max_block
    o.threads_per_chain, o.chains_per_launch = threads_per_chain, chains_per_launch
    o.ctas_per_chain = ctas_per_chain
    o.engine, o.gemm = engine, gemm
    h = C.c_void_p()
    _check(load_library().pw_plan_build(circ, C.byref(o), C.byref(h)))
    return h


def pw_plan_stats(plan) -> dict:
    s = PlanStats()
    _check(load_library().pw_plan_stats(plan, C.byref(s)))
    return {name: getattr(s, name) for name, _ in PlanStats._fields_}


def pw_plan_exec_order(plan) -> np.ndarray:
    n = pw_plan_stats(plan)["n_ops"]
    a = np.zeros(n, dtype=np.int32)
    _check(load_library().pw_plan_exec_order(plan, a.ctypes.data_as(C.POINTER(C.c_int))))
    return a


def pw_plan_destroy(plan):
    if plan:
        load_library().pw_plan_destroy(plan)


# ---------------------------------------------------------------- execution

def pw_sample(plan, seed, first_sample, n_samples, out_bits, trace=None, stream=None, want_stats=True):
    """out_bits / trace: torch CUDA tensors (int64 [n, words], float64 [n, rows, 4])."""
    st = RunStats()
    _check(load_library().pw_sample(plan, int(seed), int(first_sample), int(n_samples),
                                    C.c_void_p(out_bits.data_ptr()),
                                    C.c_void_p(trace.data_ptr()) if trace is not None else None,
                                    _stream_ptr(stream), C.byref(st) if want_stats else None))
    return {"near_boundary": st.near_boundary, "zero_mass": st.zero_mass, "launches": st.launches,
            "dense_passes": st.dense_passes, "dense_ms": st.dense_ms, "dense_bytes": st.dense_bytes,
            "dense_flops": st.dense_flops}


def pw_plan_autotune(plan, trial_samples=0, stream=None) -> int:
    """Time every threads-per-chain value on this device and keep the fastest
    in the plan; returns it."""
    chosen = C.c_int(0)
    _check(load_library().pw_plan_autotune(plan, int(trial_samples), _stream_ptr(stream), C.byref(chosen)))
    return chosen.value


def pw_autotune(circ, trial_samples=0, cache_path=None, stream=None, **base):
    """Search the plan options that change only the schedule (engine,
    max_block, order, threads_per_chain, chains_per_launch) for circuit
    `circ`; keyword arguments are pw_plan_build's options (nonzero ones stay
    fixed). Returns (options dict for pw_plan_build, samples/s, from_cache)."""
    b = PlanOpts()
    for name, v in base.items():
        setattr(b, name, v)
    o = PlanOpts()
    rate = C.c_double(0.0)
    hit = C.c_int(0)
    _check(load_library().pw_autotune(circ, C.byref(b), int(trial_samples),
                                      cache_path.encode() if cache_path else None, _stream_ptr(stream),
                                      C.byref(o), C.byref(rate), C.byref(hit)))
    opts = {name: getattr(o, name) for name, _ in PlanOpts._fields_ if name != "reserved"}
    return opts, rate.value, bool(hit.value)


def pw_sample_static(plan, seed, first_sample, n_samples, out_bits, stream=None, want_stats=True):
    """Allocation-free sampling: out_bits is a torch CUDA int64 [n, words] tensor."""
    st = RunStats()
    _check(load_library().pw_sample_static(plan, int(seed), int(first_sample), int(n_samples),
                                           C.c_void_p(out_bits.data_ptr()), _stream_ptr(stream),
                                           C.byref(st) if want_stats else None))
    return {"near_boundary": st.near_boundary, "zero_mass": st.zero_mass, "launches": st.launches}


def pw_device_fma_rate(precision=PW_PREC_FP32, stream=None) -> float:
    """Measured FP32 or FP64 FMA rate of the current device's CUDA cores, TFLOP/s."""
    r = C.c_double(0.0)
    _check(load_library().pw_device_fma_rate(int(precision), _stream_ptr(stream), C.byref(r)))
    return r.value


def make_dense_desc(width_bits, tile_pos, row_pos, swizzled=0, diag_pos=()):
    """pw_dense_desc from bit lists (diag_pos: one list of bits per factor)."""
    d = DenseDesc()
    d.width_bits = int(width_bits)
    d.tile_bits = len(tile_pos)
    for j, b in enumerate(tile_pos):
        d.tile_pos[j] = int(b)
    for j, b in enumerate(row_pos):
        d.row_pos[j] = int(b)
    d.swizzled = int(swizzled)
    d.n_diag = len(diag_pos)
    for i, bits in enumerate(diag_pos):
        d.diag_bits[i] = len(bits)
        for j, b in enumerate(bits):
            d.diag_pos[i][j] = int(b)
    return d


def pw_dense_apply(gemm, desc, n_tensors, tensors, ops, diag=None, stream=None):
    """tensors: torch CUDA complex64 [n, 2^W] (in place); ops: complex64 [n, 2^k, 2^k];
    diag: complex64 [n, n_diag, 32] or None."""
    _check(load_library().pw_dense_apply(int(gemm), C.byref(desc), int(n_tensors),
                                         C.c_void_p(tensors.data_ptr()) if tensors is not None else None,
                                         C.c_void_p(ops.data_ptr()) if ops is not None else None,
                                         C.c_void_p(diag.data_ptr()) if diag is not None else None,
                                         _stream_ptr(stream)))


def pw_set_allocator(alloc=None, free=None):
    """Register Python callables alloc(bytes, device) -> int pointer (0 for
    failure) and free(ptr, device) for the library's internal device buffers;
    no arguments restores cudaMalloc / cudaFree."""
    lib = load_library()
    if alloc is None and free is None:
        _check(lib.pw_set_allocator(_ALLOC_FN(), _FREE_FN(), None))
        _ALLOCATOR_REFS.clear()
        return

    def _a(nbytes, device, stream, ctx):
        try:
            return int(alloc(int(nbytes), int(device))) or None
        except Exception:   # (an exception cannot cross the C ABI: report no memory)
            return None

    def _f(ptr, device, stream, ctx):
        try:
            free(int(ptr), int(device))
        except Exception:
            pass

    fa, ff = _ALLOC_FN(_a), _FREE_FN(_f)
    _check(lib.pw_set_allocator(fa, ff, None))
    _ALLOCATOR_REFS[:] = [fa, ff]


def use_torch_allocator():
    """Route the library's internal device buffers through torch's caching
    allocator (torch.cuda.memory_allocated() then accounts for them)."""
    import torch

    def alloc(nbytes, device):
        return torch.cuda.caching_allocator_alloc(nbytes, device=device)

    def free(ptr, device):
        torch.cuda.caching_allocator_delete(ptr)

    pw_set_allocator(alloc, free)


def pw_sample_host(plan, seed, first_sample, n_samples, out_bits: np.ndarray, trace: np.ndarray | None = None):
    """Host-buffer variant: out_bits uint64 [n, words], trace float64 [n, rows, 4] or None."""
    assert out_bits.dtype == np.uint64 and out_bits.flags["C_CONTIGUOUS"]
    st = RunStats()
    _check(load_library().pw_sample_host(plan, int(seed), int(first_sample), int(n_samples),
                                         C.c_void_p(out_bits.ctypes.data),
                                         C.c_void_p(trace.ctypes.data) if trace is not None else None,
                                         C.byref(st)))
    return {"near_boundary": st.near_boundary, "zero_mass": st.zero_mass, "launches": st.launches}


def pw_amplitudes(plan, prefix_ops, bits, amp_out, stream=None):
    """bits: torch CUDA int64 [n_strings, words]; amp_out: torch CUDA float64 [n_strings, 2]."""
    _check(load_library().pw_amplitudes(plan, int(prefix_ops), int(bits.shape[0]), C.c_void_p(bits.data_ptr()),
                                        C.c_void_p(amp_out.data_ptr()), _stream_ptr(stream)))


def pw_qaoa_amp_grad(n, edges, weights, h, p, gammas, betas, bits, grad_out, amp_out=None, precision=PW_PREC_FP32,
                     order=PW_ORDER_AUTO, stream=None):
    """Exact d amp / d (gammas, betas) of the noiseless QAOA circuit.

    bits: torch CUDA int64 [n_strings, words]; grad_out: torch CUDA float64
    [n_strings, 2p, 2] (gammas first); amp_out: None or float64 [n_strings, 2].
    """
    e, ep = _iarr(edges)
    w, wp = _darr(weights)
    g, gp = _darr(gammas)
    b, bp = _darr(betas)
    hh, hp = _darr(h) if h is not None else (None, None)
    o = PlanOpts()
    o.precision, o.order = precision, order
    _check(load_library().pw_qaoa_amp_grad(int(n), len(e) // 2, ep, wp, hp, int(p), gp, bp, C.byref(o),
                                           int(bits.shape[0]), C.c_void_p(bits.data_ptr()),
                                           C.c_void_p(amp_out.data_ptr()) if amp_out is not None else None,
                                           C.c_void_p(grad_out.data_ptr()), _stream_ptr(stream)))


def pw_amp_grad(circ, n_params, param_of_op, dmats, bits, grad_out, amp_out=None, precision=PW_PREC_FP32,
                order=PW_ORDER_AUTO, stream=None):
    """Exact d amp / d theta of a parameterised circuit (product rule).

    param_of_op: int [n_ops] (-1 = no parameter); dmats: the derivative matrices
    of the parameterised operations in operation order (a list of 2^m x 2^m
    complex arrays); bits: torch CUDA int64 [n_strings, words]; grad_out: torch
    CUDA float64 [n_strings, n_params, 2]; amp_out: None or float64 [n_strings, 2].
    """
    q, qp = _iarr(param_of_op)
    flat = [np.asarray(D, dtype=np.complex128).ravel() for D in dmats]
    if flat:
        d, dp_ = _cplx(np.concatenate(flat))
    else:
        d, dp_ = None, None
    o = PlanOpts()
    o.precision, o.order = precision, order
    _check(load_library().pw_amp_grad(circ, int(n_params), qp, dp_, C.byref(o), int(bits.shape[0]),
                                      C.c_void_p(bits.data_ptr()),
                                      C.c_void_p(amp_out.data_ptr()) if amp_out is not None else None,
                                      C.c_void_p(grad_out.data_ptr()), _stream_ptr(stream)))


def pw_qaoa_cost_grad(n, edges, weights, h, p, gammas, betas, bits, out, precision=PW_PREC_FP32, order=PW_ORDER_AUTO,
                      stream=None):
    """Score-function estimate of d E[C] / d (gammas, betas) from sampled bits.

    bits: torch CUDA int64 [n_samples, words]; out: torch CUDA float64 [1 + 2p]
    (mean cost, then the gammas' and the betas' derivatives).
    """
    e, ep = _iarr(edges)
    w, wp = _darr(weights)
    g, gp = _darr(gammas)
    b, bp = _darr(betas)
    hh, hp = _darr(h) if h is not None else (None, None)
    o = PlanOpts()
    o.precision, o.order = precision, order
    _check(load_library().pw_qaoa_cost_grad(int(n), len(e) // 2, ep, wp, hp, int(p), gp, bp, C.byref(o),
                                            int(bits.shape[0]), C.c_void_p(bits.data_ptr()),
                                            C.c_void_p(out.data_ptr()), _stream_ptr(stream)))


# ------------------------------------------------------------ bit packing

def pack_bits(bits: np.ndarray) -> np.ndarray:
    """uint8 [count, n] -> uint64 [count, ceil(n/64)], qubit q at bit q%64 of word q//64."""
    bits = np.asarray(bits, dtype=np.uint64)
    count, n = bits.shape
    words = (n + 63) // 64
    out = np.zeros((count, words), dtype=np.uint64)
    for q in range(n):
        out[:, q // 64] |= bits[:, q] << np.uint64(q % 64)
    return out


def unpack_bits(words: np.ndarray, n: int) -> np.ndarray:
    """Inverse of pack_bits (accepts int64 or uint64 words)."""
    w = np.asarray(words).view(np.uint64) if np.asarray(words).dtype == np.int64 else np.asarray(words, np.uint64)
    out = np.zeros((w.shape[0], n), dtype=np.uint8)
    for q in range(n):
        out[:, q] = ((w[:, q // 64] >> np.uint64(q % 64)) & np.uint64(1)).astype(np.uint8)
    return out
