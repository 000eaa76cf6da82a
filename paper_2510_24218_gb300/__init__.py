"""GB300-native pilot-wave exact sampler (arXiv 2510.24218).

The compute path is the C-ABI library ``libpw.so`` (CUDA for sm_103a plus the
C++ planner); this package only marshals arguments to it. Importing the
package fails loudly when the library has not been built: there is no CPU
fallback.
"""
from .native import (PwError, pw_amp_grad, pw_amplitudes, pw_device_fma_rate, pw_dense_apply, make_dense_desc,
                     pw_set_allocator, use_torch_allocator,
                     PW_GEMM_FP32, PW_GEMM_BF16, PW_GEMM_SPLIT2, PW_GEMM_SPLIT3, PW_ENGINE_AUTO, PW_ENGINE_ONCHIP, PW_ENGINE_HBM, pw_circuit_add_gate, pw_circuit_add_kraus,  # noqa: F401
                     pw_circuit_create, pw_circuit_destroy, pw_circuit_num_ops, pw_circuit_qaoa,
                     pw_last_error, pw_autotune, pw_plan_autotune, pw_plan_build, pw_plan_destroy, pw_plan_exec_order, pw_plan_stats,
                     pw_qaoa_amp_grad, pw_qaoa_cost_grad, pw_sample, pw_sample_host, pw_sample_static, library_path, load_library, pack_bits, unpack_bits,
                     PW_PREC_FP32, PW_PREC_FP64, PW_ORDER_AUTO, PW_ORDER_NATURAL)

__all__ = [n for n in dir() if n.startswith("pw_") or n.startswith("PW_")] + [
    "PwError", "library_path", "load_library", "pack_bits", "unpack_bits", "make_dense_desc", "use_torch_allocator"]
