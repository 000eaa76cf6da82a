"""torch.autograd binding of the QAOA amplitude derivatives.

``qaoa_amplitudes(gammas, betas, ...)`` returns amp(C, x) for the given
bitstrings as a float64 CUDA tensor [K, 2] (re, im); its backward pass applies
the exact derivatives of ``pw_qaoa_amp_grad`` (computed in the forward call)
to the incoming gradient. The angles are host (CPU) float64 tensors: they
parameterise the circuit the library plans.
"""
from __future__ import annotations

import numpy as np
import torch

from . import native as N


class _QaoaAmplitudes(torch.autograd.Function):
    @staticmethod
    def forward(ctx, gammas, betas, n, edges, weights, h, bits, precision):
        p = int(gammas.numel())
        amp = torch.empty((bits.shape[0], 2), dtype=torch.float64, device=bits.device)
        grad = torch.empty((bits.shape[0], 2 * p, 2), dtype=torch.float64, device=bits.device)
        N.pw_qaoa_amp_grad(n, edges, weights, h, p, gammas.detach().numpy(), betas.detach().numpy(), bits, grad,
                           amp_out=amp, precision=precision,
                           stream=torch.cuda.current_stream(bits.device).cuda_stream)
        ctx.save_for_backward(grad)
        ctx.p = p
        return amp

    @staticmethod
    def backward(ctx, g_amp):
        (grad,) = ctx.saved_tensors
        # a real loss L of amp = a + ib: dL/dtheta = sum_k (dL/da da/dtheta + dL/db db/dtheta)
        d = torch.einsum("kc,kjc->j", g_amp.to(torch.float64), grad).cpu()
        return d[:ctx.p], d[ctx.p:], None, None, None, None, None, None


def qaoa_amplitudes(gammas: torch.Tensor, betas: torch.Tensor, n: int, edges, weights, h, bits: torch.Tensor,
                    precision: int = N.PW_PREC_FP64) -> torch.Tensor:
    """Differentiable amplitudes of the noiseless QAOA circuit (App. D).

    gammas, betas: CPU float64 tensors [p]; edges/weights/h as for
    pw_circuit_qaoa (h may be None); bits: CUDA int64 [K, ceil(n/64)] packed
    bitstrings. Returns a CUDA float64 tensor [K, 2].
    """
    if gammas.device.type != "cpu" or betas.device.type != "cpu":
        raise ValueError("angles must be CPU tensors")
    return _QaoaAmplitudes.apply(gammas.to(torch.float64), betas.to(torch.float64), int(n),
                                 np.asarray(edges), np.asarray(weights, dtype=np.float64),
                                 None if h is None else np.asarray(h, dtype=np.float64), bits, int(precision))


class _CircuitAmplitudes(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, build, n, bits, precision):
        gates, param_of_op, dmats = build(theta.detach().numpy())
        circ = N.pw_circuit_create(n)
        try:
            for qubits, A in gates:
                N.pw_circuit_add_gate(circ, qubits, A)
            amp = torch.empty((bits.shape[0], 2), dtype=torch.float64, device=bits.device)
            grad = torch.empty((bits.shape[0], theta.numel(), 2), dtype=torch.float64, device=bits.device)
            N.pw_amp_grad(circ, theta.numel(), param_of_op, dmats, bits, grad, amp_out=amp, precision=precision,
                          stream=torch.cuda.current_stream(bits.device).cuda_stream)
        finally:
            N.pw_circuit_destroy(circ)
        ctx.save_for_backward(grad)
        return amp

    @staticmethod
    def backward(ctx, g_amp):
        (grad,) = ctx.saved_tensors
        return torch.einsum("kc,kjc->j", g_amp.to(torch.float64), grad).cpu(), None, None, None, None


def circuit_amplitudes(theta: torch.Tensor, build, n: int, bits: torch.Tensor,
                       precision: int = N.PW_PREC_FP64) -> torch.Tensor:
    """Differentiable amplitudes of a parameterised noiseless circuit.

    theta: CPU float64 tensor [P]; build(theta as numpy) returns (gates,
    param_of_op, dmats): the gate list as (qubits, matrix) pairs, the parameter
    index of every gate (-1 for none) and the derivative matrices of the
    parameterised gates in gate order (see pw_amp_grad). bits: CUDA int64
    [K, ceil(n/64)]. Returns a CUDA float64 tensor [K, 2] (re, im).
    """
    if theta.device.type != "cpu":
        raise ValueError("parameters must be a CPU tensor")
    return _CircuitAmplitudes.apply(theta.to(torch.float64), build, int(n), bits, int(precision))
