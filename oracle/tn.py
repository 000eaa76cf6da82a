"""amp(C_t, i) = <i|U_t ... U_1|0^n> by plain variable elimination (oracle).

The circuit is turned into a tensor network as App. A describes: every qubit
carries a wire variable; an m-qubit gate is a tensor on its input and output
wires, except that on every qubit where the gate is diagonal its output leg is
identified with its input leg (no new variable). The first wire of every qubit
is fixed to 0 (the initial state) and the last one to the bit of i (or left
open). The amplitude is the sum over all free variables of the product of all
factors; it is evaluated here by eliminating one variable at a time (multiply
the factors that contain it, sum it out), smallest resulting factor first.
Any elimination order gives the same sum; this is the definition evaluated in
an order that keeps intermediate tables small.
"""
from __future__ import annotations

import string

import numpy as np

_LETTERS = string.ascii_letters


def _diag_on(T: np.ndarray, m: int, i: int) -> bool:
    """T has axes (out_0..out_{m-1}, in_0..in_{m-1}); diagonal on qubit i?"""
    idx_off = [slice(None)] * (2 * m)
    for a in range(2):
        idx = list(idx_off)
        idx[i] = a
        idx[m + i] = 1 - a
        if np.any(T[tuple(idx)] != 0):
            return False
    return True


def build_network(n: int, ops):
    """Variables and factors of the network for a gate list.

    Returns (factors, first_var, last_var): factors is a list of
    (var_tuple, table); first_var[q] / last_var[q] are the wire variables at
    the start and the end of qubit q.
    """
    nvar = 0
    cur = []
    for _ in range(n):
        cur.append(nvar)
        nvar += 1
    first = list(cur)
    factors = []
    for op in ops:
        assert op.kind == "gate"
        q = op.qubits
        m = len(q)
        U = op.mat
        # reorder to axes (out_0..out_{m-1}, in_0..in_{m-1}) with q_0 least significant
        T = U.reshape([2] * (2 * m))
        T = np.transpose(T, [m - 1 - i for i in range(m)] + [2 * m - 1 - i for i in range(m)])
        in_vars = [cur[qq] for qq in q]
        out_vars = []
        for i in range(m):
            if _diag_on(T, m, i):
                out_vars.append(in_vars[i])
            else:
                out_vars.append(nvar)
                nvar += 1
        all_vars = out_vars + in_vars
        uniq = []
        for v in all_vars:
            if v not in uniq:
                uniq.append(v)
        lt = {v: _LETTERS[k] for k, v in enumerate(uniq)}
        sub_in = "".join(lt[v] for v in all_vars)
        sub_out = "".join(lt[v] for v in uniq)
        table = np.einsum(f"{sub_in}->{sub_out}", T)
        factors.append((tuple(uniq), np.array(table)))
        for i in range(m):
            cur[q[i]] = out_vars[i]
    return factors, first, list(cur), nvar


def _slice(factors, fixed: dict):
    out = []
    for vars_, t in factors:
        idx = []
        keep = []
        for v in vars_:
            if v in fixed:
                idx.append(fixed[v])
            else:
                idx.append(slice(None))
                keep.append(v)
        out.append((tuple(keep), t[tuple(idx)]))
    return out


def contract(factors, open_vars):
    """Sum out every variable not in open_vars; return the table over open_vars."""
    factors = [(v, t) for v, t in factors]
    open_set = set(open_vars)
    while True:
        cand = {}
        for vars_, _ in factors:
            for v in vars_:
                if v not in open_set:
                    cand.setdefault(v, set()).update(vars_)
        if not cand:
            break
        best = min(cand, key=lambda v: (len(cand[v]) - 1, v))
        inv = [(vv, t) for vv, t in factors if best in vv]
        rest = [(vv, t) for vv, t in factors if best not in vv]
        uni = sorted(cand[best])
        lt = {v: _LETTERS[k] for k, v in enumerate(uni)}
        out_vars = tuple(v for v in uni if v != best)
        args = []
        for vv, t in inv:
            args.append(t)
            args.append([uni.index(v) for v in vv])
        res = np.einsum(*args, [uni.index(v) for v in out_vars])
        rest.append((out_vars, res))
        factors = rest
    # multiply what is left (tables over open variables and scalars), one
    # factor at a time
    k = len(open_vars)
    res = np.ones([2] * k, dtype=complex)
    for vv, t in factors:
        res = np.einsum(res, list(range(k)), t, [open_vars.index(v) for v in vv], list(range(k)))
    return res


def amplitudes(n: int, ops, bits, open_qubits=()):
    """<x|C|0^n> with x = ``bits`` on all qubits except ``open_qubits``.

    Returns an array with one axis per open qubit (axis i <-> open_qubits[i]),
    or a scalar when nothing is open.
    """
    factors, first, last, _ = build_network(n, ops)
    fixed = {}
    for q in range(n):
        fixed[first[q]] = 0
    open_vars = []
    for q in range(n):
        if q in open_qubits:
            continue
        v = last[q]
        if v in fixed and fixed[v] != int(bits[q]):
            # the wire never left the initial value yet x asks for the other one
            return np.zeros([2] * len(open_qubits), dtype=complex) if open_qubits else 0.0 + 0.0j
        fixed[v] = int(bits[q])
    for q in open_qubits:
        v = last[q]
        if v in fixed:
            raise ValueError("open qubit whose wire is fixed by the initial state")
        open_vars.append(v)
    fs = _slice(factors, fixed)
    res = contract(fs, open_vars)
    if open_qubits:
        return np.asarray(res, dtype=complex)
    return complex(res)
