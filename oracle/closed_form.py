"""Closed-form p=1 QAOA correlators (oracle pin for large n).

For |psi> = exp(-i beta sum_j X_j) exp(-i gamma sum_e w_e Z_u Z_v) |+>^n
(App. D with h = 0), conjugating Z_u Z_v by the mixer gives
c^2 Z_uZ_v + c s (Z_u Y_v + Y_u Z_v) + s^2 Y_u Y_v with c = cos 2beta,
s = sin 2beta. Averaging each term over the phase state gives

  <Z_u Z_v> = 1/2 sin(4 beta) sin(2 gamma w_uv)
                  [prod_{k in N(u)\\v} cos(2 gamma w_uk) + prod_{k in N(v)\\u} cos(2 gamma w_vk)]
            + 1/2 sin^2(2 beta) [prod_k cos(2 gamma (w_uk - w_vk)) - prod_k cos(2 gamma (w_uk + w_vk))]

where the last products run over k not in {u, v} with w = 0 on non-edges.
A test checks it against the dense state vector before it is used as a pin
at large n.
"""
from __future__ import annotations

import math

import numpy as np


def zz_p1(n, edges, weights, gamma, beta, pairs=None):
    """<Z_u Z_v> for every pair in ``pairs`` (default: the edges)."""
    W = {}
    nbr = [dict() for _ in range(n)]
    for (u, v), w in zip(edges, weights):
        u, v = int(u), int(v)
        nbr[u][v] = nbr[u].get(v, 0.0) + float(w)
        nbr[v][u] = nbr[v].get(u, 0.0) + float(w)
    if pairs is None:
        pairs = [(int(u), int(v)) for u, v in edges]
    s4, s2sq = math.sin(4 * beta), math.sin(2 * beta) ** 2
    out = []
    for u, v in pairs:
        wuv = nbr[u].get(v, 0.0)
        pu = math.prod(math.cos(2 * gamma * w) for k, w in nbr[u].items() if k != v)
        pv = math.prod(math.cos(2 * gamma * w) for k, w in nbr[v].items() if k != u)
        ks = (set(nbr[u]) | set(nbr[v])) - {u, v}
        pm = math.prod(math.cos(2 * gamma * (nbr[u].get(k, 0.0) - nbr[v].get(k, 0.0))) for k in ks)
        pp = math.prod(math.cos(2 * gamma * (nbr[u].get(k, 0.0) + nbr[v].get(k, 0.0))) for k in ks)
        out.append(0.5 * s4 * math.sin(2 * gamma * wuv) * (pu + pv) + 0.5 * s2sq * (pm - pp))
    return np.array(out)
