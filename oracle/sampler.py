"""The pilot-wave Markov chain, written out as the paper states it (oracle).

Alg. 1 (Sec. 2): Sample(C) starts from s = 0^n and applies UpdateState after
every gate. A monomial gate (permutation times diagonal) moves s
deterministically to sigma(s); any other gate restricts the move to the block
of s given by BlockDecompose and draws the new state inside it with
probability |amp(C_t, y)|^2 / sum_block |amp|^2 (zero-mass block: stay).

Alg. 2 (App. A): NoisySample keeps a frame x of pending X gates. A unitary gate
G is conjugated by X on every qubit with x[q] = 1 (PropagateX), appended to the
simulated circuit C'' and followed by UpdateState when non-diagonal. A noise
operation draws its Kraus index from Eq. (5), factorises the drawn operator into
single-qubit factors, turns each anti-diagonal factor M into the diagonal
M sigma_X while flipping x[q], and appends the (frame-conjugated) diagonal
factor. The sample is s XOR x.

Readings of points the paper leaves open:
* randomness: u = Philox4x32-10(key=seed, ctr=(sample, op_id, purpose)) mapped
  to a 53-bit double; UpdateState takes the smallest candidate y (ascending
  local index) with u * P < sum_{y' <= y} p_{y'}; the Kraus draw uses the same
  rule over the Kraus list order;
* Eq. (5) is evaluated at the true bit c = s[q] XOR x[q];
* operation ids are positions in the input circuit; the execution order may
  permute commuting gates (a list of (op_id, op) pairs is accepted).
"""
from __future__ import annotations

import numpy as np

from . import circuit as C
from . import statevector as SV
from . import tn as TN
from .philox import PURPOSE_KRAUS, PURPOSE_UPDATE, draw

NEAR_BOUNDARY = 1e-6


class Stats:
    def __init__(self):
        self.near_boundary = 0
        self.zero_mass = 0
        self.amp_calls = 0
        self.updates = 0


def _choose(probs, u):
    """Smallest index i with u * P < cumulative sum up to i; None if P == 0."""
    P = float(sum(probs))
    if P == 0.0:
        return None, False
    cum = 0.0
    pick = len(probs) - 1
    for i, p in enumerate(probs):
        cum += p
        if u * P < cum:
            pick = i
            break
    near = False
    cum = 0.0
    for p in probs[:-1]:
        cum += p
        if abs(u * P - cum) < NEAR_BOUNDARY * P:
            near = True
    return pick, near


def update_state(A, qubits, s, amp_fn, u_fn, stats: Stats, trace=None):
    """UpdateState (Alg. 1) for the last gate (A, qubits) of the prefix.

    amp_fn(list_of_bitstrings) -> complex amplitudes of the prefix circuit;
    u_fn() -> the uniform for this step (called only when a draw is needed).
    """
    x = C.local_index(s, qubits)
    if C.is_monomial(A):
        return C.set_local(s, qubits, C.monomial_image(A, x))
    block = C.block_decompose_local(A, x)
    if len(block) == 1:
        return C.set_local(s, qubits, block[0])
    cands = [C.set_local(s, qubits, y) for y in block]
    amps = amp_fn(cands)
    stats.amp_calls += len(cands)
    stats.updates += 1
    probs = [abs(a) ** 2 for a in amps]
    u = u_fn()
    pick, near = _choose(probs, u)
    if trace is not None:
        trace.append((tuple(block), [complex(a) for a in amps], u))
    if near:
        stats.near_boundary += 1
    if pick is None:
        stats.zero_mass += 1
        return s
    return cands[pick]


def _ordered(ops, order):
    if order is None:
        return list(enumerate(ops))
    return [(int(i), ops[int(i)]) for i in order]


# ---------------------------------------------------------------------------
# Alg. 1 with dense state-vector amplitudes: chains advance gate by gate in
# lockstep so that psi_t is computed once per gate for all of them.
# ---------------------------------------------------------------------------

def sample_sv(n, ops, seed, sample_ids, order=None, stats=None, traces=None):
    """Sample(C) for every id in ``sample_ids`` (ideal circuit, n small)."""
    stats = stats or Stats()
    seq = _ordered(ops, order)
    S = [np.zeros(n, dtype=np.uint8) for _ in sample_ids]
    psi = SV.zero_state(n)
    for op_id, op in seq:
        assert op.kind == "gate"
        psi = SV.apply(psi, n, op.qubits, op.mat)
        for k, sid in enumerate(sample_ids):
            def amp_fn(cands, psi=psi):
                return [psi[sum(int(b) << q for q, b in enumerate(c))] for c in cands]
            u_fn = (lambda sid=sid, op_id=op_id: draw(seed, sid, op_id, PURPOSE_UPDATE))
            tr = traces[k] if traces is not None else None
            S[k] = update_state(op.mat, op.qubits, S[k], amp_fn, u_fn, stats, tr)
    return np.array(S, dtype=np.uint8), stats


def sample_tn(n, ops, seed, sample_id, order=None, stats=None, trace=None, follow=None):
    """Sample(C) for one chain with amplitudes from variable elimination.

    Both candidates of a gate are obtained from one contraction with the
    target qubit's final wire left open. ``follow`` (optional list of
    bitstrings, one per sampling step) replaces the drawn state by the given
    one after each step, so that the oracle can check another sampler's
    amplitudes along that sampler's own path.
    """
    stats = stats or Stats()
    seq = _ordered(ops, order)
    s = np.zeros(n, dtype=np.uint8)
    prefix = []
    step = 0
    for op_id, op in seq:
        assert op.kind == "gate"
        prefix.append(op)

        def amp_fn(cands, qubits=op.qubits, pre=list(prefix)):
            if len(qubits) == 1:
                t = TN.amplitudes(n, pre, cands[0], open_qubits=(qubits[0],))
                out = []
                for c in cands:
                    out.append(t[int(c[qubits[0]])])
                return out
            return [TN.amplitudes(n, pre, c) for c in cands]

        u_fn = (lambda op_id=op_id: draw(seed, sample_id, op_id, PURPOSE_UPDATE))
        before = stats.updates
        s = update_state(op.mat, op.qubits, s, amp_fn, u_fn, stats, trace)
        if follow is not None and stats.updates > before:
            s = np.array(follow[step], dtype=np.uint8)
            step += 1
    return s, stats


# ---------------------------------------------------------------------------
# Alg. 2 (NoisySample) with the simulated circuit C'' kept as a state vector
# ---------------------------------------------------------------------------

def propagate_x(x, qubits, G):
    """PropagateX: G <- X_q G X_q for every qubit q of G with x[q] = 1."""
    m = len(qubits)
    out = np.array(G, copy=True)
    for i, q in enumerate(qubits):
        if x[q]:
            P = np.zeros((1 << m, 1 << m))
            for a in range(1 << m):
                P[a ^ (1 << i), a] = 1
            out = P @ out @ P
    return out


class _SVCircuit:
    """C'' as a gate list together with its (unnormalised) state C''|0^n>."""

    def __init__(self, n):
        self.n = n
        self.gates = []
        self.psi = SV.zero_state(n)

    def add(self, qubits, G):
        self.gates.append(C.gate(qubits, G))
        self.psi = SV.apply(self.psi, self.n, qubits, G)

    def amps(self, cands):
        return [self.psi[sum(int(b) << q for q, b in enumerate(c))] for c in cands]


class _TNCircuit(_SVCircuit):
    """C'' as a gate list, amplitudes by variable elimination (larger n)."""

    def __init__(self, n):
        self.n = n
        self.gates = []

    def add(self, qubits, G):
        self.gates.append(C.gate(qubits, G))

    def amps(self, cands):
        qubits = self._last_qubits
        if len(qubits) == 1:
            t = TN.amplitudes(self.n, self.gates, cands[0], open_qubits=(qubits[0],))
            return [t[int(c[qubits[0]])] for c in cands]
        return [TN.amplitudes(self.n, self.gates, c) for c in cands]


def noisy_sample(n, ops, seed, sample_id, order=None, backend="sv", stats=None, trace=None,
                 events=None):
    """NoisySample (Alg. 2) for one chain; returns s XOR x."""
    stats = stats or Stats()
    seq = _ordered(ops, order)
    Cpp = _SVCircuit(n) if backend == "sv" else _TNCircuit(n)
    s = np.zeros(n, dtype=np.uint8)
    x = np.zeros(n, dtype=np.uint8)

    def add_gate(qubits, G, op_id):
        nonlocal s
        G2 = propagate_x(x, qubits, G)
        Cpp.add(qubits, G2)
        Cpp._last_qubits = qubits
        if not C.is_diagonal(G2):
            u_fn = (lambda: draw(seed, sample_id, op_id, PURPOSE_UPDATE))
            s = update_state(G2, qubits, s, Cpp.amps, u_fn, stats, trace)

    for op_id, op in seq:
        if op.kind == "gate":
            add_gate(op.qubits, op.mat, op_id)
            continue
        c = C.local_index(s ^ x, op.qubits)               # true bits (Eq. 5 reading)
        probs = [float(np.sum(np.abs(E[:, c]) ** 2)) for E in op.mats]
        u = draw(seed, sample_id, op_id, PURPOSE_KRAUS)
        i, _ = _choose(probs, u)
        if events is not None:
            events.append((op_id, i))
        E = op.mats[i]
        for M, q in C.lsm_factorize(E, op.qubits):
            MX = M @ C.SIGMA_X
            if C.is_diagonal(MX) and not C.is_diagonal(M):
                x[q] ^= 1
                M = MX
            add_gate((q,), M, op_id)
    return s ^ x, stats


# ---------------------------------------------------------------------------
# Exact output distribution of the chains (tiny circuits; pins Eq. 1)
# ---------------------------------------------------------------------------

def transition_kernel(n, A, qubits, psi_t):
    """Row-stochastic matrix P[x, y] = p_t(x -> y) of UpdateState for gate (A, q)."""
    dim = 1 << n
    P = np.zeros((dim, dim))
    for xg in range(dim):
        bits = [(xg >> q) & 1 for q in range(n)]
        xl = C.local_index(bits, qubits)
        if C.is_monomial(A):
            y = C.set_local(bits, qubits, C.monomial_image(A, xl))
            P[xg, sum(int(b) << q for q, b in enumerate(y))] = 1.0
            continue
        block = C.block_decompose_local(A, xl)
        ys = [sum(int(b) << q for q, b in enumerate(C.set_local(bits, qubits, yl))) for yl in block]
        w = np.array([abs(psi_t[y]) ** 2 for y in ys])
        if w.sum() == 0.0:
            P[xg, xg] = 1.0
        else:
            P[xg, ys] = w / w.sum()
    return P


def exact_chain_distributions(n, ops):
    """Distribution of s_t for t = 0..T obtained by applying the kernels of
    UpdateState one after another, next to |psi_t|^2 for every t."""
    dim = 1 << n
    p = np.zeros(dim)
    p[0] = 1.0
    psi = SV.zero_state(n)
    chain, exact = [p.copy()], [np.abs(psi) ** 2]
    for op in ops:
        psi = SV.apply(psi, n, op.qubits, op.mat)
        p = p @ transition_kernel(n, op.mat, op.qubits, psi)
        chain.append(p.copy())
        exact.append(np.abs(psi) ** 2)
    return chain, exact


def exact_noisy_distribution(n, ops, kraus_rule="true_bit"):
    """Exact output distribution of Alg. 2 by following every branch.

    Each UpdateState branch y has probability p_y / P and each Kraus branch i
    has probability from Eq. (5). ``kraus_rule`` = "true_bit" evaluates Eq. (5)
    at s XOR x (the reading used here); "s_only" evaluates it at s (the other
    reading, kept so a test can show that it disagrees with the density matrix).
    """
    out = np.zeros(1 << n)

    def rec(k, s, x, psi, weight):
        if weight == 0.0:
            return
        if k == len(ops):
            y = s ^ x
            out[sum(int(b) << q for q, b in enumerate(y))] += weight
            return
        op = ops[k]
        if op.kind == "gate":
            for s2, x2, psi2, w2 in _branches_gate(op.qubits, op.mat, s, x, psi):
                rec(k + 1, s2, x2, psi2, weight * w2)
            return
        bits = s ^ x if kraus_rule == "true_bit" else s
        c = C.local_index(bits, op.qubits)
        for E in op.mats:
            pr = float(np.sum(np.abs(E[:, c]) ** 2))
            if pr == 0.0:
                continue
            branches = [(s, x.copy(), psi, 1.0)]
            for M, q in C.lsm_factorize(E, op.qubits):
                nb = []
                for s1, x1, psi1, w1 in branches:
                    x1 = x1.copy()
                    MX = M @ C.SIGMA_X
                    Mq = M
                    if C.is_diagonal(MX) and not C.is_diagonal(M):
                        x1[q] ^= 1
                        Mq = MX
                    for b in _branches_gate((q,), Mq, s1, x1, psi1):
                        nb.append((b[0], b[1], b[2], w1 * b[3]))
                branches = nb
            for s2, x2, psi2, w2 in branches:
                rec(k + 1, s2, x2, psi2, weight * pr * w2)

    def _branches_gate(qubits, G, s, x, psi):
        G2 = propagate_x(x, qubits, G)
        psi2 = SV.apply(psi, n, qubits, G2)
        if C.is_diagonal(G2):
            return [(s, x, psi2, 1.0)]
        xl = C.local_index(s, qubits)
        if C.is_monomial(G2):
            return [(C.set_local(s, qubits, C.monomial_image(G2, xl)), x, psi2, 1.0)]
        block = C.block_decompose_local(G2, xl)
        cands = [C.set_local(s, qubits, y) for y in block]
        w = np.array([abs(psi2[sum(int(b) << q for q, b in enumerate(c))]) ** 2 for c in cands])
        if w.sum() == 0.0:
            return [(s, x, psi2, 1.0)]
        return [(c, x, psi2, float(wi / w.sum())) for c, wi in zip(cands, w) if wi > 0]

    rec(0, np.zeros(n, dtype=np.uint8), np.zeros(n, dtype=np.uint8), SV.zero_state(n), 1.0)
    return out
