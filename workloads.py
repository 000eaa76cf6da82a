"""Seeded synthetic inputs shared by the oracle tests and the GPU path.

This module only draws graphs, weights, angles and noise strengths. It holds
none of the sampler's arithmetic: no gate matrices, no amplitudes, no random
numbers that the sampler itself consumes (those come from the counter-based
generator that each side implements on its own).

Workload shapes follow the paper's QAOA experiments (App. D: an H layer, then
p cost layers of RZZ gates and p mixer layers of RX gates on Ising/MaxCut
graphs; Sec. 4.3: grid, heavy-hex and random 3-regular topologies). The
paper's own instances, seeds and transferred angles are not available, so
every instance here is drawn from a fixed seed with numpy's PCG64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class QaoaSpec:
    """A QAOA instance: graph, weights, fields, angles and an optional noise model.

    Gate order convention shared by both implementations: H on qubits 0..n-1;
    then for each layer l: one RZZ(2*gamma_l*w_e) per edge in list order
    (each followed by a two-qubit depolarizing channel when depol2 > 0),
    one RZ(2*gamma_l*h_j) per qubit when h is given, one RX(2*beta_l) per
    qubit 0..n-1, then one amplitude-damping channel per qubit 0..n-1 when
    ad_gamma > 0.
    """
    n: int
    edges: np.ndarray          # int64 [E, 2], u < v
    weights: np.ndarray        # float64 [E]
    gammas: np.ndarray         # float64 [p]
    betas: np.ndarray          # float64 [p]
    h: np.ndarray | None = None
    depol2: float = 0.0
    ad_gamma: float = 0.0
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def p(self) -> int:
        return int(len(self.gammas))


def grid_edges(rows: int, cols: int) -> np.ndarray:
    """Square-lattice edges, qubits numbered row-major, pairs sorted."""
    e = []
    for r in range(rows):
        for c in range(cols):
            q = r * cols + c
            if c + 1 < cols:
                e.append((q, q + 1))
            if r + 1 < rows:
                e.append((q, q + cols))
    return np.array(sorted(e), dtype=np.int64).reshape(-1, 2)


def kings_edges(rows: int, cols: int) -> np.ndarray:
    """King's-graph edges (the square lattice plus both diagonals of every
    plaquette), qubits numbered row-major, pairs sorted."""
    e = []
    for r in range(rows):
        for c in range(cols):
            q = r * cols + c
            for dr, dc in ((0, 1), (1, -1), (1, 0), (1, 1)):
                rr, cc = r + dr, c + dc
                if 0 <= rr < rows and 0 <= cc < cols:
                    e.append(tuple(sorted((q, rr * cols + cc))))
    return np.array(sorted(e), dtype=np.int64).reshape(-1, 2)


def chimera_edges(m: int, n: int, t: int = 4) -> np.ndarray:
    """Chimera C(m, n, t) edges: an m x n array of unit cells, each the
    complete bipartite graph K_{t,t} between its 'vertical' and 'horizontal'
    qubits; vertical qubits couple to the cell below, horizontal ones to the
    cell to the right. Qubit (i, j, side, k) is numbered ((i n + j) 2 + side) t + k."""
    def q(i, j, side, k):
        return ((i * n + j) * 2 + side) * t + k
    e = []
    for i in range(m):
        for j in range(n):
            for a in range(t):
                for b in range(t):
                    e.append((q(i, j, 0, a), q(i, j, 1, b)))
                if i + 1 < m:
                    e.append((q(i, j, 0, a), q(i + 1, j, 0, a)))
                if j + 1 < n:
                    e.append((q(i, j, 1, a), q(i, j + 1, 1, a)))
    return np.array(sorted(tuple(sorted(x)) for x in e), dtype=np.int64).reshape(-1, 2)


def gaussian_ising(name: str, n: int, e: np.ndarray, p: int, seed: int, with_h: bool = False) -> QaoaSpec:
    """QAOA on an Ising instance with Gaussian couplings (and fields), angles
    U[0, pi) from the same seed (the topologies of Sec. 4.3's timing study)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.normal(size=len(e))
    h = rng.normal(size=n) if with_h else None
    g, b = uniform_angles(p, seed=seed)
    return QaoaSpec(n=n, edges=e, weights=w, gammas=g, betas=b, h=h, name=name)


def kings_10x10_p1() -> QaoaSpec:
    """p=1 QAOA on the 10x10 King's graph (100 qubits), Gaussian couplings."""
    return gaussian_ising("qaoa_p1_kings10x10", 100, kings_edges(10, 10), 1, seed=6)


def chimera_c444_p1() -> QaoaSpec:
    """p=1 QAOA on Chimera C(4, 4, 4) (128 qubits), Gaussian couplings."""
    return gaussian_ising("qaoa_p1_chimera444", 128, chimera_edges(4, 4, 4), 1, seed=7)


def random_regular_edges(n: int, d: int, seed: int, max_tries: int = 10000) -> np.ndarray:
    """Random d-regular simple graph: configuration model with rejection."""
    if (n * d) % 2:
        raise ValueError("n*d must be even")
    rng = np.random.Generator(np.random.PCG64(seed))
    for _ in range(max_tries):
        stubs = np.repeat(np.arange(n), d)
        rng.shuffle(stubs)
        pairs = stubs.reshape(-1, 2)
        if np.any(pairs[:, 0] == pairs[:, 1]):
            continue
        pairs = np.sort(pairs, axis=1)
        if len({(int(a), int(b)) for a, b in pairs}) != len(pairs):
            continue
        return np.array(sorted((int(a), int(b)) for a, b in pairs), dtype=np.int64)
    raise RuntimeError("no simple regular graph found")


def heavy_hex_edges(n_target: int, row_len: int = 40) -> tuple[int, np.ndarray]:
    """Heavy-hex-like lattice: linear rows joined by single bridge qubits.

    Rows of ``row_len`` qubits; between rows r and r+1 a bridge qubit sits at
    every column c with c % 4 == 0 (r even) or c % 4 == 2 (r odd). Qubits are
    numbered row by row, each row's bridges following it. Rows are added until
    at least ``n_target`` qubits exist, then the highest-numbered qubits are
    dropped (which keeps the graph connected).
    """
    edges = []
    nq = 0
    prev_row = None
    r = 0
    while True:
        row = list(range(nq, nq + row_len))
        nq += row_len
        for a, b in zip(row[:-1], row[1:]):
            edges.append((a, b))
        if prev_row is not None:
            offs = 0 if (r - 1) % 2 == 0 else 2
            for c in range(offs, row_len, 4):
                bq = prev_bridges[c]
                edges.append((prev_row[c], bq))
                edges.append((bq, row[c]))
        if nq >= n_target:
            break
        offs = 0 if r % 2 == 0 else 2
        prev_bridges = {}
        for c in range(offs, row_len, 4):
            prev_bridges[c] = nq
            nq += 1
        prev_row = row
        r += 1
    keep = [(a, b) for a, b in edges if a < n_target and b < n_target]
    return n_target, np.array(sorted((min(a, b), max(a, b)) for a, b in keep), dtype=np.int64)


def uniform_angles(p: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """(gamma_1..p, beta_1..p) drawn uniformly from [0, pi)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = rng.uniform(0.0, math.pi, size=p)
    b = rng.uniform(0.0, math.pi, size=p)
    return g, b


# ----------------------------------------------------------------------------
# The five workloads (sizes of the paper's experiments, synthetic instances)
# ----------------------------------------------------------------------------

def maxcut_3reg_n12() -> QaoaSpec:
    """Ideal p=1 MaxCut, n=12 random 3-regular (seed 1), gamma=0.4, beta=0.3."""
    e = random_regular_edges(12, 3, seed=1)
    return QaoaSpec(n=12, edges=e, weights=np.ones(len(e)), gammas=np.array([0.4]),
                    betas=np.array([0.3]), name="qaoa_p1_3reg_n12")


def grid_6x6_p2() -> QaoaSpec:
    """Ideal p=2 MaxCut on a 6x6 grid (36 qubits), angles U[0,pi) seed 2."""
    e = grid_edges(6, 6)
    g, b = uniform_angles(2, seed=2)
    return QaoaSpec(n=36, edges=e, weights=np.ones(len(e)), gammas=g, betas=b,
                    name="qaoa_p2_grid6x6", extra={"rows": 6, "cols": 6})


def grid_8x8_p2_noisy(depol2: float = 1e-3, ad_gamma: float = 1e-3) -> QaoaSpec:
    """Noisy p=2 QAOA on an 8x8 grid (64 qubits), angles seed 3,
    two-qubit depolarizing after each RZZ, amplitude damping per qubit per layer."""
    e = grid_edges(8, 8)
    g, b = uniform_angles(2, seed=3)
    return QaoaSpec(n=64, edges=e, weights=np.ones(len(e)), gammas=g, betas=b,
                    depol2=depol2, ad_gamma=ad_gamma, name="qaoa_p2_grid8x8_noisy",
                    extra={"rows": 8, "cols": 8})


def gradient_instances(count: int = 512, nmin: int = 20, nmax: int = 48, p: int = 3) -> list[QaoaSpec]:
    """Batched-gradient workload: random 3-regular graphs, n uniform over even
    values in [nmin, nmax] (instance i uses seed 4+i), p=3 angles U[0,pi)."""
    out = []
    for i in range(count):
        rng = np.random.Generator(np.random.PCG64(4 + i))
        n = int(rng.choice(np.arange(nmin, nmax + 1, 2)))
        e = random_regular_edges(n, 3, seed=4 + i)
        g, b = uniform_angles(p, seed=4 + i)
        out.append(QaoaSpec(n=n, edges=e, weights=np.ones(len(e)), gammas=g, betas=b,
                            name=f"qaoa_p{p}_3reg_n{n}_i{i}"))
    return out


def heavy_hex_400_p1() -> QaoaSpec:
    """Ideal p=1 QAOA on a 400-qubit heavy-hex-like lattice, weights +-1 and
    angles from seed 5."""
    n, e = heavy_hex_edges(400)
    rng = np.random.Generator(np.random.PCG64(5))
    w = rng.choice(np.array([-1.0, 1.0]), size=len(e))
    g, b = uniform_angles(1, seed=5)
    return QaoaSpec(n=n, edges=e, weights=w, gammas=g, betas=b, name="qaoa_p1_heavyhex400")


def random_qaoa(n: int, p: int, seed: int, degree: int = 3, with_h: bool = False,
                depol2: float = 0.0, ad_gamma: float = 0.0) -> QaoaSpec:
    """Small random instances for parity tests (Gaussian weights and fields)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if degree == 3 and n % 2 == 0 and n >= 4:
        e = random_regular_edges(n, 3, seed=seed)
    else:
        e = np.array([(i, i + 1) for i in range(n - 1)], dtype=np.int64).reshape(-1, 2)
    w = rng.normal(size=len(e))
    h = rng.normal(size=n) if with_h else None
    g = rng.uniform(0.0, math.pi, size=p)
    b = rng.uniform(0.0, math.pi, size=p)
    return QaoaSpec(n=n, edges=e, weights=w, gammas=g, betas=b, h=h, depol2=depol2,
                    ad_gamma=ad_gamma, name=f"random_qaoa_n{n}_p{p}_s{seed}")


def random_bitstrings(count: int, n: int, seed: int) -> np.ndarray:
    """Uniform random bitstrings as uint8 [count, n]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, 2, size=(count, n), dtype=np.uint8)
