"""Small systems with complete reference sets, and the 3x4 grid workload.

Everything here is exhaustive or closed-form, sized so that all K^n states can
be enumerated.  The larger seeded workloads live in ``large.py``.
"""
from __future__ import annotations

import dataclasses
import itertools
from typing import Optional

import numpy as np


@dataclasses.dataclass
class Problem:
    """One classification problem: pmf (n x K, fp64, rows sum to 1) and the
    lower (failure, S <= m') and upper (survival, S >= m'+1) reference states,
    each an R x n uint8 matrix of component states."""

    name: str
    pmf: np.ndarray
    ref_L: np.ndarray
    ref_U: np.ndarray
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pmf.shape[0])

    @property
    def K(self) -> int:
        return int(self.pmf.shape[1])

    @property
    def R_L(self) -> int:
        return int(self.ref_L.shape[0])

    @property
    def R_U(self) -> int:
        return int(self.ref_U.shape[0])


def binary_pmf(p_fail) -> np.ndarray:
    """pmf rows (P(X_i = 0), P(X_i = 1)) with state 0 = failed, 1 = working."""
    p_fail = np.asarray(p_fail, dtype=np.float64).reshape(-1)
    return np.stack([p_fail, 1.0 - p_fail], axis=1)


def grid_graph(rows: int, cols: int):
    """Undirected rows x cols grid.  Node (r, c) has index r*cols + c.  Edges:
    the horizontal ones row-major, then the vertical ones row-major."""
    edges = []
    for r in range(rows):
        for c in range(cols - 1):
            edges.append((r * cols + c, r * cols + c + 1))
    for r in range(rows - 1):
        for c in range(cols):
            edges.append((r * cols + c, (r + 1) * cols + c))
    return rows * cols, edges


def _state_index_strides(n: int, K: int) -> np.ndarray:
    """Index of state x in itertools.product order: sum_i x_i K^(n-1-i)."""
    return (K ** np.arange(n - 1, -1, -1)).astype(np.int64)


def all_states(n: int, K: int) -> np.ndarray:
    return np.array(list(itertools.product(range(K), repeat=n)), dtype=np.uint8).reshape(-1, n)


def st_connectivity_all_states(n_nodes: int, edges, s: int, t: int) -> np.ndarray:
    """Phi(x) = 1 if s and t are joined by working edges (x_e = 1), else 0, for
    every x in {0,1}^|E| (product order).  Vectorised label propagation."""
    n = len(edges)
    X = all_states(n, 2).astype(bool)
    reach = np.zeros((X.shape[0], n_nodes), dtype=bool)
    reach[:, s] = True
    while True:
        before = reach.copy()
        for e, (u, v) in enumerate(edges):
            up = X[:, e]
            reach[:, v] |= reach[:, u] & up
            reach[:, u] |= reach[:, v] & up
        if np.array_equal(before, reach):
            break
    return reach[:, t].astype(np.int32)


def reference_sets_from_phi(phi: np.ndarray, n: int, K: int, m_prime: int = 0):
    """Complete reference sets (Sec. 2.2, Eqs. (2)-(3)) from Phi over all K^n
    states in product order.  Lower: states with Phi <= m' whose every single
    upward step leaves the set (maximal); upper: states with Phi >= m'+1 whose
    every single downward step leaves the set (minimal).  For a coherent Phi a
    single-step check is enough."""
    phi = np.asarray(phi)
    X = all_states(n, K)
    stride = _state_index_strides(n, K)
    idx = np.arange(X.shape[0], dtype=np.int64)
    low = phi <= m_prime
    is_lower_ref = low.copy()
    is_upper_ref = ~low
    for i in range(n):
        can_up = X[:, i] < K - 1
        up_idx = np.where(can_up, idx + stride[i], idx)
        is_lower_ref &= ~can_up | ~low[up_idx]
        can_dn = X[:, i] > 0
        dn_idx = np.where(can_dn, idx - stride[i], idx)
        is_upper_ref &= ~can_dn | low[dn_idx]
    return X[is_lower_ref].copy(), X[is_upper_ref].copy()


def c1_grid(p_fail: float = 0.1) -> Problem:
    """3x4 grid, 12 nodes, 17 edges; s = (0,0), t = (2,3); every edge fails
    with probability p_fail; complete path (upper) and cut (lower) references
    by enumeration of all 2^17 states."""
    n_nodes, edges = grid_graph(3, 4)
    s, t = 0, 11
    phi = st_connectivity_all_states(n_nodes, edges, s, t)
    ref_L, ref_U = reference_sets_from_phi(phi, len(edges), 2, 0)
    return Problem("c1_grid3x4", binary_pmf(np.full(len(edges), p_fail)), ref_L, ref_U,
                   dict(n_nodes=n_nodes, edges=edges, s=s, t=t, phi_all=phi))


def series_system(p_fail) -> Problem:
    """Works iff every component works.  Upper: the all-ones state.  Lower:
    one failed component, all others working."""
    pmf = binary_pmf(p_fail)
    n = pmf.shape[0]
    ref_U = np.ones((1, n), dtype=np.uint8)
    ref_L = np.ones((n, n), dtype=np.uint8) - np.eye(n, dtype=np.uint8)
    return Problem("series", pmf, ref_L, ref_U)


def parallel_system(p_fail) -> Problem:
    """Works iff some component works.  Upper: one working component.  Lower:
    the all-zeros state."""
    pmf = binary_pmf(p_fail)
    n = pmf.shape[0]
    return Problem("parallel", pmf, np.zeros((1, n), dtype=np.uint8), np.eye(n, dtype=np.uint8))


def k_out_of_n_system(n: int, k: int, p_fail) -> Problem:
    """Works iff at least k of n components work.  Upper: every k-subset
    working (others failed).  Lower: every (k-1)-subset working (others
    failed)."""
    pmf = binary_pmf(np.broadcast_to(np.asarray(p_fail, dtype=np.float64), (n,)))
    ups = []
    for sub in itertools.combinations(range(n), k):
        r = np.zeros(n, dtype=np.uint8)
        r[list(sub)] = 1
        ups.append(r)
    lows = []
    for sub in itertools.combinations(range(n), k - 1):
        r = np.zeros(n, dtype=np.uint8)
        r[list(sub)] = 1
        lows.append(r)
    return Problem("k_out_of_n", pmf, np.array(lows, dtype=np.uint8).reshape(-1, n),
                   np.array(ups, dtype=np.uint8).reshape(-1, n), dict(k=k))


def random_small_system(n: int, K: int, M_S: int, seed: int, m_prime: Optional[int] = None) -> Problem:
    """Random coherent multi-state system small enough to enumerate:
    Phi(x) = min(M_S - 1, floor(sum_i w_i x_i / c)) with random w_i >= 0
    (monotone in every component), a random pmf, and complete reference sets
    for threshold m' (default 0)."""
    rng = np.random.default_rng(seed)
    w = rng.integers(0, 4, size=n)
    total = int(w.sum()) * (K - 1)
    c = max(1, total // M_S + 1)
    X = all_states(n, K)
    phi = np.minimum(M_S - 1, (X.astype(np.int64) @ w) // c)
    mp = 0 if m_prime is None else m_prime
    ref_L, ref_U = reference_sets_from_phi(phi, n, K, mp)
    pmf = rng.dirichlet(np.ones(K), size=n)
    return Problem("random_small", pmf, ref_L, ref_U, dict(phi_all=phi, m_prime=mp, w=w, c=c))
