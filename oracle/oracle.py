"""Python front end of the RSR oracle (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the cpu_baseline / reference
legs of ``bench.py`` may import this module.  The product library never does.

The heavy loops live in ``rsr_oracle.c`` (plain C, compiled here with gcc); this
module loads it with ctypes and adds the brute-force enumerations used to pin the
oracle on tiny systems:

* ``exact_probability``: P(S <= m') by summing P(x) over every state
  (Sec. 2.1: the "most straightforward approach", exponential in n);
* ``exact_gradient``: dP(S <= m')/dq_{i,k} = P(S <= m' | X_i = k), the partial
  derivative of the multilinear polynomial sum_x 1[Phi(x) <= m'] prod_j q_{j,x_j}.

The oracle shares no code with ``paper_2604_17066_gb300`` and never imports it.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rsr_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile rsr_oracle.c into liboracle.so next to it (plain gcc -O2)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i32, i64, u32, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
            lib.orc_philox4x32_10.argtypes = [P, P, P]
            lib.orc_thresholds.argtypes = [i32, i32, P, P]
            lib.orc_state_from_uniform.argtypes = [u32, i32, P]
            lib.orc_state_from_uniform.restype = i32
            lib.orc_sample.argtypes = [i32, i32, P, u64, u64, i64, P]
            lib.orc_classify.argtypes = [i32, i64, P, i64, P, i64, P, P, P]
            lib.orc_estimate.argtypes = [P, i64, i64, P]
            lib.orc_grad_counts.argtypes = [i32, i32, i64, P, P, P, i64, P]
            lib.orc_grad.argtypes = [i32, i32, i64, P, P, P, P]
            lib.orc_count_overlaps.argtypes = [i32, i64, P, i64, P]
            lib.orc_count_overlaps.restype = i64
            lib.orc_phi.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, P, P]
            lib.orc_phi.restype = ctypes.c_int
            lib.orc_resolve.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, P, ctypes.c_int, i64, P, P]
            lib.orc_resolve.restype = i64
            lib.orc_boundary_search.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_int, P, ctypes.c_int, ctypes.c_int, P, P, P, P]
            lib.orc_search_order.argtypes = [u64, u64, ctypes.c_int, P]
            lib.orc_boundary_search.restype = ctypes.c_int
            lib.orc_nondominated.argtypes = [ctypes.c_int, i64, P, ctypes.c_int, P]
            lib.orc_levels.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, P, i64, P, P]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# thin wrappers
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block: 4 uint32 words from a 4-word counter and 2-word key."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def thresholds(pmf: np.ndarray) -> np.ndarray:
    """Integer inverse-CDF thresholds T[i, k-1] = min(2^32, floor(2^32 * sum_{j<k} q_ij))."""
    pmf = np.ascontiguousarray(pmf, dtype=np.float64)
    n, K = pmf.shape
    T = np.zeros((n, K - 1), dtype=np.uint64)
    _load().orc_thresholds(n, K, _p(pmf), _p(T))
    return T


def state_from_uniform(u: int, T_row: np.ndarray) -> int:
    T_row = np.ascontiguousarray(T_row, dtype=np.uint64)
    return int(_load().orc_state_from_uniform(int(u) & 0xFFFFFFFF, T_row.size + 1, _p(T_row)))


def sample(pmf: np.ndarray, seed: int, offset: int, N: int) -> np.ndarray:
    """N x n uint8 states of samples offset .. offset+N-1 (Philox counter layout in rsr_oracle.c)."""
    pmf = np.ascontiguousarray(pmf, dtype=np.float64)
    n, K = pmf.shape
    T = thresholds(pmf)
    X = np.zeros((N, n), dtype=np.uint8)
    if N:
        _load().orc_sample(n, K, _p(T), int(seed), int(offset), int(N), _p(X))
    return X


def classify(X: np.ndarray, ref_L: np.ndarray, ref_U: np.ndarray):
    """Labels (0 = I^L, 1 = I^U, 2 = I^u) and counts [|I^L|, |I^U|, |I^u|] (Algorithm 1)."""
    X = np.ascontiguousarray(X, dtype=np.uint8)
    N, n = X.shape
    ref_L = np.ascontiguousarray(ref_L, dtype=np.uint8).reshape(-1, n)
    ref_U = np.ascontiguousarray(ref_U, dtype=np.uint8).reshape(-1, n)
    labels = np.zeros(N, dtype=np.uint8)
    counts = np.zeros(3, dtype=np.int64)
    _load().orc_classify(n, N, _p(X), ref_L.shape[0], _p(ref_L), ref_U.shape[0], _p(ref_U),
                         _p(labels), _p(counts))
    return labels, counts


ESTIMATE_FIELDS = ("pL", "pU", "pu", "P_lower", "P_upper",
                   "cov_pL", "cov_pU", "cov_pu", "cov_lower", "cov_upper")


def estimate(counts3, N: int, n_u_lower: int = 0) -> dict:
    c = np.ascontiguousarray(counts3, dtype=np.int64)
    out = np.zeros(10, dtype=np.float64)
    _load().orc_estimate(_p(c), int(N), int(n_u_lower), _p(out))
    return dict(zip(ESTIMATE_FIELDS, out.tolist()))


def grad_counts(X: np.ndarray, labels: np.ndarray, K: int, u_lower_idx=None) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.uint8)
    N, n = X.shape
    labels = np.ascontiguousarray(labels, dtype=np.uint8)
    idx = np.ascontiguousarray([] if u_lower_idx is None else u_lower_idx, dtype=np.int64)
    C = np.zeros((n, K), dtype=np.int64)
    _load().orc_grad_counts(n, K, N, _p(X), _p(labels), _p(idx), idx.size, _p(C))
    return C


def grad(C: np.ndarray, N: int, pmf: np.ndarray):
    """(g_hat, se) with g_hat[i,k] = (C[i,k]/N)/q[i,k], se = sqrt(p(1-p)/N)/q."""
    C = np.ascontiguousarray(C, dtype=np.int64)
    pmf = np.ascontiguousarray(pmf, dtype=np.float64)
    n, K = pmf.shape
    g = np.zeros((n, K), dtype=np.float64)
    se = np.zeros((n, K), dtype=np.float64)
    _load().orc_grad(n, K, int(N), _p(C), _p(pmf), _p(g), _p(se))
    return g, se


def count_overlaps(ref_L: np.ndarray, ref_U: np.ndarray) -> int:
    """Number of (r^L, r^U) pairs with r^U <= r^L componentwise."""
    ref_L = np.ascontiguousarray(ref_L, dtype=np.uint8)
    ref_U = np.ascontiguousarray(ref_U, dtype=np.uint8)
    n = ref_L.shape[1] if ref_L.ndim == 2 else ref_U.shape[1]
    return int(_load().orc_count_overlaps(n, ref_L.shape[0], _p(ref_L), ref_U.shape[0], _p(ref_U)))


# --------------------------------------------------------------------------
# Stage 2: Phi on the unclassified samples (Sec. 3.5)
# --------------------------------------------------------------------------
PHI_ST_CONNECTIVITY = 0
PHI_ST_MAXFLOW_LEVELS = 1
PHI_GLOBAL_CONNECTIVITY = 2
PHI_GLOBAL_CONN_LEVEL = 3


def _graph_args(edges, thresholds):
    e = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 2)
    src = np.ascontiguousarray(e[:, 0])
    dst = np.ascontiguousarray(e[:, 1])
    thr = np.ascontiguousarray([] if thresholds is None else thresholds, dtype=np.int32)
    return src, dst, thr


def phi(kind: int, n_nodes: int, edges, s: int, t: int, x, thresholds=None) -> int:
    """System function of one state: s-t connectivity (kind 0) or the s-t
    max-flow level #{l : flow >= thresholds[l]} (kind 1)."""
    src, dst, thr = _graph_args(edges, thresholds)
    xs = np.ascontiguousarray(x, dtype=np.uint8)
    return int(_load().orc_phi(kind, n_nodes, src.size, _p(src), _p(dst), s, t, thr.size, _p(thr), _p(xs)))


def resolve(kind: int, n_nodes: int, edges, s: int, t: int, X, labels, m_prime: int = 0, thresholds=None):
    """Stage 2: labels 2 become 3 (Phi <= m') or 4; returns (new labels, #3)."""
    src, dst, thr = _graph_args(edges, thresholds)
    X = np.ascontiguousarray(X, dtype=np.uint8)
    lab = np.array(labels, dtype=np.uint8, copy=True)
    lower = _load().orc_resolve(kind, n_nodes, src.size, _p(src), _p(dst), s, t, thr.size, _p(thr), m_prime,
                                X.shape[0], _p(X), _p(lab))
    return lab, int(lower)


def levels(kind: int, n_nodes: int, edges, s: int, t: int, X, thresholds=None) -> np.ndarray:
    """Phi(x_h) for every row of X (uint8 system levels)."""
    src, dst, thr = _graph_args(edges, thresholds)
    X = np.ascontiguousarray(X, dtype=np.uint8)
    out = np.zeros(X.shape[0], dtype=np.uint8)
    if X.shape[0]:
        _load().orc_levels(kind, n_nodes, src.size, _p(src), _p(dst), s, t, thr.size, _p(thr), X.shape[0], _p(X),
                           _p(out))
    return out


def level_pmf(pmf, kind: int, n_nodes: int, edges, s: int, t: int, seed: int, offset: int, N: int, n_levels: int,
              thresholds=None):
    """(counts[m] = #{h : Phi(x_h) = m}, levels) for samples offset .. offset+N-1."""
    X = sample(pmf, seed, offset, N)
    lv = levels(kind, n_nodes, edges, s, t, X, thresholds)
    return np.bincount(lv, minlength=n_levels).astype(np.int64), lv


# --------------------------------------------------------------------------
# Stage 1: reference-state search (Sec. 3.4, 3.5)
# --------------------------------------------------------------------------
SEARCH_INDEX_ORDER = 0
SEARCH_PERMUTED = 1


def search_order(seed: int, h: int, n: int) -> np.ndarray:
    """Visiting order of the permuted search from (global) sample h."""
    out = np.zeros(n, dtype=np.int32)
    _load().orc_search_order(int(seed), int(h), n, _p(out))
    return out


def boundary_search(kind: int, n_nodes: int, edges, s: int, t: int, x, K: int, m_prime: int = 0,
                    thresholds=None, order=None):
    """Componentwise boundary search from state x: (side, reference, #Phi evaluations),
    side 0 = lower reference (Phi(x) <= m'), 1 = upper.  order: None = index order,
    else the visiting order of the components."""
    src, dst, thr = _graph_args(edges, thresholds)
    xs = np.ascontiguousarray(x, dtype=np.uint8)
    out = np.zeros_like(xs)
    ev = np.zeros(1, dtype=np.int64)
    od = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
    side = _load().orc_boundary_search(kind, n_nodes, src.size, _p(src), _p(dst), s, t, thr.size, _p(thr),
                                       m_prime, K, _p(xs), _p(out), _p(ev), None if od is None else _p(od))
    return int(side), out, int(ev[0])


def nondominated(refs, upper: bool) -> np.ndarray:
    """keep mask of the non-dominated references of one side (first of equal ones kept)."""
    refs = np.ascontiguousarray(refs, dtype=np.uint8)
    R = refs.shape[0]
    keep = np.zeros(R, dtype=np.uint8)
    if R:
        _load().orc_nondominated(refs.shape[1], R, _p(refs), 1 if upper else 0, _p(keep))
    return keep.astype(bool)


def stage1(pmf, kind: int, n_nodes: int, edges, s: int, t: int, seed: int, N: int, max_starts: int,
           eps_u: float, R_max: int, max_rounds: int, m_prime: int = 0, thresholds=None,
           ref_L=None, ref_U=None, order: int = SEARCH_INDEX_ORDER):
    """Stage 1 of the RSR workflow (Sec. 3.5), with many searches per round.

    Round r draws samples r*N .. r*N+N-1 (Philox stream `seed`) and classifies
    them against the current references.  It stops when the unclassified
    fraction is below eps_u, when R_L + R_U >= R_max, or after max_rounds.
    Otherwise the first min(max_starts, #unclassified, R_max - R) unclassified
    samples in index order (a uniform random choice, the samples being i.i.d.)
    each start a componentwise boundary search.  The new references are
    appended to their side in start order, and each side is reduced to its
    non-dominated elements (order kept).  order = SEARCH_PERMUTED visits the
    components of the search from sample h (global index) in search_order(seed, h).

    Returns dict(ref_L, ref_U, history=[(n_unclassified, R_L, R_U, n_starts)],
    stop=0 converged | 1 R_max | 2 max_rounds, phi_evals)."""
    pmf = np.asarray(pmf, dtype=np.float64)
    n, K = pmf.shape
    L = np.zeros((0, n), np.uint8) if ref_L is None else np.array(ref_L, dtype=np.uint8).reshape(-1, n)
    U = np.zeros((0, n), np.uint8) if ref_U is None else np.array(ref_U, dtype=np.uint8).reshape(-1, n)
    hist = []
    evals = 0
    stop = 2
    for r in range(max_rounds):
        X = sample(pmf, seed, r * N, N)
        lab, cnt = classify(X, L, U)
        n_u = int(cnt[2])
        R = L.shape[0] + U.shape[0]
        if n_u < eps_u * N:
            hist.append((n_u, L.shape[0], U.shape[0], 0))
            stop = 0
            break
        if R >= R_max:
            hist.append((n_u, L.shape[0], U.shape[0], 0))
            stop = 1
            break
        starts = np.flatnonzero(lab == 2)[:min(max_starts, R_max - R)]
        hist.append((n_u, L.shape[0], U.shape[0], int(starts.size)))
        newL, newU = [], []
        for h in starts:
            od = search_order(seed, r * N + int(h), n) if order == SEARCH_PERMUTED else None
            side, ref, ev = boundary_search(kind, n_nodes, edges, s, t, X[h], K, m_prime, thresholds, od)
            evals += ev
            (newL if side == 0 else newU).append(ref)
        if newL:
            L = np.concatenate([L, np.array(newL, dtype=np.uint8)])
            L = L[nondominated(L, upper=False)]
        if newU:
            U = np.concatenate([U, np.array(newU, dtype=np.uint8)])
            U = U[nondominated(U, upper=True)]
    return dict(ref_L=L, ref_U=U, history=hist, stop=stop, phi_evals=evals)


# --------------------------------------------------------------------------
# brute force over all K^n states (tiny systems only)
# --------------------------------------------------------------------------
def all_states(n: int, K: int) -> np.ndarray:
    """Every state of {0..K-1}^n, row-major with component 0 slowest."""
    return np.array(list(itertools.product(range(K), repeat=n)), dtype=np.uint8).reshape(-1, n)


def exact_probability(pmf: np.ndarray, states: np.ndarray, in_event: np.ndarray) -> float:
    """sum over states of prod_i q_{i,x_i} * 1[event] (Sec. 2.1, full enumeration)."""
    pmf = np.asarray(pmf, dtype=np.float64)
    n = pmf.shape[0]
    prob = np.ones(states.shape[0], dtype=np.float64)
    for i in range(n):
        prob *= pmf[i, states[:, i]]
    return float(prob[np.asarray(in_event, dtype=bool)].sum())


def exact_gradient(pmf: np.ndarray, states: np.ndarray, in_event: np.ndarray) -> np.ndarray:
    """dP(event)/dq_{i,k} = sum_{x: x_i = k} 1[event] prod_{j != i} q_{j,x_j}."""
    pmf = np.asarray(pmf, dtype=np.float64)
    n, K = pmf.shape
    ev = np.asarray(in_event, dtype=bool)
    g = np.zeros((n, K), dtype=np.float64)
    for i in range(n):
        others = np.ones(states.shape[0], dtype=np.float64)
        for j in range(n):
            if j != i:
                others *= pmf[j, states[:, j]]
        for k in range(K):
            sel = ev & (states[:, i] == k)
            g[i, k] = others[sel].sum()
    return g
