"""Seeded stand-ins for the paper's large workloads (inputs only).

c2_rgg    binary s-t connectivity on a 119-node / 295-edge random geometric
          graph (the size of the paper's Graph 2, Sec. 2.4 / 4.1); references
          grown by componentwise boundary search (Sec. 3.4) from random states
c3_dnf    classifier stress: a random monotone DNF over n = 300 components with
          2e5 non-dominated terms (upper references) and 5e4 greedy minimal
          cuts (lower references); "hundreds of thousands of reference states"
          as in Sec. 4.4
c4_flow   multi-state flow network: 40 nodes, 100 arcs, capacity states
          {0,1,2,3}, system state = max-flow level in {0,1,2} (Sec. 3.5, 4.5)
c5_batch  256 hazard scenarios: random geometric graphs of 50-300 edges with
          distance-dependent failure probabilities and 1e2-1e5 references

The heavy loops are in gen.c (OpenMP); results are cached under .cache/.
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import math
import os
import subprocess
import threading

import numpy as np

from .systems import Problem, binary_pmf

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libwlgen.so")
CACHE = os.environ.get("RSR_WORKLOAD_CACHE", os.path.join(_ROOT, ".cache", "workloads"))
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64
            lib.wl_dnf_terms.argtypes = [i32, i64, i32, i32, u64, P]
            lib.wl_dnf_terms.restype = i64
            lib.wl_greedy_cuts.argtypes = [i32, i64, P, i64, u64, i64, P]
            lib.wl_greedy_cuts.restype = i64
            lib.wl_st_boundary.argtypes = [i32, i32, P, P, i32, i32, P, u64, i64, i64, i64, P, P, P, P]
            lib.wl_flow_boundary.argtypes = [i32, i32, P, P, i32, i32, i32, P, i32, i32, i32, u64, i64, i64,
                                             i64, P, P, P, P]
            lib.wl_flow_values.argtypes = [i32, i32, P, P, i32, i32, i64, P, P]
            lib.wl_st_paths_cuts.argtypes = [i32, i32, P, P, i32, i32, u64, i64, i64, i64, P, P, P, P]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _cached(name: str, params: dict, make):
    key = hashlib.sha1(json.dumps([name, params], sort_keys=True).encode()).hexdigest()[:16]
    path = os.path.join(CACHE, "%s_%s.npz" % (name, key))
    if os.path.exists(path):
        with np.load(path, allow_pickle=False) as z:
            return {k: z[k] for k in z.files}
    out = make()
    os.makedirs(CACHE, exist_ok=True)
    tmp = path + ".tmp%d.npz" % os.getpid()
    np.savez(tmp, **out)
    os.replace(tmp, path)
    return out


# ------------------------------------------------------------------ graphs
def rgg_graph(n_nodes: int, n_edges: int, seed: int):
    """Nodes uniform in the unit square; edges = Euclidean minimum spanning
    tree plus the shortest remaining pairs, exactly n_edges, ordered by length
    (ties by node pair).  s = highest-degree node (lowest index on ties), t =
    the node farthest from s in hops (lowest index on ties)."""
    from scipy.sparse.csgraph import minimum_spanning_tree
    rng = np.random.default_rng(seed)
    pos = rng.random((n_nodes, 2))
    iu, ju = np.triu_indices(n_nodes, 1)
    d = np.hypot(*(pos[iu] - pos[ju]).T)
    D = np.zeros((n_nodes, n_nodes))
    D[iu, ju] = d
    mst = minimum_spanning_tree(D).tocoo()
    chosen = set((min(a, b), max(a, b)) for a, b in zip(mst.row.tolist(), mst.col.tolist()))
    for k in np.lexsort((ju, iu, d)):
        if len(chosen) >= n_edges:
            break
        chosen.add((int(iu[k]), int(ju[k])))
    edges = sorted(chosen, key=lambda e: (float(np.hypot(*(pos[e[0]] - pos[e[1]]))), e))
    deg = np.zeros(n_nodes, dtype=np.int64)
    for a, b in edges:
        deg[a] += 1
        deg[b] += 1
    s = int(np.argmax(deg))
    adj = [[] for _ in range(n_nodes)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    hop = np.full(n_nodes, -1)
    hop[s] = 0
    frontier = [s]
    while frontier:
        nxt = []
        for v in frontier:
            for w in adj[v]:
                if hop[w] < 0:
                    hop[w] = hop[v] + 1
                    nxt.append(w)
        frontier = nxt
    t = int(np.argmax(hop))
    return pos, np.array(edges, dtype=np.int32).reshape(-1, 2), s, t


def st_boundary_refs(n_nodes, edges, s, t, p_fail, seed, n_draws, max_L, max_U):
    lib = _load()
    n = edges.shape[0]
    eu = np.ascontiguousarray(edges[:, 0], dtype=np.int32)
    ev = np.ascontiguousarray(edges[:, 1], dtype=np.int32)
    pf = np.ascontiguousarray(p_fail, dtype=np.float64)
    out_L = np.zeros((max_L, n), dtype=np.uint8)
    out_U = np.zeros((max_U, n), dtype=np.uint8)
    nL, nU = ctypes.c_int64(0), ctypes.c_int64(0)
    lib.wl_st_boundary(n_nodes, n, _p(eu), _p(ev), s, t, _p(pf), seed, n_draws, max_L, max_U,
                       _p(out_L), ctypes.byref(nL), _p(out_U), ctypes.byref(nU))
    return out_L[:nL.value].copy(), out_U[:nU.value].copy()


def st_paths_cuts(n_nodes, edges, s, t, seed, n_draws, max_L, max_U):
    lib = _load()
    n = edges.shape[0]
    eu = np.ascontiguousarray(edges[:, 0], dtype=np.int32)
    ev = np.ascontiguousarray(edges[:, 1], dtype=np.int32)
    out_L = np.zeros((max_L, n), dtype=np.uint8)
    out_U = np.zeros((max_U, n), dtype=np.uint8)
    nL, nU = ctypes.c_int64(0), ctypes.c_int64(0)
    lib.wl_st_paths_cuts(n_nodes, n, _p(eu), _p(ev), s, t, seed, n_draws, max_L, max_U,
                         _p(out_L), ctypes.byref(nL), _p(out_U), ctypes.byref(nU))
    return out_L[:nL.value].copy(), out_U[:nU.value].copy()


# ------------------------------------------------------------------ C2
def c2_rgg(seed: int = 2, n_nodes: int = 119, n_edges: int = 295, n_draws: int = 20000,
           max_refs: int = 10000) -> Problem:
    def make():
        pos, edges, s, t = rgg_graph(n_nodes, n_edges, seed)
        rng = np.random.default_rng(seed + 1000)
        pf = rng.uniform(0.01, 0.2, size=n_edges)
        ref_L, ref_U = st_boundary_refs(n_nodes, edges, s, t, pf, seed + 2000, n_draws, max_refs // 2,
                                        max_refs // 2)
        return dict(pos=pos, edges=edges, st=np.array([s, t]), pf=pf, ref_L=ref_L, ref_U=ref_U)
    z = _cached("c2_rgg", dict(seed=seed, n=n_nodes, e=n_edges, d=n_draws, m=max_refs, v=1), make)
    s, t = (int(v) for v in z["st"])
    return Problem("c2_rgg119_295", binary_pmf(z["pf"]), z["ref_L"], z["ref_U"],
                   dict(n_nodes=n_nodes, edges=z["edges"], pos=z["pos"], s=s, t=t))


# ------------------------------------------------------------------ C3
def dnf_terms(n: int, R: int, lo: int, hi: int, seed: int) -> np.ndarray:
    out = np.zeros((R, n), dtype=np.uint8)
    r = _load().wl_dnf_terms(n, R, lo, hi, seed, _p(out))
    if r != R:
        raise RuntimeError("dnf generation failed")
    return out


def greedy_cuts(terms: np.ndarray, R_L: int, seed: int, max_draws: int) -> np.ndarray:
    terms = np.ascontiguousarray(terms, dtype=np.uint8)
    R, n = terms.shape
    out = np.zeros((R_L, n), dtype=np.uint8)
    got = _load().wl_greedy_cuts(n, R, _p(terms), R_L, seed, max_draws, _p(out))
    return out[:got].copy()


def c3_dnf(n: int = 300, R_U: int = 200000, R_L: int = 50000, lo: int = 8, hi: int = 40,
           p_up: float = 0.9, seed: int = 3) -> Problem:
    """Upper references = the DNF terms (1 on the term), ordered by size (so by
    decreasing P(X >= r) under equal component probabilities; order does not
    change labels); lower references = distinct minimal hitting sets (0 on the
    cut, 1 elsewhere)."""
    def make():
        terms = dnf_terms(n, R_U, lo, hi, seed)
        order = np.argsort(terms.sum(1), kind="stable")
        terms = terms[order]
        cuts = greedy_cuts(terms, R_L, seed + 1, max_draws=4 * R_L)
        return dict(ref_U=terms, ref_L=cuts)
    z = _cached("c3_dnf", dict(n=n, RU=R_U, RL=R_L, lo=lo, hi=hi, seed=seed, v=1), make)
    return Problem("c3_dnf%d_%d_%d" % (n, R_U, R_L), binary_pmf(np.full(n, 1.0 - p_up)), z["ref_L"], z["ref_U"],
                   dict(p_up=p_up))


# ------------------------------------------------------------------ C4
def random_digraph(n_nodes: int, n_arcs: int, seed: int):
    """Uniform random simple directed graph, redrawn until t is reachable from
    s; s = highest total degree (lowest index), t = farthest in directed hops
    from s (lowest index)."""
    rng = np.random.default_rng(seed)
    while True:
        pairs = [(a, b) for a in range(n_nodes) for b in range(n_nodes) if a != b]
        pick = rng.choice(len(pairs), size=n_arcs, replace=False)
        arcs = np.array(sorted(pairs[k] for k in pick), dtype=np.int32)
        deg = np.bincount(arcs.ravel(), minlength=n_nodes)
        s = int(np.argmax(deg))
        hop = np.full(n_nodes, -1)
        hop[s] = 0
        frontier = [s]
        while frontier:
            nxt = []
            for v in frontier:
                for b in arcs[arcs[:, 0] == v, 1]:
                    if hop[b] < 0:
                        hop[b] = hop[v] + 1
                        nxt.append(int(b))
            frontier = nxt
        t = int(np.argmax(hop))
        if hop[t] > 0:
            return arcs, s, t


def flow_values(n_nodes, arcs, s, t, X) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.uint8)
    out = np.zeros(X.shape[0], dtype=np.int32)
    au = np.ascontiguousarray(arcs[:, 0], dtype=np.int32)
    av = np.ascontiguousarray(arcs[:, 1], dtype=np.int32)
    _load().wl_flow_values(n_nodes, arcs.shape[0], _p(au), _p(av), s, t, X.shape[0], _p(X), _p(out))
    return out


def c4_flow(m_prime: int = 0, seed: int = 4, n_nodes: int = 40, n_arcs: int = 100,
            pmf_row=(0.05, 0.15, 0.3, 0.5), n_draws: int = 20000, max_refs: int = 20000) -> Problem:
    """Arc capacities are the component states {0..3}; S = 0 if the s-t max
    flow f < ceil(f_max/3), 1 if f < ceil(2 f_max/3), else 2, with f_max the
    flow at full capacity.  s = highest total degree; t = the node with the
    largest full-capacity flow from s.  References for the threshold m'."""
    K = len(pmf_row)

    def make():
        arcs, s, _ = random_digraph(n_nodes, n_arcs, seed)
        full = np.full((1, n_arcs), K - 1, dtype=np.uint8)
        # sink: the node with the largest full-capacity flow from s (lowest index on ties)
        flows = [int(flow_values(n_nodes, arcs, s, v, full)[0]) if v != s else -1 for v in range(n_nodes)]
        t = int(np.argmax(flows))
        fmax = flows[t]
        l1, l2 = -(-fmax // 3), -(-2 * fmax // 3)
        pmf = np.tile(np.asarray(pmf_row, dtype=np.float64), (n_arcs, 1))
        lib = _load()
        au = np.ascontiguousarray(arcs[:, 0])
        av = np.ascontiguousarray(arcs[:, 1])
        out_L = np.zeros((max_refs // 2, n_arcs), dtype=np.uint8)
        out_U = np.zeros((max_refs // 2, n_arcs), dtype=np.uint8)
        nL, nU = ctypes.c_int64(0), ctypes.c_int64(0)
        lib.wl_flow_boundary(n_nodes, n_arcs, _p(au), _p(av), s, t, K, _p(pmf), l1, l2, m_prime,
                             seed + 100 + m_prime, n_draws, max_refs // 2, max_refs // 2,
                             _p(out_L), ctypes.byref(nL), _p(out_U), ctypes.byref(nU))
        return dict(arcs=arcs, st=np.array([s, t]), levels=np.array([fmax, l1, l2]), pmf=pmf,
                    ref_L=out_L[:nL.value].copy(), ref_U=out_U[:nU.value].copy())
    z = _cached("c4_flow", dict(seed=seed, mp=m_prime, n=n_nodes, a=n_arcs, pmf=list(pmf_row), d=n_draws,
                                m=max_refs, v=2), make)
    s, t = (int(v) for v in z["st"])
    fmax, l1, l2 = (int(v) for v in z["levels"])
    return Problem("c4_flow40_100_m%d" % m_prime, z["pmf"], z["ref_L"], z["ref_U"],
                   dict(arcs=z["arcs"], n_nodes=n_nodes, s=s, t=t, fmax=fmax, l1=l1, l2=l2, m_prime=m_prime))


# ------------------------------------------------------------------ C5
def c5_batch(S: int = 256, seed0: int = 1000, n_lo: int = 50, n_hi: int = 300, R_lo: float = 1e2,
             R_hi: float = 1e5):
    """S hazard scenarios (seeds seed0..seed0+S-1): a random geometric graph with
    n ~ U{n_lo..n_hi} edges on round(0.4 n) nodes, an epicentre uniform in the
    square, p_f = 1/(1 + exp((d - 0.25)/0.05)) clipped to [1e-4, 0.5] with d the
    edge-midpoint distance, and R ~ log-uniform [R_lo, R_hi] references (half
    minimal path sets, half minimal cuts, fewer if fewer are found)."""
    probs = []
    for j in range(S):
        sd = seed0 + j

        def make(sd=sd):
            rng = np.random.default_rng(sd)
            n = int(rng.integers(n_lo, n_hi + 1))
            nn = int(round(0.4 * n))
            R = int(round(math.exp(rng.uniform(math.log(R_lo), math.log(R_hi)))))
            epi = rng.random(2)
            pos, edges, s, t = rgg_graph(nn, n, sd)
            mid = 0.5 * (pos[edges[:, 0]] + pos[edges[:, 1]])
            d = np.hypot(*(mid - epi).T)
            pf = np.clip(1.0 / (1.0 + np.exp((d - 0.25) / 0.05)), 1e-4, 0.5)
            ref_L, ref_U = st_paths_cuts(nn, edges, s, t, sd + 7, 4 * R, R - R // 2, R // 2)
            return dict(pf=pf, edges=edges, st=np.array([s, t]), ref_L=ref_L, ref_U=ref_U)
        z = _cached("c5_scn", dict(seed=sd, nlo=n_lo, nhi=n_hi, Rlo=R_lo, Rhi=R_hi, v=1), make)
        probs.append(Problem("c5_scenario_%d" % sd, binary_pmf(z["pf"]), z["ref_L"], z["ref_U"],
                             dict(edges=z["edges"], s=int(z["st"][0]), t=int(z["st"][1]), seed=sd)))
    return probs
