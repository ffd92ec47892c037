"""Pins of the oracle's Stage 2 (Sec. 3.5): its system functions against
networkx (s-t connectivity by has_path, s-t max flow by maximum_flow_value),
and the consistency that resolving the unclassified samples of a partial
reference set with Phi reproduces the classification by the complete set."""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

nx = pytest.importorskip("networkx")


def test_connectivity_matches_networkx():
    import workloads.large as L
    p = L.c2_rgg()
    edges, s, t, nn = p.meta["edges"], p.meta["s"], p.meta["t"], p.meta["n_nodes"]
    rng = np.random.default_rng(0)
    for trial in range(150):
        x = (rng.random(p.n) > rng.uniform(0.05, 0.6)).astype(np.uint8)
        G = nx.Graph()
        G.add_nodes_from(range(nn))
        G.add_edges_from(edges[x == 1].tolist())
        assert O.phi(O.PHI_ST_CONNECTIVITY, nn, edges, s, t, x) == int(nx.has_path(G, s, t))


def test_max_flow_levels_match_networkx():
    import workloads.large as L
    p = L.c4_flow(0)
    arcs, s, t, nn = p.meta["arcs"], p.meta["s"], p.meta["t"], p.meta["n_nodes"]
    thr = [p.meta["l1"], p.meta["l2"]]
    rng = np.random.default_rng(1)
    for trial in range(120):
        x = rng.integers(0, 4, size=p.n).astype(np.uint8)
        G = nx.DiGraph()
        G.add_nodes_from(range(nn))
        for (u, v), c in zip(arcs.tolist(), x.tolist()):
            if G.has_edge(u, v):
                G[u][v]["capacity"] += c
            else:
                G.add_edge(u, v, capacity=c)
        f = nx.maximum_flow_value(G, s, t)
        level = int(f >= thr[0]) + int(f >= thr[1])
        assert O.phi(O.PHI_ST_MAXFLOW_LEVELS, nn, arcs, s, t, x, thresholds=thr) == level


def test_stage2_with_partial_references_reproduces_complete_classification():
    p = W.c1_grid()
    X = O.sample(p.pmf, 3, 0, 20000)
    full, _ = O.classify(X, p.ref_L, p.ref_U)
    lab, cnt = O.classify(X, p.ref_L[::3], p.ref_U[::4])
    assert cnt[2] > 100
    res, n_lower = O.resolve(O.PHI_ST_CONNECTIVITY, p.meta["n_nodes"], p.meta["edges"], p.meta["s"], p.meta["t"],
                             X, lab)
    final = np.where(res == 3, 0, np.where(res == 4, 1, res))
    assert np.array_equal(final, full)
    assert n_lower == int(np.sum((lab == 2) & (full == 0)))
    est = O.estimate(cnt, X.shape[0], n_lower)
    assert est["P_lower"] == np.mean(full == 0)
