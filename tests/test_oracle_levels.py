"""Pins for the oracle's system-state pmf over all levels (Sec. 3.5 at every
boundary; Sec. 4.5-4.6 multi-state examples).

* The level of every state of small systems equals networkx's (maximum flow
  levels; global connectivity with edge connectivity), exhaustively.
* The Monte Carlo histogram is within a few standard errors of the exact pmf
  computed by enumeration.
* The histogram agrees, count for count, with the paper's per-boundary
  procedure on the same samples: classification against the complete
  reference sets of boundary m' followed by Stage 2 gives #{S <= m'}.
"""
import numpy as np
import pytest

from oracle import oracle as O
from workloads import systems as W

nx = pytest.importorskip("networkx")


def _flow_system(K=3, thresholds=(2, 4)):
    # two routes s=0 -> t=4 with a cross arc: flows 0..4 all occur
    n_nodes, arcs = 5, [(0, 1), (0, 2), (1, 3), (2, 3), (1, 2), (3, 4), (2, 4)]
    X = W.all_states(len(arcs), K)
    lv = np.zeros(X.shape[0], dtype=np.int64)
    for j, x in enumerate(X):
        G = nx.DiGraph()
        G.add_nodes_from(range(n_nodes))
        for (a, b), c in zip(arcs, x):
            G.add_edge(a, b, capacity=int(c))
        f = nx.maximum_flow_value(G, 0, 4)
        lv[j] = sum(f >= l for l in thresholds)
    pmf = np.random.default_rng(2).dirichlet(np.ones(K), size=len(arcs))
    return n_nodes, arcs, X, lv, pmf, list(thresholds)


def test_levels_of_every_state_match_networkx_flow():
    n_nodes, arcs, X, lv, pmf, thr = _flow_system()
    got = O.levels(O.PHI_ST_MAXFLOW_LEVELS, n_nodes, arcs, 0, 4, X, thr)
    assert np.array_equal(got, lv)
    assert set(np.unique(lv)) == {0, 1, 2}


def test_connectivity_levels_of_every_state_match_networkx():
    n_nodes, edges = W.grid_graph(2, 3)
    edges = edges + [(0, 4)]                      # 8 edges: some states are bridgeless
    X = W.all_states(len(edges), 2)
    for x in X:
        G = nx.Graph()
        G.add_nodes_from(range(n_nodes))
        G.add_edges_from(e for e, xe in zip(edges, x) if xe)
        want = 0 if not nx.is_connected(G) else min(2, nx.edge_connectivity(G))
        assert O.levels(O.PHI_GLOBAL_CONN_LEVEL, n_nodes, edges, 0, 0, x[None, :])[0] == want


def test_monte_carlo_pmf_within_error_of_the_exact_pmf():
    n_nodes, arcs, X, lv, pmf, thr = _flow_system()
    exact = np.array([O.exact_probability(pmf, X, lv == m) for m in range(3)])
    assert abs(exact.sum() - 1.0) < 1e-12
    N = 40000
    counts, _ = O.level_pmf(pmf, O.PHI_ST_MAXFLOW_LEVELS, n_nodes, arcs, 0, 4, 17, 0, N, 3, thr)
    assert counts.sum() == N
    se = np.sqrt(exact * (1 - exact) / N)
    assert np.all(np.abs(counts / N - exact) < 4.5 * se)


def test_histogram_equals_the_per_boundary_stage2_counts():
    n_nodes, arcs, X, lv, pmf, thr = _flow_system()
    n, K = len(arcs), 3
    N = 20000
    counts, levels = O.level_pmf(pmf, O.PHI_ST_MAXFLOW_LEVELS, n_nodes, arcs, 0, 4, 5, 1000, N, 3, thr)
    S = O.sample(pmf, 5, 1000, N)
    for m_prime in (0, 1):
        ref_L, ref_U = W.reference_sets_from_phi(lv, n, K, m_prime)
        # partial sets, so that Stage 2 has work to do
        lab, cnt = O.classify(S, ref_L[::2], ref_U[::3])
        res, n_lower = O.resolve(O.PHI_ST_MAXFLOW_LEVELS, n_nodes, arcs, 0, 4, S, lab, m_prime, thr)
        assert cnt[2] > 0
        assert cnt[0] + n_lower == counts[: m_prime + 1].sum()
        assert np.array_equal(np.isin(res, (0, 3)), levels <= m_prime)
