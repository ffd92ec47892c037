"""Pins for the Stage 1 oracle (reference-state search, Sec. 3.4-3.5) and the
system functions of the global-connectivity experiments (Sec. 4.3, 4.6).

Independent checks: networkx's connectivity, edge connectivity and maximum
flow; the complete reference sets of small systems enumerated state by state
(``workloads.systems.reference_sets_from_phi``, a single-step maximality
test); and the structure the paper's search guarantees for a coherent Phi
(the result dominates the start, lies on the start's side and is a boundary
state, i.e. an element of the complete set).
"""
import numpy as np
import pytest

from oracle import oracle as O
from workloads import systems as W

nx = pytest.importorskip("networkx")


def _random_simple_graph(rng, n_nodes, n_edges):
    pairs = [(a, b) for a in range(n_nodes) for b in range(a + 1, n_nodes)]
    pick = rng.choice(len(pairs), size=min(n_edges, len(pairs)), replace=False)
    return [pairs[k] for k in sorted(pick)]


def test_global_connectivity_phi_matches_networkx():
    rng = np.random.default_rng(11)
    checked = {0: 0, 1: 0, 2: 0}
    for _ in range(60):
        n_nodes = int(rng.integers(2, 9))
        edges = _random_simple_graph(rng, n_nodes, int(rng.integers(1, 3 * n_nodes)))
        for _ in range(12):
            x = (rng.random(len(edges)) < 0.75).astype(np.uint8)
            G = nx.Graph()
            G.add_nodes_from(range(n_nodes))
            G.add_edges_from(e for e, xe in zip(edges, x) if xe)
            conn = nx.is_connected(G)
            assert O.phi(O.PHI_GLOBAL_CONNECTIVITY, n_nodes, edges, 0, 0, x) == int(conn)
            level = 0 if not conn else min(2, nx.edge_connectivity(G))
            assert O.phi(O.PHI_GLOBAL_CONN_LEVEL, n_nodes, edges, 0, 0, x) == level
            checked[level] += 1
    assert min(checked.values()) > 20      # every level was exercised


def _grid():
    p = W.c1_grid()
    m = p.meta
    return p, m["n_nodes"], m["edges"], m["s"], m["t"], m["phi_all"]


def _state_index(x, K):
    return int(np.dot(np.asarray(x, dtype=np.int64), K ** np.arange(len(x) - 1, -1, -1)))


def test_boundary_search_on_the_grid_reaches_the_complete_sets():
    p, n_nodes, edges, s, t, phi_all = _grid()
    Lset = {bytes(r) for r in p.ref_L}
    Uset = {bytes(r) for r in p.ref_U}
    rng = np.random.default_rng(5)
    starts = np.concatenate([(rng.random((400, p.n)) < 0.8).astype(np.uint8), p.ref_L, p.ref_U])
    for x in starts:
        side, r, ev = O.boundary_search(O.PHI_ST_CONNECTIVITY, n_nodes, edges, s, t, x, 2)
        assert side == (0 if phi_all[_state_index(x, 2)] <= 0 else 1)
        if side == 0:
            assert bytes(r) in Lset and np.all(r >= x)
        else:
            assert bytes(r) in Uset and np.all(r <= x)
        assert 1 <= ev <= 1 + p.n
    # a reference state is its own search result
    for r in p.ref_L[:10]:
        assert np.array_equal(O.boundary_search(0, n_nodes, edges, s, t, r, 2)[1], r)


def _lex_extreme(X, phi, x, m_prime, lower):
    """Brute force: visiting components in index order makes the search return
    the lexicographically largest state y >= x with Phi(y) <= m' (lower side;
    component 0 most significant), and the smallest y <= x with Phi(y) >= m'+1
    (upper side).  Product order is lexicographic, so these are the largest /
    smallest enumeration indices of the feasible states."""
    if lower:
        ok = np.all(X >= x, axis=1) & (phi <= m_prime)
        return X[np.flatnonzero(ok).max()]
    ok = np.all(X <= x, axis=1) & (phi >= m_prime + 1)
    return X[np.flatnonzero(ok).min()]


def test_boundary_search_visits_components_in_index_order_on_the_grid():
    p, n_nodes, edges, s, t, phi_all = _grid()
    X = W.all_states(p.n, 2)
    rng = np.random.default_rng(6)
    for x in (rng.random((60, p.n)) < 0.8).astype(np.uint8):
        side, r, _ = O.boundary_search(O.PHI_ST_CONNECTIVITY, n_nodes, edges, s, t, x, 2)
        assert np.array_equal(r, _lex_extreme(X, phi_all, x, 0, side == 0))


def _small_flow_system(K=3, thresholds=(2, 4)):
    # two routes s=0 -> t=4 with a cross arc: flows 0..4 all occur
    n_nodes, arcs = 5, [(0, 1), (0, 2), (1, 3), (2, 3), (1, 2), (3, 4), (2, 4)]
    s, t = 0, 4
    X = W.all_states(len(arcs), K)
    phi = np.zeros(X.shape[0], dtype=np.int64)
    for j, x in enumerate(X):
        G = nx.DiGraph()
        G.add_nodes_from(range(n_nodes))
        for (a, b), c in zip(arcs, x):
            G.add_edge(a, b, capacity=int(c))
        f = nx.maximum_flow_value(G, s, t)
        phi[j] = sum(f >= l for l in thresholds)
    return n_nodes, arcs, s, t, X, phi, thresholds


@pytest.mark.parametrize("m_prime", [0, 1])
def test_boundary_search_multistate_flow_from_every_state(m_prime):
    K = 3
    n_nodes, arcs, s, t, X, phi, thr = _small_flow_system(K)
    n = len(arcs)
    ref_L, ref_U = W.reference_sets_from_phi(phi, n, K, m_prime)
    assert set(np.unique(phi)) == {0, 1, 2} and len(ref_L) >= 3 and len(ref_U) >= 3
    Lset = {bytes(r) for r in ref_L}
    Uset = {bytes(r) for r in ref_U}
    for j, x in enumerate(X):
        side, r, ev = O.boundary_search(O.PHI_ST_MAXFLOW_LEVELS, n_nodes, arcs, s, t, x, K, m_prime, thr)
        assert side == (0 if phi[j] <= m_prime else 1)
        if side == 0:
            assert bytes(r) in Lset and np.all(r >= x)
        else:
            assert bytes(r) in Uset and np.all(r <= x)
        assert 1 <= ev <= 1 + n * (K - 1)
        assert np.array_equal(r, _lex_extreme(X, phi, x, m_prime, side == 0))


def test_nondominated_keeps_exactly_the_maximal_and_minimal_states():
    p, n_nodes, edges, s, t, phi_all = _grid()
    X = W.all_states(p.n, 2)
    rng = np.random.default_rng(8)
    for upper, ref, mask in ((False, p.ref_L, phi_all == 0), (True, p.ref_U, phi_all == 1)):
        pool = X[mask]
        extra = pool[rng.choice(pool.shape[0], 1500, replace=False)]
        rows = np.concatenate([extra, ref, ref[:7], extra[:5]])    # with duplicates
        rows = rows[rng.permutation(rows.shape[0])]
        keep = O.nondominated(rows, upper)
        kept = rows[keep]
        assert {bytes(r) for r in kept} == {bytes(r) for r in ref}
        assert kept.shape[0] == ref.shape[0]                      # one copy of each
        # the first occurrence of each reference is the one kept
        first = {}
        for j, r in enumerate(rows):
            first.setdefault(bytes(r), j)
        assert sorted(np.flatnonzero(keep)) == sorted(first[bytes(r)] for r in ref)


def test_stage1_on_the_grid_converges_to_boundary_states():
    p, n_nodes, edges, s, t, phi_all = _grid()
    N = 4000
    res = O.stage1(p.pmf, O.PHI_ST_CONNECTIVITY, n_nodes, edges, s, t, seed=3, N=N, max_starts=4,
                   eps_u=0.5 / N, R_max=1000, max_rounds=200)
    assert res["stop"] == 0 and res["history"][-1][0] == 0
    Lset = {bytes(r) for r in p.ref_L}
    Uset = {bytes(r) for r in p.ref_U}
    assert all(bytes(r) in Lset for r in res["ref_L"])
    assert all(bytes(r) in Uset for r in res["ref_U"])
    assert O.nondominated(res["ref_L"], False).all() and O.nondominated(res["ref_U"], True).all()
    # references only accumulate: boundary states never dominate one another
    R = [h[1] + h[2] for h in res["history"]]
    assert all(b >= a for a, b in zip(R, R[1:]))
    # the found sets leave little unclassified probability over the whole space
    X = W.all_states(p.n, 2)
    lab, _ = O.classify(X, res["ref_L"], res["ref_U"])
    pu = O.exact_probability(p.pmf, X, lab == 2)
    assert pu < 2e-3


def test_stage1_stops_at_the_reference_limit():
    p, n_nodes, edges, s, t, _ = _grid()
    res = O.stage1(p.pmf, O.PHI_ST_CONNECTIVITY, n_nodes, edges, s, t, seed=4, N=2000, max_starts=6,
                   eps_u=0.5 / 2000, R_max=10, max_rounds=50)
    assert res["stop"] == 1
    assert res["ref_L"].shape[0] + res["ref_U"].shape[0] == 10


def test_stage1_multistate_flow_finds_complete_set_elements():
    K = 3
    n_nodes, arcs, s, t, X, phi, thr = _small_flow_system(K)
    n = len(arcs)
    rng = np.random.default_rng(2)
    pmf = rng.dirichlet(np.ones(K), size=n)
    ref_L, ref_U = W.reference_sets_from_phi(phi, n, K, 1)
    res = O.stage1(pmf, O.PHI_ST_MAXFLOW_LEVELS, n_nodes, arcs, s, t, seed=9, N=3000, max_starts=3,
                   eps_u=0.5 / 3000, R_max=10_000, max_rounds=300, m_prime=1, thresholds=thr)
    assert res["stop"] == 0
    assert {bytes(r) for r in res["ref_L"]} <= {bytes(r) for r in ref_L}
    assert {bytes(r) for r in res["ref_U"]} <= {bytes(r) for r in ref_U}


def test_search_order_is_a_uniform_permutation():
    seen = {}
    for h in range(24000):
        o = O.search_order(7, h, 4)
        assert sorted(o.tolist()) == [0, 1, 2, 3]
        seen[tuple(o)] = seen.get(tuple(o), 0) + 1
    assert len(seen) == 24
    counts = np.array(list(seen.values()), dtype=np.float64)
    chi2 = ((counts - 1000.0) ** 2 / 1000.0).sum()
    assert chi2 < 49.7                     # 99.9% quantile of chi^2 with 23 degrees of freedom
    big = O.search_order(3, 12345, 300)
    assert sorted(big.tolist()) == list(range(300))
    assert not np.array_equal(big, O.search_order(3, 12346, 300))
    assert not np.array_equal(big, O.search_order(4, 12345, 300))


def test_permuted_search_is_the_lexicographic_extreme_in_the_visiting_order():
    p, n_nodes, edges, s, t, phi_all = _grid()
    X = W.all_states(p.n, 2)
    rng = np.random.default_rng(16)
    for k, x in enumerate((rng.random((40, p.n)) < 0.75).astype(np.uint8)):
        order = O.search_order(9, k, p.n)
        side, r, _ = O.boundary_search(O.PHI_ST_CONNECTIVITY, n_nodes, edges, s, t, x, 2, order=order)
        # component order[0] is the most significant: relabel and reuse the index-order characterisation
        Xp = X[:, order]
        key = Xp.astype(np.int64) @ (2 ** np.arange(p.n - 1, -1, -1)).astype(np.int64)
        if side == 0:
            ok = np.all(X >= x, axis=1) & (phi_all <= 0)
            want = X[np.flatnonzero(ok)[np.argmax(key[ok])]]
        else:
            ok = np.all(X <= x, axis=1) & (phi_all >= 1)
            want = X[np.flatnonzero(ok)[np.argmin(key[ok])]]
        assert np.array_equal(r, want)


def test_stage1_permuted_order_converges_to_boundary_states():
    p, n_nodes, edges, s, t, _ = _grid()
    N = 4000
    res = O.stage1(p.pmf, O.PHI_ST_CONNECTIVITY, n_nodes, edges, s, t, seed=3, N=N, max_starts=4,
                   eps_u=0.5 / N, R_max=1000, max_rounds=200, order=O.SEARCH_PERMUTED)
    assert res["stop"] == 0
    assert all(bytes(r) in {bytes(q) for q in p.ref_L} for r in res["ref_L"])
    assert all(bytes(r) in {bytes(q) for q in p.ref_U} for r in res["ref_U"])


def test_global_lowering_search_is_reverse_order_kruskal():
    """The search that lowers a connected state under global connectivity (remove
    each working edge, in the visiting order, if the graph stays connected)
    keeps exactly the spanning tree that Kruskal's algorithm builds from the
    working edges taken in reverse visiting order: reverse deletion with the
    visit positions as distinct weights.  The CUDA search uses this one-pass
    form; here the oracle's literal step-by-step search is compared with an
    independent union-find Kruskal on random connected graphs and orders, and
    its Phi-evaluation count is 1 + the number of working edges."""
    rng = np.random.default_rng(12)
    for trial in range(40):
        nn = int(rng.integers(4, 14))
        # a random spanning tree plus random extra edges
        edges = [(int(rng.integers(0, v)), v) for v in range(1, nn)]
        for _ in range(int(rng.integers(0, 3 * nn))):
            a, b = (int(v) for v in rng.choice(nn, size=2, replace=False))
            edges.append((a, b))
        n = len(edges)
        x = np.ones(n, dtype=np.uint8)
        x[n - 1 - rng.choice(n - (nn - 1), size=int(rng.integers(0, n - nn + 2)), replace=False)] = 0
        x[: nn - 1] = 1    # the spanning tree stays working: the start is connected
        order = rng.permutation(n).astype(np.int32)
        side, ref, ev = O.boundary_search(2, nn, edges, 0, 0, x, 2, order=order)
        assert side == 1
        parent = list(range(nn))

        def find(v):
            while parent[v] != v:
                parent[v] = parent[parent[v]]
                v = parent[v]
            return v
        want = np.zeros(n, dtype=np.uint8)
        for i in order[::-1]:
            if x[i]:
                ru, rv = find(edges[i][0]), find(edges[i][1])
                if ru != rv:
                    parent[ru] = rv
                    want[i] = 1
        assert np.array_equal(ref, want), trial
        assert int(ref.sum()) == nn - 1
        assert ev == 1 + int(x.sum())
