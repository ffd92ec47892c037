"""GPU parity of Stage 1 on the device (Sec. 3.4-3.5) and of the global
connectivity system functions (Sec. 4.3, 4.6), through the C ABI:

* rsr_resolve with Phi = global connectivity / connectivity level: labels,
  counts and the lower-index set equal the oracle's;
* rsr_boundary_search: every reference and side equals the oracle's search
  from the same sample, and the total number of Phi evaluations is equal;
* rsr_nondominated: keep masks equal the oracle's on sets with duplicates and
  dominated rows, both sides;
* rsr_stage1: the round history (n_u, R_L, R_U, starts), the stop reason, the
  Phi evaluations and the final reference buffers, row by row, equal the
  oracle's Stage 1 loop; at the C2 size the references found are boundary
  states (checked one by one by the oracle's Phi).
"""
import numpy as np
import pytest
import torch

import workloads as W
from helpers import POPC, TC, make_session
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _grid():
    p = W.c1_grid()
    m = p.meta
    return p, m["n_nodes"], m["edges"], m["s"], m["t"]


def _random_graph(seed, n_nodes=30, n_edges=80):
    rng = np.random.default_rng(seed)
    # a spanning path keeps the graph connected at full state, then random extra edges
    order = rng.permutation(n_nodes)
    edges = {(int(min(a, b)), int(max(a, b))) for a, b in zip(order[:-1], order[1:])}
    while len(edges) < n_edges:
        a, b = (int(v) for v in rng.integers(0, n_nodes, 2))
        if a != b:
            edges.add((min(a, b), max(a, b)))
    return n_nodes, sorted(edges)


def _small_flow(K=3):
    # two routes s=0 -> t=4 with a cross arc: flows 0..4 all occur
    n_nodes, arcs = 5, [(0, 1), (0, 2), (1, 3), (2, 3), (1, 2), (3, 4), (2, 4)]
    pmf = np.random.default_rng(2).dirichlet(np.ones(K), size=len(arcs))
    return n_nodes, arcs, 0, 4, pmf, (2, 4)


# ---------------------------------------------------------------- Stage 2 with the global kinds
@pytest.mark.parametrize("kind,m_prime,n_edges,p_f", [(2, 0, 40, 0.12), (3, 0, 40, 0.12), (3, 1, 80, 0.2)])
def test_resolve_global_connectivity_kinds(rsr, kind, m_prime, n_edges, p_f):
    nn, edges = _random_graph(7, 30, n_edges)
    n = len(edges)
    pmf = W.binary_pmf(np.full(n, p_f))
    # one trivial lower reference (everything failed): nearly every sample stays unclassified
    prob = W.Problem("global", pmf, np.zeros((1, n), np.uint8), np.zeros((0, n), np.uint8))
    N = 8000
    sess = make_session(rsr, prob)
    out = sess.classify(5, 100, N, labels=True, grad=False)
    labels = out["labels"]
    u_idx, c2 = rsr.rsr_resolve(sess.problem, rsr.System(kind, nn, edges, 0, 0, (), m_prime), 5, 100, N, labels,
                                sess.ws)
    torch.cuda.synchronize()
    X = O.sample(pmf, 5, 100, N)
    lab, cnt = O.classify(X, prob.ref_L, prob.ref_U)
    res, n_lower = O.resolve(kind, nn, edges, 0, 0, X, lab, m_prime=m_prime)
    assert np.array_equal(labels.cpu().numpy(), res)
    assert c2.cpu().tolist() == [n_lower, int(cnt[2]) - n_lower]
    assert np.array_equal(np.sort(u_idx[:n_lower].cpu().numpy()), np.nonzero(res == 3)[0])
    assert 0.2 * N < n_lower < 0.8 * N            # both outcomes are frequent
    assert rsr.rsr_workspace_status(sess.ws)[1] == 0


# ---------------------------------------------------------------- boundary search
def _check_search(rsr, pmf, kind, nn, edges, s, t, seed, offset, starts, m_prime=0, thr=(), order=0):
    K = pmf.shape[1]
    P = rsr.Problem(pmf, np.zeros((0, pmf.shape[0]), np.uint8), np.ones((1, pmf.shape[0]), np.uint8) * (K - 1))
    sys_ = rsr.System(kind, nn, edges, s, t, thr, m_prime)
    st = torch.as_tensor(np.asarray(starts, dtype=np.int64), device="cuda")
    refs, side, ev = rsr.rsr_boundary_search(P, sys_, seed, offset, st, order=order)
    torch.cuda.synchronize()
    refs, side, ev = refs.cpu().numpy(), side.cpu().numpy(), int(ev.item())
    total = 0
    for j, h in enumerate(starts):
        x = O.sample(pmf, seed, offset + int(h), 1)[0]
        od = O.search_order(seed, offset + int(h), pmf.shape[0]) if order else None
        sd, r, e = O.boundary_search(kind, nn, edges, s, t, x, K, m_prime, list(thr) if thr else None, od)
        assert side[j] == sd, j
        assert np.array_equal(refs[j], r), j
        total += e
    assert ev == total


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("kind", [0, 2, 3])
def test_boundary_search_grid(rsr, kind, order):
    p, nn, edges, s, t = _grid()
    pmf = W.binary_pmf(np.full(p.n, 0.3))
    m_prime = 1 if kind == 3 else 0
    _check_search(rsr, pmf, kind, nn, edges, s, t, 11, 7, np.arange(0, 600, 3), m_prime, order=order)


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("m_prime", [0, 1])
def test_boundary_search_small_flow(rsr, m_prime, order):
    nn, arcs, s, t, pmf, thr = _small_flow()
    _check_search(rsr, pmf, 1, nn, arcs, s, t, 3, 0, np.arange(257), m_prime, thr, order=order)


@pytest.mark.parametrize("order", [0, 1])
def test_boundary_search_c4_flow(rsr, order):
    import workloads.large as L
    p = L.c4_flow(0)
    m = p.meta
    _check_search(rsr, p.pmf, 1, m["n_nodes"], m["arcs"], m["s"], m["t"], 4, 5000, np.arange(0, 130 * 7, 7), 0,
                  (m["l1"], m["l2"]), order=order)


@pytest.mark.parametrize("order", [0, 1])
def test_boundary_search_c2_graph(rsr, order):
    import workloads.large as L
    p = L.c2_rgg()
    m = p.meta
    _check_search(rsr, p.pmf, 0, m["n_nodes"], m["edges"], m["s"], m["t"], 1, 0, np.arange(0, 200 * 13, 13),
                  order=order)


# ---------------------------------------------------------------- non-dominance
@pytest.mark.parametrize("upper", [False, True])
@pytest.mark.parametrize("n,K,R", [(17, 2, 700), (50, 4, 3000), (300, 2, 1100), (13, 16, 513)])
def test_nondominated_matches_oracle(rsr, upper, n, K, R):
    rng = np.random.default_rng(n * 7 + K + int(upper))
    base = rng.integers(0, K, size=(R // 2, n)).astype(np.uint8)
    # dominated variants: move a few entries towards the dominated side
    var = base.copy()
    for r in range(var.shape[0]):
        idx = rng.choice(n, size=min(n, 3), replace=False)
        var[r, idx] = (np.maximum(var[r, idx].astype(int) - 1, 0) if not upper
                       else np.minimum(var[r, idx].astype(int) + 1, K - 1)).astype(np.uint8)
    rows = np.concatenate([base, var[: R - base.shape[0] - 20], base[:20]])    # plus duplicates
    rows = rows[rng.permutation(rows.shape[0])]
    keep, n_keep = rsr.rsr_nondominated(torch.as_tensor(rows, device="cuda"), K, upper)
    torch.cuda.synchronize()
    want = O.nondominated(rows, upper)
    assert np.array_equal(keep.cpu().numpy().astype(bool), want)
    assert int(n_keep.item()) == int(want.sum())
    assert 0 < want.sum() < rows.shape[0]


def test_nondominated_empty_and_single(rsr):
    keep, n_keep = rsr.rsr_nondominated(torch.zeros((0, 5), dtype=torch.uint8, device="cuda"), 3, False)
    assert keep.numel() == 0 and int(n_keep.item()) == 0
    keep, n_keep = rsr.rsr_nondominated(torch.ones((1, 5), dtype=torch.uint8, device="cuda"), 3, True)
    assert keep.cpu().tolist() == [1] and int(n_keep.item()) == 1


# ---------------------------------------------------------------- Stage 1 loop
def _check_stage1(rsr, pmf, kind, nn, edges, s, t, seed, N, B, eps_u, R_max, rounds, m_prime=0, thr=(),
                  path=POPC, ref_L=None, ref_U=None, order=0):
    sys_ = rsr.System(kind, nn, edges, s, t, thr, m_prime)
    got = rsr.rsr_stage1(pmf, sys_, seed, N, B, eps_u, R_max, rounds, ref_L=ref_L, ref_U=ref_U, path=path,
                         order=order)
    want = O.stage1(pmf, kind, nn, edges, s, t, seed, N, B, eps_u, R_max, rounds, m_prime=m_prime,
                    thresholds=list(thr) if thr else None, ref_L=ref_L, ref_U=ref_U, order=order)
    assert got["stop"] == want["stop"]
    assert np.array_equal(got["history"], np.array(want["history"], dtype=np.int64).reshape(-1, 4))
    assert np.array_equal(got["ref_L"].cpu().numpy(), want["ref_L"])
    assert np.array_equal(got["ref_U"].cpu().numpy(), want["ref_U"])
    assert got["phi_evals"] == want["phi_evals"]
    return got


def test_stage1_grid_converges_like_the_oracle(rsr):
    p, nn, edges, s, t = _grid()
    got = _check_stage1(rsr, p.pmf, 0, nn, edges, s, t, 3, 4000, 4, 0.5 / 4000, 1000, 200)
    assert got["stop"] == 0


@pytest.mark.parametrize("path", [POPC, TC])
def test_stage1_grid_many_starts_per_round(rsr, path):
    p, nn, edges, s, t = _grid()
    pmf = W.binary_pmf(np.full(p.n, 0.25))
    _check_stage1(rsr, pmf, 0, nn, edges, s, t, 8, 3000, 64, 1e-3, 1000, 30, path=path)


def test_stage1_reference_limit_and_initial_references(rsr):
    p, nn, edges, s, t = _grid()
    got = _check_stage1(rsr, p.pmf, 0, nn, edges, s, t, 4, 2000, 6, 0.5 / 2000, 10, 50)
    assert got["stop"] == 1 and got["ref_L"].shape[0] + got["ref_U"].shape[0] == 10
    # starting from part of the complete sets
    _check_stage1(rsr, p.pmf, 0, nn, edges, s, t, 5, 3000, 5, 0.5 / 3000, 500, 40, ref_L=p.ref_L[:9],
                  ref_U=p.ref_U[:4])


def test_stage1_round_limit(rsr):
    p, nn, edges, s, t = _grid()
    pmf = W.binary_pmf(np.full(p.n, 0.3))
    got = _check_stage1(rsr, pmf, 0, nn, edges, s, t, 6, 2000, 3, 1e-9, 1000, 4)
    assert got["stop"] == 2 and got["rounds"] == 4


@pytest.mark.parametrize("m_prime", [0, 1])
def test_stage1_multistate_flow(rsr, m_prime):
    nn, arcs, s, t, pmf, thr = _small_flow()
    _check_stage1(rsr, pmf, 1, nn, arcs, s, t, 9, 3000, 3, 0.5 / 3000, 10000, 300, m_prime, thr)


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("kind,m_prime", [(2, 0), (3, 1)])
def test_stage1_global_connectivity_grid(rsr, kind, m_prime, order):
    p, nn, edges, s, t = _grid()
    pmf = W.binary_pmf(np.full(p.n, 0.05))
    _check_stage1(rsr, pmf, kind, nn, edges, s, t, 12, 5000, 16, 1e-3, 3000, 25, m_prime, order=order)


@pytest.mark.parametrize("order", [0, 1])
def test_stage1_c2_graph_parity(rsr, order):
    import workloads.large as L
    p = L.c2_rgg()
    m = p.meta
    _check_stage1(rsr, p.pmf, 0, m["n_nodes"], m["edges"], m["s"], m["t"], 2, 20000, 64, 1e-4, 2000, 6,
                  order=order)


def test_stage1_multistate_flow_permuted(rsr):
    nn, arcs, s, t, pmf, thr = _small_flow()
    _check_stage1(rsr, pmf, 1, nn, arcs, s, t, 9, 3000, 3, 0.5 / 3000, 10000, 300, 1, thr, order=1)


def test_stage1_c2_full_size_finds_boundary_states(rsr):
    """Bench configuration: rounds of 10^6 samples, up to 1024 searches per
    round, until the unclassified fraction is below 10^-5.  Every reference is
    a boundary state: Phi <= m' at r and Phi > m' after any single increase
    (lower), and symmetrically for upper references (checked on a sample)."""
    import workloads.large as L
    p = L.c2_rgg()
    m = p.meta
    nn, edges, s, t = m["n_nodes"], m["edges"], m["s"], m["t"]
    got = rsr.rsr_stage1(p.pmf, rsr.System(0, nn, edges, s, t), 2, 1_000_000, 1024, 1e-5, 20000, 40)
    hist = got["history"]
    assert got["rounds"] == hist.shape[0] and hist[0][0] == 1_000_000
    assert hist[-1][0] < hist[1][0] / 20                    # the unclassified count falls steeply
    assert got["stop"] != 0 or hist[-1][0] < 10
    rng = np.random.default_rng(0)
    for refs, lower in ((got["ref_L"].cpu().numpy(), True), (got["ref_U"].cpu().numpy(), False)):
        assert O.nondominated(refs, not lower).all()
        for r in refs[rng.choice(refs.shape[0], min(40, refs.shape[0]), replace=False)]:
            assert (O.phi(0, nn, edges, s, t, r) <= 0) == lower
            for i in range(p.n):
                if (lower and r[i] == 1) or (not lower and r[i] == 0):
                    continue
                y = r.copy()
                y[i] = 1 - y[i]
                assert (O.phi(0, nn, edges, s, t, y) <= 0) != lower


# ---------------------------------------------------------------- at the size limits
def _big_graph(seed, n_nodes, n_edges):
    rng = np.random.default_rng(seed)
    order = rng.permutation(n_nodes)
    edges = [(int(a), int(b)) for a, b in zip(order[:-1], order[1:])]      # spanning path
    seen = {tuple(sorted(e)) for e in edges}
    while len(edges) < n_edges:
        a, b = (int(v) for v in rng.integers(0, n_nodes, 2))
        if a != b and tuple(sorted((a, b))) not in seen:
            seen.add(tuple(sorted((a, b))))
            edges.append((a, b))
    return edges


@pytest.mark.parametrize("kind", [0, 2])
def test_search_and_resolve_at_1024_nodes_and_components(rsr, kind):
    """n_nodes = 1024 and n = 1024 edges: the shared-memory graph, node bitsets,
    parent words and adjacency lists at their limits."""
    nn = 1024
    edges = _big_graph(5, nn, 1024)
    pmf = W.binary_pmf(np.full(len(edges), 0.003))
    s, t = (0, nn - 1) if kind == 0 else (0, 0)
    _check_search(rsr, pmf, kind, nn, edges, s, t, 3, 0, np.arange(0, 24 * 5, 5), order=1)
    prob = W.Problem("big", pmf, np.zeros((1, len(edges)), np.uint8), np.zeros((0, len(edges)), np.uint8))
    N = 3000
    sess = make_session(rsr, prob)
    out = sess.classify(2, 0, N, labels=True, grad=False)
    _, c2 = rsr.rsr_resolve(sess.problem, rsr.System(kind, nn, edges, s, t), 2, 0, N, out["labels"], sess.ws)
    torch.cuda.synchronize()
    X = O.sample(pmf, 2, 0, N)
    lab, _ = O.classify(X, prob.ref_L, prob.ref_U)
    res, n_lower = O.resolve(kind, nn, edges, s, t, X, lab)
    assert np.array_equal(out["labels"].cpu().numpy(), res)
    assert int(c2[0].item()) == n_lower


def test_search_max_flow_at_1024_thermometer_bits(rsr):
    """K = 3, n = 512 arcs: n(K-1) = 1024 thermometer bits, the sampler's limit."""
    rng = np.random.default_rng(9)
    nn = 200
    arcs = []
    seen = set()
    while len(arcs) < 512:
        a, b = (int(v) for v in rng.integers(0, nn, 2))
        if a != b and (a, b) not in seen:
            seen.add((a, b))
            arcs.append((a, b))
    pmf = rng.dirichlet(np.ones(3), size=512)
    deg = np.bincount(np.array(arcs).ravel(), minlength=nn)
    s = int(np.argmax(deg))
    t = int(np.argsort(deg)[-2])
    for m_prime in (0, 1):
        _check_search(rsr, pmf, 1, nn, arcs, s, t, 6, 0, np.arange(40), m_prime, (2, 4), order=1)


@pytest.mark.parametrize("upper", [False, True])
def test_nondominated_at_32_words(rsr, upper):
    rng = np.random.default_rng(31)
    rows = rng.integers(0, 2, size=(700, 1024)).astype(np.uint8)
    rows[::7] = rows[1::7] if upper else rows[::7]          # duplicates
    rows[3::11] = np.maximum(rows[3::11], rows[4::11][: rows[3::11].shape[0]]) if not upper else rows[3::11]
    keep, n_keep = rsr.rsr_nondominated(torch.as_tensor(rows, device="cuda"), 2, upper)
    torch.cuda.synchronize()
    want = O.nondominated(rows, upper)
    assert np.array_equal(keep.cpu().numpy().astype(bool), want)
    assert int(n_keep.item()) == int(want.sum())


def test_boundary_search_without_starts(rsr):
    p, nn, edges, s, t = _grid()
    P = rsr.Problem(p.pmf, p.ref_L, p.ref_U)
    refs, side, ev = rsr.rsr_boundary_search(P, rsr.System(0, nn, edges, s, t), 1, 0,
                                             torch.zeros(0, dtype=torch.int64, device="cuda"))
    torch.cuda.synchronize()
    assert refs.shape == (0, p.n) and side.numel() == 0 and int(ev.item()) == 0
