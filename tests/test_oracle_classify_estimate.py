"""Pins of the oracle's classification (Algorithm 1) and estimators (Sec. 3.3).

* the paper's worked example (Sec. 3.2): the printed encodings give violation
  counts V = H Rbar^T, and "some V = 0" must agree with the oracle's direct
  componentwise test;
* the 3x4 grid: every one of the 2^17 states, with complete path/cut
  references, is labelled exactly as networkx's s-t connectivity says, and
  nothing is unclassified;
* the exact grid failure probability, by enumeration with exact rationals;
* closed forms for series, parallel and k-out-of-n systems;
* c.o.v. against a 50-digit decimal evaluation of the formula;
* coherence invariants (partition, reference order and duplicates, adding
  references, monotonicity, precedence).
"""
import json
import os
from decimal import Decimal, getcontext
from fractions import Fraction
from math import comb

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _nx_phi_all(n_nodes, edges, s, t):
    nx = pytest.importorskip("networkx")
    n = len(edges)
    phi = np.zeros(1 << n, dtype=np.int32)
    for idx in range(1 << n):
        G = nx.Graph()
        G.add_nodes_from(range(n_nodes))
        for e, (u, v) in enumerate(edges):
            if (idx >> (n - 1 - e)) & 1:
                G.add_edge(u, v)
        phi[idx] = 1 if nx.has_path(G, s, t) else 0
    return phi


@pytest.fixture(scope="module")
def grid():
    p = W.c1_grid()
    phi_nx = _nx_phi_all(p.meta["n_nodes"], p.meta["edges"], p.meta["s"], p.meta["t"])
    return p, phi_nx


# ---------------------------------------------------------------- worked example
def test_worked_example_encodings_and_labels():
    g = json.load(open(os.path.join(GOLD, "worked_example.json")))
    K = g["K"]
    ref_L = np.array(g["ref_L"], dtype=np.uint8)
    ref_U = np.array(g["ref_U"], dtype=np.uint8)
    X = np.array(g["samples"], dtype=np.uint8)
    labels, counts = O.classify(X, ref_L, ref_U)
    assert labels.tolist() == g["expected_labels"]
    # the paper's matrix form: V_{h,r} = flat(H_h) . flat(1 - R_r); classified iff some V = 0
    H = [np.array(h) for h in g["H_encoded"]]
    RL = [np.array(r) for r in g["R_L_encoded"]]
    RU = [np.array(r) for r in g["R_U_encoded"]]
    for h, Hm in enumerate(H):
        VL = [int((Hm.ravel() * (1 - R.ravel())).sum()) for R in RL]
        VU = [int((Hm.ravel() * (1 - R.ravel())).sum()) for R in RU]
        lab = 0 if 0 in VL else (1 if 0 in VU else 2)
        assert lab == labels[h]
    # printed encodings are the thermometer / one-hot maps of the printed states
    for r, R in zip(ref_L, RL):
        assert np.array_equal(R, np.array([[1 if m <= r[i] else 0 for m in range(K)] for i in range(2)]))
    for r, R in zip(ref_U, RU):
        assert np.array_equal(R, np.array([[1 if m >= r[i] else 0 for m in range(K)] for i in range(2)]))
    # Sec. 3.3: V(H_1, .) = (1, 1, 1) and V(H_2, R^U_1) = 0
    assert [int((H[0].ravel() * (1 - R.ravel())).sum()) for R in RL + RU] == [1, 1, 1]
    assert int((H[1].ravel() * (1 - RL[0].ravel())).sum()) == 2
    assert int((H[1].ravel() * (1 - RU[0].ravel())).sum()) == 0


def test_worked_example_counts():
    g = json.load(open(os.path.join(GOLD, "worked_example.json")))["count_example"]
    est = O.estimate(g["counts"], g["H"])
    assert [est["pL"], est["pU"], est["pu"]] == g["p"]


# ---------------------------------------------------------------- grid, exhaustive
def test_grid_reference_counts(grid):
    p, _ = grid
    assert (p.R_U, p.R_L) == (38, 81)


def test_grid_exhaustive_classification_equals_phi(grid):
    p, phi_nx = grid
    X = O.all_states(p.n, 2)
    labels, counts = O.classify(X, p.ref_L, p.ref_U)
    assert counts[2] == 0
    assert np.array_equal(labels, np.where(phi_nx == 0, 0, 1).astype(np.uint8))


def test_grid_exact_probability(grid):
    p, phi_nx = grid
    X = O.all_states(p.n, 2)
    # exact rational: sum over failed states of 0.1^#down 0.9^#up
    down = (X == 0).sum(axis=1)
    total = Fraction(0)
    for d in range(p.n + 1):
        cnt = int(np.sum((phi_nx == 0) & (down == d)))
        total += cnt * Fraction(1, 10) ** d * Fraction(9, 10) ** (p.n - d)
    assert total == Fraction(274067481066877, 10 ** 16)
    assert O.exact_probability(p.pmf, X, phi_nx == 0) == pytest.approx(float(total), rel=1e-13)


def test_grid_monte_carlo_estimate_within_4se(grid):
    p, _ = grid
    N = 100000
    X = O.sample(p.pmf, seed=1, offset=0, N=N)
    labels, counts = O.classify(X, p.ref_L, p.ref_U)
    est = O.estimate(counts, N)
    exact = 274067481066877 / 10 ** 16
    se = np.sqrt(exact * (1 - exact) / N)
    assert counts.sum() == N and counts[2] == 0
    assert abs(est["pL"] - exact) <= 4 * se


# ---------------------------------------------------------------- closed forms
def _mc(problem, N, seed):
    X = O.sample(problem.pmf, seed=seed, offset=0, N=N)
    labels, counts = O.classify(X, problem.ref_L, problem.ref_U)
    return X, labels, counts


def test_series_closed_form():
    p_fail = np.array([0.05, 0.1, 0.2, 0.02, 0.15])
    prob = W.series_system(p_fail)
    N = 60000
    _, _, counts = _mc(prob, N, 5)
    assert counts[2] == 0
    exact_up = float(np.prod(1 - p_fail))
    assert abs(counts[1] / N - exact_up) <= 4 * np.sqrt(exact_up * (1 - exact_up) / N)


def test_parallel_closed_form():
    p_fail = np.array([0.5, 0.6, 0.7, 0.4])
    prob = W.parallel_system(p_fail)
    N = 60000
    _, _, counts = _mc(prob, N, 6)
    assert counts[2] == 0
    exact_down = float(np.prod(p_fail))
    assert abs(counts[0] / N - exact_down) <= 4 * np.sqrt(exact_down * (1 - exact_down) / N)


def test_k_out_of_n_binomial_tail():
    n, k, pf = 7, 4, 0.3
    prob = W.k_out_of_n_system(n, k, pf)
    N = 60000
    _, _, counts = _mc(prob, N, 7)
    assert counts[2] == 0
    exact_up = sum(comb(n, j) * (1 - pf) ** j * pf ** (n - j) for j in range(k, n + 1))
    assert abs(counts[1] / N - exact_up) <= 4 * np.sqrt(exact_up * (1 - exact_up) / N)


def test_k_out_of_n_exhaustive():
    n, k = 6, 3
    prob = W.k_out_of_n_system(n, k, 0.5)
    X = O.all_states(n, 2)
    labels, _ = O.classify(X, prob.ref_L, prob.ref_U)
    assert np.array_equal(labels, np.where(X.sum(1) >= k, 1, 0).astype(np.uint8))


# ---------------------------------------------------------------- estimator arithmetic
@pytest.mark.parametrize("counts,N,nul", [
    ((3, 4, 3), 10, 0), ((1, 999998, 1), 10 ** 6, 1), ((274067, 725933, 0), 10 ** 7, 0),
    ((0, 5, 5), 10, 2), ((10, 0, 0), 10, 0), ((12345, 67890, 777), 81012, 300),
])
def test_estimate_against_decimal(counts, N, nul):
    getcontext().prec = 50
    est = O.estimate(counts, N, nul)
    exact = {
        "pL": Decimal(counts[0]) / N, "pU": Decimal(counts[1]) / N, "pu": Decimal(counts[2]) / N,
        "P_lower": Decimal(counts[0] + nul) / N, "P_upper": Decimal(counts[1] + counts[2] - nul) / N,
    }
    for key, val in exact.items():
        assert est[key] == float(val)
        cov_key = {"pL": "cov_pL", "pU": "cov_pU", "pu": "cov_pu",
                   "P_lower": "cov_lower", "P_upper": "cov_upper"}[key]
        if val == 0:
            assert est[cov_key] == float("inf")
        else:
            # delta = sqrt((1-p)/(H p)) evaluated exactly from the fp64 p (1 - p is then exact
            # in fp64 too); the fp64 result is within a few ulps of that value
            pr = Decimal(float(val))
            cov = ((1 - pr) / (N * pr)).sqrt()
            assert est[cov_key] == pytest.approx(float(cov), rel=4e-16, abs=0)


def test_cov_special_values():
    est = O.estimate((0, 10, 0), 10)
    assert est["cov_pL"] == float("inf") and est["cov_pU"] == 0.0


# ---------------------------------------------------------------- invariants
def test_precedence_lower_wins():
    # inconsistent references: upper (1,0) lies below lower (1,1); the sample (1,0) satisfies both
    ref_L = np.array([[1, 1]], dtype=np.uint8)
    ref_U = np.array([[1, 0]], dtype=np.uint8)
    labels, _ = O.classify(np.array([[1, 0], [0, 1], [1, 1]], dtype=np.uint8), ref_L, ref_U)
    assert labels.tolist() == [0, 0, 0]
    assert O.count_overlaps(ref_L, ref_U) == 1
    p = W.c1_grid()
    assert O.count_overlaps(p.ref_L, p.ref_U) == 0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_invariants_random_multistate(seed):
    prob = W.random_small_system(n=5, K=4, M_S=3, seed=seed)
    rng = np.random.default_rng(seed)
    X = O.sample(prob.pmf, seed=seed, offset=0, N=3000)
    labels, counts = O.classify(X, prob.ref_L, prob.ref_U)
    assert counts.sum() == X.shape[0]
    assert np.array_equal(np.bincount(labels, minlength=3), counts)
    # complete references: labels equal Phi <= m'
    stride = prob.K ** np.arange(prob.n - 1, -1, -1)
    phi = prob.meta["phi_all"][X.astype(np.int64) @ stride]
    assert counts[2] == 0
    assert np.array_equal(labels, np.where(phi <= prob.meta["m_prime"], 0, 1))
    # reference order and duplicates do not change labels
    pL = prob.ref_L[rng.permutation(prob.R_L)]
    pU = np.concatenate([prob.ref_U, prob.ref_U[: max(1, prob.R_U // 2)]])[::-1]
    assert np.array_equal(O.classify(X, pL, pU)[0], labels)
    # a partial reference set never classifies more; adding references never grows I^u
    half_L, half_U = prob.ref_L[: prob.R_L // 2], prob.ref_U[: prob.R_U // 2]
    lab_half, c_half = O.classify(X, half_L, half_U)
    assert c_half[2] >= counts[2]
    assert np.all((lab_half == 2) | (lab_half == labels))
    # monotonicity: raising a component never moves a sample from upper to lower
    Xup = X.copy()
    i = seed % prob.n
    Xup[:, i] = np.minimum(prob.K - 1, Xup[:, i] + 1)
    lab_up, _ = O.classify(Xup, prob.ref_L, prob.ref_U)
    assert not np.any((labels == 1) & (lab_up == 0))
