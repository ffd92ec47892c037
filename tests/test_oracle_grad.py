"""Pins of the oracle's score-function gradient of P(S <= m').

dP(F)/dq_{i,k} (unconstrained partial of the multilinear polynomial
sum_x 1_F(x) prod_j q_{j,x_j}) equals P(F | X_i = k).  Pins:
* brute-force enumeration reproduces the textbook Birnbaum importances of
  series and parallel systems (prod_{j != i} p_j and prod_{j != i} (1 - p_j));
* Euler's identity for multilinear polynomials: sum_k q_{i,k} dP/dq_{i,k} = P(F);
* the Monte Carlo estimate agrees with the enumerated gradient of the 3x4 grid
  within 3 standard errors per entry (with a multiplicity allowance and a
  chi-square bound over the 34 entries), and with central finite differences along the
  simplex (direction e_{i,0} - e_{i,1}) taken with common random numbers.
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O


def test_bruteforce_series_birnbaum():
    p_fail = np.array([0.1, 0.2, 0.3, 0.05])
    prob = W.series_system(p_fail)
    X = O.all_states(prob.n, 2)
    fail = X.min(axis=1) == 0
    g = O.exact_gradient(prob.pmf, X, fail)
    rel = 1 - p_fail
    for i in range(prob.n):
        others = np.prod(np.delete(rel, i))
        assert g[i, 0] == pytest.approx(1.0, abs=1e-15)
        assert g[i, 1] == pytest.approx(1 - others, abs=1e-15)
        assert g[i, 0] - g[i, 1] == pytest.approx(others, abs=1e-15)


def test_bruteforce_parallel_birnbaum():
    p_fail = np.array([0.4, 0.5, 0.6])
    prob = W.parallel_system(p_fail)
    X = O.all_states(prob.n, 2)
    fail = X.max(axis=1) == 0
    g = O.exact_gradient(prob.pmf, X, fail)
    for i in range(prob.n):
        others = np.prod(np.delete(p_fail, i))
        assert g[i, 0] == pytest.approx(others, abs=1e-15)
        assert g[i, 1] == pytest.approx(0.0, abs=1e-15)


def test_bruteforce_euler_identity_multistate():
    prob = W.random_small_system(n=4, K=3, M_S=3, seed=4)
    X = O.all_states(prob.n, prob.K)
    stride = prob.K ** np.arange(prob.n - 1, -1, -1)
    fail = prob.meta["phi_all"][X.astype(np.int64) @ stride] <= 0
    P = O.exact_probability(prob.pmf, X, fail)
    g = O.exact_gradient(prob.pmf, X, fail)
    for i in range(prob.n):
        assert float(np.dot(prob.pmf[i], g[i])) == pytest.approx(P, rel=1e-13)


@pytest.fixture(scope="module")
def grid_mc():
    p = W.c1_grid()
    N = 200000
    X = O.sample(p.pmf, seed=1, offset=0, N=N)
    labels, counts = O.classify(X, p.ref_L, p.ref_U)
    C = O.grad_counts(X, labels, p.K)
    g, se = O.grad(C, N, p.pmf)
    return p, N, X, labels, counts, C, g, se


def test_grad_counts_rows_sum_to_failures(grid_mc):
    p, N, X, labels, counts, C, g, se = grid_mc
    assert np.all(C.sum(axis=1) == counts[0])
    # C[i, 1] is the number of failed samples with component i working
    assert np.array_equal(C[:, 1], X[labels == 0].astype(np.int64).sum(axis=0))


def test_grad_matches_bruteforce_within_3se(grid_mc):
    p, N, X, labels, counts, C, g, se = grid_mc
    Xall = O.all_states(p.n, 2)
    fail = p.meta["phi_all"] == 0
    g_exact = O.exact_gradient(p.pmf, Xall, fail)
    z = (g - g_exact) / se
    # 34 entries: each within 3 SE except for the few that chance allows (P(|z| > 3) = 0.27%
    # per entry, so 2 of 34 is already a 0.4% event), none beyond 4.5 SE, and a
    # chi-square bound on sum z^2 (34 degrees of freedom, 99.9% quantile 65.2)
    assert np.sum(np.abs(z) > 3.0) <= 2, z
    assert np.all(np.abs(z) <= 4.5), z
    assert float(np.sum(z * z)) <= 65.2


def test_grad_matches_crn_central_differences(grid_mc):
    p, N, X, labels, counts, C, g, se = grid_mc
    h = 0.02
    for i in (0, 5, 9, 16):
        pmf_p, pmf_m = p.pmf.copy(), p.pmf.copy()
        pmf_p[i] += [h, -h]
        pmf_m[i] -= [h, -h]
        lab_p, _ = O.classify(O.sample(pmf_p, seed=1, offset=0, N=N), p.ref_L, p.ref_U)
        lab_m, _ = O.classify(O.sample(pmf_m, seed=1, offset=0, N=N), p.ref_L, p.ref_U)
        D = ((lab_p == 0).astype(np.float64) - (lab_m == 0).astype(np.float64)) / (2 * h)
        fd, se_fd = D.mean(), D.std() / np.sqrt(N)
        deriv = g[i, 0] - g[i, 1]
        se_d = np.sqrt(se[i, 0] ** 2 + se[i, 1] ** 2)
        assert abs(fd - deriv) <= 3 * np.hypot(se_fd, se_d), (i, fd, deriv)


def test_grad_zero_probability_state_gives_nan():
    C = np.array([[0, 5]], dtype=np.int64)
    g, se = O.grad(C, 10, np.array([[0.0, 1.0]]))
    assert np.isnan(g[0, 0]) and g[0, 1] == 0.5
