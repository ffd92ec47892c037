"""GPU parity of the bit-packed (CUDA-core) path against the oracle.

Labels, counts and gradient counts must be bit-exact on the same seeded
samples; estimates and gradients identical in fp64 (they are computed from
identical integers with the same formulas).  Sizes: small enough for the
oracle, large enough to span several 256-sample tiles, several 256-reference
chunks and a ragged tail.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu

from helpers import POPC, make_session, random_refs_problem, run  # noqa: E402


@pytest.mark.parametrize("n,K,N,offset", [(17, 2, 777, 0), (100, 4, 1025, 1 << 40), (68, 16, 300, 5),
                                          (295, 2, 513, 123456789)])
def test_sampler_bit_exact(rsr, n, K, N, offset):
    rng = np.random.default_rng(n)
    pmf = rng.dirichlet(np.ones(K), size=n)
    pmf[0] = [0.0] * (K - 1) + [1.0]       # degenerate component: always the top state
    prob = W.Problem("s", pmf, np.zeros((1, n), np.uint8), np.zeros((0, n), np.uint8))
    sess = make_session(rsr, prob)
    got = rsr.rsr_sample(sess.problem, 0xABCDEF0123, offset, N, sess.ws).cpu().numpy()
    want = O.sample(pmf, 0xABCDEF0123, offset, N)
    assert np.array_equal(got, want)


def test_grid_exhaustive_given_states(rsr):
    p = W.c1_grid()
    X = O.all_states(p.n, 2)
    sess = make_session(rsr, p)
    got = run(sess, 0, 0, X.shape[0], samples=torch.from_numpy(X).cuda(), grad=False)
    lab, cnt = O.classify(X, p.ref_L, p.ref_U)
    assert np.array_equal(got["labels"], lab)
    assert np.array_equal(got["counts3"], cnt)
    assert cnt[2] == 0 and np.array_equal(lab, np.where(p.meta["phi_all"] == 0, 0, 1))


@pytest.mark.parametrize("dense", [False, True])
def test_grid_philox_parity(rsr, dense):
    p = W.c1_grid()
    N = 100000
    sess = make_session(rsr, p, dense=dense)
    got = run(sess, 1, 0, N)
    X = O.sample(p.pmf, 1, 0, N)
    lab, cnt = O.classify(X, p.ref_L, p.ref_U)
    assert np.array_equal(got["labels"], lab)
    assert np.array_equal(got["counts3"], cnt)
    C = O.grad_counts(X, lab, p.K)
    assert np.array_equal(got["grad_counts"].reshape(p.n, p.K), C)
    assert rsr.rsr_estimate(got["counts3"], N) == O.estimate(cnt, N)
    g, se = rsr.rsr_grad(sess.problem, 1, 0, N, torch.from_numpy(got["grad_counts"]).cuda(), sess.ws)
    g_o, se_o = O.grad(C, N, p.pmf)
    np.testing.assert_allclose(g, g_o, rtol=1e-12, atol=0)
    np.testing.assert_allclose(se, se_o, rtol=1e-12, atol=0)
    if dense:
        assert got["exec_tests"][0] == N * (p.R_L + p.R_U)
        # dense mode issues one and-or per word of every reference test (the grid: one word)
        assert got["exec_tests"][1] == N * (p.R_L + p.R_U) * 1
    else:
        assert got["exec_tests"][0] < N * (p.R_L + p.R_U)
        assert 0 < got["exec_tests"][1] < N * (p.R_L + p.R_U)


@pytest.mark.parametrize("n,K,R_L,R_U,N", [(295, 2, 300, 700, 5000), (100, 4, 600, 300, 3001),
                                           (40, 5, 1, 513, 2049), (300, 2, 0, 257, 1000),
                                           (300, 2, 300, 0, 1000), (3, 3, 2, 2, 1)])
@pytest.mark.parametrize("dense", [False, True])
def test_random_refs_parity(rsr, n, K, R_L, R_U, N, dense):
    prob = random_refs_problem(n, K, R_L, R_U, seed=n * 7 + K)
    sess = make_session(rsr, prob, dense=dense)
    got = run(sess, 77, 1000, N)
    X = O.sample(prob.pmf, 77, 1000, N)
    lab, cnt = O.classify(X, prob.ref_L, prob.ref_U)
    assert np.array_equal(got["labels"], lab)
    assert np.array_equal(got["counts3"], cnt)
    assert np.array_equal(got["grad_counts"].reshape(n, K), O.grad_counts(X, lab, K))


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_multistate_complete_and_inconsistent_refs(rsr, seed):
    prob = W.random_small_system(n=6, K=4, M_S=3, seed=seed)
    # add an upper reference that lies below a lower reference: precedence decides
    extra_U = prob.ref_L[:1].copy()
    extra_U[0, 0] = 0
    prob_bad = W.Problem("bad", prob.pmf, prob.ref_L, np.concatenate([prob.ref_U, extra_U]))
    assert O.count_overlaps(prob_bad.ref_L, prob_bad.ref_U) > 0
    for pr, overlapping in ((prob, False), (prob_bad, True)):
        sess = make_session(rsr, pr)
        assert sess.overlap() == overlapping
        got = run(sess, seed, 3, 4099)
        X = O.sample(pr.pmf, seed, 3, 4099)
        lab, cnt = O.classify(X, pr.ref_L, pr.ref_U)
        assert np.array_equal(got["labels"], lab)
        assert np.array_equal(got["counts3"], cnt)


def test_grad_correction_with_resolved_unclassified(rsr):
    prob = random_refs_problem(60, 3, 6, 3, seed=5)   # labels 790 / 1860 / 350 (oracle)
    N = 3000
    sess = make_session(rsr, prob)
    got = run(sess, 9, 0, N)
    X = O.sample(prob.pmf, 9, 0, N)
    lab, cnt = O.classify(X, prob.ref_L, prob.ref_U)
    unl = np.nonzero(lab == 2)[0]
    assert unl.size > 10
    resolved = unl[::3].astype(np.int64)     # pretend Phi put every third one at S <= m'
    gc = torch.from_numpy(got["grad_counts"]).cuda()
    g, se = rsr.rsr_grad(sess.problem, 9, 0, N, gc, sess.ws, u_lower_idx=torch.from_numpy(resolved).cuda())
    C = O.grad_counts(X, lab, prob.K, u_lower_idx=resolved)
    assert np.array_equal(gc.cpu().numpy().reshape(prob.n, prob.K), C)
    g_o, se_o = O.grad(C, N, prob.pmf)
    np.testing.assert_allclose(g, g_o, rtol=1e-12, atol=0)
    est = rsr.rsr_estimate(got["counts3"], N, resolved.size)
    assert est == O.estimate(cnt, N, resolved.size)


def test_pmf_change_requires_update_and_reuses_refs(rsr):
    p = W.c1_grid()
    sess = make_session(rsr, p)
    new_pmf = p.pmf.copy()
    new_pmf[3] = [0.3, 0.7]
    sess.problem.pmf = new_pmf
    with pytest.raises(rsr.RSRError):
        sess.classify(1, 0, 10)
    sess.set_pmf(new_pmf)
    got = run(sess, 1, 0, 20000)
    X = O.sample(new_pmf, 1, 0, 20000)
    lab, cnt = O.classify(X, p.ref_L, p.ref_U)
    assert np.array_equal(got["labels"], lab)


def test_zero_samples_is_a_no_op(rsr):
    p = W.c1_grid()
    sess = make_session(rsr, p)
    got = run(sess, 1, 0, 0)
    assert got["counts3"].tolist() == [0, 0, 0]


def test_autograd_function_matches_oracle(rsr):
    p = W.c1_grid()
    N = 50000
    sess = make_session(rsr, p)
    q = torch.tensor(p.pmf, dtype=torch.float64, requires_grad=True)
    P = rsr.RSRProb.apply(q, sess, 4, 0, N)
    P.backward()
    X = O.sample(p.pmf, 4, 0, N)
    lab, cnt = O.classify(X, p.ref_L, p.ref_U)
    assert P.item() == O.estimate(cnt, N)["P_lower"]
    g_o, _ = O.grad(O.grad_counts(X, lab, p.K), N, p.pmf)
    np.testing.assert_allclose(q.grad.numpy(), g_o, rtol=1e-12, atol=0)


@pytest.mark.parametrize("n", [1, 7, 8, 37, 64, 300])
def test_binary_sampler_edge_thresholds(rsr, n):
    """Binary states are drawn with 32-bit thresholds plus a 'never' bit (T = 2^32);
    a lower reference at the top state labels every sample I^L, so the gradient
    counts are the per-component state counts of all N samples: they must equal
    the oracle's exactly, for the single-problem and the batched kernels."""
    rng = np.random.default_rng(n)
    p1 = rng.uniform(0, 1, size=n)
    edge = [0.0, 1.0, 2.0 ** -32, 1 - 2.0 ** -32, 0.5, 1 - 2.0 ** -33, 2.0 ** -33]
    p1[:min(n, len(edge))] = edge[:min(n, len(edge))]
    pmf = np.stack([1 - p1, p1], axis=1)
    ref_L = np.ones((1, n), np.uint8)
    ref_U = rng.integers(0, 2, size=(3, n)).astype(np.uint8)
    prob = W.Problem("edges", pmf, ref_L, ref_U)
    N = 3001
    X = O.sample(pmf, 12, 99, N)
    lab, cnt = O.classify(X, ref_L, ref_U)
    C = O.grad_counts(X, lab, 2)
    assert cnt[0] == N
    got = run(make_session(rsr, prob), 12, 99, N)
    assert np.array_equal(got["grad_counts"].reshape(n, 2), C)
    b = rsr.Batch([rsr.Problem(pmf, ref_L, ref_U, path=POPC)], [12], [99], [N])
    rsr.rsr_batch(b)
    torch.cuda.synchronize()
    assert np.array_equal(b.grad_counts[0].cpu().numpy().reshape(n, 2), C)
    assert np.array_equal(b.counts3[0].cpu().numpy(), cnt)


def test_measured_integer_peaks_are_plausible(rsr):
    """rsr_measure_int_peak (the bit-packed roofline's denominator) returns rates
    between 16 and 256 thread-ops per SM per cycle at 0.5-3 GHz."""
    m = rsr.rsr_measure_int_peak()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for k in ("lop3_ops_per_s", "imad_ops_per_s"):
        assert sms * 16 * 0.5e9 < m[k] < sms * 256 * 3e9, (k, m[k])


def test_measured_philox_rate_is_plausible(rsr):
    """rsr_measure_philox_rate (the samplers' generator alone) returns between
    0.1 and 16 Philox4x32-10 blocks per SM per cycle at 0.5-3 GHz: each block is
    20 wide products and about 40 other integer ops."""
    rate = rsr.rsr_measure_philox_rate()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert sms * 0.1 * 0.5e9 < rate < sms * 16 * 3e9, rate
