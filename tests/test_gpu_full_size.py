"""Parity at full workload sizes, in the launch configurations bench.py times.

The oracle cannot classify millions of samples against 2.5e5 references, so
it re-derives a seeded random subset of rows one by one (its own Philox
sampler and first-match loops); the rest is checked through properties that
hold at any size: the label histogram equals the counts, dense and early-exit
labels agree, the two classifier paths agree, and the gradient counts are the
per-state histogram of the I^L rows of the materialised samples.
"""
import numpy as np
import pytest
import torch

from helpers import POPC, TC, make_session, run, tc_executed_tests
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def oracle_rows(prob, seed, offset, idx):
    X = np.concatenate([O.sample(prob.pmf, seed, offset + int(i), 1) for i in idx])
    lab, _ = O.classify(X, prob.ref_L, prob.ref_U)
    return lab


def check_subset(prob, labels, seed, offset, n_check, rng_seed):
    rng = np.random.default_rng(rng_seed)
    N = labels.size
    idx = np.unique(np.concatenate([rng.integers(0, N, n_check), [0, N - 1]]))
    want = oracle_rows(prob, seed, offset, idx)
    assert np.array_equal(labels[idx], want)


@pytest.fixture(scope="module")
def c3():
    import workloads.large as L
    return L.c3_dnf()


def test_c3_dense_tc_full_size(rsr, c3):
    N = 4_000_000
    got = run(make_session(rsr, c3, path=TC, dense=True), 1, 0, N)
    assert np.array_equal(np.bincount(got["labels"], minlength=3), got["counts3"])
    check_subset(c3, got["labels"], 1, 0, 1500, 3)
    assert got["exec_tests"][0] == tc_executed_tests(c3.n, c3.K, c3.R_L, c3.R_U, N, dense=True)
    # early exit gives the same labels
    got_ee = run(make_session(rsr, c3, path=TC, dense=False), 1, 0, N)
    assert np.array_equal(got_ee["labels"], got["labels"])
    assert np.array_equal(got_ee["grad_counts"], got["grad_counts"])


def test_c3_popc_matches_tc_on_a_slice(rsr, c3):
    N = 200_000
    a = run(make_session(rsr, c3, path=POPC, dense=False), 5, 123, N)
    b = run(make_session(rsr, c3, path=TC, dense=False), 5, 123, N)
    assert np.array_equal(a["labels"], b["labels"])
    check_subset(c3, a["labels"], 5, 123, 300, 4)


@pytest.mark.parametrize("path", [POPC, TC])
def test_c2_full_size(rsr, path):
    import workloads.large as L
    p = L.c2_rgg()
    N = 1_000_000
    got = run(make_session(rsr, p, path=path), 1, 0, N)
    assert np.array_equal(np.bincount(got["labels"], minlength=3), got["counts3"])
    check_subset(p, got["labels"], 1, 0, 3000, 5)
    # gradient counts = per-state histogram of the I^L rows (materialised samples)
    sess = make_session(rsr, p, path=path)
    X = rsr.rsr_sample(sess.problem, 1, 0, N, sess.ws).cpu().numpy()
    L_rows = X[got["labels"] == 0]
    C = np.stack([np.bincount(L_rows[:, i], minlength=2) for i in range(p.n)])
    assert np.array_equal(got["grad_counts"].reshape(p.n, 2), C)


@pytest.mark.parametrize("m_prime", [0, 1])
@pytest.mark.parametrize("path", [POPC, TC])
def test_c4_multistate_full_size(rsr, m_prime, path):
    import workloads.large as L
    p = L.c4_flow(m_prime)
    N = 1_000_000
    got = run(make_session(rsr, p, path=path), 4, 0, N)
    assert np.array_equal(np.bincount(got["labels"], minlength=3), got["counts3"])
    check_subset(p, got["labels"], 4, 0, 3000, 6 + m_prime)
    dense = run(make_session(rsr, p, path=path, dense=True), 4, 0, N)
    assert np.array_equal(dense["labels"], got["labels"])


def test_c5_batched_full_size(rsr):
    """The 256 hazard scenarios at N = 2e5 each, in the batched launch the bench
    times: per scenario the label histogram equals the counts, a seeded subset of
    rows equals the oracle's, and the labels equal those of the launch without the
    upper index; every fourth scenario also equals the single-problem path."""
    import workloads.large as L
    probs = L.c5_batch()
    S, N = len(probs), 200_000
    seeds, offsets = [1000 + s for s in range(S)], [0] * S
    out = {}
    for index in (True, False):
        P = [rsr.Problem(p.pmf, p.ref_L, p.ref_U, path=POPC, index=index) for p in probs]
        b = rsr.Batch(P, seeds, offsets, [N] * S)
        rsr.rsr_batch(b)
        torch.cuda.synchronize()
        out[index] = ([t.cpu().numpy() for t in b.labels], b.counts3.cpu().numpy())
        del b
    labels, counts = out[True]
    for s, p in enumerate(probs):
        assert np.array_equal(np.bincount(labels[s], minlength=3), counts[s]), s
        assert np.array_equal(labels[s], out[False][0][s]), s
        check_subset(p, labels[s], seeds[s], offsets[s], 40, 100 + s)
    for s in range(0, S, 4):
        got = run(make_session(rsr, probs[s]), seeds[s], offsets[s], N, grad=False)
        assert np.array_equal(got["labels"], labels[s]), s
