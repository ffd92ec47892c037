"""GPU parity of the single-problem bit-packed path in stages: the first pass
walks k0 chunk steps per tile and queues the samples still unresolved in one of
the workspace's two deep queues, each later pass takes them 256 at a time and
walks four times as far, queueing again, the last to the end (at any N under a
test flag; by default from 2^19 samples, as in the full-size tests).  Labels, counts and
gradient counts equal the oracle's and the one-pass kernel's (a workspace
without a queue), with Philox samples and with given states, when the queue
overflows (its tiles finish the walk themselves), and after rsr_autotune picks
the first pass's budget."""
import numpy as np
import pytest
import torch

from helpers import POPC, deep_refs_problem, run, sparse_match_problem
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def session_with_queue(rsr, prob, n_queue, index=True):
    """A prepared workspace whose deep queue holds n_queue entries (0: none),
    for a problem that runs staged passes whatever N (test flag; without it calls
    of fewer than 2^19 samples run one pass)."""
    from paper_2604_17066_gb300._lib import RSR_FLAG_TEST_TWO_PASS
    P = rsr.Problem(prob.pmf, prob.ref_L, prob.ref_U, path=POPC, index=index)
    P.extra_flags = RSR_FLAG_TEST_TWO_PASS
    s = rsr.Session.__new__(rsr.Session)
    s.problem, s.stream = P, None
    s.ws = rsr.alloc_workspace(P, n_queue)
    rsr.rsr_prepare(P, s.ws)
    return s


def oracle_of(prob, seed, offset, N, X=None):
    X = O.sample(prob.pmf, seed, offset, N) if X is None else X
    lab, cnt = O.classify(X, prob.ref_L, prob.ref_U)
    return lab, cnt, O.grad_counts(X, lab, prob.K)


PROBS = {
    # unresolved samples after the first chunks in every tile
    "sparse": lambda: sparse_match_problem(80, 300, 3000, 6, 24, seed=5),
    # first matches thousands of references deep, multi-state
    "deep_k3": lambda: deep_refs_problem(100, 3, 30, 2000, seed=77),
    "deep_k5": lambda: deep_refs_problem(47, 5, 7, 1500, seed=78),
    # 122 chunk steps: stages [0, 2), [2, 8), [8, 32), [32, 122)
    "many_chunks": lambda: sparse_match_problem(80, 300, 30000, 6, 24, seed=6),
}


@pytest.mark.parametrize("name", sorted(PROBS))
def test_two_pass_matches_oracle_and_one_pass(rsr, name):
    prob = PROBS[name]()
    N = 12001
    lab, cnt, C = oracle_of(prob, 3, 1 << 30, N)
    for n_queue in (0, 1 << 20, 300):   # one pass; a queue for every sample; a queue that overflows
        got = run(session_with_queue(rsr, prob, n_queue), 3, 1 << 30, N)
        assert np.array_equal(got["labels"], lab), n_queue
        assert np.array_equal(got["counts3"], cnt), n_queue
        assert np.array_equal(got["grad_counts"].reshape(prob.n, prob.K), C), n_queue
    # without the index the staged passes hold as well
    got = run(session_with_queue(rsr, prob, 1 << 20, index=False), 3, 1 << 30, N)
    assert np.array_equal(got["labels"], lab)


def test_two_pass_with_given_states(rsr):
    prob = PROBS["deep_k3"]()
    N = 5000
    X = O.sample(prob.pmf, 11, 0, N)
    lab, cnt, C = oracle_of(prob, 0, 0, N, X=X)
    given = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    got = run(session_with_queue(rsr, prob, 1 << 20), 0, 0, N, samples=given)
    assert np.array_equal(got["labels"], lab)
    assert np.array_equal(got["counts3"], cnt)
    assert np.array_equal(got["grad_counts"].reshape(prob.n, prob.K), C)


def test_two_pass_after_autotune(rsr):
    prob = PROBS["sparse"]()
    sess = session_with_queue(rsr, prob, 1 << 20)
    assert rsr.rsr_autotune(sess.problem, sess.ws) in (1, 2)   # the bit-packed path also gets its k0 tuned
    N = 30000
    lab, cnt, C = oracle_of(prob, 8, 77, N)
    got = run(sess, 8, 77, N)
    assert np.array_equal(got["labels"], lab)
    assert np.array_equal(got["counts3"], cnt)
    assert np.array_equal(got["grad_counts"].reshape(prob.n, prob.K), C)


def test_two_pass_with_an_overlapping_pair(rsr):
    """An upper reference below a lower one: every lower chunk comes first
    (lower takes precedence, Algorithm 1), so the first pass's k0 steps are all
    lower chunks and the deferred samples resume there."""
    import workloads as W
    prob = sparse_match_problem(80, 600, 3000, 6, 24, seed=21)   # three lower chunks, rarely matched
    extra_U = prob.ref_L[:1].copy()
    extra_U[0, :5] = 0
    bad = W.Problem("overlapping", prob.pmf, prob.ref_L, np.concatenate([prob.ref_U, extra_U]))
    assert O.count_overlaps(bad.ref_L, bad.ref_U) > 0
    sess = session_with_queue(rsr, bad, 1 << 20)
    assert sess.overlap()
    N = 9000
    lab, cnt, C = oracle_of(bad, 6, 123, N)
    got = run(sess, 6, 123, N)
    assert np.array_equal(got["labels"], lab)
    assert np.array_equal(got["counts3"], cnt)
    assert np.array_equal(got["grad_counts"].reshape(bad.n, bad.K), C)
