"""GPU parity of the bit-packed classifiers with and without the component-major
index of the upper set (RSR_FLAG_NO_INDEX).

The index changes how a chunk of 256 upper references is tested (one 256-bit OR
per decisive zero bit of the sample instead of 256 reference tests), never the
answer: labels, counts and gradient counts must equal the oracle's bit for bit
in both modes.  The problems are built so that first matches lie deep in the
upper set (many chunks, the per-lane and the one-sample-per-warp index tests,
unclassified samples that visit every chunk), with ragged last chunks, fewer
upper references than the directly tested prefix, multi-state components whose
thermometer runs straddle 32-bit words, and an overlapping (precedence) pair.
"""
import numpy as np
import pytest
import torch

import workloads as W
from helpers import POPC, deep_refs_problem, run
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def session(rsr, prob, index):
    return rsr.Session(rsr.Problem(prob.pmf, prob.ref_L, prob.ref_U, path=POPC, index=index))


def check(rsr, prob, seed, offset, N, samples=None):
    X = samples if samples is not None else O.sample(prob.pmf, seed, offset, N)
    lab, cnt = O.classify(X, prob.ref_L, prob.ref_U)
    C = O.grad_counts(X, lab, prob.K)
    tests = {}
    for index in (True, False):
        given = torch.from_numpy(np.ascontiguousarray(X)).cuda() if samples is not None else None
        got = run(session(rsr, prob, index), seed, offset, N, samples=given)
        assert np.array_equal(got["labels"], lab), index
        assert np.array_equal(got["counts3"], cnt), index
        assert np.array_equal(got["grad_counts"].reshape(prob.n, prob.K), C), index
        tests[index] = int(got["exec_tests"][0])
    return cnt, tests


@pytest.mark.parametrize("n,K,R_L,R_U,N", [(295, 2, 40, 3000, 4000), (100, 4, 30, 1000, 3000),
                                           (68, 16, 10, 600, 2000), (33, 3, 5, 17, 1000),
                                           (300, 2, 0, 256, 1000), (300, 2, 20, 257, 1000),
                                           (10, 2, 3, 5, 700), (1, 2, 1, 1, 100), (47, 5, 7, 1500, 2500)])
def test_index_parity_deep_first_matches(rsr, n, K, R_L, R_U, N):
    prob = deep_refs_problem(n, K, R_L, R_U, seed=1000 + n * K)
    cnt, tests = check(rsr, prob, 5, 1 << 33, N)
    assert cnt.sum() == N


def test_index_parity_mostly_unclassified(rsr):
    # demanding upper references and no lower ones: almost every sample is
    # unclassified and sees every chunk (oracle: 4 upper matches in 3000)
    prob = deep_refs_problem(200, 2, 0, 2000, seed=4, lo=40, hi=80)
    cnt, _ = check(rsr, prob, 8, 0, 3000)
    assert cnt[2] > 2900


def test_index_parity_given_extreme_states(rsr):
    prob = deep_refs_problem(90, 4, 12, 900, seed=6)
    rng = np.random.default_rng(6)
    X = rng.integers(0, 4, size=(1000, 90)).astype(np.uint8)
    X[0] = 3          # at least every upper reference
    X[1] = 0          # below everything
    X[2] = 2
    X[3] = prob.ref_U[700]   # exactly the 701st upper reference
    X[4] = prob.ref_U[899]   # the last one (ragged last chunk)
    check(rsr, prob, 0, 0, X.shape[0], samples=X)


def test_index_parity_with_overlapping_pair(rsr):
    prob = deep_refs_problem(64, 3, 20, 800, seed=9)
    extra_U = prob.ref_L[:1].copy()
    extra_U[0, 5] = 0
    extra_U[0, :3] = 0
    bad = W.Problem("bad", prob.pmf, prob.ref_L, np.concatenate([prob.ref_U, extra_U]))
    assert O.count_overlaps(bad.ref_L, bad.ref_U) > 0
    assert session(rsr, bad, True).overlap()
    check(rsr, bad, 3, 17, 3000)


def test_batch_index_parity(rsr):
    probs = [deep_refs_problem(n, K, RL, RU, seed=n + K) for n, K, RL, RU in
             [(295, 2, 40, 3000), (100, 4, 30, 1000), (33, 3, 5, 17), (10, 2, 3, 5), (120, 2, 0, 700)]]
    probs.append(W.c1_grid())
    Ns = [3000, 2000, 1000, 700, 1500, 5000]
    seeds = [40 + s for s in range(len(probs))]
    offsets = [11 * s for s in range(len(probs))]
    for index in (True, False):
        P = [rsr.Problem(p.pmf, p.ref_L, p.ref_U, path=POPC, index=index) for p in probs]
        b = rsr.Batch(P, seeds, offsets, Ns)
        rsr.rsr_batch(b)
        torch.cuda.synchronize()
        counts = b.counts3.cpu().numpy()
        for s, p in enumerate(probs):
            X = O.sample(p.pmf, seeds[s], offsets[s], Ns[s])
            lab, cnt = O.classify(X, p.ref_L, p.ref_U)
            assert np.array_equal(b.labels[s].cpu().numpy(), lab), (index, s)
            assert np.array_equal(counts[s], cnt), (index, s)
            assert np.array_equal(b.grad_counts[s].cpu().numpy().reshape(p.n, p.K),
                                  O.grad_counts(X, lab, p.K)), (index, s)


def hazard_problem(n, R_L, R_U, seed):
    """A hazard footprint: 40 components fail with probability 0.3-0.5, the rest
    with 1e-3, so the index is built in clustered order (binary components, the
    32nd most failure-prone component far above the median).  Upper references
    are random subsets that mostly include footprint components, so first
    matches lie deep and chunk AND rows rule out whole chunks."""
    rng = np.random.default_rng(seed)
    pf = np.full(n, 1e-3)
    hot = rng.choice(n, size=40, replace=False)
    pf[hot] = rng.uniform(0.3, 0.5, size=40)
    pmf = np.stack([pf, 1 - pf], axis=1)
    ref_U = np.zeros((R_U, n), np.uint8)
    for r in range(R_U):
        k_hot = int(rng.integers(8, 20))
        ref_U[r, rng.choice(hot, size=k_hot, replace=False)] = 1
        ref_U[r, rng.choice(n, size=int(rng.integers(3, 15)), replace=False)] = 1
    ref_L = np.ones((R_L, n), np.uint8)
    for r in range(R_L):
        ref_L[r, rng.choice(hot, size=int(rng.integers(8, 16)), replace=False)] = 0
    return W.Problem("hazard", pmf, ref_L, ref_U)


@pytest.mark.parametrize("n,R_L,R_U,N", [(150, 30, 3000, 4000), (290, 200, 2049, 3000), (64, 0, 1100, 2000)])
def test_index_parity_clustered_order(rsr, n, R_L, R_U, N):
    prob = hazard_problem(n, R_L, R_U, seed=n + R_U)
    cnt, _ = check(rsr, prob, 21, 1 << 20, N)
    assert cnt[1] > 0 and cnt.sum() == N


def test_batch_index_parity_clustered_order(rsr):
    probs = [hazard_problem(n, RL, RU, seed=7 * n) for n, RL, RU in [(150, 30, 3000), (64, 0, 1100), (200, 50, 600)]]
    Ns = [3000, 2000, 1000]
    seeds = [3, 4, 5]
    offsets = [0, 1 << 30, 17]
    P = [rsr.Problem(p.pmf, p.ref_L, p.ref_U, path=POPC) for p in probs]
    b = rsr.Batch(P, seeds, offsets, Ns)
    rsr.rsr_batch(b)
    torch.cuda.synchronize()
    counts = b.counts3.cpu().numpy()
    for s, p in enumerate(probs):
        X = O.sample(p.pmf, seeds[s], offsets[s], Ns[s])
        lab, cnt = O.classify(X, p.ref_L, p.ref_U)
        assert np.array_equal(b.labels[s].cpu().numpy(), lab), s
        assert np.array_equal(counts[s], cnt), s
        assert np.array_equal(b.grad_counts[s].cpu().numpy().reshape(p.n, p.K), O.grad_counts(X, lab, p.K)), s


def _random_problem(rng):
    """A random mix of the shapes the kernels branch on: binary or multi-state,
    concentrated or spread failure probabilities (clustered index order or not),
    shallow or deep first matches, empty sets, ragged chunks."""
    K = int(rng.choice([2, 2, 3, 4, 5]))
    n = int(rng.integers(1, min(300, 512 // (K - 1)) + 1))
    if K == 2 and rng.random() < 0.5:
        pf = np.full(n, 1e-3)
        hot = rng.choice(n, size=min(n, 40), replace=False)
        pf[hot] = rng.uniform(0.2, 0.5, size=hot.size)
        pmf = np.stack([pf, 1 - pf], axis=1)
    else:
        pmf = rng.dirichlet(np.ones(K), size=n)
        pmf[:, -1] += rng.uniform(0.5, 3.0)
        pmf /= pmf.sum(1, keepdims=True)
    R_U = int(rng.choice([0, 1, 15, 17, 255, 256, 257, int(rng.integers(300, 2500))]))
    R_L = int(rng.choice([0, 1, int(rng.integers(2, 400))]))
    if R_L + R_U == 0:
        R_U = 1
    lo, hi = (1, 6) if rng.random() < 0.5 else (8, 30)
    ref_U = np.zeros((R_U, n), np.uint8)
    for r in range(R_U):
        idx = rng.choice(n, size=min(n, int(rng.integers(lo, hi + 1))), replace=False)
        ref_U[r, idx] = rng.integers(1, K, size=idx.size)
    ref_L = np.full((R_L, n), K - 1, np.uint8)
    for r in range(R_L):
        idx = rng.choice(n, size=min(n, int(rng.integers(1, 6))), replace=False)
        ref_L[r, idx] = rng.integers(0, K - 1, size=idx.size)
    return W.Problem("random", pmf, ref_L, ref_U)


def test_index_parity_randomized(rsr):
    rng = np.random.default_rng(2026)
    probs = [_random_problem(rng) for _ in range(24)]
    Ns = [int(rng.integers(1, 3000)) for _ in probs]
    for s, (p, N) in enumerate(zip(probs, Ns)):
        check(rsr, p, 100 + s, int(rng.integers(0, 1 << 40)), N)
    # the same problems in one batched launch, with and without the index
    seeds = [300 + s for s in range(len(probs))]
    offsets = [int(x) for x in rng.integers(0, 1 << 40, size=len(probs))]
    for index in (True, False):
        P = [rsr.Problem(p.pmf, p.ref_L, p.ref_U, path=POPC, index=index) for p in probs]
        b = rsr.Batch(P, seeds, offsets, Ns)
        rsr.rsr_batch(b)
        torch.cuda.synchronize()
        counts = b.counts3.cpu().numpy()
        for s, p in enumerate(probs):
            X = O.sample(p.pmf, seeds[s], offsets[s], Ns[s])
            lab, cnt = O.classify(X, p.ref_L, p.ref_U)
            assert np.array_equal(b.labels[s].cpu().numpy(), lab), (index, s)
            assert np.array_equal(counts[s], cnt), (index, s)
            assert np.array_equal(b.grad_counts[s].cpu().numpy().reshape(p.n, p.K),
                                  O.grad_counts(X, lab, p.K)), (index, s)
