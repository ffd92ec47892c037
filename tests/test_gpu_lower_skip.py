"""GPU parity of the lower chunk skip: lower references in guard order beyond
the first chunk, per-chunk AND and guard rows, lanes a chunk's rows rule out
passing over it.  The problems have many lower chunks, a hazard-like pmf (a few
failure-prone components), few upper references (most samples walk the lower
set far), multi-state encodings, duplicated references and a reference at the
top state (no forbidden bit, which turns its chunk's guard test off).  Labels,
counts and gradient counts equal the oracle's on the single-problem path (with
and without the skip) and in a batch."""
import numpy as np
import pytest
import torch

import workloads as W
from helpers import POPC, run
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def hazard_lower_problem(n, K, R_L, R_U, seed, top_ref=False, dups=0):
    rng = np.random.default_rng(seed)
    # most components rarely leave the top state; a footprint of n/8 often does
    pmf = np.zeros((n, K))
    weak = rng.choice(n, size=max(1, n // 8), replace=False)
    for i in range(n):
        p_low = 0.3 if i in weak else 0.01
        pmf[i, :-1] = p_low / (K - 1)
        pmf[i, -1] = 1.0 - p_low
    ref_L = np.full((R_L, n), K - 1, dtype=np.uint8)
    for r in range(R_L):
        # 3-8 entries below the top, mostly inside the footprint
        k = int(rng.integers(3, 9))
        pool = weak if rng.random() < 0.6 else np.arange(n)
        idx = rng.choice(pool, size=min(k, pool.size), replace=False)
        ref_L[r, idx] = rng.integers(0, K - 1, size=idx.size)
    if dups:
        ref_L = np.concatenate([ref_L, ref_L[rng.integers(0, R_L, size=dups)]])
    if top_ref:
        ref_L = np.concatenate([ref_L[: R_L // 2], np.full((1, n), K - 1, dtype=np.uint8), ref_L[R_L // 2:]])
    ref_U = np.zeros((R_U, n), dtype=np.uint8)
    for r in range(R_U):
        idx = rng.choice(n, size=min(n, int(rng.integers(n // 3, n // 2 + 1))), replace=False)
        ref_U[r, idx] = rng.integers(1, K, size=idx.size)
    return W.Problem("hazard_lower", pmf, ref_L, ref_U)


CASES = [  # n, K, R_L, R_U, top_ref, dups, N
    (120, 2, 1500, 40, False, 0, 20000),
    (96, 3, 1200, 25, False, 300, 12000),
    (64, 4, 900, 10, False, 0, 9000),
    (200, 2, 2100, 0, False, 0, 7001),
    (80, 2, 700, 30, True, 0, 5000),
]


def oracle_of(prob, seed, offset, N):
    X = O.sample(prob.pmf, seed, offset, N)
    lab, cnt = O.classify(X, prob.ref_L, prob.ref_U)
    return lab, cnt, O.grad_counts(X, lab, prob.K)


@pytest.mark.parametrize("n,K,R_L,R_U,top_ref,dups,N", CASES)
def test_lower_skip_single_problem(rsr, n, K, R_L, R_U, top_ref, dups, N):
    prob = hazard_lower_problem(n, K, R_L, R_U, seed=31 * n + K, top_ref=top_ref, dups=dups)
    lab, cnt, C = oracle_of(prob, 9, 1 << 20, N)
    if not top_ref:
        assert cnt[2] > 0 and cnt[0] > 0     # samples that walk every lower chunk, and lower matches
    for index in (True, False):
        P = rsr.Problem(prob.pmf, prob.ref_L, prob.ref_U, path=POPC, index=index)
        got = run(rsr.Session(P), 9, 1 << 20, N)
        assert np.array_equal(got["labels"], lab), index
        assert np.array_equal(got["counts3"], cnt), index
        assert np.array_equal(got["grad_counts"].reshape(prob.n, prob.K), C), index


def test_lower_skip_in_a_batch(rsr):
    probs = [hazard_lower_problem(n, K, R_L, R_U, seed=31 * n + K, top_ref=t, dups=d)
             for n, K, R_L, R_U, t, d, _ in CASES]
    Ns = [c[-1] for c in CASES]
    seeds = [50 + s for s in range(len(probs))]
    offsets = [3 * s for s in range(len(probs))]
    P = [rsr.Problem(p.pmf, p.ref_L, p.ref_U, path=POPC) for p in probs]
    b = rsr.Batch(P, seeds, offsets, Ns)
    rsr.rsr_batch(b)
    torch.cuda.synchronize()
    counts = b.counts3.cpu().numpy()
    for s, p in enumerate(probs):
        lab, cnt, C = oracle_of(p, seeds[s], offsets[s], Ns[s])
        assert np.array_equal(b.labels[s].cpu().numpy(), lab), s
        assert np.array_equal(counts[s], cnt), s
        assert np.array_equal(b.grad_counts[s].cpu().numpy().reshape(p.n, p.K), C), s
