"""Shared helpers of the GPU parity tests (no GPU needed to import)."""
import numpy as np

import workloads as W

POPC, TC = 1, 2


def random_refs_problem(n, K, R_L, R_U, seed):
    """Partial, random (not boundary) references with a mix of outcomes: lower
    references sit near the top state with a few low entries, upper references
    near state 0 with a few high entries."""
    rng = np.random.default_rng(seed)
    pmf = rng.dirichlet(np.ones(K) * 0.5, size=n)
    pmf[:, -1] += 2.0
    pmf /= pmf.sum(1, keepdims=True)
    ref_L = np.full((R_L, n), K - 1, dtype=np.uint8)
    for r in range(R_L):
        idx = rng.choice(n, size=min(n, int(rng.integers(1, 4))), replace=False)
        ref_L[r, idx] = rng.integers(0, K - 1, size=idx.size)
    ref_U = np.zeros((R_U, n), dtype=np.uint8)
    for r in range(R_U):
        idx = rng.choice(n, size=min(n, int(rng.integers(3, 12))), replace=False)
        ref_U[r, idx] = rng.integers(1, K, size=idx.size)
    return W.Problem("random_refs", pmf, ref_L, ref_U)


def tc_kpad(n, K):
    kenc = n * (K - 1)
    return ((kenc + (kenc + 15) // 16 + 31) // 32) * 32


def make_session(rsr, prob, path=POPC, dense=False):
    P = rsr.Problem(prob.pmf, prob.ref_L, prob.ref_U, path=path, dense=dense)
    return rsr.Session(P)


def run(sess, seed, offset, N, samples=None, grad=True):
    import torch
    out = sess.classify(seed, offset, N, samples=samples, labels=True, grad=grad, count_tests=True)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}


def tc_executed_tests(n, K, R_L, R_U, N, dense=True):
    """Reference tests the tensor-core path executes.  Dense mode runs on CTA
    pairs: 256-sample pair blocks times 256-reference tiles.  Early exit runs one
    CTA per MMA: at most 128-sample blocks times BN-reference tiles (BN = 256 when
    a row fits in 320 bytes, else 128), padding included."""
    if dense:
        tiles = -(-R_L // 256) + -(-R_U // 256)
        return (-(-N // 256)) * 256 * tiles * 256
    bn = 256 if tc_kpad(n, K) <= 320 else 128
    tiles = -(-R_L // bn) + -(-R_U // bn)
    return (-(-N // 128)) * 128 * tiles * bn


def deep_refs_problem(n, K, R_L, R_U, seed, lo=8, hi=30):
    """Upper references that few samples reach: each asks for a random subset of
    lo..hi components to be at or above a random state >= 1, so a sample's first
    match (if any) lies deep in the upper set and many samples stay
    unclassified.  Lower references as in random_refs_problem."""
    rng = np.random.default_rng(seed)
    pmf = rng.dirichlet(np.ones(K), size=n)
    pmf[:, -1] += 1.0
    pmf /= pmf.sum(1, keepdims=True)
    ref_L = np.full((R_L, n), K - 1, dtype=np.uint8)
    for r in range(R_L):
        idx = rng.choice(n, size=min(n, int(rng.integers(1, 4))), replace=False)
        ref_L[r, idx] = rng.integers(0, K - 1, size=idx.size)
    ref_U = np.zeros((R_U, n), dtype=np.uint8)
    for r in range(R_U):
        idx = rng.choice(n, size=min(n, int(rng.integers(lo, hi + 1))), replace=False)
        ref_U[r, idx] = rng.integers(1, K, size=idx.size)
    return W.Problem("deep_refs", pmf, ref_L, ref_U)


def sparse_match_problem(n, R_L, R_U, lo, hi, seed, down=20):
    """Binary components with P(up) = 1/2; each lower reference needs `down`
    given components failed (almost never met) and each upper reference a
    random set of lo..hi given components working, so the samples that match
    only a large set, or nothing, walk deep into the upper set."""
    rng = np.random.default_rng(seed)
    pmf = np.tile([0.5, 0.5], (n, 1))
    ref_L = np.ones((R_L, n), dtype=np.uint8)
    for r in range(R_L):
        ref_L[r, rng.choice(n, size=down, replace=False)] = 0
    ref_U = np.zeros((R_U, n), dtype=np.uint8)
    for r in range(R_U):
        ref_U[r, rng.choice(n, size=int(rng.integers(lo, hi + 1)), replace=False)] = 1
    return W.Problem("sparse_match", pmf, ref_L, ref_U)
