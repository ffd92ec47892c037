"""rsr_classify_static: the entry point for callers that cannot allocate
device memory (its workspace is a 4 MiB device array owned by the library).

Called twice in a row through the C ABI, it must return exactly what the
caller-workspace entry point (rsr_prepare + rsr_classify, bit-packed path)
returns, and what the oracle's own sampler, first-match loops and gradient
counts give: labels, counts and gradient counts are integers, compared exactly.
The first call uses references with an overlapping (upper below lower) pair,
the second a consistent set, so the second call also shows that the shared
array's header is re-initialised.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import workloads as W
from helpers import POPC, random_refs_problem
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _via_workspace(rsr, prob, seed, offset, N):
    P = rsr.Problem(prob.pmf, prob.ref_L, prob.ref_U, path=POPC)
    sess = rsr.Session(P)
    out = sess.classify(seed, offset, N, labels=True, grad=True)
    torch.cuda.synchronize()
    return {k: out[k].cpu().numpy() for k in ("labels", "counts3", "grad_counts")}


def _via_static(rsr, prob, seed, offset, N):
    P = rsr.Problem(prob.pmf, prob.ref_L, prob.ref_U, path=POPC)
    counts = torch.zeros(3, dtype=torch.int64, device="cuda")
    labels = torch.empty(N, dtype=torch.uint8, device="cuda")
    grad = torch.zeros(P.n * P.K, dtype=torch.int64, device="cuda")
    rsr.rsr_classify_static(P, seed, offset, N, counts, labels=labels, grad_counts=grad)
    torch.cuda.synchronize()
    return {"labels": labels.cpu().numpy(), "counts3": counts.cpu().numpy(), "grad_counts": grad.cpu().numpy()}


def test_static_scratch_matches_workspace_path_twice_in_a_row(rsr):
    first = W.random_small_system(n=6, K=4, M_S=3, seed=1)
    extra_U = first.ref_L[:1].copy()
    extra_U[0, 0] = 0
    first = W.Problem("overlapping", first.pmf, first.ref_L, np.concatenate([first.ref_U, extra_U]))
    second = random_refs_problem(295, 2, 300, 700, seed=9)
    for prob, seed, offset, N in ((first, 3, 11, 5000), (second, 4, 1 << 33, 7001)):
        want = _via_workspace(rsr, prob, seed, offset, N)
        got = _via_static(rsr, prob, seed, offset, N)
        for key in ("labels", "counts3", "grad_counts"):
            assert np.array_equal(got[key], want[key]), key
        X = O.sample(prob.pmf, seed, offset, N)
        lab, cnt = O.classify(X, prob.ref_L, prob.ref_U)
        assert np.array_equal(got["labels"], lab)
        assert np.array_equal(got["counts3"], cnt)
        assert np.array_equal(got["grad_counts"].reshape(prob.n, prob.K), O.grad_counts(X, lab, prob.K))


def test_static_scratch_rejects_problems_beyond_its_size(rsr):
    # 300 components -> 10 words per reference; 120000 references need > 4 MiB
    n, R = 300, 120000
    prob = W.Problem("too_big", np.tile([0.1, 0.9], (n, 1)), np.ones((R, n), np.uint8), np.zeros((0, n), np.uint8))
    P = rsr.Problem(prob.pmf, prob.ref_L, prob.ref_U, path=POPC)
    counts = torch.zeros(3, dtype=torch.int64, device="cuda")
    with pytest.raises(rsr.RSRError) as e:
        rsr.rsr_classify_static(P, 1, 0, 10, counts)
    assert e.value.status == -3
