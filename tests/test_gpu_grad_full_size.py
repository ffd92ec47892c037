"""Gradient parity at full workload sizes, in the launch configurations that
bench.py times.

Gradient counts C[i, k] = #{h in I^L : x_{h,i} = k} are compared with the
per-state histogram of the I^L rows of the materialised samples (rsr_sample,
whose states equal the oracle's sampler bit for bit), and the labels with the
oracle's own first-match loops on seeded row subsets.  On the multi-state flow
network the 400-probability deliverable runs through the oracle end to end at
N = 1e6: its sampler, first-match labels, max-flow Stage 2, gradient counts and
fp64 gradient and standard error.
"""
import numpy as np
import pytest
import torch

from helpers import POPC, TC, make_session
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def lower_histogram(rsr, sess, seed, offset, labels_dev, lower_codes=(0,), slice_n=1_000_000):
    """n x K int64 histogram of the states of the samples whose label is in
    lower_codes, from rsr_sample's materialised states, slice by slice."""
    p = sess.problem
    N = labels_dev.numel()
    C = torch.zeros((p.n, p.K), dtype=torch.int64, device="cuda")
    for a in range(0, N, slice_n):
        m = min(slice_n, N - a)
        X = rsr.rsr_sample(p, seed, offset + a, m, sess.ws)
        lab = labels_dev[a:a + m]
        sel = torch.zeros(m, dtype=torch.bool, device="cuda")
        for c in lower_codes:
            sel |= lab == c
        rows = X[sel]
        for k in range(p.K):
            C[:, k] += (rows == k).sum(0, dtype=torch.int64)
        del X, rows
    torch.cuda.synchronize()
    return C.cpu().numpy()


def oracle_rows(prob, seed, offset, idx):
    X = np.concatenate([O.sample(prob.pmf, seed, offset + int(i), 1) for i in idx])
    lab, _ = O.classify(X, prob.ref_L, prob.ref_U)
    return lab


@pytest.fixture(scope="module")
def c3():
    import workloads.large as L
    return L.c3_dnf()


@pytest.mark.parametrize("p_up", [0.9, 0.01])
def test_c3_dense_tc_gradient_counts_full_size(rsr, c3, p_up):
    """The 200k-reference classifier, N = 4e6, dense tensor-core launch.  At the
    workload's p_up = 0.9 no sample lies below a failure reference (a minimal
    cut of ~145 components), so every count is 0; p_up = 0.01 on the same
    references puts most samples in I^L and exercises every count."""
    import workloads as W
    N, seed = 4_000_000, 21
    prob = W.Problem("c3_p%.2f" % p_up, W.binary_pmf(np.full(c3.n, 1.0 - p_up)), c3.ref_L, c3.ref_U)
    sess = make_session(rsr, prob, path=TC, dense=True)
    out = sess.classify(seed, 0, N, labels=True, grad=True)
    torch.cuda.synchronize()
    counts = out["counts3"].cpu().numpy()
    labels = out["labels"]
    assert np.array_equal(np.bincount(labels.cpu().numpy(), minlength=3), counts)
    C = lower_histogram(rsr, sess, seed, 0, labels)
    got = out["grad_counts"].cpu().numpy().reshape(prob.n, prob.K)
    assert np.array_equal(got, C)
    assert np.all(got.sum(1) == counts[0])
    if p_up < 0.5:
        assert counts[0] > N // 2 and np.all(got[:, 1] > 0)
    rng = np.random.default_rng(31)
    idx = np.unique(np.concatenate([rng.integers(0, N, 400), [0, N - 1]]))
    assert np.array_equal(labels.cpu().numpy()[idx], oracle_rows(prob, seed, 0, idx))
    # the fp64 gradient from these counts is the oracle's formula on the same integers
    g, se = rsr.rsr_grad(sess.problem, seed, 0, N, out["grad_counts"], sess.ws)
    g_o, se_o = O.grad(C, N, prob.pmf)
    np.testing.assert_allclose(g, g_o, rtol=1e-12, atol=0)
    np.testing.assert_allclose(se, se_o, rtol=1e-12, atol=0)


@pytest.mark.parametrize("path", [POPC, TC])
def test_c4_gradient_of_400_probabilities_full_size(rsr, path):
    """C4 at m' = 0, N = 1e6: dP(S <= 0)/dq_{i,k} for all 100 x 4 state
    probabilities, after Stage 2 on the device, equals the oracle's."""
    import workloads.large as L
    p = L.c4_flow(0)
    N, seed = 1_000_000, 4
    thr = [p.meta["l1"], p.meta["l2"]]
    sess = make_session(rsr, p, path=path)
    out = sess.classify(seed, 0, N, labels=True, grad=True)
    system = rsr.System(rsr.RSR_PHI_ST_MAXFLOW_LEVELS, p.meta["n_nodes"], p.meta["arcs"], p.meta["s"],
                        p.meta["t"], thr, 0)
    labels = out["labels"]
    u_idx, c2 = rsr.rsr_resolve(sess.problem, system, seed, 0, N, labels, sess.ws)
    torch.cuda.synchronize()
    n_lower = int(c2[0].item())
    g, se = rsr.rsr_grad(sess.problem, seed, 0, N, out["grad_counts"], sess.ws, u_lower_idx=u_idx[:n_lower])
    assert rsr.rsr_workspace_status(sess.ws)[1] == 0
    # the oracle, end to end on the same seeded stream
    X = O.sample(p.pmf, seed, 0, N)
    lab, cnt = O.classify(X, p.ref_L, p.ref_U)
    res, n_lower_o = O.resolve(O.PHI_ST_MAXFLOW_LEVELS, p.meta["n_nodes"], p.meta["arcs"], p.meta["s"], p.meta["t"],
                               X, lab, m_prime=0, thresholds=thr)
    assert np.array_equal(labels.cpu().numpy(), res)
    assert np.array_equal(out["counts3"].cpu().numpy(), cnt) and n_lower == n_lower_o
    C_o = O.grad_counts(X, lab, p.K, u_lower_idx=np.nonzero(res == 3)[0])
    # rsr_grad adds the Stage-2 samples' states to the counts in place
    assert np.array_equal(out["grad_counts"].cpu().numpy().reshape(p.n, p.K), C_o)
    g_o, se_o = O.grad(C_o, N, p.pmf)
    assert g.shape == (100, 4) and np.all(np.isfinite(g))
    np.testing.assert_allclose(g, g_o, rtol=1e-12, atol=0)
    np.testing.assert_allclose(se, se_o, rtol=1e-12, atol=0)
    # the estimate behind the gradient
    assert rsr.rsr_estimate(out["counts3"].cpu().numpy(), N, n_lower) == O.estimate(cnt, N, n_lower_o)


def test_c5_batched_gradient_counts_every_scenario(rsr):
    """The 256 hazard scenarios at N = 2e5 each in the batched launch: every
    scenario's gradient counts equal the histogram of its I^L rows, and
    rsr_batch_grad equals the oracle's fp64 gradient on those counts."""
    import workloads.large as L
    probs = L.c5_batch()
    S, N = len(probs), 200_000
    seeds, offsets = [1000 + s for s in range(S)], [0] * S
    P = [rsr.Problem(p.pmf, p.ref_L, p.ref_U, path=POPC) for p in probs]
    b = rsr.Batch(P, seeds, offsets, [N] * S)
    rsr.rsr_batch(b)
    torch.cuda.synchronize()
    g, se = rsr.rsr_batch_grad(b)
    counts = b.counts3.cpu().numpy()
    n_nonzero = 0
    for s, p in enumerate(probs):
        sess = make_session(rsr, p)
        C = lower_histogram(rsr, sess, seeds[s], offsets[s], b.labels[s])
        got = b.grad_counts[s].cpu().numpy().reshape(p.n, p.K)
        assert np.array_equal(got, C), s
        assert np.all(got.sum(1) == counts[s, 0]), s
        n_nonzero += int(counts[s, 0] > 0)
        g_o, se_o = O.grad(C, N, p.pmf)
        np.testing.assert_allclose(g[s], g_o, rtol=1e-12, atol=0)
        np.testing.assert_allclose(se[s], se_o, rtol=1e-12, atol=0)
        del sess
    assert n_nonzero > S // 2
