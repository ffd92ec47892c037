"""GPU parity of the batched persistent launch (many scenarios, one kernel):
every scenario's labels, counts and gradient counts equal the single-problem
path's and the oracle's; replays (direct and from a CUDA graph) advance to the
next window of samples; autotuning never touches the caller's outputs."""
import numpy as np
import pytest
import torch

import workloads as W
from helpers import POPC, make_session, random_refs_problem, run
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def scenarios():
    probs = [random_refs_problem(n, K, RL, RU, seed=11 * n + K)
             for n, K, RL, RU in [(50, 2, 20, 40), (300, 2, 300, 700), (120, 3, 40, 1), (17, 2, 1, 1),
                                  (200, 2, 600, 5), (64, 4, 30, 30), (33, 2, 0, 9), (96, 5, 7, 0)]]
    probs.append(W.c1_grid())
    Ns = [1000, 5000, 257, 1, 3001, 2048, 700, 999, 20000]
    seeds = [100 + s for s in range(len(probs))]
    offsets = [7 * s for s in range(len(probs))]
    return probs, seeds, offsets, Ns


def make_batch(rsr, probs, seeds, offsets, Ns):
    P = [rsr.Problem(p.pmf, p.ref_L, p.ref_U, path=POPC) for p in probs]
    return rsr.Batch(P, seeds, offsets, Ns)


def test_batch_matches_oracle_and_single_path(rsr):
    probs, seeds, offsets, Ns = scenarios()
    b = make_batch(rsr, probs, seeds, offsets, Ns)
    rsr.rsr_batch(b)
    torch.cuda.synchronize()
    counts = b.counts3.cpu().numpy()
    for s, p in enumerate(probs):
        X = O.sample(p.pmf, seeds[s], offsets[s], Ns[s])
        lab, cnt = O.classify(X, p.ref_L, p.ref_U)
        assert np.array_equal(b.labels[s].cpu().numpy(), lab), s
        assert np.array_equal(counts[s], cnt), s
        assert np.array_equal(b.grad_counts[s].cpu().numpy().reshape(p.n, p.K), O.grad_counts(X, lab, p.K)), s
        single = run(make_session(rsr, p), seeds[s], offsets[s], Ns[s])
        assert np.array_equal(single["labels"], lab)


def test_batch_grad_matches_oracle(rsr):
    probs, seeds, offsets, Ns = scenarios()
    b = make_batch(rsr, probs, seeds, offsets, Ns)
    rsr.rsr_batch(b)
    torch.cuda.synchronize()
    g, se = rsr.rsr_batch_grad(b)
    for s, p in enumerate(probs):
        X = O.sample(p.pmf, seeds[s], offsets[s], Ns[s])
        lab, _ = O.classify(X, p.ref_L, p.ref_U)
        g_o, se_o = O.grad(O.grad_counts(X, lab, p.K), Ns[s], p.pmf)
        np.testing.assert_allclose(g[s], g_o, rtol=1e-12, atol=0, equal_nan=True)
        np.testing.assert_allclose(se[s], se_o, rtol=1e-12, atol=0, equal_nan=True)


def test_batch_replay_and_graph_capture(rsr):
    probs, seeds, offsets, Ns = scenarios()
    b = make_batch(rsr, probs, seeds, offsets, Ns)
    rsr.rsr_batch(b)                     # round 0
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    b.counts3.zero_()
    for t in b.grad_counts:
        t.zero_()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=stream):
        rsr.rsr_batch(b, stream=torch.cuda.current_stream())
    # capture does not run the kernel; each replay is the next round
    for rnd in (1, 2):
        b.counts3.zero_()
        for t in b.grad_counts:
            t.zero_()
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        counts = b.counts3.cpu().numpy()
        for s, p in enumerate(probs):
            X = O.sample(p.pmf, seeds[s], offsets[s] + rnd * Ns[s], Ns[s])
            lab, cnt = O.classify(X, p.ref_L, p.ref_U)
            assert np.array_equal(counts[s], cnt), (rnd, s)
            assert np.array_equal(b.labels[s].cpu().numpy(), lab), (rnd, s)
            assert np.array_equal(b.grad_counts[s].cpu().numpy().reshape(p.n, p.K), O.grad_counts(X, lab, p.K))


def test_batch_autotune_leaves_outputs_alone(rsr):
    probs, seeds, offsets, Ns = scenarios()
    b = make_batch(rsr, probs, seeds, offsets, Ns)
    grid, order = rsr.rsr_batch_autotune(b)
    assert grid >= 1 and order in (0, 1)
    torch.cuda.synchronize()
    assert int(b.counts3.abs().sum()) == 0
    assert all(int(t.abs().sum()) == 0 for t in b.grad_counts)
    rsr.rsr_batch(b)                      # still round 0 after tuning
    torch.cuda.synchronize()
    counts = b.counts3.cpu().numpy()
    for s, p in enumerate(probs):
        X = O.sample(p.pmf, seeds[s], offsets[s], Ns[s])
        _, cnt = O.classify(X, p.ref_L, p.ref_U)
        assert np.array_equal(counts[s], cnt)


def test_batch_requires_matching_prepare(rsr):
    probs, seeds, offsets, Ns = scenarios()
    b = make_batch(rsr, probs, seeds, offsets, Ns)
    b.seeds[0] += 1                       # arguments no longer match the prepared work list
    with pytest.raises(rsr.RSRError):
        rsr.rsr_batch(b)


def test_single_problem_autotune_picks_a_path(rsr):
    p = random_refs_problem(300, 2, 3000, 9000, seed=3)
    sess = make_session(rsr, p, path=0, dense=True)
    chosen = rsr.rsr_autotune(sess.problem, sess.ws)
    assert chosen in (1, 2)
    got = run(sess, 2, 0, 4096)
    X = O.sample(p.pmf, 2, 0, 4096)
    lab, _ = O.classify(X, p.ref_L, p.ref_U)
    assert np.array_equal(got["labels"], lab)
