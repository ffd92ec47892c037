"""GPU parity of the batched persistent launches (many scenarios; a tile pass
and later stages over the queued deep samples): every scenario's labels,
counts and gradient counts equal the single-problem path's and the oracle's,
including a scenario whose samples mostly reach a later stage and one that
overflows its deep queue; replays (direct and from a CUDA graph) advance to the
next window of samples; autotuning never touches the caller's outputs; the
cycle-profiled launch gives the same outputs."""
import numpy as np
import pytest
import torch

import workloads as W
from helpers import POPC, make_session, random_refs_problem, run, sparse_match_problem
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def scenarios():
    probs = [random_refs_problem(n, K, RL, RU, seed=11 * n + K)
             for n, K, RL, RU in [(50, 2, 20, 40), (300, 2, 300, 700), (120, 3, 40, 1), (17, 2, 1, 1),
                                  (200, 2, 600, 5), (64, 4, 30, 30), (33, 2, 0, 9), (96, 5, 7, 0)]]
    probs.append(W.c1_grid())
    # 2 + 12 reference chunks; samples that match only large upper references, or
    # nothing (about 10%), are still unresolved after the first pass's 8 chunks
    probs.append(sparse_match_problem(80, 300, 3000, 6, 24, seed=5))
    Ns = [1000, 5000, 257, 1, 3001, 2048, 700, 999, 20000, 40000]
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


def test_batch_profile_keeps_outputs_and_counts_items(rsr):
    """rsr_batch_profile gives rsr_batch's outputs for the same round, and its
    cycle profile counts one tile-pass item per 256 samples of each scenario,
    positive cycles in each part of an item, and later-stage items only where
    samples outlast the first pass's chunk budget (the sparse scenario)."""
    probs, seeds, offsets, Ns = scenarios()
    b1 = make_batch(rsr, probs, seeds, offsets, Ns)
    b2 = make_batch(rsr, probs, seeds, offsets, Ns)
    for _ in range(2):   # rounds 0 and 1
        rsr.rsr_batch(b1)
        prof = rsr.rsr_batch_profile(b2).cpu().numpy()
        torch.cuda.synchronize()
        assert np.array_equal(b1.counts3.cpu().numpy(), b2.counts3.cpu().numpy())
        for s in range(len(probs)):
            assert np.array_equal(b1.labels[s].cpu().numpy(), b2.labels[s].cpu().numpy()), s
            assert np.array_equal(b1.grad_counts[s].cpu().numpy(), b2.grad_counts[s].cpu().numpy()), s
        for s, N in enumerate(Ns):
            assert prof[s, 0] == (N + 255) // 256, s
            assert (prof[s, 1:4] > 0).all(), s
            assert (prof[s, 5:8] > 0).all() if prof[s, 4] > 0 else (prof[s, 5:8] == 0).all(), s
        assert prof[9, 4] > 0   # the sparse scenario queues samples for a later stage


def test_batch_items_of_three_tiles_match_oracle(rsr):
    """First-pass work items of three consecutive tiles (the test hook; a ragged
    last item where a scenario's tile count is not a multiple of three) give
    the oracle's labels, counts and gradient counts, with later stages and
    cycle profile unchanged in meaning."""
    from paper_2604_17066_gb300._lib import RSR_FLAG_TEST_TILES3
    probs, seeds, offsets, Ns = scenarios()
    P = [rsr.Problem(p.pmf, p.ref_L, p.ref_U, path=POPC) for p in probs]
    for k, pp in enumerate(P):
        if k % 3 != 2:           # most scenarios on three-tile items, the rest on one-tile items
            pp.extra_flags = RSR_FLAG_TEST_TILES3
    b = rsr.Batch(P, seeds, offsets, Ns)
    for r in range(2):
        prof = rsr.rsr_batch_profile(b).cpu().numpy()
        torch.cuda.synchronize()
        counts = b.counts3.cpu().numpy()
        for s, p in enumerate(probs):
            X = O.sample(p.pmf, seeds[s], offsets[s] + r * Ns[s], Ns[s])
            lab, cnt = O.classify(X, p.ref_L, p.ref_U)
            assert np.array_equal(b.labels[s].cpu().numpy(), lab), (r, s)
            assert prof[s, 0] == (Ns[s] + 255) // 256, (r, s)
            if r == 0:
                assert np.array_equal(counts[s], cnt), s
                assert np.array_equal(b.grad_counts[s].cpu().numpy().reshape(p.n, p.K),
                                      O.grad_counts(X, lab, p.K)), s


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
    grid, order, k0, n_tc, staged, tiles = rsr.rsr_batch_autotune(b)
    assert grid >= 1 and order in (0, 1) and k0 in (0, 2, 4, 8, 16, 32) and n_tc == 0 and staged in (0, 1)
    assert tiles in (1, 2, 4, 8)
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


def test_batch_deep_queue_overflow_falls_back_to_the_tile(rsr):
    """A scenario with more unresolved samples after the first pass's chunk
    budget than its deep queue holds (1024 entries under the test flag; a queue
    otherwise holds one entry per sample): the first tiles queue their samples,
    the tiles that find the queue full finish their walk themselves, and every
    label and count still equals the oracle's."""
    from paper_2604_17066_gb300._lib import RSR_FLAG_TEST_DEEP_CAP
    probs = [sparse_match_problem(64, 200, 4000, 10, 30, seed=8), random_refs_problem(50, 2, 20, 40, seed=9)]
    seeds, offsets, Ns = [41, 42], [0, 5], [100000, 3000]
    P = [rsr.Problem(p.pmf, p.ref_L, p.ref_U, path=POPC) for p in probs]
    P[0].extra_flags = RSR_FLAG_TEST_DEEP_CAP
    b = rsr.Batch(P, seeds, offsets, Ns)
    rsr.rsr_batch(b)
    torch.cuda.synchronize()
    counts = b.counts3.cpu().numpy()
    X = O.sample(probs[0].pmf, seeds[0], offsets[0], Ns[0])
    lab, cnt = O.classify(X, probs[0].ref_L, probs[0].ref_U)
    assert cnt[2] > 40 * 1024       # far more unresolved samples than the queue holds
    for s, p in enumerate(probs):
        if s:
            X = O.sample(p.pmf, seeds[s], offsets[s], Ns[s])
            lab, cnt = O.classify(X, p.ref_L, p.ref_U)
        assert np.array_equal(b.labels[s].cpu().numpy(), lab), s
        assert np.array_equal(counts[s], cnt), s
        assert np.array_equal(b.grad_counts[s].cpu().numpy().reshape(p.n, p.K), O.grad_counts(X, lab, p.K)), s


def mixed_scenarios():
    """Dense scenarios on the tensor cores (path TC), dense scenarios left to the
    autotuner (path AUTO), and bit-packed ones, with ragged sample counts and a
    multi-state encoding."""
    spec = [  # n, K, R_L, R_U, N, path, dense
        (295, 2, 300, 700, 5000, 2, True), (100, 4, 600, 300, 3001, 2, True), (40, 5, 1, 513, 2049, 0, True),
        (120, 3, 130, 129, 257, 0, True), (300, 2, 3000, 9000, 4096, 0, True), (50, 2, 20, 40, 1000, 1, False),
        (64, 4, 30, 30, 2048, 0, False), (200, 2, 600, 5, 1, 2, True)]
    probs = [random_refs_problem(n, K, RL, RU, seed=13 * n + K) for n, K, RL, RU, _, _, _ in spec]
    Ns = [sp[4] for sp in spec]
    paths = [sp[5] for sp in spec]
    dense = [sp[6] for sp in spec]
    seeds = [300 + s for s in range(len(probs))]
    offsets = [11 * s for s in range(len(probs))]
    return probs, seeds, offsets, Ns, paths, dense


def make_mixed_batch(rsr, probs, seeds, offsets, Ns, paths, dense):
    P = [rsr.Problem(p.pmf, p.ref_L, p.ref_U, path=pa, dense=de) for p, pa, de in zip(probs, paths, dense)]
    return rsr.Batch(P, seeds, offsets, Ns)


def check_batch_round(rsr, b, probs, seeds, offsets, Ns, rnd):
    counts = b.counts3.cpu().numpy()
    for s, p in enumerate(probs):
        X = O.sample(p.pmf, seeds[s], offsets[s] + rnd * Ns[s], Ns[s])
        lab, cnt = O.classify(X, p.ref_L, p.ref_U)
        assert np.array_equal(b.labels[s].cpu().numpy(), lab), (rnd, s)
        assert np.array_equal(counts[s], cnt), (rnd, s)
        assert np.array_equal(b.grad_counts[s].cpu().numpy().reshape(p.n, p.K), O.grad_counts(X, lab, p.K)), (rnd, s)


def test_mixed_path_batch_matches_oracle_before_and_after_autotune(rsr):
    """Tensor-core and bit-packed scenarios in one batch: every scenario equals
    the oracle, before tuning (the reference-count rule) and after (timed paths,
    k0, order, grid and tiles per item), on graph replays of the tuned batch,
    and on a cycle-profiled launch (zero rows for tensor-core scenarios)."""
    probs, seeds, offsets, Ns, paths, dense = mixed_scenarios()
    b = make_mixed_batch(rsr, probs, seeds, offsets, Ns, paths, dense)
    rsr.rsr_batch(b)
    torch.cuda.synchronize()
    check_batch_round(rsr, b, probs, seeds, offsets, Ns, 0)
    b2 = make_mixed_batch(rsr, probs, seeds, offsets, Ns, paths, dense)
    grid, order, k0, n_tc, staged, tiles = rsr.rsr_batch_autotune(b2)
    assert n_tc >= 3                      # the three scenarios that ask for the tensor cores
    torch.cuda.synchronize()
    assert int(b2.counts3.abs().sum()) == 0
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        rsr.rsr_batch(b2, stream=torch.cuda.current_stream())
    for rnd in (0, 1):
        b2.counts3.zero_()
        for t in b2.grad_counts:
            t.zero_()
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        check_batch_round(rsr, b2, probs, seeds, offsets, Ns, rnd)
    # the cycle-profiled launches continue the rounds; tensor-core scenarios keep zero rows
    b2.counts3.zero_()
    for t in b2.grad_counts:
        t.zero_()
    prof = rsr.rsr_batch_profile(b2).cpu().numpy()
    torch.cuda.synchronize()
    check_batch_round(rsr, b2, probs, seeds, offsets, Ns, 2)
    for s, pa in enumerate(paths):
        if pa == 2:
            assert (prof[s] == 0).all(), s
        elif pa == 1:
            assert prof[s, 0] == (Ns[s] + 255) // 256 and (prof[s, 1:4] > 0).all(), s


def test_tuning_cache_round_trip(rsr, tmp_path, monkeypatch):
    """With RSR_TUNE_CACHE set, rsr_autotune writes its decision to the JSON
    cache keyed by device and shape (read back here as text)."""
    import json
    path = tmp_path / "tune.json"
    monkeypatch.setenv("RSR_TUNE_CACHE", str(path))
    p = random_refs_problem(96, 2, 700, 2100, seed=17)
    sess = make_session(rsr, p, path=0, dense=True)
    chosen = rsr.rsr_autotune(sess.problem, sess.ws)
    d = json.loads(path.read_text())
    keys = [k for k in d if k.startswith("path/") and "/n96/K2/" in k]
    assert keys and d[keys[0]] == [chosen]
