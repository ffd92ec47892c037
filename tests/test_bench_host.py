"""Host-side checks of bench.py's CPU baseline (no GPU): the oracle spread over
spawned processes, each on a contiguous slice of the sample stream, returns the
same counts and gradient counts as one process classifying the whole range."""
import numpy as np

from oracle import oracle as O


def test_oracle_pool_matches_one_process():
    import bench
    import workloads.large as L
    prob = L.c2_rgg()
    seed, offset, n = 3, 12345, 6001
    pool = bench.OraclePool("c2", workers=3)
    try:
        rate, dt = pool.run(prob, seed, offset, n)
    finally:
        pool.close()
    assert rate > 0 and dt > 0
    X = O.sample(prob.pmf, seed, offset, n)
    lab, cnt = O.classify(X, prob.ref_L, prob.ref_U)
    assert np.array_equal(pool.last_counts, cnt)
    assert np.array_equal(pool.last_grad_counts, O.grad_counts(X, lab, prob.K))
