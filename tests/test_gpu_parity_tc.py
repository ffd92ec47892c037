"""GPU parity of the tensor-core (tcgen05 FP8 contraction) path against the
oracle: labels, counts and gradient counts bit-exact on the same seeded
samples, in dense mode (every reference; the CTA-pair kernel) and early-exit
mode (one CTA per MMA), across several reference tiles, several sample blocks
and ragged tails, for binary and multi-state encodings, with and without
overlapping reference pairs."""
import numpy as np
import pytest
import torch

import workloads as W
from helpers import TC, make_session, random_refs_problem, run, tc_executed_tests, tc_kpad
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def check(rsr, prob, seed, offset, N, dense, samples=None):
    sess = make_session(rsr, prob, path=TC, dense=dense)
    got = run(sess, seed, offset, N, samples=None if samples is None else torch.from_numpy(samples).cuda())
    X = O.sample(prob.pmf, seed, offset, N) if samples is None else samples
    lab, cnt = O.classify(X, prob.ref_L, prob.ref_U)
    assert np.array_equal(got["counts3"], cnt), (got["counts3"], cnt)
    assert np.array_equal(got["labels"], lab)
    assert np.array_equal(got["grad_counts"].reshape(prob.n, prob.K), O.grad_counts(X, lab, prob.K))
    full = tc_executed_tests(prob.n, prob.K, prob.R_L, prob.R_U, N, dense=dense)
    if dense:
        assert got["exec_tests"][0] == full
    else:
        assert got["exec_tests"][0] <= full
    return got


@pytest.mark.parametrize("dense", [True, False])
def test_tc_grid_philox(rsr, dense):
    check(rsr, W.c1_grid(), 1, 0, 100000, dense)


def test_tc_grid_exhaustive(rsr):
    p = W.c1_grid()
    check(rsr, p, 0, 0, 1 << p.n, True, samples=O.all_states(p.n, 2))


@pytest.mark.parametrize("n,K,R_L,R_U,N", [(295, 2, 300, 700, 5000), (100, 4, 600, 300, 3001),
                                           (40, 5, 1, 513, 2049), (300, 2, 0, 257, 1000),
                                           (300, 2, 300, 0, 1000), (3, 3, 2, 2, 1), (120, 3, 130, 129, 257),
                                           (120, 4, 300, 600, 3001)])   # 384-byte rows: 128-wide B tiles
@pytest.mark.parametrize("dense", [True, False])
def test_tc_random_refs(rsr, n, K, R_L, R_U, N, dense):
    assert tc_kpad(n, K) <= 512
    check(rsr, random_refs_problem(n, K, R_L, R_U, seed=n * 7 + K), 77, 1000, N, dense)


@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("dense", [True, False])
def test_tc_multistate_with_overlaps(rsr, seed, dense):
    prob = W.random_small_system(n=6, K=4, M_S=3, seed=seed)
    extra_U = prob.ref_L[:1].copy()
    extra_U[0, 0] = 0
    bad = W.Problem("bad", prob.pmf, prob.ref_L, np.concatenate([prob.ref_U, extra_U]))
    for pr in (prob, bad):
        check(rsr, pr, seed, 3, 4099, dense)


def test_tc_rejects_too_wide_encodings(rsr):
    prob = random_refs_problem(68, 16, 3, 3, seed=1)   # 1020 thermometer bits
    P = rsr.Problem(prob.pmf, prob.ref_L, prob.ref_U, path=TC)
    with pytest.raises(rsr.RSRError) as e:
        rsr.Session(P)
    assert e.value.status == -5


def test_tc_bounded_waits_time_out_and_leave_the_context_usable(rsr):
    """Failure detection on the device without a fault: with the test hook the
    reference producer never starts, every bounded wait runs out (about 10 ms),
    the kernel records RSR_ERR_TIMEOUT, frees its tensor memory and returns."""
    from paper_2604_17066_gb300._lib import RSR_FLAG_TEST_STALL
    prob = random_refs_problem(120, 3, 130, 129, seed=2)
    P = rsr.Problem(prob.pmf, prob.ref_L, prob.ref_U, path=TC)
    sess = rsr.Session(P)
    P.extra_flags = RSR_FLAG_TEST_STALL
    sess.classify(1, 0, 4096)
    torch.cuda.synchronize()
    overlap, err = rsr.rsr_workspace_status(sess.ws)
    assert err == -4
    # the context still works: a normal run on a fresh workspace matches the oracle
    P.extra_flags = 0
    check(rsr, prob, 1, 0, 4096, dense=False)


def test_tc_pair_kernel_bounded_waits_time_out_and_leave_the_context_usable(rsr):
    """The same failure detection on the dense CTA-pair kernel: neither CTA's
    producer starts, the leader's and the peer's waits run out, both CTAs agree
    to stop at their cluster barrier, free the pair's tensor memory and return."""
    from paper_2604_17066_gb300._lib import RSR_FLAG_TEST_STALL
    prob = random_refs_problem(120, 3, 130, 129, seed=3)
    P = rsr.Problem(prob.pmf, prob.ref_L, prob.ref_U, path=TC, dense=True)
    sess = rsr.Session(P)
    P.extra_flags = RSR_FLAG_TEST_STALL
    sess.classify(1, 0, 4096)
    torch.cuda.synchronize()
    overlap, err = rsr.rsr_workspace_status(sess.ws)
    assert err == -4
    P.extra_flags = 0
    check(rsr, prob, 1, 0, 4096, dense=True)


@pytest.mark.parametrize("pair", [False, True])
def test_measured_fp8_peak_is_plausible(rsr, pair):
    """rsr_measure_fp8_peak (the tensor roofline's denominator) returns rates
    within the range a GB300 can reach, on single CTAs and on CTA pairs: above
    half of the nominal 4.5 PFLOP/s dense FP8 figure and below twice it."""
    m = rsr.rsr_measure_fp8_peak(0.2, cta_pair=pair)
    for key in ("burst_flops_per_s", "sustained_flops_per_s"):
        assert 2.25e15 < m[key] < 9e15, m
