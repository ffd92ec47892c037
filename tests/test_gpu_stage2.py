"""GPU parity of Stage 2 on the device (rsr_resolve, Sec. 3.5): every
unclassified sample is relabelled exactly as the oracle's Phi says (3 = S <= m',
4 = S >= m'+1), the counts match, the set of lower indices matches (their
order is free), and the gradient with the Stage-2 correction matches."""
import numpy as np
import pytest
import torch

import workloads as W
from helpers import POPC, TC, make_session
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def run_stage2(rsr, prob, system_args, seed, offset, N, path=POPC, cap=None):
    sess = make_session(rsr, prob, path=path)
    out = sess.classify(seed, offset, N, labels=True, grad=True)
    system = rsr.System(*system_args)
    labels = out["labels"]
    u_idx, c2 = rsr.rsr_resolve(sess.problem, system, seed, offset, N, labels, sess.ws,
                                u_lower_idx=None if cap is None else torch.empty(cap, dtype=torch.int64,
                                                                                 device="cuda"))
    torch.cuda.synchronize()
    return sess, out, labels.cpu().numpy(), u_idx, c2.cpu().numpy()


def oracle_stage2(prob, kind, nn, edges, s, t, seed, offset, N, thr=None, m_prime=0):
    X = O.sample(prob.pmf, seed, offset, N)
    lab, cnt = O.classify(X, prob.ref_L, prob.ref_U)
    res, n_lower = O.resolve(kind, nn, edges, s, t, X, lab, m_prime=m_prime, thresholds=thr)
    return X, lab, cnt, res, n_lower


def check(rsr, prob, kind, nn, edges, s, t, seed, offset, N, thr=(), m_prime=0, path=POPC):
    sess, out, labels, u_idx, c2 = run_stage2(rsr, prob, (kind, nn, edges, s, t, list(thr), m_prime), seed,
                                              offset, N, path=path)
    X, lab, cnt, res, n_lower = oracle_stage2(prob, kind, nn, edges, s, t, seed, offset, N,
                                              thr=list(thr) if thr else None, m_prime=m_prime)
    assert np.array_equal(labels, res)
    assert c2.tolist() == [n_lower, int(cnt[2]) - n_lower]
    got_idx = np.sort(u_idx[:n_lower].cpu().numpy())
    assert np.array_equal(got_idx, np.nonzero(res == 3)[0])
    # estimates and the Stage-2 gradient
    counts = out["counts3"].cpu().numpy()
    assert rsr.rsr_estimate(counts, N, n_lower) == O.estimate(cnt, N, n_lower)
    g, _ = rsr.rsr_grad(sess.problem, seed, offset, N, out["grad_counts"], sess.ws, u_lower_idx=u_idx[:n_lower])
    g_o, _ = O.grad(O.grad_counts(X, lab, prob.K, u_lower_idx=np.nonzero(res == 3)[0]), N, prob.pmf)
    np.testing.assert_allclose(g, g_o, rtol=1e-12, atol=0)
    overlap, err = rsr.rsr_workspace_status(sess.ws)
    assert err == 0
    return n_lower, int(cnt[2])


def test_grid_partial_references_resolve_to_complete_labels(rsr):
    p = W.c1_grid()
    part = W.Problem("grid_partial", p.pmf, p.ref_L[::3], p.ref_U[::4])
    n_lower, n_u = check(rsr, part, 0, p.meta["n_nodes"], p.meta["edges"], p.meta["s"], p.meta["t"], 3, 0, 50000)
    assert n_u > 100 and n_lower > 0


@pytest.mark.parametrize("path", [POPC, TC])
def test_c2_connectivity_stage2(rsr, path):
    import workloads.large as L
    p = L.c2_rgg()
    n_lower, n_u = check(rsr, p, 0, p.meta["n_nodes"], p.meta["edges"], p.meta["s"], p.meta["t"], 1, 0, 200000,
                         path=path)
    assert n_u > 1000


@pytest.mark.parametrize("m_prime", [0, 1])
def test_c4_maxflow_stage2(rsr, m_prime):
    import workloads.large as L
    p = L.c4_flow(m_prime)
    thr = (p.meta["l1"], p.meta["l2"])
    n_lower, n_u = check(rsr, p, 1, p.meta["n_nodes"], p.meta["arcs"], p.meta["s"], p.meta["t"], 4, 0, 100000,
                         thr=thr, m_prime=m_prime)
    assert n_u > 0


def test_lower_index_overflow_is_flagged_and_counts_stay_exact(rsr):
    p = W.c1_grid()
    part = W.Problem("grid_partial", p.pmf, p.ref_L[::3], p.ref_U[::4])
    sess, out, labels, u_idx, c2 = run_stage2(
        rsr, part, (0, p.meta["n_nodes"], p.meta["edges"], p.meta["s"], p.meta["t"], [], 0), 3, 0, 50000, cap=4)
    X, lab, cnt, res, n_lower = oracle_stage2(part, 0, p.meta["n_nodes"], p.meta["edges"], p.meta["s"], p.meta["t"],
                                              3, 0, 50000)
    assert n_lower > 4
    assert c2.tolist() == [n_lower, int(cnt[2]) - n_lower]
    assert np.array_equal(labels, res)
    assert rsr.rsr_workspace_status(sess.ws)[1] == 4


def test_grad_rejects_bad_index_without_touching_counts_then_recovers(rsr):
    """rsr_grad checks its listed indices before any count changes: a call with
    an index outside [0, N) fails with RSR_ERR_INVALID_ARG and leaves the counts
    as they were, and the next valid call on the same workspace succeeds (the
    check is per call, not a sticky workspace state)."""
    p = W.c1_grid()
    part = W.Problem("grid_partial", p.pmf, p.ref_L[::3], p.ref_U[::4])
    args = (0, p.meta["n_nodes"], p.meta["edges"], p.meta["s"], p.meta["t"], [], 0)
    sess, out, labels, u_idx, c2 = run_stage2(rsr, part, args, 3, 0, 50000)
    n_lower = int(c2[0])
    before = out["grad_counts"].clone()
    bad = u_idx[:n_lower].clone()
    bad[n_lower // 2] = 50000
    with pytest.raises(rsr.RSRError) as e:
        rsr.rsr_grad(sess.problem, 3, 0, 50000, out["grad_counts"], sess.ws, u_lower_idx=bad)
    assert e.value.status == -1
    assert torch.equal(out["grad_counts"], before)
    g, _ = rsr.rsr_grad(sess.problem, 3, 0, 50000, out["grad_counts"], sess.ws, u_lower_idx=u_idx[:n_lower])
    X, lab, cnt, res, n_lower_o = oracle_stage2(part, *args[:5], 3, 0, 50000)
    g_o, _ = O.grad(O.grad_counts(X, lab, part.K, u_lower_idx=np.nonzero(res == 3)[0]), 50000, part.pmf)
    np.testing.assert_allclose(g, g_o, rtol=1e-12, atol=0)
