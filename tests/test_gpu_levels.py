"""GPU parity of the system-state pmf over all levels (rsr_level_pmf; Sec. 3.5
at every boundary, Sec. 4.5-4.6): per-sample levels, level counts, the
per-boundary classification counts and the number of samples that needed Phi
equal the oracle's on the same seeded samples; the cumulative counts agree with
the single-boundary Stage 2 path (rsr_resolve)."""
import numpy as np
import pytest
import torch

import workloads as W
from helpers import POPC, TC, make_session
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _check(rsr, pmf, boundaries, kind, nn, edges, s, t, thr, seed, offset, N, path=POPC):
    """boundaries: list of (ref_L, ref_U) for m' = 0, 1, ..."""
    nb = len(boundaries)
    sessions = [make_session(rsr, W.Problem("b%d" % b, pmf, L, U), path=path) for b, (L, U) in enumerate(boundaries)]
    system = rsr.System(kind, nn, edges, s, t, thr, 0)
    out = rsr.rsr_level_pmf(sessions, system, seed, offset, N)
    torch.cuda.synchronize()
    want_counts, want_levels = O.level_pmf(pmf, kind, nn, edges, s, t, seed, offset, N, nb + 1,
                                           list(thr) if thr else None)
    assert np.array_equal(out["levels"].cpu().numpy(), want_levels)
    assert np.array_equal(out["level_counts"].cpu().numpy(), want_counts)
    X = O.sample(pmf, seed, offset, N)
    lo = np.zeros(N, dtype=np.int64)
    hi = np.full(N, nb, dtype=np.int64)
    for b, (L, U) in enumerate(boundaries):
        lab, cnt = O.classify(X, L, U)
        assert np.array_equal(out["counts3"][b].cpu().numpy(), cnt)
        hi = np.where(lab == 0, np.minimum(hi, b), hi)
        lo = np.where(lab == 1, np.maximum(lo, b + 1), lo)
    assert int(out["n_phi"].item()) == int((lo < hi).sum())
    assert np.all((want_levels >= lo) & (want_levels <= hi))
    for S in sessions:
        assert rsr.rsr_workspace_status(S.ws)[1] == 0
    return out, sessions, system


def test_level_pmf_c4_three_levels(rsr):
    import workloads.large as L
    p0, p1 = L.c4_flow(0), L.c4_flow(1)
    m = p0.meta
    out, sessions, _ = _check(rsr, p0.pmf, [(p0.ref_L, p0.ref_U), (p1.ref_L, p1.ref_U)], 1, m["n_nodes"],
                              m["arcs"], m["s"], m["t"], (m["l1"], m["l2"]), 4, 0, 30000)
    lc = out["level_counts"].cpu().numpy()
    assert np.all(lc > 0)
    # cumulative counts = the single-boundary Stage 2 result of each boundary
    for b in range(2):
        S = sessions[b]
        res = S.classify(4, 0, 30000, labels=True, grad=False)
        sys_b = rsr.System(1, m["n_nodes"], m["arcs"], m["s"], m["t"], (m["l1"], m["l2"]), b)
        _, c2 = rsr.rsr_resolve(S.problem, sys_b, 4, 0, 30000, res["labels"], S.ws)
        torch.cuda.synchronize()
        assert int(res["counts3"][0].item()) + int(c2[0].item()) == lc[: b + 1].sum()


@pytest.mark.parametrize("path", [POPC, TC])
def test_level_pmf_small_flow_partial_references(rsr, path):
    n_nodes, arcs = 5, [(0, 1), (0, 2), (1, 3), (2, 3), (1, 2), (3, 4), (2, 4)]
    K, thr = 3, (2, 4)
    X = W.all_states(len(arcs), K)
    lv = O.levels(1, n_nodes, arcs, 0, 4, X, list(thr))
    pmf = np.random.default_rng(2).dirichlet(np.ones(K), size=len(arcs))
    bds = []
    for mp in (0, 1):
        L, U = W.reference_sets_from_phi(lv, len(arcs), K, mp)
        bds.append((L[::2], U[::2]))
    out, _, _ = _check(rsr, pmf, bds, 1, n_nodes, arcs, 0, 4, thr, 9, 77, 50001, path=path)
    assert int(out["n_phi"].item()) > 100


def test_level_pmf_global_connectivity_levels(rsr):
    p = W.c1_grid()
    nn, edges = p.meta["n_nodes"], p.meta["edges"]
    X = W.all_states(p.n, 2)
    lv = O.levels(O.PHI_GLOBAL_CONN_LEVEL, nn, edges, 0, 0, X)
    pmf = W.binary_pmf(np.full(p.n, 0.08))
    bds = []
    for mp in (0, 1):
        L, U = W.reference_sets_from_phi(lv, p.n, 2, mp)
        bds.append((L[::3], U[::5]))
    out, _, _ = _check(rsr, pmf, bds, O.PHI_GLOBAL_CONN_LEVEL, nn, edges, 0, 0, (), 3, 0, 40000)
    assert np.all(out["level_counts"].cpu().numpy() > 0)


def test_level_pmf_binary_st_connectivity_and_empty(rsr):
    p = W.c1_grid()
    m = p.meta
    _check(rsr, p.pmf, [(p.ref_L[::4], p.ref_U[::4])], 0, m["n_nodes"], m["edges"], m["s"], m["t"], (), 2, 5, 20000)
    sessions = [make_session(rsr, p)]
    out = rsr.rsr_level_pmf(sessions, rsr.System(0, m["n_nodes"], m["edges"], m["s"], m["t"]), 1, 0, 0)
    assert out["level_counts"].cpu().tolist() == [0, 0]
