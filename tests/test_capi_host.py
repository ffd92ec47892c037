"""C ABI checks that need no GPU: the library loads, exports every entry point
include/rsr.h declares, rejects bad arguments before touching CUDA, and its
host-side estimators agree with the oracle's."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_entry_points():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"RSR_API\s+[\w\s\*]+?\b(rsr_\w+)\s*\(", text)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2604_17066_gb300 import _lib, build
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = set(_header_entry_points())
    for required in ("rsr_classify", "rsr_estimate", "rsr_grad", "rsr_batch", "rsr_prepare",
                     "rsr_workspace_size", "rsr_sample", "rsr_status_string"):
        assert required in names, required


def test_every_declared_symbol_is_exported(lib):
    from paper_2604_17066_gb300 import _lib
    for name in _header_entry_points():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, "binding lacks " + name


def test_flags_match_the_header():
    from paper_2604_17066_gb300 import _lib
    text = open(os.path.join(ROOT, "include", "rsr.h")).read()
    for name in ("RSR_FLAG_DENSE", "RSR_FLAG_NO_INDEX", "RSR_FLAG_TEST_STALL", "RSR_FLAG_TEST_DEEP_CAP",
                 "RSR_FLAG_TEST_TWO_PASS", "RSR_FLAG_TEST_TILES3"):
        m = re.search(r"#define\s+%s\s+(0x[0-9a-fA-F]+|\d+)u" % name, text)
        assert m, name
        assert int(m.group(1), 0) == getattr(_lib, name), name


def _problem_struct(n=4, K=2, R_L=1, R_U=1, pmf=None, path=0):
    from paper_2604_17066_gb300._lib import rsr_problem
    pmf = np.full((n, K), 1.0 / K) if pmf is None else pmf
    s = rsr_problem()
    s.n, s.K, s.R_L, s.R_U, s.path = n, K, R_L, R_U, path
    s.pmf = pmf.ctypes.data
    s.ref_L = 0x1000 if R_L else None   # never dereferenced: validation fails or only sizes are computed
    s.ref_U = 0x2000 if R_U else None
    return s, pmf


def test_workspace_size_and_validation(lib):
    s, pmf = _problem_struct(n=300, K=2, R_L=50000, R_U=200000)
    size = lib.rsr_workspace_size(ctypes.byref(s), 0)
    # thresholds + 10 bit-words per reference + FP8 rows of 320 bytes per reference (padded to 128)
    # + the component-major index of the upper set (10 words per upper reference, chunks of 256)
    assert size >= 300 * 8 + 250000 * 10 * 4 + 250000 * 320 + 782 * 256 * 10 * 4
    assert size % 256 == 0
    bad = [
        _problem_struct(n=0),
        _problem_struct(K=1),
        _problem_struct(R_L=0, R_U=0),
        _problem_struct(pmf=np.array([[0.5, 0.6]] * 4)),       # row sums to 1.1
        _problem_struct(pmf=np.array([[-0.1, 1.1]] * 4)),      # negative probability
        _problem_struct(path=7),
    ]
    for s_bad, pmf_bad in bad:
        assert lib.rsr_workspace_size(ctypes.byref(s_bad), 0) == 0
        assert lib.rsr_prepare(ctypes.byref(s_bad), None, 0, None) in (-1,)
    big, pmf_big = _problem_struct(n=600, K=3)   # 1200 thermometer bits > 1024
    assert lib.rsr_prepare(ctypes.byref(big), None, 0, None) == -5
    ok, pmf_ok = _problem_struct()
    assert lib.rsr_prepare(ctypes.byref(ok), None, 0, None) == -3       # no workspace
    assert lib.rsr_prepare(ctypes.byref(ok), 0x1008, 1 << 20, None) == -3   # misaligned workspace
    assert lib.rsr_status_string(-6) == b"workspace not prepared for this problem/pmf"


@pytest.mark.parametrize("counts,N,nul", [
    ((3, 4, 3), 10, 0), ((1, 999998, 1), 10 ** 6, 1), ((0, 7, 0), 7, 0), ((12345, 67890, 777), 81012, 300),
])
def test_estimate_matches_oracle(lib, counts, N, nul):
    from paper_2604_17066_gb300 import api
    got = api.rsr_estimate(counts, N, nul)
    want = O.estimate(counts, N, nul)
    for k, v in want.items():
        assert got[k] == v or (np.isnan(got[k]) and np.isnan(v)), k


def test_estimate_rejects_inconsistent_counts(lib):
    from paper_2604_17066_gb300 import api
    from paper_2604_17066_gb300._lib import RSRError
    with pytest.raises(RSRError):
        api.rsr_estimate((1, 2, 3), 7)          # counts do not sum to N
    with pytest.raises(RSRError):
        api.rsr_estimate((1, 2, 3), 6, 4)       # more resolved than unclassified


def _system_struct(kind=0, n_nodes=4, s=0, t=3, levels=(), m_prime=0):
    from paper_2604_17066_gb300._lib import rsr_system
    g = rsr_system()
    g.kind, g.n_nodes, g.s, g.t, g.m_prime = kind, n_nodes, s, t, m_prime
    g.src, g.dst = 0x3000, 0x4000            # never dereferenced on the host
    g.n_levels = len(levels)
    for i, v in enumerate(levels):
        g.level_thr[i] = v
    return g


def test_stage1_entry_points_reject_bad_arguments(lib):
    from paper_2604_17066_gb300 import _lib
    E_ARG, E_WS, E_UNS = _lib.RSR_ERR_INVALID_ARG, _lib.RSR_ERR_WORKSPACE, _lib.RSR_ERR_UNSUPPORTED
    s, pmf = _problem_struct(n=4, K=2, R_L=0, R_U=0)
    P = ctypes.c_void_p
    # search workspace: header + counter (512 B) + thresholds rounded to 256 B
    assert lib.rsr_search_workspace_size(ctypes.byref(s)) == 512 + 256
    good = _system_struct()
    fake = P(0x10000)                                 # 256-aligned, never dereferenced
    args = lambda g, ws_bytes=4096, order=0: (ctypes.byref(s), ctypes.byref(g), 1, 0, fake, 2, fake, fake, None,
                                              order, fake, ws_bytes, None)
    assert lib.rsr_boundary_search(*args(good, order=2)) == E_ARG                   # unknown visiting order
    assert lib.rsr_boundary_search(*args(_system_struct(kind=7))) == E_ARG            # unknown Phi
    assert lib.rsr_boundary_search(*args(_system_struct(n_nodes=2000))) == E_UNS      # too many nodes
    assert lib.rsr_boundary_search(*args(_system_struct(t=4))) == E_ARG               # t out of range
    assert lib.rsr_boundary_search(*args(_system_struct(kind=1, levels=(3, 2)))) == E_ARG   # not ascending
    assert lib.rsr_boundary_search(*args(good, ws_bytes=100)) == E_WS
    s3, _ = _problem_struct(n=4, K=3, R_L=0, R_U=0)
    assert lib.rsr_boundary_search(ctypes.byref(s3), ctypes.byref(good), 1, 0, fake, 2, fake, fake, None, 0, fake,
                                   4096, None) == E_ARG                               # connectivity needs K = 2
    # non-dominance scratch: one 32-bit word bucket per reference, 256-byte rounded
    assert lib.rsr_nondominated_scratch_size(4, 2, 100) == 512
    assert lib.rsr_nondominated_scratch_size(300, 2, 1000) == 40192   # 1000 x 10 words x 4 B, rounded
    assert lib.rsr_nondominated_scratch_size(0, 2, 10) == 0
    assert lib.rsr_nondominated(4, 2, 10, fake, 0, fake, None, fake, 4096, None) == E_ARG     # n_keep NULL
    assert lib.rsr_nondominated(4, 2, 10, fake, 0, fake, fake, fake, 16, None) == E_WS
    # Stage 1 options
    opts = _lib.rsr_stage1_opts()
    opts.seed, opts.N, opts.max_starts, opts.eps_u, opts.R_max, opts.max_rounds = 1, 1000, 8, 1e-5, 64, 10
    assert lib.rsr_stage1_workspace_size(ctypes.byref(s), ctypes.byref(opts)) > 0
    for field, bad in (("N", 0), ("max_starts", 0), ("R_max", 0), ("max_rounds", 0), ("eps_u", -1.0),
                       ("search_order", 5)):
        old = getattr(opts, field)
        setattr(opts, field, bad)
        assert lib.rsr_stage1_workspace_size(ctypes.byref(s), ctypes.byref(opts)) == 0, field
        setattr(opts, field, old)
    s_big, _ = _problem_struct(n=4, K=2, R_L=65, R_U=0)   # more initial rows than R_max
    assert lib.rsr_stage1_workspace_size(ctypes.byref(s_big), ctypes.byref(opts)) == 0
    res = _lib.rsr_stage1_result()
    assert lib.rsr_stage1(ctypes.byref(s), ctypes.byref(good), ctypes.byref(opts), fake, fake, None,
                          ctypes.byref(res), fake, 16, None) == E_WS


def test_classify_plan_on_the_host(lib):
    """rsr_classify_plan reports the launches rsr_classify makes: one pass, or
    with deep queues from 2^19 samples (or under the test flag) one pass per
    stage (24 chunk steps at k0 = 2: steps [0, 2), [2, 8), [8, 24)), none for
    N = 0, one on the dense path; a workspace below the layout is refused."""
    from paper_2604_17066_gb300 import _lib
    s, pmf = _problem_struct(n=100, K=2, R_L=3000, R_U=3000, path=_lib.RSR_PATH_POPC)
    base = lib.rsr_workspace_size(ctypes.byref(s), 0)
    queue = lib.rsr_workspace_size(ctypes.byref(s), 1 << 20)
    assert queue >= base + 2 * 8 * (1 << 20) and queue % 256 == 0
    out = np.zeros(3, dtype=np.int32)

    def plan(N, ws_bytes):
        st = lib.rsr_classify_plan(ctypes.byref(s), N, ws_bytes, out.ctypes.data)
        return st, tuple(int(v) for v in out)

    assert plan(1 << 20, base) == (0, (_lib.RSR_PATH_POPC, 1, 0))        # no queue: one pass
    assert plan(1 << 20, queue) == (0, (_lib.RSR_PATH_POPC, 3, 2))       # staged passes, default k0
    assert plan((1 << 19) - 1, queue) == (0, (_lib.RSR_PATH_POPC, 1, 0))  # small calls: one pass
    assert plan(0, queue)[1][1] == 0
    s.flags = _lib.RSR_FLAG_TEST_TWO_PASS
    assert plan(1000, queue) == (0, (_lib.RSR_PATH_POPC, 3, 2))
    s.flags = _lib.RSR_FLAG_DENSE
    assert plan(1 << 20, queue)[1][1] == 1
    s.flags = 0
    assert plan(1 << 20, base - 256)[0] == _lib.RSR_ERR_WORKSPACE
    assert plan(-1, queue)[0] == _lib.RSR_ERR_INVALID_ARG


def test_batch_profile_rejects_bad_arguments(lib):
    """rsr_batch_profile checks its cycle array and the batch's arguments on the
    host, before any CUDA call."""
    from paper_2604_17066_gb300 import _lib
    s, pmf = _problem_struct(n=4, K=2, R_L=0, R_U=0)
    fake = ctypes.c_void_p(0x10000)                    # never dereferenced
    seeds = (ctypes.c_uint64 * 1)(1)
    offs = (ctypes.c_uint64 * 1)(0)
    Ns = (ctypes.c_int64 * 1)(1000)
    call = lambda S, cycles: lib.rsr_batch_profile(ctypes.byref(s), S, seeds, offs, Ns, None, fake, None, fake,
                                                   1 << 20, None, cycles)
    assert call(1, None) == _lib.RSR_ERR_INVALID_ARG   # no cycle array
    assert call(0, fake) == _lib.RSR_ERR_INVALID_ARG   # no scenario
