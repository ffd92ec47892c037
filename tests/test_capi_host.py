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
    assert size >= 300 * 8 + 250000 * 10 * 4 + 250000 * 320
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
