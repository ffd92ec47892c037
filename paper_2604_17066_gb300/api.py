"""Python binding of librsr: the C entry points under the same names, taking
torch tensors for device buffers (argument marshalling only), plus a small
session object and a torch.autograd.Function for the score-function gradient.

Every step of the hot path runs in librsr's CUDA kernels; nothing here computes
on the host beyond building argument structs.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np
import torch

from . import _lib
from ._lib import (RSR_FLAG_DENSE, RSR_FLAG_NO_INDEX, RSR_PATH_AUTO, RSR_PATH_POPC, RSR_PATH_TC,  # noqa: F401
                   RSR_PHI_GLOBAL_CONN_LEVEL, RSR_PHI_GLOBAL_CONNECTIVITY, RSR_PHI_ST_CONNECTIVITY,
                   RSR_PHI_ST_MAXFLOW_LEVELS, RSR_SEARCH_INDEX_ORDER, RSR_SEARCH_PERMUTED, RSRError, check,
                   rsr_estimate_out,
                   rsr_problem, rsr_system)


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


class Problem:
    """pmf (host, n x K fp64) and reference states (device uint8) of one
    threshold m'.  Keeps the buffers alive for as long as the C struct points
    at them."""

    def __init__(self, pmf, ref_L, ref_U, path: int = RSR_PATH_AUTO, dense: bool = False,
                 device: Optional[torch.device] = None, index: bool = True):
        self.pmf = np.ascontiguousarray(pmf, dtype=np.float64)
        if self.pmf.ndim != 2:
            raise ValueError("pmf must be n x K")
        n = self.pmf.shape[0]
        dev = device or torch.device("cuda", torch.cuda.current_device())
        self.ref_L = torch.as_tensor(np.asarray(ref_L, dtype=np.uint8).reshape(-1, n)).to(dev).contiguous()
        self.ref_U = torch.as_tensor(np.asarray(ref_U, dtype=np.uint8).reshape(-1, n)).to(dev).contiguous()
        self.path = int(path)
        self.dense = bool(dense)
        self.index = bool(index)   # bit-packed path: upper set through its component-major index
        self.extra_flags = 0   # further RSR_FLAG_* bits (e.g. the failure-detection test hook)

    @property
    def n(self) -> int:
        return int(self.pmf.shape[0])

    @property
    def K(self) -> int:
        return int(self.pmf.shape[1])

    @property
    def R_L(self) -> int:
        return int(self.ref_L.shape[0])

    @property
    def R_U(self) -> int:
        return int(self.ref_U.shape[0])

    def struct(self) -> rsr_problem:
        s = rsr_problem()
        s.n, s.K = self.n, self.K
        s.pmf = self.pmf.ctypes.data
        s.R_L, s.R_U = self.R_L, self.R_U
        s.ref_L = self.ref_L.data_ptr() if self.R_L else None
        s.ref_U = self.ref_U.data_ptr() if self.R_U else None
        s.path = self.path
        s.flags = ((RSR_FLAG_DENSE if self.dense else 0) | (0 if self.index else RSR_FLAG_NO_INDEX) |
                   int(self.extra_flags))
        return s


# ---------------------------------------------------------------------------
# the C entry points, same names
# ---------------------------------------------------------------------------
def rsr_workspace_size(problem: Problem, N: int = 0) -> int:
    s = problem.struct()
    size = _lib.load().rsr_workspace_size(ctypes.byref(s), int(N))
    if size == 0:
        raise RSRError(_lib.RSR_ERR_INVALID_ARG, "rsr_workspace_size")
    return int(size)


def alloc_workspace(problem: Problem, N: int = 0) -> torch.Tensor:
    ws = torch.empty(rsr_workspace_size(problem, N) + 256, dtype=torch.uint8, device="cuda")
    off = (-ws.data_ptr()) % 256
    return ws[off:off + rsr_workspace_size(problem, N)]


def rsr_prepare(problem: Problem, ws: torch.Tensor, stream=None) -> None:
    s = problem.struct()
    check(_lib.load().rsr_prepare(ctypes.byref(s), _ptr(ws), ws.numel(), _stream(stream)), "rsr_prepare")


def rsr_update_pmf(problem: Problem, ws: torch.Tensor, stream=None) -> None:
    s = problem.struct()
    check(_lib.load().rsr_update_pmf(ctypes.byref(s), _ptr(ws), ws.numel(), _stream(stream)), "rsr_update_pmf")


def rsr_classify(problem: Problem, seed: int, offset: int, N: int, ws: torch.Tensor,
                 counts3: torch.Tensor, samples: Optional[torch.Tensor] = None,
                 labels: Optional[torch.Tensor] = None, grad_counts: Optional[torch.Tensor] = None,
                 exec_tests: Optional[torch.Tensor] = None, stream=None) -> None:
    s = problem.struct()
    check(_lib.load().rsr_classify(ctypes.byref(s), int(seed), int(offset), int(N), _ptr(samples), _ptr(labels),
                                   _ptr(counts3), _ptr(grad_counts), _ptr(exec_tests), _ptr(ws), ws.numel(),
                                   _stream(stream)), "rsr_classify")


def rsr_classify_plan(problem: Problem, N: int, ws: torch.Tensor):
    """(path, kernel launches, k0) that rsr_classify would use for N samples
    in the prepared workspace ws (host only)."""
    out = np.zeros(3, dtype=np.int32)
    s = problem.struct()
    check(_lib.load().rsr_classify_plan(ctypes.byref(s), int(N), ws.numel(), out.ctypes.data), "rsr_classify_plan")
    return int(out[0]), int(out[1]), int(out[2])


def rsr_estimate(counts3, N: int, n_u_lower: int = 0) -> dict:
    c = np.ascontiguousarray(np.asarray(counts3, dtype=np.int64).reshape(3))
    out = rsr_estimate_out()
    check(_lib.load().rsr_estimate(c.ctypes.data, int(N), int(n_u_lower), ctypes.byref(out)), "rsr_estimate")
    return {name: getattr(out, name) for name, _ in rsr_estimate_out._fields_}


def rsr_grad(problem: Problem, seed: int, offset: int, N: int, grad_counts: torch.Tensor, ws: torch.Tensor,
             u_lower_idx: Optional[torch.Tensor] = None, stream=None):
    s = problem.struct()
    g = np.zeros((problem.n, problem.K), dtype=np.float64)
    se = np.zeros_like(g)
    m = 0 if u_lower_idx is None else int(u_lower_idx.numel())
    check(_lib.load().rsr_grad(ctypes.byref(s), int(seed), int(offset), int(N), _ptr(grad_counts),
                               _ptr(u_lower_idx) if m else None, m, g.ctypes.data, se.ctypes.data, _ptr(ws),
                               ws.numel(), _stream(stream)), "rsr_grad")
    return g, se


def rsr_sample(problem: Problem, seed: int, offset: int, N: int, ws: torch.Tensor,
               states: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    if states is None:
        states = torch.empty((N, problem.n), dtype=torch.uint8, device="cuda")
    s = problem.struct()
    check(_lib.load().rsr_sample(ctypes.byref(s), int(seed), int(offset), int(N), _ptr(states), _ptr(ws),
                                 ws.numel(), _stream(stream)), "rsr_sample")
    return states


def rsr_workspace_status(ws: torch.Tensor, stream=None):
    out = np.zeros(2, dtype=np.int32)
    check(_lib.load().rsr_workspace_status(_ptr(ws), out.ctypes.data, _stream(stream)), "rsr_workspace_status")
    return int(out[0]), int(out[1])


# ---------------------------------------------------------------------------
# convenience layer
# ---------------------------------------------------------------------------
class Session:
    """A prepared workspace for one Problem: classify batches of samples,
    estimate, and differentiate, reusing the encoded references (the references
    stay valid when the pmf changes, Sec. 5)."""

    def __init__(self, problem: Problem, stream=None, max_samples: int = 1 << 20):
        # the workspace holds a deep queue for calls of up to max_samples samples
        # (the bit-packed path's later stages; larger calls defer fewer samples)
        self.problem = problem
        self.stream = stream
        self.ws = alloc_workspace(problem, max_samples)
        rsr_prepare(problem, self.ws, stream)

    def set_pmf(self, pmf) -> None:
        self.problem.pmf = np.ascontiguousarray(pmf, dtype=np.float64)
        rsr_update_pmf(self.problem, self.ws, self.stream)

    def classify(self, seed: int, offset: int, N: int, samples: Optional[torch.Tensor] = None,
                 labels: bool = True, grad: bool = False, count_tests: bool = False) -> dict:
        dev = self.ws.device
        out = {"counts3": torch.zeros(3, dtype=torch.int64, device=dev)}
        out["labels"] = torch.empty(N, dtype=torch.uint8, device=dev) if labels else None
        out["grad_counts"] = (torch.zeros(self.problem.n * self.problem.K, dtype=torch.int64, device=dev)
                              if grad else None)
        out["exec_tests"] = torch.zeros(2, dtype=torch.int64, device=dev) if count_tests else None
        rsr_classify(self.problem, seed, offset, N, self.ws, out["counts3"], samples, out["labels"],
                     out["grad_counts"], out["exec_tests"], self.stream)
        return out

    def overlap(self) -> bool:
        return rsr_workspace_status(self.ws, self.stream)[0] != 0


class RSRProb(torch.autograd.Function):
    """P_hat(S <= m') from N samples as a differentiable function of the pmf.

    forward(pmf, session, seed, offset, N) -> 0-d fp64 tensor; backward gives
    grad_output * dP/dq_{i,k} from the same samples (score function, computed
    by rsr_grad from the per-state counts of I^L samples)."""

    @staticmethod
    def forward(ctx, pmf: torch.Tensor, session: Session, seed: int, offset: int, N: int):
        session.set_pmf(pmf.detach().cpu().numpy())
        out = session.classify(seed, offset, N, labels=False, grad=True)
        counts = out["counts3"].cpu().numpy()
        est = rsr_estimate(counts, N)
        ctx.session, ctx.seed, ctx.offset, ctx.N = session, seed, offset, N
        ctx.grad_counts = out["grad_counts"]
        return torch.tensor(est["P_lower"], dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_output):
        g, _ = rsr_grad(ctx.session.problem, ctx.seed, ctx.offset, ctx.N, ctx.grad_counts, ctx.session.ws,
                        stream=ctx.session.stream)
        return grad_output * torch.from_numpy(g), None, None, None, None


# ---------------------------------------------------------------------------
# batched launch
# ---------------------------------------------------------------------------
class Batch:
    """S problems (scenarios) prepared in one workspace and classified by one
    persistent launch per rsr_batch call.  Outputs live on the device:
    labels[s] (N_s uint8, optional), counts3 (S x 3 int64) and grad_counts[s]
    (n_s*K_s int64, optional); counts are accumulated (zero them between
    launches if needed)."""

    def __init__(self, problems, seeds, offsets, Ns, labels: bool = True, grad: bool = True, stream=None):
        self.problems = list(problems)
        S = len(self.problems)
        self.S = S
        self.stream = stream
        self._structs = (rsr_problem * S)(*[p.struct() for p in self.problems])
        self.seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
        self.offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        self.Ns = np.ascontiguousarray(Ns, dtype=np.int64)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.counts3 = torch.zeros((S, 3), dtype=torch.int64, device=dev)
        self.labels = [torch.empty(int(n), dtype=torch.uint8, device=dev) for n in self.Ns] if labels else None
        self.grad_counts = ([torch.zeros(p.n * p.K, dtype=torch.int64, device=dev) for p in self.problems]
                            if grad else None)
        self._lab_ptrs = (ctypes.c_void_p * S)(*[t.data_ptr() for t in self.labels]) if labels else None
        self._grad_ptrs = (ctypes.c_void_p * S)(*[t.data_ptr() for t in self.grad_counts]) if grad else None
        size = _lib.load().rsr_batch_workspace_size(self._structs, S, self.Ns.ctypes.data)
        if size == 0:
            raise RSRError(_lib.RSR_ERR_INVALID_ARG, "rsr_batch_workspace_size")
        raw = torch.empty(size + 256, dtype=torch.uint8, device=dev)
        off = (-raw.data_ptr()) % 256
        self.ws = raw[off:off + size]
        self._args = None
        rsr_batch_prepare(self)

    def args(self):
        return (self._structs, self.S, self.seeds.ctypes.data, self.offsets.ctypes.data, self.Ns.ctypes.data,
                ctypes.cast(self._lab_ptrs, ctypes.c_void_p) if self._lab_ptrs is not None else None,
                self.counts3.data_ptr(),
                ctypes.cast(self._grad_ptrs, ctypes.c_void_p) if self._grad_ptrs is not None else None,
                self.ws.data_ptr(), self.ws.numel())


def rsr_batch_prepare(batch: Batch, stream=None) -> None:
    check(_lib.load().rsr_batch_prepare(*batch.args(), _stream(stream if stream is not None else batch.stream)),
          "rsr_batch_prepare")


def rsr_batch(batch: Batch, stream=None) -> None:
    check(_lib.load().rsr_batch(*batch.args(), _stream(stream if stream is not None else batch.stream)),
          "rsr_batch")


def rsr_batch_profile(batch: Batch, stream=None) -> torch.Tensor:
    """rsr_batch (same outputs; advances the round) with a cycle profile of the
    bit-packed launches: a device int64 [S, 8] tensor, per scenario the tile
    pass's tiles and its set-up, sampling and chunk-walk SM cycles (summed over
    items, clock64 of each item's block), then the same four for the later
    stages (groups of queued samples).  Tensor-core scenarios keep zeros."""
    st = stream if stream is not None else batch.stream
    cycles = torch.empty((batch.S, 8), dtype=torch.int64, device=batch.counts3.device)
    check(_lib.load().rsr_batch_profile(*batch.args(), _stream(st), cycles.data_ptr()), "rsr_batch_profile")
    return cycles


def rsr_batch_autotune(batch: Batch, stream=None):
    """Tunes the batch's launches; returns (grid, order, k0, n_tc, staged, tiles):
    blocks of the bit-packed persistent grid, work order (0 = longest scenarios
    first, 1 = as given), the first pass's reference-chunk budget (0 = one
    pass), the number of scenarios on the tensor-core pair kernel, whether the
    later passes are staged (1) or one stage to the end (0), and the
    consecutive 256-sample tiles per first-pass work item."""
    chosen = np.zeros(6, dtype=np.int32)
    check(_lib.load().rsr_batch_autotune(*batch.args(), _stream(stream if stream is not None else batch.stream),
                                         chosen.ctypes.data), "rsr_batch_autotune")
    return tuple(int(x) for x in chosen)


def rsr_batch_grad(batch: Batch, stream=None):
    """FP64 gradients and standard errors of every scenario from the batch's
    gradient counts: lists of n_s x K_s arrays."""
    if batch.grad_counts is None:
        raise ValueError("batch was built without gradient counts")
    g = [np.zeros((p.n, p.K), dtype=np.float64) for p in batch.problems]
    se = [np.zeros_like(x) for x in g]
    gp = (ctypes.c_void_p * batch.S)(*[x.ctypes.data for x in g])
    sp = (ctypes.c_void_p * batch.S)(*[x.ctypes.data for x in se])
    check(_lib.load().rsr_batch_grad(batch._structs, batch.S, batch.Ns.ctypes.data,
                                     ctypes.cast(batch._grad_ptrs, ctypes.c_void_p), ctypes.cast(gp, ctypes.c_void_p),
                                     ctypes.cast(sp, ctypes.c_void_p),
                                     _stream(stream if stream is not None else batch.stream)), "rsr_batch_grad")
    return g, se


def rsr_autotune(problem: Problem, ws: torch.Tensor, stream=None) -> int:
    s = problem.struct()
    chosen = ctypes.c_int32(0)
    check(_lib.load().rsr_autotune(ctypes.byref(s), _ptr(ws), ws.numel(), _stream(stream), ctypes.byref(chosen)),
          "rsr_autotune")
    return int(chosen.value)


def rsr_classify_static(problem: Problem, seed: int, offset: int, N: int, counts3: torch.Tensor,
                        samples: Optional[torch.Tensor] = None, labels: Optional[torch.Tensor] = None,
                        grad_counts: Optional[torch.Tensor] = None, stream=None) -> None:
    """rsr_classify_static: classification whose workspace is a 4 MiB device
    array owned by the library, for callers that cannot allocate device
    memory (see include/rsr.h)."""
    s = problem.struct()
    check(_lib.load().rsr_classify_static(ctypes.byref(s), int(seed), int(offset), int(N), _ptr(samples),
                                          _ptr(labels), _ptr(counts3), _ptr(grad_counts), _stream(stream)),
          "rsr_classify_static")


class System:
    """A built-in system function Phi with its threshold m': s-t connectivity
    or global connectivity (level) over undirected edges (binary components),
    or s-t max-flow levels over directed arcs (component state = capacity).
    edges: n x 2 node indices, one row per component."""

    def __init__(self, kind: int, n_nodes: int, edges, s: int, t: int, level_thr=(), m_prime: int = 0,
                 device: Optional[torch.device] = None):
        e = np.asarray(edges, dtype=np.int32).reshape(-1, 2)
        dev = device or torch.device("cuda", torch.cuda.current_device())
        self.src = torch.from_numpy(np.ascontiguousarray(e[:, 0])).to(dev)
        self.dst = torch.from_numpy(np.ascontiguousarray(e[:, 1])).to(dev)
        self.kind, self.n_nodes, self.s, self.t = int(kind), int(n_nodes), int(s), int(t)
        self.level_thr = [int(v) for v in level_thr]
        self.m_prime = int(m_prime)

    def struct(self) -> rsr_system:
        st = rsr_system()
        st.kind, st.n_nodes = self.kind, self.n_nodes
        st.src, st.dst = self.src.data_ptr(), self.dst.data_ptr()
        st.s, st.t = self.s, self.t
        st.n_levels = len(self.level_thr)
        for i, v in enumerate(self.level_thr):
            st.level_thr[i] = v
        st.m_prime = self.m_prime
        return st


def rsr_resolve(problem: Problem, system: System, seed: int, offset: int, N: int, labels: torch.Tensor,
                ws: torch.Tensor, u_lower_idx: Optional[torch.Tensor] = None, counts2: Optional[torch.Tensor] = None,
                stream=None):
    """Stage 2: relabel unclassified samples 3 (S <= m') or 4 by evaluating Phi
    on the device; returns (u_lower_idx, counts2) device tensors."""
    dev = labels.device
    if u_lower_idx is None:
        u_lower_idx = torch.empty(max(int(N), 1), dtype=torch.int64, device=dev)
    if counts2 is None:
        counts2 = torch.zeros(2, dtype=torch.int64, device=dev)
    s = problem.struct()
    g = system.struct()
    check(_lib.load().rsr_resolve(ctypes.byref(s), ctypes.byref(g), int(seed), int(offset), int(N), _ptr(labels),
                                  _ptr(u_lower_idx), u_lower_idx.numel(), _ptr(counts2), _ptr(ws), ws.numel(),
                                  _stream(stream)), "rsr_resolve")
    return u_lower_idx, counts2


# ---------------------------------------------------------------------------
# Stage 1: boundary search, reference-set maintenance, the round loop
# ---------------------------------------------------------------------------
def _aligned(nbytes: int, device) -> torch.Tensor:
    buf = torch.empty(int(nbytes) + 256, dtype=torch.uint8, device=device)
    off = (-buf.data_ptr()) % 256
    return buf[off:off + int(nbytes)]


def rsr_boundary_search(problem: Problem, system: System, seed: int, offset: int, starts: torch.Tensor,
                        ws: Optional[torch.Tensor] = None, phi_evals: Optional[torch.Tensor] = None,
                        order: int = _lib.RSR_SEARCH_INDEX_ORDER, stream=None):
    """Componentwise boundary search from samples offset + starts[j]; returns
    (refs [n_starts x n] uint8, side [n_starts] uint8, phi_evals [1] int64) on the device."""
    dev = starts.device
    s = problem.struct()
    lib = _lib.load()
    if ws is None:
        size = lib.rsr_search_workspace_size(ctypes.byref(s))
        if size == 0:
            raise RSRError(_lib.RSR_ERR_INVALID_ARG, "rsr_search_workspace_size")
        ws = _aligned(size, dev)
    S = int(starts.numel())
    refs = torch.empty((S, problem.n), dtype=torch.uint8, device=dev)
    side = torch.empty(S, dtype=torch.uint8, device=dev)
    if phi_evals is None:
        phi_evals = torch.zeros(1, dtype=torch.int64, device=dev)
    g = system.struct()
    check(lib.rsr_boundary_search(ctypes.byref(s), ctypes.byref(g), int(seed), int(offset), _ptr(starts), S,
                                  _ptr(refs), _ptr(side), _ptr(phi_evals), int(order), _ptr(ws), ws.numel(),
                                  _stream(stream)),
          "rsr_boundary_search")
    return refs, side, phi_evals


def rsr_nondominated(refs: torch.Tensor, K: int, upper: bool, stream=None):
    """keep mask (uint8) of the non-dominated references of one set, and the kept count (device int64[1])."""
    R, n = (int(v) for v in refs.shape)
    lib = _lib.load()
    size = lib.rsr_nondominated_scratch_size(n, int(K), R)
    if size == 0:
        raise RSRError(_lib.RSR_ERR_INVALID_ARG, "rsr_nondominated_scratch_size")
    scratch = _aligned(size, refs.device)
    keep = torch.empty(R, dtype=torch.uint8, device=refs.device)
    n_keep = torch.zeros(1, dtype=torch.int64, device=refs.device)
    check(lib.rsr_nondominated(n, int(K), R, _ptr(refs) if R else None, 1 if upper else 0,
                               _ptr(keep) if R else None, _ptr(n_keep), _ptr(scratch), scratch.numel(),
                               _stream(stream)), "rsr_nondominated")
    return keep, n_keep


def rsr_stage1(pmf, system: System, seed: int, N: int, max_starts: int, eps_u: float, R_max: int,
               max_rounds: int, ref_L=None, ref_U=None, path: int = RSR_PATH_POPC, stream=None,
               device: Optional[torch.device] = None, order: int = _lib.RSR_SEARCH_INDEX_ORDER):
    """Stage 1 on the device.  Returns dict(ref_L, ref_U (device uint8),
    history (rounds x 4 int64: n_u, R_L, R_U, starts), rounds, stop, n_u_last,
    phi_evals)."""
    pmf = np.ascontiguousarray(pmf, dtype=np.float64)
    n = pmf.shape[0]
    dev = device or torch.device("cuda", torch.cuda.current_device())
    L0 = np.zeros((0, n), np.uint8) if ref_L is None else np.asarray(ref_L, dtype=np.uint8).reshape(-1, n)
    U0 = np.zeros((0, n), np.uint8) if ref_U is None else np.asarray(ref_U, dtype=np.uint8).reshape(-1, n)
    bufL = torch.zeros((int(R_max), n), dtype=torch.uint8, device=dev)
    bufU = torch.zeros((int(R_max), n), dtype=torch.uint8, device=dev)
    if L0.shape[0]:
        bufL[:L0.shape[0]] = torch.from_numpy(np.ascontiguousarray(L0)).to(dev)
    if U0.shape[0]:
        bufU[:U0.shape[0]] = torch.from_numpy(np.ascontiguousarray(U0)).to(dev)
    prob = rsr_problem()
    prob.n, prob.K = n, pmf.shape[1]
    prob.pmf = pmf.ctypes.data
    prob.R_L, prob.R_U = L0.shape[0], U0.shape[0]
    prob.ref_L = prob.ref_U = None
    prob.path, prob.flags = int(path), 0
    opts = _lib.rsr_stage1_opts()
    opts.seed, opts.N, opts.max_starts = int(seed), int(N), int(max_starts)
    opts.eps_u, opts.R_max, opts.max_rounds = float(eps_u), int(R_max), int(max_rounds)
    opts.search_order = int(order)
    lib = _lib.load()
    size = lib.rsr_stage1_workspace_size(ctypes.byref(prob), ctypes.byref(opts))
    if size == 0:
        raise RSRError(_lib.RSR_ERR_INVALID_ARG, "rsr_stage1_workspace_size")
    ws = _aligned(size, dev)
    hist = np.zeros((int(max_rounds), 4), dtype=np.int64)
    res = _lib.rsr_stage1_result()
    g = system.struct()
    check(lib.rsr_stage1(ctypes.byref(prob), ctypes.byref(g), ctypes.byref(opts), _ptr(bufL), _ptr(bufU),
                         hist.ctypes.data, ctypes.byref(res), _ptr(ws), ws.numel(), _stream(stream)), "rsr_stage1")
    return dict(ref_L=bufL[:res.R_L], ref_U=bufU[:res.R_U], history=hist[:res.rounds], rounds=res.rounds,
                stop=res.stop, n_u_last=res.n_u_last, phi_evals=res.phi_evals)


def rsr_level_pmf(sessions, system: System, seed: int, offset: int, N: int, levels: bool = True, stream=None):
    """System-state pmf over all levels in one call: sessions[b] is a prepared
    Session of boundary m' = b.  Returns dict(level_counts [M_S], levels [N] or
    None, counts3 [n_boundaries x 3], n_phi) as device tensors."""
    nb = len(sessions)
    dev = sessions[0].ws.device
    structs = (rsr_problem * nb)(*[S.problem.struct() for S in sessions])
    ws_ptrs = (ctypes.c_void_p * nb)(*[_ptr(S.ws) for S in sessions])
    ws_sizes = (ctypes.c_size_t * nb)(*[S.ws.numel() for S in sessions])
    scratch = torch.empty(max(nb * int(N), 1), dtype=torch.uint8, device=dev)
    lv = torch.empty(max(int(N), 1), dtype=torch.uint8, device=dev) if levels else None
    counts3 = torch.zeros((nb, 3), dtype=torch.int64, device=dev)
    level_counts = torch.zeros(nb + 1, dtype=torch.int64, device=dev)
    n_phi = torch.zeros(1, dtype=torch.int64, device=dev)
    g = system.struct()
    check(_lib.load().rsr_level_pmf(structs, nb, ws_ptrs, ws_sizes, ctypes.byref(g), int(seed), int(offset), int(N),
                                    _ptr(scratch), _ptr(lv), _ptr(counts3), _ptr(level_counts), _ptr(n_phi),
                                    _stream(stream)), "rsr_level_pmf")
    return dict(level_counts=level_counts, levels=None if lv is None else lv[:int(N)], counts3=counts3,
                n_phi=n_phi)


def rsr_measure_int_peak(stream=None) -> dict:
    """rsr_measure_int_peak: measured LOP3 and IMAD.WIDE thread-ops per second
    of the current GPU (the bit-packed classifiers' roofline denominator)."""
    lop3 = ctypes.c_double(0.0)
    imad = ctypes.c_double(0.0)
    check(_lib.load().rsr_measure_int_peak(ctypes.addressof(lop3), ctypes.addressof(imad), _stream(stream)),
          "rsr_measure_int_peak")
    return {"lop3_ops_per_s": lop3.value, "imad_ops_per_s": imad.value}


def rsr_measure_philox_rate(stream=None) -> float:
    """rsr_measure_philox_rate: Philox4x32-10 blocks per second of the library's
    generator on the current GPU."""
    rate = ctypes.c_double(0.0)
    check(_lib.load().rsr_measure_philox_rate(ctypes.addressof(rate), _stream(stream)), "rsr_measure_philox_rate")
    return rate.value


def rsr_measure_fp8_peak(seconds: float = 0.0, cta_pair: bool = False, stream=None) -> dict:
    """rsr_measure_fp8_peak: measured dense FP8 tensor-core rate of the current
    GPU (tcgen05.mma kind::f8f6f4, E4M3 operands, FP32 accumulation), in
    flop/s, for single CTAs (M = 128) or CTA pairs (cta_group::2, M = 256): the
    fastest single ~16 ms launch (burst) and, for seconds > 0, back-to-back
    launches for that long (sustained; 0.0 when skipped)."""
    burst = ctypes.c_double(0.0)
    sustained = ctypes.c_double(0.0)
    check(_lib.load().rsr_measure_fp8_peak(1 if cta_pair else 0, float(seconds), ctypes.addressof(burst),
                                           ctypes.addressof(sustained), _stream(stream)), "rsr_measure_fp8_peak")
    return {"burst_flops_per_s": burst.value, "sustained_flops_per_s": sustained.value}
