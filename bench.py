"""Benchmark of the RSR hot path on GB300 (one JSON line on rank 0).

Default workload: the 200k-reference classifier (n = 300 binary components,
R_U = 2e5 DNF terms, R_L = 5e4 greedy cuts, N = 4e6 Philox samples per GPU,
p_up = 0.9), classified in dense mode (every sample against every reference,
the paper's O(H N M R) product, Sec. 3.3 complexity) on the tensor-core path,
with the fused gradient counts and the fp64 estimates and gradient (one step =
every hot-path step: thresholds, sampling, encoding, classification,
estimates, gradient).  Extra keys report the same workload with early exit,
forward-only vs forward+gradient, and the 119-node / 295-edge graph workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "samples classified/s and dominance tests/s vs roofline; fwd vs fwd+grad"
UNIT = "samples/s"


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _captured_traffic(workload_tag):
    """DRAM bytes per launch of the dense tensor-core kernel from the committed
    ncu record, if its sources are unchanged since the capture (else None)."""
    import hashlib
    rec = os.path.join(ROOT, "profiles", "classify_tc2_c3_dense_traffic.json")
    try:
        d = json.load(open(rec))
        h = hashlib.sha1()
        for src in d["sources"]:
            h.update(open(os.path.join(ROOT, src), "rb").read())
        if h.hexdigest() != d["source_sha1"]:
            return None
        if not workload_tag.startswith(d["workload"].split()[0]) or "_N" in workload_tag.split("p0.9")[-1]:
            return None
        return float(d["dram_bytes_read"]) + float(d["dram_bytes_write"])
    except (OSError, KeyError, ValueError):
        return None


def _workload(name):
    import workloads.large as L
    if name == "c3":
        p = L.c3_dnf()
        return p, 4_000_000, "c3_dnf300_refs200000U+50000L_N4e6_p0.9"
    if name == "c2":
        p = L.c2_rgg()
        return p, 1_000_000, "c2_rgg119n295e_N1e6"
    if name == "c4":
        p = L.c4_flow(0)
        return p, 1_000_000, "c4_flow40n100a_K4_m0_N1e6"
    raise ValueError(name)


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.proc = None
        self.uuid = uuid

    def __enter__(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd[1:1] = ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]
        return False

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}

    def power_max(self):
        pw = []
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            try:
                pw.append(float(f[3]))
            except (IndexError, ValueError):
                continue
        return max(pw) if pw else None


def measure_fp8_peak(rsr, torch, uuid, seconds=3.0):
    """The tensor roofline's denominator, measured on this GPU: librsr's own
    back-to-back tcgen05 FP8 MMA loops (rsr_measure_fp8_peak), on single CTAs
    (M = 128) and on CTA pairs (cta_group::2, M = 256), each a burst with the SM
    clock sampled while it ran, plus a sustained run of the pair variant; the
    peak is the larger burst.  cuBLASLt's FP8 GEMM (torch._scaled_mm, 8192^3)
    is a cross-check."""
    out = {}
    for key, pair in (("cta1", False), ("cta_pair", True)):
        with Clocks(uuid) as ck:
            torch.cuda.synchronize()
            r = rsr.rsr_measure_fp8_peak(0.0, cta_pair=pair)
        out["burst_tflops_" + key] = r["burst_flops_per_s"] / 1e12
        out["burst_clocks_" + key] = ck.summary()
    out["burst_tflops"] = max(out["burst_tflops_cta1"], out["burst_tflops_cta_pair"])
    with Clocks(uuid) as ck:
        torch.cuda.synchronize()
        r = rsr.rsr_measure_fp8_peak(seconds, cta_pair=True)
    out["sustained_tflops"] = r["sustained_flops_per_s"] / 1e12
    out["sustained_clocks"] = ck.summary()
    out["sustained_power_w_max"] = ck.power_max()
    try:
        n = 8192
        a = (torch.rand(n, n, device="cuda") - 0.5).to(torch.float8_e4m3fn)
        b = (torch.rand(n, n, device="cuda") - 0.5).to(torch.float8_e4m3fn)
        one = torch.ones((), device="cuda")
        best = 1e30
        for _ in range(6):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            e[0].record()
            torch._scaled_mm(a, b.t(), scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
            e[1].record()
            torch.cuda.synchronize()
            best = min(best, e[0].elapsed_time(e[1]))
        out["cublaslt_fp8_8192_tflops"] = 2.0 * n ** 3 / (best / 1000.0) / 1e12
        del a, b
    except Exception as exc:  # the cross-check is optional; the measured peak above stands alone
        out["cublaslt_fp8_8192_tflops"] = None
        out["cublaslt_error"] = str(exc)[:200]
    return out


def _stage1_timed(rsr, torch, pmf, system, B, R_max, rounds, order):
    rsr.rsr_stage1(pmf, system, 99, 10000, 16, 1e-5, 64, 2, order=order)      # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s1 = rsr.rsr_stage1(pmf, system, 2, 1_000_000, B, 1e-5, R_max, rounds, order=order)
    torch.cuda.synchronize()
    return s1, time.perf_counter() - t0


def _stage1_summary(s1, dt):
    h = s1["history"]
    return {"s": dt, "rounds": int(s1["rounds"]), "stop": int(s1["stop"]),
            "refs": [int(s1["ref_L"].shape[0]), int(s1["ref_U"].shape[0])],
            "final_pu": float(h[-1][0]) / 1e6, "phi_evals": int(s1["phi_evals"])}


def bench_pipeline(rsr, torch, reps=5, quick=False):
    """The paper's whole workflow on a 119-node / 295-edge graph with every
    edge failing with probability 0.05 (Sec. 2.4, 4.1): Stage 1 from no
    references to an unclassified fraction below 1e-5 (rounds of 10^6 samples,
    64 searches per round, permuted visiting order; the paper's index order is
    reported beside it), then Stage 2 on a fresh 10^6 samples with the
    references found (classification + Phi of the unclassified samples on the
    device).  Also Stage 1 for global connectivity (Sec. 4.3) of a 59-node /
    262-edge graph.  Timed with CUDA events (Stage 2) and the host clock around
    the synchronous Stage 1 calls."""
    import workloads.large as L
    from workloads.systems import binary_pmf
    p = L.c2_rgg()
    m = p.meta
    pmf = binary_pmf(np.full(p.n, 0.05))
    system = rsr.System(rsr.RSR_PHI_ST_CONNECTIVITY, m["n_nodes"], m["edges"], m["s"], m["t"])
    s1_idx, t_idx = (None, 0.0) if quick else _stage1_timed(rsr, torch, pmf, system, 64, 10_000, 2000,
                                                           rsr.RSR_SEARCH_INDEX_ORDER)
    s1, t_s1 = _stage1_timed(rsr, torch, pmf, system, 64, 10_000, 2000, rsr.RSR_SEARCH_PERMUTED)
    P = rsr.Problem(pmf, s1["ref_L"].cpu().numpy(), s1["ref_U"].cpu().numpy(), path=rsr.RSR_PATH_POPC)
    sess = rsr.Session(P)
    N = 1_000_000
    dev = torch.device("cuda")
    counts = torch.zeros(3, dtype=torch.int64, device=dev)
    labels = torch.empty(N, dtype=torch.uint8, device=dev)
    uidx = torch.empty(N, dtype=torch.int64, device=dev)
    c2 = torch.zeros(2, dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    times, est = [], None
    for k in range(reps + 2):
        flush.fill_(k)
        counts.zero_()
        c2.zero_()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        off = (1000 + k) * N
        e[0].record(stream)
        rsr.rsr_classify(P, 7, off, N, sess.ws, counts, None, labels, None, None, stream)
        rsr.rsr_resolve(P, system, 7, off, N, labels, sess.ws, u_lower_idx=uidx, counts2=c2, stream=stream)
        e[1].record(stream)
        torch.cuda.synchronize()
        if k >= 2:
            times.append(e[0].elapsed_time(e[1]))
        est = rsr.rsr_estimate(counts.cpu().numpy(), N, int(c2[0].item()))
    out = {
        "graph": "119 nodes / 295 edges, p_f = 0.05 (synthetic stand-in for the paper's Graph 2)",
        "stage1": _stage1_summary(s1, t_s1),
        "stage2_ms_1e6_samples": sum(times) / len(times), "stage2_P_S_le_0": est["P_lower"],
        "stage2_unclassified": est["pu"],
    }
    if quick:
        return out
    # global connectivity of a 59-node / 262-edge graph (Sec. 4.3), permuted order
    _, e1, _, _ = L.rgg_graph(59, 262, 1)
    pmf1 = binary_pmf(np.full(262, 0.05))
    g_sys = rsr.System(rsr.RSR_PHI_GLOBAL_CONNECTIVITY, 59, e1, 0, 0)
    s1g, t_g = _stage1_timed(rsr, torch, pmf1, g_sys, 1024, 100_000, 400, rsr.RSR_SEARCH_PERMUTED)
    # global connectivity of the 119/295 graph (the paper's hardest case): 60 rounds of 8192 searches
    g2_sys = rsr.System(rsr.RSR_PHI_GLOBAL_CONNECTIVITY, m["n_nodes"], m["edges"], 0, 0)
    s1g2, t_g2 = _stage1_timed(rsr, torch, pmf, g2_sys, 8192, 200_000, 60, rsr.RSR_SEARCH_PERMUTED)
    return {
        **out,
        "stage1_index_order": _stage1_summary(s1_idx, t_idx),
        "global_connectivity_59_262": _stage1_summary(s1g, t_g),
        "global_connectivity_119_295": _stage1_summary(s1g2, t_g2),
        "paper_context": "Table 3 Graph 2 (another graph, desktop CPU + T400): 288 references, reference "
                         "search 0.0571 h, probability evaluation 9.33 s; Tables 4-5 Graph 1 global "
                         "connectivity: 8680 references in 17.2 h (desktop), 6757 in 1.12 h (2 V100, 96 workers); "
                         "Graph 2 global connectivity: 560597 references in 4.77 h (2 V100, 96 workers), "
                         "unclassified 2.22e-3",
    }


def bench_levels(rsr, torch, N=1_000_000, reps=5):
    """System-state pmf over all levels of the C4 flow network (three levels,
    boundaries m' = 0 and 1; Sec. 4.5) in one rsr_level_pmf call, against the
    per-boundary path (classification + Stage 2 for each boundary).  CUDA
    events; a 256 MB L2 flush between repetitions."""
    import workloads.large as L
    p0, p1 = L.c4_flow(0), L.c4_flow(1)
    m = p0.meta
    sessions, paths = [], []
    for p in (p0, p1):                               # the autotuner picks each boundary's classifier
        P = rsr.Problem(p.pmf, p.ref_L, p.ref_U, path=rsr.RSR_PATH_AUTO)
        probe = rsr.Session(P)
        P.path = rsr.rsr_autotune(P, probe.ws)
        del probe
        sessions.append(rsr.Session(P))
        paths.append("tcgen05" if P.path == rsr.RSR_PATH_TC else "popc")
    system = rsr.System(rsr.RSR_PHI_ST_MAXFLOW_LEVELS, m["n_nodes"], m["arcs"], m["s"], m["t"],
                        (m["l1"], m["l2"]), 0)
    per_b = [rsr.System(rsr.RSR_PHI_ST_MAXFLOW_LEVELS, m["n_nodes"], m["arcs"], m["s"], m["t"],
                        (m["l1"], m["l2"]), b) for b in range(2)]
    dev = torch.device("cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    labels = torch.empty(N, dtype=torch.uint8, device=dev)
    counts = torch.zeros(3, dtype=torch.int64, device=dev)
    st = torch.cuda.current_stream()
    t_one, t_sep, out = [], [], None
    for k in range(reps + 2):
        flush.fill_(k)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(st)
        out = rsr.rsr_level_pmf(sessions, system, 3, k * N, N, levels=False, stream=st)
        e[1].record(st)
        flush.fill_(k + 1)
        e[2].record(st)
        for b in range(2):
            counts.zero_()
            rsr.rsr_classify(sessions[b].problem, 3, k * N, N, sessions[b].ws, counts, None, labels, None, None, st)
            rsr.rsr_resolve(sessions[b].problem, per_b[b], 3, k * N, N, labels, sessions[b].ws, stream=st)
        e[3].record(st)
        torch.cuda.synchronize()
        if k >= 2:
            t_one.append(e[0].elapsed_time(e[1]))
            t_sep.append(e[2].elapsed_time(e[3]))
    lc = out["level_counts"].cpu().numpy()
    return {"workload": "c4_flow40n100a_K4_levels3_N1e6", "paths": paths, "level_pmf_ms": sum(t_one) / len(t_one),
            "per_boundary_classify_resolve_ms": sum(t_sep) / len(t_sep),
            "P_S_eq": (lc / N).tolist(), "samples_needing_phi": int(out["n_phi"].item())}


def bench_batch(rsr, torch, N=200_000, reps=5):
    """256 hazard scenarios (n = 50..300 edges, 1e2..1e5 references, N samples
    each): the batched launches (tile pass + deep pass) replayed from a CUDA
    graph vs the per-scenario path on prepared workspaces.  Two comparisons:
    kernels only (the batched launches vs one rsr_classify per scenario), and a
    forward+gradient round
    (batched launch + rsr_batch_grad vs rsr_classify + rsr_grad per scenario,
    each rsr_grad reading its counts back)."""
    import workloads.large as L
    probs = L.c5_batch()
    S = len(probs)
    P = [rsr.Problem(p.pmf, p.ref_L, p.ref_U, path=rsr.RSR_PATH_POPC) for p in probs]
    seeds, offsets, Ns = [1000 + s for s in range(S)], [0] * S, [N] * S
    t0 = time.perf_counter()
    b = rsr.Batch(P, seeds, offsets, Ns, labels=True, grad=True)
    grid, order, k0, n_tc, staged, tiles = rsr.rsr_batch_autotune(b)
    prep_s = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        rsr.rsr_batch(b, stream=torch.cuda.current_stream())
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    for _ in range(reps):
        g.replay()
    ev[1].record()
    torch.cuda.synchronize()
    batched_ms = ev[0].elapsed_time(ev[1]) / reps
    t0 = time.perf_counter()
    for _ in range(reps):
        g.replay()
        rsr.rsr_batch_grad(b)
    batched_round_ms = 1000 * (time.perf_counter() - t0) / reps
    # where a block's time goes: one cycle-profiled launch set (the same kernels with
    # clock64 marks per item; outside the timed region)
    torch.cuda.synchronize()
    prof = rsr.rsr_batch_profile(b).cpu().numpy().astype(np.float64)
    R_s = np.array([p.R_L + p.R_U for p in P], dtype=np.float64)
    heavy = R_s >= 1e4
    first, later = prof[:, 1:4].sum(axis=0), prof[:, 5:8].sum(axis=0)
    walk = prof[:, 3] + prof[:, 7]
    tot = first.sum() + later.sum()
    cycle_profile = {
        "tile_pass_share": float(first.sum() / tot),
        "tile_pass_setup_sample_walk": [float(x) for x in first / first.sum()],
        "later_stages_setup_sample_walk": [float(x) for x in later / max(later.sum(), 1.0)],
        "sample_share": float((first[1] + later[1]) / tot),
        "walk_share": float((first[2] + later[2]) / tot),
        "heavy_scenarios_R_ge_1e4": int(heavy.sum()),
        "heavy_share_of_walk": float(walk[heavy].sum() / walk.sum()),
        "heavy_share_of_samples": float(heavy.sum() / len(P)),
        "later_stage_groups": int(prof[:, 4].sum()), "tiles": int(prof[:, 0].sum()),
    }
    # per-scenario path
    sessions = [rsr.Session(p) for p in P]
    cur = torch.cuda.current_stream()
    cnt = torch.zeros(3, dtype=torch.int64, device="cuda")
    lab = torch.empty(N, dtype=torch.uint8, device="cuda")
    grads = [torch.zeros(p.n * p.K, dtype=torch.int64, device="cuda") for p in P]

    def plain(r, with_grad):
        for s_, (p, se) in enumerate(zip(P, sessions)):
            rsr.rsr_classify(p, seeds[s_], offsets[s_] + r * N, N, se.ws, cnt, None, lab, grads[s_], None, cur)
            if with_grad:
                rsr.rsr_grad(p, seeds[s_], offsets[s_] + r * N, N, grads[s_], se.ws, stream=cur)

    plain(0, False)
    torch.cuda.synchronize()
    ev[0].record()
    for r in range(reps):
        plain(1 + r, False)
    ev[1].record()
    torch.cuda.synchronize()
    plain_ms = ev[0].elapsed_time(ev[1]) / reps
    # the same per-scenario launches, each timed by its own events: the sum of kernel
    # durations, and what is left of plain_ms between them (launch gaps)
    pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in P]
    for s_, (p, se) in enumerate(zip(P, sessions)):
        pev[s_][0].record(cur)
        rsr.rsr_classify(p, seeds[s_], offsets[s_] + 20 * N, N, se.ws, cnt, None, lab, grads[s_], None, cur)
        pev[s_][1].record(cur)
    torch.cuda.synchronize()
    per_launch = [a.elapsed_time(b_) for a, b_ in pev]
    kernel_sum_ms = float(sum(per_launch))
    t0 = time.perf_counter()
    for r in range(reps):
        plain(10 + r, True)
    torch.cuda.synchronize()
    plain_round_ms = 1000 * (time.perf_counter() - t0) / reps
    # the same batched launch with the upper sets scanned reference by reference
    Pn = [rsr.Problem(p.pmf, p.ref_L, p.ref_U, path=rsr.RSR_PATH_POPC, index=False) for p in probs]
    bn = rsr.Batch(Pn, seeds, offsets, Ns, labels=True, grad=True)
    rsr.rsr_batch_autotune(bn)
    for _ in range(2):
        rsr.rsr_batch(bn)
    torch.cuda.synchronize()
    ev[0].record()
    for _ in range(reps):
        rsr.rsr_batch(bn)
    ev[1].record()
    torch.cuda.synchronize()
    no_index_ms = ev[0].elapsed_time(ev[1]) / reps
    del bn
    R = [p.R_L + p.R_U for p in P]
    # the generator alone: the Philox4x32-10 blocks both paths draw, at the measured rate
    philox_blocks = sum(N * ((p.n + 3) // 4) for p in P)
    philox_ms = 1e3 * philox_blocks / rsr.rsr_measure_philox_rate()
    return {"workload": "c5_256_scenarios_N%d" % N, "scenarios": S, "refs_total": int(sum(R)),
            "philox_blocks": philox_blocks, "philox_floor_ms": philox_ms,
            "batched_no_index_ms": no_index_ms,
            "batched_ms": batched_ms, "per_scenario_ms": plain_ms, "speedup_kernels": plain_ms / batched_ms,
            "per_scenario_kernel_sum_ms": kernel_sum_ms, "per_scenario_gaps_ms": plain_ms - kernel_sum_ms,
            "per_scenario_launch_ms_max": max(per_launch), "per_scenario_launch_ms_median": statistics.median(per_launch),
            "batched_fwd_grad_round_ms": batched_round_ms, "per_scenario_fwd_grad_round_ms": plain_round_ms,
            "speedup_fwd_grad_round": plain_round_ms / batched_round_ms,
            "samples_per_s": S * N / (batched_ms / 1000.0), "autotune_grid": grid,
            "autotune_order": "longest-first" if order == 0 else "as-given", "autotune_k0": k0,
            "autotune_staged": staged, "autotune_tiles_per_item": tiles, "autotune_tc_scenarios": n_tc,
            "cycle_profile": cycle_profile, "prepare_s": prep_s}


def popc_roofline(rsr, n, K, n_samples, kern_ms, word_ops, meas=None):
    """Roofline of the bit-packed classifier on the operations it issues:
    per Philox4x32-10 block 20 wide products (IMAD.WIDE) and 60 logic / add ops,
    n(K-1) threshold compares per sample, and the 32-bit logic operations on
    reference data that the kernel counted (exec_tests[1]: scan words, AND-row
    words, index rows).  Peak: this mix at the LOP3 and IMAD.WIDE rates measured
    on this GPU (time bound = max(ALU ops / LOP3 rate, IMAD ops / IMAD rate))."""
    meas = meas or rsr.rsr_measure_int_peak()
    if "philox_blocks_per_s" not in meas:
        meas = dict(meas, philox_blocks_per_s=rsr.rsr_measure_philox_rate())
    blocks = n_samples * ((n + 3) // 4)
    imad_ops = 20.0 * blocks
    alu_ops = 60.0 * blocks + n_samples * n * (K - 1) + float(word_ops)
    ops = imad_ops + alu_ops
    t_bound = max(alu_ops / meas["lop3_ops_per_s"], imad_ops / meas["imad_ops_per_s"])
    achieved = ops / (kern_ms / 1000.0) / 1e12
    peak = ops / t_bound / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
            "traffic": None, "issued_word_ops": float(word_ops), "philox_blocks": float(blocks),
            "measured_lop3_tops": meas["lop3_ops_per_s"] / 1e12,
            "measured_imad_wide_tops": meas["imad_ops_per_s"] / 1e12,
            "measured_philox_blocks_per_s": meas["philox_blocks_per_s"],
            "philox_floor_ms": 1e3 * blocks / meas["philox_blocks_per_s"],
            "note": "integer-op model on issued operations (per Philox block 20 IMAD.WIDE + 60 ALU ops, n(K-1) "
                    "compares per sample, the kernel's own count of logic operations on reference data); peak = "
                    "this mix at the LOP3 and IMAD.WIDE rates measured on this GPU (rsr_measure_int_peak)"}


def bench_c2_popc(rsr, torch, meas, reps=5):
    """The 119-node / 295-edge workload (1840 references, N = 1e6, early exit)
    on the bit-packed classifier alone: kernel time and its roofline on issued
    operations (classifier only; the --workload c2 line adds Stage 2 and the
    gradient)."""
    import workloads.large as L
    p = L.c2_rgg()
    N = 1_000_000
    P = rsr.Problem(p.pmf, p.ref_L, p.ref_U, path=rsr.RSR_PATH_POPC)
    sess = rsr.Session(P)
    rsr.rsr_autotune(P, sess.ws)   # the first-pass budget (k0) of the two-pass kernel
    counts = torch.zeros(3, dtype=torch.int64, device="cuda")
    ex = torch.zeros(2, dtype=torch.int64, device="cuda")
    labels = torch.empty(N, dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ts, ops = [], []
    for k in range(reps + 2):
        flush.fill_(k & 0xFF)
        counts.zero_()
        ex.zero_()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record()
        rsr.rsr_classify(P, 1, k * N, N, sess.ws, counts, None, labels, None, ex)
        e[1].record()
        torch.cuda.synchronize()
        if k >= 2:
            ts.append(e[0].elapsed_time(e[1]))
            ops.append(int(ex[1].item()))
    ms = statistics.median(ts)
    roof = popc_roofline(rsr, P.n, P.K, N, ms, statistics.median(ops), meas)
    return {"workload": "c2_rgg119n295e_N1e6 classifier (early exit, bit-packed)", "classifier_ms": ms,
            "samples_per_s": N / (ms / 1000.0), "roofline": roof}


_ORACLE_PROB = None


def _oracle_init(name):
    """Worker start-up (spawned process): load the workload once."""
    global _ORACLE_PROB
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    _ORACLE_PROB = _workload(name)[0]


def _oracle_slice(args):
    """One worker's share: the oracle's sampler, first-match classification and
    gradient counts on samples [offset, offset + n) of the stream."""
    seed, offset, n = args
    from oracle import oracle as O
    prob = _ORACLE_PROB
    t0 = time.perf_counter()
    X = O.sample(prob.pmf, seed, offset, n)
    lab, cnt = O.classify(X, prob.ref_L, prob.ref_U)
    C = O.grad_counts(X, lab, prob.K)
    return cnt, C, time.perf_counter() - t0


class OraclePool:
    """The oracle as it stands on every host core: one spawned process per core,
    each classifying a contiguous slice of the same sample stream (the Philox
    counters make slices independent); the counts are summed and the estimates
    and fp64 gradient computed once.  Spawned, so it is safe after CUDA use."""

    def __init__(self, name, workers=None):
        import multiprocessing as mp
        self.workers = workers or os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.workers, initializer=_oracle_init, initargs=(name,))
        # the initializer loads the workload in every worker; a first small map starts
        # them all and loads the oracle library outside the timed runs
        self.pool.map(_oracle_slice, [(1, 0, 16)] * self.workers, chunksize=1)

    def run(self, prob, seed, offset, n_total):
        from oracle import oracle as O
        per = -(-n_total // self.workers)
        parts = [(seed, offset + k * per, min(per, n_total - k * per)) for k in range(self.workers)
                 if n_total - k * per > 0]
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_slice, parts)
        cnt = sum(r[0] for r in res)
        C = sum(r[1] for r in res)
        O.grad(C, n_total, prob.pmf)
        O.estimate(cnt, n_total)
        dt = time.perf_counter() - t0
        self.last_counts, self.last_grad_counts = cnt, C
        return n_total / dt, dt

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(prob, seed, n_sample, offset=0):
    """The oracle as it stands, single-threaded, on a bounded sample."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    X = O.sample(prob.pmf, seed, offset, n_sample)
    lab, cnt = O.classify(X, prob.ref_L, prob.ref_U)
    C = O.grad_counts(X, lab, prob.K)
    O.grad(C, n_sample, prob.pmf)
    O.estimate(cnt, n_sample)
    dt = time.perf_counter() - t0
    return n_sample / dt, dt


def c5_cpu_baseline(N_each=5000, stride=16):
    """The oracle as it stands on one host core over a bounded sample of the
    batched workload: N_each samples of every stride-th scenario."""
    import workloads.large as L
    probs = L.c5_batch()
    tot_n, tot_t, k = 0, 0.0, 0
    for s in range(0, len(probs), stride):
        _, dt = cpu_baseline(probs[s], 1000 + s, N_each)
        tot_n += N_each
        tot_t += dt
        k += 1
    return {"value": tot_n / tot_t, "unit": "samples/s", "cores": 1, "kind": "oracle",
            "sample": "%d samples of each of %d scenarios (every %dth of 256), one core, %.1f s"
                      % (N_each, k, stride, tot_t)}


def run_reference(args):
    """--impl reference: the oracle timed on the host cores on the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    prob, N, wname = _workload(args.workload)
    pool = OraclePool(args.workload)
    n_sample = args.ref_samples * pool.workers
    for _ in range(args.warmup):
        pool.run(prob, 1, 0, min(n_sample, 2000 * pool.workers))
    times = []
    for k in range(args.steps):
        _, dt = pool.run(prob, 1, k * n_sample, n_sample)
        times.append(dt)
    pool.close()
    ms = 1000.0 * sum(times) / len(times)
    value = n_sample / (ms / 1000.0)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": wname, "sample_per_step": n_sample, "mode": "oracle (first-match loops)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.workers, "kind": "oracle",
                         "sample": "%d samples per step of %s on %d processes" % (n_sample, wname, pool.workers)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_pipeline(args):
    """--workload pipeline: the whole workflow of bench_pipeline as its own line
    (value = seconds of Stage 1 + Stage 2 on the 119/295 graph, permuted
    visiting order).  Used for the kernel launch lists of Stage 1 / Stage 2."""
    import torch
    from paper_2604_17066_gb300 import api as rsr
    from paper_2604_17066_gb300 import build as rsr_build
    rsr_build.build()
    torch.cuda.set_device(0)
    res = None
    with Clocks(None) as clk:
        res = bench_pipeline(rsr, torch, reps=max(1, args.steps), quick=args.quick)
    total = res["stage1"]["s"] + res["stage2_ms_1e6_samples"] / 1000.0
    line = {"metric": "RSR workflow time: Stage 1 to p_u < 1e-5 from no references + Stage 2 on 1e6 samples",
            "value": total, "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": 1,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u32 bit-packed",
            "data": "synthetic", "config": {"workload": "pipeline_rgg119n295e_pf0.05"},
            "clocks": clk.summary(), "pipeline": res}
    print(json.dumps(line), flush=True)
    return 0


def run_batch_line(args):
    """--workload c5: the 256-scenario batch on its own line (value = samples/s of
    the batched launch, beside the per-scenario path).  With --quick: prepare,
    two warm-up launches and one timed launch, no autotuning and no graph, then
    one pass of the per-scenario path (the launch lists and captures of the
    batched kernels and of the per-scenario launches)."""
    import torch
    from paper_2604_17066_gb300 import api as rsr
    from paper_2604_17066_gb300 import build as rsr_build
    rsr_build.build()
    torch.cuda.set_device(0)
    N = args.samples or 200_000
    with Clocks(None) as clk:
        if args.quick:
            import workloads.large as L
            probs = L.c5_batch()
            S = len(probs)
            b = rsr.Batch([rsr.Problem(p.pmf, p.ref_L, p.ref_U, path=rsr.RSR_PATH_POPC) for p in probs],
                          [1000 + s for s in range(S)], [0] * S, [N] * S)
            for _ in range(2):
                rsr.rsr_batch(b)
            torch.cuda.synchronize()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            e[0].record()
            rsr.rsr_batch(b)
            e[1].record()
            torch.cuda.synchronize()
            ms = e[0].elapsed_time(e[1])
            # one pass of the per-scenario path over the same scenarios (launch list comparison)
            P = [rsr.Problem(p.pmf, p.ref_L, p.ref_U, path=rsr.RSR_PATH_POPC) for p in probs]
            sessions = [rsr.Session(pp) for pp in P]
            cnt = torch.zeros(3, dtype=torch.int64, device="cuda")
            lab = torch.empty(N, dtype=torch.uint8, device="cuda")
            torch.cuda.synchronize()
            e[0].record()
            for s_, (pp, se) in enumerate(zip(P, sessions)):
                rsr.rsr_classify(pp, 1000 + s_, 0, N, se.ws, cnt, None, lab)
            e[1].record()
            torch.cuda.synchronize()
            res = {"workload": "c5_256_scenarios_N%d" % N, "batched_ms": ms, "samples_per_s": S * N / (ms / 1e3),
                   "per_scenario_ms": e[0].elapsed_time(e[1])}
        else:
            res = bench_batch(rsr, torch, N=N)
    line = {"metric": "batched classification of 256 hazard scenarios: samples/s of one persistent launch",
            "value": res["samples_per_s"], "unit": "samples/s", "n_gpus": 1, "steps": 1 if args.quick else 5,
            "warmup": 2, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32 bit-packed", "data": "synthetic", "config": {"workload": res["workload"]},
            "clocks": clk.summary(), "batch": res}
    if not args.quick:
        line["cpu_baseline"] = c5_cpu_baseline()
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c3", "c2", "c4", "c5", "pipeline"])
    ap.add_argument("--ref-samples", type=int, default=8000)
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 256-scenario batched comparison")
    ap.add_argument("--samples", type=int, default=0, help="override samples per GPU (profiling runs)")
    ap.add_argument("--early-exit", action="store_true",
                    help="time the C3 line in production mode (early exit) instead of dense mode")
    ap.add_argument("--quick", action="store_true",
                    help="--workload pipeline: only the permuted-order Stage 1 and Stage 2; --workload c5: "
                         "one batched launch after two warm-ups (profiling runs)")
    args = ap.parse_args()
    if args.workload == "c5":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batched line has no oracle arm; the "
                              "oracle is timed on the C3 line"}), flush=True)
            return 0
        return run_batch_line(args)
    if args.workload == "pipeline":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the workflow line has no oracle arm; "
                              "the oracle's Stage 1 is timed by the tests only"}), flush=True)
            return 0
        return run_pipeline(args)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2604_17066_gb300 import api as rsr
    from paper_2604_17066_gb300 import build as rsr_build
    from paper_2604_17066_gb300.shard import combine_counts, shard_range
    rsr_build.build()

    prob, N, wname = _workload(args.workload)
    if args.samples > 0:
        N = args.samples
        wname += "_N%d" % N
    if args.early_exit and args.workload == "c3":
        wname += "_early_exit"
    path = rsr.RSR_PATH_TC if args.workload == "c3" else rsr.RSR_PATH_POPC
    P = rsr.Problem(prob.pmf, prob.ref_L, prob.ref_U, path=path,
                    dense=(args.workload == "c3" and not args.early_exit))
    if args.workload == "c4":
        # multi-state: let the autotuner pick the classifier path for this problem
        P.path = rsr.RSR_PATH_AUTO
        probe = rsr.Session(P)
        path = rsr.rsr_autotune(P, probe.ws)
        P.path = path
        del probe
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    sess = rsr.Session(P)
    torch.cuda.synchronize()
    prep_ms = 1000 * (time.perf_counter() - t0)
    if args.workload == "c2":
        # the bit-packed path's first-pass budget, tuned on this problem (not timed)
        rsr.rsr_autotune(P, sess.ws)
    overlap = sess.overlap()
    offset, n_rank = shard_range(N, rank, world)
    dev = torch.device("cuda", local)
    counts = torch.zeros(3, dtype=torch.int64, device=dev)
    gcounts = torch.zeros(P.n * P.K, dtype=torch.int64, device=dev)
    labels = torch.empty(n_rank, dtype=torch.uint8, device=dev)
    exec_t = torch.zeros(2, dtype=torch.int64, device=dev)   # executed tests, issued word operations
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    # Stage 2 (Sec. 3.5) for the graph workloads: Phi on the unclassified samples, on the device
    system = None
    if args.workload == "c2":
        system = rsr.System(rsr.RSR_PHI_ST_CONNECTIVITY, prob.meta["n_nodes"], prob.meta["edges"],
                            prob.meta["s"], prob.meta["t"])
    elif args.workload == "c4":
        system = rsr.System(rsr.RSR_PHI_ST_MAXFLOW_LEVELS, prob.meta["n_nodes"], prob.meta["arcs"],
                            prob.meta["s"], prob.meta["t"], (prob.meta["l1"], prob.meta["l2"]), prob.meta["m_prime"])
    uidx = torch.empty(n_rank, dtype=torch.int64, device=dev)
    c2 = torch.zeros(2, dtype=torch.int64, device=dev)
    stage2_ms = []

    classify_launches = rsr.rsr_classify_plan(P, n_rank, sess.ws)[1]

    def step(k, grad=True, ev=None):
        counts.zero_()
        gcounts.zero_()
        off = offset + k * N * world
        if ev is not None:
            ev[0].record(stream)
        rsr.rsr_classify(P, 1, off, n_rank, sess.ws, counts, None, labels,
                         gcounts if grad else None, exec_t, stream)
        if ev is not None:
            ev[1].record(stream)
        n_ul = 0
        if system is not None:
            c2.zero_()
            rsr.rsr_resolve(P, system, 1, off, n_rank, labels, sess.ws, u_lower_idx=uidx, counts2=c2, stream=stream)
            if ev is not None:
                ev[4].record(stream)
            n_ul = int(c2[0].item())
        if grad:
            rsr.rsr_grad(P, 1, off, n_rank, gcounts, sess.ws, u_lower_idx=uidx[:n_ul] if n_ul else None,
                         stream=stream)
        est = rsr.rsr_estimate(counts.cpu().numpy(), n_rank, n_ul)
        # classify (one launch, one per stage on the bit-packed path's staged passes), resolve,
        # and rsr_grad's index check and correction
        step.last_launches = classify_launches + (system is not None) + (2 if (grad and n_ul > 0) else 0)
        return est

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    launches = 0
    kern_ms = []
    step_ms = []
    exec_t.zero_()
    with Clocks(uuid) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(k & 0xFF)                      # L2 flush between timed steps (not timed)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            ev[2].record(stream)
            est = step(args.warmup + k, grad=True, ev=ev)
            ev[3].record(stream)
            torch.cuda.synchronize()
            launches += step.last_launches
            kern_ms.append(ev[0].elapsed_time(ev[1]))
            step_ms.append(ev[2].elapsed_time(ev[3]))
            if system is not None:
                stage2_ms.append(ev[1].elapsed_time(ev[4]))
    torch.cuda.synchronize()
    exec_tests = int(exec_t[0].item())
    exec_ops = int(exec_t[1].item())
    total_ms = sum(step_ms)
    if world > 1:
        # the estimate of the last timed step over every rank's samples: the integer counts
        # (and the Stage-2 lower count) add up exactly across ranks
        tot = torch.cat([counts, c2[:1] if system is not None else torch.zeros(1, dtype=torch.int64, device=dev)])
        combine_counts(tot)
        tot_h = tot.cpu().numpy()
        est = rsr.rsr_estimate(tot_h[:3], world * n_rank, int(tot_h[3]))
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    ms_step = total_ms / args.steps
    value = world * n_rank / (ms_step / 1000.0)

    # roofline of the classifier kernel.  Tensor path: algorithmic flops 2*n(K-1) per
    # dominance test (all N*(R_L+R_U) tests in dense mode, the executed ones otherwise).
    # Bit-packed path: an integer-op model, 80 ops per Philox4x32-10 block (10 rounds of two
    # 32x32->64 products, two 3-input xors, two key adds), n(K-1) threshold compares per
    # sample, ceil(n(K-1)/32) + 1 ops per executed test; peak = SMs x 128 lanes x max clock.
    peaks, peak_src = _peaks()
    R = P.R_L + P.R_U
    kenc = P.n * (P.K - 1)
    kern_avg = sum(kern_ms) / len(kern_ms)
    tests_per_launch = n_rank * R
    exec_per_launch = exec_tests / args.steps
    if path == rsr.RSR_PATH_TC:
        work_tests = tests_per_launch if P.dense else exec_per_launch
        flops = 2.0 * kenc * work_tests
        achieved = flops / (kern_avg / 1000.0) / 1e12
        kpad = ((kenc + (kenc + 15) // 16 + 31) // 32) * 32       # FP8 row incl. bias columns, padded to 32
        achieved_exec = 2.0 * kpad * exec_per_launch / (kern_avg / 1000.0) / 1e12
        fp8 = measure_fp8_peak(rsr, torch, uuid)
        peak = fp8["burst_tflops"]
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "frac_executed": achieved_exec / peak,
                "achieved_executed": achieved_exec,
                "traffic": _captured_traffic(wname) if P.dense else None,
                "peak_measured": fp8,
                "note": "peak = measured FP8 tcgen05 burst of this GPU, the larger of single-CTA and CTA-pair "
                        "MMA loops (rsr_measure_fp8_peak: back-to-back kind::f8f6f4 MMAs from shared memory, "
                        "one CTA per SM); frac = algorithmic flops "
                        "2*n(K-1)*%s tests / kernel time / peak; frac_executed counts the executed tests at "
                        "the padded row of %d bytes" % ("N*(R_L+R_U)" if P.dense else "executed", kpad)}
    else:
        roof = popc_roofline(rsr, P.n, P.K, n_rank, kern_avg, exec_ops / args.steps)

    extras = {}
    if rank == 0 and not args.no_extras:
        # forward only (no gradient counts)
        fw = []
        for k in range(3):
            flush.fill_(k)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            e[0].record(stream)
            step(100 + k, grad=False)
            e[1].record(stream)
            torch.cuda.synchronize()
            fw.append(e[0].elapsed_time(e[1]))
        extras["fwd_ms"] = sum(fw) / len(fw)
        extras["fwd_grad_ms"] = ms_step
        extras["fwd_grad_over_fwd"] = ms_step / extras["fwd_ms"]
        # early exit (production mode) on the same references, both classifier paths
        if args.workload == "c3":
            ee_all = {}
            for pname, pth, idx in (("tc", rsr.RSR_PATH_TC, True), ("popc", rsr.RSR_PATH_POPC, True),
                                    ("popc_no_index", rsr.RSR_PATH_POPC, False)):
                P2 = rsr.Problem(prob.pmf, prob.ref_L, prob.ref_U, path=pth, dense=False, index=idx)
                s2 = rsr.Session(P2)
                ee = []
                ex = torch.zeros(2, dtype=torch.int64, device=dev)
                for k in range(4):
                    flush.fill_(k)
                    counts.zero_()
                    ex.zero_()
                    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                    e[0].record(stream)
                    rsr.rsr_classify(P2, 1, 7 * N + k * N, N, s2.ws, counts, None, labels, gcounts, ex, stream)
                    e[1].record(stream)
                    torch.cuda.synchronize()
                    ee.append(e[0].elapsed_time(e[1]))
                ee_ms = statistics.median(ee[1:])
                ee_all[pname] = {"ms": ee_ms, "samples_per_s": N / (ee_ms / 1000.0),
                                 "nominal_tests_per_s": N * R / (ee_ms / 1000.0),
                                 "executed_tests_per_sample": int(ex[0].item()) / N}
                del s2
            extras["early_exit"] = ee_all
        if path == rsr.RSR_PATH_POPC:
            # the classifier kernel alone, with and without the upper index
            for key, idx in (("classifier_ms", True), ("classifier_no_index_ms", False)):
                P3 = rsr.Problem(prob.pmf, prob.ref_L, prob.ref_U, path=path, dense=P.dense, index=idx)
                s3 = rsr.Session(P3)
                tk = []
                for k in range(5):
                    flush.fill_(k)
                    counts.zero_()
                    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                    e[0].record(stream)
                    rsr.rsr_classify(P3, 1, 13 * N + k * N, n_rank, s3.ws, counts, None, labels, None, None, stream)
                    e[1].record(stream)
                    torch.cuda.synchronize()
                    tk.append(e[0].elapsed_time(e[1]))
                extras[key] = statistics.median(tk[1:])
                del s3
        extras["prepare_ms"] = prep_ms
        extras["overlap_pairs"] = bool(overlap)
        if stage2_ms:
            extras["stage2"] = {"resolve_ms": sum(stage2_ms) / len(stage2_ms), "n_u": int(c2.sum().item()),
                                "note": "Phi evaluated on the device for every unclassified sample; the step "
                                        "estimate is the Stage-2 P(S<=m')"}
        if args.workload == "c3":
            extras["c2_popc"] = bench_c2_popc(rsr, torch, rsr.rsr_measure_int_peak())
        extras["pipeline_119_295"] = bench_pipeline(rsr, torch)
        extras["level_pmf_c4"] = bench_levels(rsr, torch)
        if args.workload == "c3" and not args.no_batch:
            extras["batch_c5"] = bench_batch(rsr, torch, N=200_000)
            extras["batch_c5_N2e4"] = bench_batch(rsr, torch, N=20_000)

    # end to end through the public API: pmf -> thresholds (H2D), classify, results (D2H)
    e2e = None
    if rank == 0:
        lab_host = torch.empty(n_rank, dtype=torch.uint8, pin_memory=True)
        cnt_host = torch.empty(3, dtype=torch.int64, pin_memory=True)
        times = []
        for k in range(3):
            flush.fill_(k)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sess.set_pmf(prob.pmf)                     # host thresholds -> device
            counts.zero_()
            gcounts.zero_()
            off_k = 11 * N + k * N
            rsr.rsr_classify(P, 1, off_k, n_rank, sess.ws, counts, None, labels, gcounts, None, stream)
            n_ul = 0
            if system is not None:
                c2.zero_()
                rsr.rsr_resolve(P, system, 1, off_k, n_rank, labels, sess.ws, u_lower_idx=uidx, counts2=c2,
                                stream=stream)
                n_ul = int(c2[0].item())
            lab_host.copy_(labels, non_blocking=True)
            cnt_host.copy_(counts, non_blocking=True)
            g, se = rsr.rsr_grad(P, 1, off_k, n_rank, gcounts, sess.ws,
                                 u_lower_idx=uidx[:n_ul] if n_ul else None, stream=stream)   # syncs
            rsr.rsr_estimate(cnt_host.numpy(), n_rank, n_ul)
            times.append(time.perf_counter() - t0)
        e2e_s = statistics.median(times)
        e2e = {"value": n_rank / e2e_s, "unit": UNIT, "h2d_bytes_per_step": P.n * (P.K - 1) * 8,
               "d2h_bytes_per_step": n_rank + 3 * 8 + P.n * P.K * 8 + (16 if system is not None else 0)}

    cpu = None
    if rank == 0:
        n_s = 20000 if args.workload == "c3" else 100000
        v1, dt1 = cpu_baseline(prob, 1, n_s, offset=5 * N)
        pool = OraclePool(args.workload)
        n_all = n_s * pool.workers
        v, dt = pool.run(prob, 1, 5 * N, n_all)
        pool.close()
        cpu = {"value": v, "unit": UNIT, "cores": pool.workers, "kind": "oracle",
               "sample": "%d samples of %s on %d processes (oracle first-match loops, %.1f s); one core: "
                         "%.4g samples/s on %d samples (%.1f s)" % (n_all, wname, pool.workers, dt, v1, n_s, dt1),
               "single_core_value": v1}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "fp8-e4m3 0/1 operands, fp32 accumulate (exact integers)"
            if path == rsr.RSR_PATH_TC else "u32 bit-packed", "data": "synthetic",
            "config": {"workload": wname, "n": P.n, "K": P.K, "R_L": P.R_L, "R_U": P.R_U, "N_per_gpu": n_rank,
                       "mode": "dense" if P.dense else "early-exit",
                       "path": "tcgen05" if path == rsr.RSR_PATH_TC else "popc",
                       "l2": "flushed between timed steps (256 MB write)", "parallelism": "samples%d" % world},
            "dominance_tests_per_s": world * n_rank * R / (ms_step / 1000.0),
            "executed_tests": exec_tests,
            "kernel_ms": kern_avg,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "estimate": est,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
