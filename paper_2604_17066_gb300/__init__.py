"""GB300-native (sm_103a) hot path of Reference-state System Reliability
(arXiv 2604.17066): Monte Carlo samples classified against lower / upper
reference states, estimates and score-function gradients, behind the C ABI of
librsr.so (include/rsr.h).

The CUDA library is loaded lazily on first use; importing the package needs no
GPU.  There is no CPU fallback: the entry points raise if librsr.so is missing.
"""
from __future__ import annotations

__all__ = [
    "Problem", "Session", "RSRProb", "RSRError", "alloc_workspace",
    "rsr_workspace_size", "rsr_prepare", "rsr_update_pmf", "rsr_classify", "rsr_classify_plan", "rsr_estimate",
    "rsr_grad", "rsr_sample", "rsr_workspace_status",
    "Batch", "rsr_batch_prepare", "rsr_batch", "rsr_batch_profile", "rsr_batch_autotune", "rsr_autotune",
    "rsr_classify_static", "rsr_batch_grad", "System", "rsr_resolve",
    "rsr_boundary_search", "rsr_nondominated", "rsr_stage1", "rsr_level_pmf", "rsr_measure_int_peak", "rsr_measure_fp8_peak",
    "rsr_measure_philox_rate",
    "RSR_PHI_ST_CONNECTIVITY", "RSR_PHI_ST_MAXFLOW_LEVELS", "RSR_PHI_GLOBAL_CONNECTIVITY",
    "RSR_PHI_GLOBAL_CONN_LEVEL", "RSR_SEARCH_INDEX_ORDER", "RSR_SEARCH_PERMUTED",
    "RSR_PATH_AUTO", "RSR_PATH_POPC", "RSR_PATH_TC", "RSR_FLAG_DENSE", "RSR_FLAG_NO_INDEX",
]


def __getattr__(name):
    if name in __all__:
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
