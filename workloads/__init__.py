"""Seeded synthetic inputs for the RSR hot path.

This package produces *inputs only*: component pmfs, systems (graphs, DNF
terms, flow networks) and their reference states.  It holds none of the hot
path's arithmetic (no thresholds, no sampler, no classification, no estimates,
no gradients), and it is the one module that both the CUDA library's tests and
the independent oracle read from.

The paper's own graphs and data are not available; these generators stand in
for its workloads with the same shapes (Sec. 2.4 random graphs of 59/262 and
119/295; Sec. 4.4 hundreds of thousands of reference states; Sec. 4.5
multi-state systems).  Reference states follow Sec. 2.2: a lower reference is
a maximal state with Phi <= m' (a minimal cut set in the binary case: 0 on the
cut, 1 elsewhere), an upper reference a minimal state with Phi >= m'+1 (a
minimal path set: 1 on the path, 0 elsewhere).
"""
from __future__ import annotations

from .systems import (  # noqa: F401
    Problem,
    binary_pmf,
    all_states,
    grid_graph,
    st_connectivity_all_states,
    reference_sets_from_phi,
    c1_grid,
    series_system,
    parallel_system,
    k_out_of_n_system,
    random_small_system,
)
