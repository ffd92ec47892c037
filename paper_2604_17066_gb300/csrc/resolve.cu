// resolve.cu -- system-function kernels: Stage 2 (Sec. 3.5), where Phi is
// evaluated for every unclassified sample, which closes the estimate of
// P(S <= m') without the host; and the componentwise boundary search of
// Stage 1 (Sec. 3.4), which turns unclassified samples into new reference
// states.
//
// Built-in system functions (the families of the paper's experiments):
//   RSR_PHI_ST_CONNECTIVITY   binary components are undirected edges; Phi = 1
//                             iff s reaches t over working edges (x_e = 1)
//   RSR_PHI_ST_MAXFLOW_LEVELS components are directed arcs with capacity x_a;
//                             Phi = #{l : maxflow(s -> t) >= thr_l}
//   RSR_PHI_GLOBAL_CONNECTIVITY  Phi = 1 iff the working edges connect all
//                             nodes (Sec. 4.3)
//   RSR_PHI_GLOBAL_CONN_LEVEL Phi = 0 disconnected, 1 connected with a bridge
//                             (some pair has one edge-disjoint path), 2 no
//                             bridge (Sec. 4.6; Menger)
// One warp per sample: its states are regenerated from Philox (lane-strided
// blocks), then
//   s-t connectivity: label propagation over a shared-memory bitset, one edge
//                 per lane per sweep, until t is reached or nothing changes;
//   max flow:     Ford-Fulkerson; each augmenting path is found by a
//                 warp-parallel search of the residual graph (parents claimed
//                 with atomicCAS, so they form a tree rooted at s) and pushed
//                 by one lane; it stops as soon as the flow reaches the
//                 threshold that decides S <= m';
//   global:       a level-synchronous breadth-first tree from node 0 (parent
//                 word = depth << 16 | edge); bridges by covering: every
//                 non-tree working edge walks its two ends up to their common
//                 ancestor and marks the tree edges it passes, and a tree edge
//                 left unmarked is a bridge.
// Stage 2 rewrites labels 2 to 3 (Phi <= m') or 4 (Phi >= m'+1) and appends
// the local indices of the 3s to u_lower_idx (in no particular order) for
// rsr_grad.  The search raises (Phi <= m') or lowers (Phi >= m'+1) the
// components in index order one state at a time, undoing the step that
// crosses the boundary, exactly as Sec. 3.4 describes.
#include <algorithm>

#include <cuda_runtime.h>

#include "rsr.h"
#include "rsr_internal.cuh"
#include "rsr_launch.h"

namespace rsr {

namespace {

constexpr int kWarps = 4;          // warps per block, one sample each at a time
// Stage 2 and the level pmf are latency-bound: compiled for 12 resident blocks
// (48 warps) per SM, which their shared memory allows for graphs of the
// experiments' size (C4's Stage 2: 0.24 -> 0.22 ms against 8 blocks).
constexpr int kMaxNodes = 1024;
constexpr int kMaxLevels = 9;      // system levels: at most 8 boundaries

struct Sys {
    int32_t kind, n_nodes, s, t, n_levels, m_prime;
    int32_t thr[8];
    const int32_t *src, *dst;
};

// One warp's scratch, as pointers into dynamic shared memory sized by the
// system (SysSmem, SearchSmem), so that small graphs leave room for more
// resident warps.
struct WarpScratch {
    uint8_t *x;        // [n] component states of the sample
    uint32_t *vis;     // [ceil(max(n, n_nodes) / 32)] reached nodes, or a witness edge mask (search)
    int32_t *parent;   // [n_nodes] claimed residual arc (max flow) / tree parent, -1 = unreached
    int16_t *flow;     // [max(n, n_nodes)] arc flows (max flow), covered marks (bridges), a node queue (search)
};

// Dynamic shared memory of resolve_kernel / levels_kernel: the block's graph
// (src, dst: int32 [n]) and thresholds (uint64 [n (K-1)]), then per warp x
// (uint8 [n]), vis (uint32 [ceil(m / 32)]), parent (int32 [n_nodes]) and flow
// (int16 [m]), m = max(n, n_nodes), every region 16-byte aligned.
struct SysSmem {
    size_t off_src, off_dst, off_thr, off_warps, warp_bytes, off_x, off_vis, off_parent, off_flow, total;
};
__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }
__host__ __device__ inline SysSmem sys_smem(int n, int km1, int n_nodes, int warps) {
    SysSmem L{};
    size_t o = 0;
    L.off_src = o;
    o = align16(o + sizeof(int32_t) * (size_t)n);
    L.off_dst = o;
    o = align16(o + sizeof(int32_t) * (size_t)n);
    L.off_thr = o;
    o = align16(o + sizeof(unsigned long long) * (size_t)n * km1);
    L.off_warps = o;
    size_t w = 0;
    L.off_x = w;
    w = align16(w + (size_t)n);
    const int m = n > n_nodes ? n : n_nodes;   // vis and flow also serve as edge arrays / node queues
    L.off_vis = w;
    w = align16(w + sizeof(uint32_t) * (size_t)((m + 31) / 32));
    L.off_parent = w;
    w = align16(w + sizeof(int32_t) * (size_t)n_nodes);
    L.off_flow = w;
    w = align16(w + sizeof(int16_t) * (size_t)m);
    L.warp_bytes = w;
    L.total = o + w * (size_t)warps;
    return L;
}
// The search kernel's dynamic shared memory: SysSmem's regions, then the
// block's adjacency (off, cur: int32 [n_nodes + 1]; adj: int16 [2n]; one
// frontier counter per warp) and per warp a visiting order (int16 [n]) and a
// saved flow / second frontier buffer (int16 [max(n, n_nodes)]).
struct SearchSmem {
    SysSmem sys;
    size_t off_off, off_cur, off_adj, off_cnt, off_ord, off_bak, warp_bytes, total;
};
__host__ __device__ inline SearchSmem search_smem(int n, int km1, int n_nodes, int warps) {
    SearchSmem L{};
    L.sys = sys_smem(n, km1, n_nodes, warps);
    const int m = n > n_nodes ? n : n_nodes;
    size_t o = L.sys.total;
    L.off_off = o;
    o = align16(o + sizeof(int32_t) * (size_t)(n_nodes + 1));
    L.off_cur = o;
    o = align16(o + sizeof(int32_t) * (size_t)(n_nodes + 1));
    L.off_adj = o;
    o = align16(o + sizeof(int16_t) * 2 * (size_t)n);
    L.off_cnt = o;
    o = align16(o + sizeof(int32_t) * (size_t)warps);
    L.off_ord = o;
    L.warp_bytes = align16(sizeof(int16_t) * (size_t)n) + align16(sizeof(int16_t) * (size_t)m);
    L.off_bak = align16(sizeof(int16_t) * (size_t)n);   // within a warp's slice
    L.total = o + L.warp_bytes * (size_t)warps;
    return L;
}

__device__ inline WarpScratch warp_view(unsigned char *dyn, const SysSmem &L, int warp) {
    unsigned char *b = dyn + L.off_warps + L.warp_bytes * (size_t)warp;
    return WarpScratch{b + L.off_x, reinterpret_cast<uint32_t *>(b + L.off_vis),
                       reinterpret_cast<int32_t *>(b + L.off_parent), reinterpret_cast<int16_t *>(b + L.off_flow)};
}

__device__ __forceinline__ bool bit(const uint32_t *v, int i) { return (v[i >> 5] >> (i & 31)) & 1u; }

__device__ __forceinline__ int vload(const int32_t *p) { return *(const volatile int32_t *)p; }

// Breadth-first tree from `root` over working edges, level by level: in sweep d
// only nodes of depth d-1 expand, so depths are exact.  parent[v] = depth << 16
// | edge (0xFFFF at the root), -1 unreached.  Stops early once `stop` (>= 0) is
// reached.  Returns the number of reached nodes.
__device__ int bfs_tree(const Sys &g, int n, WarpScratch &w, const int32_t *s_src, const int32_t *s_dst,
                        int root = 0, int stop = -1) {
    const int lane = threadIdx.x & 31;
    for (int v = lane; v < g.n_nodes; v += 32) w.parent[v] = -1;
    __syncwarp();
    if (lane == 0) w.parent[root] = 0xFFFF;
    __syncwarp();
    int reached = 1;
    for (int d = 1; d < g.n_nodes; ++d) {
        if (stop >= 0 && vload(&w.parent[stop]) != -1) break;
        int claimed = 0;
        for (int e = lane; e < n; e += 32) {
            if (!w.x[e]) continue;
            const int u = s_src[e], v = s_dst[e];
            const int pu = vload(&w.parent[u]), pv = vload(&w.parent[v]);
            if (pu != -1 && (pu >> 16) == d - 1 && pv == -1) {
                if (atomicCAS(&w.parent[v], -1, (d << 16) | e) == -1) ++claimed;
            } else if (pv != -1 && (pv >> 16) == d - 1 && pu == -1) {
                if (atomicCAS(&w.parent[u], -1, (d << 16) | e) == -1) ++claimed;
            }
        }
        claimed = __reduce_add_sync(0xffffffffu, claimed);
        __syncwarp();
        if (claimed == 0) break;
        reached += claimed;
    }
    return reached;
}

// With a spanning tree from bfs_tree that reached every node: true iff no
// working edge is a bridge.
__device__ bool bridgeless(const Sys &g, int n, WarpScratch &w, const int32_t *s_src, const int32_t *s_dst,
                           int32_t *err) {
    const int lane = threadIdx.x & 31;
    for (int e = lane; e < n; e += 32) w.flow[e] = 0;   // "covered" marks of tree edges
    __syncwarp();
    for (int e = lane; e < n; e += 32) {
        if (!w.x[e]) continue;
        int a = s_src[e], b = s_dst[e];
        if (a == b || (w.parent[a] & 0xFFFF) == e || (w.parent[b] & 0xFFFF) == e) continue;   // loop / tree edge
        for (int guard = 0; a != b && guard < 2 * g.n_nodes; ++guard) {
            const int qa = w.parent[a], qb = w.parent[b];
            if ((qa & 0xFFFF) >= n && (qb & 0xFFFF) >= n) {
                atomicMax(err, 3);   // both at the root yet apart: cannot happen; recorded, walk stopped
                break;
            }
            if ((qa >> 16) >= (qb >> 16) && (qa & 0xFFFF) < n) {
                const int ea = qa & 0xFFFF;
                w.flow[ea] = 1;
                a = s_src[ea] == a ? s_dst[ea] : s_src[ea];
            } else if ((qb & 0xFFFF) < n) {
                const int eb = qb & 0xFFFF;
                w.flow[eb] = 1;
                b = s_src[eb] == b ? s_dst[eb] : s_src[eb];
            } else {
                const int ea = qa & 0xFFFF;   // b is the root, a is not
                w.flow[ea] = 1;
                a = s_src[ea] == a ? s_dst[ea] : s_src[ea];
            }
        }
    }
    __syncwarp();
    bool ok = true;
    for (int v = lane + 1; v < g.n_nodes; v += 32) {
        const int e = w.parent[v] & 0xFFFF;
        if (e >= n || w.flow[e] == 0) ok = false;
    }
    return __all_sync(0xffffffffu, ok);
}

// One augmenting path s -> t in the residual graph of the flow in w.flow
// (capacities w.x), found by a warp-parallel search; parents (2a forward,
// 2a+1 backward arc) are claimed with atomicCAS, so they form a tree rooted at
// s.  True if t was reached.
__device__ bool residual_path(const Sys &g, int n, WarpScratch &w, const int32_t *s_src, const int32_t *s_dst) {
    const int lane = threadIdx.x & 31;
    for (int v = lane; v < g.n_nodes; v += 32) w.parent[v] = -1;
    __syncwarp();
    if (lane == 0) w.parent[g.s] = -2;
    __syncwarp();
    for (int sweep = 0; sweep <= g.n_nodes; ++sweep) {
        bool changed = false;
        for (int a = lane; a < n; a += 32) {
            const int u = s_src[a], v = s_dst[a];
            const int pu = vload(&w.parent[u]), pv = vload(&w.parent[v]);
            if (pu != -1 && pv == -1 && w.flow[a] < (int)w.x[a]) {
                if (atomicCAS(&w.parent[v], -1, 2 * a) == -1) changed = true;
            } else if (pv != -1 && pu == -1 && w.flow[a] > 0) {
                if (atomicCAS(&w.parent[u], -1, 2 * a + 1) == -1) changed = true;
            }
        }
        __syncwarp();
        if (vload(&w.parent[g.t]) != -1) return true;
        if (!__any_sync(0xffffffffu, changed)) return false;
    }
    return vload(&w.parent[g.t]) != -1;
}

// Push `amount` (> 0: the bottleneck is computed; < 0: exactly -amount is
// taken back) along the path of residual_path.  Lane 0 works; returns the
// amount pushed (warp-uniform), 0 on a broken chain (recorded).
__device__ int push_path(const Sys &g, WarpScratch &w, const int32_t *s_src, const int32_t *s_dst, int amount,
                         int32_t *err) {
    const int lane = threadIdx.x & 31;
    int pushed = 0;
    if (lane == 0) {
        int b = amount;
        int v = g.t, guard = 0;
        if (amount > 0) {
            b = 0x7fffffff;
            while (v != g.s && guard++ <= g.n_nodes) {
                const int pa = w.parent[v], a = pa >> 1;
                const int r = (pa & 1) ? (int)w.flow[a] : (int)w.x[a] - (int)w.flow[a];
                b = r < b ? r : b;
                v = (pa & 1) ? s_dst[a] : s_src[a];
            }
            if (v != g.s) {
                atomicMax(err, 3);  // a broken parent chain cannot happen; recorded, not pushed
                b = 0;
            }
            if (amount < b) b = amount;
        }
        v = g.t;
        guard = 0;
        while (b != 0 && v != g.s && guard++ <= g.n_nodes) {
            const int pa = w.parent[v], a = pa >> 1;
            w.flow[a] += (pa & 1) ? -b : b;
            v = (pa & 1) ? s_dst[a] : s_src[a];
        }
        pushed = b;
    }
    pushed = __shfl_sync(0xffffffffu, pushed, 0);
    __syncwarp();
    return pushed;
}

// Ford-Fulkerson from zero flow, stopping once the flow reaches `target`.
// Returns the flow value; w.flow holds the flow.
__device__ int maxflow_to(const Sys &g, int n, WarpScratch &w, const int32_t *s_src, const int32_t *s_dst,
                          int target, int32_t *err) {
    const int lane = threadIdx.x & 31;
    for (int a = lane; a < n; a += 32) w.flow[a] = 0;
    __syncwarp();
    int total = 0;
    while (total < target) {
        if (!residual_path(g, n, w, s_src, s_dst)) break;
        const int push = push_path(g, w, s_src, s_dst, 0x7fffffff, err);
        if (push <= 0) break;
        total += push;
    }
    return total;
}

// Phi(x) <= m' ?  (warp-uniform result; x in w.x)
__device__ bool phi_le(const Sys &g, int n, WarpScratch &w, const int32_t *s_src, const int32_t *s_dst,
                       int32_t *err) {
    const int lane = threadIdx.x & 31;
    const int nw = (g.n_nodes + 31) / 32;
    if (g.kind == RSR_PHI_GLOBAL_CONNECTIVITY || g.kind == RSR_PHI_GLOBAL_CONN_LEVEL) {
        const int top = g.kind == RSR_PHI_GLOBAL_CONNECTIVITY ? 1 : 2;
        if (g.m_prime >= top) return true;
        if (bfs_tree(g, n, w, s_src, s_dst) < g.n_nodes) return true;        // Phi = 0
        if (g.m_prime == 0) return false;                                    // Phi >= 1
        return !bridgeless(g, n, w, s_src, s_dst, err);                      // m' = 1: Phi = 1 ?
    }
    if (g.kind == RSR_PHI_ST_CONNECTIVITY) {
        if (g.m_prime >= 1) return true;
        for (int i = lane; i < nw; i += 32) w.vis[i] = 0u;
        __syncwarp();
        if (lane == 0) w.vis[g.s >> 5] |= 1u << (g.s & 31);
        __syncwarp();
        for (int sweep = 0; sweep <= g.n_nodes; ++sweep) {
            bool changed = false;
            for (int e = lane; e < n; e += 32) {
                if (!w.x[e]) continue;
                const int u = s_src[e], v = s_dst[e];
                const bool bu = bit(w.vis, u), bv = bit(w.vis, v);
                if (bu != bv) {
                    const int o = bu ? v : u;
                    atomicOr(&w.vis[o >> 5], 1u << (o & 31));
                    changed = true;
                }
            }
            __syncwarp();
            if (bit(w.vis, g.t)) return false;  // connected: Phi = 1 > m' = 0
            if (!__any_sync(0xffffffffu, changed)) break;
        }
        return true;
    }
    // max flow; the decision needs only whether the flow reaches thr[m'] (ascending thresholds)
    const int target = g.m_prime < g.n_levels ? g.thr[g.m_prime] : 0x7fffffff;
    return maxflow_to(g, n, w, s_src, s_dst, target, err) < target;
}

// Graph and sampler thresholds into shared memory (whole block).
__device__ void stage_system(const ClassifyParams &p, const Sys &g, int32_t *s_src, int32_t *s_dst,
                             unsigned long long *s_thr, int32_t *err) {
    for (int i = threadIdx.x; i < p.n; i += blockDim.x) {
        int u = g.src[i], v = g.dst[i];
        if (u < 0 || u >= g.n_nodes || v < 0 || v >= g.n_nodes) {
            atomicMax(err, 2);  // node index out of range: the edge is dropped
            u = v = 0;
        }
        s_src[i] = u;
        s_dst[i] = v;
    }
    for (int i = threadIdx.x; i < p.n * p.km1; i += blockDim.x) s_thr[i] = p.thr[i];
    __syncthreads();
}

// States of sample offset + hl into w.x (whole warp).
__device__ void regen_sample(const ClassifyParams &p, int64_t hl, WarpScratch &w, const unsigned long long *s_thr) {
    const int lane = threadIdx.x & 31;
    const uint32_t key0 = (uint32_t)p.seed, key1 = (uint32_t)(p.seed >> 32);
    const uint64_t h = p.offset + (uint64_t)hl;
    for (int q = lane; 4 * q < p.n; q += 32) {
        const U32x4 r = philox4x32_10((uint32_t)h, (uint32_t)(h >> 32), (uint32_t)q, 0u, key0, key1);
        const uint32_t us[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int i = 4 * q + c;
            if (i < p.n) w.x[i] = (uint8_t)state_from_uniform(us[c], s_thr + (size_t)i * p.km1, p.km1);
        }
    }
    __syncwarp();
}

__global__ void __launch_bounds__(kWarps * 32, 12) resolve_kernel(const ClassifyParams p, const Sys g, uint8_t *labels,
                                                              int64_t *u_lower_idx, int64_t cap,
                                                              unsigned long long *counts2) {
    extern __shared__ __align__(16) unsigned char s_dyn[];
    const SysSmem L = sys_smem(p.n, p.km1, g.n_nodes, kWarps);
    int32_t *s_src = reinterpret_cast<int32_t *>(s_dyn + L.off_src);
    int32_t *s_dst = reinterpret_cast<int32_t *>(s_dyn + L.off_dst);
    unsigned long long *s_thr = reinterpret_cast<unsigned long long *>(s_dyn + L.off_thr);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t *err = &p.hdr->error;
    stage_system(p, g, s_src, s_dst, s_thr, err);
    WarpScratch w = warp_view(s_dyn, L, warp);
    const int64_t warps_total = (int64_t)gridDim.x * kWarps;
    for (int64_t base = ((int64_t)blockIdx.x * kWarps + warp) * 32; base < p.N; base += warps_total * 32) {
        const int64_t mine = base + lane;
        const bool unl = mine < p.N && labels[mine] == 2;
        unsigned todo = __ballot_sync(0xffffffffu, unl);
        while (todo) {
            const int src_lane = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t hl = base + src_lane;
            regen_sample(p, hl, w, s_thr);
            const bool lower = phi_le(g, p.n, w, s_src, s_dst, err);
            if (lane == 0) {
                labels[hl] = lower ? 3 : 4;
                if (lower) {
                    const unsigned long long pos = atomicAdd(&counts2[0], 1ull);
                    if ((int64_t)pos < cap) u_lower_idx[pos] = hl;
                    else atomicMax(err, 4);  // index list full: counts stay exact
                } else {
                    atomicAdd(&counts2[1], 1ull);
                }
            }
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------------------
// Incremental Phi for the search.  Every step of the componentwise search asks
// whether one more raise (lower side) or lowering (upper side) of component i
// crosses the boundary.  Where the system function allows, the answer comes
// from state kept across steps instead of a new evaluation from scratch; the
// answer is the same, so the references and the evaluation counts are too.
//   s-t / global connectivity, raising (Phi = 0 kept): union-find over the
//     working edges; an added edge crosses iff it joins s's and t's components
//     (s-t) or the last two components (global).
//   s-t / global connectivity, lowering (Phi = 1 kept): a witness (an s-t path,
//     a spanning tree) in the edge bitmask; deleting an edge outside it keeps
//     Phi; deleting a witness edge triggers a breadth-first search that also
//     rebuilds the witness.
//   max flow, raising (flow < target kept, w.flow a maximum flow): one unit of
//     capacity raises the maximum flow by at most one, so one residual path
//     search decides; a path that reaches the target is pushed back.
//   max flow, lowering (flow >= target kept, w.flow a feasible flow): if the
//     arc carries less than its capacity the flow stays feasible; otherwise the
//     flow is recomputed up to the target, from a saved copy if that fails.
// Other cases (the connectivity grade, m' beyond the levels) evaluate Phi.
// ---------------------------------------------------------------------------
enum SearchMode { kGeneric = 0, kDsuSt, kPathSt, kDsuGlobal, kTreeGlobal, kFlowRaise, kFlowLower };

// Adjacency of the block's graph (compressed rows in shared memory): the edges
// of node v are adj[off[v] .. off[v+1]).  Built once per block.
struct Csr {
    int32_t *off;     // [n_nodes + 1]
    int32_t *cur;     // [n_nodes] fill cursors
    int16_t *adj;     // [2 n]
};

__device__ void build_csr(const Sys &g, int n, const int32_t *s_src, const int32_t *s_dst, Csr c) {
    for (int v = threadIdx.x; v <= g.n_nodes; v += blockDim.x) c.off[v] = 0;
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        atomicAdd(&c.off[s_src[e] + 1], 1);
        atomicAdd(&c.off[s_dst[e] + 1], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int v = 0; v < g.n_nodes; ++v) c.off[v + 1] += c.off[v];
    __syncthreads();
    for (int v = threadIdx.x; v < g.n_nodes; v += blockDim.x) c.cur[v] = c.off[v];
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        c.adj[atomicAdd(&c.cur[s_src[e]], 1)] = (int16_t)e;
        c.adj[atomicAdd(&c.cur[s_dst[e]], 1)] = (int16_t)e;
    }
    __syncthreads();
}

// Breadth-first tree from `root` over working edges, frontier by frontier over
// the adjacency lists: each level touches only the edges of its frontier, so a
// search costs O(edges) instead of O(levels x edges).  Same parent encoding as
// bfs_tree (depth << 16 | edge, 0xFFFF at the root, -1 unreached); stops once
// `stop` (>= 0) is reached.  qa, qb: per-warp frontier buffers [n_nodes];
// *cnt: a per-warp counter.  Returns the number of reached nodes.
__device__ int bfs_csr(const Sys &g, WarpScratch &w, const int32_t *s_src, const int32_t *s_dst, const Csr &c,
                       int root, int stop, int16_t *qa, int16_t *qb, int *cnt) {
    const int lane = threadIdx.x & 31;
    for (int v = lane; v < g.n_nodes; v += 32) w.parent[v] = -1;
    __syncwarp();
    if (lane == 0) {
        w.parent[root] = 0xFFFF;
        qa[0] = (int16_t)root;
        *cnt = 0;
    }
    __syncwarp();
    int nf = 1, reached = 1;
    for (int d = 1; nf > 0 && d < g.n_nodes; ++d) {
        if (stop >= 0 && vload(&w.parent[stop]) != -1) break;
        for (int f = lane; f < nf; f += 32) {
            const int v = qa[f];
            for (int k = c.off[v]; k < c.off[v + 1]; ++k) {
                const int e = c.adj[k];
                if (!w.x[e]) continue;
                const int u = s_src[e] == v ? s_dst[e] : s_src[e];
                if (vload(&w.parent[u]) == -1 && atomicCAS(&w.parent[u], -1, (d << 16) | e) == -1)
                    qb[atomicAdd(cnt, 1)] = (int16_t)u;
            }
        }
        __syncwarp();
        nf = *(volatile int *)cnt;
        __syncwarp();
        if (lane == 0) *cnt = 0;
        reached += nf;
        int16_t *t = qa;
        qa = qb;
        qb = t;
        __syncwarp();
    }
    return reached;
}

__device__ __forceinline__ int dsu_find(int32_t *par, int v) {
    while (par[v] != v) {
        par[v] = par[par[v]];
        v = par[v];
    }
    return v;
}

__device__ __forceinline__ void set_edge_bit(uint32_t *bits, int e) { atomicOr(&bits[e >> 5], 1u << (e & 31)); }

// Witness bitmask of the tree in w.parent: the path t -> root (s-t) or every tree edge (global).
__device__ void build_witness(const Sys &g, int n, WarpScratch &w, const int32_t *s_src, const int32_t *s_dst,
                              bool path_only, int32_t *err) {
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < (n + 31) / 32; i += 32) w.vis[i] = 0u;
    __syncwarp();
    if (path_only) {
        if (lane == 0) {
            int v = g.t, guard = 0;
            while (v != g.s && guard++ <= g.n_nodes) {
                const int e = w.parent[v] & 0xFFFF;
                if (e >= n) {
                    atomicMax(err, 3);
                    break;
                }
                w.vis[e >> 5] |= 1u << (e & 31);
                v = s_src[e] == v ? s_dst[e] : s_src[e];
            }
        }
    } else {
        for (int v = lane; v < g.n_nodes; v += 32) {
            const int e = w.parent[v] & 0xFFFF;
            if (e < n) set_edge_bit(w.vis, e);
        }
    }
    __syncwarp();
}

// With w.parent a spanning tree of the working graph (depth << 16 | edge,
// 0xFFFF at the root) and its tree edge e just removed (w.x[e] = 0): is there a
// working non-tree edge with one end below e and the other above?  The nodes
// below e are marked in w.flow (int16 per node) by walking each node up to the
// depth of e's lower end.  Warp-uniform.
__device__ bool tree_edge_has_cover(const Sys &g, int n, WarpScratch &w, const int32_t *s_src, const int32_t *s_dst,
                                    int e) {
    const int lane = threadIdx.x & 31;
    const int a = s_src[e], b = s_dst[e];
    const int c = (w.parent[a] & 0xFFFF) == e ? a : b;   // the lower end
    const int dc = w.parent[c] >> 16;
    for (int v = lane; v < g.n_nodes; v += 32) {
        int y = v;
        for (int guard = 0; (w.parent[y] >> 16) > dc && guard < g.n_nodes; ++guard) {
            const int pe = w.parent[y] & 0xFFFF;
            y = s_src[pe] == y ? s_dst[pe] : s_src[pe];
        }
        w.flow[v] = (int16_t)(y == c ? 1 : 0);
    }
    __syncwarp();
    bool found = false;
    for (int f = lane; f < n && !found; f += 32) {
        if (f == e || !w.x[f] || ((w.vis[f >> 5] >> (f & 31)) & 1u)) continue;
        found = w.flow[s_src[f]] != w.flow[s_dst[f]];
    }
    found = __any_sync(0xffffffffu, found);
    __syncwarp();
    return found;
}

struct SearchBufs {
    Csr csr;
    int16_t *qa, *qb;   // frontier buffers (the flow arrays; connectivity does not use them)
    int *cnt;
};

__device__ int search_setup(const Sys &g, int n, bool lower, WarpScratch &w, const int32_t *s_src,
                            const int32_t *s_dst, int *state, int32_t *err, const SearchBufs &sb) {
    const int lane = threadIdx.x & 31;
    const bool st = g.kind == RSR_PHI_ST_CONNECTIVITY, gl = g.kind == RSR_PHI_GLOBAL_CONNECTIVITY;
    if ((st || gl) && g.m_prime == 0) {
        if (lower) {
            // union-find over the working edges (lane 0); state = components (global)
            for (int v = lane; v < g.n_nodes; v += 32) w.parent[v] = v;
            __syncwarp();
            int comps = g.n_nodes;
            if (lane == 0) {
                for (int e = 0; e < n; ++e) {
                    if (!w.x[e]) continue;
                    const int ru = dsu_find(w.parent, s_src[e]), rv = dsu_find(w.parent, s_dst[e]);
                    if (ru != rv) {
                        w.parent[ru] = rv;
                        --comps;
                    }
                }
            }
            *state = __shfl_sync(0xffffffffu, comps, 0);
            __syncwarp();
            return st ? kDsuSt : kDsuGlobal;
        }
        bfs_csr(g, w, s_src, s_dst, sb.csr, st ? g.s : 0, st ? g.t : -1, sb.qa, sb.qb, sb.cnt);
        build_witness(g, n, w, s_src, s_dst, st, err);
        return st ? kPathSt : kTreeGlobal;
    }
    if (g.kind == RSR_PHI_ST_MAXFLOW_LEVELS && g.m_prime < g.n_levels) {
        // the decision left w.flow at a maximum flow (< target) or a feasible flow (>= target)
        int total = 0;
        if (lane == 0) {
            for (int a = 0; a < n; ++a) {
                if (s_src[a] == g.s) total += w.flow[a];
                if (s_dst[a] == g.s) total -= w.flow[a];
            }
        }
        *state = __shfl_sync(0xffffffffu, total, 0);
        return lower ? kFlowRaise : kFlowLower;
    }
    return kGeneric;
}

// One search step on component i: raise (lower side) or lower it by one state.
// Keeps the step and returns true if Phi stays on the start's side; otherwise
// undoes it and returns false.  Warp-uniform.
__device__ bool try_step(const Sys &g, int n, int mode, bool lower, int i, WarpScratch &w, int16_t *bak,
                         const int32_t *s_src, const int32_t *s_dst, int *state, int32_t *err,
                         const SearchBufs &sb) {
    const int lane = threadIdx.x & 31;
    const int d = lower ? 1 : -1;
    switch (mode) {
        case kDsuSt:
        case kDsuGlobal: {
            int keep = 1, comps = *state;
            if (lane == 0) {
                const int ru = dsu_find(w.parent, s_src[i]), rv = dsu_find(w.parent, s_dst[i]);
                if (ru != rv) {
                    if (mode == kDsuSt) {
                        const int rs = dsu_find(w.parent, g.s), rt = dsu_find(w.parent, g.t);
                        keep = !((ru == rs && rv == rt) || (ru == rt && rv == rs));
                    } else {
                        keep = comps > 2;
                    }
                    if (keep) {
                        w.parent[ru] = rv;
                        --comps;
                    }
                }
                if (keep) w.x[i] = 1;
            }
            keep = __shfl_sync(0xffffffffu, keep, 0);
            *state = __shfl_sync(0xffffffffu, comps, 0);
            __syncwarp();
            return keep != 0;
        }
        case kPathSt:
        case kTreeGlobal: {
            const bool on = (w.vis[i >> 5] >> (i & 31)) & 1u;
            __syncwarp();
            if (lane == 0) w.x[i] = 0;
            __syncwarp();
            if (!on) return true;
            bool ok;
            if (mode == kPathSt) {
                bfs_csr(g, w, s_src, s_dst, sb.csr, g.s, g.t, sb.qa, sb.qb, sb.cnt);
                ok = vload(&w.parent[g.t]) != -1;
            } else {
                // w.parent is the witness spanning tree (depth << 16 | edge).  Removing
                // its edge i splits it into the subtree below i and the rest; the
                // working graph stays connected iff another working edge joins the two.
                // Only then is the tree rebuilt; a bridge costs no search.
                if (!tree_edge_has_cover(g, n, w, s_src, s_dst, i)) {
                    if (lane == 0) w.x[i] = 1;
                    __syncwarp();
                    return false;
                }
                ok = bfs_csr(g, w, s_src, s_dst, sb.csr, 0, -1, sb.qa, sb.qb, sb.cnt) == g.n_nodes;
            }
            if (ok) {
                build_witness(g, n, w, s_src, s_dst, mode == kPathSt, err);
            } else {
                if (lane == 0) w.x[i] = 1;
                __syncwarp();
            }
            return ok;
        }
        case kFlowRaise: {
            const int target = g.thr[g.m_prime];
            if (lane == 0) w.x[i] += 1;
            __syncwarp();
            if (!residual_path(g, n, w, s_src, s_dst)) return true;     // maximum flow unchanged
            const int pushed = push_path(g, w, s_src, s_dst, 1, err);
            if (*state + pushed < target) {
                *state += pushed;
                return true;
            }
            push_path(g, w, s_src, s_dst, -pushed, err);                 // take the unit back
            if (lane == 0) w.x[i] -= 1;
            __syncwarp();
            return false;
        }
        case kFlowLower: {
            const int target = g.thr[g.m_prime];
            const bool fits = (int)w.flow[i] < (int)w.x[i];
            __syncwarp();
            if (lane == 0) w.x[i] -= 1;
            __syncwarp();
            if (fits) return true;                                       // the flow stays feasible
            for (int a = lane; a < n; a += 32) bak[a] = w.flow[a];
            __syncwarp();
            const int tot = maxflow_to(g, n, w, s_src, s_dst, target, err);
            if (tot >= target) {
                *state = tot;
                return true;
            }
            for (int a = lane; a < n; a += 32) w.flow[a] = bak[a];
            if (lane == 0) w.x[i] += 1;
            __syncwarp();
            return false;
        }
        default: {
            __syncwarp();
            if (lane == 0) w.x[i] += d;
            __syncwarp();
            const bool ok = phi_le(g, n, w, s_src, s_dst, err) == lower;
            if (!ok) {
                __syncwarp();
                if (lane == 0) w.x[i] -= d;
                __syncwarp();
            }
            return ok;
        }
    }
}

// Permuted visiting order from sample h: Fisher-Yates over 0..n-1 driven by
// Philox4x32-10 (key = seed, counter (h lo, h hi, floor(i/4), 1)); for
// i = n-1 down to 1, j = (u * (i+1)) >> 32 with u = word (i mod 4).  One lane.
__device__ void search_order(const ClassifyParams &p, uint64_t h, int16_t *ord) {
    const uint32_t key0 = (uint32_t)p.seed, key1 = (uint32_t)(p.seed >> 32);
    for (int i = 0; i < p.n; ++i) ord[i] = (int16_t)i;
    U32x4 blk{0u, 0u, 0u, 0u};
    int cur = -1;
    for (int i = p.n - 1; i >= 1; --i) {
        if ((i >> 2) != cur) {
            cur = i >> 2;
            blk = philox4x32_10((uint32_t)h, (uint32_t)(h >> 32), (uint32_t)cur, 1u, key0, key1);
        }
        const uint32_t u = (i & 3) == 0 ? blk.x : (i & 3) == 1 ? blk.y : (i & 3) == 2 ? blk.z : blk.w;
        const int j = (int)(((unsigned long long)u * (unsigned long long)(i + 1)) >> 32);
        const int16_t tmp = ord[i];
        ord[i] = ord[j];
        ord[j] = tmp;
    }
}

// Componentwise boundary search (Sec. 3.4) from samples offset + starts[j];
// order_mode 0 visits components in index order, 1 in search_order.
__global__ void __launch_bounds__(kWarps * 32) search_kernel(const ClassifyParams p, const Sys g,
                                                             const int64_t *starts, int64_t n_starts,
                                                             uint8_t *refs_out, uint8_t *side_out,
                                                             unsigned long long *evals, int order_mode) {
    extern __shared__ __align__(16) unsigned char s_dyn[];   // SearchSmem
    const SearchSmem L = search_smem(p.n, p.km1, g.n_nodes, kWarps);
    int32_t *s_src = reinterpret_cast<int32_t *>(s_dyn + L.sys.off_src);
    int32_t *s_dst = reinterpret_cast<int32_t *>(s_dyn + L.sys.off_dst);
    unsigned long long *s_thr = reinterpret_cast<unsigned long long *>(s_dyn + L.sys.off_thr);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t *err = &p.hdr->error;
    stage_system(p, g, s_src, s_dst, s_thr, err);
    WarpScratch w = warp_view(s_dyn, L.sys, warp);
    int16_t *ord = reinterpret_cast<int16_t *>(s_dyn + L.off_ord + L.warp_bytes * (size_t)warp);
    int16_t *bak = reinterpret_cast<int16_t *>(s_dyn + L.off_ord + L.warp_bytes * (size_t)warp + L.off_bak);
    SearchBufs sb;
    sb.csr.off = reinterpret_cast<int32_t *>(s_dyn + L.off_off);
    sb.csr.cur = reinterpret_cast<int32_t *>(s_dyn + L.off_cur);
    sb.csr.adj = reinterpret_cast<int16_t *>(s_dyn + L.off_adj);
    sb.cnt = reinterpret_cast<int *>(s_dyn + L.off_cnt) + warp;
    sb.qa = w.flow;
    sb.qb = bak;
    const bool csr = g.kind == RSR_PHI_ST_CONNECTIVITY || g.kind == RSR_PHI_GLOBAL_CONNECTIVITY;
    if (csr) build_csr(g, p.n, s_src, s_dst, sb.csr);
    const int top = p.K - 1;
    for (int64_t j = (int64_t)blockIdx.x * kWarps + warp; j < n_starts; j += (int64_t)gridDim.x * kWarps) {
        regen_sample(p, starts[j], w, s_thr);
        if (order_mode) {
            if (lane == 0) search_order(p, p.offset + (uint64_t)starts[j], ord);
            __syncwarp();
        }
        const bool lower = phi_le(g, p.n, w, s_src, s_dst, err);
        unsigned long long ev = 1;
        if (!lower && g.kind == RSR_PHI_GLOBAL_CONNECTIVITY && g.m_prime == 0) {
            // Lowering a connected state: each working edge, in the visiting order, is
            // removed if the graph stays connected without it.  That is reverse deletion
            // with the visit positions as distinct weights, and it keeps exactly the
            // spanning tree that Kruskal's algorithm builds from the working edges taken
            // in reverse visiting order (the unique minimum spanning tree for those
            // weights).  One union-find pass gives the same state; the count of Phi
            // evaluations is unchanged: one decision per working edge.
            for (int v = lane; v < g.n_nodes; v += 32) w.parent[v] = v;
            __syncwarp();
            if (lane == 0) {
                for (int step = p.n - 1; step >= 0; --step) {
                    const int i = order_mode ? (int)ord[step] : step;
                    if (!w.x[i]) continue;
                    ++ev;
                    const int ru = dsu_find(w.parent, s_src[i]), rv = dsu_find(w.parent, s_dst[i]);
                    if (ru != rv) w.parent[ru] = rv;
                    else w.x[i] = 0;
                }
            }
            __syncwarp();
        } else {
        int state = 0;
        const int mode = search_setup(g, p.n, lower, w, s_src, s_dst, &state, err, sb);
        for (int step = 0; step < p.n; ++step) {
            const int i = order_mode ? (int)ord[step] : step;
            if (lower) {
                while (w.x[i] < top) {
                    ++ev;
                    if (!try_step(g, p.n, mode, true, i, w, bak, s_src, s_dst, &state, err, sb)) break;
                }
            } else {
                while (w.x[i] > 0) {
                    ++ev;
                    if (!try_step(g, p.n, mode, false, i, w, bak, s_src, s_dst, &state, err, sb)) break;
                }
            }
        }
        }
        __syncwarp();
        for (int i = lane; i < p.n; i += 32) refs_out[(size_t)j * p.n + i] = w.x[i];
        if (lane == 0) {
            side_out[j] = lower ? 0 : 1;
            atomicAdd(evals, ev);
        }
        __syncwarp();
    }
}

// Phi(x) given that it lies in [lo, hi] (lo < hi).  Max flow: one computation up
// to the top open threshold, then S = the first m' in [lo, hi) whose threshold
// the flow does not reach.  Connectivity grade: connectivity once, bridges once.
// Otherwise decisions Phi <= m' from lo upwards.
__device__ int phi_in_bracket(const Sys &g, int n, WarpScratch &w, const int32_t *s_src, const int32_t *s_dst,
                              int lo, int hi, int32_t *err) {
    if (g.kind == RSR_PHI_ST_MAXFLOW_LEVELS && hi <= g.n_levels) {
        const int f = maxflow_to(g, n, w, s_src, s_dst, g.thr[hi - 1], err);
        int S = lo;
        while (S < hi && f >= g.thr[S]) ++S;
        return S;
    }
    if (g.kind == RSR_PHI_GLOBAL_CONN_LEVEL) {
        int S;
        if (bfs_tree(g, n, w, s_src, s_dst) < g.n_nodes) S = 0;
        else S = bridgeless(g, n, w, s_src, s_dst, err) ? 2 : 1;
        return S < lo ? lo : (S > hi ? hi : S);
    }
    for (int m = lo; m < hi; ++m) {
        Sys gm = g;
        gm.m_prime = m;
        if (phi_le(gm, n, w, s_src, s_dst, err)) return m;
    }
    return hi;
}

// System-state level of every sample from the labels of nb boundaries
// (labels[b*N + h], boundary m' = b): a lower match at b bounds S <= b, an
// upper match S >= b+1.  Where the bounds meet the level is known; otherwise
// Phi decides, boundary by boundary from the lowest open one.
__global__ void __launch_bounds__(kWarps * 32, 12) levels_kernel(const ClassifyParams p, const Sys g, int nb,
                                                             const uint8_t *labels, uint8_t *levels_out,
                                                             unsigned long long *level_counts,
                                                             unsigned long long *n_phi) {
    extern __shared__ __align__(16) unsigned char s_dyn[];
    const SysSmem L = sys_smem(p.n, p.km1, g.n_nodes, kWarps);
    int32_t *s_src = reinterpret_cast<int32_t *>(s_dyn + L.off_src);
    int32_t *s_dst = reinterpret_cast<int32_t *>(s_dyn + L.off_dst);
    unsigned long long *s_thr = reinterpret_cast<unsigned long long *>(s_dyn + L.off_thr);
    __shared__ unsigned long long s_hist[kMaxLevels];
    __shared__ unsigned long long s_phi;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t *err = &p.hdr->error;
    if (threadIdx.x < kMaxLevels) s_hist[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) s_phi = 0ull;
    stage_system(p, g, s_src, s_dst, s_thr, err);
    WarpScratch w = warp_view(s_dyn, L, warp);
    const int64_t warps_total = (int64_t)gridDim.x * kWarps;
    for (int64_t base = ((int64_t)blockIdx.x * kWarps + warp) * 32; base < p.N; base += warps_total * 32) {
        const int64_t h = base + lane;
        const bool valid = h < p.N;
        int lo = 0, hi = nb;
        if (valid) {
            for (int b = 0; b < nb; ++b) {
                const uint8_t lab = labels[(size_t)b * p.N + h];
                if (lab == 0) hi = b < hi ? b : hi;
                else if (lab == 1) lo = b + 1 > lo ? b + 1 : lo;
            }
            if (lo > hi) {
                atomicMax(err, 5);   // a lower and an upper bound that exclude each other: inconsistent references
            } else if (lo == hi) {
                if (levels_out) levels_out[h] = (uint8_t)lo;
                atomicAdd(&s_hist[lo], 1ull);
            }
        }
        unsigned todo = __ballot_sync(0xffffffffu, valid && lo < hi);
        while (todo) {
            const int src_lane = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t hs = base + src_lane;
            const int slo = __shfl_sync(0xffffffffu, lo, src_lane), shi = __shfl_sync(0xffffffffu, hi, src_lane);
            regen_sample(p, hs, w, s_thr);
            const int S = phi_in_bracket(g, p.n, w, s_src, s_dst, slo, shi, err);
            if (lane == 0) {
                if (levels_out) levels_out[hs] = (uint8_t)S;
                atomicAdd(&s_hist[S], 1ull);
                atomicAdd(&s_phi, 1ull);
            }
            __syncwarp();
        }
    }
    __syncthreads();
    if (threadIdx.x <= nb && s_hist[threadIdx.x]) atomicAdd(&level_counts[threadIdx.x], s_hist[threadIdx.x]);
    if (threadIdx.x == 0 && n_phi && s_phi) atomicAdd(n_phi, s_phi);
}

}  // namespace

namespace {
Sys make_sys(const rsr_system &sys) {
    Sys g{};
    g.kind = sys.kind;
    g.n_nodes = sys.n_nodes;
    g.s = sys.s;
    g.t = sys.t;
    g.n_levels = sys.n_levels;
    g.m_prime = sys.m_prime;
    for (int l = 0; l < 8; ++l) g.thr[l] = sys.level_thr[l];
    g.src = sys.src;
    g.dst = sys.dst;
    return g;
}
}  // namespace

// The largest dynamic shared memory the two Stage-2 kernels can ask for (n and
// n_nodes at their limits), allowed once per device.
cudaError_t allow_dynamic_smem() {
    static int done[64] = {0};
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return e;
    if (d >= 0 && d < 64 && done[d]) return cudaSuccess;
    const int mx = (int)sys_smem(kMaxKenc, 1, kMaxNodes, kWarps).total;   // n (K-1) <= kMaxKenc, n <= kMaxKenc
    if ((e = cudaFuncSetAttribute(resolve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(levels_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)) != cudaSuccess)
        return e;
    if (d >= 0 && d < 64) done[d] = 1;
    return cudaSuccess;
}

cudaError_t launch_resolve(const ClassifyParams &p, const rsr_system &sys, uint8_t *labels, int64_t *u_lower_idx,
                           int64_t cap, unsigned long long *counts2, cudaStream_t s) {
    if (p.N <= 0) return cudaSuccess;
    const Sys g = make_sys(sys);
    const size_t smem = sys_smem(p.n, p.km1, g.n_nodes, kWarps).total;
    cudaError_t e = allow_dynamic_smem();
    if (e != cudaSuccess) return e;
    const int64_t warps = (p.N + 31) / 32;
    const int64_t grid = std::min<int64_t>((warps + kWarps - 1) / kWarps, (int64_t)device_sm_count() * 16);
    resolve_kernel<<<(unsigned)grid, kWarps * 32, smem, s>>>(p, g, labels, u_lower_idx, cap, counts2);
    return cudaGetLastError();
}

cudaError_t launch_search(const ClassifyParams &p, const rsr_system &sys, const int64_t *starts, int64_t n_starts,
                          uint8_t *refs_out, uint8_t *side_out, unsigned long long *evals, int order_mode,
                          cudaStream_t s) {
    if (n_starts <= 0) return cudaSuccess;
    // the largest layout (n and n_nodes at their limits) is allowed once per device
    static int attr_set[64] = {0};
    const int d = [] { int v = 0; cudaGetDevice(&v); return v; }();
    if (d >= 0 && d < 64 && !attr_set[d]) {
        const int mx = (int)search_smem(kMaxKenc, 1, kMaxNodes, kWarps).total;
        const cudaError_t e = cudaFuncSetAttribute(search_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        if (e != cudaSuccess) return e;
        attr_set[d] = 1;
    }
    const Sys g = make_sys(sys);
    const size_t smem = search_smem(p.n, p.km1, g.n_nodes, kWarps).total;
    const int64_t grid = std::min<int64_t>((n_starts + kWarps - 1) / kWarps, (int64_t)device_sm_count() * 16);
    search_kernel<<<(unsigned)grid, kWarps * 32, smem, s>>>(p, g, starts, n_starts, refs_out, side_out, evals,
                                                             order_mode);
    return cudaGetLastError();
}

cudaError_t launch_levels(const ClassifyParams &p, const rsr_system &sys, int nb, const uint8_t *labels,
                          uint8_t *levels_out, unsigned long long *level_counts, unsigned long long *n_phi,
                          cudaStream_t s) {
    if (p.N <= 0) return cudaSuccess;
    if (nb < 1 || nb >= kMaxLevels) return cudaErrorInvalidValue;
    const Sys g = make_sys(sys);
    const size_t smem = sys_smem(p.n, p.km1, g.n_nodes, kWarps).total;
    cudaError_t e = allow_dynamic_smem();
    if (e != cudaSuccess) return e;
    const int64_t warps = (p.N + 31) / 32;
    const int64_t grid = std::min<int64_t>((warps + kWarps - 1) / kWarps, (int64_t)device_sm_count() * 16);
    levels_kernel<<<(unsigned)grid, kWarps * 32, smem, s>>>(p, g, nb, labels, levels_out, level_counts, n_phi);
    return cudaGetLastError();
}

int resolve_max_nodes() { return kMaxNodes; }

}  // namespace rsr
