// resolve.cu -- Stage 2 on the device (Sec. 3.5): the system function Phi is
// evaluated for every unclassified sample, which closes the estimate of
// P(S <= m') without the host.
//
// Built-in system functions (the two families of the paper's experiments):
//   RSR_PHI_ST_CONNECTIVITY   binary components are undirected edges; Phi = 1
//                             iff s reaches t over working edges (x_e = 1)
//   RSR_PHI_ST_MAXFLOW_LEVELS components are directed arcs with capacity x_a;
//                             Phi = #{l : maxflow(s -> t) >= thr_l}
// One warp per unclassified sample: its states are regenerated from Philox
// (lane-strided blocks), then
//   connectivity: label propagation over a shared-memory bitset, one edge per
//                 lane per sweep, until t is reached or nothing changes;
//   max flow:     Ford-Fulkerson; each augmenting path is found by a
//                 warp-parallel search of the residual graph (parents claimed
//                 with atomicCAS, so they form a tree rooted at s) and pushed
//                 by one lane; it stops as soon as the flow reaches the
//                 threshold that decides S <= m'.
// Labels 2 become 3 (Phi <= m') or 4 (Phi >= m'+1); the local indices of the
// 3s are appended to u_lower_idx (in no particular order) for rsr_grad.
#include <cuda_runtime.h>

#include "rsr.h"
#include "rsr_internal.cuh"
#include "rsr_launch.h"

namespace rsr {

namespace {

constexpr int kWarps = 4;          // warps per block, one sample each at a time
constexpr int kMaxNodes = 1024;

struct Sys {
    int32_t kind, n_nodes, s, t, n_levels, m_prime;
    int32_t thr[8];
    const int32_t *src, *dst;
};

struct WarpScratch {
    uint8_t x[kMaxKenc];           // component states of the sample
    uint32_t vis[kMaxNodes / 32];  // reached nodes (connectivity)
    int32_t parent[kMaxNodes];     // claimed residual arc (max flow), -1 = unreached
    int16_t flow[kMaxKenc];        // arc flows (max flow)
};

__device__ __forceinline__ bool bit(const uint32_t *v, int i) { return (v[i >> 5] >> (i & 31)) & 1u; }

// Phi(x) <= m' ?
__device__ bool resolve_lower(const Sys &g, int n, WarpScratch &w, const int32_t *s_src, const int32_t *s_dst,
                              int32_t *err) {
    const int lane = threadIdx.x & 31;
    const int nw = (g.n_nodes + 31) / 32;
    if (g.kind == RSR_PHI_ST_CONNECTIVITY) {
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
    for (int a = lane; a < n; a += 32) w.flow[a] = 0;
    __syncwarp();
    int total = 0;
    while (total < target) {
        for (int v = lane; v < g.n_nodes; v += 32) w.parent[v] = -1;
        __syncwarp();
        if (lane == 0) w.parent[g.s] = -2;
        __syncwarp();
        bool reached = false;
        for (int sweep = 0; sweep <= g.n_nodes; ++sweep) {
            bool changed = false;
            for (int a = lane; a < n; a += 32) {
                const int u = s_src[a], v = s_dst[a];
                const int pu = ((volatile int32_t *)w.parent)[u], pv = ((volatile int32_t *)w.parent)[v];
                if (pu != -1 && pv == -1 && w.flow[a] < (int)w.x[a]) {
                    if (atomicCAS(&w.parent[v], -1, 2 * a) == -1) changed = true;
                } else if (pv != -1 && pu == -1 && w.flow[a] > 0) {
                    if (atomicCAS(&w.parent[u], -1, 2 * a + 1) == -1) changed = true;
                }
            }
            __syncwarp();
            if (((volatile int32_t *)w.parent)[g.t] != -1) {
                reached = true;
                break;
            }
            if (!__any_sync(0xffffffffu, changed)) break;
        }
        if (!reached) break;
        int push = 0;
        if (lane == 0) {
            int b = 0x7fffffff, v = g.t, guard = 0;
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
            v = g.t;
            guard = 0;
            while (b > 0 && v != g.s && guard++ <= g.n_nodes) {
                const int pa = w.parent[v], a = pa >> 1;
                w.flow[a] += (pa & 1) ? -b : b;
                v = (pa & 1) ? s_dst[a] : s_src[a];
            }
            push = b;
        }
        push = __shfl_sync(0xffffffffu, push, 0);
        __syncwarp();
        if (push <= 0) break;
        total += push;
    }
    return total < target;
}

__global__ void __launch_bounds__(kWarps * 32) resolve_kernel(const ClassifyParams p, const Sys g, uint8_t *labels,
                                                              int64_t *u_lower_idx, int64_t cap,
                                                              unsigned long long *counts2) {
    __shared__ WarpScratch ws[kWarps];
    __shared__ int32_t s_src[kMaxKenc], s_dst[kMaxKenc];
    __shared__ unsigned long long s_thr[kMaxKenc];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int32_t *err = &p.hdr->error;
    for (int i = tid; i < p.n; i += blockDim.x) {
        int u = g.src[i], v = g.dst[i];
        if (u < 0 || u >= g.n_nodes || v < 0 || v >= g.n_nodes) {
            atomicMax(err, 2);  // node index out of range: the edge is dropped
            u = v = 0;
        }
        s_src[i] = u;
        s_dst[i] = v;
    }
    for (int i = tid; i < p.n * p.km1; i += blockDim.x) s_thr[i] = p.thr[i];
    __syncthreads();
    WarpScratch &w = ws[warp];
    const uint32_t key0 = (uint32_t)p.seed, key1 = (uint32_t)(p.seed >> 32);
    const int64_t warps_total = (int64_t)gridDim.x * kWarps;
    for (int64_t base = ((int64_t)blockIdx.x * kWarps + warp) * 32; base < p.N; base += warps_total * 32) {
        const int64_t mine = base + lane;
        const bool unl = mine < p.N && labels[mine] == 2;
        unsigned todo = __ballot_sync(0xffffffffu, unl);
        while (todo) {
            const int src_lane = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t hl = base + src_lane;
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
            const bool lower = resolve_lower(g, p.n, w, s_src, s_dst, err);
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

}  // namespace

cudaError_t launch_resolve(const ClassifyParams &p, const rsr_system &sys, uint8_t *labels, int64_t *u_lower_idx,
                           int64_t cap, unsigned long long *counts2, cudaStream_t s) {
    if (p.N <= 0) return cudaSuccess;
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
    const int64_t warps = (p.N + 31) / 32;
    const int64_t grid = std::min<int64_t>((warps + kWarps - 1) / kWarps, (int64_t)device_sm_count() * 8);
    resolve_kernel<<<(unsigned)grid, kWarps * 32, 0, s>>>(p, g, labels, u_lower_idx, cap, counts2);
    return cudaGetLastError();
}

int resolve_max_nodes() { return kMaxNodes; }

}  // namespace rsr
