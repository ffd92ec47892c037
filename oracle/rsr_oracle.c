/*
 * rsr_oracle.c -- plain, slow, obviously correct CPU oracle for the RSR hot path
 * (Reference-state System Reliability, arXiv 2604.17066).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may load, call or link
 * this file: only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference legs of bench.py use it.  It shares no code, header, table or
 * constant generator with the CUDA library in paper_2604_17066_gb300/csrc.
 *
 * Every loop follows the definition it cites, one sample and one reference at a
 * time, with no blocking, encoding or reordering.  Floating point is IEEE fp64.
 *
 * Definitions followed (paper section / equation):
 *   - problem setting, componentwise order, coherence: Sec. 2.1-2.2, Eq. (1)
 *   - lower / upper reference sets L(m'), U(m'): Sec. 2.2, Eqs. (2)-(3)
 *   - classification into I^L, I^U, I^u, lower taking precedence: Sec. 3.3,
 *     the p^L / p^U / p^u definitions and Algorithm 1
 *   - count estimators p_hat = |I|/H and c.o.v. sqrt((1-p)/(H p)): Sec. 3.3
 *   - Stage 2 estimate of P(S <= m') after resolving I^u with Phi: Sec. 3.5
 *   - componentwise boundary search for new reference states: Sec. 3.4
 *   - non-dominated reference sets: Sec. 2.2, Eqs. (2)-(3)
 *   - system functions of the experiments: s-t connectivity (Sec. 4.1-4.2),
 *     global connectivity (Sec. 4.3), s-t maximum-flow levels (d-MC / d-MP
 *     systems, Sec. 2.2) and the three-state global connectivity level (Sec. 4.6)
 * Not in the paper (defined by this library, see the function comments):
 *   - the sampler (Philox4x32-10 counter layout and integer inverse-CDF
 *     thresholds); the paper only states that P(X) is available (Sec. 3.1)
 *   - the score-function gradient of P(S <= m') with respect to the
 *     component-state probabilities q_{i,k}
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11).  Ten rounds; each round multiplies counter      */
/* words 0 and 2 by the two Philox-4x32 multipliers, takes the 64-bit        */
/* products apart into high and low halves, xors the high halves with the    */
/* other two counter words and the round key, and permutes the words.  The   */
/* key is bumped by the two Weyl constants between rounds.                   */
/* ------------------------------------------------------------------------ */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += ORC_PHILOX_W0;
            k1 += ORC_PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* Sampler thresholds (not in the paper; Sec. 3.1 only assumes P(X) can be    */
/* sampled).  For component i with pmf q_{i,0..K-1}:                         */
/*   c_{i,k} = q_{i,0} + ... + q_{i,k-1}   (fp64, summed left to right)       */
/*   T_{i,k} = min(2^32, floor(2^32 * c_{i,k}))     for k = 1..K-1            */
/* stored row-major as T[i*(K-1) + (k-1)].                                    */
/* ------------------------------------------------------------------------ */
void orc_thresholds(int32_t n, int32_t K, const double *pmf, uint64_t *T)
{
    for (int32_t i = 0; i < n; ++i) {
        double c = 0.0;
        for (int32_t k = 1; k < K; ++k) {
            c = c + pmf[(size_t)i * K + (k - 1)];
            double scaled = floor(ldexp(c, 32));
            uint64_t t;
            if (scaled <= 0.0)
                t = 0;
            else if (scaled >= 4294967296.0)
                t = 4294967296ull;
            else
                t = (uint64_t)scaled;
            T[(size_t)i * (K - 1) + (k - 1)] = t;
        }
    }
}

/* State of one component from one uniform 32-bit word u:                     */
/*   x = #{ k in 1..K-1 : u >= T_{i,k} }                                      */
int32_t orc_state_from_uniform(uint32_t u, int32_t K, const uint64_t *T_row)
{
    int32_t x = 0;
    for (int32_t k = 1; k < K; ++k)
        if ((uint64_t)u >= T_row[k - 1])
            x = x + 1;
    return x;
}

/* Sample h (global index = offset + local index), component i:               */
/*   u_{h,i} = word (i mod 4) of Philox4x32-10(                                */
/*               key = (seed mod 2^32, seed div 2^32),                         */
/*               ctr = (h mod 2^32, h div 2^32, floor(i/4), 0))                */
/* X is N x n row-major uint8.                                                 */
void orc_sample(int32_t n, int32_t K, const uint64_t *T, uint64_t seed, uint64_t offset,
                int64_t N, uint8_t *X)
{
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    for (int64_t s = 0; s < N; ++s) {
        uint64_t h = offset + (uint64_t)s;
        for (int32_t i = 0; i < n; ++i) {
            uint32_t ctr[4] = {(uint32_t)(h & 0xffffffffu), (uint32_t)(h >> 32),
                               (uint32_t)(i / 4), 0u};
            uint32_t words[4];
            orc_philox4x32_10(ctr, key, words);
            uint32_t u = words[i % 4];
            X[(size_t)s * n + i] = (uint8_t)orc_state_from_uniform(u, K, T + (size_t)i * (K - 1));
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Componentwise order (Eq. (1)): x <= r  iff  x_i <= r_i for every i.        */
/* ------------------------------------------------------------------------ */
static int orc_leq(int32_t n, const uint8_t *x, const uint8_t *r)
{
    for (int32_t i = 0; i < n; ++i)
        if (x[i] > r[i])
            return 0;
    return 1;
}

/* Classification (Sec. 3.3, Algorithm 1).  Sample h is in I^L if some lower  */
/* reference r satisfies x_h <= r; otherwise in I^U if some upper reference r  */
/* satisfies r <= x_h; otherwise in I^u.  Lower takes precedence.              */
/* labels: 0 = I^L (S <= m'), 1 = I^U (S >= m'+1), 2 = I^u (unclassified).     */
/* counts3 receives |I^L|, |I^U|, |I^u|.                                       */
void orc_classify(int32_t n, int64_t N, const uint8_t *X,
                  int64_t R_L, const uint8_t *ref_L,
                  int64_t R_U, const uint8_t *ref_U,
                  uint8_t *labels, int64_t *counts3)
{
    counts3[0] = 0; counts3[1] = 0; counts3[2] = 0;
    for (int64_t h = 0; h < N; ++h) {
        const uint8_t *x = X + (size_t)h * n;
        int label = 2;
        for (int64_t r = 0; r < R_L && label == 2; ++r)
            if (orc_leq(n, x, ref_L + (size_t)r * n))
                label = 0;
        for (int64_t r = 0; r < R_U && label == 2; ++r)
            if (orc_leq(n, ref_U + (size_t)r * n, x))
                label = 1;
        labels[h] = (uint8_t)label;
        counts3[label] += 1;
    }
}

/* ------------------------------------------------------------------------ */
/* Estimates (Sec. 3.3 count estimators and c.o.v.; Sec. 3.5 Stage 2).        */
/*   p_hat^L = c_L/H, p_hat^U = c_U/H, p_hat^u = c_u/H                         */
/*   P_hat(S <= m') = (c_L + n_u_lower)/H, where n_u_lower is the number of    */
/*   unclassified samples that Phi resolved to S <= m' (0 before Stage 2)      */
/*   P_hat(S >= m'+1) = (c_U + (c_u - n_u_lower))/H                            */
/*   delta_hat(p) = sqrt((1 - p)/(H p)); +inf at p = 0 (IEEE division).         */
/* out: [pL, pU, pu, P_lower, P_upper, cov_pL, cov_pU, cov_pu, cov_lower,     */
/*       cov_upper]                                                            */
/* ------------------------------------------------------------------------ */
static double orc_cov(double p, double H)
{
    return sqrt((1.0 - p) / (H * p));
}

void orc_estimate(const int64_t counts3[3], int64_t N, int64_t n_u_lower, double *out)
{
    double H = (double)N;
    double pL = (double)counts3[0] / H;
    double pU = (double)counts3[1] / H;
    double pu = (double)counts3[2] / H;
    double P_lower = (double)(counts3[0] + n_u_lower) / H;
    double P_upper = (double)(counts3[1] + (counts3[2] - n_u_lower)) / H;
    out[0] = pL;
    out[1] = pU;
    out[2] = pu;
    out[3] = P_lower;
    out[4] = P_upper;
    out[5] = orc_cov(pL, H);
    out[6] = orc_cov(pU, H);
    out[7] = orc_cov(pu, H);
    out[8] = orc_cov(P_lower, H);
    out[9] = orc_cov(P_upper, H);
}

/* ------------------------------------------------------------------------ */
/* Score-function gradient (not in the paper).  With independent components,  */
/*   P(F) = sum_x 1_F(x) prod_j q_{j,x_j}                                      */
/* is multilinear in the q's, and its unconstrained partial derivative is      */
/*   dP(F)/dq_{i,k} = E[ 1_F(X) 1{X_i = k} ] / q_{i,k} = P(F | X_i = k).        */
/* F is the event S <= m' (samples labelled I^L plus the unclassified samples  */
/* that Phi resolved to S <= m').                                              */
/*                                                                             */
/* orc_grad_counts: C[i*K + k] = #{ h in F : x_{h,i} = k }, F given by labels  */
/* (label 0) plus the listed unclassified indices.                             */
/* ------------------------------------------------------------------------ */
void orc_grad_counts(int32_t n, int32_t K, int64_t N, const uint8_t *X, const uint8_t *labels,
                     const int64_t *u_lower_idx, int64_t n_u_lower, int64_t *C)
{
    for (int64_t j = 0; j < (int64_t)n * K; ++j)
        C[j] = 0;
    for (int64_t h = 0; h < N; ++h) {
        if (labels[h] != 0)
            continue;
        for (int32_t i = 0; i < n; ++i)
            C[(size_t)i * K + X[(size_t)h * n + i]] += 1;
    }
    for (int64_t j = 0; j < n_u_lower; ++j) {
        int64_t h = u_lower_idx[j];
        for (int32_t i = 0; i < n; ++i)
            C[(size_t)i * K + X[(size_t)h * n + i]] += 1;
    }
}

/* Estimator g_hat_{i,k} = (C_{i,k}/H) / q_{i,k}.  Each sample contributes     */
/* Y = 1_F 1{x_i = k} / q_{i,k}, a Bernoulli(p) variable scaled by 1/q with     */
/* p = C/H, so its standard error is sqrt(p (1 - p) / H) / q.  q = 0 gives      */
/* IEEE results (0/0 = NaN).                                                   */
void orc_grad(int32_t n, int32_t K, int64_t N, const int64_t *C, const double *pmf,
              double *g, double *se)
{
    double H = (double)N;
    for (int64_t j = 0; j < (int64_t)n * K; ++j) {
        double p = (double)C[j] / H;
        double q = pmf[j];
        g[j] = p / q;
        se[j] = sqrt(p * (1.0 - p) / H) / q;
    }
}

/* Consistency of a reference pair (Sec. 3.3, note on precedence): the label   */
/* sets can overlap only if some upper reference r^U lies below some lower     */
/* reference r^L (r^U <= r^L); a sample between them satisfies both.  Returns  */
/* the number of such (r^L, r^U) pairs.                                        */
int64_t orc_count_overlaps(int32_t n, int64_t R_L, const uint8_t *ref_L,
                           int64_t R_U, const uint8_t *ref_U)
{
    int64_t c = 0;
    for (int64_t a = 0; a < R_L; ++a)
        for (int64_t b = 0; b < R_U; ++b)
            if (orc_leq(n, ref_U + (size_t)b * n, ref_L + (size_t)a * n))
                c += 1;
    return c;
}

/* ------------------------------------------------------------------------ */
/* Stage 2 (Sec. 3.5): the system function Phi is evaluated for the          */
/* unclassified samples, and P(S <= m') is estimated from |I^L| plus the      */
/* unclassified samples with Phi <= m'.  Two system functions of the paper's  */
/* experiments:                                                               */
/*   kind 0, s-t connectivity (Sec. 2.2 example, Sec. 4.1): component e is an */
/*     undirected edge (src[e], dst[e]) that works when x_e = 1;              */
/*     Phi = 1 if s reaches t over working edges, else 0;                     */
/*   kind 1, s-t maximum flow (Sec. 2.2, d-MC/d-MP systems): component a is a */
/*     directed arc src[a] -> dst[a] with capacity x_a; f = max flow s -> t;  */
/*     Phi = #{ l : f >= thr[l] } for the level thresholds thr[0..L-1].       */
/* Labels 2 are rewritten to 3 (Phi <= m') or 4 (Phi >= m'+1); the function   */
/* returns the number of 3s.                                                  */
/* ------------------------------------------------------------------------ */
static int orc_st_connected(int n_nodes, int n_edges, const int32_t *src, const int32_t *dst, int s, int t,
                            const uint8_t *x, int32_t *queue, uint8_t *seen)
{
    for (int v = 0; v < n_nodes; ++v) seen[v] = 0;
    int head = 0, tail = 0;
    queue[tail++] = s;
    seen[s] = 1;
    while (head < tail) {
        int v = queue[head++];
        if (v == t) return 1;
        for (int e = 0; e < n_edges; ++e) {
            if (!x[e]) continue;
            int w = -1;
            if (src[e] == v) w = dst[e];
            else if (dst[e] == v) w = src[e];
            if (w >= 0 && !seen[w]) {
                seen[w] = 1;
                queue[tail++] = w;
            }
        }
    }
    return 0;
}

/* Ford-Fulkerson with breadth-first augmenting paths (Edmonds-Karp). */
static int orc_max_flow(int n_nodes, int n_arcs, const int32_t *src, const int32_t *dst, int s, int t,
                        const uint8_t *cap, int32_t *flow, int32_t *queue, int32_t *parent_arc, int8_t *parent_dir)
{
    for (int a = 0; a < n_arcs; ++a) flow[a] = 0;
    int total = 0;
    while (1) {
        for (int v = 0; v < n_nodes; ++v) parent_arc[v] = -2;
        parent_arc[s] = -1;
        int head = 0, tail = 0;
        queue[tail++] = s;
        while (head < tail && parent_arc[t] == -2) {
            int v = queue[head++];
            for (int a = 0; a < n_arcs; ++a) {
                if (src[a] == v && parent_arc[dst[a]] == -2 && flow[a] < cap[a]) {
                    parent_arc[dst[a]] = a;
                    parent_dir[dst[a]] = 1;
                    queue[tail++] = dst[a];
                } else if (dst[a] == v && parent_arc[src[a]] == -2 && flow[a] > 0) {
                    parent_arc[src[a]] = a;
                    parent_dir[src[a]] = -1;
                    queue[tail++] = src[a];
                }
            }
        }
        if (parent_arc[t] == -2) break;
        int bottleneck = 1 << 30;
        for (int v = t; v != s;) {
            int a = parent_arc[v];
            int r = parent_dir[v] > 0 ? cap[a] - flow[a] : flow[a];
            if (r < bottleneck) bottleneck = r;
            v = parent_dir[v] > 0 ? src[a] : dst[a];
        }
        for (int v = t; v != s;) {
            int a = parent_arc[v];
            flow[a] += parent_dir[v] > 0 ? bottleneck : -bottleneck;
            v = parent_dir[v] > 0 ? src[a] : dst[a];
        }
        total += bottleneck;
    }
    return total;
}

/* Number of nodes reached from node 0 over working edges, edge `skip` left out
 * (skip = -1: none).  Breadth-first search over the undirected edge list. */
static int orc_reached_from_0(int n_nodes, int n_edges, const int32_t *src, const int32_t *dst,
                              const uint8_t *x, int skip, int32_t *queue, uint8_t *seen)
{
    for (int v = 0; v < n_nodes; ++v) seen[v] = 0;
    int head = 0, tail = 0;
    queue[tail++] = 0;
    seen[0] = 1;
    while (head < tail) {
        int v = queue[head++];
        for (int e = 0; e < n_edges; ++e) {
            if (!x[e] || e == skip) continue;
            int w = -1;
            if (src[e] == v) w = dst[e];
            else if (dst[e] == v) w = src[e];
            if (w >= 0 && !seen[w]) {
                seen[w] = 1;
                queue[tail++] = w;
            }
        }
    }
    return tail;
}

/* Further system functions (binary components = undirected edges):
 *   kind 2, global connectivity (Sec. 4.3): Phi = 1 if every node is
 *     connected to every other over working edges, else 0;
 *   kind 3, global connectivity level (Sec. 4.6): Phi = 0 if disconnected,
 *     1 if connected but some pair of nodes has only one edge-disjoint path,
 *     2 if every pair has two or more.  By Menger's theorem the last case is
 *     "no single working edge disconnects the graph", which is tested here by
 *     removing each working edge in turn. */
int orc_phi(int kind, int n_nodes, int n, const int32_t *src, const int32_t *dst, int s, int t,
            int n_thr, const int32_t *thr, const uint8_t *x)
{
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_nodes + n + 1));
    uint8_t *seen = (uint8_t *)malloc((size_t)n_nodes + 1);
    int32_t *flow = (int32_t *)malloc(sizeof(int32_t) * (size_t)n + 4);
    int32_t *parent_arc = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_nodes + 4);
    int8_t *parent_dir = (int8_t *)malloc((size_t)n_nodes + 4);
    int phi;
    if (kind == 0) {
        phi = orc_st_connected(n_nodes, n, src, dst, s, t, x, queue, seen);
    } else if (kind == 1) {
        int f = orc_max_flow(n_nodes, n, src, dst, s, t, x, flow, queue, parent_arc, parent_dir);
        phi = 0;
        for (int l = 0; l < n_thr; ++l)
            if (f >= thr[l]) phi += 1;
    } else {
        phi = orc_reached_from_0(n_nodes, n, src, dst, x, -1, queue, seen) == n_nodes ? 1 : 0;
        if (kind == 3 && phi == 1) {
            phi = 2;
            for (int e = 0; e < n && phi == 2; ++e)
                if (x[e] && orc_reached_from_0(n_nodes, n, src, dst, x, e, queue, seen) < n_nodes) phi = 1;
        }
    }
    free(queue); free(seen); free(flow); free(parent_arc); free(parent_dir);
    return phi;
}

int64_t orc_resolve(int kind, int n_nodes, int n, const int32_t *src, const int32_t *dst, int s, int t,
                    int n_thr, const int32_t *thr, int m_prime, int64_t N, const uint8_t *X, uint8_t *labels)
{
    int64_t lower = 0;
    for (int64_t h = 0; h < N; ++h) {
        if (labels[h] != 2) continue;
        int phi = orc_phi(kind, n_nodes, n, src, dst, s, t, n_thr, thr, X + (size_t)h * n);
        if (phi <= m_prime) {
            labels[h] = 3;
            lower += 1;
        } else {
            labels[h] = 4;
        }
    }
    return lower;
}

/* ------------------------------------------------------------------------ */
/* Componentwise boundary search (Sec. 3.4).  From a state x with           */
/* Phi(x) <= m', the components are visited in index order; each is raised  */
/* one state at a time, Phi re-evaluated after every step, until it reaches */
/* the top state K-1 or the step makes Phi > m', in which case that step is */
/* undone and the next component is visited.  A state with Phi(x) >= m'+1  */
/* is lowered in the same way.  The final state is a lower (side 0) or      */
/* upper (side 1) boundary reference state.  *phi_evals receives the number */
/* of Phi evaluations, the first one included.                              */
/* ------------------------------------------------------------------------ */
/* Visiting order of the permuted search (not in the paper, which visits in   */
/* index order): a Fisher-Yates shuffle of 0..n-1 driven by Philox4x32-10    */
/* with key = seed and counter (h lo, h hi, floor(i/4), 1) -- counter word 3  */
/* = 1 keeps it apart from the sampler's words (word 3 = 0).  For i = n-1    */
/* down to 1: u = word (i mod 4) of block floor(i/4), j = (u * (i+1)) >> 32  */
/* (an exact integer multiply-shift), swap order[i] and order[j].            */
void orc_search_order(uint64_t seed, uint64_t h, int n, int32_t *order)
{
    for (int i = 0; i < n; ++i) order[i] = i;
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int i = n - 1; i >= 1; --i) {
        const uint32_t ctr[4] = {(uint32_t)h, (uint32_t)(h >> 32), (uint32_t)(i / 4), 1u};
        uint32_t words[4];
        orc_philox4x32_10(ctr, key, words);
        const uint32_t u = words[i % 4];
        const int j = (int)(((uint64_t)u * (uint64_t)(i + 1)) >> 32);
        const int32_t tmp = order[i];
        order[i] = order[j];
        order[j] = tmp;
    }
}

/* order = NULL: index order 0..n-1 (Sec. 3.4); otherwise the components are
 * visited as order[0], order[1], ... */
int orc_boundary_search(int kind, int n_nodes, int n, const int32_t *src, const int32_t *dst, int s, int t,
                        int n_thr, const int32_t *thr, int m_prime, int K, const uint8_t *x_in, uint8_t *x_out,
                        int64_t *phi_evals, const int32_t *order)
{
    int64_t evals = 0;
    for (int i = 0; i < n; ++i) x_out[i] = x_in[i];
    const int lower = orc_phi(kind, n_nodes, n, src, dst, s, t, n_thr, thr, x_out) <= m_prime;
    evals += 1;
    for (int step = 0; step < n; ++step) {
        const int i = order ? order[step] : step;
        if (lower) {
            while (x_out[i] < K - 1) {
                x_out[i] += 1;
                evals += 1;
                if (orc_phi(kind, n_nodes, n, src, dst, s, t, n_thr, thr, x_out) > m_prime) {
                    x_out[i] -= 1;
                    break;
                }
            }
        } else {
            while (x_out[i] > 0) {
                x_out[i] -= 1;
                evals += 1;
                if (orc_phi(kind, n_nodes, n, src, dst, s, t, n_thr, thr, x_out) <= m_prime) {
                    x_out[i] += 1;
                    break;
                }
            }
        }
    }
    if (phi_evals) *phi_evals = evals;
    return lower ? 0 : 1;
}

/* ------------------------------------------------------------------------ */
/* Non-dominated references (Sec. 2.2, Eqs. (2)-(3)).  A lower reference    */
/* r_j is redundant when another lower reference r_i satisfies r_j <= r_i   */
/* componentwise; an upper reference r_j when another upper reference r_i   */
/* satisfies r_j >= r_i.  Of identical references only the first (lowest    */
/* index) is kept.  keep[j] = 1 for the references that remain.             */
/* ------------------------------------------------------------------------ */
void orc_nondominated(int n, int64_t R, const uint8_t *refs, int upper, uint8_t *keep)
{
    for (int64_t j = 0; j < R; ++j) {
        const uint8_t *rj = refs + (size_t)j * n;
        keep[j] = 1;
        for (int64_t i = 0; i < R && keep[j]; ++i) {
            if (i == j) continue;
            const uint8_t *ri = refs + (size_t)i * n;
            int dominated = 1, equal = 1;
            for (int k = 0; k < n; ++k) {
                if (upper ? (rj[k] < ri[k]) : (rj[k] > ri[k])) dominated = 0;
                if (rj[k] != ri[k]) equal = 0;
            }
            if (dominated && (!equal || i < j)) keep[j] = 0;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* System-state pmf over all levels (Sec. 3.5 applied at every boundary,    */
/* Sec. 4.5-4.6): P(S = m) is estimated by #{h : Phi(x_h) = m} / H.  The    */
/* oracle takes the definition directly: Phi of every sample.               */
/* ------------------------------------------------------------------------ */
void orc_levels(int kind, int n_nodes, int n, const int32_t *src, const int32_t *dst, int s, int t, int n_thr,
                const int32_t *thr, int64_t N, const uint8_t *X, uint8_t *levels)
{
    for (int64_t h = 0; h < N; ++h)
        levels[h] = (uint8_t)orc_phi(kind, n_nodes, n, src, dst, s, t, n_thr, thr, X + (size_t)h * n);
}
