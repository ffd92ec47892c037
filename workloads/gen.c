/*
 * gen.c -- seeded generators of synthetic RSR inputs (systems and their
 * reference states).  Input generation only: no sampler, classifier,
 * estimator or gradient of the hot path lives here.
 *
 * Randomness: splitmix64 to seed, xoshiro256** to draw; every output item j
 * has its own stream seeded from (seed, j), so results do not depend on the
 * number of OpenMP threads.
 *
 * Contents
 *   wl_dnf_terms      random monotone DNF: R non-dominated terms (subsets)
 *   wl_greedy_cuts    minimal hitting sets of the DNF terms (greedy + prune)
 *   wl_st_boundary    s-t connectivity references by componentwise boundary
 *                     search from random states (Sec. 3.4)
 *   wl_flow_boundary  max-flow level references by the same search, K states
 *   wl_st_paths_cuts  random minimal s-t path sets and minimal s-t cuts
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ RNG */
typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64(uint64_t *x)
{
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void rng_seed(rng_t *r, uint64_t seed, uint64_t stream)
{
    uint64_t x = seed ^ (stream * 0xD1B54A32D192ED03ull);
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}

static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t rng_next(rng_t *r)
{
    uint64_t *s = r->s;
    uint64_t result = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = rotl(s[3], 45);
    return result;
}

static inline double rng_uniform(rng_t *r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }

static inline int64_t rng_below(rng_t *r, int64_t n) { return (int64_t)(rng_uniform(r) * (double)n); }

static void shuffle_int(rng_t *r, int *a, int n)
{
    for (int i = n - 1; i > 0; --i) {
        int j = (int)rng_below(r, i + 1);
        int t = a[i]; a[i] = a[j]; a[j] = t;
    }
}

/* -------------------------------------------------------- hashing / sets */
static uint64_t hash_bytes(const uint8_t *p, int n)
{
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < n; ++i) { h ^= p[i]; h *= 1099511628211ull; }
    return h ? h : 1;
}

typedef struct {
    uint64_t *keys;   /* 0 = empty */
    int64_t *rows;
    int64_t cap;
} hset_t;

static void hset_init(hset_t *h, int64_t expect)
{
    int64_t cap = 16;
    while (cap < expect * 2) cap <<= 1;
    h->cap = cap;
    h->keys = (uint64_t *)calloc((size_t)cap, sizeof(uint64_t));
    h->rows = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
}

static void hset_free(hset_t *h) { free(h->keys); free(h->rows); }

/* insert row (n bytes) if absent; rows stored in `store` (n bytes each) */
static int hset_insert(hset_t *h, const uint8_t *row, int n, uint8_t *store, int64_t *count)
{
    uint64_t k = hash_bytes(row, n);
    int64_t i = (int64_t)(k & (uint64_t)(h->cap - 1));
    while (h->keys[i]) {
        if (h->keys[i] == k && memcmp(store + (size_t)h->rows[i] * n, row, (size_t)n) == 0) return 0;
        i = (i + 1) & (h->cap - 1);
    }
    h->keys[i] = k;
    h->rows[i] = *count;
    memcpy(store + (size_t)(*count) * n, row, (size_t)n);
    *count += 1;
    return 1;
}

/* ================================================================ DNF terms */
/* Terms are subsets of {0..n-1} with size uniform in [lo, hi]; a term that is  */
/* a superset of another is dropped; draws continue until R remain.             */
/* out: R x n uint8, 1 on the term.                                             */
#define WMAX 16  /* n <= 1024 */

typedef struct { uint64_t w[WMAX]; } bits_t;

static int is_subset(const bits_t *a, const bits_t *b, int nw)
{
    for (int i = 0; i < nw; ++i) if (a->w[i] & ~b->w[i]) return 0;
    return 1;
}

int64_t wl_dnf_terms(int n, int64_t R, int lo, int hi, uint64_t seed, uint8_t *out)
{
    if (n > 64 * WMAX || lo < 2 || hi > n || lo > hi) return -1;
    const int nw = (n + 63) / 64;
    int64_t cap = R + R / 4 + 64;
    bits_t *T = (bits_t *)calloc((size_t)cap, sizeof(bits_t));
    int *size = (int *)calloc((size_t)cap, sizeof(int));
    int *first2 = (int *)calloc((size_t)cap * 2, sizeof(int));
    char *alive = (char *)calloc((size_t)cap, 1);
    int *perm = (int *)malloc(sizeof(int) * n);
    int64_t have = 0, drawn = 0;
    while (1) {
        /* draw until `have` candidates exist */
        int64_t start = have;
        while (have < R) {
            if (have >= cap) {  /* grow */
                int64_t nc = cap * 2;
                T = (bits_t *)realloc(T, (size_t)nc * sizeof(bits_t));
                size = (int *)realloc(size, (size_t)nc * sizeof(int));
                first2 = (int *)realloc(first2, (size_t)nc * 2 * sizeof(int));
                alive = (char *)realloc(alive, (size_t)nc);
                cap = nc;
            }
            rng_t r;
            rng_seed(&r, seed, (uint64_t)drawn++);
            int k = lo + (int)rng_below(&r, hi - lo + 1);
            for (int i = 0; i < n; ++i) perm[i] = i;
            /* partial Fisher-Yates: first k entries are a uniform k-subset */
            for (int i = 0; i < k; ++i) {
                int j = i + (int)rng_below(&r, n - i);
                int t = perm[i]; perm[i] = perm[j]; perm[j] = t;
            }
            memset(&T[have], 0, sizeof(bits_t));
            int m1 = n, m2 = n;
            for (int i = 0; i < k; ++i) {
                int e = perm[i];
                T[have].w[e >> 6] |= 1ull << (e & 63);
                if (e < m1) { m2 = m1; m1 = e; } else if (e < m2) m2 = e;
            }
            size[have] = k;
            first2[2 * have] = m1;
            first2[2 * have + 1] = m2;
            alive[have] = 1;
            ++have;
        }
        /* index terms by their two smallest elements */
        int64_t nkeys = (int64_t)n * n;
        int64_t *head = (int64_t *)malloc((size_t)(nkeys + 1) * sizeof(int64_t));
        int64_t *list = (int64_t *)malloc((size_t)have * sizeof(int64_t));
        memset(head, 0, (size_t)(nkeys + 1) * sizeof(int64_t));
        for (int64_t j = 0; j < have; ++j) head[(int64_t)first2[2 * j] * n + first2[2 * j + 1] + 1]++;
        for (int64_t q = 0; q < nkeys; ++q) head[q + 1] += head[q];
        int64_t *fill = (int64_t *)malloc((size_t)nkeys * sizeof(int64_t));
        memcpy(fill, head, (size_t)nkeys * sizeof(int64_t));
        for (int64_t j = 0; j < have; ++j) list[fill[(int64_t)first2[2 * j] * n + first2[2 * j + 1]]++] = j;
        free(fill);
        /* a term dies if some other term is a subset of it (ties: the later index dies) */
        char *dead = (char *)calloc((size_t)have, 1);
        #pragma omp parallel for schedule(dynamic, 256)
        for (int64_t j = 0; j < have; ++j) {
            int elems[64 * WMAX];
            int m = 0;
            for (int e = 0; e < n; ++e) if (T[j].w[e >> 6] >> (e & 63) & 1) elems[m++] = e;
            int found = 0;
            for (int a = 0; a < m && !found; ++a)
                for (int b = a + 1; b < m && !found; ++b) {
                    int64_t key = (int64_t)elems[a] * n + elems[b];
                    for (int64_t q = head[key]; q < head[key + 1]; ++q) {
                        int64_t o = list[q];
                        if (o == j || size[o] > size[j]) continue;
                        if (size[o] == size[j] && o > j) continue;  /* duplicate: keep the earlier */
                        if (is_subset(&T[o], &T[j], nw)) { found = 1; break; }
                    }
                }
            dead[j] = (char)found;
        }
        int64_t w = 0;
        for (int64_t j = 0; j < have; ++j) {
            if (dead[j]) continue;
            T[w] = T[j]; size[w] = size[j];
            first2[2 * w] = first2[2 * j]; first2[2 * w + 1] = first2[2 * j + 1];
            ++w;
        }
        free(dead); free(head); free(list);
        (void)start;
        if (w == have) break;   /* nothing removed: exactly R non-dominated terms */
        have = w;
    }
    for (int64_t j = 0; j < R; ++j)
        for (int e = 0; e < n; ++e) out[(size_t)j * n + e] = (uint8_t)(T[j].w[e >> 6] >> (e & 63) & 1);
    free(T); free(size); free(first2); free(alive); free(perm);
    return R;
}

/* ============================================================ greedy cuts */
/* A cut H hits every term.  Greedy: components in a random order are added   */
/* until every term is hit; then, in another random order, a component is     */
/* removed when every term it hits is hit by another member.  Output row =     */
/* 0 on the cut, 1 elsewhere (a maximal failed state).  Distinct cuts only.    */
int64_t wl_greedy_cuts(int n, int64_t R_terms, const uint8_t *terms, int64_t R_L, uint64_t seed,
                       int64_t max_draws, uint8_t *out)
{
    /* posting lists: component -> terms containing it */
    int64_t *phead = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t t = 0; t < R_terms; ++t)
        for (int e = 0; e < n; ++e) if (terms[(size_t)t * n + e]) phead[e + 1]++;
    for (int e = 0; e < n; ++e) phead[e + 1] += phead[e];
    int32_t *plist = (int32_t *)malloc((size_t)phead[n] * sizeof(int32_t));
    int64_t *pfill = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    memcpy(pfill, phead, (size_t)n * sizeof(int64_t));
    for (int64_t t = 0; t < R_terms; ++t)
        for (int e = 0; e < n; ++e) if (terms[(size_t)t * n + e]) plist[pfill[e]++] = (int32_t)t;
    free(pfill);

    hset_t hs;
    hset_init(&hs, R_L);
    int64_t count = 0, draw = 0;
    const int64_t batch = 1024;
    uint8_t *rows = (uint8_t *)malloc((size_t)batch * n);
    while (count < R_L && draw < max_draws) {
        int64_t nb = batch;
        if (draw + nb > max_draws) nb = max_draws - draw;
        #pragma omp parallel
        {
            uint8_t *cnt = (uint8_t *)malloc((size_t)R_terms);
            int *order = (int *)malloc(sizeof(int) * n);
            char *inH = (char *)malloc((size_t)n);
            #pragma omp for schedule(dynamic, 4)
            for (int64_t b = 0; b < nb; ++b) {
                rng_t r;
                rng_seed(&r, seed, (uint64_t)(draw + b));
                memset(cnt, 0, (size_t)R_terms);
                memset(inH, 0, (size_t)n);
                for (int i = 0; i < n; ++i) order[i] = i;
                shuffle_int(&r, order, n);
                int64_t hit = 0;
                for (int i = 0; i < n && hit < R_terms; ++i) {
                    int e = order[i];
                    inH[e] = 1;
                    for (int64_t q = phead[e]; q < phead[e + 1]; ++q) {
                        int32_t t = plist[q];
                        if (cnt[t] == 0) ++hit;
                        if (cnt[t] < 255) cnt[t]++;
                    }
                }
                shuffle_int(&r, order, n);
                for (int i = 0; i < n; ++i) {
                    int e = order[i];
                    if (!inH[e]) continue;
                    int needed = 0;
                    for (int64_t q = phead[e]; q < phead[e + 1]; ++q)
                        if (cnt[plist[q]] == 1) { needed = 1; break; }
                    if (needed) continue;
                    inH[e] = 0;
                    for (int64_t q = phead[e]; q < phead[e + 1]; ++q) cnt[plist[q]]--;
                }
                uint8_t *row = rows + (size_t)b * n;
                for (int e = 0; e < n; ++e) row[e] = inH[e] ? 0 : 1;
                if (hit < R_terms) row[0] = 2;  /* marker: terms left unhit (impossible for lo >= 1) */
            }
            free(cnt); free(order); free(inH);
        }
        for (int64_t b = 0; b < nb && count < R_L; ++b) {
            if (rows[(size_t)b * n] == 2) continue;
            hset_insert(&hs, rows + (size_t)b * n, n, out, &count);
        }
        draw += nb;
    }
    free(rows); free(phead); free(plist);
    hset_free(&hs);
    return count;
}

/* ====================================================== s-t connectivity */
typedef struct {
    int n_nodes, n_edges, s, t;
    const int32_t *eu, *ev;
    int32_t *adj_head, *adj_edge, *adj_to;   /* CSR over both directions */
} graph_t;

static void graph_build(graph_t *g, int n_nodes, int n_edges, const int32_t *eu, const int32_t *ev, int s, int t)
{
    g->n_nodes = n_nodes; g->n_edges = n_edges; g->s = s; g->t = t; g->eu = eu; g->ev = ev;
    g->adj_head = (int32_t *)calloc((size_t)n_nodes + 1, sizeof(int32_t));
    g->adj_edge = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)n_edges);
    g->adj_to = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)n_edges);
    for (int e = 0; e < n_edges; ++e) { g->adj_head[eu[e] + 1]++; g->adj_head[ev[e] + 1]++; }
    for (int v = 0; v < n_nodes; ++v) g->adj_head[v + 1] += g->adj_head[v];
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_nodes);
    memcpy(fill, g->adj_head, sizeof(int32_t) * (size_t)n_nodes);
    for (int e = 0; e < n_edges; ++e) {
        g->adj_edge[fill[eu[e]]] = e; g->adj_to[fill[eu[e]]++] = ev[e];
        g->adj_edge[fill[ev[e]]] = e; g->adj_to[fill[ev[e]]++] = eu[e];
    }
    free(fill);
}

static void graph_free(graph_t *g) { free(g->adj_head); free(g->adj_edge); free(g->adj_to); }

/* Phi(x) = 1 iff s reaches t over edges with x_e = 1 (undirected).  */
static int st_connected(const graph_t *g, const uint8_t *x, int32_t *stack, char *seen)
{
    memset(seen, 0, (size_t)g->n_nodes);
    int sp = 0;
    stack[sp++] = g->s;
    seen[g->s] = 1;
    while (sp) {
        int v = stack[--sp];
        if (v == g->t) return 1;
        for (int q = g->adj_head[v]; q < g->adj_head[v + 1]; ++q) {
            if (!x[g->adj_edge[q]]) continue;
            int w = g->adj_to[q];
            if (!seen[w]) { seen[w] = 1; stack[sp++] = w; }
        }
    }
    return 0;
}

/* Boundary search from random states (Sec. 3.4): Phi(x) = 1 -> decrement     */
/* components in index order, reverting a step that makes Phi = 0 (a minimal  */
/* path set, an upper reference); Phi(x) = 0 -> increment, reverting a step   */
/* that makes Phi = 1 (a maximal failed state, a lower reference).            */
/* Random states: x_e = 1 with probability 1 - pf[e].  Distinct refs only.     */
void wl_st_boundary(int n_nodes, int n_edges, const int32_t *eu, const int32_t *ev, int s, int t,
                    const double *pf, uint64_t seed, int64_t n_draws, int64_t max_L, int64_t max_U,
                    uint8_t *out_L, int64_t *nL, uint8_t *out_U, int64_t *nU)
{
    graph_t g;
    graph_build(&g, n_nodes, n_edges, eu, ev, s, t);
    const int n = n_edges;
    hset_t hL, hU;
    hset_init(&hL, max_L);
    hset_init(&hU, max_U);
    *nL = 0; *nU = 0;
    const int64_t batch = 4096;
    uint8_t *rows = (uint8_t *)malloc((size_t)batch * n);
    char *kind = (char *)malloc((size_t)batch);
    for (int64_t d0 = 0; d0 < n_draws && (*nL < max_L || *nU < max_U); d0 += batch) {
        int64_t nb = n_draws - d0 < batch ? n_draws - d0 : batch;
        #pragma omp parallel
        {
            int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_nodes);
            char *seen = (char *)malloc((size_t)n_nodes);
            #pragma omp for schedule(dynamic, 16)
            for (int64_t b = 0; b < nb; ++b) {
                rng_t r;
                rng_seed(&r, seed, (uint64_t)(d0 + b));
                uint8_t *x = rows + (size_t)b * n;
                for (int e = 0; e < n; ++e) x[e] = rng_uniform(&r) < pf[e] ? 0 : 1;
                int phi = st_connected(&g, x, stack, seen);
                kind[b] = (char)phi;
                for (int e = 0; e < n; ++e) {
                    if (phi && x[e]) {
                        x[e] = 0;
                        if (!st_connected(&g, x, stack, seen)) x[e] = 1;
                    } else if (!phi && !x[e]) {
                        x[e] = 1;
                        if (st_connected(&g, x, stack, seen)) x[e] = 0;
                    }
                }
            }
            free(stack); free(seen);
        }
        for (int64_t b = 0; b < nb; ++b) {
            if (kind[b] && *nU < max_U) hset_insert(&hU, rows + (size_t)b * n, n, out_U, nU);
            if (!kind[b] && *nL < max_L) hset_insert(&hL, rows + (size_t)b * n, n, out_L, nL);
        }
    }
    free(rows); free(kind);
    hset_free(&hL); hset_free(&hU);
    graph_free(&g);
}

/* ============================================================ max-flow */
/* Directed arcs a: u[a] -> v[a] with capacity x[a] (the component state).     */
/* Edmonds-Karp on the residual graph; small integer capacities.               */
typedef struct {
    int n_nodes, n_arcs, s, t;
    const int32_t *au, *av;
    int32_t *head, *nxt, *to;   /* residual arcs 2a (forward) and 2a+1 (backward) */
} fgraph_t;

static void fgraph_build(fgraph_t *g, int n_nodes, int n_arcs, const int32_t *au, const int32_t *av, int s, int t)
{
    g->n_nodes = n_nodes; g->n_arcs = n_arcs; g->s = s; g->t = t; g->au = au; g->av = av;
    g->head = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_nodes);
    g->nxt = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)n_arcs);
    g->to = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)n_arcs);
    for (int v = 0; v < n_nodes; ++v) g->head[v] = -1;
    for (int a = 0; a < n_arcs; ++a) {
        g->to[2 * a] = av[a]; g->nxt[2 * a] = g->head[au[a]]; g->head[au[a]] = 2 * a;
        g->to[2 * a + 1] = au[a]; g->nxt[2 * a + 1] = g->head[av[a]]; g->head[av[a]] = 2 * a + 1;
    }
}

static void fgraph_free(fgraph_t *g) { free(g->head); free(g->nxt); free(g->to); }

static int max_flow(const fgraph_t *g, const uint8_t *x, int32_t *cap, int32_t *prev, int32_t *queue)
{
    for (int a = 0; a < g->n_arcs; ++a) { cap[2 * a] = x[a]; cap[2 * a + 1] = 0; }
    int flow = 0;
    while (1) {
        for (int v = 0; v < g->n_nodes; ++v) prev[v] = -1;
        prev[g->s] = -2;
        int qh = 0, qt = 0;
        queue[qt++] = g->s;
        while (qh < qt && prev[g->t] == -1) {
            int v = queue[qh++];
            for (int e = g->head[v]; e >= 0; e = g->nxt[e]) {
                if (cap[e] > 0 && prev[g->to[e]] == -1) { prev[g->to[e]] = e; queue[qt++] = g->to[e]; }
            }
        }
        if (prev[g->t] == -1) break;
        int bott = 1 << 30;
        for (int v = g->t; v != g->s; v = g->to[prev[v] ^ 1]) if (cap[prev[v]] < bott) bott = cap[prev[v]];
        for (int v = g->t; v != g->s; v = g->to[prev[v] ^ 1]) { cap[prev[v]] -= bott; cap[prev[v] ^ 1] += bott; }
        flow += bott;
    }
    return flow;
}

static int flow_level(int f, int l1, int l2) { return f < l1 ? 0 : (f < l2 ? 1 : 2); }

/* System state S = level of the s-t max flow (thresholds l1 <= l2).  For the  */
/* threshold m': lower refs are maximal states with S <= m' (increment search), */
/* upper refs minimal states with S >= m'+1 (decrement search).  Random states  */
/* draw each arc state from pmf (n_arcs x K, rows sum to 1).                    */
void wl_flow_boundary(int n_nodes, int n_arcs, const int32_t *au, const int32_t *av, int s, int t, int K,
                      const double *pmf, int l1, int l2, int m_prime, uint64_t seed, int64_t n_draws,
                      int64_t max_L, int64_t max_U, uint8_t *out_L, int64_t *nL, uint8_t *out_U, int64_t *nU)
{
    fgraph_t g;
    fgraph_build(&g, n_nodes, n_arcs, au, av, s, t);
    const int n = n_arcs;
    hset_t hL, hU;
    hset_init(&hL, max_L);
    hset_init(&hU, max_U);
    *nL = 0; *nU = 0;
    const int64_t batch = 2048;
    uint8_t *rows = (uint8_t *)malloc((size_t)batch * n);
    char *kind = (char *)malloc((size_t)batch);
    for (int64_t d0 = 0; d0 < n_draws && (*nL < max_L || *nU < max_U); d0 += batch) {
        int64_t nb = n_draws - d0 < batch ? n_draws - d0 : batch;
        #pragma omp parallel
        {
            int32_t *cap = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)n_arcs);
            int32_t *prev = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_nodes);
            int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_nodes);
            #pragma omp for schedule(dynamic, 8)
            for (int64_t b = 0; b < nb; ++b) {
                rng_t r;
                rng_seed(&r, seed, (uint64_t)(d0 + b));
                uint8_t *x = rows + (size_t)b * n;
                for (int a = 0; a < n; ++a) {
                    double u = rng_uniform(&r), c = 0.0;
                    int k = 0;
                    for (; k < K - 1; ++k) { c += pmf[(size_t)a * K + k]; if (u < c) break; }
                    x[a] = (uint8_t)k;
                }
                int low = flow_level(max_flow(&g, x, cap, prev, queue), l1, l2) <= m_prime;
                kind[b] = (char)low;
                for (int a = 0; a < n; ++a) {
                    if (low) {
                        while (x[a] < K - 1) {
                            x[a]++;
                            if (flow_level(max_flow(&g, x, cap, prev, queue), l1, l2) > m_prime) { x[a]--; break; }
                        }
                    } else {
                        while (x[a] > 0) {
                            x[a]--;
                            if (flow_level(max_flow(&g, x, cap, prev, queue), l1, l2) <= m_prime) { x[a]++; break; }
                        }
                    }
                }
            }
            free(cap); free(prev); free(queue);
        }
        for (int64_t b = 0; b < nb; ++b) {
            if (kind[b] && *nL < max_L) hset_insert(&hL, rows + (size_t)b * n, n, out_L, nL);
            if (!kind[b] && *nU < max_U) hset_insert(&hU, rows + (size_t)b * n, n, out_U, nU);
        }
    }
    free(rows); free(kind);
    hset_free(&hL); hset_free(&hU);
    fgraph_free(&g);
}

/* Max-flow of every given state (n_states x n_arcs), for checks. */
void wl_flow_values(int n_nodes, int n_arcs, const int32_t *au, const int32_t *av, int s, int t,
                    int64_t n_states, const uint8_t *X, int32_t *flow)
{
    fgraph_t g;
    fgraph_build(&g, n_nodes, n_arcs, au, av, s, t);
    #pragma omp parallel
    {
        int32_t *cap = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)n_arcs);
        int32_t *prev = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_nodes);
        int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_nodes);
        #pragma omp for schedule(static)
        for (int64_t j = 0; j < n_states; ++j) flow[j] = max_flow(&g, X + (size_t)j * n_arcs, cap, prev, queue);
        free(cap); free(prev); free(queue);
    }
    fgraph_free(&g);
}

/* ======================================= random minimal s-t paths and cuts */
/* Paths: Dijkstra from s under random edge weights exp(U) (O(V^2), small     */
/* graphs); the path's edge set is a minimal path set.  Cuts: grow a random    */
/* node set S from s (random-weight Dijkstra order, t excluded) to a random    */
/* size, take T = component of t in G - S, and cut = edges between V - T and   */
/* T; both sides are connected, so the cut is minimal.                         */
void wl_st_paths_cuts(int n_nodes, int n_edges, const int32_t *eu, const int32_t *ev, int s, int t,
                      uint64_t seed, int64_t n_draws, int64_t max_L, int64_t max_U,
                      uint8_t *out_L, int64_t *nL, uint8_t *out_U, int64_t *nU)
{
    graph_t g;
    graph_build(&g, n_nodes, n_edges, eu, ev, s, t);
    const int n = n_edges;
    hset_t hL, hU;
    hset_init(&hL, max_L);
    hset_init(&hU, max_U);
    *nL = 0; *nU = 0;
    const int64_t batch = 8192;
    uint8_t *rows = (uint8_t *)malloc((size_t)batch * n);
    for (int64_t d0 = 0; d0 < n_draws && (*nL < max_L || *nU < max_U); d0 += batch) {
        int64_t nb = n_draws - d0 < batch ? n_draws - d0 : batch;
        #pragma omp parallel
        {
            double *w = (double *)malloc(sizeof(double) * (size_t)n);
            double *dist = (double *)malloc(sizeof(double) * (size_t)n_nodes);
            int32_t *pe = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_nodes);
            char *done = (char *)malloc((size_t)n_nodes);
            int32_t *orderv = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_nodes);
            char *inS = (char *)malloc((size_t)n_nodes);
            char *inT = (char *)malloc((size_t)n_nodes);
            int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_nodes);
            #pragma omp for schedule(dynamic, 64)
            for (int64_t b = 0; b < nb; ++b) {
                rng_t r;
                rng_seed(&r, seed, (uint64_t)(d0 + b));
                uint8_t *x = rows + (size_t)b * n;
                const int want_path = (int)((d0 + b) & 1);
                for (int e = 0; e < n; ++e) w[e] = exp(3.0 * rng_uniform(&r));
                for (int v = 0; v < n_nodes; ++v) { dist[v] = 1e300; pe[v] = -1; done[v] = 0; }
                dist[s] = 0.0;
                int nord = 0;
                for (int it = 0; it < n_nodes; ++it) {
                    int best = -1;
                    for (int v = 0; v < n_nodes; ++v)
                        if (!done[v] && dist[v] < 1e299 && (best < 0 || dist[v] < dist[best])) best = v;
                    if (best < 0) break;
                    done[best] = 1;
                    orderv[nord++] = best;
                    for (int q = g.adj_head[best]; q < g.adj_head[best + 1]; ++q) {
                        int e = g.adj_edge[q], u = g.adj_to[q];
                        if (!done[u] && dist[best] + w[e] < dist[u]) { dist[u] = dist[best] + w[e]; pe[u] = e; }
                    }
                }
                if (want_path) {
                    memset(x, 0, (size_t)n);
                    if (pe[t] < 0) { x[0] = 2; continue; }
                    for (int v = t; v != s;) {
                        int e = pe[v];
                        x[e] = 1;
                        v = (eu[e] == v) ? ev[e] : eu[e];
                    }
                } else {
                    /* S = first k nodes of the Dijkstra order without t */
                    int cand = 0;
                    for (int i = 0; i < nord; ++i) if (orderv[i] != t) ++cand;
                    int k = 1 + (int)rng_below(&r, cand > 1 ? cand : 1);
                    memset(inS, 0, (size_t)n_nodes);
                    for (int i = 0, taken = 0; i < nord && taken < k; ++i)
                        if (orderv[i] != t) { inS[orderv[i]] = 1; ++taken; }
                    /* T = component of t in G - S */
                    memset(inT, 0, (size_t)n_nodes);
                    int sp = 0;
                    stack[sp++] = t; inT[t] = 1;
                    while (sp) {
                        int v = stack[--sp];
                        for (int q = g.adj_head[v]; q < g.adj_head[v + 1]; ++q) {
                            int u = g.adj_to[q];
                            if (!inS[u] && !inT[u]) { inT[u] = 1; stack[sp++] = u; }
                        }
                    }
                    for (int e = 0; e < n; ++e) x[e] = (inT[eu[e]] != inT[ev[e]]) ? 0 : 1;
                }
            }
            free(w); free(dist); free(pe); free(done); free(orderv); free(inS); free(inT); free(stack);
        }
        for (int64_t b = 0; b < nb; ++b) {
            uint8_t *x = rows + (size_t)b * n;
            if (x[0] == 2) continue;
            if (((d0 + b) & 1) && *nU < max_U) hset_insert(&hU, x, n, out_U, nU);
            if (!((d0 + b) & 1) && *nL < max_L) hset_insert(&hL, x, n, out_L, nL);
        }
    }
    free(rows);
    hset_free(&hL); hset_free(&hU);
    graph_free(&g);
}
