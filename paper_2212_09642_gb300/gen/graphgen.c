/*
 * Seeded synthetic graph generators (input side only).
 *
 * These produce the undirected simple graphs whose Laplacians are the
 * density matrices rho = L / tr(L) of Section 2 (eq. graph_laplacian).  The
 * file holds none of the entropy method's arithmetic: it only draws edges
 * and assembles a symmetric CSR pattern (sorted columns, no self-loops, no
 * duplicate entries).  Both the CPU oracle and the GPU path consume its
 * output.
 *
 * Families (Section 6 uses SuiteSparse networks that are not available here;
 * these stand in for them):
 *   - Erdos-Renyi G(n, p): exact Bernoulli(p) per unordered pair, drawn by
 *     geometric skipping over the pair index (Batagelj & Brandes 2005).
 *   - Barabasi-Albert: seed clique on m+1 nodes, every new node attaches to
 *     m distinct earlier nodes chosen with probability proportional to their
 *     degree (sampling uniformly from the list of edge endpoints).
 *   - Watts-Strogatz: ring lattice with k/2 neighbours per side, each lattice
 *     edge rewired with probability beta to a uniform non-self target;
 *     duplicate edges created by rewiring are merged at CSR assembly.
 *   - Random geometric graph in the unit square with radius r, built with a
 *     cell grid of side >= r; node order is generation order (no locality).
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) as a stream
 * generator.  All floating point here is plain IEEE double without
 * contraction (compiled with -ffp-contract=off), so graphs are identical on
 * x86-64 and aarch64 hosts, except ER geometric skips which call log().
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct { uint64_t s; } rng_t;

static uint64_t rng_next(rng_t *r) {
    uint64_t z = (r->s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
/* uniform double in [0, 1) with 53 random bits */
static double rng_unif(rng_t *r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }
/* uniform integer in [0, bound) by 64x64->128 multiply-high (bias < 2^-64 * bound) */
static uint64_t rng_below(rng_t *r, uint64_t bound) {
    return (uint64_t)(((__uint128_t)rng_next(r) * (__uint128_t)bound) >> 64);
}

/* ------------------------------------------------------------------ */
/* Edge buffers grow geometrically.                                    */
typedef struct { int64_t *u, *v; int64_t len, cap; } edges_t;

static int edges_push(edges_t *e, int64_t a, int64_t b) {
    if (e->len == e->cap) {
        int64_t nc = e->cap ? e->cap * 2 : 1024;
        int64_t *nu = (int64_t *)realloc(e->u, (size_t)nc * sizeof(int64_t));
        if (!nu) return -1;
        e->u = nu;
        int64_t *nv = (int64_t *)realloc(e->v, (size_t)nc * sizeof(int64_t));
        if (!nv) return -1;
        e->v = nv;
        e->cap = nc;
    }
    e->u[e->len] = a; e->v[e->len] = b; e->len++;
    return 0;
}

void gg_free(void *p) { free(p); }

/* Erdos-Renyi G(n, p).  Unordered pairs (v, w), w < v, are enumerated by the
 * linear index k = v (v - 1) / 2 + w; the gaps between selected indices are
 * geometric with success probability p. */
int gg_erdos_renyi(int64_t n, double p, uint64_t seed, int64_t **eu, int64_t **ev, int64_t *ne) {
    rng_t r = {seed};
    edges_t e = {0};
    if (p <= 0.0 || n < 2) { *eu = NULL; *ev = NULL; *ne = 0; return 0; }
    const double lq = log(1.0 - p);
    int64_t v = 1, w = -1;
    for (;;) {
        double u = rng_unif(&r);
        int64_t skip = (p >= 1.0) ? 0 : (int64_t)floor(log(1.0 - u) / lq);
        w += 1 + skip;
        while (w >= v && v < n) { w -= v; v++; }
        if (v >= n) break;
        if (edges_push(&e, v, w)) return -1;
    }
    *eu = e.u; *ev = e.v; *ne = e.len;
    return 0;
}

/* Barabasi-Albert preferential attachment with m edges per new node. */
int gg_barabasi_albert(int64_t n, int64_t m, uint64_t seed, int64_t **eu, int64_t **ev, int64_t *ne) {
    rng_t r = {seed};
    edges_t e = {0};
    if (m < 1 || n < m + 1) return -2;
    int64_t max_end = 2 * ((m + 1) * m / 2 + (n - m - 1) * m);
    int64_t *ends = (int64_t *)malloc((size_t)max_end * sizeof(int64_t));
    int64_t *pick = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    if (!ends || !pick) { free(ends); free(pick); return -1; }
    int64_t nend = 0;
    for (int64_t a = 0; a <= m; a++)
        for (int64_t b = 0; b < a; b++) {
            if (edges_push(&e, a, b)) return -1;
            ends[nend++] = a; ends[nend++] = b;
        }
    for (int64_t t = m + 1; t < n; t++) {
        int64_t got = 0;
        while (got < m) {
            int64_t cand = ends[rng_below(&r, (uint64_t)nend)];
            int dup = 0;
            for (int64_t q = 0; q < got; q++) if (pick[q] == cand) { dup = 1; break; }
            if (!dup) pick[got++] = cand;
        }
        for (int64_t q = 0; q < m; q++) {
            if (edges_push(&e, t, pick[q])) return -1;
            ends[nend++] = t; ends[nend++] = pick[q];
        }
    }
    free(ends); free(pick);
    *eu = e.u; *ev = e.v; *ne = e.len;
    return 0;
}

/* Watts-Strogatz small world: ring lattice of degree k (even), rewiring prob beta. */
int gg_watts_strogatz(int64_t n, int64_t k, double beta, uint64_t seed, int64_t **eu, int64_t **ev, int64_t *ne) {
    rng_t r = {seed};
    edges_t e = {0};
    if (k < 2 || (k & 1) || n <= k) return -2;
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = 1; j <= k / 2; j++) {
            int64_t t = (i + j) % n;
            if (rng_unif(&r) < beta) {
                int64_t w;
                do { w = (int64_t)rng_below(&r, (uint64_t)n); } while (w == i);
                t = w;
            }
            if (edges_push(&e, i, t)) return -1;
        }
    *eu = e.u; *ev = e.v; *ne = e.len;
    return 0;
}

/* Random geometric graph: n uniform points in [0,1)^2, edge iff distance <= radius. */
int gg_random_geometric(int64_t n, double radius, uint64_t seed, int64_t **eu, int64_t **ev, int64_t *ne) {
    rng_t r = {seed};
    edges_t e = {0};
    double *x = (double *)malloc((size_t)n * sizeof(double));
    double *y = (double *)malloc((size_t)n * sizeof(double));
    if (!x || !y) { free(x); free(y); return -1; }
    for (int64_t i = 0; i < n; i++) { x[i] = rng_unif(&r); y[i] = rng_unif(&r); }
    int64_t g = (int64_t)floor(1.0 / radius);
    if (g < 1) g = 1;
    if (g > 65536) g = 65536;
    int64_t ncell = g * g;
    int64_t *head = (int64_t *)malloc((size_t)(ncell + 1) * sizeof(int64_t));
    int64_t *order = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *cellof = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!head || !order || !cellof) return -1;
    memset(head, 0, (size_t)(ncell + 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) {
        int64_t cx = (int64_t)(x[i] * (double)g), cy = (int64_t)(y[i] * (double)g);
        if (cx >= g) cx = g - 1;
        if (cy >= g) cy = g - 1;
        cellof[i] = cy * g + cx;
        head[cellof[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; c++) head[c + 1] += head[c];
    {
        int64_t *fill = (int64_t *)malloc((size_t)ncell * sizeof(int64_t));
        if (!fill) return -1;
        memcpy(fill, head, (size_t)ncell * sizeof(int64_t));
        for (int64_t i = 0; i < n; i++) order[fill[cellof[i]]++] = i;
        free(fill);
    }
    const double r2 = radius * radius;
    for (int64_t i = 0; i < n; i++) {
        int64_t cx = cellof[i] % g, cy = cellof[i] / g;
        for (int64_t dy = -1; dy <= 1; dy++)
            for (int64_t dx = -1; dx <= 1; dx++) {
                int64_t ax = cx + dx, ay = cy + dy;
                if (ax < 0 || ay < 0 || ax >= g || ay >= g) continue;
                int64_t c = ay * g + ax;
                for (int64_t q = head[c]; q < head[c + 1]; q++) {
                    int64_t j = order[q];
                    if (j >= i) continue;
                    double ddx = x[i] - x[j], ddy = y[i] - y[j];
                    double d2 = ddx * ddx + ddy * ddy;
                    if (d2 <= r2 && edges_push(&e, i, j)) return -1;
                }
            }
    }
    free(x); free(y); free(head); free(order); free(cellof);
    *eu = e.u; *ev = e.v; *ne = e.len;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Symmetric CSR assembly: both directions of every edge, self-loops
 * dropped, columns sorted ascending, duplicates merged.  rowptr has n+1
 * entries (int64), col has rowptr[n] entries (int32). */
static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

int gg_edges_to_csr(int64_t n, const int64_t *eu, const int64_t *ev, int64_t ne,
                    int64_t **rowptr_out, int32_t **col_out) {
    int64_t *rp = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
    if (!rp) return -1;
    for (int64_t q = 0; q < ne; q++) {
        int64_t a = eu[q], b = ev[q];
        if (a == b || a < 0 || b < 0 || a >= n || b >= n) continue;
        rp[a + 1]++; rp[b + 1]++;
    }
    for (int64_t i = 0; i < n; i++) rp[i + 1] += rp[i];
    int32_t *col = (int32_t *)malloc((size_t)(rp[n] > 0 ? rp[n] : 1) * sizeof(int32_t));
    int64_t *fill = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!col || !fill) { free(rp); free(col); free(fill); return -1; }
    memcpy(fill, rp, (size_t)n * sizeof(int64_t));
    for (int64_t q = 0; q < ne; q++) {
        int64_t a = eu[q], b = ev[q];
        if (a == b || a < 0 || b < 0 || a >= n || b >= n) continue;
        col[fill[a]++] = (int32_t)b;
        col[fill[b]++] = (int32_t)a;
    }
    /* sort each row, merge duplicates, compact in place */
    int64_t w = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t lo = rp[i], hi = rp[i + 1];
        int64_t len = hi - lo;
        if (len > 1) {
            if (len <= 16) {
                for (int64_t a = lo + 1; a < hi; a++) {
                    int32_t key = col[a];
                    int64_t b = a - 1;
                    while (b >= lo && col[b] > key) { col[b + 1] = col[b]; b--; }
                    col[b + 1] = key;
                }
            } else {
                qsort(col + lo, (size_t)len, sizeof(int32_t), cmp_i32);
            }
        }
        int64_t start = w;
        for (int64_t a = lo; a < hi; a++)
            if (w == start || col[w - 1] != col[a]) col[w++] = col[a];
        rp[i] = start;
    }
    rp[n] = w;
    free(fill);
    *rowptr_out = rp;
    *col_out = col;
    return 0;
}
