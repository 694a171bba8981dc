/*
 * Seeded synthetic graph generators and the CSR builder.
 *
 * This file produces INPUTS only: undirected graphs in CSR form and source
 * lists.  It holds none of the betweenness-centrality arithmetic, so both the
 * CUDA library and the CPU oracle may consume what it writes.
 *
 * Graph conventions (Sec. VI, "directed graphs were converted to undirected"):
 * every graph is returned symmetric, with no self-loops, no duplicate entries
 * and rows sorted ascending; row_ptr and col are int32 (nnz < 2^31).
 *
 * Randomness: one counter-based generator, SplitMix64 (Steele, Lea, Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014): value i of
 * stream (seed, id) is the SplitMix64 output mixer applied to
 * key + (i + 1) * 0x9E3779B97F4A7C15.  Only integer arithmetic is used, so the
 * same seed gives the same bytes on x86-64 and AArch64.
 *
 * Memory returned in gg_csr / gg_i32 is malloc'd here; release with gg_free_*.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GG_GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Key of stream `id` under `seed`. */
static inline uint64_t gg_key(uint64_t seed, uint64_t id) {
    return sm64_mix(sm64_mix(seed + GG_GOLDEN) ^ (id * 0xD1B54A32D192ED03ULL + 1));
}

static inline uint64_t gg_at(uint64_t key, uint64_t i) {
    return sm64_mix(key + (i + 1) * GG_GOLDEN);
}

uint64_t gg_rng(uint64_t seed, uint64_t id, uint64_t i) { return gg_at(gg_key(seed, id), i); }

/* Uniform integer in [0, range) by the multiply-high method (Lemire 2019,
 * without the rejection step: bias below range / 2^64). */
static inline uint64_t gg_bounded(uint64_t r, uint64_t range) {
    return (uint64_t)(((__uint128_t)r * (__uint128_t)range) >> 64);
}

enum { ST_ER = 1, ST_RMAT = 2, ST_PERM = 3, ST_GRID = 4, ST_SRC = 5, ST_TRI = 6, ST_RGG = 7, ST_WEIGHT = 8 };

typedef struct {
    int32_t n;
    int64_t nnz;
    int32_t *row_ptr; /* n + 1 */
    int32_t *col;     /* nnz */
} gg_csr;

void gg_free_csr(gg_csr *g) {
    if (!g) return;
    free(g->row_ptr);
    free(g->col);
    g->row_ptr = NULL;
    g->col = NULL;
}
void gg_free_ptr(void *p) { free(p); }

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Edge list -> symmetric, sorted, deduplicated, loop-free CSR.
 * Returns 0, or -1 on a bad vertex id / allocation failure / nnz >= 2^31. */
int gg_from_edges(int32_t n, int64_t m, const int32_t *u, const int32_t *v, gg_csr *out) {
    memset(out, 0, sizeof(*out));
    if (n < 0 || m < 0) return -1;
    int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!deg) return -1;
    for (int64_t e = 0; e < m; ++e) {
        int32_t a = u[e], b = v[e];
        if (a < 0 || b < 0 || a >= n || b >= n) { free(deg); return -1; }
        if (a == b) continue;
        deg[a]++;
        deg[b]++;
    }
    int64_t *off = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!off) { free(deg); return -1; }
    off[0] = 0;
    for (int32_t i = 0; i < n; ++i) off[i + 1] = off[i] + deg[i];
    int64_t total = off[n];
    int32_t *tmp = (int32_t *)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
    if (!tmp) { free(deg); free(off); return -1; }
    memset(deg, 0, ((size_t)n + 1) * sizeof(int64_t));
    for (int64_t e = 0; e < m; ++e) {
        int32_t a = u[e], b = v[e];
        if (a == b) continue;
        tmp[off[a] + deg[a]++] = b;
        tmp[off[b] + deg[b]++] = a;
    }
    /* sort + dedup each row in place, recording the kept length in deg[] */
    int64_t nnz = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t *row = tmp + off[i];
        int64_t len = deg[i];
        if (len > 1) qsort(row, (size_t)len, sizeof(int32_t), cmp_i32);
        int64_t k = 0;
        for (int64_t j = 0; j < len; ++j)
            if (k == 0 || row[j] != row[k - 1]) row[k++] = row[j];
        deg[i] = k;
        nnz += k;
    }
    if (nnz >= ((int64_t)1 << 31)) { free(deg); free(off); free(tmp); return -1; }
    out->n = n;
    out->nnz = nnz;
    out->row_ptr = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    out->col = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    if (!out->row_ptr || !out->col) { gg_free_csr(out); free(deg); free(off); free(tmp); return -1; }
    int64_t p = 0;
    out->row_ptr[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        memcpy(out->col + p, tmp + off[i], (size_t)deg[i] * sizeof(int32_t));
        p += deg[i];
        out->row_ptr[i + 1] = (int32_t)p;
    }
    free(deg);
    free(off);
    free(tmp);
    return 0;
}

/* Erdos-Renyi G(n, p): each of the n(n-1)/2 pairs is an edge iff its draw is
 * below thr = floor(p * 2^64).  O(n^2) draws, meant for n up to ~10^5. */
int gg_er(int32_t n, uint64_t thr, uint64_t seed, gg_csr *out) {
    uint64_t key = gg_key(seed, ST_ER);
    int64_t cap = 1024, m = 0;
    int32_t *eu = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    int32_t *ev = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    if (!eu || !ev) { free(eu); free(ev); return -1; }
    uint64_t idx = 0;
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t j = i + 1; j < n; ++j, ++idx) {
            if (gg_at(key, idx) < thr) {
                if (m == cap) {
                    cap *= 2;
                    int32_t *nu = (int32_t *)realloc(eu, (size_t)cap * sizeof(int32_t));
                    int32_t *nv = (int32_t *)realloc(ev, (size_t)cap * sizeof(int32_t));
                    if (!nu || !nv) { free(nu ? nu : eu); free(nv ? nv : ev); return -1; }
                    eu = nu;
                    ev = nv;
                }
                eu[m] = i;
                ev[m] = j;
                ++m;
            }
        }
    }
    int rc = gg_from_edges(n, m, eu, ev, out);
    free(eu);
    free(ev);
    return rc;
}

/* Seeded uniform permutation of [0, n) (Fisher-Yates, Durstenfeld form). */
int gg_permutation(int32_t n, uint64_t seed, uint64_t stream, int32_t *perm) {
    uint64_t key = gg_key(seed, stream);
    for (int32_t i = 0; i < n; ++i) perm[i] = i;
    for (int32_t i = n - 1; i > 0; --i) {
        int32_t j = (int32_t)gg_bounded(gg_at(key, (uint64_t)i), (uint64_t)i + 1);
        int32_t t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
    }
    return 0;
}

/* R-MAT (Chakrabarti, Zhan, Faloutsos, SDM 2004) without noise: edge e picks
 * one quadrant per bit with probabilities a, b, c, d; thresholds are given as
 * 32-bit fixed point (ta = floor(a 2^32), tab = floor((a+b) 2^32), ...).
 * permute != 0 relabels vertices by a seeded permutation so that hubs are
 * spread over the id range. */
int gg_rmat(int32_t scale, int32_t edge_factor, uint32_t ta, uint32_t tab, uint32_t tabc,
            uint64_t seed, int32_t permute, gg_csr *out) {
    memset(out, 0, sizeof(*out));
    if (scale < 1 || scale > 30 || edge_factor < 1) return -1;
    int32_t n = (int32_t)1 << scale;
    int64_t m = (int64_t)edge_factor * n;
    int32_t *eu = (int32_t *)malloc((size_t)m * sizeof(int32_t));
    int32_t *ev = (int32_t *)malloc((size_t)m * sizeof(int32_t));
    int32_t *perm = permute ? (int32_t *)malloc((size_t)n * sizeof(int32_t)) : NULL;
    if (!eu || !ev || (permute && !perm)) { free(eu); free(ev); free(perm); return -1; }
    uint64_t key = gg_key(seed, ST_RMAT);
    int64_t draws_per_edge = (scale + 1) / 2;
    for (int64_t e = 0; e < m; ++e) {
        uint32_t a = 0, b = 0;
        for (int32_t lvl = 0; lvl < scale; ++lvl) {
            uint64_t r64 = gg_at(key, (uint64_t)(e * draws_per_edge + lvl / 2));
            uint32_t r = (lvl & 1) ? (uint32_t)(r64 >> 32) : (uint32_t)r64;
            uint32_t bu, bv;
            if (r < ta) { bu = 0; bv = 0; }
            else if (r < tab) { bu = 0; bv = 1; }
            else if (r < tabc) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            a = (a << 1) | bu;
            b = (b << 1) | bv;
        }
        eu[e] = (int32_t)a;
        ev[e] = (int32_t)b;
    }
    if (permute) {
        gg_permutation(n, seed, ST_PERM, perm);
        for (int64_t e = 0; e < m; ++e) {
            eu[e] = perm[eu[e]];
            ev[e] = perm[ev[e]];
        }
    }
    int rc = gg_from_edges(n, m, eu, ev, out);
    free(eu);
    free(ev);
    free(perm);
    return rc;
}

/* Connected components by BFS; comp[v] = component index in discovery order
 * (by smallest vertex id).  Returns the number of components. */
static int32_t components(const gg_csr *g, int32_t *comp, int32_t *queue) {
    for (int32_t v = 0; v < g->n; ++v) comp[v] = -1;
    int32_t nc = 0;
    for (int32_t s = 0; s < g->n; ++s) {
        if (comp[s] >= 0) continue;
        int32_t head = 0, tail = 0;
        queue[tail++] = s;
        comp[s] = nc;
        while (head < tail) {
            int32_t x = queue[head++];
            for (int32_t p = g->row_ptr[x]; p < g->row_ptr[x + 1]; ++p) {
                int32_t y = g->col[p];
                if (comp[y] < 0) { comp[y] = nc; queue[tail++] = y; }
            }
        }
        ++nc;
    }
    return nc;
}

/* Component label of every vertex (comp[n], labels in discovery order from
 * the smallest vertex id).  Returns the number of components, -1 when out
 * of memory. */
int32_t gg_components(const gg_csr *g, int32_t *comp) {
    if (g->n == 0) return 0;
    int32_t *queue = (int32_t *)malloc((size_t)g->n * sizeof(int32_t));
    if (!queue) return -1;
    int32_t nc = components(g, comp, queue);
    free(queue);
    return nc;
}

/* Largest connected component (ties: the one holding the smallest id), with
 * vertices relabelled compactly in increasing old-id order. old_id (optional,
 * n entries) receives the old id of each kept vertex. */
int gg_lcc(const gg_csr *g, gg_csr *out, int32_t *old_id) {
    memset(out, 0, sizeof(*out));
    int32_t n = g->n;
    if (n == 0) {
        out->row_ptr = (int32_t *)calloc(1, sizeof(int32_t));
        out->col = (int32_t *)malloc(sizeof(int32_t));
        return out->row_ptr && out->col ? 0 : -1;
    }
    int32_t *comp = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!comp || !queue) { free(comp); free(queue); return -1; }
    int32_t nc = components(g, comp, queue);
    int64_t *size = (int64_t *)calloc((size_t)nc, sizeof(int64_t));
    if (!size) { free(comp); free(queue); return -1; }
    for (int32_t v = 0; v < n; ++v) size[comp[v]]++;
    int32_t best = 0;
    for (int32_t c = 1; c < nc; ++c)
        if (size[c] > size[best]) best = c;
    int32_t *newid = queue; /* reuse */
    int32_t k = 0;
    for (int32_t v = 0; v < n; ++v) {
        if (comp[v] == best) {
            if (old_id) old_id[k] = v;
            newid[v] = k++;
        } else {
            newid[v] = -1;
        }
    }
    int64_t nnz = 0;
    for (int32_t v = 0; v < n; ++v)
        if (newid[v] >= 0) nnz += g->row_ptr[v + 1] - g->row_ptr[v];
    out->n = k;
    out->nnz = nnz;
    out->row_ptr = (int32_t *)malloc(((size_t)k + 1) * sizeof(int32_t));
    out->col = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    if (!out->row_ptr || !out->col) { gg_free_csr(out); free(comp); free(queue); free(size); return -1; }
    int64_t p = 0;
    out->row_ptr[0] = 0;
    for (int32_t v = 0, r = 0; v < n; ++v) {
        if (newid[v] < 0) continue;
        /* relabelling is monotone, so each row stays sorted */
        for (int32_t q = g->row_ptr[v]; q < g->row_ptr[v + 1]; ++q) out->col[p++] = newid[g->col[q]];
        out->row_ptr[++r] = (int32_t)p;
    }
    free(comp);
    free(queue);
    free(size);
    return 0;
}

/* side x side 4-neighbour grid; remove_count edges removed uniformly without
 * replacement (partial Fisher-Yates over edge indices); keep_lcc keeps the
 * largest component, relabelled in row-major order.  Vertex (i, j) = i*side+j
 * before relabelling.  Edge index: horizontal (i,j)-(i,j+1) -> i*(side-1)+j,
 * vertical (i,j)-(i+1,j) -> side*(side-1) + i*side + j. */
int gg_grid(int32_t side, int64_t remove_count, uint64_t seed, int32_t keep_lcc, gg_csr *out) {
    memset(out, 0, sizeof(*out));
    if (side < 1 || (int64_t)side * side >= ((int64_t)1 << 31)) return -1;
    int64_t H = (int64_t)side * (side - 1);
    int64_t E = 2 * H;
    if (remove_count < 0 || remove_count > E) return -1;
    int64_t *idx = (int64_t *)malloc((size_t)(E > 0 ? E : 1) * sizeof(int64_t));
    uint8_t *removed = (uint8_t *)calloc((size_t)(E > 0 ? E : 1), 1);
    if (!idx || !removed) { free(idx); free(removed); return -1; }
    for (int64_t e = 0; e < E; ++e) idx[e] = e;
    uint64_t key = gg_key(seed, ST_GRID);
    for (int64_t i = 0; i < remove_count; ++i) {
        int64_t j = i + (int64_t)gg_bounded(gg_at(key, (uint64_t)i), (uint64_t)(E - i));
        int64_t t = idx[i];
        idx[i] = idx[j];
        idx[j] = t;
        removed[idx[i]] = 1;
    }
    int64_t m = E - remove_count;
    int32_t *eu = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    int32_t *ev = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    if (!eu || !ev) { free(idx); free(removed); free(eu); free(ev); return -1; }
    int64_t q = 0;
    for (int64_t e = 0; e < E; ++e) {
        if (removed[e]) continue;
        int32_t a, b;
        if (e < H) {
            int32_t i = (int32_t)(e / (side - 1)), j = (int32_t)(e % (side - 1));
            a = i * side + j;
            b = a + 1;
        } else {
            int64_t f = e - H;
            int32_t i = (int32_t)(f / side), j = (int32_t)(f % side);
            a = i * side + j;
            b = a + side;
        }
        eu[q] = a;
        ev[q] = b;
        ++q;
    }
    free(idx);
    free(removed);
    gg_csr full;
    int rc = gg_from_edges(side * side, m, eu, ev, &full);
    free(eu);
    free(ev);
    if (rc) return rc;
    if (!keep_lcc) { *out = full; return 0; }
    rc = gg_lcc(&full, out, NULL);
    gg_free_csr(&full);
    return rc;
}

/* Planar triangulation of a side x side point lattice (a Delaunay-like
 * planar graph): the 4-neighbour grid edges plus one diagonal per unit cell,
 * (i,j)-(i+1,j+1) or (i,j+1)-(i+1,j) by one random bit per cell.  Interior
 * vertices have degree 4 + (diagonals at their 4 cells), 6 on average; the
 * graph is connected.  Vertex (i, j) = i*side + j. */
int gg_tri(int32_t side, uint64_t seed, gg_csr *out) {
    memset(out, 0, sizeof(*out));
    if (side < 1 || (int64_t)side * side >= ((int64_t)1 << 31)) return -1;
    int64_t cells = (int64_t)(side - 1) * (side - 1);
    int64_t m = 2 * (int64_t)side * (side - 1) + cells;
    int32_t *eu = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    int32_t *ev = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    if (!eu || !ev) { free(eu); free(ev); return -1; }
    uint64_t key = gg_key(seed, ST_TRI);
    int64_t q = 0;
    for (int32_t i = 0; i < side; ++i)
        for (int32_t j = 0; j < side; ++j) {
            int32_t a = i * side + j;
            if (j + 1 < side) { eu[q] = a; ev[q] = a + 1; ++q; }
            if (i + 1 < side) { eu[q] = a; ev[q] = a + side; ++q; }
            if (i + 1 < side && j + 1 < side) {
                uint64_t bit = gg_at(key, (uint64_t)i * (uint64_t)(side - 1) + (uint64_t)j) >> 63;
                if (bit) { eu[q] = a + 1; ev[q] = a + side; }
                else { eu[q] = a; ev[q] = a + side + 1; }
                ++q;
            }
        }
    int rc = gg_from_edges(side * side, q, eu, ev, out);
    free(eu);
    free(ev);
    return rc;
}

static uint64_t isqrt64(uint64_t x) {
    uint64_t r = 0;
    for (int b = 31; b >= 0; --b) {
        uint64_t t = r | (1ULL << b);
        if ((__uint128_t)t * t <= x) r = t;
    }
    return r;
}

/* Random geometric graph: n points with independent uniform 32-bit integer
 * coordinates (x, y) in [0, 2^32)^2, an edge between two points whose squared
 * Euclidean distance is below r2 (exact integer arithmetic).  Points are
 * binned into square cells of side >= sqrt(r2) and numbered in cell order
 * (row-major over cells, generation order within a cell), so that vertex ids
 * follow space; keep_lcc keeps the largest component, renumbered in order. */
int gg_rgg(int32_t n, uint64_t r2, uint64_t seed, int32_t keep_lcc, gg_csr *out) {
    memset(out, 0, sizeof(*out));
    if (n < 1 || r2 == 0) return -1;
    uint64_t r = isqrt64(r2);
    if ((__uint128_t)r * r < r2) ++r; /* ceil(sqrt(r2)) */
    uint64_t cs = r > 0 ? r : 1;     /* cell side */
    uint64_t C = ((1ULL << 32) + cs - 1) / cs;
    uint64_t cmax = isqrt64((uint64_t)n);  /* at most about n cells */
    if (cmax < 1) cmax = 1;
    if (C > cmax) C = cmax, cs = ((1ULL << 32) + C - 1) / C;
    uint32_t *px = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    uint32_t *py = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    int64_t *cstart = (int64_t *)calloc((size_t)(C * C + 1), sizeof(int64_t));
    int32_t *order = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!px || !py || !cstart || !order) {
        free(px); free(py); free(cstart); free(order);
        return -1;
    }
    uint64_t key = gg_key(seed, ST_RGG);
    for (int32_t i = 0; i < n; ++i) {
        px[i] = (uint32_t)(gg_at(key, 2 * (uint64_t)i) >> 32);
        py[i] = (uint32_t)(gg_at(key, 2 * (uint64_t)i + 1) >> 32);
        cstart[(py[i] / cs) * C + px[i] / cs + 1]++;
    }
    for (uint64_t c = 0; c < C * C; ++c) cstart[c + 1] += cstart[c];
    {
        int64_t *fill = (int64_t *)malloc((size_t)(C * C) * sizeof(int64_t));
        if (!fill) { free(px); free(py); free(cstart); free(order); return -1; }
        memcpy(fill, cstart, (size_t)(C * C) * sizeof(int64_t));
        for (int32_t i = 0; i < n; ++i) {
            int64_t p = fill[(py[i] / cs) * C + px[i] / cs]++;
            order[p] = i;
        }
        free(fill);
    }
    /* edges between points of neighbouring cells, each pair once (a < b) */
    int64_t cap = 1024, m = 0;
    int32_t *eu = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    int32_t *ev = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    int rc = (eu && ev) ? 0 : -1;
    for (int64_t p = 0; p < n && rc == 0; ++p) {
        int32_t i = order[p];
        int64_t cx = px[i] / cs, cy = py[i] / cs;
        for (int64_t dy = -1; dy <= 1 && rc == 0; ++dy)
            for (int64_t dx = -1; dx <= 1; ++dx) {
                int64_t ux = cx + dx, uy = cy + dy;
                if (ux < 0 || uy < 0 || ux >= (int64_t)C || uy >= (int64_t)C) continue;
                int64_t c = uy * (int64_t)C + ux;
                for (int64_t q = cstart[c]; q < cstart[c + 1]; ++q) {
                    if (q <= p) continue;
                    int32_t j = order[q];
                    int64_t ddx = (int64_t)px[i] - (int64_t)px[j], ddy = (int64_t)py[i] - (int64_t)py[j];
                    uint64_t adx = (uint64_t)(ddx < 0 ? -ddx : ddx), ady = (uint64_t)(ddy < 0 ? -ddy : ddy);
                    __uint128_t d2 = (__uint128_t)adx * adx + (__uint128_t)ady * ady;
                    if (d2 >= (__uint128_t)r2) continue;
                    if (m == cap) {
                        cap *= 2;
                        int32_t *nu = (int32_t *)realloc(eu, (size_t)cap * sizeof(int32_t));
                        int32_t *nv = nu ? (int32_t *)realloc(ev, (size_t)cap * sizeof(int32_t)) : NULL;
                        if (nu) eu = nu;
                        if (nv) ev = nv;
                        if (!nu || !nv) { rc = -1; break; }
                    }
                    eu[m] = (int32_t)p;
                    ev[m] = (int32_t)q;
                    ++m;
                }
            }
    }
    free(px); free(py); free(cstart); free(order);
    gg_csr full;
    if (rc == 0) rc = gg_from_edges(n, m, eu, ev, &full);
    free(eu);
    free(ev);
    if (rc) return rc;
    if (!keep_lcc) { *out = full; return 0; }
    rc = gg_lcc(&full, out, NULL);
    gg_free_csr(&full);
    return rc;
}

/* 3-D mesh with the 27-point stencil (a banded, KKT-like sparsity pattern):
 * nx x ny x nz points, each joined to every other point whose coordinates
 * differ by at most 1 in each dimension (26 neighbours inside).  Vertex
 * (x, y, z) = (x*ny + y)*nz + z. */
int gg_mesh27(int32_t nx, int32_t ny, int32_t nz, gg_csr *out) {
    memset(out, 0, sizeof(*out));
    if (nx < 1 || ny < 1 || nz < 1) return -1;
    int64_t n = (int64_t)nx * ny * nz;
    if (n >= ((int64_t)1 << 31) || 13 * n >= ((int64_t)1 << 31)) return -1;
    int64_t cap = 13 * n + 1, m = 0;
    int32_t *eu = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    int32_t *ev = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    if (!eu || !ev) { free(eu); free(ev); return -1; }
    for (int32_t x = 0; x < nx; ++x)
        for (int32_t y = 0; y < ny; ++y)
            for (int32_t z = 0; z < nz; ++z) {
                int32_t a = (x * ny + y) * nz + z;
                for (int dx = -1; dx <= 1; ++dx)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dz = -1; dz <= 1; ++dz) {
                            int32_t X = x + dx, Y = y + dy, Z = z + dz;
                            if (X < 0 || Y < 0 || Z < 0 || X >= nx || Y >= ny || Z >= nz) continue;
                            int32_t b = (X * ny + Y) * nz + Z;
                            if (b <= a) continue;
                            eu[m] = a;
                            ev[m] = b;
                            ++m;
                        }
            }
    int rc = gg_from_edges((int32_t)n, m, eu, ev, out);
    free(eu);
    free(ev);
    return rc;
}

/* Edge weights for a symmetric CSR: the undirected edge {u, v} gets
 * 1 + (value (min(u,v) * n + max(u,v)) of the weight stream, bounded to
 * [0, max_weight)), so both of its entries carry the same weight. */
int gg_weights(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t max_weight, uint64_t seed,
               int32_t *out) {
    if (n < 0 || max_weight < 1) return -1;
    uint64_t key = gg_key(seed, ST_WEIGHT);
    for (int32_t u = 0; u < n; ++u)
        for (int32_t p = row_ptr[u]; p < row_ptr[u + 1]; ++p) {
            int32_t v = col[p];
            uint64_t a = (uint64_t)(u < v ? u : v), b = (uint64_t)(u < v ? v : u);
            out[p] = 1 + (int32_t)gg_bounded(gg_at(key, a * (uint64_t)n + b), (uint64_t)max_weight);
        }
    return 0;
}

/* k distinct sources drawn uniformly from [0, n) (partial Fisher-Yates). */
int gg_sample_sources(int32_t n, int64_t k, uint64_t seed, int32_t *out) {
    if (k < 0 || k > n) return -1;
    int32_t *pool = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!pool) return -1;
    for (int32_t i = 0; i < n; ++i) pool[i] = i;
    uint64_t key = gg_key(seed, ST_SRC);
    for (int64_t i = 0; i < k; ++i) {
        int64_t j = i + (int64_t)gg_bounded(gg_at(key, (uint64_t)i), (uint64_t)(n - i));
        int32_t t = pool[i];
        pool[i] = pool[j];
        pool[j] = t;
        out[i] = pool[i];
    }
    free(pool);
    return 0;
}
