/*
 * ORACLE - test infrastructure, not part of the product.
 *
 * Plain, single-threaded, deliberately unoptimised Brandes betweenness
 * centrality for unweighted undirected graphs in CSR form.  Only the tests,
 * the smoke check and the benchmark's CPU-baseline leg may load this code;
 * the CUDA library never links or calls it, and it shares no code with it.
 *
 * What it computes, per source s, in the paper's order (Sec. II):
 *   forward phase  - Algorithm 1's level-by-level BFS: level[0] = {s},
 *                    dist[s] = 0, sigma[s] = 1, every other vertex dist -1,
 *                    sigma 0, empty pred set; for each v in level[cur] and each
 *                    neighbour w: an undiscovered w joins level[cur+1] with
 *                    dist[v]+1; if dist[w] == dist[v]+1 then sigma[w] +=
 *                    sigma[v] and v joins pred[w].
 *   backward phase - Algorithm 1's reverse sweep from the deepest level down
 *                    to level 1: for u in level[cur], for v in pred[u],
 *                    delta[v] += sigma[v]/sigma[u] * (1 + delta[u])  (Eq. 2).
 *   accumulation   - BC[v] += delta_s(v) for every v != s (the sum that
 *                    follows Eq. 2: BC[v] = sum over s != v of delta_s(v)).
 *
 * Readings where the paper is silent:
 *   - sigma is kept EXACT as a multi-limb unsigned integer (64-bit limbs);
 *     the reported sigma is the value mod 2^64 plus a flag "sigma >= 2^64".
 *   - the ratio sigma[v]/sigma[u] is formed from the two exact integers, each
 *     rounded once to a 53-bit mantissa (round to nearest, ties to even) with
 *     an unbounded binary exponent, then divided in double precision and
 *     rescaled by the exponent difference.  Below 2^1024 this is exactly
 *     (double)sigma[v] / (double)sigma[u].
 *   - sources are taken in list order, duplicates counted with multiplicity;
 *     no n/k rescaling; unreachable vertices keep dist -1, sigma 0, delta 0.
 *   - BC counts ordered pairs (no factor 1/2), as Eq. 1 sums over s and t.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct {
    uint64_t *limb; /* arena */
    size_t cap, used;
} arena_t;

static int64_t arena_alloc(arena_t *a, size_t nlimbs) {
    if (a->used + nlimbs > a->cap) {
        size_t nc = a->cap ? a->cap : 1024;
        while (a->used + nlimbs > nc) nc *= 2;
        uint64_t *p = (uint64_t *)realloc(a->limb, nc * sizeof(uint64_t));
        if (!p) return -1;
        a->limb = p;
        a->cap = nc;
    }
    int64_t off = (int64_t)a->used;
    memset(a->limb + off, 0, nlimbs * sizeof(uint64_t));
    a->used += nlimbs;
    return off;
}

/* number of significant limbs of x[0..len) */
static int32_t big_len(const uint64_t *x, int32_t len) {
    while (len > 0 && x[len - 1] == 0) --len;
    return len;
}

/* dst[0..dcap) += src[0..slen), dcap > slen; the true sum fits in dcap limbs */
static void big_add(uint64_t *dst, int32_t dcap, const uint64_t *src, int32_t slen) {
    uint64_t carry = 0;
    int32_t i = 0;
    for (; i < slen; ++i) {
        uint64_t a = dst[i], b = src[i];
        uint64_t s = a + b;
        uint64_t c1 = s < a;
        uint64_t s2 = s + carry;
        uint64_t c2 = s2 < s;
        dst[i] = s2;
        carry = c1 | c2;
    }
    for (; carry && i < dcap; ++i) {
        dst[i] += 1;
        carry = dst[i] == 0;
    }
}

static int clz64(uint64_t x) { return x ? __builtin_clzll(x) : 64; }

/* x = mant * 2^exp with mant in [1, 2) holding the correctly rounded 53-bit
 * significand of the exact integer x (round to nearest, ties to even). */
void oracle_big_to_scaled(const uint64_t *x, int32_t len, double *mant, int64_t *exp) {
    len = big_len(x, len);
    if (len == 0) { *mant = 0.0; *exp = 0; return; }
    int32_t t = len - 1;
    uint64_t hi = x[t];
    int nb = 64 - clz64(hi);                 /* significant bits in the top limb */
    int64_t bits = (int64_t)64 * t + nb;     /* total significant bits */
    uint64_t top;                            /* the leading 64 bits, MSB set */
    int sticky = 0;
    if (nb == 64) {
        top = hi;
        for (int32_t i = t - 1; i >= 0; --i) sticky |= x[i] != 0;
    } else if (t > 0) {
        top = (hi << (64 - nb)) | (x[t - 1] >> nb);
        sticky = (x[t - 1] << (64 - nb)) != 0;
        for (int32_t i = t - 2; i >= 0; --i) sticky |= x[i] != 0;
    } else {
        top = hi << (64 - nb);
    }
    uint64_t keep = top >> 11;               /* 53 bits */
    uint64_t rem = top & 0x7FFULL;
    if (rem > 0x400ULL || (rem == 0x400ULL && (sticky || (keep & 1)))) {
        keep += 1;
        if (keep == (1ULL << 53)) { keep = 1ULL << 52; bits += 1; }
    }
    *mant = ldexp((double)keep, -52);
    *exp = bits - 1;
}

/* sigma[v] / sigma[u] from sigma[v] (exact integer) and the rounded
 * (mu, eu) of sigma[u], as described in the header. */
static double ratio(const uint64_t *sv, int32_t lv, double mu, int64_t eu) {
    double mv;
    int64_t ev;
    oracle_big_to_scaled(sv, lv, &mv, &ev);
    int64_t d = ev - eu;
    if (d < -4000) return 0.0;
    return ldexp(mv / mu, (int)d);
}

/*
 * Brandes BC over the k listed sources, ADDED into bc[0..n).
 * For the sources whose positions are listed in dump_idx[0..n_dump), the
 * per-vertex state is written row by row (row i = dump_idx[i]):
 *   dump_dist[i*n + v]  (int32, -1 unreachable)   may be NULL
 *   dump_sigma[i*n + v] (sigma mod 2^64)          may be NULL
 *   dump_ovf[i*n + v]   (1 iff sigma >= 2^64)     may be NULL
 *   dump_delta[i*n + v] (delta_s(v); at v = s the recurrence's value, which
 *                        is not added to BC)     may be NULL
 * Returns 0; -1 on invalid input; -2 on allocation failure.
 */
int oracle_bc(int32_t n, const int32_t *row_ptr, const int32_t *col, int64_t k, const int32_t *sources,
              double *bc, int64_t n_dump, const int64_t *dump_idx, int32_t *dump_dist,
              uint64_t *dump_sigma, uint8_t *dump_ovf, double *dump_delta) {
    if (n < 0 || k < 0) return -1;
    for (int64_t i = 0; i < k; ++i)
        if (sources[i] < 0 || sources[i] >= n) return -1;
    if (n == 0) return 0;
    int64_t nnz = row_ptr[n];
    int32_t *dist = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int64_t *soff = (int64_t *)malloc((size_t)n * sizeof(int64_t)); /* sigma limbs offset */
    int32_t *scap = (int32_t *)malloc((size_t)n * sizeof(int32_t)); /* sigma limbs allocated */
    int32_t *order = (int32_t *)malloc((size_t)n * sizeof(int32_t)); /* vertices by level */
    int64_t *lstart = (int64_t *)malloc(((size_t)n + 2) * sizeof(int64_t)); /* level boundaries */
    int32_t *npred = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *pred = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t)); /* pred[w] in row w's slots */
    double *delta = (double *)malloc((size_t)n * sizeof(double));
    arena_t ar = {0, 0, 0};
    int rc = 0;
    if (!dist || !soff || !scap || !order || !lstart || !npred || !pred || !delta) { rc = -2; goto done; }

    for (int64_t si = 0; si < k; ++si) {
        int32_t s = sources[si];
        /* ---- forward phase (Algorithm 1) ---- */
        for (int32_t v = 0; v < n; ++v) { dist[v] = -1; scap[v] = 0; soff[v] = -1; npred[v] = 0; }
        ar.used = 0;
        dist[s] = 0;
        soff[s] = arena_alloc(&ar, 1);
        if (soff[s] < 0) { rc = -2; goto done; }
        ar.limb[soff[s]] = 1;
        scap[s] = 1;
        int64_t head = 0, tail = 0; /* level[cur] = order[lstart[cur] .. lstart[cur+1]) */
        int32_t nlev = 0;
        order[tail++] = s;
        lstart[0] = 0;
        while (head < tail) {          /* while level[curLevel] is not empty */
            int64_t lend = tail;
            lstart[nlev + 1] = lend;
            /* widest sigma at this level: every sigma of level cur is final now */
            int32_t maxlen = 1;
            for (int64_t q = head; q < lend; ++q) {
                int32_t v = order[q];
                int32_t l = big_len(ar.limb + soff[v], scap[v]);
                if (l > maxlen) maxlen = l;
            }
            for (int64_t q = head; q < lend; ++q) {
                int32_t v = order[q];
                for (int32_t p = row_ptr[v]; p < row_ptr[v + 1]; ++p) {
                    int32_t w = col[p];
                    if (dist[w] == -1) {
                        order[tail++] = w;      /* level[cur+1] gets w */
                        dist[w] = dist[v] + 1;
                        int64_t off = arena_alloc(&ar, (size_t)maxlen + 1);
                        if (off < 0) { rc = -2; goto done; }
                        soff[w] = off;
                        scap[w] = maxlen + 1;
                    }
                    if (dist[w] == dist[v] + 1) {
                        big_add(ar.limb + soff[w], scap[w], ar.limb + soff[v], big_len(ar.limb + soff[v], scap[v]));
                        pred[row_ptr[w] + npred[w]++] = v;
                    }
                }
            }
            head = lend;
            ++nlev;
        }
        /* ---- backward phase (Algorithm 1, Eq. 2) ---- */
        for (int32_t v = 0; v < n; ++v) delta[v] = 0.0;
        for (int32_t cur = nlev - 1; cur > 0; --cur) {
            for (int64_t q = lstart[cur]; q < lstart[cur + 1]; ++q) {
                int32_t u = order[q];
                double mu;
                int64_t eu;
                oracle_big_to_scaled(ar.limb + soff[u], scap[u], &mu, &eu);
                for (int32_t j = 0; j < npred[u]; ++j) {
                    int32_t v = pred[row_ptr[u] + j];
                    delta[v] += ratio(ar.limb + soff[v], scap[v], mu, eu) * (1.0 + delta[u]);
                }
            }
        }
        /* ---- BC[v] += delta_s(v), v != s ---- */
        for (int32_t v = 0; v < n; ++v)
            if (v != s) bc[v] += delta[v];
        /* ---- optional dumps ---- */
        for (int64_t di = 0; di < n_dump; ++di) {
            if (dump_idx[di] != si) continue;
            for (int32_t v = 0; v < n; ++v) {
                size_t at = (size_t)di * (size_t)n + (size_t)v;
                int reach = dist[v] >= 0;
                const uint64_t *sv = reach ? ar.limb + soff[v] : NULL;
                int32_t lv = reach ? big_len(sv, scap[v]) : 0;
                if (dump_dist) dump_dist[at] = dist[v];
                if (dump_sigma) dump_sigma[at] = lv > 0 ? sv[0] : 0;
                if (dump_ovf) dump_ovf[at] = (uint8_t)(lv > 1);
                if (dump_delta) dump_delta[at] = delta[v];
            }
        }
    }
done:
    free(dist); free(soff); free(scap); free(order); free(lstart); free(npred); free(pred); free(delta);
    free(ar.limb);
    return rc;
}

/*
 * Weighted form (the SSSP case the paper's forward phase names beside BFS,
 * Sec. IV-C: "BFS/SSSP"): undirected edges with positive integer weights,
 * weight[p] belonging to the CSR entry col[p] (symmetric: the two entries of
 * an edge carry the same weight).  Per source s:
 *   distances   - Dijkstra from s (binary heap, lazy deletion); the settle
 *                 order lists the reached vertices by nondecreasing distance.
 *   sigma       - in settle order, for w != s: sigma[w] = sum of sigma[v]
 *                 over the neighbours v with dist[v] + weight(v, w) ==
 *                 dist[w] (its shortest-path predecessors, all settled
 *                 before w since weights are >= 1); sigma[s] = 1; exact.
 *   backward    - in reverse settle order, for each such predecessor v of w:
 *                 delta[v] += sigma[v]/sigma[w] * (1 + delta[w])  (Eq. 2).
 *   accumulation, dumps, ratio rounding: as in oracle_bc.
 * Distances are int64 here; the dumps hold them as int32 (-1 unreachable),
 * and a distance above 2^31 - 1 is an error (-3).
 */
typedef struct {
    int64_t d;
    int32_t v;
} heap_item;

static void heap_push(heap_item *h, int64_t *len, int64_t d, int32_t v) {
    int64_t i = (*len)++;
    h[i].d = d;
    h[i].v = v;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h[p].d <= h[i].d) break;
        heap_item t = h[p]; h[p] = h[i]; h[i] = t;
        i = p;
    }
}

static heap_item heap_pop(heap_item *h, int64_t *len) {
    heap_item top = h[0];
    h[0] = h[--(*len)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < *len && h[l].d < h[m].d) m = l;
        if (r < *len && h[r].d < h[m].d) m = r;
        if (m == i) break;
        heap_item t = h[m]; h[m] = h[i]; h[i] = t;
        i = m;
    }
    return top;
}

int oracle_bc_weighted(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *weight, int64_t k,
                       const int32_t *sources, double *bc, int64_t n_dump, const int64_t *dump_idx,
                       int32_t *dump_dist, uint64_t *dump_sigma, uint8_t *dump_ovf, double *dump_delta) {
    if (n < 0 || k < 0) return -1;
    for (int64_t i = 0; i < k; ++i)
        if (sources[i] < 0 || sources[i] >= n) return -1;
    if (n == 0) return 0;
    int64_t nnz = row_ptr[n];
    for (int64_t p = 0; p < nnz; ++p)
        if (weight[p] < 1) return -1;
    int64_t *dist = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    uint8_t *done_v = (uint8_t *)malloc((size_t)n);
    int64_t *soff = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int32_t *scap = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *order = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    double *delta = (double *)malloc((size_t)n * sizeof(double));
    heap_item *heap = (heap_item *)malloc((size_t)(nnz + 2) * sizeof(heap_item));
    arena_t ar = {0, 0, 0};
    int rc = 0;
    if (!dist || !done_v || !soff || !scap || !order || !delta || !heap) { rc = -2; goto done; }

    for (int64_t si = 0; si < k; ++si) {
        int32_t s = sources[si];
        for (int32_t v = 0; v < n; ++v) { dist[v] = -1; done_v[v] = 0; soff[v] = -1; scap[v] = 0; }
        ar.used = 0;
        /* ---- distances: Dijkstra ---- */
        int64_t hl = 0, nset = 0;
        dist[s] = 0;
        heap_push(heap, &hl, 0, s);
        while (hl > 0) {
            heap_item it = heap_pop(heap, &hl);
            int32_t u = it.v;
            if (done_v[u] || it.d != dist[u]) continue; /* stale entry */
            done_v[u] = 1;
            order[nset++] = u;
            for (int32_t p = row_ptr[u]; p < row_ptr[u + 1]; ++p) {
                int32_t w = col[p];
                int64_t nd = dist[u] + (int64_t)weight[p];
                if (!done_v[w] && (dist[w] < 0 || nd < dist[w])) {
                    dist[w] = nd;
                    heap_push(heap, &hl, nd, w);
                }
            }
        }
        for (int64_t q = 0; q < nset; ++q)
            if (dist[order[q]] > 2147483647LL) { rc = -3; goto done; }
        /* ---- sigma in settle order, from the predecessors ---- */
        soff[s] = arena_alloc(&ar, 1);
        if (soff[s] < 0) { rc = -2; goto done; }
        ar.limb[soff[s]] = 1;
        scap[s] = 1;
        for (int64_t q = 1; q < nset; ++q) {
            int32_t w = order[q];
            int32_t maxlen = 1;
            for (int32_t p = row_ptr[w]; p < row_ptr[w + 1]; ++p) {
                int32_t v = col[p];
                if (dist[v] >= 0 && dist[v] + (int64_t)weight[p] == dist[w]) {
                    int32_t l = big_len(ar.limb + soff[v], scap[v]);
                    if (l > maxlen) maxlen = l;
                }
            }
            int64_t off = arena_alloc(&ar, (size_t)maxlen + 1);
            if (off < 0) { rc = -2; goto done; }
            soff[w] = off;
            scap[w] = maxlen + 1;
            for (int32_t p = row_ptr[w]; p < row_ptr[w + 1]; ++p) {
                int32_t v = col[p];
                if (dist[v] >= 0 && dist[v] + (int64_t)weight[p] == dist[w])
                    big_add(ar.limb + soff[w], scap[w], ar.limb + soff[v], big_len(ar.limb + soff[v], scap[v]));
            }
        }
        /* ---- backward (Eq. 2) in reverse settle order ---- */
        for (int32_t v = 0; v < n; ++v) delta[v] = 0.0;
        for (int64_t q = nset - 1; q > 0; --q) {
            int32_t w = order[q];
            double mw;
            int64_t ew;
            oracle_big_to_scaled(ar.limb + soff[w], scap[w], &mw, &ew);
            for (int32_t p = row_ptr[w]; p < row_ptr[w + 1]; ++p) {
                int32_t v = col[p];
                if (dist[v] >= 0 && dist[v] + (int64_t)weight[p] == dist[w])
                    delta[v] += ratio(ar.limb + soff[v], scap[v], mw, ew) * (1.0 + delta[w]);
            }
        }
        for (int32_t v = 0; v < n; ++v)
            if (v != s) bc[v] += delta[v];
        for (int64_t di = 0; di < n_dump; ++di) {
            if (dump_idx[di] != si) continue;
            for (int32_t v = 0; v < n; ++v) {
                size_t at = (size_t)di * (size_t)n + (size_t)v;
                int reach = dist[v] >= 0;
                const uint64_t *sv = reach ? ar.limb + soff[v] : NULL;
                int32_t lv = reach ? big_len(sv, scap[v]) : 0;
                if (dump_dist) dump_dist[at] = (int32_t)dist[v];
                if (dump_sigma) dump_sigma[at] = lv > 0 ? sv[0] : 0;
                if (dump_ovf) dump_ovf[at] = (uint8_t)(lv > 1);
                if (dump_delta) dump_delta[at] = delta[v];
            }
        }
    }
done:
    free(dist); free(done_v); free(soff); free(scap); free(order); free(delta); free(heap);
    free(ar.limb);
    return rc;
}
