/*
 * graphgen.c -- seeded synthetic graphs and personalization seed sets.
 *
 * These are the inputs that both the CUDA path and the oracle consume.  Nothing
 * here computes any part of the PageRank / D-iteration method: the output is a
 * CSR of out-links (row_ptr[n+1], col_idx[L], int32) and lists of seed nodes.
 *
 * Random numbers come from a counter-based generator built on the SplitMix64
 * finaliser (Steele, Lea & Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): draw(seed, stream, ctr) hashes the triple, so every
 * row / edge owns an independent stream and the output does not depend on the
 * number of OpenMP threads or on the machine.
 *
 * Graph families (the paper's workloads, Section 4.1, use power-law source and
 * destination choices; the families below are the synthetic stand-ins):
 *   uniform : out-degree uniform in {0..dmax}, targets uniform over the other
 *             nodes, no self-loops, no duplicates.
 *   zipf    : an exact floor(frac*n) dangling set chosen by a seeded
 *             permutation; other out-degrees Zipf(alpha) on k>=1 clipped at kmax;
 *             targets drawn with probability proportional to rank^-beta where
 *             ranks are assigned to node ids by a second seeded permutation;
 *             self-loops and duplicates are re-drawn, so each row keeps its drawn
 *             out-degree.
 *   rmat    : R-MAT (Chakrabarti, Zhan & Faloutsos 2004) with quadrant
 *             probabilities (a,b,c,1-a-b-c), edge_factor*2^scale draws, no noise,
 *             no id permutation, self-loops kept, duplicates optionally removed.
 * Every row of every CSR produced here is sorted ascending.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef uint64_t u64;
typedef int32_t i32;
typedef int64_t i64;

static inline u64 mix64(u64 z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* value number `ctr` of stream `stream` under `seed` */
static inline u64 draw(u64 seed, u64 stream, u64 ctr) {
    return mix64(mix64(seed * 0x9e3779b97f4a7c15ULL + stream) + (ctr + 1) * 0x9e3779b97f4a7c15ULL);
}

static inline double unit(u64 x) { return (double)(x >> 11) * 0x1.0p-53; }

/* integer in [0, m) by the multiply-high method (bias below 2^-32 for m < 2^32) */
static inline u64 below(u64 x, u64 m) { return (u64)(((unsigned __int128)x * m) >> 64); }

/* stream namespaces so that different uses of one seed never share a stream */
enum { S_DEG = 1, S_ROW = 2, S_PERM1 = 3, S_PERM2 = 4, S_EDGE = 5, S_SEEDS = 6 };
#define STREAM(kind, id) (((u64)(kind) << 56) ^ (u64)(id))

static int cmp_i32(const void *a, const void *b) {
    i32 x = *(const i32 *)a, y = *(const i32 *)b;
    return (x > y) - (x < y);
}

/* Fisher-Yates permutation of [0,n) driven by one stream */
static void permutation(u64 seed, int kind, i32 n, i32 *perm) {
    for (i32 i = 0; i < n; ++i) perm[i] = i;
    for (i32 i = n - 1; i > 0; --i) {
        i32 j = (i32)below(draw(seed, STREAM(kind, 0), (u64)i), (u64)i + 1);
        i32 t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
}

static void exclusive_scan_deg(i32 n, const i32 *deg, i32 *row_ptr) {
    i64 acc = 0;
    for (i32 i = 0; i < n; ++i) { row_ptr[i] = (i32)acc; acc += deg[i]; }
    row_ptr[n] = (i32)acc;
}

/* ------------------------------------------------------------------ uniform */

/* out-degrees U{0..dmax}; returns total edges, or -1 if it overflows int32 */
i64 gg_uniform_degrees(i32 n, i32 dmax, u64 seed, i32 *row_ptr) {
    if (n <= 0 || dmax < 0) return -1;
    if (dmax > n - 1) dmax = n - 1;
    i32 *deg = (i32 *)malloc(sizeof(i32) * (size_t)n);
    if (!deg) return -1;
    for (i32 i = 0; i < n; ++i) deg[i] = (i32)below(draw(seed, STREAM(S_DEG, i), 0), (u64)dmax + 1);
    i64 tot = 0;
    for (i32 i = 0; i < n; ++i) tot += deg[i];
    if (tot > INT32_MAX) { free(deg); return -1; }
    exclusive_scan_deg(n, deg, row_ptr);
    free(deg);
    return tot;
}

static int row_contains(const i32 *row, i32 len, i32 v) {
    for (i32 k = 0; k < len; ++k) if (row[k] == v) return 1;
    return 0;
}

void gg_uniform_fill(i32 n, u64 seed, const i32 *row_ptr, i32 *col_idx) {
    #pragma omp parallel for schedule(dynamic, 256)
    for (i32 i = 0; i < n; ++i) {
        i32 *row = col_idx + row_ptr[i];
        i32 len = row_ptr[i + 1] - row_ptr[i];
        u64 ctr = 0;
        for (i32 k = 0; k < len; ++k) {
            for (;;) {
                i32 t = (i32)below(draw(seed, STREAM(S_ROW, i), ctr++), (u64)n);
                if (t == i || row_contains(row, k, t)) continue;
                row[k] = t;
                break;
            }
        }
        qsort(row, (size_t)len, sizeof(i32), cmp_i32);
    }
}

/* --------------------------------------------------------------------- zipf */

/* Hurwitz-style tail of zeta: sum_{m>=M} m^-s by Euler-Maclaurin (s > 1) */
static double zeta_tail(double s, double M) {
    return pow(M, 1.0 - s) / (s - 1.0) + 0.5 * pow(M, -s) + s * pow(M, -s - 1.0) / 12.0;
}

/* smallest index k with cdf[k] > u, or len if none */
static i64 search_cdf(const double *cdf, i64 len, double u) {
    i64 lo = 0, hi = len;
    while (lo < hi) {
        i64 mid = lo + (hi - lo) / 2;
        if (cdf[mid] > u) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/* Out-degrees for the zipf family.  Returns total edges (or -1). */
i64 gg_zipf_degrees(i32 n, double alpha, i32 kmax, double dangling_frac, u64 seed, i32 *row_ptr) {
    if (n <= 0 || kmax < 1 || alpha <= 1.0 || dangling_frac < 0 || dangling_frac > 1) return -1;
    if (kmax > n - 1) kmax = n - 1;
    if (kmax < 1) return -1;
    i32 *deg = (i32 *)malloc(sizeof(i32) * (size_t)n);
    i32 *perm = (i32 *)malloc(sizeof(i32) * (size_t)n);
    double *cdf = (double *)malloc(sizeof(double) * (size_t)kmax);
    if (!deg || !perm || !cdf) { free(deg); free(perm); free(cdf); return -1; }
    /* P(k) = k^-alpha / zeta(alpha), k >= 1; cdf[k-1] = P(K <= k) for k < kmax */
    double head = 0.0;
    for (i32 k = 1; k <= kmax - 1; ++k) head += pow((double)k, -alpha);
    double zeta = head + zeta_tail(alpha, (double)kmax);
    double acc = 0.0;
    for (i32 k = 1; k <= kmax - 1; ++k) { acc += pow((double)k, -alpha); cdf[k - 1] = acc / zeta; }
    permutation(seed, S_PERM1, n, perm);
    i32 ndang = (i32)floor(dangling_frac * (double)n);
    #pragma omp parallel for schedule(static)
    for (i32 r = 0; r < n; ++r) {
        i32 i = perm[r];
        if (r < ndang) { deg[i] = 0; continue; }
        double u = unit(draw(seed, STREAM(S_DEG, i), 0));
        i64 k = search_cdf(cdf, kmax - 1, u) + 1;   /* k in [1, kmax]; tail mass lands on kmax */
        deg[i] = (i32)k;
    }
    i64 tot = 0;
    for (i32 i = 0; i < n; ++i) tot += deg[i];
    free(perm); free(cdf);
    if (tot > INT32_MAX) { free(deg); return -1; }
    exclusive_scan_deg(n, deg, row_ptr);
    free(deg);
    return tot;
}

/* Targets for the zipf family: P(target = rank_perm[r-1]) proportional to r^-beta. */
int gg_zipf_fill(i32 n, double beta, u64 seed, const i32 *row_ptr, i32 *col_idx) {
    double *cdf = (double *)malloc(sizeof(double) * (size_t)n);
    i32 *perm = (i32 *)malloc(sizeof(i32) * (size_t)n);
    if (!cdf || !perm) { free(cdf); free(perm); return -1; }
    double acc = 0.0;
    for (i32 r = 1; r <= n; ++r) { acc += pow((double)r, -beta); cdf[r - 1] = acc; }
    for (i32 r = 0; r < n; ++r) cdf[r] /= acc;
    cdf[n - 1] = 2.0; /* every u < 1 lands inside */
    permutation(seed, S_PERM2, n, perm);
    #pragma omp parallel for schedule(dynamic, 64)
    for (i32 i = 0; i < n; ++i) {
        i32 *row = col_idx + row_ptr[i];
        i32 len = row_ptr[i + 1] - row_ptr[i];
        if (len == 0) continue;
        u64 ctr = 0;
        for (i32 k = 0; k < len; ++k) {
            i32 t;
            do { t = perm[search_cdf(cdf, n, unit(draw(seed, STREAM(S_ROW, i), ctr++)))]; } while (t == i);
            row[k] = t;
        }
        /* re-draw duplicates until the row holds len distinct targets */
        for (;;) {
            qsort(row, (size_t)len, sizeof(i32), cmp_i32);
            i32 ndup = 0;
            for (i32 k = 1; k < len; ++k) if (row[k] == row[k - 1]) ++ndup;
            if (ndup == 0) break;
            i32 w = 0;
            for (i32 k = 0; k < len; ++k) if (k == 0 || row[k] != row[k - 1]) row[w++] = row[k];
            for (i32 k = w; k < len; ++k) {
                i32 t;
                do { t = perm[search_cdf(cdf, n, unit(draw(seed, STREAM(S_ROW, i), ctr++)))]; } while (t == i);
                row[k] = t;
            }
        }
    }
    free(cdf); free(perm);
    return 0;
}

/* --------------------------------------------------------------------- rmat */

static inline void rmat_edge(u64 seed, i64 e, int scale, double a, double ab, double abc, i32 *s, i32 *t) {
    u64 src = 0, dst = 0;
    for (int l = 0; l < scale; ++l) {
        double u = unit(draw(seed, STREAM(S_EDGE, e), (u64)l));
        int sb, db;
        if (u < a) { sb = 0; db = 0; }
        else if (u < ab) { sb = 0; db = 1; }
        else if (u < abc) { sb = 1; db = 0; }
        else { sb = 1; db = 1; }
        src = (src << 1) | (u64)sb;
        dst = (dst << 1) | (u64)db;
    }
    *s = (i32)src; *t = (i32)dst;
}

/*
 * R-MAT CSR in one call.  The caller passes row_ptr[n+1] (n = 2^scale) and a
 * col_idx buffer of capacity edge_factor*n; returns the realised edge count L
 * (<= capacity) or -1.  Rows are sorted; with dedup != 0 duplicates are removed.
 */
i64 gg_rmat(int scale, i32 edge_factor, double a, double b, double c, u64 seed, int dedup,
            i32 *row_ptr, i32 *col_idx) {
    if (scale < 1 || scale > 30 || edge_factor < 1) return -1;
    i64 n = (i64)1 << scale;
    i64 m = (i64)edge_factor * n;
    if (m > INT32_MAX) return -1;
    double ab = a + b, abc = a + b + c;
    i32 *src = (i32 *)malloc(sizeof(i32) * (size_t)m);
    i32 *dst = (i32 *)malloc(sizeof(i32) * (size_t)m);
    i32 *cnt = (i32 *)calloc((size_t)n + 1, sizeof(i32));
    if (!src || !dst || !cnt) { free(src); free(dst); free(cnt); return -1; }
    #pragma omp parallel for schedule(static)
    for (i64 e = 0; e < m; ++e) rmat_edge(seed, e, scale, a, ab, abc, &src[e], &dst[e]);
    for (i64 e = 0; e < m; ++e) cnt[src[e]]++;
    i64 acc = 0;
    for (i64 i = 0; i < n; ++i) { i32 cdeg = cnt[i]; row_ptr[i] = (i32)acc; acc += cdeg; }
    row_ptr[n] = (i32)acc;
    /* fill rows in edge order (sequential: stable and deterministic) */
    memset(cnt, 0, sizeof(i32) * (size_t)(n + 1));
    for (i64 e = 0; e < m; ++e) { i32 s = src[e]; col_idx[row_ptr[s] + cnt[s]++] = dst[e]; }
    free(src); free(dst);
    #pragma omp parallel for schedule(dynamic, 1024)
    for (i64 i = 0; i < n; ++i) {
        i32 len = row_ptr[i + 1] - row_ptr[i];
        qsort(col_idx + row_ptr[i], (size_t)len, sizeof(i32), cmp_i32);
    }
    if (dedup) {
        /* compact in place: rows only move left */
        i64 w = 0;
        for (i64 i = 0; i < n; ++i) {
            i32 beg = row_ptr[i], end = row_ptr[i + 1];
            row_ptr[i] = (i32)w;
            for (i32 k = beg; k < end; ++k)
                if (k == beg || col_idx[k] != col_idx[k - 1]) col_idx[w++] = col_idx[k];
        }
        row_ptr[n] = (i32)w;
        acc = w;
    }
    free(cnt);
    return acc;
}

/* ---------------------------------------------------------------- seed sets */

/*
 * Personalization seed sets for query q: size uniform in {smin..smax}, members
 * distinct and uniform over [0,n).  out must hold smax ints; returns the size.
 */
/*
 * An edited copy of a graph (an "updated" web graph): every edge is kept unless
 * its draw falls below drop, and `extra` new edges, drawn as (source, target)
 * pairs uniform over the nodes, are appended to their source rows.  Writes row_ptr2[n+1] and col_idx2
 * (capacity cap); returns the edge count, or -1 if cap is too small.
 */
i64 gg_modify(i32 n, const i32 *row_ptr, const i32 *col_idx, double drop, i64 extra, u64 seed,
              i32 *row_ptr2, i32 *col_idx2, i64 cap) {
    i32 *add = (i32 *)calloc((size_t)n, sizeof(i32));
    for (i64 k = 0; k < extra; ++k) add[below(draw(seed, 21, 2 * (u64)k), (u64)n)] += 1;
    i64 at = 0;
    i64 k_next = 0;
    /* the k-th extra edge goes to the k-th slot of its source, in draw order */
    i32 **tgt = (i32 **)calloc((size_t)n, sizeof(i32 *));
    i32 *fill = (i32 *)calloc((size_t)n, sizeof(i32));
    for (i32 i = 0; i < n; ++i)
        if (add[i]) tgt[i] = (i32 *)malloc(sizeof(i32) * (size_t)add[i]);
    for (; k_next < extra; ++k_next) {
        i32 src = (i32)below(draw(seed, 21, 2 * (u64)k_next), (u64)n);
        tgt[src][fill[src]++] = (i32)below(draw(seed, 21, 2 * (u64)k_next + 1), (u64)n);
    }
    row_ptr2[0] = 0;
    for (i32 i = 0; i < n; ++i) {
        for (i32 e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            if (unit(draw(seed, 20, (u64)e)) < drop) continue;
            if (at >= cap) { at = -1; goto done; }
            col_idx2[at++] = col_idx[e];
        }
        for (i32 k = 0; k < add[i]; ++k) {
            if (at >= cap) { at = -1; goto done; }
            col_idx2[at++] = tgt[i][k];
        }
        row_ptr2[i + 1] = (i32)at;
    }
done:
    for (i32 i = 0; i < n; ++i) free(tgt[i]);
    free(tgt); free(fill); free(add);
    return at;
}

i32 gg_seed_set(i32 n, i32 smin, i32 smax, u64 seed, i64 q, i32 *out) {
    if (n <= 0 || smin < 1 || smax < smin) return -1;
    if (smax > n) smax = n;
    if (smin > smax) smin = smax;
    u64 ctr = 0;
    i32 sz = smin + (i32)below(draw(seed, STREAM(S_SEEDS, q), ctr++), (u64)(smax - smin + 1));
    for (i32 k = 0; k < sz; ++k) {
        for (;;) {
            i32 t = (i32)below(draw(seed, STREAM(S_SEEDS, q), ctr++), (u64)n);
            if (row_contains(out, k, t)) continue;
            out[k] = t;
            break;
        }
    }
    qsort(out, (size_t)sz, sizeof(i32), cmp_i32);
    return sz;
}

/* raw stream access, for tests of the generator itself */
double gg_unit(u64 seed, u64 stream, u64 ctr) { return unit(draw(seed, stream, ctr)); }
