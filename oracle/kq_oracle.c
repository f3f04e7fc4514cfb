/*
 * kq_oracle.c -- plain FP64 CPU reference for exact k-means colour quantization
 * (Weighted Sort-Means, Celebi 2011).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header, table or
 * helper with the CUDA path; the two agree only through the paper and the
 * written readings below.
 *
 * Because the paper states that Weighted Sort-Means gives the same result as
 * conventional k-means from the same centres (Section 2.2), the oracle is the
 * plain definition: dense weighted Lloyd over the unique colours, every distance
 * in FP64, every sum an exact 64-bit integer.  Nothing here is blocked, fused or
 * reordered.
 *
 * Readings where the paper is silent (each one is also listed in the design notes):
 *  - colours are 24-bit keys (R<<16)|(G<<8)|B; the unique colours are kept in
 *    ascending key order;
 *  - weights are integer pixel counts (the paper divides them by N; centres and
 *    the relative convergence test do not change under that scaling);
 *  - ties in every argmin go to the lowest centre index;
 *  - an empty cluster keeps its previous centre;
 *  - SSE_i is the weighted SSE of iteration i's assignment against the centres
 *    that entered iteration i; the run stops after iteration i when
 *    SSE_i == 0 or (i > 1 and (SSE_{i-1} - SSE_i) / SSE_i <= eps); eps < 0
 *    disables the test (a fixed number of iterations, as in Section 3.2);
 *  - when K >= N' every scheme returns the N' unique colours in key order and
 *    fills the remaining centres with copies of the last one;
 *  - random draws use the counter-based SplitMix64 stream defined at
 *    or_rand() and the integer range reduction of or_below().
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_API __attribute__((visibility("default")))

enum { OR_FGY = 0, OR_LBG = 1, OR_MMX = 2, OR_DEN = 3, OR_VAR = 4, OR_SFF = 5, OR_KPP = 6, OR_WU = 8 };

/* ------------------------------------------------------------------------- */
/* Random numbers: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014).  The n-th  */
/* output of the generator seeded with s is mix(s + n * gamma).  Stream `st`   */
/* counter `i` is output number n = st * 2^32 + i + 1.                         */
/* ------------------------------------------------------------------------- */
OR_API uint64_t or_rand(uint64_t seed, uint32_t stream, uint32_t ctr)
{
    uint64_t n = ((uint64_t)stream << 32) + (uint64_t)ctr + 1u;
    uint64_t z = seed + n * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* An integer in [0, m): the high 64 bits of the 128-bit product u * m. */
OR_API uint64_t or_below(uint64_t u, uint64_t m)
{
    return (uint64_t)(((unsigned __int128)u * (unsigned __int128)m) >> 64);
}

static void key_rgb(uint32_t key, int64_t *r, int64_t *g, int64_t *b)
{
    *r = (key >> 16) & 255u;
    *g = (key >> 8) & 255u;
    *b = key & 255u;
}

static int64_t key_dist2(uint32_t a, uint32_t b)
{
    int64_t ar, ag, ab, br, bg, bb;
    key_rgb(a, &ar, &ag, &ab);
    key_rgb(b, &br, &bg, &bb);
    return (ar - br) * (ar - br) + (ag - bg) * (ag - bg) + (ab - bb) * (ab - bb);
}

/* ------------------------------------------------------------------------- */
/* Unique-colour sampling with weights (Section 2.2, items 1 and 2): a count   */
/* per 24-bit colour, then the colours with a nonzero count in ascending key   */
/* order.  Returns N'; writes at most `cap` entries.                           */
/* ------------------------------------------------------------------------- */
OR_API int64_t or_histogram(const uint8_t *rgb, int64_t n, uint32_t *keys, uint32_t *weights, int64_t cap)
{
    uint32_t *cnt = (uint32_t *)calloc((size_t)1 << 24, sizeof(uint32_t));
    if (!cnt) return -1;
    for (int64_t i = 0; i < n; ++i) {
        uint32_t key = ((uint32_t)rgb[3 * i] << 16) | ((uint32_t)rgb[3 * i + 1] << 8) | rgb[3 * i + 2];
        cnt[key] += 1u;
    }
    int64_t u = 0;
    for (uint32_t key = 0; key < (1u << 24); ++key) {
        if (cnt[key]) {
            if (u < cap) {
                keys[u] = key;
                weights[u] = cnt[key];
            }
            ++u;
        }
    }
    free(cnt);
    return u;
}

/* ------------------------------------------------------------------------- */
/* Assignment step (Algorithm 1, the argmin over all K centres; Algorithm 2    */
/* reaches the same labels).  Squared Euclidean distance in FP64, lowest index */
/* on ties.  d1/d2 (nullable) receive the best and second-best distances.      */
/* Returns the weighted SSE of Eq. 1 for this assignment.                      */
/* ------------------------------------------------------------------------- */
OR_API double or_assign(const uint32_t *keys, const uint32_t *w, int64_t n, int K, const double *c,
                        uint8_t *labels, double *d1, double *d2)
{
    double sse = 0.0;
    /* The second build of this file (-fopenmp, used only to time the oracle on
       all host cores) splits the colours over threads; the sum then depends on
       the thread count, so the parity tests use the serial build. */
#ifdef _OPENMP
#pragma omp parallel for reduction(+ : sse) schedule(static)
#endif
    for (int64_t i = 0; i < n; ++i) {
        int64_t r, g, b;
        key_rgb(keys[i], &r, &g, &b);
        double best = INFINITY, second = INFINITY;
        int arg = 0;
        for (int k = 0; k < K; ++k) {
            double dr = (double)r - c[3 * k], dg = (double)g - c[3 * k + 1], db = (double)b - c[3 * k + 2];
            double d = dr * dr + dg * dg + db * db;
            if (d < best) {
                second = best;
                best = d;
                arg = k;
            } else if (d < second) {
                second = d;
            }
        }
        labels[i] = (uint8_t)arg;
        if (d1) d1[i] = best;
        if (d2) d2[i] = second;
        sse += (double)w[i] * best;
    }
    return sse;
}

/* ------------------------------------------------------------------------- */
/* Update step (Algorithm 2, the weighted mean of each cluster): exact int64   */
/* sums S_k = sum w*x and W_k = sum w, then c_k = S_k / W_k in FP64.  An empty */
/* cluster keeps its centre.  sums (nullable) receives K x {S_r,S_g,S_b,W}.    */
/* ------------------------------------------------------------------------- */
OR_API void or_update(const uint32_t *keys, const uint32_t *w, int64_t n, int K, const uint8_t *labels,
                      const double *c_in, double *c_out, int64_t *sums)
{
    int64_t *s = (int64_t *)calloc((size_t)K * 4, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        int64_t r, g, b;
        key_rgb(keys[i], &r, &g, &b);
        int k = labels[i];
        s[4 * k + 0] += (int64_t)w[i] * r;
        s[4 * k + 1] += (int64_t)w[i] * g;
        s[4 * k + 2] += (int64_t)w[i] * b;
        s[4 * k + 3] += (int64_t)w[i];
    }
    for (int k = 0; k < K; ++k) {
        if (s[4 * k + 3] > 0) {
            for (int ch = 0; ch < 3; ++ch) c_out[3 * k + ch] = (double)s[4 * k + ch] / (double)s[4 * k + 3];
        } else {
            for (int ch = 0; ch < 3; ++ch) c_out[3 * k + ch] = c_in[3 * k + ch];
        }
    }
    if (sums) memcpy(sums, s, (size_t)K * 4 * sizeof(int64_t));
    free(s);
}

/* Convergence test of Section 3.3 (Linde, Buzo and Gray): relative SSE drop. */
static int converged_after(int iter, double prev, double cur, double eps)
{
    if (eps < 0.0) return 0;
    if (cur == 0.0) return 1;
    if (iter <= 1) return 0;
    return (prev - cur) / cur <= eps;
}

/* ------------------------------------------------------------------------- */
/* Weighted Lloyd (Algorithm 2 without the pruning, which leaves the result    */
/* unchanged).  centers: in = seeds, out = final.  labels: the last            */
/* assignment.  sse_hist (nullable, max_iter entries).  Returns the number of  */
/* iterations run; *converged is set when the relative test fired.             */
/* ------------------------------------------------------------------------- */
OR_API int or_lloyd(const uint32_t *keys, const uint32_t *w, int64_t n, int K, double *centers, double eps,
                    int max_iter, uint8_t *labels, double *sse_hist, int *converged, int64_t *sums)
{
    double *next = (double *)malloc(sizeof(double) * 3 * (size_t)K);
    double prev = 0.0;
    int it = 0;
    if (converged) *converged = 0;
    while (it < max_iter) {
        double sse = or_assign(keys, w, n, K, centers, labels, NULL, NULL);
        ++it;
        if (sse_hist) sse_hist[it - 1] = sse;
        or_update(keys, w, n, K, labels, centers, next, sums);
        memcpy(centers, next, sizeof(double) * 3 * (size_t)K);
        if (converged_after(it, prev, sse, eps)) {
            if (converged) *converged = 1;
            break;
        }
        prev = sse;
    }
    free(next);
    return it;
}

/* ------------------------------------------------------------------------- */
/* Palette: each centre rounded half-up to 0..255.  For a cluster with pixels  */
/* this is floor((2 S + W) / (2 W)) in exact integers; for an empty cluster it */
/* is floor(c + 0.5) of the held centre, clamped.                              */
/* ------------------------------------------------------------------------- */
OR_API void or_palette(const int64_t *sums, const double *c, int K, uint8_t *pal)
{
    for (int k = 0; k < K; ++k) {
        int64_t W = sums ? sums[4 * k + 3] : 0;
        for (int ch = 0; ch < 3; ++ch) {
            int64_t v;
            if (W > 0) {
                v = (2 * sums[4 * k + ch] + W) / (2 * W);
            } else {
                double f = floor(c[3 * k + ch] + 0.5);
                v = f < 0.0 ? 0 : (f > 255.0 ? 255 : (int64_t)f);
            }
            pal[3 * k + ch] = (uint8_t)v;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Pixel mapping (Section 1: each pixel to its nearest palette colour; Section */
/* 2.1: a full search of the palette) with integer distances and the lowest    */
/* index on ties.  sse_num (nullable) = sum of squared errors, the numerator   */
/* of the MSE of Section 3.1 (Eq. 2).                                          */
/* ------------------------------------------------------------------------- */
OR_API void or_map(const uint8_t *rgb, int64_t n, const uint8_t *pal, int K, uint8_t *idx, int64_t *sse_num)
{
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t best = INT64_MAX;
        int arg = 0;
        for (int k = 0; k < K; ++k) {
            int64_t dr = (int64_t)rgb[3 * i] - pal[3 * k];
            int64_t dg = (int64_t)rgb[3 * i + 1] - pal[3 * k + 1];
            int64_t db = (int64_t)rgb[3 * i + 2] - pal[3 * k + 2];
            int64_t d = dr * dr + dg * dg + db * db;
            if (d < best) {
                best = d;
                arg = k;
            }
        }
        idx[i] = (uint8_t)arg;
        total += best;
    }
    if (sse_num) *sse_num = total;
}

/* ========================================================================= */
/* Seeding: the generic initialization schemes of Section 2.3.                */
/* ========================================================================= */

static void centre_from_key(double *c, uint32_t key)
{
    int64_t r, g, b;
    key_rgb(key, &r, &g, &b);
    c[0] = (double)r;
    c[1] = (double)g;
    c[2] = (double)b;
}

/* Partial Fisher-Yates: the first `count` entries of a uniformly random     */
/* permutation of 0..n-1, drawn from stream `stream`, written to out.        */
static void partial_shuffle(int64_t n, int64_t count, uint64_t seed, uint32_t stream, int64_t *out)
{
    int64_t *a = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) a[i] = i;
    for (int64_t j = 0; j < count; ++j) {
        int64_t r = j + (int64_t)or_below(or_rand(seed, stream, (uint32_t)j), (uint64_t)(n - j));
        int64_t t = a[j];
        a[j] = a[r];
        a[r] = t;
        out[j] = a[j];
    }
    free(a);
}

/* Forgy: K distinct data points drawn uniformly (Algorithm 2, first line). */
static void seed_fgy(const uint32_t *keys, int64_t n, int K, uint64_t seed, double *c)
{
    int64_t *pick = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
    partial_shuffle(n, K, seed, 1, pick);
    for (int k = 0; k < K; ++k) centre_from_key(c + 3 * k, keys[pick[k]]);
    free(pick);
}

/* Minmax over the points `idx[0..m-1]` (ascending unique-colour indices):   */
/* the first centre is idx[first]; each next centre is the point whose       */
/* smallest distance to the chosen centres is largest (lowest index on ties).*/
static void maxmin_select(const uint32_t *keys, const int64_t *idx, int64_t m, int64_t first, int K, double *c)
{
    int64_t *mind = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    int64_t cur = idx[first];
    centre_from_key(c, keys[cur]);
    for (int64_t i = 0; i < m; ++i) mind[i] = INT64_MAX;
    for (int k = 1; k < K; ++k) {
        int64_t best = -1, arg = 0;
        for (int64_t i = 0; i < m; ++i) {
            int64_t d = key_dist2(keys[idx[i]], keys[cur]);
            if (d < mind[i]) mind[i] = d;
            if (mind[i] > best) {
                best = mind[i];
                arg = i;
            }
        }
        cur = idx[arg];
        centre_from_key(c + 3 * k, keys[cur]);
    }
    free(mind);
}

/* Minmax (MMX): first centre uniform over the unique colours. */
static void seed_mmx(const uint32_t *keys, int64_t n, int K, uint64_t seed, double *c)
{
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) idx[i] = i;
    int64_t first = (int64_t)or_below(or_rand(seed, 3, 0), (uint64_t)n);
    maxmin_select(keys, idx, n, first, K, c);
    free(idx);
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* Subset size of Subset Farthest First: min(N', max(K, ceil(2 K ln K))). */
OR_API int64_t or_sff_size(int64_t n, int K)
{
    int64_t s = (int64_t)ceil(2.0 * (double)K * log((double)K));
    if (s < K) s = K;
    if (s > n) s = n;
    return s;
}

/* Subset Farthest First (SFF): minmax on a uniform random subset. */
static void seed_sff(const uint32_t *keys, int64_t n, int K, uint64_t seed, double *c)
{
    int64_t s = or_sff_size(n, K);
    int64_t *sub = (int64_t *)malloc(sizeof(int64_t) * (size_t)s);
    partial_shuffle(n, s, seed, 4, sub);
    qsort(sub, (size_t)s, sizeof(int64_t), cmp_i64);
    int64_t first = (int64_t)or_below(or_rand(seed, 5, 0), (uint64_t)s);
    maxmin_select(keys, sub, s, first, K, c);
    free(sub);
}

/* K-means++ (KPP): first centre drawn with probability w_i / sum w; centre */
/* r drawn with probability w_i D(x_i)^2 / sum w D^2, where D is the        */
/* distance to the nearest chosen centre.  Integer arithmetic throughout:   */
/* t = below(u, total), choose the first i whose running sum exceeds t.     */
static void seed_kpp(const uint32_t *keys, const uint32_t *w, int64_t n, int K, uint64_t seed, double *c)
{
    int64_t *d2 = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) total += (int64_t)w[i];
    int64_t t = (int64_t)or_below(or_rand(seed, 2, 0), (uint64_t)total), run = 0, cur = n - 1;
    for (int64_t i = 0; i < n; ++i) {
        run += (int64_t)w[i];
        if (run > t) {
            cur = i;
            break;
        }
    }
    centre_from_key(c, keys[cur]);
    for (int64_t i = 0; i < n; ++i) d2[i] = INT64_MAX;
    for (int k = 1; k < K; ++k) {
        total = 0;
        for (int64_t i = 0; i < n; ++i) {
            int64_t d = key_dist2(keys[i], keys[cur]);
            if (d < d2[i]) d2[i] = d;
            total += (int64_t)w[i] * d2[i];
        }
        t = (int64_t)or_below(or_rand(seed, 2, (uint32_t)k), (uint64_t)total);
        run = 0;
        cur = n - 1;
        for (int64_t i = 0; i < n; ++i) {
            run += (int64_t)w[i] * d2[i];
            if (run > t) {
                cur = i;
                break;
            }
        }
        centre_from_key(c + 3 * k, keys[cur]);
    }
    free(d2);
}

/* Maximum variance (VAR): the channel of largest pixel-weighted variance     */
/* (compared exactly as W*sum(w x^2) - (sum w x)^2, ties to R, then G); the   */
/* unique colours sorted ascending on it (ties by key); K equal-count groups  */
/* [floor(g N'/K), floor((g+1) N'/K)); each centre is the group's middle     */
/* element, index floor((lo + hi - 1) / 2).                                  */
static const uint32_t *g_sort_keys;
static int g_sort_shift;
static int cmp_channel(const void *a, const void *b)
{
    uint32_t ka = g_sort_keys[*(const int64_t *)a], kb = g_sort_keys[*(const int64_t *)b];
    uint32_t va = (ka >> g_sort_shift) & 255u, vb = (kb >> g_sort_shift) & 255u;
    if (va != vb) return va < vb ? -1 : 1;
    return (ka > kb) - (ka < kb);
}

OR_API int or_var_channel(const uint32_t *keys, const uint32_t *w, int64_t n)
{
    __int128 W = 0, s1[3] = {0, 0, 0}, s2[3] = {0, 0, 0};
    for (int64_t i = 0; i < n; ++i) {
        int64_t x[3];
        key_rgb(keys[i], &x[0], &x[1], &x[2]);
        W += w[i];
        for (int ch = 0; ch < 3; ++ch) {
            s1[ch] += (__int128)w[i] * x[ch];
            s2[ch] += (__int128)w[i] * x[ch] * x[ch];
        }
    }
    int best = 0;
    __int128 bv = W * s2[0] - s1[0] * s1[0];
    for (int ch = 1; ch < 3; ++ch) {
        __int128 v = W * s2[ch] - s1[ch] * s1[ch];
        if (v > bv) {
            bv = v;
            best = ch;
        }
    }
    return best;
}

static void seed_var(const uint32_t *keys, const uint32_t *w, int64_t n, int K, double *c)
{
    int ch = or_var_channel(keys, w, n);
    int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) ord[i] = i;
    g_sort_keys = keys;
    g_sort_shift = 16 - 8 * ch;
    qsort(ord, (size_t)n, sizeof(int64_t), cmp_channel);
    for (int g = 0; g < K; ++g) {
        int64_t lo = (int64_t)g * n / K, hi = (int64_t)(g + 1) * n / K;
        centre_from_key(c + 3 * g, keys[ord[(lo + hi - 1) / 2]]);
    }
    free(ord);
}

/* Density-based (DEN): 64 uniform cells (4 levels per channel, cell index    */
/* (R>>6)*16 + (G>>6)*4 + (B>>6)).  Seats are apportioned to cells in          */
/* proportion to their pixel counts by largest remainder (ties to the lower    */
/* cell); a cell whose share exceeds its unique-colour count is fixed at that  */
/* count and the rest is apportioned again among the other cells.  Inside each */
/* cell the centres are a uniform draw without replacement (stream 16 + cell). */
OR_API void or_den_quota(const int64_t *cellw, const int64_t *celln, int K, int64_t *q)
{
    int fixed[64];
    memset(fixed, 0, sizeof(fixed));
    for (;;) {
        int64_t seats = K, wa = 0;
        for (int c = 0; c < 64; ++c) {
            if (fixed[c]) seats -= celln[c];
            else if (celln[c] > 0) wa += cellw[c];
        }
        int64_t rem[64], given = 0;
        for (int c = 0; c < 64; ++c) {
            q[c] = 0;
            rem[c] = -1;
            if (fixed[c]) {
                q[c] = celln[c];
            } else if (celln[c] > 0 && wa > 0) {
                q[c] = seats * cellw[c] / wa;
                rem[c] = seats * cellw[c] % wa;
                given += q[c];
            }
        }
        for (int64_t left = seats - given; left > 0; --left) {
            int arg = -1;
            for (int c = 0; c < 64; ++c)
                if (rem[c] >= 0 && (arg < 0 || rem[c] > rem[arg])) arg = c;
            q[arg] += 1;
            rem[arg] = -1;
        }
        int grew = 0;
        for (int c = 0; c < 64; ++c) {
            if (!fixed[c] && q[c] > celln[c]) {
                fixed[c] = 1;
                grew = 1;
            }
        }
        if (!grew) return;
    }
}

static int den_cell(uint32_t key)
{
    return (int)(((key >> 22) & 3u) * 16u + ((key >> 14) & 3u) * 4u + ((key >> 6) & 3u));
}

static void seed_den(const uint32_t *keys, const uint32_t *w, int64_t n, int K, uint64_t seed, double *c)
{
    int64_t cellw[64], celln[64], q[64];
    memset(cellw, 0, sizeof(cellw));
    memset(celln, 0, sizeof(celln));
    for (int64_t i = 0; i < n; ++i) {
        int cc = den_cell(keys[i]);
        cellw[cc] += (int64_t)w[i];
        celln[cc] += 1;
    }
    or_den_quota(cellw, celln, K, q);
    int k = 0;
    for (int cc = 0; cc < 64; ++cc) {
        if (q[cc] == 0) continue;
        int64_t *members = (int64_t *)malloc(sizeof(int64_t) * (size_t)celln[cc]);
        int64_t *pick = (int64_t *)malloc(sizeof(int64_t) * (size_t)q[cc]);
        int64_t m = 0;
        for (int64_t i = 0; i < n; ++i)
            if (den_cell(keys[i]) == cc) members[m++] = i;
        partial_shuffle(m, q[cc], seed, 16u + (uint32_t)cc, pick);
        for (int64_t j = 0; j < q[cc]; ++j) centre_from_key(c + 3 * (k++), keys[members[pick[j]]]);
        free(members);
        free(pick);
    }
}

/* Exact per-cluster SSE about the cluster mean, as the fraction num / W with  */
/* num = W * sum(w |x|^2) - |S|^2.  Used to rank clusters for a partial split. */
static int sse_greater(__int128 na, int64_t wa, __int128 nb, int64_t wb)
{
    /* compare na/wa > nb/wb with wa, wb > 0 (an empty cluster ranks lowest) */
    if (wa == 0) return 0;
    if (wb == 0) return 1;
    /* na * wb and nb * wa stay below 2^127 for images up to 2^26 pixels */
    return na * (__int128)wb > nb * (__int128)wa;
}

/* Splitting (LBG): the centroid, then each centre c split into c - eps and    */
/* c + eps (c - eps keeps index j, c + eps takes index m + j), each round       */
/* refined by full Lloyd.  When K is not a power of two the last round splits   */
/* only the K - m clusters of largest weighted SSE (ties to the lower index),   */
/* taken in ascending index order.                                              */
static void seed_lbg(const uint32_t *keys, const uint32_t *w, int64_t n, int K, double lbg_eps, double conv_eps,
                     int max_iter, double *c)
{
    uint8_t *labels = (uint8_t *)malloc((size_t)n);
    int64_t *sums = (int64_t *)calloc((size_t)K * 4, sizeof(int64_t));
    int64_t W = 0, s[3] = {0, 0, 0};
    for (int64_t i = 0; i < n; ++i) {
        int64_t x[3];
        key_rgb(keys[i], &x[0], &x[1], &x[2]);
        W += (int64_t)w[i];
        for (int ch = 0; ch < 3; ++ch) s[ch] += (int64_t)w[i] * x[ch];
    }
    for (int ch = 0; ch < 3; ++ch) c[ch] = (double)s[ch] / (double)W;
    int m = 1;
    while (m < K) {
        int split = (2 * m <= K) ? m : K - m;
        int *chosen = (int *)malloc(sizeof(int) * (size_t)m);
        if (split == m) {
            for (int j = 0; j < m; ++j) chosen[j] = 1;
        } else {
            /* rank clusters of the current assignment by exact SSE */
            __int128 *num = (__int128 *)calloc((size_t)m, sizeof(__int128));
            int64_t *cw = (int64_t *)calloc((size_t)m, sizeof(int64_t));
            int64_t *cs = (int64_t *)calloc((size_t)m * 3, sizeof(int64_t));
            __int128 *sq = (__int128 *)calloc((size_t)m, sizeof(__int128));
            for (int64_t i = 0; i < n; ++i) {
                int64_t x[3];
                key_rgb(keys[i], &x[0], &x[1], &x[2]);
                int k = labels[i];
                cw[k] += (int64_t)w[i];
                for (int ch = 0; ch < 3; ++ch) cs[3 * k + ch] += (int64_t)w[i] * x[ch];
                sq[k] += (__int128)w[i] * (x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
            }
            for (int k = 0; k < m; ++k) {
                __int128 s2 = 0;
                for (int ch = 0; ch < 3; ++ch) s2 += (__int128)cs[3 * k + ch] * cs[3 * k + ch];
                num[k] = (__int128)cw[k] * sq[k] - s2;
            }
            for (int j = 0; j < m; ++j) chosen[j] = 0;
            for (int t = 0; t < split; ++t) {
                int arg = -1;
                for (int k = 0; k < m; ++k) {
                    if (chosen[k]) continue;
                    if (arg < 0 || sse_greater(num[k], cw[k], num[arg], cw[arg])) arg = k;
                }
                chosen[arg] = 1;
            }
            free(num);
            free(cw);
            free(cs);
            free(sq);
        }
        int q = 0;
        for (int j = 0; j < m; ++j) {
            if (!chosen[j]) continue;
            for (int ch = 0; ch < 3; ++ch) {
                double base = c[3 * j + ch];
                c[3 * (m + q) + ch] = base + lbg_eps;
                c[3 * j + ch] = base - lbg_eps;
            }
            ++q;
        }
        free(chosen);
        m += split;
        or_lloyd(keys, w, n, m, c, conv_eps, max_iter, labels, NULL, NULL, sums);
    }
    free(labels);
    free(sums);
}

/* ------------------------------------------------------------------------- */
/* WU: greedy orthogonal bipartitioning (Wu 1991), the preclustering method   */
/* of Section 3.3 that initializes WSM-WU.  Colours fall in a 32 x 32 x 32     */
/* grid of cells (5 bits per channel).  A box is a range of cells [lo, hi) on  */
/* each axis.  Starting from the whole grid, the box with the largest weighted */
/* variance (sum over its colours of w |x - mean|^2) is split by the           */
/* axis-aligned cut between cells that minimizes the sum of the two halves'    */
/* variances -- equivalently, maximizes |S_a|^2/W_a + |S_b|^2/W_b -- until K   */
/* boxes exist or no box can be split.  The centres are the box means.         */
/* Readings: the moments use the colours' full 8-bit values; ties go to the    */
/* lower box index, to R before G before B and to the lower cut position; a    */
/* cut must leave pixels on both sides; a box that cannot be cut gets variance */
/* 0; when fewer than K boxes result, the remaining centres copy the last      */
/* box's mean.  FP64 evaluation order: term(m) = ((Sr*Sr + Sg*Sg) + Sb*Sb)/W   */
/* with every operation rounded, criterion = term(a) + term(b), variance =     */
/* Q - term(m).  Box moments here are plain sums over the box's cells.         */
/* ------------------------------------------------------------------------- */
typedef struct {
    int lo[3], hi[3];
} wu_box;

typedef struct {
    int64_t w, s[3], q;
} wu_mom;

static int wu_cell(uint32_t key)
{
    return (int)(((key >> 19) & 31u) * 1024u + ((key >> 11) & 31u) * 32u + ((key >> 3) & 31u));
}

static void wu_add(wu_mom *a, const wu_mom *b)
{
    a->w += b->w;
    a->q += b->q;
    for (int ch = 0; ch < 3; ++ch) a->s[ch] += b->s[ch];
}

static void wu_sub(wu_mom *out, const wu_mom *a, const wu_mom *b)
{
    out->w = a->w - b->w;
    out->q = a->q - b->q;
    for (int ch = 0; ch < 3; ++ch) out->s[ch] = a->s[ch] - b->s[ch];
}

static void wu_moments(const wu_mom *cell, const wu_box *b, wu_mom *m)
{
    memset(m, 0, sizeof(*m));
    for (int r = b->lo[0]; r < b->hi[0]; ++r)
        for (int g = b->lo[1]; g < b->hi[1]; ++g)
            for (int bb = b->lo[2]; bb < b->hi[2]; ++bb) wu_add(m, &cell[r * 1024 + g * 32 + bb]);
}

static double wu_term(const wu_mom *m)
{
    const double sr = (double)m->s[0], sg = (double)m->s[1], sb = (double)m->s[2];
    return ((sr * sr + sg * sg) + sb * sb) / (double)m->w;
}

static double wu_variance(const wu_mom *cell, const wu_box *b)
{
    const int vol = (b->hi[0] - b->lo[0]) * (b->hi[1] - b->lo[1]) * (b->hi[2] - b->lo[2]);
    if (vol <= 1) return 0.0;
    wu_mom m;
    wu_moments(cell, b, &m);
    if (m.w == 0) return 0.0;
    return (double)m.q - wu_term(&m);
}

OR_API int or_wu(const uint32_t *keys, const uint32_t *w, int64_t n, int K, double *c)
{
    if (n <= 0 || K <= 0) return -1;
    wu_mom *cell = (wu_mom *)calloc(32768, sizeof(wu_mom));
    wu_box *box = (wu_box *)malloc((size_t)K * sizeof(wu_box));
    double *vv = (double *)malloc((size_t)K * sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        int64_t r, g, b;
        key_rgb(keys[i], &r, &g, &b);
        wu_mom *m = &cell[wu_cell(keys[i])];
        m->w += w[i];
        m->s[0] += (int64_t)w[i] * r;
        m->s[1] += (int64_t)w[i] * g;
        m->s[2] += (int64_t)w[i] * b;
        m->q += (int64_t)w[i] * (r * r + g * g + b * b);
    }
    for (int ax = 0; ax < 3; ++ax) {
        box[0].lo[ax] = 0;
        box[0].hi[ax] = 32;
    }
    vv[0] = wu_variance(cell, &box[0]);
    int nb = 1, next = 0;
    while (nb < K && vv[next] > 0.0) {
        wu_mom whole;
        wu_moments(cell, &box[next], &whole);
        double best = -1.0;
        int bax = -1, bpos = -1;
        for (int ax = 0; ax < 3; ++ax) {
            wu_mom half;
            memset(&half, 0, sizeof(half));
            for (int p = box[next].lo[ax] + 1; p < box[next].hi[ax]; ++p) {
                /* half = the box's cells with coordinate < p on this axis */
                wu_box slab = box[next];
                slab.lo[ax] = p - 1;
                slab.hi[ax] = p;
                wu_mom plane;
                wu_moments(cell, &slab, &plane);
                wu_add(&half, &plane);
                wu_mom rest;
                wu_sub(&rest, &whole, &half);
                if (half.w == 0 || rest.w == 0) continue;
                const double f = wu_term(&half) + wu_term(&rest);
                if (f > best) {
                    best = f;
                    bax = ax;
                    bpos = p;
                }
            }
        }
        if (bax < 0) {
            vv[next] = 0.0;
        } else {
            box[nb] = box[next];
            box[nb].lo[bax] = bpos;
            box[next].hi[bax] = bpos;
            vv[next] = wu_variance(cell, &box[next]);
            vv[nb] = wu_variance(cell, &box[nb]);
            ++nb;
        }
        next = 0;
        for (int k = 1; k < nb; ++k)
            if (vv[k] > vv[next]) next = k;
    }
    for (int k = 0; k < nb; ++k) {
        wu_mom m;
        wu_moments(cell, &box[k], &m);
        for (int ch = 0; ch < 3; ++ch) c[3 * k + ch] = (double)m.s[ch] / (double)m.w;
    }
    for (int k = nb; k < K; ++k) memcpy(c + 3 * k, c + 3 * (nb - 1), 3 * sizeof(double));
    free(cell);
    free(box);
    free(vv);
    return nb;
}

/* ------------------------------------------------------------------------- */
/* Entry point for seeding.  K_eff = min(K, N'); for K >= N' the centres are   */
/* the unique colours in key order, padded with copies of the last one.        */
/* Returns K_eff, or -1 for an unknown scheme.                                 */
/* ------------------------------------------------------------------------- */
OR_API int or_seed(const uint32_t *keys, const uint32_t *w, int64_t n, int K, int scheme, uint64_t seed,
                   double lbg_eps, double conv_eps, int max_iter, double *c)
{
    if (n <= 0 || K <= 0) return -1;
    if (K >= n) {
        for (int64_t i = 0; i < n; ++i) centre_from_key(c + 3 * i, keys[i]);
        for (int k = (int)n; k < K; ++k) memcpy(c + 3 * k, c + 3 * (n - 1), 3 * sizeof(double));
        return (int)n;
    }
    switch (scheme) {
    case OR_FGY: seed_fgy(keys, n, K, seed, c); break;
    case OR_LBG: seed_lbg(keys, w, n, K, lbg_eps, conv_eps, max_iter, c); break;
    case OR_MMX: seed_mmx(keys, n, K, seed, c); break;
    case OR_DEN: seed_den(keys, w, n, K, seed, c); break;
    case OR_VAR: seed_var(keys, w, n, K, c); break;
    case OR_SFF: seed_sff(keys, n, K, seed, c); break;
    case OR_KPP: seed_kpp(keys, w, n, K, seed, c); break;
    case OR_WU: or_wu(keys, w, n, K, c); break;
    default: return -1;
    }
    return K;
}

/* ========================================================================= */
/* CIE L*a*b* (Section 2.1 names L*a*b* beside RGB as a colour space for      */
/* k-means).  An 8-bit sRGB colour (IEC 61966-2-1) is made linear, taken to   */
/* CIE XYZ by the sRGB matrix (D65), and to CIE 1976 L*a*b* relative to the   */
/* D65 white.  Points are kept in fixed point, OR_LAB_SCALE units per         */
/* L*a*b* unit (rounded to nearest, ties to even), so that the weighted sums  */
/* of a cluster stay exact integers as in RGB.                                */
/* ========================================================================= */
#define OR_LAB_SCALE 256.0

static double srgb_linear(int v8)
{
    double v = (double)v8 / 255.0;
    return v <= 0.04045 ? v / 12.92 : pow((v + 0.055) / 1.055, 2.4);
}

static double lab_f(double t)
{
    const double d = 6.0 / 29.0;
    return t > d * d * d ? cbrt(t) : t / (3.0 * d * d) + 4.0 / 29.0;
}

static double lab_finv(double t)
{
    const double d = 6.0 / 29.0;
    return t > d ? t * t * t : 3.0 * d * d * (t - 4.0 / 29.0);
}

/* L*, a*, b* of one 24-bit colour (FP64, every operation separately rounded). */
OR_API void or_lab(uint32_t key, double *lab)
{
    int64_t r8, g8, b8;
    key_rgb(key, &r8, &g8, &b8);
    double r = srgb_linear((int)r8), g = srgb_linear((int)g8), b = srgb_linear((int)b8);
    double X = (0.4124564 * r + 0.3575761 * g) + 0.1804375 * b;
    double Y = (0.2126729 * r + 0.7151522 * g) + 0.0721750 * b;
    double Z = (0.0193339 * r + 0.1191920 * g) + 0.9503041 * b;
    double fx = lab_f(X / 0.95047), fy = lab_f(Y / 1.0), fz = lab_f(Z / 1.08883);
    lab[0] = 116.0 * fy - 16.0;
    lab[1] = 500.0 * (fx - fy);
    lab[2] = 200.0 * (fy - fz);
}

/* Fixed-point L*a*b* points of n colours: pts[4 i + c] = rint(lab_c * 256), c < 3; pts[4 i + 3] = 0. */
OR_API void or_lab_points(const uint32_t *keys, int64_t n, int32_t *pts)
{
    for (int64_t i = 0; i < n; ++i) {
        double lab[3];
        or_lab(keys[i], lab);
        for (int c = 0; c < 3; ++c) pts[4 * i + c] = (int32_t)llrint(lab[c] * OR_LAB_SCALE);
        pts[4 * i + 3] = 0;
    }
}

/* The sRGB colour of each of K centres given in fixed-point L*a*b* units: the  */
/* inverse of or_lab, each channel clamped to [0, 1] and rounded half up to     */
/* 0..255.                                                                      */
OR_API void or_lab_palette(const double *centers, int K, uint8_t *pal)
{
    for (int k = 0; k < K; ++k) {
        double L = centers[3 * k] / OR_LAB_SCALE, a = centers[3 * k + 1] / OR_LAB_SCALE,
               bb = centers[3 * k + 2] / OR_LAB_SCALE;
        double fy = (L + 16.0) / 116.0;
        double fx = fy + a / 500.0, fz = fy - bb / 200.0;
        double X = 0.95047 * lab_finv(fx), Y = 1.0 * lab_finv(fy), Z = 1.08883 * lab_finv(fz);
        double lin[3];
        lin[0] = (3.2404542 * X - 1.5371385 * Y) - 0.4985314 * Z;
        lin[1] = (-0.9692660 * X + 1.8760108 * Y) + 0.0415560 * Z;
        lin[2] = (0.0556434 * X - 0.2040259 * Y) + 1.0572252 * Z;
        for (int c = 0; c < 3; ++c) {
            double v = lin[c];
            v = v <= 0.0031308 ? 12.92 * v : 1.055 * pow(v, 1.0 / 2.4) - 0.055;
            v = v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
            pal[3 * k + c] = (uint8_t)floor(v * 255.0 + 0.5);
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Weighted Lloyd on fixed-point 3-D points (L*a*b* here): the steps of        */
/* or_assign / or_update / or_lloyd with the point's three integer coordinates */
/* in place of a colour's three bytes.  Distances in FP64, sums exact int64.   */
/* ------------------------------------------------------------------------- */
OR_API double or_assign_points(const int32_t *pts, const uint32_t *w, int64_t n, int K, const double *c,
                               uint8_t *labels, double *d1, double *d2)
{
    double sse = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double best = INFINITY, second = INFINITY;
        int arg = 0;
        for (int k = 0; k < K; ++k) {
            double dx = (double)pts[4 * i] - c[3 * k], dy = (double)pts[4 * i + 1] - c[3 * k + 1],
                   dz = (double)pts[4 * i + 2] - c[3 * k + 2];
            double d = dx * dx + dy * dy + dz * dz;
            if (d < best) {
                second = best;
                best = d;
                arg = k;
            } else if (d < second) {
                second = d;
            }
        }
        labels[i] = (uint8_t)arg;
        if (d1) d1[i] = best;
        if (d2) d2[i] = second;
        sse += (double)w[i] * best;
    }
    return sse;
}

OR_API void or_update_points(const int32_t *pts, const uint32_t *w, int64_t n, int K, const uint8_t *labels,
                             const double *c_in, double *c_out, int64_t *sums)
{
    int64_t *s = (int64_t *)calloc((size_t)K * 4, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        int k = labels[i];
        for (int ch = 0; ch < 3; ++ch) s[4 * k + ch] += (int64_t)w[i] * (int64_t)pts[4 * i + ch];
        s[4 * k + 3] += (int64_t)w[i];
    }
    for (int k = 0; k < K; ++k) {
        for (int ch = 0; ch < 3; ++ch)
            c_out[3 * k + ch] = s[4 * k + 3] > 0 ? (double)s[4 * k + ch] / (double)s[4 * k + 3] : c_in[3 * k + ch];
    }
    if (sums) memcpy(sums, s, (size_t)K * 4 * sizeof(int64_t));
    free(s);
}

OR_API int or_lloyd_points(const int32_t *pts, const uint32_t *w, int64_t n, int K, double *centers, double eps,
                           int max_iter, uint8_t *labels, double *sse_hist, int *converged, int64_t *sums)
{
    double *next = (double *)malloc(sizeof(double) * 3 * (size_t)K);
    double prev = 0.0;
    int it = 0;
    if (converged) *converged = 0;
    while (it < max_iter) {
        double sse = or_assign_points(pts, w, n, K, centers, labels, NULL, NULL);
        ++it;
        if (sse_hist) sse_hist[it - 1] = sse;
        or_update_points(pts, w, n, K, labels, centers, next, sums);
        memcpy(centers, next, sizeof(double) * 3 * (size_t)K);
        if (converged_after(it, prev, sse, eps)) {
            if (converged) *converged = 1;
            break;
        }
        prev = sse;
    }
    free(next);
    return it;
}

/* Forgy seeds among the points: the K indices or_seed's Forgy draws (stream 1), */
/* each centre that point's coordinates; K >= n gives the n points in order,     */
/* padded with copies of the last.                                               */
OR_API void or_seed_points_fgy(const int32_t *pts, int64_t n, int K, uint64_t seed, double *c)
{
    if ((int64_t)K >= n) {
        for (int k = 0; k < K; ++k)
            for (int ch = 0; ch < 3; ++ch)
                c[3 * k + ch] = n == 0 ? 0.0 : (double)pts[4 * (k < n ? k : n - 1) + ch];
        return;
    }
    int64_t *pick = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
    partial_shuffle(n, K, seed, 1, pick);
    for (int k = 0; k < K; ++k)
        for (int ch = 0; ch < 3; ++ch) c[3 * k + ch] = (double)pts[4 * pick[k] + ch];
    free(pick);
}
