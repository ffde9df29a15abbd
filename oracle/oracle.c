/*
 * Oracle for the level-blocked matrix power kernel (MPK) of
 * "Cache Blocking of Distributed-Memory Parallel Matrix Power Kernels" (Lacey et al.).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code, header or
 * helper with the CUDA library; it is plain, slow, serial C written to be checked
 * against the paper by eye.
 *
 * Floating point: every row sum is evaluated in the stored order of the row, one
 * rounding per term, as s <- fma(a_ij, x_j, s) starting from s = +0.0 (C99 fma,
 * correctly rounded).  Build with -ffp-contract=off so that no other expression is
 * fused behind our back.
 *
 * Index conventions: CSR with int32 row pointers (n+1) and column indices; dense
 * blocks are n x m row-major (the m right-hand sides of one row are contiguous);
 * the power sequence Y is (p+1) x n x m with Y[0] = X.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 3

/* One row of y = A x for m right-hand sides (Sec. 3: y_k = A x with x = y_{k-1}). */
static void row_times_block(const int32_t *rp, const int32_t *ci, const double *va, int32_t m,
                            const double *x, int64_t i, double *y)
{
    for (int32_t r = 0; r < m; ++r) y[r] = 0.0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
        const double a = va[e];
        const double *xr = x + (int64_t)ci[e] * m;
        for (int32_t r = 0; r < m; ++r) y[r] = fma(a, xr[r], y[r]);
    }
}

/*
 * Matrix power kernel, Sec. 3 and Alg. 1 without the halo exchange: y_0 = x and
 * y_k = A y_{k-1} for k = 1..p ("back-to-back SpMVs", the definition of MPK).
 * Y must hold (p+1)*n*m doubles.
 */
int orc_mpk(int32_t n, const int32_t *rp, const int32_t *ci, const double *va, int32_t m,
            const double *X, int32_t p, double *Y)
{
    if (n < 0 || m < 1 || p < 0) return ORC_EINVAL;
    const int64_t nm = (int64_t)n * m;
    memcpy(Y, X, sizeof(double) * (size_t)nm);
    for (int32_t k = 1; k <= p; ++k) {
        const double *xin = Y + (int64_t)(k - 1) * nm;
        double *yout = Y + (int64_t)k * nm;
        for (int64_t i = 0; i < n; ++i) row_times_block(rp, ci, va, m, xin, i, yout + i * m);
    }
    return ORC_OK;
}

/*
 * orc_mpk with the rows of each power shared out over the host's cores (OpenMP, when the
 * oracle is built with it): the same row body, so the same bits as orc_mpk.  A timing leg of
 * the CPU baseline only; the tests check it against orc_mpk.  *threads receives the number of
 * threads that ran.
 */
int orc_mpk_omp(int32_t n, const int32_t *rp, const int32_t *ci, const double *va, int32_t m,
                const double *X, int32_t p, double *Y, int32_t *threads)
{
    if (n < 0 || m < 1 || p < 0) return ORC_EINVAL;
    const int64_t nm = (int64_t)n * m;
    memcpy(Y, X, sizeof(double) * (size_t)nm);
    int32_t used = 1;
    for (int32_t k = 1; k <= p; ++k) {
        const double *xin = Y + (int64_t)(k - 1) * nm;
        double *yout = Y + (int64_t)k * nm;
#ifdef _OPENMP
#pragma omp parallel
        {
#pragma omp single
            used = omp_get_num_threads();
#pragma omp for schedule(static)
            for (int64_t i = 0; i < n; ++i) row_times_block(rp, ci, va, m, xin, i, yout + i * m);
        }
#else
        for (int64_t i = 0; i < n; ++i) row_times_block(rp, ci, va, m, xin, i, yout + i * m);
#endif
    }
    *threads = used;
    return ORC_OK;
}

/*
 * Host load bandwidth, for the context line of the CPU baseline (the paper's roofline of
 * Sec. 6 takes the saturated load bandwidth b_s): `reps` sums over buf[0..n) by all
 * threads; returns the sum so that the loads cannot be dropped.
 */
double orc_load_sum(const double *buf, int64_t n, int32_t reps)
{
    double total = 0.0;
    for (int32_t r = 0; r < reps; ++r) {
        double s = 0.0;
#ifdef _OPENMP
#pragma omp parallel for reduction(+ : s) schedule(static)
#endif
        for (int64_t i = 0; i < n; ++i) s += buf[i];
        total += s;
    }
    return total;
}

/*
 * Single-precision accumulation of the same powers (Sec. 3's MPK, y_k = A y_{k-1}, with a
 * narrower arithmetic): the vectors stay binary64, each row sum runs in binary32 over the
 * binary32 roundings of its inputs, and its result is stored widened (exactly) to binary64:
 *     s = +0.0f;  s = fmaf(a_ij, (float) y_{k-1}[j], s)   in stored order,   y_k[i] = (double) s,
 * (float) rounding to nearest-even and fmaf rounding once.  From power 2 on the inputs are
 * widened binary32 values, so only X is actually rounded.  The matrix values must be exact
 * in binary32 (va holds them as doubles; each converts exactly); ORC_EINVAL otherwise.
 */
int orc_mpk_acc32(int32_t n, const int32_t *rp, const int32_t *ci, const double *va, int32_t m,
                  const double *X, int32_t p, double *Y)
{
    if (n < 0 || m < 1 || p < 0) return ORC_EINVAL;
    for (int64_t e = 0; e < (n > 0 ? rp[n] : 0); ++e)
        if ((double)(float)va[e] != va[e]) return ORC_EINVAL;
    const int64_t nm = (int64_t)n * m;
    float *xf = malloc(sizeof(float) * (size_t)(nm > 0 ? nm : 1));
    float *s = malloc(sizeof(float) * (size_t)m);
    if (!xf || !s) { free(xf); free(s); return ORC_ENOMEM; }
    memcpy(Y, X, sizeof(double) * (size_t)nm);
    for (int32_t k = 1; k <= p; ++k) {
        const double *xin = Y + (int64_t)(k - 1) * nm;
        double *yout = Y + (int64_t)k * nm;
        for (int64_t t = 0; t < nm; ++t) xf[t] = (float)xin[t];
        for (int64_t i = 0; i < n; ++i) {
            for (int32_t r = 0; r < m; ++r) s[r] = 0.0f;
            for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
                const float a = (float)va[e];
                const float *xr = xf + (int64_t)ci[e] * m;
                for (int32_t r = 0; r < m; ++r) s[r] = fmaf(a, xr[r], s[r]);
            }
            for (int32_t r = 0; r < m; ++r) yout[i * m + r] = (double)s[r];
        }
    }
    free(xf); free(s);
    return ORC_OK;
}

/*
 * Same powers accumulated in long double with separate multiply and add: an
 * independent, more precise evaluation used only to bound the rounding error of
 * orc_mpk on small cases.
 */
int orc_mpk_longdouble(int32_t n, const int32_t *rp, const int32_t *ci, const double *va,
                       const double *x, int32_t p, double *Y)
{
    if (n < 0 || p < 0) return ORC_EINVAL;
    long double *a = malloc(sizeof(long double) * (size_t)(n > 0 ? n : 1));
    long double *b = malloc(sizeof(long double) * (size_t)(n > 0 ? n : 1));
    if (!a || !b) { free(a); free(b); return ORC_ENOMEM; }
    for (int64_t i = 0; i < n; ++i) { a[i] = x[i]; Y[i] = x[i]; }
    for (int32_t k = 1; k <= p; ++k) {
        for (int64_t i = 0; i < n; ++i) {
            long double s = 0.0L;
            for (int64_t e = rp[i]; e < rp[i + 1]; ++e) s += (long double)va[e] * a[ci[e]];
            b[i] = s;
            Y[(int64_t)k * n + i] = (double)s;
        }
        long double *t = a; a = b; b = t;
    }
    free(a); free(b);
    return ORC_OK;
}

/*
 * BFS levels of the graph G(A) (Sec. 3, the level definition and its prose):
 *  - the graph is the pattern of A + A^T without self-loops; values are ignored and
 *    a non-symmetric A is treated as symmetric in the graph only (Sec. 3 endnote);
 *  - L(0) = {root}; L(i+1) = neighbours of L(i) not yet touched;
 *  - if the search runs dry with vertices left (a disconnected graph, on which the
 *    paper is silent), the smallest untouched vertex starts the next level;
 *  - the permutation ("BFS reordering") lists vertices by level, and inside a level
 *    by ascending original index, which is the order Fig. 1(c) shows.
 * Outputs: level_of[n], perm[n] (new -> old), iperm[n] (old -> new),
 * level_ptr[nlevels+1] (caller gives room for n+1), *nlevels.
 */
int orc_levels(int32_t n, const int32_t *rp, const int32_t *ci, int32_t root, int32_t *level_of,
               int32_t *perm, int32_t *iperm, int32_t *level_ptr, int32_t *nlevels)
{
    if (n < 0 || (n > 0 && (root < 0 || root >= n))) return ORC_EINVAL;
    *nlevels = 0;
    level_ptr[0] = 0;
    if (n == 0) return ORC_OK;
    const int64_t nnz = rp[n];
    /* symmetrised adjacency, duplicates allowed */
    int64_t *deg = calloc((size_t)n + 1, sizeof(int64_t));
    if (!deg) return ORC_ENOMEM;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
            if (ci[e] != i) { deg[i + 1]++; deg[ci[e] + 1]++; }
    for (int64_t i = 0; i < n; ++i) deg[i + 1] += deg[i];
    int32_t *adj = malloc(sizeof(int32_t) * (size_t)(deg[n] > 0 ? deg[n] : 1));
    int64_t *fill = malloc(sizeof(int64_t) * (size_t)n);
    int32_t *queue = malloc(sizeof(int32_t) * (size_t)n);
    if (!adj || !fill || !queue) { free(deg); free(adj); free(fill); free(queue); return ORC_ENOMEM; }
    (void)nnz;
    memcpy(fill, deg, sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
            if (ci[e] != i) { adj[fill[i]++] = ci[e]; adj[fill[ci[e]]++] = (int32_t)i; }
    for (int64_t i = 0; i < n; ++i) level_of[i] = -1;

    /* level-synchronous search: queue[head..tail) holds the current level */
    int64_t head = 0, tail = 0, next_unvisited = 0;
    int32_t lev = 0;
    level_of[root] = 0;
    queue[tail++] = root;
    while (head < n) {
        if (head == tail) { /* disconnected: restart at the smallest untouched vertex */
            while (level_of[next_unvisited] >= 0) ++next_unvisited;
            level_of[next_unvisited] = lev + 1;
            queue[tail++] = (int32_t)next_unvisited;
        }
        const int64_t level_end = tail;
        lev = level_of[queue[head]];
        for (; head < level_end; ++head) {
            const int32_t v = queue[head];
            for (int64_t e = deg[v]; e < deg[v + 1]; ++e) {
                const int32_t u = adj[e];
                if (level_of[u] < 0) { level_of[u] = lev + 1; queue[tail++] = u; }
            }
        }
    }
    int32_t L = 0;
    for (int64_t i = 0; i < n; ++i) if (level_of[i] + 1 > L) L = level_of[i] + 1;
    /* counting sort by level; scanning ids in ascending order keeps each level ascending */
    for (int32_t l = 0; l <= L; ++l) level_ptr[l] = 0;
    for (int64_t i = 0; i < n; ++i) level_ptr[level_of[i] + 1]++;
    for (int32_t l = 0; l < L; ++l) level_ptr[l + 1] += level_ptr[l];
    for (int32_t l = 0; l < L; ++l) fill[l] = level_ptr[l];
    for (int64_t i = 0; i < n; ++i) {
        const int64_t pos = fill[level_of[i]]++;
        perm[pos] = (int32_t)i;
        iperm[i] = (int32_t)pos;
    }
    *nlevels = L;
    free(deg); free(adj); free(fill); free(queue);
    return ORC_OK;
}

/*
 * Symmetric permutation P A P^T (Sec. 3, "BFS reordering"): new row r is old row
 * perm[r]; each entry keeps its position inside the row (original stored order) and
 * its column is relabelled through iperm.  Outputs must hold n+1 / nnz entries.
 */
int orc_permute(int32_t n, const int32_t *rp, const int32_t *ci, const double *va,
                const int32_t *perm, const int32_t *iperm, int32_t *prp, int32_t *pci, double *pva)
{
    if (n < 0) return ORC_EINVAL;
    prp[0] = 0;
    for (int64_t r = 0; r < n; ++r) {
        const int32_t old = perm[r];
        const int32_t len = rp[old + 1] - rp[old];
        prp[r + 1] = prp[r] + len;
        for (int32_t t = 0; t < len; ++t) {
            pci[prp[r] + t] = iperm[ci[rp[old] + t]];
            pva[prp[r] + t] = va[rp[old] + t];
        }
    }
    return ORC_OK;
}

/*
 * Level grouping under a cache budget (Sec. 3 reuse window and Sec. 6 parameter C):
 * scan the levels left to right and put the next level into the current group while
 * the group's bytes stay <= budget; otherwise start a new group.  A level that alone
 * exceeds the budget forms its own group.  The bytes a level needs are its CSR data
 * and its rows' entries of the two vectors one power reads and writes:
 *   bytes(level) = (val_bytes + 4) * nnz(level) + 4 * rows(level) + 16 * m * rows(level).
 * rp is the row pointer of the permuted matrix (levels are consecutive row ranges).
 * group_ptr (room for nlevels+1) receives level indices; *ngroups the count.
 */
int orc_groups(int32_t nlevels, const int32_t *level_ptr, const int32_t *rp, int32_t val_bytes,
               int32_t m, int64_t budget, int32_t *group_ptr, int32_t *ngroups)
{
    if (nlevels < 0 || val_bytes <= 0 || m < 1) return ORC_EINVAL;
    int32_t G = 0;
    int64_t cur = 0;
    group_ptr[0] = 0;
    for (int32_t l = 0; l < nlevels; ++l) {
        const int64_t rows = level_ptr[l + 1] - level_ptr[l];
        const int64_t nz = (int64_t)rp[level_ptr[l + 1]] - rp[level_ptr[l]];
        const int64_t b = ((int64_t)val_bytes + 4) * nz + 4 * rows + 16 * (int64_t)m * rows;
        if (l > 0 && cur + b <= budget) {
            cur += b;
        } else {
            if (l > 0) group_ptr[++G] = l;
            cur = b;
        }
    }
    if (nlevels > 0) group_ptr[++G] = nlevels;
    *ngroups = G;
    return ORC_OK;
}

/*
 * Groups with bulky levels split (the recursion stage s_m of Sec. 6, read as: a level too large
 * for the budget is broken into pieces): levels are grouped as in orc_groups while they fit
 * the budget; a level whose bytes exceed it closes the current group and is cut into pieces
 * of consecutive rows, each piece taking rows while its bytes stay <= budget (at least one
 * row), each piece a group of its own; the next level starts a new group.  A row costs
 * (val_bytes + 4) * nnz(row) + 4 + 16 * m bytes, so a level costs what orc_groups charges.
 * group_rows (room for n+1) receives the first row of every group and n; *ngroups the count.
 */
int orc_groups_split(int32_t nlevels, const int32_t *level_ptr, const int32_t *rp, int32_t val_bytes, int32_t m,
                     int64_t budget, int32_t *group_rows, int32_t *ngroups)
{
    if (nlevels < 0 || val_bytes <= 0 || m < 1) return ORC_EINVAL;
    int32_t G = 0;
    int64_t cur = 0;
    group_rows[0] = 0;
    for (int32_t l = 0; l < nlevels; ++l) {
        const int64_t rows = level_ptr[l + 1] - level_ptr[l];
        const int64_t nz = (int64_t)rp[level_ptr[l + 1]] - rp[level_ptr[l]];
        const int64_t b = ((int64_t)val_bytes + 4) * nz + 4 * rows + 16 * (int64_t)m * rows;
        if (b > budget) {
            if (l > 0 && group_rows[G] != level_ptr[l]) group_rows[++G] = level_ptr[l];
            int64_t piece = 0;
            for (int32_t r = level_ptr[l]; r < level_ptr[l + 1]; ++r) {
                const int64_t rb = ((int64_t)val_bytes + 4) * (rp[r + 1] - rp[r]) + 4 + 16 * (int64_t)m;
                if (r > level_ptr[l] && piece + rb > budget) {
                    group_rows[++G] = r;
                    piece = 0;
                }
                piece += rb;
            }
            if (l + 1 < nlevels) group_rows[++G] = level_ptr[l + 1];
            cur = 0;
            continue;
        }
        if (l > 0 && group_rows[G] == level_ptr[l]) {  /* a new group starts here (after a bulky level) */
            cur = b;
        } else if (l > 0 && cur + b <= budget) {
            cur += b;
        } else {
            if (l > 0) group_rows[++G] = level_ptr[l];
            cur = b;
        }
    }
    if (nlevels > 0) group_rows[++G] = level_ptr[nlevels];
    *ngroups = G;
    return ORC_OK;
}

/*
 * Serial level-blocked MPK over groups that need not follow the +-1 rule of whole levels
 * (split levels): cell (g, k) runs in the order of its wave w(g, k), where w(g, 1) = 3 + g
 * and w(g, k) = max{ w(g', k-1) : group g reads a row of group g' } + 2; cells are visited by
 * increasing (w, k, g).  Every cell's inputs lie on smaller waves, so the result equals
 * back-to-back SpMV bit for bit (rows keep their summation order); Y[1..p] are only written,
 * so NaN-filled outputs expose any early read.  Arguments as orc_lb_mpk (skew replaced by the
 * wave rule).
 */
int orc_lb_mpk_waves(int32_t n, const int32_t *rp, const int32_t *ci, const double *va, int32_t m,
                     const double *X, int32_t p, int32_t G, const int32_t *group_rows, double *Y)
{
    if (n < 0 || m < 1 || p < 0 || G < 0) return ORC_EINVAL;
    const int64_t nm = (int64_t)n * m;
    memcpy(Y, X, sizeof(double) * (size_t)nm);
    if (p == 0 || G == 0) return ORC_OK;
    int32_t *group_of = malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *lo = malloc(sizeof(int32_t) * (size_t)G), *hi = malloc(sizeof(int32_t) * (size_t)G);
    int64_t *w = malloc(sizeof(int64_t) * (size_t)G * (size_t)p);
    if (!group_of || !lo || !hi || !w) { free(group_of); free(lo); free(hi); free(w); return ORC_ENOMEM; }
    for (int32_t g = 0; g < G; ++g)
        for (int32_t r = group_rows[g]; r < group_rows[g + 1]; ++r) group_of[r] = g;
    /* the groups each group reads form a contiguous hull here only as a bound; the wave takes the
       maximum over the groups actually read */
    for (int32_t g = 0; g < G; ++g) w[g] = 3 + g;
    for (int32_t k = 2; k <= p; ++k)
        for (int32_t g = 0; g < G; ++g) {
            int64_t mx = 0;
            for (int32_t r = group_rows[g]; r < group_rows[g + 1]; ++r)
                for (int32_t e = rp[r]; e < rp[r + 1]; ++e) {
                    const int64_t v = w[(int64_t)(k - 2) * G + group_of[ci[e]]];
                    if (v > mx) mx = v;
                }
            w[(int64_t)(k - 1) * G + g] = mx + 2;
        }
    int64_t wmax = 0;
    for (int64_t t = 0; t < (int64_t)G * p; ++t) if (w[t] > wmax) wmax = w[t];
    for (int64_t wave = 0; wave <= wmax; ++wave)
        for (int32_t k = 1; k <= p; ++k)
            for (int32_t g = 0; g < G; ++g) {
                if (w[(int64_t)(k - 1) * G + g] != wave) continue;
                const double *xin = Y + (int64_t)(k - 1) * nm;
                double *yout = Y + (int64_t)k * nm;
                for (int64_t i = group_rows[g]; i < group_rows[g + 1]; ++i)
                    row_times_block(rp, ci, va, m, xin, i, yout + i * m);
            }
    free(group_of); free(lo); free(hi); free(w);
    return ORC_OK;
}

/*
 * Execution order of the Lp diagram (Sec. 3, Fig. 2): cells (i, p) with level i in
 * 0..L-1 and power p in 1..pm are visited line by line, i + skew*p increasing, and inside
 * one line from bottom-right to top-left, i.e. p ascending.  skew = 1 gives the paper's
 * diagonals i + p = const.  Every line with skew >= 1 visits (i-1, p-1), (i, p-1) and
 * (i+1, p-1) before (i, p), since those lie on earlier lines (or, for skew = 1, earlier on
 * the same line).  skew = 0 visits all powers of level 0, then of level 1, ...: that order
 * breaks the rule ((i, 2) runs before (i+1, 1)) and exists so that tests can show a wrong
 * order being caught.  labels[(p-1)*L + i] receives the 0-based step of cell (i, p).
 */
int orc_lp_labels(int32_t L, int32_t pm, int32_t skew, int32_t *labels)
{
    if (L < 0 || pm < 0 || skew < 0) return ORC_EINVAL;
    int32_t step = 0;
    for (int32_t d = skew; d <= L - 1 + skew * pm; ++d)     /* d = i + skew * p */
        for (int32_t p = 1; p <= pm; ++p) {
            const int32_t i = d - skew * p;
            if (i >= 0 && i < L) labels[(p - 1) * L + i] = step++;
        }
    return ORC_OK;
}

/*
 * Serial level-blocked MPK (Sec. 3): the groups of the permuted matrix are promoted
 * power by power in the Lp-diagram order of orc_lp_labels (with the given skew),
 * computing every row of a cell with the same row body as orc_mpk.  Because no row
 * changes its summation order, the result equals back-to-back SpMV on the permuted matrix
 * bit for bit; a cell that ran before its dependencies (groups g-1, g, g+1 at power p-1)
 * would read values that are not yet set.  Y (p+1)*n*m in permuted order, Y[0] = X
 * (permuted order).  group_rows[G+1] are row offsets of the groups.  Y[1..p] are only
 * written, never cleared, so a caller that fills them with NaN sees every early read.
 */
int orc_lb_mpk(int32_t n, const int32_t *rp, const int32_t *ci, const double *va, int32_t m,
               const double *X, int32_t p, int32_t G, const int32_t *group_rows, int32_t skew, double *Y)
{
    if (n < 0 || m < 1 || p < 0 || G < 0 || skew < 0) return ORC_EINVAL;
    const int64_t nm = (int64_t)n * m;
    memcpy(Y, X, sizeof(double) * (size_t)nm);
    for (int32_t d = skew; d <= G - 1 + skew * p; ++d)
        for (int32_t k = 1; k <= p; ++k) {
            const int32_t g = d - skew * k;
            if (g < 0 || g >= G) continue;
            const double *xin = Y + (int64_t)(k - 1) * nm;
            double *yout = Y + (int64_t)k * nm;
            for (int64_t i = group_rows[g]; i < group_rows[g + 1]; ++i)
                row_times_block(rp, ci, va, m, xin, i, yout + i * m);
        }
    return ORC_OK;
}

/*
 * Chebyshev expansion (Sec. 7, Eqs. for the time step and the recurrence), with the
 * matrix rescaled as A' = (A - shift I) / scale:
 *   v_0 = x,  v_1 = A' x,  v_{k+1} = 2 A' v_k - v_{k-1},
 *   out = sum_{k=0..degree} c_k v_k.
 * With alpha = 2/scale and beta = -2 shift/scale, 2 A' v = alpha (A v) + beta v, and
 * A' v = (alpha/2)(A v) + (beta/2) v.  Each row is evaluated as
 *   w      = sum_j a_ij v_k[j]                      (stored order, fma per term)
 *   v_1    = fma(1/scale, w, (-shift/scale) * v_0)
 *   v_{k+1}= fma(alpha, w, fma(beta, v_k, -v_{k-1}))
 *   acc    = c_0 * v_0, then acc = fma(c_k, v_k, acc)
 * Complex coefficients (coeff_im != NULL) act on pairs of right-hand sides
 * (columns 2j, 2j+1 = real, imaginary part of one complex vector):
 *   acc_re = fma(cr, v_re, acc_re); acc_re = fma(-ci, v_im, acc_re);
 *   acc_im = fma(cr, v_im, acc_im); acc_im = fma(ci, v_re, acc_im).
 * out holds n*m doubles.
 */
int orc_cheb(int32_t n, const int32_t *rp, const int32_t *ci, const double *va, int32_t m,
             const double *X, int32_t degree, const double *coeff_re, const double *coeff_im,
             double scale, double shift, double *out)
{
    if (n < 0 || m < 1 || degree < 0 || scale == 0.0) return ORC_EINVAL;
    if (coeff_im && (m % 2)) return ORC_EINVAL;
    const int64_t nm = (int64_t)n * m;
    const double alpha = 2.0 / scale, beta = -2.0 * shift / scale;
    const double halpha = 1.0 / scale, hbeta = -shift / scale;
    double *vprev = malloc(sizeof(double) * (size_t)(nm > 0 ? nm : 1));
    double *vcur = malloc(sizeof(double) * (size_t)(nm > 0 ? nm : 1));
    double *vnext = malloc(sizeof(double) * (size_t)(nm > 0 ? nm : 1));
    double *w = malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    if (!vprev || !vcur || !vnext || !w) { free(vprev); free(vcur); free(vnext); free(w); return ORC_ENOMEM; }
    memcpy(vcur, X, sizeof(double) * (size_t)nm);
    /* k = 0 term */
    for (int64_t t = 0; t < nm; ++t) out[t] = coeff_re[0] * vcur[t];
    if (coeff_im)
        for (int64_t i = 0; i < n; ++i)
            for (int32_t r = 0; r < m; r += 2) {
                const int64_t o = i * m + r;
                out[o] = fma(-coeff_im[0], vcur[o + 1], out[o]);
                out[o + 1] = coeff_re[0] * vcur[o + 1];
                out[o + 1] = fma(coeff_im[0], vcur[o], out[o + 1]);
            }
    for (int32_t k = 0; k < degree; ++k) {
        for (int64_t i = 0; i < n; ++i) {
            row_times_block(rp, ci, va, m, vcur, i, w);
            for (int32_t r = 0; r < m; ++r) {
                const int64_t o = i * m + r;
                vnext[o] = (k == 0) ? fma(halpha, w[r], hbeta * vcur[o])
                                    : fma(alpha, w[r], fma(beta, vcur[o], -vprev[o]));
            }
        }
        const double cr = coeff_re[k + 1];
        if (!coeff_im) {
            for (int64_t t = 0; t < nm; ++t) out[t] = fma(cr, vnext[t], out[t]);
        } else {
            const double cim = coeff_im[k + 1];
            for (int64_t i = 0; i < n; ++i)
                for (int32_t r = 0; r < m; r += 2) {
                    const int64_t o = i * m + r;
                    out[o] = fma(cr, vnext[o], out[o]);
                    out[o] = fma(-cim, vnext[o + 1], out[o]);
                    out[o + 1] = fma(cr, vnext[o + 1], out[o + 1]);
                    out[o + 1] = fma(cim, vnext[o], out[o + 1]);
                }
        }
        double *t = vprev; vprev = vcur; vcur = vnext; vnext = t;
    }
    free(vprev); free(vcur); free(vnext); free(w);
    return ORC_OK;
}

/*
 * The Chebyshev expansion of orc_cheb with the matrix-vector product accumulated in binary32
 * (as orc_mpk_acc32: w = sum fmaf(a_ij, (float) v_k[j], w) in stored order, widened exactly)
 * while the recurrence v_{k+1} = fma(alpha, w, fma(beta, v_k, -v_{k-1})), the vectors and the
 * accumulator stay binary64: the three-term recurrence, whose stability needs it, keeps
 * double precision.  Same arguments and layout as orc_cheb.
 */
int orc_cheb_acc32(int32_t n, const int32_t *rp, const int32_t *ci, const double *va, int32_t m,
                   const double *X, int32_t degree, const double *coeff_re, const double *coeff_im,
                   double scale, double shift, double *out)
{
    if (n < 0 || m < 1 || degree < 0 || scale == 0.0) return ORC_EINVAL;
    if (coeff_im && (m % 2)) return ORC_EINVAL;
    for (int64_t e = 0; e < (n > 0 ? rp[n] : 0); ++e)
        if ((double)(float)va[e] != va[e]) return ORC_EINVAL;
    const int64_t nm = (int64_t)n * m;
    const double alpha = 2.0 / scale, beta = -2.0 * shift / scale;
    const double halpha = 1.0 / scale, hbeta = -shift / scale;
    double *vprev = malloc(sizeof(double) * (size_t)(nm > 0 ? nm : 1));
    double *vcur = malloc(sizeof(double) * (size_t)(nm > 0 ? nm : 1));
    double *vnext = malloc(sizeof(double) * (size_t)(nm > 0 ? nm : 1));
    float *vf = malloc(sizeof(float) * (size_t)(nm > 0 ? nm : 1));
    float *w = malloc(sizeof(float) * (size_t)m);
    if (!vprev || !vcur || !vnext || !vf || !w) {
        free(vprev); free(vcur); free(vnext); free(vf); free(w);
        return ORC_ENOMEM;
    }
    memcpy(vcur, X, sizeof(double) * (size_t)nm);
    for (int64_t t = 0; t < nm; ++t) out[t] = coeff_re[0] * vcur[t];
    if (coeff_im)
        for (int64_t i = 0; i < n; ++i)
            for (int32_t r = 0; r < m; r += 2) {
                const int64_t o = i * m + r;
                out[o] = fma(-coeff_im[0], vcur[o + 1], out[o]);
                out[o + 1] = coeff_re[0] * vcur[o + 1];
                out[o + 1] = fma(coeff_im[0], vcur[o], out[o + 1]);
            }
    for (int32_t k = 0; k < degree; ++k) {
        for (int64_t t = 0; t < nm; ++t) vf[t] = (float)vcur[t];
        for (int64_t i = 0; i < n; ++i) {
            for (int32_t r = 0; r < m; ++r) w[r] = 0.0f;
            for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
                const float a = (float)va[e];
                const float *xr = vf + (int64_t)ci[e] * m;
                for (int32_t r = 0; r < m; ++r) w[r] = fmaf(a, xr[r], w[r]);
            }
            for (int32_t r = 0; r < m; ++r) {
                const int64_t o = i * m + r;
                const double wd = (double)w[r];
                vnext[o] = (k == 0) ? fma(halpha, wd, hbeta * vcur[o]) : fma(alpha, wd, fma(beta, vcur[o], -vprev[o]));
            }
        }
        const double cr = coeff_re[k + 1];
        if (!coeff_im) {
            for (int64_t t = 0; t < nm; ++t) out[t] = fma(cr, vnext[t], out[t]);
        } else {
            const double cim = coeff_im[k + 1];
            for (int64_t i = 0; i < n; ++i)
                for (int32_t r = 0; r < m; r += 2) {
                    const int64_t o = i * m + r;
                    out[o] = fma(cr, vnext[o], out[o]);
                    out[o] = fma(-cim, vnext[o + 1], out[o]);
                    out[o + 1] = fma(cr, vnext[o + 1], out[o + 1]);
                    out[o + 1] = fma(cim, vnext[o], out[o + 1]);
                }
        }
        double *t = vprev; vprev = vcur; vcur = vnext; vnext = t;
    }
    free(vprev); free(vcur); free(vnext); free(vf); free(w);
    return ORC_OK;
}

/*
 * Bessel functions of the first kind J_0..J_kmax at x >= 0 by Miller's backward
 * recurrence (J.C.P. Miller, 1952): start far above kmax with J_{N+1} = 0,
 * J_N = tiny, recur J_{k-1} = (2k/x) J_k - J_{k+1} downward and normalise with
 * J_0 + 2 sum_{j>=1} J_{2j} = 1.  Inputs for the Chebyshev time step of Sec. 7,
 * whose coefficients are J_0(dt) and 2 (-i)^k J_k(dt).
 */
int orc_bessel_j(int32_t kmax, double x, double *J)
{
    if (kmax < 0 || x < 0.0) return ORC_EINVAL;
    if (x == 0.0) { for (int32_t k = 0; k <= kmax; ++k) J[k] = (k == 0) ? 1.0 : 0.0; return ORC_OK; }
    int32_t N = kmax + 40 + (int32_t)(2.0 * x);
    if (N % 2) ++N;
    long double *b = calloc((size_t)N + 2, sizeof(long double));
    if (!b) return ORC_ENOMEM;
    long double jp1 = 0.0L, j = 1e-300L, norm = 0.0L;
    for (int32_t k = N; k >= 1; --k) {
        b[k] = j;
        const long double jm1 = (2.0L * k / (long double)x) * j - jp1;
        jp1 = j; j = jm1;
        if (fabsl(j) > 1e250L) { /* rescale to stay in range */
            for (int32_t t = k; t <= N; ++t) b[t] *= 1e-250L;
            j *= 1e-250L; jp1 *= 1e-250L;
        }
    }
    b[0] = j;
    norm = b[0];
    for (int32_t k = 2; k <= N; k += 2) norm += 2.0L * b[k];
    for (int32_t k = 0; k <= kmax; ++k) J[k] = (double)(b[k] / norm);
    free(b);
    return ORC_OK;
}
