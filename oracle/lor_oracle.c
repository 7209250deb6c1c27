/*
 * lor_oracle.c -- plain, slow, obviously correct CPU oracle for the
 * longest-overlap-region path (suffix array, LCP array, LCP of arbitrary
 * suffixes, longest common substring by dynamic programming).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header or table with the CUDA
 * path.
 *
 * Every routine is the plain definition written out:
 *   - suffix order: Section 3 ("LCP and related algorithm"), the suffix-array
 *     definition S[SA[0]..] < S[SA[1]..] < ... (Table 1 is its worked
 *     example).  The end of the text compares smaller than every symbol, so a
 *     proper prefix sorts first (Table 1: suffix "C" precedes "CTAC").
 *   - LCP array: Section 3, LCP table under Table 1: lcp[0] = 0 and lcp[k] is
 *     the common-prefix length of the suffixes at ranks k-1 and k.
 *   - LCP of two arbitrary suffixes: Section 3, the identity
 *     lcp(S_pos_i, S_pos_j) = min over the adjacent LCPs between them; here
 *     computed directly by comparing the two suffixes symbol by symbol.
 *   - longest common substring of two sequences by the O(n*m) dynamic program
 *     (a brute force independent of suffix arrays) -- used to pin the
 *     overlap that the method derives from SA + LCP (Section 3, "longest
 *     overlap prefix of two sequences").
 *   - one query against a reference: for every query suffix, its longest
 *     prefix occurring in the reference, by binary search over the
 *     reference's sorted suffixes with direct comparisons (the longest match
 *     is with one of the two suffixes around the insertion point).
 *
 * Sorting uses a plain top-down merge sort with a direct suffix comparison.
 * The pthread variant only splits the same merge sort across threads.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* ---- suffix comparison (Section 3, suffix-array definition) ------------ */

static int suffix_cmp(const uint8_t *t, int64_t n, int64_t a, int64_t b)
{
    if (a == b) return 0;
    int64_t la = n - a, lb = n - b;
    int64_t m = la < lb ? la : lb;
    int c = memcmp(t + a, t + b, (size_t)m);   /* unsigned byte order */
    if (c != 0) return c;
    return la < lb ? -1 : 1;                   /* shorter suffix is smaller */
}

/* Length of the common prefix of T[a..n) and T[b..n). */
static int64_t lcp_direct(const uint8_t *t, int64_t n, int64_t a, int64_t b)
{
    if (a == b) return n - a;
    int64_t h = 0;
    while (a + h < n && b + h < n && t[a + h] == t[b + h]) h++;
    return h;
}

/* ---- merge sort of suffix start positions ------------------------------- */

static void msort(const uint8_t *t, int64_t n, int32_t *a, int32_t *tmp,
                  int64_t lo, int64_t hi)
{
    if (hi - lo < 2) return;
    int64_t mid = lo + (hi - lo) / 2;
    msort(t, n, a, tmp, lo, mid);
    msort(t, n, a, tmp, mid, hi);
    int64_t i = lo, j = mid, k = lo;
    while (i < mid && j < hi)
        tmp[k++] = (suffix_cmp(t, n, a[i], a[j]) <= 0) ? a[i++] : a[j++];
    while (i < mid) tmp[k++] = a[i++];
    while (j < hi) tmp[k++] = a[j++];
    memcpy(a + lo, tmp + lo, (size_t)(hi - lo) * sizeof(int32_t));
}

typedef struct {
    const uint8_t *t; int64_t n; int32_t *a; int32_t *tmp; int64_t lo, hi;
} sort_job;

static void *sort_worker(void *arg)
{
    sort_job *j = (sort_job *)arg;
    msort(j->t, j->n, j->a, j->tmp, j->lo, j->hi);
    return NULL;
}

typedef struct {
    const uint8_t *t; int64_t n; const int32_t *src; int32_t *dst;
    int64_t lo, mid, hi;
} merge_job;

static void *merge_worker(void *arg)
{
    merge_job *m = (merge_job *)arg;
    int64_t i = m->lo, j = m->mid, k = m->lo;
    while (i < m->mid && j < m->hi)
        m->dst[k++] = (suffix_cmp(m->t, m->n, m->src[i], m->src[j]) <= 0)
                          ? m->src[i++] : m->src[j++];
    while (i < m->mid) m->dst[k++] = m->src[i++];
    while (j < m->hi) m->dst[k++] = m->src[j++];
    return NULL;
}

/*
 * Suffix array of T[0..n): sa[k] = start of the k-th smallest suffix.
 * nthreads <= 1 runs single-threaded.  Returns 0 on success, -1 on bad
 * arguments or allocation failure.
 */
int oracle_suffix_array(const uint8_t *t, int64_t n, int32_t *sa, int nthreads)
{
    if (n < 0 || (n > 0 && (!t || !sa))) return -1;
    for (int64_t i = 0; i < n; i++) sa[i] = (int32_t)i;
    if (n < 2) return 0;
    int32_t *tmp = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!tmp) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 64) nthreads = 64;
    int p = 1;
    while (p * 2 <= nthreads && (int64_t)p * 2 <= n) p *= 2;
    if (p == 1) {
        msort(t, n, sa, tmp, 0, n);
        free(tmp);
        return 0;
    }
    /* p chunks sorted in parallel, then log2(p) rounds of pairwise merges. */
    int64_t bounds[65];
    for (int c = 0; c <= p; c++) bounds[c] = n * c / p;
    pthread_t th[64];
    sort_job sj[64];
    for (int c = 0; c < p; c++) {
        sj[c] = (sort_job){t, n, sa, tmp, bounds[c], bounds[c + 1]};
        pthread_create(&th[c], NULL, sort_worker, &sj[c]);
    }
    for (int c = 0; c < p; c++) pthread_join(th[c], NULL);
    int32_t *src = sa, *dst = tmp;
    for (int width = 1; width < p; width *= 2) {
        merge_job mj[64];
        int nm = 0;
        for (int c = 0; c < p; c += 2 * width) {
            int64_t lo = bounds[c];
            int64_t mid = bounds[c + width < p ? c + width : p];
            int64_t hi = bounds[c + 2 * width < p ? c + 2 * width : p];
            mj[nm] = (merge_job){t, n, src, dst, lo, mid, hi};
            pthread_create(&th[nm], NULL, merge_worker, &mj[nm]);
            nm++;
        }
        for (int c = 0; c < nm; c++) pthread_join(th[c], NULL);
        int32_t *s = src; src = dst; dst = s;
    }
    if (src != sa) memcpy(sa, src, (size_t)n * sizeof(int32_t));
    free(tmp);
    return 0;
}

/* ---- LCP array (Section 3, LCP table: lcp[0] = 0) ------------------------ */

typedef struct {
    const uint8_t *t; int64_t n; const int32_t *sa; const int64_t *sa64; int32_t *lcp; int64_t lo, hi;
    int too_long;
} lcp_job;

/* SA entry k of a job (int32 or int64 array). */
static int64_t job_sa(const int32_t *sa, const int64_t *sa64, int64_t k)
{
    return sa64 ? sa64[k] : (int64_t)sa[k];
}

static void *lcp_worker(void *arg)
{
    lcp_job *j = (lcp_job *)arg;
    for (int64_t k = j->lo; k < j->hi; k++) {
        int64_t h = (k == 0) ? 0
                             : lcp_direct(j->t, j->n, job_sa(j->sa, j->sa64, k - 1), job_sa(j->sa, j->sa64, k));
        if (h > INT32_MAX) { j->too_long = 1; h = INT32_MAX; }
        j->lcp[k] = (int32_t)h;
    }
    return NULL;
}

static int lcp_array_any(const uint8_t *t, int64_t n, const int32_t *sa, const int64_t *sa64, int32_t *lcp,
                         int nthreads)
{
    if (n < 0 || (n > 0 && (!t || !(sa || sa64) || !lcp))) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 64) nthreads = 64;
    pthread_t th[64];
    lcp_job jb[64];
    for (int c = 0; c < nthreads; c++) {
        jb[c] = (lcp_job){t, n, sa, sa64, lcp, n * c / nthreads, n * (c + 1) / nthreads, 0};
        pthread_create(&th[c], NULL, lcp_worker, &jb[c]);
    }
    int too_long = 0;
    for (int c = 0; c < nthreads; c++) {
        pthread_join(th[c], NULL);
        too_long |= jb[c].too_long;
    }
    return too_long ? -2 : 0;
}

int oracle_lcp_array(const uint8_t *t, int64_t n, const int32_t *sa, int32_t *lcp,
                     int nthreads)
{
    return lcp_array_any(t, n, sa, NULL, lcp, nthreads);
}

/* The same with an int64 suffix array (texts past 2^31 symbols); -2 when an
 * LCP value does not fit int32. */
int oracle_lcp_array64(const uint8_t *t, int64_t n, const int64_t *sa, int32_t *lcp, int nthreads)
{
    return lcp_array_any(t, n, NULL, sa, lcp, nthreads);
}

/* ---- check a given suffix array by direct comparison -------------------- */
/*
 * A permutation of [0,n) whose adjacent entries are strictly increasing
 * suffixes is the suffix array (Section 3 definition).  Returns -1 when sa
 * is the suffix array; otherwise the first rank k at which the definition
 * fails (k = n signals "not a permutation").
 */
typedef struct {
    const uint8_t *t; int64_t n; const int32_t *sa; const int64_t *sa64; int64_t lo, hi; int64_t bad;
} chk_job;

static void *chk_worker(void *arg)
{
    chk_job *j = (chk_job *)arg;
    j->bad = -1;
    for (int64_t k = j->lo < 1 ? 1 : j->lo; k < j->hi; k++) {
        if (suffix_cmp(j->t, j->n, job_sa(j->sa, j->sa64, k - 1), job_sa(j->sa, j->sa64, k)) >= 0) {
            j->bad = k;
            return NULL;
        }
    }
    return NULL;
}

static int64_t check_suffix_array_any(const uint8_t *t, int64_t n, const int32_t *sa, const int64_t *sa64,
                                      int nthreads)
{
    if (n <= 0) return -1;
    uint8_t *seen = (uint8_t *)calloc((size_t)n, 1);
    if (!seen) return n;
    for (int64_t k = 0; k < n; k++) {
        int64_t p = job_sa(sa, sa64, k);
        if (p < 0 || p >= n || seen[p]) { free(seen); return n; }
        seen[p] = 1;
    }
    free(seen);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 64) nthreads = 64;
    pthread_t th[64];
    chk_job jb[64];
    for (int c = 0; c < nthreads; c++) {
        jb[c] = (chk_job){t, n, sa, sa64, n * c / nthreads, n * (c + 1) / nthreads, -1};
        pthread_create(&th[c], NULL, chk_worker, &jb[c]);
    }
    int64_t bad = -1;
    for (int c = 0; c < nthreads; c++) {
        pthread_join(th[c], NULL);
        if (jb[c].bad >= 0 && (bad < 0 || jb[c].bad < bad)) bad = jb[c].bad;
    }
    return bad;
}

int64_t oracle_check_suffix_array(const uint8_t *t, int64_t n, const int32_t *sa,
                                  int nthreads)
{
    return check_suffix_array_any(t, n, sa, NULL, nthreads);
}

int64_t oracle_check_suffix_array64(const uint8_t *t, int64_t n, const int64_t *sa, int nthreads)
{
    return check_suffix_array_any(t, n, NULL, sa, nthreads);
}

/* ---- LCP of arbitrary suffix pairs (Section 3, lcp identity; direct) ---- */

int oracle_lcp_pairs(const uint8_t *t, int64_t n, const int32_t *p, const int32_t *q,
                     int64_t nq, int32_t *out)
{
    for (int64_t i = 0; i < nq; i++) {
        if (p[i] < 0 || p[i] >= n || q[i] < 0 || q[i] >= n) return -1;
        out[i] = (int32_t)lcp_direct(t, n, p[i], q[i]);
    }
    return 0;
}

int oracle_lcp_pairs64(const uint8_t *t, int64_t n, const int64_t *p, const int64_t *q, int64_t nq, int64_t *out)
{
    for (int64_t i = 0; i < nq; i++) {
        if (p[i] < 0 || p[i] >= n || q[i] < 0 || q[i] >= n) return -1;
        out[i] = lcp_direct(t, n, p[i], q[i]);
    }
    return 0;
}

/* ---- longest common substring by dynamic programming --------------------- */
/*
 * D[i][j] = length of the longest common suffix of a[0..i] and b[0..j]
 *         = (a[i] == b[j]) ? D[i-1][j-1] + 1 : 0.
 * The longest common substring length is max D.  When mark_a / mark_b are
 * given (sizes na / nb, zero-filled by the caller), every start position
 * i - L + 1 (resp. j - L + 1) of a cell with D == L > 0 is set to 1.
 * Returns L (>= 0), or -1 on allocation failure.
 */
int64_t oracle_lcs_dp(const uint8_t *a, int64_t na, const uint8_t *b, int64_t nb,
                      uint8_t *mark_a, uint8_t *mark_b)
{
    if (na <= 0 || nb <= 0) return 0;
    int32_t *prev = (int32_t *)calloc((size_t)nb + 1, sizeof(int32_t));
    int32_t *cur = (int32_t *)calloc((size_t)nb + 1, sizeof(int32_t));
    if (!prev || !cur) { free(prev); free(cur); return -1; }
    int64_t best = 0;
    for (int64_t i = 0; i < na; i++) {
        cur[0] = 0;
        for (int64_t j = 0; j < nb; j++) {
            int32_t v = (a[i] == b[j]) ? prev[j] + 1 : 0;
            cur[j + 1] = v;
            if (v > best) best = v;
        }
        int32_t *s = prev; prev = cur; cur = s;
    }
    if (best > 0 && (mark_a || mark_b)) {
        memset(prev, 0, ((size_t)nb + 1) * sizeof(int32_t));
        for (int64_t i = 0; i < na; i++) {
            cur[0] = 0;
            for (int64_t j = 0; j < nb; j++) {
                int32_t v = (a[i] == b[j]) ? prev[j] + 1 : 0;
                cur[j + 1] = v;
                if (v == best) {
                    if (mark_a) mark_a[i - best + 1] = 1;
                    if (mark_b) mark_b[j - best + 1] = 1;
                }
            }
            int32_t *s = prev; prev = cur; cur = s;
        }
    }
    free(prev);
    free(cur);
    return best;
}

/* Common prefix length of a[0..na) and b[0..nb). */
static int64_t common_prefix(const uint8_t *a, int64_t na, const uint8_t *b, int64_t nb)
{
    int64_t l = 0;
    while (l < na && l < nb && a[l] == b[l]) l++;
    return l;
}

/* Longest substring of q shared with r (r's suffix array sa_r given, by
 * direct comparison of suffixes): out[0] = its length L, out[1] = the
 * smallest offset in q where a length-L match starts, out[2] = the smallest
 * offset in r holding q[out[1] .. out[1] + L); -1 for both when L = 0. */
int oracle_multi_query_one(const uint8_t *r, int64_t rn, const int32_t *sa_r, const uint8_t *q, int64_t qn,
                           int64_t *out)
{
    int64_t best = 0, bq = -1;
    for (int64_t i = 0; i < qn && rn > 0; i++) {
        /* first reference suffix not smaller than q[i..] */
        int64_t lo = 0, hi = rn;
        while (lo < hi) {
            const int64_t mid = (lo + hi) / 2;
            const int64_t x = sa_r[mid];
            const int64_t l = common_prefix(r + x, rn - x, q + i, qn - i);
            int less; /* r[x..] < q[i..] */
            if (l == rn - x) less = (l < qn - i); /* proper prefix sorts first */
            else if (l == qn - i) less = 0;
            else less = r[x + l] < q[i + l];
            if (less) lo = mid + 1;
            else hi = mid;
        }
        int64_t m = 0;
        if (lo < rn) {
            const int64_t x = sa_r[lo];
            const int64_t l = common_prefix(r + x, rn - x, q + i, qn - i);
            if (l > m) m = l;
        }
        if (lo > 0) {
            const int64_t x = sa_r[lo - 1];
            const int64_t l = common_prefix(r + x, rn - x, q + i, qn - i);
            if (l > m) m = l;
        }
        if (m > best) {
            best = m;
            bq = i;
        }
    }
    out[0] = best;
    out[1] = best > 0 ? bq : -1;
    out[2] = -1;
    if (best > 0) {
        for (int64_t x = 0; x + best <= rn; x++)
            if (memcmp(r + x, q + bq, (size_t)best) == 0) {
                out[2] = x;
                break;
            }
    }
    return 0;
}
