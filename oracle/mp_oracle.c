/*
 * FP64 CPU oracle for the matrix-profile sweep of Akbarinia & Cloez,
 * "Efficient Matrix Profile Computation Using Different Distance Functions"
 * (arXiv:1901.05708).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code with the CUDA library.
 *
 * Indexing is 0-based throughout.  With N = n - m + 1 subsequences, the pair
 * (i, j) is a candidate iff |i - j| > excl ("exclusion zone"; excl = 0 gives
 * the paper's own rule, which only drops the self-match).
 *
 * Every function fills two arrays of length N:
 *   P[i]  the matrix-profile value (a distance, Def. 2.4), or a "score"
 *         (the quantity the paper compares before its final root) when
 *         raw != 0: the squared Euclidean distance, the p-th power of the
 *         p-norm distance, or the squared z-normalised distance.
 *   I[i]  the index of the nearest neighbour, -1 when there is none.
 *
 * Tie-break (what the strict "<" of Algorithms 1-3 produces).  The loops
 * run over diagonals k = j - i ascending and, inside one diagonal, over i
 * ascending, and each distance first updates P[i] then P[i + k].  Target x
 * therefore meets, for each k, first its left neighbour x - k (as the
 * column of row x - k) and then its right neighbour x + k; the first of a
 * run of equal scores wins.  Equivalently: among equal scores the smallest
 * |i - j| wins, and for equal |i - j| the left neighbour wins.  The brute
 * force below visits candidates in exactly that order.
 *
 * Readings of the paper taken here (each is also listed in the design notes):
 *  - Algorithm 1 iterates k = 1..n-m-1 and Algorithms 2/3 k = 1..n-m+1; all
 *    diagonals that exist are k = excl+1 .. N-1, which is what is used.
 *  - The anchor partner written T_{k,m} (and the update target P[k]) is
 *    T_{1+k,m} (target P[1+k]), consistent with the recurrence indices.
 *  - Algorithm 2's anchor C = sum t_{1+l} t_{k+l} is read as t_{1+l} t_{1+k+l}.
 *  - The p-norm terms carry an absolute value, |t_i - t_j|^p, for real p >= 1.
 *  - A window is flat when its centred sum of squares S_i is at most
 *    2^-40 times its raw sum of squares; a flat window has no z-normalised
 *    distance: it gets P = +inf, I = -1 and is never a candidate.
 *  - Rounding can push rho slightly outside [-1, 1]; DZ^2 is clamped to
 *    [0, 4m].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_EUCLID = 0, ORC_PNORM = 1, ORC_ZNORM = 2 };
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2 };

#define ORC_FLAT_REL 0x1p-40

/* ---- compensated (Neumaier) summation -------------------------------- */
typedef struct { double s, c; } nsum_t;

static inline void nadd(nsum_t *a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else                       a->c += (x - t) + a->s;
    a->s = t;
}
static inline double nval(const nsum_t *a) { return a->s + a->c; }

/* |x|^p with the two integer powers that must be exact written out, so that
 * p = 2 reproduces the Euclidean score bit for bit (the paper notes that
 * the Euclidean distance is the p = 2 case of the p-norm). */
static inline double powabs(double x, double p) {
    if (p == 1.0) return fabs(x);
    if (p == 2.0) return x * x;
    return pow(fabs(x), p);
}

static int check_args(int64_t n, int32_t m, int64_t excl) {
    if (n < 1 || m < 1 || (int64_t)m > n || excl < 0) return ORC_EINVAL;
    return ORC_OK;
}

/* ---- per-window statistics (definition of mu_i and sigma_i, Sec. 2) ---- */
/* Two passes: mean, then centred sum of squares S_i = m sigma_i^2. */
int orc_window_stats(const double *T, int64_t n, int32_t m,
                     double *mu, double *S, uint8_t *flat) {
    if (check_args(n, m, 0)) return ORC_EINVAL;
    int64_t N = n - m + 1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; i++) {
        nsum_t a = {0, 0}, q = {0, 0}, r = {0, 0};
        for (int32_t l = 0; l < m; l++) nadd(&a, T[i + l]);
        double mean = nval(&a) / m;
        for (int32_t l = 0; l < m; l++) {
            double d = T[i + l] - mean;
            nadd(&q, d * d);
            nadd(&r, T[i + l] * T[i + l]);
        }
        mu[i] = mean;
        S[i] = nval(&q);
        flat[i] = (uint8_t)(S[i] <= ORC_FLAT_REL * nval(&r));
    }
    return ORC_OK;
}

/* ---- direct distance of one pair (Eqs. for D, DP and DZ, Sec. 2) ------- */
/* Score of the pair, i.e. the quantity under the final root.  For ZNORM the
 * caller supplies mu / S from orc_window_stats; flat windows give +inf. */
static double pair_score(const double *T, int32_t m, int dist, double p,
                         int64_t i, int64_t j,
                         const double *mu, const double *S, const uint8_t *flat) {
    nsum_t acc = {0, 0};
    if (dist == ORC_EUCLID) {
        for (int32_t l = 0; l < m; l++) {
            double d = T[i + l] - T[j + l];
            nadd(&acc, d * d);
        }
        return nval(&acc);
    }
    if (dist == ORC_PNORM) {
        for (int32_t l = 0; l < m; l++) nadd(&acc, powabs(T[i + l] - T[j + l], p));
        return nval(&acc);
    }
    /* z-normalised: population sigma, sigma = sqrt(S / m) */
    if (flat[i] || flat[j]) return INFINITY;
    double si = sqrt(S[i] / m), sj = sqrt(S[j] / m);
    for (int32_t l = 0; l < m; l++) {
        double d = (T[i + l] - mu[i]) / si - (T[j + l] - mu[j]) / sj;
        nadd(&acc, d * d);
    }
    return nval(&acc);
}

static double finish(int dist, double p, double score) {
    if (!isfinite(score)) return INFINITY;
    if (dist == ORC_PNORM) {
        if (p == 1.0) return score;
        return pow(score, 1.0 / p);
    }
    return sqrt(score < 0 ? 0 : score);
}

static void finish_all(int dist, double p, int64_t N, double *P, int raw) {
    if (raw) return;
    for (int64_t i = 0; i < N; i++) P[i] = finish(dist, p, P[i]);
}

/* Stats for ZNORM, NULLs otherwise.  Returns ORC_ENOMEM on failure. */
static int make_stats(const double *T, int64_t n, int32_t m, int dist,
                      double **mu, double **S, uint8_t **flat) {
    *mu = NULL; *S = NULL; *flat = NULL;
    if (dist != ORC_ZNORM) return ORC_OK;
    int64_t N = n - m + 1;
    *mu = (double *)malloc(sizeof(double) * N);
    *S = (double *)malloc(sizeof(double) * N);
    *flat = (uint8_t *)malloc(N);
    if (!*mu || !*S || !*flat) { free(*mu); free(*S); free(*flat); return ORC_ENOMEM; }
    orc_window_stats(T, n, m, *mu, *S, *flat);
    return ORC_OK;
}

/* ---- nested-loop brute force (the naive algorithm, Sec. 1) ------------- */
/* For each target x the candidates are visited in the paper's arrival order:
 * k = excl+1, excl+2, ..., and for each k the left neighbour before the
 * right one; a candidate replaces the current best only if strictly smaller. */
int orc_brute(const double *T, int64_t n, int32_t m, int64_t excl, int dist,
              double p, int raw, double *P, int64_t *I) {
    if (check_args(n, m, excl) || dist < 0 || dist > 2 || p < 1.0) return ORC_EINVAL;
    int64_t N = n - m + 1;
    double *mu, *S; uint8_t *flat;
    if (make_stats(T, n, m, dist, &mu, &S, &flat)) return ORC_ENOMEM;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t x = 0; x < N; x++) {
        double best = INFINITY;
        int64_t arg = -1;
        if (!(dist == ORC_ZNORM && flat[x])) {
            for (int64_t k = excl + 1; k < N; k++) {
                if (x - k >= 0) {
                    double s = pair_score(T, m, dist, p, x, x - k, mu, S, flat);
                    if (s < best) { best = s; arg = x - k; }
                }
                if (x + k < N) {
                    double s = pair_score(T, m, dist, p, x, x + k, mu, S, flat);
                    if (s < best) { best = s; arg = x + k; }
                }
            }
        }
        P[x] = best;
        I[x] = arg;
    }
    finish_all(dist, p, N, P, raw);
    free(mu); free(S); free(flat);
    return ORC_OK;
}

/* Brute force restricted to a list of rows.  Besides the best score P and
 * its index I it returns P2, the best score among candidates j with
 * |j - I| > excl (the runner-up outside the trivial-match zone of the
 * winner), +inf if there is none.  Used to decide where I is unique. */
int orc_brute_rows(const double *T, int64_t n, int32_t m, int64_t excl, int dist,
                   double p, int raw, const int64_t *rows, int64_t nrows,
                   double *P, int64_t *I, double *P2) {
    if (check_args(n, m, excl) || dist < 0 || dist > 2 || p < 1.0) return ORC_EINVAL;
    int64_t N = n - m + 1;
    for (int64_t r = 0; r < nrows; r++)
        if (rows[r] < 0 || rows[r] >= N) return ORC_EINVAL;
    double *mu, *S; uint8_t *flat;
    if (make_stats(T, n, m, dist, &mu, &S, &flat)) return ORC_ENOMEM;
    int fail = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < nrows; r++) {
        int64_t x = rows[r];
        double *prof = (double *)malloc(sizeof(double) * N);
        if (!prof) {
#pragma omp atomic write
            fail = 1;
            continue;
        }
        double best = INFINITY;
        int64_t arg = -1;
        for (int64_t j = 0; j < N; j++) prof[j] = INFINITY;
        if (!(dist == ORC_ZNORM && flat[x])) {
            for (int64_t k = excl + 1; k < N; k++) {
                if (x - k >= 0) {
                    double s = pair_score(T, m, dist, p, x, x - k, mu, S, flat);
                    prof[x - k] = s;
                    if (s < best) { best = s; arg = x - k; }
                }
                if (x + k < N) {
                    double s = pair_score(T, m, dist, p, x, x + k, mu, S, flat);
                    prof[x + k] = s;
                    if (s < best) { best = s; arg = x + k; }
                }
            }
        }
        double second = INFINITY;
        if (arg >= 0)
            for (int64_t j = 0; j < N; j++) {
                int64_t dj = j > arg ? j - arg : arg - j;
                if (dj > excl && prof[j] < second) second = prof[j];
            }
        P[r] = raw ? best : finish(dist, p, best);
        P2[r] = raw ? second : finish(dist, p, second);
        I[r] = arg;
        free(prof);
    }
    free(mu); free(S); free(flat);
    return fail ? ORC_ENOMEM : ORC_OK;
}

/* Distance (or score, raw != 0) of explicit pairs (i[r], j[r]). */
int orc_pair_dist(const double *T, int64_t n, int32_t m, int dist, double p, int raw,
                  const int64_t *ii, const int64_t *jj, int64_t npairs, double *out) {
    if (check_args(n, m, 0) || dist < 0 || dist > 2 || p < 1.0) return ORC_EINVAL;
    int64_t N = n - m + 1;
    for (int64_t r = 0; r < npairs; r++)
        if (ii[r] < 0 || ii[r] >= N || jj[r] < 0 || jj[r] >= N) return ORC_EINVAL;
    double *mu, *S; uint8_t *flat;
    if (make_stats(T, n, m, dist, &mu, &S, &flat)) return ORC_ENOMEM;
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < npairs; r++) {
        double s = pair_score(T, m, dist, p, ii[r], jj[r], mu, S, flat);
        out[r] = raw ? s : finish(dist, p, s);
    }
    free(mu); free(S); free(flat);
    return ORC_OK;
}

/* ---- the incremental algorithms (Algorithms 1, 3 and 2) ----------------- */
/*
 * The diagonal loop is split over threads (OpenMP) with thread-private
 * profiles.  Each thread takes diagonals in ascending order, so inside a
 * thread every target still sees its candidates in the paper's order; the
 * final merge keeps, per target, the smallest score and, among equal scores,
 * the smallest key 2k + [neighbour on the right], which is the same rule.
 * The result is therefore identical to a single-threaded run.
 *
 * Only diagonals k in [k_lo, k_hi) are swept (clipped to excl+1 .. N-1), so
 * that disjoint diagonal ranges can be computed separately and merged.
 */
typedef struct {
    double *P;
    int64_t *key; /* 2k + side of the current best; INT64_MAX = none */
} prof_t;

static inline void offer(prof_t *pr, int64_t x, double s, int64_t key) {
    if (s < pr->P[x]) { pr->P[x] = s; pr->key[x] = key; }
}

static int prof_alloc(prof_t *pr, int64_t N) {
    pr->P = (double *)malloc(sizeof(double) * N);
    pr->key = (int64_t *)malloc(sizeof(int64_t) * N);
    if (!pr->P || !pr->key) { free(pr->P); free(pr->key); return ORC_ENOMEM; }
    for (int64_t x = 0; x < N; x++) { pr->P[x] = INFINITY; pr->key[x] = INT64_MAX; }
    return ORC_OK;
}

/* variant of the diagonal body */
enum { SWEEP_EUCLID = 0, SWEEP_PNORM = 1, SWEEP_ZRAW = 2, SWEEP_ZCENTRED = 3 };

typedef struct {
    const double *T;
    int32_t m;
    double p;
    const double *mu, *S;
    const uint8_t *flat;
} sweep_ctx;

/* Squared z-normalised distance from Lemma 3's five sums. */
static inline double dz2_from_sums(double A, double B, double AA, double BB, double C, int32_t m) {
    double rho = (C - A * B / m) / sqrt((AA - A * A / m) * (BB - B * B / m));
    double d = 2.0 * m * (1.0 - rho);
    /* NaN (a negative variance term after cancellation) stays NaN: the
     * strict "<" of the algorithm then never takes it, as in the paper. */
    if (d < 0) d = 0;
    if (d > 4.0 * m) d = 4.0 * m;
    return d;
}

static inline double dz2_from_cov(double cov, double Si, double Sj, int32_t m) {
    double rho = cov / sqrt(Si * Sj);
    double d = 2.0 * m * (1.0 - rho);
    if (d < 0) d = 0;
    if (d > 4.0 * m) d = 4.0 * m;
    return d;
}

/* One diagonal k: anchor at i = 0 from the definition, then the O(1) update
 * along i = 1 .. N-1-k (Lemma 1 / Lemma 2 / Lemma 3). */
static void sweep_diagonal(const sweep_ctx *c, int variant, int64_t N, int64_t k, prof_t *pr) {
    const double *T = c->T;
    const int32_t m = c->m;
    const int64_t kl = 2 * k, kr = 2 * k + 1; /* left / right neighbour keys */
    if (variant == SWEEP_EUCLID || variant == SWEEP_PNORM) {
        const double p = variant == SWEEP_EUCLID ? 2.0 : c->p;
        nsum_t a = {0, 0};
        for (int32_t l = 0; l < m; l++) nadd(&a, powabs(T[l] - T[k + l], p));
        double s = nval(&a);
        offer(pr, 0, s, kr);
        offer(pr, k, s, kl);
        for (int64_t i = 1; i + k < N; i++) {
            s = s - powabs(T[i - 1] - T[i - 1 + k], p) + powabs(T[i + m - 1] - T[i + m - 1 + k], p);
            offer(pr, i, s, kr);
            offer(pr, i + k, s, kl);
        }
        return;
    }
    const uint8_t *flat = c->flat;
    if (variant == SWEEP_ZRAW) {
        /* Algorithm 2: the five running sums of Lemma 3 */
        double A = 0, B = 0, AA = 0, BB = 0, C = 0;
        for (int32_t l = 0; l < m; l++) {
            A += T[l];
            B += T[k + l];
            AA += T[l] * T[l];
            BB += T[k + l] * T[k + l];
            C += T[l] * T[k + l];
        }
        if (!flat[0] && !flat[k]) {
            double d = dz2_from_sums(A, B, AA, BB, C, m);
            offer(pr, 0, d, kr);
            offer(pr, k, d, kl);
        }
        for (int64_t i = 1; i + k < N; i++) {
            double lo = T[i - 1], hi = T[i + m - 1];
            double lo2 = T[i - 1 + k], hi2 = T[i + m - 1 + k];
            A = A - lo + hi;
            B = B - lo2 + hi2;
            AA = AA - lo * lo + hi * hi;
            BB = BB - lo2 * lo2 + hi2 * hi2;
            C = C - lo * lo2 + hi * hi2;
            if (flat[i] || flat[i + k]) continue;
            double d = dz2_from_sums(A, B, AA, BB, C, m);
            offer(pr, i, d, kr);
            offer(pr, i + k, d, kl);
        }
        return;
    }
    /* SWEEP_ZCENTRED: the same sweep on the centred covariance
     *   cov_{i,j} = sum_l (t_{i+l} - mu_i)(t_{j+l} - mu_j) = C_{i,j} - m mu_i mu_j,
     * updated by  cov_{i+1,j+1} = cov_{i,j} + df_i dg_j + df_j dg_i  with
     *   df_i = (t_{i+m} - t_i) / 2,   dg_i = (t_{i+m} - mu_{i+1}) + (t_i - mu_i),
     * which follows from Lemma 3's sums (C, A = m mu) by expanding both sides;
     * rho = cov / sqrt(S_i S_j) and DZ^2 = 2m(1 - rho) as in Lemma 3. */
    const double *mu = c->mu, *S = c->S;
    nsum_t a = {0, 0};
    for (int32_t l = 0; l < m; l++) nadd(&a, (T[l] - mu[0]) * (T[k + l] - mu[k]));
    double cov = nval(&a);
    if (!flat[0] && !flat[k]) {
        double d = dz2_from_cov(cov, S[0], S[k], m);
        offer(pr, 0, d, kr);
        offer(pr, k, d, kl);
    }
    for (int64_t i = 1; i + k < N; i++) {
        int64_t j = i + k;
        double dfi = 0.5 * (T[i - 1 + m] - T[i - 1]);
        double dfj = 0.5 * (T[j - 1 + m] - T[j - 1]);
        double dgi = (T[i - 1 + m] - mu[i]) + (T[i - 1] - mu[i - 1]);
        double dgj = (T[j - 1 + m] - mu[j]) + (T[j - 1] - mu[j - 1]);
        cov = cov + dfi * dgj + dfj * dgi;
        if (flat[i] || flat[j]) continue;
        double d = dz2_from_cov(cov, S[i], S[j], m);
        offer(pr, i, d, kr);
        offer(pr, j, d, kl);
    }
}

static int sweep(const double *T, int64_t n, int32_t m, int64_t excl, double p, int variant,
                 int64_t k_lo, int64_t k_hi, int raw, double *P, int64_t *I) {
    if (check_args(n, m, excl) || p < 1.0) return ORC_EINVAL;
    int64_t N = n - m + 1;
    int dist = variant == SWEEP_EUCLID ? ORC_EUCLID : variant == SWEEP_PNORM ? ORC_PNORM : ORC_ZNORM;
    double *mu, *S; uint8_t *flat;
    if (make_stats(T, n, m, dist, &mu, &S, &flat)) return ORC_ENOMEM;
    sweep_ctx ctx = {T, m, p, mu, S, flat};
    int64_t k0 = excl + 1 > k_lo ? excl + 1 : k_lo;
    int64_t k1 = N < k_hi ? N : k_hi;

    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    prof_t *pr = (prof_t *)calloc((size_t)nthr, sizeof(prof_t));
    if (!pr) { free(mu); free(S); free(flat); return ORC_ENOMEM; }
    int fail = 0;
    for (int t = 0; t < nthr; t++)
        if (prof_alloc(&pr[t], N)) fail = 1;
    if (!fail) {
#pragma omp parallel num_threads(nthr)
        {
            int tid = 0;
#ifdef _OPENMP
            tid = omp_get_thread_num();
#endif
#pragma omp for schedule(dynamic, 8)
            for (int64_t k = k0; k < k1; k++) sweep_diagonal(&ctx, variant, N, k, &pr[tid]);
        }
        /* deterministic merge: smallest score, then smallest key */
        for (int64_t x = 0; x < N; x++) {
            double best = INFINITY;
            int64_t bkey = INT64_MAX;
            for (int t = 0; t < nthr; t++) {
                double s = pr[t].P[x];
                int64_t key = pr[t].key[x];
                if (s < best || (s == best && key < bkey)) { best = s; bkey = key; }
            }
            P[x] = best;
            if (bkey == INT64_MAX) I[x] = -1;
            else {
                int64_t k = bkey >> 1;
                I[x] = (bkey & 1) ? x + k : x - k;
            }
        }
        finish_all(dist, p, N, P, raw);
    }
    for (int t = 0; t < nthr; t++) { free(pr[t].P); free(pr[t].key); }
    free(pr);
    free(mu); free(S); free(flat);
    return fail ? ORC_ENOMEM : ORC_OK;
}

/* Algorithm 1 (AAMP, pure Euclidean). */
int orc_aamp(const double *T, int64_t n, int32_t m, int64_t excl, int64_t k_lo, int64_t k_hi,
             int raw, double *P, int64_t *I) {
    return sweep(T, n, m, excl, 2.0, SWEEP_EUCLID, k_lo, k_hi, raw, P, I);
}

/* Algorithm 3 (AAMP for the p-norm distance). */
int orc_pnorm(const double *T, int64_t n, int32_t m, int64_t excl, double p, int64_t k_lo,
              int64_t k_hi, int raw, double *P, int64_t *I) {
    if (p < 1.0) return ORC_EINVAL;
    return sweep(T, n, m, excl, p, SWEEP_PNORM, k_lo, k_hi, raw, P, I);
}

/* Algorithm 2 (ACAMP) with the paper's five raw running sums. */
int orc_acamp(const double *T, int64_t n, int32_t m, int64_t excl, int64_t k_lo, int64_t k_hi,
              int raw, double *P, int64_t *I) {
    return sweep(T, n, m, excl, 2.0, SWEEP_ZRAW, k_lo, k_hi, raw, P, I);
}

/* ACAMP on the centred covariance (same sweep, cancellation-free sums). */
int orc_acamp_centred(const double *T, int64_t n, int32_t m, int64_t excl, int64_t k_lo,
                      int64_t k_hi, int raw, double *P, int64_t *I) {
    return sweep(T, n, m, excl, 2.0, SWEEP_ZCENTRED, k_lo, k_hi, raw, P, I);
}

/* Polish: P[i] = d(i, I[i]) recomputed from the definition (I[i] = -1 keeps
 * P[i] = +inf). */
int orc_polish(const double *T, int64_t n, int32_t m, int dist, double p, int raw,
               const int64_t *I, double *P) {
    if (check_args(n, m, 0) || dist < 0 || dist > 2 || p < 1.0) return ORC_EINVAL;
    int64_t N = n - m + 1;
    for (int64_t x = 0; x < N; x++)
        if (I[x] < -1 || I[x] >= N) return ORC_EINVAL;
    double *mu, *S; uint8_t *flat;
    if (make_stats(T, n, m, dist, &mu, &S, &flat)) return ORC_ENOMEM;
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < N; x++) {
        if (I[x] < 0) { P[x] = INFINITY; continue; }
        double s = pair_score(T, m, dist, p, x, I[x], mu, S, flat);
        P[x] = raw ? s : finish(dist, p, s);
    }
    free(mu); free(S); free(flat);
    return ORC_OK;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
