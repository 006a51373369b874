/*
 * bn_oracle.c -- plain CPU FP64 oracle for exact Bayesian-network edge
 * posteriors (Chen, Tian, Nikolova, Aluru: "A Parallel Algorithm for Exact
 * Bayesian Structure Discovery in Bayesian Networks", arXiv 1408.1664).
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the CPU
 * baseline leg of the benchmark are the only callers.  The product (the CUDA
 * library) never links, loads or calls this file, and this file includes no
 * header of the product: the two share no code.
 *
 * What it computes, step by step, following the serial algorithm of Section
 * 2.2 (Algorithm 1), in the natural-log domain and in double precision:
 *
 *   1. counts N_jk of every family (i, G), |G| <= d, by a direct loop over the
 *      samples, and the BDeu local score  log B_i(G) = log rho(|G|) +
 *      log p(x_i | x_G)  (Eq. 6; the paper leaves p unspecified, Section 2.1,
 *      this oracle reads it as BDeu with equivalent sample size `ess`);
 *   2. A_i(S) = q_i(S) sum_{G subset S, |G|<=d} B_i(G)  (Eq. 7) by the
 *      truncated upward zeta transform of Definition 1, run serially one
 *      dimension j = 1..n at a time with the guards of Algorithm 2;
 *   3. F(S) = sum_{i in S} A_i(S-{i}) F(S-{i}), F(empty) = 1  (Eq. 9),
 *      lattice level by lattice level (Section 3.1.1);
 *   4. R(S) = sum_{i in S} A_i(V-S) R(S-{i}), R(empty) = 1  (Eq. 10);
 *   5. Gamma_v(G) = sum_{G subset S subset V-{v}} q_v(S) F(S) R(V-{v}-S)
 *      (Eq. 12) by the truncated downward zeta transform of Definition 2, run
 *      serially with the guards of Algorithm 3;
 *   6. P(u->v, D) = sum_{G: u in G, |G|<=d} B_v(G) Gamma_v(G)  (Eq. 11);
 *   7. P(u->v | D) = P(u->v, D) / F(V)  (Algorithm 1, last step).
 *
 * Conventions: variable i (0-based) is bit i of a subset mask (the paper's
 * variable i+1 is its bit i, Section 3.1.1).  A zero value is -INFINITY in
 * the log domain.  The output matrix is n x n row-major with
 * post[u*n + v] = P(u->v | D) and a zero diagonal.  Families of node i are
 * listed by |G|, then by increasing mask value (colexicographic order).  The
 * parent configuration of a family is a mixed-radix number with the
 * lowest-numbered parent least significant; cell index = config * r_i + x_i.
 *
 * A single modular feature f (Eqs. 5-9): B_i carries f_i, P(f, D) = F(V)
 * computed from those B_i, and P(f | D) = P(f, D) / P(D)
 * (orc_feature_posterior).
 *
 * Readings where the paper is silent: BDeu local scores (alpha_jk =
 * ess/(r_i q_i), alpha_j = ess/q_i); rho_i(G) = exp(log_rho[|G|] + log_w[i,G])
 * (log_rho per parent-set size and log_w per family, each zero when NULL);
 * q_i(S) = exp(log_q[i * n + |S|]), a function of the size of the
 * predecessor set (all ones when log_q is NULL); an in-degree bound d > n-1
 * is the same as d = n-1.
 *
 * Loops over independent nodes i and endpoints v, and over the subsets of
 * one lattice level, carry OpenMP pragmas; the arithmetic is unchanged by
 * them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

static int popc(uint32_t x) { return __builtin_popcount(x); }

/* log(exp(a) + exp(b)) with exp(-inf) = 0. */
static double lse(double a, double b)
{
    if (a == -INFINITY) return b;
    if (b == -INFINITY) return a;
    if (a < b) { double t = a; a = b; b = t; }
    return a + log1p(exp(b - a));
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int64_t binom(int n, int k)
{
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int t = 1; t <= k; t++) r = r * (n - k + t) / t;
    return r;
}

static int clamp_d(int n, int d) { return d > n - 1 ? n - 1 : d; }

/* Number of candidate parent sets G of one node, G subset V-{i}, |G| <= d. */
int64_t orc_num_families(int n, int d)
{
    if (n < 1 || d < 0) return 0;
    d = clamp_d(n, d);
    int64_t k = 0;
    for (int s = 0; s <= d; s++) k += binom(n - 1, s);
    return k;
}

/* Canonical family list of node i: by size, then by increasing mask value.
 * Every k-subset of V-{i} is visited by stepping through the k-subsets of the
 * n-1 other positions in increasing order (the "next larger integer with the
 * same number of ones" step) and re-inserting a zero bit at position i, which
 * keeps the order.  Returns the number of families written. */
int64_t orc_family_list(int n, int d, int i, uint32_t* masks)
{
    d = clamp_d(n, d);
    int64_t idx = 0;
    const int np = n - 1;
    const uint32_t low = (1u << i) - 1u;
    for (int k = 0; k <= d; k++) {
        if (k == 0) { masks[idx++] = 0; continue; }
        uint64_t c = (1ull << k) - 1ull;           /* smallest k-subset */
        while (c < (1ull << np)) {
            uint32_t cc = (uint32_t)c;
            masks[idx++] = (cc & low) | ((cc & ~low) << 1);
            uint64_t u = c & (~c + 1ull);          /* lowest set bit */
            uint64_t v = c + u;
            c = v + (((v ^ c) / u) >> 2);
        }
    }
    return idx;
}

/* Number of cells q * r_i of family (i, G). */
int64_t orc_family_cells(int n, const uint8_t* arity, int i, uint32_t G)
{
    int64_t q = 1;
    for (int p = 0; p < n; p++)
        if (G >> p & 1u) q *= arity[p];
    return q * arity[i];
}

/* Contingency counts N[config * r_i + x_i] of family (i, G) by a direct loop
 * over the m samples (Section 2.1: the local score costs O(m)). */
void orc_family_counts(int n, int m, const uint8_t* data, const uint8_t* arity,
                       int i, uint32_t G, int64_t* N)
{
    const int64_t cells = orc_family_cells(n, arity, i, G);
    memset(N, 0, (size_t)cells * sizeof(int64_t));
    for (int s = 0; s < m; s++) {
        const uint8_t* row = data + (size_t)s * n;
        int64_t cfg = 0, stride = 1;
        for (int p = 0; p < n; p++) {
            if (G >> p & 1u) { cfg += row[p] * stride; stride *= arity[p]; }
        }
        N[cfg * arity[i] + row[i]] += 1;
    }
}

/* BDeu log marginal likelihood of one family from its counts:
 *   sum_j [lgamma(a_j) - lgamma(a_j + N_j)]
 *     + sum_jk [lgamma(a_jk + N_jk) - lgamma(a_jk)],
 * a_j = ess / q, a_jk = ess / (q r). */
double orc_bdeu(int r, int64_t q, const int64_t* N, double ess)
{
    const double a_j = ess / (double)q;
    const double a_jk = ess / ((double)q * (double)r);
    double score = 0.0;
    for (int64_t j = 0; j < q; j++) {
        int64_t Nj = 0;
        for (int k = 0; k < r; k++) {
            const int64_t c = N[j * r + k];
            Nj += c;
            score += lgamma(a_jk + (double)c) - lgamma(a_jk);
        }
        score += lgamma(a_j) - lgamma(a_j + (double)Nj);
    }
    return score;
}

/* log B_i(G) = log rho(|G|) + BDeu(i, G)   (Eq. 6 with f = 1). */
double orc_family_score(int n, int m, const uint8_t* data, const uint8_t* arity,
                        double ess, const double* log_rho, int i, uint32_t G)
{
    const int64_t cells = orc_family_cells(n, arity, i, G);
    int64_t* N = (int64_t*)malloc((size_t)cells * sizeof(int64_t));
    if (!N) return NAN;
    orc_family_counts(n, m, data, arity, i, G, N);
    const double s = orc_bdeu(arity[i], cells / arity[i], N, ess);
    free(N);
    return s + (log_rho ? log_rho[popc(G)] : 0.0);
}

static int validate(int n, int d, int m, const uint8_t* data, const uint8_t* arity)
{
    if (n < 1 || n > 31 || d < 0 || m < 0 || !arity) return ORC_EINVAL;
    if (m > 0 && !data) return ORC_EINVAL;
    for (int i = 0; i < n; i++) if (arity[i] < 1) return ORC_EINVAL;
    for (size_t s = 0; s < (size_t)m * n; s++)
        if (data[s] >= arity[s % n]) return ORC_EINVAL;
    return ORC_OK;
}

/* Step 1 of Algorithm 1: all local scores, layout [i * K + f], families in
 * canonical order. */
int orc_scores(int n, int d, int m, const uint8_t* data, const uint8_t* arity,
               double ess, const double* log_rho, uint32_t* mask_out,
               double* logB_out)
{
    int rc = validate(n, d, m, data, arity);
    if (rc) return rc;
    const int64_t K = orc_num_families(n, d);
    for (int i = 0; i < n; i++) orc_family_list(n, d, i, mask_out + (size_t)i * K);
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t x = 0; x < (int64_t)n * K; x++) {
        const int i = (int)(x / K);
        logB_out[x] = orc_family_score(n, m, data, arity, ess, log_rho, i, mask_out[x]);
    }
    return ORC_OK;
}

/* Definition 1 via Algorithm 2 run serially: t(T) = sum_{S subset T, |S|<=d}
 * s(S) for every T subset V, |V| = n, in the log domain.  Iteration j sums
 * dimension j; entries outside the guard of line 3 are not computed in that
 * iteration (they are never read afterwards) and are left at zero. */
int orc_upzeta(int n, int d, const double* s, double* t)
{
    const size_t N = (size_t)1 << n;
    const uint32_t full = (uint32_t)(N - 1);
    double* prev = (double*)malloc(N * sizeof(double));
    double* next = (double*)malloc(N * sizeof(double));
    if (!prev || !next) { free(prev); free(next); return ORC_ENOMEM; }
    for (size_t S = 0; S < N; S++) prev[S] = popc((uint32_t)S) <= d ? s[S] : -INFINITY;
    for (int j = 1; j <= n; j++) {
        const uint32_t bit = 1u << (j - 1);
        const uint32_t from_j = full & ~(bit - 1u);          /* {j, ..., n}   */
        const uint32_t after_j = full & ~((bit << 1) - 1u);  /* {j+1, ..., n} */
        for (size_t Sx = 0; Sx < N; Sx++) {
            const uint32_t S = (uint32_t)Sx;
            if (popc(S & after_j) > d) { next[S] = -INFINITY; continue; }
            double v = -INFINITY;
            if (popc(S & from_j) <= d) v = prev[S];
            if (S & bit) v = lse(v, prev[S & ~bit]);
            next[S] = v;
        }
        double* tmp = prev; prev = next; next = tmp;
    }
    memcpy(t, prev, N * sizeof(double));
    free(prev); free(next);
    return ORC_OK;
}

/* Definition 2 via Algorithm 3 run serially: t(T) = sum_{T subset S subset V}
 * s(S) for every T with |T| <= d (other entries are left at zero). */
int orc_downzeta(int n, int d, const double* s, double* t)
{
    const size_t N = (size_t)1 << n;
    double* prev = (double*)malloc(N * sizeof(double));
    double* next = (double*)malloc(N * sizeof(double));
    if (!prev || !next) { free(prev); free(next); return ORC_ENOMEM; }
    memcpy(prev, s, N * sizeof(double));
    for (int j = 1; j <= n; j++) {
        const uint32_t bit = 1u << (j - 1);
        const uint32_t upto_j = (bit << 1) - 1u;              /* {1, ..., j} */
        for (size_t Sx = 0; Sx < N; Sx++) {
            const uint32_t S = (uint32_t)Sx;
            if (popc(S & upto_j) > d) { next[S] = -INFINITY; continue; }
            double v = prev[S];
            if (!(S & bit)) v = lse(v, prev[S | bit]);
            next[S] = v;
        }
        double* tmp = prev; prev = next; next = tmp;
    }
    memcpy(t, prev, N * sizeof(double));
    free(prev); free(next);
    return ORC_OK;
}

/* Eq. 9, lattice level by level: F(empty) = 1, then every S of size l from
 * the F values of size l-1.  A is [i * 2^n + S] with A_i(S) for S not
 * containing i. */
void orc_forward(int n, const double* A, double* F)
{
    const size_t N = (size_t)1 << n;
    F[0] = 0.0;
    for (int l = 1; l <= n; l++) {
        #pragma omp parallel for schedule(static)
        for (size_t Sx = 1; Sx < N; Sx++) {
            const uint32_t S = (uint32_t)Sx;
            if (popc(S) != l) continue;
            double v = -INFINITY;
            for (int i = 0; i < n; i++) {
                if (!(S >> i & 1u)) continue;
                const uint32_t Si = S & ~(1u << i);
                v = lse(v, A[(size_t)i * N + Si] + F[Si]);
            }
            F[S] = v;
        }
    }
}

/* Eq. 10, lattice level by level: R(empty) = 1,
 * R(S) = sum_{i in S} A_i(V-S) R(S-{i}). */
void orc_backward(int n, const double* A, double* R)
{
    const size_t N = (size_t)1 << n;
    const uint32_t full = (uint32_t)(N - 1);
    R[0] = 0.0;
    for (int l = 1; l <= n; l++) {
        #pragma omp parallel for schedule(static)
        for (size_t Sx = 1; Sx < N; Sx++) {
            const uint32_t S = (uint32_t)Sx;
            if (popc(S) != l) continue;
            double v = -INFINITY;
            for (int i = 0; i < n; i++) {
                if (!(S >> i & 1u)) continue;
                v = lse(v, A[(size_t)i * N + (full & ~S)] + R[S & ~(1u << i)]);
            }
            R[S] = v;
        }
    }
}

int orc_edge_posteriors_ext(int n, int d, int m, const uint8_t* data,
                            const uint8_t* arity, double ess, const double* log_rho,
                            const double* log_q, const double* log_w,
                            double* post, double* log_PD, double* A_out,
                            double* F_out, double* R_out, double* Gamma_out,
                            double* logB_out, uint32_t* mask_out);

/* Step 2 for every node: A_i = q_i * (truncated upward zeta transform of B_i
 * over V), with s(S) = 0 for S containing i (footnote to Section 3.1.2) and
 * A_i(S) = 0 there.  A is [i * 2^n + S]; logB / masks are [i * K + f]. */
static int build_A(int n, int d, int64_t K, const uint32_t* masks, const double* logB,
                   const double* log_q, double* A)
{
    const size_t N = (size_t)1 << n;
    int rc = ORC_OK;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < n; i++) {
        double* s = (double*)malloc(N * sizeof(double));
        double* Ai = A + (size_t)i * N;
        if (!s) { rc = ORC_ENOMEM; continue; }
        for (size_t S = 0; S < N; S++) s[S] = -INFINITY;
        for (int64_t f = 0; f < K; f++) s[masks[(size_t)i * K + f]] = logB[(size_t)i * K + f];
        if (orc_upzeta(n, d, s, Ai)) rc = ORC_ENOMEM;
        for (size_t S = 0; S < N; S++) {
            if (S >> i & 1u) Ai[S] = -INFINITY;
            else if (log_q) Ai[S] += log_q[(size_t)i * n + popc((uint32_t)S)];   /* Eq. 7 */
        }
        free(s);
    }
    return rc;
}

/* Algorithm 1 end to end.  post: n*n; log_PD: log F(V) = log P(D).
 * Optional stage outputs (NULL to skip): A_out [n * 2^n] (A_i(S), zero where
 * i is in S), F_out / R_out [2^n], Gamma_out [n * K] and logB_out / mask_out
 * [n * K] in canonical family order. */
int orc_edge_posteriors(int n, int d, int m, const uint8_t* data,
                        const uint8_t* arity, double ess, const double* log_rho,
                        double* post, double* log_PD, double* A_out,
                        double* F_out, double* R_out, double* Gamma_out,
                        double* logB_out, uint32_t* mask_out)
{
    return orc_edge_posteriors_ext(n, d, m, data, arity, ess, log_rho, NULL, NULL, post,
                                   log_PD, A_out, F_out, R_out, Gamma_out, logB_out,
                                   mask_out);
}

/* As orc_edge_posteriors, with the order prior q_i(S) by size (log_q, n*n,
 * row i: log q_i for |S| = 0..n-1) and per-family log weights (log_w, n*K in
 * canonical family order, added to log B_i(G)); either may be NULL. */
int orc_edge_posteriors_ext(int n, int d, int m, const uint8_t* data,
                            const uint8_t* arity, double ess, const double* log_rho,
                            const double* log_q, const double* log_w,
                            double* post, double* log_PD, double* A_out,
                            double* F_out, double* R_out, double* Gamma_out,
                            double* logB_out, uint32_t* mask_out)
{
    int rc = validate(n, d, m, data, arity);
    if (rc) return rc;
    d = clamp_d(n, d);
    const size_t N = (size_t)1 << n;
    const uint32_t full = (uint32_t)(N - 1);
    const int64_t K = orc_num_families(n, d);

    uint32_t* masks = (uint32_t*)malloc((size_t)n * K * sizeof(uint32_t));
    double* logB = (double*)malloc((size_t)n * K * sizeof(double));
    double* A = (double*)malloc((size_t)n * N * sizeof(double));
    double* F = (double*)malloc(N * sizeof(double));
    double* R = (double*)malloc(N * sizeof(double));
    double* G = (double*)malloc((size_t)n * K * sizeof(double));
    if (!masks || !logB || !A || !F || !R || !G) { rc = ORC_ENOMEM; goto done; }

    /* Step 1: local scores, times the per-family weights. */
    rc = orc_scores(n, d, m, data, arity, ess, log_rho, masks, logB);
    if (rc) goto done;
    if (log_w)
        for (int64_t x = 0; x < (int64_t)n * K; x++) logB[x] += log_w[x];

    /* Step 2. */
    rc = build_A(n, d, K, masks, logB, log_q, A);
    if (rc) goto done;

    /* Steps 3 and 4. */
    orc_forward(n, A, F);
    orc_backward(n, A, R);

    /* Steps 5-7 for every endpoint v. */
    #pragma omp parallel for schedule(dynamic, 1)
    for (int v = 0; v < n; v++) {
        const uint32_t bv = 1u << v;
        double* s = (double*)malloc(N * sizeof(double));
        double* t = (double*)malloc(N * sizeof(double));
        if (!s || !t) { free(s); free(t); rc = ORC_ENOMEM; continue; }
        for (size_t Sx = 0; Sx < N; Sx++) {
            const uint32_t S = (uint32_t)Sx;
            s[S] = (S & bv) ? -INFINITY : F[S] + R[(full & ~bv) & ~S];
            if (log_q && !(S & bv)) s[S] += log_q[(size_t)v * n + popc(S)];   /* Eq. 12 */
        }
        if (orc_downzeta(n, d, s, t)) rc = ORC_ENOMEM;
        for (int64_t f = 0; f < K; f++) G[(size_t)v * K + f] = t[masks[(size_t)v * K + f]];
        for (int u = 0; u < n; u++) {
            if (u == v) { post[u * n + v] = 0.0; continue; }
            double joint = -INFINITY;                    /* log P(u->v, D) */
            for (int64_t f = 0; f < K; f++) {
                const size_t x = (size_t)v * K + f;
                if (masks[x] >> u & 1u) joint = lse(joint, logB[x] + G[x]);
            }
            post[u * n + v] = exp(joint - F[full]);
        }
        free(s); free(t);
    }
    if (rc) goto done;

    if (log_PD) *log_PD = F[full];
    if (A_out) memcpy(A_out, A, (size_t)n * N * sizeof(double));
    if (F_out) memcpy(F_out, F, N * sizeof(double));
    if (R_out) memcpy(R_out, R, N * sizeof(double));
    if (Gamma_out) memcpy(Gamma_out, G, (size_t)n * K * sizeof(double));
    if (logB_out) memcpy(logB_out, logB, (size_t)n * K * sizeof(double));
    if (mask_out) memcpy(mask_out, masks, (size_t)n * K * sizeof(uint32_t));
done:
    free(masks); free(logB); free(A); free(F); free(R); free(G);
    return rc;
}

/* One modular feature f = prod_i f_i(G_i) (Eqs. 5-9): with B^f_i(G) =
 * B_i(G) f_i(G) (log_f, n*K in canonical family order, log f_i(G); -inf for
 * f_i(G) = 0), P(f, D) = F^f(V) from the recursion of Eq. 9 over the A^f_i of
 * Eq. 7, and P(f | D) = F^f(V) / F(V) (the second run with f = 1).  log_q,
 * log_w and log_rho as in orc_edge_posteriors_ext.  Outputs: *p = P(f | D),
 * *log_PfD = log P(f, D) (either may be NULL). */
int orc_feature_posterior(int n, int d, int m, const uint8_t* data, const uint8_t* arity,
                          double ess, const double* log_rho, const double* log_q,
                          const double* log_w, const double* log_f, double* p,
                          double* log_PfD)
{
    int rc = validate(n, d, m, data, arity);
    if (rc) return rc;
    if (!log_f) return ORC_EINVAL;
    d = clamp_d(n, d);
    const size_t N = (size_t)1 << n;
    const uint32_t full = (uint32_t)(N - 1);
    const int64_t K = orc_num_families(n, d);
    uint32_t* masks = (uint32_t*)malloc((size_t)n * K * sizeof(uint32_t));
    double* logB = (double*)malloc((size_t)n * K * sizeof(double));
    double* logBf = (double*)malloc((size_t)n * K * sizeof(double));
    double* A = (double*)malloc((size_t)n * N * sizeof(double));
    double* F = (double*)malloc(N * sizeof(double));
    double lpd = 0.0, lpfd = 0.0;
    if (!masks || !logB || !logBf || !A || !F) { rc = ORC_ENOMEM; goto done; }
    rc = orc_scores(n, d, m, data, arity, ess, log_rho, masks, logB);
    if (rc) goto done;
    for (int64_t x = 0; x < (int64_t)n * K; x++) {
        if (log_w) logB[x] += log_w[x];
        logBf[x] = logB[x] + log_f[x];                  /* B_i(G) f_i(G) */
    }
    rc = build_A(n, d, K, masks, logB, log_q, A);       /* f = 1: P(D) */
    if (rc) goto done;
    orc_forward(n, A, F);
    lpd = F[full];
    rc = build_A(n, d, K, masks, logBf, log_q, A);      /* P(f, D) */
    if (rc) goto done;
    orc_forward(n, A, F);
    lpfd = F[full];
    if (p) *p = exp(lpfd - lpd);
    if (log_PfD) *log_PfD = lpfd;
done:
    free(masks); free(logB); free(logBf); free(A); free(F);
    return rc;
}
