/*
 * agp_oracle.c -- plain, slow FP64 CPU oracle for Approximate Graph Propagation
 * (Wang et al., "Approximate Graph Propagation", KDD'21, arXiv:2106.03058).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, loads or calls this file; only
 * the test suite, the smoke check and the CPU-baseline leg of the benchmark do. It shares no code,
 * header, table or constant with the CUDA library.
 *
 * Every function follows a passage of the paper and is written for a reader who checks it against
 * the paper by eye: no blocking, no fusion, no reordering beyond what the cited passage states.
 * All floating point is FP64.
 *
 *   ora_philox4x32_10  Philox4x32-10 counter-based generator (Salmon et al., SC'11, Section 4).
 *   ora_build_csr      Section 4 "Pre-sorting adjacency list by degrees": undirected CSR whose
 *                      rows are sorted by neighbour degree (ties by neighbour id).
 *   ora_build_csr_directed  the same for a directed graph (Section 4, "Propagation on directed
 *                      graph", transposed adjacency): rows are out-neighbours, degrees out-degrees.
 *   ora_build_csr_directed_in  the untransposed adjacency of that passage (single-target PPR): rows
 *                      are in-neighbours, degrees still out-degrees.
 *   ora_tail_sums      Def. 3.1: Y_i = sum_{k>=i} w_k, for the weight sequences of Table 1.
 *   ora_basic          Algorithm 1 (Basic Propagation), exact truncated sum.
 *   ora_randomized     Algorithm 2 (Randomized Propagation), subset sampling done neighbour by
 *                      neighbour as its definition states (each remaining neighbour independently).
 *   ora_randomized_groups  Algorithm 2 with the Section 4 "Subset Sampling" scheme: degree groups
 *                      [2^k, 2^{k+1}), a Binomial(|G_k|, p*) count, uniform choice without
 *                      replacement, rejection with probability 1 - p_v/p*.
 *   ora_power_lambda   largest eigenvalue of A by FP64 power iteration (Katz needs beta < 1/lambda_1,
 *                      Table 1 / Section 2).
 *   ora_sweep_conductance  the local-clustering sweep of Section 6: nodes by pi(v)/d_v, the prefix
 *                      of least conductance.
 *
 * Readings where the paper is silent (listed in the design notes as well):
 *   - isolated nodes (d_u = 0) have D^{-1} := 0, so their residue is reserved and never pushed;
 *   - the push test is "increment >= eps" (the proof of Lemma 4.1 uses >=; the text uses >);
 *   - adjacency ties on degree are broken by ascending neighbour id.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",   */
/* SC'11. Round: (hi0,lo0) = M0*c0, (hi1,lo1) = M1*c2; c' = (hi1^c1^k0, lo1, hi0^c3^k1, lo0);  */
/* the key is bumped by the Weyl constants before every round but the first.                   */
/* ------------------------------------------------------------------------------------------ */
void ora_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A uniform in the open interval (0, 1) from the first Philox word of counter (c0,c1,c2,c3). */
static double uniform01(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3)
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    ora_philox4x32_10(ctr, key, out);
    return ((double)out[0] + 0.5) / 4294967296.0;
}

/* ------------------------------------------------------------------------------------------ */
/* CSR builder. Section 4, "Pre-sorting adjacency list by degrees": N_u = {v_1..v_du} stored so */
/* that d_{v_1} <= ... <= d_{v_du}. The graph is undirected (Algorithm 2 input): every input    */
/* edge (u,v) gives v in N_u and u in N_v; repeated edges are merged; input self-loops are      */
/* dropped. With add_self_loops, every node gets exactly one self-loop afterwards, counted once */
/* in its degree (the self-looped graph of SGC, Section 1).                                     */
/* ------------------------------------------------------------------------------------------ */
static const int32_t *g_sort_deg; /* degree array used by the row comparator */

static int cmp_by_id(const void *pa, const void *pb)
{
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    return (a > b) - (a < b);
}

static int cmp_by_degree_then_id(const void *pa, const void *pb)
{
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    int32_t da = g_sort_deg[a], db = g_sort_deg[b];
    if (da != db) return (da > db) - (da < db);
    return (a > b) - (a < b);
}

/* Returns nnz, or -1 on a bad argument. rowptr has n+1 entries; colidx must hold
 * 2*m (+ n with add_self_loops) entries (m (+ n) when directed); deg has n entries.
 * directed = 0: undirected graph as above. directed = 1: "Propagation on directed graph"
 * (end of Section 4) with the transposed adjacency of PageRank, PPR, HKPR and Katz: r^(i+1)(v)
 * sums over the in-neighbours u of v, so the push list of u is its out-neighbours, each edge
 * (u, v) gives v in N_u only, and d_u is the out-degree. Rows are sorted by (d_out(v), v).
 * directed = 2: the untransposed adjacency of the same passage (single-target PPR): r^(i+1)(v)
 * sums over the out-neighbours u of v, so the push list of u is its in-neighbours, while d stays
 * the out-degree; rows are sorted by (d_out(v), v) and their length is the in-degree. */
static int64_t build_csr(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, int add_self_loops,
                         int directed, int64_t *rowptr, int32_t *colidx, int32_t *deg)
{
    if (n < 0 || m < 0) return -1;
    for (int64_t e = 0; e < m; ++e)
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return -1;

    /* 1. count the kept directions of every non-loop edge */
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t e = 0; e < m; ++e) {
        if (src[e] == dst[e]) continue;
        if (directed != 2) cnt[src[e]]++;
        if (directed != 1) cnt[dst[e]]++;
    }
    int64_t *start = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    start[0] = 0;
    for (int64_t u = 0; u < n; ++u) start[u + 1] = start[u] + cnt[u] + (add_self_loops ? 1 : 0);
    int32_t *tmp = (int32_t *)malloc((size_t)(start[n] > 0 ? start[n] : 1) * sizeof(int32_t));
    int64_t *fill = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    for (int64_t u = 0; u < n; ++u) fill[u] = start[u];
    for (int64_t e = 0; e < m; ++e) {
        if (src[e] == dst[e]) continue;
        if (directed != 2) tmp[fill[src[e]]++] = dst[e];
        if (directed != 1) tmp[fill[dst[e]]++] = src[e];
    }
    if (add_self_loops)
        for (int64_t u = 0; u < n; ++u) tmp[fill[u]++] = (int32_t)u;

    /* 2. merge repeated neighbours: sort each row by id and keep the first of each run */
    int64_t *rowlen = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    for (int64_t u = 0; u < n; ++u) {
        int64_t len = fill[u] - start[u];
        qsort(tmp + start[u], (size_t)len, sizeof(int32_t), cmp_by_id);
        int64_t k = 0;
        for (int64_t j = 0; j < len; ++j)
            if (j == 0 || tmp[start[u] + j] != tmp[start[u] + j - 1]) tmp[start[u] + k++] = tmp[start[u] + j];
        rowlen[u] = k;
    }

    /* 3. degrees: the row length, except for in-neighbour rows, whose nodes keep their out-degree
     *    (the number of rows a node appears in) */
    for (int64_t u = 0; u < n; ++u) deg[u] = directed == 2 ? 0 : (int32_t)rowlen[u];
    if (directed == 2)
        for (int64_t u = 0; u < n; ++u)
            for (int64_t j = 0; j < rowlen[u]; ++j) deg[tmp[start[u] + j]]++;

    /* 4. compact into the output and sort every row by (degree, id) */
    rowptr[0] = 0;
    for (int64_t u = 0; u < n; ++u) rowptr[u + 1] = rowptr[u] + rowlen[u];
    for (int64_t u = 0; u < n; ++u)
        memcpy(colidx + rowptr[u], tmp + start[u], (size_t)rowlen[u] * sizeof(int32_t));
    g_sort_deg = deg;
    for (int64_t u = 0; u < n; ++u)
        qsort(colidx + rowptr[u], (size_t)rowlen[u], sizeof(int32_t), cmp_by_degree_then_id);
    g_sort_deg = NULL;

    int64_t nnz = rowptr[n];
    free(cnt); free(start); free(tmp); free(fill); free(rowlen);
    return nnz;
}

int64_t ora_build_csr(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                      int add_self_loops, int64_t *rowptr, int32_t *colidx, int32_t *deg)
{
    return build_csr(n, m, src, dst, add_self_loops, 0, rowptr, colidx, deg);
}

int64_t ora_build_csr_directed(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                               int add_self_loops, int64_t *rowptr, int32_t *colidx, int32_t *deg)
{
    return build_csr(n, m, src, dst, add_self_loops, 1, rowptr, colidx, deg);
}

int64_t ora_build_csr_directed_in(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                                  int add_self_loops, int64_t *rowptr, int32_t *colidx, int32_t *deg)
{
    return build_csr(n, m, src, dst, add_self_loops, 2, rowptr, colidx, deg);
}

/* ------------------------------------------------------------------------------------------ */
/* Weights and tail sums, Def. 3.1: Y_i = sum_{k >= i} w_k. Table 1 gives the weight sequences. */
/*   kind 0 FINITE:     the caller's w_0..w_L, zero beyond L, so Y_i = sum_{k=i..L} w_k.         */
/*   kind 1 PPR(alpha): w_i = alpha (1-alpha)^i, infinite tail, Y_i = (1-alpha)^i.              */
/*   kind 2 HKPR(t):    w_i = e^{-t} t^i / i!, infinite tail summed from far out inwards.        */
/*   kind 3 KATZ(beta): w_i = beta^i, infinite tail Y_i = beta^i / (1 - beta).                   */
/*   kind 4 TRANSITION: w_L = 1, all others 0, so Y_i = 1 for i <= L.                          */
/* Output: w[0..L] and Y[0..L+1] (Y_{L+1} is the tail beyond the truncation).                  */
/* ------------------------------------------------------------------------------------------ */
int ora_tail_sums(int kind, int L, double param, const double *w_in, double *w, double *Y)
{
    if (L < 0) return -1;
    switch (kind) {
    case 0:
        for (int i = 0; i <= L; ++i) w[i] = w_in[i];
        Y[L + 1] = 0.0;
        for (int i = L; i >= 0; --i) Y[i] = Y[i + 1] + w[i];
        return 0;
    case 1: {
        double alpha = param;
        if (!(alpha > 0.0 && alpha <= 1.0)) return -1;
        for (int i = 0; i <= L; ++i) w[i] = alpha * pow(1.0 - alpha, i);
        for (int i = 0; i <= L + 1; ++i) Y[i] = pow(1.0 - alpha, i);
        return 0;
    }
    case 2: {
        double t = param;
        if (!(t > 0.0)) return -1;
        /* w_k = exp(-t + k ln t - lgamma(k+1)); sum the tail from K (where w_K < 1e-300, past
         * the mode) down to i so that the smallest terms are added first. */
        int K = L + 2;
        while (K < 100000 && (K < t + 1.0 || -t + K * log(t) - lgamma(K + 1.0) > -690.0)) ++K;
        double acc = 0.0;
        for (int k = K; k >= 0; --k) {
            double wk = exp(-t + k * log(t) - lgamma(k + 1.0));
            acc += wk;
            if (k <= L + 1) Y[k] = acc;
            if (k <= L) w[k] = wk;
        }
        return 0;
    }
    case 3: {
        double beta = param;
        if (!(beta > 0.0 && beta < 1.0)) return -1;
        for (int i = 0; i <= L; ++i) w[i] = pow(beta, i);
        for (int i = 0; i <= L + 1; ++i) Y[i] = pow(beta, i) / (1.0 - beta);
        return 0;
    }
    case 4:
        for (int i = 0; i <= L; ++i) w[i] = (i == L) ? 1.0 : 0.0;
        for (int i = 0; i <= L; ++i) Y[i] = 1.0;
        Y[L + 1] = 0.0;
        return 0;
    default:
        return -1;
    }
}

/* d^{-p} with the reading D^{-p} := 0 at degree 0 for p > 0; D^0 = I, so p = 0 gives 1 at any
 * degree. (Undirected: a neighbour has degree >= 1, and a node of degree 0 pushes nothing, so
 * only the directed case meets degree 0 here: a node without out-edges still receives pushes
 * when a = 0.) */
static double deg_pow_neg(int32_t d, double p)
{
    if (p == 0.0) return 1.0;
    if (d == 0) return 0.0;
    return pow((double)d, -p);
}

/* ratio num/den with 0/0 := 0 (a zero tail stops the propagation) */
static double safe_ratio(double num, double den)
{
    return den > 0.0 ? num / den : 0.0;
}

/* ------------------------------------------------------------------------------------------ */
/* Algorithm 1 (Basic Propagation). r^(0) = x; for i = 0..L-1 every u with r^(i)(u) != 0 pushes */
/* (Y_{i+1}/Y_i) r^(i)(u) / (d_v^a d_u^b) to every v in N_u and reserves (w_i/Y_i) r^(i)(u);   */
/* finally q^(L) = (w_L/Y_L) r^(L). The result is sum_{i<=L} w_i (D^-a A D^-b)^i x / Y_0 * Y_0  */
/* -- the Y's cancel (Def. 3.1), so any positive rescaling of w gives the same output.         */
/* frontier_sizes (optional, L+1 entries): |{u : r^(i)(u) != 0}| per level.                    */
/* ------------------------------------------------------------------------------------------ */
int ora_basic(int64_t n, const int64_t *rowptr, const int32_t *colidx, const int32_t *deg,
              double a, double b, int L, const double *w, const double *Y,
              const double *x, double *pi, int64_t *frontier_sizes)
{
    double *r = (double *)calloc((size_t)n, sizeof(double));
    double *rn = (double *)calloc((size_t)n, sizeof(double));
    for (int64_t u = 0; u < n; ++u) { r[u] = x[u]; pi[u] = 0.0; }
    for (int i = 0; i < L; ++i) {
        double push = safe_ratio(Y[i + 1], Y[i]);
        double keep = safe_ratio(w[i], Y[i]);
        int64_t nz = 0;
        for (int64_t u = 0; u < n; ++u) {
            if (r[u] == 0.0) continue;
            ++nz;
            double du_b = deg_pow_neg(deg[u], b);
            for (int64_t e = rowptr[u]; e < rowptr[u + 1]; ++e) {
                int32_t v = colidx[e];
                rn[v] += push * r[u] * du_b * deg_pow_neg(deg[v], a);
            }
            pi[u] += keep * r[u];
        }
        if (frontier_sizes) frontier_sizes[i] = nz;
        double *t = r; r = rn; rn = t;
        memset(rn, 0, (size_t)n * sizeof(double));
    }
    double keepL = safe_ratio(w[L], Y[L]);
    int64_t nz = 0;
    for (int64_t u = 0; u < n; ++u) {
        if (r[u] != 0.0) ++nz;
        pi[u] += keepL * r[u];
    }
    if (frontier_sizes) frontier_sizes[L] = nz;
    free(r); free(rn);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Algorithm 2 (Randomized Propagation) with subset sampling done by its definition: each       */
/* remaining neighbour v of u is kept independently with probability                            */
/*     p_v = (1/eps) (Y_{i+1}/Y_i) r(u) / (d_u^b d_v^a),                                       */
/* and adds eps to r^(i+1)(v) when kept. Neighbours whose increment is >= eps are pushed        */
/* deterministically. Input x >= 0 with ||x||_1 <= 1 (Algorithm 2 input). The uniform for        */
/* neighbour slot j of u at level i is Philox word 0 of counter (u, i, j, 0x4F524131) under the */
/* 64-bit key `seed`.                                                                          */
/* stats (optional, 3 + (L+1) entries): [0] deterministic pushes, [1] Bernoulli trials,        */
/* [2] accepted samples, [3+i] |{u : r^(i)(u) != 0}|.                                          */
/* ------------------------------------------------------------------------------------------ */
int ora_randomized(int64_t n, const int64_t *rowptr, const int32_t *colidx, const int32_t *deg,
                   double a, double b, int L, const double *w, const double *Y, double eps,
                   const double *x, uint64_t seed, double *pi, int64_t *stats)
{
    double *r = (double *)calloc((size_t)n, sizeof(double));
    double *rn = (double *)calloc((size_t)n, sizeof(double));
    int64_t det = 0, trials = 0, accepted = 0;
    for (int64_t u = 0; u < n; ++u) { r[u] = x[u]; pi[u] = 0.0; }
    for (int i = 0; i < L; ++i) {
        double push = safe_ratio(Y[i + 1], Y[i]);
        double keep = safe_ratio(w[i], Y[i]);
        int64_t nz = 0;
        for (int64_t u = 0; u < n; ++u) {
            if (r[u] == 0.0) continue;
            ++nz;
            double du_b = deg_pow_neg(deg[u], b);
            for (int64_t e = rowptr[u]; e < rowptr[u + 1]; ++e) {
                int32_t v = colidx[e];
                double inc = push * r[u] * du_b * deg_pow_neg(deg[v], a);
                if (inc >= eps) {
                    rn[v] += inc;
                    ++det;
                } else if (inc > 0.0) {
                    double pv = inc / eps;
                    ++trials;
                    uint32_t j = (uint32_t)(e - rowptr[u]);
                    if (uniform01(seed, (uint32_t)u, (uint32_t)i, j, 0x4F524131u) < pv) {
                        rn[v] += eps;
                        ++accepted;
                    }
                }
            }
            pi[u] += keep * r[u];
        }
        if (stats) stats[3 + i] = nz;
        double *t = r; r = rn; rn = t;
        memset(rn, 0, (size_t)n * sizeof(double));
    }
    double keepL = safe_ratio(w[L], Y[L]);
    int64_t nz = 0;
    for (int64_t u = 0; u < n; ++u) {
        if (r[u] != 0.0) ++nz;
        pi[u] += keepL * r[u];
    }
    if (stats) {
        stats[0] = det; stats[1] = trials; stats[2] = accepted; stats[3 + L] = nz;
    }
    free(r); free(rn);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Binomial(N, p) by inversion: walk the pmf from 0 upwards until the uniform is covered.       */
/* pmf(0) = (1-p)^N, pmf(k+1) = pmf(k) (N-k)/(k+1) p/(1-p). Plain and exact up to rounding.    */
/* ------------------------------------------------------------------------------------------ */
static int64_t binomial_inversion(int64_t N, double p, double U)
{
    if (p <= 0.0 || N == 0) return 0;
    if (p >= 1.0) return N;
    double pmf = pow(1.0 - p, (double)N), cdf = pmf;
    int64_t k = 0;
    while (U > cdf && k < N) {
        pmf *= (double)(N - k) / (double)(k + 1) * p / (1.0 - p);
        ++k;
        cdf += pmf;
        if (pmf == 0.0 && cdf < U) break;
    }
    return k;
}

/* ------------------------------------------------------------------------------------------ */
/* Algorithm 2 with the paper's Subset Sampling scheme (Section 4): the remaining neighbours of */
/* u are split into groups G_k = {v : d_v in [2^k, 2^{k+1})}; in G_k draw ell ~ Binomial(|G_k|, */
/* p*), choose ell members uniformly without replacement, and reject each with probability      */
/* 1 - p_v/p*. p* is the largest probability among the remaining members of the group (the one */
/* of smallest degree), which keeps p* <= 1. Uniforms: counter (u, i, k, 0x47525053 + draw).   */
/* ------------------------------------------------------------------------------------------ */
int ora_randomized_groups(int64_t n, const int64_t *rowptr, const int32_t *colidx,
                          const int32_t *deg, double a, double b, int L, const double *w,
                          const double *Y, double eps, const double *x, uint64_t seed,
                          double *pi, int64_t *stats)
{
    double *r = (double *)calloc((size_t)n, sizeof(double));
    double *rn = (double *)calloc((size_t)n, sizeof(double));
    int64_t maxd = 1;
    for (int64_t u = 0; u < n; ++u) if (deg[u] > maxd) maxd = deg[u];
    int64_t *pick = (int64_t *)malloc((size_t)maxd * sizeof(int64_t));
    int64_t det = 0, trials = 0, accepted = 0;
    for (int64_t u = 0; u < n; ++u) { r[u] = x[u]; pi[u] = 0.0; }
    for (int i = 0; i < L; ++i) {
        double push = safe_ratio(Y[i + 1], Y[i]);
        double keep = safe_ratio(w[i], Y[i]);
        int64_t nz = 0;
        for (int64_t u = 0; u < n; ++u) {
            if (r[u] == 0.0) continue;
            ++nz;
            double du_b = deg_pow_neg(deg[u], b);
            int64_t e = rowptr[u], end = rowptr[u + 1];
            /* deterministic prefix: neighbours are in ascending degree, so inc decreases */
            while (e < end) {
                double inc = push * r[u] * du_b * deg_pow_neg(deg[colidx[e]], a);
                if (!(inc >= eps)) break;
                rn[colidx[e]] += inc;
                ++det;
                ++e;
            }
            /* remaining neighbours, group by group */
            while (e < end) {
                int32_t dfirst = deg[colidx[e]];
                int g = 0;
                while ((1LL << (g + 1)) <= dfirst) ++g;
                int64_t gend = e;
                while (gend < end && deg[colidx[gend]] < (1LL << (g + 1))) ++gend;
                double pstar = push * r[u] * du_b * deg_pow_neg(dfirst, a) / eps;
                int64_t size = gend - e;
                if (pstar > 0.0) {
                    uint32_t draw = 0;
                    double U = uniform01(seed, (uint32_t)u, (uint32_t)i, (uint32_t)g, 0x47525053u + draw++);
                    int64_t ell = binomial_inversion(size, pstar, U);
                    /* ell members uniformly without replacement: partial Fisher-Yates */
                    for (int64_t t = 0; t < size; ++t) pick[t] = e + t;
                    for (int64_t t = 0; t < ell; ++t) {
                        double V = uniform01(seed, (uint32_t)u, (uint32_t)i, (uint32_t)g, 0x47525053u + draw++);
                        int64_t s = t + (int64_t)(V * (double)(size - t));
                        if (s >= size) s = size - 1;
                        int64_t tmp = pick[t]; pick[t] = pick[s]; pick[s] = tmp;
                        int64_t slot = pick[t];
                        double pv = push * r[u] * du_b * deg_pow_neg(deg[colidx[slot]], a) / eps;
                        double A = uniform01(seed, (uint32_t)u, (uint32_t)i, (uint32_t)g, 0x47525053u + draw++);
                        ++trials;
                        if (A < pv / pstar) {
                            rn[colidx[slot]] += eps;
                            ++accepted;
                        }
                    }
                }
                e = gend;
            }
            pi[u] += keep * r[u];
        }
        if (stats) stats[3 + i] = nz;
        double *t = r; r = rn; rn = t;
        memset(rn, 0, (size_t)n * sizeof(double));
    }
    double keepL = safe_ratio(w[L], Y[L]);
    int64_t nz = 0;
    for (int64_t u = 0; u < n; ++u) {
        if (r[u] != 0.0) ++nz;
        pi[u] += keepL * r[u];
    }
    if (stats) {
        stats[0] = det; stats[1] = trials; stats[2] = accepted; stats[3 + L] = nz;
    }
    free(pick); free(r); free(rn);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Largest eigenvalue of the adjacency matrix by FP64 power iteration on A + I (the shift keeps  */
/* bipartite graphs from oscillating); returns lambda_1(A). Katz needs beta < 1/lambda_1        */
/* (Section 2, Katz row of Table 1); the experiments take beta = 0.85/lambda_1.                */
/* ------------------------------------------------------------------------------------------ */
double ora_power_lambda(int64_t n, const int64_t *rowptr, const int32_t *colidx, int iters,
                        double tol)
{
    if (n == 0) return 0.0;
    double *x = (double *)malloc((size_t)n * sizeof(double));
    double *y = (double *)malloc((size_t)n * sizeof(double));
    for (int64_t u = 0; u < n; ++u) x[u] = 1.0 / sqrt((double)n);
    double lam = 0.0;
    for (int it = 0; it < iters; ++it) {
        for (int64_t u = 0; u < n; ++u) {
            double s = x[u];
            for (int64_t e = rowptr[u]; e < rowptr[u + 1]; ++e) s += x[colidx[e]];
            y[u] = s;
        }
        double nrm = 0.0, rq = 0.0;
        for (int64_t u = 0; u < n; ++u) { nrm += y[u] * y[u]; rq += x[u] * y[u]; }
        nrm = sqrt(nrm);
        double prev = lam;
        lam = rq - 1.0; /* Rayleigh quotient of A + I at the unit vector x, minus the shift */
        for (int64_t u = 0; u < n; ++u) x[u] = nrm > 0.0 ? y[u] / nrm : 0.0;
        if (it > 0 && fabs(lam - prev) <= tol * fabs(lam)) break;
    }
    free(x); free(y);
    return lam;
}

/* ------------------------------------------------------------------------------------------ */
/* Sweep for local clustering (Section 6, local clustering with HKPR): order the nodes by        */
/* pi(v)/d_v, largest first, and return the prefix S_i with the smallest conductance            */
/* Phi(S) = |cut(S)| / min(vol(S), 2m - vol(S)), vol(S) = sum of d_v over S, 2m = sum of all d.  */
/* Readings: only nodes with pi(v) > 0 and d_v > 0 are swept (a zero score gives no order, and    */
/* d_v = 0 gives no score); ties on the score go to the smaller id; prefixes run over i = 1 ..   */
/* min(swept, n - 1); a prefix whose min(vol, 2m - vol) is 0 is skipped. The graph is the        */
/* undirected CSR of ora_build_csr. Returns the best prefix size (0 when no prefix qualifies);    */
/* order (n entries, may be NULL) receives the swept nodes in order, phi_out the conductance.     */
/* ------------------------------------------------------------------------------------------ */
static const double *g_sweep_score;

static int cmp_sweep(const void *pa, const void *pb)
{
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    double sa = g_sweep_score[a], sb = g_sweep_score[b];
    if (sa != sb) return sa > sb ? -1 : 1;
    return (a > b) - (a < b);
}

int64_t ora_sweep_conductance(int64_t n, const int64_t *rowptr, const int32_t *colidx, const int32_t *deg,
                              const double *pi, int32_t *order, double *phi_out)
{
    if (n <= 0) return 0;
    double *score = (double *)malloc((size_t)n * sizeof(double));
    int32_t *nodes = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    char *in_s = (char *)calloc((size_t)n, 1);
    double two_m = 0.0;
    int64_t k = 0;
    for (int64_t v = 0; v < n; ++v) {
        two_m += (double)deg[v];
        score[v] = deg[v] > 0 ? pi[v] / (double)deg[v] : 0.0;
        if (deg[v] > 0 && pi[v] > 0.0) nodes[k++] = (int32_t)v;
    }
    g_sweep_score = score;
    qsort(nodes, (size_t)k, sizeof(int32_t), cmp_sweep);
    g_sweep_score = NULL;
    int64_t last = k < n - 1 ? k : n - 1;
    double vol = 0.0, cut = 0.0, best = INFINITY;
    int64_t best_i = 0;
    for (int64_t i = 0; i < last; ++i) {
        int32_t v = nodes[i];
        /* adding v: its edges into S stop being cut, its other edges start being cut */
        int64_t inside = 0;
        for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e)
            if (in_s[colidx[e]] && colidx[e] != v) ++inside;
        int64_t loops = 0;
        for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e) loops += colidx[e] == v;
        in_s[v] = 1;
        vol += (double)deg[v];
        cut += (double)(deg[v] - loops - 2 * inside);
        double den = vol < two_m - vol ? vol : two_m - vol;
        if (den > 0.0 && cut / den < best) {
            best = cut / den;
            best_i = i + 1;
        }
    }
    if (order)
        for (int64_t i = 0; i < n; ++i) order[i] = i < k ? nodes[i] : -1;
    if (phi_out) *phi_out = best_i > 0 ? best : NAN;
    free(score); free(nodes); free(in_s);
    return best_i;
}
