/*
 * agp.h -- C ABI of the GB300 library for Approximate Graph Propagation
 * (Wang, He, Wei, Wang, Yuan, Du, Wen: "Approximate Graph Propagation", KDD'21, arXiv:2106.03058).
 *
 * The library estimates the graph propagation vector of Eq. (1), Section 2,
 *
 *     pi = sum_{i=0..L} w_i (D^-a A D^-b)^i x ,
 *
 * with the level-by-level randomized push of Algorithm 2 (Section 4): at level i every node u with
 * a non-zero residue r^(i)(u) reserves (w_i/Y_i) r^(i)(u) (Def. 3.1, Y_i = sum_{k>=i} w_k),
 * pushes the increment (Y_{i+1}/Y_i) r^(i)(u) / (d_u^b d_v^a) to every neighbour v for which that
 * increment is >= eps (a prefix of the degree-sorted adjacency list, Section 4 "Pre-sorting"), and
 * subset-samples every other neighbour with probability increment/eps, adding eps when sampled
 * (Section 4 "Subset Sampling"). eps = 0 gives Algorithm 1 (exact propagation).
 *
 * Conventions shared by every entry point:
 *  - Every call returns an int status (AGP_OK = 0 or one of the AGP_E* codes below). No call
 *    aborts, traps or exits the process. agp_last_error_detail() gives a message for the last
 *    failure on the calling thread.
 *  - Device pointers are CUDA device addresses on the graph's device; host pointers are ordinary
 *    process memory (pageable or pinned). Each argument states which one it takes.
 *  - The caller owns every input and output buffer. The library owns the graph (device CSR and
 *    its work buffers) until agp_graph_destroy, and serving results until agp_serve_release.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Calls are stream-ordered and
 *    return once their work is enqueued, except where an entry point says it synchronises.
 *  - One graph handle must not be used by two host threads at the same time.
 *  - Node ids are int32 in [0, n). Degrees count distinct neighbours.
 */
#ifndef AGP_H
#define AGP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define AGP_API __attribute__((visibility("default")))
#else
#define AGP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------- */
#define AGP_OK 0
#define AGP_EINVAL 1     /* an argument is out of range or inconsistent                       */
#define AGP_ENOMEM 2     /* a device or host allocation failed                                 */
#define AGP_ECUDA 3      /* a CUDA runtime call failed (detail names it)                       */
#define AGP_EBUDGET 4    /* the request does not fit the configured memory budget              */
#define AGP_EAGAIN 5     /* serving: the result is not ready yet                               */
#define AGP_ETIMEDOUT 6  /* a bounded wait ran out                                             */
#define AGP_ECANCELED 7  /* serving: the request was cancelled                                 */
#define AGP_EINTERNAL 8  /* a device-side consistency check failed (capacity, bounds)          */

/* Human-readable name of a status code (static storage). */
AGP_API const char *agp_strerror(int code);
/* Message describing the last failure on the calling thread (thread-local storage, valid until
 * the next failing call on this thread). Empty string if none. */
AGP_API const char *agp_last_error_detail(void);
/* Library version as 10000*major + 100*minor + patch. */
AGP_API int agp_version(void);

/* ---- graph -------------------------------------------------------------------------------- */
typedef struct agp_graph_s *agp_graph_t;

#define AGP_ADD_SELF_LOOPS 0x1u  /* add one self-loop per node, counted once in its degree        */
#define AGP_EDGES_ON_DEVICE 0x2u /* src/dst are device pointers (else host pointers)               */
#define AGP_DIRECTED 0x4u        /* directed graph, out-neighbour rows: see below                  */
#define AGP_DIRECTED_IN 0x8u     /* directed graph, in-neighbour rows: see below                   */

/*
 * Build the device CSR of an undirected graph: Section 4 "Pre-sorting adjacency list by degrees".
 * Every input edge (src[e], dst[e]) makes each endpoint a neighbour of the other; repeated edges
 * are merged and input self-loops dropped. With AGP_ADD_SELF_LOOPS every node then gets exactly
 * one self-loop (the self-looped graph of SGC/GCN, Section 1). Each adjacency list N_u is stored
 * in ascending (d_v, v) order, so the neighbours of small degree form a prefix.
 * AGP_DIRECTED: Section 4, "Propagation on directed graph", with the transposed adjacency that the
 * paper uses for PageRank, PPR, HKPR and Katz: pi = sum_i w_i (D^-a A^T D^-b)^i x, D the out-degree
 * matrix. Each edge (src[e], dst[e]) is directed src -> dst; N_u is the out-neighbour list of u and
 * d_u its out-degree (rowptr, colidx and deg of agp_graph_info are these), so the propagation
 * pushes along out-edges. Queries on a directed graph need a = 0 (AGP_EINVAL otherwise): a node
 * without out-edges would have d^-a undefined. A node without out-edges keeps what reaches it as
 * reserve and passes nothing on (D^-1 := 0).
 * AGP_DIRECTED_IN: the untransposed adjacency of the same passage (single-target PPR, a = 1, b = 0):
 * pi = sum_i w_i (D^-a A D^-b)^i x with (A y)(u) = sum_{v : u -> v} y(v) and D the out-degree matrix.
 * In push form a node v passes r(v) / (d_v^b d_u^a) to every in-neighbour u (u -> v), so N_v is the
 * in-neighbour list of v, sorted by (d_u, u), while deg[] stays the out-degree: a row's length
 * (rowptr[v+1] - rowptr[v], the in-degree) is not its node's degree here. Any a, b is valid (every
 * push target has an out-edge); a node without out-edges pushes nothing when b > 0 (D^-b := 0).
 * The two directed flags exclude each other.
 *   n        number of nodes, 0 <= n < 2^31
 *   n_edges  number of input edges (>= 0)
 *   src,dst  n_edges int32 ids each, host or device memory (AGP_EDGES_ON_DEVICE); not retained
 *   device   CUDA device ordinal that will hold the graph
 *   stream   stream for the build; the call synchronises it before returning
 *   out      receives the handle
 * Errors: AGP_EINVAL (bad n, id out of range), AGP_ENOMEM, AGP_ECUDA.
 */
AGP_API int agp_build_graph(int64_t n, int64_t n_edges, const int32_t *src, const int32_t *dst,
                    uint32_t flags, int device, void *stream, agp_graph_t *out);

/* Sizes and device arrays of a built graph (library-owned, valid until agp_graph_destroy):
 * rowptr int64[n+1], colidx int32[nnz], deg int32[n] (row lengths, except with AGP_DIRECTED_IN where
 * deg holds out-degrees). Any output pointer may be NULL. */
AGP_API int agp_graph_info(agp_graph_t g, int64_t *n, int64_t *nnz, const int64_t **rowptr,
                   const int32_t **colidx, const int32_t **deg);

/* Free the graph and every work buffer it owns. Synchronises the device first. */
AGP_API int agp_graph_destroy(agp_graph_t g);

/* Device memory (bytes) the graph may use for query work buffers; 0 = default (60% of the free
 * device memory at the first query). Work buffers are sized from it and reused across calls. */
AGP_API int agp_graph_set_memory_budget(agp_graph_t g, int64_t bytes);

/* Lanes (sign parts of queries or feature columns) propagated together in one wave; 0 = automatic:
 * as many as keep their residue vectors within ~96 MB of L2. agp_autotune picks it by timing. */
AGP_API int agp_graph_set_wave_lanes(agp_graph_t g, int32_t lanes);

/* Lanes per residue group: 1, 2 or 4 (0 = automatic: 4 when the wave width is a multiple of 4,
 * else 2 when it is even, else 1). The residues of a group's lanes are interleaved per node, so a
 * frontier node's row is walked once for all lanes of the group that hold it, and their increments
 * at a neighbour leave as one vector reduction. Results do not depend on it (a lane's random draws
 * are its own). The plain path always uses 1. agp_autotune picks it by timing. */
AGP_API int agp_graph_set_group_width(agp_graph_t g, int32_t width);

/* Direction of a level. On an undirected graph a lane whose frontier volume (sum of d_u over
 * r^(i)(u) != 0) is at least nnz >> shift computes level i by pulling: every node v walks its row
 * once for the lane's group and adds, per edge (u, v) with r(u) != 0, what Algorithm 2 pushes along
 * it (the deterministic increment when it passes the push test, else eps with the sampling
 * probability, the trial drawn from a stream keyed by (u, v, level)). There are no atomics; the
 * estimator and its distribution are those of the push. Smaller frontiers push. The decision is the
 * lane's own, so a lane's result does not depend on its batch. shift in [0, 62]; -1 = never pull
 * (the default). Pulling walks every edge and draws a trial for each sampled one, while pushing
 * skips through sparse tails: it pays only where nearly every edge of the graph carries a
 * deterministic increment (exact or large-residue levels); on the batched benchmark's eps = 1e-8
 * Katz levels it was several times slower. Directed graphs always push. */
AGP_API int agp_graph_set_pull_threshold(agp_graph_t g, int32_t shift);

/* Columns per tile of exact feature propagation (agp_feature_propagate with eps = 0 on an undirected
 * graph): 8, 16 or 32 (0 = automatic: the widest whose n x T FP32 residue block stays within 64 MB,
 * half of L2, at least 8). */
AGP_API int agp_graph_set_column_tile(agp_graph_t g, int32_t columns);

/* ---- propagation parameters ---------------------------------------------------------------- */
/* Weight sequences of Table 1. FINITE takes w_0..w_L from `w`; the others are generated with
 * their infinite tails Y_i = sum_{k>=i} w_k (Def. 3.1):
 *   PPR(param = alpha):  w_i = alpha (1-alpha)^i            (PageRank, PPR, APPNP)
 *   HKPR(param = t):     w_i = e^-t t^i / i!                (heat kernel PageRank, GDC)
 *   KATZ(param = beta):  w_i = beta^i, 0 < beta < 1         (Katz; beta < 1/lambda_1 for convergence)
 *   TRANSITION:          w_L = 1, other w_i = 0             (L-hop transition probability, SGC)   */
#define AGP_W_FINITE 0
#define AGP_W_PPR 1
#define AGP_W_HKPR 2
#define AGP_W_KATZ 3
#define AGP_W_TRANSITION 4

#define AGP_MAX_LEVELS 64 /* L <= AGP_MAX_LEVELS - 1 */

typedef struct {
    double a, b;          /* Laplacian parameters, each in [0, 1] (Eq. 1)                         */
    int32_t L;            /* number of levels, 0 <= L < AGP_MAX_LEVELS                            */
    int32_t kind;         /* AGP_W_*                                                              */
    double param;         /* alpha, t or beta for PPR, HKPR, KATZ                                 */
    const double *w;      /* FINITE only: host array of L+1 non-negative weights, sum > 0        */
    double eps;           /* error parameter of Algorithm 2, >= 0; 0 = exact (Algorithm 1)        */
    uint64_t seed;        /* random stream of this query (see agp_query_batch for shared params)  */
} agp_params_t;

/* Per-query counters (Theorem 4.3 counts cost as deterministic pushes plus accepted samples). */
typedef struct {
    int64_t frontier[AGP_MAX_LEVELS]; /* |{u : r^(i)(u) != 0}| per level, summed over sign parts */
    int64_t det_edge_ops;             /* deterministic pushes (Algorithm 2, push loop)           */
    int64_t samples_drawn;            /* candidate positions reached by the geometric skips      */
    int64_t samples_accepted;         /* samples that added eps                                  */
    /* the same counters split by the kernel that did the work (0 = expand, 1 = push, 2 = sample;
     * see agp_profile_read): [kernel][0 deterministic pushes, 1 trials, 2 accepted, 3 frontier
     * appends]                                                                                   */
    int64_t by_kernel[3][4];
    int32_t levels;                   /* L + 1 entries of `frontier` are meaningful              */
    float done_ms;                    /* AGP_QUERY_TIMES: device time from the start of the call's
                                         first wave to the end of the wave that finished this query
                                         (CUDA events); 0 otherwise                              */
} agp_stats_t;

/* Memory-location flags of the query entry points. */
#define AGP_INPUT_ON_DEVICE 0x1u  /* x_off / x_idx / x_val are device pointers                */
#define AGP_OUTPUT_ON_DEVICE 0x2u /* pi_out is a device pointer                                */
#define AGP_PLAIN 0x4u            /* plain path: one query per launch sequence, host-synchronised
                                     frontier sizes (the baseline the batched path is measured
                                     against); same kernels, same results                      */
#define AGP_COLLECT_STATS 0x8u    /* fill `stats` (adds counter atomics to the kernels)        */
#define AGP_PROFILE 0x10u         /* record CUDA events around every kernel of the level loop
                                     (inside the captured graph as well); read the per-kernel
                                     device time with agp_profile_read                          */
#define AGP_QUERY_TIMES 0x80u     /* fill stats[q].done_ms: one CUDA event per wave (no counter
                                     atomics); needs stats                                      */
#define AGP_SAMPLER_GROUPS 0x100u /* subset sampling by the paper's scheme (Section 4): per degree
                                     group a Binomial(|G_k|, p*) count of trials at uniformly chosen
                                     positions, each kept with p_v / p*, instead of geometric skips
                                     and per-position trials (same distribution; for the sampler's
                                     ablation). Such lanes always push                           */
#define AGP_EPS_ABSOLUTE 0x20u    /* eps is in the raw units of the signal: a sign part x+- runs
                                     with eps / ||x+-||_1 on its normalised residues. Default
                                     (flag clear): eps applies to the normalised residues, the
                                     convention of Section 3 and Algorithm 2                     */

/*
 * Batched queries (Algorithm 2 per query). Query q has the sparse signal
 *     x_q = sum_{t = x_off[q] .. x_off[q+1]-1} x_val[t] * e_{x_idx[t]}
 * (x_val == NULL means all ones; repeated indices add up). Negative entries are handled as
 * Section 3 states: x = x+ + x-, each part normalised to unit L1 norm and propagated with its own
 * random stream, pi = ||x+||_1 pi(x+/||x+||_1) - ||x-||_1 pi(x-/||x-||_1). Weights are normalised
 * by Y_0 and the result rescaled (Section 3, "Assumptions on w_i"). eps applies to the normalised
 * residues.
 *   params    n_params == 1: shared by all queries, and query q draws its random numbers from the
 *             stream (seed, q), so queries of one batch do not repeat one another's draws; n_params
 *             == Q: one per query (host memory), each query drawing from its own seed alone, so a
 *             query gives the same draws in any batch and at any position
 *   x_off     Q+1 int64 offsets; x_idx / x_val as above; host or device (AGP_INPUT_ON_DEVICE)
 *   pi_out    Q rows of ld_out >= n floats, row q = estimate of pi for query q (dense FP32);
 *             host or device (AGP_OUTPUT_ON_DEVICE). Every entry of each row [0, n) is written.
 *   stats     NULL or Q entries (host memory): counters with AGP_COLLECT_STATS, completion times
 *             with AGP_QUERY_TIMES (either flag needs stats)
 * The call synchronises `stream` when pi_out or stats are host memory.
 * Errors: AGP_EINVAL (parameter out of range, index out of range when inputs are on the host),
 * AGP_ENOMEM / AGP_EBUDGET (work buffers), AGP_ECUDA, AGP_EINTERNAL (device-side check).
 */
AGP_API int agp_query_batch(agp_graph_t g, const agp_params_t *params, int32_t n_params, int32_t Q,
                    const int64_t *x_off, const int32_t *x_idx, const float *x_val,
                    float *pi_out, int64_t ld_out, uint32_t flags, agp_stats_t *stats,
                    void *stream);

/* One query: agp_query_batch with Q = 1. */
AGP_API int agp_query(agp_graph_t g, const agp_params_t *params, int64_t x_nnz, const int32_t *x_idx,
              const float *x_val, float *pi_out, uint32_t flags, agp_stats_t *stats,
              void *stream);

/*
 * Batched queries with dense signals (Algorithm 2 per query; Table 1's PageRank row uses x = 1/n):
 * query q has the dense signal x_q(u) = X[q * ldx + u], u < n, in FP32, or in bfloat16 (raw 16-bit
 * patterns) with AGP_DENSE_BF16. Sign parts, normalisation, eps and output are as for
 * agp_query_batch; the parts' L1 norms are reduced in a fixed order (no atomics), so they do not
 * depend on scheduling.
 *   X        Q rows of ldx >= n elements; host or device (AGP_INPUT_ON_DEVICE). Host rows are
 *            copied to the graph's device staging first.
 *   pi_out   Q rows of ld_out >= n floats; host or device (AGP_OUTPUT_ON_DEVICE)
 *   flags    AGP_INPUT_ON_DEVICE, AGP_OUTPUT_ON_DEVICE, AGP_PLAIN, AGP_COLLECT_STATS, AGP_PROFILE,
 *            AGP_QUERY_TIMES, AGP_EPS_ABSOLUTE, AGP_DENSE_BF16, AGP_SAMPLER_GROUPS
 * The call synchronises `stream` once after the norms, and at the end when pi_out or stats are host
 * memory. Errors as agp_query_batch (a non-finite entry of X: AGP_EINVAL).
 */
#define AGP_DENSE_BF16 0x40u
AGP_API int agp_query_dense(agp_graph_t g, const agp_params_t *params, int32_t n_params, int32_t Q, const void *X,
                            int64_t ldx, float *pi_out, int64_t ld_out, uint32_t flags, agp_stats_t *stats,
                            void *stream);

/*
 * Feature propagation for GNNs (Section 5.2; SGC, APPNP and GDC rows of Table 1): every column
 * c of X is a graph signal, Z[:, c] = estimate of sum_i w_i (D^-a A D^-b)^i X[:, c]. Columns are
 * split into sign parts and normalised as in agp_query_batch; eps applies per normalised part
 * (flags AGP_PLAIN, AGP_PROFILE, AGP_SAMPLER_GROUPS and AGP_EPS_ABSOLUTE; with the last, eps is in X's
 * raw units).
 *   X       device, n rows x d columns of bfloat16 (raw 16-bit patterns), row stride ldx >= d
 *   Z       device, n rows x d columns of FP32, row stride ldz >= d; fully written
 *   seed    of params: column c part s uses the stream (seed, c, s)
 * d = 0 (or n = 0) returns AGP_OK without touching X or Z, which may then be NULL.
 * eps = 0 on an undirected graph (without AGP_PLAIN) takes the exact path: Algorithm 1, Z = sum_i w_i
 * P^i X, computed over tiles of columns (agp_graph_set_column_tile) by pulling over the symmetric rows,
 * without sign parts or atomics; it keeps two n x T FP32 blocks with the graph.
 * Errors as agp_query_batch.
 */
AGP_API int agp_feature_propagate(agp_graph_t g, const agp_params_t *params, const uint16_t *X,
                          int64_t d, int64_t ldx, float *Z, int64_t ldz, uint32_t flags,
                          void *stream);

/*
 * Katz spectral bound (Table 1, Katz row; the experiments use beta = 0.85 / lambda_1): lambda_1
 * of A by FP64 power iteration on the device (iterating A + I so that bipartite graphs converge),
 * stopping when the Rayleigh quotient changes by <= tol relatively or after `iters` steps.
 * beta = fraction / lambda_1. Synchronises `stream`. Outputs are host pointers (may be NULL).
 * On a directed graph (AGP_DIRECTED) the iteration runs on the out-neighbour rows, i.e. on A,
 * whose spectral radius is that of A^T; it may need more steps to converge than on a symmetric A.
 */
AGP_API int agp_katz_beta(agp_graph_t g, double fraction, int32_t iters, double tol, double *beta,
                  double *lambda1, void *stream);

/* ---- serving ----------------------------------------------------------------------------------- */
/*
 * Continuous-batching server over a resident graph. Requests (single-source proximity queries or
 * BF16 feature blocks) are admitted into lanes ("slots") as lanes and result memory free up; every
 * sweep advances every admitted lane by one level of Algorithm 2 in shared launches, so requests
 * that arrive while others run join the next sweep. Each lane keeps its own level, coefficients and
 * random stream, so a request's result does not depend on what it shares sweeps with (up to FP32
 * atomic summation order). A host thread owned by the server drives the device on its own stream.
 */
typedef struct agp_server_s *agp_server_t;

#define AGP_SERVE_BATCHED 0     /* continuous batching (default)                                     */
#define AGP_SERVE_FIFO_PLAIN 1  /* baseline: one request at a time on the plain path, arrival order  */

#define AGP_ADMIT_COST 0  /* cheapest estimated cost first, with aging (default)                     */
#define AGP_ADMIT_FIFO 1  /* arrival order                                                           */

typedef struct {
    int32_t mode;             /* AGP_SERVE_*                                                        */
    int32_t max_lanes;        /* slots (lanes) per pool; 0 = max(8 x automatic wave width, 128)     */
    int64_t result_budget;    /* bytes of result buffers of admitted, unreleased requests; 0 = 4 GiB */
    int32_t results_on_host;  /* 1: results are copied to library-owned pinned host memory          */
    int32_t admission;        /* AGP_ADMIT_* (batched mode). Requests are split by estimated cost
                                 into a light pool (below 2^23 ~ 8.4e6 operations) and a heavy pool,
                                 each with max_lanes slots, its own workspace, stream and sweeps, so
                                 light sweeps never wait for heavy lanes. Heavy sweeps yield: one
                                 starts only while the light pool is idle, or once a heavy request
                                 has waited over 30 s (then its sweeps run beside the light ones
                                 until it is done). The estimate is the edge
                                 bound of the proof of Theorem 4.3, (1/eps) sum_{i=1..L} (Y_i/Y_0)
                                 ||P^i x||_1 (the mass bounded per weight kind), plus one frontier
                                 item per non-zero residue and level ((L+1) n/2 per sign part of a
                                 feature column). Within a pool a request's priority is cost / (1 +
                                 seconds waited), compared between the oldest waiting requests of its
                                 cost classes (floor(log2 cost)); a request that has waited over 30 s
                                 is admitted next, nothing else of its pool starting until its slots
                                 are free                                                           */
} agp_serve_config_t;

#define AGP_REQ_X_ON_DEVICE 0x1u   /* X is a device pointer that stays valid until the request is done */
#define AGP_REQ_EPS_ABSOLUTE 0x2u  /* eps in the raw units of the signal, as AGP_EPS_ABSOLUTE          */

typedef struct {
    agp_params_t params;      /* a, b, L, weights, eps, seed                                         */
    int32_t source;           /* >= 0: x = e_source; -1: feature request                            */
    int32_t cols;             /* feature request: number of columns (1..1024)                        */
    const uint16_t *X;        /* feature request: BF16 matrix n x cols, row stride ldx; host memory
                                 is copied by agp_serve_submit, device memory (AGP_REQ_X_ON_DEVICE)
                                 is read in place                                                    */
    int64_t ldx;
    int64_t deadline_us;      /* > 0: a request not admitted within this many microseconds of its
                                 submission finishes with AGP_ETIMEDOUT                              */
    uint32_t flags;           /* AGP_REQ_*                                                           */
    int32_t reserved;
} agp_request_t;

typedef struct {
    int32_t status;           /* AGP_OK, AGP_ETIMEDOUT, AGP_ECANCELED or an error code               */
    int32_t on_host;          /* 1: `pi` is host memory, 0: device memory                           */
    const float *pi;          /* library-owned: n floats (query) or n x cols row-major (features);  */
    int64_t n, cols;          /*   valid until agp_serve_release                                     */
    double queue_us;          /* submission -> admission                                             */
    double latency_us;        /* submission -> result ready                                          */
} agp_result_t;

/* Create a server over graph g (which must outlive it). Errors: AGP_EINVAL, AGP_ENOMEM, AGP_ECUDA. */
AGP_API int agp_serve_create(agp_graph_t g, const agp_serve_config_t *config, agp_server_t *out);
/* Queue a request; thread-safe. Validation errors are returned immediately (AGP_EINVAL). */
AGP_API int agp_serve_submit(agp_server_t s, const agp_request_t *req, uint64_t *ticket);
/* AGP_OK and *out filled when done (out->status tells how it ended), AGP_EAGAIN while pending. */
AGP_API int agp_serve_poll(agp_server_t s, uint64_t ticket, agp_result_t *out);
/* Wait up to timeout_us (< 0: no limit) for a result; AGP_ETIMEDOUT if it is still pending. */
AGP_API int agp_serve_wait(agp_server_t s, uint64_t ticket, int64_t timeout_us, agp_result_t *out);
/* Wait up to timeout_us (< 0: no limit) for the next request to finish, in completion order:
 * *ticket and *out are filled (AGP_OK), or AGP_ETIMEDOUT when none finished in time. Every finished
 * request is reported once; one released before it is reported is skipped. A client that takes its
 * results this way can release each as it arrives, which keeps the result budget free for
 * admissions. The queue of unreported completions is pruned of released requests, so a client that
 * never calls this function does not make it grow without bound. */
AGP_API int agp_serve_next(agp_server_t s, int64_t timeout_us, uint64_t *ticket, agp_result_t *out);
/* Free the result buffer of a finished request (pending requests: AGP_EINVAL). */
AGP_API int agp_serve_release(agp_server_t s, uint64_t ticket);
/* Cancel: a queued request finishes at once, an admitted one at the next sweep, with AGP_ECANCELED. */
AGP_API int agp_serve_cancel(agp_server_t s, uint64_t ticket);
/* Counters: completed requests, sweeps run, lanes in flight now, requests queued now. */
AGP_API int agp_serve_stats(agp_server_t s, int64_t *completed, int64_t *sweeps, int32_t *lanes_active,
                            int32_t *queued);
/* Stop the server thread (finishing nothing further), free everything. */
AGP_API int agp_serve_destroy(agp_server_t s);

/*
 * Autotuner of the wave width and the group width: runs the given batch (arguments as
 * agp_query_batch, output on the device) once per candidate pair (lanes from `candidates`,
 * n_candidates > 0, NULL = powers of two up to the batch's lane count; group width 1, 2 or 4
 * dividing the lanes), times each second run with CUDA events, keeps the fastest pair on the graph
 * (agp_graph_set_wave_lanes, agp_graph_set_group_width) and returns it. With the environment
 * variable AGP_TUNE_CACHE naming a file, results are cached there, keyed by graph size and parameter
 * signature, and a cached entry is used without timing. best_lanes / best_width / best_ms: host
 * pointers (may be NULL; best_ms = -1 for a cached entry).
 */
AGP_API int agp_autotune(agp_graph_t g, const agp_params_t *params, int32_t n_params, int32_t Q,
                         const int64_t *x_off, const int32_t *x_idx, const float *x_val, float *pi_out,
                         int64_t ld_out, uint32_t flags, const int32_t *candidates, int32_t n_candidates,
                         int32_t *best_lanes, int32_t *best_width, double *best_ms, void *stream);

/*
 * Kernel accounting of a graph handle since the last reset.
 *   ms[5], launches[5]  (host, may be NULL): device time in milliseconds and number of launches of
 *                       the level-loop steps measured under AGP_PROFILE, in the order
 *                       0 = compact (residue vectors -> ascending frontier item list, 3 kernels),
 *                       1 = expand (reserve, threshold, short pushes, light sampling),
 *                       2 = push (long deterministic prefixes, per-position dense tails),
 *                       3 = sample (sparse heavy tails), 4 = level end
 *   kernel_launches     (host, may be NULL): every kernel the library launched for this graph
 *                       (graph nodes included), with or without AGP_PROFILE
 *   reset               non-zero: clear the counters after reading
 */
AGP_API int agp_profile_read(agp_graph_t g, double *ms, int64_t *launches, int64_t *kernel_launches,
                             int reset);

/*
 * lambda_1 of A without any allocation. The paper has no counterpart: this is a deployment variant
 * of agp_katz_beta's power iteration for callers that may not allocate device memory while they
 * run (their device memory belongs to another allocator, or they avoid cudaMalloc/cudaFree
 * because those synchronise the device). It reads a CSR owned by the caller and keeps its iterate
 * vectors in a fixed array compiled into the library (64 MiB on every GPU that loads it, until the
 * process exits); it calls no cudaMalloc, cudaFree or other allocating routine.
 *   n       number of nodes, 1 <= n <= 4194304 (larger graphs: AGP_EINVAL; use agp_katz_beta)
 *   rowptr  device int64[n+1], colidx device int32[rowptr[n]] (undirected CSR as agp_graph_info
 *           returns it); caller-owned, only read
 *   iters, tol as agp_katz_beta; lambda1: host output
 *   stream  the call enqueues on it and synchronises it every iteration
 * Every call looks up the array's device address on the current device (cudaGetSymbolAddress, which
 * allocates nothing), so a device reset or another current context is handled. The first call on a
 * device may load the library's device code there: make that first call before any stream capture.
 * All calls share the one array and each starts by
 * re-initialising it, so calls that overlap on the GPU (other threads or streams) race: callers
 * must serialise them.
 */
AGP_API int agp_katz_lambda_noalloc(int64_t n, const int64_t *rowptr, const int32_t *colidx, int32_t iters,
                                    double tol, double *lambda1, void *stream);

/*
 * Threshold of the deterministic prefix (Algorithm 2 push condition, Section 4 pre-sorting):
 * for each t < count, k_out[t] = #{ j : c[t] / d_{v_j}^a >= eps } over the degree-sorted
 * N_{nodes[t]} = {v_1, ...}, with the comparison taken in FP64 from the FP32 value c[t]
 * (c = (Y_{i+1}/Y_i) r(u) / d_u^b as the push kernel computes it). a == 0 gives d_u or 0.
 * Exposes the step the push kernel uses, for parity checks. nodes, c, k_out: device arrays.
 */
AGP_API int agp_threshold(agp_graph_t g, double a, double eps, int64_t count, const int32_t *nodes,
                  const float *c, int32_t *k_out, void *stream);

/*
 * Local-clustering sweep (Section 6, local clustering with HKPR): the nodes are ordered by
 * pi(v)/d_v, largest first, and the prefix S_i of least conductance
 *     Phi(S_i) = cut(S_i) / min(vol(S_i), 2m - vol(S_i)),  vol(S) = sum_{v in S} d_v,
 * is found. Readings: only nodes with pi(v) > 0 and d_v > 0 are swept; ties on the score go to the
 * smaller id (the score is the FP64 quotient of the FP32 pi); prefixes run over i = 1..min(swept,
 * n - 1); a prefix with min(vol, 2m - vol) = 0 is skipped; a self-loop counts once in d_v and never
 * crosses the cut. The first prefix of least conductance wins.
 *   g          an undirected graph (AGP_EINVAL for directed ones)
 *   pi         device, n floats (a row of agp_query_batch output)
 *   order      device, n int32 or NULL: the swept nodes in order, -1 after them
 *   phi        device, n - 1 doubles or NULL: Phi(S_i) at [i - 1] for i = 1..min(swept, n - 1), +inf
 *              where skipped, 0 after
 *   best_size, best_phi, swept: host outputs (may be NULL): the best prefix size (0 if none
 *              qualifies, best_phi then NaN) and the number of swept nodes
 * Allocates device scratch for the call (O(n)) and synchronises `stream`.
 * Errors: AGP_EINVAL, AGP_ENOMEM, AGP_ECUDA.
 */
AGP_API int agp_sweep(agp_graph_t g, const float *pi, int32_t *order, double *phi, int64_t *best_size,
                      double *best_phi, int64_t *swept, void *stream);

/*
 * Sparse output: the k largest entries of each of Q result rows (serving and local-clustering
 * consumers need the top of pi, not a dense n-vector; returning k pairs instead of n floats cuts
 * device-to-host traffic by n / (2k)). Row q's entries are ordered by value, largest first, ties by
 * ascending node id (-0 counts as +0); the first k of that order are written to val[q * ldo + j],
 * idx[q * ldo + j], j < k. Exact: a radix select over the (value, id) order, one CTA per row, then a
 * sort of the k keys.
 *   pi       device, Q rows of ld >= n floats (an output of agp_query_batch / agp_query_dense); rows
 *            must not hold NaN
 *   k        1 <= k <= min(n, 2048)
 *   val, idx device, Q rows of ldo >= k entries, caller-owned
 * Stream-ordered, no synchronisation, no allocation. Errors: AGP_EINVAL, AGP_ECUDA.
 */
AGP_API int agp_topk(const float *pi, int64_t n, int64_t ld, int32_t Q, int32_t k, float *val, int32_t *idx,
                     int64_t ldo, void *stream);

/*
 * Approximation quality of an estimate against a reference (Section 6, local clustering with HKPR,
 * and the Katz experiments of the appendix): MaxError = max_v |pi_est(v)/d_v - pi_ref(v)/d_v|
 * (normalised by the degree) and Precision@k = |V_k ∩ V_hat_k| / k, where V_k and V_hat_k are the k
 * nodes of largest normalised reference and estimated value. With deg = NULL both use the plain
 * values (the Katz form of MaxError). A node with d_v = 0 has normalised value 0. MaxError is taken
 * in FP64 from the FP32 inputs. The top-k sets use agp_topk's order (value descending, ties by
 * ascending id) on the FP32 normalised values, so they are unique.
 *   pi_est, pi_ref  device FP32 n-vectors (no NaN)
 *   deg             device int32 n-vector (a graph's degrees, see agp_graph_info) or NULL
 *   k               1 <= k <= min(n, 2048), read only when precision_at_k is not NULL
 *   max_error       host, required; precision_at_k host or NULL
 * Allocates device scratch for the call (two n-vectors when normalising for Precision@k) and
 * synchronises the stream. Errors: AGP_EINVAL, AGP_ENOMEM, AGP_ECUDA.
 */
AGP_API int agp_compare(const float *pi_est, const float *pi_ref, int64_t n, const int32_t *deg, int32_t k,
                        double *max_error, double *precision_at_k, void *stream);

/*
 * Level coefficients of Def. 3.1 as the level pipeline computes them on the device (FP64), for a
 * signal part of unit L1 norm: with Y_i = sum_{k>=i} w_k,
 *     keep[i] = Y_0 * w_i / Y_i   (reserve factor of level i: pi(u) += keep[i] * r^(i)(u)),
 *     push[i] = Y_{i+1} / Y_i     (factor of every increment pushed at level i; 0 at i = L),
 * for i = 0..L, and *y0 = Y_0 (the normaliser of Section 3, "Assumptions on w_i"). Entries after a
 * zero tail are zero (nothing reaches those levels). The level kernels store keep (times the sign
 * part's norm) and push rounded to FP32. Exposes the step for parity checks.
 *   params  as for agp_query_batch (host); keep, push: host arrays of L+1 doubles; y0 may be NULL
 *   device  CUDA device ordinal to compute on; stream: enqueued there and synchronised
 * Allocates a few hundred bytes of device memory for the call.
 * Errors: AGP_EINVAL (parameters out of range, NULL arrays), AGP_ECUDA.
 */
AGP_API int agp_coefficients(const agp_params_t *params, double *keep, double *push, double *y0, int device,
                             void *stream);

#ifdef __cplusplus
}
#endif
#endif /* AGP_H */
