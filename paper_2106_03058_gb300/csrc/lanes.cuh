// lanes.cuh -- lane state of the level pipeline, shared by batched queries and the server.
//
// A lane is one propagation problem with a non-negative, L1-normalised signal (one sign part of a
// query or of a feature column, Section 3). Lanes own one dense FP32 residue vector (r^(i) until the
// level's compaction empties it, then r^(i+1)) and a coefficient row; their reserves accumulate at
// out[u * su].
#pragma once

#include <functional>
#include <vector>

#include "agp_internal.cuh"

namespace agp {

constexpr int kMaxLevels = AGP_MAX_LEVELS;
constexpr int kChunk = 512;          // prefix edges per chunk record (one warp)
constexpr int kMinBlocks = 4;        // resident CTAs per SM the level kernels are compiled for
constexpr int kCompactBlocks = 4;    // resident CTAs per SM of the compaction kernels; their grid is
                                     // this many per SM, so that every range is resident at once
constexpr int kCountBatch = 8;       // units per step of the count pass (loads in flight per thread)
constexpr int kInlineDet = 64;       // prefixes up to this length are pushed inline by the expansion
constexpr float kLightSamples = 16.f; // tails expected to yield at most this many trials stay inline
constexpr int kMinSeg = 256;         // shortest tail segment of a segment record
constexpr float kSegSamples = 64.f;  // expected trials of one segment record (a thread's share of a
                                     // heavy tail; its setup is a chain of dependent loads)
constexpr float kDenseP = 0.25f;     // tails whose largest probability is >= this are sampled per position
constexpr uint32_t kOffsetsOnHost = 0x80000000u;  // internal query flag: x_off is host memory even
                                                   // when x_idx / x_val are on the device
constexpr uint32_t kSampleTag = 0x53414D50u;  // Philox counter word of the skip sampler
constexpr uint32_t kDenseTag = 0x44534E53u;   // Philox counter word of the per-position sampler
constexpr uint32_t kPullTag = 0x50554C4Cu;    // Philox counter word of the edge trials of a pull level

struct LaneParam {
    double eps_d;     // eps (FP64) for the push/sample decision
    float eps;        // eps (FP32), the sampled increment
    float a, b;       // FP32 exponents for the increments
    double a_d;       // FP64 exponent a for the push/sample decision
    int32_t a_mode;   // 0: a = 0, 1: a = 1, 2: a = 1/2, 3: general
    int32_t b_mode;
    int32_t L;
    int32_t out_row;  // query / column index (statistics and bookkeeping)
    int32_t sampler;  // 0: geometric skips / per-position trials; 1: the paper's Binomial-count scheme
    uint32_t key0, key1;
    float *out;       // pi(u) of this lane accumulates at out[u * su]
    int64_t su;
    // derived by lane_param_derive (FP32 forms of the FP64 decision; the GPU's FP64 rate is low)
    float eps_up;          // smallest float f with (double)f >= eps_d: for a = 0, c >= eps_up is
                           // exactly (double)c >= eps_d
    float eps_lo, eps_hi;  // FP32 bracket of eps wider than the FP32 error of c / d^a
    float inv_eps;         // 1 / eps in FP32, for the sampling probabilities c / (eps d^a)
    int32_t screen;        // 1: decide in FP32 outside [eps_lo, eps_hi), FP64 only inside
};

// eps of a lane from an eps in raw signal units (AGP_EPS_ABSOLUTE): the lane runs on the sign part
// x+-/||x+-||_1, whose residues are those of the raw problem divided by ||x+-||_1 (the ratios
// Y_{i+1}/Y_i do not depend on the scale of w).
inline double lane_eps_absolute(double eps, double norm) { return norm > 0.0 ? eps / norm : eps; }

// Fill the derived fields of a lane whose eps_d, a_d and a_mode are set. For a in {1, 1/2} the FP32
// quotient c / d^a (correctly rounded division and square root) is within 2 ulp (2.4e-7 relative) of
// the exact value, for general 0 < a <= 1 (powf) well within 2^-16; the bracket is 2^-20 (resp.
// 2^-16) wide on each side, so a decision made outside it equals the FP64 one.
inline void lane_param_derive(LaneParam &P)
{
    const double e = P.eps_d;
    float f = (float)e;
    if ((double)f < e) f = nextafterf(f, INFINITY);
    P.eps_up = f;
    const double m = (P.a_mode == 3) ? 0x1p-16 : 0x1p-20;
    P.eps_lo = (float)(e * (1.0 - m));
    P.eps_hi = (float)(e * (1.0 + m));
    P.inv_eps = e > 0.0 ? (float)(1.0 / e) : 0.f;
    const bool a_ok = P.a_mode == 1 || P.a_mode == 2 || (P.a_mode == 3 && P.a_d > 0.0 && P.a_d <= 1.0);
    P.screen = (a_ok && e >= 1e-30 && e <= 1e30) ? 1 : 0;
}

struct LaneStats {
    unsigned long long frontier[kMaxLevels];
    unsigned long long by_kernel[3][4];  // [expand, push, sample][det, drawn, accepted, unused];
                                         // push counts the per-position tail sampler too
};

struct Ctrl {
    unsigned long long n_items;  // frontier size of the current level (set by the compaction)
    unsigned long long n_det, n_smp;  // walk-chunk and segment records of the current level
    unsigned int error;          // 1: frontier overflow, 2: chunk overflow, 4: segment overflow, 16: bad level
    unsigned int lanes_used;     // lanes [0, lanes_used) hold work; the compaction scans only those
    unsigned int scan_mode;      // compaction of the next level: 0 one pass (sparse frontier), 1 two passes
    unsigned long long prev_items;  // frontier size of the previous level (growth of the frontier)
};

constexpr int kProfKernels = 5;  // compact, expand, push, sample, level end
constexpr int kKernelsPerLevel = 9;  // compaction 3, expansion 3 (expand, record scan, record emit),
                                     // push, sample, level end
constexpr int kScanUnit = 1024;  // floats of a group's residue block scanned by one CTA step (256 x float4)
constexpr int kMaxGroupWidth = 4;  // lanes per group: a node's residues of a group fill one float4

// Residue layout: lanes are taken W at a time (W = 1, 2 or 4: the workspace's group width) into
// groups; group g owns the block R[g][ldR][W] (node-major, the W lanes of a node contiguous), so one
// frontier item is one (group, node) with W residues, its row is walked once for all W lanes, and
// the lanes' increments at a neighbour leave as one vector reduction.
struct KArgs {
    DevGraph g;
    int ubits;
    uint32_t umask;
    int W;                    // lanes per group
    int rows_in;              // rows are in-neighbour lists (deg[] is not the row length)
    int groups;               // the wave may hold lanes of the paper's group sampler
    float *C;                 // [G / W][ldR][W]: c(u) of the lanes that pull this level (else 0)
    unsigned long long *lane_count;  // [G] frontier volume (sum of d_u) of each lane, from the compaction
    int32_t *pull;            // [G] 1: the lane pulls this level; [G + g]: group g has a pulling lane
    int64_t pull_min;         // frontier volume from which a lane pulls (> nnz: never)
    const int32_t *rows[3];   // rows by length class (pull levels)
    int64_t row_count[3];
    float *R;                 // [G / W][ldR][W]
    uint32_t *items;          // current frontier, ascending (group << ubits | u)
    float *rval;              // [item][W]: r^(i)(u) of the group's lanes
    int64_t ldR;              // nodes per group block (n rounded up to kScanUnit / W)
    int64_t units;            // kScanUnit-float units per group block
    int64_t *part;            // per-range counts / offsets of the compaction
    int part_blocks;          // compaction ranges (blocks)
    float *c_item;            // [item][W] c = (Y_{i+1}/Y_i) r / d_u^b per lane (records only)
    int32_t *k_item;          // [item][W] deterministic prefix length per lane
    int32_t *seg_item;        // [item][W] sparse-tail segment length per lane
    uint32_t *flag_item;      // [item] bit j: lane j's tail is dense (per-position trials in the walk);
                              // bit 8 + j: lane j is in the walk; bit 16 + j: lane j has segments
    uint2 *nrec;              // per item: (walk chunks, sparse-tail segments)
    unsigned long long *rpart;  // [2][grid] per-block record counts / offsets
    uint2 *det_rec, *smp_rec;   // walk-chunk records (item, chunk), segment records (item, segment)
    unsigned long long cap_items, cap_det, cap_smp;
    const LaneParam *lanes;
    const float2 *coef;       // [G][kMaxLevels] (keep_i = scale * w_i/Y_i, push_i = Y_{i+1}/Y_i)
    int32_t *level;           // [G], -1 = idle
    LaneStats *stats;
    int collect;
    int G;
    int grid;                 // blocks of the grid-stride level kernels (8 per SM of the device)
    Ctrl *ctrl;
};

struct Workspace {
    int device = 0;
    int G = 0;
    int W = 1;                         // lanes per group (G is a multiple of W)
    int grid = 0;                      // grid-stride blocks of the device (rpart holds 2 rows of it)
    int64_t n = 0;
    unsigned long long cap_items = 0, cap_det = 0, cap_smp = 0;
    float *R = nullptr;
    uint32_t *items = nullptr;
    float *rval = nullptr;
    int64_t ldR = 0;
    int64_t *part = nullptr;
    int part_blocks = 1;
    float *c_item = nullptr;
    int32_t *k_item = nullptr;
    int32_t *seg_item = nullptr;
    uint32_t *flag_item = nullptr;
    uint2 *nrec = nullptr;
    unsigned long long *rpart = nullptr;
    uint2 *det_rec = nullptr, *smp_rec = nullptr;
    float *C = nullptr;
    unsigned long long *lane_count = nullptr;
    int32_t *pull = nullptr;
    LaneParam *lanes = nullptr;
    float2 *coef = nullptr;
    int32_t *level = nullptr;
    LaneStats *stats = nullptr;
    Ctrl *ctrl = nullptr;
    Ctrl *h_ctrl = nullptr;            // pinned
    LaneParam *h_lanes = nullptr;      // pinned
    // per-wave staging (grown on demand): device block for coefficient specs, weights and seed maps,
    // and a pinned host block it is filled from (so uploads need no stream synchronisation)
    void *stage = nullptr;
    size_t stage_bytes = 0;
    void *h_stage = nullptr;
    size_t h_stage_bytes = 0;
    int prof_levels = 0;           // AGP_PROFILE: levels whose events are not read yet
    bool pending = false;          // a wave was launched and not checked yet
    float *out_stage = nullptr;
    size_t out_stage_bytes = 0;
    // captured wave graph
    cudaGraphExec_t graph = nullptr;
    int graph_levels = -1;
    int graph_collect = -1;
    int graph_profile = -1;
    int graph_groups = -1;
    int64_t graph_pull = -2;   // pull threshold the graph was captured with (-1: pull off)
    // AGP_PROFILE events: [level][kernel][begin/end]
    cudaEvent_t ev[kMaxLevels][kProfKernels][2] = {};
    bool ev_ready = false;
    size_t bytes = 0;
};

struct CoefSpec {
    int32_t lane;      // workspace lane whose coefficient row is written
    int32_t kind, L;
    double param;
    int32_t w_off;     // FINITE: offset of w_0..w_L in the weight array
    double scale;      // sign * ||x_part||_1 (the Y_0 factor is applied here)
};

// Where a query call takes its work buffers: the graph's own (ws == nullptr) or a fixed workspace
// (the server's), with the staging buffer of its per-call inputs.
struct ExecCtx {
    Workspace *ws;
    void **stage;
    size_t *stage_bytes;
};

// ---- host helpers of propagate.cu shared with serve.cu -------------------------------------------
int query_batch_ctx(agp_graph_s *g, ExecCtx *ctx, const agp_params_t *params, int32_t n_params, int32_t Q,
                    const int64_t *x_off, const int32_t *x_idx, const float *x_val, float *pi_out,
                    int64_t ld_out, uint32_t flags, agp_stats_t *stats, cudaStream_t s);
int run_queries(agp_graph_s *g, ExecCtx *ctx, const agp_params_t *params, int32_t n_params, int32_t Q,
                const std::vector<double> &norms,
                const std::function<int(const KArgs &A, const int32_t *d_aux, cudaStream_t st)> &seed,
                float *pi_out, int64_t ld_out, uint32_t flags, agp_stats_t *stats, cudaStream_t s);
int feature_propagate_ctx(agp_graph_s *g, ExecCtx *ctx, const agp_params_t *params, const uint16_t *X, int64_t d,
                          int64_t ldx, float *Z, int64_t ldz, uint32_t flags, cudaStream_t s);
int exponent_mode(double p);
int validate_params(const agp_params_t &p);
int validate_params_for(const agp_graph_s *g, const agp_params_t &p);
void lane_key(uint64_t seed, uint64_t stream, int part, uint32_t &k0, uint32_t &k1);
size_t bytes_per_lane(const agp_graph_s *g);
int lane_capacity(const agp_graph_s *g);
// Group width of a wave of G lanes: 4 when G is a multiple of 4, else 2 when even, else 1.
inline int group_width(int G) { return (G % 4 == 0) ? 4 : (G % 2 == 0) ? 2 : 1; }
// grid > 0: blocks of the grid-stride level kernels (default 8 per SM); a smaller grid leaves SM
// slots to kernels of other streams (the server's heavy pool)
int create_workspace(agp_graph_s *g, int G, int W, Workspace **out, int grid = 0);
void drop_workspace(agp_graph_s *g);
KArgs make_args(agp_graph_s *g, Workspace *ws, int collect);
int blocks_for(unsigned long long work, int per_block);
void launch_level(const KArgs &A, cudaStream_t s, int expand_blocks, int push_blocks, int sample_blocks,
                  cudaEvent_t (*ev)[2] = nullptr);
void launch_compact(const KArgs &A, cudaStream_t s);
int capture_levels(const KArgs &A, int levels, cudaGraphExec_t *out);
void launch_coef(const CoefSpec *spec, const double *wts, float2 *coef, int nspec, cudaStream_t s);
void launch_seed_sources(const KArgs &A, const int32_t *lanes, const int32_t *sources, int count, cudaStream_t s);
void launch_colnorms_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ldx, double *norms, cudaStream_t s);
void launch_seed_dense_bf16(const KArgs &A, const uint16_t *X, int64_t ldx, const int32_t *lane_of,
                            const int32_t *col_of, const int32_t *part_of, const double *norms, int nl, cudaStream_t s);
int grow(void **p, size_t *have, size_t need);

}  // namespace agp
