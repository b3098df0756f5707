// propagate.cu -- the level-by-level randomized push of Algorithm 2 on the GPU.
//
// Unit of work: a "lane" = one propagation problem with a non-negative, L1-normalised signal (one
// sign part of one query or of one feature column, Section 3 "Assumption on graph signal"). A
// wave runs up to G lanes at once; every lane keeps two dense FP32 residue vectors (r^(i) and
// r^(i+1), swapped by level parity) and accumulates its reserve straight into the caller's output.
//
// One level of one lane, for every u with r^(i)(u) != 0 (Algorithm 2, inner loop):
//   k_expand   reads and clears r^(i)(u); reserve pi(u) += (w_i/Y_i) r^(i)(u);
//              c = (Y_{i+1}/Y_i) r^(i)(u) / d_u^b; deterministic prefix length k(u) = number of
//              neighbours with c / d_v^a >= eps (binary search over the degree-sorted row, or all
//              or nothing when a = 0); short prefixes and light tails are done by the same thread,
//              long prefixes become 1024-edge chunk records, heavy tails become segment records.
//   k_push     one warp per chunk record: r^(i+1)(v) += c / d_v^a for the prefix neighbours.
//   k_sample   one thread per segment record: subset sampling of the tail, Section 4: neighbours
//              are grouped by degree in [2^g, 2^{g+1}); in a group every position is a Bernoulli
//              trial with the group's largest probability p* (geometric skips, so the cost is the
//              number of trials reached, not the group size) and a reached neighbour is kept with
//              probability p_v/p*; a kept neighbour gets r^(i+1)(v) += eps.
//   k_level_end   swaps the frontier buffers and advances every lane's level.
// The frontier of the next level is built during the pushes: the thread whose atomic add finds the
// residue at zero appends (lane, v). Increments below FLT_MIN are dropped so that this first-touch
// test is exact. Sizes stay on the device; kernels are grid-stride loops over device-side counts,
// so a whole wave can be captured in one CUDA graph.
#include <cooperative_groups.h>

#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include "agp_internal.cuh"

namespace cg = cooperative_groups;

namespace agp {

constexpr int kMaxLevels = AGP_MAX_LEVELS;
constexpr int kChunk = 1024;         // prefix edges per chunk record (one warp)
constexpr int kInlineDet = 32;       // prefixes up to this length stay with the expanding thread
constexpr float kLightSamples = 4.f; // tails expected to yield at most this many trials stay inline
constexpr int kMinSeg = 256;         // shortest tail segment of a segment record
constexpr uint32_t kSampleTag = 0x53414D50u;

struct LaneParam {
    double eps_d;     // eps (FP64) for the push/sample decision
    float eps;        // eps (FP32), the sampled increment
    float a, b;       // FP32 exponents for the increments
    double a_d;       // FP64 exponent a for the push/sample decision
    int32_t a_mode;   // 0: a = 0, 1: a = 1, 2: a = 1/2, 3: general
    int32_t b_mode;
    int32_t L;
    int32_t out_row;
    uint32_t key0, key1;
};

struct LaneStats {
    unsigned long long frontier[kMaxLevels];
    unsigned long long by_kernel[3][4];  // [expand, push, sample][det, drawn, accepted, appends]
};

struct OutDesc {
    float *out;
    int64_t su, sr;   // pi(lane row, u) lives at out[u * su + row * sr]
};

struct Ctrl {
    unsigned long long n_items[2];
    unsigned long long n_det, n_smp;
    unsigned int cur;
    unsigned int error;  // 1: frontier overflow, 2: chunk overflow, 4: segment overflow, 8: bad index
    OutDesc od;
};

struct KArgs {
    DevGraph g;
    int ubits;
    uint32_t umask;
    float *R;                 // [2][G][n]
    size_t par_stride;        // G * n
    uint32_t *items0, *items1;
    float *c_item;
    int2 *k_item;             // (prefix length, tail segment length)
    uint2 *det_rec, *smp_rec;
    unsigned long long cap_items, cap_det, cap_smp;
    const LaneParam *lanes;
    const float2 *coef;       // [G][kMaxLevels] (keep_i = scale * w_i/Y_i, push_i = Y_{i+1}/Y_i)
    int32_t *level;           // [G], -1 = idle
    LaneStats *stats;
    int collect;
    int G;
    Ctrl *ctrl;
};

struct Workspace {
    int device = 0;
    int G = 0;
    int64_t n = 0;
    unsigned long long cap_items = 0, cap_det = 0, cap_smp = 0;
    float *R = nullptr;
    uint32_t *items[2] = {nullptr, nullptr};
    float *c_item = nullptr;
    int2 *k_item = nullptr;
    uint2 *det_rec = nullptr, *smp_rec = nullptr;
    LaneParam *lanes = nullptr;
    float2 *coef = nullptr;
    int32_t *level = nullptr;
    LaneStats *stats = nullptr;
    Ctrl *ctrl = nullptr;
    Ctrl *h_ctrl = nullptr;            // pinned
    LaneParam *h_lanes = nullptr;      // pinned
    // per-call staging (grown on demand)
    void *stage = nullptr;
    size_t stage_bytes = 0;
    float *out_stage = nullptr;
    size_t out_stage_bytes = 0;
    // captured wave graph
    cudaGraphExec_t graph = nullptr;
    int graph_levels = -1;
    int graph_collect = -1;
    int graph_profile = -1;
    // AGP_PROFILE events: [level][kernel][begin/end]
    cudaEvent_t ev[kMaxLevels][4][2] = {};
    bool ev_ready = false;
    size_t bytes = 0;
};

// ------------------------------------------------------------------------------------ helpers
__device__ __forceinline__ float deg_pow_neg_f(int32_t d, int mode, float p)
{
    // d^-p in FP32 for d >= 1
    switch (mode) {
    case 0: return 1.f;
    case 1: return __frcp_rn((float)d);
    case 2: return __frcp_rn(__fsqrt_rn((float)d));
    default: return powf((float)d, -p);
    }
}

__device__ __forceinline__ float apply_deg(float c, int32_t d, int mode, float p)
{
    // c / d^p in FP32
    switch (mode) {
    case 0: return c;
    case 1: return __fdiv_rn(c, (float)d);
    case 2: return __fdiv_rn(c, __fsqrt_rn((float)d));
    default: return c * powf((float)d, -p);
    }
}

// push condition of Algorithm 2 in FP64 from the FP32 value c: c / d^a >= eps
__device__ __forceinline__ bool push_test(float c, int32_t d, int mode, double a, double eps)
{
    const double cd = (double)c;
    switch (mode) {
    case 0: return cd >= eps;
    case 1: return cd / (double)d >= eps;
    case 2: return cd / sqrt((double)d) >= eps;
    default: return cd / pow((double)d, a) >= eps;
    }
}

// k(u): length of the deterministic prefix of the degree-sorted row (Section 4 pre-sorting).
__device__ __forceinline__ int det_prefix(float c, const LaneParam &P, const int32_t *row, int d,
                                          const int32_t *deg)
{
    if (P.eps_d == 0.0) return d;
    if (P.a_mode == 0) return ((double)c >= P.eps_d) ? d : 0;
    if (!push_test(c, deg[row[0]], P.a_mode, P.a_d, P.eps_d)) return 0;
    if (push_test(c, deg[row[d - 1]], P.a_mode, P.a_d, P.eps_d)) return d;
    int lo = 1, hi = d - 1;  // first failing position is in [1, d-1]
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (push_test(c, deg[row[mid]], P.a_mode, P.a_d, P.eps_d)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void append_item(const KArgs &A, uint32_t item, unsigned int buf, int lane, int lvl_next,
                                            int kern)
{
    cg::coalesced_group grp = cg::coalesced_threads();
    unsigned long long base = 0;
    if (grp.thread_rank() == 0) base = atomicAdd(&A.ctrl->n_items[buf], (unsigned long long)grp.size());
    base = grp.shfl(base, 0);
    const unsigned long long pos = base + grp.thread_rank();
    uint32_t *dst = buf ? A.items1 : A.items0;
    if (pos < A.cap_items) dst[pos] = item;
    else atomicOr(&A.ctrl->error, 1u);
    if (A.collect) {
        if (lvl_next < kMaxLevels) atomicAdd(&A.stats[lane].frontier[lvl_next], 1ull);
        if (kern >= 0) atomicAdd(&A.stats[lane].by_kernel[kern][3], 1ull);
    }
}

// r^(i+1)(v) += inc, first toucher appends (lane, v) to the next frontier
__device__ __forceinline__ void push_to(const KArgs &A, float *Rn, int lane, int32_t v, float inc,
                                        unsigned int nxt, int lvl_next, int kern)
{
    if (!(inc >= FLT_MIN)) return;
    const float old = atomicAdd(Rn + v, inc);
    if (old == 0.f) append_item(A, ((uint32_t)lane << A.ubits) | (uint32_t)v, nxt, lane, lvl_next, kern);
}

struct Uniforms {
    uint32_t c0, c1, k0, k1, blk;
    Philox4 cache;
    int used;
    __device__ Uniforms(uint32_t u, uint32_t lvl, uint32_t seg, uint32_t k0_, uint32_t k1_)
        : c0(u), c1(lvl | (seg << 8)), k0(k0_), k1(k1_), blk(0), used(4) {}
    __device__ float next()
    {
        if (used == 4) {
            cache = philox4x32_10(c0, c1, blk++, kSampleTag, k0, k1);
            used = 0;
        }
        const uint32_t b = (used == 0) ? cache.x : (used == 1) ? cache.y : (used == 2) ? cache.z : cache.w;
        ++used;
        return u01_open(b);
    }
};

// Subset sampling of row positions [j0, j1) (Section 4), stream (u, level, seg) of the lane.
__device__ void sample_range(const KArgs &A, const LaneParam &P, float *Rn, int lane, int32_t u, int lvl,
                             uint32_t seg, const int32_t *row, int j0, int j1, float c, unsigned int nxt,
                             unsigned long long &drawn, unsigned long long &accepted, int kern)
{
    Uniforms U((uint32_t)u, (uint32_t)lvl, seg, P.key0, P.key1);
    const float ce = (float)((double)c / P.eps_d);  // c / eps
    int j = j0;
    while (j < j1) {
        int gend = j1;
        float pstar;
        if (P.a_mode == 0) {
            pstar = ce;
        } else {
            const int32_t dj = A.g.deg[row[j]];
            pstar = apply_deg(ce, dj, P.a_mode, P.a);  // largest probability in the group
            const int g = 31 - __clz(dj);
            const int32_t glim = (g >= 30) ? INT_MAX : (1 << (g + 1));
            int lo = j + 1, hi = j1;  // first position with degree >= 2^{g+1}
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (A.g.deg[row[mid]] < glim) lo = mid + 1;
                else hi = mid;
            }
            gend = lo;
        }
        pstar = fminf(pstar, 1.f);
        if (!(pstar > 0.f)) { j = gend; continue; }
        const float lq = (pstar < 1.f) ? log1pf(-pstar) : -INFINITY;
        while (true) {
            const float skip = (pstar < 1.f) ? floorf(logf(U.next()) / lq) : 0.f;
            if (!(skip < (float)(gend - j))) { j = gend; break; }
            j += (int)skip;
            ++drawn;
            const int32_t v = row[j];
            bool keep = true;
            if (P.a_mode != 0) {
                const float pv = apply_deg(ce, A.g.deg[v], P.a_mode, P.a);
                keep = U.next() * pstar < pv;
            }
            if (keep) {
                ++accepted;
                push_to(A, Rn, lane, v, P.eps, nxt, lvl + 1, kern);
            }
            if (++j >= gend) break;
        }
    }
}

// ------------------------------------------------------------------------------------ kernels
__global__ void __launch_bounds__(kBlock) k_expand(KArgs A)
{
    Ctrl *ctrl = A.ctrl;
    const unsigned int cur = ctrl->cur, nxt = cur ^ 1u;
    const unsigned long long n_items = min(ctrl->n_items[cur], A.cap_items);
    const uint32_t *items = cur ? A.items1 : A.items0;
    const OutDesc od = ctrl->od;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long idx = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; idx < n_items; idx += stride) {
        const uint32_t item = items[idx];
        const int lane = (int)(item >> A.ubits);
        const int32_t u = (int32_t)(item & A.umask);
        const int lvl = A.level[lane];
        if (lvl < 0 || lvl >= kMaxLevels) {
            atomicOr(&ctrl->error, 16u);
            continue;
        }
        const LaneParam P = A.lanes[lane];
        float *Rc = A.R + (size_t)(lvl & 1) * A.par_stride + (size_t)lane * A.g.n;
        float *Rn = A.R + (size_t)((lvl + 1) & 1) * A.par_stride + (size_t)lane * A.g.n;
        const float r = Rc[u];
        Rc[u] = 0.f;
        const float2 cf = A.coef[lane * kMaxLevels + lvl];
        // reserve: q^(i)(u) = (w_i / Y_i) r^(i)(u), added to pi (scale folded into cf.x)
        atomicAdd(od.out + (int64_t)u * od.su + (int64_t)P.out_row * od.sr, cf.x * r);
        if (lvl >= P.L) continue;
        const int32_t d = A.g.deg[u];
        if (d == 0) continue;
        const float c = apply_deg(cf.y * r, d, P.b_mode, P.b);  // (Y_{i+1}/Y_i) r / d_u^b
        if (!(c > 0.f)) continue;
        const int32_t *row = A.g.colidx + A.g.rowptr[u];
        const int k = det_prefix(c, P, row, d, A.g.deg);
        unsigned long long drawn = 0, accepted = 0;
        if (k > 0) {
            if (k <= kInlineDet) {
                for (int j = 0; j < k; ++j) {
                    const int32_t v = row[j];
                    const float inc = (P.a_mode == 0) ? c : apply_deg(c, A.g.deg[v], P.a_mode, P.a);
                    push_to(A, Rn, lane, v, inc, nxt, lvl + 1, 0);
                }
                if (A.collect) atomicAdd(&A.stats[lane].by_kernel[0][0], (unsigned long long)k);
            } else {
                const int nrec = (k + kChunk - 1) / kChunk;
                const unsigned long long base = atomicAdd(&ctrl->n_det, (unsigned long long)nrec);
                for (int t = 0; t < nrec; ++t) {
                    if (base + t < A.cap_det) A.det_rec[base + t] = make_uint2((uint32_t)idx, (uint32_t)t);
                    else atomicOr(&ctrl->error, 2u);
                }
            }
        }
        const int tail = d - k;
        int seglen = 0;
        if (tail > 0) {
            const float ce = (float)((double)c / P.eps_d);
            const float p0 = fminf(1.f, (P.a_mode == 0) ? ce : apply_deg(ce, A.g.deg[row[k]], P.a_mode, P.a));
            const float expect = p0 * (float)tail;  // upper bound on the trials reached
            if (expect <= kLightSamples) {
                sample_range(A, P, Rn, lane, u, lvl, 0u, row, k, d, c, nxt, drawn, accepted, 0);
            } else {
                int nseg = (int)fminf(ceilf(expect / kLightSamples), (float)((tail + kMinSeg - 1) / kMinSeg));
                nseg = max(nseg, 1);
                seglen = (tail + nseg - 1) / nseg;
                nseg = (tail + seglen - 1) / seglen;
                const unsigned long long base = atomicAdd(&ctrl->n_smp, (unsigned long long)nseg);
                for (int t = 0; t < nseg; ++t) {
                    if (base + t < A.cap_smp) A.smp_rec[base + t] = make_uint2((uint32_t)idx, (uint32_t)t);
                    else atomicOr(&ctrl->error, 4u);
                }
            }
        }
        if (k > kInlineDet || seglen > 0) {
            A.c_item[idx] = c;
            A.k_item[idx] = make_int2(k, seglen);
        }
        if (A.collect && (drawn | accepted)) {
            atomicAdd(&A.stats[lane].by_kernel[0][1], drawn);
            atomicAdd(&A.stats[lane].by_kernel[0][2], accepted);
        }
    }
}

__global__ void __launch_bounds__(kBlock) k_push(KArgs A)
{
    Ctrl *ctrl = A.ctrl;
    const unsigned int cur = ctrl->cur, nxt = cur ^ 1u;
    const unsigned long long n_det = min(ctrl->n_det, A.cap_det);
    const uint32_t *items = cur ? A.items1 : A.items0;
    const int lane_id = threadIdx.x & 31;
    const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    for (unsigned long long rec = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5; rec < n_det; rec += nwarps) {
        const uint2 R = A.det_rec[rec];
        const uint32_t item = items[R.x];
        const int lane = (int)(item >> A.ubits);
        const int32_t u = (int32_t)(item & A.umask);
        const int lvl = A.level[lane];
        const LaneParam P = A.lanes[lane];
        float *Rn = A.R + (size_t)((lvl + 1) & 1) * A.par_stride + (size_t)lane * A.g.n;
        const float c = A.c_item[R.x];
        const int k = A.k_item[R.x].x;
        const int j0 = (int)R.y * kChunk, j1 = min(k, j0 + kChunk);
        const int32_t *row = A.g.colidx + A.g.rowptr[u];
        for (int j = j0 + lane_id; j < j1; j += 32) {
            const int32_t v = row[j];
            const float inc = (P.a_mode == 0) ? c : apply_deg(c, A.g.deg[v], P.a_mode, P.a);
            push_to(A, Rn, lane, v, inc, nxt, lvl + 1, 1);
        }
        if (A.collect && lane_id == 0) atomicAdd(&A.stats[lane].by_kernel[1][0], (unsigned long long)(j1 - j0));
    }
}

__global__ void __launch_bounds__(kBlock) k_sample(KArgs A)
{
    Ctrl *ctrl = A.ctrl;
    const unsigned int cur = ctrl->cur, nxt = cur ^ 1u;
    const unsigned long long n_smp = min(ctrl->n_smp, A.cap_smp);
    const uint32_t *items = cur ? A.items1 : A.items0;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long rec = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; rec < n_smp; rec += stride) {
        const uint2 R = A.smp_rec[rec];
        const uint32_t item = items[R.x];
        const int lane = (int)(item >> A.ubits);
        const int32_t u = (int32_t)(item & A.umask);
        const int lvl = A.level[lane];
        const LaneParam P = A.lanes[lane];
        float *Rn = A.R + (size_t)((lvl + 1) & 1) * A.par_stride + (size_t)lane * A.g.n;
        const float c = A.c_item[R.x];
        const int2 ks = A.k_item[R.x];
        const int d = A.g.deg[u];
        const int j0 = ks.x + (int)R.y * ks.y, j1 = min(d, j0 + ks.y);
        const int32_t *row = A.g.colidx + A.g.rowptr[u];
        unsigned long long drawn = 0, accepted = 0;
        sample_range(A, P, Rn, lane, u, lvl, R.y, row, j0, j1, c, nxt, drawn, accepted, 2);
        if (A.collect && (drawn | accepted)) {
            atomicAdd(&A.stats[lane].by_kernel[2][1], drawn);
            atomicAdd(&A.stats[lane].by_kernel[2][2], accepted);
        }
    }
}

__global__ void k_level_end(KArgs A)
{
    Ctrl *ctrl = A.ctrl;
    const unsigned int cur = ctrl->cur;
    for (int l = threadIdx.x; l < A.G; l += blockDim.x) {
        const int lvl = A.level[l];
        if (lvl >= 0) A.level[l] = (lvl < A.lanes[l].L) ? lvl + 1 : -1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ctrl->n_items[cur] = 0;
        ctrl->cur = cur ^ 1u;
        ctrl->n_det = 0;
        ctrl->n_smp = 0;
    }
}

// ---- coefficients (Def. 3.1), FP64 on the device -------------------------------------------
struct CoefSpec {
    int32_t kind, L;
    double param;
    int32_t w_off;     // FINITE: offset of w_0..w_L in the weight array
    double scale;      // sign * ||x_part||_1 (the Y_0 factor is applied here)
};

__global__ void k_coef(const CoefSpec *spec, const double *wts, float2 *coef, int nlanes)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nlanes) return;
    const CoefSpec S = spec[l];
    const int L = S.L;
    double w[kMaxLevels], Y[kMaxLevels + 1];
    switch (S.kind) {
    case AGP_W_FINITE: {
        for (int i = 0; i <= L; ++i) w[i] = wts[S.w_off + i];
        double acc = 0.0;  // smallest terms last in the list are added first
        Y[L + 1] = 0.0;
        for (int i = L; i >= 0; --i) { acc += w[i]; Y[i] = acc; }
        break;
    }
    case AGP_W_PPR: {
        const double al = S.param;
        for (int i = 0; i <= L + 1; ++i) {
            const double t = pow(1.0 - al, (double)i);
            if (i <= L) w[i] = al * t;
            Y[i] = t;
        }
        break;
    }
    case AGP_W_HKPR: {
        const double t = S.param;
        int K = L + 2;
        while (K < 100000 && (K < t + 1.0 || -t + K * log(t) - lgamma(K + 1.0) > -690.0)) ++K;
        double acc = 0.0;
        for (int k = K; k >= 0; --k) {
            const double wk = exp(-t + k * log(t) - lgamma(k + 1.0));
            acc += wk;
            if (k <= L + 1) Y[k] = acc;
            if (k <= L) w[k] = wk;
        }
        break;
    }
    case AGP_W_KATZ: {
        const double be = S.param;
        for (int i = 0; i <= L + 1; ++i) {
            const double t = pow(be, (double)i);
            if (i <= L) w[i] = t;
            Y[i] = t / (1.0 - be);
        }
        break;
    }
    default: {  // TRANSITION
        for (int i = 0; i <= L; ++i) { w[i] = (i == L) ? 1.0 : 0.0; Y[i] = 1.0; }
        Y[L + 1] = 0.0;
        break;
    }
    }
    const double Y0 = Y[0];
    for (int i = 0; i < kMaxLevels; ++i) {
        float keep = 0.f, push = 0.f;
        if (i <= L && Y[i] > 0.0) {
            keep = (float)(S.scale * Y0 * (w[i] / Y[i]));
            push = (i < L) ? (float)(Y[i + 1] / Y[i]) : 0.f;
        }
        coef[l * kMaxLevels + i] = make_float2(keep, push);
    }
}

// ---- seeds -------------------------------------------------------------------------------------
__device__ __forceinline__ int query_of(const int64_t *off, int Q, int64_t t)
{
    int lo = 0, hi = Q;  // last q with off[q] <= t
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void k_norms_sparse(const int64_t *off, const int32_t *idx, const float *val, int Q,
                               int64_t n, double *norms, unsigned int *bad)
{
    const int64_t total = off[Q];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int q = query_of(off, Q, t);
        const float x = val ? val[t] : 1.f;
        const int32_t u = idx[t];
        if (u < 0 || u >= n || !isfinite(x)) { atomicOr(bad, 1u); continue; }
        if (x == 0.f) continue;
        atomicAdd(&norms[2 * q + (x < 0.f ? 1 : 0)], (double)fabsf(x));
    }
}

__global__ void k_seed_sparse(KArgs A, const int64_t *off, const int32_t *idx, const float *val, int Q,
                              const int32_t *lane_of, const double *norms)
{
    const unsigned int cur = A.ctrl->cur;
    const int64_t total = off[Q];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int q = query_of(off, Q, t);
        const float x = val ? val[t] : 1.f;
        if (x == 0.f) continue;
        const int part = x < 0.f ? 1 : 0;
        const int lane = lane_of[2 * q + part];
        if (lane < 0) continue;
        const int32_t u = idx[t];
        if (u < 0 || u >= A.g.n) continue;
        float *R0 = A.R + (size_t)lane * A.g.n;  // level 0 lives in parity 0
        const float r0 = (float)((double)fabsf(x) / norms[2 * q + part]);
        push_to(A, R0, lane, u, r0, cur, 0, -1);
    }
}

__global__ void k_colnorms_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ldx, int64_t rows_per_block,
                                double *norms)
{
    const int64_t r0 = blockIdx.x * rows_per_block, r1 = min(n, r0 + rows_per_block);
    for (int64_t c = threadIdx.x; c < d; c += blockDim.x) {
        double sp = 0.0, sn = 0.0;
        for (int64_t u = r0; u < r1; ++u) {
            const float x = __uint_as_float((uint32_t)X[u * ldx + c] << 16);
            if (x > 0.f) sp += x;
            else if (x < 0.f) sn -= x;
        }
        if (sp != 0.0) atomicAdd(&norms[2 * c], sp);
        if (sn != 0.0) atomicAdd(&norms[2 * c + 1], sn);
    }
}

// lane l of the wave takes column col_of[l], sign part part_of[l]
__global__ void k_seed_dense_bf16(KArgs A, const uint16_t *X, int64_t ldx, const int32_t *col_of,
                                  const int32_t *part_of, const double *norms, int nl)
{
    const unsigned int cur = A.ctrl->cur;
    const int64_t total = A.g.n * nl;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(t % nl);
        const int64_t u = t / nl;
        const int col = col_of[l];
        const float x = __uint_as_float((uint32_t)X[u * ldx + col] << 16);
        const int part = part_of[l];
        if (!((part == 0 && x > 0.f) || (part == 1 && x < 0.f))) continue;
        float *R0 = A.R + (size_t)l * A.g.n;
        const float r0 = (float)((double)fabsf(x) / norms[2 * col + part]);
        push_to(A, R0, l, (int32_t)u, r0, cur, 0, -1);
    }
}

__global__ void k_threshold(DevGraph g, double a, int a_mode, double eps, int64_t count, const int32_t *nodes,
                            const float *c, int32_t *k_out)
{
    LaneParam P;
    P.eps_d = eps;
    P.eps = (float)eps;
    P.a = (float)a;
    P.b = 0.f;
    P.a_d = a;
    P.a_mode = a_mode;
    P.b_mode = 0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = nodes[t];
        int k = 0;
        if (u >= 0 && u < g.n) {
            const int d = g.deg[u];
            if (d > 0 && c[t] > 0.f) k = det_prefix(c[t], P, g.colidx + g.rowptr[u], d, g.deg);
        }
        k_out[t] = k;
    }
}

// ------------------------------------------------------------------------------------ host side
namespace {

int exponent_mode(double p)
{
    if (p == 0.0) return 0;
    if (p == 1.0) return 1;
    if (p == 0.5) return 2;
    return 3;
}

int validate_params(const agp_params_t &p)
{
    if (!(p.a >= 0.0 && p.a <= 1.0 && p.b >= 0.0 && p.b <= 1.0)) return fail(AGP_EINVAL, "params: a and b must be in [0, 1]");
    if (p.L < 0 || p.L >= kMaxLevels) return fail(AGP_EINVAL, "params: L must be in [0, 63]");
    if (!(p.eps >= 0.0) || std::isinf(p.eps)) return fail(AGP_EINVAL, "params: eps must be finite and >= 0");
    if (p.eps != 0.0 && p.eps < 1e-30) return fail(AGP_EINVAL, "params: eps must be 0 or >= 1e-30");
    switch (p.kind) {
    case AGP_W_FINITE: {
        if (!p.w) return fail(AGP_EINVAL, "params: FINITE weights need w");
        double s = 0.0;
        for (int i = 0; i <= p.L; ++i) {
            if (!(p.w[i] >= 0.0) || std::isinf(p.w[i])) return fail(AGP_EINVAL, "params: weights must be finite and >= 0");
            s += p.w[i];
        }
        if (!(s > 0.0)) return fail(AGP_EINVAL, "params: weights sum to 0");
        return AGP_OK;
    }
    case AGP_W_PPR:
        if (!(p.param > 0.0 && p.param <= 1.0)) return fail(AGP_EINVAL, "params: PPR alpha must be in (0, 1]");
        return AGP_OK;
    case AGP_W_HKPR:
        if (!(p.param > 0.0 && p.param < 1000.0)) return fail(AGP_EINVAL, "params: HKPR t must be in (0, 1000)");
        return AGP_OK;
    case AGP_W_KATZ:
        if (!(p.param > 0.0 && p.param < 1.0)) return fail(AGP_EINVAL, "params: Katz beta must be in (0, 1)");
        return AGP_OK;
    case AGP_W_TRANSITION:
        return AGP_OK;
    default:
        return fail(AGP_EINVAL, "params: unknown weight kind");
    }
}

uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Lane key: a function of (seed, stream, part) only, so that a query's samples do not depend on
// the batch it runs in.
void lane_key(uint64_t seed, uint64_t stream, int part, uint32_t &k0, uint32_t &k1)
{
    const uint64_t k = splitmix64(seed ^ splitmix64(2 * stream + (uint64_t)part + 1));
    k0 = (uint32_t)k;
    k1 = (uint32_t)(k >> 32);
}

template <class T> int dev_alloc(T **p, size_t count, size_t &acc)
{
    const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(AGP_ENOMEM, "cudaMalloc(" + std::to_string(bytes) + ") for query work buffers: " + cudaGetErrorString(e));
    }
    acc += bytes;
    return AGP_OK;
}

size_t bytes_per_lane(const agp_graph_s *g)
{
    const size_t n = (size_t)g->n;
    const double avg = g->n ? (double)g->nnz / (double)g->n : 0.0;
    // R (2 x 4) + items (2 x 4) + c (4) + k (8) + chunk and segment records (8 + 8, with the
    // extra records of long rows) per (lane, node)
    return n * (8 + 8 + 4 + 8) + (size_t)(n * 8 * (1.0 + avg / kChunk)) + (size_t)(n * 8 * (1.0 + avg / kMinSeg)) + 4096;
}

int lane_capacity(const agp_graph_s *g)
{
    const int by_bits = (g->ubits >= 31) ? 1 : (int)std::min<int64_t>(4096, 1ll << (32 - g->ubits));
    const int64_t by_items = g->n ? (int64_t)(4294967295ull / (uint64_t)g->n) : 4096;
    return (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)by_bits, by_items, 4096}));
}

}  // namespace

void free_workspace(Workspace *ws)
{
    if (!ws) return;
    if (ws->graph) cudaGraphExecDestroy(ws->graph);
    if (ws->ev_ready)
        for (int l = 0; l < kMaxLevels; ++l)
            for (int k = 0; k < 4; ++k)
                for (int e = 0; e < 2; ++e) cudaEventDestroy(ws->ev[l][k][e]);
    cudaFree(ws->R);
    cudaFree(ws->items[0]);
    cudaFree(ws->items[1]);
    cudaFree(ws->c_item);
    cudaFree(ws->k_item);
    cudaFree(ws->det_rec);
    cudaFree(ws->smp_rec);
    cudaFree(ws->lanes);
    cudaFree(ws->coef);
    cudaFree(ws->level);
    cudaFree(ws->stats);
    cudaFree(ws->ctrl);
    cudaFree(ws->stage);
    cudaFree(ws->out_stage);
    cudaFreeHost(ws->h_ctrl);
    cudaFreeHost(ws->h_lanes);
    delete ws;
}

namespace {

int ensure_workspace(agp_graph_s *g, int lanes_wanted, Workspace **out)
{
    const int cap = lane_capacity(g);
    int G = std::max(1, std::min(lanes_wanted, cap));
    int64_t budget = g->mem_budget;
    if (budget <= 0) {
        size_t fr = 0, tot = 0;
        AGP_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
        const size_t have = g->ws ? g->ws->bytes : 0;
        budget = (int64_t)((double)(fr + have) * 0.6);
    }
    const int by_budget = (int)std::min<int64_t>(cap, std::max<int64_t>(0, budget / (int64_t)bytes_per_lane(g)));
    if (by_budget < 1) return fail(AGP_EBUDGET, "memory budget too small for one propagation lane");
    G = std::min(G, by_budget);
    if (g->ws && g->ws->G >= G) {
        *out = g->ws;
        return AGP_OK;
    }
    if (g->ws) {
        AGP_CUDA_TRY(cudaDeviceSynchronize());
        free_workspace(g->ws);
        g->ws = nullptr;
    }
    Workspace *ws = new Workspace();
    ws->device = g->device;
    ws->G = G;
    ws->n = g->n;
    const unsigned long long n = (unsigned long long)std::max<int64_t>(g->n, 1);
    ws->cap_items = (unsigned long long)G * n;
    ws->cap_det = ws->cap_items + (unsigned long long)G * (unsigned long long)g->nnz / kChunk + 1;
    ws->cap_smp = ws->cap_items + (unsigned long long)G * (unsigned long long)g->nnz / kMinSeg + 1;
    size_t acc = 0;
    int rc = AGP_OK;
    auto A = [&](int r) { if (rc == AGP_OK) rc = r; };
    A(dev_alloc(&ws->R, (size_t)2 * G * n, acc));
    A(dev_alloc(&ws->items[0], ws->cap_items, acc));
    A(dev_alloc(&ws->items[1], ws->cap_items, acc));
    A(dev_alloc(&ws->c_item, ws->cap_items, acc));
    A(dev_alloc(&ws->k_item, ws->cap_items, acc));
    A(dev_alloc(&ws->det_rec, ws->cap_det, acc));
    A(dev_alloc(&ws->smp_rec, ws->cap_smp, acc));
    A(dev_alloc(&ws->lanes, (size_t)G, acc));
    A(dev_alloc(&ws->coef, (size_t)G * kMaxLevels, acc));
    A(dev_alloc(&ws->level, (size_t)G, acc));
    A(dev_alloc(&ws->stats, (size_t)G, acc));
    A(dev_alloc(&ws->ctrl, 1, acc));
    if (rc == AGP_OK && cudaMallocHost((void **)&ws->h_ctrl, sizeof(Ctrl)) != cudaSuccess) rc = fail(AGP_ENOMEM, "cudaMallocHost");
    if (rc == AGP_OK && cudaMallocHost((void **)&ws->h_lanes, sizeof(LaneParam) * G) != cudaSuccess) rc = fail(AGP_ENOMEM, "cudaMallocHost");
    if (rc == AGP_OK) {
        cudaError_t e = cudaMemset(ws->R, 0, sizeof(float) * (size_t)2 * G * n);
        if (e == cudaSuccess) e = cudaMemset(ws->level, 0xff, sizeof(int32_t) * G);
        if (e == cudaSuccess) e = cudaMemset(ws->ctrl, 0, sizeof(Ctrl));
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) rc = fail(AGP_ECUDA, std::string("workspace init: ") + cudaGetErrorString(e));
    }
    if (rc != AGP_OK) {
        free_workspace(ws);
        return rc;
    }
    ws->bytes = acc;
    g->ws = ws;
    *out = ws;
    return AGP_OK;
}

int grow(void **p, size_t *have, size_t need)
{
    if (*have >= need) return AGP_OK;
    cudaFree(*p);
    *p = nullptr;
    *have = 0;
    need = std::max<size_t>(need, 4096);
    cudaError_t e = cudaMalloc(p, need);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(AGP_ENOMEM, std::string("staging buffer: ") + cudaGetErrorString(e));
    }
    *have = need;
    return AGP_OK;
}

KArgs make_args(agp_graph_s *g, Workspace *ws, int collect)
{
    KArgs A;
    A.g = g->dev();
    A.ubits = g->ubits;
    A.umask = (g->ubits >= 32) ? 0xffffffffu : ((1u << g->ubits) - 1u);
    A.R = ws->R;
    A.par_stride = (size_t)ws->G * (size_t)std::max<int64_t>(g->n, 1);
    A.items0 = ws->items[0];
    A.items1 = ws->items[1];
    A.c_item = ws->c_item;
    A.k_item = ws->k_item;
    A.det_rec = ws->det_rec;
    A.smp_rec = ws->smp_rec;
    A.cap_items = ws->cap_items;
    A.cap_det = ws->cap_det;
    A.cap_smp = ws->cap_smp;
    A.lanes = ws->lanes;
    A.coef = ws->coef;
    A.level = ws->level;
    A.stats = ws->stats;
    A.collect = collect;
    A.G = ws->G;
    A.ctrl = ws->ctrl;
    return A;
}

int ensure_events(Workspace *ws)
{
    if (ws->ev_ready) return AGP_OK;
    for (int l = 0; l < kMaxLevels; ++l)
        for (int k = 0; k < 4; ++k)
            for (int e = 0; e < 2; ++e) AGP_CUDA_TRY(cudaEventCreate(&ws->ev[l][k][e]));
    ws->ev_ready = true;
    return AGP_OK;
}

// One level: expand, push, sample, level end. With `ev` (profiling) every kernel is bracketed by
// event records on the same stream.
void launch_level(const KArgs &A, cudaStream_t s, int expand_blocks, int push_blocks, int sample_blocks,
                  cudaEvent_t (*ev)[2] = nullptr)
{
    if (ev) cudaEventRecord(ev[0][0], s);
    k_expand<<<expand_blocks, kBlock, 0, s>>>(A);
    if (ev) { cudaEventRecord(ev[0][1], s); cudaEventRecord(ev[1][0], s); }
    k_push<<<push_blocks, kBlock, 0, s>>>(A);
    if (ev) { cudaEventRecord(ev[1][1], s); cudaEventRecord(ev[2][0], s); }
    k_sample<<<sample_blocks, kBlock, 0, s>>>(A);
    if (ev) { cudaEventRecord(ev[2][1], s); cudaEventRecord(ev[3][0], s); }
    k_level_end<<<1, kBlock, 0, s>>>(A);
    if (ev) cudaEventRecord(ev[3][1], s);
}

int blocks_for(unsigned long long work, int per_block)
{
    const unsigned long long b = (work + per_block - 1) / per_block;
    return (int)std::max<unsigned long long>(1, std::min<unsigned long long>(b, (unsigned long long)kGridStrideBlocks * 4));
}

// Accumulate the profiled kernel times of levels [0, levels) (the stream has been synchronised).
void read_profile(agp_graph_s *g, Workspace *ws, int levels, const bool *ran)
{
    for (int l = 0; l < levels; ++l)
        for (int k = 0; k < 4; ++k) {
            if (ran && !ran[l * 4 + k]) continue;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ws->ev[l][k][0], ws->ev[l][k][1]) == cudaSuccess) {
                g->prof_ms[k] += ms;
                g->prof_launches[k] += 1;
            } else {
                cudaGetLastError();
            }
        }
}

// Run the levels of the current wave (lanes already seeded, level 0 frontier in items[cur]).
int run_levels(agp_graph_s *g, Workspace *ws, const KArgs &A, int max_L, bool plain, bool profile, cudaStream_t s)
{
    if (profile) AGP_TRY(ensure_events(ws));
    if (plain) {
        bool ran[kMaxLevels * 4] = {};
        int levels = 0;
        for (int lvl = 0; lvl <= max_L; ++lvl) {
            AGP_CUDA_TRY(cudaMemcpyAsync(ws->h_ctrl, ws->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
            AGP_CUDA_TRY(cudaStreamSynchronize(s));
            const unsigned long long items = std::min(ws->h_ctrl->n_items[ws->h_ctrl->cur], ws->cap_items);
            if (items == 0) break;
            auto rec = [&](int k, int e) { if (profile) cudaEventRecord(ws->ev[lvl][k][e], s); };
            rec(0, 0);
            k_expand<<<blocks_for(items, kBlock), kBlock, 0, s>>>(A);
            rec(0, 1);
            ran[lvl * 4 + 0] = true;
            AGP_CUDA_TRY(cudaMemcpyAsync(ws->h_ctrl, ws->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
            AGP_CUDA_TRY(cudaStreamSynchronize(s));
            const unsigned long long nd = std::min(ws->h_ctrl->n_det, ws->cap_det), ns = std::min(ws->h_ctrl->n_smp, ws->cap_smp);
            g->kernel_launches += 2 + (nd ? 1 : 0) + (ns ? 1 : 0);
            if (nd) { rec(1, 0); k_push<<<blocks_for(nd, kBlock / 32), kBlock, 0, s>>>(A); rec(1, 1); ran[lvl * 4 + 1] = true; }
            if (ns) { rec(2, 0); k_sample<<<blocks_for(ns, kBlock), kBlock, 0, s>>>(A); rec(2, 1); ran[lvl * 4 + 2] = true; }
            rec(3, 0);
            k_level_end<<<1, kBlock, 0, s>>>(A);
            rec(3, 1);
            ran[lvl * 4 + 3] = true;
            levels = lvl + 1;
            AGP_CUDA_TRY(cudaGetLastError());
        }
        if (profile) {
            AGP_CUDA_TRY(cudaStreamSynchronize(s));
            read_profile(g, ws, levels, ran);
        }
        return AGP_OK;
    }
    if (!ws->graph || ws->graph_levels != max_L || ws->graph_collect != A.collect || ws->graph_profile != (int)profile) {
        if (ws->graph) {
            cudaGraphExecDestroy(ws->graph);
            ws->graph = nullptr;
        }
        cudaStream_t cs;
        AGP_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            for (int lvl = 0; lvl <= max_L; ++lvl)
                launch_level(A, cs, kGridStrideBlocks, kGridStrideBlocks, kGridStrideBlocks, profile ? ws->ev[lvl] : nullptr);
            e = cudaStreamEndCapture(cs, &graph);
        }
        if (e == cudaSuccess) {
            e = cudaGraphInstantiate(&ws->graph, graph, 0);
            cudaGraphDestroy(graph);
        }
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) {
            ws->graph = nullptr;
            return fail(AGP_ECUDA, std::string("capturing the level loop: ") + cudaGetErrorString(e));
        }
        ws->graph_levels = max_L;
        ws->graph_collect = A.collect;
        ws->graph_profile = (int)profile;
    }
    AGP_CUDA_TRY(cudaGraphLaunch(ws->graph, s));
    g->kernel_launches += 4 * (max_L + 1);
    if (profile) {
        AGP_CUDA_TRY(cudaStreamSynchronize(s));
        read_profile(g, ws, max_L + 1, nullptr);
    }
    return AGP_OK;
}

int check_ctrl(Workspace *ws, cudaStream_t s)
{
    AGP_CUDA_TRY(cudaMemcpyAsync(ws->h_ctrl, ws->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    AGP_CUDA_TRY(cudaStreamSynchronize(s));
    if (ws->h_ctrl->error & 8u) return fail(AGP_EINVAL, "signal index outside [0, n) or non-finite value");
    if (ws->h_ctrl->error) return fail(AGP_EINTERNAL, "device work list overflow (flags " + std::to_string(ws->h_ctrl->error) + ")");
    return AGP_OK;
}

struct LaneSpec {
    int query;       // output row
    int part;        // 0: x+, 1: x-
    double norm;
    int params;      // index into params
};

int prepare_wave(agp_graph_s *g, Workspace *ws, const std::vector<LaneSpec> &lanes, size_t first, int count,
                 const agp_params_t *params, uint64_t stream_base_is_query, cudaStream_t s,
                 std::vector<CoefSpec> &cs, std::vector<double> &wts, int *max_L)
{
    cs.assign(count, CoefSpec{});
    wts.clear();
    *max_L = 0;
    for (int l = 0; l < count; ++l) {
        const LaneSpec &ls = lanes[first + l];
        const agp_params_t &p = params[ls.params];
        LaneParam &P = ws->h_lanes[l];
        P.eps_d = p.eps;
        P.eps = (float)p.eps;
        P.a = (float)p.a;
        P.b = (float)p.b;
        P.a_d = p.a;
        P.a_mode = exponent_mode(p.a);
        P.b_mode = exponent_mode(p.b);
        P.L = p.L;
        P.out_row = ls.query;
        lane_key(p.seed, stream_base_is_query ? (uint64_t)ls.query : 0ull, ls.part, P.key0, P.key1);
        CoefSpec &c = cs[l];
        c.kind = p.kind;
        c.L = p.L;
        c.param = p.param;
        c.scale = (ls.part ? -1.0 : 1.0) * ls.norm;
        c.w_off = 0;
        if (p.kind == AGP_W_FINITE) {
            c.w_off = (int32_t)wts.size();
            for (int i = 0; i <= p.L; ++i) wts.push_back(p.w[i]);
        }
        *max_L = std::max(*max_L, p.L);
    }
    // device copies: lane params, coefficient specs, weights (staging area)
    const size_t cs_bytes = sizeof(CoefSpec) * count, w_bytes = sizeof(double) * std::max<size_t>(wts.size(), 1);
    AGP_TRY(grow(&ws->stage, &ws->stage_bytes, cs_bytes + w_bytes + 256));
    char *st = (char *)ws->stage;
    CoefSpec *d_cs = (CoefSpec *)st;
    double *d_w = (double *)(st + ((cs_bytes + 15) / 16) * 16);
    AGP_CUDA_TRY(cudaMemcpyAsync(ws->lanes, ws->h_lanes, sizeof(LaneParam) * count, cudaMemcpyHostToDevice, s));
    AGP_CUDA_TRY(cudaMemcpyAsync(d_cs, cs.data(), cs_bytes, cudaMemcpyHostToDevice, s));
    if (!wts.empty()) AGP_CUDA_TRY(cudaMemcpyAsync(d_w, wts.data(), sizeof(double) * wts.size(), cudaMemcpyHostToDevice, s));
    k_coef<<<(count + 127) / 128, 128, 0, s>>>(d_cs, d_w, ws->coef, count);
    // all wave lanes start at level 0, the other lanes idle
    std::vector<int32_t> lv(ws->G, -1);
    for (int l = 0; l < count; ++l) lv[l] = 0;
    AGP_CUDA_TRY(cudaMemcpyAsync(ws->level, lv.data(), sizeof(int32_t) * ws->G, cudaMemcpyHostToDevice, s));
    AGP_CUDA_TRY(cudaMemsetAsync(ws->stats, 0, sizeof(LaneStats) * ws->G, s));
    // the copies above read host memory that lives until the next synchronisation point
    AGP_CUDA_TRY(cudaStreamSynchronize(s));
    return AGP_OK;
}

int set_ctrl(Workspace *ws, float *out, int64_t su, int64_t sr, cudaStream_t s)
{
    Ctrl *h = ws->h_ctrl;
    std::memset(h, 0, sizeof(Ctrl));
    h->od.out = out;
    h->od.su = su;
    h->od.sr = sr;
    AGP_CUDA_TRY(cudaMemcpyAsync(ws->ctrl, h, sizeof(Ctrl), cudaMemcpyHostToDevice, s));
    AGP_CUDA_TRY(cudaStreamSynchronize(s));
    return AGP_OK;
}

int collect_stats(Workspace *ws, const std::vector<LaneSpec> &lanes, size_t first, int count, agp_stats_t *stats,
                  cudaStream_t s)
{
    std::vector<LaneStats> h(count);
    AGP_CUDA_TRY(cudaMemcpyAsync(h.data(), ws->stats, sizeof(LaneStats) * count, cudaMemcpyDeviceToHost, s));
    AGP_CUDA_TRY(cudaStreamSynchronize(s));
    for (int l = 0; l < count; ++l) {
        agp_stats_t &S = stats[lanes[first + l].query];
        for (int i = 0; i < kMaxLevels; ++i) S.frontier[i] += (int64_t)h[l].frontier[i];
        for (int k = 0; k < 3; ++k) {
            for (int c = 0; c < 4; ++c) S.by_kernel[k][c] += (int64_t)h[l].by_kernel[k][c];
            S.det_edge_ops += (int64_t)h[l].by_kernel[k][0];
            S.samples_drawn += (int64_t)h[l].by_kernel[k][1];
            S.samples_accepted += (int64_t)h[l].by_kernel[k][2];
        }
    }
    return AGP_OK;
}

}  // namespace

// ------------------------------------------------------------------------------------ queries
int query_batch(agp_graph_s *g, const agp_params_t *params, int32_t n_params, int32_t Q,
                const int64_t *x_off, const int32_t *x_idx, const float *x_val, float *pi_out,
                int64_t ld_out, uint32_t flags, agp_stats_t *stats, cudaStream_t s)
{
    if (!g) return fail(AGP_EINVAL, "graph is NULL");
    if (Q < 0) return fail(AGP_EINVAL, "Q < 0");
    if (Q == 0) return AGP_OK;
    if (!params || !(n_params == 1 || n_params == Q)) return fail(AGP_EINVAL, "n_params must be 1 or Q");
    if (!x_off || !pi_out) return fail(AGP_EINVAL, "x_off / pi_out NULL");
    if (ld_out < g->n) return fail(AGP_EINVAL, "ld_out < n");
    if (flags & ~(AGP_INPUT_ON_DEVICE | AGP_OUTPUT_ON_DEVICE | AGP_PLAIN | AGP_COLLECT_STATS | AGP_PROFILE))
        return fail(AGP_EINVAL, "unknown flag");
    if ((flags & AGP_COLLECT_STATS) && !stats) return fail(AGP_EINVAL, "AGP_COLLECT_STATS needs stats");
    for (int i = 0; i < n_params; ++i) AGP_TRY(validate_params(params[i]));
    AGP_CUDA_TRY(cudaSetDevice(g->device));
    const bool plain = flags & AGP_PLAIN;
    const bool profile = flags & AGP_PROFILE;
    const int collect = (flags & AGP_COLLECT_STATS) ? 1 : 0;
    const int64_t n = g->n;

    // --- inputs on the device
    int64_t total = 0;
    if (flags & AGP_INPUT_ON_DEVICE) {
        AGP_CUDA_TRY(cudaMemcpyAsync(&total, x_off + Q, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        AGP_CUDA_TRY(cudaStreamSynchronize(s));
    } else {
        total = x_off[Q];
        if (x_off[0] != 0) return fail(AGP_EINVAL, "x_off[0] must be 0");
        for (int q = 0; q < Q; ++q)
            if (x_off[q + 1] < x_off[q]) return fail(AGP_EINVAL, "x_off must be non-decreasing");
    }
    if (total < 0) return fail(AGP_EINVAL, "negative signal size");
    if (total > 0 && !x_idx) return fail(AGP_EINVAL, "x_idx NULL");

    const size_t off_b = sizeof(int64_t) * (Q + 1), idx_b = sizeof(int32_t) * std::max<int64_t>(total, 1),
                 val_b = x_val ? sizeof(float) * std::max<int64_t>(total, 1) : 0, norm_b = sizeof(double) * 2 * Q,
                 map_b = sizeof(int32_t) * 2 * Q;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t need = al(off_b) + al(idx_b) + al(val_b) + al(norm_b) + al(map_b) + al(sizeof(unsigned int));
    AGP_TRY(grow(&g->in_stage, &g->in_bytes, need));
    char *p = (char *)g->in_stage;
    int64_t *d_off = (int64_t *)p; p += al(off_b);
    int32_t *d_idx = (int32_t *)p; p += al(idx_b);
    float *d_val = x_val ? (float *)p : nullptr; p += al(val_b);
    double *d_norm = (double *)p; p += al(norm_b);
    int32_t *d_map = (int32_t *)p; p += al(map_b);
    unsigned int *d_bad = (unsigned int *)p;
    const int64_t *off_src = x_off;
    const int32_t *idx_src = x_idx;
    const float *val_src = x_val;
    if (flags & AGP_INPUT_ON_DEVICE) {
        off_src = x_off; idx_src = x_idx; val_src = x_val;
    } else {
        AGP_CUDA_TRY(cudaMemcpyAsync(d_off, x_off, off_b, cudaMemcpyHostToDevice, s));
        if (total) AGP_CUDA_TRY(cudaMemcpyAsync(d_idx, x_idx, sizeof(int32_t) * total, cudaMemcpyHostToDevice, s));
        if (x_val && total) AGP_CUDA_TRY(cudaMemcpyAsync(d_val, x_val, sizeof(float) * total, cudaMemcpyHostToDevice, s));
        off_src = d_off; idx_src = d_idx; val_src = d_val;
    }
    // --- a2: norms of the sign parts (Section 3)
    AGP_CUDA_TRY(cudaMemsetAsync(d_norm, 0, norm_b, s));
    AGP_CUDA_TRY(cudaMemsetAsync(d_bad, 0, sizeof(unsigned int), s));
    if (total) {
        k_norms_sparse<<<blocks_for((unsigned long long)total, kBlock), kBlock, 0, s>>>(off_src, idx_src, val_src, Q, n, d_norm, d_bad);
        g->kernel_launches += 1;
    }
    AGP_CUDA_TRY(cudaGetLastError());
    std::vector<double> norms(2 * Q);
    unsigned int bad = 0;
    AGP_CUDA_TRY(cudaMemcpyAsync(norms.data(), d_norm, norm_b, cudaMemcpyDeviceToHost, s));
    AGP_CUDA_TRY(cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, s));
    AGP_CUDA_TRY(cudaStreamSynchronize(s));
    if (bad) return fail(AGP_EINVAL, "signal index outside [0, n) or non-finite value");

    // --- lanes: one per non-empty sign part
    std::vector<LaneSpec> lanes;
    for (int q = 0; q < Q; ++q)
        for (int part = 0; part < 2; ++part)
            if (norms[2 * q + part] > 0.0) lanes.push_back(LaneSpec{q, part, norms[2 * q + part], n_params == 1 ? 0 : q});
    Workspace *ws = nullptr;
    AGP_TRY(ensure_workspace(g, plain ? 1 : (int)std::max<size_t>(1, lanes.size()), &ws));

    // --- output rows start at zero
    float *out = pi_out;
    const bool host_out = !(flags & AGP_OUTPUT_ON_DEVICE);
    int64_t ld = ld_out;
    if (host_out) {
        AGP_TRY(grow((void **)&ws->out_stage, &ws->out_stage_bytes, sizeof(float) * (size_t)Q * (size_t)std::max<int64_t>(n, 1)));
        out = ws->out_stage;
        ld = n;
    }
    if (n > 0) AGP_CUDA_TRY(cudaMemset2DAsync(out, sizeof(float) * ld, 0, sizeof(float) * n, Q, s));

    if (stats) std::memset(stats, 0, sizeof(agp_stats_t) * Q);
    const KArgs A = make_args(g, ws, collect);
    const int G = plain ? 1 : ws->G;
    std::vector<CoefSpec> cs;
    std::vector<double> wts;
    for (size_t first = 0; first < lanes.size(); first += G) {
        const int count = (int)std::min<size_t>(G, lanes.size() - first);
        int max_L = 0;
        AGP_TRY(prepare_wave(g, ws, lanes, first, count, params, 0, s, cs, wts, &max_L));
        std::vector<int32_t> map(2 * Q, -1);
        for (int l = 0; l < count; ++l) map[2 * lanes[first + l].query + lanes[first + l].part] = l;
        AGP_CUDA_TRY(cudaMemcpyAsync(d_map, map.data(), map_b, cudaMemcpyHostToDevice, s));
        AGP_TRY(set_ctrl(ws, out, 1, ld, s));
        k_seed_sparse<<<blocks_for((unsigned long long)total, kBlock), kBlock, 0, s>>>(A, off_src, idx_src, val_src, Q, d_map, d_norm);
        g->kernel_launches += 2;  // coefficients + seed
        AGP_CUDA_TRY(cudaGetLastError());
        AGP_TRY(run_levels(g, ws, A, max_L, plain, profile, s));
        AGP_TRY(check_ctrl(ws, s));
        if (collect) AGP_TRY(collect_stats(ws, lanes, first, count, stats, s));
    }
    if (collect)
        for (int q = 0; q < Q; ++q) stats[q].levels = params[n_params == 1 ? 0 : q].L + 1;
    if (host_out) {
        if (n > 0) AGP_CUDA_TRY(cudaMemcpy2DAsync(pi_out, sizeof(float) * ld_out, out, sizeof(float) * n, sizeof(float) * n, Q, cudaMemcpyDeviceToHost, s));
        AGP_CUDA_TRY(cudaStreamSynchronize(s));
    }
    AGP_CUDA_TRY(cudaGetLastError());
    return AGP_OK;
}

int feature_propagate(agp_graph_s *g, const agp_params_t *params, const uint16_t *X, int64_t d, int64_t ldx,
                      float *Z, int64_t ldz, uint32_t flags, cudaStream_t s)
{
    if (!g || !params || !X || !Z) return fail(AGP_EINVAL, "NULL argument");
    if (d < 0 || ldx < d || ldz < d) return fail(AGP_EINVAL, "need d >= 0, ldx >= d, ldz >= d");
    if (flags & ~(AGP_PLAIN | AGP_PROFILE)) return fail(AGP_EINVAL, "unknown flag");
    AGP_TRY(validate_params(*params));
    const bool profile = flags & AGP_PROFILE;
    if (d == 0 || g->n == 0) return AGP_OK;
    AGP_CUDA_TRY(cudaSetDevice(g->device));
    const bool plain = flags & AGP_PLAIN;
    const int64_t n = g->n;
    Workspace *ws = nullptr;
    AGP_TRY(ensure_workspace(g, plain ? 1 : (int)std::min<int64_t>(2 * d, 4096), &ws));
    // column norms of the sign parts
    const size_t norm_b = sizeof(double) * 2 * d, map_b = sizeof(int32_t) * 2 * 4096;
    AGP_TRY(grow(&g->in_stage, &g->in_bytes, norm_b + 2 * map_b + 512));
    double *d_norm = (double *)g->in_stage;
    int32_t *d_col = (int32_t *)((char *)g->in_stage + (norm_b + 255) / 256 * 256);
    int32_t *d_part = d_col + 4096;
    AGP_CUDA_TRY(cudaMemsetAsync(d_norm, 0, norm_b, s));
    const int64_t rows_per_block = std::max<int64_t>(64, (n + kGridStrideBlocks - 1) / kGridStrideBlocks);
    k_colnorms_bf16<<<(int)((n + rows_per_block - 1) / rows_per_block), kBlock, 0, s>>>(X, n, d, ldx, rows_per_block, d_norm);
    g->kernel_launches += 1;
    AGP_CUDA_TRY(cudaGetLastError());
    std::vector<double> norms(2 * d);
    AGP_CUDA_TRY(cudaMemcpyAsync(norms.data(), d_norm, norm_b, cudaMemcpyDeviceToHost, s));
    AGP_CUDA_TRY(cudaStreamSynchronize(s));
    AGP_CUDA_TRY(cudaMemset2DAsync(Z, sizeof(float) * ldz, 0, sizeof(float) * d, n, s));
    std::vector<LaneSpec> lanes;
    for (int64_t c = 0; c < d; ++c)
        for (int part = 0; part < 2; ++part)
            if (norms[2 * c + part] > 0.0) lanes.push_back(LaneSpec{(int)c, part, norms[2 * c + part], 0});
    const KArgs A = make_args(g, ws, 0);
    const int G = plain ? 1 : std::min(ws->G, 4096);
    std::vector<CoefSpec> cs;
    std::vector<double> wts;
    for (size_t first = 0; first < lanes.size(); first += G) {
        const int count = (int)std::min<size_t>(G, lanes.size() - first);
        int max_L = 0;
        AGP_TRY(prepare_wave(g, ws, lanes, first, count, params, 1, s, cs, wts, &max_L));
        std::vector<int32_t> col(count), part(count);
        for (int l = 0; l < count; ++l) { col[l] = lanes[first + l].query; part[l] = lanes[first + l].part; }
        AGP_CUDA_TRY(cudaMemcpyAsync(d_col, col.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, s));
        AGP_CUDA_TRY(cudaMemcpyAsync(d_part, part.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, s));
        AGP_TRY(set_ctrl(ws, Z, ldz, 1, s));
        k_seed_dense_bf16<<<kGridStrideBlocks, kBlock, 0, s>>>(A, X, ldx, d_col, d_part, d_norm, count);
        g->kernel_launches += 2;  // coefficients + seed
        AGP_CUDA_TRY(cudaGetLastError());
        AGP_TRY(run_levels(g, ws, A, max_L, plain, profile, s));
        AGP_TRY(check_ctrl(ws, s));
    }
    return AGP_OK;
}

int threshold(agp_graph_s *g, double a, double eps, int64_t count, const int32_t *nodes, const float *c,
              int32_t *k_out, cudaStream_t s)
{
    if (!g) return fail(AGP_EINVAL, "graph is NULL");
    if (!(a >= 0.0 && a <= 1.0) || !(eps >= 0.0)) return fail(AGP_EINVAL, "a in [0,1], eps >= 0");
    if (count < 0 || (count > 0 && (!nodes || !c || !k_out))) return fail(AGP_EINVAL, "bad arrays");
    if (count == 0) return AGP_OK;
    AGP_CUDA_TRY(cudaSetDevice(g->device));
    k_threshold<<<blocks_for((unsigned long long)count, kBlock), kBlock, 0, s>>>(g->dev(), a, exponent_mode(a), eps, count, nodes, c, k_out);
    AGP_CUDA_TRY(cudaGetLastError());
    return AGP_OK;
}

}  // namespace agp
