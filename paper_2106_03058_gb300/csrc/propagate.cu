// propagate.cu -- the level-by-level randomized push of Algorithm 2 on the GPU.
//
// Unit of work: a "lane" = one propagation problem with a non-negative, L1-normalised signal (one
// sign part of one query or of one feature column, Section 3 "Assumption on graph signal"). A
// wave runs up to G lanes at once; every lane keeps one dense FP32 residue vector and accumulates
// its reserve straight into the caller's output. The compaction at the start of a level moves
// r^(i) out of the vector (into the frontier list) and leaves it zero, so the pushes of the level
// build r^(i+1) in the same vector: one n-vector per lane is all that must stay in L2.
//
// One level of all lanes of a wave (Algorithm 2, inner loop over u with r^(i)(u) != 0):
//   k_compact_count / _scan / _emit   dense scan of the lanes' residue vectors: the frontier
//              F_i = {(lane, u) : r^(i)(u) != 0} as an ascending item list with the values
//              r^(i)(u); the vectors are cleared as they are read. Dense levels count, scan and
//              emit (two reads); sparse levels emit to per-block staging, scan and move (one read).
//   k_expand   one thread per item: reserve pi(u) += (w_i/Y_i) r^(i)(u); c = (Y_{i+1}/Y_i) r / d_u^b;
//              deterministic prefix length k(u) = number of neighbours with c / d_v^a >= eps
//              (binary search over the degree-sorted row, all or nothing when a = 0). Short
//              prefixes (pushed by the whole warp at group width 1) and light tails (few expected
//              trials) are done inline; long prefixes, dense tails (p >= 1/4) and heavy sparse
//              tails become records.
//   k_push     one warp per 512-position record: r^(i+1)(v) += c / d_v^a over a prefix chunk, or
//              one Bernoulli trial per position of a dense-tail chunk (kept: += eps).
//   k_sample   one thread per segment record of a sparse tail: subset sampling (Section 4) with
//              neighbours grouped by degree in [2^g, 2^{g+1}); every position of a group is a trial
//              with the group's largest probability p* (geometric skips, so the cost is the number
//              of trials reached) and a reached neighbour is kept with probability p_v / p*.
//   k_level_end   advances the lanes' levels and resets the record counters.
// Pushes are fire-and-forget atomic adds. Sizes stay on the device; kernels are grid-stride loops
// over device-side counts, so a wave's levels are captured in one CUDA graph.
#include <cooperative_groups.h>
#include <cooperative_groups/scan.h>

#include <algorithm>
#include <cfloat>
#include <climits>
#include <limits>
#include <cmath>
#include <cstring>
#include <functional>
#include <vector>

#include "lanes.cuh"

namespace cg = cooperative_groups;

namespace agp {

// ------------------------------------------------------------------------------------ helpers
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

// push condition of Algorithm 2, c / d^a >= eps, as evaluated in FP64 from the FP32 value c. The
// FP32 screen decides every case outside the bracket [eps_lo, eps_hi); only the rare values inside
// it take the FP64 path (see lane_param_derive).
__device__ __forceinline__ bool push_test(float c, int32_t d, const LaneParam &P)
{
    if (P.a_mode == 0) return c >= P.eps_up;
    if (P.screen) {
        const float q = apply_deg(c, d, P.a_mode, P.a);
        if (q >= P.eps_hi) return true;
        if (q < P.eps_lo) return false;
    }
    const double cd = (double)c;
    switch (P.a_mode) {
    case 1: return cd / (double)d >= P.eps_d;
    case 2: return cd / sqrt((double)d) >= P.eps_d;
    default: return cd / pow((double)d, P.a_d) >= P.eps_d;
    }
}

// k(u): length of the deterministic prefix of the degree-sorted row (Section 4 pre-sorting).
__device__ __forceinline__ int det_prefix(float c, const LaneParam &P, const int32_t *row, int d,
                                          const int32_t *deg)
{
    if (P.eps_d == 0.0) return d;
    if (P.a_mode == 0) return (c >= P.eps_up) ? d : 0;
    if (!push_test(c, __ldg(deg + __ldg(row)), P)) return 0;
    if (push_test(c, __ldg(deg + __ldg(row + d - 1)), P)) return d;
    int lo = 1, hi = d - 1;  // first failing position is in [1, d-1]
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (push_test(c, __ldg(deg + __ldg(row + mid)), P)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// ---- pushes --------------------------------------------------------------------------------------
// Neighbour lists are streamed: the CSR is several times larger than L2, while the residue vectors
// that take the random atomic adds fit in it. Neighbour-list loads are therefore marked evict-first
// in L2, so that they do not displace the residue vectors.
__device__ __forceinline__ int32_t ld_col(const int32_t *p)
{
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    int32_t v;
    asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}

// Pushes are fire-and-forget reductions (no value returned, so no thread waits on them), written
// as red.global explicitly: for a pointer loaded from memory (an output row of the lane parameters)
// the compiler cannot prove the global space and would issue a returning generic atomic. The next
// frontier is not tracked during the pushes: each level starts by scanning the residue vectors (see
// k_compact_*), which finds F_i = {u : r^(i)(u) != 0} exactly. No kernel reads what it reduces into,
// so the reductions carry no memory clobber: values the kernel holds (lane parameters, the walk's
// lane states) stay in registers across them.
__device__ __forceinline__ void red_add(float *p, float v)
{
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "f"(v));
}

// The W residues of one node are contiguous and W-float aligned (vectors start 4 KB-aligned), so the
// increments of several lanes at one neighbour go out as one vector reduction.
__device__ __forceinline__ void red_add_v2(float *p, float a, float b)
{
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(__cvta_generic_to_global(p)), "f"(a), "f"(b));
}

__device__ __forceinline__ void red_add_v4(float *p, float a, float b, float c, float d)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(__cvta_generic_to_global(p)), "f"(a), "f"(b),
                 "f"(c), "f"(d));
}

__device__ __forceinline__ void push_to(float *p, float inc)
{
    if (inc != 0.f) red_add(p, inc);
}

// Increments inc[0..W) of the W lanes of a group at neighbour v (Rg: the group's residue block). One
// non-zero lane takes a scalar reduction, several a vector one.
template <int W>
__device__ __forceinline__ void push_node(float *Rg, int32_t v, const float (&inc)[W])
{
    float *p = Rg + (size_t)v * W;
    if constexpr (W == 1) {
        push_to(p, inc[0]);
    } else {
        int nz = 0, last = 0;
#pragma unroll
        for (int j = 0; j < W; ++j)
            if (inc[j] != 0.f) {
                ++nz;
                last = j;
            }
        if (nz == 1) {
            red_add(p + last, inc[last]);
        } else if (nz > 1) {
            if constexpr (W == 2) red_add_v2(p, inc[0], inc[1]);
            else red_add_v4(p, inc[0], inc[1], inc[2], inc[3]);
        }
    }
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

// The paper's subset-sampling scheme (Section 4) for positions [j, gend) of one degree group whose
// largest probability is pstar: the number of trials is Binomial(m, pstar), the trial positions are
// chosen uniformly without replacement, and a reached neighbour is kept with probability p_v / pstar.
// The group is taken in chunks of at most min(64, 10 / pstar) positions: the inversion then starts
// from (1 - pstar)^m >= e^-10.6 (representable in FP32), and Floyd's algorithm keeps the chosen set
// in a 64-bit mask. Chunks are independent, so the positions are still independent Bernoulli(pstar)
// trials, which is the distribution the scheme draws.
template <int W>
__device__ __forceinline__ void sample_group_paper(const KArgs &A, const LaneParam &P, float *Rs, Uniforms &U,
                                                   const int32_t *row, int j, int gend, float pstar, float ce,
                                                   unsigned long long &drawn, unsigned long long &accepted)
{
    const int chunk = (pstar >= 1.f) ? 64 : max(1, (int)fminf(10.f / pstar, 64.f));
    for (int c0 = j; c0 < gend; c0 += chunk) {
        const int m = min(chunk, gend - c0);
        int cnt = m;  // pstar = 1: every position is a trial
        if (pstar < 1.f) {
            const float x = U.next();
            const float ratio = pstar / (1.f - pstar);
            float pk = expf((float)m * log1pf(-pstar));  // Binomial pmf at 0
            float F = pk;
            cnt = 0;
            while (x > F && cnt < m) {
                pk *= (float)(m - cnt) / (float)(cnt + 1) * ratio;
                ++cnt;
                F += pk;
            }
        }
        uint64_t chosen = 0;  // Floyd: for t = m - cnt .. m - 1 pick r in [0, t], or t if r is taken
        for (int t = m - cnt; t < m; ++t) {
            const int r = min((int)(U.next() * (float)(t + 1)), t);
            chosen |= ((chosen >> r) & 1ull) ? (1ull << t) : (1ull << r);
        }
        while (chosen) {
            const int pos = c0 + __ffsll((long long)chosen) - 1;
            chosen &= chosen - 1;
            const int32_t v = ld_col(row + pos);
            ++drawn;
            bool keep = true;
            if (P.a_mode != 0) keep = U.next() * pstar < apply_deg(ce, A.g.deg[v], P.a_mode, P.a);
            if (keep) {
                ++accepted;
                push_to(Rs + (size_t)v * W, P.eps);
            }
        }
    }
}

// Subset sampling of row positions [j0, j1) (Section 4), stream (u, level, seg) of the lane. Rs is
// the lane's residue at node 0 (group block + slot); node v's residue is Rs[v * W].
template <int kSampleBatch, int W, bool kGroups = false>
__device__ void sample_range(const KArgs &A, const LaneParam &P, float *Rs, int32_t u, int lvl, uint32_t seg,
                             const int32_t *row, int j0, int j1, float c, unsigned long long &drawn,
                             unsigned long long &accepted)
{
    Uniforms U((uint32_t)u, (uint32_t)lvl, seg, P.key0, P.key1);
    const float ce = c * P.inv_eps;  // c / eps
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
        if constexpr (kGroups) {  // AGP_SAMPLER_GROUPS: the paper's Binomial-count scheme for this group
            sample_group_paper<W>(A, P, Rs, U, row, j, gend, pstar, ce, drawn, accepted);
            j = gend;
            continue;
        }
        // geometric skip: floor(ln U / ln(1 - p*)) positions are passed over before the next trial.
        // Trials are taken kSampleBatch at a time: their uniforms are drawn first, in the order of
        // one trial after the other (skip, then the acceptance uniform when a > 0), so that the
        // neighbour loads of a batch are in flight together.
        const float rlq = (pstar < 1.f) ? 1.f / log1pf(-pstar) : 0.f;
        bool more = true;
        while (more) {
            int pos[kSampleBatch];
            float acc[kSampleBatch];
            int cnt = 0;
#pragma unroll
            for (int t = 0; t < kSampleBatch; ++t) {
                if (!more) continue;
                const float skip = (pstar < 1.f) ? floorf(logf(U.next()) * rlq) : 0.f;
                if (!(skip < (float)(gend - j))) {
                    j = gend;
                    more = false;
                    continue;
                }
                j += (int)skip;
                pos[t] = j;
                acc[t] = (P.a_mode != 0) ? U.next() : 0.f;
                cnt = t + 1;
                if (++j >= gend) more = false;
            }
            int32_t v[kSampleBatch];
#pragma unroll
            for (int t = 0; t < kSampleBatch; ++t)
                if (t < cnt) v[t] = ld_col(row + pos[t]);
#pragma unroll
            for (int t = 0; t < kSampleBatch; ++t) {
                if (t >= cnt) continue;
                ++drawn;
                bool keep = true;
                if (P.a_mode != 0) keep = acc[t] * pstar < apply_deg(ce, A.g.deg[v[t]], P.a_mode, P.a);
                if (keep) {
                    ++accepted;
                    push_to(Rs + (size_t)v[t] * W, P.eps);
                }
            }
        }
    }
}

// ---- row walks: deterministic prefixes and dense tails of all lanes of a group at once -------------
// A lane's part of the walk of row N_u: positions j < k (the deterministic prefix) get c / d_{v_j}^a;
// if its tail is dense, every position j >= k is an independent Bernoulli trial with probability
// p_j = (c / eps) / d_{v_j}^a (subset sampling by definition, Section 4) and adds eps when kept. The
// uniform of position j is word j & 3 of the Philox block (u, level, j >> 2, kDenseTag) under the
// lane's key, so a lane's draws do not depend on the other lanes of its group or on who walks.
struct WalkLane {
    float c, ce, eps, a;
    int k;          // deterministic prefix length; positions [k, d) are trials when `dense`
    int a_mode;
    int dense;      // 1: dense tail; -1: the lane takes no part in the walk
    int lvl;
    uint32_t key0, key1;
};

__device__ __forceinline__ WalkLane walk_lane(const LaneParam &P, float c, int k, bool dense, int lvl)
{
    WalkLane L;
    L.c = c;
    L.ce = c * P.inv_eps;
    L.eps = P.eps;
    L.a = P.a;
    L.k = k;
    L.a_mode = P.a_mode;
    L.dense = dense ? 1 : 0;
    L.lvl = lvl;
    L.key0 = P.key0;
    L.key1 = P.key1;
    return L;
}

__device__ __forceinline__ WalkLane idle_walk_lane()
{
    WalkLane L{};
    L.dense = -1;
    return L;
}

// Increment of one lane at walk position pos (neighbour degree dv), with the lane's uniform word.
__device__ __forceinline__ float walk_inc(const WalkLane &L, int pos, int32_t dv, uint32_t word, unsigned int &acc)
{
    if (pos < L.k) return (L.a_mode == 0) ? L.c : apply_deg(L.c, dv, L.a_mode, L.a);
    if (L.dense > 0) {
        const float p = (L.a_mode == 0) ? L.ce : apply_deg(L.ce, dv, L.a_mode, L.a);
        if (u01_open(word) < p) {
            ++acc;
            return L.eps;
        }
    }
    return 0.f;
}

// Positions [p0, p1) of the walk (p0 a multiple of 4, p1 - p0 <= 4) for the W lanes L[0..W) (shared
// or local memory). acc[j] counts lane j's kept dense-tail trials.
template <int W>
__device__ __forceinline__ void walk4(const KArgs &A, float *Rg, const WalkLane *L, int32_t u, const int32_t *row,
                                      int p0, int p1, bool need_deg, unsigned int (&acc)[W])
{
    int32_t v[4], dv[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        v[t] = 0;
        dv[t] = 1;
        if (p0 + t < p1) v[t] = ld_col(row + p0 + t);
    }
    if (need_deg)
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (p0 + t < p1) dv[t] = A.g.deg[v[t]];
    float inc[4][W];
#pragma unroll
    for (int j = 0; j < W; ++j) {
#pragma unroll
        for (int t = 0; t < 4; ++t) inc[t][j] = 0.f;
        const int k = L[j].k;
        const int dn = L[j].dense;
        if (dn < 0 || (dn == 0 && k <= p0)) continue;  // no part in these positions
        Philox4 q{0u, 0u, 0u, 0u};
        if (dn > 0 && p1 > k)
            q = philox4x32_10((uint32_t)u, (uint32_t)L[j].lvl, (uint32_t)(p0 >> 2), kDenseTag, L[j].key0, L[j].key1);
        const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (p0 + t < p1) inc[t][j] = walk_inc(L[j], p0 + t, dv[t], w4[t], acc[j]);
    }
#pragma unroll
    for (int t = 0; t < 4; ++t)
        if (p0 + t < p1) push_node<W>(Rg, v[t], inc[t]);
}

// The walk of one lane alone over positions [0, J) (a short row, done by the expanding thread):
// the same increments and uniforms as in a group walk, scalar reductions.
template <int W>
__device__ __forceinline__ void walk_lane_inline(const KArgs &A, float *Rs, const WalkLane &L, int32_t u,
                                                 const int32_t *row, int J, unsigned int &acc)
{
    for (int p0 = 0; p0 < J; p0 += 4) {
        const int p1 = min(p0 + 4, J);
        Philox4 q{0u, 0u, 0u, 0u};
        if (L.dense > 0 && p1 > L.k)
            q = philox4x32_10((uint32_t)u, (uint32_t)L.lvl, (uint32_t)(p0 >> 2), kDenseTag, L.key0, L.key1);
        const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
        int32_t v[4];
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (p0 + t < p1) v[t] = ld_col(row + p0 + t);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (p0 + t >= p1) break;
            const int32_t dv = (L.a_mode != 0) ? A.g.deg[v[t]] : 1;
            push_to(Rs + (size_t)v[t] * W, walk_inc(L, p0 + t, dv, w4[t], acc));
        }
    }
}

// ------------------------------------------------------------------------------------ kernels
// ---- frontier compaction: F_i = {(group, u) : r^(i)(u) != 0 for a lane of the group} ------------
// The residue blocks of the groups holding lanes [0, lanes_used) are cut into units of kScanUnit
// floats (1024 / W nodes); the units are split into part_blocks contiguous ranges. Pass 1 counts the
// frontier items of every range, pass 2 scans the counts, pass 3 writes (group << ubits | u) and the
// W residues of every item, and clears the block. Groups whose lanes are all idle are skipped (their
// residues are zero).
__device__ __forceinline__ void compact_range(const KArgs &A, int64_t &begin, int64_t &end)
{
    const int groups = (min((int)A.ctrl->lanes_used, A.G) + A.W - 1) / A.W;
    const int64_t U = (int64_t)groups * A.units;
    const int64_t per = (U + A.part_blocks - 1) / A.part_blocks;
    begin = (int64_t)blockIdx.x * per;
    end = min(U, begin + per);
}

// Position of a unit: its group and its index in the group's block. A block's units are
// consecutive, so the cursor is set once by a division and then advanced unit by unit.
struct UnitCursor {
    int grp;
    int64_t uig;
};

__device__ __forceinline__ UnitCursor unit_cursor(const KArgs &A, int64_t unit)
{
    UnitCursor c;
    c.grp = (int)(unit / A.units);
    c.uig = unit - (int64_t)c.grp * A.units;
    return c;
}

__device__ __forceinline__ void unit_next(const KArgs &A, UnitCursor &c)
{
    if (++c.uig == A.units) {
        c.uig = 0;
        ++c.grp;
    }
}

template <int W>
__device__ __forceinline__ float4 *unit_at(const KArgs &A, const UnitCursor &c, int64_t &off_f, bool &live)
{
    live = false;
#pragma unroll
    for (int j = 0; j < W; ++j) live |= __ldg(A.level + c.grp * W + j) >= 0;
    off_f = c.uig * kScanUnit;  // float offset of the unit in its group block
    return (float4 *)(A.R + (size_t)c.grp * A.ldR * W + off_f);
}

// frontier items in one float4 of a group block: nodes with a non-zero lane
template <int W>
__device__ __forceinline__ int nz_items(float4 v)
{
    if constexpr (W == 4) return (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f) ? 1 : 0;
    else if constexpr (W == 2) return (v.x != 0.f || v.y != 0.f) + (v.z != 0.f || v.w != 0.f);
    else return (v.x != 0.f) + (v.y != 0.f) + (v.z != 0.f) + (v.w != 0.f);
}

// Exclusive scan across a block of 1024 threads (32 warps): warp shuffles, then one warp scans the
// warp totals. `sm` holds 32 entries; *total receives the block sum. Contains two barriers; the
// caller must not reuse `sm` before a further barrier.
__device__ __forceinline__ unsigned long long block_scan_1024(unsigned long long v, unsigned long long *sm,
                                                               unsigned long long *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = sm[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        sm[lane] = w;  // inclusive prefix of the warp totals
    }
    __syncthreads();
    *total = sm[31];
    return (warp > 0 ? sm[warp - 1] : 0ull) + x - v;
}

template <int W, bool kLocal>
__device__ __forceinline__ void compact_emit_body(const KArgs &A);
__device__ __forceinline__ bool compact_one_pass(const KArgs &A);

template <int W>
__global__ void __launch_bounds__(kBlock, kCompactBlocks) k_compact_count(KArgs A)
{
    if (compact_one_pass(A)) {
        compact_emit_body<W, true>(A);
        return;
    }
    __shared__ unsigned long long red[kBlock / 32];
    __shared__ unsigned long long slot_n[kBlock / 32][W];
    int64_t begin, end;
    compact_range(A, begin, end);
    unsigned long long c = 0;
    const int lane_id = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // without pull levels the pass only counts: kCountBatch units at a time, so that as many loads
    // of each thread are in flight together
    const int64_t batched_end = A.C ? begin : end;
    UnitCursor cur = unit_cursor(A, begin);
    for (int64_t u0 = begin; u0 < batched_end; u0 += kCountBatch) {
        float4 v[kCountBatch];
#pragma unroll
        for (int j = 0; j < kCountBatch; ++j) {
            v[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (u0 + j < end) {
                int64_t off_f;
                bool live;
                const float4 *p = unit_at<W>(A, cur, off_f, live);
                if (live) v[j] = p[threadIdx.x];
            }
            unit_next(A, cur);
        }
#pragma unroll
        for (int j = 0; j < kCountBatch; ++j) c += nz_items<W>(v[j]);
    }
    for (int64_t unit = A.C ? begin : end; unit < end; ++unit, unit_next(A, cur)) {
        const int grp = cur.grp;
        int64_t off_f;
        bool live;
        const float4 *p = unit_at<W>(A, cur, off_f, live);
        if (!live) continue;  // uniform over the block
        const float4 v = p[threadIdx.x];
        c += nz_items<W>(v);
        if (A.C) {
            // the C block of a group that pulled the previous level is cleared here, before this
            // level's expansion writes it again
            if (A.pull[A.G + grp]) reinterpret_cast<float4 *>(A.C + (size_t)grp * A.ldR * W + off_f)[threadIdx.x] =
                make_float4(0.f, 0.f, 0.f, 0.f);
            // frontier volume per lane, sum of d_u over r(u) != 0 (the pull decision of the level)
            const float e[4] = {v.x, v.y, v.z, v.w};
            const int64_t node0 = (off_f + 4 * threadIdx.x) / W;
            unsigned long long ns[W];
#pragma unroll
            for (int sl = 0; sl < W; ++sl) {
                ns[sl] = 0;
#pragma unroll
                for (int k = sl; k < 4; k += W) {
                    const int64_t nd = node0 + k / W;
                    if (e[k] != 0.f && nd < A.g.n) ns[sl] += (unsigned long long)(A.g.rowptr[nd + 1] - A.g.rowptr[nd]);
                }
                for (int o = 16; o > 0; o >>= 1) ns[sl] += __shfl_down_sync(0xffffffffu, ns[sl], o);
                if (lane_id == 0) slot_n[warp][sl] = ns[sl];
            }
            __syncthreads();
            if (threadIdx.x < W) {
                unsigned long long t = 0;
                for (int w = 0; w < kBlock / 32; ++w) t += slot_n[w][threadIdx.x];
                if (t) atomicAdd(&A.lane_count[grp * W + threadIdx.x], t);
            }
            __syncthreads();
        }
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int k = 0; k < kBlock / 32; ++k) t += red[k];
        A.part[blockIdx.x] = (int64_t)t;
    }
}

// Pass 2 (one block of 1024 threads): exclusive scan of the range counts; the total is the
// frontier size.
__global__ void __launch_bounds__(1024) k_compact_scan(KArgs A)
{
    __shared__ unsigned long long sm[32];
    const int t = threadIdx.x, nb = A.part_blocks;
    const int chunk = (nb + blockDim.x - 1) / blockDim.x;
    const int b0 = min(nb, t * chunk), b1 = min(nb, b0 + chunk);
    unsigned long long s = 0;
    for (int b = b0; b < b1; ++b) s += (unsigned long long)A.part[b];
    unsigned long long total;
    unsigned long long run = block_scan_1024(s, sm, &total);
    for (int b = b0; b < b1; ++b) {
        const int64_t v = A.part[b];
        A.part[b] = (int64_t)run;
        run += (unsigned long long)v;
    }
    if (t == 0) {
        A.ctrl->n_items = total;
        A.part[nb] = (int64_t)total;
    }
    if (A.C) {
        // pull or push, per lane, from its own frontier size (so a lane's mode does not depend on the
        // other lanes of its batch); a lane at its last level pushes nothing
        for (int l = t; l < A.G; l += blockDim.x) {
            const unsigned long long vol = A.lane_count[l];
            A.lane_count[l] = 0;
            const int lvl = A.level[l];
            A.pull[l] = (lvl >= 0 && lvl < A.lanes[l].L && vol > 0 && (int64_t)vol >= A.pull_min && !A.lanes[l].sampler)
                            ? 1 : 0;
        }
        __syncthreads();
        for (int gi = t; gi < A.G / A.W; gi += blockDim.x) {
            int any = 0;
            for (int sl = 0; sl < A.W; ++sl) any |= A.pull[gi * A.W + sl];
            A.pull[A.G + gi] = any;
        }
    }
}

// Pass 3: units are taken four at a time. The four float4 loads of a thread are issued together,
// and one block scan of the four per-thread counts (packed in 16-bit fields of a 64-bit word: a
// unit holds at most 1024 items, so no field carries into the next) places every item. The warp
// totals are double-buffered, so a batch needs a single __syncthreads.
//
// kLocal (the one-pass form, for sparse frontiers): the same pass runs first, without a count pass,
// and writes the items of block b to its own stretch of a staging list, slot begin_b * (1024 / W)
// onwards (a block's units hold at most that many items), and its count to part[b]; after the scan
// of the counts, k_compact_emit moves each block's items to their place (compact_gather). The
// residues are read once instead of twice, and the items are moved once more: 4 + 24 rho bytes per
// (lane, node) at frontier density rho (W = 1) against 8 + 8 rho, the better choice below rho = 1/4.
// The staging list is the c_item / k_item storage, which the expansion of the level rewrites.
constexpr int kEmitBatch = 4;
// Residues of the units u0 .. u0 + kEmitBatch - 1 (cursor at u0); returns the cursor after them.
template <int W>
__device__ __forceinline__ UnitCursor load_batch(const KArgs &A, UnitCursor cur, int64_t u0, int64_t end,
                                                 float4 (&v)[kEmitBatch])
{
#pragma unroll
    for (int j = 0; j < kEmitBatch; ++j) {
        v[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (u0 + j < end) {
            int64_t off_f;
            bool live;
            const float4 *p = unit_at<W>(A, cur, off_f, live);
            if (live) v[j] = p[threadIdx.x];
        }
        unit_next(A, cur);
    }
    return cur;
}

template <int W, bool kLocal>
__device__ __forceinline__ void compact_emit_body(const KArgs &A)
{
    __shared__ unsigned long long wsum[2][kBlock / 32];
    int64_t begin, end;
    compact_range(A, begin, end);
    const int lane_id = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *items = kLocal ? reinterpret_cast<uint32_t *>(A.k_item) + begin * (kScanUnit / W) : A.items;
    float *rval = kLocal ? A.c_item + begin * (kScanUnit / W) * W : A.rval;
    unsigned long long run = kLocal ? 0ull : (unsigned long long)A.part[blockIdx.x];
    int parity = 0;
    // the next batch's residues are loaded while the current one is scanned and written
    float4 v_next[kEmitBatch];
    UnitCursor cur = unit_cursor(A, begin);  // at u0
    UnitCursor nxt = load_batch<W>(A, cur, begin, end, v_next);  // at u0 + kEmitBatch
    for (int64_t u0 = begin; u0 < end; u0 += kEmitBatch, parity ^= 1) {
        float4 v[kEmitBatch];
        float4 *ptr[kEmitBatch];
        int grps[kEmitBatch];
        int64_t offs[kEmitBatch];
        unsigned long long packed = 0;
#pragma unroll
        for (int j = 0; j < kEmitBatch; ++j) {
            v[j] = v_next[j];
            ptr[j] = nullptr;
            grps[j] = cur.grp;
            offs[j] = 0;
            if (u0 + j < end) {
                bool live;
                float4 *p = unit_at<W>(A, cur, offs[j], live);
                if (live) ptr[j] = p;
            }
            unit_next(A, cur);
        }
        // cur is now at u0 + kEmitBatch (= nxt); prefetch the batch after it
        nxt = load_batch<W>(A, nxt, u0 + kEmitBatch, end, v_next);
#pragma unroll
        for (int j = 0; j < kEmitBatch; ++j) packed |= (unsigned long long)nz_items<W>(v[j]) << (16 * j);
        unsigned long long x = packed;  // inclusive warp scan of the packed counts
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane_id >= o) x += y;
        }
        if (lane_id == 31) wsum[parity][warp] = x;
        __syncthreads();
        unsigned long long before = 0, total = 0;
        for (int k = 0; k < kBlock / 32; ++k) {
            const unsigned long long w = wsum[parity][k];
            if (k < warp) before += w;
            total += w;
        }
        const unsigned long long excl = before + x - packed;
        unsigned long long unit_base = run;
#pragma unroll
        for (int j = 0; j < kEmitBatch; ++j) {
            const unsigned int c = (unsigned int)(packed >> (16 * j)) & 0xFFFFu;
            unsigned long long off = unit_base + ((excl >> (16 * j)) & 0xFFFFull);
            unit_base += (total >> (16 * j)) & 0xFFFFull;
            if (c == 0) continue;
            const int grp = grps[j];
            const uint32_t hi = (uint32_t)grp << A.ubits;
            const uint32_t node0 = (uint32_t)((offs[j] + 4 * threadIdx.x) / W);  // first node of this float4
            const float e[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
#pragma unroll
            for (int k = 0; k < 4 / W; ++k) {
                bool any = false;
#pragma unroll
                for (int s = 0; s < W; ++s) any |= e[k * W + s] != 0.f;
                if (!any) continue;
                // the staging stretch of a block holds all of its units' nodes: no overflow there
                if (kLocal || off < A.cap_items) {
                    items[off] = hi | (node0 + (uint32_t)k);
                    if constexpr (W == 4) reinterpret_cast<float4 *>(rval)[off] = v[j];
                    else if constexpr (W == 2)
                        reinterpret_cast<float2 *>(rval)[off] = make_float2(e[2 * k], e[2 * k + 1]);
                    else rval[off] = e[k];
                } else {
                    atomicOr(&A.ctrl->error, 1u);
                }
                ++off;
                if (A.collect)
#pragma unroll
                    for (int s = 0; s < W; ++s)
                        if (e[k * W + s] != 0.f) {
                            const int lane = grp * W + s;
                            const int lvl = A.level[lane];
                            if (lvl >= 0 && lvl < kMaxLevels) atomicAdd(&A.stats[lane].frontier[lvl], 1ull);
                        }
            }
            ptr[j][threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        run = unit_base;
    }
    if (kLocal && threadIdx.x == 0) A.part[blockIdx.x] = (int64_t)run;
}

// The one-pass form's last step: block b copies its staged items (count part[b + 1] - part[b]
// after the scan) to items[part[b] ...), in order.
template <int W>
__device__ __forceinline__ void compact_gather(const KArgs &A)
{
    int64_t begin, end;
    compact_range(A, begin, end);
    const unsigned long long n_items = min(A.ctrl->n_items, A.cap_items);
    const unsigned long long o0 = (unsigned long long)A.part[blockIdx.x];
    const unsigned long long o1 = min((unsigned long long)A.part[blockIdx.x + 1], n_items);
    const uint32_t *src_i = reinterpret_cast<const uint32_t *>(A.k_item) + begin * (kScanUnit / W);
    const float *src_r = A.c_item + begin * (kScanUnit / W) * W;
    for (unsigned long long i = threadIdx.x; o0 + i < o1; i += kBlock) {
        A.items[o0 + i] = src_i[i];
        if constexpr (W == 4) reinterpret_cast<float4 *>(A.rval)[o0 + i] = reinterpret_cast<const float4 *>(src_r)[i];
        else if constexpr (W == 2) reinterpret_cast<float2 *>(A.rval)[o0 + i] = reinterpret_cast<const float2 *>(src_r)[i];
        else A.rval[o0 + i] = src_r[i];
    }
}

// The level's compaction form, decided at the end of the previous level (k_level_end) from its
// frontier density; pull levels keep the two-pass form (their count pass also sums volumes).
__device__ __forceinline__ bool compact_one_pass(const KArgs &A) { return !A.C && A.ctrl->scan_mode == 0; }

template <int W>
__global__ void __launch_bounds__(kBlock, kCompactBlocks) k_compact_emit(KArgs A)
{
    if (compact_one_pass(A)) compact_gather<W>(A);
    else compact_emit_body<W, false>(A);
}

// Record counts of one frontier item: x = walk chunks (kChunk positions of the row walk that covers
// the deterministic prefixes and dense tails of the item's walking lanes), y = sparse-tail segments
// (over all lanes of the item). A lane whose own walk is short (<= kInlineDet positions) is walked
// here, alone. Written for every item; k_rec_* turn them into record lists without a shared counter.
// flag_item bits: j = lane j's tail is dense, 8 + j = lane j is in the walk, 16 + j = lane j has
// segments; c_item / k_item / seg_item are written for the lanes named there.
// A short deterministic prefix left to the warp (group width 1): the row, its length and the
// lane's increment parameters. len = 0: none.
struct InlinePush {
    int64_t e0;
    float c, a;
    int len, a_mode, grp;
};

template <int W>
__device__ __forceinline__ uint2 expand_item(const KArgs &A, unsigned long long idx, InlinePush &ip)
{
    Ctrl *ctrl = A.ctrl;
    // every array read here is written only by earlier kernels: read-only path
    const uint32_t item = __ldg(A.items + idx);
    const int grp = (int)(item >> A.ubits);
    const int32_t u = (int32_t)(item & A.umask);
    const int64_t e0 = __ldg(A.g.rowptr + u);
    const int d = (int)(__ldg(A.g.rowptr + u + 1) - e0);  // row length
    const int32_t du = A.rows_in ? __ldg(A.g.deg + u) : d;  // d_u of the normalisation (the row length
                                                            // except on in-neighbour rows)
    float *Rg = A.R + (size_t)grp * A.ldR * W;  // r^(i+1): the compaction emptied r^(i)
    const int32_t *row = A.g.colidx + e0;
    int J = 0, nseg = 0;
    uint32_t flags = 0;
    // the lanes one after the other (a rolled loop keeps the per-lane state out of spilled registers)
#pragma unroll 1
    for (int j = 0; j < W; ++j) {
        const float rj = __ldg(A.rval + idx * W + j);  // the compaction read r^(i)(u) and cleared it
        if (rj == 0.f) continue;
        const int lane = grp * W + j;
        const int lvl = __ldg(A.level + lane);
        if (lvl < 0 || lvl >= kMaxLevels) {
            atomicOr(&ctrl->error, 16u);
            continue;
        }
        const LaneParam &P = A.lanes[lane];
        const float2 cf = __ldg(A.coef + lane * kMaxLevels + lvl);
        // reserve: q^(i)(u) = (w_i / Y_i) r^(i)(u), added to pi (scale folded into cf.x)
        red_add(P.out + (int64_t)u * P.su, cf.x * rj);
        // nothing to push: the last level, an empty row, or d_u = 0 with b > 0 (D^-b := 0)
        if (lvl >= P.L || d == 0 || (du == 0 && P.b_mode != 0)) continue;
        const float c = apply_deg(cf.y * rj, du, P.b_mode, P.b);  // (Y_{i+1}/Y_i) r / d_u^b
        if (!(c > 0.f)) continue;
        if (A.C && A.pull[lane]) {  // this level pulls: the targets gather c(u) (k_pull_*)
            A.C[((size_t)grp * A.ldR + u) * W + j] = c;
            continue;
        }
        const int k = det_prefix(c, P, row, d, A.g.deg);
        const int tail = d - k;
        bool is_dense = false;
        int seglen = 0;
        unsigned long long drawn = 0, accepted = 0;
        if (tail > 0) {
            const float ce = c * P.inv_eps;
            const float p0 = fminf(1.f, (P.a_mode == 0) ? ce : apply_deg(ce, A.g.deg[row[k]], P.a_mode, P.a));
            const float expect = p0 * (float)tail;  // upper bound on the trials reached
            if (expect <= kLightSamples && !P.sampler) {
                sample_range<2, W>(A, P, Rg + j, u, lvl, 0u, row, k, d, c, drawn, accepted);
            } else if (p0 >= kDenseP && !P.sampler) {
                is_dense = true;  // most positions are kept: one Bernoulli per position in the walk
            } else {
                int ns = (int)fminf(ceilf(expect / kSegSamples), (float)((tail + kMinSeg - 1) / kMinSeg));
                ns = max(ns, 1);
                seglen = (tail + ns - 1) / ns;
                nseg += (tail + seglen - 1) / seglen;
            }
        }
        // a short deterministic prefix is pushed here; a longer one, and every dense tail, joins the
        // group's walk (warps, coalesced neighbour loads, one reduction per neighbour for the group)
        const int wlen = is_dense ? d : k;
        bool in_walk = false;
        if (wlen > 0) {
            if (!is_dense && wlen <= kInlineDet) {
                if constexpr (W == 1) {
                    // pushed by the whole warp after the items (warp_inline_push)
                    ip.e0 = e0;
                    ip.c = c;
                    ip.a = P.a;
                    ip.len = wlen;
                    ip.a_mode = P.a_mode;
                    ip.grp = grp;
                } else {
                    unsigned int acc = 0;
                    walk_lane_inline<W>(A, Rg + j, walk_lane(P, c, k, false, lvl), u, row, wlen, acc);
                }
                if (A.collect) atomicAdd(&A.stats[lane].by_kernel[0][0], (unsigned long long)k);
            } else {
                in_walk = true;
                J = max(J, wlen);
            }
        }
        if (in_walk || seglen > 0) {
            A.c_item[idx * W + j] = c;
            A.k_item[idx * W + j] = k;
            A.seg_item[idx * W + j] = seglen;
            flags |= (in_walk ? (1u << (8 + j)) : 0u) | ((in_walk && is_dense) ? (1u << j) : 0u) |
                     (seglen > 0 ? (1u << (16 + j)) : 0u);
        }
        if (A.collect && (drawn | accepted)) {
            atomicAdd(&A.stats[lane].by_kernel[0][1], drawn);
            atomicAdd(&A.stats[lane].by_kernel[0][2], accepted);
        }
    }
    const uint2 nrec = make_uint2(J > 0 ? (unsigned int)((J + kChunk - 1) / kChunk) : 0u, (unsigned int)nseg);
    if (nrec.x | nrec.y) A.flag_item[idx] = flags;
    return nrec;
}

// The short deterministic prefixes of a warp's 32 items (group width 1), pushed by the whole warp:
// the prefixes are laid end to end and every lane takes four consecutive outputs of each round of
// 128, so a round's neighbour loads are mostly coalesced and no lane waits for the longest prefix.
// Output p belongs to the first lane whose inclusive prefix-length sum exceeds p (a five-step search
// over the lanes' sums). The increments are those of the lane's own walk, c / d_v^a.
__device__ __forceinline__ void warp_inline_push(const KArgs &A, const InlinePush &ip)
{
    const int lane_id = threadIdx.x & 31;
    unsigned int incl = (unsigned int)ip.len;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane_id >= o) incl += y;
    }
    const unsigned int total = __shfl_sync(0xffffffffu, incl, 31);
    const unsigned int excl = incl - (unsigned int)ip.len;
    for (unsigned int p0 = 0; p0 < total; p0 += 128) {
        int owner[4];
        unsigned int pos[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const unsigned int p = p0 + 4 * lane_id + t;
            int lo = 0;
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) {
                const unsigned int v = __shfl_sync(0xffffffffu, incl, lo + s - 1);
                if (v <= p) lo += s;
            }
            owner[t] = lo;
            pos[t] = p - __shfl_sync(0xffffffffu, excl, lo);
        }
        int32_t v[4];
        float c[4], a[4];
        int am[4];
        float *Rg[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int64_t e0 = __shfl_sync(0xffffffffu, ip.e0, owner[t]);
            c[t] = __shfl_sync(0xffffffffu, ip.c, owner[t]);
            a[t] = __shfl_sync(0xffffffffu, ip.a, owner[t]);
            am[t] = __shfl_sync(0xffffffffu, ip.a_mode, owner[t]);
            const int grp = __shfl_sync(0xffffffffu, ip.grp, owner[t]);
            Rg[t] = A.R + (size_t)grp * A.ldR;
            v[t] = (p0 + 4 * lane_id + t < total) ? ld_col(A.g.colidx + e0 + pos[t]) : -1;
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (v[t] < 0) continue;
            const float inc = (am[t] == 0) ? c[t] : apply_deg(c[t], A.g.deg[v[t]], am[t], a[t]);
            push_to(Rg[t] + v[t], inc);
        }
    }
}

// Items are split into contiguous block ranges, a multiple of kBlock long (k_rec_emit walks the
// same ranges). Returns [begin, end) of this block.
__device__ __forceinline__ void item_range(const KArgs &A, unsigned long long &begin, unsigned long long &end)
{
    const unsigned long long n = min(A.ctrl->n_items, A.cap_items);
    const unsigned long long per = ((n + gridDim.x - 1) / gridDim.x + kBlock - 1) / kBlock * kBlock;
    begin = (unsigned long long)blockIdx.x * per;
    end = min(n, begin + per);
}

template <int W>
__global__ void __launch_bounds__(kBlock, kMinBlocks) k_expand(KArgs A)
{
    // block totals of the two record kinds, gathered without a closing barrier: every warp adds its
    // totals, and the last warp to finish writes them (warps that finish early leave at once)
    __shared__ unsigned long long tot_s[2];
    __shared__ unsigned int warps_done;
    if (threadIdx.x < 2) tot_s[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) warps_done = 0u;
    __syncthreads();
    unsigned long long begin, end;
    item_range(A, begin, end);
    // per-thread record totals (32-bit: a thread's items have far fewer than 2^32 records; the
    // block sums are 64-bit)
    unsigned int tot[2] = {0u, 0u};
    // warp-uniform trip count: the whole warp takes part in the inline pushes of every round
    for (unsigned long long base = begin; base < end; base += kBlock) {
        const unsigned long long idx = base + threadIdx.x;
        InlinePush ip{0, 0.f, 0.f, 0, 0, 0};
        if (idx < end) {
            const uint2 nr = expand_item<W>(A, idx, ip);
            A.nrec[idx] = nr;
            tot[0] += nr.x;
            tot[1] += nr.y;
        }
        if constexpr (W == 1) warp_inline_push(A, ip);
    }
    // block totals of the two record kinds, for k_rec_scan
    unsigned long long wt[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        wt[t] = tot[t];
        for (int o = 16; o > 0; o >>= 1) wt[t] += __shfl_down_sync(0xffffffffu, wt[t], o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&tot_s[0], wt[0]);
        atomicAdd(&tot_s[1], wt[1]);
        __threadfence_block();  // the sums before the count of finished warps
        if (atomicAdd(&warps_done, 1u) == kBlock / 32 - 1) {
            __threadfence_block();
            A.rpart[blockIdx.x] = atomicAdd(&tot_s[0], 0ull);
            A.rpart[(size_t)gridDim.x + blockIdx.x] = atomicAdd(&tot_s[1], 0ull);
        }
    }
}

// One block of 1024 threads: exclusive scan of the per-block record counts of k_expand (two kinds,
// each a row of nb entries); the totals become the record list sizes.
__global__ void __launch_bounds__(1024) k_rec_scan(KArgs A, int nb)
{
    __shared__ unsigned long long sm[32];
    const int t = threadIdx.x;
    const int chunk = (nb + blockDim.x - 1) / blockDim.x;
    const int b0 = min(nb, t * chunk), b1 = min(nb, b0 + chunk);
    for (int kind = 0; kind < 2; ++kind) {
        unsigned long long *row = A.rpart + (size_t)kind * nb;
        unsigned long long s = 0;
        for (int b = b0; b < b1; ++b) s += row[b];
        unsigned long long total;
        unsigned long long run = block_scan_1024(s, sm, &total);
        for (int b = b0; b < b1; ++b) {
            const unsigned long long v = row[b];
            row[b] = run;
            run += v;
        }
        if (t == 0) {
            if (kind == 0) A.ctrl->n_det = total;
            else A.ctrl->n_smp = total;
        }
        __syncthreads();  // sm is reused by the next kind
    }
}

// Writes the records of every item at its block's offset plus its place in the block: walk chunks
// (item, chunk) and sparse-tail segments (item, segment over the item's lanes), in item order. Same
// grid and ranges as k_expand.
__global__ void __launch_bounds__(kBlock) k_rec_emit(KArgs A)
{
    __shared__ unsigned int wsum[2][2][kBlock / 32];
    unsigned long long begin, end;
    item_range(A, begin, end);
    const int lane_id = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long base[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) base[t] = A.rpart[(size_t)t * gridDim.x + blockIdx.x];
    int parity = 0;
    // the counts of the next tile are loaded while the current one is scanned and written
    uint2 nr_next = (begin + threadIdx.x < end) ? A.nrec[begin + threadIdx.x] : make_uint2(0u, 0u);
    for (unsigned long long tile = begin; tile < end; tile += kBlock, parity ^= 1) {
        const unsigned long long idx = tile + threadIdx.x;
        const uint2 nr = nr_next;
        const unsigned long long nidx = idx + kBlock;
        nr_next = (nidx < end) ? A.nrec[nidx] : make_uint2(0u, 0u);
        const unsigned int cnt[2] = {nr.x, nr.y};
        unsigned int x[2];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            x[t] = cnt[t];  // inclusive warp scan
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned int y = __shfl_up_sync(0xffffffffu, x[t], o);
                if (lane_id >= o) x[t] += y;
            }
            if (lane_id == 31) wsum[parity][t][warp] = x[t];
        }
        __syncthreads();
        const uint32_t idx0 = (uint32_t)(tile + (threadIdx.x & ~31u));  // item of the warp's lane 0
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            unsigned long long before = 0, all = 0;
            for (int w = 0; w < kBlock / 32; ++w) {
                const unsigned int v = wsum[parity][t][w];
                if (w < warp) before += v;
                all += v;
            }
            // the warp's records are written by consecutive lanes (a hub item has hundreds): output p
            // of the warp belongs to the first lane whose inclusive count exceeds p, found by a
            // five-step search over the lanes' counts
            const unsigned int wtotal = __shfl_sync(0xffffffffu, x[t], 31);
            const unsigned int excl = x[t] - cnt[t];
            uint2 *rec = t == 0 ? A.det_rec : A.smp_rec;
            const unsigned long long cap = t == 0 ? A.cap_det : A.cap_smp;
            const unsigned long long wbase = base[t] + before;
            for (unsigned int p0 = 0; p0 < wtotal; p0 += 32) {
                const unsigned int p = p0 + lane_id;
                int lo = 0;
#pragma unroll
                for (int s = 16; s > 0; s >>= 1) {
                    const unsigned int v = __shfl_sync(0xffffffffu, x[t], lo + s - 1);
                    if (v <= p) lo += s;
                }
                const unsigned int r = p - __shfl_sync(0xffffffffu, excl, lo);
                if (p < wtotal) {
                    if (wbase + p < cap) rec[wbase + p] = make_uint2(idx0 + (uint32_t)lo, r);
                    else atomicOr(&A.ctrl->error, t == 0 ? 2u : 4u);
                }
            }
            base[t] += all;
        }
    }
}

// One warp per walk chunk: positions [chunk * kChunk, ...) of the item's row walk, 4 consecutive
// positions per thread (one Philox block per dense lane), coalesced neighbour loads. The record's
// lane states sit in shared memory, one slot per warp.
template <int W>
__global__ void __launch_bounds__(kBlock, kMinBlocks) k_push(KArgs A)
{
    __shared__ WalkLane sL[kBlock / 32][W];
    const unsigned long long n_rec = min(A.ctrl->n_det, A.cap_det);
    const int lane_id = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    for (unsigned long long rec = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5; rec < n_rec; rec += nwarps) {
        const uint2 Rc = A.det_rec[rec];
        const unsigned long long idx = Rc.x;
        const uint32_t item = A.items[idx];
        const int grp = (int)(item >> A.ubits);
        const int32_t u = (int32_t)(item & A.umask);
        const int64_t e0 = A.g.rowptr[u];
        const int d = (int)(A.g.rowptr[u + 1] - e0);  // row length
        const uint32_t flags = A.flag_item[idx];
        // the record's lane states: in registers for a single lane, else in the warp's shared slot
        WalkLane L1[1];
        const WalkLane *Ls = L1;
        if constexpr (W == 1) {
            L1[0] = walk_lane(A.lanes[grp], A.c_item[idx], A.k_item[idx], flags & 1u, A.level[grp]);
        } else {
            __syncwarp();
            if (lane_id < W) {
                const int j = lane_id;
                WalkLane L = idle_walk_lane();
                if ((flags >> (8 + j)) & 1u) {
                    const int lane = grp * W + j;
                    L = walk_lane(A.lanes[lane], A.c_item[idx * W + j], A.k_item[idx * W + j], (flags >> j) & 1u,
                                  A.level[lane]);
                }
                sL[warp][j] = L;
            }
            __syncwarp();
            Ls = sL[warp];
        }
        int J = 0;
        bool need_deg = false;
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const WalkLane &L = Ls[j];
            if (L.dense < 0) continue;
            J = max(J, L.dense > 0 ? d : L.k);
            need_deg |= L.a_mode != 0;
        }
        float *Rg = A.R + (size_t)grp * A.ldR * W;
        const int32_t *row = A.g.colidx + e0;
        const int c0 = (int)Rc.y * kChunk, c1 = min(J, c0 + kChunk);
        unsigned int acc[W] = {};
        for (int p0 = c0 + 4 * lane_id; p0 < c1; p0 += 128) walk4<W>(A, Rg, Ls, u, row, p0, min(p0 + 4, c1), need_deg, acc);
        if (A.collect) {
#pragma unroll
            for (int j = 0; j < W; ++j) {
                const WalkLane &L = Ls[j];
                if (L.dense < 0) continue;
                const int lane = grp * W + j;
                if (lane_id == 0) {
                    const int det = max(0, min(L.k, c1) - c0);
                    const int trials = (L.dense > 0) ? max(0, c1 - max(c0, L.k)) : 0;
                    atomicAdd(&A.stats[lane].by_kernel[1][0], (unsigned long long)det);
                    atomicAdd(&A.stats[lane].by_kernel[1][1], (unsigned long long)trials);
                }
                if (acc[j]) atomicAdd(&A.stats[lane].by_kernel[1][2], (unsigned long long)acc[j]);
            }
        }
    }
}

// One thread per sparse-tail segment: record (item, s), s counting the segments of the item's lanes
// in slot order.
// kGroups: the wave may hold lanes of the paper's group sampler (AGP_SAMPLER_GROUPS); the default
// instantiation carries no code of that scheme
template <int W, bool kGroups>
__global__ void __launch_bounds__(kBlock, kMinBlocks) k_sample(KArgs A)
{
    const unsigned long long n_smp = min(A.ctrl->n_smp, A.cap_smp);
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long rec = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; rec < n_smp; rec += stride) {
        const uint2 Rc = A.smp_rec[rec];
        const unsigned long long idx = Rc.x;
        const uint32_t item = A.items[idx];
        const int grp = (int)(item >> A.ubits);
        const int32_t u = (int32_t)(item & A.umask);
        const int64_t e0 = A.g.rowptr[u];
        const int d = (int)(A.g.rowptr[u + 1] - e0);  // row length
        const uint32_t flags = A.flag_item[idx];
        int s = (int)Rc.y, slot = -1, k = 0, seglen = 0;
#pragma unroll
        for (int j = 0; j < W; ++j) {
            if (slot >= 0 || !((flags >> (16 + j)) & 1u)) continue;
            const int sl = A.seg_item[idx * W + j];
            const int kj = A.k_item[idx * W + j];
            const int ns = (d - kj + sl - 1) / sl;
            if (s < ns) {
                slot = j;
                k = kj;
                seglen = sl;
            } else {
                s -= ns;
            }
        }
        if (slot < 0) {
            atomicOr(&A.ctrl->error, 4u);
            continue;
        }
        const int lane = grp * W + slot;
        const int lvl = A.level[lane];
        const LaneParam &P = A.lanes[lane];
        float *Rs = A.R + (size_t)grp * A.ldR * W + slot;
        const float c = A.c_item[idx * W + slot];
        const int j0 = k + s * seglen, j1 = min(d, j0 + seglen);
        const int32_t *row = A.g.colidx + e0;
        unsigned long long drawn = 0, accepted = 0;
        if (kGroups && P.sampler) sample_range<4, W, true>(A, P, Rs, u, lvl, (uint32_t)s, row, j0, j1, c, drawn, accepted);
        else sample_range<4, W>(A, P, Rs, u, lvl, (uint32_t)s, row, j0, j1, c, drawn, accepted);
        if (A.collect && (drawn | accepted)) {
            atomicAdd(&A.stats[lane].by_kernel[2][1], drawn);
            atomicAdd(&A.stats[lane].by_kernel[2][2], accepted);
        }
    }
}

// ---- pull levels -------------------------------------------------------------------------------
// A lane whose frontier covers a large part of the graph spends most of a pushed level on random
// reductions into r^(i+1). On an undirected graph the row of v lists exactly the nodes that push to
// v, so the same level can be computed by the targets: every node v walks its row once for the
// group, gathers c(u) of the pulling lanes (published by the expansion in the C block) and adds, per
// lane and edge, what Algorithm 2 adds there: c(u) / d_v^a when that increment passes the push test,
// else eps with probability (c(u) / eps) / d_v^a. The trial of edge (u, v) uses word 0 of the Philox
// block (u, v, level, kPullTag) under the lane's key. The sums land in the lane's own slot of R with
// plain stores: no other kernel writes a pulling lane's slot during the level, and the compaction
// left it zero.
struct PullLane {
    LaneParam P;
    int lvl;
    int on;
};

template <int W>
__device__ __forceinline__ void pull_edge(const PullLane *L, float4 cu4, int32_t u, int32_t v, int32_t dv,
                                          float (&acc)[W], unsigned int (&cnt)[W][3])
{
    const float cu[4] = {cu4.x, cu4.y, cu4.z, cu4.w};
#pragma unroll
    for (int j = 0; j < W; ++j) {
        const float c = cu[j];
        if (!L[j].on || !(c > 0.f)) continue;
        const LaneParam &P = L[j].P;
        if (P.eps_d == 0.0 || push_test(c, dv, P)) {
            acc[j] += (P.a_mode == 0) ? c : apply_deg(c, dv, P.a_mode, P.a);
            ++cnt[j][0];
        } else {
            const float p = (P.a_mode == 0) ? c * P.inv_eps : apply_deg(c * P.inv_eps, dv, P.a_mode, P.a);
            const Philox4 q = philox4x32_10((uint32_t)u, (uint32_t)v, (uint32_t)L[j].lvl, kPullTag, P.key0, P.key1);
            ++cnt[j][1];
            if (u01_open(q.x) < p) {
                acc[j] += P.eps;
                ++cnt[j][2];
            }
        }
    }
}

template <int W>
__device__ __forceinline__ float4 load_c(const float *Cg, int32_t u)
{
    if constexpr (W == 4) return __ldg(reinterpret_cast<const float4 *>(Cg) + u);
    else if constexpr (W == 2) {
        const float2 c = __ldg(reinterpret_cast<const float2 *>(Cg) + u);
        return make_float4(c.x, c.y, 0.f, 0.f);
    } else {
        return make_float4(__ldg(Cg + u), 0.f, 0.f, 0.f);
    }
}

template <int W>
__device__ __forceinline__ void pull_store(const KArgs &A, const PullLane *L, float *Rg, int32_t v,
                                           const float (&acc)[W])
{
#pragma unroll
    for (int j = 0; j < W; ++j)
        if (L[j].on && acc[j] != 0.f) Rg[(size_t)v * W + j] = acc[j];
}

template <int W>
__device__ __forceinline__ void pull_stats(const KArgs &A, int grp, const PullLane *L, const unsigned int (&cnt)[W][3])
{
    if (!A.collect) return;
#pragma unroll
    for (int j = 0; j < W; ++j)
        if (L[j].on && (cnt[j][0] | cnt[j][1])) {
            LaneStats &S = A.stats[grp * W + j];
            atomicAdd(&S.by_kernel[1][0], (unsigned long long)cnt[j][0]);
            atomicAdd(&S.by_kernel[1][1], (unsigned long long)cnt[j][1]);
            atomicAdd(&S.by_kernel[1][2], (unsigned long long)cnt[j][2]);
        }
}

// the group's lane states into shared memory (threads 0..W-1), read by every thread of the block
template <int W>
__device__ __forceinline__ void pull_lanes(const KArgs &A, int grp, PullLane *L)
{
    if (threadIdx.x < W) {
        const int lane = grp * W + threadIdx.x;
        L[threadIdx.x].on = A.pull[lane];
        L[threadIdx.x].lvl = A.level[lane];
        L[threadIdx.x].P = A.lanes[lane];
    }
}

// CLS 0: short rows, a thread each; 1: medium rows, a warp each; 2: long rows, a block each
template <int W, int CLS>
__global__ void __launch_bounds__(kBlock) k_pull(KArgs A)
{
    if (!A.C) return;
    __shared__ float part[kBlock / 32][W];
    __shared__ PullLane L[W];
    const int groups = (min((int)A.ctrl->lanes_used, A.G) + W - 1) / W;
    const int64_t count = A.row_count[CLS];
    const int32_t *rows = A.rows[CLS];
    const int lane_id = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int grp = 0; grp < groups; ++grp) {
        if (!A.pull[A.G + grp]) continue;  // uniform over the grid
        __syncthreads();  // the previous group's states are no longer read
        pull_lanes<W>(A, grp, L);
        __syncthreads();
        const float *Cg = A.C + (size_t)grp * A.ldR * W;
        float *Rg = A.R + (size_t)grp * A.ldR * W;
        unsigned int cnt[W][3] = {};
        if constexpr (CLS == 0) {
            for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < count; r += (int64_t)gridDim.x * blockDim.x) {
                const int32_t v = rows[r];
                const int64_t e0 = A.g.rowptr[v], e1 = A.g.rowptr[v + 1];
                const int32_t dv = (int32_t)(e1 - e0);
                float acc[W] = {};
                for (int64_t e = e0; e < e1; ++e) {
                    const int32_t u = ld_col(A.g.colidx + e);
                    pull_edge<W>(L, load_c<W>(Cg, u), u, v, dv, acc, cnt);
                }
                pull_store<W>(A, L, Rg, v, acc);
            }
        } else if constexpr (CLS == 1) {
            const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
            for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < count; r += nw) {
                const int32_t v = rows[r];
                const int64_t e0 = A.g.rowptr[v], e1 = A.g.rowptr[v + 1];
                const int32_t dv = (int32_t)(e1 - e0);
                float acc[W] = {};
                for (int64_t e = e0 + lane_id; e < e1; e += 32) {
                    const int32_t u = ld_col(A.g.colidx + e);
                    pull_edge<W>(L, load_c<W>(Cg, u), u, v, dv, acc, cnt);
                }
#pragma unroll
                for (int j = 0; j < W; ++j)
                    for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_down_sync(0xffffffffu, acc[j], o);
                if (lane_id == 0) pull_store<W>(A, L, Rg, v, acc);
            }
        } else {
            for (int64_t r = blockIdx.x; r < count; r += gridDim.x) {
                const int32_t v = rows[r];
                const int64_t e0 = A.g.rowptr[v], e1 = A.g.rowptr[v + 1];
                const int32_t dv = (int32_t)(e1 - e0);
                float acc[W] = {};
                for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
                    const int32_t u = ld_col(A.g.colidx + e);
                    pull_edge<W>(L, load_c<W>(Cg, u), u, v, dv, acc, cnt);
                }
#pragma unroll
                for (int j = 0; j < W; ++j) {
                    for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_down_sync(0xffffffffu, acc[j], o);
                    if (lane_id == 0) part[warp][j] = acc[j];
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    float tot[W];
#pragma unroll
                    for (int j = 0; j < W; ++j) {
                        tot[j] = 0.f;
                        for (int w = 0; w < kBlock / 32; ++w) tot[j] += part[w][j];
                    }
                    pull_store<W>(A, L, Rg, v, tot);
                }
                __syncthreads();
            }
        }
        pull_stats<W>(A, grp, L, cnt);
    }
}

__global__ void k_level_end(KArgs A)
{
    Ctrl *ctrl = A.ctrl;
    for (int l = threadIdx.x; l < A.G; l += blockDim.x) {
        const int lvl = A.level[l];
        if (lvl >= 0) A.level[l] = (lvl < A.lanes[l].L) ? lvl + 1 : -1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ctrl->n_det = 0;
        ctrl->n_smp = 0;
        // the next level's compaction form: the frontier density predicted as this level's, times
        // its growth over the previous level when it grew; one pass below a predicted 1/6 of the
        // scanned (group, node) pairs (the break-even of the two forms is 1/4)
        const unsigned long long groups = (min((int)ctrl->lanes_used, A.G) + A.W - 1) / A.W;
        const unsigned long long items = ctrl->n_items, prev = ctrl->prev_items;
        const double grow = (prev > 0 && items > prev) ? (double)items / (double)prev : 1.0;
        ctrl->scan_mode = ((double)items * grow * 6.0 < (double)(groups * (unsigned long long)A.ldR)) ? 0u : 1u;
        ctrl->prev_items = items;
    }
}

// ---- seeds -------------------------------------------------------------------------------------
// Residue of `lane` at node u: lane / W is its group, lane % W its slot in the group's block.
__device__ __forceinline__ float *lane_res(const KArgs &A, int lane, int64_t u)
{
    return A.R + ((size_t)(lane / A.W) * A.ldR + (size_t)u) * A.W + (lane % A.W);
}

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
    const int64_t total = off[Q];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int q = query_of(off, Q, t);
        const float x = val ? val[t] : 1.f;
        if (x == 0.f) continue;
        const int part = x < 0.f ? 1 : 0;
        const int lane = lane_of[2 * q + part];
        const int32_t u = idx[t];
        if (lane < 0 || u < 0 || u >= A.g.n) continue;
        push_to(lane_res(A, lane, u), (float)((double)fabsf(x) / norms[2 * q + part]));
    }
}

// one-hot seeds x = e_source (already normalised) for lanes[t]
__global__ void k_seed_sources(KArgs A, const int32_t *lanes, const int32_t *sources, int count)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) {
        const int lane = lanes[t];
        const int32_t u = sources[t];
        if (u >= 0 && u < A.g.n) push_to(lane_res(A, lane, u), 1.f);
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

// seed l (lane lane_of[l], or l when lane_of is NULL) takes column col_of[l], sign part part_of[l]
__global__ void k_seed_dense_bf16(KArgs A, const uint16_t *X, int64_t ldx, const int32_t *lane_of, const int32_t *col_of,
                                  const int32_t *part_of, const double *norms, int nl)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) A.ctrl->scan_mode = 1u;  // dense seeds: two-pass compaction
    const int64_t total = A.g.n * nl;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(t % nl);
        const int64_t u = t / nl;
        const int col = col_of[l];
        const float x = __uint_as_float((uint32_t)X[u * ldx + col] << 16);
        const int part = part_of[l];
        if (!((part == 0 && x > 0.f) || (part == 1 && x < 0.f))) continue;
        const int lane = lane_of ? lane_of[l] : l;
        push_to(lane_res(A, lane, u), (float)((double)fabsf(x) / norms[2 * col + part]));
    }
}

// ---- dense signal rows (agp_query_dense) ----------------------------------------------------------
__device__ __forceinline__ float load_x(const float *X, int64_t i) { return X[i]; }
__device__ __forceinline__ float load_x(const uint16_t *X, int64_t i) { return __uint_as_float((uint32_t)X[i] << 16); }

// Sign-part norms of the rows of X in a fixed order, so they do not depend on scheduling: row q is
// cut into `chunks` ranges (blockIdx.x), each reduced by one block (per-thread sums in index order,
// then a shuffle tree and the warp totals in order) into part[(q * chunks + c) * 2 + {0: x+, 1: x-}];
// k_rownorm_sum adds a row's ranges in order. Non-finite entries set *bad.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_rownorm_part(const T *X, int64_t ldx, int64_t n, int chunks, double *part,
                                                         unsigned int *bad)
{
    __shared__ double sm[2][kBlock / 32];
    const int q = blockIdx.y, c = blockIdx.x;
    const int64_t per = (n + chunks - 1) / chunks, r0 = (int64_t)c * per, r1 = min(n, r0 + per);
    double sp = 0.0, sn = 0.0;
    for (int64_t u = r0 + threadIdx.x; u < r1; u += kBlock) {
        const float x = load_x(X, (int64_t)q * ldx + u);
        if (!isfinite(x)) atomicOr(bad, 1u);
        else if (x > 0.f) sp += (double)x;
        else if (x < 0.f) sn -= (double)x;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sp += __shfl_down_sync(0xffffffffu, sp, o);
        sn += __shfl_down_sync(0xffffffffu, sn, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sm[0][threadIdx.x >> 5] = sp;
        sm[1][threadIdx.x >> 5] = sn;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double t = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) t += sm[threadIdx.x][w];
        part[((size_t)q * chunks + c) * 2 + threadIdx.x] = t;
    }
}

__global__ void k_rownorm_sum(const double *part, int chunks, int Q, double *norms)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;  // t = 2q + sign part
    if (t >= 2 * Q) return;
    const int q = t >> 1, sgn = t & 1;
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += part[((size_t)q * chunks + c) * 2 + sgn];
    norms[t] = s;
}

// r^(0) of the lanes of dense rows: entry (q, u) of sign part s goes to lane lane_of[2q + s] as
// |x| / ||x_s||_1 (each (lane, u) receives exactly one value, so the seed is order-free).
template <typename T>
__global__ void k_seed_dense_rows(KArgs A, const T *X, int64_t ldx, int Q, const int32_t *lane_of, const double *norms)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) A.ctrl->scan_mode = 1u;  // dense seeds: two-pass compaction
    const int64_t n = A.g.n, total = (int64_t)Q * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(t / n);
        const int64_t u = t - (int64_t)q * n;
        const float x = load_x(X, (int64_t)q * ldx + u);
        if (!(x != 0.f) || !isfinite(x)) continue;
        const int part = x < 0.f ? 1 : 0;
        const int lane = lane_of[2 * q + part];
        if (lane < 0) continue;
        push_to(lane_res(A, lane, u), (float)((double)fabsf(x) / norms[2 * q + part]));
    }
}

__global__ void k_threshold(DevGraph g, LaneParam P, int64_t count, const int32_t *nodes, const float *c,
                            int32_t *k_out)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = nodes[t];
        int k = 0;
        if (u >= 0 && u < g.n) {
            const int d = (int)(g.rowptr[u + 1] - g.rowptr[u]);  // row length
            if (d > 0 && c[t] > 0.f) k = det_prefix(c[t], P, g.colidx + g.rowptr[u], d, g.deg);
        }
        k_out[t] = k;
    }
}

// ------------------------------------------------------------------------------------ host side
int exponent_mode(double p)
{
    if (p == 0.0) return 0;
    if (p == 1.0) return 1;
    if (p == 0.5) return 2;
    return 3;
}

// Parameters checked against the graph they run on: a directed graph with out-neighbour rows
// (AGP_DIRECTED) needs a = 0, because a node without out-edges would have d^-a undefined as a push
// target. With in-neighbour rows (AGP_DIRECTED_IN) every push target has an out-edge, and a source
// without out-edges pushes nothing when b > 0 (D^-b := 0), so any a, b is valid.
int validate_params_for(const agp_graph_s *g, const agp_params_t &p)
{
    AGP_TRY(validate_params(p));
    if (g->directed == 1 && p.a != 0.0) return fail(AGP_EINVAL, "params: a directed graph needs a = 0");
    return AGP_OK;
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
    // per (lane, node): R (4), the item's residue, c, k and segment length (16), and the lane's share
    // of the item id, flags and record counts (16, as if every lane were its own group); walk-chunk
    // records (8, with the extra records of long rows) and segment records (8, likewise)
    // (+ 4 for the c(u) block of pull levels)
    return n * (4 + 4 + 16 + 16) + (size_t)(n * 8 * (1.0 + avg / kChunk)) + (size_t)(n * 8 * (1.0 + avg / kMinSeg)) + 8192;
}

// Lanes a workspace can hold: the group index of an item has 32 - ubits bits, and the item lists
// are indexed with 32-bit record fields.
int lane_capacity(const agp_graph_s *g)
{
    const int by_bits = (g->ubits >= 31) ? 1 : (int)std::min<int64_t>(4096, 1ll << (32 - g->ubits));
    const int64_t by_items = g->n ? (int64_t)(4294967295ull / (uint64_t)g->n) : 4096;
    return (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)by_bits, by_items, 4096}));
}

void free_workspace(Workspace *ws)
{
    if (!ws) return;
    if (ws->graph) cudaGraphExecDestroy(ws->graph);
    if (ws->ev_ready)
        for (int l = 0; l < kMaxLevels; ++l)
            for (int k = 0; k < kProfKernels; ++k)
                for (int e = 0; e < 2; ++e) cudaEventDestroy(ws->ev[l][k][e]);
    cudaFree(ws->R);
    cudaFree(ws->items);
    cudaFree(ws->rval);
    cudaFree(ws->part);
    cudaFree(ws->c_item);
    cudaFree(ws->k_item);
    cudaFree(ws->seg_item);
    cudaFree(ws->flag_item);
    cudaFree(ws->nrec);
    cudaFree(ws->rpart);
    cudaFree(ws->det_rec);
    cudaFree(ws->smp_rec);
    cudaFree(ws->C);
    cudaFree(ws->lane_count);
    cudaFree(ws->pull);
    cudaFree(ws->lanes);
    cudaFree(ws->coef);
    cudaFree(ws->level);
    cudaFree(ws->stats);
    cudaFree(ws->ctrl);
    cudaFree(ws->stage);
    cudaFreeHost(ws->h_stage);
    cudaFree(ws->out_stage);
    cudaFreeHost(ws->h_ctrl);
    cudaFreeHost(ws->h_lanes);
    delete ws;
}

// Lanes in flight per wave. Every lane scatters atomics into its own residues; the automatic choice
// keeps the residue blocks of all lanes in flight within ~96 MB of the 129 MB L2, so that the
// random reductions are served by L2 rather than DRAM (measured: 16 lanes of 4M nodes ran slower
// than one lane at a time), rounded down to a multiple of 4 lanes (one full group) when it is 4 or
// more.
int wave_lanes(const agp_graph_s *g)
{
    if (g->wave_lanes > 0) return g->wave_lanes;
    const int64_t per_lane = 4 * std::max<int64_t>(g->n, 1);
    int64_t l = std::max<int64_t>(1, std::min<int64_t>(4096, (96ll << 20) / per_lane));
    if (l >= 4) l = l / 4 * 4;
    return (int)l;
}

// Lanes that fit the graph's memory budget (default: 60% of the free device memory, counting the
// memory already held by the graph's current work buffers).
int lanes_for_budget(agp_graph_s *g, int64_t held, int *lanes)
{
    int64_t budget = g->mem_budget;
    if (budget <= 0) {
        size_t fr = 0, tot = 0;
        AGP_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
        budget = (int64_t)((double)(fr + held) * 0.6);
    }
    *lanes = (int)std::min<int64_t>(lane_capacity(g), std::max<int64_t>(0, budget / (int64_t)bytes_per_lane(g)));
    if (*lanes < 1) return fail(AGP_EBUDGET, "memory budget too small for one propagation lane");
    return AGP_OK;
}

int create_workspace(agp_graph_s *g, int G, int W, Workspace **out, int grid)
{
    if (W != 1 && W != 2 && W != 4) return fail(AGP_EINTERNAL, "group width must be 1, 2 or 4");
    G = (G + W - 1) / W * W;
    Workspace *ws = new Workspace();
    ws->device = g->device;
    ws->G = G;
    ws->W = W;
    ws->n = g->n;
    const unsigned long long n = (unsigned long long)std::max<int64_t>(g->n, 1);
    const unsigned long long groups = (unsigned long long)(G / W), nnz = (unsigned long long)g->nnz;
    const int64_t node_unit = kScanUnit / W;  // nodes per scanned unit of a group block
    ws->ldR = ((int64_t)n + node_unit - 1) / node_unit * node_unit;
    // one item per (group, node); the one-pass compaction stages a block's items at its units'
    // node offsets, so the item storage covers every node slot of the blocks (ldR per group)
    ws->cap_items = groups * (unsigned long long)ws->ldR;
    // a row is walked at most once per group and level: ceil(d_u / kChunk) <= 1 + d_u / kChunk chunks
    ws->cap_det = ws->cap_items + groups * nnz / kChunk + 1;
    // segments of a lane's tail: at most 1 + d_u / kMinSeg per (lane, node)
    ws->cap_smp = (unsigned long long)G * n + (unsigned long long)G * nnz / kMinSeg + 1;
    size_t acc = 0;
    int rc = AGP_OK;
    auto A = [&](int r) { if (rc == AGP_OK) rc = r; };
    const int64_t units = (int64_t)groups * (ws->ldR * W / kScanUnit);
    ws->grid = grid > 0 ? grid : grid_stride_blocks();
    // compaction ranges: one resident CTA each (kCompactBlocks per SM), at most the workspace's grid
    ws->part_blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>({(int64_t)ws->grid, (int64_t)kCompactBlocks * sm_count(), units}));
    A(dev_alloc(&ws->R, (size_t)G * ws->ldR, acc));
    A(dev_alloc(&ws->items, ws->cap_items, acc));
    A(dev_alloc(&ws->rval, ws->cap_items * W, acc));
    A(dev_alloc(&ws->part, (size_t)ws->part_blocks + 1, acc));
    A(dev_alloc(&ws->c_item, ws->cap_items * W, acc));
    A(dev_alloc(&ws->k_item, ws->cap_items * W, acc));
    A(dev_alloc(&ws->seg_item, ws->cap_items * W, acc));
    A(dev_alloc(&ws->flag_item, ws->cap_items, acc));
    A(dev_alloc(&ws->nrec, ws->cap_items, acc));
    A(dev_alloc(&ws->rpart, (size_t)2 * ws->grid, acc));
    A(dev_alloc(&ws->det_rec, ws->cap_det, acc));
    A(dev_alloc(&ws->smp_rec, ws->cap_smp, acc));
    // pull levels (undirected graphs, when enabled): c(u) block beside R, per-lane frontier counts
    // and modes
    if (!g->directed && g->pull_shift >= 0) {
        A(dev_alloc(&ws->C, (size_t)G * ws->ldR, acc));
        A(dev_alloc(&ws->lane_count, (size_t)G, acc));
        A(dev_alloc(&ws->pull, (size_t)2 * G, acc));
        if (rc == AGP_OK) rc = ensure_row_lists(g, 0);
    }
    A(dev_alloc(&ws->lanes, (size_t)G, acc));
    A(dev_alloc(&ws->coef, (size_t)G * kMaxLevels, acc));
    A(dev_alloc(&ws->level, (size_t)G, acc));
    A(dev_alloc(&ws->stats, (size_t)G, acc));
    A(dev_alloc(&ws->ctrl, 1, acc));
    if (rc == AGP_OK && cudaMallocHost((void **)&ws->h_ctrl, sizeof(Ctrl)) != cudaSuccess) rc = fail(AGP_ENOMEM, "cudaMallocHost");
    if (rc == AGP_OK && cudaMallocHost((void **)&ws->h_lanes, sizeof(LaneParam) * G) != cudaSuccess) rc = fail(AGP_ENOMEM, "cudaMallocHost");
    if (rc == AGP_OK) {
        cudaError_t e = cudaMemset(ws->R, 0, sizeof(float) * (size_t)G * ws->ldR);
        if (e == cudaSuccess && ws->C) e = cudaMemset(ws->C, 0, sizeof(float) * (size_t)G * ws->ldR);
        if (e == cudaSuccess && ws->lane_count) e = cudaMemset(ws->lane_count, 0, sizeof(unsigned long long) * G);
        if (e == cudaSuccess && ws->pull) e = cudaMemset(ws->pull, 0, sizeof(int32_t) * 2 * G);
        if (e == cudaSuccess) e = cudaMemset(ws->level, 0xff, sizeof(int32_t) * G);
        if (e == cudaSuccess) e = cudaMemset(ws->ctrl, 0, sizeof(Ctrl));
        if (e == cudaSuccess) e = cudaMemset(ws->stats, 0, sizeof(LaneStats) * G);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) rc = fail(AGP_ECUDA, std::string("workspace init: ") + cudaGetErrorString(e));
    }
    if (rc != AGP_OK) {
        free_workspace(ws);
        return rc;
    }
    ws->bytes = acc;
    *out = ws;
    return AGP_OK;
}

// A wave that failed part-way may leave residues or frontier bits behind; its buffers are freed
// so that the next call starts from freshly zeroed ones.
void drop_workspace(agp_graph_s *g)
{
    cudaDeviceSynchronize();
    cudaGetLastError();
    free_workspace(g->ws);
    free_workspace(g->ws2);
    free_workspace(g->ws_plain);
    g->ws = nullptr;
    g->ws2 = nullptr;
    g->ws_plain = nullptr;
}

// The graph's work buffers for waves of `lanes_wanted` lanes: the batched workspace (group width
// from the wave width), or for the plain path a one-lane workspace of its own (group width 1, so
// the baseline scans one lane's residues, not a group's).
int ensure_workspace(agp_graph_s *g, int lanes_wanted, bool plain, Workspace **out)
{
    if (plain) {
        if (!g->ws_plain) AGP_TRY(create_workspace(g, 1, 1, &g->ws_plain));
        *out = g->ws_plain;
        return AGP_OK;
    }
    int by_budget = 0;
    AGP_TRY(lanes_for_budget(g, g->ws ? (int64_t)g->ws->bytes : 0, &by_budget));
    int G = std::max(1, std::min(lanes_wanted, by_budget));
    int W;
    if (g->group_width > 0) {  // the graph's setting: whole groups of that width
        W = std::min(g->group_width, std::max(1, by_budget));
        while (W > 1 && W > G) W /= 2;
        G = (G + W - 1) / W * W;
    } else {
        if (G >= 3) {  // whole groups of four lanes: round up when the budget allows, else down
            const int up = (G + 3) / 4 * 4;
            G = (up <= by_budget) ? up : std::max(G / 4 * 4, std::min(G, 2));
        }
        W = group_width(G);
    }
    if (g->ws && g->ws->G >= G && g->ws->W == W) {
        *out = g->ws;
        return AGP_OK;
    }
    if (g->ws) {
        AGP_CUDA_TRY(cudaDeviceSynchronize());
        free_workspace(g->ws);
        g->ws = nullptr;
        free_workspace(g->ws2);
        g->ws2 = nullptr;
    }
    AGP_TRY(create_workspace(g, G, W, &g->ws));
    *out = g->ws;
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

int grow_pinned(void **p, size_t *have, size_t need)
{
    if (*have >= need) return AGP_OK;
    cudaFreeHost(*p);
    *p = nullptr;
    *have = 0;
    need = std::max<size_t>(need, 4096);
    if (cudaMallocHost(p, need) != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(AGP_ENOMEM, "pinned staging buffer");
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
    A.W = ws->W;
    A.R = ws->R;
    A.items = ws->items;
    A.rval = ws->rval;
    A.ldR = ws->ldR;
    A.units = ws->ldR * ws->W / kScanUnit;
    A.part = ws->part;
    A.part_blocks = ws->part_blocks;
    A.c_item = ws->c_item;
    A.k_item = ws->k_item;
    A.seg_item = ws->seg_item;
    A.flag_item = ws->flag_item;
    A.nrec = ws->nrec;
    A.rpart = ws->rpart;
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
    A.grid = ws->grid;
    A.rows_in = g->directed == 2 ? 1 : 0;
    A.groups = 0;
    // pull levels off (the default): no frontier volumes, pull decisions or pull launches at all
    const bool pull_on = ws->C && g->pull_shift >= 0 && g->pull_shift < 63;
    A.C = pull_on ? ws->C : nullptr;
    A.lane_count = pull_on ? ws->lane_count : nullptr;
    A.pull = pull_on ? ws->pull : nullptr;
    A.pull_min = pull_on ? std::max<int64_t>(1, g->nnz >> g->pull_shift) : std::numeric_limits<int64_t>::max();
    for (int c = 0; c < 3; ++c) {
        A.rows[c] = g->row_list[c];
        A.row_count[c] = g->row_count[c];
    }
    A.ctrl = ws->ctrl;
    return A;
}

int ensure_events(Workspace *ws)
{
    if (ws->ev_ready) return AGP_OK;
    for (int l = 0; l < kMaxLevels; ++l)
        for (int k = 0; k < kProfKernels; ++k)
            for (int e = 0; e < 2; ++e) AGP_CUDA_TRY(cudaEventCreate(&ws->ev[l][k][e]));
    ws->ev_ready = true;
    return AGP_OK;
}

// Frontier compaction: residue blocks of the groups -> ascending item list, size in ctrl->n_items.
template <int W> void launch_compact_w(const KArgs &A, cudaStream_t s)
{
    k_compact_count<W><<<A.part_blocks, kBlock, 0, s>>>(A);
    k_compact_scan<<<1, 1024, 0, s>>>(A);
    k_compact_emit<W><<<A.part_blocks, kBlock, 0, s>>>(A);
}

// Expansion and its record lists (sizes in ctrl->n_det, n_smp). k_expand and k_rec_emit must run on
// the same grid: they walk the same item ranges.
template <int W> void launch_expand_w(const KArgs &A, cudaStream_t s)
{
    k_expand<W><<<A.grid, kBlock, 0, s>>>(A);
    k_rec_scan<<<1, 1024, 0, s>>>(A, A.grid);
    k_rec_emit<<<A.grid, kBlock, 0, s>>>(A);
}

template <int W> void launch_push_w(const KArgs &A, cudaStream_t s, int blocks) { k_push<W><<<blocks, kBlock, 0, s>>>(A); }
template <int W> void launch_sample_w(const KArgs &A, cudaStream_t s, int blocks)
{
    if (A.groups) k_sample<W, true><<<blocks, kBlock, 0, s>>>(A);
    else k_sample<W, false><<<blocks, kBlock, 0, s>>>(A);
}
template <int W> void launch_pull_w(const KArgs &A, cudaStream_t s)
{
    k_pull<W, 0><<<A.grid, kBlock, 0, s>>>(A);
    k_pull<W, 1><<<A.grid, kBlock, 0, s>>>(A);
    k_pull<W, 2><<<(int)std::max<int64_t>(1, std::min<int64_t>(A.row_count[2], A.grid)), kBlock, 0, s>>>(A);
}

#define AGP_BY_WIDTH(fn, ...)                         \
    do {                                              \
        if (A.W == 4) fn<4>(__VA_ARGS__);             \
        else if (A.W == 2) fn<2>(__VA_ARGS__);        \
        else fn<1>(__VA_ARGS__);                      \
    } while (0)

void launch_compact(const KArgs &A, cudaStream_t s) { AGP_BY_WIDTH(launch_compact_w, A, s); }
void launch_expand(const KArgs &A, cudaStream_t s) { AGP_BY_WIDTH(launch_expand_w, A, s); }
void launch_push(const KArgs &A, cudaStream_t s, int blocks) { AGP_BY_WIDTH(launch_push_w, A, s, blocks); }
void launch_sample(const KArgs &A, cudaStream_t s, int blocks) { AGP_BY_WIDTH(launch_sample_w, A, s, blocks); }
void launch_pull(const KArgs &A, cudaStream_t s)
{
    if (A.C) AGP_BY_WIDTH(launch_pull_w, A, s);
}

// One level: compact, expand, push, sample, level end. With `ev` (profiling) every step is
// bracketed by event records on the same stream.
void launch_level(const KArgs &A, cudaStream_t s, int expand_blocks, int push_blocks, int sample_blocks,
                  cudaEvent_t (*ev)[2])
{
    (void)expand_blocks;
    // External records become event nodes when captured into a graph (plain records during
    // capture only express dependencies and never fire).
    auto rec = [&](cudaEvent_t e) { cudaEventRecordWithFlags(e, s, cudaEventRecordExternal); };
    if (ev) rec(ev[0][0]);
    launch_compact(A, s);
    if (ev) { rec(ev[0][1]); rec(ev[1][0]); }
    launch_expand(A, s);
    if (ev) { rec(ev[1][1]); rec(ev[2][0]); }
    launch_push(A, s, push_blocks);
    if (ev) { rec(ev[2][1]); rec(ev[3][0]); }
    launch_sample(A, s, sample_blocks);
    launch_pull(A, s);
    if (ev) { rec(ev[3][1]); rec(ev[4][0]); }
    k_level_end<<<1, kBlock, 0, s>>>(A);
    if (ev) rec(ev[4][1]);
}

int blocks_for(unsigned long long work, int per_block)
{
    const unsigned long long b = (work + per_block - 1) / per_block;
    return (int)std::max<unsigned long long>(1, std::min<unsigned long long>(b, (unsigned long long)grid_stride_blocks() * 4));
}

// Accumulate the profiled kernel times of levels [0, levels) (the stream has been synchronised).
void read_profile(agp_graph_s *g, Workspace *ws, int levels, const bool *ran)
{
    for (int l = 0; l < levels; ++l)
        for (int k = 0; k < kProfKernels; ++k) {
            if (ran && !ran[l * kProfKernels + k]) continue;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ws->ev[l][k][0], ws->ev[l][k][1]) == cudaSuccess) {
                g->prof_ms[k] += ms;
                g->prof_launches[k] += 1;
            } else {
                cudaGetLastError();
            }
        }
}

// Capture `levels` consecutive levels (expand, push, sample, level end) into an executable graph.
int capture_levels_ev(const KArgs &A, int levels, Workspace *ws_events, cudaGraphExec_t *out)
{
    cudaStream_t cs;
    AGP_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int lvl = 0; lvl < levels; ++lvl)
            launch_level(A, cs, A.grid, A.grid, A.grid,
                         ws_events ? ws_events->ev[lvl] : nullptr);
        e = cudaStreamEndCapture(cs, &graph);
    }
    if (e == cudaSuccess) {
        e = cudaGraphInstantiate(out, graph, 0);
        cudaGraphDestroy(graph);
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        *out = nullptr;
        return fail(AGP_ECUDA, std::string("capturing the level loop: ") + cudaGetErrorString(e));
    }
    return AGP_OK;
}

int capture_levels(const KArgs &A, int levels, cudaGraphExec_t *out) { return capture_levels_ev(A, levels, nullptr, out); }

void launch_seed_sources(const KArgs &A, const int32_t *lanes, const int32_t *sources, int count, cudaStream_t s)
{
    if (count > 0) k_seed_sources<<<blocks_for((unsigned long long)count, kBlock), kBlock, 0, s>>>(A, lanes, sources, count);
}

void launch_colnorms_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ldx, double *norms, cudaStream_t s)
{
    if (n <= 0 || d <= 0) return;
    const int grid = grid_stride_blocks();
    const int64_t rows_per_block = std::max<int64_t>(64, (n + grid - 1) / grid);
    k_colnorms_bf16<<<(int)((n + rows_per_block - 1) / rows_per_block), kBlock, 0, s>>>(X, n, d, ldx, rows_per_block, norms);
}

void launch_seed_dense_bf16(const KArgs &A, const uint16_t *X, int64_t ldx, const int32_t *lane_of,
                            const int32_t *col_of, const int32_t *part_of, const double *norms, int nl, cudaStream_t s)
{
    if (nl > 0) k_seed_dense_bf16<<<A.grid, kBlock, 0, s>>>(A, X, ldx, lane_of, col_of, part_of, norms, nl);
}

// Run the levels of the current wave (lanes already seeded, level 0 frontier in items[cur]).
int run_levels(agp_graph_s *g, Workspace *ws, const KArgs &A, int max_L, bool plain, bool profile, cudaStream_t s)
{
    ws->prof_levels = 0;
    if (profile) AGP_TRY(ensure_events(ws));
    if (plain) {
        bool ran[kMaxLevels * kProfKernels] = {};
        int levels = 0;
        for (int lvl = 0; lvl <= max_L; ++lvl) {
            auto rec = [&](int k, int e) { if (profile) cudaEventRecord(ws->ev[lvl][k][e], s); };
            rec(0, 0);
            launch_compact(A, s);
            rec(0, 1);
            ran[lvl * kProfKernels + 0] = true;
            levels = lvl + 1;
            AGP_CUDA_TRY(cudaMemcpyAsync(ws->h_ctrl, ws->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
            AGP_CUDA_TRY(cudaStreamSynchronize(s));
            __atomic_fetch_add(&g->kernel_launches, (int64_t)(3), __ATOMIC_RELAXED);
            const unsigned long long items = std::min(ws->h_ctrl->n_items, ws->cap_items);
            if (items == 0) break;
            rec(1, 0);
            launch_expand(A, s);
            rec(1, 1);
            ran[lvl * kProfKernels + 1] = true;
            AGP_CUDA_TRY(cudaMemcpyAsync(ws->h_ctrl, ws->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
            AGP_CUDA_TRY(cudaStreamSynchronize(s));
            const unsigned long long nd = std::min(ws->h_ctrl->n_det, ws->cap_det),
                                     ns = std::min(ws->h_ctrl->n_smp, ws->cap_smp);
            __atomic_fetch_add(&g->kernel_launches, (int64_t)(4 + (nd ? 1 : 0) + (ns ? 1 : 0)), __ATOMIC_RELAXED);
            if (nd) { rec(2, 0); launch_push(A, s, blocks_for(nd, kBlock / 32)); rec(2, 1); ran[lvl * kProfKernels + 2] = true; }
            if (ns) { rec(3, 0); launch_sample(A, s, blocks_for(ns, kBlock)); rec(3, 1); ran[lvl * kProfKernels + 3] = true; }
            launch_pull(A, s);
            if (A.C) __atomic_fetch_add(&g->kernel_launches, (int64_t)3, __ATOMIC_RELAXED);
            rec(4, 0);
            k_level_end<<<1, kBlock, 0, s>>>(A);
            rec(4, 1);
            ran[lvl * kProfKernels + 4] = true;
            AGP_CUDA_TRY(cudaGetLastError());
        }
        if (profile) {
            AGP_CUDA_TRY(cudaStreamSynchronize(s));
            read_profile(g, ws, levels, ran);
        }
        return AGP_OK;
    }
    const int64_t pull_key = A.C ? A.pull_min : -1;
    if (!ws->graph || ws->graph_levels != max_L || ws->graph_collect != A.collect || ws->graph_profile != (int)profile ||
        ws->graph_groups != A.groups || ws->graph_pull != pull_key) {
        if (ws->graph) {
            cudaGraphExecDestroy(ws->graph);
            ws->graph = nullptr;
        }
        AGP_TRY(capture_levels_ev(A, max_L + 1, profile ? ws : nullptr, &ws->graph));
        ws->graph_levels = max_L;
        ws->graph_collect = A.collect;
        ws->graph_profile = (int)profile;
        ws->graph_groups = A.groups;
        ws->graph_pull = pull_key;
    }
    AGP_CUDA_TRY(cudaGraphLaunch(ws->graph, s));
    __atomic_fetch_add(&g->kernel_launches, (int64_t)((kKernelsPerLevel + (A.C ? 3 : 0)) * (max_L + 1)), __ATOMIC_RELAXED);
    ws->prof_levels = profile ? max_L + 1 : 0;  // read when the wave is checked
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

// Lane parameters, coefficients and levels of a wave, plus `aux` (int32 seed map of the caller),
// uploaded from the workspace's pinned staging on stream s. The workspace must be idle (its
// previous wave checked), which is what makes reusing the pinned staging safe without a sync.
int prepare_wave(agp_graph_s *g, Workspace *ws, const std::vector<LaneSpec> &lanes, size_t first, int count,
                 const agp_params_t *params, uint64_t stream_base_is_query, bool eps_absolute, bool sampler_groups, float *out, int64_t su,
                 int64_t sr, const std::vector<int32_t> &aux, int32_t **d_aux, cudaStream_t s, int *max_L)
{
    *max_L = 0;
    size_t nw = 0;
    for (int l = 0; l < count; ++l) {
        const agp_params_t &p = params[lanes[first + l].params];
        if (p.kind == AGP_W_FINITE) nw += (size_t)p.L + 1;
    }
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t lp_b = sizeof(LaneParam) * count, cs_b = sizeof(CoefSpec) * count, w_b = sizeof(double) * std::max<size_t>(nw, 1),
                 lv_b = sizeof(int32_t) * ws->G, aux_b = sizeof(int32_t) * std::max<size_t>(aux.size(), 1);
    const size_t total = al(lp_b) + al(cs_b) + al(w_b) + al(lv_b) + al(aux_b);
    AGP_TRY(grow(&ws->stage, &ws->stage_bytes, total));
    AGP_TRY(grow_pinned(&ws->h_stage, &ws->h_stage_bytes, total));
    char *h = (char *)ws->h_stage;
    LaneParam *h_lp = (LaneParam *)h;
    CoefSpec *h_cs = (CoefSpec *)(h + al(lp_b));
    double *h_w = (double *)(h + al(lp_b) + al(cs_b));
    int32_t *h_lv = (int32_t *)(h + al(lp_b) + al(cs_b) + al(w_b));
    int32_t *h_aux = (int32_t *)(h + al(lp_b) + al(cs_b) + al(w_b) + al(lv_b));
    size_t w_used = 0;
    for (int l = 0; l < count; ++l) {
        const LaneSpec &ls = lanes[first + l];
        const agp_params_t &p = params[ls.params];
        LaneParam &P = h_lp[l];
        P.eps_d = eps_absolute ? lane_eps_absolute(p.eps, ls.norm) : p.eps;
        P.eps = (float)P.eps_d;
        P.a = (float)p.a;
        P.b = (float)p.b;
        P.a_d = p.a;
        P.a_mode = exponent_mode(p.a);
        P.b_mode = exponent_mode(p.b);
        P.L = p.L;
        P.out_row = ls.query;
        P.sampler = sampler_groups ? 1 : 0;
        P.out = out + (int64_t)ls.query * sr;
        P.su = su;
        lane_param_derive(P);
        lane_key(p.seed, stream_base_is_query ? (uint64_t)ls.query : 0ull, ls.part, P.key0, P.key1);
        CoefSpec &c = h_cs[l];
        c = CoefSpec{};
        c.lane = l;
        c.kind = p.kind;
        c.L = p.L;
        c.param = p.param;
        c.scale = (ls.part ? -1.0 : 1.0) * ls.norm;
        c.w_off = 0;
        if (p.kind == AGP_W_FINITE) {
            c.w_off = (int32_t)w_used;
            for (int i = 0; i <= p.L; ++i) h_w[w_used++] = p.w[i];
        }
        *max_L = std::max(*max_L, p.L);
    }
    for (int l = 0; l < ws->G; ++l) h_lv[l] = l < count ? 0 : -1;  // wave lanes start at level 0
    std::copy(aux.begin(), aux.end(), h_aux);
    char *d = (char *)ws->stage;
    AGP_CUDA_TRY(cudaMemcpyAsync(d, h, total, cudaMemcpyHostToDevice, s));
    AGP_CUDA_TRY(cudaMemcpyAsync(ws->lanes, d, lp_b, cudaMemcpyDeviceToDevice, s));
    launch_coef((const CoefSpec *)(d + al(lp_b)), (const double *)(d + al(lp_b) + al(cs_b)), ws->coef, count, s);
    AGP_CUDA_TRY(cudaMemcpyAsync(ws->level, d + al(lp_b) + al(cs_b) + al(w_b), lv_b, cudaMemcpyDeviceToDevice, s));
    AGP_CUDA_TRY(cudaMemsetAsync(ws->stats, 0, sizeof(LaneStats) * ws->G, s));
    *d_aux = (int32_t *)(d + al(lp_b) + al(cs_b) + al(w_b) + al(lv_b));
    return AGP_OK;
}

int reset_ctrl(Workspace *ws, int lanes_used, cudaStream_t s)
{
    Ctrl *h = ws->h_ctrl;  // pinned; the workspace's previous wave has been checked
    std::memset(h, 0, sizeof(Ctrl));
    h->lanes_used = (unsigned int)lanes_used;
    AGP_CUDA_TRY(cudaMemcpyAsync(ws->ctrl, h, sizeof(Ctrl), cudaMemcpyHostToDevice, s));
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

// ------------------------------------------------------------------------------------ wave pipeline
// What a call does per wave besides the common steps: its seed map (uploaded with the wave's
// parameters) and its seed kernel.
struct WaveJob {
    float *out;
    int64_t su, sr;
    uint64_t stream_base_is_query;
    bool eps_absolute = false;  // eps in raw signal units: a lane uses eps / ||x+-||_1
    bool sampler_groups = false;  // AGP_SAMPLER_GROUPS
    std::function<void(size_t first, int count, std::vector<int32_t> &aux)> make_aux;
    std::function<int(const KArgs &A, int count, const int32_t *d_aux, cudaStream_t st)> seed;
    // optional: called on the wave's stream after its levels, once every earlier wave is complete
    // on that stream too (result rows that are final can be copied out while later waves compute)
    std::function<int(size_t first, int count, cudaStream_t st)> after_wave;
    // optional (AGP_QUERY_TIMES): done_ms[lanes[i].query] = device time from the first wave's start to
    // the end of the wave that ran lane i, largest over the query's lanes
    agp_stats_t *times = nullptr;
};

// Runs the waves (G lanes each) of a call. Unless the call is on the plain path or on a fixed
// workspace, two waves are in flight: wave w uses workspace w % 2 on stream w % 2 (the caller's
// stream and a side stream forked from it), so the latency-bound expansion of one wave overlaps
// the L2-bound pushes of the other. A workspace's wave is checked (errors, profile, statistics)
// only when the workspace is needed again or at the end.
int run_waves(agp_graph_s *g, ExecCtx *ctx, Workspace *ws0, const std::vector<LaneSpec> &lanes,
              const agp_params_t *params, int G, bool plain, bool profile, int collect, agp_stats_t *stats,
              cudaStream_t s, const WaveJob &job)
{
    const bool two = !plain && !ctx->ws && lanes.size() > (size_t)G;
    Workspace *wss[2] = {ws0, nullptr};
    cudaStream_t ss[2] = {s, nullptr};
    if (two) {
        if (g->ws2 && (g->ws2->G < ws0->G || g->ws2->W != ws0->W)) {
            AGP_CUDA_TRY(cudaDeviceSynchronize());
            free_workspace(g->ws2);
            g->ws2 = nullptr;
        }
        if (!g->ws2) AGP_TRY(create_workspace(g, ws0->G, ws0->W, &g->ws2));
        if (!g->side) {
            AGP_CUDA_TRY(cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking));
            AGP_CUDA_TRY(cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming));
            AGP_CUDA_TRY(cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming));
        }
        wss[1] = g->ws2;
        ss[1] = g->side;
        AGP_CUDA_TRY(cudaEventRecord(g->ev_fork, s));
        AGP_CUDA_TRY(cudaStreamWaitEvent(g->side, g->ev_fork, 0));
    }
    size_t wfirst[2] = {0, 0};
    int wcount[2] = {0, 0};
    // AGP_QUERY_TIMES: event 0 at the start, event 1 + w at the end of wave w
    const size_t n_waves = (lanes.size() + G - 1) / G;
    if (job.times) {
        while (g->wave_ev.size() < n_waves + 1) {
            cudaEvent_t e;
            AGP_CUDA_TRY(cudaEventCreate(&e));
            g->wave_ev.push_back(e);
        }
        AGP_CUDA_TRY(cudaEventRecord(g->wave_ev[0], s));
        if (two) AGP_CUDA_TRY(cudaStreamWaitEvent(g->side, g->wave_ev[0], 0));
    }
    auto finish = [&](int k) -> int {
        Workspace *W = wss[k];
        if (!W || !W->pending) return AGP_OK;
        W->pending = false;
        int rc = check_ctrl(W, ss[k]);
        if (rc == AGP_OK && W->prof_levels > 0) {
            read_profile(g, W, W->prof_levels, nullptr);
            W->prof_levels = 0;
        }
        if (rc == AGP_OK && collect) rc = collect_stats(W, lanes, wfirst[k], wcount[k], stats, ss[k]);
        return rc;
    };
    int rc = AGP_OK;
    size_t first = 0;
    for (int w = 0; first < lanes.size(); first += G, ++w) {
        const int k = two ? (w & 1) : 0;
        Workspace *W = wss[k];
        const cudaStream_t st = ss[k];
        if ((rc = finish(k)) != AGP_OK) break;
        const int count = (int)std::min<size_t>(G, lanes.size() - first);
        std::vector<int32_t> aux;
        job.make_aux(first, count, aux);
        int32_t *d_aux = nullptr;
        int max_L = 0;
        if ((rc = prepare_wave(g, W, lanes, first, count, params, job.stream_base_is_query, job.eps_absolute,
                               job.sampler_groups, job.out,
                               job.su, job.sr, aux, &d_aux, st, &max_L)) != AGP_OK)
            break;
        if ((rc = reset_ctrl(W, count, st)) != AGP_OK) break;
        KArgs A = make_args(g, W, collect);
        A.groups = job.sampler_groups ? 1 : 0;
        if ((rc = job.seed(A, count, d_aux, st)) != AGP_OK) break;
        __atomic_fetch_add(&g->kernel_launches, (int64_t)2, __ATOMIC_RELAXED);  // coefficients + seed
        if ((rc = run_levels(g, W, A, max_L, plain, profile, st)) != AGP_OK) break;
        if (job.after_wave) {
            if (!g->ev_wave[k]) AGP_CUDA_TRY(cudaEventCreateWithFlags(&g->ev_wave[k], cudaEventDisableTiming));
            if (two && w > 0) AGP_CUDA_TRY(cudaStreamWaitEvent(st, g->ev_wave[k ^ 1], 0));
            if ((rc = job.after_wave(first, count, st)) != AGP_OK) break;
            AGP_CUDA_TRY(cudaEventRecord(g->ev_wave[k], st));
        }
        if (job.times) AGP_CUDA_TRY(cudaEventRecord(g->wave_ev[1 + w], st));
        W->pending = true;
        wfirst[k] = first;
        wcount[k] = count;
    }
    for (int k = 0; k < 2; ++k) {
        const int r2 = finish(k);
        if (rc == AGP_OK) rc = r2;
    }
    if (two) {
        cudaEventRecord(g->ev_join, g->side);
        cudaStreamWaitEvent(s, g->ev_join, 0);
    }
    if (rc == AGP_OK && job.times && n_waves > 0) {
        if (cudaStreamSynchronize(s) != cudaSuccess) rc = fail(AGP_ECUDA, "waiting for the waves");
        for (size_t w = 0; rc == AGP_OK && w < n_waves; ++w) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, g->wave_ev[0], g->wave_ev[1 + w]) != cudaSuccess) {
                rc = fail(AGP_ECUDA, "reading the wave events");
                break;
            }
            const size_t end = std::min(lanes.size(), (w + 1) * (size_t)G);
            for (size_t i = w * (size_t)G; i < end; ++i) {
                float &d = job.times[lanes[i].query].done_ms;
                d = std::max(d, ms);
            }
        }
    }
    if (rc != AGP_OK) {
        if (!ctx->ws) drop_workspace(g);
        else wss[0]->pending = false;
    }
    return rc;
}

// ------------------------------------------------------------------------------------ queries
int query_batch(agp_graph_s *g, const agp_params_t *params, int32_t n_params, int32_t Q,
                const int64_t *x_off, const int32_t *x_idx, const float *x_val, float *pi_out,
                int64_t ld_out, uint32_t flags, agp_stats_t *stats, cudaStream_t s)
{
    if (!g) return fail(AGP_EINVAL, "graph is NULL");
    ExecCtx ctx{nullptr, &g->in_stage, &g->in_bytes};
    return query_batch_ctx(g, &ctx, params, n_params, Q, x_off, x_idx, x_val, pi_out, ld_out, flags, stats, s);
}

int query_batch_ctx(agp_graph_s *g, ExecCtx *ctx, const agp_params_t *params, int32_t n_params, int32_t Q,
                    const int64_t *x_off, const int32_t *x_idx, const float *x_val, float *pi_out,
                    int64_t ld_out, uint32_t flags, agp_stats_t *stats, cudaStream_t s)
{
    if (!g) return fail(AGP_EINVAL, "graph is NULL");
    if (Q < 0) return fail(AGP_EINVAL, "Q < 0");
    if (Q == 0) return AGP_OK;
    if (!params || !(n_params == 1 || n_params == Q)) return fail(AGP_EINVAL, "n_params must be 1 or Q");
    if (!x_off || !pi_out) return fail(AGP_EINVAL, "x_off / pi_out NULL");
    if (ld_out < g->n) return fail(AGP_EINVAL, "ld_out < n");
    if (flags & ~(AGP_INPUT_ON_DEVICE | AGP_OUTPUT_ON_DEVICE | AGP_PLAIN | AGP_COLLECT_STATS | AGP_PROFILE |
                  AGP_QUERY_TIMES | AGP_EPS_ABSOLUTE | AGP_SAMPLER_GROUPS | kOffsetsOnHost))
        return fail(AGP_EINVAL, "unknown flag");
    // offsets on the device only when the inputs are and the caller did not pass them from the host
    const bool off_dev = (flags & AGP_INPUT_ON_DEVICE) && !(flags & kOffsetsOnHost);
    if ((flags & (AGP_COLLECT_STATS | AGP_QUERY_TIMES)) && !stats)
        return fail(AGP_EINVAL, "AGP_COLLECT_STATS / AGP_QUERY_TIMES need stats");
    for (int i = 0; i < n_params; ++i) AGP_TRY(validate_params_for(g, params[i]));
    AGP_CUDA_TRY(cudaSetDevice(g->device));
    const int64_t n = g->n;

    // --- inputs on the device
    int64_t total = 0;
    if (off_dev) {
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
    AGP_TRY(grow(ctx->stage, ctx->stage_bytes, need));
    char *p = (char *)*ctx->stage;
    int64_t *d_off = (int64_t *)p; p += al(off_b);
    int32_t *d_idx = (int32_t *)p; p += al(idx_b);
    float *d_val = x_val ? (float *)p : nullptr; p += al(val_b);
    double *d_norm = (double *)p; p += al(norm_b);
    p += al(map_b);
    unsigned int *d_bad = (unsigned int *)p;
    const int64_t *off_src = x_off;
    const int32_t *idx_src = x_idx;
    const float *val_src = x_val;
    if (flags & AGP_INPUT_ON_DEVICE) {
        off_src = x_off; idx_src = x_idx; val_src = x_val;
        if (!off_dev) {
            AGP_CUDA_TRY(cudaMemcpyAsync(d_off, x_off, off_b, cudaMemcpyHostToDevice, s));
            off_src = d_off;
        }
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
        __atomic_fetch_add(&g->kernel_launches, (int64_t)(1), __ATOMIC_RELAXED);
    }
    AGP_CUDA_TRY(cudaGetLastError());
    std::vector<double> norms(2 * Q);
    unsigned int bad = 0;
    AGP_CUDA_TRY(cudaMemcpyAsync(norms.data(), d_norm, norm_b, cudaMemcpyDeviceToHost, s));
    AGP_CUDA_TRY(cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, s));
    AGP_CUDA_TRY(cudaStreamSynchronize(s));
    if (bad) return fail(AGP_EINVAL, "signal index outside [0, n) or non-finite value");

    auto seed = [&](const KArgs &A, const int32_t *d_aux, cudaStream_t st) -> int {
        k_seed_sparse<<<blocks_for((unsigned long long)total, kBlock), kBlock, 0, st>>>(A, off_src, idx_src, val_src, Q,
                                                                                       d_aux, d_norm);
        AGP_CUDA_TRY(cudaGetLastError());
        return AGP_OK;
    };
    return run_queries(g, ctx, params, n_params, Q, norms, seed, pi_out, ld_out, flags, stats, s);
}

// The lanes of Q queries whose sign-part norms are known (norms[2q + part], host): one lane per
// non-empty part, waves of lanes, output rows zeroed first and, for host output, copied back as their
// queries finish. `seed` adds the normalised signal parts of a wave's lanes to their residue vectors
// (d_aux: lane of part (q, s) at 2q + s, or -1).
int run_queries(agp_graph_s *g, ExecCtx *ctx, const agp_params_t *params, int32_t n_params, int32_t Q,
                const std::vector<double> &norms,
                const std::function<int(const KArgs &A, const int32_t *d_aux, cudaStream_t st)> &seed,
                float *pi_out, int64_t ld_out, uint32_t flags, agp_stats_t *stats, cudaStream_t s)
{
    const bool plain = flags & AGP_PLAIN;
    const bool profile = flags & AGP_PROFILE;
    const int collect = (flags & AGP_COLLECT_STATS) ? 1 : 0;
    const int64_t n = g->n;
    // --- lanes: one per non-empty sign part
    std::vector<LaneSpec> lanes;
    for (int q = 0; q < Q; ++q)
        for (int part = 0; part < 2; ++part)
            if (norms[2 * q + part] > 0.0) lanes.push_back(LaneSpec{q, part, norms[2 * q + part], n_params == 1 ? 0 : q});
    Workspace *ws = ctx->ws;
    if (!ws) AGP_TRY(ensure_workspace(g, (int)std::min<size_t>(std::max<size_t>(1, lanes.size()), (size_t)wave_lanes(g)), plain, &ws));

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
    const int G = plain ? 1 : std::min(ws->G, ctx->ws ? ws->G : wave_lanes(g));
    WaveJob job;
    job.out = out;
    job.su = 1;
    job.sr = ld;
    // n_params == Q: a query's random stream depends on its own seed, not on its position, so it draws
    // the same numbers in any batch; n_params == 1: the queries share one seed, and query q draws
    // from the stream (seed, q), so that they do not repeat one another's draws on common nodes
    job.stream_base_is_query = (n_params == 1) ? 1 : 0;
    job.eps_absolute = flags & AGP_EPS_ABSOLUTE;
    job.sampler_groups = flags & AGP_SAMPLER_GROUPS;
    if (flags & AGP_QUERY_TIMES) job.times = stats;
    job.make_aux = [&](size_t first, int count, std::vector<int32_t> &aux) {
        aux.assign(2 * (size_t)Q, -1);
        for (int l = 0; l < count; ++l) aux[2 * lanes[first + l].query + lanes[first + l].part] = l;
    };
    job.seed = [&](const KArgs &A, int count, const int32_t *d_aux, cudaStream_t st) -> int {
        (void)count;
        return seed(A, d_aux, st);
    };
    // host output: the rows of the queries whose lanes have all run are copied after each wave, on
    // that wave's stream, so the copies overlap the next waves (lanes are sorted by query)
    int64_t next_q = 0;
    auto copy_rows = [&](int64_t q_end, cudaStream_t st) -> int {
        if (n > 0 && q_end > next_q)
            AGP_CUDA_TRY(cudaMemcpy2DAsync(pi_out + next_q * ld_out, sizeof(float) * ld_out, out + next_q * n,
                                           sizeof(float) * n, sizeof(float) * n, (size_t)(q_end - next_q),
                                           cudaMemcpyDeviceToHost, st));
        next_q = std::max(next_q, q_end);
        return AGP_OK;
    };
    if (host_out)
        job.after_wave = [&](size_t first, int count, cudaStream_t st) -> int {
            const size_t end = first + (size_t)count;
            return copy_rows(end < lanes.size() ? (int64_t)lanes[end].query : (int64_t)Q, st);
        };
    AGP_TRY(run_waves(g, ctx, ws, lanes, params, G, plain, profile, collect, stats, s, job));
    if (collect)
        for (int q = 0; q < Q; ++q) stats[q].levels = params[n_params == 1 ? 0 : q].L + 1;
    if (host_out) {
        AGP_TRY(copy_rows(Q, s));  // queries without lanes (zero signals) after the last wave
        AGP_CUDA_TRY(cudaStreamSynchronize(s));
    }
    AGP_CUDA_TRY(cudaGetLastError());
    return AGP_OK;
}

// ------------------------------------------------------------------------------------ dense signals
int query_dense(agp_graph_s *g, const agp_params_t *params, int32_t n_params, int32_t Q, const void *X, int64_t ldx,
                float *pi_out, int64_t ld_out, uint32_t flags, agp_stats_t *stats, cudaStream_t s)
{
    if (!g) return fail(AGP_EINVAL, "graph is NULL");
    if (Q < 0) return fail(AGP_EINVAL, "Q < 0");
    if (Q == 0) return AGP_OK;
    if (!params || !(n_params == 1 || n_params == Q)) return fail(AGP_EINVAL, "n_params must be 1 or Q");
    const int64_t n = g->n;
    if (ldx < n || ld_out < n) return fail(AGP_EINVAL, "ldx and ld_out must be >= n");
    if (n > 0 && (!X || !pi_out)) return fail(AGP_EINVAL, "X / pi_out NULL");
    if (flags & ~(AGP_INPUT_ON_DEVICE | AGP_OUTPUT_ON_DEVICE | AGP_PLAIN | AGP_COLLECT_STATS | AGP_PROFILE |
                  AGP_QUERY_TIMES | AGP_EPS_ABSOLUTE | AGP_DENSE_BF16 | AGP_SAMPLER_GROUPS))
        return fail(AGP_EINVAL, "unknown flag");
    if ((flags & (AGP_COLLECT_STATS | AGP_QUERY_TIMES)) && !stats)
        return fail(AGP_EINVAL, "AGP_COLLECT_STATS / AGP_QUERY_TIMES need stats");
    for (int i = 0; i < n_params; ++i) AGP_TRY(validate_params_for(g, params[i]));
    AGP_CUDA_TRY(cudaSetDevice(g->device));
    if (n == 0) return AGP_OK;
    const bool bf16 = flags & AGP_DENSE_BF16;
    const size_t esz = bf16 ? 2 : 4;
    const int chunks = (int)std::max<int64_t>(1, std::min<int64_t>(256, (n + 65535) / 65536));
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const bool host_in = !(flags & AGP_INPUT_ON_DEVICE);
    const size_t x_b = host_in ? al(esz * (size_t)Q * (size_t)n) : 0;
    const size_t part_b = al(sizeof(double) * 2 * (size_t)Q * chunks), norm_b = al(sizeof(double) * 2 * Q);
    ExecCtx ctx{nullptr, &g->in_stage, &g->in_bytes};
    AGP_TRY(grow(ctx.stage, ctx.stage_bytes, x_b + part_b + norm_b + 256));
    char *p = (char *)*ctx.stage;
    const void *Xd = X;
    int64_t ld = ldx;
    if (host_in) {  // rows are packed to stride n on the device
        AGP_CUDA_TRY(cudaMemcpy2DAsync(p, esz * n, X, esz * ldx, esz * n, Q, cudaMemcpyHostToDevice, s));
        Xd = p;
        ld = n;
    }
    double *d_part = (double *)(p + x_b), *d_norm = (double *)(p + x_b + part_b);
    unsigned int *d_bad = (unsigned int *)(p + x_b + part_b + norm_b);
    AGP_CUDA_TRY(cudaMemsetAsync(d_bad, 0, sizeof(unsigned int), s));
    const dim3 grid(chunks, Q);
    if (bf16) k_rownorm_part<<<grid, kBlock, 0, s>>>((const uint16_t *)Xd, ld, n, chunks, d_part, d_bad);
    else k_rownorm_part<<<grid, kBlock, 0, s>>>((const float *)Xd, ld, n, chunks, d_part, d_bad);
    k_rownorm_sum<<<(2 * Q + 127) / 128, 128, 0, s>>>(d_part, chunks, Q, d_norm);
    __atomic_fetch_add(&g->kernel_launches, (int64_t)2, __ATOMIC_RELAXED);
    AGP_CUDA_TRY(cudaGetLastError());
    std::vector<double> norms(2 * Q);
    unsigned int bad = 0;
    AGP_CUDA_TRY(cudaMemcpyAsync(norms.data(), d_norm, sizeof(double) * 2 * Q, cudaMemcpyDeviceToHost, s));
    AGP_CUDA_TRY(cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, s));
    AGP_CUDA_TRY(cudaStreamSynchronize(s));
    if (bad) return fail(AGP_EINVAL, "non-finite value in a dense signal");
    auto seed = [&](const KArgs &A, const int32_t *d_aux, cudaStream_t st) -> int {
        if (bf16) k_seed_dense_rows<<<A.grid, kBlock, 0, st>>>(A, (const uint16_t *)Xd, ld, Q, d_aux, d_norm);
        else k_seed_dense_rows<<<A.grid, kBlock, 0, st>>>(A, (const float *)Xd, ld, Q, d_aux, d_norm);
        AGP_CUDA_TRY(cudaGetLastError());
        return AGP_OK;
    };
    return run_queries(g, &ctx, params, n_params, Q, norms, seed, pi_out, ld_out, flags, stats, s);
}

int feature_propagate(agp_graph_s *g, const agp_params_t *params, const uint16_t *X, int64_t d, int64_t ldx,
                      float *Z, int64_t ldz, uint32_t flags, cudaStream_t s)
{
    if (!g) return fail(AGP_EINVAL, "graph is NULL");
    ExecCtx ctx{nullptr, &g->in_stage, &g->in_bytes};
    return feature_propagate_ctx(g, &ctx, params, X, d, ldx, Z, ldz, flags, s);
}

int feature_propagate_ctx(agp_graph_s *g, ExecCtx *ctx, const agp_params_t *params, const uint16_t *X, int64_t d,
                          int64_t ldx, float *Z, int64_t ldz, uint32_t flags, cudaStream_t s)
{
    if (!g || !params) return fail(AGP_EINVAL, "NULL argument");
    if (d < 0 || ldx < d || ldz < d) return fail(AGP_EINVAL, "need d >= 0, ldx >= d, ldz >= d");
    if (flags & ~(AGP_PLAIN | AGP_PROFILE | AGP_EPS_ABSOLUTE | AGP_SAMPLER_GROUPS)) return fail(AGP_EINVAL, "unknown flag");
    AGP_TRY(validate_params_for(g, *params));
    const bool profile = flags & AGP_PROFILE;
    if (d == 0 || g->n == 0) return AGP_OK;  // nothing to read or write: X and Z may be NULL
    if (!X || !Z) return fail(AGP_EINVAL, "NULL argument");
    AGP_CUDA_TRY(cudaSetDevice(g->device));
    const bool plain = flags & AGP_PLAIN;
    const int64_t n = g->n;
    // eps = 0 on an undirected graph: exact propagation (Algorithm 1) over column tiles, pulling over
    // the symmetric rows (no atomics); the plain path and directed graphs keep the lane pipeline
    if (params->eps == 0.0 && !plain && !g->directed && !ctx->ws)
        return feature_exact_tiled(g, params, X, d, ldx, Z, ldz, s);
    Workspace *ws = ctx->ws;
    if (!ws) AGP_TRY(ensure_workspace(g, (int)std::min<int64_t>({2 * d, 4096, (int64_t)wave_lanes(g)}), plain, &ws));
    // column norms of the sign parts
    const size_t norm_b = sizeof(double) * 2 * d;
    AGP_TRY(grow(ctx->stage, ctx->stage_bytes, norm_b + 256));
    double *d_norm = (double *)*ctx->stage;
    AGP_CUDA_TRY(cudaMemsetAsync(d_norm, 0, norm_b, s));
    launch_colnorms_bf16(X, n, d, ldx, d_norm, s);
    __atomic_fetch_add(&g->kernel_launches, (int64_t)(1), __ATOMIC_RELAXED);
    AGP_CUDA_TRY(cudaGetLastError());
    std::vector<double> norms(2 * d);
    AGP_CUDA_TRY(cudaMemcpyAsync(norms.data(), d_norm, norm_b, cudaMemcpyDeviceToHost, s));
    AGP_CUDA_TRY(cudaStreamSynchronize(s));
    AGP_CUDA_TRY(cudaMemset2DAsync(Z, sizeof(float) * ldz, 0, sizeof(float) * d, n, s));
    std::vector<LaneSpec> lanes;
    for (int64_t c = 0; c < d; ++c)
        for (int part = 0; part < 2; ++part)
            if (norms[2 * c + part] > 0.0) lanes.push_back(LaneSpec{(int)c, part, norms[2 * c + part], 0});
    const int G = plain ? 1 : std::min({ws->G, 4096, ctx->ws ? ws->G : wave_lanes(g)});
    WaveJob job;
    job.out = Z;
    job.su = ldz;
    job.sr = 1;
    job.stream_base_is_query = 1;  // column c of part s draws from the stream (seed, c, s)
    job.eps_absolute = flags & AGP_EPS_ABSOLUTE;
    job.sampler_groups = flags & AGP_SAMPLER_GROUPS;
    job.make_aux = [&](size_t first, int count, std::vector<int32_t> &aux) {
        aux.resize(2 * (size_t)count);
        for (int l = 0; l < count; ++l) {
            aux[l] = lanes[first + l].query;          // column
            aux[count + l] = lanes[first + l].part;   // sign part
        }
    };
    job.seed = [&](const KArgs &A, int count, const int32_t *d_aux, cudaStream_t st) -> int {
        launch_seed_dense_bf16(A, X, ldx, nullptr, d_aux, d_aux + count, d_norm, count, st);
        AGP_CUDA_TRY(cudaGetLastError());
        return AGP_OK;
    };
    AGP_TRY(run_waves(g, ctx, ws, lanes, params, G, plain, profile, 0, nullptr, s, job));
    return AGP_OK;
}

int threshold(agp_graph_s *g, double a, double eps, int64_t count, const int32_t *nodes, const float *c,
              int32_t *k_out, cudaStream_t s)
{
    if (!g) return fail(AGP_EINVAL, "graph is NULL");
    if (!(a >= 0.0 && a <= 1.0) || !(eps >= 0.0)) return fail(AGP_EINVAL, "a in [0,1], eps >= 0");
    if (g->directed == 1 && a != 0.0) return fail(AGP_EINVAL, "a directed graph needs a = 0");
    if (count < 0 || (count > 0 && (!nodes || !c || !k_out))) return fail(AGP_EINVAL, "bad arrays");
    if (count == 0) return AGP_OK;
    AGP_CUDA_TRY(cudaSetDevice(g->device));
    LaneParam P{};
    P.eps_d = eps;
    P.eps = (float)eps;
    P.a = (float)a;
    P.a_d = a;
    P.a_mode = exponent_mode(a);
    lane_param_derive(P);
    k_threshold<<<blocks_for((unsigned long long)count, kBlock), kBlock, 0, s>>>(g->dev(), P, count, nodes, c, k_out);
    AGP_CUDA_TRY(cudaGetLastError());
    return AGP_OK;
}

}  // namespace agp
