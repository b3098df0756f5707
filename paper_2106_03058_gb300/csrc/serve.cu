// serve.cu -- continuous-batching server: admission into lanes, shared level sweeps, completion.
//
// The server keeps requests in two pools of lanes ("slots"): light requests and heavy ones, split by
// the estimated cost of Theorem 4.3's bound. Each pool owns a lane workspace, a stream and a captured
// sweep: one level of Algorithm 2 for every lane of the pool (compact / expand / push / sample /
// level end). Lanes carry their own level, coefficients, L and random key, so requests admitted at
// different times share sweeps. A host thread drives both pools:
//   1. it admits waiting requests of each pool (cost-aware or FIFO) while the pool's free slots and
//      the result memory allow, seeds them and starts them at level 0 (the heavy pool only between
//      its sweeps),
//   2. it launches the heavy pool's sweep without waiting for it, then runs light sweeps back to
//      back on the light pool's higher-priority stream, retiring finished light requests after each,
//   3. when the heavy sweep's event has fired, it retires finished heavy requests and starts the next
//      heavy sweep.
// A light request therefore never waits for a sweep of heavy lanes (eps = 1e-9, L = 40: ~140 ms a
// level on the 4M-node graph), only for its own pool's short sweeps; the heavy pool's kernels use a
// quarter of the usual grid, so the light kernels find free SM slots while they run. Waits of host
// threads on results are bounded by the caller's timeout.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lanes.cuh"

namespace agp {
namespace {

using Clock = std::chrono::steady_clock;

double now_us()
{
    return std::chrono::duration<double, std::micro>(Clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t ticket = 0;
    agp_request_t r{};
    std::vector<double> w;          // FINITE weights (copied)
    std::vector<uint16_t> X;        // feature block (copied)
    double t_submit = 0, t_admit = 0, t_done = 0;
    int status = AGP_OK;
    bool done = false, cancelled = false, released = false, cut = false, counted = false;
    int lanes_left = 0;
    double cost = 0.0;              // estimated operations (admission priority)
    int pool = 0;                   // kLight or kHeavy
    bool in_queue = false;          // waiting for admission (queue entries of other requests are dropped lazily)
    int refs = 0;                   // queue entries that still point at this request
    bool zombie = false;            // released while queue entries remained: deleted with the last one
    std::vector<int> slots;
    float *d_out = nullptr;         // device result (n or n * cols floats)
    float *h_out = nullptr;         // pinned host copy when results live on the host
    size_t bytes = 0;
};

constexpr int kLight = 0, kHeavy = 1;

// One pool of lanes with its own workspace, stream, sweep and seed staging. free_slots is guarded
// by the server mutex; the rest belongs to the server thread.
struct Pool {
    Workspace *ws = nullptr;
    KArgs A{};
    cudaStream_t stream = nullptr;
    cudaGraphExec_t sweep = nullptr;
    cudaEvent_t done = nullptr;    // end of the sweep in flight
    bool in_flight = false;
    std::vector<Request *> slot_owner;
    std::vector<int> free_slots;
    std::vector<int32_t> h_level;
    int active_lanes = 0;
    int32_t *d_seed_lane = nullptr, *d_seed_src = nullptr;
    CoefSpec *d_spec = nullptr;
    double *d_w = nullptr;
    size_t d_w_cap = 0;
    uint16_t *d_X = nullptr;
    size_t d_X_cap = 0;
    double *d_norm = nullptr;
    int32_t *d_col = nullptr, *d_part = nullptr, *d_lane_of = nullptr;
};

}  // namespace
}  // namespace agp

struct agp_server_s {
    agp_graph_s *g = nullptr;
    agp_serve_config_t cfg{};
    agp::Pool pool[2];
    int npools = 2;                 // 1 in FIFO-plain mode (its one-lane workspace)
    std::thread th;
    std::mutex m;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    uint64_t next_ticket = 1;
    // Waiting requests. `queue[p]` is pool p's arrival order (FIFO admission, the oldest request, the
    // FIFO plain mode); `cls[c]` holds the requests of cost class c = floor(log2 cost), in arrival
    // order (a class belongs to one pool). Entries of requests that left the queue (admitted,
    // cancelled, expired) are dropped lazily when they reach a front, so every operation is O(1) or
    // O(classes) however long the queue grows.
    std::deque<agp::Request *> queue[2];
    std::deque<agp::Request *> cls[64];
    std::vector<agp::Request *> with_deadline;  // waiting requests that carry a deadline
    int64_t queued = 0;                          // waiting requests
    int64_t queued_pool[2] = {0, 0};
    std::unordered_map<uint64_t, agp::Request *> all;
    int64_t result_bytes[2] = {0, 0};  // result bytes of admitted, unreleased requests, per pool
    std::deque<uint64_t> done_q;     // tickets of finished requests, in completion order (agp_serve_next)
    int64_t completed = 0, sweeps = 0;
    std::unordered_map<size_t, std::vector<void *>> free_dev, free_host;  // result buffers by size
    int64_t pooled_bytes = 0;
    void *fifo_stage = nullptr;  // input staging of the FIFO-plain path (never the graph's own)
    size_t fifo_stage_bytes = 0;
    int fatal = AGP_OK;
};

namespace agp {
namespace {

constexpr int kMaxCols = 1024;
constexpr int kCostClasses = 64;
constexpr int kHeavyClass = 23;        // cost classes >= this (estimated operations >= 2^23 ~ 8.4e6) are heavy:
                                       // a sweep of a full light pool then stays at a few milliseconds
constexpr double kAgingUs = 1e6;       // a request's priority doubles every second it waits
constexpr double kStarveUs = 30e6;     // a request waiting longer than this reserves the lanes it needs

// Estimated operations of a request: the edge operations bounded in the proof of Theorem 4.3,
// E[pushes + samples] <= (1/eps) sum_{i=1..L} (Y_i / Y_0) ||P^i x||_1, plus the frontier items, one
// per non-zero residue and level (the bound leaves them out; a dense feature column starts with n of
// them and keeps most of them). The mass ||P^i x||_1 is 1 for the column-stochastic presets (a = 0,
// b = 1 and one-hot x) and is bounded by the number of levels otherwise; eps = 0 (exact) counts as
// the full graph per level.
double estimate_cost(const agp_request_t &r, int64_t n, int64_t nnz)
{
    const agp_params_t &p = r.params;
    const int L = p.L;
    double mass;
    const bool stochastic = p.a == 0.0 && p.b == 1.0;
    switch (p.kind) {
    case AGP_W_PPR: mass = stochastic ? std::min((double)L, (1.0 - p.param) / p.param) : L; break;
    case AGP_W_HKPR: mass = stochastic ? std::min((double)L, p.param) : L; break;
    case AGP_W_KATZ: mass = (double)L * 10.0; break;  // mass grows like (beta lambda_1)^i times the source's reach
    default: mass = L; break;
    }
    const double parts = r.source >= 0 ? 1.0 : 2.0 * r.cols;
    const double per_lane = p.eps > 0.0 ? mass / p.eps : (double)L * (double)nnz;
    const double support = r.source >= 0 ? 1.0 : 0.5 * (double)n;  // non-zeros of a sign part of x
    return parts * (std::min(per_lane, (double)(L + 1) * (double)nnz) + (double)(L + 1) * support) + 1e5;
}

int cost_class(double cost)
{
    const int c = cost >= 1.0 ? (int)std::floor(std::log2(cost)) : 0;
    return std::min(kCostClasses - 1, std::max(0, c));
}

void finish(agp_server_s *S, Request *q, int status)
{
    q->status = status;
    q->done = true;
    q->t_done = now_us();
    ++S->completed;
    S->done_q.push_back(q->ticket);
    // a client that waits ticket by ticket never takes these: drop the entries of released requests
    // once the queue is much longer than the requests still held, so it stays bounded
    if (S->done_q.size() > 2 * S->all.size() + 1024) {
        std::deque<uint64_t> keep;
        for (const uint64_t t : S->done_q) {
            auto it = S->all.find(t);
            if (it != S->all.end() && !it->second->released) keep.push_back(t);
        }
        S->done_q.swap(keep);
    }
    S->cv_done.notify_all();
}

void free_result(agp_server_s *S, Request *q, bool destroy = false);

// Result buffers are pooled by size: cudaMalloc and cudaFree synchronise the whole device, so an
// allocation per admitted request (or a free per released one) would stall every sweep in flight,
// the heavy pool's included, until it ends. A released buffer goes back to its size's free list
// (while the pooled bytes stay within the result budget) and the next request of that size takes it.
int alloc_result(agp_server_s *S, Request *q, cudaStream_t st)
{
    const int64_t n = S->g->n;
    const size_t elems = (size_t)n * (size_t)(q->r.source >= 0 ? 1 : q->r.cols);
    q->bytes = std::max<size_t>(elems * sizeof(float), 16);
    {
        std::lock_guard<std::mutex> lk(S->m);
        auto take = [&](std::unordered_map<size_t, std::vector<void *>> &pool, void **out) {
            auto it = pool.find(q->bytes);
            if (it == pool.end() || it->second.empty()) return false;
            *out = it->second.back();
            it->second.pop_back();
            S->pooled_bytes -= (int64_t)q->bytes;
            return true;
        };
        void *p = nullptr;
        if (take(S->free_dev, &p)) q->d_out = (float *)p;
        if (S->cfg.results_on_host && take(S->free_host, &p)) q->h_out = (float *)p;
    }
    if (!q->d_out && cudaMalloc((void **)&q->d_out, q->bytes) != cudaSuccess) {
        cudaGetLastError();
        q->d_out = nullptr;
        return fail(AGP_ENOMEM, "server: result buffer");
    }
    if (S->cfg.results_on_host && !q->h_out && cudaMallocHost((void **)&q->h_out, q->bytes) != cudaSuccess) {
        cudaGetLastError();
        free_result(S, q);
        return fail(AGP_ENOMEM, "server: pinned result buffer");
    }
    AGP_CUDA_TRY(cudaMemsetAsync(q->d_out, 0, q->bytes, st));
    return AGP_OK;
}

// Return q's buffers to the size pools (freed outright past the result budget, or at destroy).
void free_result(agp_server_s *S, Request *q, bool destroy)
{
    bool keep = false;
    if (!destroy) {
        std::lock_guard<std::mutex> lk(S->m);
        const int64_t add = (int64_t)q->bytes * ((q->d_out ? 1 : 0) + (q->h_out ? 1 : 0));
        if (S->pooled_bytes + add <= S->cfg.result_budget) {
            if (q->d_out) S->free_dev[q->bytes].push_back(q->d_out);
            if (q->h_out) S->free_host[q->bytes].push_back(q->h_out);
            S->pooled_bytes += add;
            keep = true;
        }
    }
    if (!keep) {
        if (q->d_out) cudaFree(q->d_out);
        if (q->h_out) cudaFreeHost(q->h_out);
    }
    q->d_out = nullptr;
    q->h_out = nullptr;
}

// Fill lane `slot` of pool P for request q (column `col` / sign `part`, L1 norm `norm`); returns its
// CoefSpec.
CoefSpec start_lane(Pool &P, Request *q, int slot, int col, int part, double norm, int w_off)
{
    const agp_params_t &p = q->r.params;
    LaneParam L{};
    L.eps_d = (q->r.flags & AGP_REQ_EPS_ABSOLUTE) ? lane_eps_absolute(p.eps, norm) : p.eps;
    L.eps = (float)L.eps_d;
    L.a = (float)p.a;
    L.b = (float)p.b;
    L.a_d = p.a;
    L.a_mode = exponent_mode(p.a);
    L.b_mode = exponent_mode(p.b);
    L.L = p.L;
    L.out_row = col;
    if (q->r.source >= 0) {
        L.out = q->d_out;
        L.su = 1;
    } else {
        L.out = q->d_out + col;
        L.su = q->r.cols;
    }
    lane_key(p.seed, q->r.source >= 0 ? 0ull : (uint64_t)col, part, L.key0, L.key1);
    lane_param_derive(L);
    P.ws->h_lanes[slot] = L;
    CoefSpec c{};
    c.lane = slot;
    c.kind = p.kind;
    c.L = p.L;
    c.param = p.param;
    c.w_off = w_off;
    c.scale = (part ? -1.0 : 1.0) * norm;
    return c;
}

// One queue entry of q is gone; a released request is deleted with its last entry.
void unref(Request *q)
{
    if (--q->refs == 0 && q->zombie) delete q;
}

// Drop the entries of requests that no longer wait from the front of d.
void pop_dead(std::deque<Request *> &d)
{
    while (!d.empty() && !d.front()->in_queue) {
        Request *q = d.front();
        d.pop_front();
        unref(q);
    }
}

// q stops waiting (admitted or finished); its queue entries are dropped lazily.
void dequeue(agp_server_s *S, Request *q)
{
    if (q->in_queue) {
        q->in_queue = false;
        --S->queued;
        --S->queued_pool[q->pool];
    }
}

// Every queue entry (stop and fatal paths). Requests stay owned by S->all unless released.
void drain_queues(agp_server_s *S)
{
    auto drain = [](std::deque<Request *> &d) {
        while (!d.empty()) {
            Request *q = d.front();
            d.pop_front();
            q->in_queue = false;
            unref(q);
        }
    };
    for (auto &d : S->queue) drain(d);
    for (auto &d : S->cls) drain(d);
    for (Request *q : S->with_deadline) {
        q->in_queue = false;
        unref(q);
    }
    S->with_deadline.clear();
    S->queued = 0;
    S->queued_pool[0] = S->queued_pool[1] = 0;
}

// Waiting requests past their deadline finish with AGP_ETIMEDOUT (cancelled waiting requests are
// finished by agp_serve_cancel itself). Called with S->m held.
void expire_waiting(agp_server_s *S, double t)
{
    size_t keep = 0;
    for (Request *q : S->with_deadline) {
        if (q->in_queue && t - q->t_submit > (double)q->r.deadline_us) {
            dequeue(S, q);
            finish(S, q, AGP_ETIMEDOUT);
        }
        if (q->in_queue) S->with_deadline[keep++] = q;
        else unref(q);
    }
    S->with_deadline.resize(keep);
}

int need_of(const Request *q) { return q->r.source >= 0 ? 1 : 2 * q->r.cols; }

// Admit queued requests of pool p while its slots and the result memory allow. Called by the server
// thread, between sweeps of that pool.
int admit(agp_server_s *S, int p)
{
    Pool &P = S->pool[p];
    std::vector<Request *> take;
    std::vector<int> cut;
    {
        std::lock_guard<std::mutex> lk(S->m);
        // cancelled requests in flight: their lanes stop after the next sweep (L lowered to 0, so
        // the lanes only reserve what they hold and finish)
        for (int sl = 0; sl < (int)P.slot_owner.size(); ++sl) {
            Request *q = P.slot_owner[sl];
            if (q && q->cancelled && !q->cut) cut.push_back(sl);
        }
        for (int sl : cut) P.slot_owner[sl]->cut = true;
        const double t = now_us();
        expire_waiting(S, t);
        const bool fifo = S->cfg.admission == AGP_ADMIT_FIFO;
        const int c_lo = (p == kHeavy) ? kHeavyClass : 0, c_hi = (p == kHeavy) ? kCostClasses : kHeavyClass;
        auto fits = [&](const Request *q) { return (int)P.free_slots.size() >= need_of(q); };
        while (S->queued_pool[p] > 0) {
            // FIFO: the pool's oldest request. Cost-aware: among the oldest request of every cost
            // class of the pool (floor(log2 cost)), the one that fits now with the best aged priority
            // cost / (1 + seconds waited). Within a class requests start in arrival order. A request
            // that has waited past kStarveUs goes next under either policy, and nothing else of its
            // pool starts until its slots are free (no starvation of wide requests).
            pop_dead(S->queue[p]);
            if (S->queue[p].empty()) break;
            Request *q = nullptr;
            std::deque<Request *> *from = nullptr;
            Request *oldest = S->queue[p].front();
            if (fifo || t - oldest->t_submit > kStarveUs) {
                if (!fits(oldest)) break;
                q = oldest;
                from = &S->queue[p];
            } else {
                double best = 0.0;
                for (int c = c_lo; c < c_hi; ++c) {
                    std::deque<Request *> &d = S->cls[c];
                    pop_dead(d);
                    if (d.empty() || !fits(d.front())) continue;
                    Request *h = d.front();
                    const double prio = h->cost / (1.0 + (t - h->t_submit) / kAgingUs);
                    if (!q || prio < best) {
                        q = h;
                        best = prio;
                        from = &d;
                    }
                }
                if (!q) break;
            }
            const int need = need_of(q);
            const int64_t bytes = (int64_t)S->g->n * (q->r.source >= 0 ? 1 : q->r.cols) * (int64_t)sizeof(float);
            // each pool has half of the result budget, so that requests of one pool that hold their
            // results (waiting to run, or unreleased) never keep the other from admitting
            const int64_t budget = S->npools == 2 ? S->cfg.result_budget / 2 : S->cfg.result_budget;
            if (S->result_bytes[p] + bytes > budget && S->result_bytes[p] > 0) break;
            from->pop_front();
            unref(q);  // still owned by S->all: not released while it waits
            dequeue(S, q);
            q->t_admit = t;
            q->slots.clear();
            for (int k = 0; k < need; ++k) {
                // the lowest free slot: admitted lanes pack into as few groups of four as possible,
                // so more of them share row walks
                auto lo = std::min_element(P.free_slots.begin(), P.free_slots.end());
                q->slots.push_back(*lo);
                *lo = P.free_slots.back();
                P.free_slots.pop_back();
            }
            S->result_bytes[p] += bytes;
            q->counted = true;
            take.push_back(q);
        }
    }
    static const int32_t zero_L = 0;
    for (int sl : cut)
        AGP_CUDA_TRY(cudaMemcpyAsync(&P.ws->lanes[sl].L, &zero_L, sizeof(int32_t), cudaMemcpyHostToDevice, P.stream));
    if (take.empty()) return AGP_OK;
    std::vector<CoefSpec> specs;
    std::vector<double> wts;
    std::vector<int32_t> seed_lane, seed_src;
    std::vector<int32_t> start;  // slots that start at level 0
    std::vector<int> give_back;
    for (Request *q : take) {
        int w_off = 0;
        if (q->r.params.kind == AGP_W_FINITE) {
            w_off = (int)wts.size();
            wts.insert(wts.end(), q->w.begin(), q->w.end());
        }
        int rc = alloc_result(S, q, P.stream);
        if (rc != AGP_OK) {
            std::lock_guard<std::mutex> lk(S->m);
            for (int sl : q->slots) P.free_slots.push_back(sl);
            S->result_bytes[p] -= (int64_t)q->bytes;
            q->slots.clear();
            finish(S, q, rc);
            continue;
        }
        if (q->r.source >= 0) {
            const int slot = q->slots[0];
            specs.push_back(start_lane(P, q, slot, 0, 0, 1.0, w_off));
            seed_lane.push_back(slot);
            seed_src.push_back(q->r.source);
            start.push_back(slot);
            P.slot_owner[slot] = q;
            q->lanes_left = 1;
            continue;
        }
        // feature block: column norms of the sign parts decide which lanes run
        const int cols = q->r.cols;
        const bool x_dev = q->r.flags & AGP_REQ_X_ON_DEVICE;
        const uint16_t *X = x_dev ? q->r.X : P.d_X;
        const int64_t ldx = x_dev ? q->r.ldx : cols;
        const size_t xb = x_dev ? 0 : sizeof(uint16_t) * (size_t)S->g->n * cols;
        if (xb > P.d_X_cap) {
            cudaFree(P.d_X);
            P.d_X = nullptr;
            P.d_X_cap = 0;
            if (cudaMalloc((void **)&P.d_X, xb) != cudaSuccess) {
                cudaGetLastError();
                free_result(S, q);  // takes the server lock itself
                std::lock_guard<std::mutex> lk(S->m);
                for (int sl : q->slots) P.free_slots.push_back(sl);
                S->result_bytes[p] -= (int64_t)q->bytes;
                finish(S, q, fail(AGP_ENOMEM, "server: feature staging"));
                continue;
            }
            P.d_X_cap = xb;
        }
        if (!x_dev) {
            AGP_CUDA_TRY(cudaMemcpyAsync(P.d_X, q->X.data(), xb, cudaMemcpyHostToDevice, P.stream));
            X = P.d_X;
        }
        AGP_CUDA_TRY(cudaMemsetAsync(P.d_norm, 0, sizeof(double) * 2 * cols, P.stream));
        launch_colnorms_bf16(X, S->g->n, cols, ldx, P.d_norm, P.stream);
        std::vector<double> norms(2 * cols);
        AGP_CUDA_TRY(cudaMemcpyAsync(norms.data(), P.d_norm, sizeof(double) * 2 * cols, cudaMemcpyDeviceToHost, P.stream));
        AGP_CUDA_TRY(cudaStreamSynchronize(P.stream));
        std::vector<int32_t> lane_of, col_of, part_of;
        size_t used = 0;
        for (int c = 0; c < cols; ++c)
            for (int part = 0; part < 2; ++part) {
                if (!(norms[2 * c + part] > 0.0)) continue;
                const int slot = q->slots[used++];
                specs.push_back(start_lane(P, q, slot, c, part, norms[2 * c + part], w_off));
                lane_of.push_back(slot);
                col_of.push_back(c);
                part_of.push_back(part);
                start.push_back(slot);
                P.slot_owner[slot] = q;
            }
        {
            std::lock_guard<std::mutex> lk(S->m);
            for (size_t k = used; k < q->slots.size(); ++k) give_back.push_back(q->slots[k]);
            q->slots.resize(used);
        }
        q->lanes_left = (int)used;
        if (used == 0) {
            AGP_CUDA_TRY(cudaStreamSynchronize(P.stream));
            if (q->h_out) std::memset(q->h_out, 0, q->bytes);
            std::lock_guard<std::mutex> lk(S->m);
            finish(S, q, AGP_OK);
            continue;
        }
        // parameters and coefficients must be on the device before the dense seed
        for (size_t k = 0; k < lane_of.size(); ++k)
            AGP_CUDA_TRY(cudaMemcpyAsync(P.ws->lanes + lane_of[k], P.ws->h_lanes + lane_of[k], sizeof(LaneParam),
                                         cudaMemcpyHostToDevice, P.stream));
        AGP_CUDA_TRY(cudaMemcpyAsync(P.d_lane_of, lane_of.data(), sizeof(int32_t) * lane_of.size(), cudaMemcpyHostToDevice, P.stream));
        AGP_CUDA_TRY(cudaMemcpyAsync(P.d_col, col_of.data(), sizeof(int32_t) * col_of.size(), cudaMemcpyHostToDevice, P.stream));
        AGP_CUDA_TRY(cudaMemcpyAsync(P.d_part, part_of.data(), sizeof(int32_t) * part_of.size(), cudaMemcpyHostToDevice, P.stream));
        launch_seed_dense_bf16(P.A, X, ldx, P.d_lane_of, P.d_col, P.d_part, P.d_norm, (int)lane_of.size(), P.stream);
        AGP_CUDA_TRY(cudaStreamSynchronize(P.stream));  // d_X and the seed staging are reused
    }
    if (!give_back.empty()) {
        std::lock_guard<std::mutex> lk(S->m);
        for (int sl : give_back) P.free_slots.push_back(sl);
    }
    if (!specs.empty()) {
        // lane parameters, coefficients and levels
        for (const CoefSpec &c : specs)
            AGP_CUDA_TRY(cudaMemcpyAsync(P.ws->lanes + c.lane, P.ws->h_lanes + c.lane, sizeof(LaneParam),
                                         cudaMemcpyHostToDevice, P.stream));
        if (wts.size() > P.d_w_cap) {
            cudaFree(P.d_w);
            if (cudaMalloc((void **)&P.d_w, sizeof(double) * wts.size()) != cudaSuccess) {
                cudaGetLastError();
                P.d_w = nullptr;
                P.d_w_cap = 0;
                return fail(AGP_ENOMEM, "server: weight staging");
            }
            P.d_w_cap = wts.size();
        }
        if (!wts.empty()) AGP_CUDA_TRY(cudaMemcpyAsync(P.d_w, wts.data(), sizeof(double) * wts.size(), cudaMemcpyHostToDevice, P.stream));
        AGP_CUDA_TRY(cudaMemcpyAsync(P.d_spec, specs.data(), sizeof(CoefSpec) * specs.size(), cudaMemcpyHostToDevice, P.stream));
        launch_coef(P.d_spec, P.d_w, P.ws->coef, (int)specs.size(), P.stream);
        const int32_t zero = 0;
        for (int32_t sl : start)
            AGP_CUDA_TRY(cudaMemcpyAsync(P.ws->level + sl, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, P.stream));
        if (!seed_lane.empty()) {
            AGP_CUDA_TRY(cudaMemcpyAsync(P.d_seed_lane, seed_lane.data(), sizeof(int32_t) * seed_lane.size(), cudaMemcpyHostToDevice, P.stream));
            AGP_CUDA_TRY(cudaMemcpyAsync(P.d_seed_src, seed_src.data(), sizeof(int32_t) * seed_src.size(), cudaMemcpyHostToDevice, P.stream));
            launch_seed_sources(P.A, P.d_seed_lane, P.d_seed_src, (int)seed_lane.size(), P.stream);
        }
        AGP_CUDA_TRY(cudaGetLastError());
        AGP_CUDA_TRY(cudaStreamSynchronize(P.stream));  // host staging vectors go out of scope
        P.active_lanes += (int)start.size();
    }
    return AGP_OK;
}

// Lanes of pool p whose level went to -1 are finished; complete requests whose lanes are all
// finished. Synchronises the pool's stream.
int retire(agp_server_s *S, int p)
{
    Pool &P = S->pool[p];
    AGP_CUDA_TRY(cudaMemcpyAsync(P.h_level.data(), P.ws->level, sizeof(int32_t) * P.ws->G, cudaMemcpyDeviceToHost, P.stream));
    AGP_CUDA_TRY(cudaStreamSynchronize(P.stream));
    std::vector<Request *> ready;
    for (int sl = 0; sl < P.ws->G; ++sl) {
        Request *q = P.slot_owner[sl];
        if (!q || P.h_level[sl] >= 0) continue;
        P.slot_owner[sl] = nullptr;
        --P.active_lanes;
        {
            std::lock_guard<std::mutex> lk(S->m);
            P.free_slots.push_back(sl);
        }
        if (--q->lanes_left == 0) ready.push_back(q);
    }
    for (Request *q : ready)
        if (q->h_out) AGP_CUDA_TRY(cudaMemcpyAsync(q->h_out, q->d_out, q->bytes, cudaMemcpyDeviceToHost, P.stream));
    if (!ready.empty()) AGP_CUDA_TRY(cudaStreamSynchronize(P.stream));
    std::lock_guard<std::mutex> lk(S->m);
    for (Request *q : ready) finish(S, q, q->cancelled ? AGP_ECANCELED : AGP_OK);
    return AGP_OK;
}

int launch_sweep(agp_server_s *S, int p)
{
    Pool &P = S->pool[p];
    AGP_CUDA_TRY(cudaGraphLaunch(P.sweep, P.stream));
    AGP_CUDA_TRY(cudaEventRecord(P.done, P.stream));
    P.in_flight = true;
    std::lock_guard<std::mutex> lk(S->m);
    ++S->sweeps;
    return AGP_OK;
}

void run_fifo_plain(agp_server_s *S, Request *q)
{
    Pool &P = S->pool[0];
    int rc = alloc_result(S, q, P.stream);
    if (rc == AGP_OK) {
        q->t_admit = now_us();
        // the server's own one-lane workspace and staging: the graph's buffers stay the caller's
        ExecCtx ctx{P.ws, &S->fifo_stage, &S->fifo_stage_bytes};
        if (q->r.source >= 0) {
            const int64_t off[2] = {0, 1};
            rc = query_batch_ctx(S->g, &ctx, &q->r.params, 1, 1, off, &q->r.source, nullptr, q->d_out, S->g->n,
                                 AGP_OUTPUT_ON_DEVICE | AGP_PLAIN, nullptr, P.stream);
        } else if (q->r.flags & AGP_REQ_X_ON_DEVICE) {
            rc = feature_propagate_ctx(S->g, &ctx, &q->r.params, q->r.X, q->r.cols, q->r.ldx, q->d_out, q->r.cols,
                                       AGP_PLAIN, P.stream);
        } else {
            const size_t xb = sizeof(uint16_t) * (size_t)S->g->n * q->r.cols;
            if (xb > P.d_X_cap) {
                cudaFree(P.d_X);
                P.d_X_cap = 0;
                if (cudaMalloc((void **)&P.d_X, xb) != cudaSuccess) {
                    cudaGetLastError();
                    P.d_X = nullptr;
                    rc = fail(AGP_ENOMEM, "server: feature staging");
                } else {
                    P.d_X_cap = xb;
                }
            }
            if (rc == AGP_OK && cudaMemcpyAsync(P.d_X, q->X.data(), xb, cudaMemcpyHostToDevice, P.stream) != cudaSuccess)
                rc = fail(AGP_ECUDA, "server: feature copy");
            if (rc == AGP_OK)
                rc = feature_propagate_ctx(S->g, &ctx, &q->r.params, P.d_X, q->r.cols, q->r.cols, q->d_out, q->r.cols,
                                           AGP_PLAIN, P.stream);
        }
        if (rc == AGP_OK && q->h_out && cudaMemcpyAsync(q->h_out, q->d_out, q->bytes, cudaMemcpyDeviceToHost, P.stream) != cudaSuccess)
            rc = fail(AGP_ECUDA, "server: result copy");
        if (cudaStreamSynchronize(P.stream) != cudaSuccess && rc == AGP_OK) rc = fail(AGP_ECUDA, "server: sync");
    }
    std::lock_guard<std::mutex> lk(S->m);
    finish(S, q, q->cancelled ? AGP_ECANCELED : rc);
}

// The heavy pool yields to the light one. Its kernels share the SMs, the L2 and HBM with the light
// sweeps, and one dense level of a wide feature block keeps them busy for a large fraction of a
// second, which slows every light request in flight by as much. So a heavy sweep starts only while
// the light pool has no lanes in flight (after its admissions), or once a heavy request (waiting or
// in flight) has waited past kStarveUs, from which point its sweeps run beside the light ones until
// it is done.
bool heavy_may_run(agp_server_s *S)
{
    Pool &Lp = S->pool[kLight], &Hp = S->pool[kHeavy];
    if (Lp.active_lanes == 0) return true;
    std::lock_guard<std::mutex> lk(S->m);
    const double t = now_us();
    for (const Request *q : Hp.slot_owner)
        if (q && t - q->t_submit > kStarveUs) return true;
    pop_dead(S->queue[kHeavy]);
    return !S->queue[kHeavy].empty() && t - S->queue[kHeavy].front()->t_submit > kStarveUs;
}

// One step of the batched server thread: admit to the light pool; keep a heavy sweep in flight
// while the heavy pool may run (retiring and admitting between its sweeps, never waiting for it
// here); then sweep and retire the light pool. *busy: some pool has work.
int serve_step(agp_server_s *S, bool *busy)
{
    Pool &Lp = S->pool[kLight], &Hp = S->pool[kHeavy];
    *busy = false;
    if (Hp.in_flight) {
        const cudaError_t e = cudaEventQuery(Hp.done);
        if (e == cudaSuccess) {
            Hp.in_flight = false;
            AGP_TRY(retire(S, kHeavy));
        } else if (e != cudaErrorNotReady) {
            return fail(AGP_ECUDA, std::string("server: heavy sweep: ") + cudaGetErrorString(e));
        }
    }
    AGP_TRY(admit(S, kLight));
    if (!Hp.in_flight && heavy_may_run(S)) {
        AGP_TRY(admit(S, kHeavy));
        if (Hp.active_lanes > 0) AGP_TRY(launch_sweep(S, kHeavy));
    }
    *busy = Hp.in_flight;
    if (Lp.active_lanes > 0) {
        AGP_TRY(launch_sweep(S, kLight));
        AGP_TRY(retire(S, kLight));  // synchronises the light stream
        Lp.in_flight = false;
        *busy = true;
    }
    return AGP_OK;
}

void server_main(agp_server_s *S)
{
    cudaSetDevice(S->g->device);
    if (S->cfg.mode == AGP_SERVE_FIFO_PLAIN) {
        while (true) {
            Request *q = nullptr;
            {
                std::unique_lock<std::mutex> lk(S->m);
                S->cv_work.wait(lk, [&] { return S->stop || S->queued > 0; });
                if (S->stop) return;
                expire_waiting(S, now_us());
                pop_dead(S->queue[0]);
                if (S->queue[0].empty()) continue;
                q = S->queue[0].front();
                S->queue[0].pop_front();
                unref(q);
                dequeue(S, q);
            }
            run_fifo_plain(S, q);
        }
    }
    bool busy = true;
    while (true) {
        {
            std::unique_lock<std::mutex> lk(S->m);
            if (S->stop) return;
            if (!busy && S->queued == 0) {
                S->cv_work.wait_for(lk, std::chrono::milliseconds(2), [&] { return S->stop || S->queued > 0; });
            } else if (S->pool[kLight].active_lanes == 0 && S->pool[kHeavy].in_flight && S->queued_pool[kLight] == 0) {
                // only a heavy sweep runs: wake for a light arrival, or poll its event again shortly
                S->cv_work.wait_for(lk, std::chrono::microseconds(200),
                                    [&] { return S->stop || S->queued_pool[kLight] > 0; });
            }
            if (S->stop) return;
        }
        const int rc = serve_step(S, &busy);
        if (rc != AGP_OK) {
            // a device error ends the server: fail everything pending and in flight
            std::lock_guard<std::mutex> lk(S->m);
            S->fatal = rc;
            for (auto &kv : S->all)
                if (!kv.second->done) finish(S, kv.second, rc);
            drain_queues(S);
            return;
        }
    }
}

int create_pool(agp_server_s *S, Pool &P, int lanes, int W, int priority, int grid)
{
    agp_graph_s *g = S->g;
    AGP_TRY(create_workspace(g, lanes, W, &P.ws, grid));
    AGP_CUDA_TRY(cudaStreamCreateWithPriority(&P.stream, cudaStreamNonBlocking, priority));
    AGP_CUDA_TRY(cudaEventCreateWithFlags(&P.done, cudaEventDisableTiming));
    // every slot may hold work: the compaction scans all of them
    const unsigned int used = (unsigned int)P.ws->G;
    AGP_CUDA_TRY(cudaMemcpy(&P.ws->ctrl->lanes_used, &used, sizeof(used), cudaMemcpyHostToDevice));
    P.A = make_args(g, P.ws, 0);
    if (S->cfg.mode != AGP_SERVE_FIFO_PLAIN) AGP_TRY(capture_levels(P.A, 1, &P.sweep));
    auto dalloc = [&](void **p, size_t b) -> int {
        if (cudaMalloc(p, b) != cudaSuccess) {
            cudaGetLastError();
            return fail(AGP_ENOMEM, "server staging");
        }
        return AGP_OK;
    };
    const int G = P.ws->G;
    AGP_TRY(dalloc((void **)&P.d_seed_lane, sizeof(int32_t) * G));
    AGP_TRY(dalloc((void **)&P.d_seed_src, sizeof(int32_t) * G));
    AGP_TRY(dalloc((void **)&P.d_spec, sizeof(CoefSpec) * G));
    AGP_TRY(dalloc((void **)&P.d_norm, sizeof(double) * 2 * kMaxCols));
    AGP_TRY(dalloc((void **)&P.d_col, sizeof(int32_t) * 2 * kMaxCols));
    AGP_TRY(dalloc((void **)&P.d_part, sizeof(int32_t) * 2 * kMaxCols));
    AGP_TRY(dalloc((void **)&P.d_lane_of, sizeof(int32_t) * 2 * kMaxCols));
    P.slot_owner.assign(G, nullptr);
    P.h_level.assign(G, -1);
    for (int sl = G - 1; sl >= 0; --sl) P.free_slots.push_back(sl);
    return AGP_OK;
}

void destroy_pool(Pool &P)
{
    if (P.sweep) cudaGraphExecDestroy(P.sweep);
    free_workspace(P.ws);
    cudaFree(P.d_seed_lane);
    cudaFree(P.d_seed_src);
    cudaFree(P.d_spec);
    cudaFree(P.d_w);
    cudaFree(P.d_X);
    cudaFree(P.d_norm);
    cudaFree(P.d_col);
    cudaFree(P.d_part);
    cudaFree(P.d_lane_of);
    if (P.done) cudaEventDestroy(P.done);
    if (P.stream) cudaStreamDestroy(P.stream);
    P = Pool{};
}

}  // namespace

int serve_create(agp_graph_s *g, const agp_serve_config_t *cfg, agp_server_s **out)
{
    if (!g || !out) return fail(AGP_EINVAL, "NULL argument");
    *out = nullptr;
    agp_serve_config_t c{};
    if (cfg) c = *cfg;
    if (c.mode != AGP_SERVE_BATCHED && c.mode != AGP_SERVE_FIFO_PLAIN) return fail(AGP_EINVAL, "unknown serve mode");
    if (c.max_lanes < 0 || c.result_budget < 0) return fail(AGP_EINVAL, "negative limit");
    if (c.admission != AGP_ADMIT_COST && c.admission != AGP_ADMIT_FIFO) return fail(AGP_EINVAL, "unknown admission policy");
    if (c.result_budget == 0) c.result_budget = 4ll << 30;
    AGP_CUDA_TRY(cudaSetDevice(g->device));
    agp_server_s *S = new agp_server_s();
    S->g = g;
    // default: room for the widest feature block (2 x 64 columns) next to 8 waves of queries
    int lanes = c.max_lanes > 0 ? c.max_lanes : std::min(lane_capacity(g), std::max(8 * wave_lanes(g), 128));
    lanes = std::max(lanes, 2);
    // batched slots come in groups of four lanes that share row walks (the level pipeline's layout)
    int W = 4;
    if (c.mode == AGP_SERVE_FIFO_PLAIN) lanes = W = 1;
    else lanes = (lanes + 3) / 4 * 4;
    c.max_lanes = lanes;
    S->cfg = c;
    int lo = 0, hi = 0;
    int rc = AGP_OK;
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) {
        cudaGetLastError();
        lo = hi = 0;
    }
    S->npools = (c.mode == AGP_SERVE_FIFO_PLAIN) ? 1 : 2;
    // The GPU is shared between the pools: the heavy pool's level kernels run 2 blocks per SM (all
    // resident at once, half of the slots at the kernels' register use), so its grid-stride blocks never
    // hold every slot for a whole heavy kernel; the light pool's kernels, on the highest-priority
    // stream, take the other slots and run beside them.
    for (int p = 0; p < S->npools && rc == AGP_OK; ++p)
        rc = create_pool(S, S->pool[p], lanes, W, p == kLight ? hi : lo, p == kHeavy ? 2 * sm_count() : 0);
    if (rc != AGP_OK) {
        serve_destroy(S);
        return rc;
    }
    S->th = std::thread(server_main, S);
    *out = S;
    return AGP_OK;
}

int serve_submit(agp_server_s *S, const agp_request_t *req, uint64_t *ticket)
{
    if (!S || !req || !ticket) return fail(AGP_EINVAL, "NULL argument");
    AGP_TRY(validate_params_for(S->g, req->params));
    const int64_t n = S->g->n;
    if (req->source >= 0) {
        if (req->source >= n) return fail(AGP_EINVAL, "source outside [0, n)");
    } else {
        if (req->cols < 1 || req->cols > kMaxCols) return fail(AGP_EINVAL, "feature request needs 1..1024 columns");
        if (!req->X || req->ldx < req->cols) return fail(AGP_EINVAL, "feature request needs X and ldx >= cols");
        if (S->cfg.mode == AGP_SERVE_BATCHED && 2 * req->cols > S->cfg.max_lanes)
            return fail(AGP_EBUDGET, "feature request needs more lanes than the server has");
    }
    Request *q = new Request();
    q->r = *req;
    if (req->params.kind == AGP_W_FINITE) {
        q->w.assign(req->params.w, req->params.w + req->params.L + 1);
        q->r.params.w = nullptr;
    }
    if (req->flags & ~(AGP_REQ_X_ON_DEVICE | AGP_REQ_EPS_ABSOLUTE)) {
        delete q;
        return fail(AGP_EINVAL, "unknown request flag");
    }
    if (req->source < 0 && !(req->flags & AGP_REQ_X_ON_DEVICE)) {
        q->X.resize((size_t)n * req->cols);
        for (int64_t u = 0; u < n; ++u)
            std::memcpy(q->X.data() + (size_t)u * req->cols, req->X + (size_t)u * req->ldx, sizeof(uint16_t) * req->cols);
        q->r.X = nullptr;
    }
    q->t_submit = now_us();
    q->cost = estimate_cost(q->r, S->g->n, S->g->nnz);
    const int cc = cost_class(q->cost);
    q->pool = (S->npools == 2 && cc >= kHeavyClass) ? kHeavy : kLight;
    {
        std::lock_guard<std::mutex> lk(S->m);
        if (S->fatal != AGP_OK) {
            delete q;
            return fail(S->fatal, "server stopped after a device error");
        }
        q->ticket = S->next_ticket++;
        S->all[q->ticket] = q;
        q->in_queue = true;
        ++S->queued;
        ++S->queued_pool[q->pool];
        S->queue[q->pool].push_back(q);
        S->cls[cc].push_back(q);
        q->refs = 2;
        if (q->r.deadline_us > 0) {
            S->with_deadline.push_back(q);
            ++q->refs;
        }
    }
    S->cv_work.notify_one();
    *ticket = q->ticket;
    return AGP_OK;
}

static void fill_result(const agp_server_s *S, const Request *q, agp_result_t *out)
{
    out->status = q->status;
    out->on_host = q->h_out ? 1 : 0;
    out->pi = q->h_out ? q->h_out : q->d_out;
    out->n = S->g->n;
    out->cols = q->r.source >= 0 ? 1 : q->r.cols;
    out->queue_us = q->t_admit > 0 ? q->t_admit - q->t_submit : q->t_done - q->t_submit;
    out->latency_us = q->t_done - q->t_submit;
}

int serve_poll(agp_server_s *S, uint64_t ticket, agp_result_t *out)
{
    if (!S || !out) return fail(AGP_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->m);
    auto it = S->all.find(ticket);
    if (it == S->all.end() || it->second->released) return fail(AGP_EINVAL, "unknown ticket");
    if (!it->second->done) return AGP_EAGAIN;
    fill_result(S, it->second, out);
    return AGP_OK;
}

int serve_wait(agp_server_s *S, uint64_t ticket, int64_t timeout_us, agp_result_t *out)
{
    if (!S || !out) return fail(AGP_EINVAL, "NULL argument");
    std::unique_lock<std::mutex> lk(S->m);
    auto it = S->all.find(ticket);
    if (it == S->all.end() || it->second->released) return fail(AGP_EINVAL, "unknown ticket");
    Request *q = it->second;
    auto ready = [&] { return q->done; };
    if (timeout_us < 0) {
        S->cv_done.wait(lk, ready);
    } else if (!S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
        return AGP_ETIMEDOUT;
    }
    fill_result(S, q, out);
    return AGP_OK;
}

int serve_next(agp_server_s *S, int64_t timeout_us, uint64_t *ticket, agp_result_t *out)
{
    if (!S || !ticket || !out) return fail(AGP_EINVAL, "NULL argument");
    std::unique_lock<std::mutex> lk(S->m);
    const auto until = std::chrono::steady_clock::now() + std::chrono::microseconds(std::max<int64_t>(0, timeout_us));
    while (true) {
        // requests released before they were reported are skipped
        while (!S->done_q.empty()) {
            const uint64_t t = S->done_q.front();
            S->done_q.pop_front();
            auto it = S->all.find(t);
            if (it == S->all.end() || it->second->released) continue;
            *ticket = t;
            fill_result(S, it->second, out);
            return AGP_OK;
        }
        if (timeout_us < 0) {
            S->cv_done.wait(lk);
        } else if (S->cv_done.wait_until(lk, until) == std::cv_status::timeout && S->done_q.empty()) {
            return AGP_ETIMEDOUT;
        }
    }
}

int serve_release(agp_server_s *S, uint64_t ticket)
{
    if (!S) return fail(AGP_EINVAL, "NULL argument");
    Request *q = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->m);
        auto it = S->all.find(ticket);
        if (it == S->all.end()) return fail(AGP_EINVAL, "unknown ticket");
        if (!it->second->done) return fail(AGP_EINVAL, "request still pending");
        q = it->second;
        S->all.erase(it);
        if (q->counted)
            S->result_bytes[q->pool] -= (int64_t)(q->r.source >= 0 ? 1 : q->r.cols) * S->g->n * (int64_t)sizeof(float);
    }
    free_result(S, q);  // nobody deletes q meanwhile: it is not a zombie yet
    {
        std::lock_guard<std::mutex> lk(S->m);
        if (q->refs > 0) {
            q->zombie = true;  // queue entries remain: deleted with the last one
            q = nullptr;
        }
    }
    delete q;
    S->cv_work.notify_one();
    return AGP_OK;
}

int serve_cancel(agp_server_s *S, uint64_t ticket)
{
    if (!S) return fail(AGP_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->m);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return fail(AGP_EINVAL, "unknown ticket");
    Request *q = it->second;
    if (q->done) return AGP_OK;
    q->cancelled = true;
    if (q->in_queue) {  // still waiting: finished now, its queue entries are dropped lazily
        dequeue(S, q);
        finish(S, q, AGP_ECANCELED);
        return AGP_OK;
    }
    S->cv_work.notify_one();  // in flight: the server thread stops its lanes before the next sweep
    return AGP_OK;
}

int serve_stats(agp_server_s *S, int64_t *completed, int64_t *sweeps, int32_t *lanes_active, int32_t *queued)
{
    if (!S) return fail(AGP_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->m);
    if (completed) *completed = S->completed;
    if (sweeps) *sweeps = S->sweeps;
    if (lanes_active) *lanes_active = S->pool[0].active_lanes + S->pool[1].active_lanes;
    if (queued) *queued = (int32_t)std::min<int64_t>(S->queued, INT32_MAX);
    return AGP_OK;
}

int serve_destroy(agp_server_s *S)
{
    if (!S) return AGP_OK;
    {
        std::lock_guard<std::mutex> lk(S->m);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    for (Pool &P : S->pool)
        if (P.stream) cudaStreamSynchronize(P.stream);
    {
        std::lock_guard<std::mutex> lk(S->m);
        drain_queues(S);  // released requests go with their last queue entry
        for (auto &kv : S->all) {
            if (!kv.second->done) finish(S, kv.second, AGP_ECANCELED);
            free_result(S, kv.second, true);
            delete kv.second;
        }
        S->all.clear();
    }
    for (Pool &P : S->pool) destroy_pool(P);
    for (auto &kv : S->free_dev)
        for (void *p : kv.second) cudaFree(p);
    for (auto &kv : S->free_host)
        for (void *p : kv.second) cudaFreeHost(p);
    cudaFree(S->fifo_stage);
    delete S;
    return AGP_OK;
}

}  // namespace agp
