// tune.cu -- autotuner of the wave width (lanes propagated together) and of the group width (lanes
// whose residues are interleaved, so that one row walk and one vector reduction serve them), with a
// file cache.
//
// The wave width trades parallelism (more lanes per launch) against L2 residency of the lanes'
// residue vectors, which receive random reductions; the group width trades shared row walks and
// fewer, wider reductions against longer per-item work. The best pair depends on the graph and on
// the query mix, so it is measured: each candidate runs the caller's batch twice and the second run
// is timed with CUDA events on the caller's stream.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "agp_internal.cuh"

namespace agp {
namespace {

std::string signature(const agp_graph_s *g, const agp_params_t *p, int32_t n_params, int32_t Q)
{
    std::ostringstream k;
    k << "n" << g->n << "_m" << g->nnz << "_d" << g->max_deg << "_Q" << Q;
    for (int i = 0; i < n_params && i < 4; ++i)
        k << "_k" << p[i].kind << "L" << p[i].L << "e" << p[i].eps << "a" << p[i].a << "b" << p[i].b;
    return k.str();
}

bool cache_lookup(const std::string &key, int *lanes, int *width)
{
    const char *path = std::getenv("AGP_TUNE_CACHE");
    if (!path || !*path) return false;
    std::ifstream f(path);
    std::string k;
    int v, w;
    double ms;
    while (f >> k >> v >> w >> ms)
        if (k == key) {
            *lanes = v;
            *width = w;
            return true;
        }
    return false;
}

void cache_store(const std::string &key, int lanes, int width, double ms)
{
    const char *path = std::getenv("AGP_TUNE_CACHE");
    if (!path || !*path) return;
    std::ofstream f(path, std::ios::app);
    f << key << " " << lanes << " " << width << " " << ms << "\n";
}

}  // namespace

int autotune(agp_graph_s *g, const agp_params_t *params, int32_t n_params, int32_t Q, const int64_t *x_off,
             const int32_t *x_idx, const float *x_val, float *pi_out, int64_t ld_out, uint32_t flags,
             const int32_t *candidates, int32_t n_candidates, int32_t *best_lanes, int32_t *best_width,
             double *best_ms, cudaStream_t s)
{
    if (!g) return fail(AGP_EINVAL, "graph is NULL");
    if (!(flags & AGP_OUTPUT_ON_DEVICE)) return fail(AGP_EINVAL, "agp_autotune needs AGP_OUTPUT_ON_DEVICE");
    if (flags & (AGP_PLAIN | AGP_COLLECT_STATS | AGP_PROFILE)) return fail(AGP_EINVAL, "agp_autotune: only the batched path is tuned");
    const std::string key = signature(g, params, n_params, Q) + "_v2";
    int cached = 0, cached_w = 0;
    if (cache_lookup(key, &cached, &cached_w) && cached > 0) {
        g->wave_lanes = cached;
        g->group_width = cached_w;
        if (best_lanes) *best_lanes = cached;
        if (best_width) *best_width = cached_w;
        if (best_ms) *best_ms = -1.0;
        return AGP_OK;
    }
    std::vector<int32_t> cand;
    if (candidates && n_candidates > 0) {
        cand.assign(candidates, candidates + n_candidates);
    } else {
        for (int c = 1; c <= 2 * std::max(Q, 1); c *= 2) cand.push_back(c);
    }
    cudaEvent_t e0, e1;
    AGP_CUDA_TRY(cudaEventCreate(&e0));
    AGP_CUDA_TRY(cudaEventCreate(&e1));
    int best = -1, best_w = 0;
    float best_t = 0.f;
    int rc = AGP_OK;
    const int32_t saved = g->wave_lanes, saved_w = g->group_width;
    for (int32_t c : cand) {
        if (c < 1) continue;
        for (int w : {1, 2, 4}) {
            if (c % w != 0) continue;
            g->wave_lanes = c;
            g->group_width = w;
            rc = query_batch(g, params, n_params, Q, x_off, x_idx, x_val, pi_out, ld_out, flags, nullptr, s);
            if (rc != AGP_OK) break;
            cudaEventRecord(e0, s);
            rc = query_batch(g, params, n_params, Q, x_off, x_idx, x_val, pi_out, ld_out, flags, nullptr, s);
            if (rc != AGP_OK) break;
            cudaEventRecord(e1, s);
            float t = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
                rc = fail(AGP_ECUDA, "agp_autotune: event timing failed");
                break;
            }
            if (best < 0 || t < best_t) {
                best = c;
                best_w = w;
                best_t = t;
            }
        }
        if (rc != AGP_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != AGP_OK || best < 0) {
        g->wave_lanes = saved;
        g->group_width = saved_w;
        return rc != AGP_OK ? rc : fail(AGP_EINVAL, "agp_autotune: no valid candidate");
    }
    g->wave_lanes = best;
    g->group_width = best_w;
    cache_store(key, best, best_w, best_t);
    if (best_lanes) *best_lanes = best;
    if (best_width) *best_width = best_w;
    if (best_ms) *best_ms = best_t;
    return AGP_OK;
}

}  // namespace agp
