// api.cu -- the extern "C" entry points of include/agp.h, error reporting and the Katz bound.
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "lanes.cuh"

namespace agp {

namespace {
thread_local std::string g_detail;
}

void set_error_detail(const std::string &msg) { g_detail = msg; }

int fail(int code, const std::string &msg)
{
    g_detail = msg;
    return code;
}

int sm_count()
{
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 152;
    }
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v <= 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            v = 152;
        }
        cache[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

// ---- Katz spectral bound: lambda_1(A) by FP64 power iteration on A + I --------------------------
namespace {

__global__ void k_spmv_shift(DevGraph g, const double *x, double *y)
{
    // one warp per row: y(u) = x(u) + sum_{v in N_u} x(v)
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; u < g.n; u += nw) {
        double s = 0.0;
        for (int64_t e = g.rowptr[u] + lane; e < g.rowptr[u + 1]; e += 32) s += x[g.colidx[e]];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) y[u] = x[u] + s;
    }
}

__global__ void k_dots(const double *x, const double *y, int64_t n, double *acc)
{
    __shared__ double s_yy[kBlock / 32], s_xy[kBlock / 32];
    double yy = 0.0, xy = 0.0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        yy += y[u] * y[u];
        xy += x[u] * y[u];
    }
    for (int o = 16; o > 0; o >>= 1) {
        yy += __shfl_down_sync(0xffffffffu, yy, o);
        xy += __shfl_down_sync(0xffffffffu, xy, o);
    }
    if ((threadIdx.x & 31) == 0) { s_yy[threadIdx.x >> 5] = yy; s_xy[threadIdx.x >> 5] = xy; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) { a += s_yy[w]; b += s_xy[w]; }
        atomicAdd(&acc[0], a);
        atomicAdd(&acc[1], b);
    }
}

__global__ void k_fill(double *x, int64_t n, double v)
{
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) x[u] = v;
}

__global__ void k_scale(const double *y, double *x, int64_t n, const double *acc)
{
    const double nrm = sqrt(acc[0]);
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) x[u] = y[u] * inv;
}

}  // namespace

int katz_beta(agp_graph_s *g, double fraction, int iters, double tol, double *beta, double *lambda1,
              cudaStream_t s)
{
    if (!g) return fail(AGP_EINVAL, "graph is NULL");
    if (!(fraction > 0.0) || iters < 1 || !(tol >= 0.0)) return fail(AGP_EINVAL, "need fraction > 0, iters >= 1, tol >= 0");
    AGP_CUDA_TRY(cudaSetDevice(g->device));
    const int64_t n = g->n;
    if (n == 0) return fail(AGP_EINVAL, "empty graph");
    double *x = nullptr, *y = nullptr, *acc = nullptr;
    auto cleanup = [&]() { cudaFree(x); cudaFree(y); cudaFree(acc); };
    if (cudaMalloc(&x, sizeof(double) * n) != cudaSuccess || cudaMalloc(&y, sizeof(double) * n) != cudaSuccess ||
        cudaMalloc(&acc, sizeof(double) * 2) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return fail(AGP_ENOMEM, "katz_beta: device allocation");
    }
    k_fill<<<grid_stride_blocks(), kBlock, 0, s>>>(x, n, 1.0 / std::sqrt((double)n));
    double lam = 0.0, prev = 0.0, h[2];
    int rc = AGP_OK;
    for (int it = 0; it < iters; ++it) {
        k_spmv_shift<<<grid_stride_blocks(), kBlock, 0, s>>>(g->dev(), x, y);
        cudaMemsetAsync(acc, 0, sizeof(double) * 2, s);
        k_dots<<<grid_stride_blocks(), kBlock, 0, s>>>(x, y, n, acc);
        k_scale<<<grid_stride_blocks(), kBlock, 0, s>>>(y, x, n, acc);
        if (cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            rc = fail(AGP_ECUDA, std::string("katz_beta: ") + cudaGetErrorString(cudaGetLastError()));
            break;
        }
        prev = lam;
        lam = h[1] - 1.0;  // Rayleigh quotient of A + I at the unit iterate, minus the shift
        if (it > 0 && std::fabs(lam - prev) <= tol * std::fabs(lam)) break;
    }
    cleanup();
    if (rc != AGP_OK) return rc;
    if (!(lam > 0.0)) return fail(AGP_EINVAL, "graph has no edges (lambda_1 = 0)");
    if (lambda1) *lambda1 = lam;
    if (beta) *beta = fraction / lam;
    return AGP_OK;
}

// ---- lambda_1 without allocations ----------------------------------------------------------------
// Some callers cannot allocate device memory once they are running: processes whose device memory
// is owned by another allocator (a framework's caching pool or a fixed arena that must account for
// every byte), and latency-critical services that avoid cudaMalloc/cudaFree because those calls
// synchronise the device and stall the other streams. For them, agp_katz_lambda_noalloc runs the
// same FP64 power iteration as agp_katz_beta on a CSR the caller owns, with its two iterate vectors
// and accumulators in the fixed device array below instead of freshly allocated buffers.
//
// The array is part of the loaded library: every GPU that loads it holds these 64 MiB until the
// process exits. Host code must not use the symbol as an address (on the host it names a stand-in
// variable); the device address is looked up with cudaGetSymbolAddress on every call, with the
// caller's device current. The lookup allocates nothing, and doing it per call (rather than caching
// it per device ordinal) keeps the address right after a device reset or when the caller has made
// another context current on the same ordinal.
constexpr int64_t kNoAllocMaxNodes = 4194304;  // 2^22 nodes: x and y of 32 MiB each
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocMaxNodes + 64];

namespace {

int noalloc_scratch(double **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return fail(AGP_ECUDA, std::string("cudaGetSymbolAddress(no-alloc scratch): ") + cudaGetErrorString(e));
    *out = (double *)p;
    return AGP_OK;
}

}  // namespace

int katz_lambda_noalloc(int64_t n, const int64_t *rowptr, const int32_t *colidx, int iters, double tol,
                        double *lambda1, cudaStream_t s)
{
    if (n <= 0) return fail(AGP_EINVAL, "agp_katz_lambda_noalloc: n must be >= 1");
    if (n > kNoAllocMaxNodes)
        return fail(AGP_EINVAL, "agp_katz_lambda_noalloc: n = " + std::to_string(n) +
                                    " exceeds the fixed scratch of 4194304 nodes; use agp_katz_beta");
    if (!rowptr || !colidx || !lambda1) return fail(AGP_EINVAL, "agp_katz_lambda_noalloc: NULL argument");
    if (iters < 1 || !(tol >= 0.0)) return fail(AGP_EINVAL, "agp_katz_lambda_noalloc: need iters >= 1, tol >= 0");
    double *base = nullptr;
    AGP_TRY(noalloc_scratch(&base));
    double *x = base, *y = base + kNoAllocMaxNodes, *acc = base + 2 * kNoAllocMaxNodes;
    DevGraph g{n, 0, rowptr, colidx, nullptr};
    // the scratch keeps the previous call's contents: x is re-initialised, acc cleared per step
    k_fill<<<grid_stride_blocks(), kBlock, 0, s>>>(x, n, 1.0 / std::sqrt((double)n));
    AGP_CUDA_TRY(cudaGetLastError());
    double lam = 0.0, prev = 0.0, h[2] = {0.0, 0.0};
    for (int it = 0; it < iters; ++it) {
        k_spmv_shift<<<grid_stride_blocks(), kBlock, 0, s>>>(g, x, y);
        AGP_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(double) * 2, s));
        k_dots<<<grid_stride_blocks(), kBlock, 0, s>>>(x, y, n, acc);
        k_scale<<<grid_stride_blocks(), kBlock, 0, s>>>(y, x, n, acc);
        AGP_CUDA_TRY(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
        AGP_CUDA_TRY(cudaStreamSynchronize(s));
        prev = lam;
        lam = h[1] - 1.0;  // Rayleigh quotient of A + I at the unit iterate, minus the shift
        if (it > 0 && std::fabs(lam - prev) <= tol * std::fabs(lam)) break;
    }
    if (!(lam > 0.0)) return fail(AGP_EINVAL, "agp_katz_lambda_noalloc: graph has no edges (lambda_1 = 0)");
    *lambda1 = lam;
    return AGP_OK;
}

}  // namespace agp

// ------------------------------------------------------------------------------------ C ABI
extern "C" {

const char *agp_strerror(int code)
{
    switch (code) {
    case AGP_OK: return "AGP_OK";
    case AGP_EINVAL: return "AGP_EINVAL";
    case AGP_ENOMEM: return "AGP_ENOMEM";
    case AGP_ECUDA: return "AGP_ECUDA";
    case AGP_EBUDGET: return "AGP_EBUDGET";
    case AGP_EAGAIN: return "AGP_EAGAIN";
    case AGP_ETIMEDOUT: return "AGP_ETIMEDOUT";
    case AGP_ECANCELED: return "AGP_ECANCELED";
    case AGP_EINTERNAL: return "AGP_EINTERNAL";
    default: return "AGP_UNKNOWN";
    }
}

const char *agp_last_error_detail(void) { return agp::g_detail.c_str(); }

int agp_version(void) { return 10000; }

int agp_build_graph(int64_t n, int64_t n_edges, const int32_t *src, const int32_t *dst, uint32_t flags,
                    int device, void *stream, agp_graph_t *out)
{
    return agp::build_graph(n, n_edges, src, dst, flags, device, (cudaStream_t)stream, out);
}

int agp_graph_info(agp_graph_t g, int64_t *n, int64_t *nnz, const int64_t **rowptr, const int32_t **colidx,
                   const int32_t **deg)
{
    if (!g) return agp::fail(AGP_EINVAL, "graph is NULL");
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    if (rowptr) *rowptr = g->rowptr;
    if (colidx) *colidx = g->colidx;
    if (deg) *deg = g->deg;
    return AGP_OK;
}

int agp_graph_destroy(agp_graph_t g)
{
    if (!g) return AGP_OK;
    cudaSetDevice(g->device);
    cudaDeviceSynchronize();
    agp::free_workspace(g->ws);
    agp::free_workspace(g->ws2);
    agp::free_workspace(g->ws_plain);
    if (g->side) cudaStreamDestroy(g->side);
    if (g->ev_fork) cudaEventDestroy(g->ev_fork);
    if (g->ev_join) cudaEventDestroy(g->ev_join);
    for (int k = 0; k < 2; ++k)
        if (g->ev_wave[k]) cudaEventDestroy(g->ev_wave[k]);
    for (cudaEvent_t e : g->wave_ev) cudaEventDestroy(e);
    for (int c = 0; c < 3; ++c) cudaFree(g->row_list[c]);
    cudaFree(g->tile_buf);
    cudaFree(g->rowptr);
    cudaFree(g->colidx);
    cudaFree(g->deg);
    cudaFree(g->in_stage);
    delete g;
    return AGP_OK;
}

int agp_graph_set_memory_budget(agp_graph_t g, int64_t bytes)
{
    if (!g) return agp::fail(AGP_EINVAL, "graph is NULL");
    if (bytes < 0) return agp::fail(AGP_EINVAL, "budget < 0");
    g->mem_budget = bytes;
    return AGP_OK;
}

int agp_graph_set_wave_lanes(agp_graph_t g, int32_t lanes)
{
    if (!g) return agp::fail(AGP_EINVAL, "graph is NULL");
    if (lanes < 0) return agp::fail(AGP_EINVAL, "lanes < 0");
    g->wave_lanes = lanes;
    return AGP_OK;
}

int agp_autotune(agp_graph_t g, const agp_params_t *params, int32_t n_params, int32_t Q, const int64_t *x_off,
                 const int32_t *x_idx, const float *x_val, float *pi_out, int64_t ld_out, uint32_t flags,
                 const int32_t *candidates, int32_t n_candidates, int32_t *best_lanes, int32_t *best_width,
                 double *best_ms, void *stream)
{
    return agp::autotune(g, params, n_params, Q, x_off, x_idx, x_val, pi_out, ld_out, flags, candidates, n_candidates,
                         best_lanes, best_width, best_ms, (cudaStream_t)stream);
}

int agp_graph_set_pull_threshold(agp_graph_t g, int32_t shift)
{
    if (!g) return agp::fail(AGP_EINVAL, "graph is NULL");
    if (shift < -1 || shift > 62) return agp::fail(AGP_EINVAL, "pull threshold shift must be in [-1, 62]");
    // workspaces made while pulling was off have no c(u) blocks: they are rebuilt at the next call
    const bool need_c = shift >= 0 && !g->directed;
    if (need_c && ((g->ws && !g->ws->C) || (g->ws2 && !g->ws2->C) || (g->ws_plain && !g->ws_plain->C)))
        agp::drop_workspace(g);
    g->pull_shift = shift;
    return AGP_OK;
}

int agp_graph_set_column_tile(agp_graph_t g, int32_t columns)
{
    if (!g) return agp::fail(AGP_EINVAL, "graph is NULL");
    if (columns != 0 && columns != 8 && columns != 16 && columns != 32)
        return agp::fail(AGP_EINVAL, "column tile must be 0, 8, 16 or 32");
    g->column_tile = columns;
    return AGP_OK;
}

int agp_graph_set_group_width(agp_graph_t g, int32_t width)
{
    if (!g) return agp::fail(AGP_EINVAL, "graph is NULL");
    if (width != 0 && width != 1 && width != 2 && width != 4) return agp::fail(AGP_EINVAL, "group width must be 0, 1, 2 or 4");
    g->group_width = width;
    return AGP_OK;
}

int agp_query_batch(agp_graph_t g, const agp_params_t *params, int32_t n_params, int32_t Q, const int64_t *x_off,
                    const int32_t *x_idx, const float *x_val, float *pi_out, int64_t ld_out, uint32_t flags,
                    agp_stats_t *stats, void *stream)
{
    if (flags & agp::kOffsetsOnHost) return agp::fail(AGP_EINVAL, "unknown flag");
    return agp::query_batch(g, params, n_params, Q, x_off, x_idx, x_val, pi_out, ld_out, flags, stats,
                            (cudaStream_t)stream);
}

int agp_query(agp_graph_t g, const agp_params_t *params, int64_t x_nnz, const int32_t *x_idx, const float *x_val,
              float *pi_out, uint32_t flags, agp_stats_t *stats, void *stream)
{
    if (!g) return agp::fail(AGP_EINVAL, "graph is NULL");
    if (x_nnz < 0) return agp::fail(AGP_EINVAL, "x_nnz < 0");
    if (flags & agp::kOffsetsOnHost) return agp::fail(AGP_EINVAL, "unknown flag");
    // the two offsets are known here: they are passed from the host even when the signal is on the
    // device (no per-call device allocation or synchronisation)
    if (flags & AGP_INPUT_ON_DEVICE) flags |= agp::kOffsetsOnHost;
    const int64_t h_off[2] = {0, x_nnz};
    return agp::query_batch(g, params, 1, 1, h_off, x_idx, x_val, pi_out, g->n, flags, stats, (cudaStream_t)stream);
}

int agp_query_dense(agp_graph_t g, const agp_params_t *params, int32_t n_params, int32_t Q, const void *X, int64_t ldx,
                    float *pi_out, int64_t ld_out, uint32_t flags, agp_stats_t *stats, void *stream)
{
    return agp::query_dense(g, params, n_params, Q, X, ldx, pi_out, ld_out, flags, stats, (cudaStream_t)stream);
}

int agp_feature_propagate(agp_graph_t g, const agp_params_t *params, const uint16_t *X, int64_t d, int64_t ldx,
                          float *Z, int64_t ldz, uint32_t flags, void *stream)
{
    return agp::feature_propagate(g, params, X, d, ldx, Z, ldz, flags, (cudaStream_t)stream);
}

int agp_katz_beta(agp_graph_t g, double fraction, int32_t iters, double tol, double *beta, double *lambda1,
                  void *stream)
{
    return agp::katz_beta(g, fraction, iters, tol, beta, lambda1, (cudaStream_t)stream);
}

int agp_profile_read(agp_graph_t g, double *ms, int64_t *launches, int64_t *kernel_launches, int reset)
{
    if (!g) return agp::fail(AGP_EINVAL, "graph is NULL");
    for (int k = 0; k < 5; ++k) {
        if (ms) ms[k] = g->prof_ms[k];
        if (launches) launches[k] = g->prof_launches[k];
    }
    if (kernel_launches) *kernel_launches = g->kernel_launches;
    if (reset) {
        for (int k = 0; k < 5; ++k) { g->prof_ms[k] = 0.0; g->prof_launches[k] = 0; }
        g->kernel_launches = 0;
    }
    return AGP_OK;
}

int agp_katz_lambda_noalloc(int64_t n, const int64_t *rowptr, const int32_t *colidx, int32_t iters, double tol,
                            double *lambda1, void *stream)
{
    return agp::katz_lambda_noalloc(n, rowptr, colidx, iters, tol, lambda1, (cudaStream_t)stream);
}

int agp_coefficients(const agp_params_t *params, double *keep, double *push, double *y0, int device, void *stream)
{
    return agp::coefficients(params, keep, push, y0, device, (cudaStream_t)stream);
}

int agp_sweep(agp_graph_t g, const float *pi, int32_t *order, double *phi, int64_t *best_size, double *best_phi,
              int64_t *swept, void *stream)
{
    return agp::sweep(g, pi, order, phi, best_size, best_phi, swept, (cudaStream_t)stream);
}

int agp_topk(const float *pi, int64_t n, int64_t ld, int32_t Q, int32_t k, float *val, int32_t *idx, int64_t ldo,
             void *stream)
{
    return agp::topk(pi, n, ld, Q, k, val, idx, ldo, (cudaStream_t)stream);
}

int agp_compare(const float *pi_est, const float *pi_ref, int64_t n, const int32_t *deg, int32_t k, double *max_error,
                double *precision_at_k, void *stream)
{
    return agp::compare(pi_est, pi_ref, n, deg, k, max_error, precision_at_k, (cudaStream_t)stream);
}

int agp_threshold(agp_graph_t g, double a, double eps, int64_t count, const int32_t *nodes, const float *c,
                  int32_t *k_out, void *stream)
{
    return agp::threshold(g, a, eps, count, nodes, c, k_out, (cudaStream_t)stream);
}

int agp_serve_create(agp_graph_t g, const agp_serve_config_t *config, agp_server_t *out)
{
    return agp::serve_create(g, config, out);
}
int agp_serve_submit(agp_server_t s, const agp_request_t *req, uint64_t *ticket) { return agp::serve_submit(s, req, ticket); }
int agp_serve_poll(agp_server_t s, uint64_t ticket, agp_result_t *out) { return agp::serve_poll(s, ticket, out); }
int agp_serve_wait(agp_server_t s, uint64_t ticket, int64_t timeout_us, agp_result_t *out)
{
    return agp::serve_wait(s, ticket, timeout_us, out);
}
int agp_serve_next(agp_server_t s, int64_t timeout_us, uint64_t *ticket, agp_result_t *out)
{
    return agp::serve_next(s, timeout_us, ticket, out);
}
int agp_serve_release(agp_server_t s, uint64_t ticket) { return agp::serve_release(s, ticket); }
int agp_serve_cancel(agp_server_t s, uint64_t ticket) { return agp::serve_cancel(s, ticket); }
int agp_serve_stats(agp_server_t s, int64_t *completed, int64_t *sweeps, int32_t *lanes_active, int32_t *queued)
{
    return agp::serve_stats(s, completed, sweeps, lanes_active, queued);
}
int agp_serve_destroy(agp_server_t s) { return agp::serve_destroy(s); }

}  // extern "C"
