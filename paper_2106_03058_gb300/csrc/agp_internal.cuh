// agp_internal.cuh -- shared declarations of the CUDA library (not part of the public ABI).
//
// Notation follows the paper (Wang et al., KDD'21): a, b Laplacian parameters, w_i weights,
// Y_i = sum_{k>=i} w_k (Def. 3.1), r^(i) residue, pi reserve/estimate, eps error parameter.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/agp.h"

namespace agp {

// ---------------------------------------------------------------- error plumbing
void set_error_detail(const std::string &msg);
int fail(int code, const std::string &msg);

#define AGP_CUDA_TRY(expr)                                                                   \
    do {                                                                                     \
        cudaError_t _e = (expr);                                                             \
        if (_e != cudaSuccess)                                                               \
            return ::agp::fail(AGP_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)

#define AGP_TRY(expr)                    \
    do {                                 \
        int _rc = (expr);                \
        if (_rc != AGP_OK) return _rc;   \
    } while (0)

// ---------------------------------------------------------------- launch geometry
// Grid-stride kernels use a multiple of the SM count (152 on GB300, read from the device) so that
// every SM gets the same number of resident blocks.
constexpr int kBlock = 256;
// SMs of the current device (cudaDevAttrMultiProcessorCount, cached per device ordinal).
int sm_count();
// Grid of the grid-stride kernels: 8 blocks of kBlock threads per SM.
inline int grid_stride_blocks() { return 8 * sm_count(); }

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11): ten rounds
// of (hi0,lo0) = M0*c0, (hi1,lo1) = M1*c2, c' = (hi1^c1^k0, lo1, hi0^c3^k1, lo0), with the key
// advanced by the Weyl increments before every round after the first.
struct Philox4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return Philox4{c0, c1, c2, c3};
}

// 32 random bits -> uniform in the open interval (0, 1).
__device__ __forceinline__ float u01_open(uint32_t bits)
{
    return ((float)(bits >> 8) + 0.5f) * (1.0f / 16777216.0f);
}

// ---------------------------------------------------------------- graph
struct DevGraph {
    int64_t n;
    int64_t nnz;
    const int64_t *rowptr;  // n+1
    const int32_t *colidx;  // nnz, each row in ascending (d_v, v)
    const int32_t *deg;     // n
};

struct Workspace;  // query work buffers (propagate.cu)
struct ServeState; // serving (serve.cu)

}  // namespace agp

struct agp_server_s;

struct agp_graph_s {
    int device = 0;
    int64_t n = 0, nnz = 0;
    int32_t max_deg = 0;
    int directed = 0;              // 1: rows are out-neighbour lists, deg out-degrees (AGP_DIRECTED);
                                   // 2: rows are in-neighbour lists, deg out-degrees (AGP_DIRECTED_IN)
    int ubits = 1;                 // bits of a node id inside a packed (lane, node) item
    int64_t *rowptr = nullptr;
    int32_t *colidx = nullptr;
    int32_t *deg = nullptr;
    int64_t mem_budget = 0;        // 0 = default
    int32_t wave_lanes = 0;        // lanes in flight per wave, 0 = automatic (L2 residency)
    int32_t group_width = 0;       // lanes per residue group (1, 2, 4), 0 = automatic
    agp::Workspace *ws = nullptr;
    agp::Workspace *ws2 = nullptr; // second workspace: two waves in flight on two streams
    agp::Workspace *ws_plain = nullptr;  // one-lane workspace of the plain path
    cudaStream_t side = nullptr;   // stream of the second wave slot
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_wave[2] = {nullptr, nullptr};  // end of the last wave on stream k (result copies)
    void *in_stage = nullptr;      // device staging of per-call inputs (grown on demand)
    size_t in_bytes = 0;
    double prof_ms[5] = {0, 0, 0, 0, 0};   // AGP_PROFILE: device time per level-loop step
    int64_t prof_launches[5] = {0, 0, 0, 0, 0};
    int64_t kernel_launches = 0;           // all kernels launched for this graph
    std::vector<cudaEvent_t> wave_ev;      // AGP_QUERY_TIMES: call start + one event per wave
    int32_t *row_list[3] = {nullptr, nullptr, nullptr};  // rows by length class (feature tiles, pull levels)
    int64_t row_count[3] = {0, 0, 0};
    int32_t column_tile = 0;               // columns per tile of exact feature propagation, 0 = automatic
    int32_t pull_shift = -1;               // a lane pulls a level whose frontier volume (sum of d_u) is
                                           // >= nnz >> pull_shift (undirected graphs); < 0: never
    void *tile_buf = nullptr;              // residue blocks of the column tiles (grown on demand)
    size_t tile_bytes = 0;
    agp::DevGraph dev() const { return agp::DevGraph{n, nnz, rowptr, colidx, deg}; }
};

namespace agp {
int build_graph(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, uint32_t flags,
                int device, cudaStream_t stream, agp_graph_s **out);
void free_workspace(Workspace *ws);
int katz_beta(agp_graph_s *g, double fraction, int iters, double tol, double *beta,
              double *lambda1, cudaStream_t stream);
int katz_lambda_noalloc(int64_t n, const int64_t *rowptr, const int32_t *colidx, int iters, double tol,
                        double *lambda1, cudaStream_t stream);
int sweep(agp_graph_s *g, const float *pi, int32_t *order_out, double *phi_out, int64_t *best_size, double *best_phi,
          int64_t *swept, cudaStream_t s);
int topk(const float *pi, int64_t n, int64_t ld, int32_t Q, int32_t k, float *val, int32_t *idx, int64_t ldo,
         cudaStream_t s);
int compare(const float *pi_est, const float *pi_ref, int64_t n, const int32_t *deg, int32_t k, double *max_error,
            double *precision_at_k, cudaStream_t s);
int coefficients(const agp_params_t *p, double *keep, double *push, double *y0, int device, cudaStream_t s);
int validate_params(const agp_params_t &p);
int threshold(agp_graph_s *g, double a, double eps, int64_t count, const int32_t *nodes,
              const float *c, int32_t *k_out, cudaStream_t stream);
int wave_lanes(const agp_graph_s *g);
int autotune(agp_graph_s *g, const agp_params_t *params, int32_t n_params, int32_t Q, const int64_t *x_off,
             const int32_t *x_idx, const float *x_val, float *pi_out, int64_t ld_out, uint32_t flags,
             const int32_t *candidates, int32_t n_candidates, int32_t *best_lanes, int32_t *best_width,
             double *best_ms, cudaStream_t s);
int query_batch(agp_graph_s *g, const agp_params_t *params, int32_t n_params, int32_t Q,
                const int64_t *x_off, const int32_t *x_idx, const float *x_val, float *pi_out,
                int64_t ld_out, uint32_t flags, agp_stats_t *stats, cudaStream_t stream);
int query_dense(agp_graph_s *g, const agp_params_t *params, int32_t n_params, int32_t Q, const void *X, int64_t ldx,
                float *pi_out, int64_t ld_out, uint32_t flags, agp_stats_t *stats, cudaStream_t stream);
int feature_exact_tiled(agp_graph_s *g, const agp_params_t *p, const uint16_t *X, int64_t d, int64_t ldx, float *Z,
                        int64_t ldz, cudaStream_t s);
int column_tile(const agp_graph_s *g);
int ensure_row_lists(agp_graph_s *g, cudaStream_t s);
int exponent_mode(double p);
int feature_propagate(agp_graph_s *g, const agp_params_t *params, const uint16_t *X, int64_t d,
                      int64_t ldx, float *Z, int64_t ldz, uint32_t flags, cudaStream_t stream);

// serving (serve.cu)
int serve_create(agp_graph_s *g, const agp_serve_config_t *cfg, agp_server_s **out);
int serve_submit(agp_server_s *s, const agp_request_t *req, uint64_t *ticket);
int serve_poll(agp_server_s *s, uint64_t ticket, agp_result_t *out);
int serve_wait(agp_server_s *s, uint64_t ticket, int64_t timeout_us, agp_result_t *out);
int serve_next(agp_server_s *s, int64_t timeout_us, uint64_t *ticket, agp_result_t *out);
int serve_release(agp_server_s *s, uint64_t ticket);
int serve_cancel(agp_server_s *s, uint64_t ticket);
int serve_stats(agp_server_s *s, int64_t *completed, int64_t *sweeps, int32_t *lanes_active, int32_t *queued);
int serve_destroy(agp_server_s *s);

// device-wide primitives (sort_scan.cu)
// Exclusive prefix sum of `count` uint32 flags into int64 offsets; total written to *d_total.
int exclusive_scan_u32(const uint32_t *in, int64_t *out, int64_t count, int64_t *d_total,
                       void *scratch, size_t scratch_bytes, cudaStream_t stream);
size_t exclusive_scan_scratch_bytes(int64_t count);
// Stable LSD radix sort of 64-bit keys (optionally carrying 32-bit values) on key bits
// [0, key_bits). Buffers are ping-ponged; the result ends in (*keys_out, *vals_out), which is
// one of the two buffer pairs given.
int radix_sort_u64(uint64_t *keys_a, uint64_t *keys_b, uint32_t *vals_a, uint32_t *vals_b,
                   int64_t count, int key_bits, uint64_t **keys_out, uint32_t **vals_out,
                   void *scratch, size_t scratch_bytes, cudaStream_t stream);
size_t radix_sort_scratch_bytes(int64_t count);

}  // namespace agp
