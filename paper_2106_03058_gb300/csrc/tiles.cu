// tiles.cu -- exact feature propagation (eps = 0) over column tiles.
//
// At eps = 0 Algorithm 2 pushes every residue to every neighbour: it is Algorithm 1, the truncated
// sum Z = sum_{i<=L} w_i P^i X with P = D^-a A D^-b. For a dense feature matrix every node is in every
// level's frontier, so the level is a sparse-times-dense product. On an undirected graph the rows of
// the CSR are also the columns of A, so the level can pull instead of push: node u reads its
// neighbours' residues and writes its own, with no atomics and one walk of N_u for all columns of a
// tile. The recursion is the lane pipeline's own (Def. 3.1 coefficients):
//     S_i = D^-b R_i,   R_{i+1} = rho_i D^-a A S_i,   Z += keep_{i+1} R_{i+1},   R_0 = X, Z = keep_0 X,
// with keep_i = Y_0 w_i / Y_i and rho_i = Y_{i+1} / Y_i, so R_i = (Y_i / Y_0) P^i X and Z gets w_i P^i X.
// S (already scaled by d^-b) is what neighbours read, so the per-edge work is one gather of T floats.
//
// A tile holds T columns (T = 8, 16 or 32; one column per thread). Its S block, n x T floats, is
// kept small enough to stay in L2 (T = 8 for 2.5M nodes is 80 MB of the 129 MB), so the neighbour
// gathers (T x 4 bytes, one or a few 32-byte sectors) are served by L2 and HBM carries only the CSR
// stream, the S writes and the Z read-modify-write. Rows are split by length into three lists built
// once per graph: short rows (d <= 32) take T threads each, medium rows (d <= 4096) a warp, long rows
// (the hubs of a power-law graph) a block of 8 warps, so no warp waits on a hub.
#include <algorithm>
#include <vector>

#include "lanes.cuh"

namespace agp {
namespace {

constexpr int kShortRow = 32;
constexpr int kMediumRow = 4096;
constexpr int kLongBlock = 256;

__device__ __forceinline__ float deg_scale(int32_t d, int mode)
{
    // d^-p for p in {0, 1, 1/2} (mode 3, general p, is passed in as the precomputed factor table)
    switch (mode) {
    case 0: return 1.f;
    case 1: return d > 0 ? __frcp_rn((float)d) : 0.f;
    default: return d > 0 ? __frcp_rn(__fsqrt_rn((float)d)) : 0.f;
    }
}

struct TileArgs {
    DevGraph g;
    const float *fa, *fb;     // per-node d^-a, d^-b (general exponents), or NULL for modes 0-2
    int a_mode, b_mode;
    const float *S_in;        // [n][T]
    float *S_out;             // [n][T]
    float *Z;                 // caller's Z, columns [c0, c0 + width) of rows of stride ldz
    int64_t ldz;
    int c0, width;            // first column and valid columns of the tile
    float rho, keep;          // rho_i and keep_{i+1}
};

__device__ __forceinline__ float fac_a(const TileArgs &P, int32_t u, int32_t d)
{
    return P.fa ? P.fa[u] : deg_scale(d, P.a_mode);
}
__device__ __forceinline__ float fac_b(const TileArgs &P, int32_t u, int32_t d)
{
    return P.fb ? P.fb[u] : deg_scale(d, P.b_mode);
}

// finish row u: R = rho d_u^-a acc, Z += keep R, S_out = d_u^-b R (thread j holds column j)
template <int T>
__device__ __forceinline__ void finish_row(const TileArgs &P, int32_t u, int j, float acc)
{
    const int32_t d = P.g.deg[u];
    const float R = P.rho * fac_a(P, u, d) * acc;
    if (j < P.width) {
        float *z = P.Z + (int64_t)u * P.ldz + P.c0 + j;
        *z += P.keep * R;
    }
    P.S_out[(size_t)u * T + j] = fac_b(P, u, d) * R;
}

// short rows: T threads per row, 32 / T rows per warp
template <int T>
__global__ void __launch_bounds__(kBlock) k_tile_short(TileArgs P, const int32_t *rows, int64_t count)
{
    const int j = threadIdx.x % T;
    const int64_t sub = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / T;
    const int64_t nsub = (int64_t)gridDim.x * blockDim.x / T;
    for (int64_t r = sub; r < count; r += nsub) {
        const int32_t u = rows[r];
        const int64_t e0 = P.g.rowptr[u], e1 = P.g.rowptr[u + 1];
        float acc = 0.f;
        int64_t e = e0;
        for (; e + 4 <= e1; e += 4) {
            const int32_t v0 = P.g.colidx[e], v1 = P.g.colidx[e + 1], v2 = P.g.colidx[e + 2], v3 = P.g.colidx[e + 3];
            const float s0 = P.S_in[(size_t)v0 * T + j], s1 = P.S_in[(size_t)v1 * T + j];
            const float s2 = P.S_in[(size_t)v2 * T + j], s3 = P.S_in[(size_t)v3 * T + j];
            acc += s0;
            acc += s1;
            acc += s2;
            acc += s3;
        }
        for (; e < e1; ++e) acc += P.S_in[(size_t)P.g.colidx[e] * T + j];
        finish_row<T>(P, u, j, acc);
    }
}

// medium rows: a warp per row, its 32 / T sub-groups take every (32 / T)-th neighbour, then the
// partial sums of the sub-groups are added with shuffles
template <int T>
__global__ void __launch_bounds__(kBlock) k_tile_medium(TileArgs P, const int32_t *rows, int64_t count)
{
    constexpr int G = 32 / T;
    const int lane = threadIdx.x & 31, j = lane % T, gsub = lane / T;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = w; r < count; r += nw) {
        const int32_t u = rows[r];
        const int64_t e0 = P.g.rowptr[u], e1 = P.g.rowptr[u + 1];
        float acc = 0.f;
        int64_t e = e0 + gsub;
        for (; e + 3 * G < e1; e += 4 * G) {
            const int32_t v0 = P.g.colidx[e], v1 = P.g.colidx[e + G], v2 = P.g.colidx[e + 2 * G], v3 = P.g.colidx[e + 3 * G];
            const float s0 = P.S_in[(size_t)v0 * T + j], s1 = P.S_in[(size_t)v1 * T + j];
            const float s2 = P.S_in[(size_t)v2 * T + j], s3 = P.S_in[(size_t)v3 * T + j];
            acc += s0;
            acc += s1;
            acc += s2;
            acc += s3;
        }
        for (; e < e1; e += G) acc += P.S_in[(size_t)P.g.colidx[e] * T + j];
#pragma unroll
        for (int o = T; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (gsub == 0) finish_row<T>(P, u, j, acc);
    }
}

// long rows: a block per row, partial sums of its 8 warps added in shared memory
template <int T>
__global__ void __launch_bounds__(kLongBlock) k_tile_long(TileArgs P, const int32_t *rows, int64_t count)
{
    constexpr int G = kLongBlock / T;  // sub-groups of the block
    __shared__ float part[kLongBlock / 32][T];
    const int t = threadIdx.x, j = t % T, gsub = t / T, lane = t & 31, warp = t >> 5;
    for (int64_t r = blockIdx.x; r < count; r += gridDim.x) {
        const int32_t u = rows[r];
        const int64_t e0 = P.g.rowptr[u], e1 = P.g.rowptr[u + 1];
        float acc = 0.f;
        int64_t e = e0 + gsub;
        for (; e + 3 * G < e1; e += 4 * G) {
            const int32_t v0 = P.g.colidx[e], v1 = P.g.colidx[e + G], v2 = P.g.colidx[e + 2 * G], v3 = P.g.colidx[e + 3 * G];
            const float s0 = P.S_in[(size_t)v0 * T + j], s1 = P.S_in[(size_t)v1 * T + j];
            const float s2 = P.S_in[(size_t)v2 * T + j], s3 = P.S_in[(size_t)v3 * T + j];
            acc += s0;
            acc += s1;
            acc += s2;
            acc += s3;
        }
        for (; e < e1; e += G) acc += P.S_in[(size_t)P.g.colidx[e] * T + j];
#pragma unroll
        for (int o = T; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane < T) part[warp][j] = acc;
        __syncthreads();
        if (t < T) {
            float s = 0.f;
            for (int w2 = 0; w2 < kLongBlock / 32; ++w2) s += part[w2][t];
            finish_row<T>(P, u, t, s);
        }
        __syncthreads();
    }
}

// level 0 of a tile: R_0 = X (BF16 -> FP32), Z = keep_0 X, S_0 = d^-b X; columns past the tile's
// width are zero
template <int T>
__global__ void k_tile_init(TileArgs P, const uint16_t *X, int64_t ldx, int64_t n)
{
    const int64_t total = n * T;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = t / T;
        const int j = (int)(t - u * T);
        float x = 0.f;
        if (j < P.width) {
            x = __uint_as_float((uint32_t)X[u * ldx + P.c0 + j] << 16);
            P.Z[u * P.ldz + P.c0 + j] = P.keep * x;
        }
        P.S_out[(size_t)u * T + j] = fac_b(P, (int32_t)u, P.g.deg[u]) * x;
    }
}

__global__ void k_deg_pow(const int32_t *deg, int64_t n, float p, float *out)
{
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        out[u] = deg[u] > 0 ? powf((float)deg[u], -p) : (p == 0.f ? 1.f : 0.f);
}

__global__ void k_row_class(const int32_t *deg, int64_t n, int cls, uint32_t *flag)
{
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = deg[u];
        const int c = d <= kShortRow ? 0 : (d <= kMediumRow ? 1 : 2);
        flag[u] = (d > 0 && c == cls) ? 1u : 0u;
    }
}

__global__ void k_row_scatter(const uint32_t *flag, const int64_t *pos, int64_t n, int32_t *out)
{
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        if (flag[u]) out[pos[u]] = (int32_t)u;
}

__global__ void k_zero_rows(float *Z, int64_t ldz, int64_t n, int c0, int width, const int32_t *deg, float *S, int T)
{
    // rows without neighbours keep Z = keep_0 X after level 0 and have R = 0 afterwards
    (void)Z; (void)ldz; (void)c0; (void)width;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        if (deg[u] == 0)
            for (int j = 0; j < T; ++j) S[(size_t)u * T + j] = 0.f;
}

template <int T>
int run_tiles(agp_graph_s *g, const double *keep, const double *rho, int L, const uint16_t *X, int64_t d, int64_t ldx,
              float *Z, int64_t ldz, float *S0, float *S1, const float *fa, const float *fb, int a_mode, int b_mode,
              cudaStream_t s)
{
    const int64_t n = g->n;
    const int grid = grid_stride_blocks();
    const int64_t cnt[3] = {g->row_count[0], g->row_count[1], g->row_count[2]};
    for (int64_t c0 = 0; c0 < d; c0 += T) {
        TileArgs P;
        P.g = g->dev();
        P.fa = fa;
        P.fb = fb;
        P.a_mode = a_mode;
        P.b_mode = b_mode;
        P.Z = Z;
        P.ldz = ldz;
        P.c0 = (int)c0;
        P.width = (int)std::min<int64_t>(T, d - c0);
        P.rho = 0.f;
        P.keep = (float)keep[0];
        P.S_in = nullptr;
        P.S_out = S0;
        k_tile_init<T><<<grid, kBlock, 0, s>>>(P, X, ldx, n);
        float *in = S0, *out = S1;
        for (int i = 0; i < L && rho[i] != 0.0; ++i) {
            P.S_in = in;
            P.S_out = out;
            P.rho = (float)rho[i];
            P.keep = (float)keep[i + 1];
            // every row with neighbours is in exactly one list; isolated rows get S = 0 (nothing
            // reaches them, and their Z keeps level 0)
            k_zero_rows<<<grid, kBlock, 0, s>>>(Z, ldz, n, P.c0, P.width, g->deg, out, T);
            if (cnt[0]) k_tile_short<T><<<grid, kBlock, 0, s>>>(P, g->row_list[0], cnt[0]);
            if (cnt[1]) k_tile_medium<T><<<grid, kBlock, 0, s>>>(P, g->row_list[1], cnt[1]);
            if (cnt[2]) k_tile_long<T><<<(int)std::min<int64_t>(cnt[2], grid), kLongBlock, 0, s>>>(P, g->row_list[2], cnt[2]);
            std::swap(in, out);
        }
        AGP_CUDA_TRY(cudaGetLastError());
    }
    return AGP_OK;
}

}  // namespace

// Rows of the graph by length class (built once, kept with the graph): short (d <= 32), medium
// (d <= 4096), long; rows without neighbours are in none. Used by the exact feature tiles and by
// the pull levels of the propagation.
int ensure_row_lists(agp_graph_s *g, cudaStream_t s)
{
    if (g->row_list[0] || g->n == 0) return AGP_OK;
    const int64_t n = g->n;
    const int grid = grid_stride_blocks();
    uint32_t *flag = nullptr;
    int64_t *pos = nullptr;
    void *scratch = nullptr;
    const size_t sb = exclusive_scan_scratch_bytes(n);
    int rc = AGP_OK;
    if (cudaMalloc(&flag, sizeof(uint32_t) * n) != cudaSuccess || cudaMalloc(&pos, sizeof(int64_t) * (n + 1)) != cudaSuccess ||
        cudaMalloc(&scratch, sb) != cudaSuccess)
        rc = fail(AGP_ENOMEM, "row lists: device scratch");
    for (int c = 0; c < 3 && rc == AGP_OK; ++c) {
        k_row_class<<<grid, kBlock, 0, s>>>(g->deg, n, c, flag);
        rc = exclusive_scan_u32(flag, pos, n, pos + n, scratch, sb, s);
        int64_t cnt = 0;
        if (rc == AGP_OK && (cudaMemcpyAsync(&cnt, pos + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                             cudaStreamSynchronize(s) != cudaSuccess))
            rc = fail(AGP_ECUDA, "row lists: count");
        if (rc == AGP_OK && cudaMalloc(&g->row_list[c], sizeof(int32_t) * std::max<int64_t>(cnt, 1)) != cudaSuccess)
            rc = fail(AGP_ENOMEM, "row lists");
        if (rc == AGP_OK) {
            k_row_scatter<<<grid, kBlock, 0, s>>>(flag, pos, n, g->row_list[c]);
            g->row_count[c] = cnt;
        }
    }
    if (rc == AGP_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = fail(AGP_ECUDA, "row lists");
    cudaFree(flag);
    cudaFree(pos);
    cudaFree(scratch);
    if (rc != AGP_OK) {
        cudaGetLastError();
        for (int c = 0; c < 3; ++c) {
            cudaFree(g->row_list[c]);
            g->row_list[c] = nullptr;
            g->row_count[c] = 0;
        }
    }
    return rc;
}

// Column tile width: the graph's setting, else the widest of 8 / 16 / 32 whose S block stays within
// 64 MB (half of L2), at least 8.
int column_tile(const agp_graph_s *g)
{
    if (g->column_tile > 0) return g->column_tile;
    int T = 32;
    while (T > 8 && (int64_t)T * 4 * std::max<int64_t>(g->n, 1) > (64ll << 20)) T /= 2;
    return T;
}

int feature_exact_tiled(agp_graph_s *g, const agp_params_t *p, const uint16_t *X, int64_t d, int64_t ldx, float *Z,
                        int64_t ldz, cudaStream_t s)
{
    const int L = p->L;
    std::vector<double> keep(L + 1), rho(L + 1);
    double y0 = 0.0;
    AGP_TRY(coefficients(p, keep.data(), rho.data(), &y0, g->device, s));
    AGP_TRY(ensure_row_lists(g, s));
    const int T = column_tile(g);
    const int64_t n = g->n;
    const int a_mode = exponent_mode(p->a), b_mode = exponent_mode(p->b);
    const bool general = a_mode == 3 || b_mode == 3;
    const size_t sbytes = sizeof(float) * (size_t)n * T;
    AGP_TRY(grow(&g->tile_buf, &g->tile_bytes, 2 * sbytes + (general ? 2 * sizeof(float) * (size_t)n : 0) + 1024));
    float *S0 = (float *)g->tile_buf, *S1 = S0 + (size_t)n * T;
    float *fa = nullptr, *fb = nullptr;
    if (general) {  // general exponents: per-node factor tables (modes 0-2 are computed inline)
        fa = S1 + (size_t)n * T;
        fb = fa + n;
        const int grid = grid_stride_blocks();
        k_deg_pow<<<grid, kBlock, 0, s>>>(g->deg, n, (float)p->a, fa);
        k_deg_pow<<<grid, kBlock, 0, s>>>(g->deg, n, (float)p->b, fb);
    }
    int rc;
    switch (T) {
    case 8: rc = run_tiles<8>(g, keep.data(), rho.data(), L, X, d, ldx, Z, ldz, S0, S1, fa, fb, a_mode, b_mode, s); break;
    case 16: rc = run_tiles<16>(g, keep.data(), rho.data(), L, X, d, ldx, Z, ldz, S0, S1, fa, fb, a_mode, b_mode, s); break;
    default: rc = run_tiles<32>(g, keep.data(), rho.data(), L, X, d, ldx, Z, ldz, S0, S1, fa, fb, a_mode, b_mode, s); break;
    }
    const int64_t launches = (d + T - 1) / T * (1 + (int64_t)L * 4);
    __atomic_fetch_add(&g->kernel_launches, launches, __ATOMIC_RELAXED);
    return rc;
}

}  // namespace agp
