// sweep.cu -- the local-clustering sweep of Section 6 (local clustering with HKPR) on the GPU.
//
// Given a propagation result pi, the nodes are ordered by pi(v)/d_v, largest first, and the prefix
// S_i of least conductance Phi(S_i) = cut(S_i) / min(vol(S_i), 2m - vol(S_i)) is returned. Readings
// where the paper is silent: only nodes with pi(v) > 0 and d_v > 0 are swept; ties on the score go to
// the smaller id; prefixes run over i = 1 .. min(swept, n - 1); a prefix with min(vol, 2m - vol) = 0
// is skipped; a self-loop counts once in d_v and never crosses the cut.
//
// Steps (all on the device):
//   1. flag the swept nodes and compact them in id order (scan), with the key ~bits(pi(v)/d_v): the
//      FP64 score of the FP32 pi, whose bit pattern ascends with the value for positive doubles;
//   2. a stable radix sort of the keys gives the sweep order (ties keep ascending id);
//   3. rank[v] = position of v; one warp per swept node counts its neighbours of smaller rank
//      (edges inside the prefix when v joins) and its self-loops;
//   4. prefix sums of d_v, d_v - loops_v and inside_v give vol(S_i) and cut(S_i) = sum (d - loops)
//      - 2 sum inside as exact integers; Phi_i in FP64; the first least Phi_i wins.
#include <cmath>
#include <vector>

#include "agp_internal.cuh"

namespace agp {
namespace {

__global__ void k_sweep_flag(const float *pi, const int32_t *deg, int64_t n, uint32_t *flag)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        flag[v] = (deg[v] > 0 && pi[v] > 0.f) ? 1u : 0u;
}

__global__ void k_sweep_keys(const float *pi, const int32_t *deg, int64_t n, const uint32_t *flag, const int64_t *pos,
                             uint64_t *keys, uint32_t *vals)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[v]) continue;
        const double score = (double)pi[v] / (double)deg[v];  // > 0
        keys[pos[v]] = ~(uint64_t)__double_as_longlong(score);  // descending score
        vals[pos[v]] = (uint32_t)v;
    }
}

__global__ void k_sweep_rank(const uint32_t *order, int64_t K, int32_t *rank)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < K; i += (int64_t)gridDim.x * blockDim.x)
        rank[order[i]] = (int32_t)i;
}

// one warp per swept node: neighbours already in the prefix when it joins, and its self-loops
__global__ void k_sweep_count(DevGraph g, const uint32_t *order, int64_t K, const int32_t *rank, uint32_t *deg_i,
                              uint32_t *open_i, uint32_t *inside_i)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < K; i += nw) {
        const int32_t v = (int32_t)order[i];
        uint32_t inside = 0, loops = 0;
        for (int64_t e = g.rowptr[v] + lane; e < g.rowptr[v + 1]; e += 32) {
            const int32_t w = g.colidx[e];
            if (w == v) ++loops;
            else if (rank[w] < (int32_t)i) ++inside;
        }
        for (int o = 16; o > 0; o >>= 1) {
            inside += __shfl_down_sync(0xffffffffu, inside, o);
            loops += __shfl_down_sync(0xffffffffu, loops, o);
        }
        if (lane == 0) {
            const uint32_t d = (uint32_t)g.deg[v];
            deg_i[i] = d;
            open_i[i] = d - loops;
            inside_i[i] = inside;
        }
    }
}

// Phi of prefix i (1 <= i <= last) into phi[i - 1]; +inf where min(vol, 2m - vol) = 0
__global__ void k_sweep_phi(const int64_t *vol, const int64_t *open, const int64_t *inside, int64_t last, int64_t two_m,
                            double *phi)
{
    for (int64_t i = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= last; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = vol[i], cut = open[i] - 2 * inside[i];
        const int64_t den = v < two_m - v ? v : two_m - v;
        phi[i - 1] = den > 0 ? (double)cut / (double)den : INFINITY;
    }
}

// first index of the least phi (one block of 1024 threads); out = [best index or -1, phi]
__global__ void __launch_bounds__(1024) k_sweep_argmin(const double *phi, int64_t last, double *out)
{
    __shared__ double sv[1024];
    __shared__ int64_t si[1024];
    double bv = INFINITY;
    int64_t bi = -1;
    for (int64_t i = threadIdx.x; i < last; i += blockDim.x)
        if (phi[i] < bv) {  // strict: the first of equal values in this thread's (ascending) indices
            bv = phi[i];
            bi = i;
        }
    sv[threadIdx.x] = bv;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = 512; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            const double ov = sv[threadIdx.x + s];
            const int64_t oi = si[threadIdx.x + s];
            if (oi >= 0 && (ov < sv[threadIdx.x] || (ov == sv[threadIdx.x] && (si[threadIdx.x] < 0 || oi < si[threadIdx.x])))) {
                sv[threadIdx.x] = ov;
                si[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = (double)si[0];
        out[1] = sv[0];
    }
}

struct Scratch {
    std::vector<void *> ptrs;
    ~Scratch()
    {
        for (void *p : ptrs) cudaFree(p);
    }
    template <class T> int get(T **p, size_t count)
    {
        void *q = nullptr;
        if (cudaMalloc(&q, std::max<size_t>(count * sizeof(T), 16)) != cudaSuccess) {
            cudaGetLastError();
            return fail(AGP_ENOMEM, "agp_sweep: device scratch");
        }
        ptrs.push_back(q);
        *p = (T *)q;
        return AGP_OK;
    }
};

}  // namespace

int sweep(agp_graph_s *g, const float *pi, int32_t *order_out, double *phi_out, int64_t *best_size, double *best_phi,
          int64_t *swept, cudaStream_t s)
{
    if (!g || !pi) return fail(AGP_EINVAL, "agp_sweep: NULL argument");
    if (g->directed) return fail(AGP_EINVAL, "agp_sweep: conductance needs an undirected graph");
    AGP_CUDA_TRY(cudaSetDevice(g->device));
    const int64_t n = g->n;
    if (best_size) *best_size = 0;
    if (best_phi) *best_phi = NAN;
    if (swept) *swept = 0;
    if (n == 0) return AGP_OK;
    const int grid = grid_stride_blocks();
    Scratch S;
    uint32_t *flag = nullptr;
    int64_t *pos = nullptr;
    AGP_TRY(S.get(&flag, n));
    AGP_TRY(S.get(&pos, n + 1));
    const size_t scan_b = exclusive_scan_scratch_bytes(n + 1);
    void *scan_scratch = nullptr;
    AGP_TRY(S.get((char **)&scan_scratch, scan_b));
    k_sweep_flag<<<grid, kBlock, 0, s>>>(pi, g->deg, n, flag);
    AGP_TRY(exclusive_scan_u32(flag, pos, n, pos + n, scan_scratch, scan_b, s));
    int64_t K = 0;
    AGP_CUDA_TRY(cudaMemcpyAsync(&K, pos + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    AGP_CUDA_TRY(cudaStreamSynchronize(s));
    if (order_out) AGP_CUDA_TRY(cudaMemsetAsync(order_out, 0xff, sizeof(int32_t) * n, s));  // -1 past the swept nodes
    const int64_t last = std::min<int64_t>(K, n - 1);
    if (phi_out && n > 1) AGP_CUDA_TRY(cudaMemsetAsync(phi_out, 0, sizeof(double) * (n - 1), s));
    if (swept) *swept = K;
    if (K == 0) return AGP_OK;
    uint64_t *ka = nullptr, *kb = nullptr, *kout = nullptr;
    uint32_t *va = nullptr, *vb = nullptr, *vout = nullptr;
    AGP_TRY(S.get(&ka, K));
    AGP_TRY(S.get(&kb, K));
    AGP_TRY(S.get(&va, K));
    AGP_TRY(S.get(&vb, K));
    const size_t sort_b = radix_sort_scratch_bytes(K);
    void *sort_scratch = nullptr;
    AGP_TRY(S.get((char **)&sort_scratch, sort_b));
    k_sweep_keys<<<grid, kBlock, 0, s>>>(pi, g->deg, n, flag, pos, ka, va);
    AGP_CUDA_TRY(cudaGetLastError());
    AGP_TRY(radix_sort_u64(ka, kb, va, vb, K, 64, &kout, &vout, sort_scratch, sort_b, s));
    int32_t *rank = nullptr;
    uint32_t *dg = nullptr, *op = nullptr, *in = nullptr;
    int64_t *vol = nullptr, *ops = nullptr, *ins = nullptr;
    double *phi = nullptr, *res = nullptr;
    AGP_TRY(S.get(&rank, n));
    AGP_TRY(S.get(&dg, K));
    AGP_TRY(S.get(&op, K));
    AGP_TRY(S.get(&in, K));
    AGP_TRY(S.get(&vol, K + 1));
    AGP_TRY(S.get(&ops, K + 1));
    AGP_TRY(S.get(&ins, K + 1));
    AGP_TRY(S.get(&phi, std::max<int64_t>(last, 1)));
    AGP_TRY(S.get(&res, 2));
    AGP_CUDA_TRY(cudaMemsetAsync(rank, 0x7f, sizeof(int32_t) * n, s));  // not swept: larger than every rank
    k_sweep_rank<<<grid, kBlock, 0, s>>>(vout, K, rank);
    k_sweep_count<<<grid, kBlock, 0, s>>>(g->dev(), vout, K, rank, dg, op, in);
    AGP_CUDA_TRY(cudaGetLastError());
    AGP_TRY(exclusive_scan_u32(dg, vol, K, vol + K, scan_scratch, scan_b, s));
    AGP_TRY(exclusive_scan_u32(op, ops, K, ops + K, scan_scratch, scan_b, s));
    AGP_TRY(exclusive_scan_u32(in, ins, K, ins + K, scan_scratch, scan_b, s));
    if (order_out) AGP_CUDA_TRY(cudaMemcpyAsync(order_out, vout, sizeof(int32_t) * K, cudaMemcpyDeviceToDevice, s));
    double h[2] = {-1.0, NAN};
    if (last > 0) {
        k_sweep_phi<<<grid, kBlock, 0, s>>>(vol, ops, ins, last, g->nnz, phi);
        k_sweep_argmin<<<1, 1024, 0, s>>>(phi, last, res);
        AGP_CUDA_TRY(cudaGetLastError());
        if (phi_out) AGP_CUDA_TRY(cudaMemcpyAsync(phi_out, phi, sizeof(double) * last, cudaMemcpyDeviceToDevice, s));
        AGP_CUDA_TRY(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, s));
    }
    AGP_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t bi = (int64_t)h[0];
    if (bi >= 0 && std::isfinite(h[1])) {
        if (best_size) *best_size = bi + 1;
        if (best_phi) *best_phi = h[1];
    }
    return AGP_OK;
}

}  // namespace agp
