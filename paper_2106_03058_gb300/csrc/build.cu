// build.cu -- device CSR builder: Section 4, "Pre-sorting adjacency list by degrees".
//
// The paper sorts (u, v, d_v) tuples by d_v with a counting sort and appends v to N_u in that
// order, so that every N_u is in ascending neighbour degree. On the GPU the same order is reached
// with two stable LSD radix sorts over the whole edge list:
//   1. key (u, v): groups each row and exposes repeated edges as equal neighbours (merged);
//   2. key (u, d_v) with value v: stable, so ties on degree keep ascending v.
// Input self-loops are dropped; with AGP_ADD_SELF_LOOPS one loop per node is added before the
// sorts and counts once in the degree. With AGP_DIRECTED (Section 4, "Propagation on directed
// graph", transposed adjacency) only u -> v is kept, so rows are out-neighbour lists and degrees
// out-degrees. With AGP_DIRECTED_IN (the untransposed adjacency of the same passage, single-target
// PPR) only v -> u is kept: rows are in-neighbour lists, while the degrees stay out-degrees (the
// number of rows a node appears in), so a row's length is not its node's degree.
#include <algorithm>
#include <vector>

#include "agp_internal.cuh"

namespace agp {
namespace {

// Two keys per input edge: (u, v) and, for an undirected graph, (v, u); a directed graph keeps
// only u -> v (directed = 1) or only its reverse v -> u (directed = 2); a slot it does not keep
// holds the sentinel and is dropped with the loops.
__global__ void k_expand_edges(const int32_t *src, const int32_t *dst, int64_t m, int64_t n, int ubits,
                               uint64_t sentinel, int directed, uint64_t *keys, unsigned int *bad)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = src[e], v = dst[e];
        const bool ok = u >= 0 && u < n && v >= 0 && v < n;
        if (!ok) atomicOr(bad, 1u);
        const bool keep = ok && u != v;
        keys[2 * e] = (keep && directed != 2) ? (((uint64_t)u << ubits) | (uint64_t)v) : sentinel;
        keys[2 * e + 1] = (keep && directed != 1) ? (((uint64_t)v << ubits) | (uint64_t)u) : sentinel;
    }
}

__global__ void k_self_loops(int64_t n, int ubits, uint64_t *keys)
{
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        keys[u] = ((uint64_t)u << ubits) | (uint64_t)u;
}

__global__ void k_unique_flags(const uint64_t *keys, int64_t count, uint64_t sentinel, uint32_t *flag)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        flag[i] = (k != sentinel && (i == 0 || keys[i - 1] != k)) ? 1u : 0u;
    }
}

// Unique keys to the front of `uniq`; rowlen[u] counts row u. With `outdeg` (in-neighbour rows),
// outdeg[v] counts the rows v appears in.
__global__ void k_compact_unique(const uint64_t *keys, const uint32_t *flag, const int64_t *pos, int64_t count,
                                 int ubits, uint64_t *uniq, int32_t *rowlen, int32_t *outdeg)
{
    const uint64_t mask = (1ull << ubits) - 1ull;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[i]) continue;
        const uint64_t k = keys[i];
        uniq[pos[i]] = k;
        atomicAdd(&rowlen[(int64_t)(k >> ubits)], 1);
        if (outdeg) atomicAdd(&outdeg[(int64_t)(k & mask)], 1);
    }
}

__global__ void k_max_deg(const int32_t *deg, int64_t n, int32_t *out)
{
    int32_t mx = 0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        mx = max(mx, deg[u]);
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}

__global__ void k_degree_keys(const uint64_t *uniq, int64_t nnz, int ubits, int dbits, const int32_t *deg,
                              uint64_t *key2, uint32_t *val)
{
    const uint64_t mask = (1ull << ubits) - 1ull;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = uniq[p];
        const uint64_t u = k >> ubits, v = k & mask;
        key2[p] = (u << dbits) | (uint64_t)deg[v];
        val[p] = (uint32_t)v;
    }
}

int bits_for(int64_t x)  // smallest b >= 1 with 2^b > x - 1, i.e. values in [0, x) fit
{
    int b = 1;
    while (b < 63 && (1ll << b) < x) ++b;
    return b;
}

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() { reset(); }
    void reset()
    {
        if (p) cudaFree(p);
        p = nullptr;
    }
    int alloc(size_t bytes)
    {
        if (bytes == 0) bytes = 16;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            return fail(AGP_ENOMEM, "cudaMalloc(" + std::to_string(bytes) + ") in graph build: " + cudaGetErrorString(e));
        }
        return AGP_OK;
    }
    template <class T> T *as() const { return (T *)p; }
    void *release() { void *q = p; p = nullptr; return q; }
};

}  // namespace

int build_graph(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, uint32_t flags,
                int device, cudaStream_t stream, agp_graph_s **out)
{
    if (!out) return fail(AGP_EINVAL, "agp_build_graph: out is NULL");
    *out = nullptr;
    if (n < 0 || n >= (1ll << 31)) return fail(AGP_EINVAL, "agp_build_graph: n must be in [0, 2^31)");
    if (m < 0) return fail(AGP_EINVAL, "agp_build_graph: n_edges < 0");
    if (m > 0 && (!src || !dst)) return fail(AGP_EINVAL, "agp_build_graph: src/dst NULL");
    if (flags & ~(AGP_ADD_SELF_LOOPS | AGP_EDGES_ON_DEVICE | AGP_DIRECTED | AGP_DIRECTED_IN))
        return fail(AGP_EINVAL, "agp_build_graph: unknown flag");
    if ((flags & AGP_DIRECTED) && (flags & AGP_DIRECTED_IN))
        return fail(AGP_EINVAL, "agp_build_graph: AGP_DIRECTED and AGP_DIRECTED_IN exclude each other");
    const int directed = (flags & AGP_DIRECTED) ? 1 : (flags & AGP_DIRECTED_IN) ? 2 : 0;
    AGP_CUDA_TRY(cudaSetDevice(device));

    const bool loops = flags & AGP_ADD_SELF_LOOPS;
    const int ubits = bits_for(std::max<int64_t>(n, 2));
    const uint64_t sentinel = 1ull << (2 * ubits);
    const int64_t E = 2 * m + (loops ? n : 0);
    const int grid = grid_stride_blocks();

    DevBuf d_src, d_dst;
    const int32_t *s = src, *t = dst;
    if (!(flags & AGP_EDGES_ON_DEVICE) && m > 0) {
        AGP_TRY(d_src.alloc(sizeof(int32_t) * m));
        AGP_TRY(d_dst.alloc(sizeof(int32_t) * m));
        AGP_CUDA_TRY(cudaMemcpyAsync(d_src.p, src, sizeof(int32_t) * m, cudaMemcpyHostToDevice, stream));
        AGP_CUDA_TRY(cudaMemcpyAsync(d_dst.p, dst, sizeof(int32_t) * m, cudaMemcpyHostToDevice, stream));
        s = d_src.as<int32_t>();
        t = d_dst.as<int32_t>();
    }

    DevBuf keys_a, keys_b, flagb, pos, scratch, bad, total, maxd;
    AGP_TRY(keys_a.alloc(sizeof(uint64_t) * E));
    AGP_TRY(keys_b.alloc(sizeof(uint64_t) * E));
    const size_t scratch_bytes = std::max(radix_sort_scratch_bytes(E), exclusive_scan_scratch_bytes(std::max(E, n)));
    AGP_TRY(scratch.alloc(scratch_bytes));
    AGP_TRY(bad.alloc(sizeof(unsigned int)));
    AGP_TRY(total.alloc(sizeof(int64_t)));
    AGP_TRY(maxd.alloc(sizeof(int32_t)));
    AGP_CUDA_TRY(cudaMemsetAsync(bad.p, 0, sizeof(unsigned int), stream));
    AGP_CUDA_TRY(cudaMemsetAsync(maxd.p, 0, sizeof(int32_t), stream));
    if (m > 0) k_expand_edges<<<grid, kBlock, 0, stream>>>(s, t, m, n, ubits, sentinel, directed, keys_a.as<uint64_t>(), bad.as<unsigned int>());
    if (loops && n > 0) k_self_loops<<<grid, kBlock, 0, stream>>>(n, ubits, keys_a.as<uint64_t>() + 2 * m);
    AGP_CUDA_TRY(cudaGetLastError());
    unsigned int h_bad = 0;
    AGP_CUDA_TRY(cudaMemcpyAsync(&h_bad, bad.p, sizeof(h_bad), cudaMemcpyDeviceToHost, stream));
    AGP_CUDA_TRY(cudaStreamSynchronize(stream));
    if (h_bad) return fail(AGP_EINVAL, "agp_build_graph: edge endpoint outside [0, n)");
    d_src.reset();
    d_dst.reset();

    // sort 1: (u, v); the sentinel bit sorts dropped edges to the end
    uint64_t *sorted = nullptr;
    AGP_TRY(radix_sort_u64(keys_a.as<uint64_t>(), keys_b.as<uint64_t>(), nullptr, nullptr, E, 2 * ubits + 1,
                           &sorted, nullptr, scratch.p, scratch_bytes, stream));
    uint64_t *other = (sorted == keys_a.as<uint64_t>()) ? keys_b.as<uint64_t>() : keys_a.as<uint64_t>();

    // merge repeated neighbours
    AGP_TRY(flagb.alloc(sizeof(uint32_t) * E));
    AGP_TRY(pos.alloc(sizeof(int64_t) * E));
    if (E > 0) k_unique_flags<<<grid, kBlock, 0, stream>>>(sorted, E, sentinel, flagb.as<uint32_t>());
    AGP_TRY(exclusive_scan_u32(flagb.as<uint32_t>(), pos.as<int64_t>(), E, total.as<int64_t>(), scratch.p, scratch_bytes, stream));
    int64_t nnz = 0;
    AGP_CUDA_TRY(cudaMemcpyAsync(&nnz, total.p, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));

    DevBuf rowptr, degb, lenb, colA, colB;
    AGP_TRY(degb.alloc(sizeof(int32_t) * std::max<int64_t>(n, 1)));
    AGP_TRY(rowptr.alloc(sizeof(int64_t) * (n + 1)));
    AGP_CUDA_TRY(cudaMemsetAsync(degb.p, 0, sizeof(int32_t) * std::max<int64_t>(n, 1), stream));
    if (directed == 2) {  // row lengths (in-degrees) apart from the degrees (out-degrees)
        AGP_TRY(lenb.alloc(sizeof(int32_t) * std::max<int64_t>(n, 1)));
        AGP_CUDA_TRY(cudaMemsetAsync(lenb.p, 0, sizeof(int32_t) * std::max<int64_t>(n, 1), stream));
    }
    int32_t *rowlen = directed == 2 ? lenb.as<int32_t>() : degb.as<int32_t>();
    AGP_CUDA_TRY(cudaStreamSynchronize(stream));
    // unique keys go to the front of the spare key buffer
    if (E > 0)
        k_compact_unique<<<grid, kBlock, 0, stream>>>(sorted, flagb.as<uint32_t>(), pos.as<int64_t>(), E, ubits, other, rowlen,
                                                      directed == 2 ? degb.as<int32_t>() : nullptr);
    AGP_CUDA_TRY(cudaGetLastError());
    flagb.reset();
    pos.reset();

    // rowptr = exclusive scan of row lengths
    AGP_TRY(exclusive_scan_u32((const uint32_t *)rowlen, rowptr.as<int64_t>(), n, rowptr.as<int64_t>() + n, scratch.p, scratch_bytes, stream));
    if (n > 0) k_max_deg<<<grid, kBlock, 0, stream>>>(degb.as<int32_t>(), n, maxd.as<int32_t>());
    int32_t max_deg = 0;
    AGP_CUDA_TRY(cudaMemcpyAsync(&max_deg, maxd.p, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    AGP_CUDA_TRY(cudaStreamSynchronize(stream));
    const int dbits = bits_for((int64_t)max_deg + 1);

    // sort 2: stable by (u, d_v), value v
    AGP_TRY(colA.alloc(sizeof(uint32_t) * std::max<int64_t>(nnz, 1)));
    AGP_TRY(colB.alloc(sizeof(uint32_t) * std::max<int64_t>(nnz, 1)));
    uint64_t *key2 = sorted;  // sort-1 output is no longer needed
    if (nnz > 0) k_degree_keys<<<grid, kBlock, 0, stream>>>(other, nnz, ubits, dbits, degb.as<int32_t>(), key2, colA.as<uint32_t>());
    AGP_CUDA_TRY(cudaGetLastError());
    uint64_t *k2out = nullptr;
    uint32_t *vout = nullptr;
    AGP_TRY(radix_sort_u64(key2, other, colA.as<uint32_t>(), colB.as<uint32_t>(), nnz, ubits + dbits, &k2out, &vout,
                           scratch.p, scratch_bytes, stream));
    AGP_CUDA_TRY(cudaStreamSynchronize(stream));

    agp_graph_s *g = new agp_graph_s();
    g->device = device;
    g->n = n;
    g->nnz = nnz;
    g->max_deg = max_deg;
    g->directed = directed;
    g->ubits = ubits;
    g->rowptr = (int64_t *)rowptr.release();
    g->deg = (int32_t *)degb.release();
    g->colidx = (int32_t *)((vout == colA.as<uint32_t>()) ? colA.release() : colB.release());
    *out = g;
    return AGP_OK;
}

}  // namespace agp
