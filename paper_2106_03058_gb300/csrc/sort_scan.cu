// sort_scan.cu -- device-wide exclusive scan and stable LSD radix sort used by the graph builder.
//
// Both use contiguous partitions: a fixed number of blocks (a multiple of the SM count), each
// owning one contiguous range of the input, so that per-block histograms/partials are small and
// stability follows from processing every range front to back.
#include <algorithm>

#include "agp_internal.cuh"

namespace agp {
namespace {

constexpr int kPartBlocks = 608;  // partitions (4 per SM on a 152-SM GB300; any count is correct)
constexpr int kRadix = 256;
constexpr int kWarps = kBlock / 32;

int partitions_for(int64_t count)
{
    int64_t nb = (count + 4095) / 4096;
    return (int)std::max<int64_t>(1, std::min<int64_t>(kPartBlocks, nb));
}

int64_t per_partition(int64_t count, int nb)
{
    int64_t per = (count + nb - 1) / nb;
    return (per + kBlock - 1) / kBlock * kBlock;
}

// ---------------------------------------------------------------- scan
__global__ void k_scan_partial(const uint32_t *in, int64_t count, int64_t per, int64_t *partial)
{
    __shared__ uint64_t red[kWarps];
    const int64_t begin = (int64_t)blockIdx.x * per;
    const int64_t end = min(count, begin + per);
    uint64_t s = 0;
    for (int64_t i = begin + threadIdx.x; i < end; i += blockDim.x) s += in[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t t = 0;
        for (int w = 0; w < kWarps; ++w) t += red[w];
        partial[blockIdx.x] = (int64_t)t;
    }
}

// Exclusive scan of nb (<= 1024 * 64) partials by one block; writes the grand total.
__global__ void k_scan_partials(int64_t *partial, int nb, int64_t *total)
{
    __shared__ int64_t sums[1024];
    const int t = threadIdx.x;
    const int chunk = (nb + blockDim.x - 1) / blockDim.x;
    const int b0 = t * chunk, b1 = min(nb, b0 + chunk);
    int64_t s = 0;
    for (int b = b0; b < b1; ++b) s += partial[b];
    sums[t] = s;
    __syncthreads();
    if (t == 0) {
        int64_t run = 0;
        for (int k = 0; k < (int)blockDim.x; ++k) {
            int64_t v = sums[k];
            sums[k] = run;
            run += v;
        }
        *total = run;
    }
    __syncthreads();
    int64_t run = sums[t];
    for (int b = b0; b < b1; ++b) {
        int64_t v = partial[b];
        partial[b] = run;
        run += v;
    }
}

__global__ void k_scan_final(const uint32_t *in, int64_t *out, int64_t count, int64_t per,
                             const int64_t *partial)
{
    __shared__ uint64_t wsum[kWarps];
    __shared__ uint64_t run_s;
    const int64_t begin = (int64_t)blockIdx.x * per;
    const int64_t end = min(count, begin + per);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) run_s = (uint64_t)partial[blockIdx.x];
    __syncthreads();
    for (int64_t base = begin; base < end; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const uint64_t v = (i < end) ? in[i] : 0;
        uint64_t x = v;  // inclusive warp scan
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        uint64_t before = run_s;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        if (i < end) out[i] = (int64_t)(before + x - v);
        __syncthreads();
        if (threadIdx.x == 0) {
            uint64_t t = 0;
            for (int w = 0; w < kWarps; ++w) t += wsum[w];
            run_s += t;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- radix sort
__global__ void k_radix_hist(const uint64_t *keys, int64_t count, int64_t per, int shift,
                             uint32_t *counts, int nb)
{
    __shared__ uint32_t hist[kRadix];
    hist[threadIdx.x] = 0;
    __syncthreads();
    const int64_t begin = (int64_t)blockIdx.x * per;
    const int64_t end = min(count, begin + per);
    for (int64_t i = begin + threadIdx.x; i < end; i += blockDim.x)
        atomicAdd(&hist[(uint32_t)(keys[i] >> shift) & 255u], 1u);
    __syncthreads();
    counts[(int64_t)threadIdx.x * nb + blockIdx.x] = hist[threadIdx.x];
}

// Exclusive scan of the digit-major count table (digit d of block b at d*nb + b) by one block.
__global__ void k_radix_offsets(const uint32_t *counts, uint64_t *offsets, int entries)
{
    __shared__ uint64_t sums[1024];
    const int t = threadIdx.x;
    const int chunk = (entries + blockDim.x - 1) / blockDim.x;
    const int e0 = t * chunk, e1 = min(entries, e0 + chunk);
    uint64_t s = 0;
    for (int e = e0; e < e1; ++e) s += counts[e];
    sums[t] = s;
    __syncthreads();
    if (t == 0) {
        uint64_t run = 0;
        for (int k = 0; k < (int)blockDim.x; ++k) {
            uint64_t v = sums[k];
            sums[k] = run;
            run += v;
        }
    }
    __syncthreads();
    uint64_t run = sums[t];
    for (int e = e0; e < e1; ++e) {
        offsets[e] = run;
        run += counts[e];
    }
}

// Stable scatter: each block walks its range in rounds of 256 consecutive keys. The rank of a key
// is the block's running offset for its digit, plus the keys of that digit in earlier warps of
// the round, plus the lower lanes of its own warp with the same digit.
__global__ void k_radix_scatter(const uint64_t *keys_in, const uint32_t *vals_in, uint64_t *keys_out,
                                uint32_t *vals_out, int64_t count, int64_t per, int shift,
                                const uint64_t *offsets, int nb)
{
    __shared__ uint64_t run[kRadix];
    __shared__ uint32_t wcnt[kWarps][kRadix];
    __shared__ uint32_t tot[kRadix];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    run[t] = offsets[(int64_t)t * nb + blockIdx.x];
    for (int w = 0; w < kWarps; ++w) wcnt[w][t] = 0;
    __syncthreads();
    const int64_t begin = (int64_t)blockIdx.x * per;
    const int64_t end = min(count, begin + per);
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (int64_t base = begin; base < end; base += blockDim.x) {
        const int64_t i = base + t;
        const bool valid = i < end;
        const uint64_t key = valid ? keys_in[i] : 0ull;
        const uint32_t val = (valid && vals_in) ? vals_in[i] : 0u;
        const uint32_t d = valid ? ((uint32_t)(key >> shift) & 255u) : 0x100u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & lt_mask);
        if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        {
            uint32_t s = 0;
            for (int w = 0; w < kWarps; ++w) {
                uint32_t c = wcnt[w][t];
                wcnt[w][t] = s;
                s += c;
            }
            tot[t] = s;
        }
        __syncthreads();
        if (valid) {
            const uint64_t pos = run[d] + wcnt[warp][d] + rank;
            keys_out[pos] = key;
            if (vals_out) vals_out[pos] = val;
        }
        __syncthreads();
        run[t] += tot[t];
        for (int w = 0; w < kWarps; ++w) wcnt[w][t] = 0;
        __syncthreads();
    }
}

}  // namespace

size_t exclusive_scan_scratch_bytes(int64_t) { return sizeof(int64_t) * kPartBlocks + 256; }

int exclusive_scan_u32(const uint32_t *in, int64_t *out, int64_t count, int64_t *d_total,
                       void *scratch, size_t scratch_bytes, cudaStream_t stream)
{
    if (scratch_bytes < exclusive_scan_scratch_bytes(count))
        return fail(AGP_EINTERNAL, "exclusive_scan_u32: scratch too small");
    if (count == 0) {
        AGP_CUDA_TRY(cudaMemsetAsync(d_total, 0, sizeof(int64_t), stream));
        return AGP_OK;
    }
    const int nb = partitions_for(count);
    const int64_t per = per_partition(count, nb);
    int64_t *partial = (int64_t *)scratch;
    k_scan_partial<<<nb, kBlock, 0, stream>>>(in, count, per, partial);
    k_scan_partials<<<1, 1024, 0, stream>>>(partial, nb, d_total);
    k_scan_final<<<nb, kBlock, 0, stream>>>(in, out, count, per, partial);
    AGP_CUDA_TRY(cudaGetLastError());
    return AGP_OK;
}

size_t radix_sort_scratch_bytes(int64_t)
{
    return (size_t)kRadix * kPartBlocks * (sizeof(uint32_t) + sizeof(uint64_t)) + 256;
}

int radix_sort_u64(uint64_t *keys_a, uint64_t *keys_b, uint32_t *vals_a, uint32_t *vals_b,
                   int64_t count, int key_bits, uint64_t **keys_out, uint32_t **vals_out,
                   void *scratch, size_t scratch_bytes, cudaStream_t stream)
{
    if (scratch_bytes < radix_sort_scratch_bytes(count))
        return fail(AGP_EINTERNAL, "radix_sort_u64: scratch too small");
    uint64_t *kin = keys_a, *kout = keys_b;
    uint32_t *vin = vals_a, *vout = vals_b;
    if (count > 0) {
        const int nb = partitions_for(count);
        const int64_t per = per_partition(count, nb);
        uint32_t *counts = (uint32_t *)scratch;
        uint64_t *offsets = (uint64_t *)((char *)scratch + (size_t)kRadix * kPartBlocks * sizeof(uint32_t));
        for (int shift = 0; shift < key_bits; shift += 8) {
            k_radix_hist<<<nb, kRadix, 0, stream>>>(kin, count, per, shift, counts, nb);
            k_radix_offsets<<<1, 1024, 0, stream>>>(counts, offsets, kRadix * nb);
            k_radix_scatter<<<nb, kBlock, 0, stream>>>(kin, vin, kout, vout, count, per, shift, offsets, nb);
            std::swap(kin, kout);
            std::swap(vin, vout);
        }
        AGP_CUDA_TRY(cudaGetLastError());
    }
    *keys_out = kin;
    if (vals_out) *vals_out = vin;
    return AGP_OK;
}

}  // namespace agp
