// topk.cu -- sparse output of a propagation: the k largest entries of each result row.
//
// Serving and local-clustering consumers want the few largest entries of pi, not a dense n-vector.
// For every row this kernel selects the k entries that come first in the order (value descending,
// node id ascending) and writes them in that order. The order is a 64-bit key per entry:
//     key = (desc(value) << 32) | id,
// where desc maps a float to a 32-bit integer whose ascending order is the float's descending order
// (with -0 taken as +0). Keys are unique, so the k smallest keys are exactly the wanted entries.
//
// One CTA per row runs a radix select over the key, 11 bits at a time from the top: a pass scans the
// row, histograms the next digit of the keys that match the digits fixed so far, and in the same scan
// emits the keys that the previous pass proved to be inside (their digit below the boundary digit).
// The boundary digit b* is where the running count reaches k; when its bin holds exactly the keys
// still needed, the next scan emits them and the selection ends, otherwise b* is fixed and the next
// pass looks at the next digit. A row is read once per pass (at most six, usually two or three), and
// no scratch memory is needed besides the k keys in shared memory, which a bitonic sort orders.
#include <cstdint>

#include "agp_internal.cuh"

namespace agp {
namespace {

constexpr int kTopkThreads = 1024;
constexpr int kTopkMax = 2048;      // largest k (the keys sit in shared memory)
constexpr int kDigitBits = 11;
constexpr int kBins = 1 << kDigitBits;

__device__ __forceinline__ uint32_t desc_key(float x)
{
    uint32_t b = __float_as_uint(x);
    if ((b << 1) == 0u) b = 0u;                      // -0 sorts as +0
    const uint32_t asc = (b & 0x80000000u) ? ~b : (b | 0x80000000u);  // ascending order of floats
    return ~asc;                                     // descending
}

__device__ __forceinline__ float key_value(uint64_t key)
{
    const uint32_t asc = ~(uint32_t)(key >> 32);
    const uint32_t b = (asc & 0x80000000u) ? (asc & 0x7fffffffu) : ~asc;
    return __uint_as_float(b);
}

// digit of `key` at bit offset `shift` (the lowest bits of the last digit when fewer remain)
__device__ __forceinline__ uint32_t digit_of(uint64_t key, int shift)
{
    return (uint32_t)((shift >= 0 ? (key >> shift) : (key << -shift)) & (kBins - 1));
}

__global__ void __launch_bounds__(kTopkThreads) k_topk_rows(const float *pi, int64_t n, int64_t ld, int k, float *val,
                                                            int32_t *idx, int64_t ldo)
{
    __shared__ uint32_t hist[kBins];
    __shared__ uint64_t keys[kTopkMax];
    __shared__ uint32_t n_out;
    __shared__ int s_bstar, s_done;
    __shared__ uint32_t s_needed;
    const int row = blockIdx.x;
    const float *x = pi + (size_t)row * ld;
    const int t = threadIdx.x, lane = t & 31;
    if (t == 0) n_out = 0;
    for (int i = t; i < kTopkMax; i += kTopkThreads) keys[i] = ~0ull;
    uint64_t prefix = 0;        // key bits fixed so far (above `fixed_shift`)
    int fixed = 0;              // number of fixed top bits
    uint32_t needed = (uint32_t)k;
    int emit_digit = -1;        // keys matching the previous prefix with digit < emit_digit are emitted
    uint64_t emit_prefix = 0;
    int emit_fixed = 0;
    bool emit_all_bin = false;  // the previous pass's boundary bin is wholly needed
    for (int pass = 0; pass <= 64 / kDigitBits + 1; ++pass) {
        const int shift = 64 - fixed - kDigitBits;  // bit offset of this pass's digit
        for (int b = t; b < kBins; b += kTopkThreads) hist[b] = 0;
        __syncthreads();
        const bool histo = !emit_all_bin && fixed < 64;
        // warp-uniform scan (every lane runs every step, out-of-range lanes inactive), so that equal
        // digits of a warp make one shared-memory add and emitted keys one slot reservation: a row
        // often holds millions of equal keys in their top digits (entries that are exactly zero)
        for (int64_t base = 0; base < n; base += kTopkThreads) {
            const int64_t i = base + t;
            const bool valid = i < n;
            const uint64_t key = valid ? (((uint64_t)desc_key(x[i]) << 32) | (uint64_t)(uint32_t)i) : ~0ull;
            bool emit = false;
            if (valid && emit_digit >= 0) {
                // what the previous pass proved inside: same prefix, digit below its boundary (or equal
                // to it when the whole boundary bin is needed)
                const bool match = emit_fixed == 0 || (key >> (64 - emit_fixed)) == (emit_prefix >> (64 - emit_fixed));
                if (match) {
                    const uint32_t dg = digit_of(key, 64 - emit_fixed - kDigitBits);
                    emit = dg < (uint32_t)emit_digit || (emit_all_bin && dg == (uint32_t)emit_digit);
                }
            }
            const unsigned eb = __ballot_sync(0xffffffffu, emit);
            if (eb) {
                uint32_t first = 0;
                if (lane == __ffs(eb) - 1) first = atomicAdd(&n_out, (uint32_t)__popc(eb));
                first = __shfl_sync(0xffffffffu, first, __ffs(eb) - 1);
                if (emit) {
                    const uint32_t slot = first + (uint32_t)__popc(eb & ((1u << lane) - 1u));
                    if (slot < (uint32_t)kTopkMax) keys[slot] = key;
                }
            }
            const bool in_h = valid && histo && (fixed == 0 || (key >> (64 - fixed)) == (prefix >> (64 - fixed)));
            const uint32_t dg = in_h ? digit_of(key, shift) : 0xffffffffu;
            const unsigned same = __match_any_sync(0xffffffffu, dg);
            if (in_h && lane == __ffs(same) - 1) atomicAdd(&hist[dg], (uint32_t)__popc(same));
        }
        __syncthreads();
        if (!histo) break;
        // boundary digit: the first bin at which the running count reaches `needed` (one thread; 2048 bins)
        if (t == 0) {
            uint32_t run = 0;
            int bstar = kBins - 1;
            for (int b = 0; b < kBins; ++b) {
                if (run + hist[b] >= needed) {
                    bstar = b;
                    break;
                }
                run += hist[b];
            }
            s_bstar = bstar;
            s_needed = needed - run;                  // still needed from the boundary bin
            s_done = (hist[bstar] == needed - run) ? 1 : 0;
        }
        __syncthreads();
        const int bstar = s_bstar;
        const uint32_t need_b = s_needed;
        emit_prefix = prefix;
        emit_fixed = fixed;
        emit_digit = bstar;
        emit_all_bin = s_done != 0;
        // the boundary bin becomes the new prefix
        const int digit_bits = (shift >= 0) ? kDigitBits : kDigitBits + shift;
        const uint64_t dig = (uint64_t)bstar >> (shift >= 0 ? 0 : -shift);
        prefix |= (shift >= 0) ? ((uint64_t)bstar << shift) : dig;
        fixed += digit_bits;
        needed = need_b;
        __syncthreads();
    }
    __syncthreads();
    // bitonic sort of the k keys (ascending), padded with all-ones keys to a power of two
    int m = 1;
    while (m < k) m <<= 1;
    for (int i = t; i < m; i += kTopkThreads)
        if (i >= k) keys[i] = ~0ull;
    __syncthreads();
    for (int size = 2; size <= m; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = t; i < m; i += kTopkThreads) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const uint64_t a = keys[i], b = keys[j];
                    if ((a > b) == up) {
                        keys[i] = b;
                        keys[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = t; i < k; i += kTopkThreads) {
        const uint64_t key = keys[i];
        val[(size_t)row * ldo + i] = key_value(key);
        idx[(size_t)row * ldo + i] = (int32_t)(uint32_t)key;
    }
}

}  // namespace

int topk(const float *pi, int64_t n, int64_t ld, int32_t Q, int32_t k, float *val, int32_t *idx, int64_t ldo,
         cudaStream_t s)
{
    if (Q < 0 || n < 0) return fail(AGP_EINVAL, "agp_topk: Q and n must be >= 0");
    if (Q == 0) return AGP_OK;
    if (k < 1 || k > kTopkMax || k > n) return fail(AGP_EINVAL, "agp_topk: need 1 <= k <= min(n, 2048)");
    if (n >= (1ll << 31)) return fail(AGP_EINVAL, "agp_topk: n must be < 2^31");
    if (ld < n || ldo < k) return fail(AGP_EINVAL, "agp_topk: need ld >= n and ldo >= k");
    if (!pi || !val || !idx) return fail(AGP_EINVAL, "agp_topk: NULL array");
    k_topk_rows<<<Q, kTopkThreads, 0, s>>>(pi, n, ld, k, val, idx, ldo);
    AGP_CUDA_TRY(cudaGetLastError());
    return AGP_OK;
}

}  // namespace agp
