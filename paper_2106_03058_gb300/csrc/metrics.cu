// metrics.cu -- the approximation-quality measures of the paper's experiments, on the GPU.
//
// Section 6 (local clustering with HKPR) measures an estimate against the exact propagation by
//   MaxError     = max_v | pi(v) / d_v - pi_hat(v) / d_v |   (normalised by the degree; the Katz
//                  experiments use the plain values, max_v | pi(v) - pi_hat(v) |), and
//   Precision@k  = | V_k ∩ V_hat_k | / k, with V_k and V_hat_k the k nodes of largest normalised
//                  exact and estimated value.
// Here the normalised value of a node with d_v = 0 is 0. MaxError is taken in FP64 from the FP32
// inputs. The top-k sets use the order of agp_topk (value descending, then id ascending) on the FP32
// normalised values (correctly rounded division), so the sets are unique.
#include <cmath>
#include <cstring>

#include "agp_internal.cuh"

namespace agp {
namespace {

__device__ __forceinline__ double norm_value(float x, const int32_t *deg, int64_t v)
{
    if (!deg) return (double)x;
    const int32_t d = deg[v];
    return d > 0 ? (double)x / (double)d : 0.0;
}

// largest |a - b| (normalised) as the bit pattern of a non-negative double, which orders like the
// value; one atomicMax per warp
__global__ void k_max_abs_diff(const float *a, const float *b, const int32_t *deg, int64_t n,
                               unsigned long long *out)
{
    double m = 0.0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(norm_value(a[v], deg, v) - norm_value(b[v], deg, v)));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// FP32 normalised values x(v) = pi(v) / d_v (0 when d_v = 0), the keys of the top-k sets
__global__ void k_normalise(const float *pi, const int32_t *deg, int64_t n, float *out)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = deg[v];
        out[v] = d > 0 ? __fdiv_rn(pi[v], (float)d) : 0.f;
    }
}

// |A ∩ B| of two sets of k distinct ids: one block; every id of A is searched in B
__global__ void __launch_bounds__(1024) k_overlap(const int32_t *ida, const int32_t *idb, int k, unsigned int *count)
{
    __shared__ int32_t sb[2048];
    for (int i = threadIdx.x; i < k; i += blockDim.x) sb[i] = idb[i];
    __syncthreads();
    unsigned int c = 0;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const int32_t x = ida[i];
        for (int j = 0; j < k; ++j) c += (sb[j] == x) ? 1u : 0u;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(count, c);
}

struct Scratch {
    void *p = nullptr;
    ~Scratch()
    {
        if (p) cudaFree(p);
    }
};

}  // namespace

int compare(const float *pi_est, const float *pi_ref, int64_t n, const int32_t *deg, int32_t k, double *max_error,
            double *precision_at_k, cudaStream_t s)
{
    if (!pi_est || !pi_ref || !max_error) return fail(AGP_EINVAL, "agp_compare: NULL argument");
    if (n < 1) return fail(AGP_EINVAL, "agp_compare: n must be >= 1");
    if (precision_at_k && (k < 1 || k > 2048 || k > n)) return fail(AGP_EINVAL, "agp_compare: need 1 <= k <= min(n, 2048)");
    if (precision_at_k && n >= (1ll << 31)) return fail(AGP_EINVAL, "agp_compare: n must be < 2^31");
    // scratch: the max (8 B), the overlap count (4 B, padded), and for Precision@k two normalised
    // vectors and two id lists
    const size_t head = 256;
    const size_t vec = precision_at_k && deg ? ((size_t)n * sizeof(float) + 255) / 256 * 256 : 0;
    const size_t ids = precision_at_k ? ((size_t)k * (sizeof(int32_t) + sizeof(float)) + 255) / 256 * 256 : 0;
    Scratch S;
    if (cudaMalloc(&S.p, head + 2 * vec + 2 * ids) != cudaSuccess) {
        cudaGetLastError();
        return fail(AGP_ENOMEM, "agp_compare: device scratch");
    }
    char *base = (char *)S.p;
    unsigned long long *d_max = (unsigned long long *)base;
    unsigned int *d_count = (unsigned int *)(base + 8);
    AGP_CUDA_TRY(cudaMemsetAsync(base, 0, head, s));
    const int grid = grid_stride_blocks();
    k_max_abs_diff<<<grid, kBlock, 0, s>>>(pi_est, pi_ref, deg, n, d_max);
    AGP_CUDA_TRY(cudaGetLastError());
    if (precision_at_k) {
        const float *ke = pi_est, *kr = pi_ref;
        if (deg) {
            float *ne = (float *)(base + head), *nr = (float *)(base + head + vec);
            k_normalise<<<grid, kBlock, 0, s>>>(pi_est, deg, n, ne);
            k_normalise<<<grid, kBlock, 0, s>>>(pi_ref, deg, n, nr);
            AGP_CUDA_TRY(cudaGetLastError());
            ke = ne;
            kr = nr;
        }
        char *ib = base + head + 2 * vec;
        int32_t *id_e = (int32_t *)ib, *id_r = (int32_t *)(ib + ids);
        float *val_e = (float *)(ib + (size_t)k * sizeof(int32_t)), *val_r = (float *)(ib + ids + (size_t)k * sizeof(int32_t));
        AGP_TRY(topk(ke, n, n, 1, k, val_e, id_e, k, s));
        AGP_TRY(topk(kr, n, n, 1, k, val_r, id_r, k, s));
        k_overlap<<<1, 1024, 0, s>>>(id_e, id_r, k, d_count);
        AGP_CUDA_TRY(cudaGetLastError());
    }
    unsigned long long h_max = 0;
    unsigned int h_count = 0;
    AGP_CUDA_TRY(cudaMemcpyAsync(&h_max, d_max, sizeof(h_max), cudaMemcpyDeviceToHost, s));
    AGP_CUDA_TRY(cudaMemcpyAsync(&h_count, d_count, sizeof(h_count), cudaMemcpyDeviceToHost, s));
    AGP_CUDA_TRY(cudaStreamSynchronize(s));
    double m;
    std::memcpy(&m, &h_max, sizeof(m));
    *max_error = m;
    if (precision_at_k) *precision_at_k = (double)h_count / (double)k;
    return AGP_OK;
}

}  // namespace agp
