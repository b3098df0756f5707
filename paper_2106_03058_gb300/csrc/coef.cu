// coef.cu -- the level coefficients of Def. 3.1, FP64 on the device.
//
// The level pipeline needs two numbers per lane and level i = 0..L, both ratios of the tail sums
// Y_i = sum_{k>=i} w_k of Def. 3.1:
//   f_i   = w_i / Y_i        the share of r^(i) that level i keeps as reserve,
//   rho_i = Y_{i+1} / Y_i    the factor every increment pushed at level i carries,
// and the normaliser Y_0 of Section 3 ("Assumptions on w_i": propagate with w / Y_0, rescale the
// result by Y_0). The stored reserve factor of a lane is keep_i = s * Y_0 * f_i with s = sign *
// ||x_part||_1 (the signal part's norm, Section 3 "Assumption on graph signal").
//
// They are computed as ratios, never as quotients of two separately summed tails:
//   PPR(alpha)   w_i = alpha (1-alpha)^i: f_i = alpha, rho_i = 1 - alpha, Y_0 = 1.
//   KATZ(beta)   w_i = beta^i:            f_i = 1 - beta, rho_i = beta, Y_0 = 1 / (1 - beta).
//   TRANSITION   w_L = 1:                 f_i = [i = L], rho_i = 1 for i < L, Y_0 = 1.
//   HKPR(t)      w_i = e^-t t^i / i!:     Y_0 = 1 (a Poisson law). Writing S_i = Y_i / w_i,
//                S_i = 1 + t/(i+1) S_{i+1}, so f_i = 1/S_i obeys the downward recurrence
//                f_i = (i+1) f_{i+1} / ((i+1) f_{i+1} + t), rho_i = t / ((i+1) f_{i+1} + t).
//                It is started at an index K >= 2t, where S_K = sum_{j>=0} prod_{m=1..j} t/(K+m)
//                converges geometrically (ratio <= 1/2). Each step maps a relative error e of
//                f_{i+1} to at most e t / ((i+1) f_{i+1} + t) < e, so errors shrink downwards, and
//                no step overflows or cancels, however small w_i / Y_i gets for i << t.
//   FINITE       the caller's w_0..w_L: suffix sums with Neumaier's compensated summation, then
//                f_i = w_i / Y_i and rho_i = Y_{i+1} / Y_i (zero once the tail is zero: the
//                propagation stops, Algorithm 2 has nothing left to push).
#include <cmath>
#include <vector>

#include "lanes.cuh"

namespace agp {

namespace {

// One coefficient row: f[0..L], rho[0..L] (rho_L = 0: nothing is pushed after the last level) and
// Y_0. Entries above L are not written.
__device__ void coef_row(const CoefSpec &S, const double *wts, double *f, double *rho, double *y0)
{
    const int L = S.L;
    switch (S.kind) {
    case AGP_W_PPR: {
        const double al = S.param;
        for (int i = 0; i <= L; ++i) {
            f[i] = al;
            rho[i] = 1.0 - al;
        }
        *y0 = 1.0;
        break;
    }
    case AGP_W_KATZ: {
        const double be = S.param;
        for (int i = 0; i <= L; ++i) {
            f[i] = 1.0 - be;
            rho[i] = be;
        }
        *y0 = 1.0 / (1.0 - be);
        break;
    }
    case AGP_W_HKPR: {
        const double t = S.param;
        int K = L + 1;
        if ((double)K < 2.0 * t) K = (int)ceil(2.0 * t);
        // S_K by its series: term_j = term_{j-1} * t / (K + j), each at most half the previous one
        double sum = 1.0, term = 1.0;
        for (int j = 1; j < 4096; ++j) {
            term *= t / (double)(K + j);
            sum += term;
            if (term <= 1e-18 * sum) break;
        }
        double fn = 1.0 / sum;  // f_K
        for (int i = K - 1; i >= 0; --i) {
            const double x = (double)(i + 1) * fn;  // (i+1) f_{i+1}
            const double fi = x / (x + t);
            if (i <= L) {
                f[i] = fi;
                rho[i] = t / (x + t);
            }
            fn = fi;
        }
        *y0 = 1.0;
        break;
    }
    case AGP_W_FINITE: {
        // Y_i for i = L..0, compensated; rho_i needs Y_{i+1}, so walk downwards keeping it
        double s = 0.0, comp = 0.0, next = 0.0;  // next = Y_{i+1}
        for (int i = L; i >= 0; --i) {
            const double w = wts[S.w_off + i];
            const double t = s + w;
            comp += (fabs(s) >= fabs(w)) ? (s - t) + w : (w - t) + s;
            s = t;
            const double Yi = s + comp;
            f[i] = Yi > 0.0 ? w / Yi : 0.0;
            rho[i] = (Yi > 0.0 && i < L) ? next / Yi : 0.0;
            next = Yi;
        }
        *y0 = next;
        break;
    }
    default: {  // AGP_W_TRANSITION
        for (int i = 0; i <= L; ++i) {
            f[i] = (i == L) ? 1.0 : 0.0;
            rho[i] = (i < L) ? 1.0 : 0.0;
        }
        *y0 = 1.0;
        break;
    }
    }
    rho[L] = 0.0;
    // once a tail is zero nothing reaches the later levels: their entries are zero
    for (int i = 1; i <= L; ++i)
        if (rho[i - 1] == 0.0) {
            f[i] = 0.0;
            rho[i] = 0.0;
        }
}

// One thread per lane: the lane's row of (keep_i, rho_i) in FP32, zero above L.
__global__ void k_coef(const CoefSpec *spec, const double *wts, float2 *coef, int nlanes)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nlanes) return;
    const CoefSpec S = spec[l];
    double f[kMaxLevels], rho[kMaxLevels], y0 = 0.0;
    coef_row(S, wts, f, rho, &y0);
    for (int i = 0; i < kMaxLevels; ++i) {
        float2 c = make_float2(0.f, 0.f);
        if (i <= S.L) c = make_float2((float)(S.scale * (y0 * f[i])), (float)rho[i]);
        coef[S.lane * kMaxLevels + i] = c;
    }
}

// The same row in FP64 for one parameter set (unit signal norm): out = [keep 0..L | rho 0..L | Y_0].
__global__ void k_coef_fp64(CoefSpec S, const double *wts, double *out)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double f[kMaxLevels], rho[kMaxLevels], y0 = 0.0;
    coef_row(S, wts, f, rho, &y0);
    for (int i = 0; i <= S.L; ++i) {
        out[i] = y0 * f[i];
        out[S.L + 1 + i] = rho[i];
    }
    out[2 * (S.L + 1)] = y0;
}

}  // namespace

void launch_coef(const CoefSpec *spec, const double *wts, float2 *coef, int nspec, cudaStream_t s)
{
    if (nspec > 0) k_coef<<<(nspec + 127) / 128, 128, 0, s>>>(spec, wts, coef, nspec);
}

int coefficients(const agp_params_t *p, double *keep, double *push, double *y0, int device, cudaStream_t s)
{
    if (!p || !keep || !push) return fail(AGP_EINVAL, "agp_coefficients: NULL argument");
    AGP_TRY(validate_params(*p));
    AGP_CUDA_TRY(cudaSetDevice(device));
    const int L = p->L;
    CoefSpec S{};
    S.lane = 0;
    S.kind = p->kind;
    S.L = L;
    S.param = p->param;
    S.w_off = 0;
    S.scale = 1.0;
    const size_t nw = (p->kind == AGP_W_FINITE) ? (size_t)L + 1 : 1;
    const size_t nout = 2 * ((size_t)L + 1) + 1;
    double *d = nullptr;
    AGP_CUDA_TRY(cudaMalloc(&d, sizeof(double) * (nw + nout)));
    std::vector<double> h(nout, 0.0);
    int rc = AGP_OK;
    cudaError_t e = cudaSuccess;
    if (p->kind == AGP_W_FINITE)
        e = cudaMemcpyAsync(d, p->w, sizeof(double) * nw, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_coef_fp64<<<1, 32, 0, s>>>(S, d, d + nw);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d + nw, sizeof(double) * nout, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = fail(AGP_ECUDA, std::string("agp_coefficients: ") + cudaGetErrorString(e));
    cudaFree(d);
    if (rc != AGP_OK) return rc;
    for (int i = 0; i <= L; ++i) {
        keep[i] = h[i];
        push[i] = h[L + 1 + i];
    }
    if (y0) *y0 = h[2 * (L + 1)];
    return AGP_OK;
}

}  // namespace agp
