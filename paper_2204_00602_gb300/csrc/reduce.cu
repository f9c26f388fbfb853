// Reductions over output distributions: sum of P(S), total variation
// distance (Eq. bosonsampling: 1/2 sum |p - q|), KL(q || p), and the gradient
// of the KL loss with respect to the amplitudes.
//
// Deterministic: each block reduces a fixed slice of the outputs with a
// shared-memory tree, and one block adds the block partials in index order.

#include <cmath>

#include "pcv_common.cuh"

namespace pcv {
namespace {

constexpr int kThreads = 256;
constexpr int kBlocksPerBatch = 256;     // slices per distribution

__device__ double block_sum(double v, double* sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = kThreads / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// grid (kBlocksPerBatch, B): partial sums of p, |p - q|, q log(q/p)
__global__ void __launch_bounds__(kThreads) stats_partial_kernel(const double* __restrict__ p, const double* __restrict__ q,
                                                                 int64_t N, int q_batched, double* __restrict__ part)
{
    __shared__ double sh[kThreads];
    const int b = blockIdx.y;
    const double* pb = p + (size_t)b * N;
    const double* qb = q ? q + (q_batched ? (size_t)b * N : 0) : nullptr;
    const int64_t per = (N + gridDim.x - 1) / gridDim.x;
    const int64_t lo = (int64_t)blockIdx.x * per, hi = min(N, lo + per);
    double s = 0, tv = 0, kl = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kThreads) {
        const double pi = pb[i];
        s += pi;
        if (qb) {
            const double qi = qb[i];
            tv += fabs(pi - qi);
            if (qi > 0) kl += qi * (log(qi) - log(pi));
        }
    }
    s = block_sum(s, sh);
    tv = block_sum(tv, sh);
    kl = block_sum(kl, sh);
    if (threadIdx.x == 0) {
        double* o = part + ((size_t)b * gridDim.x + blockIdx.x) * 3;
        o[0] = s;
        o[1] = tv;
        o[2] = kl;
    }
}

// grid (B): fixed-order sum of the partials -> out[b*3 + {sum p, TVD, KL}]
__global__ void __launch_bounds__(kThreads) stats_final_kernel(const double* __restrict__ part, int nparts, double* out)
{
    __shared__ double sh[kThreads];
    const int b = blockIdx.x;
    double v[3] = {0, 0, 0};
    for (int i = threadIdx.x; i < nparts; i += kThreads)
        for (int c = 0; c < 3; ++c) v[c] += part[((size_t)b * nparts + i) * 3 + c];
    for (int c = 0; c < 3; ++c) v[c] = block_sum(v[c], sh);
    if (threadIdx.x == 0) {
        out[b * 3 + 0] = v[0];
        out[b * 3 + 1] = 0.5 * v[1];
        out[b * 3 + 2] = v[2];
    }
}

// dL/da for L = scale * KL(q || p), p = |a|^2: with the dL/dRe + i dL/dIm
// convention, dL/da = 2 a dL/dp and dL/dp = -scale_b q / p (scale_b = scale * bscale[b]).
__global__ void kl_grad_kernel(const double* __restrict__ p, const double* __restrict__ q, const double2* __restrict__ amp,
                               int64_t N, int q_batched, const double* __restrict__ bscale, double scale,
                               double2* __restrict__ grad)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (i >= N) return;
    if (bscale) scale *= bscale[b];
    const size_t o = (size_t)b * N + i;
    const double qi = q[(q_batched ? (size_t)b * N : 0) + i];
    double2 g = make_double2(0.0, 0.0);
    if (qi > 0) {
        const double dp = -scale * qi / p[o];
        g = make_double2(2.0 * amp[o].x * dp, 2.0 * amp[o].y * dp);
    }
    grad[o] = g;
}

// dL/da = 2 a dL/dp for p = |a|^2 (dL/dRe + i dL/dIm convention).
__global__ void prob_grad_kernel(const double* __restrict__ gp, const double2* __restrict__ amp, int64_t count,
                                 double2* __restrict__ gamp)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double g = 2.0 * gp[i];
    gamp[i] = make_double2(g * amp[i].x, g * amp[i].y);
}

}  // namespace

cudaError_t launch_prob_grad(const double* gp, const double2* amp, int64_t count, double2* gamp, cudaStream_t s)
{
    prob_grad_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(gp, amp, count, gamp);
    note_launches(1);
    return cudaGetLastError();
}

int64_t stats_workspace(int B) { return (int64_t)B * kBlocksPerBatch * 3 * sizeof(double); }

cudaError_t launch_stats(const double* p, const double* q, int64_t N, int B, int q_batched, double* out,
                         double* ws, cudaStream_t s)
{
    stats_partial_kernel<<<dim3(kBlocksPerBatch, B), kThreads, 0, s>>>(p, q, N, q_batched, ws);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    stats_final_kernel<<<B, kThreads, 0, s>>>(ws, kBlocksPerBatch, out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_kl_grad(const double* p, const double* q, const double2* amp, int64_t N, int B, int q_batched,
                           const double* bscale, double scale, double2* grad, cudaStream_t s)
{
    kl_grad_kernel<<<dim3((unsigned)((N + 255) / 256), B), 256, 0, s>>>(p, q, amp, N, q_batched, bscale, scale, grad);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace pcv
