// Plain Glynn/Gray-code permanent kernels: one permanent per group of G
// threads (G = 1..32, a warp at most) or per block (optionally split over
// several blocks with a deterministic second pass).
//
// Glynn's formula (Sec. 3.2.3 names it for the Naive back-end), applied to the
// columns of A = U_{T,S} (Eq. eqperm; Perm(A) = Perm(A^T)):
//   Perm(A) = 2^{-(n-1)} sum_{d in {+-1}^n, d_0 = +1} (prod_k d_k) prod_i x_i(d),
//   x_i(d) = sum_j d_j A[i][j].
// The 2^{n-1} sign vectors are visited in reflected Gray-code order: step k
// flips d_{b+1} with b = ctz(k), so each step changes every x_i by +-2 A[i][b+1]
// and the sign prod_k d_k alternates.  Each thread runs a contiguous chunk of
// steps whose start is a multiple of the chunk length; it rebuilds x from
// scratch at its chunk start, so rounding does not drift across chunks.
//
// FP64 instructions per Gray step and permanent: 2n (row-sum update, DFMA
// with +-2) + 4(n-1) (product) + 2 (signed accumulate) = 6n - 2.

#include "pcv_common.cuh"

namespace pcv {
namespace {

struct GlynnArgs {
    const double2* U;
    int m;
    int cols[PCV_MAX_PHOTONS];
    double norm_t;
    const uint8_t* out_occ;   // explicit outputs [count][m], or nullptr: unrank idx0 + o
    MultisetTable mc;
    int64_t idx0, count;
    double2* amp;
    double* prob;
    int use_smem;
};

// Rows of U_{T,S} for output o: the non-decreasing photon -> output-mode list.
// Returns false when the output's photon number is not N.  norm_s = 1/sqrt(prod s_i!).
template <int N>
__device__ __forceinline__ bool decode_output(const GlynnArgs& a, int64_t o, int* rows, double& norm_s)
{
    bool ok = true;
    if (a.out_occ) {
        const uint8_t* occ = a.out_occ + o * a.m;
        int r = -1, left = 0;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            while (left == 0 && r + 1 < a.m) { ++r; left = occ[r]; }
            if (left == 0) { ok = false; rows[i] = 0; }
            else { rows[i] = r; --left; }
        }
        if (left != 0) ok = false;
        for (int q = r + 1; q < a.m && ok; ++q) if (occ[q]) ok = false;
    } else {
        int64_t idx = a.idx0 + o;
        int v = 0;
#pragma unroll
        for (int p = 0; p < N; ++p) {
            for (;;) {
                const int64_t c = a.mc(a.m - v, N - p - 1);
                if (idx < c) break;
                idx -= c;
                ++v;
            }
            rows[p] = v;
        }
    }
    double f = 1.0;
    int run = 1;
#pragma unroll
    for (int i = 1; i < N; ++i) {
        run = (rows[i] == rows[i - 1]) ? run + 1 : 1;
        f *= (double)run;
    }
    norm_s = 1.0 / sqrt(f);
    return ok;
}

__device__ __forceinline__ void write_result(const GlynnArgs& a, int64_t o, double2 acc, int n, double norm_s, bool ok)
{
    double2 v = make_double2(0.0, 0.0);
    if (ok) {
        const double sc = ldexp(norm_s * a.norm_t, -(n - 1));
        v = make_double2(acc.x * sc, acc.y * sc);
    }
    if (a.amp) a.amp[o] = v;
    if (a.prob) a.prob[o] = fma(v.x, v.x, v.y * v.y);
}

// -------------------------------------------------- G threads per permanent
template <int N, int G>
__global__ void __launch_bounds__(256) glynn_group_kernel(const GlynnArgs a)
{
    extern __shared__ double2 sU[];
    const double2* U = a.U;
    if (a.use_smem) {
        for (int i = threadIdx.x; i < a.m * a.m; i += blockDim.x) sU[i] = a.U[i];
        __syncthreads();
        U = sU;
    }
    const int lg = threadIdx.x & (G - 1);
    const int64_t o = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    int rows[N];
    double norm_s = 1.0;
    const bool live = o < a.count;
    const bool ok = live && decode_output<N>(a, o, rows, norm_s);

    constexpr uint32_t L = (1u << (N - 1)) / G;   // Gray steps per thread
    double2 acc = make_double2(0.0, 0.0);
    if (ok) {
        int roff[N];
#pragma unroll
        for (int i = 0; i < N; ++i) roff[i] = rows[i] * a.m;
        const uint32_t k0 = (uint32_t)lg * L;
        const uint32_t g0 = k0 ^ (k0 >> 1);
        double2 x[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            double2 s = U[roff[i] + a.cols[0]];
#pragma unroll
            for (int j = 1; j < N; ++j) caxpy(s, ((g0 >> (j - 1)) & 1u) ? -1.0 : 1.0, U[roff[i] + a.cols[j]]);
            x[i] = s;
        }
        double par = (__popc(g0) & 1) ? -1.0 : 1.0;
        for (uint32_t st = 0; st < L; ++st) {
            double2 p = x[0];
#pragma unroll
            for (int i = 1; i < N; ++i) p = cmul(p, x[i]);
            caxpy(acc, par, p);
            par = -par;
            if (st + 1 < L) {
                const uint32_t kk = k0 + st + 1;
                const int b = __ffs(kk) - 1;
                const double sd = ((kk >> (b + 1)) & 1u) ? 2.0 : -2.0;
                const int col = a.cols[b + 1];
#pragma unroll
                for (int i = 0; i < N; ++i) caxpy(x[i], sd, U[roff[i] + col]);
            }
        }
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
    }
    if (lg == 0 && live) write_result(a, o, acc, N, norm_s, ok);
}

// ------------------------------------------- one block (x splits) per permanent
constexpr int kBlockThreads = 256;

template <int N>
__global__ void __launch_bounds__(kBlockThreads) glynn_block_kernel(const GlynnArgs a, int splits, double2* partial)
{
    __shared__ double2 sA[N * N];          // sA[j*N + i] = A[i][j] = U[rows[i]][cols[j]]
    __shared__ double2 sred[kBlockThreads / 32];
    __shared__ int srows[N];
    __shared__ int sok;
    __shared__ double snorm;
    const int64_t o = blockIdx.x / splits;
    const int sp = blockIdx.x % splits;
    if (threadIdx.x == 0) {
        int rows[N];
        double ns;
        sok = decode_output<N>(a, o, rows, ns);
        snorm = ns;
#pragma unroll
        for (int i = 0; i < N; ++i) srows[i] = rows[i];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < N * N; q += blockDim.x) {
        const int j = q / N, i = q % N;
        sA[q] = a.U[(size_t)srows[i] * a.m + a.cols[j]];
    }
    __syncthreads();

    double2 acc = make_double2(0.0, 0.0);
    if (sok) {
        const uint32_t units = (uint32_t)splits * kBlockThreads;
        const uint32_t L = (1u << (N - 1)) / units;
        const uint32_t k0 = ((uint32_t)sp * kBlockThreads + threadIdx.x) * L;
        const uint32_t g0 = k0 ^ (k0 >> 1);
        double2 x[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            double2 s = sA[i];
#pragma unroll
            for (int j = 1; j < N; ++j) caxpy(s, ((g0 >> (j - 1)) & 1u) ? -1.0 : 1.0, sA[j * N + i]);
            x[i] = s;
        }
        double par = (__popc(g0) & 1) ? -1.0 : 1.0;
        for (uint32_t st = 0; st < L; ++st) {
            double2 p = x[0];
#pragma unroll
            for (int i = 1; i < N; ++i) p = cmul(p, x[i]);
            caxpy(acc, par, p);
            par = -par;
            if (st + 1 < L) {
                const uint32_t kk = k0 + st + 1;
                const int b = __ffs(kk) - 1;
                const double sd = ((kk >> (b + 1)) & 1u) ? 2.0 : -2.0;
                const double2* col = sA + (b + 1) * N;
#pragma unroll
                for (int i = 0; i < N; ++i) caxpy(x[i], sd, col[i]);
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
    }
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 t = sred[0];
        for (int w = 1; w < kBlockThreads / 32; ++w) t = cadd(t, sred[w]);
        if (splits == 1) write_result(a, o, t, N, snorm, sok);
        else partial[o * splits + sp] = t;
    }
}

// Second pass of a split permanent: fixed-order sum of the block partials.
template <int N>
__global__ void glynn_finalize_kernel(const GlynnArgs a, int splits, const double2* partial)
{
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= a.count) return;
    int rows[N];
    double ns;
    const bool ok = decode_output<N>(a, o, rows, ns);
    double2 t = partial[o * splits];
    for (int q = 1; q < splits; ++q) t = cadd(t, partial[o * splits + q]);
    write_result(a, o, t, N, ns, ok);
}

__global__ void multiset_table_kernel(int64_t* t, int amax, int kmax)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a > amax) return;
    unsigned __int128 c = 1;                  // C(a+k-1, k) by the multiplicative recurrence
    bool sat = false;
    t[a * (kmax + 1)] = 1;
    for (int k = 1; k <= kmax; ++k) {
        if (!sat) {
            c = c * (unsigned __int128)(a + k - 1) / (unsigned __int128)k;
            if (c > (unsigned __int128)INT64_MAX) sat = true;
        }
        t[a * (kmax + 1) + k] = sat ? INT64_MAX : (int64_t)c;
    }
}

// n = 0: the empty output has amplitude 1, every other output 0.
__global__ void n0_kernel(const uint8_t* out_occ, int m, int64_t count, double2* amp, double* prob)
{
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= count) return;
    bool empty = true;
    if (out_occ) for (int r = 0; r < m; ++r) empty &= (out_occ[o * m + r] == 0);
    if (amp) amp[o] = make_double2(empty ? 1.0 : 0.0, 0.0);
    if (prob) prob[o] = empty ? 1.0 : 0.0;
}

GlynnArgs make_args(const Plan& p, const double2* U, const uint8_t* out_occ, const int64_t* mc_table,
                    int64_t idx0, int64_t count, double2* amp, double* prob)
{
    GlynnArgs a;
    a.U = U;
    a.m = p.m;
    for (int i = 0; i < PCV_MAX_PHOTONS; ++i) a.cols[i] = p.cols[i];
    a.norm_t = p.norm_t;
    a.out_occ = out_occ;
    a.mc.t = mc_table;
    a.mc.kmax = p.n;
    a.idx0 = idx0;
    a.count = count;
    a.amp = amp;
    a.prob = prob;
    a.use_smem = 0;
    return a;
}

template <int N, int G>
cudaError_t group_launch(GlynnArgs a, cudaStream_t s)
{
    if constexpr ((1 << (N - 1)) < G) {
        return cudaErrorInvalidValue;
    } else {
        const int threads = 256;
        const int64_t tot = a.count * G;
        const int64_t blocks = (tot + threads - 1) / threads;
        size_t smem = 0;
        if ((size_t)a.m * a.m * sizeof(double2) <= 48 * 1024) {
            a.use_smem = 1;
            smem = (size_t)a.m * a.m * sizeof(double2);
        }
        glynn_group_kernel<N, G><<<(unsigned)blocks, threads, smem, s>>>(a);
        note_launches(1);
        return cudaGetLastError();
    }
}

template <int N>
cudaError_t group_dispatch_g(GlynnArgs a, int G, cudaStream_t s)
{
    switch (G) {
    case 1: return group_launch<N, 1>(a, s);
    case 2: return group_launch<N, 2>(a, s);
    case 4: return group_launch<N, 4>(a, s);
    case 8: return group_launch<N, 8>(a, s);
    case 16: return group_launch<N, 16>(a, s);
    case 32: return group_launch<N, 32>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int N>
cudaError_t block_launch(GlynnArgs a, int splits, double2* partial, cudaStream_t s)
{
    const int64_t blocks = a.count * splits;
    glynn_block_kernel<N><<<(unsigned)blocks, kBlockThreads, 0, s>>>(a, splits, partial);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || splits == 1) return e;
    glynn_finalize_kernel<N><<<(unsigned)((a.count + 255) / 256), 256, 0, s>>>(a, splits, partial);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace

int glynn_block_threads() { return kBlockThreads; }

cudaError_t build_multiset_table(int64_t* t, int amax, int kmax, cudaStream_t s)
{
    multiset_table_kernel<<<(amax + 1 + 127) / 128, 128, 0, s>>>(t, amax, kmax);
    note_launches(1);
    return cudaGetLastError();
}

#define PCV_CASE_N(n, call) case n: return call<n>

cudaError_t launch_glynn_group(const Plan& p, const double2* U, const uint8_t* out_occ,
                               const int64_t* mc_table, int64_t idx0, int64_t count,
                               double2* amp, double* prob, int G, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    if (p.n == 0) {
        n0_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(out_occ, p.m, count, amp, prob);
        note_launches(1);
        return cudaGetLastError();
    }
    GlynnArgs a = make_args(p, U, out_occ, mc_table, idx0, count, amp, prob);
    switch (p.n) {
    case 1: return group_dispatch_g<1>(a, G, s);
    case 2: return group_dispatch_g<2>(a, G, s);
    case 3: return group_dispatch_g<3>(a, G, s);
    case 4: return group_dispatch_g<4>(a, G, s);
    case 5: return group_dispatch_g<5>(a, G, s);
    case 6: return group_dispatch_g<6>(a, G, s);
    case 7: return group_dispatch_g<7>(a, G, s);
    case 8: return group_dispatch_g<8>(a, G, s);
    case 9: return group_dispatch_g<9>(a, G, s);
    case 10: return group_dispatch_g<10>(a, G, s);
    case 11: return group_dispatch_g<11>(a, G, s);
    case 12: return group_dispatch_g<12>(a, G, s);
    case 13: return group_dispatch_g<13>(a, G, s);
    case 14: return group_dispatch_g<14>(a, G, s);
    case 15: return group_dispatch_g<15>(a, G, s);
    case 16: return group_dispatch_g<16>(a, G, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_glynn_block(const Plan& p, const double2* U, const uint8_t* out_occ,
                               const int64_t* mc_table, int64_t idx0, int64_t count,
                               double2* amp, double* prob, int splits, double2* partial,
                               cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    GlynnArgs a = make_args(p, U, out_occ, mc_table, idx0, count, amp, prob);
    switch (p.n) {
    case 9: return block_launch<9>(a, splits, partial, s);
    case 10: return block_launch<10>(a, splits, partial, s);
    case 11: return block_launch<11>(a, splits, partial, s);
    case 12: return block_launch<12>(a, splits, partial, s);
    case 13: return block_launch<13>(a, splits, partial, s);
    case 14: return block_launch<14>(a, splits, partial, s);
    case 15: return block_launch<15>(a, splits, partial, s);
    case 16: return block_launch<16>(a, splits, partial, s);
    case 17: return block_launch<17>(a, splits, partial, s);
    case 18: return block_launch<18>(a, splits, partial, s);
    case 19: return block_launch<19>(a, splits, partial, s);
    case 20: return block_launch<20>(a, splits, partial, s);
    case 21: return block_launch<21>(a, splits, partial, s);
    case 22: return block_launch<22>(a, splits, partial, s);
    case 23: return block_launch<23>(a, splits, partial, s);
    case 24: return block_launch<24>(a, splits, partial, s);
    case 25: return block_launch<25>(a, splits, partial, s);
    case 26: return block_launch<26>(a, splits, partial, s);
    case 27: return block_launch<27>(a, splits, partial, s);
    case 28: return block_launch<28>(a, splits, partial, s);
    case 29: return block_launch<29>(a, splits, partial, s);
    case 30: return block_launch<30>(a, splits, partial, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace pcv
