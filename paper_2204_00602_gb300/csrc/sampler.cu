// Exact boson sampling by the algorithm the paper's CliffordClifford2017
// back-end implements (Sec. 3.2.3: "adapted Glynn algorithm to efficiently
// compute n simultaneous sub-permanents", O(n 2^n + m n^2) per sample).
//
// With A the m x n matrix of the input photons' columns of U (randomly
// permuted per sample), photon positions are drawn one at a time.  After
// r_1..r_{k-1} have been drawn, the next position i has weight
//     w_i = | sum_{l<k} A[i][l] Perm(A[r_1..r_{k-1}; {0..k-1} \ l]) |^2,
// the Laplace expansion along the new row of Perm(A[r_1..r_{k-1}, i; 0..k-1]).
// The k leave-one-column-out permanents come from one Glynn sum over the
// k-1 rows: with x_j(d) = sum_i d_i M[i][j] and leave-one-out products,
//     Perm(M_{-l}) = 2^{-(k-2)} sum_{d, d_1=+1} (prod d) prod_{j != l} x_j(d).
// One warp per sample: lanes split the Gray-code sequence of sign vectors
// (shuffle reduction), then the m weights, then an inverse-CDF draw with a
// warp prefix sum.  The random numbers (column permutation, one uniform per
// photon) are inputs, so a sample is a deterministic function of them.

#include "pcv_common.cuh"

namespace pcv {
namespace {

constexpr int kSampWarps = 4;

struct SampArgs {
    const double2* U;         // m x m
    int m, n;
    int cols[PCV_MAX_PHOTONS];
    const uint8_t* perm;      // [count][n] column permutation per sample
    const double* uni;        // [count][n] uniforms in [0, 1)
    int64_t count;
    uint8_t* out;             // [count][m] occupations
};

template <int NMAX>
__global__ void __launch_bounds__(32 * kSampWarps) sampler_kernel(const SampArgs a)
{
    extern __shared__ double2 sA[];           // A[i][l] = U[i][cols[l]], m x n
    const int m = a.m, n = a.n;
    for (int q = threadIdx.x; q < m * n; q += blockDim.x) {
        const int i = q / n, l = q % n;
        sA[q] = a.U[(size_t)i * m + a.cols[l]];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t smp = (int64_t)blockIdx.x * kSampWarps + warp;
    if (smp >= a.count) return;
    const uint8_t* perm = a.perm + smp * n;
    const double* uni = a.uni + smp * n;
    int rows[NMAX];                            // drawn positions
    int pc[NMAX];                              // permuted column order
#pragma unroll
    for (int l = 0; l < NMAX; ++l) pc[l] = l < n ? min((int)perm[l], n - 1) : 0;   // clamp keeps reads in bounds

    for (int k = 1; k <= n; ++k) {
        // ---- leave-one-out permanents P_l of M = A[rows[0..k-2]; pc[0..k-1]]
        double2 P[NMAX];
#pragma unroll
        for (int l = 0; l < NMAX; ++l) P[l] = make_double2(0.0, 0.0);
        if (k == 1) {
            P[0] = make_double2(lane == 0 ? 1.0 : 0.0, 0.0);
        } else {
            const int R = k - 1;                                // rows of M
            const uint32_t steps = 1u << (R - 1);               // sign vectors with d_0 = +1
            const uint32_t per = steps >= 32 ? steps / 32 : 1;
            const uint32_t k0 = (uint32_t)lane * per;
            if (k0 < steps) {
                uint32_t g = k0 ^ (k0 >> 1);
                double2 x[NMAX];
#pragma unroll
                for (int j = 0; j < NMAX; ++j) {
                    if (j >= k) continue;
                    double2 s = sA[rows[0] * n + pc[j]];
                    for (int i = 1; i < R; ++i) caxpy(s, ((g >> (i - 1)) & 1u) ? -1.0 : 1.0, sA[rows[i] * n + pc[j]]);
                    x[j] = s;
                }
                double par = (__popc(g) & 1) ? -1.0 : 1.0;
                for (uint32_t st = 0; st < per; ++st) {
                    // leave-one-out products of x_0..x_{k-1}
                    double2 pre = make_double2(par, 0.0);
                    double2 pres[NMAX];
#pragma unroll
                    for (int j = 0; j < NMAX; ++j) {
                        if (j >= k) continue;
                        pres[j] = pre;
                        pre = cmul(pre, x[j]);
                    }
                    double2 suf = make_double2(1.0, 0.0);
#pragma unroll
                    for (int j = NMAX - 1; j >= 0; --j) {
                        if (j >= k) continue;
                        const double2 t = cmul(pres[j], suf);
                        P[j] = cadd(P[j], t);
                        suf = cmul(suf, x[j]);
                    }
                    if (st + 1 < per) {
                        const uint32_t kk = k0 + st + 1;
                        const int b = __ffs(kk) - 1;
                        const double sd = ((kk >> (b + 1)) & 1u) ? 2.0 : -2.0;
                        const int rr = rows[b + 1];
#pragma unroll
                        for (int j = 0; j < NMAX; ++j)
                            if (j < k) caxpy(x[j], sd, sA[rr * n + pc[j]]);
                        par = -par;
                    }
                }
            }
            const double sc = ldexp(1.0, -(R - 1));
#pragma unroll
            for (int j = 0; j < NMAX; ++j) {
                if (j >= k) continue;
                for (int off = 16; off > 0; off >>= 1) {
                    P[j].x += __shfl_xor_sync(0xffffffffu, P[j].x, off);
                    P[j].y += __shfl_xor_sync(0xffffffffu, P[j].y, off);
                }
                P[j].x *= sc;
                P[j].y *= sc;
            }
        }
        if (k == 1) {                                   // every lane needs P_0 = 1
            P[0] = make_double2(1.0, 0.0);
        }
        // ---- weights of the m candidate positions, inverse-CDF draw
        double wloc[4];
        double part = 0.0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int i = lane + 32 * c;
            double w = 0.0;
            if (i < m) {
                double2 s = make_double2(0.0, 0.0);
#pragma unroll
                for (int j = 0; j < NMAX; ++j)
                    if (j < k) cmac(s, sA[i * n + pc[j]], P[j]);
                w = fma(s.x, s.x, s.y * s.y);
            }
            wloc[c] = w;
            part += w;
        }
        // total and lane prefix of the per-lane sums (modes lane, lane+32, ... belong to lane)
        double incl = part;
        for (int off = 1; off < 32; off <<= 1) {
            const double v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += v;
        }
        const double total = __shfl_sync(0xffffffffu, incl, 31);
        const double target = uni[k - 1] * total;
        // the lane whose cumulative range holds the target picks within its modes
        const double before = incl - part;
        int pick = -1;
        if (target >= before && target < incl) {
            double acc = before;
            int lastpos = -1;
            for (int c = 0; c < 4; ++c) {
                const int i = lane + 32 * c;
                if (i >= m) break;
                if (wloc[c] > 0.0) lastpos = i;
                acc += wloc[c];
                if (target < acc) { pick = i; break; }
            }
            if (pick < 0) pick = lastpos;          // rounding: this lane's last mode with weight
        }
        const unsigned ball = __ballot_sync(0xffffffffu, pick >= 0);
        int chosen;
        if (ball) {
            const int src = __ffs(ball) - 1;
            chosen = __shfl_sync(0xffffffffu, pick, src);
        } else {                                        // rounding at the top end: last mode with weight
            int last = -1;
            for (int c = 3; c >= 0 && last < 0; --c) {
                const int i = lane + 32 * c;
                if (i < m && wloc[c] > 0.0) last = i;
            }
            int best = last;
            for (int off = 16; off > 0; off >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, off));
            chosen = best < 0 ? 0 : best;
        }
        rows[k - 1] = chosen;
    }
    for (int i = lane; i < m; i += 32) {
        int c = 0;
        for (int p = 0; p < n; ++p) c += rows[p] == i;
        a.out[smp * m + i] = (uint8_t)c;
    }
}

}  // namespace

cudaError_t launch_sampler(const Plan& p, const double2* U, const uint8_t* perm, const double* uni, int64_t count,
                           uint8_t* out, cudaStream_t s)
{
    SampArgs a;
    a.U = U;
    a.m = p.m;
    a.n = p.n;
    for (int j = 0; j < PCV_MAX_PHOTONS; ++j) a.cols[j] = p.cols[j];
    a.perm = perm;
    a.uni = uni;
    a.count = count;
    a.out = out;
    const size_t smem = (size_t)p.m * p.n * sizeof(double2);
    const unsigned blocks = (unsigned)((count + kSampWarps - 1) / kSampWarps);
    cudaError_t e;
    if (p.n <= 8) {
        if (smem > 48 * 1024 &&
            (e = cudaFuncSetAttribute(sampler_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        sampler_kernel<8><<<blocks, 32 * kSampWarps, smem, s>>>(a);
    } else {
        if (smem > 48 * 1024 &&
            (e = cudaFuncSetAttribute(sampler_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        sampler_kernel<16><<<blocks, 32 * kSampWarps, smem, s>>>(a);
    }
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace pcv
