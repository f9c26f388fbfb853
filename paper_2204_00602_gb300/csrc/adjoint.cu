// Adjoint of the amplitude: dL/dU from dL/da for many outputs (explicit
// outputs of one U, or every output of the distribution of a batch of U).
//
// With Glynn's sign vector d on the columns of A = U_{T,S} (Eq. eqperm) and
// row sums x_i(d) = sum_j d_j A[i][j],
//     dPerm/dA[i][j] = 2^{-(n-1)} sum_d sigma(d) d_j prod_{i' != i} x_{i'}(d),
// the permanent of the minor of (i, j) written as a Glynn sum over the same
// Gray-code sequence as the forward kernel.  Each thread walks all 2^{n-1}
// sign vectors of one output, forms the leave-one-out products of its row
// sums from prefix and suffix products, and accumulates the n x n matrix
// G[i][j] in registers.  U[k][l] sits at every (i, j) with r_i = k and
// c_j = l, so with the dL/dRe + i dL/dIm convention
//     dL/dU[k][l] += gbar_S * conj(norm_S * sum_{r_i = k, c_j = l} G[i][j]).
// Contributions are summed per block in shared memory and per block into
// dL/dU with FP64 atomics (the summation order of these adds is not fixed).

#include "pcv_common.cuh"

namespace pcv {
namespace {

struct AdjArgs {
    const double2* U;        // [B][m][m]
    int m;
    int cols[PCV_MAX_PHOTONS];
    double norm_t;
    const uint8_t* out_occ;  // explicit outputs [count][m], or nullptr: canonical index o
    MultisetTable mc;
    int64_t count;           // outputs per batch entry
    const double2* gbar;     // [B][count]
    double2* gradU;          // [B][m][m], accumulated
};

template <int N>
__device__ __forceinline__ bool decode(const AdjArgs& a, int64_t o, int* rows, double& norm_s)
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
        int64_t idx = o;
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

template <int N>
__global__ void __launch_bounds__(128) adjoint_kernel(const AdjArgs a)
{
    extern __shared__ double2 sG[];     // [m][m] block accumulator
    const int b = blockIdx.y;
    const int m = a.m;
    for (int i = threadIdx.x; i < m * m; i += blockDim.x) sG[i] = make_double2(0.0, 0.0);
    __syncthreads();
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int rows[N];
    double norm_s = 1.0;
    bool ok = o < a.count && decode<N>(a, o, rows, norm_s);
    double2 g = make_double2(0.0, 0.0);
    if (ok) g = a.gbar[(size_t)b * a.count + o];
    if (ok && (g.x != 0.0 || g.y != 0.0)) {
        const double2* U = a.U + (size_t)b * m * m;
        double2 x[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {          // sign vector 0: all d_j = +1
            double2 s = U[rows[i] * m + a.cols[0]];
#pragma unroll
            for (int j = 1; j < N; ++j) s = cadd(s, U[rows[i] * m + a.cols[j]]);
            x[i] = s;
        }
        double2 G[N][N];
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = 0; j < N; ++j) G[i][j] = make_double2(0.0, 0.0);
        uint32_t gc = 0;                       // Gray code of the current sign vector
        double par = 1.0;                      // sigma(d) = prod_j d_j
        const uint32_t steps = 1u << (N - 1);
        for (uint32_t st = 0; st < steps; ++st) {
            double sj[N];                      // sigma(d) d_j
            sj[0] = par;
#pragma unroll
            for (int j = 1; j < N; ++j) sj[j] = ((gc >> (j - 1)) & 1u) ? -par : par;
            double2 pre[N];
            pre[0] = make_double2(1.0, 0.0);
            if (N > 1) pre[1] = x[0];
#pragma unroll
            for (int i = 2; i < N; ++i) pre[i] = cmul(pre[i - 1], x[i - 1]);
            double2 suf = make_double2(1.0, 0.0);
#pragma unroll
            for (int i = N - 1; i >= 0; --i) {
                const double2 L = (i == N - 1) ? pre[i] : (i == 0 ? suf : cmul(pre[i], suf));
#pragma unroll
                for (int j = 0; j < N; ++j) caxpy(G[i][j], sj[j], L);
                if (i > 0) suf = (i == N - 1) ? x[i] : cmul(suf, x[i]);
            }
            if (st + 1 < steps) {
                const uint32_t kk = st + 1;
                const int bb = __ffs(kk) - 1;
                const uint32_t gn = kk ^ (kk >> 1);
                const double sd = ((gn >> bb) & 1u) ? -2.0 : 2.0;
                const int col = a.cols[bb + 1];
#pragma unroll
                for (int i = 0; i < N; ++i) caxpy(x[i], sd, U[rows[i] * m + col]);
                gc = gn;
                par = -par;
            }
        }
        const double c = ldexp(norm_s * a.norm_t, -(N - 1));
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = 0; j < N; ++j) {
                // g * conj(c G)
                const double2 h = make_double2(c * G[i][j].x, -c * G[i][j].y);
                const double2 v = cmul(g, h);
                double2* dst = sG + rows[i] * m + a.cols[j];
                atomicAdd(&dst->x, v.x);
                atomicAdd(&dst->y, v.y);
            }
    }
    __syncthreads();
    double2* out = a.gradU + (size_t)b * m * m;
    for (int i = threadIdx.x; i < m * m; i += blockDim.x) {
        const double2 v = sG[i];
        if (v.x != 0.0) atomicAdd(&out[i].x, v.x);
        if (v.y != 0.0) atomicAdd(&out[i].y, v.y);
    }
}

template <int N>
cudaError_t adj_launch(const AdjArgs& a, int B, cudaStream_t s)
{
    const size_t smem = (size_t)a.m * a.m * sizeof(double2);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(adjoint_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)((a.count + 127) / 128), (unsigned)B);
    adjoint_kernel<N><<<grid, 128, smem, s>>>(a);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace

int adjoint_max_photons() { return 8; }

cudaError_t launch_adjoint(const Plan& p, const double2* U, int B, const uint8_t* out_occ, const int64_t* mc_table,
                           int64_t count, const double2* gbar, double2* gradU, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(gradU, 0, (size_t)B * p.m * p.m * sizeof(double2), s);
    if (e != cudaSuccess || count == 0 || p.n == 0) return e;
    AdjArgs a;
    a.U = U;
    a.m = p.m;
    for (int j = 0; j < PCV_MAX_PHOTONS; ++j) a.cols[j] = p.cols[j];
    a.norm_t = p.norm_t;
    a.out_occ = out_occ;
    a.mc.t = mc_table;
    a.mc.kmax = p.n;
    a.count = count;
    a.gbar = gbar;
    a.gradU = gradU;
    switch (p.n) {
    case 1: return adj_launch<1>(a, B, s);
    case 2: return adj_launch<2>(a, B, s);
    case 3: return adj_launch<3>(a, B, s);
    case 4: return adj_launch<4>(a, B, s);
    case 5: return adj_launch<5>(a, B, s);
    case 6: return adj_launch<6>(a, B, s);
    case 7: return adj_launch<7>(a, B, s);
    case 8: return adj_launch<8>(a, B, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace pcv
