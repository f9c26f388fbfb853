// Full output distribution by photon-by-photon state expansion, the approach
// of the paper's SLOS back-end (Sec. 3.2.3: the full computation path unfolded
// in memory, O(n C(m+n-1, n)) time and memory), written for the GPU.
//
// The output state is prod_j (sum_r U[r][c_j] a_r^dagger) |0> / sqrt(prod t!)
// (Eq. eqperm's amplitudes are its coefficients).  With
// |psi_k> = prod_{j<=k} (sum_r U[r][c_j] a_r^dagger) |0> = sum_{s in S_{m,k}} B_k(s) |s>
// and a_r^dagger |s - e_r> = sqrt(s_r) |s>,
//     B_k(s) = sum_{r : s_r >= 1} U[r][c_k] sqrt(s_r) B_{k-1}(s - e_r),
// B_0 = 1, and a(S) = B_n(S) / sqrt(prod t!).  The kernels carry
// C_k(s) = B_k(s) / sqrt(prod_r s_r!) instead: since (s - e_r)! differs from
// s! by the factor s_r, the square roots cancel and
//     C_k(s) = sum_{r : s_r >= 1} U[r][c_k] C_{k-1}(s - e_r),
// a plain gather with one complex multiply-add per distinct occupied mode
// and no square root; the last level applies
// a(S) = C_n(S) sqrt(prod s!) / sqrt(prod t!).  One thread per state s of
// S_{m,k} (canonical order); the last level is the distribution in
// canonical order.

#include <cmath>

#include "pcv_common.cuh"

namespace pcv {
namespace {

// CUM[a][k] = sum_{v < a} MC(m - v, k): the rank contribution of all lists
// whose current position is below a.
__global__ void cum_table_kernel(const int64_t* __restrict__ mc, int m, int kmax, int64_t* __restrict__ cum)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > kmax) return;
    int64_t acc = 0;
    for (int a = 0; a <= m; ++a) {
        cum[a * (kmax + 1) + k] = acc;
        if (a < m) acc += mc[(m - a) * (kmax + 1) + k];
    }
}

struct SlosArgs {
    const double2* U;          // [B][m][m]
    int m, n, k;               // level being built
    int col;                   // input mode of photon k
    int kmax;                  // table width - 1
    const int64_t* mc;         // multiset counts MC[a][k] = C(a+k-1, k)
    const int64_t* cum;        // prefix sums of MC over the first position
    int64_t count;             // states of level k
    int64_t prev_stride, cur_stride;
    const double2* prev;       // [B][C(m+k-2, k-1)]
    double2* cur;              // [B][count] (intermediate levels)
    double norm_t;             // last level: 1/sqrt(prod t!)
    double sqrtfact[PCV_MAX_PHOTONS + 1];   // sqrt(j!)
    double2* amp;              // last level outputs (or null)
    double* prob;
};

template <int KMAX>
__global__ void __launch_bounds__(256) slos_level_kernel(const SlosArgs a)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.count) return;
    const int b = blockIdx.y;
    const int k = a.k, m = a.m, W = a.kmax + 1;
    // unrank i in S_{m,k}
    int modes[KMAX];
    {
        int64_t idx = i;
        int v = 0;
        for (int p = 0; p < k; ++p) {
            const int rest = k - p - 1;
            for (;;) {
                const int64_t c = a.mc[(m - v) * W + rest];
                if (idx < c) break;
                idx -= c;
                ++v;
            }
            modes[p] = v;
        }
    }
    const double2* U = a.U + (size_t)b * m * m;
    const double2* prev = a.prev + (size_t)b * a.prev_stride;
    // Predecessor of position p (the list without modes[p]) in S_{m,k-1}:
    //   rank_p = A_p + J_p + B_p, with
    //   A_p = sum_{q<p} CUM[modes_q][k-2-q] - CUM[modes_{q-1}][k-2-q]   (positions before p keep their index)
    //   J_p = CUM[modes_{p+1}][k-2-p] - CUM[modes_{p-1}][k-2-p]         (the position after p, shifted down)
    //   B_p = sum_{q>=p+2} CUM[modes_q][k-1-q] - CUM[modes_{q-1}][k-1-q] (later positions, shifted down)
    // with modes_{-1} = 0; B is a suffix sum, so all predecessors cost O(k).
    int64_t suffix = 0;                        // B for the current p, starting from the full sum over q >= 2
    for (int q = 2; q < k; ++q) suffix += a.cum[modes[q] * W + (k - 1 - q)] - a.cum[modes[q - 1] * W + (k - 1 - q)];
    double2 acc = make_double2(0.0, 0.0);
    int64_t pre = 0;                           // A_p
    int mult = 0;
    double sfac = 1.0;                         // sqrt(prod s!) (used by the last level)
    for (int p = 0; p < k; ++p) {
        const int r = modes[p];
        mult = (p > 0 && modes[p - 1] == r) ? mult + 1 : 1;
        const bool last = !(p + 1 < k && modes[p + 1] == r);   // one term per distinct mode, at its last copy
        if (last) {
            const int before = p > 0 ? modes[p - 1] : 0;
            const int64_t junction = p + 1 < k ? a.cum[modes[p + 1] * W + (k - 2 - p)] - a.cum[before * W + (k - 2 - p)] : 0;
            const int64_t rk = pre + junction + suffix;
            cmac(acc, U[(size_t)r * m + a.col], prev[rk]);
            if (mult > 1) sfac *= a.sqrtfact[mult];
        }
        // advance to p + 1: A gains position p at rest k-2-p; B loses position p+2
        if (p + 1 < k) {
            const int pm = p > 0 ? modes[p - 1] : 0;
            pre += a.cum[r * W + (k - 2 - p)] - a.cum[pm * W + (k - 2 - p)];
            if (p + 2 < k) suffix -= a.cum[modes[p + 2] * W + (k - 3 - p)] - a.cum[modes[p + 1] * W + (k - 3 - p)];
        }
    }
    if (a.amp || a.prob) {
        const double sc = sfac * a.norm_t;
        const double2 v = make_double2(acc.x * sc, acc.y * sc);
        if (a.amp) a.amp[(size_t)b * a.cur_stride + i] = v;
        if (a.prob) a.prob[(size_t)b * a.cur_stride + i] = fma(v.x, v.x, v.y * v.y);
    } else {
        a.cur[(size_t)b * a.cur_stride + i] = acc;
    }
}

__global__ void slos_init_kernel(double2* lvl0, int64_t stride, int B)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) lvl0[(size_t)b * stride] = make_double2(1.0, 0.0);
}

int64_t mset_s(int w, int k)
{
    if (k == 0) return 1;
    if (w <= 0) return 0;
    unsigned __int128 c = 1;
    for (int i = 1; i <= k; ++i) {
        c = c * (unsigned __int128)(w - 1 + i) / (unsigned __int128)i;
        if (c > (unsigned __int128)INT64_MAX) return -1;
    }
    return (int64_t)c;
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

template <int KMAX>
cudaError_t slos_levels(SlosArgs a, int B, const Plan& p, double2* buf0, double2* buf1, int64_t half,
                        double* prob, double2* amp, cudaStream_t s)
{
    double2* prev = buf0;
    double2* cur = buf1;
    for (int k = 1; k <= p.n; ++k) {
        a.k = k;
        a.col = p.cols[k - 1];
        a.count = mset_s(p.m, k);
        a.prev = prev;
        a.prev_stride = half;
        a.cur = cur;
        a.cur_stride = k == p.n ? a.count : half;
        const bool last = k == p.n;
        a.amp = last ? amp : nullptr;
        a.prob = last ? prob : nullptr;
        if (last && !amp && !prob) return cudaErrorInvalidValue;
        dim3 grid((unsigned)((a.count + 255) / 256), (unsigned)B);
        slos_level_kernel<KMAX><<<grid, 256, 0, s>>>(a);
        note_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        double2* t = prev;
        prev = cur;
        cur = t;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t build_cum_table(const int64_t* mc, int m, int kmax, int64_t* cum, cudaStream_t s)
{
    cum_table_kernel<<<(kmax + 32) / 32, 32, 0, s>>>(mc, m, kmax, cum);
    note_launches(1);
    return cudaGetLastError();
}

// Workspace: MC and CUM tables, then two level buffers of the largest
// intermediate level per batch entry.
int64_t slos_workspace(int B, int m, int n)
{
    int64_t half = 1;
    for (int k = 0; k < n; ++k) {
        const int64_t c = mset_s(m, k);
        if (c < 0) return -1;
        half = c > half ? c : half;
    }
    return (int64_t)(2 * al256((size_t)(m + 1) * (n + 1) * sizeof(int64_t)) +
                     2 * al256((size_t)B * half * sizeof(double2)));
}

cudaError_t launch_slos(const Plan& p, int B, const double2* U, double* prob, double2* amp, void* ws, cudaStream_t s)
{
    const int m = p.m, n = p.n;
    int64_t half = 1;
    for (int k = 0; k < n; ++k) {
        const int64_t c = mset_s(m, k);
        half = c > half ? c : half;
    }
    char* w = (char*)ws;
    int64_t* mc = (int64_t*)w;          w += al256((size_t)(m + 1) * (n + 1) * sizeof(int64_t));
    int64_t* cum = (int64_t*)w;         w += al256((size_t)(m + 1) * (n + 1) * sizeof(int64_t));
    double2* buf0 = (double2*)w;        w += al256((size_t)B * half * sizeof(double2));
    double2* buf1 = (double2*)w;
    cudaError_t e = build_multiset_table(mc, m, n, s);
    if (e != cudaSuccess) return e;
    if ((e = build_cum_table(mc, m, n, cum, s)) != cudaSuccess) return e;
    slos_init_kernel<<<(B + 127) / 128, 128, 0, s>>>(buf0, half, B);
    note_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    SlosArgs a;
    a.U = U;
    a.m = m;
    a.n = n;
    a.kmax = n;
    a.mc = mc;
    a.cum = cum;
    a.norm_t = p.norm_t;
    {
        double f = 1.0;
        a.sqrtfact[0] = 1.0;
        for (int j = 1; j <= PCV_MAX_PHOTONS; ++j) {
            f *= j;
            a.sqrtfact[j] = std::sqrt(f);
        }
    }
    if (n <= 8) return slos_levels<8>(a, B, p, buf0, buf1, half, prob, amp, s);
    if (n <= 16) return slos_levels<16>(a, B, p, buf0, buf1, half, prob, amp, s);
    return slos_levels<PCV_MAX_PHOTONS>(a, B, p, buf0, buf1, half, prob, amp, s);
}

}  // namespace pcv
