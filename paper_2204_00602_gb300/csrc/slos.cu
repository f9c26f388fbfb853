// Full output distribution by photon-by-photon state expansion, the approach
// of the paper's SLOS back-end (Sec. 3.2.3: the full computation path unfolded
// in memory, O(n C(m+n-1, n)) time and memory), written for the GPU.
//
// The output state is prod_j (sum_r U[r][c_j] a_r^dagger) |0> / sqrt(prod t!)
// (Eq. eqperm's amplitudes are its coefficients).  With
// |psi_k> = prod_{j<=k} (sum_r U[r][c_j] a_r^dagger) |0> = sum_{s in S_{m,k}} B_k(s) |s>
// and a_r^dagger |s - e_r> = sqrt(s_r) |s>,
//     B_k(s) = sum_{r : s_r >= 1} U[r][c_k] sqrt(s_r) B_{k-1}(s - e_r),
// B_0 = 1, and a(S) = B_n(S) / sqrt(prod t!).  Each level k is a gather: one
// thread per state s of S_{m,k} (canonical order) adds one complex
// multiply-add per distinct occupied mode.  The last level is the
// distribution in canonical order.

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
    double2 acc = make_double2(0.0, 0.0);
    // for each distinct mode r (its last occurrence at position p): predecessor
    // = the list without position p (still sorted), ranked in S_{m,k-1}
    for (int p = 0; p < k; ++p) {
        if (p + 1 < k && modes[p + 1] == modes[p]) continue;
        const int r = modes[p];
        int mult = 1;
        for (int q = p - 1; q >= 0 && modes[q] == r; --q) ++mult;
        int64_t rk = 0;
        int prevm = 0, pos = 0;
        for (int q = 0; q < k; ++q) {
            if (q == p) continue;
            const int rest = (k - 1) - pos - 1;
            rk += a.cum[modes[q] * W + rest] - a.cum[prevm * W + rest];
            prevm = modes[q];
            ++pos;
        }
        double2 u = U[(size_t)r * m + a.col];
        if (mult > 1) {
            const double sq = sqrt((double)mult);
            u.x *= sq;
            u.y *= sq;
        }
        cmac(acc, u, prev[rk]);
    }
    if (a.amp || a.prob) {
        const double2 v = make_double2(acc.x * a.norm_t, acc.y * a.norm_t);
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
    if (n <= 8) return slos_levels<8>(a, B, p, buf0, buf1, half, prob, amp, s);
    if (n <= 16) return slos_levels<16>(a, B, p, buf0, buf1, half, prob, amp, s);
    return slos_levels<PCV_MAX_PHOTONS>(a, B, p, buf0, buf1, half, prob, amp, s);
}

}  // namespace pcv
