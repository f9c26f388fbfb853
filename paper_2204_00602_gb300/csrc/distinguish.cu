// Output distributions of partially distinguishable photons.
//
// Photons of one class are identical. Photons of different classes have
// orthogonal internal states, and the detectors count photons per mode only.
// Each class then evolves on its own, and the distribution of the total
// occupation is the multiset convolution of the classes' distributions:
//     P(S) = sum_{S_1 + S_2 = S} P_1(S_1) P_2(S_2),
// where each P_g is Eq. eqperm for that class's photons alone. A single
// photon entering in mode c lands in mode r with probability |U[r][c]|^2, so
// convolving with it is a gather over the occupied modes of S:
//     C(S) = sum_{r : s_r >= 1} A(S - e_r) |U[r][c]|^2.
// The source model mixes such terms with weights: the photon is absent,
// pure (in the one class of pure photons) or noisy (a class of its own).
// The host loop in pcv_api.cu sequences the launches; the kernels here
// compute one convolution step.
//
// Layout: a distribution over S_{m,k} is a dense float64 vector in canonical
// order. Ranks use the CUM table built by build_cum_table (O(k) per rank),
// and unranking uses the multiset-count table MC.

#include "pcv_common.cuh"

namespace pcv {
namespace {

struct RankTables {
    const int64_t* mc;     // MC[a*W + k] = C(a+k-1, k)
    const int64_t* cum;    // CUM[a*W + k] = sum_{v<a} MC[(m-v)*W + k]
    int m, W;              // W = kmax + 1
};

template <int KMAX>
__device__ __forceinline__ void unrank_modes(const RankTables& t, int k, int64_t idx, int* modes)
{
    int v = 0;
    for (int p = 0; p < k; ++p) {
        const int rest = k - p - 1;
        for (;;) {
            const int64_t c = t.mc[(t.m - v) * t.W + rest];
            if (idx < c) break;
            idx -= c;
            ++v;
        }
        modes[p] = v;
    }
}

// Rank in S_{m,len} of the sorted list holding cnt[j] copies of mode dm[j].
__device__ __forceinline__ int64_t rank_counts(const RankTables& t, const int* dm, const int* cnt, int d, int len)
{
    int64_t r = 0;
    int prev = 0, pos = 0;
    for (int j = 0; j < d; ++j) {
        for (int q = 0; q < cnt[j]; ++q) {
            const int rest = len - pos - 1;
            r += t.cum[dm[j] * t.W + rest] - t.cum[prev * t.W + rest];
            prev = dm[j];
            ++pos;
        }
    }
    return r;
}

// out(S) = alpha in_same(S) + beta sum_{r: s_r >= 1} in_prev(S - e_r) |U[r][c]|^2,
// S in S_{m,k}; in_same (S_{m,k}) and in_prev (S_{m,k-1}) may be null.
struct PhotonStep {
    RankTables t;
    int k, c;
    const double2* U;
    const double* in_same;
    const double* in_prev;
    double alpha, beta;
    double* out;
    int64_t count;
};

template <int KMAX>
__global__ void __launch_bounds__(256) photon_step_kernel(const PhotonStep a)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.count) return;
    double acc = a.in_same ? a.alpha * a.in_same[i] : 0.0;
    if (a.in_prev && a.k >= 1) {
        int modes[KMAX];
        unrank_modes<KMAX>(a.t, a.k, i, modes);
        const int m = a.t.m, W = a.t.W, k = a.k;
        double g = 0.0;
        for (int p = 0; p < k; ++p) {
            if (p + 1 < k && modes[p + 1] == modes[p]) continue;     // last copy of each occupied mode
            // rank of the list without position p, in S_{m,k-1}
            int64_t rk = 0;
            int prev = 0, pos = 0;
            for (int q = 0; q < k; ++q) {
                if (q == p) continue;
                const int rest = (k - 1) - pos - 1;
                rk += a.t.cum[modes[q] * W + rest] - a.t.cum[prev * W + rest];
                prev = modes[q];
                ++pos;
            }
            const double2 u = a.U[(size_t)modes[p] * m + a.c];
            g = fma(fma(u.x, u.x, u.y * u.y), a.in_prev[rk], g);
        }
        acc = fma(a.beta, g, acc);
    }
    a.out[i] = acc;
}

// C(S) = sum over S_1 <= S with |S_1| = a of A(S_1) B(S - S_1), S in S_{m,a+b}.
// The sub-multisets are the bounded compositions k_j in [0, mu_j] with
// sum k_j = a over the distinct modes of S, visited in lexicographic order:
// the successor raises the last k_j that still has room while something
// remains to its right, then refills the right part as low as it can go.
struct ClassConv {
    RankTables t;
    int a, b;
    const double* A;       // S_{m,a}
    const double* B;       // S_{m,b}
    double* C;             // S_{m,a+b}
    int64_t count;
};

template <int KMAX>
__global__ void __launch_bounds__(256) class_conv_kernel(const ClassConv g)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.count) return;
    const int n = g.a + g.b;
    int modes[KMAX];
    unrank_modes<KMAX>(g.t, n, i, modes);
    int dm[KMAX], mu[KMAX], cap[KMAX + 1], k[KMAX], rest[KMAX];
    int d = 0;
    for (int p = 0; p < n; ++p) {
        if (p == 0 || modes[p] != modes[p - 1]) {
            dm[d] = modes[p];
            mu[d] = 0;
            ++d;
        }
        mu[d - 1] += 1;
    }
    cap[d] = 0;
    for (int j = d - 1; j >= 0; --j) cap[j] = cap[j + 1] + mu[j];
    int rem = g.a;
    for (int j = 0; j < d; ++j) {
        k[j] = max(0, rem - cap[j + 1]);
        rem -= k[j];
    }
    double acc = 0.0;
    for (;;) {
        for (int j = 0; j < d; ++j) rest[j] = mu[j] - k[j];
        const int64_t r1 = rank_counts(g.t, dm, k, d, g.a);
        const int64_t r2 = rank_counts(g.t, dm, rest, d, g.b);
        acc = fma(g.A[r1], g.B[r2], acc);
        int j = d - 2, suf = k[d - 1];
        while (j >= 0 && !(k[j] < mu[j] && suf >= 1)) {
            suf += k[j];
            --j;
        }
        if (j < 0) break;
        k[j] += 1;
        rem = suf - 1;
        for (int q = j + 1; q < d; ++q) {
            k[q] = max(0, rem - cap[q + 1]);
            rem -= k[q];
        }
    }
    g.C[i] = acc;
}

// acc[i] += w x[i]
__global__ void scale_add_kernel(double* __restrict__ acc, const double* __restrict__ x, double w, int64_t count)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) acc[i] = fma(w, x[i], acc[i]);
}

__global__ void set_one_kernel(double* p) { *p = 1.0; }

unsigned blocks_for(int64_t count) { return (unsigned)((count + 255) / 256); }

}  // namespace

cudaError_t launch_photon_step(const int64_t* mc, const int64_t* cum, int m, int kmax, int k, const double2* U, int c,
                               const double* in_same, const double* in_prev, double alpha, double beta, double* out,
                               int64_t count, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    PhotonStep a;
    a.t = RankTables{mc, cum, m, kmax + 1};
    a.k = k;
    a.c = c;
    a.U = U;
    a.in_same = in_same;
    a.in_prev = in_prev;
    a.alpha = alpha;
    a.beta = beta;
    a.out = out;
    a.count = count;
    if (k <= 16) photon_step_kernel<16><<<blocks_for(count), 256, 0, s>>>(a);
    else photon_step_kernel<PCV_MAX_PHOTONS><<<blocks_for(count), 256, 0, s>>>(a);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_class_conv(const int64_t* mc, const int64_t* cum, int m, int kmax, int a, int b, const double* A,
                              const double* B, double* C, int64_t count, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    ClassConv g;
    g.t = RankTables{mc, cum, m, kmax + 1};
    g.a = a;
    g.b = b;
    g.A = A;
    g.B = B;
    g.C = C;
    g.count = count;
    if (a + b <= 16) class_conv_kernel<16><<<blocks_for(count), 256, 0, s>>>(g);
    else class_conv_kernel<PCV_MAX_PHOTONS><<<blocks_for(count), 256, 0, s>>>(g);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_scale_add(double* acc, const double* x, double w, int64_t count, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    scale_add_kernel<<<blocks_for(count), 256, 0, s>>>(acc, x, w, count);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_set_one(double* p, cudaStream_t s)
{
    set_one_kernel<<<1, 1, 0, s>>>(p);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace pcv
