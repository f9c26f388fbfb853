// Full output distribution by a factorised Glynn sum.
//
// Put Glynn's sign vector on the input photons (columns of U_{T,S}, Eq.
// eqperm).  The row sum of output row i then depends only on the output mode
// r_i:  y_r(d) = sum_j d_j U[r][c_j].  Every output S therefore shares the
// same m row sums per sign vector d, and
//     a(S) = norm_t 2^{-(n-1)} sum_d sigma(d) prod_r y_r(d)^{s_r} / sqrt(s_r!).
// Split the modes at h: S = (P on modes [0,h), Q on modes [h,m)).  With
//     alpha_P(d) = sigma(d) 2^{-(n-1)} norm_t prod_{r<h} y_r^{P_r}/sqrt(P_r!),
//     beta_Q(d)  = prod_{r>=h} y_r^{Q_r}/sqrt(Q_r!),
// every output is a(S) = sum_d alpha_P(d) beta_Q(d): for each k = |P| this is
// a complex matrix product over the sign vectors, one complex multiply-add
// (4 DFMA) per output and sign vector, instead of the 6n-2 FP64 instructions
// of a Gray step of the plain per-output kernel.
//
// Pipeline per chunk of KC sign vectors (all vectors at once when the
// workspace allows):
//   row_sums_kernel y_r(d) by Gray-code row-sum updates (one column per step)
//   level_kernel   alpha/beta tables level by level: entry(P) = entry(P minus
//                  its last mode) * y_last / sqrt(multiplicity)
//   gemm_kernel    a(S) = sum_d alpha_P(d) beta_Q(d), written at the
//                  canonical index lowbase(P) + rank(Q)
//
// The canonical index of S (lexicographic order of the non-decreasing mode
// list) splits as lowbase(P) + rank of Q among the (n-k)-multisets over
// [h, m), because all outputs whose first k photons are P and whose others
// lie in [h, m) are contiguous in that order.

#include <algorithm>

#include "pcv_common.cuh"

namespace pcv {
namespace {

constexpr int kYRun = 32;          // sign vectors per row_sums_kernel thread

struct ColList { int c[PCV_MAX_PHOTONS]; };

__global__ void row_sums_kernel(const double2* __restrict__ U, int m, int n, ColList cols,
                                int64_t d0, int kc, double2* __restrict__ Y)
{
    // thread -> (row r, run of kYRun consecutive sign vectors)
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int runs = (kc + kYRun - 1) / kYRun;
    if (t >= (int64_t)m * runs) return;
    const int r = (int)(t % m);
    const int run = (int)(t / m);
    const double2* Ur = U + (size_t)r * m;
    const int64_t dstart = d0 + (int64_t)run * kYRun;
    const int len = min(kYRun, kc - run * kYRun);
    uint64_t g = (uint64_t)dstart ^ ((uint64_t)dstart >> 1);
    double2 y = __ldg(Ur + cols.c[0]);
    for (int j = 1; j < n; ++j) caxpy(y, ((g >> (j - 1)) & 1u) ? -1.0 : 1.0, __ldg(Ur + cols.c[j]));
    for (int q = 0; q < len; ++q) {
        Y[(int64_t)(run * kYRun + q) * m + r] = y;
        if (q + 1 < len) {                       // Gray step to d+1: flip one sign
            const uint64_t kk = (uint64_t)(dstart + q + 1);
            const int b = __ffsll((long long)kk) - 1;
            const double sd = ((kk >> (b + 1)) & 1u) ? 2.0 : -2.0;
            caxpy(y, sd, __ldg(Ur + cols.c[b + 1]));
        }
    }
}

struct LevelArgs {
    MultisetTable mc;      // global table, a <= m, k <= n
    int m, n, h;
    int side;              // 0 = low modes [0,h), 1 = high modes [h,m)
    int k;                 // level (multiset size)
    int64_t count;         // entries of this level
    int64_t off, poff;     // table offsets of level k and k-1
    int64_t width;         // row length of the table (all levels)
    int kc;
    int64_t d0;
    double lead;           // low side level 0: 2^{-(n-1)} norm_t
    const double2* Y;
    double2* T;
    int64_t* lowbase;      // low side: canonical base index of each P (level k == n - |Q| pairing)
};

__global__ void level_kernel(const LevelArgs a)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.count) return;
    const int w = a.side == 0 ? a.h : a.m - a.h;
    const int shift = a.side == 0 ? 0 : a.h;
    if (a.k == 0) {
        for (int q = 0; q < a.kc; ++q) {
            double v = 1.0;
            if (a.side == 0) {
                const uint64_t d = (uint64_t)(a.d0 + q);
                v = (__popcll(d ^ (d >> 1)) & 1) ? -a.lead : a.lead;
            }
            a.T[(int64_t)q * a.width] = make_double2(v, 0.0);
        }
        if (a.side == 0 && a.lowbase) {
            int64_t r = 0;
            if (a.n > 0) for (int v = 0; v < a.h; ++v) r += a.mc(a.m - v, a.n - 1);
            a.lowbase[0] = r;
        }
        return;
    }
    // Level-local multiset tables count C(w' + k - 1, k) for w' <= w; the global
    // table (a <= m) covers them.
    int modes[PCV_MAX_PHOTONS];
    {
        int64_t idx = i;
        int v = 0;
        for (int p = 0; p < a.k; ++p) {
            const int rest = a.k - p - 1;
            for (;;) {
                const int64_t c = a.mc(w - v, rest);
                if (idx < c) break;
                idx -= c;
                ++v;
            }
            modes[p] = v;
        }
    }
    const int64_t parent = rank_multiset(a.mc, w, a.k - 1, modes);
    const int last = modes[a.k - 1];
    int mult = 1;
    for (int p = a.k - 2; p >= 0 && modes[p] == last; --p) ++mult;
    const double sc = mult > 1 ? inv_sqrt_int(mult) : 1.0;
    const int r = last + shift;

    if (a.side == 0 && a.lowbase) {
        // canonical index of the first output with prefix P and the rest in [h, m)
        int64_t base = 0;
        int prev = 0;
        for (int p = 0; p < a.k; ++p) {
            for (int v = prev; v < modes[p]; ++v) base += a.mc(a.m - v, a.n - p - 1);
            prev = modes[p];
        }
        if (a.k < a.n)
            for (int v = prev; v < a.h; ++v) base += a.mc(a.m - v, a.n - a.k - 1);
        a.lowbase[a.off + i] = base;
    }

    const double2* __restrict__ Tp = a.T + a.poff + parent;
    const double2* __restrict__ Yr = a.Y + r;
    double2* __restrict__ Tout = a.T + a.off + i;
    if (mult > 1) {
        for (int q = 0; q < a.kc; ++q) {
            double2 y = Yr[(int64_t)q * a.m];
            y.x *= sc;
            y.y *= sc;
            Tout[(int64_t)q * a.width] = cmul(Tp[(int64_t)q * a.width], y);
        }
    } else {
        for (int q = 0; q < a.kc; ++q)
            Tout[(int64_t)q * a.width] = cmul(Tp[(int64_t)q * a.width], Yr[(int64_t)q * a.m]);
    }
}

struct GemmArgs {
    const double2* Tlow;   // [kc][wlow], level k at column lowoff
    const double2* Thigh;  // [kc][whigh], level n-k at column highoff
    int64_t wlow, whigh, lowoff, highoff;
    int64_t M, N;          // entries of the two levels
    const int64_t* lowbase;
    int kc;
    int first, last;       // first / last chunk of sign vectors
    double2* acc;          // running sums (= amp when the caller wants amplitudes)
    double2* amp;
    double* prob;
};

constexpr int kStrip = 4;               // outputs per thread
constexpr int kWarps = 8;               // rows of a block tile

// QSTRIP: a warp owns one P (alpha broadcast); its lanes own 4 Q's each
// (strided by 32 so loads and stores coalesce).  !QSTRIP: the same with the
// roles of P and Q exchanged.
template <bool QSTRIP>
__global__ void __launch_bounds__(256) gemm_kernel(const GemmArgs a)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nfixed = QSTRIP ? a.M : a.N;
    const int64_t nstrip = QSTRIP ? a.N : a.M;
    const int64_t strip_tiles = (nstrip + 32 * kStrip - 1) / (32 * kStrip);
    const int64_t tile = blockIdx.x;
    const int64_t fixed = (tile / strip_tiles) * kWarps + warp;     // P (QSTRIP) or Q
    if (fixed >= nfixed) return;
    const int64_t s0 = (tile % strip_tiles) * (32 * kStrip) + lane;
    int64_t sidx[kStrip];
    bool sv[kStrip];
#pragma unroll
    for (int t = 0; t < kStrip; ++t) {
        sidx[t] = s0 + 32 * t;
        sv[t] = sidx[t] < nstrip;
    }
    int64_t oidx[kStrip];
#pragma unroll
    for (int t = 0; t < kStrip; ++t) {
        if (!sv[t]) { oidx[t] = 0; continue; }
        oidx[t] = QSTRIP ? a.lowbase[a.lowoff + fixed] + sidx[t]
                         : a.lowbase[a.lowoff + sidx[t]] + fixed;
    }
    double2 acc[kStrip];
#pragma unroll
    for (int t = 0; t < kStrip; ++t)
        acc[t] = (a.first || !sv[t]) ? make_double2(0.0, 0.0) : a.acc[oidx[t]];

    const double2* __restrict__ F = QSTRIP ? a.Tlow + a.lowoff + fixed : a.Thigh + a.highoff + fixed;
    const double2* __restrict__ S = QSTRIP ? a.Thigh + a.highoff : a.Tlow + a.lowoff;
    const int64_t wF = QSTRIP ? a.wlow : a.whigh;
    const int64_t wS = QSTRIP ? a.whigh : a.wlow;
    int64_t sclamp[kStrip];
#pragma unroll
    for (int t = 0; t < kStrip; ++t) sclamp[t] = sv[t] ? sidx[t] : 0;

#pragma unroll 2
    for (int q = 0; q < a.kc; ++q) {
        const double2 f = __ldg(F + (int64_t)q * wF);
        const double2* __restrict__ Sq = S + (int64_t)q * wS;
#pragma unroll
        for (int t = 0; t < kStrip; ++t) {
            if (sv[t]) cmac(acc[t], f, __ldg(Sq + sclamp[t]));
        }
    }
#pragma unroll
    for (int t = 0; t < kStrip; ++t) {
        if (!sv[t]) continue;
        if (!a.last) { a.acc[oidx[t]] = acc[t]; continue; }
        if (a.amp) a.amp[oidx[t]] = acc[t];
        if (a.prob) a.prob[oidx[t]] = fma(acc[t].x, acc[t].x, acc[t].y * acc[t].y);
    }
}

int64_t binom_host(int a, int b)
{
    if (b < 0 || a < 0 || b > a) return 0;
    unsigned __int128 c = 1;
    for (int i = 1; i <= b; ++i) {
        c = c * (unsigned __int128)(a - b + i) / (unsigned __int128)i;
        if (c > (unsigned __int128)INT64_MAX) return -1;
    }
    return (int64_t)c;
}

// multisets of size k over w modes
int64_t mset(int w, int k) { return k == 0 ? 1 : (w <= 0 ? 0 : binom_host(w + k - 1, k)); }

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// Plan the workspace: fixed parts, then the largest power-of-two chunk of
// sign vectors whose tables fit.  Returns the bytes used (or -1 on overflow).
int64_t dist_plan(const Plan& p, int64_t ws_bytes, bool need_acc, DistPlan* dp)
{
    const int m = p.m, n = p.n;
    dp->h = std::max(1, m / 2);
    const int wl = dp->h, wh = m - dp->h;
    int64_t lo = 0, hi = 0;
    for (int k = 0; k <= n + 1; ++k) {
        dp->lowoff[k] = lo;
        dp->highoff[k] = hi;
        if (k <= n) {
            const int64_t a = mset(wl, k), b = mset(wh, k);
            if (a < 0 || b < 0) return -1;
            lo += a;
            hi += b;
        }
    }
    dp->wlow = lo;
    dp->whigh = hi;
    const int64_t total = mset(m, n);
    if (total < 0) return -1;
    dp->ws_table = align256((size_t)(m + 1) * (n + 1) * sizeof(int64_t));
    dp->ws_base = align256((size_t)lo * sizeof(int64_t));
    dp->ws_acc = need_acc ? align256((size_t)total * sizeof(double2)) : 0;
    const size_t fixed = dp->ws_table + dp->ws_base + dp->ws_acc;
    const size_t per_d = (size_t)(m + lo + hi) * sizeof(double2);
    const int64_t dmax = n > 0 ? (1ll << (n - 1)) : 1;
    // default plan: all sign vectors if the tables stay under 4 GiB
    const size_t cap = ws_bytes < 0 ? ((size_t)4 << 30) : (size_t)std::max<int64_t>(0, ws_bytes - (int64_t)fixed - 3 * 256);
    int64_t kc = dmax;
    while (kc > 1 && (size_t)kc * per_d > cap) kc >>= 1;
    dp->kc = (int)kc;
    dp->ws_y = align256((size_t)kc * m * sizeof(double2));
    dp->ws_T = align256((size_t)kc * lo * sizeof(double2)) + align256((size_t)kc * hi * sizeof(double2));
    dp->ws_total = fixed + dp->ws_y + dp->ws_T;
    return (int64_t)dp->ws_total;
}

cudaError_t launch_glynn_dist(const Plan& p, const DistPlan& dp, const double2* U,
                              double* prob, double2* amp, void* ws, cudaStream_t s)
{
    const int m = p.m, n = p.n;
    char* w = (char*)ws;
    int64_t* table = (int64_t*)w;            w += dp.ws_table;
    int64_t* lowbase = (int64_t*)w;          w += dp.ws_base;
    double2* accbuf = dp.ws_acc ? (double2*)w : amp;  w += dp.ws_acc;
    double2* Y = (double2*)w;                w += dp.ws_y;
    double2* Tlow = (double2*)w;             w += align256((size_t)dp.kc * dp.wlow * sizeof(double2));
    double2* Thigh = (double2*)w;

    cudaError_t e = build_multiset_table(table, m, n, s);
    if (e != cudaSuccess) return e;
    MultisetTable mc{table, n};
    ColList cols;
    for (int j = 0; j < PCV_MAX_PHOTONS; ++j) cols.c[j] = p.cols[j];

    const int64_t dtot = 1ll << (n - 1);
    const int nchunks = (int)(dtot / dp.kc);
    const double lead = ldexp(p.norm_t, -(n - 1));
    for (int ch = 0; ch < nchunks; ++ch) {
        const int64_t d0 = (int64_t)ch * dp.kc;
        stage_begin(kStageTables, s);
        {
            const int runs = (dp.kc + kYRun - 1) / kYRun;
            const int64_t th = (int64_t)m * runs;
            row_sums_kernel<<<(unsigned)((th + 127) / 128), 128, 0, s>>>(U, m, n, cols, d0, dp.kc, Y);
            note_launches(1);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        for (int side = 0; side < 2; ++side) {
            const int wside = side == 0 ? dp.h : m - dp.h;
            for (int k = 0; k <= n; ++k) {
                LevelArgs la;
                la.mc = mc;
                la.m = m; la.n = n; la.h = dp.h;
                la.side = side;
                la.k = k;
                la.count = mset(wside, k);
                if (la.count == 0) continue;
                la.off = side == 0 ? dp.lowoff[k] : dp.highoff[k];
                la.poff = k > 0 ? (side == 0 ? dp.lowoff[k - 1] : dp.highoff[k - 1]) : 0;
                la.width = side == 0 ? dp.wlow : dp.whigh;
                la.kc = dp.kc;
                la.d0 = d0;
                la.lead = lead;
                la.Y = Y;
                la.T = side == 0 ? Tlow : Thigh;
                la.lowbase = (side == 0 && ch == 0) ? lowbase : nullptr;
                level_kernel<<<(unsigned)((la.count + 127) / 128), 128, 0, s>>>(la);
                note_launches(1);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
            }
        }
        stage_end(kStageTables, s);
        stage_begin(kStageGemm, s);
        for (int k = 0; k <= n; ++k) {
            GemmArgs g;
            g.M = mset(dp.h, k);
            g.N = mset(m - dp.h, n - k);
            if (g.M == 0 || g.N == 0) continue;
            g.Tlow = Tlow; g.Thigh = Thigh;
            g.wlow = dp.wlow; g.whigh = dp.whigh;
            g.lowoff = dp.lowoff[k]; g.highoff = dp.highoff[n - k];
            g.lowbase = lowbase;
            g.kc = dp.kc;
            g.first = ch == 0;
            g.last = ch == nchunks - 1;
            g.acc = accbuf;
            g.amp = amp;
            g.prob = prob;
            const bool qstrip = g.N >= g.M;
            const int64_t nstrip = qstrip ? g.N : g.M, nfixed = qstrip ? g.M : g.N;
            const int64_t tiles = ((nstrip + 32 * kStrip - 1) / (32 * kStrip)) * ((nfixed + kWarps - 1) / kWarps);
            if (tiles > INT32_MAX) return cudaErrorInvalidConfiguration;
            const unsigned grid = (unsigned)tiles;
            if (qstrip) gemm_kernel<true><<<grid, 256, 0, s>>>(g);
            else        gemm_kernel<false><<<grid, 256, 0, s>>>(g);
            note_launches(1);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        stage_end(kStageGemm, s);
    }
    return cudaSuccess;
}

}  // namespace pcv
