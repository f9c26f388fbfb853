// Full output distribution by a factorised Glynn sum, for a batch of B
// unitaries sharing one input state.
//
// Put Glynn's sign vector on the input photons (columns of U_{T,S}, Eq.
// eqperm).  The row sum of output row i then depends only on the output mode
// r_i:  y_r(d) = sum_j d_j U[r][c_j].  Every output S therefore shares the
// same m row sums per sign vector d, and
//     a(S) = norm_t 2^{-(n-1)} sum_d sigma(d) prod_r y_r(d)^{s_r} / sqrt(s_r!).
// Split the modes at h: S = (P on modes [0,h), Q on modes [h,m)).  With
//     alpha_P(d) = sigma(d) 2^{-(n-1)} norm_t prod_{r<h} y_r^{P_r}/sqrt(P_r!),
//     beta_Q(d)  = prod_{r>=h} y_r^{Q_r}/sqrt(Q_r!),
// every output is a(S) = sum_d alpha_P(d) beta_Q(d): for each k = |P| a
// complex matrix product over the sign vectors.  The product uses three real
// multiply-adds per output and sign vector (Gauss's three-multiplication
// form, with alpha_re + alpha_im and beta_re + beta_im stored beside the
// tables):
//     t1 += a_re b_re,  t2 += a_im b_im,  t3 += (a_re + a_im)(b_re + b_im),
//     Re a(S) = t1 - t2,  Im a(S) = t3 - t1 - t2,
// 3 DFMA instead of the 6n - 2 FP64 instructions of a Gray step of the plain
// per-output kernel.
//
// Pipeline per chunk of KC sign vectors (all of them when the workspace
// allows):
//   row_sums_kernel  y_r(d) by Gray-code row-sum updates (one column per step)
//   level_kernel     alpha/beta tables level by level: entry(P) = entry(P minus
//                    its last mode) * y_last / sqrt(multiplicity)
//   gemm_kernel      one launch over every k: a(S) = sum_d alpha_P beta_Q,
//                    written at the canonical index lowbase(P) + rank(Q)
//
// The canonical index of S (lexicographic order of the non-decreasing mode
// list) splits as lowbase(P) + rank of Q among the (n-k)-multisets over
// [h, m): all outputs whose first k photons are P and whose other photons lie
// in [h, m) are contiguous in that order.

#include <algorithm>

#include "pcv_common.cuh"

namespace pcv {
namespace {

constexpr int kYRun = 32;          // sign vectors per row_sums_kernel thread
constexpr int kLevelGroup = 8;     // sign vectors per level_kernel thread
constexpr int kStrip = 4;          // outputs per gemm_kernel thread
constexpr int kWarps = 8;          // rows of a gemm block tile

struct ColList { int c[PCV_MAX_PHOTONS]; };

__global__ void row_sums_kernel(const double2* __restrict__ Ub, int m, int n, ColList cols,
                                int64_t d0, int kc, double2* __restrict__ Yb, int64_t ystride)
{
    // thread -> (row r, run of kYRun consecutive sign vectors); blockIdx.y = batch entry
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int runs = (kc + kYRun - 1) / kYRun;
    if (t >= (int64_t)m * runs) return;
    const double2* U = Ub + (size_t)blockIdx.y * m * m;
    double2* Y = Yb + (size_t)blockIdx.y * ystride;
    const int r = (int)(t % m);
    const int run = (int)(t / m);
    const double2* Ur = U + (size_t)r * m;
    const int64_t dstart = d0 + (int64_t)run * kYRun;
    const int len = min(kYRun, kc - run * kYRun);
    const uint64_t g = (uint64_t)dstart ^ ((uint64_t)dstart >> 1);
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
    const double2* Y;      // [batch][kc][m]
    int64_t ystride;
    double2* T;            // [batch][kc][width]
    double* Tsum;          // [batch][kc][width]: re + im of T
    int64_t tstride;
    int64_t* lowbase;      // low side: canonical base index of each P (written once)
    // Edge mode (partial != null): the level is not stored; each thread adds
    // sum_q F(q) entry(q) over its sign vectors, F being the single entry of
    // the other side, and writes the sum to partial[entry * ngroups + group].
    const double2* F;
    int64_t wF;
    double2* partial;
    int ngroups;
};

__global__ void level_kernel(const LevelArgs a)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.count) return;
    const int q0 = blockIdx.y * kLevelGroup;
    const int q1 = min(a.kc, q0 + kLevelGroup);
    const int b = blockIdx.z;
    double2* T = a.T + (size_t)b * a.tstride;
    double* Ts = a.Tsum + (size_t)b * a.tstride;
    const double2* Y = a.Y + (size_t)b * a.ystride;
    const bool write_base = a.side == 0 && a.lowbase && blockIdx.y == 0 && b == 0;
    if (a.k == 0) {
        for (int q = q0; q < q1; ++q) {
            double v = 1.0;
            if (a.side == 0) {
                const uint64_t d = (uint64_t)(a.d0 + q);
                v = (__popcll(d ^ (d >> 1)) & 1) ? -a.lead : a.lead;
            }
            T[(int64_t)q * a.width] = make_double2(v, 0.0);
            Ts[(int64_t)q * a.width] = v;
        }
        if (write_base) {
            int64_t r = 0;
            if (a.n > 0) for (int v = 0; v < a.h; ++v) r += a.mc(a.m - v, a.n - 1);
            a.lowbase[0] = r;
        }
        return;
    }
    const int w = a.side == 0 ? a.h : a.m - a.h;
    const int shift = a.side == 0 ? 0 : a.h;
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

    if (write_base) {
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

    if (a.partial) {
        double2 acc = make_double2(0.0, 0.0);
        for (int q = q0; q < q1; ++q) {
            double2 y = Y[(int64_t)q * a.m + r];
            if (mult > 1) { y.x *= sc; y.y *= sc; }
            const double2 v = cmul(T[(int64_t)q * a.width + a.poff + parent], y);
            cmac(acc, a.F[(int64_t)q * a.wF], v);
        }
        if (b == 0) a.partial[i * a.ngroups + blockIdx.y] = acc;
        return;
    }
    for (int q = q0; q < q1; ++q) {
        double2 y = Y[(int64_t)q * a.m + r];
        if (mult > 1) { y.x *= sc; y.y *= sc; }
        const double2 v = cmul(T[(int64_t)q * a.width + a.poff + parent], y);
        T[(int64_t)q * a.width + a.off + i] = v;
        Ts[(int64_t)q * a.width + a.off + i] = v.x + v.y;
    }
}

// Edge mode's second pass: the sign-vector groups of each entry added in a
// fixed order, written at its canonical index.
__global__ void edge_reduce_kernel(const double2* __restrict__ partial, int64_t count, int ngroups,
                                   const int64_t* __restrict__ lowbase, int64_t lowidx, int strip_is_low,
                                   int64_t lo, int64_t hi, double2* __restrict__ amp, double* __restrict__ prob)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int64_t o = strip_is_low ? lowbase[lowidx + i] : lowbase[lowidx] + i;
    if (o < lo || o >= hi) return;
    double2 v = partial[i * ngroups];
    for (int g = 1; g < ngroups; ++g) v = cadd(v, partial[i * ngroups + g]);
    if (amp) amp[o - lo] = v;
    if (prob) prob[o - lo] = fma(v.x, v.x, v.y * v.y);
}

struct GemmArgs {
    const double2* Tlow;   // [batch][kc][wlow]
    const double* Slow;
    const double2* Thigh;  // [batch][kc][whigh]
    const double* Shigh;
    int64_t wlow, whigh, tstride_low, tstride_high;
    int64_t lowoff[PCV_MAX_PHOTONS + 1], highoff[PCV_MAX_PHOTONS + 1];  // per k: level k low, level n-k high
    int64_t M[PCV_MAX_PHOTONS + 1], N[PCV_MAX_PHOTONS + 1];
    // entries of the fixed and strip sides this launch covers, per k: one of
    // them is the range of P whose outputs meet [lo, hi), the other complete
    int64_t fb[PCV_MAX_PHOTONS + 1], fe[PCV_MAX_PHOTONS + 1], sb[PCV_MAX_PHOTONS + 1], se[PCV_MAX_PHOTONS + 1];
    int64_t tile0[PCV_MAX_PHOTONS + 2];   // first tile of each k
    int nk;
    const int64_t* lowbase;
    int kc;
    int first, last;       // first / last chunk of sign vectors
    int64_t lo, hi;        // outputs written: canonical [lo, hi), at o - lo
    int64_t out_stride;    // outputs per batch entry (hi - lo)
    double2* acc;          // running sums between chunks (= amp when amplitudes are wanted)
    double2* amp;
    double* prob;
};

// A warp owns one "fixed" entry (P if N >= M, else Q: the shorter side, so
// the strip side fills whole warps); its lanes own 4 strip entries each,
// strided by 32 so loads and stores coalesce.
__global__ void __launch_bounds__(256) gemm_kernel(const GemmArgs a)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t tile = blockIdx.x;
    int k = 0;
    while (k + 1 < a.nk && a.tile0[k + 1] <= tile) ++k;
    const int64_t M = a.M[k], N = a.N[k];
    const bool qstrip = N >= M;
    const int64_t strip_tiles = (a.se[k] - a.sb[k] + 32 * kStrip - 1) / (32 * kStrip);
    const int64_t lt = tile - a.tile0[k];
    const int64_t fixed = a.fb[k] + (lt / strip_tiles) * kWarps + warp;
    if (fixed >= a.fe[k]) return;
    const int64_t nstrip = a.se[k];
    const int64_t s0 = a.sb[k] + (lt % strip_tiles) * (32 * kStrip) + lane;
    const int b = blockIdx.y;

    const double2* Tl = a.Tlow + (size_t)b * a.tstride_low + a.lowoff[k];
    const double* Sl = a.Slow + (size_t)b * a.tstride_low + a.lowoff[k];
    const double2* Th = a.Thigh + (size_t)b * a.tstride_high + a.highoff[k];
    const double* Sh = a.Shigh + (size_t)b * a.tstride_high + a.highoff[k];
    const double2* __restrict__ F = qstrip ? Tl + fixed : Th + fixed;
    const double* __restrict__ Fs = qstrip ? Sl + fixed : Sh + fixed;
    const double2* __restrict__ S = qstrip ? Th : Tl;
    const double* __restrict__ Ss = qstrip ? Sh : Sl;
    const int64_t wF = qstrip ? a.wlow : a.whigh;
    const int64_t wS = qstrip ? a.whigh : a.wlow;

    int64_t sidx[kStrip], oidx[kStrip];
    bool sv[kStrip];
#pragma unroll
    for (int t = 0; t < kStrip; ++t) {
        sidx[t] = s0 + 32 * t;
        sv[t] = sidx[t] < nstrip;
        if (!sv[t]) sidx[t] = 0;
        oidx[t] = qstrip ? a.lowbase[a.lowoff[k] + fixed] + sidx[t] : a.lowbase[a.lowoff[k] + sidx[t]] + fixed;
    }
    double t1[kStrip], t2[kStrip], t3[kStrip];
#pragma unroll
    for (int t = 0; t < kStrip; ++t) t1[t] = t2[t] = t3[t] = 0.0;

#pragma unroll 2
    for (int q = 0; q < a.kc; ++q) {
        const double2 f = __ldg(F + (int64_t)q * wF);
        const double fs = __ldg(Fs + (int64_t)q * wF);
        const double2* __restrict__ Sq = S + (int64_t)q * wS;
        const double* __restrict__ Ssq = Ss + (int64_t)q * wS;
#pragma unroll
        for (int t = 0; t < kStrip; ++t) {
            const double2 v = __ldg(Sq + sidx[t]);
            const double vs = __ldg(Ssq + sidx[t]);
            t1[t] = fma(f.x, v.x, t1[t]);
            t2[t] = fma(f.y, v.y, t2[t]);
            t3[t] = fma(fs, vs, t3[t]);
        }
    }
    double2* acc = a.acc ? a.acc + (size_t)b * a.out_stride : nullptr;
    double2* amp = a.amp ? a.amp + (size_t)b * a.out_stride : nullptr;
    double* prob = a.prob ? a.prob + (size_t)b * a.out_stride : nullptr;
#pragma unroll
    for (int t = 0; t < kStrip; ++t) {
        if (!sv[t] || oidx[t] < a.lo || oidx[t] >= a.hi) continue;
        const int64_t o = oidx[t] - a.lo;
        double2 v = make_double2(t1[t] - t2[t], t3[t] - t1[t] - t2[t]);
        if (!a.first) v = cadd(v, acc[o]);
        if (!a.last) { acc[o] = v; continue; }
        if (amp) amp[o] = v;
        if (prob) prob[o] = fma(v.x, v.x, v.y * v.y);
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

struct Layout {
    size_t status, table, base, acc, y, tl, sl, th, sh, total;
};

Layout layout(int m, int n, int B, int64_t lo, int64_t hi, int64_t total, bool need_acc, int64_t kc)
{
    Layout L;
    L.status = 256;                          // the call's status word (pcv_distribution_status)
    L.table = align256((size_t)(m + 1) * (n + 1) * sizeof(int64_t));
    L.base = align256((size_t)lo * sizeof(int64_t));
    L.acc = need_acc ? align256((size_t)B * total * sizeof(double2)) : 0;
    L.y = align256((size_t)B * kc * m * sizeof(double2));
    L.tl = align256((size_t)B * kc * lo * sizeof(double2));
    L.sl = align256((size_t)B * kc * lo * sizeof(double));
    L.th = align256((size_t)B * kc * hi * sizeof(double2));
    L.sh = align256((size_t)B * kc * hi * sizeof(double));
    L.total = L.status + L.table + L.base + L.acc + L.y + L.tl + L.sl + L.th + L.sh;
    return L;
}

// Host copies of the multiset walks: unrank a size-k multiset over w modes,
// and the rank of a non-decreasing mode list.
void host_unrank(int w, int k, int64_t idx, int* modes)
{
    int v = 0;
    for (int p = 0; p < k; ++p) {
        for (;;) {
            const int64_t c = mset(w - v, k - p - 1);
            if (idx < c) break;
            idx -= c;
            ++v;
        }
        modes[p] = v;
    }
}

int64_t host_rank(int w, int k, const int* modes)
{
    int64_t r = 0;
    int prev = 0;
    for (int p = 0; p < k; ++p) {
        for (int v = prev; v < modes[p]; ++v) r += mset(w - v, k - p - 1);
        prev = modes[p];
    }
    return r;
}

}  // namespace

int64_t host_lowbase(int m, int n, int h, int k, int64_t rank)
{
    int modes[PCV_MAX_PHOTONS];
    host_unrank(h, k, rank, modes);
    int64_t base = 0;
    int prev = 0;
    for (int p = 0; p < k; ++p) {
        for (int v = prev; v < modes[p]; ++v) base += mset(m - v, n - p - 1);
        prev = modes[p];
    }
    if (k < n)
        for (int v = prev; v < h; ++v) base += mset(m - v, n - k - 1);
    return base;
}

int64_t host_parent_rank(int w, int k, int64_t rank)
{
    int modes[PCV_MAX_PHOTONS];
    host_unrank(w, k, rank, modes);
    return host_rank(w, k - 1, modes);
}

void p_ranges(int m, int n, int h, int64_t lo, int64_t hi, PRanges* r)
{
    for (int k = 0; k <= n; ++k) {
        const int64_t cnt = mset(h, k), blk = mset(m - h, n - k);
        r->pa[k] = r->pb[k] = 0;
        if (cnt <= 0 || blk <= 0 || lo >= hi) continue;
        // lowbase grows with P's rank at a fixed level: bisect for the first
        // block that ends after lo and the first that starts at or after hi
        int64_t a0 = 0, a1 = cnt;
        while (a0 < a1) {
            const int64_t mid = a0 + (a1 - a0) / 2;
            if (host_lowbase(m, n, h, k, mid) + blk > lo) a1 = mid;
            else a0 = mid + 1;
        }
        int64_t b0 = a0, b1 = cnt;
        while (b0 < b1) {
            const int64_t mid = b0 + (b1 - b0) / 2;
            if (host_lowbase(m, n, h, k, mid) >= hi) b1 = mid;
            else b0 = mid + 1;
        }
        r->pa[k] = a0;
        r->pb[k] = b0;
    }
}

// Plan the workspace: the largest power-of-two chunk of sign vectors whose
// tables fit into ws_bytes (ws_bytes < 0: the default budget of 8 GiB).
// Returns the bytes used, or -1 on overflow.
int64_t dist_plan(const Plan& p, int B, int64_t ws_bytes, bool need_acc, DistPlan* dp)
{
    const int m = p.m, n = p.n;
    dp->h = std::max(1, m / 2);
    dp->B = B;
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
    dp->total = total;
    const int64_t dmax = n > 0 ? (1ll << (n - 1)) : 1;
    const size_t budget = ws_bytes < 0 ? ((size_t)8 << 30) : (size_t)ws_bytes;
    int64_t kc = dmax;
    while (kc > 1 && layout(m, n, B, lo, hi, total, need_acc && kc < dmax, kc).total > budget) kc >>= 1;
    const Layout L = layout(m, n, B, lo, hi, total, need_acc && kc < dmax, kc);
    dp->kc = (int)kc;
    dp->ws_status = L.status;
    dp->ws_table = L.table;
    dp->ws_base = L.base;
    dp->ws_acc = L.acc;
    dp->ws_y = L.y;
    dp->ws_tl = L.tl;
    dp->ws_sl = L.sl;
    dp->ws_th = L.th;
    dp->ws_sh = L.sh;
    dp->ws_total = L.total;
    dp->lo = 0;
    dp->hi = total;
    return (int64_t)L.total;
}

int64_t dist_plan_tc(const Plan& p, bool need_amp_buffer, DistPlan* dp)
{
    if (dist_plan(p, 1, INT64_MAX / 4, false, dp) < 0) return -1;
    const int64_t dmax = p.n > 0 ? (1ll << (p.n - 1)) : 1;
    if (dp->kc != dmax) return -1;
    (void)need_amp_buffer;                   // the products go to their own buffer
    dp->ws_acc = 0;
    dp->tc = true;
    // n >= 2 with both sides non-empty: tables, digits and every output block
    // in glynn_tc.cu (no FP64 tables in this file's layout); else (n = 1 or
    // m = 1, no block has entries on both sides) only the single-entry blocks
    // in FP64: the tables of levels < n and edge-mode partial sums of the
    // larger level n, reused by both sides
    const bool tc_all = p.n >= 2 && p.m - dp->h >= 1;
    if (tc_all) {
        dp->ws_tl = dp->ws_sl = dp->ws_th = dp->ws_sh = 0;
        dp->ws_tc = (size_t)tc_workspace(p.m, p.n, dp->h, (int)dmax, dp->total);
        dp->ws_edge = 0;
    } else {
        dp->ws_tc = 0;
        const int64_t ln = std::max(mset(dp->h, p.n), mset(p.m - dp->h, p.n));
        dp->ws_edge = align256((size_t)ln * ((dmax + kLevelGroup - 1) / kLevelGroup) * sizeof(double2));
    }
    dp->ws_total = dp->ws_status + dp->ws_table + dp->ws_base + dp->ws_acc + dp->ws_y + dp->ws_tl + dp->ws_sl +
                   dp->ws_th + dp->ws_sh + dp->ws_tc + dp->ws_edge;
    return (int64_t)dp->ws_total;
}

cudaError_t launch_glynn_dist(const Plan& p, const DistPlan& dp, const double2* U,
                              double* prob, double2* amp, void* ws, cudaStream_t s)
{
    const int m = p.m, n = p.n, B = dp.B;
    char* w = (char*)ws;
    int* status = (int*)w;                   w += dp.ws_status;
    int64_t* table = (int64_t*)w;            w += dp.ws_table;
    int64_t* lowbase = (int64_t*)w;          w += dp.ws_base;
    double2* accbuf = dp.ws_acc ? (double2*)w : amp;  w += dp.ws_acc;
    double2* Y = (double2*)w;                w += dp.ws_y;
    double2* Tlow = (double2*)w;             w += dp.ws_tl;
    double* Slow = (double*)w;               w += dp.ws_sl;
    double2* Thigh = (double2*)w;            w += dp.ws_th;
    double* Shigh = (double*)w;              w += dp.ws_sh;
    void* tcws = w;
    if (dp.tc && (B != 1 || dp.kc != (1ll << (n - 1)))) return cudaErrorInvalidValue;

    // the status word starts each call at zero; a tensor-core kernel whose
    // bounded wait gives up writes its role code there
    cudaError_t e = cudaMemsetAsync(status, 0, 16, s);     // time-out word, tensor-core tile counter
    if (e != cudaSuccess) return e;
    if ((e = build_multiset_table(table, m, n, s)) != cudaSuccess) return e;
    MultisetTable mc{table, n};
    ColList cols;
    for (int j = 0; j < PCV_MAX_PHOTONS; ++j) cols.c[j] = p.cols[j];

    const int64_t dtot = 1ll << (n - 1);
    const int nchunks = (int)(dtot / dp.kc);
    const double lead = ldexp(p.norm_t, -(n - 1));
    const int64_t ystride = (int64_t)dp.kc * m;
    const int64_t tl_stride = (int64_t)dp.kc * dp.wlow, th_stride = (int64_t)dp.kc * dp.whigh;

    GemmArgs g;
    g.Tlow = Tlow; g.Slow = Slow; g.Thigh = Thigh; g.Shigh = Shigh;
    g.wlow = dp.wlow; g.whigh = dp.whigh;
    g.tstride_low = tl_stride; g.tstride_high = th_stride;
    g.lowbase = lowbase;
    g.kc = dp.kc;
    const int64_t lo = dp.lo, hi = dp.hi < 0 ? dp.total : dp.hi;
    g.lo = lo;
    g.hi = hi;
    g.out_stride = hi - lo;
    PRanges pr;
    p_ranges(m, n, dp.h, lo, hi, &pr);
    g.acc = accbuf;
    g.amp = amp;
    g.prob = prob;
    g.nk = 0;
    int64_t tiles = 0;
    for (int k = 0; k <= n; ++k) {
        const int64_t M = mset(dp.h, k), N = mset(m - dp.h, n - k);
        if (M == 0 || N == 0 || pr.pa[k] >= pr.pb[k]) continue;
        const bool qstrip = N >= M;
        // the P side (fixed when qstrip) covers only the P whose outputs meet [lo, hi)
        g.fb[g.nk] = qstrip ? pr.pa[k] : 0;
        g.fe[g.nk] = qstrip ? pr.pb[k] : N;
        g.sb[g.nk] = qstrip ? 0 : pr.pa[k];
        g.se[g.nk] = qstrip ? N : pr.pb[k];
        g.lowoff[g.nk] = dp.lowoff[k];
        g.highoff[g.nk] = dp.highoff[n - k];
        g.M[g.nk] = M;
        g.N[g.nk] = N;
        g.tile0[g.nk] = tiles;
        tiles += ((g.se[g.nk] - g.sb[g.nk] + 32 * kStrip - 1) / (32 * kStrip)) *
                 ((g.fe[g.nk] - g.fb[g.nk] + kWarps - 1) / kWarps);
        g.nk++;
    }
    g.tile0[g.nk] = tiles;
    if (tiles > INT32_MAX) return cudaErrorInvalidConfiguration;

    for (int ch = 0; ch < nchunks; ++ch) {
        const int64_t d0 = (int64_t)ch * dp.kc;
        stage_begin(kStageTables, s);
        {
            const int runs = (dp.kc + kYRun - 1) / kYRun;
            const int64_t th = (int64_t)m * runs;
            dim3 grid((unsigned)((th + 127) / 128), (unsigned)B);
            row_sums_kernel<<<grid, 128, 0, s>>>(U, m, n, cols, d0, dp.kc, Y, ystride);
            note_launches(1);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        if (dp.tc && n >= 2 && m - dp.h >= 1) {
            // tables, digits and products on the tensor-core path
            TcInputs ti;
            ti.K = (int)dp.kc; ti.n = n; ti.m = m; ti.h = dp.h;
            for (int k = 0; k <= PCV_MAX_PHOTONS + 1; ++k) {
                ti.lowoff[k] = dp.lowoff[k];
                ti.highoff[k] = dp.highoff[k];
            }
            ti.lowbase = lowbase;
            ti.Y = Y;
            ti.mc = mc;
            ti.lead = lead;
            ti.total = dp.total;
            ti.amp = amp;
            ti.prob = prob;
            ti.ws = tcws;
            ti.error = status;
            ti.next_tile = (unsigned long long*)((char*)status + 8);
            ti.lo = lo;
            ti.hi = hi;
            if ((e = launch_tc_tables(ti, s)) != cudaSuccess) return e;
            stage_end(kStageTables, s);
            if ((e = launch_tc_products(ti, s)) != cudaSuccess) return e;
            continue;
        }
        for (int side = 0; side < 2; ++side) {
            const int wside = side == 0 ? dp.h : m - dp.h;
            for (int k = 0; k <= n; ++k) {
                if (dp.tc && k == n) continue;     // folded into the edge products below
                LevelArgs la;
                la.F = nullptr;
                la.wF = 0;
                la.partial = nullptr;
                la.ngroups = 0;
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
                la.ystride = ystride;
                la.T = side == 0 ? Tlow : Thigh;
                la.Tsum = side == 0 ? Slow : Shigh;
                la.tstride = side == 0 ? tl_stride : th_stride;
                la.lowbase = (side == 0 && ch == 0) ? lowbase : nullptr;
                dim3 grid((unsigned)((la.count + 127) / 128), (unsigned)((dp.kc + kLevelGroup - 1) / kLevelGroup),
                          (unsigned)B);
                level_kernel<<<grid, 128, 0, s>>>(la);
                note_launches(1);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
            }
        }
        stage_end(kStageTables, s);
        if (dp.tc) {
            // n = 1 or m = 1: the k = 0 and k = n blocks (one entry on one side) in FP64:
            // level n of each side is never stored; the level kernel multiplies
            // each new entry by the other side's single entry (level 0) and sums
            // over its sign vectors, and a second pass adds the groups
            stage_begin(kStageEdge, s);
            const int ngroups = (int)((dp.kc + kLevelGroup - 1) / kLevelGroup);
            double2* partial = (double2*)((char*)tcws + dp.ws_tc);
            for (int side = 0; side < 2; ++side) {
                const int wside = side == 0 ? dp.h : m - dp.h;
                LevelArgs la;
                la.mc = mc;
                la.m = m; la.n = n; la.h = dp.h;
                la.side = side;
                la.k = n;
                la.count = mset(wside, n);
                if (la.count == 0) continue;
                la.off = side == 0 ? dp.lowoff[n] : dp.highoff[n];
                la.poff = side == 0 ? dp.lowoff[n - 1] : dp.highoff[n - 1];
                la.width = side == 0 ? dp.wlow : dp.whigh;
                la.kc = dp.kc;
                la.d0 = 0;
                la.lead = lead;
                la.Y = Y;
                la.ystride = ystride;
                la.T = side == 0 ? Tlow : Thigh;
                la.Tsum = side == 0 ? Slow : Shigh;
                la.tstride = side == 0 ? tl_stride : th_stride;
                la.lowbase = side == 0 ? lowbase : nullptr;
                la.F = side == 0 ? Thigh + dp.highoff[0] : Tlow + dp.lowoff[0];
                la.wF = side == 0 ? dp.whigh : dp.wlow;
                la.partial = partial;
                la.ngroups = ngroups;
                dim3 grid((unsigned)((la.count + 127) / 128), (unsigned)ngroups, 1);
                level_kernel<<<grid, 128, 0, s>>>(la);
                // low side level n: the block k = n (Q empty), outputs lowbase(P);
                // high side level n: the block k = 0 (P empty), outputs lowbase({}) + rank(Q)
                edge_reduce_kernel<<<(unsigned)((la.count + 255) / 256), 256, 0, s>>>(
                    partial, la.count, ngroups, lowbase, side == 0 ? dp.lowoff[n] : dp.lowoff[0], side == 0 ? 1 : 0,
                    lo, hi, amp, prob);
                note_launches(2);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
            }
            stage_end(kStageEdge, s);
            continue;
        }
        stage_begin(kStageGemm, s);
        g.first = ch == 0;
        g.last = ch == nchunks - 1;
        if (tiles > 0) {                      // none when [lo, hi) is empty
            gemm_kernel<<<dim3((unsigned)tiles, (unsigned)B), 256, 0, s>>>(g);
            note_launches(1);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        stage_end(kStageGemm, s);
    }
    return cudaSuccess;
}

}  // namespace pcv
