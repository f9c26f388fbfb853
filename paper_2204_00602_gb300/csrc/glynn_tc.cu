// The factorised full distribution with its products on the BF16 tensor
// cores, in exact integer arithmetic: table levels, digit splitting and the
// products of every block k = 0..n.
//
// With the row sums y_r(d) (glynn_dist.cu), every output is
//     a(S) = sum_d alpha_P(d) beta_Q(d),
// for each k a complex matrix product over the K = 2^{n-1} sign vectors, done
// as three real products (Gauss): t1 = Ar Br, t2 = Ai Bi, t3 = (Ar+Ai)(Br+Bi),
// Re a = t1 - t2, Im a = t3 - t1 - t2.  Here each real product runs on the
// tensor cores without losing FP64 accuracy, by splitting every table value
// into integer digits (the error-free splitting idea of Ozaki, Ogita, Oishi
// and Rump, 2012):
//
//   * each row gets an exponent E with max_d |x(d)| <= 2^{E-1}; X =
//     round(x 2^{56-E}) is an integer with |X| <= 2^55, written as 8
//     balanced base-128 digits,
//         X = sum_{i=0..7} D_i 128^{7-i},   |D_i| <= 64,
//     so x = 2^E sum_i D_i 2^{-7(i+1)} up to 2^{E-56} (FP64 accuracy).  A
//     table entry's re and im share one exponent one bit higher (54 bits
//     each), and its third operand is the integer X_re + X_im; the per-mode
//     vectors of the single-entry columns keep one exponent per product;
//   * a digit is an integer of at most 7 bits, exact in BF16, and a product of
//     two is at most 2^12; over K <= 512 sign vectors a digit-pair product
//     sums to at most 2^21, and the 8 pairs (i, j) of one diagonal i + j = d
//     to at most 2^24, so an FP32 accumulator holds every partial sum of a
//     diagonal exactly, in any order the tensor core adds them;
//   * diagonals d = 0..7 are kept (36 digit pairs); the dropped ones weigh
//     2^{-56} and less relative to the row and column scales;
//   * the 8 diagonal sums (exact integers) are combined on the integer pipe
//     into Z = hi 2^28 + lo, hi = sum_{d<4} acc_d 128^{3-d}, lo = sum_{d>=4}
//     acc_d 128^{7-d}, and x_t = Z 2^{E_row + E_col - 63} is rounded once to
//     FP64 with integer operations (scale_packed).
//
// Kernels:
//   tc_level_kernel     table levels 1..n-1 of each side, built in FP64 from
//                       the parent level and written as BF16 digits, laid out
//                       [t][digit][entry][K] for TMA (levels <= n-2 also keep
//                       their complex entries as the next level's parents);
//   split_exp_kernel, split_digits_kernel, edge_vectors_kernel,
//   edge_info_kernel    the single-entry blocks (k = 0, k = n): level n is
//                       level n-1 times y_r / sqrt(multiplicity), so these
//                       blocks are products of level n-1 with one vector per
//                       mode; the vectors are split here, and each level n-1
//                       entry gets its output index and scale;
//   tc_product_kernel   one persistent CTA per SM walking 128 x N output
//                       tiles of one block each (N = 16..64; the single-entry
//                       columns ride in the tile of the block k = 1 or n-1
//                       with the same rows when both fit), eleven warps:
//   warp 0  row-operand TMA: per 64-wide K block, the 8 digit slices of the
//           row operand one at a time (16 KB slots, six in flight, digits in
//           the order 0 7 1 6 2 5 3 4), 128B swizzle;
//   warp 10 column-operand TMA: per K block the 8 digit slices of the
//           column operand (N rows each, packed one after the other in a
//           64 KB set, double-buffered);
//   warp 1  MMA issuer: the accumulator of diagonal d sits at TMEM columns
//           d N .. d N + N - 1, so the products of row digit i with column
//           digits j = j0 .. j1 land on the contiguous columns (i + j0) N ..
//           (i + j1 + 1) N - 1: one tcgen05.mma kind::f16 (M=128, K=16) with
//           the packed column slices j0 .. j1 as a single operand of width
//           (j1 - j0 + 1) N <= 256 covers them all.  A row slice is then read
//           from shared memory once or twice per K step instead of 8 - i
//           times; commits free the slots;
//   warps 2-9  drain: after each of the three products, tcgen05.ld of the 8
//           diagonals (warp w owns TMEM lanes 32 (w mod 4) .., two warps per
//           lane group split the columns) and the integer combination; the
//           accumulators are then handed back to the MMA, and the rounding
//           and stores follow.  t1 and t2 are stored at the output's
//           canonical index in a [2][outputs] buffer; after t3 the thread
//           that stored them forms the amplitude and |a|^2 in place.  Tile
//           rows are high-side entries wherever there are 128 of them, so a
//           warp's 32 lanes hold consecutive outputs and its stores coalesce.
// Every mbarrier wait is bounded; on a time-out the kernel records an error
// code and returns after releasing its tensor memory.

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "pcv_common.cuh"
#include "tc_ptx.cuh"

namespace pcv {
namespace {

constexpr int kDigits = 8;
constexpr int TBM = 128, TBN = 64, TBK = 64;
constexpr int kASlots = 6, kBSets = 2;
constexpr uint32_t kABytes = TBM * TBK * 2;             // 16 KB: one digit slice of the row operand
constexpr uint32_t kRowBytes = TBK * 2;                 // one 64-wide K row of a slice: 128 B
constexpr uint32_t kBBytes = kDigits * TBN * kRowBytes; // 64 KB: all digit slices of the column operand
constexpr int kBSub = 16;                               // rows per column load when N < 64
constexpr uint32_t kSmemBytes = kBSets * kBBytes + kASlots * kABytes + 1024;
constexpr int kColWarp = 10;                             // its lane 0 loads the column operand
constexpr int kThreads = 352;                            // warp 0 row loads, 1 MMA, 2-9 drain, 10 column loads
constexpr uint32_t kTmemCols = 512;
constexpr long long kMaxPolls = 1ll << 26;               // default bound of one mbarrier wait
constexpr int kNoExp = -100000;                          // an all-zero row

// ------------------------------------------------------------ splitting

__device__ __forceinline__ int exp_field(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

// E_t(entry) for t = re, im, re+im: the smallest E with max |x| <= 2^{E-1}
// (from the largest exponent field; a power of two costs one spare bit).
// (T, Sm: [K][stride] tables from their first digitised entry; w entries.)
// One warp per entry, lanes over the sign vectors.
__global__ void split_exp_kernel(const double2* __restrict__ T, const double* __restrict__ Sm, int64_t stride,
                                 int64_t w, int K, int* __restrict__ ex)
{
    const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (e >= w) return;                                    // whole warps
    int f0 = 0, f1 = 0, f2 = 0;
    for (int d = lane; d < K; d += 32) {
        const double2 v = T[(int64_t)d * stride + e];
        f0 = max(f0, exp_field(v.x));
        f1 = max(f1, exp_field(v.y));
        f2 = max(f2, exp_field(Sm[(int64_t)d * stride + e]));
    }
    f0 = __reduce_max_sync(0xffffffffu, f0);
    f1 = __reduce_max_sync(0xffffffffu, f1);
    f2 = __reduce_max_sync(0xffffffffu, f2);
    if (lane == 0) {
        ex[e] = f0 ? f0 - 1021 : kNoExp;
        ex[w + e] = f1 ? f1 - 1021 : kNoExp;
        ex[2 * w + e] = f2 ? f2 - 1021 : kNoExp;
    }
}

// X = round(x 2^{56-E}) as a signed integer, |X| <= 2^55 (the magnitude
// rounded half up; 0 for x = 0 or an all-zero row), for |x| <= 2^{E-1}.  With
// the 53-bit mantissa m, X = m 2^{sh} for sh = e - 1019 - E <= 3 (e the
// exponent field): one right shift of 16 m by s = 4 - sh >= 1, rounded half
// up, covers every case without branches.
__device__ __forceinline__ long long fixed_of(double x, int E)
{
    const long long bits = __double_as_longlong(x);
    const int ef = (int)((bits >> 52) & 0x7FF);
    const unsigned long long m16 = ((unsigned long long)(bits & ((1ll << 52) - 1)) | (1ull << 52)) << 4;
    const int s = min(max(4 - (ef - 1019 - E), 1), 64);
    unsigned long long M = s < 64 ? (m16 + (1ull << (s - 1))) >> s : 0ull;
    if (ef == 0 || E == kNoExp) M = 0;
    return bits < 0 ? -(long long)M : (long long)M;
}

// Balanced base-128 digits of X, most significant first, X = sum_i D_i
// 128^{7-i}: with C = 64 (1 + 128 + ... + 128^7), the word P = X + C is
// non-negative and below 2^57, and D_i = u_i - 64 for its 7-bit fields u_i
// (the top field, bits 49 and up, unmasked), so |D_i| <= 64 with no carry
// chain.  The digits are formed in FP32 (below), exactly; their low 16 bits
// are zero, so the high half of each is D_i in BF16.
constexpr unsigned long long kDigitOffset = 0x0081020408102040ull;   // 64 in every 7-bit field

__device__ __forceinline__ unsigned long long digit_word(long long X) { return (unsigned long long)(X + (long long)kDigitOffset); }

// The digits on the FP32 pipe (twice the lanes of the integer pipe), from
// three pieces of P that FP32 holds exactly: piece 0 = P >> 42 (< 2^15)
// gives digits 0 and 1, piece 1 = bits 21..41 digits 2..4, piece 2 = bits
// 0..20 digits 5..7.  For 0 <= x < 2^22, RD(x + 2^23) - 2^23 = floor(x), and
// subtracting 2^23 + 64 instead gives the balanced digit; every other step is
// a fused multiply-add of integers below 2^24, exact.
template <int PIECE>
__device__ __forceinline__ void piece_digits(unsigned long long P, float* d)
{
    const uint32_t lo = (uint32_t)P, hi = (uint32_t)(P >> 32);
    if constexpr (PIECE == 0) {
        const float v = __uint_as_float(0x4B000000u | (hi >> 10)) - 8388608.0f;
        d[0] = __fmaf_rd(v, 0.0078125f, 8388608.0f) - 8388672.0f;              // floor(v / 2^7) - 64
        d[1] = fmaf(d[0], -128.0f, v - 8256.0f);                                 // v mod 2^7 - 64
    } else {
        const uint32_t u = PIECE == 1 ? (__funnelshift_r(lo, hi, 21) & 0x1FFFFFu) : (lo & 0x1FFFFFu);
        const float v = __uint_as_float(0x4B000000u | u) - 8388608.0f;
        d[0] = __fmaf_rd(v, 6.103515625e-05f, 8388608.0f) - 8388672.0f;         // floor(v / 2^14) - 64
        const float r = fmaf(d[0], -16384.0f, v - 1048576.0f);                   // v mod 2^14
        d[1] = __fmaf_rd(r, 0.0078125f, 8388608.0f) - 8388672.0f;              // floor(r / 2^7) - 64
        d[2] = fmaf(d[1], -128.0f, r - 8256.0f);                                 // r mod 2^7 - 64
    }
}

// The digits of one piece of RUN words, each digit plane a store of RUN
// consecutive BF16 values (planes dstride elements apart); two digits share
// a 32-bit word, the first in its low half.
template <int PIECE, int RUN>
__device__ __forceinline__ void store_piece(__nv_bfloat16* dst, int64_t dstride, const unsigned long long* pk)
{
    constexpr int ND = PIECE == 0 ? 2 : 3;
    float d[RUN][3];
#pragma unroll
    for (int j = 0; j < RUN; ++j) piece_digits<PIECE>(pk[j], d[j]);
#pragma unroll
    for (int k = 0; k < ND; ++k) {
        uint32_t wv[RUN / 2];
#pragma unroll
        for (int u = 0; u < RUN / 2; ++u)
            wv[u] = __byte_perm(__float_as_uint(d[2 * u][k]), __float_as_uint(d[2 * u + 1][k]), 0x7632);
        __nv_bfloat16* q = dst + k * dstride;
        if constexpr (RUN == 8) *reinterpret_cast<uint4*>(q) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        else if constexpr (RUN == 4) *reinterpret_cast<uint2*>(q) = make_uint2(wv[0], wv[1]);
        else *reinterpret_cast<uint32_t*>(q) = wv[0];
    }
}

// ------------------------------------------------------------ fused tables

// One level k >= 1 of one side's factor table, built and split in one pass
// (the tables are never stored in the [sign vector][entry] layout of the
// FP64 path): entry(P)(d) = entry(P minus its last mode r)(d) y_r(d) /
// sqrt(multiplicity of r in P), level 0 being sigma(d) 2^{-(n-1)} norm_t on
// the low side and 1 on the high side.  Kpad / 128 warps per entry P (one
// for Kpad <= 128), each lane holding 4 sign vectors (2 at Kpad = 64; those
// >= K are zero): the entry's exponent (one for re, im and re + im) is a
// maximum over its warps, so the digits [3][8][entry][Kpad] are written in
// the same pass.  Levels below
// n - 1 also keep the complex entries, entry-major [entry][K], as the parents
// of the next level.  Low side: writes lowbase of each entry.
struct TcLevelArgs {
    MultisetTable mc;
    int m, n, h, side, k, K, Kpad;
    int64_t count;                       // entries of level k
    double lead;                         // 2^{-(n-1)} norm_t
    const double2* Ys;                   // [n-1][m][K]: y_r(d) / sqrt(mult), mult = 1 .. n-1
    const double2* parent;               // level k-1, [entry][K] (k >= 2)
    double2* out;                        // level k, [entry][K], or null
    int64_t dig_off, wdig;               // entry offset of level k in the digit tensor; its entries
    __nv_bfloat16* digits;               // [3][8][wdig][Kpad]
    int* ex;                             // [3][wdig]
    int64_t* lowbase;                    // low side: at lowoff_k + entry, else null
    int64_t lowoff_k;
};

// Ys[mult-1][r][d] = y_r(d) / sqrt(mult) (mult = 1: y_r(d) itself), the
// factor a level entry whose last mode r occurs mult times takes from its
// parent; sign vectors contiguous per (mult, r).
__global__ void scaled_rowsums_kernel(const double2* __restrict__ Y, int m, int K, int nmult, double2* __restrict__ Ys)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nmult * m * K) return;
    const int mu = (int)(i / ((int64_t)m * K));
    const int64_t rem = i % ((int64_t)m * K);
    const int r = (int)(rem / K), q = (int)(rem % K);
    double2 y = Y[(int64_t)q * m + r];
    if (mu > 0) {
        const double sc = inv_sqrt_int(mu + 1);
        y.x *= sc;
        y.y *= sc;
    }
    Ys[i] = y;
}


template <int PER, int WPE>
__global__ void __launch_bounds__(128) tc_level_kernel(const TcLevelArgs a)
{
    // WPE warps per entry (4 / WPE entries per block), warp `part` holding
    // sign vectors part 32 PER .. (part + 1) 32 PER - 1
    __shared__ int s_f[4][3];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int part = warp % WPE;
    const int64_t e = (int64_t)blockIdx.x * (4 / WPE) + warp / WPE;
    const bool valid = e < a.count;
    const int w = a.side == 0 ? a.h : a.m - a.h;
    const int shift = a.side == 0 ? 0 : a.h;
    int mult = 1, r = 0;
    int64_t parent = 0;
    if (valid) {
        // unrank P (non-decreasing modes, lexicographic order) and, in the same
        // walk, the rank of P minus its last mode among (k-1)-multisets, the
        // run length of the last mode, and (low side) the canonical index of
        // the first output with prefix P and the rest in [h, m)
        const bool want_base = a.lowbase && lane == 0 && part == 0;
        int64_t idx = e, base = 0;
        int v = 0, prevmode = -1;
        for (int p = 0; p < a.k; ++p) {
            const int rest = a.k - p - 1;
            for (;;) {
                const int64_t c = a.mc(w - v, rest);
                if (idx < c) break;
                idx -= c;
                if (p < a.k - 1) parent += a.mc(w - v, a.k - 2 - p);
                if (want_base) base += a.mc(a.m - v, a.n - p - 1);
                ++v;
            }
            mult = v == prevmode ? mult + 1 : 1;
            prevmode = v;
        }
        r = v + shift;
        if (want_base) {
            if (a.k < a.n)
                for (int u = v; u < a.h; ++u) base += a.mc(a.m - u, a.n - a.k - 1);
            a.lowbase[a.lowoff_k + e] = base;
        }
    }
    const double2* yr = a.Ys + ((int64_t)(mult - 1) * a.m + r) * a.K;
    // lane l holds runs of RUN consecutive sign vectors, run j0 / RUN at
    // j0 32 + l RUN of this warp's range, so that each 16-byte digit store of
    // a warp covers 512 contiguous bytes
    constexpr int RUN = PER < 8 ? PER : 8;
    const int qbase = part * 32 * PER;
    double2 v[PER];
    int fc = 0;                                            // largest exponent field of re and im
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int q = qbase + (j / RUN) * 32 * RUN + lane * RUN + (j % RUN);
        v[j] = make_double2(0.0, 0.0);
        if (valid && q < a.K) {
            const double2 y = yr[q];
            double2 pv;
            if (a.k == 1) {
                double lv = 1.0;
                if (a.side == 0) {
                    const uint64_t d = (uint64_t)q;
                    lv = (__popcll(d ^ (d >> 1)) & 1) ? -a.lead : a.lead;
                }
                pv = make_double2(lv, 0.0);
            } else {
                pv = a.parent[parent * a.K + q];
            }
            v[j] = cmul(pv, y);
            if (a.out) a.out[e * a.K + q] = v[j];
        }
        fc = max(fc, max(exp_field(v[j].x), exp_field(v[j].y)));
    }
    fc = __reduce_max_sync(0xffffffffu, fc);
    if constexpr (WPE > 1) {
        if (lane == 0) s_f[warp][0] = fc;
        __syncthreads();
        const int w0 = warp - part;
#pragma unroll
        for (int u = 0; u < WPE; ++u) fc = max(fc, s_f[w0 + u][0]);
    }
    if (!valid) return;
    const int64_t ent = a.dig_off + e;
    // One exponent for re, im and re + im of the entry, one bit above their
    // largest: |re|, |im| <= 2^{E-2}, so |X_re|, |X_im| <= 2^54 and the third
    // operand X_re + X_im (|.| <= 2^55) is formed exactly in integers; the
    // third product then equals t1 + t2 + the imaginary part exactly.
    const int E = fc ? fc - 1020 : kNoExp;
    if (lane == 0 && part == 0)
        for (int t = 0; t < 3; ++t) a.ex[(int64_t)t * a.wdig + ent] = E;
#pragma unroll
    for (int j0 = 0; j0 < PER; j0 += RUN) {
        long long xr[RUN], xi[RUN];
#pragma unroll
        for (int j = 0; j < RUN; ++j) {
            xr[j] = fixed_of(v[j0 + j].x, E);
            xi[j] = fixed_of(v[j0 + j].y, E);
        }
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            unsigned long long pk[RUN];
#pragma unroll
            for (int j = 0; j < RUN; ++j) pk[j] = digit_word(t == 0 ? xr[j] : (t == 1 ? xi[j] : xr[j] + xi[j]));
            const int64_t plane = a.wdig * a.Kpad;                 // elements between digit planes
            __nv_bfloat16* d0 = a.digits + ((int64_t)t * kDigits * a.wdig + ent) * a.Kpad + qbase + j0 * 32 + lane * RUN;
            store_piece<0, RUN>(d0, plane, pk);
            store_piece<1, RUN>(d0 + 2 * plane, plane, pk);
            store_piece<2, RUN>(d0 + 5 * plane, plane, pk);
        }
    }
}

// One warp: 4 consecutive entries x 32 consecutive sign vectors (lane ->
// entry lane & 3, sign vectors 4 (lane >> 2) .. + 3).  Loads take 64-byte
// segments of the tables; each product and digit is one 8-byte store per
// lane (64-byte segments along K of the digit tensors).  No shared memory.
__global__ void __launch_bounds__(256) split_digits_kernel(const double2* __restrict__ T, const double* __restrict__ Sm,
                                                           int64_t stride, int64_t w, int K, int Kpad,
                                                           const int* __restrict__ ex, __nv_bfloat16* __restrict__ out)
{
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int ndg = Kpad / 32;
    const int64_t eg = gw / ndg;
    const int dg = (int)(gw % ndg);
    const int64_t e = eg * 4 + (lane & 3);
    const int d0 = dg * 32 + (lane >> 2) * 4;
    if (e >= w) return;
    double vr[4], vi[4], vs[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int d = d0 + u;
        if (d < K) {
            const double2 v = T[(int64_t)d * stride + e];
            vr[u] = v.x;
            vi[u] = v.y;
            vs[u] = Sm[(int64_t)d * stride + e];
        } else {
            vr[u] = vi[u] = vs[u] = 0.0;
        }
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        const int E = ex[(int64_t)t * w + e];
        unsigned long long pk[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) pk[u] = digit_word(fixed_of(t == 0 ? vr[u] : (t == 1 ? vi[u] : vs[u]), E));
        const int64_t plane = (int64_t)w * Kpad;
        __nv_bfloat16* q = out + ((int64_t)t * kDigits * w + e) * Kpad + d0;
        store_piece<0, 4>(q, plane, pk);
        store_piece<1, 4>(q + 2 * plane, plane, pk);
        store_piece<2, 4>(q + 5 * plane, plane, pk);
    }
}

// ------------------------------------------------------------ products

constexpr int kMaxBlocks = PCV_MAX_PHOTONS + 2;     // k = 1 .. n-1 and the two single-entry blocks

struct TcProdArgs {
    int nk;                                   // blocks with outputs
    int kblocks;                              // 64-wide K blocks
    int64_t tile0[kMaxBlocks + 1];            // first tile of each block
    int64_t tiles;                            // all tiles
    int rows_low[kMaxBlocks];                 // 1: rows are low-side entries P, columns high-side Q
    // Columns of a block: [0, ncol) from the other side's table levels
    // (col_off), then [ecol0, ecol0 + ecols) single-entry columns (see below);
    // a block k = 1 or k = n-1 whose rows are level n-1 carries the
    // single-entry columns of that side when both fit one tile
    int ncol[kMaxBlocks], ecol0[kMaxBlocks], ecols[kMaxBlocks];
    int tn[kMaxBlocks];                       // tile width (16..64)
    // tiles cover rows [rows0, rows) and columns [cols0, cols) of the block:
    // all of it, or the rows or columns of the P whose outputs meet [lo, hi)
    int64_t rows0[kMaxBlocks], rows[kMaxBlocks], cols0[kMaxBlocks], cols[kMaxBlocks];
    int64_t row_off[kMaxBlocks], col_off[kMaxBlocks];   // entry offsets in the digit tensors
    int64_t lowoff[kMaxBlocks];               // level offset of P (for lowbase)
    const int64_t* lowbase;
    const int* ex_low;                        // [3][wlow]
    const int* ex_high;                       // [3][whigh]
    int64_t wlow, whigh;
    // Single-entry blocks, by the side s of their rows (0 low, 1 high): the
    // rows are the level n-1 entries R' of side s, the columns the modes r of
    // side s with the vectors v_r of that side (digits under the v maps), and
    // the output of (R', r), r >= max R', is entry R' + r of level n:
    // index efirst[s][R'] + r - max R', scaled by esc[s][R'] when r = max R'.
    const int* ex_v[2];                       // [3][modes of side s]
    const int64_t* efirst[2];
    const int* emax[2];
    const double* esc[2];
    double* xt;                               // [2][hi - lo]: the real products t1, t2 per output
    int64_t lo, hi;                           // outputs [lo, hi) are written, at o - lo
    double2* amp;                             // amplitudes, or null
    double* prob;                             // probabilities, or null
    int* error;                               // set to the role that gave up (1 producer, 2 MMA, 3 drain,
                                              // 4 clean-up), or null
    long long max_polls;                      // bound of one mbarrier wait
};

using tcx::mbar_arrive;
using tcx::mbar_expect_tx;
using tcx::mbar_init;
using tcx::mbar_wait;
using tcx::mma_bf16;
using tcx::mma_commit;
using tcx::sdesc_sw128;
using tcx::tma_load_4d;

__device__ __forceinline__ double pow2(int e)      // 2^e for -1022 <= e <= 1023
{
    return __longlong_as_double((long long)(1023 + e) << 52);
}

// RN(Z 2^s) for the exact integer Z = zh 2^28 + zl (0 <= zl < 2^28, |Z| <
// 2^75), from 64-bit integer operations only (FP64 arithmetic is scarce on
// this part): |Z| is shifted so that its leading one is bit 63 of a word, the
// top 53 bits are kept and rounded to nearest even, with the bits shifted out
// of the word as a sticky bit.  Z = hi 2^28 + lo is the combination of the
// diagonal sums, so this is the value fma(lo, 2^s, hi 2^{s+28}) rounds to.
// Returns false if the result would not be a normal number; the caller then
// takes the FP64 expression.
__device__ __forceinline__ bool scale_packed(long long zh, uint32_t zl, int s, double& out)
{
    const bool neg = zh < 0;
    unsigned long long mh;                                 // |Z| = mh 2^28 + ml
    uint32_t ml;
    if (!neg) {
        mh = (unsigned long long)zh;
        ml = zl;
    } else if (zl == 0) {
        mh = (unsigned long long)(-zh);
        ml = 0;
    } else {
        mh = (unsigned long long)(-zh) - 1;
        ml = (1u << 28) - zl;
    }
    if (mh == 0) {
        if (ml == 0) {
            out = 0.0;
            return true;
        }
        mh = ml;
        ml = 0;
        s -= 28;
    }
    const int lz = __clzll((long long)mh);
    const int sh = lz - 28;
    unsigned long long T = mh << lz;
    bool sticky = false;
    if (sh >= 0) {
        T |= (unsigned long long)ml << sh;
    } else {
        T |= (unsigned long long)(ml >> (-sh));
        sticky = (ml & ((1u << (-sh)) - 1)) != 0;
    }
    unsigned long long mant = T >> 11;
    const uint32_t rb = (uint32_t)(T & 0x7FF);
    if (rb > 0x400 || (rb == 0x400 && (sticky || (mant & 1)))) ++mant;
    int ef = s + (64 - lz + 28) + 1022;                    // |Z| has 64 - lz + 28 bits
    if (mant >> 53) {
        mant >>= 1;
        ++ef;
    }
    if (ef < 1 || ef > 2046) return false;
    out = __longlong_as_double((long long)(((unsigned long long)neg << 63) | ((unsigned long long)ef << 52) |
                                           (mant & ((1ull << 52) - 1))));
    return true;
}

// Row digits in the order 0, 7, 1, 6, 2, 5, 3, 4: digit i is multiplied by
// 8 - i column digits, so alternating long and short products keeps the MMA
// time between consecutive row-digit loads even (the slots then stay about
// equally far ahead of the MMA).  Digit 0 comes first: its products start
// every diagonal.
__device__ __forceinline__ int slice_order(int ii) { return (ii & 1) ? kDigits - 1 - (ii >> 1) : (ii >> 1); }

// A tile's place: k block, first row and column, width, and which side the
// rows come from.  Tiles are numbered k block by k block, column tiles
// fastest, so CTAs that run at the same time share row digits.
struct TileInfo {
    int kb, tn;
    int64_t r0, c0;
    bool rl;
    int rentry, centry;
};

__device__ __forceinline__ TileInfo tile_info(const TcProdArgs& a, int64_t tile)
{
    TileInfo ti;
    int kb = 0;
    while (kb + 1 < a.nk && a.tile0[kb + 1] <= tile) ++kb;
    ti.kb = kb;
    ti.tn = a.tn[kb];
    const int64_t ctiles = (a.cols[kb] - a.cols0[kb] + ti.tn - 1) / ti.tn;
    const int64_t lt = tile - a.tile0[kb];
    ti.r0 = a.rows0[kb] + (lt / ctiles) * TBM;
    ti.c0 = a.cols0[kb] + (lt % ctiles) * ti.tn;
    ti.rl = a.rows_low[kb] != 0;
    ti.rentry = (int)(a.row_off[kb] + ti.r0);
    ti.centry = (int)(a.col_off[kb] + ti.c0);
    return ti;
}

// Persistent: CTA b takes tiles b, b + grid, b + 2 grid, ...  The work of a
// CTA is a sequence of chunks q = (tile, product t, 64-wide K block c); the
// producer issues chunk q + 1's column digits after chunk q's third row digit
// (by then chunk q - 1, the last user of that buffer, is nearly done), and
// the next tile's loads while the drain finishes the last one.
__global__ void __launch_bounds__(kThreads, 1)
tc_product_kernel(const __grid_constant__ CUtensorMap low_rows, const __grid_constant__ CUtensorMap low_cols,
                  const __grid_constant__ CUtensorMap high_rows, const __grid_constant__ CUtensorMap high_cols,
                  const __grid_constant__ CUtensorMap low_cols16, const __grid_constant__ CUtensorMap high_cols16,
                  const __grid_constant__ CUtensorMap vlow16, const __grid_constant__ CUtensorMap vhigh16,
                  const TcProdArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* bset = base;                                // kBSets x 64 KB
    unsigned char* aslot = base + kBSets * kBBytes;            // kASlots x 16 KB
    __shared__ __align__(8) uint64_t bfull[kBSets], bempty[kBSets], afull[kASlots], aempty[kASlots];
    __shared__ __align__(8) uint64_t accfull, accempty, mma_done;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nkb = a.kblocks;
    const int64_t my_tiles = a.tiles > (int64_t)blockIdx.x ? (a.tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const uint32_t nchunks = (uint32_t)(my_tiles * 3 * nkb);      // < 2^31 (checked on the host)

    if (tid == 0) {
        for (int s = 0; s < kBSets; ++s) {
            mbar_init(&bfull[s], 1);
            mbar_init(&bempty[s], 1);
        }
        for (int s = 0; s < kASlots; ++s) {
            mbar_init(&afull[s], 1);
            mbar_init(&aempty[s], 1);
        }
        mbar_init(&accfull, 1);
        mbar_init(&accempty, 256);
        mbar_init(&mma_done, 1);
        s_fail = 0;
        tcx::mbar_fence_init();
        tcx::prefetch_tmap(&low_rows);
        tcx::prefetch_tmap(&low_cols);
        tcx::prefetch_tmap(&high_rows);
        tcx::prefetch_tmap(&high_cols);
        tcx::prefetch_tmap(&low_cols16);
        tcx::prefetch_tmap(&high_cols16);
        tcx::prefetch_tmap(&vlow16);
        tcx::prefetch_tmap(&vhigh16);
    }
    if (warp == 1) tcx::tmem_alloc(&tmem_base, kTmemCols);
    tcx::fence_before_sync();
    __syncthreads();
    tcx::fence_after_sync();
    const uint32_t tmem = tmem_base;
    const long long polls = a.max_polls;

    if (tid == 0) {
        // ---------------- row-operand producer: for every chunk q = (tile,
        // product t, K block c), in that nesting, the 8 digit slices of the
        // row tile, one per slot, in the MMA's digit order
        uint32_t na = 0;                                              // row slices issued
        for (int64_t it = 0; it < my_tiles && !s_fail; ++it) {
            const TileInfo ti = tile_info(a, blockIdx.x + it * gridDim.x);
            const CUtensorMap* rmap = ti.rl ? &low_rows : &high_rows;
            for (int t = 0; t < 3 && !s_fail; ++t) {
                for (int c = 0; c < nkb && !s_fail; ++c) {
                    for (int ii = 0; ii < kDigits; ++ii) {
                        const uint32_t as = na % kASlots;
                        if (na >= (uint32_t)kASlots && !mbar_wait(&aempty[as], ((na / kASlots) - 1) & 1, polls)) {
                            s_fail = 1;
                            break;
                        }
                        mbar_expect_tx(&afull[as], kABytes);
                        tma_load_4d(aslot + as * kABytes, rmap, &afull[as], c * TBK, ti.rentry, slice_order(ii), t);
                        ++na;
                    }
                }
            }
        }
        // every load issued lands in this CTA's shared memory: wait for the
        // ones no consumer waited for before the CTA may exit
        if (!tcx::wait_issued(afull, kASlots, na) && !s_fail) s_fail = 4;
    } else if (tid == kColWarp * 32) {
        // ---------------- column-operand producer: for every chunk, the digit
        // slices of the column tile packed one after the other in a set
        // (double-buffered), so a slow set never holds up the row slices
        uint32_t q = 0;                                               // column sets issued
        for (int64_t it = 0; it < my_tiles && !s_fail; ++it) {
            const TileInfo tb = tile_info(a, blockIdx.x + it * gridDim.x);
            for (int t = 0; t < 3 && !s_fail; ++t) {
                for (int c = 0; c < nkb && !s_fail; ++c, ++q) {
                    const uint32_t bs = q % kBSets;
                    if (q >= kBSets && !mbar_wait(&bempty[bs], ((q / kBSets) - 1) & 1, polls)) {
                        s_fail = 1;
                        break;
                    }
                    // slice j at rows j N .. j N + N - 1 of the set: one 64-row
                    // box, or N / 16 boxes of 16 rows
                    unsigned char* dst = bset + bs * kBBytes;
                    mbar_expect_tx(&bfull[bs], (uint32_t)(kDigits * tb.tn) * kRowBytes);
                    if (tb.tn == TBN && a.ecols[tb.kb] == 0) {
                        const CUtensorMap* cmap = tb.rl ? &high_cols : &low_cols;
                        for (int j = 0; j < kDigits; ++j)
                            tma_load_4d(dst + j * TBN * kRowBytes, cmap, &bfull[bs], c * TBK, tb.centry, j, t);
                    } else {
                        // 16-row boxes; those at or past ecol0 come from the
                        // vectors of the single-entry columns (ecol0 is a
                        // multiple of 16)
                        const int e0 = a.ecol0[tb.kb];
                        const CUtensorMap* nmap = tb.rl ? &high_cols16 : &low_cols16;
                        const CUtensorMap* vmap = tb.rl ? &vlow16 : &vhigh16;
                        for (int j = 0; j < kDigits; ++j)
                            for (int r = 0; r < tb.tn; r += kBSub) {
                                const int lc = (int)tb.c0 + r;
                                if (lc < e0)
                                    tma_load_4d(dst + (j * tb.tn + r) * kRowBytes, nmap, &bfull[bs], c * TBK,
                                                tb.centry + r, j, t);
                                else
                                    tma_load_4d(dst + (j * tb.tn + r) * kRowBytes, vmap, &bfull[bs], c * TBK,
                                                lc - e0, j, t);
                            }
                    }
                }
            }
        }
        if (!tcx::wait_issued(bfull, kBSets, q) && !s_fail) s_fail = 4;
    } else if (tid == 32) {
        // ---------------- MMA issuer
        uint32_t na = 0, q = 0, g = 0;                               // slices, chunks, passes
        for (int64_t it = 0; it < my_tiles && !s_fail; ++it) {
            const int tn = tile_info(a, blockIdx.x + it * gridDim.x).tn;
            const int per = min(kDigits, 256 / tn);                      // column slices per MMA
            for (int t = 0; t < 3 && !s_fail; ++t, ++g) {
                if (g > 0 && !mbar_wait(&accempty, (g - 1) & 1, polls)) {
                    s_fail = 2;
                    break;
                }
                tcx::fence_after_sync();
                for (int c = 0; c < nkb && !s_fail; ++c, ++q) {
                    const uint32_t bs = q % kBSets;
                    if (!mbar_wait(&bfull[bs], (q / kBSets) & 1, polls)) {
                        s_fail = 2;
                        break;
                    }
                    // descriptors are linear in the address (16-byte units in
                    // the low bits): one per slice, plus 2 per 16-wide K step
                    const uint64_t db0 = sdesc_sw128(bset + bs * kBBytes);
                    for (int ii = 0; ii < kDigits; ++ii) {
                        const int i = slice_order(ii);
                        const uint32_t as = na % kASlots;
                        if (!mbar_wait(&afull[as], (na / kASlots) & 1, polls)) {
                            s_fail = 2;
                            break;
                        }
                        tcx::fence_after_sync();
                        const uint64_t da = sdesc_sw128(aslot + as * kABytes);
                        const uint32_t first = (c == 0 && ii == 0) ? 0u : 1u;
                        for (int j0 = 0; j0 < kDigits - i; j0 += per) {
                            const int ns = min(per, kDigits - i - j0);
                            const uint32_t idesc = tcx::idesc_bf16(TBM, ns * tn);
                            const uint32_t acc_t = tmem + (uint32_t)((i + j0) * tn);
                            const uint64_t db = db0 + (uint64_t)((j0 * tn * kRowBytes) >> 4);
                            mma_bf16(acc_t, da, db, idesc, first);
                            mma_bf16(acc_t, da + 2, db + 2, idesc, 1u);
                            mma_bf16(acc_t, da + 4, db + 4, idesc, 1u);
                            mma_bf16(acc_t, da + 6, db + 6, idesc, 1u);
                        }
                        mma_commit(&aempty[as]);
                        ++na;
                    }
                    mma_commit(&bempty[bs]);
                }
                if (!s_fail) mma_commit(&accfull);
            }
        }
        // the MMAs issued are complete before the tensor memory is released
        if (na > 0) {
            mma_commit(&mma_done);
            if (!mbar_wait(&mma_done, 0, tcx::kCleanupPolls) && !s_fail) s_fail = 4;
        }
    } else if (warp >= 2 && warp < kColWarp) {
        // ---------------- drain: warp w owns TMEM lanes 32 (w mod 4) .. + 31;
        // warps 2-5 take the 16-column chunks at 0 and 32, warps 6-9 those at
        // 16 and 48 (so a 32-wide tile keeps all eight busy)
        const int q4 = warp & 3;
        const int cbase = warp < 6 ? 0 : 16;
        bool alive = true;
        for (int64_t it = 0; it < my_tiles && alive; ++it) {
            const TileInfo ti = tile_info(a, blockIdx.x + it * gridDim.x);
            const int kb = ti.kb, tn = ti.tn;
            const bool rl = ti.rl;
            const int64_t row = ti.r0 + q4 * 32 + lane;
            const bool rv = row < a.rows[kb];
            const int side = rl ? 0 : 1;
            const int* ex_r = rl ? a.ex_low : a.ex_high;
            const int* ex_c = rl ? a.ex_high : a.ex_low;
            const int* ex_e = a.ex_v[side];
            const int64_t wr = rl ? a.wlow : a.whigh, wc = rl ? a.whigh : a.wlow;
            const int ncol = a.ncol[kb], e0 = a.ecol0[kb], necol = a.ecols[kb];
            int64_t pbase = 0;                     // lowbase(P) of a low-side row
            int64_t ebase = 0;                     // efirst(R') - max R' of a level n-1 row
            int emx = 0;
            double esc = 1.0;
            if (rv && necol > 0) {
                emx = a.emax[side][row];
                esc = a.esc[side][row];
                ebase = a.efirst[side][row] - emx;
            }
            if (rv && rl && ncol > 0) pbase = a.lowbase[a.lowoff[kb] + row];
            for (int t = 0; t < 3; ++t) {
                const int64_t g = it * 3 + t;
                const int er = rv ? ex_r[(int64_t)t * wr + a.row_off[kb] + row] : kNoExp;
                if (!mbar_wait(&accfull, (uint32_t)g & 1, polls)) {
                    if (lane == 0) s_fail = 3;
                    alive = false;
                    break;
                }
                tcx::fence_after_sync();
                // read the 8 diagonals of this warp's columns (16-wide chunks
                // cc = 0, 32 for warps 2-5 and 16, 48 for warps 6-9) and
                // combine them on the integer pipe into Z = zh 2^28 + zl, then
                // hand the accumulators back to the MMA; the rounding to FP64
                // and the stores come after
                long long zh[2][16];
                uint32_t zl[2][16];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int cc = cbase + 32 * h;
                    if (cc >= tn) continue;
                    long long hi[16], lo[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) hi[q] = lo[q] = 0;
#pragma unroll
                    for (int d = 0; d < kDigits; ++d) {
                        uint32_t r[16];
                        const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(d * tn + cc);
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
                            "%14,%15}, [%16];\n"
                            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                              "=r"(r[14]), "=r"(r[15])
                            : "r"(taddr));
                        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const long long v = (long long)__float2int_rn(__uint_as_float(r[q]));
                            if (d < 4) hi[q] = hi[q] * 128 + v;
                            else lo[q] = lo[q] * 128 + v;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        zh[h][q] = hi[q] + (lo[q] >> 28);
                        zl[h][q] = (uint32_t)(lo[q] & ((1ll << 28) - 1));
                    }
                }
                tcx::fence_before_sync();
                mbar_arrive(&accempty);
                // the per-column data of this warp's two 16-column chunks:
                // lane l loads that of column l mod 16 of each chunk, and the
                // loop below broadcasts it (no loads inside the loop)
                int ecl[2];
                int64_t lbl[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int64_t col = ti.c0 + cbase + 32 * h + (lane & 15);
                    const int64_t ce = col - e0;
                    ecl[h] = kNoExp;
                    lbl[h] = 0;
                    if (cbase + 32 * h < tn) {
                        if (col >= e0) {
                            if (ce < necol) ecl[h] = ex_e[(int64_t)t * necol + ce];
                        } else if (col < ncol) {
                            ecl[h] = ex_c[(int64_t)t * wc + a.col_off[kb] + col];
                            if (!rl) lbl[h] = a.lowbase[a.lowoff[kb] + col];
                        }
                    }
                }
                // t1 and t2 go to the workspace; with t3, the same thread
                // forms a = (t1 - t2) + i (t3 - t1 - t2) and |a|^2
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int cc = cbase + 32 * h;
                    if (cc >= tn) continue;
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int ec = __shfl_sync(0xffffffffu, ecl[h], q);
                        const int64_t lb = __shfl_sync(0xffffffffu, lbl[h], q);
                        const int64_t col = ti.c0 + cc + q;
                        const bool is_e = col >= e0;       // a single-entry column: mode ce of this side
                        const int64_t ce = col - e0;
                        if (!rv || (is_e ? (ce >= necol || ce < emx) : (col >= ncol))) continue;
                        double x = 0.0;
                        if (er != kNoExp && ec != kNoExp) {
                            const int sc = er + ec - 14;
                            if (!scale_packed(zh[h][q], zl[h][q], sc - 49, x))
                                x = fma((double)zl[h][q], pow2(sc - 49), (double)zh[h][q] * pow2(sc - 21));
                        }
                        const int64_t og = is_e ? ebase + ce : (rl ? pbase + col : lb + row);
                        if (og < a.lo || og >= a.hi) continue;
                        const int64_t o = og - a.lo, span = a.hi - a.lo;
                        if (t < 2) {
                            a.xt[(int64_t)t * span + o] = x;
                        } else {
                            const double t1 = a.xt[o], t2 = a.xt[span + o];
                            double re = t1 - t2, im = x - t1 - t2;
                            if (is_e && ce == emx) {           // 1 / sqrt(multiplicity of r in R' + r)
                                re *= esc;
                                im *= esc;
                            }
                            if (a.amp) a.amp[o] = make_double2(re, im);
                            if (a.prob) a.prob[o] = fma(re, re, im * im);
                        }
                    }
                }
            }
        }
    }
    tcx::fence_before_sync();
    __syncthreads();
    if (warp == 1) tcx::tmem_dealloc(tmem, kTmemCols);
    if (tid == 0 && s_fail && a.error) atomicExch(a.error, s_fail);
}

// Column vectors of the single-entry blocks, per sign vector d and mode r:
//   low side  (block k = n, rows P'):  v_r(d) = y_r(d) beta_{}(d),
//   high side (block k = 0, rows Q'):  v_r(d) = alpha_{}(d) y_{h+r}(d),
// so that sum_d entry_{R'}(d) v_r(d) is the output of R' + r up to the
// 1/sqrt(multiplicity) that level n would have applied.  [K][modes] each,
// with re + im beside them for the third product.
__global__ void edge_vectors_kernel(const double2* __restrict__ Y, int m, int h, int K, double lead,
                                    double2* __restrict__ Vl, double* __restrict__ Sl, double2* __restrict__ Vh,
                                    double* __restrict__ Sh)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)K * m) return;
    const int64_t q = i / m;
    const int r = (int)(i % m);
    const double2 y = Y[q * m + r];
    if (r < h) {                                           // beta_{}(d) = 1
        const double2 v = cmul(y, make_double2(1.0, 0.0));
        Vl[q * h + r] = v;
        Sl[q * h + r] = v.x + v.y;
    } else {                                               // alpha_{}(d) = sigma(d) 2^{-(n-1)} norm_t
        const uint64_t d = (uint64_t)q;
        const double2 t0 = make_double2((__popcll(d ^ (d >> 1)) & 1) ? -lead : lead, 0.0);
        const double2 v = cmul(t0, y);
        Vh[q * (m - h) + (r - h)] = v;
        Sh[q * (m - h) + (r - h)] = v.x + v.y;
    }
}

// Per level n-1 entry R' of one side (modes in [0, w), shifted by `shift` in
// the output): its largest mode, the canonical output index of R' + max R',
// and 1/sqrt(multiplicity of max R' in R' + max R').  Low side: the output
// index among all n-photon outputs; high side: lowbase({}) + rank of Q'+max.
__global__ void edge_info_kernel(MultisetTable mc, int m, int n, int h, int side, int64_t count,
                                 int64_t* __restrict__ first, int* __restrict__ mx, double* __restrict__ sc)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int w = side == 0 ? h : m - h;
    int modes[PCV_MAX_PHOTONS];
    unrank_multiset<PCV_MAX_PHOTONS>(mc, w, n - 1, i, modes);
    const int top = modes[n - 2];
    int mult = 1;
    for (int p = n - 2; p >= 0 && modes[p] == top; --p) ++mult;
    modes[n - 1] = top;
    int64_t o = 0;
    if (side == 0) {
        int prev = 0;
        for (int p = 0; p < n; ++p) {
            for (int v = prev; v < modes[p]; ++v) o += mc(m - v, n - p - 1);
            prev = modes[p];
        }
    } else {
        for (int v = 0; v < h; ++v) o += mc(m - v, n - 1);
        o += rank_multiset(mc, w, n, modes);
    }
    first[i] = o;
    mx[i] = top;
    sc[i] = inv_sqrt_int(mult);
}

PFN_cuTensorMapEncodeTiled_v12000 g_enc = nullptr;
std::once_flag g_enc_once;
bool g_tc_attr[64] = {};

cudaError_t get_enc()
{
    std::call_once(g_enc_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_enc = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    });
    return g_enc ? cudaSuccess : cudaErrorNotSupported;
}

// 4-D map over the digit tensor [3][8][w][Kpad] (bf16), box 64 (K) x rows.
cudaError_t make_digit_map(CUtensorMap* map, const void* base, int64_t w, int Kpad, int box_rows)
{
    const cuuint64_t dims[4] = {(cuuint64_t)Kpad, (cuuint64_t)w, (cuuint64_t)kDigits, 3};
    const cuuint64_t strides[3] = {(cuuint64_t)Kpad * 2, (cuuint64_t)w * Kpad * 2, (cuuint64_t)kDigits * w * Kpad * 2};
    const cuuint32_t box[4] = {(cuuint32_t)TBK, (cuuint32_t)box_rows, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = g_enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

int64_t binom_tc(int a, int b)
{
    if (b < 0 || a < 0 || b > a) return 0;
    unsigned __int128 c = 1;
    for (int i = 1; i <= b; ++i) c = c * (unsigned __int128)(a - b + i) / (unsigned __int128)i;
    return (int64_t)c;
}

int64_t msets_tc(int w, int k) { return k == 0 ? 1 : (w <= 0 ? 0 : binom_tc(w + k - 1, k)); }

}  // namespace

int tc_pad_k(int K) { return ((K + TBK - 1) / TBK) * TBK; }

namespace {

// Workspace layout: digits and exponents of table levels 1 .. n-1 of the two
// sides, the entry-major complex entries of levels 1 .. n-2 (parents), two
// products per output, the column vectors of the single-entry blocks (sized
// by m for both sides) with their digits and exponents, and the per-row data
// of those blocks (sized by levels 1 .. n-1).
struct TcLayout {
    int64_t lcnt, hcnt, plow, phigh;
    size_t dlow, dhigh, exlow, exhigh, tpl, tph, ys, xt, v, sv, dv, exv, efirst_l, emax_l, esc_l, efirst_h, emax_h, esc_h,
        total;
};

TcLayout tc_layout(int m, int n, int K, int64_t total, const int64_t* lowoff, const int64_t* highoff)
{
    const size_t Kp = (size_t)tc_pad_k(K);
    TcLayout L;
    L.lcnt = n >= 2 ? lowoff[n] - lowoff[1] : 0;
    L.hcnt = n >= 2 ? highoff[n] - highoff[1] : 0;
    L.plow = n >= 3 ? lowoff[n - 1] - lowoff[1] : 0;
    L.phigh = n >= 3 ? highoff[n - 1] - highoff[1] : 0;
    L.dlow = al256((size_t)3 * kDigits * L.lcnt * Kp * 2);
    L.dhigh = al256((size_t)3 * kDigits * L.hcnt * Kp * 2);
    L.exlow = al256((size_t)3 * L.lcnt * sizeof(int));
    L.exhigh = al256((size_t)3 * L.hcnt * sizeof(int));
    L.tpl = al256((size_t)L.plow * K * sizeof(double2));
    L.tph = al256((size_t)L.phigh * K * sizeof(double2));
    L.ys = al256((size_t)(n > 1 ? n - 1 : 1) * m * K * sizeof(double2));
    L.xt = al256((size_t)2 * total * sizeof(double));
    L.v = al256((size_t)K * m * sizeof(double2));
    L.sv = al256((size_t)K * m * sizeof(double));
    L.dv = al256((size_t)3 * kDigits * m * Kp * 2);
    L.exv = al256((size_t)3 * m * sizeof(int));
    L.efirst_l = al256((size_t)L.lcnt * sizeof(int64_t));
    L.emax_l = al256((size_t)L.lcnt * sizeof(int));
    L.esc_l = al256((size_t)L.lcnt * sizeof(double));
    L.efirst_h = al256((size_t)L.hcnt * sizeof(int64_t));
    L.emax_h = al256((size_t)L.hcnt * sizeof(int));
    L.esc_h = al256((size_t)L.hcnt * sizeof(double));
    L.total = L.dlow + L.dhigh + L.exlow + L.exhigh + L.tpl + L.tph + L.ys + L.xt + 2 * (L.v + L.sv + L.dv + L.exv) +
              L.efirst_l + L.emax_l + L.esc_l + L.efirst_h + L.emax_h + L.esc_h + 256;
    return L;
}

struct TcBuffers {
    __nv_bfloat16* dig[2];
    int* ex[2];
    double2* par[2];
    double2* ys;
    double* xt;
    double2* V[2];
    double* SV[2];
    __nv_bfloat16* DV[2];
    int* EXV[2];
    int64_t* efirst[2];
    int* emax[2];
    double* esc[2];
};

TcBuffers tc_buffers(const TcLayout& L, void* ws)
{
    TcBuffers B;
    char* w = (char*)ws;
    B.dig[0] = (__nv_bfloat16*)w;    w += L.dlow;
    B.dig[1] = (__nv_bfloat16*)w;    w += L.dhigh;
    B.ex[0] = (int*)w;               w += L.exlow;
    B.ex[1] = (int*)w;               w += L.exhigh;
    B.par[0] = (double2*)w;          w += L.tpl;
    B.par[1] = (double2*)w;          w += L.tph;
    B.ys = (double2*)w;              w += L.ys;
    B.xt = (double*)w;               w += L.xt;
    for (int side = 0; side < 2; ++side) {
        B.V[side] = (double2*)w;     w += L.v;
        B.SV[side] = (double*)w;     w += L.sv;
        B.DV[side] = (__nv_bfloat16*)w;  w += L.dv;
        B.EXV[side] = (int*)w;       w += L.exv;
    }
    B.efirst[0] = (int64_t*)w;       w += L.efirst_l;
    B.emax[0] = (int*)w;             w += L.emax_l;
    B.esc[0] = (double*)w;           w += L.esc_l;
    B.efirst[1] = (int64_t*)w;       w += L.efirst_h;
    B.emax[1] = (int*)w;             w += L.emax_h;
    B.esc[1] = (double*)w;           w += L.esc_h;
    return B;
}

template <int PER, int WPE>
cudaError_t launch_level(const TcLevelArgs& la, cudaStream_t s)
{
    const int64_t blocks = (la.count + (4 / WPE) - 1) / (4 / WPE);
    tc_level_kernel<PER, WPE><<<(unsigned)blocks, 128, 0, s>>>(la);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace

int64_t tc_workspace(int m, int n, int K, int64_t total, const int64_t* lowoff, const int64_t* highoff)
{
    return (int64_t)tc_layout(m, n, K, total, lowoff, highoff).total;
}

cudaError_t launch_tc_tables(const TcInputs& in, cudaStream_t s)
{
    const int K = in.K, Kp = tc_pad_k(K), n = in.n;
    if (n < 2 || Kp > 512) return cudaErrorInvalidValue;
    const TcLayout L = tc_layout(in.m, n, K, in.total, in.lowoff, in.highoff);
    const TcBuffers B = tc_buffers(L, in.ws);
    const int64_t nys = (int64_t)(n - 1) * in.m * K;
    scaled_rowsums_kernel<<<(unsigned)((nys + 255) / 256), 256, 0, s>>>(in.Y, in.m, K, n - 1, B.ys);
    note_launches(1);
    for (int side = 0; side < 2; ++side) {
        const int64_t* off = side == 0 ? in.lowoff : in.highoff;
        for (int k = 1; k < n; ++k) {
            TcLevelArgs la;
            la.mc = in.mc;
            la.m = in.m; la.n = n; la.h = in.h; la.side = side; la.k = k; la.K = K; la.Kpad = Kp;
            la.count = off[k + 1] - off[k];
            if (la.count == 0) continue;
            la.lead = in.lead;
            la.Ys = B.ys;
            la.parent = k >= 2 ? B.par[side] + (off[k - 1] - off[1]) * K : nullptr;
            la.out = k <= n - 2 ? B.par[side] + (off[k] - off[1]) * K : nullptr;
            la.dig_off = off[k] - off[1];
            la.wdig = side == 0 ? L.lcnt : L.hcnt;
            la.digits = B.dig[side];
            la.ex = B.ex[side];
            la.lowbase = side == 0 ? in.lowbase : nullptr;
            la.lowoff_k = off[k];
            cudaError_t e;
            switch (Kp / 32) {
                case 2: e = launch_level<2, 1>(la, s); break;           // Kpad = 64
                case 4: e = launch_level<4, 1>(la, s); break;           // 128
                case 8: e = launch_level<4, 2>(la, s); break;           // 256
                default: e = launch_level<4, 4>(la, s); break;          // 512
            }
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

cudaError_t launch_tc_products(const TcInputs& in, cudaStream_t s)
{
    cudaError_t e = get_enc();
    if (e != cudaSuccess) return e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && !g_tc_attr[dev]) {
        e = cudaFuncSetAttribute(tc_product_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
        if (e != cudaSuccess) return e;
        g_tc_attr[dev] = true;
    }
    const int K = in.K, Kp = tc_pad_k(K), n = in.n, m = in.m, h = in.h;
    if (n < 2 || m - h < 1) return cudaErrorInvalidValue;
    // the blocks k = 1 .. n-1 use table levels 1 .. n-1 of each side; the
    // single-entry blocks k = 0 and k = n use level n-1 of one side
    const int64_t lb = in.lowoff[1], hb = in.highoff[1];
    const TcLayout L = tc_layout(m, n, K, in.total, in.lowoff, in.highoff);
    const TcBuffers B = tc_buffers(L, in.ws);
    const int64_t lcnt = L.lcnt, hcnt = L.hcnt;
    __nv_bfloat16* dlow = B.dig[0];
    __nv_bfloat16* dhigh = B.dig[1];
    int* exlow = B.ex[0];
    int* exhigh = B.ex[1];
    double* xt = B.xt;
    double2* const* V = B.V;
    double* const* SV = B.SV;
    __nv_bfloat16* const* DV = B.DV;
    int* const* EXV = B.EXV;
    int64_t* const* efirst = B.efirst;
    int* const* emax = B.emax;
    double* const* esc = B.esc;
    // single-entry blocks: the column vectors of both sides, their digits, and
    // the output data of every level n-1 entry (timed as the split stage)
    stage_begin(kStageSplit, s);
    edge_vectors_kernel<<<(unsigned)(((int64_t)K * m + 255) / 256), 256, 0, s>>>(in.Y, m, h, K, in.lead, V[0], SV[0],
                                                                                    V[1], SV[1]);
    note_launches(1);
    for (int side = 0; side < 2; ++side) {
        const int64_t ww = side == 0 ? h : m - h;
        split_exp_kernel<<<(unsigned)((ww * 32 + 255) / 256), 256, 0, s>>>(V[side], SV[side], ww, ww, K, EXV[side]);
        const int64_t warps = ((ww + 3) / 4) * (Kp / 32);
        split_digits_kernel<<<(unsigned)((warps + 7) / 8), 256, 0, s>>>(V[side], SV[side], ww, ww, K, Kp, EXV[side],
                                                                          DV[side]);
        const int64_t cnt = side == 0 ? in.lowoff[n] - in.lowoff[n - 1] : in.highoff[n] - in.highoff[n - 1];
        edge_info_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(in.mc, m, n, h, side, cnt, efirst[side],
                                                                         emax[side], esc[side]);
        note_launches(3);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    stage_end(kStageSplit, s);
    stage_begin(kStageGemm, s);
    CUtensorMap lr, lc, hr, hc, lc16, hc16, vl16, vh16;
    if ((e = make_digit_map(&vl16, DV[0], h, Kp, kBSub)) != cudaSuccess) return e;
    if ((e = make_digit_map(&vh16, DV[1], m - h, Kp, kBSub)) != cudaSuccess) return e;
    if ((e = make_digit_map(&lr, dlow, lcnt, Kp, TBM)) != cudaSuccess) return e;
    if ((e = make_digit_map(&lc, dlow, lcnt, Kp, TBN)) != cudaSuccess) return e;
    if ((e = make_digit_map(&hr, dhigh, hcnt, Kp, TBM)) != cudaSuccess) return e;
    if ((e = make_digit_map(&hc, dhigh, hcnt, Kp, TBN)) != cudaSuccess) return e;
    if ((e = make_digit_map(&lc16, dlow, lcnt, Kp, kBSub)) != cudaSuccess) return e;
    if ((e = make_digit_map(&hc16, dhigh, hcnt, Kp, kBSub)) != cudaSuccess) return e;
    TcProdArgs a;
    a.nk = 0;
    a.kblocks = Kp / TBK;
    auto round16 = [](int64_t x) { return (int)((x + 15) / 16) * 16; };
    // outputs [lo, hi): per k the ranks of the P whose outputs meet the range
    PRanges pr;
    p_ranges(m, n, h, in.lo, in.hi, &pr);
    int64_t fullcols[kMaxBlocks];                 // columns of each block before any restriction
    for (int k = 1; k < in.n; ++k) {
        const int64_t M = msets_tc(in.h, k), N = msets_tc(in.m - in.h, in.n - k);
        if (M == 0 || N == 0) continue;
        // Rows are the high-side entries Q unless Q has fewer entries than a
        // tile's 128 rows (and P more), which would leave most rows empty.
        // With Q on the rows, the 32 lanes of a drain warp hold consecutive Q
        // of one P, i.e. consecutive canonical outputs, so each store of the
        // drain is one contiguous 256-byte run.
        const bool rl = N < TBM && M > N;
        const int64_t rows = rl ? M : N, cols = rl ? N : M;
        const bool any = pr.pa[k] < pr.pb[k];
        a.rows_low[a.nk] = rl ? 1 : 0;
        a.tn[a.nk] = cols >= TBN ? TBN : round16(cols);
        // the P side (rows when rl, else columns) restricted to [pa, pb)
        a.rows0[a.nk] = rl ? pr.pa[k] : 0;
        a.rows[a.nk] = !any ? a.rows0[a.nk] : (rl ? pr.pb[k] : rows);
        a.cols0[a.nk] = rl ? 0 : pr.pa[k];
        a.cols[a.nk] = !any ? a.cols0[a.nk] : (rl ? cols : pr.pb[k]);
        a.ncol[a.nk] = (int)std::min<int64_t>(a.cols[a.nk], INT32_MAX);
        a.ecol0[a.nk] = (int)std::min<int64_t>(cols, INT32_MAX);
        a.ecols[a.nk] = 0;
        fullcols[a.nk] = cols;
        a.row_off[a.nk] = rl ? in.lowoff[k] - lb : in.highoff[in.n - k] - hb;
        a.col_off[a.nk] = rl ? in.highoff[in.n - k] - hb : in.lowoff[k] - lb;
        a.lowoff[a.nk] = in.lowoff[k];
        a.nk++;
    }
    // the single-entry columns: rows = level n-1 of a side, columns = its
    // modes (side 0: outputs with every photon low, k = n; side 1: k = 0),
    // merged into the block with the same rows when both fit one tile.  The
    // rows that reach [lo, hi): side 0, the parents (level n-1) of the level-n
    // P in range; side 1, the parents of the Q of the block P = {} in range.
    for (int side = 0; side < 2; ++side) {
        const int64_t rows = side == 0 ? in.lowoff[n] - in.lowoff[n - 1] : in.highoff[n] - in.highoff[n - 1];
        const int ecols = side == 0 ? h : m - h;
        if (rows == 0 || ecols == 0) continue;
        int64_t r0 = 0, r1 = 0;
        if (side == 0) {
            if (pr.pa[n] < pr.pb[n]) {
                r0 = host_parent_rank(h, n, pr.pa[n]);
                r1 = host_parent_rank(h, n, pr.pb[n] - 1) + 1;
            }
        } else {
            const int64_t base = host_lowbase(m, n, h, 0, 0);
            const int64_t c = std::max(in.lo, base) - base, d = std::min(in.hi, in.total) - base;
            if (c < d) {
                r0 = host_parent_rank(m - h, n, c);
                r1 = host_parent_rank(m - h, n, d - 1) + 1;
            }
        }
        if (r0 >= r1) continue;
        const int64_t roff = side == 0 ? in.lowoff[n - 1] - lb : in.highoff[n - 1] - hb;
        int host = -1;
        for (int b = 0; b < a.nk; ++b)
            if (a.rows_low[b] == (side == 0 ? 1 : 0) && a.row_off[b] == roff && a.ecols[b] == 0 &&
                round16(fullcols[b]) + round16(ecols) <= TBN)
                host = b;
        if (host >= 0) {
            // one column tile: every column of the host block, then the modes
            a.ecol0[host] = round16(fullcols[host]);
            a.ecols[host] = ecols;
            a.ncol[host] = (int)fullcols[host];
            a.cols0[host] = 0;
            a.cols[host] = a.ecol0[host] + ecols;
            a.tn[host] = a.ecol0[host] + round16(ecols);
            if (a.rows[host] <= a.rows0[host]) {
                a.rows0[host] = r0;
                a.rows[host] = r1;
            } else {
                a.rows0[host] = std::min(a.rows0[host], r0);
                a.rows[host] = std::max(a.rows[host], r1);
            }
            continue;
        }
        a.rows_low[a.nk] = side == 0 ? 1 : 0;
        a.tn[a.nk] = ecols >= TBN ? TBN : round16(ecols);
        a.rows0[a.nk] = r0;
        a.rows[a.nk] = r1;
        a.cols0[a.nk] = 0;
        a.cols[a.nk] = ecols;
        a.ncol[a.nk] = 0;
        a.ecol0[a.nk] = 0;
        a.ecols[a.nk] = ecols;
        fullcols[a.nk] = ecols;
        a.row_off[a.nk] = roff;
        a.col_off[a.nk] = 0;
        a.lowoff[a.nk] = 0;
        a.nk++;
    }
    // blocks without tiles are dropped
    int64_t tiles = 0;
    int nb = 0;
    for (int b = 0; b < a.nk; ++b) {
        const int64_t rt = a.rows[b] > a.rows0[b] ? (a.rows[b] - a.rows0[b] + TBM - 1) / TBM : 0;
        const int64_t ct = a.cols[b] > a.cols0[b] ? (a.cols[b] - a.cols0[b] + a.tn[b] - 1) / a.tn[b] : 0;
        if (rt * ct == 0) continue;
        if (nb != b) {
            a.rows_low[nb] = a.rows_low[b];
            a.tn[nb] = a.tn[b];
            a.rows0[nb] = a.rows0[b];
            a.rows[nb] = a.rows[b];
            a.cols0[nb] = a.cols0[b];
            a.cols[nb] = a.cols[b];
            a.ncol[nb] = a.ncol[b];
            a.ecol0[nb] = a.ecol0[b];
            a.ecols[nb] = a.ecols[b];
            a.row_off[nb] = a.row_off[b];
            a.col_off[nb] = a.col_off[b];
            a.lowoff[nb] = a.lowoff[b];
        }
        a.tile0[nb] = tiles;
        tiles += rt * ct;
        ++nb;
    }
    a.nk = nb;
    a.tile0[a.nk] = tiles;
    if (tiles == 0) {
        stage_end(kStageGemm, s);
        return cudaSuccess;
    }
    if (tiles * 3 * a.kblocks > INT32_MAX || lcnt + TBM > INT32_MAX || hcnt + TBM > INT32_MAX)
        return cudaErrorInvalidConfiguration;
    a.lowbase = in.lowbase;
    a.ex_low = exlow;
    a.ex_high = exhigh;
    a.wlow = lcnt;                            // entries of the digit tensors (exponent stride)
    a.whigh = hcnt;
    a.xt = xt;
    a.lo = in.lo;
    a.hi = in.hi;
    a.amp = in.amp;
    a.prob = in.prob;
    for (int side = 0; side < 2; ++side) {
        a.ex_v[side] = EXV[side];
        a.efirst[side] = efirst[side];
        a.emax[side] = emax[side];
        a.esc[side] = esc[side];
    }
    a.error = in.error;
    a.max_polls = wait_limit(kMaxPolls);
    a.tiles = tiles;
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const unsigned grid = (unsigned)(tiles < (int64_t)sms ? tiles : sms);
    tc_product_kernel<<<grid, kThreads, kSmemBytes, s>>>(lr, lc, hr, hc, lc16, hc16, vl16, vh16, a);
    note_launches(1);
    stage_end(kStageGemm, s);
    return cudaGetLastError();
}

}  // namespace pcv
