// The factorised full distribution with its products on the BF16 tensor
// cores, in exact integer arithmetic: table levels, digit splitting and the
// products of every output block.
//
// With the row sums y_r(d) (glynn_dist.cu), every output is
//     a(S) = sum_d alpha_P(d) beta_Q(d),
// a sum over the K = 2^{n-1} sign vectors of a low-side factor (modes [0, h))
// times a high-side one, so a block of outputs is a complex matrix product,
// done as three real products (Gauss): t1 = Ar Br, t2 = Ai Bi, t3 = (Ar+Ai)
// (Br+Bi), Re a = t1 - t2, Im a = t3 - t1 - t2.  Each real product runs on the
// tensor cores without losing FP64 accuracy, by splitting every operand value
// into integer digits (the error-free splitting idea of Ozaki, Ogita, Oishi
// and Rump, 2012):
//
//   * each operand row gets an exponent E with max_d |x(d)| <= 2^{E-1}; X =
//     round(x 2^{56-E}) is an integer with |X| <= 2^55, written as 8
//     balanced base-128 digits,
//         X = sum_{i=0..7} D_i 128^{7-i},   |D_i| <= 64,
//     so x = 2^E sum_i D_i 2^{-7(i+1)} up to 2^{E-56} (FP64 accuracy).  A
//     table entry's re and im share one exponent one bit higher (54 bits
//     each), and its third operand is the integer X_re + X_im;
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
// Output blocks.  With e = min(3, n / 2) and k the photons on the low side:
//   * k = e+1 .. n-e-1: the low-side table level k times the high-side level
//     n-k (both in lexicographic order);
//   * the outputs with at least n-e photons on one side ("extension blocks"):
//     S = R ++ E, R the n-e photons of that side nearest the other side (for
//     the low side the n-e smallest modes of S, for the high side the n-e
//     largest) and E the other e photons, any modes.  Rows are the table
//     entries R of level n-e of that side, grouped by their seam mode (max R
//     low, min R high); columns are the e-multisets E over all m modes,
//     v_E(d) = prod_{x in E} y_x(d) / sqrt(prod mult!).  A row with seam
//     mode t takes the columns with min E >= t (low side) or max E <= t (high
//     side), which the column orders make a prefix: by min E descending for
//     the low side, by max E ascending for the high side.  When n = 2e the
//     high side leaves out the all-low E (those outputs are the low side's).
//     The output index splits into a row part and a column part, and where
//     E meets R at the seam mode the product carries 1/sqrt(C(mu_R + mu_E,
//     mu_E)) more (multiplicities of that mode in R and E).  The glynn sign
//     and 2^{-(n-1)} norm_t sit on the low-side entries, and on the column
//     vectors the high side's rows take.
// So no table level above n-e is built: for n = 10, levels 8 and 9 of both
// sides (three quarters of all table entries) never exist.
//
// Kernels:
//   tc_level_kernel     table levels, built in FP64 from their parent levels
//                       and written as BF16 digits, laid out [t][digit][entry]
//                       [K] for TMA; levels below n-e also keep their complex
//                       entries as the next level's parents.  The extension
//                       rows and the column vectors are levels too, in their
//                       grouped orders (seam_entries_kernel gives each entry
//                       its parent, mode and output-index part).  One launch
//                       per level number covers both sides and the columns;
//   tc_product_kernel   one persistent CTA per SM walking 128 x N output
//                       tiles of one block each (N = 16..64), eleven warps:
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
//           and stores follow (one non-inlined function per output).  t1 is
//           stored at the output's canonical index in a [2][outputs] buffer;
//           with t2 the same thread turns it into Re a and t1 + t2, and with
//           t3 it forms Im a and |a|^2.  Tiles are oriented so that a warp's
//           32 lanes hold consecutive outputs wherever a block allows it, so
//           its stores coalesce.
// Every mbarrier wait is bounded; on a time-out the kernel records an error
// code and returns after releasing its tensor memory.

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <vector>

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

// ------------------------------------------------------------ extension blocks

// Orders of the extension rows and of the column vectors: the entries of one
// level over the values [0, w), listed group by group, lexicographically
// within a group.
enum SeamOrder {
    kRowsLow = 0,     // low-side rows (level n-e over [0, h)): by largest mode, ascending
    kRowsHigh = 1,    // high-side rows (level n-e over [h, m)): by smallest mode, ascending
    kColsHigh = 2,    // columns of the high-side rows (e-multisets over m): by largest mode, ascending
    kColsLow = 3,     // columns of the low-side rows: by smallest mode, descending
};

// A table entry whose parent, last mode and multiplicity are given (the
// extension rows and the column vectors, whose orders are not lexicographic).
struct EntryInfo {
    long long parent;     // lexicographic rank of the entry without its last mode (in the parent level)
    int r;                // that last mode (global, the row of Ys)
    int mult;             // its multiplicity in the entry
};

// The output-index part and seam data of a row or a column of an extension
// block: the output of row i and column j is base_i + base_j.
struct SeamInfo {
    long long base;
    int key;              // seam mode (global): max R (low rows), min R (high rows), min E, max E
    int mu;               // multiplicity of key in the row or column
};

// Entry i of a grouped order of the k-multisets over [0, w), into
// modes[0..k).  By largest mode g = 0, 1, ...: a (k-1)-multiset over [0, g],
// then g.  By smallest mode g (ascending, or descending from w-1): g, then a
// (k-1)-multiset over [g, w).
__host__ __device__ inline void unrank_grouped(const MultisetTable& mc, bool bymax, bool desc, int w, int k, int64_t i,
                                               int* modes)
{
    for (int j = 0; j < w; ++j) {
        const int g = desc ? w - 1 - j : j;
        const int64_t c = bymax ? mc(g + 1, k - 1) : mc(w - g, k - 1);
        if (i >= c) {
            i -= c;
            continue;
        }
        if (bymax) {
            unrank_multiset<PCV_MAX_PHOTONS>(mc, g + 1, k - 1, i, modes);
            modes[k - 1] = g;
        } else {
            modes[0] = g;
            unrank_multiset<PCV_MAX_PHOTONS>(mc, w - g, k - 1, i, modes + 1);
            for (int p = 1; p < k; ++p) modes[p] += g;
        }
        return;
    }
}

// Seam data from an entry's modes s (global), with idx the canonical index of
// an n-photon output (lexicographic rank of its mode list) and C_a(b) the
// b-multisets over a values:
//   low rows R (n-e modes, t = max R):   base = idx(R ++ t^e) - Phi(t)
//   columns by min E (order kColsLow):   base = rank of E among e-multisets over m
//   high rows R (t = min R):             base = idx(0^e ++ R)
//   columns by max E (u = max E):        base = idx(E ++ u^{n-e}) - Psi(u)
// with Phi(z) = sum_{v<z} C_{m-v}(e-1), Psi(z) = sum_{v<z} C_{m-v}(n-e-1).
// In the rank sum of R ++ E (or E ++ R) only the term of the first position
// after R (after E) depends on both, as Phi(min E) - Phi(t) (Psi(t) -
// Psi(u)); every other term belongs to one of the two.
__host__ __device__ inline SeamInfo seam_of(const MultisetTable& mc, int m, int n, int e, int order, const int* s)
{
    int buf[PCV_MAX_PHOTONS];
    const int L = n - e;
    SeamInfo si;
    int mu = 0;
    if (order == kRowsLow) {
        const int t = s[L - 1];
        for (int p = 0; p < L; ++p) {
            buf[p] = s[p];
            mu += s[p] == t;
        }
        for (int p = L; p < n; ++p) buf[p] = t;
        int64_t phi = 0;
        for (int v = 0; v < t; ++v) phi += mc(m - v, e - 1);
        si.base = rank_multiset(mc, m, n, buf) - phi;
        si.key = t;
    } else if (order == kRowsHigh) {
        const int t = s[0];
        for (int p = 0; p < e; ++p) buf[p] = 0;
        for (int p = 0; p < L; ++p) {
            buf[e + p] = s[p];
            mu += s[p] == t;
        }
        si.base = rank_multiset(mc, m, n, buf);
        si.key = t;
    } else if (order == kColsLow) {
        const int t = s[0];
        for (int p = 0; p < e; ++p) mu += s[p] == t;
        si.base = rank_multiset(mc, m, e, s);
        si.key = t;
    } else {
        const int u = s[e - 1];
        for (int p = 0; p < e; ++p) {
            buf[p] = s[p];
            mu += s[p] == u;
        }
        for (int p = e; p < n; ++p) buf[p] = u;
        int64_t psi = 0;
        for (int v = 0; v < u; ++v) psi += mc(m - v, L - 1);
        si.base = rank_multiset(mc, m, n, buf) - psi;
        si.key = u;
    }
    si.mu = mu;
    return si;
}

// The modes (global) of entry i of an extension-row or column order.
__host__ __device__ inline int seam_modes(const MultisetTable& mc, int m, int n, int e, int h, int order, int64_t i,
                                          int* modes)
{
    const bool rows = order == kRowsLow || order == kRowsHigh;
    const int k = rows ? n - e : e;
    const int w = order == kRowsLow ? h : (order == kRowsHigh ? m - h : m);
    unrank_grouped(mc, order == kRowsLow || order == kColsHigh, order == kColsLow, w, k, i, modes);
    return k;
}

// The four entry lists of the extension blocks (rows of both sides, the
// column vectors in both orders), one launch: list j holds threads
// [start[j], start[j+1]).
struct SeamLists {
    int order[4];
    EntryInfo* info[4];
    SeamInfo* seam[4];
    int64_t start[5];
};

// Per entry of the extension rows or the column vectors: the parent
// (lexicographic rank without the last mode, over the same values), the
// last mode and its multiplicity, and the seam data.
__global__ void seam_entries_kernel(MultisetTable mc, int m, int n, int e, int h, const SeamLists sl)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= sl.start[4]) return;
    int j = 0;
    while (j < 3 && g >= sl.start[j + 1]) ++j;
    const int order = sl.order[j];
    const int64_t i = g - sl.start[j];
    EntryInfo* __restrict__ info = sl.info[j];
    SeamInfo* __restrict__ seam = sl.seam[j];
    int modes[PCV_MAX_PHOTONS];
    const int k = seam_modes(mc, m, n, e, h, order, i, modes);
    const int w = order == kRowsLow ? h : (order == kRowsHigh ? m - h : m);
    const int shift = order == kRowsHigh ? h : 0;
    const int last = modes[k - 1];
    int mult = 0;
    for (int p = 0; p < k; ++p) mult += modes[p] == last;
    EntryInfo ei;
    ei.parent = rank_multiset(mc, w, k - 1, modes);
    ei.r = last + shift;
    ei.mult = mult;
    info[i] = ei;
    for (int p = 0; p < k; ++p) modes[p] += shift;
    seam[i] = seam_of(mc, m, n, e, order, modes);
}

// ------------------------------------------------------------ fused tables

// One level k >= 1 of a factor table, built and split in one pass (the
// tables are never stored in the [sign vector][entry] layout of the FP64
// path): entry(P)(d) = entry(P minus its last mode r)(d) y_r(d) /
// sqrt(multiplicity of r in P), level 0 being sigma(d) 2^{-(n-1)} norm_t on
// the low side (side 0) and 1 elsewhere (high side, column vectors).  Kpad /
// 128 warps per entry P (one for Kpad <= 128), each lane holding 4 sign
// vectors (2 at Kpad = 64; those >= K are zero): the entry's exponent (one for
// re, im and re + im) is a maximum over its warps, so the digits
// [3][8][entry][Kpad] are written in the same pass.  A level that is a parent
// keeps its complex entries, entry-major [entry][K].  Entries are in
// lexicographic order (unranked here; the low side's also get lowbase), or
// take parent, mode and multiplicity from `info` (grouped orders).
struct TcLevelArgs {
    MultisetTable mc;
    int m, n, h, side, k, K, Kpad;
    int w, shift;                        // modes [0, w), at `shift` in the output (lexicographic levels)
    int64_t count;                       // entries of level k
    double lead;                         // 2^{-(n-1)} norm_t
    int sigma_out;                       // 1: entries times sigma(d) 2^{-(n-1)} norm_t (the high side's columns)
    const EntryInfo* info;               // per entry, or null (lexicographic)
    const double2* Ys;                   // [n-1][m][K]: y_r(d) / sqrt(mult), mult = 1 .. n-1
    const double2* parent;               // level k-1, [entry][K] (k >= 2)
    double2* out;                        // level k, [entry][K], or null
    int64_t dig_off, wdig;               // entry offset of level k in the digit tensor; its entries
    __nv_bfloat16* digits;               // [3][8][wdig][Kpad], or null (a parent level only)
    int* ex;                             // [3][wdig]
    int64_t* lowbase;                    // low side: at lowoff_k + entry, else null
    int64_t lowoff_k;
};

// sigma(d) 2^{-(n-1)} norm_t: the sign of sign vector d (Gray-code order)
// times the leading factor
__device__ __forceinline__ double glynn_lead(int q, double lead)
{
    const uint64_t d = (uint64_t)q;
    return (__popcll(d ^ (d >> 1)) & 1) ? -lead : lead;
}

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


// Up to four independent levels in one launch (the same level of both sides
// and of the column vectors, which need only their own parents): job j takes
// the blocks [block0[j], block0[j+1]).
constexpr int kLevelJobs = 4;
struct TcLevelBatch {
    TcLevelArgs job[kLevelJobs];
    int njobs;
    int64_t block0[kLevelJobs + 1];
};

template <int PER, int WPE>
__global__ void __launch_bounds__(128) tc_level_kernel(const __grid_constant__ TcLevelBatch b)
{
    int jb = 0;
    while (jb + 1 < b.njobs && (int64_t)blockIdx.x >= b.block0[jb + 1]) ++jb;
    const TcLevelArgs& a = b.job[jb];
    // WPE warps per entry (4 / WPE entries per block), warp `part` holding
    // sign vectors part 32 PER .. (part + 1) 32 PER - 1
    __shared__ int s_f[4][3];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int part = warp % WPE;
    const int64_t e = ((int64_t)blockIdx.x - b.block0[jb]) * (4 / WPE) + warp / WPE;
    const bool valid = e < a.count;
    const int w = a.w, shift = a.shift;
    int mult = 1, r = 0;
    int64_t parent = 0;
    if (valid && a.info) {
        const EntryInfo ei = a.info[e];
        parent = ei.parent;
        r = ei.r;
        mult = ei.mult;
    } else if (valid) {
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
            if (a.k == 1)
                pv = make_double2(a.side == 0 ? glynn_lead(q, a.lead) : 1.0, 0.0);
            else
                pv = a.parent[parent * a.K + q];
            v[j] = cmul(pv, y);
            if (a.sigma_out) {
                const double sl = glynn_lead(q, a.lead);
                v[j].x *= sl;
                v[j].y *= sl;
            }
            if (a.out) a.out[e * a.K + q] = v[j];
        }
        fc = max(fc, max(exp_field(v[j].x), exp_field(v[j].y)));
    }
    if (!a.digits) return;                                 // the same for the whole grid
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
// ------------------------------------------------------------ products

constexpr int kMaxSideBlocks = 32;                  // extension blocks per side
constexpr int kMaxBlocks = 8 + 2 * kMaxSideBlocks;  // and the level products k = e+1 .. n-e-1 (n <= 10)

struct TcProdArgs {
    int nk;                                   // blocks with tiles
    int kblocks;                              // 64-wide K blocks
    int64_t tile0[kMaxBlocks + 1];            // first tile of each block
    int64_t tiles;                            // all tiles
    // Per block: rows_low 1 if the rows come from the low side's digit tensor
    // (then the columns from the high side's, else the other way round);
    // kind 0 for a level product, 1 for an extension block; tile width
    // (16..64); the rows [rows0, rows) and columns [cols0, cols) its tiles
    // cover; entry offsets of row 0 and column 0 in the digit tensors; lowoff
    // the level offset of a level product's low-side entries (lowbase).  An
    // extension block's rows and columns take their seam data from seam[rs]
    // at ri_off + row and seam[cs] at ci_off + column, and a pair is an
    // output when the column's seam mode is >= the row's (cge = 1) or <= it.
    int rows_low[kMaxBlocks], kind[kMaxBlocks], tn[kMaxBlocks];
    int rs[kMaxBlocks], cs[kMaxBlocks], cge[kMaxBlocks];
    int64_t rows0[kMaxBlocks], rows[kMaxBlocks], cols0[kMaxBlocks], cols[kMaxBlocks];
    int64_t row_off[kMaxBlocks], col_off[kMaxBlocks], lowoff[kMaxBlocks], ri_off[kMaxBlocks], ci_off[kMaxBlocks];
    const int64_t* lowbase;
    const int* ex_low;                        // [3][wlow]
    const int* ex_high;                       // [3][whigh]
    int64_t wlow, whigh;
    // seam data: extension rows of the low (0) and high (1) side, column
    // vectors by max E (2, in the low tensor) and by min E (3, high tensor)
    const SeamInfo* seam[4];
    double* xt;                               // [2][hi - lo]: per output t1, then Re a and t1 + t2
    int64_t lo, hi;                           // outputs [lo, hi) are written, at o - lo
    double2* amp;                             // amplitudes, or null
    double* prob;                             // probabilities, or null
    int* error;                               // set to the role that gave up (1 producer, 2 MMA, 3 drain,
                                              // 4 clean-up), or null
    unsigned long long* next_tile;            // tile counter, zero at launch: CTAs take tiles in order
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

// 1/sqrt(C(a + b, b)): the seam mode's share of 1/sqrt(prod mult!) that
// neither the row (multiplicity a) nor the column (multiplicity b) carries.
__device__ __forceinline__ double seam_scale(int a, int b)
{
    int c = 1;
    for (int i = 1; i <= b; ++i) c = c * (a + i) / i;
    return inv_sqrt_int(c);
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

// The rounding and stores of one output of one product: x_t = RN(Z 2^{sc -
// 49}) (sc = E_row + E_col - 14, kNoExp for an all-zero row or column).  t1
// goes to the workspace at o; with t2 the same thread replaces it by Re a =
// t1 - t2 and stores t1 + t2 beside it, so that with t3 only Im a = t3 - (t1
// + t2) and |a|^2 remain (FP64 is scarce on this part, and the work after
// the third product is the one that holds up the next tile); the amplitude
// takes the seam factor 1/sqrt(C(a + b, b)) when smu = a << 8 | b is set.
// Not inlined: the drain calls it for each of its 32 outputs per product, and
// a single copy keeps the kernel's code, which the MMA and TMA warps share
// the instruction cache with, small (measured at m=20, n=10: products 2.51
// -> 2.28 ms; the split of the combination, 2.27 -> 2.22 ms).
__device__ __noinline__ void drain_output(double* __restrict__ xt, double2* amp, double* prob, int64_t span, int64_t o,
                                         int t, long long zh, uint32_t zl, int sc, int smu)
{
    double x = 0.0;
    if (sc != kNoExp && !scale_packed(zh, zl, sc - 49, x))
        x = fma((double)zl, pow2(sc - 49), (double)zh * pow2(sc - 21));
    if (t == 0) {
        xt[o] = x;
        return;
    }
    if (t == 1) {
        const double t1 = xt[o];
        xt[o] = t1 - x;
        xt[span + o] = t1 + x;
        return;
    }
    double re = xt[o], im = x - xt[span + o];
    if (smu) {
        const double f = seam_scale(smu >> 8, smu & 255);
        re *= f;
        im *= f;
    }
    if (amp) amp[o] = make_double2(re, im);
    if (prob) prob[o] = fma(re, re, im * im);
}

// Row digits in the order 0, 7, 1, 6, 2, 5, 3, 4: digit i is multiplied by
// 8 - i column digits, so alternating long and short products keeps the MMA
// time between consecutive row-digit loads even (the slots then stay about
// equally far ahead of the MMA).  Digit 0 comes first: its products start
// every diagonal.
__device__ __forceinline__ int slice_order(int ii) { return (ii & 1) ? kDigits - 1 - (ii >> 1) : (ii >> 1); }

// A tile's place: block, first row and column, width, and which side the
// rows come from.  Tiles are numbered block by block; within a block the
// tiles along the longer side come slowest (column tiles fastest when the
// block has at least as many rows as columns), so CTAs that run at the same
// time share the operand tile of the longer side, which is read from memory
// once, and cycle through the shorter side's operand, which stays in L2.
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
    const int64_t rtiles = (a.rows[kb] - a.rows0[kb] + TBM - 1) / TBM;
    const int64_t lt = tile - a.tile0[kb];
    const bool cfast = a.cols[kb] - a.cols0[kb] <= a.rows[kb] - a.rows0[kb];
    ti.r0 = a.rows0[kb] + (cfast ? lt / ctiles : lt % rtiles) * TBM;
    ti.c0 = a.cols0[kb] + (cfast ? lt % ctiles : lt / rtiles) * ti.tn;
    ti.rl = a.rows_low[kb] != 0;
    ti.rentry = (int)(a.row_off[kb] + ti.r0);
    ti.centry = (int)(a.col_off[kb] + ti.c0);
    return ti;
}

constexpr int kTileRing = 4;     // tiles a CTA's row producer has taken ahead of the other roles

// The next tile of this CTA from the tile ring (-1: no more tiles, -2: the
// wait gave up); every role takes every tile and hands the slot back once
// (a warp role: its lane 0 waits and reads, and the warp learns the tile by
// a shuffle, so all its lanes leave with the same answer).
__device__ __forceinline__ int64_t take_tile(uint64_t* tfull, uint64_t* tempty, const int64_t* s_tile, uint32_t it,
                                             long long polls, bool warp_role)
{
    const uint32_t slot = it % kTileRing;
    const bool leader = !warp_role || (threadIdx.x & 31) == 0;
    long long tile = -2;
    if (leader && tcx::mbar_wait(&tfull[slot], (it / kTileRing) & 1, polls)) tile = s_tile[slot];
    if (warp_role) tile = __shfl_sync(0xffffffffu, tile, 0);
    if (leader && tile != -2) tcx::mbar_arrive(&tempty[slot]);
    return tile;
}

// Persistent, one CTA per SM, tiles handed out in order by a global counter
// (the row producer takes them, a few ahead, and passes them to the other
// roles through a ring in shared memory), so a CTA that runs fast takes more
// tiles.  The work of a CTA is a sequence of chunks q = (tile, product t,
// 64-wide K block c); the row and column producers run ahead of the MMA by
// their slot rings.
__global__ void __launch_bounds__(kThreads, 1)
tc_product_kernel(const __grid_constant__ CUtensorMap low_rows, const __grid_constant__ CUtensorMap low_cols,
                  const __grid_constant__ CUtensorMap high_rows, const __grid_constant__ CUtensorMap high_cols,
                  const __grid_constant__ CUtensorMap low_cols16, const __grid_constant__ CUtensorMap high_cols16,
                  const TcProdArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* bset = base;                                // kBSets x 64 KB
    unsigned char* aslot = base + kBSets * kBBytes;            // kASlots x 16 KB
    __shared__ __align__(8) uint64_t bfull[kBSets], bempty[kBSets], afull[kASlots], aempty[kASlots];
    __shared__ __align__(8) uint64_t accfull, accempty, mma_done;
    __shared__ __align__(8) uint64_t tfull[kTileRing], tempty[kTileRing];
    __shared__ int64_t s_tile[kTileRing];
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nkb = a.kblocks;

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
        for (int s = 0; s < kTileRing; ++s) {
            mbar_init(&tfull[s], 1);
            mbar_init(&tempty[s], 2 + (kColWarp - 2));    // column producer, MMA, one per drain warp
        }
        s_fail = 0;
        tcx::mbar_fence_init();
        tcx::prefetch_tmap(&low_rows);
        tcx::prefetch_tmap(&low_cols);
        tcx::prefetch_tmap(&high_rows);
        tcx::prefetch_tmap(&high_cols);
        tcx::prefetch_tmap(&low_cols16);
        tcx::prefetch_tmap(&high_cols16);
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
        for (uint32_t it = 0; !s_fail; ++it) {
            // take the next tile and pass it on (-1: none left)
            const uint32_t slot = it % kTileRing;
            if (it >= (uint32_t)kTileRing && !mbar_wait(&tempty[slot], ((it / kTileRing) - 1) & 1, polls)) {
                s_fail = 1;
                break;
            }
            int64_t tile = (int64_t)atomicAdd(a.next_tile, 1ull);
            if (tile >= a.tiles) tile = -1;
            s_tile[slot] = tile;
            mbar_arrive(&tfull[slot]);
            if (tile < 0) break;
            const TileInfo ti = tile_info(a, tile);
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
        for (uint32_t it = 0; !s_fail; ++it) {
            const int64_t tile = take_tile(tfull, tempty, s_tile, it, polls, false);
            if (tile == -2) s_fail = 1;
            if (tile < 0) break;
            const TileInfo tb = tile_info(a, tile);
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
                    if (tb.tn == TBN) {
                        const CUtensorMap* cmap = tb.rl ? &high_cols : &low_cols;
                        for (int j = 0; j < kDigits; ++j)
                            tma_load_4d(dst + j * TBN * kRowBytes, cmap, &bfull[bs], c * TBK, tb.centry, j, t);
                    } else {
                        const CUtensorMap* nmap = tb.rl ? &high_cols16 : &low_cols16;     // 16-row boxes
                        for (int j = 0; j < kDigits; ++j)
                            for (int r = 0; r < tb.tn; r += kBSub)
                                tma_load_4d(dst + (j * tb.tn + r) * kRowBytes, nmap, &bfull[bs], c * TBK,
                                            tb.centry + r, j, t);
                    }
                }
            }
        }
        if (!tcx::wait_issued(bfull, kBSets, q) && !s_fail) s_fail = 4;
    } else if (tid == 32) {
        // ---------------- MMA issuer
        uint32_t na = 0, q = 0, g = 0;                               // slices, chunks, passes
        for (uint32_t it = 0; !s_fail; ++it) {
            const int64_t tile = take_tile(tfull, tempty, s_tile, it, polls, false);
            if (tile == -2) s_fail = 2;
            if (tile < 0) break;
            const int tn = tile_info(a, tile).tn;
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
        for (uint32_t it = 0; alive; ++it) {
            const int64_t tile = take_tile(tfull, tempty, s_tile, it, polls, true);
            if (tile == -2 && lane == 0) s_fail = 3;
            if (tile < 0) break;
            const TileInfo ti = tile_info(a, tile);
            const int kb = ti.kb, tn = ti.tn;
            const bool rl = ti.rl;
            const bool ext = a.kind[kb] != 0;
            const int64_t row = ti.r0 + q4 * 32 + lane;
            const bool rv = row < a.rows[kb];
            const int* ex_r = rl ? a.ex_low : a.ex_high;
            const int* ex_c = rl ? a.ex_high : a.ex_low;
            const int64_t wr = rl ? a.wlow : a.whigh, wc = rl ? a.whigh : a.wlow;
            const int64_t ncol = a.cols[kb];
            // The output of (row, column) is rbase + the column's base: in a
            // level product lowbase(P) + rank of Q, P being the row (rows
            // low, column base = its index) or the column (row base = its
            // index); in an extension block the two seam parts.
            int64_t rbase = row;
            int rkey = 0, rmu = 0;
            const bool cge = a.cge[kb] != 0;
            if (rv && ext) {
                const SeamInfo si = a.seam[a.rs[kb]][a.ri_off[kb] + row];
                rbase = si.base;
                rkey = si.key;
                rmu = si.mu;
            } else if (rv && rl) {
                rbase = a.lowbase[a.lowoff[kb] + row];
            }
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
                int ecl[2], ckl[2];
                int64_t cbl[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int64_t col = ti.c0 + cbase + 32 * h + (lane & 15);
                    ecl[h] = kNoExp;
                    cbl[h] = 0;
                    ckl[h] = 0;
                    if (cbase + 32 * h < tn && col < ncol) {
                        ecl[h] = ex_c[(int64_t)t * wc + a.col_off[kb] + col];
                        if (ext) {
                            const SeamInfo si = a.seam[a.cs[kb]][a.ci_off[kb] + col];
                            cbl[h] = si.base;
                            ckl[h] = si.key | (si.mu << 16);
                        } else {
                            cbl[h] = rl ? col : a.lowbase[a.lowoff[kb] + col];
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
                        const int64_t cb = __shfl_sync(0xffffffffu, cbl[h], q);
                        const int ck = ext ? __shfl_sync(0xffffffffu, ckl[h], q) : 0;
                        const int64_t col = ti.c0 + cc + q;
                        if (!rv || col >= ncol) continue;
                        // an extension pair is an output when its column lies on
                        // the row's side of the seam
                        const int ckey = ck & 0xFFFF;
                        if (ext && (cge ? ckey < rkey : ckey > rkey)) continue;
                        const int64_t og = rbase + cb;
                        if (og < a.lo || og >= a.hi) continue;
                        const int sc = (er != kNoExp && ec != kNoExp) ? er + ec - 14 : kNoExp;
                        const int smu = (ext && ckey == rkey) ? ((rmu << 8) | (ck >> 16)) : 0;
                        drain_output(a.xt, a.amp, a.prob, a.hi - a.lo, og - a.lo, t, zh[h][q], zl[h][q], sc, smu);
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

// The tables of one problem: e = min(3, n / 2) (at least 1), L = n - e.  Per
// side s (w_s modes) a digit tensor holds the lexicographic levels e+1 ..
// n-e-1 (operands of the level products), then the extension rows (level L,
// grouped by seam mode), then the column vectors in the order the other
// side's rows take them (side 0's tensor by max E, for the high-side rows;
// side 1's by min E).  FP64 entries are kept for the parents: levels 1 .. L-1
// of each side and column levels 1 .. e-1 over all m modes.
struct TcShape {
    int m, n, h, e, L, K, Kp;
    int w[2];
    int64_t lev[2][PCV_MAX_PHOTONS + 2];              // digit entry offset of lexicographic level k, or -1
    int64_t rows_off[2], nrows[2];                    // extension rows: digit entry offset, count
    int64_t cols_off[2], ncols;                       // column vectors in each tensor
    int64_t wdig[2];                                  // entries of each digit tensor
    int64_t par[2][PCV_MAX_PHOTONS + 2], npar[2];     // FP64 parents: entry offset of level k
    int64_t cpar[PCV_MAX_PHOTONS + 2], ncpar;         // FP64 column levels
};

TcShape tc_shape(int m, int n, int h, int K)
{
    TcShape S;
    S.m = m;
    S.n = n;
    S.h = h;
    S.K = K;
    S.Kp = tc_pad_k(K);
    S.e = std::max(1, std::min(3, n / 2));
    S.L = n - S.e;
    S.w[0] = h;
    S.w[1] = m - h;
    S.ncols = msets_tc(m, S.e);
    for (int s = 0; s < 2; ++s) {
        int64_t off = 0;
        for (int k = 0; k < PCV_MAX_PHOTONS + 2; ++k) S.lev[s][k] = S.par[s][k] = -1;
        for (int k = S.e + 1; k <= n - S.e - 1; ++k) {
            S.lev[s][k] = off;
            off += msets_tc(S.w[s], k);
        }
        S.rows_off[s] = off;
        S.nrows[s] = msets_tc(S.w[s], S.L);
        S.cols_off[s] = off + S.nrows[s];
        S.wdig[s] = S.cols_off[s] + S.ncols;
        int64_t p = 0;
        for (int k = 1; k < S.L; ++k) {
            S.par[s][k] = p;
            p += msets_tc(S.w[s], k);
        }
        S.npar[s] = p;
    }
    int64_t p = 0;
    for (int k = 0; k < PCV_MAX_PHOTONS + 2; ++k) S.cpar[k] = -1;
    for (int k = 1; k < S.e; ++k) {
        S.cpar[k] = p;
        p += msets_tc(m, k);
    }
    S.ncpar = p;
    return S;
}

// Workspace: per side the digits and exponents, the FP64 parents and the
// entry and seam data of the extension rows and of the column vectors; the
// FP64 column levels, Ys, and two products per output.
struct TcLayout {
    size_t dig[2], ex[2], par[2], rinfo[2], rseam[2], cinfo[2], cseam[2], cpar, ys, xt, total;
};

TcLayout tc_layout(const TcShape& S, int64_t total)
{
    const size_t Kp = (size_t)S.Kp, K = (size_t)S.K;
    TcLayout L;
    L.total = 256;
    for (int s = 0; s < 2; ++s) {
        L.dig[s] = al256((size_t)3 * kDigits * S.wdig[s] * Kp * 2);
        L.ex[s] = al256((size_t)3 * S.wdig[s] * sizeof(int));
        L.par[s] = al256((size_t)S.npar[s] * K * sizeof(double2));
        L.rinfo[s] = al256((size_t)S.nrows[s] * sizeof(EntryInfo));
        L.rseam[s] = al256((size_t)S.nrows[s] * sizeof(SeamInfo));
        L.cinfo[s] = al256((size_t)S.ncols * sizeof(EntryInfo));
        L.cseam[s] = al256((size_t)S.ncols * sizeof(SeamInfo));
        L.total += L.dig[s] + L.ex[s] + L.par[s] + L.rinfo[s] + L.rseam[s] + L.cinfo[s] + L.cseam[s];
    }
    L.cpar = al256((size_t)S.ncpar * K * sizeof(double2));
    L.ys = al256((size_t)(S.n > 1 ? S.n - 1 : 1) * S.m * K * sizeof(double2));
    L.xt = al256((size_t)2 * total * sizeof(double));
    L.total += L.cpar + L.ys + L.xt;
    return L;
}

struct TcBuffers {
    __nv_bfloat16* dig[2];
    int* ex[2];
    double2* par[2];
    EntryInfo* rinfo[2];
    SeamInfo* rseam[2];
    EntryInfo* cinfo[2];
    SeamInfo* cseam[2];
    double2* cpar;
    double2* ys;
    double* xt;
};

TcBuffers tc_buffers(const TcLayout& L, void* ws)
{
    TcBuffers B;
    char* w = (char*)ws;
    for (int s = 0; s < 2; ++s) {
        B.dig[s] = (__nv_bfloat16*)w;   w += L.dig[s];
        B.ex[s] = (int*)w;              w += L.ex[s];
        B.par[s] = (double2*)w;         w += L.par[s];
        B.rinfo[s] = (EntryInfo*)w;     w += L.rinfo[s];
        B.rseam[s] = (SeamInfo*)w;      w += L.rseam[s];
        B.cinfo[s] = (EntryInfo*)w;     w += L.cinfo[s];
        B.cseam[s] = (SeamInfo*)w;      w += L.cseam[s];
    }
    B.cpar = (double2*)w;               w += L.cpar;
    B.ys = (double2*)w;                 w += L.ys;
    B.xt = (double*)w;
    return B;
}

template <int PER, int WPE>
cudaError_t launch_level(TcLevelBatch& b, cudaStream_t s)
{
    int64_t blocks = 0;
    for (int j = 0; j < b.njobs; ++j) {
        b.block0[j] = blocks;
        blocks += (b.job[j].count + (4 / WPE) - 1) / (4 / WPE);
    }
    b.block0[b.njobs] = blocks;
    if (blocks == 0) return cudaSuccess;
    tc_level_kernel<PER, WPE><<<(unsigned)blocks, 128, 0, s>>>(b);
    note_launches(1);
    return cudaGetLastError();
}

// One launch for the jobs in b (all with the same Kpad).
cudaError_t launch_levels(TcLevelBatch& b, cudaStream_t s)
{
    if (b.njobs == 0) return cudaSuccess;
    switch (b.job[0].Kpad / 32) {
        case 2: return launch_level<2, 1>(b, s);     // Kpad = 64
        case 4: return launch_level<4, 1>(b, s);     // 128
        case 8: return launch_level<4, 2>(b, s);     // 256
        default: return launch_level<4, 4>(b, s);    // 512
    }
}

// The multiset counts on the host, in the device table's layout.
struct HostCounts {
    std::vector<int64_t> t;
    MultisetTable mc;
    HostCounts(int m, int n) : t((size_t)(m + 1) * (n + 1))
    {
        for (int a = 0; a <= m; ++a)
            for (int k = 0; k <= n; ++k) t[(size_t)a * (n + 1) + k] = msets_tc(a, k);
        mc.t = t.data();
        mc.kmax = n;
    }
};

}  // namespace

int64_t tc_workspace(int m, int n, int h, int K, int64_t total)
{
    return (int64_t)tc_layout(tc_shape(m, n, h, K), total).total;
}

cudaError_t launch_tc_tables(const TcInputs& in, cudaStream_t s)
{
    const int K = in.K, n = in.n;
    const TcShape S = tc_shape(in.m, n, in.h, K);
    if (n < 2 || S.Kp > 512) return cudaErrorInvalidValue;
    const TcLayout L = tc_layout(S, in.total);
    const TcBuffers B = tc_buffers(L, in.ws);
    const int64_t nys = (int64_t)(n - 1) * in.m * K;
    scaled_rowsums_kernel<<<(unsigned)((nys + 255) / 256), 256, 0, s>>>(in.Y, in.m, K, n - 1, B.ys);
    note_launches(1);
    auto level_args = [&](int side, int k, int w, int shift) {
        TcLevelArgs la;
        la.mc = in.mc;
        la.m = in.m; la.n = n; la.h = in.h; la.side = side; la.k = k; la.K = K; la.Kpad = S.Kp;
        la.w = w; la.shift = shift;
        la.count = 0;
        la.lead = in.lead;
        la.sigma_out = 0;
        la.info = nullptr;
        la.Ys = B.ys;
        la.parent = nullptr;
        la.out = nullptr;
        la.dig_off = 0; la.wdig = 0;
        la.digits = nullptr;
        la.ex = nullptr;
        la.lowbase = nullptr;
        la.lowoff_k = 0;
        return la;
    };
    cudaError_t e;
    // the entry lists of the extension blocks (they need only the multiset
    // counts): rows of both sides, column vectors by max E (side 0's tensor)
    // and by min E (side 1's)
    {
        SeamLists sl;
        const int orders[4] = {kRowsLow, kRowsHigh, kColsHigh, kColsLow};
        const int64_t counts[4] = {S.nrows[0], S.nrows[1], S.ncols, S.ncols};
        EntryInfo* infos[4] = {B.rinfo[0], B.rinfo[1], B.cinfo[0], B.cinfo[1]};
        SeamInfo* seams[4] = {B.rseam[0], B.rseam[1], B.cseam[0], B.cseam[1]};
        sl.start[0] = 0;
        for (int j = 0; j < 4; ++j) {
            sl.order[j] = orders[j];
            sl.info[j] = infos[j];
            sl.seam[j] = seams[j];
            sl.start[j + 1] = sl.start[j] + counts[j];
        }
        seam_entries_kernel<<<(unsigned)((sl.start[4] + 127) / 128), 128, 0, s>>>(in.mc, in.m, n, S.e, in.h, sl);
        note_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // lexicographic levels k = 1 .. L-1 of both sides (parents, with digits
    // where a level product takes them) and, for k < e, of the column vectors
    for (int k = 1; k < S.L; ++k) {
        TcLevelBatch b;
        b.njobs = 0;
        for (int side = 0; side < 2; ++side) {
            const int w = S.w[side];
            TcLevelArgs la = level_args(side, k, w, side == 0 ? 0 : in.h);
            la.count = msets_tc(w, k);
            la.parent = k >= 2 ? B.par[side] + S.par[side][k - 1] * K : nullptr;
            la.out = B.par[side] + S.par[side][k] * K;
            if (S.lev[side][k] >= 0) {
                la.digits = B.dig[side];
                la.ex = B.ex[side];
                la.dig_off = S.lev[side][k];
                la.wdig = S.wdig[side];
            }
            if (side == 0) {
                la.lowbase = in.lowbase;
                la.lowoff_k = in.lowoff[k];
            }
            b.job[b.njobs++] = la;
        }
        if (k < S.e) {
            TcLevelArgs la = level_args(2, k, in.m, 0);
            la.count = msets_tc(in.m, k);
            la.parent = k >= 2 ? B.cpar + S.cpar[k - 1] * K : nullptr;
            la.out = B.cpar + S.cpar[k] * K;
            b.job[b.njobs++] = la;
        }
        if ((e = launch_levels(b, s)) != cudaSuccess) return e;
    }
    // the extension rows (level L of each side, grouped by seam mode) and
    // the column vectors (level e over all modes) in both orders.  The glynn
    // sign and leading factor, on the low side from level 0 on, go to the
    // high side's products through their columns (side 0's tensor).
    TcLevelBatch b;
    b.njobs = 0;
    for (int side = 0; side < 2; ++side) {
        TcLevelArgs la = level_args(side, S.L, S.w[side], side == 0 ? 0 : in.h);
        la.count = S.nrows[side];
        la.info = B.rinfo[side];
        la.parent = S.L >= 2 ? B.par[side] + S.par[side][S.L - 1] * K : nullptr;
        la.digits = B.dig[side];
        la.ex = B.ex[side];
        la.dig_off = S.rows_off[side];
        la.wdig = S.wdig[side];
        b.job[b.njobs++] = la;
    }
    for (int side = 0; side < 2; ++side) {
        TcLevelArgs la = level_args(2, S.e, in.m, 0);
        la.count = S.ncols;
        la.info = B.cinfo[side];
        la.parent = S.e >= 2 ? B.cpar + S.cpar[S.e - 1] * K : nullptr;
        la.sigma_out = side == 0;
        la.digits = B.dig[side];
        la.ex = B.ex[side];
        la.dig_off = S.cols_off[side];
        la.wdig = S.wdig[side];
        b.job[b.njobs++] = la;
    }
    return launch_levels(b, s);
}

namespace {

// The output blocks of one call, the outputs [lo, hi) of `total`: a's
// per-block fields, nk, tile0 and tiles (host only; lowoff: offset of each
// low-side level in lowbase).
cudaError_t plan_tc_blocks(const TcShape& S, int64_t total, const int64_t* lowoff, int64_t lo, int64_t hi,
                           TcProdArgs& a)
{
    const int m = S.m, n = S.n, h = S.h;
    a.nk = 0;
    a.kblocks = S.Kp / TBK;
    auto width = [](int64_t cols) { return cols >= TBN ? TBN : (int)((cols + 15) / 16) * 16; };
    // outputs [lo, hi): per k the ranks of the P whose outputs meet the range
    PRanges pr;
    p_ranges(m, n, h, lo, hi, &pr);
    // level products k = e+1 .. n-e-1
    for (int k = S.e + 1; k <= n - S.e - 1; ++k) {
        const int64_t M = msets_tc(h, k), N = msets_tc(m - h, n - k);
        if (M == 0 || N == 0) continue;
        // Rows are the high-side entries Q unless Q has fewer entries than a
        // tile's 128 rows (and P more), which would leave most rows empty.
        // With Q on the rows, the 32 lanes of a drain warp hold consecutive Q
        // of one P, i.e. consecutive canonical outputs, so each store of the
        // drain is one contiguous 256-byte run.
        const bool rl = N < TBM && M > N;
        const int64_t rows = rl ? M : N, cols = rl ? N : M;
        const bool any = pr.pa[k] < pr.pb[k];
        const int b = a.nk++;
        a.rows_low[b] = rl ? 1 : 0;
        a.kind[b] = 0;
        a.tn[b] = width(cols);
        // the P side (rows when rl, else columns) restricted to [pa, pb)
        a.rows0[b] = rl ? pr.pa[k] : 0;
        a.rows[b] = !any ? a.rows0[b] : (rl ? pr.pb[k] : rows);
        a.cols0[b] = rl ? 0 : pr.pa[k];
        a.cols[b] = !any ? a.cols0[b] : (rl ? cols : pr.pb[k]);
        a.row_off[b] = rl ? S.lev[0][k] : S.lev[1][n - k];
        a.col_off[b] = rl ? S.lev[1][n - k] : S.lev[0][k];
        a.lowoff[b] = lowoff[k];
        a.rs[b] = a.cs[b] = a.cge[b] = 0;
        a.ri_off[b] = a.ci_off[b] = 0;
    }
    // Extension blocks, per side: runs of seam groups (consecutive groups
    // merged until a run holds at least `thr` extension entries; a run takes
    // the vectors E of its widest group, and each pair checks its own seam).
    // High side: the entries are the tile rows and the vectors E the columns.
    // Low side the other way round, so that there too the 32 lanes of a drain
    // warp hold consecutive outputs (consecutive E) and its stores coalesce.
    // For a part [lo, hi) of the outputs the entries and vectors are cut to
    // those with an output in range (seam data on the host: a group's
    // entries have increasing bases, so each vector's entries in range are
    // found by bisection).
    const bool whole = lo <= 0 && hi >= total;
    std::vector<SeamInfo> hrow, hcol;
    HostCounts hc_tab(whole ? 0 : m, whole ? 0 : n);
    for (int side = 0; side < 2; ++side) {
        const int w = S.w[side];
        auto gsize = [&](int g) { return side == 0 ? msets_tc(g + 1, S.L - 1) : msets_tc(w - g, S.L - 1); };
        auto gcols = [&](int g) { return side == 0 ? msets_tc(m - g, S.e) : msets_tc(g + h + 1, S.e); };
        if (!whole) {
            int modes[PCV_MAX_PHOTONS];
            const int order = side == 0 ? kRowsLow : kRowsHigh;
            const int corder = side == 0 ? kColsLow : kColsHigh;     // the vectors this side's entries take
            hrow.resize((size_t)S.nrows[side]);
            for (int64_t i = 0; i < S.nrows[side]; ++i) {
                const int k = seam_modes(hc_tab.mc, m, n, S.e, h, order, i, modes);
                if (side == 1)
                    for (int p = 0; p < k; ++p) modes[p] += h;
                hrow[(size_t)i] = seam_of(hc_tab.mc, m, n, S.e, order, modes);
            }
            hcol.resize((size_t)S.ncols);
            for (int64_t i = 0; i < S.ncols; ++i) {
                seam_modes(hc_tab.mc, m, n, S.e, h, corder, i, modes);
                hcol[(size_t)i] = seam_of(hc_tab.mc, m, n, S.e, corder, modes);
            }
        }
        const int64_t c0 = (side == 1 && n == 2 * S.e) ? msets_tc(h, S.e) : 0;   // all-low E: the low side's
        // The runs of groups: fewest tiles over at most kMaxSideBlocks runs
        // (f[i][j]: groups i.. in j runs; a run's tiles follow from its
        // entries and its widest group's vectors, in this side's orientation).
        auto run_tiles = [&](int64_t entries, int64_t vectors) {
            const int64_t rows = side == 0 ? vectors : entries, cols = side == 0 ? entries : vectors;
            const int64_t tn = width(cols);
            return ((rows + TBM - 1) / TBM) * ((cols + tn - 1) / tn);
        };
        const int64_t kInf = INT64_MAX / 4;
        const int J = kMaxSideBlocks;
        std::vector<int64_t> f((size_t)(w + 1) * (J + 1), kInf);
        std::vector<int> cut((size_t)(w + 1) * (J + 1), -1);
        f[(size_t)w * (J + 1)] = 0;
        for (int i = w - 1; i >= 0; --i) {
            int64_t ent = 0, vec = 0;
            for (int b = i; b < w; ++b) {
                ent += gsize(b);
                vec = std::max(vec, gcols(b));
                const int64_t t = run_tiles(ent, vec - c0);
                for (int j = 1; j <= J; ++j) {
                    const int64_t rest = f[(size_t)(b + 1) * (J + 1) + j - 1];
                    if (rest < kInf && t + rest < f[(size_t)i * (J + 1) + j]) {
                        f[(size_t)i * (J + 1) + j] = t + rest;
                        cut[(size_t)i * (J + 1) + j] = b;
                    }
                }
            }
        }
        int jbest = 1;
        for (int j = 1; j <= J; ++j)
            if (f[(size_t)j] < f[(size_t)jbest]) jbest = j;
        std::vector<int> run_end;                                    // last group of each run
        for (int i = 0, j = jbest; i < w; --j) {
            const int b = cut[(size_t)i * (J + 1) + j];
            run_end.push_back(b);
            i = b + 1;
        }
        int64_t rb = 0, r = 0, cend = 0;
        int g0 = 0;
        size_t ri = 0;
        for (int g = 0; g < w; ++g) {
            r += gsize(g);
            cend = std::max(cend, gcols(g));
            if (g != run_end[ri]) continue;
            ++ri;
            // entries [ea, ez) (from rb) and vectors [va, vz) of the block
            int64_t ea = 0, ez = r - rb, va = c0, vz = cend;
            if (!whole) {
                int64_t ra = INT64_MAX, rz = -1, ca = INT64_MAX, cz = -1;
                int64_t gb = rb;
                for (int gg = g0; gg <= g; ++gg) {
                    const int64_t gs = gsize(gg), nc = gcols(gg);
                    for (int64_t c = c0; c < nc && gs > 0; ++c) {
                        const int64_t cb = hcol[(size_t)c].base;
                        auto first_at_least = [&](int64_t v) {     // first entry of the group with base >= v
                            int64_t x = gb, y = gb + gs;
                            while (x < y) {
                                const int64_t mid = (x + y) / 2;
                                if (hrow[(size_t)mid].base < v) x = mid + 1; else y = mid;
                            }
                            return x;
                        };
                        const int64_t x0 = first_at_least(lo - cb), x1 = first_at_least(hi - cb);
                        if (x0 >= x1) continue;
                        ra = std::min(ra, x0);
                        rz = std::max(rz, x1);
                        ca = std::min(ca, c);
                        cz = std::max(cz, c);
                    }
                    gb += gs;
                }
                if (rz < 0) {
                    ez = ea;
                } else {
                    ea = ra - rb;
                    ez = rz - rb;
                    va = ca;
                    vz = cz + 1;
                }
            }
            if (a.nk >= kMaxBlocks) return cudaErrorInvalidConfiguration;
            const int b = a.nk++;
            a.kind[b] = 1;
            a.lowoff[b] = 0;
            a.rows_low[b] = 0;
            // a pair is an output when max E <= min R (high side; rows R,
            // columns E) or max R <= min E (low side; rows E, columns R)
            a.cge[b] = 0;
            if (side == 1) {
                a.rows0[b] = ea;
                a.rows[b] = ez;
                a.cols0[b] = va;
                a.cols[b] = vz;
                a.row_off[b] = S.rows_off[1] + rb;
                a.col_off[b] = S.cols_off[0];
                a.rs[b] = 1;
                a.ri_off[b] = rb;
                a.cs[b] = 2;
                a.ci_off[b] = 0;
            } else {
                a.rows0[b] = va;
                a.rows[b] = vz;
                a.cols0[b] = ea;
                a.cols[b] = ez;
                a.row_off[b] = S.cols_off[1];
                a.col_off[b] = S.rows_off[0] + rb;
                a.rs[b] = 3;
                a.ri_off[b] = 0;
                a.cs[b] = 0;
                a.ci_off[b] = rb;
            }
            a.tn[b] = width(a.cols[b] - a.cols0[b]);
            rb = r;
            cend = 0;
            g0 = g + 1;
        }
    }
    // A block whose last row tile holds at most 64 rows gives those rows to
    // a block of the other orientation (its columns as rows, the leftover
    // rows as one narrow column tile) when that takes fewer tiles: the
    // leftover rows of a 286-vector group, say, take 79 tiles as a row tile
    // and 40 as a column tile.  Whole distributions only; a part keeps its
    // blocks as they are (the results are the same either way).
    if (whole) {
        const int nb0 = a.nk;
        for (int b = 0; b < nb0 && a.nk < kMaxBlocks; ++b) {
            const int64_t rows = a.rows[b] - a.rows0[b], cols = a.cols[b] - a.cols0[b];
            const int64_t tail = rows % TBM;
            if (rows < TBM || tail == 0 || tail > TBN || cols <= 0) continue;
            const int64_t now = (cols + a.tn[b] - 1) / a.tn[b];          // tiles of the last row tile
            if ((cols + TBM - 1) / TBM >= now) continue;
            const int t = a.nk++;
            a.kind[t] = a.kind[b];
            a.rows_low[t] = a.rows_low[b] ? 0 : 1;
            a.rows0[t] = a.cols0[b];
            a.rows[t] = a.cols[b];
            a.cols0[t] = a.rows[b] - tail;
            a.cols[t] = a.rows[b];
            a.tn[t] = width(tail);
            a.row_off[t] = a.col_off[b];
            a.col_off[t] = a.row_off[b];
            a.lowoff[t] = a.lowoff[b];
            a.rs[t] = a.cs[b];
            a.cs[t] = a.rs[b];
            a.ri_off[t] = a.ci_off[b];
            a.ci_off[t] = a.ri_off[b];
            a.cge[t] = a.cge[b] ? 0 : 1;
            a.rows[b] -= tail;
        }
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
            a.kind[nb] = a.kind[b];
            a.tn[nb] = a.tn[b];
            a.rows0[nb] = a.rows0[b];
            a.rows[nb] = a.rows[b];
            a.cols0[nb] = a.cols0[b];
            a.cols[nb] = a.cols[b];
            a.row_off[nb] = a.row_off[b];
            a.col_off[nb] = a.col_off[b];
            a.lowoff[nb] = a.lowoff[b];
            a.rs[nb] = a.rs[b];
            a.cs[nb] = a.cs[b];
            a.cge[nb] = a.cge[b];
            a.ri_off[nb] = a.ri_off[b];
            a.ci_off[nb] = a.ci_off[b];
        }
        a.tile0[nb] = tiles;
        tiles += rt * ct;
        ++nb;
    }
    a.nk = nb;
    a.tile0[a.nk] = tiles;
    a.tiles = tiles;
    return cudaSuccess;
}

}  // namespace

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
    const int K = in.K, n = in.n, m = in.m, h = in.h;
    if (n < 2 || m - h < 1) return cudaErrorInvalidValue;
    const TcShape S = tc_shape(m, n, h, K);
    const TcLayout L = tc_layout(S, in.total);
    const TcBuffers B = tc_buffers(L, in.ws);
    if (S.wdig[0] + TBM > INT32_MAX || S.wdig[1] + TBM > INT32_MAX) return cudaErrorInvalidConfiguration;
    stage_begin(kStageGemm, s);
    CUtensorMap lr, lc, hr, hc, lc16, hc16;
    if ((e = make_digit_map(&lr, B.dig[0], S.wdig[0], S.Kp, TBM)) != cudaSuccess) return e;
    if ((e = make_digit_map(&lc, B.dig[0], S.wdig[0], S.Kp, TBN)) != cudaSuccess) return e;
    if ((e = make_digit_map(&hr, B.dig[1], S.wdig[1], S.Kp, TBM)) != cudaSuccess) return e;
    if ((e = make_digit_map(&hc, B.dig[1], S.wdig[1], S.Kp, TBN)) != cudaSuccess) return e;
    if ((e = make_digit_map(&lc16, B.dig[0], S.wdig[0], S.Kp, kBSub)) != cudaSuccess) return e;
    if ((e = make_digit_map(&hc16, B.dig[1], S.wdig[1], S.Kp, kBSub)) != cudaSuccess) return e;
    TcProdArgs a;
    if ((e = plan_tc_blocks(S, in.total, in.lowoff, in.lo, in.hi, a)) != cudaSuccess) return e;
    const int64_t tiles = a.tiles;
    if (tiles == 0) {
        stage_end(kStageGemm, s);
        return cudaSuccess;
    }
    if (tiles * 3 * a.kblocks > INT32_MAX) return cudaErrorInvalidConfiguration;
    a.lowbase = in.lowbase;
    a.ex_low = B.ex[0];
    a.ex_high = B.ex[1];
    a.wlow = S.wdig[0];                       // entries of the digit tensors (exponent stride)
    a.whigh = S.wdig[1];
    a.seam[0] = B.rseam[0];
    a.seam[1] = B.rseam[1];
    a.seam[2] = B.cseam[0];
    a.seam[3] = B.cseam[1];
    a.xt = B.xt;
    a.lo = in.lo;
    a.hi = in.hi;
    a.amp = in.amp;
    a.prob = in.prob;
    a.error = in.error;
    a.next_tile = in.next_tile;
    a.max_polls = wait_limit(kMaxPolls);
    a.tiles = tiles;
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const unsigned grid = (unsigned)(tiles < (int64_t)sms ? tiles : sms);
    tc_product_kernel<<<grid, kThreads, kSmemBytes, s>>>(lr, lc, hr, hc, lc16, hc16, a);
    note_launches(1);
    stage_end(kStageGemm, s);
    return cudaGetLastError();
}

// The products' output blocks for m modes, n photons and the outputs [lo,
// hi), written to out (host only): kTcPlanHeader values describing the digit
// tensors, then kTcPlanBlock values per block.  Returns the values needed (out
// is written only when cap holds them), or -1 if the plan fails.
int64_t tc_block_list(int m, int n, int64_t lo, int64_t hi, int64_t* out, int64_t cap)
{
    const int h = std::max(1, m / 2);
    int64_t lowoff[PCV_MAX_PHOTONS + 2];
    int64_t acc = 0;
    for (int k = 0; k < PCV_MAX_PHOTONS + 2; ++k) {
        lowoff[k] = acc;
        if (k <= n) acc += msets_tc(h, k);
    }
    const TcShape S = tc_shape(m, n, h, 1 << (n - 1));
    TcProdArgs a;
    if (plan_tc_blocks(S, msets_tc(m, n), lowoff, lo, hi, a) != cudaSuccess) return -1;
    const int64_t need = kTcPlanHeader + (int64_t)a.nk * kTcPlanBlock;
    if (!out || cap < need) return need;
    for (int64_t i = 0; i < kTcPlanHeader; ++i) out[i] = -1;
    out[0] = S.e;
    out[1] = S.L;
    out[2] = h;
    out[3] = a.nk;
    out[4] = a.tiles;
    out[5] = S.ncols;
    for (int sd = 0; sd < 2; ++sd) {
        out[6 + sd] = S.rows_off[sd];
        out[8 + sd] = S.nrows[sd];
        out[10 + sd] = S.cols_off[sd];
        out[12 + sd] = S.wdig[sd];
        for (int k = 0; k <= n && k <= 15; ++k) out[16 + 16 * sd + k] = S.lev[sd][k];
    }
    for (int b = 0; b < a.nk; ++b) {
        int64_t* o = out + kTcPlanHeader + (int64_t)b * kTcPlanBlock;
        const int64_t v[kTcPlanBlock] = {a.kind[b], a.rows_low[b], a.tn[b], a.rows0[b], a.rows[b], a.cols0[b],
                                         a.cols[b], a.row_off[b], a.col_off[b], a.lowoff[b], a.rs[b], a.cs[b],
                                         a.cge[b], a.ri_off[b], a.ci_off[b], a.tile0[b]};
        for (int i = 0; i < kTcPlanBlock; ++i) o[i] = v[i];
    }
    return need;
}

}  // namespace pcv
