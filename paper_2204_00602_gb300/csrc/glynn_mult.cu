// Glynn's sum with multiplicities, for outputs (or inputs) that put several
// photons in one mode.
//
// Such a state repeats a row (column) of U in the n x n matrix of Eq. eqperm.
// In Glynn's sum the mu_j copies of a repeated line only enter through k_j,
// the number of minus signs among them: C(mu_j, k_j) sign vectors share the
// same value, their sign product is (-1)^{k_j} and the copies add up to
// (mu_j - 2 k_j) times the line.  With the sign vectors on one side (its
// distinct modes j = 0..d-1, multiplicities mu_j) and the product over the
// other side (distinct modes i, multiplicities e_i),
//
//     Perm = 2^{-n} sum_{k_j = 0..mu_j} prod_j (-1)^{k_j} C(mu_j, k_j)
//                   prod_i ( sum_j (mu_j - 2 k_j) M[j][i] )^{e_i},
//
// prod_j (mu_j + 1) terms instead of 2^{n-1}.  The map k -> mu - k leaves a
// term unchanged (every line sum changes sign, as does the sign product when
// n is odd), so one digit, the pivot p, runs over k_p <= floor(mu_p / 2) with
// weight 2 below the middle; an odd mu_p halves the count.  The terms are
// visited in reflected mixed-radix Gray order: consecutive terms differ in one
// k_j by +-1, so the line sums move by -+2 M[j][.] (2 DFMA per other-side
// mode), the sign alternates, and the integer weight (below 2^31 for n <= 30)
// is updated exactly with one division and one multiplication on the integer
// pipe.
//
// Orientation: Perm(A) = Perm(A^T), so either side may carry the sign
// vectors; each permanent takes the side with fewer terms.  One warp per
// permanent (lanes split the term sequence), or `parts` warps per permanent
// whose partial sums are added in a fixed order.  The batched launch routes
// each output either here or to the shared-row-sum tile kernel by an FP64
// instruction-count model (glynn_tile.cu).

#include "pcv_common.cuh"

namespace pcv {
namespace {

constexpr int kMultWarps = 8;
constexpr int kMultThreads = 32 * kMultWarps;
constexpr int kBinW = PCV_MAX_PHOTONS + 1;
constexpr unsigned kFull = 0xffffffffu;

// One permanent as the warp sees it, in shared memory.
struct MultWarp {
    uint64_t T;                       // terms of the restricted sum
    double scale;                     // 2^{-n} / sqrt(prod s! prod t!)
    int d, q, piv;                    // distinct modes on the sign side / product side; pivot digit
    int moff[PCV_MAX_PHOTONS];        // element offset in U of sign-side mode j (row r*m or column c)
    int ooff[PCV_MAX_PHOTONS];        // element offset in U of product-side mode i
    uint8_t mu[PCV_MAX_PHOTONS];      // sign-side multiplicities
    uint8_t R[PCV_MAX_PHOTONS];       // radices: mu_j + 1, floor(mu_p / 2) + 1 for the pivot
    uint8_t e[PCV_MAX_PHOTONS];       // product-side multiplicities
    int omode[PCV_MAX_PHOTONS];       // decode scratch: occupied output modes
    uint8_t omu[PCV_MAX_PHOTONS];     //                 and their photon counts
};

struct MultShared {
    uint32_t binom[kBinW * kBinW];                   // C(a, k), a, k <= 30
    MultWarp w[kMultWarps];
    uint8_t digit[kMultWarps][PCV_MAX_PHOTONS][32];  // per lane: current k_j
};

__device__ void init_binom(uint32_t* binom)
{
    for (int a = threadIdx.x; a < kBinW; a += blockDim.x) {
        uint64_t c = 1;
        for (int k = 0; k < kBinW; ++k) {
            binom[a * kBinW + k] = (uint32_t)c;       // C(a, k); 0 once k > a
            c = c * (uint64_t)(a - k) / (uint64_t)(k + 1);
        }
    }
    __syncthreads();
}

// Terms of a side with multiplicities mu[0..d) and its pivot: an odd
// multiplicity if there is one (halves the count), else the largest.
__device__ __forceinline__ uint64_t side_terms(const uint8_t* mu, int d, int& piv)
{
    uint64_t t = 1;
    int odd = -1, big = 0;
    for (int j = 0; j < d; ++j) {
        t *= (uint64_t)mu[j] + 1;
        if (odd < 0 && (mu[j] & 1)) odd = j;
        if (mu[j] > mu[big]) big = j;
    }
    piv = odd >= 0 ? odd : big;
    return t / ((uint64_t)mu[piv] + 1) * ((uint64_t)mu[piv] / 2 + 1);
}

__device__ __forceinline__ uint32_t weight(const uint32_t* binom, uint32_t mu, uint32_t k, bool pivot)
{
    return binom[mu * kBinW + k] << ((pivot && 2 * k < mu) ? 1 : 0);
}

// Fills w for output `occ` of circuit c; side 0 = the side with fewer terms,
// 1 = signs on the output modes, 2 = signs on the input modes.  Returns false
// (and sets scale = 0) when the output does not hold exactly n photons.
__device__ bool mult_decode(const pcv_batch_desc& c, const uint8_t* occ, int side, MultWarp& w, int lane)
{
    const int m = c.m, n = c.n;
    int d_out = 0, tot = 0;
    for (int base = 0; base < m; base += 32) {
        const int r = base + lane;
        const int v = r < m ? occ[r] : 0;
        const unsigned mask = __ballot_sync(kFull, v > 0);
        const int pos = d_out + __popc(mask & ((1u << lane) - 1u));
        if (v > 0 && pos < PCV_MAX_PHOTONS) {
            w.omode[pos] = r;
            w.omu[pos] = (uint8_t)v;
        }
        d_out += __popc(mask);
        int s = v;
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(kFull, s, off);
        tot += s;
    }
    const bool ok = tot == n && d_out <= PCV_MAX_PHOTONS;
    __syncwarp();
    if (lane == 0) {
        if (!ok) {
            w.T = 0;
            w.scale = 0.0;
        } else {
            // input side: runs of the sorted photon -> input-mode list
            int imode[PCV_MAX_PHOTONS];
            uint8_t imu[PCV_MAX_PHOTONS];
            int d_in = 0;
            double f = 1.0;
            for (int j = 0; j < n; ++j) {
                if (j == 0 || c.cols[j] != c.cols[j - 1]) {
                    imode[d_in] = c.cols[j];
                    imu[d_in] = 0;
                    ++d_in;
                }
                imu[d_in - 1] += 1;
                f *= imu[d_in - 1];
            }
            for (int j = 0; j < d_out; ++j)
                for (int k = 2; k <= w.omu[j]; ++k) f *= k;
            int piv_out = 0, piv_in = 0;
            const uint64_t t_out = side_terms(w.omu, d_out, piv_out);
            const uint64_t t_in = side_terms(imu, d_in, piv_in);
            const bool use_in = side == 2 || (side == 0 && t_in < t_out);
            if (!use_in) {
                w.d = d_out;
                w.q = d_in;
                w.piv = piv_out;
                w.T = t_out;
                for (int j = 0; j < d_out; ++j) {
                    w.moff[j] = w.omode[j] * m;
                    w.mu[j] = w.omu[j];
                }
                for (int i = 0; i < d_in; ++i) {
                    w.ooff[i] = imode[i];
                    w.e[i] = imu[i];
                }
            } else {
                w.d = d_in;
                w.q = d_out;
                w.piv = piv_in;
                w.T = t_in;
                for (int j = 0; j < d_in; ++j) {
                    w.moff[j] = imode[j];
                    w.mu[j] = imu[j];
                }
                for (int i = 0; i < d_out; ++i) {
                    w.ooff[i] = w.omode[i] * m;
                    w.e[i] = w.omu[i];
                }
            }
            for (int j = 0; j < w.d; ++j) w.R[j] = (uint8_t)(j == w.piv ? w.mu[j] / 2 + 1 : w.mu[j] + 1);
            w.scale = ldexp(1.0 / sqrt(f), -n);
        }
    }
    __syncwarp();
    return ok;
}

// Sum of terms [g0, g1) of the restricted Gray sequence (unscaled).
template <int QMAX>
__device__ double2 mult_range(const double2* __restrict__ U, const MultWarp& w, const uint32_t* binom,
                              uint8_t (*dig)[32], uint64_t g0, uint64_t g1, int lane)
{
    double2 acc = make_double2(0.0, 0.0);
    if (g0 >= g1) return acc;
    const int d = w.d, q = w.q, piv = w.piv;
    double2 x[QMAX];
    int oo[QMAX];                               // product-side offsets, kept in registers
    bool ones = true;                           // every product-side multiplicity is 1
#pragma unroll
    for (int i = 0; i < QMAX; ++i) {
        x[i] = make_double2(0.0, 0.0);
        oo[i] = i < q ? w.ooff[i] : 0;
        if (i < q && w.e[i] != 1) ones = false;
    }
    // digits of g0: with a_j the plain mixed-radix digits and h_j the number
    // formed by the digits above j, k_j = a_j if h_j is even, R_j - 1 - a_j if
    // odd; the parity of h_j is also the direction k_j moves next.
    uint32_t down = 0, cw = 1, par = 0;
    uint64_t rest = g0;
    for (int j = 0; j < d; ++j) {
        const uint32_t R = w.R[j];
        const uint32_t a = (uint32_t)(rest % R);
        rest /= R;
        uint32_t b = a;
        if (rest & 1u) {
            b = R - 1u - a;
            down |= 1u << j;
        }
        dig[j][lane] = (uint8_t)b;
        cw *= weight(binom, w.mu[j], b, j == piv);
        par += b;
        const double f = (double)((int)w.mu[j] - 2 * (int)b);
        const double2* Uj = U + w.moff[j];
#pragma unroll
        for (int i = 0; i < QMAX; ++i)
            if (i < q) caxpy(x[i], f, ld(Uj + oo[i]));
    }
    for (uint64_t g = g0;;) {
        double2 p;
        if (ones) {
            // two independent chains (even and odd i) joined at the end: the
            // same n - 1 complex products with twice the instruction-level
            // parallelism
            double2 pa = x[0];
            double2 pb = q > 1 ? x[1] : make_double2(1.0, 0.0);
#pragma unroll
            for (int i = 2; i < QMAX; ++i) {
                if (i < q) {
                    if (i & 1) pb = cmul(pb, x[i]);
                    else pa = cmul(pa, x[i]);
                }
            }
            p = q > 1 ? cmul(pa, pb) : pa;
        } else {
            p = x[0];
            for (int t = 1; t < w.e[0]; ++t) p = cmul(p, x[0]);
#pragma unroll
            for (int i = 1; i < QMAX; ++i)
                if (i < q)
                    for (int t = 0; t < w.e[i]; ++t) p = cmul(p, x[i]);
        }
        double cf = (double)cw;
        if (par & 1u) cf = -cf;
        acc.x = fma(cf, p.x, acc.x);
        acc.y = fma(cf, p.y, acc.y);
        if (++g >= g1) break;
        // the lowest digit that can still move in its direction moves; the
        // digits below it turn around
        int j = 0;
        uint32_t b = 0, nb = 0;
        for (; j < d; ++j) {
            b = dig[j][lane];
            if ((down >> j) & 1u) {
                if (b > 0) { nb = b - 1u; break; }
            } else if (b + 1u < w.R[j]) {
                nb = b + 1u;
                break;
            }
            down ^= 1u << j;
        }
        if (j >= d) break;                      // not reached while g < T
        dig[j][lane] = (uint8_t)nb;
        const double f = nb > b ? -2.0 : 2.0;   // one more minus sign: the line sum loses 2 M[j][.]
        const double2* Uj = U + w.moff[j];
#pragma unroll
        for (int i = 0; i < QMAX; ++i)
            if (i < q) caxpy(x[i], f, ld(Uj + oo[i]));
        const bool pj = j == piv;
        cw = cw / weight(binom, w.mu[j], b, pj) * weight(binom, w.mu[j], nb, pj);
        par ^= 1u;
    }
    return acc;
}

// Part `part` of `parts` of output o's permanent, scaled; every lane returns
// the warp's sum.
__device__ double2 mult_item(const pcv_batch_desc& c, int64_t o, int part, int parts, int side, MultShared& sh,
                             int warp, int lane)
{
    MultWarp& w = sh.w[warp];
    double2 acc = make_double2(0.0, 0.0);
    if (mult_decode(c, c.outputs + o * c.m, side, w, lane)) {
        const uint64_t V = 32ull * (uint64_t)parts, v = (uint64_t)part * 32ull + (uint64_t)lane;
        const uint64_t g0 = w.T * v / V, g1 = w.T * (v + 1) / V;
        const double2* U = (const double2*)c.U;
        uint8_t (*dig)[32] = sh.digit[warp];
        if (w.q <= 8) acc = mult_range<8>(U, w, sh.binom, dig, g0, g1, lane);
        else if (w.q <= 16) acc = mult_range<16>(U, w, sh.binom, dig, g0, g1, lane);
        else if (w.q <= 24) acc = mult_range<24>(U, w, sh.binom, dig, g0, g1, lane);
        else acc = mult_range<PCV_MAX_PHOTONS>(U, w, sh.binom, dig, g0, g1, lane);
    }
    for (int off = 16; off > 0; off >>= 1) {
        acc.x += __shfl_xor_sync(kFull, acc.x, off);
        acc.y += __shfl_xor_sync(kFull, acc.y, off);
    }
    const double sc = w.scale;
    __syncwarp();                               // w is rewritten by the warp's next item
    return make_double2(acc.x * sc, acc.y * sc);
}

__device__ __forceinline__ void write_amp(const pcv_batch_desc& c, int64_t o, double2 v)
{
    if (c.amp) ((double2*)c.amp)[o] = v;
    if (c.prob) c.prob[o] = fma(v.x, v.x, v.y * v.y);
}

__global__ void __launch_bounds__(kMultThreads) glynn_mult_kernel(const pcv_batch_desc c, int parts, int side,
                                                                   double2* partial)
{
    __shared__ MultShared sh;
    init_binom(sh.binom);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * kMultWarps + warp;
    if (item >= c.n_out * parts) return;
    const int64_t o = item / parts;
    const int part = (int)(item % parts);
    const double2 v = mult_item(c, o, part, parts, side, sh, warp, lane);
    if (lane == 0) {
        if (parts == 1) write_amp(c, o, v);
        else partial[item] = v;
    }
}

__global__ void mult_finalize_kernel(const pcv_batch_desc c, int parts, const double2* partial)
{
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= c.n_out) return;
    double2 t = partial[o * parts];
    for (int p = 1; p < parts; ++p) t = cadd(t, partial[o * parts + p]);
    write_amp(c, o, t);
}

// Warps pull (circuit, output) entries of the batched launch's list one at a
// time; no warp waits for another.
__global__ void __launch_bounds__(kMultThreads) glynn_mult_persistent_kernel(const pcv_batch_desc* descs, MultQueue q)
{
    __shared__ MultShared sh;
    init_binom(sh.binom);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int total = *q.total;
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(q.counter, 1);
        it = __shfl_sync(kFull, it, 0);
        if (it >= total) break;
        const pcv_batch_desc& c = descs[q.circ[it]];
        const int64_t o = q.out[it];
        const double2 v = mult_item(c, o, 0, 1, 0, sh, warp, lane);
        if (lane == 0) write_amp(c, o, v);
    }
}

}  // namespace

cudaError_t launch_glynn_mult(const pcv_batch_desc& d, int parts, int side, double2* partial, cudaStream_t s)
{
    if (d.n_out == 0) return cudaSuccess;
    const int64_t items = d.n_out * parts;
    glynn_mult_kernel<<<(unsigned)((items + kMultWarps - 1) / kMultWarps), kMultThreads, 0, s>>>(d, parts, side, partial);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || parts == 1) return e;
    mult_finalize_kernel<<<(unsigned)((d.n_out + 255) / 256), 256, 0, s>>>(d, parts, partial);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_glynn_mult_persistent(const pcv_batch_desc* descs, const MultQueue& q, int sms, cudaStream_t s)
{
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, glynn_mult_persistent_kernel, kMultThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    glynn_mult_persistent_kernel<<<sms * per_sm, kMultThreads, 0, s>>>(descs, q);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace pcv
