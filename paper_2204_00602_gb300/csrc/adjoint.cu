// Adjoint of the amplitude: dL/dU from dL/da for many outputs (explicit
// outputs of one or B unitaries, or every output of the distributions of a
// batch of unitaries), any n <= 30, summed in a fixed order.
//
// With Glynn's sign vector d on the columns of A = U_{T,S} (Eq. eqperm) and
// row sums x_i(d) = sum_j d_j A[i][j],
//     dPerm/dA[i][j] = 2^{-(n-1)} sum_d sigma(d) d_j prod_{i' != i} x_{i'}(d),
// the permanent of the minor of (i, j) as a Glynn sum over the same Gray-code
// sequence as the forward kernels.  With w_i(d) = sigma(d) prod_{i' != i}
// x_{i'}(d), the n x n matrix G = sum_d w(d) d^T.  U[k][l] sits at every
// (i, j) with r_i = k and c_j = l, so with the dL/dRe + i dL/dIm convention
//     dL/dU[k][l] = sum_S gbar_S conj(norm_S sum_{r_i = k, c_j = l} G_S[i][j]).
//
// Kernels:
//   adjoint_thread_kernel  n <= 6: one thread per (output, batch entry) walks
//                          the whole Gray sequence with G in registers and
//                          writes H (below);
//   adjoint_part_kernel    one warp per (output, part of its Gray sequence,
//                          batch entry).  Each round every lane takes one sign
//                          vector (lane l walks its own run of the part),
//                          forms w(d) from prefix and suffix products of its
//                          row sums, and puts it in shared memory; then each
//                          lane adds the 32 sign vectors' w_i d_j into the
//                          entries of G it owns (row i, a run of columns), in
//                          lane order.  The scaled partial matrix
//                          H = gbar conj(c G) goes to the workspace.
//   adjoint_parts_kernel   (several parts per output) their H added in part order;
//   adjoint_segment_kernel per (batch entry, segment of 64 outputs, mode k,
//                          input mode l): the H entries of (k, l) summed over
//                          the segment's outputs in index order;
//   adjoint_final_kernel   per (batch entry, k, l): the segments added in
//                          order into dL/dU.
// No atomics: every sum has one fixed order, so a call gives the same bits
// every time.  Outputs are processed in chunks that fit the workspace, each
// chunk added into dL/dU after the previous one.

#include <algorithm>

#include "pcv_common.cuh"

namespace pcv {
namespace {

constexpr int kWarpsA = 4;                  // warps per block of adjoint_part_kernel
constexpr int kSeg = 64;                    // outputs per segment of the reduction
constexpr int64_t kPartSteps = 1 << 13;     // Gray steps per part when a sequence is split
constexpr int kMaxParts = 1024;
constexpr uint16_t kBadOutput = 0xFFFF;     // rows marker of an output whose photon number differs
constexpr int kThreadMaxN = 6;              // n up to this: one thread per output (G in registers)

struct ColList32 { int c[PCV_MAX_PHOTONS]; };

struct AdjArgs {
    const double2* U;            // [B][m][m]
    int m, n;
    int cols[PCV_MAX_PHOTONS];   // input modes, with repetition, non-decreasing
    double norm_t;
    const uint8_t* out_occ;      // explicit outputs [count][m], or null: canonical index o
    MultisetTable mc;
    int64_t count;               // outputs per batch entry (stride of gbar)
    int64_t o0, chunk;           // this launch: outputs [o0, o0 + chunk)
    int parts;                   // parts of each output's Gray sequence
    int64_t part_steps;          // 2^{n-1} / parts
    int q, cj;                   // lanes per row of G, columns per lane
    const double2* gbar;         // [B][count]
    double2* H;                  // [B][chunk][parts][n][n]
    uint16_t* rows;              // [chunk][n]: output modes of each row, or kBadOutput
};

// Output modes of the n rows (non-decreasing) and 1/sqrt(prod s!); false when
// an explicit output's photon number differs from n.
__device__ bool decode_rows(const AdjArgs& a, int64_t o, uint16_t* rows, double& norm_s)
{
    const int n = a.n, m = a.m;
    bool ok = true;
    if (a.out_occ) {
        const uint8_t* occ = a.out_occ + o * m;
        int i = 0;
        for (int r = 0; r < m; ++r)
            for (int c = occ[r]; c > 0; --c) {
                if (i < n) rows[i] = (uint16_t)r;
                ++i;
            }
        ok = i == n;
    } else {
        int64_t idx = o;
        int v = 0;
        for (int p = 0; p < n; ++p) {
            for (;;) {
                const int64_t c = a.mc(m - v, n - p - 1);
                if (idx < c) break;
                idx -= c;
                ++v;
            }
            rows[p] = (uint16_t)v;
        }
    }
    double f = 1.0;
    int run = 1;
    for (int i = 1; ok && i < n; ++i) {
        run = rows[i] == rows[i - 1] ? run + 1 : 1;
        f *= (double)run;
    }
    norm_s = 1.0 / sqrt(f);
    return ok;
}

// Shared memory of one warp: row sums and w of the 32 lanes (stride n + 1
// complex values), their Gray codes, and the output's rows.
__host__ __device__ inline size_t warp_smem_bytes(int n)
{
    return (size_t)2 * 32 * (n + 1) * sizeof(double2) + 32 * sizeof(uint32_t) + 64 * sizeof(uint16_t);
}

template <int CJ>
__global__ void __launch_bounds__(kWarpsA * 32) adjoint_part_kernel(const AdjArgs a)
{
    extern __shared__ double2 smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = a.n, m = a.m, st = n + 1;
    double2* xs = (double2*)((char*)smem + warp * warp_smem_bytes(n));
    double2* ws = xs + 32 * st;
    uint32_t* gcs = (uint32_t*)(ws + 32 * st);
    uint16_t* rows = (uint16_t*)(gcs + 32);

    const int64_t item = (int64_t)blockIdx.x * kWarpsA + warp;
    if (item >= a.chunk * a.parts) return;                // whole warps
    const int b = blockIdx.y;
    const int64_t oc = item / a.parts;
    const int part = (int)(item % a.parts);
    const int64_t o = a.o0 + oc;
    double norm_s = 1.0;
    if (lane == 0) {
        const bool ok = decode_rows(a, o, rows, norm_s);
        if (!ok) rows[0] = kBadOutput;
    }
    __syncwarp();
    norm_s = __shfl_sync(0xffffffffu, norm_s, 0);
    const bool ok = rows[0] != kBadOutput;
    if (b == 0 && part == 0 && lane < n) a.rows[oc * n + lane] = ok ? rows[lane] : kBadOutput;
    const double2 g = ok ? a.gbar[(int64_t)b * a.count + o] : make_double2(0.0, 0.0);
    const double2* U = a.U + (size_t)b * m * m;

    // this lane's entries of G: row i, columns j0 .. j0 + CJ - 1 (< n)
    const bool owner = lane < a.q * n;
    const int gi = owner ? lane / a.q : 0;
    const int j0 = owner ? (lane % a.q) * a.cj : n;
    double2 G[CJ];
#pragma unroll
    for (int jj = 0; jj < CJ; ++jj) G[jj] = make_double2(0.0, 0.0);

    if (g.x != 0.0 || g.y != 0.0) {
        // lane l walks steps [s0, s0 + len) of the part
        const int64_t pbase = (int64_t)part * a.part_steps;
        const int64_t per = a.part_steps >= 32 ? a.part_steps / 32 : 1;
        const bool walks = a.part_steps >= 32 || lane < a.part_steps;
        const int64_t s0 = pbase + (int64_t)lane * per;
        const int64_t rounds = per;
        double2* x = xs + lane * st;
        double2* w = ws + lane * st;
        uint32_t gc = 0;
        double sg = 1.0;                                 // sigma(d)
        if (walks) {
            gc = (uint32_t)(s0 ^ (s0 >> 1));
            sg = (__popc(gc) & 1) ? -1.0 : 1.0;
            for (int i = 0; i < n; ++i) {
                const double2* Ur = U + (size_t)rows[i] * m;
                double2 s = __ldg(Ur + a.cols[0]);
                for (int j = 1; j < n; ++j) caxpy(s, ((gc >> (j - 1)) & 1u) ? -1.0 : 1.0, __ldg(Ur + a.cols[j]));
                x[i] = s;
            }
        }
        for (int64_t r = 0; r < rounds; ++r) {
            // w_i = sigma prod_{i' != i} x_i': prefix products, then suffixes
            if (walks) {
                double2 p = make_double2(1.0, 0.0);
                for (int i = 0; i < n; ++i) {
                    w[i] = p;
                    p = cmul(p, x[i]);
                }
                double2 sfx = make_double2(sg, 0.0);
                for (int i = n - 1; i >= 0; --i) {
                    w[i] = cmul(w[i], sfx);
                    sfx = cmul(sfx, x[i]);
                }
            } else {
                for (int i = 0; i < n; ++i) w[i] = make_double2(0.0, 0.0);
            }
            gcs[lane] = gc;
            __syncwarp();
            if (owner) {
                for (int l2 = 0; l2 < 32; ++l2) {
                    const double2 wv = ws[l2 * st + gi];
                    const uint32_t g2 = gcs[l2];
#pragma unroll
                    for (int jj = 0; jj < CJ; ++jj) {
                        const int j = j0 + jj;
                        if (jj < a.cj && j < n) {
                            const bool neg = j > 0 && ((g2 >> (j - 1)) & 1u);
                            G[jj].x += neg ? -wv.x : wv.x;
                            G[jj].y += neg ? -wv.y : wv.y;
                        }
                    }
                }
            }
            __syncwarp();
            if (walks && r + 1 < rounds) {               // Gray step to the next sign vector
                const uint64_t kk = (uint64_t)(s0 + r + 1);
                const int bb = __ffsll((long long)kk) - 1;
                const uint32_t gn = (uint32_t)(kk ^ (kk >> 1));
                const double sd = ((gn >> bb) & 1u) ? -2.0 : 2.0;
                const int col = a.cols[bb + 1];
                for (int i = 0; i < n; ++i) caxpy(x[i], sd, __ldg(U + (size_t)rows[i] * m + col));
                gc = gn;
                sg = -sg;
            }
        }
    }
    if (!owner) return;
    // H = gbar conj(c G), c = norm_S norm_T 2^{-(n-1)}
    const double c = ldexp(norm_s * a.norm_t, -(n - 1));
    double2* H = a.H + (((size_t)b * a.chunk + oc) * a.parts + part) * n * n + (size_t)gi * n;
#pragma unroll
    for (int jj = 0; jj < CJ; ++jj) {
        const int j = j0 + jj;
        if (jj < a.cj && j < n) H[j] = cmul(g, make_double2(c * G[jj].x, -c * G[jj].y));
    }
}

// Small n: one thread per output walks all 2^{n-1} sign vectors in Gray
// order with the n x n Glynn sums of the minors in registers, and writes H as
// adjoint_part_kernel does with one part.  Every lane does useful FP64 work
// (FP64 is scarce on this part; the warp form leaves lanes idle when n is
// small): measured at n = 6, 2.4x faster over 792K outputs and 1.3x over 32K.
template <int N>
__global__ void __launch_bounds__(128) adjoint_thread_kernel(const AdjArgs a)
{
    const int64_t oc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (oc >= a.chunk) return;
    const int b = blockIdx.y;
    const int64_t o = a.o0 + oc;
    const int m = a.m;
    uint16_t rows[N];
    double norm_s = 1.0;
    const bool ok = decode_rows(a, o, rows, norm_s);
    if (b == 0)
        for (int i = 0; i < N; ++i) a.rows[oc * N + i] = ok ? rows[i] : kBadOutput;
    double2* H = a.H + ((size_t)b * a.chunk + oc) * N * N;
    const double2 g = ok ? a.gbar[(int64_t)b * a.count + o] : make_double2(0.0, 0.0);
    if (g.x == 0.0 && g.y == 0.0) {
        for (int e = 0; e < N * N; ++e) H[e] = make_double2(0.0, 0.0);
        return;
    }
    const double2* U = a.U + (size_t)b * m * m;
    double2 x[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {                         // sign vector 0: every sign +1
        double2 sum = __ldg(U + (size_t)rows[i] * m + a.cols[0]);
        for (int j = 1; j < N; ++j) sum = cadd(sum, __ldg(U + (size_t)rows[i] * m + a.cols[j]));
        x[i] = sum;
    }
    double2 G[N][N];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) G[i][j] = make_double2(0.0, 0.0);
    uint32_t gc = 0;
    double sg = 1.0;                                      // sigma(d)
    const uint32_t steps = 1u << (N - 1);
    for (uint32_t st = 0; st < steps; ++st) {
        // w_i = sigma prod_{i' != i} x_i': prefix products, then suffixes
        double2 pre[N];
        pre[0] = make_double2(1.0, 0.0);
#pragma unroll
        for (int i = 1; i < N; ++i) pre[i] = cmul(pre[i - 1], x[i - 1]);
        double2 sfx = make_double2(sg, 0.0);
#pragma unroll
        for (int i = N - 1; i >= 0; --i) {
            const double2 w = cmul(pre[i], sfx);
            sfx = cmul(sfx, x[i]);
            G[i][0] = cadd(G[i][0], w);
#pragma unroll
            for (int j = 1; j < N; ++j) caxpy(G[i][j], ((gc >> (j - 1)) & 1u) ? -1.0 : 1.0, w);
        }
        if (st + 1 < steps) {                             // Gray step to the next sign vector
            const uint32_t kk = st + 1;
            const int bb = __ffs((int)kk) - 1;
            const uint32_t gn = kk ^ (kk >> 1);
            const double sd = ((gn >> bb) & 1u) ? -2.0 : 2.0;
            const int col = a.cols[bb + 1];
#pragma unroll
            for (int i = 0; i < N; ++i) caxpy(x[i], sd, __ldg(U + (size_t)rows[i] * m + col));
            gc = gn;
            sg = -sg;
        }
    }
    // H = gbar conj(c G), c = norm_S norm_T 2^{-(n-1)}
    const double c = ldexp(norm_s * a.norm_t, -(N - 1));
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) H[i * N + j] = cmul(g, make_double2(c * G[i][j].x, -c * G[i][j].y));
}

// H of each output summed over its parts, in part order, into part 0's place
// of a [B][chunk][n][n] array.
__global__ void adjoint_parts_kernel(const double2* __restrict__ H, int64_t chunk, int parts, int nn, int B,
                                     double2* __restrict__ Hs)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)B * chunk * nn) return;
    const int64_t bo = t / nn;
    const int e = (int)(t % nn);
    const double2* src = H + bo * parts * nn + e;
    double2 v = src[0];
    for (int p = 1; p < parts; ++p) v = cadd(v, src[(int64_t)p * nn]);
    Hs[t] = v;
}

struct SegArgs {
    const double2* H;            // [B][chunk][n][n]
    const uint16_t* rows;        // [chunk][n]
    int64_t chunk;
    int n, m, B, din, nseg;
    int jb[PCV_MAX_PHOTONS], je[PCV_MAX_PHOTONS];   // columns j of input mode li: [jb, je)
    double2* seg;                // [B][nseg][m][din]
};

// (b, segment, k, li): sum over the segment's outputs in order of the H
// entries with row mode k and the columns of input mode li.
__global__ void adjoint_segment_kernel(const SegArgs a)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per_b = (int64_t)a.nseg * a.m * a.din;
    if (t >= per_b * a.B) return;
    const int b = (int)(t / per_b);
    const int64_t rem = t % per_b;
    const int sg = (int)(rem / ((int64_t)a.m * a.din));
    const int k = (int)((rem / a.din) % a.m);
    const int li = (int)(rem % a.din);
    const int n = a.n;
    double2 acc = make_double2(0.0, 0.0);
    const int64_t e = min((int64_t)(sg + 1) * kSeg, a.chunk);
    for (int64_t oc = (int64_t)sg * kSeg; oc < e; ++oc) {
        const uint16_t* r = a.rows + oc * n;
        if (r[0] == kBadOutput) continue;
        const double2* Ho = a.H + ((size_t)b * a.chunk + oc) * n * n;
        for (int i = 0; i < n; ++i) {
            if (r[i] != k) continue;
            for (int j = a.jb[li]; j < a.je[li]; ++j) acc = cadd(acc, Ho[i * n + j]);
        }
    }
    a.seg[t] = acc;
}

// (b, k, li): dL/dU[b][k][l] += the segments in order.
__global__ void adjoint_final_kernel(const double2* __restrict__ seg, int B, int nseg, int m, int din, ColList32 lmode,
                                     double2* __restrict__ gradU)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)B * m * din) return;
    const int b = (int)(t / ((int64_t)m * din));
    const int k = (int)((t / din) % m);
    const int li = (int)(t % din);
    double2 v = make_double2(0.0, 0.0);
    for (int s = 0; s < nseg; ++s) v = cadd(v, seg[(((int64_t)b * nseg + s) * m + k) * din + li]);
    double2* dst = gradU + ((size_t)b * m + k) * m + lmode.c[li];
    *dst = cadd(*dst, v);
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

template <int N>
cudaError_t launch_thread(const AdjArgs& a, int B, cudaStream_t s)
{
    dim3 grid((unsigned)((a.chunk + 127) / 128), (unsigned)B);
    adjoint_thread_kernel<N><<<grid, 128, 0, s>>>(a);
    note_launches(1);
    return cudaGetLastError();
}

template <int CJ>
cudaError_t launch_part(const AdjArgs& a, int B, cudaStream_t s)
{
    const size_t smem = kWarpsA * warp_smem_bytes(a.n);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(adjoint_part_kernel<CJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t items = a.chunk * a.parts;
    dim3 grid((unsigned)((items + kWarpsA - 1) / kWarpsA), (unsigned)B);
    adjoint_part_kernel<CJ><<<grid, kWarpsA * 32, smem, s>>>(a);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace

AdjPlan adjoint_plan(int m, int n, int B, int64_t count, int64_t ws_bytes)
{
    AdjPlan p{};
    const int64_t K = n > 0 ? (1ll << (n - 1)) : 1;
    p.parts = (int)std::min<int64_t>(kMaxParts, std::max<int64_t>(1, K / kPartSteps));
    p.part_steps = K / p.parts;
    int q = std::max(1, std::min(n, 32 / std::max(n, 1)));
    p.cj = (n + q - 1) / q;
    p.q = (n + p.cj - 1) / p.cj;
    p.table = al256((size_t)(m + 1) * (n + 1) * sizeof(int64_t));
    const size_t nn16 = (size_t)n * n * sizeof(double2);
    auto bytes = [&](int64_t C) {
        const int64_t nseg = (C + kSeg - 1) / kSeg;
        return p.table + al256((size_t)B * C * p.parts * nn16) + (p.parts > 1 ? al256((size_t)B * C * nn16) : 0) +
               al256((size_t)C * n * sizeof(uint16_t)) + al256((size_t)B * nseg * m * n * sizeof(double2));
    };
    // default: every output in one chunk up to a 256 MiB budget
    const size_t budget = ws_bytes < 0 ? std::max<size_t>(bytes(1), (size_t)256 << 20) : (size_t)ws_bytes;
    int64_t C = std::max<int64_t>(1, count);
    if (bytes(C) > budget) {
        int64_t lo = 1, hi = C;
        while (lo < hi) {                      // the largest chunk that fits
            const int64_t mid = lo + (hi - lo + 1) / 2;
            if (bytes(mid) <= budget) lo = mid;
            else hi = mid - 1;
        }
        C = lo;
    }
    p.chunk = C;
    p.total = bytes(C);
    p.min_total = bytes(1);
    return p;
}

int adjoint_max_photons() { return PCV_MAX_PHOTONS; }

cudaError_t launch_adjoint(const Plan& pl, const double2* U, int B, const uint8_t* out_occ, int64_t count,
                           const double2* gbar, double2* gradU, void* ws, const AdjPlan& ap, cudaStream_t s)
{
    const int m = pl.m, n = pl.n;
    cudaError_t e = cudaMemsetAsync(gradU, 0, (size_t)B * m * m * sizeof(double2), s);
    if (e != cudaSuccess || count == 0 || n == 0) return e;
    char* w = (char*)ws;
    int64_t* table = (int64_t*)w;
    w += ap.table;
    const size_t nn16 = (size_t)n * n * sizeof(double2);
    const int64_t C = ap.chunk;
    double2* H = (double2*)w;
    w += al256((size_t)B * C * ap.parts * nn16);
    double2* Hs = ap.parts > 1 ? (double2*)w : H;
    if (ap.parts > 1) w += al256((size_t)B * C * nn16);
    uint16_t* rows = (uint16_t*)w;
    w += al256((size_t)C * n * sizeof(uint16_t));
    double2* seg = (double2*)w;
    if (!out_occ && (e = build_multiset_table(table, m, n, s)) != cudaSuccess) return e;

    AdjArgs a;
    a.U = U;
    a.m = m;
    a.n = n;
    for (int j = 0; j < PCV_MAX_PHOTONS; ++j) a.cols[j] = pl.cols[j];
    a.norm_t = pl.norm_t;
    a.out_occ = out_occ;
    a.mc.t = table;
    a.mc.kmax = n;
    a.count = count;
    a.parts = ap.parts;
    a.part_steps = ap.part_steps;
    a.q = ap.q;
    a.cj = ap.cj;
    a.gbar = gbar;
    a.H = H;
    a.rows = rows;
    // the distinct input modes and their column ranges
    SegArgs sa;
    ColList32 lmode;
    int din = 0;
    for (int j = 0; j < n; ++j) {
        if (j == 0 || pl.cols[j] != pl.cols[j - 1]) {
            lmode.c[din] = pl.cols[j];
            sa.jb[din] = j;
            ++din;
        }
        sa.je[din - 1] = j + 1;
    }
    sa.rows = rows;
    sa.n = n;
    sa.m = m;
    sa.B = B;
    sa.din = din;
    sa.seg = seg;
    sa.H = Hs;
    for (int64_t o0 = 0; o0 < count; o0 += C) {
        const int64_t cc = std::min<int64_t>(C, count - o0);
        a.o0 = o0;
        a.chunk = cc;
        if (ap.parts == 1 && n <= kThreadMaxN) {
            switch (n) {
            case 1: e = launch_thread<1>(a, B, s); break;
            case 2: e = launch_thread<2>(a, B, s); break;
            case 3: e = launch_thread<3>(a, B, s); break;
            case 4: e = launch_thread<4>(a, B, s); break;
            case 5: e = launch_thread<5>(a, B, s); break;
            default: e = launch_thread<6>(a, B, s); break;
            }
        } else switch (ap.cj) {
        case 1: e = launch_part<1>(a, B, s); break;
        case 2: e = launch_part<2>(a, B, s); break;
        case 3: case 4: e = launch_part<4>(a, B, s); break;
        case 5: case 6: case 7: case 8: e = launch_part<8>(a, B, s); break;
        default: e = launch_part<32>(a, B, s); break;
        }
        if (e != cudaSuccess) return e;
        if (ap.parts > 1) {
            const int64_t th = (int64_t)B * cc * n * n;
            adjoint_parts_kernel<<<(unsigned)((th + 255) / 256), 256, 0, s>>>(H, cc, ap.parts, n * n, B, Hs);
            note_launches(1);
        }
        sa.chunk = cc;
        sa.nseg = (int)((cc + kSeg - 1) / kSeg);
        const int64_t th = (int64_t)B * sa.nseg * m * din;
        adjoint_segment_kernel<<<(unsigned)((th + 127) / 128), 128, 0, s>>>(sa);
        const int64_t tf = (int64_t)B * m * din;
        adjoint_final_kernel<<<(unsigned)((tf + 127) / 128), 128, 0, s>>>(seg, B, sa.nseg, m, din, lmode, gradU);
        note_launches(2);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace pcv
