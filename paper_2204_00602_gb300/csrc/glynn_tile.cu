// Shared-row-sum Glynn kernels for explicit outputs: one block computes a tile
// of outputs of one (U, input) pair, and a persistent variant pulls tiles of
// many circuits of uneven size from a device work queue.
//
// With Glynn's sign vector d on the input photons (columns of U_{T,S}, Eq.
// eqperm), the row sum of output row i depends only on its output mode:
// y_r(d) = sum_j d_j U[r][c_j].  A block therefore keeps y_r(d) for all m modes
// in shared memory, advancing it one Gray step at a time (2 DFMA per mode and
// step, shared by the whole tile), and each output only forms its product
//     a(S) += sigma(d) prod_i y_{r_i}(d):  4(n-1) + 2 FP64 instructions per
// output and sign vector instead of the 6n - 2 of the plain per-output kernel.
//
// Block layout: TILE = 256 / S outputs x S contiguous ranges of sign vectors
// ("splits"); split s owns sign vectors [s L, (s+1) L), L = 2^{n-1} / S, and
// walks them in chunks of C steps whose row sums are staged in shared memory.
// The S partial sums of an output are added in a fixed order at the end, so
// results are deterministic.

#include "pcv_common.cuh"

namespace pcv {

// Splits per block as a function of n: more sign-vector parallelism for
// larger permanents, whole tiles of 256 outputs for small ones.
__host__ __device__ int tile_splits(int n)
{
    if (n <= 10) return 1;
    if (n <= 13) return 2;
    if (n <= 16) return 4;
    return 8;
}

namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 4;            // Gray steps staged per split and pass
constexpr int kMaxModes = 128;       // modes kept in shared memory

struct TileShared {
    double2 y[8 * kChunk * kMaxModes];   // [split][step][mode] staged row sums
    double2 yrun[8 * kMaxModes];         // [split][mode] running row sums
    double2 acc[kThreads];
    uint8_t rows[kThreads * PCV_MAX_PHOTONS];
    int cols[PCV_MAX_PHOTONS];
};

// One tile of circuit c: positions [tile TILE, (tile + 1) TILE) of its
// output list, which is idx[0..count) (or the outputs 0..count-1 themselves
// when idx is null).
__device__ void tile_item(const pcv_batch_desc& c, int64_t tile, TileShared& sh, const int* idx, int64_t count)
{
    const int n = c.n, m = c.m;
    const int S = tile_splits(n);
    const int TILE = kThreads / S;
    const int tid = threadIdx.x;
    const int ol = tid % TILE, s = tid / TILE;
    const int64_t pos = tile * TILE + ol;
    const bool live = pos < count;
    const int64_t o = live ? (idx ? (int64_t)idx[pos] : pos) : 0;

    if (tid < n) sh.cols[tid] = c.cols[tid];
    double norm_t = 1.0;                  // 1/sqrt(prod t!) from the sorted photon -> input-mode list
    {
        double f = 1.0;
        int run = 1;
        for (int j = 1; j < n; ++j) {
            run = (c.cols[j] == c.cols[j - 1]) ? run + 1 : 1;
            f *= run;
        }
        norm_t = 1.0 / sqrt(f);
    }
    // decode the output: rows (output modes, non-decreasing) and 1/sqrt(prod s!)
    bool ok = live;
    double norm = 1.0;
    if (live && s == 0) {
        const uint8_t* occ = c.outputs + o * m;
        int cnt = 0;
        double f = 1.0;
        for (int r = 0; r < m; ++r) {
            const int k = occ[r];
            for (int q = 1; q <= k; ++q) {
                if (cnt < PCV_MAX_PHOTONS) sh.rows[tid * PCV_MAX_PHOTONS + cnt] = (uint8_t)r;
                ++cnt;
                f *= q;
            }
        }
        ok = cnt == n;
        norm = 1.0 / sqrt(f);
    }
    __syncthreads();
    // every split of this output reads the rows decoded by split 0
    const uint8_t* myrows = sh.rows + ol * PCV_MAX_PHOTONS;
    if (live && s != 0) {
        int cnt = 0;
        const uint8_t* occ = c.outputs + o * m;
        for (int r = 0; r < m; ++r) cnt += occ[r];
        ok = cnt == n;
    }

    const int64_t L = (1ll << (n - 1)) / S;
    const int C = L < kChunk ? (int)L : kChunk;
    // running row sums of every split at its first sign vector
    for (int q = tid; q < S * m; q += kThreads) {
        const int ss = q / m, r = q % m;
        const int64_t k0 = (int64_t)ss * L;
        const uint64_t g = (uint64_t)k0 ^ ((uint64_t)k0 >> 1);
        const double2* Ur = (const double2*)c.U + (size_t)r * m;
        double2 y = Ur[sh.cols[0]];
        for (int j = 1; j < n; ++j) caxpy(y, ((g >> (j - 1)) & 1u) ? -1.0 : 1.0, Ur[sh.cols[j]]);
        sh.yrun[ss * kMaxModes + r] = y;
    }
    double2 acc = make_double2(0.0, 0.0);
    for (int64_t base = 0; base < L; base += C) {
        __syncthreads();
        // stage C steps of row sums for every split; advance the running sums
        for (int q = tid; q < S * m; q += kThreads) {
            const int ss = q / m, r = q % m;
            double2 y = sh.yrun[ss * kMaxModes + r];
            const double2* Ur = (const double2*)c.U + (size_t)r * m;
            for (int st = 0; st < C; ++st) {
                sh.y[(ss * kChunk + st) * kMaxModes + r] = y;
                const int64_t kk = (int64_t)ss * L + base + st + 1;
                if (base + st + 1 < L) {
                    const int b = __ffsll(kk) - 1;
                    const double sd = ((kk >> (b + 1)) & 1) ? 2.0 : -2.0;
                    caxpy(y, sd, Ur[sh.cols[b + 1]]);
                }
            }
            sh.yrun[ss * kMaxModes + r] = y;
        }
        __syncthreads();
        if (ok) {
            for (int st = 0; st < C; ++st) {
                const int64_t k = (int64_t)s * L + base + st;
                const uint64_t g = (uint64_t)k ^ ((uint64_t)k >> 1);
                const double sg = (__popcll(g) & 1) ? -1.0 : 1.0;
                const double2* ys = sh.y + (s * kChunk + st) * kMaxModes;
                double2 p = ys[myrows[0]];
                for (int i = 1; i < n; ++i) p = cmul(p, ys[myrows[i]]);
                caxpy(acc, sg, p);
            }
        }
    }
    sh.acc[tid] = acc;
    __syncthreads();
    if (s == 0 && live) {
        double2 t = acc;
        for (int ss = 1; ss < S; ++ss) t = cadd(t, sh.acc[ss * TILE + ol]);
        double2 v = make_double2(0.0, 0.0);
        if (ok) {
            const double sc = ldexp(norm * norm_t, -(n - 1));
            v = make_double2(t.x * sc, t.y * sc);
        }
        if (c.amp) ((double2*)c.amp)[o] = v;
        if (c.prob) c.prob[o] = fma(v.x, v.x, v.y * v.y);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads) glynn_tile_kernel(const pcv_batch_desc c)
{
    extern __shared__ __align__(16) unsigned char smem[];
    TileShared& sh = *reinterpret_cast<TileShared*>(smem);
    tile_item(c, blockIdx.x, sh, nullptr, c.n_out);
}

// Same outputs for B unitaries: blockIdx.y selects U + b*ustride and the
// output arrays + b*ostride.
__global__ void __launch_bounds__(kThreads) glynn_tile_multi_kernel(const pcv_batch_desc c0, int64_t ustride, int64_t ostride)
{
    extern __shared__ __align__(16) unsigned char smem[];
    TileShared& sh = *reinterpret_cast<TileShared*>(smem);
    pcv_batch_desc c = c0;
    const int64_t b = blockIdx.y;
    c.U = c0.U + b * ustride;
    if (c0.amp) c.amp = c0.amp + b * ostride;
    if (c0.prob) c.prob = c0.prob + b * ostride;
    tile_item(c, blockIdx.x, sh, nullptr, c.n_out);
}

// Work queue of the batched launch: tile items (circuit, tile of the
// circuit's tile-routed outputs) in order of decreasing photon number; blocks
// pull the next item with one atomicAdd and never wait for another block.
struct Queue {
    int* counter;
    int* total;
    int* item_circ;
    int* item_tile;
    const int64_t* out_off;   // first entry of circuit c in idx
    const int* n_tile;        // tile-routed outputs of circuit c (idx[out_off[c] ...])
    const int* idx;
};

__global__ void __launch_bounds__(kThreads) glynn_persistent_kernel(const pcv_batch_desc* descs, Queue q)
{
    extern __shared__ __align__(16) unsigned char smem[];
    TileShared& sh = *reinterpret_cast<TileShared*>(smem);
    __shared__ int s_item;
    const int total = *q.total;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(q.counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= total) break;
        const int c = q.item_circ[it];
        tile_item(descs[c], q.item_tile[it], sh, q.idx + q.out_off[c], q.n_tile[c]);
    }
}

// A descriptor the kernels cannot run (n or m out of range, an input mode
// outside [0, m) or out of order) gets no work; the binding checks
// descriptors before they reach the device.
__device__ bool desc_ok(const pcv_batch_desc& d)
{
    if (d.n < 1 || d.n > PCV_MAX_PHOTONS || d.m < 1 || d.m > kMaxModes || d.n_out < 0) return false;
    for (int j = 0; j < d.n; ++j)
        if (d.cols[j] < 0 || d.cols[j] >= d.m || (j > 0 && d.cols[j] < d.cols[j - 1])) return false;
    return true;
}

// Block-wide exclusive scan of one value per thread (1024 threads at most);
// returns the thread's offset, *total the sum.  buf holds 64 values.
template <typename T>
__device__ T block_scan(T v, T* buf, T* total)
{
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = (blockDim.x + 31) >> 5;
    T incl = v;
    for (int off = 1; off < 32; off <<= 1) {
        const T t = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += t;
    }
    if (lane == 31) buf[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        T w = lane < nw ? buf[lane] : T(0);
        for (int off = 1; off < 32; off <<= 1) {
            const T t = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += t;
        }
        if (lane < nw) buf[32 + lane] = w;       // inclusive prefix over warps
    }
    __syncthreads();
    const T res = (wid ? buf[32 + wid - 1] : T(0)) + incl - v;
    *total = buf[32 + nw - 1];
    __syncthreads();
    return res;
}

// out_off[c]: exclusive prefix of the output counts of valid circuits, in
// circuit order (one block of 1024 threads).
__global__ void __launch_bounds__(1024) offsets_kernel(const pcv_batch_desc* descs, int n_circ, int64_t* out_off)
{
    __shared__ int64_t buf[64];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < n_circ; b0 += 1024) {
        const int c = b0 + threadIdx.x;
        const int64_t cnt = c < n_circ && desc_ok(descs[c]) ? descs[c].n_out : 0;
        int64_t tot = 0;
        const int64_t ex = block_scan<int64_t>(cnt, buf, &tot);
        if (c < n_circ) out_off[c] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
}

// FP64 pipe instructions of one output: the tile kernel spends 4n - 2 per
// sign vector (n - 1 complex products and the accumulation) plus its share
// 2m / TILE of the row-sum updates; Glynn's sum with multiplicities spends
// 2q + 4n - 1 per term (q line-sum updates, n - 1 complex products, the
// weight and the accumulation).
__device__ double tile_cost(int m, int n)
{
    return ldexp(1.0, n - 1) * (4.0 * n - 2.0 + 2.0 * m / (double)(kThreads / tile_splits(n)));
}

__device__ double mult_side_cost(const int* mu, int d, int q, int n)
{
    double t = 1.0;
    int odd = -1, big = 0;
    for (int j = 0; j < d; ++j) {
        t *= mu[j] + 1;
        if (odd < 0 && (mu[j] & 1)) odd = j;
        if (mu[j] > mu[big]) big = j;
    }
    const int p = odd >= 0 ? odd : big;
    t = t / (mu[p] + 1) * (mu[p] / 2 + 1);
    return t * (2.0 * q + 4.0 * n - 1.0);
}

// FP64 instructions of output o by Glynn's sum with multiplicities on its
// cheaper side; a negative value for an output outside S_{m,n} (amplitude 0).
__device__ double output_mult_cost(const pcv_batch_desc& c, int64_t o, const int* imu, int d_in)
{
    const uint8_t* occ = c.outputs + o * c.m;
    int omu[PCV_MAX_PHOTONS];
    int d_out = 0, tot = 0;
    for (int r = 0; r < c.m; ++r) {
        const int v = occ[r];
        if (v > 0 && d_out < PCV_MAX_PHOTONS) omu[d_out++] = v;
        tot += v;
    }
    if (tot != c.n) return -1.0;
    return fmin(mult_side_cost(omu, d_out, d_in, c.n), mult_side_cost(imu, d_in, d_out, c.n));
}

// One block per circuit: route each output to the tile kernel or to Glynn's
// sum with multiplicities; idx[out_off[c] ..] lists the tile outputs first
// (in order) and the others after them (in reverse order).  A tile block
// costs as much with one live output as with TILE of them, so a last,
// partly filled tile is re-routed when its outputs cost less on the
// multiplicity kernel than the whole block.
__global__ void __launch_bounds__(256) classify_kernel(const pcv_batch_desc* descs, const int64_t* out_off, int route,
                                                       int64_t cap, int* idx, int* n_tile, int* n_mult)
{
    __shared__ int buf[64];
    __shared__ int s_tile, s_mult;
    const int ci = blockIdx.x;
    const pcv_batch_desc& c = descs[ci];
    const bool valid = desc_ok(c) && out_off[ci] + c.n_out <= cap;
    if (!valid) {
        if (threadIdx.x == 0) n_tile[ci] = n_mult[ci] = 0;
        return;
    }
    const int m = c.m, n = c.n;
    const int64_t no = c.n_out;
    int* list = idx + out_off[ci];
    // input side: distinct modes and multiplicities
    int imu[PCV_MAX_PHOTONS];
    int d_in = 0;
    for (int j = 0; j < n; ++j) {
        if (j == 0 || c.cols[j] != c.cols[j - 1]) imu[d_in++] = 0;
        imu[d_in - 1] += 1;
    }
    const double ct = tile_cost(m, n);
    if (threadIdx.x == 0) s_tile = s_mult = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < no; b0 += blockDim.x) {
        const int64_t o = b0 + threadIdx.x;
        int to_mult = 0;
        if (o < no) {
            if (route == PCV_ALGO_MULT) {
                to_mult = 1;
            } else if (route == PCV_ALGO_AUTO) {
                const double cm = output_mult_cost(c, o, imu, d_in);
                to_mult = cm < ct;                    // cm < 0: not in S_{m,n}, amplitude 0
            }
        }
        int tot_m = 0;
        const int pm = block_scan<int>(to_mult, buf, &tot_m);
        const int live = o < no ? 1 : 0;
        int tot_t = 0;
        const int pt = block_scan<int>(live - to_mult, buf, &tot_t);
        if (o < no) {
            if (to_mult) list[no - 1 - (s_mult + pm)] = (int)o;
            else list[s_tile + pt] = (int)o;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_tile += tot_t;
            s_mult += tot_m;
        }
        __syncthreads();
    }
    if (route == PCV_ALGO_AUTO) {
        const int tilesz = kThreads / tile_splits(n);
        const int r = s_tile % tilesz;
        if (r > 0) {
            // the last r tile outputs sit just below the multiplicity outputs
            // in the list; moving the boundary re-routes them
            double part = 0.0;
            for (int k = threadIdx.x; k < r; k += blockDim.x)
                part += output_mult_cost(c, list[s_tile - r + k], imu, d_in);
            for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
            __shared__ double wsum[8];
            if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = part;
            __syncthreads();
            if (threadIdx.x == 0) {
                double tot = 0.0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += wsum[w];
                if (tot < ct * tilesz) {
                    s_tile -= r;
                    s_mult += r;
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        n_tile[ci] = s_tile;
        n_mult[ci] = s_mult;
    }
}

// Builds both work lists on the device (one block): a counting sort of the
// circuits by n (descending), then tile items and multiplicity entries in
// that order.
__global__ void __launch_bounds__(1024) plan_kernel(const pcv_batch_desc* descs, int n_circ, Queue q, MultQueue mq,
                                                    int* order, int* item_off, int* mult_off, const int* n_mult,
                                                    int* mult_circ, int* mult_out, int max_items)
{
    __shared__ int bucket[PCV_MAX_PHOTONS + 2];
    __shared__ int cursor[PCV_MAX_PHOTONS + 2];
    __shared__ int buf[64];
    __shared__ int carry_t, carry_m;
    const int tid = threadIdx.x;
    if (tid < PCV_MAX_PHOTONS + 2) bucket[tid] = 0;
    __syncthreads();
    for (int c = tid; c < n_circ; c += blockDim.x)
        atomicAdd(&bucket[desc_ok(descs[c]) ? descs[c].n : 0], 1);
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int n = PCV_MAX_PHOTONS; n >= 0; --n) { cursor[n] = acc; acc += bucket[n]; }
        carry_t = carry_m = 0;
    }
    __syncthreads();
    for (int c = tid; c < n_circ; c += blockDim.x)
        order[atomicAdd(&cursor[desc_ok(descs[c]) ? descs[c].n : 0], 1)] = c;
    __syncthreads();
    // exclusive scans of tile-item and entry counts over the sorted order
    for (int b0 = 0; b0 < n_circ; b0 += 1024) {
        const int p = b0 + tid;
        int ct = 0, cm = 0;
        if (p < n_circ) {
            const int c = order[p];
            const int tilesz = kThreads / tile_splits(descs[c].n);
            ct = (q.n_tile[c] + tilesz - 1) / tilesz;
            cm = n_mult[c];
        }
        int tt = 0, tm = 0;
        const int et = block_scan<int>(ct, buf, &tt);
        const int em = block_scan<int>(cm, buf, &tm);
        if (p < n_circ) {
            item_off[p] = carry_t + et;
            mult_off[p] = carry_m + em;
        }
        __syncthreads();
        if (tid == 0) {
            carry_t += tt;
            carry_m += tm;
        }
        __syncthreads();
    }
    if (tid == 0) {
        *q.total = carry_t < max_items ? carry_t : max_items;
        *q.counter = 0;
        *mq.total = carry_m;
        *mq.counter = 0;
    }
    __syncthreads();
    for (int p = 0; p < n_circ; ++p) {
        const int c = order[p];
        const int tilesz = kThreads / tile_splits(descs[c].n);
        const int cnt = (q.n_tile[c] + tilesz - 1) / tilesz;
        for (int t = tid; t < cnt; t += blockDim.x) {
            const int it = item_off[p] + t;
            if (it < max_items) {
                q.item_circ[it] = c;
                q.item_tile[it] = t;
            }
        }
        const int cm = n_mult[c];
        const int* src = q.idx + q.out_off[c] + q.n_tile[c];
        for (int t = tid; t < cm; t += blockDim.x) {
            mult_circ[mult_off[p] + t] = c;
            mult_out[mult_off[p] + t] = src[t];
        }
    }
}

uint64_t g_attr_set = 0;     // bit d: attributes set on device d

cudaError_t ensure_smem_attr()
{
    int dev = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 != cudaSuccess) return e0;
    const uint64_t bit = 1ull << (dev & 63);
    if (g_attr_set & bit) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(glynn_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TileShared));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(glynn_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TileShared));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(glynn_tile_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TileShared));
    if (e != cudaSuccess) return e;
    g_attr_set |= bit;
    return cudaSuccess;
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

__global__ void store_desc_kernel(const pcv_batch_desc d, pcv_batch_desc* out) { *out = d; }

}  // namespace

int tile_max_modes() { return kMaxModes; }

cudaError_t launch_store_desc(const pcv_batch_desc& d, pcv_batch_desc* out, cudaStream_t s)
{
    store_desc_kernel<<<1, 1, 0, s>>>(d, out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_glynn_tile(const pcv_batch_desc& d, cudaStream_t s)
{
    if (d.n_out == 0) return cudaSuccess;
    cudaError_t e = ensure_smem_attr();
    if (e != cudaSuccess) return e;
    const int tilesz = kThreads / tile_splits(d.n);
    const int64_t tiles = (d.n_out + tilesz - 1) / tilesz;
    glynn_tile_kernel<<<(unsigned)tiles, kThreads, sizeof(TileShared), s>>>(d);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_glynn_tile_multi(const pcv_batch_desc& d, int B, cudaStream_t s)
{
    if (d.n_out == 0 || B == 0) return cudaSuccess;
    cudaError_t e = ensure_smem_attr();
    if (e != cudaSuccess) return e;
    const int tilesz = kThreads / tile_splits(d.n);
    const int64_t tiles = (d.n_out + tilesz - 1) / tilesz;
    glynn_tile_multi_kernel<<<dim3((unsigned)tiles, (unsigned)B), kThreads, sizeof(TileShared), s>>>(
        d, (int64_t)d.m * d.m, d.n_out);
    note_launches(1);
    return cudaGetLastError();
}

// Workspace of the batched launch: counters, per-circuit arrays, the routed
// output lists and the tile items.
int64_t batched_workspace(int n_circ, int64_t total_outputs)
{
    const int64_t max_items = total_outputs / 32 + n_circ + 1;
    return (int64_t)(al256(4 * sizeof(int)) + 6 * al256((size_t)n_circ * sizeof(int)) +
                     al256((size_t)n_circ * sizeof(int64_t)) + 3 * al256((size_t)total_outputs * sizeof(int)) +
                     2 * al256((size_t)max_items * sizeof(int)));
}

cudaError_t launch_glynn_batched(const pcv_batch_desc* descs, int n_circ, int64_t total_outputs, void* ws,
                                 int sms, int route, cudaStream_t s)
{
    cudaError_t e = ensure_smem_attr();
    if (e != cudaSuccess) return e;
    const int64_t max_items = total_outputs / 32 + n_circ + 1;
    char* w = (char*)ws;
    int* counters = (int*)w;                          w += al256(4 * sizeof(int));
    int* order = (int*)w;                             w += al256((size_t)n_circ * sizeof(int));
    int* item_off = (int*)w;                          w += al256((size_t)n_circ * sizeof(int));
    int* mult_off = (int*)w;                          w += al256((size_t)n_circ * sizeof(int));
    int* n_tile = (int*)w;                            w += al256((size_t)n_circ * sizeof(int));
    int* n_mult = (int*)w;                            w += al256((size_t)n_circ * sizeof(int));
    w += al256((size_t)n_circ * sizeof(int));
    int64_t* out_off = (int64_t*)w;                   w += al256((size_t)n_circ * sizeof(int64_t));
    int* idx = (int*)w;                               w += al256((size_t)total_outputs * sizeof(int));
    int* mult_circ = (int*)w;                         w += al256((size_t)total_outputs * sizeof(int));
    int* mult_out = (int*)w;                          w += al256((size_t)total_outputs * sizeof(int));
    int* item_circ = (int*)w;                         w += al256((size_t)max_items * sizeof(int));
    int* item_tile = (int*)w;
    Queue q;
    q.counter = counters;
    q.total = counters + 1;
    q.item_circ = item_circ;
    q.item_tile = item_tile;
    q.out_off = out_off;
    q.n_tile = n_tile;
    q.idx = idx;
    MultQueue mq;
    mq.counter = counters + 2;
    mq.total = counters + 3;
    mq.circ = mult_circ;
    mq.out = mult_out;

    offsets_kernel<<<1, 1024, 0, s>>>(descs, n_circ, out_off);
    classify_kernel<<<n_circ, 256, 0, s>>>(descs, out_off, route, total_outputs, idx, n_tile, n_mult);
    plan_kernel<<<1, 1024, 0, s>>>(descs, n_circ, q, mq, order, item_off, mult_off, n_mult, mult_circ, mult_out,
                                   (int)max_items);
    note_launches(3);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, glynn_persistent_kernel, kThreads, sizeof(TileShared));
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    glynn_persistent_kernel<<<sms * per_sm, kThreads, sizeof(TileShared), s>>>(descs, q);
    note_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_glynn_mult_persistent(descs, mq, sms, s);
}

}  // namespace pcv
