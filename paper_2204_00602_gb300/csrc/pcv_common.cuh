// Shared device helpers of the CUDA path (complex FP64 arithmetic, multiset
// ranking, launch plumbing).  Internal to the library; the C ABI is in
// include/pcv.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pcv.h"

namespace pcv {

// ------------------------------------------------------------ complex FP64
// Complex values are double2 (x = real, y = imaginary); pcv_c64 and
// torch.complex128 have the same layout.

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// a * b: 2 DMUL + 2 DFMA
__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -(a.y * b.y)), fma(a.x, b.y, a.y * b.x));
}

// acc += a * b: 4 DFMA
__device__ __forceinline__ void cmac(double2& acc, double2 a, double2 b)
{
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}

// acc += s * a for a real scalar s: 2 DFMA
__device__ __forceinline__ void caxpy(double2& acc, double s, double2 a)
{
    acc.x = fma(s, a.x, acc.x);
    acc.y = fma(s, a.y, acc.y);
}

__device__ __forceinline__ double2 ld(const double2* p) { return __ldg(p); }

// -------------------------------------------------------- output space
// Multisets of size k over a modes: C(a+k-1, k).  The table MC[a*(kmax+1)+k]
// is built on the device (build_multiset_table) for a <= amax, k <= kmax and
// saturates at INT64_MAX.
struct MultisetTable {
    const int64_t* t;
    int kmax;
    __host__ __device__ __forceinline__ int64_t operator()(int a, int k) const { return t[a * (kmax + 1) + k]; }
};

// Canonical order of S_{w,k}: lexicographic order of the non-decreasing
// photon->mode list.  Unrank `idx` into modes[0..k) (values in [0, w)).
template <int KMAX>
__host__ __device__ __forceinline__ void unrank_multiset(MultisetTable mc, int w, int k, int64_t idx, int* modes)
{
    int v = 0;
    for (int p = 0; p < k; ++p) {
        const int rest = k - p - 1;
        for (;;) {
            const int64_t c = mc(w - v, rest);     // lists with this position = v
            if (idx < c) break;
            idx -= c;
            ++v;
        }
        modes[p] = v;
    }
}

// Rank of a non-decreasing mode list of length k over w modes.
__host__ __device__ __forceinline__ int64_t rank_multiset(MultisetTable mc, int w, int k, const int* modes)
{
    int64_t r = 0;
    int prev = 0;
    for (int p = 0; p < k; ++p) {
        const int rest = k - p - 1;
        for (int v = prev; v < modes[p]; ++v) r += mc(w - v, rest);
        prev = modes[p];
    }
    return r;
}

__device__ __forceinline__ double inv_sqrt_int(int k) { return 1.0 / sqrt((double)k); }

}  // namespace pcv

// Launch helpers implemented in the .cu files (host side).
namespace pcv {
struct Plan {           // host-side description of one (U, input) problem
    int m;
    int n;
    int cols[PCV_MAX_PHOTONS];     // input modes with repetition (photon -> input mode)
    double norm_t;                 // 1 / sqrt(prod t_j!)
};

cudaError_t build_multiset_table(int64_t* t, int amax, int kmax, cudaStream_t s);
// CUM[a*(kmax+1)+k] = sum_{v < a} MC[(m-v)*(kmax+1)+k] (a = 0..m): the rank of a
// sorted mode list of length k is sum_p CUM[mode_p][k-p-1] - CUM[mode_{p-1}][k-p-1]
// (slos.cu)
cudaError_t build_cum_table(const int64_t* mc, int m, int kmax, int64_t* cum, cudaStream_t s);

// Per-stage timing (pcv_api.cu): when enabled, stage_begin/stage_end record
// CUDA events on the launching stream around a group of launches; the times
// are read back by pcv_profile_read.  note_launches counts kernel launches.
enum Stage { kStageTables = 0, kStageGemm = 1, kStagePlain = 2, kStageSplit = 3, kStageEdge = 4, kStageCount = 8 };
void stage_begin(int stage, cudaStream_t s);
void stage_end(int stage, cudaStream_t s);
void note_launches(int64_t k);
void set_error(const char* msg);      // message returned by pcv_last_error
// Bound of one mbarrier wait in the tensor-core kernels: `dflt` unless
// pcv_set_wait_limit set another.
long long wait_limit(long long dflt);

// Plain Glynn kernels (glynn_plain.cu)
cudaError_t launch_glynn_group(const Plan& p, const double2* U, const uint8_t* out_occ,
                               const int64_t* mc_table, int64_t idx0, int64_t count,
                               double2* amp, double* prob, int G, cudaStream_t s);
cudaError_t launch_glynn_block(const Plan& p, const double2* U, const uint8_t* out_occ,
                               const int64_t* mc_table, int64_t idx0, int64_t count,
                               double2* amp, double* prob, int splits, double2* partial,
                               cudaStream_t s);
int glynn_block_threads();

// Shared-row-sum tile kernels (glynn_tile.cu)
__host__ __device__ int tile_splits(int n);
int tile_max_modes();
cudaError_t launch_glynn_tile(const pcv_batch_desc& d, cudaStream_t s);
cudaError_t launch_glynn_tile_multi(const pcv_batch_desc& d, int B, cudaStream_t s);
int64_t batched_workspace(int n_circ, int64_t total_outputs);
// copies a descriptor (passed by value) into device memory
cudaError_t launch_store_desc(const pcv_batch_desc& d, pcv_batch_desc* out, cudaStream_t s);
// route: PCV_ALGO_AUTO (per output, by FP64 instruction count), PCV_ALGO_TILE
// or PCV_ALGO_MULT (every output to that kernel)
cudaError_t launch_glynn_batched(const pcv_batch_desc* descs, int n_circ, int64_t total_outputs, void* ws,
                                 int sms, int route, cudaStream_t s);

// Glynn's sum with multiplicities (glynn_mult.cu).  side: 0 = fewer terms,
// 1 = sign vectors on the output modes, 2 = on the input modes.
struct MultQueue {
    int* counter;            // next entry
    int* total;              // entries
    const int* circ;         // circuit of entry e
    const int* out;          // output index of entry e within its circuit
};
cudaError_t launch_glynn_mult(const pcv_batch_desc& d, int parts, int side, double2* partial, cudaStream_t s);
cudaError_t launch_glynn_mult_persistent(const pcv_batch_desc* descs, const MultQueue& q, int sms, cudaStream_t s);

// Adjoint (adjoint.cu): the plan of one call (B batch entries, `count`
// outputs each) in a workspace of ws_bytes (< 0: the default budget): Gray
// sequence split in `parts` of part_steps, lanes per row q and columns per
// lane cj of the G matrix, outputs per chunk, and the bytes used.
struct AdjPlan {
    int parts;
    int64_t part_steps;
    int q, cj;
    size_t table;             // multiset table (canonical outputs)
    int64_t chunk;
    size_t total, min_total;  // bytes of this plan, of a one-output chunk
};
AdjPlan adjoint_plan(int m, int n, int B, int64_t count, int64_t ws_bytes);
int adjoint_max_photons();
// out_occ: explicit outputs [count][m] (device) or null for every output of
// S_{m,n} in canonical order; dL/dU [B][m][m] is overwritten.
cudaError_t launch_adjoint(const Plan& p, const double2* U, int B, const uint8_t* out_occ, int64_t count,
                           const double2* gbar, double2* gradU, void* ws, const AdjPlan& ap, cudaStream_t s);
// Mesh (mesh.cu), reductions (reduce.cu)
int mesh_max_modes();
cudaError_t launch_mesh_forward(const double* phases, int B, int m, double2* U, cudaStream_t s);
cudaError_t launch_mesh_backward(const double* phases, int B, int m, const double2* U, const double2* G,
                                 double* gphi, cudaStream_t s);
int64_t stats_workspace(int B);
cudaError_t launch_stats(const double* p, const double* q, int64_t N, int B, int q_batched, double* out,
                         double* ws, cudaStream_t s);
cudaError_t launch_kl_grad(const double* p, const double* q, const double2* amp, int64_t N, int B, int q_batched,
                           const double* bscale, double scale, double2* grad, cudaStream_t s);
cudaError_t launch_prob_grad(const double* gp, const double2* amp, int64_t count, double2* gamp, cudaStream_t s);

// Exact boson sampling (sampler.cu)
cudaError_t launch_sampler(const Plan& p, const double2* U, const uint8_t* perm, const double* uni, int64_t count,
                           uint8_t* out, cudaStream_t s);

// Partially distinguishable photons (distinguish.cu); mc and cum are the
// tables of S_{m,k} for k <= kmax.
cudaError_t launch_photon_step(const int64_t* mc, const int64_t* cum, int m, int kmax, int k, const double2* U, int c,
                               const double* in_same, const double* in_prev, double alpha, double beta, double* out,
                               int64_t count, cudaStream_t s);
cudaError_t launch_class_conv(const int64_t* mc, const int64_t* cum, int m, int kmax, int a, int b, const double* A,
                              const double* B, double* C, int64_t count, cudaStream_t s);
cudaError_t launch_scale_add(double* acc, const double* x, double w, int64_t count, cudaStream_t s);
cudaError_t launch_set_one(double* p, cudaStream_t s);

// Photon-by-photon state expansion (slos.cu)
int64_t slos_workspace(int B, int m, int n);
cudaError_t launch_slos(const Plan& p, int B, const double2* U, double* prob, double2* amp, void* ws, cudaStream_t s);

// Factorised full distribution (glynn_dist.cu)
struct DistPlan {
    int h;                    // modes [0,h) are the low side, [h,m) the high side
    int B;                    // batch entries (unitaries)
    int kc;                   // Glynn sign vectors per chunk
    int64_t total;            // outputs per batch entry
    int64_t wlow, whigh;      // entries of all levels per side: C(h+n, n), C(m-h+n, n)
    int64_t lowoff[PCV_MAX_PHOTONS + 2], highoff[PCV_MAX_PHOTONS + 2];
    size_t ws_status, ws_table, ws_base, ws_acc, ws_y, ws_tl, ws_sl, ws_th, ws_sh, ws_total;
    bool tc = false;          // products on the tensor cores (glynn_tc.cu)
    size_t ws_tc = 0;
    size_t ws_edge = 0;       // partial sums of the single-entry blocks (tensor-core plan)
    // The outputs computed: canonical indices [lo, hi) (the whole space by
    // default), written at prob[o - lo], amp[o - lo].
    int64_t lo = 0, hi = -1;
};

// Outputs in a canonical index range, grouped by the low-side multiset P
// (modes [0, h)): all outputs with low part P form one contiguous block of the
// canonical order, starting at lowbase(P) with msets(m - h, n - |P|) entries,
// and within one size k the blocks follow P's rank.  So [lo, hi) meets, for
// each k, the P of ranks [pa[k], pb[k]) at level k (empty when pa >= pb).
struct PRanges {
    int64_t pa[PCV_MAX_PHOTONS + 1], pb[PCV_MAX_PHOTONS + 1];
};
void p_ranges(int m, int n, int h, int64_t lo, int64_t hi, PRanges* r);
// canonical index of the first output whose low part is the level-k multiset of rank `rank`
int64_t host_lowbase(int m, int n, int h, int k, int64_t rank);
// rank at level k-1 of the level-k multiset of rank `rank` (over w modes) without its last mode
int64_t host_parent_rank(int w, int k, int64_t rank);
// The single-pass plan for the tensor-core products (B = 1): the FP64 tables
// of all sign vectors, an amplitude buffer when the caller wants
// probabilities only, and the digit tensors.  Returns the bytes, -1 on overflow.
int64_t dist_plan_tc(const Plan& p, bool need_amp_buffer, DistPlan* dp);
int64_t dist_plan(const Plan& p, int B, int64_t ws_bytes, bool need_acc, DistPlan* dp);

// Tables and products on the tensor cores with exact digit splitting
// (glynn_tc.cu): one batch entry, all K = 2^{n-1} <= 512 sign vectors in one
// pass, n >= 2 and both sides non-empty.  launch_tc_tables builds the table
// levels 1 .. n-e of both sides (e = min(3, n/2)) and the e-photon column
// vectors from the row sums and writes their digits (and lowbase of the low
// side); launch_tc_products runs every output block and writes amp / prob.
struct TcInputs {
    int K, n, m, h;
    int64_t lowoff[PCV_MAX_PHOTONS + 2], highoff[PCV_MAX_PHOTONS + 2];
    int64_t* lowbase;                             // low side, written by launch_tc_tables
    const double2* Y;                             // [K][m] row sums y_r(d)
    MultisetTable mc;                             // multiset counts (a <= m, k <= n)
    double lead;                                  // 2^{-(n-1)} norm_t
    int64_t total;                                // outputs
    double2* amp;                                 // amplitudes (written), or null
    double* prob;                                 // or null
    void* ws;                                     // tc_workspace bytes
    int* error;                                   // device flag, or null
    unsigned long long* next_tile;                // the products' tile counter, zero at the call's start
    int64_t lo, hi;                               // outputs [lo, hi), stored at [o - lo]
};
int tc_pad_k(int K);
int64_t tc_workspace(int m, int n, int h, int K, int64_t total);
cudaError_t launch_tc_tables(const TcInputs& in, cudaStream_t s);
constexpr int kTcPlanHeader = 48, kTcPlanBlock = 16;   // tc_block_list's record sizes
int64_t tc_block_list(int m, int n, int64_t lo, int64_t hi, int64_t* out, int64_t cap);
cudaError_t launch_tc_products(const TcInputs& in, cudaStream_t s);
cudaError_t launch_glynn_dist(const Plan& p, const DistPlan& dp, const double2* U,
                              double* prob, double2* amp, void* ws, cudaStream_t s);
}  // namespace pcv
