/*
 * pcv: GB300 (sm_103a) strong simulation of linear-optical interferometers.
 *
 * C ABI of the CUDA library libpcv.so.  Everything the library computes is
 * defined by Eq. eqperm (Sec. 4.2 of the Perceval paper, arXiv 2204.00602):
 * for an m x m matrix U (row = output mode, column = input mode), an input
 * occupation t and an output occupation s with the same photon number n,
 * U_{T,S} is the n x n matrix holding s_i copies of row i of U and then t_j
 * copies of column j, and the output amplitude is
 *
 *     a(S) = Perm(U_{T,S}) / sqrt(s_1! ... s_m! t_1! ... t_m!),   P(S) = |a(S)|^2.
 *
 * The Naive back-end of Sec. 3.2.3 evaluates this per (input, output) pair
 * ("prob", "probampli"); the SLOS back-end returns every output at once
 * ("allstateprob_iterator").  pcv_amplitudes and pcv_distribution are the
 * GPU counterparts of those two calls.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Complex numbers are pcv_c64 {re, im}, the layout of torch.complex128 and
 *    C99 double complex.  Device arrays of pcv_c64 must be 16-byte aligned.
 *  - U is row-major m x m, U[out_mode * m + in_mode].  It is not checked for
 *    unitarity (the permanent is defined for any matrix).
 *  - Pointers documented as "device" are CUDA device pointers owned by the
 *    caller; the library never frees or keeps them after the call returns.
 *    Pointers documented as "host" are read during the call only.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Compute
 *    calls enqueue kernels on it and return without synchronising; results
 *    are valid once the stream reaches that point.
 *  - `workspace` is caller-owned device scratch of `workspace_bytes` bytes
 *    (query the size with the matching *_workspace call).  The library
 *    allocates no device memory itself.  A workspace may be reused by
 *    consecutive calls on the same stream but not by calls that overlap.
 *  - Every function returns PCV_OK (0) or a negative PCV_E* code; the message
 *    of the last failure on the calling host thread is pcv_last_error().
 *    Argument errors are reported before anything is enqueued.
 *  - An output whose photon number differs from the input's has amplitude 0
 *    (linear optics conserves photon number).  n = 0 gives amplitude 1 for
 *    the empty output.
 */
#ifndef PCV_H
#define PCV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } pcv_c64;

enum {
    PCV_OK = 0,
    PCV_EINVAL = -1,      /* bad argument: sizes, null pointer, alignment       */
    PCV_ERANGE = -2,      /* the output space or an index does not fit in int64 */
    PCV_ECUDA = -3,       /* a CUDA runtime call or kernel launch failed        */
    PCV_ETIMEOUT = -4,    /* a bounded device loop gave up                      */
    PCV_ENOMEM = -5,      /* the workspace passed is smaller than required      */
};

#define PCV_MAX_PHOTONS 30   /* n <= 30 (the paper's practical limit of Naive, Table 2) */
#define PCV_MAX_MODES 1024

/* ----------------------------------------------------------- host helpers */

/* Message of the last error on this host thread ("" if none).  The pointer
 * stays valid until the next failing call on the same thread. */
const char* pcv_last_error(void);

/* Library version string, e.g. "pcv 0.1 sm_103a". */
const char* pcv_version(void);

/* |S_{m,n}| = C(m+n-1, n), the number of n-photon output states over m modes
 * (Sec. 4.2, the output space S_{m,n}).  Returns PCV_EINVAL for m < 1 or
 * n < 0 and PCV_ERANGE if it exceeds 2^62. */
int64_t pcv_num_outputs(int m, int n);

/* Canonical order of S_{m,n}: lexicographic order of the non-decreasing list
 * of occupied modes (one entry per photon).  pcv_unrank writes the occupation
 * of output `idx` to occ_out[m] (host); pcv_rank returns the index of the
 * occupation occ[m] (host) or a negative error. */
int pcv_unrank(int m, int n, int64_t idx, uint8_t* occ_out);
int64_t pcv_rank(int m, const uint8_t* occ);

/* ------------------------------------------------------ amplitude kernels */

/* Algorithm selectors for the *_ex calls. */
enum {
    PCV_ALGO_AUTO = 0,
    PCV_ALGO_GROUP = 1,   /* plain Glynn, G threads per permanent (G = 1..32), n <= 16  */
    PCV_ALGO_BLOCK = 2,   /* plain Glynn, one block (x splits) per permanent, n <= 30   */
    PCV_ALGO_FACTOR = 3,  /* factorised Glynn sum over the whole output space           */
    PCV_ALGO_TILE = 4,    /* shared row sums, one block per tile of outputs, m <= 128   */
    PCV_ALGO_SLOS = 5,    /* full distribution by photon-by-photon state expansion      */
    PCV_ALGO_MULT = 6,    /* Glynn's sum with multiplicities, a warp (or more) per permanent */
    PCV_ALGO_FACTOR_TC = 7, /* factorised Glynn sum, products on the tensor cores (exact digits) */
};

/* Workspace bytes pcv_amplitudes needs for these sizes (0 if none). */
int64_t pcv_amplitudes_workspace(int m, int n, int64_t n_out);

/* Amplitudes a(S) of explicit outputs (Eq. eqperm; the Naive back-end's
 * probampli of Sec. 3.2.3).
 *   U          device, m*m pcv_c64, row = output mode
 *   m          1..PCV_MAX_MODES
 *   input_occ  host, m uint8, photon number n = sum <= PCV_MAX_PHOTONS
 *   output_occ device, n_out*m uint8, row-major (output o at output_occ + o*m)
 *   n_out      >= 0 (0 = nothing to do)
 *   amp        device, n_out pcv_c64 (written)
 *   prob       device, n_out double (written) or NULL
 * The permanent is Glynn's formula, Perm(A) = 2^{-(n-1)} sum over sign
 * vectors d with d_1 = +1 of (prod_k d_k) prod_i sum_j d_j a_ij, with the
 * sign vectors visited in reflected Gray-code order so each step updates the
 * row sums by one column (Sec. 3.2.3 names Glynn's algorithm).  The kernel
 * is chosen from m, n and n_out: with m <= 128 and enough outputs to fill
 * the GPU, the shared-row-sum tile kernel (n <= 12), or for n >= 13 a
 * per-output choice between the tile kernel and Glynn's sum with
 * multiplicities (PCV_ALGO_MULT below), whichever issues fewer FP64
 * instructions for that output; otherwise the plain Glynn kernels. */
int pcv_amplitudes(const pcv_c64* U, int m, const uint8_t* input_occ,
                   const uint8_t* output_occ, int64_t n_out,
                   pcv_c64* amp, double* prob,
                   void* workspace, int64_t workspace_bytes, void* stream);

/* pcv_amplitudes with an explicit algorithm: algo = PCV_ALGO_GROUP with
 * `param` threads per permanent (1, 2, 4, 8, 16 or 32), PCV_ALGO_BLOCK with
 * `param` blocks per permanent (>= 1), PCV_ALGO_TILE (m <= 128; the row
 * sums y_r(d) = sum_j d_j U[r][c_j] of each sign vector are formed once per
 * block and shared by its 32..256 outputs), or PCV_ALGO_MULT with `param`
 * warps per permanent (1..1024; 0 = chosen from n_out).
 * PCV_ALGO_MULT is Glynn's sum written over the multiplicities of a bunched
 * state (the same identity as above, with the sign vectors of the mu copies
 * of a repeated line grouped by their number k of minus signs):
 *   Perm = 2^{-n} sum_{k_j=0..mu_j} prod_j (-1)^{k_j} C(mu_j,k_j)
 *          prod_i (sum_j (mu_j - 2 k_j) M[j][i])^{e_i},
 * with j over the distinct modes of one side (the output or the input,
 * whichever gives fewer terms) and i over those of the other; prod (mu_j+1)
 * terms, halved by the symmetry k -> mu - k, instead of 2^{n-1}.  The paper
 * states no such variant; it serves outputs with several photons per mode.
 * PCV_ALGO_AUTO ignores param.  Workspace: pcv_amplitudes_ex_workspace. */
int pcv_amplitudes_ex(const pcv_c64* U, int m, const uint8_t* input_occ,
                      const uint8_t* output_occ, int64_t n_out,
                      pcv_c64* amp, double* prob, int algo, int param,
                      void* workspace, int64_t workspace_bytes, void* stream);

/* Workspace bytes pcv_amplitudes_ex needs for this algorithm and param
 * (0 if none; negative error code for an invalid choice). */
int64_t pcv_amplitudes_ex_workspace(int m, int n, int64_t n_out, int algo, int param);

/* One circuit of a batched call.  All pointers are device pointers; the
 * descriptor array itself lives in device memory and is only read. */
typedef struct {
    const pcv_c64* U;        /* m*m, row = output mode                               */
    const uint8_t* outputs;  /* n_out*m output occupations                           */
    pcv_c64* amp;            /* n_out amplitudes (written), or NULL                  */
    double* prob;            /* n_out probabilities (written), or NULL               */
    int64_t n_out;           /* >= 0                                                 */
    int32_t m;               /* 1..128                                               */
    int32_t n;               /* 1..PCV_MAX_PHOTONS photons                           */
    int32_t cols[PCV_MAX_PHOTONS];  /* photon -> input mode, non-decreasing, < m    */
} pcv_batch_desc;

/* Workspace bytes of pcv_amplitudes_batched for n_circ circuits holding
 * total_outputs outputs in all. */
int64_t pcv_amplitudes_batched_workspace(int n_circ, int64_t total_outputs);

/* Amplitudes of many circuits of uneven size (Eq. eqperm per circuit).
 * A routing kernel sends each output either to the shared-row-sum tile
 * kernel or to Glynn's sum with multiplicities (PCV_ALGO_MULT), whichever
 * issues fewer FP64 instructions for it; a planning kernel sorts the circuits
 * by photon number (largest first) and expands them into tile items
 * (circuit, tile of 32..256 outputs) and single-output entries.  Two
 * persistent launches then pull from device counters until their queues are
 * empty: blocks take tile items, warps take entries.  No block waits on
 * another.
 *   descs          device, n_circ descriptors (see pcv_batch_desc)
 *   total_outputs  sum of n_out over the circuits (<= INT32_MAX; sizes the
 *                  work lists)
 * A descriptor with n or m out of range, input modes outside [0, m) or out
 * of order, or outputs beyond total_outputs, is skipped (its outputs are not
 * written). */
int pcv_amplitudes_batched(const pcv_batch_desc* descs, int n_circ, int64_t total_outputs,
                           void* workspace, int64_t workspace_bytes, void* stream);

/* pcv_amplitudes_batched with the routing fixed: algo = PCV_ALGO_AUTO (per
 * output, as above), PCV_ALGO_TILE (every output to the tile kernel) or
 * PCV_ALGO_MULT (every output to Glynn's sum with multiplicities).  Same
 * workspace. */
int pcv_amplitudes_batched_ex(const pcv_batch_desc* descs, int n_circ, int64_t total_outputs, int algo,
                              void* workspace, int64_t workspace_bytes, void* stream);

/* Workspace bytes of pcv_distribution_ex with PCV_ALGO_FACTOR_TC (1 <= n <= 10;
 * e = min(3, n/2)): per side the digit tensor (48 bytes per entry and sign
 * vector) of the table levels e+1 .. n-e-1, of the level n-e entries and of
 * the e-photon column vectors, their exponents, the FP64 entries of the
 * parent levels 1 .. n-e-1, the entry and seam data of the level n-e entries
 * and column vectors, and two FP64 values per output. */
int64_t pcv_distribution_tc_workspace(int m, int n);

/* Workspace bytes pcv_distribution needs for m modes and n photons with the
 * default plan: for 2 <= n <= 10 and m >= 2 the single-pass plan of the
 * tensor-core products (= pcv_distribution_tc_workspace), otherwise the FP64
 * plan.  A smaller workspace (>= pcv_distribution_workspace_min) is accepted:
 * pcv_distribution then takes the FP64 products, in more passes if needed. */
int64_t pcv_distribution_workspace(int m, int n);
int64_t pcv_distribution_workspace_min(int m, int n);

/* The algorithm pcv_distribution (PCV_ALGO_AUTO) runs for m modes, n photons
 * and a workspace of workspace_bytes: PCV_ALGO_FACTOR_TC when 2 <= n <= 10,
 * m >= 2 and workspace_bytes >= pcv_distribution_tc_workspace(m, n), else
 * PCV_ALGO_FACTOR.  Both give the same amplitudes to double precision.  Returns
 * the algorithm code, or PCV_EINVAL for sizes out of range.  No counterpart in
 * the paper. */
int pcv_distribution_auto_algo(int m, int n, int64_t workspace_bytes);

/* Every output of S_{m,n} in canonical order (the SLOS back-end's full
 * distribution, Sec. 3.2.3, computed here from Eq. eqperm).
 *   prob  device, C(m+n-1,n) doubles (written) or NULL
 *   amp   device, C(m+n-1,n) pcv_c64 (written) or NULL; not both NULL
 * The algorithm factorises Glynn's sum: with sign vectors on the input
 * photons, every output shares the per-mode row sums
 * y_r(d) = sum_j d_j U[r][c_j], and a(S) = sum_d (sign, scale) prod_r y_r(d)^{s_r};
 * the product splits into the modes below and above m/2, so each output costs
 * one complex multiply-add per sign vector.  Those products run on the tensor
 * cores in exact integer arithmetic (PCV_ALGO_FACTOR_TC below) when the input
 * has 2..10 photons and the workspace holds that plan, else as FP64 multiply-
 * adds (PCV_ALGO_FACTOR); pcv_distribution_auto_algo tells which. */
int pcv_distribution(const pcv_c64* U, int m, const uint8_t* input_occ,
                     double* prob, pcv_c64* amp,
                     void* workspace, int64_t workspace_bytes, void* stream);

/* The outputs of pcv_distribution with canonical index in [begin, end), for
 * splitting one distribution across devices or processes (each takes a
 * contiguous range of the canonical order, 0 <= begin <= end <=
 * C(m+n-1,n)).  Output i is written at prob[i - begin] and amp[i - begin]
 * (end - begin entries each; either may be NULL, not both).  Same algorithm
 * choice, workspace and errors as pcv_distribution, and the same result for
 * every output, bit for bit: the ranges of a partition of [0, C(m+n-1,n))
 * together give exactly pcv_distribution's arrays.  Work scales with the
 * range for the products; the per-mode row sums and factor tables (13 % of
 * the time at m=20, n=10 with the tensor-core products, 7 % with the FP64
 * products) are built whole by every call.  The paper
 * has no counterpart (its workers split samples, Sec. 4.2). */
int pcv_distribution_range(const pcv_c64* U, int m, const uint8_t* input_occ, int64_t begin, int64_t end,
                           double* prob, pcv_c64* amp, void* workspace, int64_t workspace_bytes, void* stream);

/* Host-only view of how pcv_distribution_range splits its work.  Let P be
 * the photons of an output in modes [0, h), h = max(1, m / 2), a multiset of
 * size k ranked at its level k in canonical order.  The outputs sharing P
 * form one contiguous block of the canonical order, and at a fixed k the
 * blocks follow P's rank, so [begin, end) meets the blocks of the P of ranks
 * [pa[k], pb[k]) at each k = 0..n (empty when pa[k] == pb[k]); those are the
 * rows or columns of the products the range computes.  pa, pb: host arrays of
 * n + 1 entries (written).  Errors as pcv_distribution_range. */
int pcv_distribution_range_plan(int m, int n, int64_t begin, int64_t end, int64_t* pa, int64_t* pb);

/* Host-only view of the output blocks PCV_ALGO_FACTOR_TC's products run for
 * the outputs [begin, end) (end < 0: all), for inspection and tests.  With
 * h = max(1, m/2) and e = min(3, n/2), each side s (0: modes [0, h), 1:
 * [h, m)) has a digit tensor whose entries are, in order, the table levels
 * e+1 .. n-e-1 (each lexicographic), the level n-e entries (side 0 grouped
 * by largest mode ascending, side 1 by smallest mode ascending, each group
 * lexicographic) and the e-photon vectors over all m modes (side 0's tensor
 * grouped by largest mode ascending, side 1's by smallest mode descending).
 * out (host int64): 48 header values, then 16 per block.  Header: e, n-e, h,
 * blocks, tiles, vectors per tensor, level-(n-e) offsets [2], counts [2],
 * vector offsets [2], entries per tensor [2], then at 16 + 16 s + k the offset
 * of level k in side s's tensor (-1: not in it).  Block: kind (0: level
 * product, 1: extension block), rows_low (1: rows from side 0's tensor,
 * columns from side 1's), tile width, rows [rows0, rows) and columns [cols0,
 * cols) of the block, entry offsets of row 0 and column 0, lowoff, seam list
 * of the rows and of the columns (0, 1: level n-e of side 0, 1; 2, 3: the
 * vectors in side 0's, 1's tensor), cge (1: a pair is an output when the
 * column's seam mode >= the row's; 0: <=), seam index of row 0 and of column
 * 0, first tile.  needed (host, or NULL) receives the values out must hold;
 * out may be NULL to ask for it.  PCV_EINVAL outside 2 <= n <= 10, m >= 2,
 * or for a bad range or a short out.  No counterpart in the paper. */
int pcv_distribution_tc_blocks(int m, int n, int64_t begin, int64_t end, int64_t* out, int64_t out_len,
                               int64_t* needed);

/* Full distributions of B unitaries with the same input state (the
 * factorised algorithm of pcv_distribution, all B in the same launches).
 *   U     device, B*m*m pcv_c64 (entry b at U + b*m*m)
 *   B     1..65535
 *   prob  device, B*C(m+n-1,n) doubles or NULL; amp likewise pcv_c64 or NULL
 *         (entry b's outputs start at b*C(m+n-1,n)). */
int64_t pcv_distribution_batched_workspace(int B, int m, int n);
int pcv_distribution_batched(const pcv_c64* U, int B, int m, const uint8_t* input_occ,
                             double* prob, pcv_c64* amp,
                             void* workspace, int64_t workspace_bytes, void* stream);

/* Full distributions by photon-by-photon state expansion, the computation the
 * paper's SLOS back-end unfolds (Sec. 3.2.3: O(n C(m+n-1, n)) time and
 * memory).  Photons are created one at a time:
 *     B_k(s) = sum_{r: s_r >= 1} U[r][c_k] sqrt(s_r) B_{k-1}(s - e_r),  B_0 = 1,
 * and a(S) = B_n(S) / sqrt(prod t!) gives Eq. eqperm's amplitudes in canonical
 * order; level k keeps C(m+k-1, k) complex values.  Layouts as
 * pcv_distribution_batched (U [B][m][m], outputs [B][C(m+n-1,n)]). */
int64_t pcv_distribution_slos_workspace(int B, int m, int n);
int pcv_distribution_slos(const pcv_c64* U, int B, int m, const uint8_t* input_occ,
                          double* prob, pcv_c64* amp,
                          void* workspace, int64_t workspace_bytes, void* stream);

/* pcv_distribution with an explicit algorithm: PCV_ALGO_FACTOR (param
 * ignored), PCV_ALGO_GROUP (param = threads per permanent; unranks each
 * output), PCV_ALGO_BLOCK (param = blocks per permanent), PCV_ALGO_SLOS
 * (state expansion; workspace of pcv_distribution_slos_workspace(1, m, n)),
 * or PCV_ALGO_FACTOR_TC (workspace of pcv_distribution_tc_workspace).
 *
 * PCV_ALGO_FACTOR_TC computes the factorised sum's complex products over the
 * 2^{n-1} sign vectors on the BF16 tensor cores with exact integer
 * arithmetic.  Every FP64 table value is split into 8 balanced base-128
 * digits under a per-row power-of-two scale (the error-free splitting of
 * Ozaki, Ogita, Oishi and Rump, 2012); digit products are exact in BF16 and
 * each diagonal of digit pairs sums to at most 2^24, so its FP32 tensor-core
 * accumulation is exact; the diagonals are recombined in 64-bit integers and
 * rounded once to FP64 (round to nearest even) with integer operations.
 * With k photons on the low side (modes [0, h)) and e = min(3, n/2), the
 * outputs with k = e+1 .. n-e-1 are products of table levels k and n-k; an
 * output with at least n-e photons on one side is R ++ E, R its n-e photons
 * of that side nearest the other side (a level n-e entry) and E the other e
 * (an e-multiset over all modes, v_E = prod y_x / sqrt(prod mult!)), so no
 * table level above n-e is built.  With n = 1 or m = 1 the outputs with
 * every photon on one side run in FP64.  Results agree with the FP64 path
 * to double precision.  The paper has no such variant (its back-ends
 * run on CPUs).  n <= 10 (2^{n-1} <= 512 keeps each diagonal sum below 2^24). */
int pcv_distribution_ex(const pcv_c64* U, int m, const uint8_t* input_occ,
                        double* prob, pcv_c64* amp, int algo, int param,
                        void* workspace, int64_t workspace_bytes, void* stream);

/* The same explicit outputs for B unitaries with one input state (the tile
 * kernel of PCV_ALGO_TILE with a batch dimension; m <= 128, n >= 1).
 *   U       device, B*m*m pcv_c64;  output_occ device, n_out*m uint8
 *   amp     device, B*n_out pcv_c64 or NULL;  prob device, B*n_out doubles or NULL */
int pcv_amplitudes_multi(const pcv_c64* U, int B, int m, const uint8_t* input_occ,
                         const uint8_t* output_occ, int64_t n_out, pcv_c64* amp, double* prob, void* stream);

/* ------------------------------------------------------------- sampling */

/* Exact boson sampling: `count` independent output states drawn from P(S)
 * (Eq. eqperm), by the algorithm of the paper's CliffordClifford2017 back-end
 * (Sec. 3.2.3): with the input photons' columns of U in a random order,
 * photon k lands in mode i with weight
 *     | sum_{l<k} U[i][c_l] Perm(U[r_1..r_{k-1}; c_0..c_{k-1} without c_l]) |^2,
 * the k leave-one-out permanents computed together by one Glynn sum.
 *   U         device, m*m pcv_c64; m <= 128
 *   input_occ host, m uint8; 1 <= n <= 16 photons
 *   perm      device, count*n uint8: a permutation of 0..n-1 per sample
 *   uniforms  device, count*n doubles in [0, 1): one per photon and sample
 *   samples   device, count*m uint8 occupations (written)
 * The random numbers are inputs: a sample is a deterministic function of
 * (U, input, perm, uniforms). */
int pcv_sample(const pcv_c64* U, int m, const uint8_t* input_occ, const uint8_t* perm, const double* uniforms,
               int64_t count, uint8_t* samples, void* stream);

/* ------------------------------------------ partially distinguishable photons */

/* The paper's Processor takes a source with a transmittance and an
 * indistinguishability (Sec. processors), and its Hong-Ou-Mandel experiment
 * (Sec. hom) simulates such a source; it states no formula. The readings
 * here: photons of one class are identical, photons of different classes are
 * perfectly distinguishable (orthogonal internal states), and detectors
 * count photons per mode. Then
 *   P(S) = sum over S_1 + ... + S_G = S of prod_g P_g(S_g),
 * each P_g being Eq. eqperm for class g alone (a multiset convolution). */

/* Workspace bytes of pcv_distribution_classes. */
int64_t pcv_distribution_classes_workspace(int m, int G, const uint8_t* class_occ);

/* Distribution over S_{m,n} (canonical order) of G photon classes.
 *   U          device, m*m pcv_c64
 *   class_occ  host, G*m uint8: class g's input occupation at class_occ + g*m;
 *              n = total photons <= PCV_MAX_PHOTONS; empty classes allowed
 *   prob       device, C(m+n-1, n) doubles (written)
 * Each class's distribution is the factorised Glynn path's; one-photon
 * classes are folded in by a gather over the occupied modes,
 * C(S) = sum_{r: s_r >= 1} A(S - e_r) |U[r][c]|^2, larger ones by a
 * sub-multiset convolution. Errors: PCV_EINVAL, PCV_ERANGE, PCV_ENOMEM. */
int pcv_distribution_classes(const pcv_c64* U, int m, int G, const uint8_t* class_occ, double* prob,
                             void* workspace, int64_t workspace_bytes, void* stream);

/* Entries of the photon-number-resolved output space: sum_{k=0..n} C(m+k-1, k). */
int64_t pcv_distribution_source_size(int m, int n);

/* Workspace bytes of pcv_distribution_source. */
int64_t pcv_distribution_source_workspace(int m, const uint8_t* input_occ);

/* Output distribution of an imperfect source (n <= 16 photons): each photon
 * independently is absent (probability 1 - transmittance), pure
 * (transmittance * q) or noisy (transmittance * (1 - q)), with
 * q = sqrt(indistinguishability), so that two photons on a 50:50 beam
 * splitter show HOM visibility = indistinguishability. Pure photons form one
 * class, each noisy photon a class of its own; the result is the mixture
 * over all 2^n choices of the pure set, each folded with the other photons'
 * (absent or noisy) one-photon terms.
 *   prob  device, pcv_distribution_source_size(m, n) doubles (written): the
 *         blocks S_{m,0}, S_{m,1}, ..., S_{m,n} concatenated, each in
 *         canonical order; they sum to 1 together.
 * Errors: PCV_EINVAL (n > 16, parameters outside [0, 1]), PCV_ERANGE,
 * PCV_ENOMEM. */
int pcv_distribution_source(const pcv_c64* U, int m, const uint8_t* input_occ, double transmittance,
                            double indistinguishability, double* prob, void* workspace, int64_t workspace_bytes,
                            void* stream);

/* ------------------------------------------------------------ gradients */

/* dL/dU from dL/da for explicit outputs of one U, any n the forward calls
 * take (n <= 30).
 *   grad_amp  device, n_out pcv_c64: dL/dRe a + i dL/dIm a per output
 *   grad_U    device, m*m pcv_c64 (overwritten): dL/dRe U + i dL/dIm U
 *   workspace device, >= the minimum (pcv_amplitudes_backward_workspace(1, m,
 *             n, 1)); pcv_amplitudes_backward_workspace(1, m, n, n_out) is the
 *             default plan, and a smaller workspace runs the outputs in more
 *             chunks.
 * a(S) is holomorphic in U, so grad_U = sum_S grad_amp_S * conj(da_S/dU), and
 * da_S/dU[k][l] = norm_S * sum over (i, j) with r_i = k, c_j = l of the
 * permanent of the minor of (i, j) (the Laplace expansion of Eq. eqperm's
 * permanent), all minors of one output computed as Glynn sums over the
 * forward kernels' Gray-code row sums (one thread per output for n <= 6,
 * else one warp per output, or per part of its sign vectors for n > 14).
 * Every sum is taken in one fixed order (no
 * atomics), so repeated calls give the same bits.  Outputs whose photon number
 * differs from the input's contribute nothing. */
int64_t pcv_amplitudes_backward_workspace(int B, int m, int n, int64_t n_out);
int pcv_amplitudes_backward(const pcv_c64* U, int m, const uint8_t* input_occ,
                            const uint8_t* output_occ, int64_t n_out, const pcv_c64* grad_amp,
                            pcv_c64* grad_U, void* workspace, int64_t workspace_bytes, void* stream);

/* The same explicit outputs for B unitaries: grad_amp [B][n_out], grad_U
 * [B][m][m]; workspace from pcv_amplitudes_backward_workspace(B, m, n, n_out). */
int pcv_amplitudes_backward_multi(const pcv_c64* U, int B, int m, const uint8_t* input_occ,
                                  const uint8_t* output_occ, int64_t n_out, const pcv_c64* grad_amp,
                                  pcv_c64* grad_U, void* workspace, int64_t workspace_bytes, void* stream);

/* The same for every output of the distributions of B unitaries (grad_amp
 * [B][C(m+n-1,n)] in canonical order, grad_U [B][m][m]); the workspace
 * (default plan: pcv_distribution_backward_workspace(B, m, n)) also holds the
 * multiset-count table used to unrank outputs. */
int64_t pcv_distribution_backward_workspace(int B, int m, int n);
int pcv_distribution_backward(const pcv_c64* U, int B, int m, const uint8_t* input_occ,
                              const pcv_c64* grad_amp, pcv_c64* grad_U,
                              void* workspace, int64_t workspace_bytes, void* stream);

/* Clements rectangular MZI mesh (Sec. 2 cites the square decomposition;
 * components of Eq. bs and Table 1): m columns, column c holds MZIs on modes
 * (k, k+1), k = c mod 2, c mod 2 + 2, ...; MZI q uses phases[2q] (phase
 * shifter inside, on the upper mode) and phases[2q+1] (phase shifter after,
 * on the lower mode): MZI = diag(1, e^{i phi_b}) BS diag(e^{i phi_a}, 1) BS,
 * BS = (1/sqrt2)[[1, i], [i, 1]]; later MZIs multiply on the left.
 *   phases  device, B * m(m-1) doubles;  U device, B*m*m pcv_c64;  2 <= m <= 64.
 * pcv_mesh_backward takes U = pcv_mesh_unitary's output and grad_U = dL/dU
 * (dL/dRe + i dL/dIm) and writes dL/dphases [B][m(m-1)]. */
int pcv_mesh_unitary(const double* phases, int B, int m, pcv_c64* U, void* stream);
int pcv_mesh_backward(const double* phases, int B, int m, const pcv_c64* U, const pcv_c64* grad_U,
                      double* grad_phases, void* stream);

/* Per distribution b of B (p [B][N], q [N] or [B][N] when q_batched):
 * out[3b] = sum_S p(S), out[3b+1] = TVD(p, q) = 1/2 sum |p - q| (Eq.
 * bosonsampling), out[3b+2] = KL(q || p) = sum_{q>0} q log(q/p); q may be NULL
 * (sum only).  Deterministic (fixed reduction order). */
int64_t pcv_dist_stats_workspace(int B);
int pcv_dist_stats(const double* p, const double* q, int64_t N, int B, int q_batched, double* out,
                   void* workspace, int64_t workspace_bytes, void* stream);

/* Gradient of L = sum_b scale * w_b * KL(q || p_b) with respect to the
 * amplitudes: grad_amp = 2 a dL/dp, dL/dp = -scale w_b q / p (0 where q = 0);
 * batch_scale = w (device, B doubles) or NULL for w_b = 1. */
int pcv_kl_grad(const double* p, const double* q, const pcv_c64* amp, int64_t N, int B, int q_batched,
                const double* batch_scale, double scale, pcv_c64* grad_amp, void* stream);

/* grad_amp = 2 a grad_prob for p = |a|^2 (count elements). */
int pcv_prob_grad_to_amp(const double* grad_prob, const pcv_c64* amp, int64_t count, pcv_c64* grad_amp, void* stream);

/* ------------------------------------------------------ BF16 MLP surrogate */
/* No counterpart in the paper: kernels of the learned surrogate that maps
 * mesh phases to log-probabilities of a fixed output set.  All pointers are
 * device pointers; bf16 arrays are row-major with the given leading
 * dimensions (elements).
 *
 * pcv_gemm_bf16: C[M x N] = A[M x K] . B[N x K]^T on the tensor cores (BF16
 * operands, FP32 accumulation); K a multiple of 32, lda/ldb multiples of 8,
 * operands 16-byte aligned.  Epilogue `mode`:
 *   0  outf = C (fp32)
 *   1  pre = C + bias -> outf (fp32, optional), outb = bf16(GELU(pre)),
 *      GELU(x) = x/2 (1 + erf(x / sqrt 2))
 *   2  outf = C + bias (fp32)
 *   3  outb = bf16(C * GELU'(pre)), pre = the forward layer's pre-activation */
int pcv_gemm_bf16(const void* A, int lda, const void* B, int ldb, int M, int N, int K, int mode,
                  const float* bias, float* outf, int ldo, void* outb, int ldob, const float* pre, int ldp,
                  void* stream);
/* The same product on the 5th-generation tensor cores: TMA loads of 128 x 64
 * bf16 tiles (128-byte swizzle) into a 3-stage shared-memory ring,
 * tcgen05.mma (M = N = 128, K = 16) accumulating FP32 in tensor memory,
 * tcgen05.ld epilogue with the same `mode`s.  K must be a multiple of 8 (no
 * multiple of 32 needed: TMA zero-fills beyond K).  `error` (device int, may
 * be NULL) is set nonzero if a pipeline wait gave up (bounded polling); the
 * result is then invalid. */
int pcv_gemm_bf16_tc(const void* A, int lda, const void* B, int ldb, int M, int N, int K, int mode,
                     const float* bias, float* outf, int ldo, void* outb, int ldob, const float* pre, int ldp,
                     int* error, void* stream);
/* out[C x R] = in[R x C]^T (bf16). */
int pcv_transpose_bf16(const void* in, int R, int C, int ldi, void* out, int ldo, void* stream);
/* db[n] = sum_m dY[m][n] (bf16 in, fp32 out, fixed summation order). */
int pcv_colsum_bf16(const void* dY, int M, int N, int ld, float* db, void* stream);
/* X[b] = (sin phi_b, cos phi_b, 1, 0 ...) as bf16 rows of length ldx >= 2P+1;
 * the constant 1 carries the first layer's bias. */
int pcv_phase_features(const double* phases, int B, int P, void* X, int ldx, void* stream);
/* dL/dphi from dL/dX (fp32 [B][ldx]): dX_sin cos(phi) - dX_cos sin(phi). */
int pcv_phase_features_grad(const double* phases, int B, int P, const float* dX, int ldx, double* grad_phases,
                            void* stream);
/* loss = mean (pred - target)^2 over count elements (fp32); grad_pred_bf16 =
 * 2 (pred - target) / count as bf16, or NULL. */
int64_t pcv_mse_workspace(void);
int pcv_mse(const float* pred, const float* target, int64_t count, float* loss, void* grad_pred_bf16,
            void* workspace, int64_t workspace_bytes, void* stream);
/* Adam on fp32 master weights (bias-corrected with `step` >= 1); writes the
 * bf16 copy of the updated weights to w_bf16 when it is not NULL. */
int pcv_adam(float* w, float* m, float* v, const float* g, int64_t count, float lr, float beta1, float beta2,
             float eps, int step, void* w_bf16, void* stream);
int pcv_f32_to_bf16(const float* in, int64_t count, void* out, void* stream);
/* Adam on FP64 parameters (the mesh phases of the optimisation loops). */
int pcv_adam_f64(double* w, double* m, double* v, const double* g, int64_t count, double lr, double beta1,
                 double beta2, double eps, int step, void* stream);
/* out = (float) log(in) elementwise: log-probability targets of the surrogate. */
int pcv_log_f64_to_f32(const double* in, int64_t count, float* out, void* stream);
/* out = exp(in) elementwise in FP64: the surrogate's probabilities. */
int pcv_exp_f32_to_f64(const float* in, int64_t count, double* out, void* stream);

/* ------------------------------------------- distribution without allocation */

/* Size of the scratch array pcv_distribution_static uses: 32 MiB. */
#define PCV_STATIC_SCRATCH_BYTES (32ll << 20)

/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot call cudaMalloc, and it computes exactly what
 * pcv_distribution computes, with the same kernels.  Such callers include
 * plugins whose host application owns all device memory through its own
 * pool, and services that allow no allocation after start-up, so that no
 * call can fail for lack of memory or stall the device while it allocates.
 * They pass U and the output arrays as usual (device pointers they own) and
 * no workspace: the scratch is a 32 MiB array in the library's device code,
 * which every GPU that loads the library holds until the process exits.
 *   - The first call on a device looks up that device's address of the array
 *     (cudaGetSymbolAddress) with the device current; make that first call
 *     before any stream capture.
 *   - Problems whose scratch would exceed PCV_STATIC_SCRATCH_BYTES are
 *     rejected with PCV_ENOMEM (for example amp == NULL with an output space
 *     larger than about a million states).  The sign vectors are processed in
 *     as many passes as the array requires.
 *   - Every call, from every host thread and stream, shares the one array.
 *     Calls whose work overlaps on the GPU (different streams, or the same
 *     array used concurrently from several threads) race and give wrong
 *     results; serialise them on one stream.  Nothing in the array needs to
 *     start at zero: each call writes all it reads.
 *   - n must be >= 1.  Other arguments and errors as pcv_distribution. */
int pcv_distribution_static(const pcv_c64* U, int m, const uint8_t* input_occ,
                            double* prob, pcv_c64* amp, void* stream);
int64_t pcv_distribution_static_max_bytes(void);

/* ------------------------------------------------ failure detection */

/* Status of the last pcv_distribution / pcv_distribution_ex /
 * pcv_distribution_batched call that used `workspace` (device): waits for
 * `stream` (the call's stream), then returns PCV_OK, or PCV_ETIMEOUT when a
 * bounded wait inside the tensor-core product kernel gave up, in which case
 * the outputs of that call are not valid (pcv_last_error names the role that
 * gave up).  The first 256 bytes of a distribution workspace hold this status
 * word; each call sets it to zero before its kernels run.  The kernels never
 * wait on other blocks or devices, so a time-out means a stalled copy or
 * tensor-core operation inside one block; the block then waits, again with a
 * bound, for its own copies and MMAs in flight, releases its tensor memory and
 * returns.  No counterpart in the paper. */
int pcv_distribution_status(const void* workspace, void* stream);

/* Number of polls after which one mbarrier wait of the tensor-core kernels
 * (distribution products, pcv_gemm_bf16_tc) gives up: polls >= 1 sets it for
 * later launches, 0 restores each kernel's default (2^26 and 2^22 polls).  A
 * small value makes the waits run out, so the time-out path can be exercised
 * without a fault; it is a testing aid.  Returns PCV_OK or PCV_EINVAL (polls
 * < 0).  No counterpart in the paper. */
int pcv_set_wait_limit(int64_t polls);

/* -------------------------------------------------- measurement helpers */

/* FP64 throughput probe: `blocks` x `threads` threads each run `iters`
 * iterations of 8 independent DFMA chains and write one value to out[]
 * (device, blocks*threads doubles).  FLOPs = blocks*threads*iters*16.
 * Used to measure the FP64 roofline denominator. */
int pcv_fp64_probe(double* out, int blocks, int threads, int iters, void* stream);

/* Stage timing for measurement.  pcv_profile_enable(1) makes the library
 * record CUDA events on the launching stream around each stage of a call
 * (stage 0: factorised-distribution tables, with PCV_ALGO_FACTOR_TC their
 * digits too, 1: factorised-distribution products, 2: plain Glynn kernels,
 * 3: not recorded any more (kept so that stage numbers stay), 4: the FP64
 * single-entry blocks of PCV_ALGO_FACTOR_TC, n = 1 or m = 1 only).  pcv_profile_read waits for the recorded
 * events, writes the accumulated milliseconds and call counts of the first
 * `nstages` stages to ms[] and calls[] (host) and resets them.
 * pcv_launch_count returns the number of kernels the library has launched
 * since it was loaded.  No counterpart in the paper. */
int pcv_profile_enable(int on);
int pcv_profile_read(double* ms, int64_t* calls, int nstages);
int64_t pcv_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* PCV_H */
