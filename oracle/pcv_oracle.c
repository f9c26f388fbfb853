/*
 * CPU FP64 oracle for linear-optical output amplitudes.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the CUDA path is checked against.  Only the tests, the smoke
 * check and the bench's CPU-baseline leg may load it.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * What it computes (Sec. 4.2, Eq. eqperm): for an m-mode unitary U (row =
 * output mode, column = input mode), input occupation t and output occupation
 * s with the same photon number n, the n x n matrix U_{T,S} takes s_i copies
 * of row i of U, then t_j copies of column j; the amplitude is
 *     a(S) = Perm(U_{T,S}) / sqrt(s_1! ... s_m! t_1! ... t_m!)
 * and P(S) = |a(S)|^2.
 *
 * The permanent is computed three ways:
 *   - Leibniz: the definition, sum over all n! permutations (small n only);
 *   - Ryser's formula (Sec. 3.2.3 names Ryser's and Glynn's algorithms):
 *       Perm(A) = (-1)^n sum_{S subset of columns} (-1)^{|S|} prod_i sum_{j in S} a_ij.
 *     Subsets are visited in reflected-Gray-code order so consecutive subsets
 *     differ by one column (the usual way Ryser's formula is evaluated); the
 *     row sums are recomputed from scratch at the start of every block of
 *     2^RYSER_BLOCK_BITS subsets so rounding does not drift, and the terms are
 *     added with Neumaier compensated summation;
 *   - the same Ryser sum in double-double arithmetic, for n >= 20 where the
 *     plain double sum loses digits to cancellation.
 *
 * Everything is plain IEEE double (double-double is built from doubles); compile without -ffast-math and with
 * -ffp-contract=off.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define RYSER_BLOCK_BITS 14

/* ---------------------------------------------------------------- Leibniz */

static cplx leibniz_rec(int n, const cplx* A, int row, uint64_t used, cplx prefix)
{
    if (row == n) return prefix;
    cplx s = 0;
    for (int j = 0; j < n; ++j)
        if (!(used & (1ull << j)))
            s += leibniz_rec(n, A, row + 1, used | (1ull << j), prefix * A[row * n + j]);
    return s;
}

/* Definition of the permanent: sum over permutations sigma of prod_i A[i][sigma(i)].
 * A is row-major n x n.  n <= 12 (n! terms). */
void oracle_perm_leibniz(int n, const double* A_ri, double* out_ri)
{
    const cplx* A = (const cplx*)A_ri;
    cplx p = (n == 0) ? 1.0 : leibniz_rec(n, A, 0, 0, 1.0);
    out_ri[0] = creal(p);
    out_ri[1] = cimag(p);
}

/* ------------------------------------------------------------------ Ryser */

typedef struct { double s, c; } nsum; /* Neumaier running sum */

static void nsum_add(nsum* a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else                       a->c += (x - t) + a->s;
    a->s = t;
}

/* Ryser terms for Gray-code indices k in [k0, k1): subset(k) = k ^ (k >> 1). */
static cplx ryser_block(int n, const cplx* A, uint64_t k0, uint64_t k1)
{
    cplx rs[64];
    uint64_t g = k0 ^ (k0 >> 1);
    for (int i = 0; i < n; ++i) {           /* row sums over the start subset, from scratch */
        rs[i] = 0;
        for (int j = 0; j < n; ++j)
            if (g & (1ull << j)) rs[i] += A[i * n + j];
    }
    nsum re = {0, 0}, im = {0, 0};
    for (uint64_t k = k0; k < k1; ++k) {
        if (k != k0) {                      /* subset(k) differs from subset(k-1) in one column */
            uint64_t gk = k ^ (k >> 1);
            int j = __builtin_ctzll(k);
            if (gk & (1ull << j)) for (int i = 0; i < n; ++i) rs[i] += A[i * n + j];
            else                  for (int i = 0; i < n; ++i) rs[i] -= A[i * n + j];
            g = gk;
        }
        if (g == 0) continue;               /* empty subset: all row sums are zero */
        cplx prod = 1.0;
        for (int i = 0; i < n; ++i) prod *= rs[i];
        int size = __builtin_popcountll(g);
        if (((n - size) & 1) != 0) prod = -prod;   /* (-1)^n (-1)^{|S|} */
        nsum_add(&re, creal(prod));
        nsum_add(&im, cimag(prod));
    }
    return (re.s + re.c) + I * (im.s + im.c);
}

/* Ryser's formula for an n x n complex matrix (row-major), n <= 40. */
void oracle_perm_ryser(int n, const double* A_ri, double* out_ri)
{
    const cplx* A = (const cplx*)A_ri;
    if (n == 0) { out_ri[0] = 1.0; out_ri[1] = 0.0; return; }
    uint64_t total = 1ull << n;
    uint64_t bs = (n > RYSER_BLOCK_BITS) ? (1ull << RYSER_BLOCK_BITS) : total;
    int64_t nblocks = (int64_t)(total / bs);
    cplx* part = (cplx*)malloc(sizeof(cplx) * (size_t)nblocks);
#ifdef _OPENMP
    int par = !omp_in_parallel() && nblocks >= 4;
#pragma omp parallel for schedule(dynamic, 1) if (par)
#endif
    for (int64_t b = 0; b < nblocks; ++b)
        part[b] = ryser_block(n, A, (uint64_t)b * bs, (uint64_t)(b + 1) * bs);
    nsum re = {0, 0}, im = {0, 0};          /* fixed order: deterministic for any thread count */
    for (int64_t b = 0; b < nblocks; ++b) { nsum_add(&re, creal(part[b])); nsum_add(&im, cimag(part[b])); }
    free(part);
    out_ri[0] = re.s + re.c;
    out_ri[1] = im.s + im.c;
}

/* -------------------------------------------------- Ryser, double-double */

/*
 * The same Ryser sum with every quantity held as an unevaluated sum of two
 * doubles, hi + lo (about 106 bits).  Ryser's terms can exceed the
 * permanent by many orders of magnitude, so in plain double the sum loses
 * digits (at n = 24, Ryser on A and on A^T can disagree in the 7th digit);
 * here the rounding error is ~1e-32 of the largest term.  The operations are
 * the published error-free transformations: Knuth's TwoSum (TAOCP Vol. 2,
 * Sec. 4.2.2) and Dekker's product with the exact remainder from a correctly
 * rounded fma, combined as in Dekker (1971) / Bailey's double-double
 * arithmetic.  Only IEEE double operations and fma() are used.
 */
typedef struct { double hi, lo; } dd;
typedef struct { dd re, im; } ddc;

static dd dd_two_sum(double a, double b)
{
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    dd r = {s, e};
    return r;
}

static dd dd_fast_two_sum(double a, double b)   /* needs |a| >= |b| or a == 0 */
{
    double s = a + b;
    dd r = {s, b - (s - a)};
    return r;
}

static dd dd_add(dd a, dd b)
{
    dd s = dd_two_sum(a.hi, b.hi);
    dd t = dd_two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = dd_fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return dd_fast_two_sum(s.hi, s.lo);
}

static dd dd_neg(dd a) { dd r = {-a.hi, -a.lo}; return r; }

static dd dd_mul(dd a, dd b)
{
    double p = a.hi * b.hi;
    double e = fma(a.hi, b.hi, -p);          /* exact remainder of the product */
    e += a.hi * b.lo + a.lo * b.hi;
    return dd_fast_two_sum(p, e);
}

static ddc ddc_add(ddc a, ddc b) { ddc r = {dd_add(a.re, b.re), dd_add(a.im, b.im)}; return r; }

static ddc ddc_mul(ddc a, ddc b)
{
    ddc r = {dd_add(dd_mul(a.re, b.re), dd_neg(dd_mul(a.im, b.im))),
             dd_add(dd_mul(a.re, b.im), dd_mul(a.im, b.re))};
    return r;
}

static ddc ddc_from(cplx z) { ddc r = {{creal(z), 0.0}, {cimag(z), 0.0}}; return r; }

static ddc ryser_block_dd(int n, const cplx* A, uint64_t k0, uint64_t k1)
{
    ddc rs[64];
    const ddc zero = {{0.0, 0.0}, {0.0, 0.0}};
    uint64_t g = k0 ^ (k0 >> 1);
    for (int i = 0; i < n; ++i) {
        rs[i] = zero;
        for (int j = 0; j < n; ++j)
            if (g & (1ull << j)) rs[i] = ddc_add(rs[i], ddc_from(A[i * n + j]));
    }
    ddc acc = zero;
    for (uint64_t k = k0; k < k1; ++k) {
        if (k != k0) {
            uint64_t gk = k ^ (k >> 1);
            int j = __builtin_ctzll(k);
            int add = (gk & (1ull << j)) != 0;
            for (int i = 0; i < n; ++i) rs[i] = ddc_add(rs[i], ddc_from(add ? A[i * n + j] : -A[i * n + j]));
            g = gk;
        }
        if (g == 0) continue;
        ddc prod = rs[0];
        for (int i = 1; i < n; ++i) prod = ddc_mul(prod, rs[i]);
        int size = __builtin_popcountll(g);
        if (((n - size) & 1) != 0) { prod.re = dd_neg(prod.re); prod.im = dd_neg(prod.im); }
        acc = ddc_add(acc, prod);
    }
    return acc;
}

/* Ryser's formula in double-double; the result rounded to double. */
void oracle_perm_ryser_dd(int n, const double* A_ri, double* out_ri)
{
    const cplx* A = (const cplx*)A_ri;
    if (n == 0) { out_ri[0] = 1.0; out_ri[1] = 0.0; return; }
    uint64_t total = 1ull << n;
    uint64_t bs = (n > RYSER_BLOCK_BITS) ? (1ull << RYSER_BLOCK_BITS) : total;
    int64_t nblocks = (int64_t)(total / bs);
    ddc* part = (ddc*)malloc(sizeof(ddc) * (size_t)nblocks);
#ifdef _OPENMP
    int par = !omp_in_parallel() && nblocks >= 4;
#pragma omp parallel for schedule(dynamic, 1) if (par)
#endif
    for (int64_t b = 0; b < nblocks; ++b)
        part[b] = ryser_block_dd(n, A, (uint64_t)b * bs, (uint64_t)(b + 1) * bs);
    ddc acc = {{0.0, 0.0}, {0.0, 0.0}};
    for (int64_t b = 0; b < nblocks; ++b) acc = ddc_add(acc, part[b]);
    free(part);
    out_ri[0] = acc.re.hi + acc.re.lo;
    out_ri[1] = acc.im.hi + acc.im.lo;
}

/* --------------------------------------------------------- Eq. eqperm */

static double factorial(int k)
{
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= (double)i;
    return f;
}

/* Build U_{T,S}: s_i copies of row i (output modes), then t_j copies of column j
 * (input modes).  Returns n, or -1 when the photon numbers differ. */
static int build_submatrix(int m, const cplx* U, const uint8_t* in_occ, const uint8_t* out_occ, cplx* A)
{
    int rows[64], cols[64], nr = 0, nc = 0;
    for (int i = 0; i < m; ++i) {
        nr += out_occ[i];
        nc += in_occ[i];
    }
    if (nr != nc || nr > 40) return -1;
    nr = nc = 0;
    for (int i = 0; i < m; ++i) for (int c = 0; c < out_occ[i]; ++c) rows[nr++] = i;
    for (int j = 0; j < m; ++j) for (int c = 0; c < in_occ[j]; ++c) cols[nc++] = j;
    for (int a = 0; a < nr; ++a)
        for (int b = 0; b < nc; ++b)
            A[a * nr + b] = U[(size_t)rows[a] * m + cols[b]];
    return nr;
}

static double occ_norm(int m, const uint8_t* in_occ, const uint8_t* out_occ)
{
    double d = 1.0;
    for (int i = 0; i < m; ++i) d *= factorial(out_occ[i]) * factorial(in_occ[i]);
    return 1.0 / sqrt(d);
}

/* a(S) for one output.  method: 0 = Ryser, 1 = Leibniz, 2 = Ryser in
 * double-double.  Different photon
 * numbers give 0 (linear optics conserves photon number). */
void oracle_amplitude(int m, const double* U_ri, const uint8_t* in_occ, const uint8_t* out_occ,
                      int method, double* out_ri)
{
    const cplx* U = (const cplx*)U_ri;
    cplx A[40 * 40];
    int n = build_submatrix(m, U, in_occ, out_occ, A);
    if (n < 0) { out_ri[0] = out_ri[1] = 0.0; return; }
    double p[2];
    if (method == 1)      oracle_perm_leibniz(n, (const double*)A, p);
    else if (method == 2) oracle_perm_ryser_dd(n, (const double*)A, p);
    else                  oracle_perm_ryser(n, (const double*)A, p);
    double nrm = occ_norm(m, in_occ, out_occ);
    out_ri[0] = p[0] * nrm;
    out_ri[1] = p[1] * nrm;
}

/* Batch over explicit outputs (row-major uint8 [n_out][m]); parallel over outputs. */
void oracle_amplitudes(int m, const double* U_ri, const uint8_t* in_occ, const uint8_t* out_occ,
                       int64_t n_out, int method, double* amp_ri)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t o = 0; o < n_out; ++o)
        oracle_amplitude(m, U_ri, in_occ, out_occ + o * m, method, amp_ri + 2 * o);
}

/* ------------------------------------------------- output space S_{m,n} */

/* |S_{m,n}| = C(m+n-1, n) by direct multiplicative evaluation; -1 on overflow. */
int64_t oracle_num_outputs(int m, int n)
{
    if (m < 1 || n < 0) return -1;
    unsigned __int128 c = 1;
    for (int k = 1; k <= n; ++k) {
        c = c * (unsigned __int128)(m - 1 + k) / (unsigned __int128)k;
        if (c > (unsigned __int128)INT64_MAX) return -1;
    }
    return (int64_t)c;
}

/* All outputs in canonical order: lexicographic order of the non-decreasing
 * list of occupied modes (photon -> mode).  Writes occupations [count][m]. */
int64_t oracle_enumerate(int m, int n, uint8_t* occ_out, int64_t cap)
{
    int modes[64];
    for (int i = 0; i < n; ++i) modes[i] = 0;
    int64_t count = 0;
    for (;;) {
        if (count < cap) {
            uint8_t* o = occ_out + count * m;
            memset(o, 0, (size_t)m);
            for (int i = 0; i < n; ++i) o[modes[i]]++;
        }
        ++count;
        int i = n - 1;                       /* rightmost position that can still grow */
        while (i >= 0 && modes[i] == m - 1) --i;
        if (i < 0) break;
        modes[i]++;
        for (int j = i + 1; j < n; ++j) modes[j] = modes[i];
    }
    return count;
}

/* Full distribution: amplitudes and probabilities of every output, canonical order. */
int oracle_distribution(int m, const double* U_ri, const uint8_t* in_occ, double* prob, double* amp_ri)
{
    int n = 0;
    for (int i = 0; i < m; ++i) n += in_occ[i];
    int64_t N = oracle_num_outputs(m, n);
    if (N < 0) return -1;
    uint8_t* occ = (uint8_t*)malloc((size_t)N * (size_t)m);
    if (!occ) return -2;
    oracle_enumerate(m, n, occ, N);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t o = 0; o < N; ++o) {
        double a[2];
        oracle_amplitude(m, U_ri, in_occ, occ + o * m, 0, a);
        if (amp_ri) { amp_ri[2 * o] = a[0]; amp_ri[2 * o + 1] = a[1]; }
        if (prob) prob[o] = a[0] * a[0] + a[1] * a[1];
    }
    free(occ);
    return 0;
}

/* ------------------------------------------------------------- gradients */

/* d a(S) / d U[k][l] for every k, l (a is holomorphic in U), written to
 * D_ri[m][m] complex.  By the Laplace expansion, dPerm(A)/dA_ij is the
 * permanent of A with row i and column j removed; U[k][l] sits at every (i, j)
 * with row i a copy of output mode k and column j a copy of input mode l. */
void oracle_amplitude_grad(int m, const double* U_ri, const uint8_t* in_occ, const uint8_t* out_occ,
                           double* D_ri)
{
    const cplx* U = (const cplx*)U_ri;
    cplx* D = (cplx*)D_ri;
    for (int64_t q = 0; q < (int64_t)m * m; ++q) D[q] = 0;
    cplx A[40 * 40], minor[40 * 40];
    int n = build_submatrix(m, U, in_occ, out_occ, A);
    if (n <= 0) return;
    int rows[64], cols[64], nr = 0, nc = 0;
    for (int i = 0; i < m; ++i) for (int c = 0; c < out_occ[i]; ++c) rows[nr++] = i;
    for (int j = 0; j < m; ++j) for (int c = 0; c < in_occ[j]; ++c) cols[nc++] = j;
    double nrm = occ_norm(m, in_occ, out_occ);
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            int mi = 0;
            for (int a = 0; a < n; ++a) {
                if (a == i) continue;
                int mj = 0;
                for (int b = 0; b < n; ++b) {
                    if (b == j) continue;
                    minor[mi * (n - 1) + mj] = A[a * n + b];
                    ++mj;
                }
                ++mi;
            }
            double p[2];
            oracle_perm_ryser(n - 1, (const double*)minor, p);
            D[(size_t)rows[i] * m + cols[j]] += (p[0] + I * p[1]) * nrm;
        }
    }
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
