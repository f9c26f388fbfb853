// BF16 MLP surrogate kernels: tensor-core GEMM with FP32 accumulation and
// fused epilogues (bias, GELU, GELU derivative), transposes, bias gradient,
// MSE loss, Adam, and the sin/cos phase features.  No counterpart in the
// paper: the surrogate maps mesh phases to log-probabilities of a fixed output
// set and is trained on data from the permanent kernels.
//
// GEMM: C[M x N] = A[M x K] . B[N x K]^T, A and B bf16 row-major with K
// contiguous (the "row.col" operand layout of mma.m16n8k16), K a multiple of
// 32.  Block tile 128 x 128 x 32, 8 warps of 64 x 32, double-buffered
// cp.async staging in padded shared memory, ldmatrix fragment loads.
// Out-of-range rows and columns are zero-filled on load and skipped on store.

#include <cuda_bf16.h>

#include <cstdio>

#include "pcv_common.cuh"

namespace pcv {
namespace {

constexpr int BM = 128, BN = 128, BK = 32, PAD = 8, LDS = BK + PAD;   // smem row = 40 bf16 = 80 B

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool pred)
{
    const int sz = pred ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(sz));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldmatrix_x4(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3, const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x)
{
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

}  // namespace

// epilogue modes
enum { kEpiF32 = 0, kEpiBiasGeluBf16 = 1, kEpiBiasF32 = 2, kEpiGeluGradBf16 = 3 };

struct GemmBf16Args {
    const __nv_bfloat16* A; int lda;
    const __nv_bfloat16* B; int ldb;
    int M, N, K;
    int mode;
    const float* bias;            // [N] (modes 1, 2)
    float* outf; int ldo;         // fp32 output (modes 0, 2) or pre-activation (mode 1, optional)
    __nv_bfloat16* outb; int ldob;  // bf16 output (modes 1, 3)
    const float* pre; int ldp;    // mode 3: forward pre-activation, out = acc * gelu'(pre)
};

namespace {

__global__ void __launch_bounds__(256) gemm_bf16_kernel(const GemmBf16Args g)
{
    __shared__ __align__(16) __nv_bfloat16 sA[2][BM * LDS];
    __shared__ __align__(16) __nv_bfloat16 sB[2][BN * LDS];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wm = warp >> 2, wn = warp & 3;           // 2 x 4 warps, 64 x 32 each
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;

    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[i][j][c] = 0.f;

    auto load = [&](int stage, int k0) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int chunk = tid + h * 256;          // 512 chunks of 16 B per operand tile
            const int row = chunk >> 2, kc = (chunk & 3) * 8;
            const int ga = m0 + row, gb = n0 + row;
            const bool pa = ga < g.M, pb = gb < g.N;
            cp_async16(&sA[stage][row * LDS + kc], g.A + (size_t)(pa ? ga : 0) * g.lda + k0 + kc, pa);
            cp_async16(&sB[stage][row * LDS + kc], g.B + (size_t)(pb ? gb : 0) * g.ldb + k0 + kc, pb);
        }
        cp_async_commit();
    };

    const int nk = g.K / BK;
    load(0, 0);
    for (int kt = 0; kt < nk; ++kt) {
        const int st = kt & 1;
        if (kt + 1 < nk) {
            load(st ^ 1, (kt + 1) * BK);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < BK; ks += 16) {
            uint32_t af[4][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = wm * 64 + i * 16 + (lane & 15);
                const int c = ks + (lane >> 4) * 8;
                ldmatrix_x4(af[i][0], af[i][1], af[i][2], af[i][3], &sA[st][r * LDS + c]);
            }
#pragma unroll
            for (int j2 = 0; j2 < 2; ++j2) {
                const int r = wn * 32 + j2 * 16 + (lane & 7) + ((lane >> 4) << 3);
                const int c = ks + ((lane >> 3) & 1) * 8;
                ldmatrix_x4(bf[2 * j2][0], bf[2 * j2][1], bf[2 * j2 + 1][0], bf[2 * j2 + 1][1], &sB[st][r * LDS + c]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j]);
        }
        __syncthreads();
    }

    // epilogue: c0,c1 at (row, col..col+1), c2,c3 at (row+8, col..col+1)
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int row = m0 + wm * 64 + i * 16 + (lane >> 2) + hh * 8;
                const int col = n0 + wn * 32 + j * 8 + (lane & 3) * 2;
                if (row >= g.M) continue;
                float v[2] = {acc[i][j][2 * hh], acc[i][j][2 * hh + 1]};
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int cc = col + e;
                    if (cc >= g.N) continue;
                    float x = v[e];
                    switch (g.mode) {
                    case kEpiF32:
                        g.outf[(size_t)row * g.ldo + cc] = x;
                        break;
                    case kEpiBiasF32:
                        g.outf[(size_t)row * g.ldo + cc] = x + g.bias[cc];
                        break;
                    case kEpiBiasGeluBf16:
                        x += g.bias[cc];
                        if (g.outf) g.outf[(size_t)row * g.ldo + cc] = x;
                        g.outb[(size_t)row * g.ldob + cc] = __float2bfloat16_rn(gelu(x));
                        break;
                    case kEpiGeluGradBf16:
                        g.outb[(size_t)row * g.ldob + cc] = __float2bfloat16_rn(x * gelu_grad(g.pre[(size_t)row * g.ldp + cc]));
                        break;
                    }
                }
            }
}

__global__ void transpose_bf16_kernel(const __nv_bfloat16* __restrict__ in, int R, int C, int ldi,
                                      __nv_bfloat16* __restrict__ out, int ldo)
{
    __shared__ __nv_bfloat16 t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = r0 + y, c = c0 + threadIdx.x;
        if (r < R && c < C) t[y][threadIdx.x] = in[(size_t)r * ldi + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int c = c0 + y, r = r0 + threadIdx.x;
        if (r < R && c < C) out[(size_t)c * ldo + r] = t[threadIdx.x][y];
    }
}

// db[n] = sum_m dY[m][n] (bf16 input, fp32 sum in a fixed order)
__global__ void colsum_bf16_kernel(const __nv_bfloat16* __restrict__ dY, int M, int N, int ld, float* __restrict__ db)
{
    __shared__ float sh[8][33];
    const int c = blockIdx.x * 32 + threadIdx.x;
    float s = 0.f;
    if (c < N)
        for (int r = threadIdx.y; r < M; r += 8) s += __bfloat162float(dY[(size_t)r * ld + c]);
    sh[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && c < N) {
        float t = 0.f;
        for (int y = 0; y < 8; ++y) t += sh[y][threadIdx.x];
        db[c] = t;
    }
}

// x = [sin phi, cos phi, 1, 0...] (bf16, row length ldx)
__global__ void features_kernel(const double* __restrict__ phases, int B, int P, __nv_bfloat16* __restrict__ X, int ldx)
{
    const int b = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ldx) return;
    float v = 0.f;
    if (j < P) v = (float)sin(phases[(size_t)b * P + j]);
    else if (j < 2 * P) v = (float)cos(phases[(size_t)b * P + j - P]);
    else if (j == 2 * P) v = 1.f;
    X[(size_t)b * ldx + j] = __float2bfloat16_rn(v);
}

// dL/dphi from dL/dx: d sin = cos, d cos = -sin
__global__ void features_grad_kernel(const double* __restrict__ phases, int B, int P, const float* __restrict__ dX,
                                     int ldx, double* __restrict__ gphi)
{
    const int b = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P) return;
    const double ph = phases[(size_t)b * P + j];
    gphi[(size_t)b * P + j] = (double)dX[(size_t)b * ldx + j] * cos(ph) - (double)dX[(size_t)b * ldx + P + j] * sin(ph);
}

// MSE: loss partials and dPred = 2 (pred - target) * scale (bf16)
__global__ void mse_kernel(const float* __restrict__ pred, const float* __restrict__ tgt, int64_t count, float scale,
                           __nv_bfloat16* __restrict__ dpred, float* __restrict__ part)
{
    __shared__ float sh[256];
    float s = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < count; i += (int64_t)gridDim.x * 256) {
        const float d = pred[i] - tgt[i];
        s += d * d;
        if (dpred) dpred[i] = __float2bfloat16_rn(2.f * d * scale);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void sum_partials_kernel(const float* __restrict__ part, int n, float scale, float* out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        float s = 0.f;
        for (int i = 0; i < n; ++i) s += part[i];
        *out = s * scale;
    }
}

__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v, const float* __restrict__ g,
                            int64_t count, float lr, float b1, float b2, float eps, float c1, float c2,
                            __nv_bfloat16* __restrict__ wb)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16_rn(wi);
}

__global__ void adam_f64_kernel(double* __restrict__ w, double* __restrict__ m, double* __restrict__ v,
                                const double* __restrict__ g, int64_t count, double lr, double b1, double b2, double eps,
                                double c1, double c2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double gi = g[i];
    const double mi = b1 * m[i] + (1.0 - b1) * gi;
    const double vi = b2 * v[i] + (1.0 - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrt(vi / c2) + eps);
}

__global__ void f32_to_bf16_kernel(const float* __restrict__ in, int64_t count, __nv_bfloat16* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = __float2bfloat16_rn(in[i]);
}

__global__ void log_f64_to_f32_kernel(const double* __restrict__ in, int64_t count, float* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = (float)log(in[i]);
}

__global__ void exp_f32_to_f64_kernel(const float* __restrict__ in, int64_t count, double* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = exp((double)in[i]);
}

}  // namespace

cudaError_t launch_exp_f32_to_f64(const float* in, int64_t count, double* out, cudaStream_t s)
{
    exp_f32_to_f64_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(in, count, out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_log_f64_to_f32(const double* in, int64_t count, float* out, cudaStream_t s)
{
    log_f64_to_f32_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(in, count, out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gemm_bf16(const GemmBf16Args& g, cudaStream_t s)
{
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM);
    gemm_bf16_kernel<<<grid, 256, 0, s>>>(g);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_transpose_bf16(const void* in, int R, int C, int ldi, void* out, int ldo, cudaStream_t s)
{
    dim3 grid((C + 31) / 32, (R + 31) / 32);
    transpose_bf16_kernel<<<grid, dim3(32, 8), 0, s>>>((const __nv_bfloat16*)in, R, C, ldi, (__nv_bfloat16*)out, ldo);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_colsum_bf16(const void* dY, int M, int N, int ld, float* db, cudaStream_t s)
{
    colsum_bf16_kernel<<<(N + 31) / 32, dim3(32, 8), 0, s>>>((const __nv_bfloat16*)dY, M, N, ld, db);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_features(const double* phases, int B, int P, void* X, int ldx, cudaStream_t s)
{
    features_kernel<<<dim3((ldx + 127) / 128, B), 128, 0, s>>>(phases, B, P, (__nv_bfloat16*)X, ldx);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_features_grad(const double* phases, int B, int P, const float* dX, int ldx, double* gphi, cudaStream_t s)
{
    features_grad_kernel<<<dim3((P + 127) / 128, B), 128, 0, s>>>(phases, B, P, dX, ldx, gphi);
    note_launches(1);
    return cudaGetLastError();
}

int mse_partials() { return 256; }

cudaError_t launch_mse(const float* pred, const float* tgt, int64_t count, float* loss, void* dpred, float* part,
                       cudaStream_t s)
{
    mse_kernel<<<256, 256, 0, s>>>(pred, tgt, count, 1.f / (float)count, (__nv_bfloat16*)dpred, part);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_partials_kernel<<<1, 32, 0, s>>>(part, 256, 1.f / (float)count, loss);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* w, float* m, float* v, const float* g, int64_t count, float lr, float b1, float b2,
                        float eps, int step, void* wb, cudaStream_t s)
{
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(w, m, v, g, count, lr, b1, b2, eps, c1, c2,
                                                                 (__nv_bfloat16*)wb);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_adam_f64(double* w, double* m, double* v, const double* g, int64_t count, double lr, double b1,
                            double b2, double eps, int step, cudaStream_t s)
{
    const double c1 = 1.0 - pow(b1, (double)step), c2 = 1.0 - pow(b2, (double)step);
    adam_f64_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(w, m, v, g, count, lr, b1, b2, eps, c1, c2);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_f32_to_bf16(const float* in, int64_t count, void* out, cudaStream_t s)
{
    f32_to_bf16_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(in, count, (__nv_bfloat16*)out);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace pcv

// ------------------------------------------------------------------- C ABI

namespace {
inline int mlp_ok(cudaError_t e, const char* where)
{
    if (e == cudaSuccess) return PCV_OK;
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
    pcv::set_error(buf);
    return PCV_ECUDA;
}
inline int mlp_bad(const char* msg)
{
    pcv::set_error(msg);
    return PCV_EINVAL;
}
}  // namespace

extern "C" {

int pcv_gemm_bf16(const void* A, int lda, const void* B, int ldb, int M, int N, int K, int mode,
                  const float* bias, float* outf, int ldo, void* outb, int ldob, const float* pre, int ldp,
                  void* stream)
{
    if (!A || !B || M < 1 || N < 1 || K < 32 || K % 32 != 0) return mlp_bad("gemm_bf16: sizes (K must be a positive multiple of 32)");
    if (lda % 8 || ldb % 8 || lda < K || ldb < K || ((uintptr_t)A % 16) || ((uintptr_t)B % 16))
        return mlp_bad("gemm_bf16: leading dimensions must be multiples of 8 >= K and operands 16-byte aligned");
    if (mode < 0 || mode > 3) return mlp_bad("gemm_bf16: unknown epilogue");
    if ((mode == 0 || mode == 2) && !outf) return mlp_bad("gemm_bf16: fp32 output missing");
    if ((mode == 1 || mode == 3) && !outb) return mlp_bad("gemm_bf16: bf16 output missing");
    if ((mode == 1 || mode == 2) && !bias) return mlp_bad("gemm_bf16: bias missing");
    if (mode == 3 && !pre) return mlp_bad("gemm_bf16: pre-activation missing");
    pcv::GemmBf16Args g;
    g.A = (const __nv_bfloat16*)A; g.lda = lda;
    g.B = (const __nv_bfloat16*)B; g.ldb = ldb;
    g.M = M; g.N = N; g.K = K; g.mode = mode;
    g.bias = bias; g.outf = outf; g.ldo = ldo; g.outb = (__nv_bfloat16*)outb; g.ldob = ldob; g.pre = pre; g.ldp = ldp;
    return mlp_ok(pcv::launch_gemm_bf16(g, (cudaStream_t)stream), "gemm_bf16");
}

int pcv_transpose_bf16(const void* in, int R, int C, int ldi, void* out, int ldo, void* stream)
{
    if (!in || !out || R < 1 || C < 1 || ldi < C || ldo < R) return mlp_bad("transpose_bf16: bad arguments");
    return mlp_ok(pcv::launch_transpose_bf16(in, R, C, ldi, out, ldo, (cudaStream_t)stream), "transpose_bf16");
}

int pcv_colsum_bf16(const void* dY, int M, int N, int ld, float* db, void* stream)
{
    if (!dY || !db || M < 1 || N < 1 || ld < N) return mlp_bad("colsum_bf16: bad arguments");
    return mlp_ok(pcv::launch_colsum_bf16(dY, M, N, ld, db, (cudaStream_t)stream), "colsum_bf16");
}

int pcv_phase_features(const double* phases, int B, int P, void* X, int ldx, void* stream)
{
    if (!phases || !X || B < 1 || B > 65535 || P < 1 || ldx < 2 * P + 1) return mlp_bad("phase_features: bad arguments");
    return mlp_ok(pcv::launch_features(phases, B, P, X, ldx, (cudaStream_t)stream), "phase_features");
}

int pcv_phase_features_grad(const double* phases, int B, int P, const float* dX, int ldx, double* grad_phases,
                            void* stream)
{
    if (!phases || !dX || !grad_phases || B < 1 || B > 65535 || P < 1 || ldx < 2 * P) return mlp_bad("phase_features_grad: bad arguments");
    return mlp_ok(pcv::launch_features_grad(phases, B, P, dX, ldx, grad_phases, (cudaStream_t)stream), "phase_features_grad");
}

int64_t pcv_mse_workspace(void) { return pcv::mse_partials() * (int64_t)sizeof(float); }

int pcv_mse(const float* pred, const float* target, int64_t count, float* loss, void* grad_pred_bf16,
            void* workspace, int64_t workspace_bytes, void* stream)
{
    if (!pred || !target || !loss || count < 1) return mlp_bad("mse: bad arguments");
    if (!workspace || workspace_bytes < pcv_mse_workspace()) return mlp_bad("mse: workspace too small");
    return mlp_ok(pcv::launch_mse(pred, target, count, loss, grad_pred_bf16, (float*)workspace, (cudaStream_t)stream), "mse");
}

int pcv_adam(float* w, float* m, float* v, const float* g, int64_t count, float lr, float beta1, float beta2,
             float eps, int step, void* w_bf16, void* stream)
{
    if (!w || !m || !v || !g || count < 1 || step < 1) return mlp_bad("adam: bad arguments");
    return mlp_ok(pcv::launch_adam(w, m, v, g, count, lr, beta1, beta2, eps, step, w_bf16, (cudaStream_t)stream), "adam");
}

int pcv_exp_f32_to_f64(const float* in, int64_t count, double* out, void* stream)
{
    if (!in || !out || count < 0) return mlp_bad("exp_f32_to_f64: bad arguments");
    if (count == 0) return PCV_OK;
    return mlp_ok(pcv::launch_exp_f32_to_f64(in, count, out, (cudaStream_t)stream), "exp_f32_to_f64");
}

int pcv_log_f64_to_f32(const double* in, int64_t count, float* out, void* stream)
{
    if (!in || !out || count < 0) return mlp_bad("log_f64_to_f32: bad arguments");
    if (count == 0) return PCV_OK;
    return mlp_ok(pcv::launch_log_f64_to_f32(in, count, out, (cudaStream_t)stream), "log_f64_to_f32");
}

int pcv_adam_f64(double* w, double* m, double* v, const double* g, int64_t count, double lr, double beta1,
                 double beta2, double eps, int step, void* stream)
{
    if (!w || !m || !v || !g || count < 1 || step < 1) return mlp_bad("adam_f64: bad arguments");
    return mlp_ok(pcv::launch_adam_f64(w, m, v, g, count, lr, beta1, beta2, eps, step, (cudaStream_t)stream), "adam_f64");
}

int pcv_f32_to_bf16(const float* in, int64_t count, void* out, void* stream)
{
    if (!in || !out || count < 0) return mlp_bad("f32_to_bf16: bad arguments");
    if (count == 0) return PCV_OK;
    return mlp_ok(pcv::launch_f32_to_bf16(in, count, out, (cudaStream_t)stream), "f32_to_bf16");
}

}  // extern "C"
