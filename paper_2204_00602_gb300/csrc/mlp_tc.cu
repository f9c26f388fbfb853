// BF16 GEMM on the 5th-generation tensor cores (tcgen05 + TMEM) with TMA
// staging, for the surrogate MLP.  C[M x N] = A[M x K] . B[N x K]^T, A and B
// bf16 row-major (K contiguous), FP32 accumulation in tensor memory, the same
// fused epilogues as the mma.sync kernel in mlp.cu (plain, bias, bias+GELU,
// GELU derivative).  No counterpart in the paper.
//
// One CTA computes a 128 x 128 tile with 128 threads:
//   thread 0    TMA producer: 64-wide K blocks of A and B (128B swizzle) into a
//               3-stage shared-memory ring, completion tracked by mbarriers;
//   thread 32   MMA issuer: tcgen05.mma.cta_group::1.kind::f16 (M=128, N=128,
//               K=16) from shared-memory descriptors into a 128-column TMEM
//               accumulator; tcgen05.commit frees each stage and finally
//               signals the epilogue;
//   all warps   epilogue: warp w reads TMEM lanes 32w..32w+31 (rows) with
//               tcgen05.ld.32x32b, turns each 32 x 32 block around in shared
//               memory and stores it row-contiguously.
// Three stages (97 KB of shared memory) let two CTAs share an SM, so one
// CTA's epilogue overlaps the other's main loop.
// Out-of-range rows, columns and K are zero-filled by TMA and skipped on
// store.  Every mbarrier wait gives up after a bounded number of polls and
// raises an error flag the host reads; TMEM is always released.

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <mutex>

#include "pcv_common.cuh"
#include "tc_ptx.cuh"

namespace pcv {

namespace {

constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 64, TC_STAGES = 3;   // 97 KB: two CTAs per SM
constexpr int TC_THREADS = 128;
constexpr uint32_t TC_STAGE_BYTES = (TC_BM + TC_BN) * TC_BK * 2;     // 32 KB per stage
constexpr uint32_t TC_TMEM_COLS = 128;
constexpr long long TC_MAX_POLLS = 1ll << 22;                        // default bound of one mbarrier wait

struct TcArgs {
    int M, N, K;
    int mode;
    const float* bias;
    float* outf; int ldo;
    __nv_bfloat16* outb; int ldob;
    const float* pre; int ldp;
    int* error;                       // set to the role that gave up (1 loads, 2 MMA, 3 epilogue, 4 clean-up)
    long long max_polls;              // bound of one mbarrier wait
};

using tcx::mbar_expect_tx;
using tcx::mbar_init;
using tcx::mbar_wait;
using tcx::sdesc_sw128;
using tcx::tma_load_2d;

__device__ __forceinline__ float gelu_tc(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_tc(float x)
{
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

__global__ void __launch_bounds__(TC_THREADS, 2)
gemm_bf16_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, const TcArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned ring of stages: [A 128x64 | B 128x64] bf16 each
    unsigned char* ring = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[TC_STAGES], empty_bar[TC_STAGES], done_bar, mma_done;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * TC_BN;
    const int nk = (a.K + TC_BK - 1) / TC_BK;

    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
        mbar_init(&mma_done, 1);
        s_fail = 0;
        tcx::mbar_fence_init();
        tcx::prefetch_tmap(&mapA);
        tcx::prefetch_tmap(&mapB);
    }
    if (warp == 1) tcx::tmem_alloc(&tmem_base, TC_TMEM_COLS);
    tcx::fence_before_sync();
    __syncthreads();
    tcx::fence_after_sync();
    const uint32_t tmem = tmem_base;
    const long long polls = a.max_polls;

    if (tid == 0) {
        // ---------------- TMA producer
        int issued = 0;
        for (int kt = 0; kt < nk && !s_fail; ++kt) {
            const int s = kt % TC_STAGES;
            if (kt >= TC_STAGES && !mbar_wait(&empty_bar[s], ((kt / TC_STAGES) - 1) & 1, polls)) { s_fail = 1; break; }
            unsigned char* sa = ring + s * TC_STAGE_BYTES;
            unsigned char* sb = sa + TC_BM * TC_BK * 2;
            mbar_expect_tx(&full_bar[s], TC_STAGE_BYTES);
            tma_load_2d(sa, &mapA, &full_bar[s], kt * TC_BK, m0);
            tma_load_2d(sb, &mapB, &full_bar[s], kt * TC_BK, n0);
            ++issued;
        }
        // the loads issued land in this CTA's shared memory before it may exit
        if (!tcx::wait_issued(full_bar, TC_STAGES, (uint32_t)issued) && !s_fail) s_fail = 4;
    } else if (tid == 32) {
        // ---------------- MMA issuer
        const uint32_t idesc = tcx::idesc_bf16(TC_BM, TC_BN);
        bool all = true;
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % TC_STAGES;
            if (!mbar_wait(&full_bar[s], (kt / TC_STAGES) & 1, polls)) { s_fail = 2; all = false; break; }
            tcx::fence_after_sync();
            const unsigned char* sa = ring + s * TC_STAGE_BYTES;
            const unsigned char* sb = sa + TC_BM * TC_BK * 2;
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk) {
                const uint64_t ad = sdesc_sw128(sa + kk * 32);      // 16 bf16 = 32 B along K
                const uint64_t bd = sdesc_sw128(sb + kk * 32);
                tcx::mma_bf16(tmem, ad, bd, idesc, (kt > 0 || kk > 0) ? 1u : 0u);
            }
            tcx::mma_commit(&empty_bar[s]);
        }
        // a complete accumulation goes to the epilogue; in every case the MMAs
        // issued finish before the tensor memory is released
        if (all) tcx::mma_commit(&done_bar);
        tcx::mma_commit(&mma_done);
        if (!mbar_wait(&mma_done, 0, tcx::kCleanupPolls) && !s_fail) s_fail = 4;
    }

    // ---------------- epilogue (all warps)
    const bool ok = mbar_wait(&done_bar, 0, polls);
    if (!ok && lane == 0) s_fail = 3;
    tcx::fence_after_sync();
    __syncwarp();
    if (ok) {
        // Each warp moves its 32 rows x 32 columns through a padded shared tile
        // (the drained stage ring) so that global stores are row-contiguous.
        float* stage = reinterpret_cast<float*>(ring) + warp * (32 * 33);
#pragma unroll 1
        for (int c0 = 0; c0 < TC_BN; c0 += 32) {
            uint32_t r[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
            for (int j = 0; j < 32; ++j) stage[lane * 33 + j] = __uint_as_float(r[j]);   // row = lane
            __syncwarp();
            const int col = n0 + c0 + lane;
            if (col < a.N) {
#pragma unroll 4
                for (int rr = 0; rr < 32; ++rr) {
                    const int row = m0 + warp * 32 + rr;
                    if (row >= a.M) break;
                    float x = stage[rr * 33 + lane];
                    switch (a.mode) {
                    case 0: a.outf[(size_t)row * a.ldo + col] = x; break;
                    case 2: a.outf[(size_t)row * a.ldo + col] = x + a.bias[col]; break;
                    case 1:
                        x += a.bias[col];
                        if (a.outf) a.outf[(size_t)row * a.ldo + col] = x;
                        a.outb[(size_t)row * a.ldob + col] = __float2bfloat16_rn(gelu_tc(x));
                        break;
                    case 3:
                        a.outb[(size_t)row * a.ldob + col] =
                            __float2bfloat16_rn(x * gelu_grad_tc(a.pre[(size_t)row * a.ldp + col]));
                        break;
                    }
                }
            }
            __syncwarp();
        }
    }
    tcx::fence_before_sync();
    __syncthreads();
    if (warp == 1) tcx::tmem_dealloc(tmem, TC_TMEM_COLS);
    if (tid == 0 && s_fail && a.error) atomicExch(a.error, s_fail);
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
bool g_attr_done[64] = {};

cudaError_t get_encode()
{
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    });
    return g_encode ? cudaSuccess : cudaErrorNotSupported;
}

// 2-D bf16 tensor map over rows x K (row stride ld elements), box 64 x 128, 128B swizzle.
cudaError_t make_map(CUtensorMap* map, const void* base, int rows, int K, int ld)
{
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)TC_BM};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
                                estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

size_t gemm_tc_smem() { return (size_t)TC_STAGES * TC_STAGE_BYTES + 1024; }

cudaError_t launch_gemm_bf16_tc(const void* A, int lda, const void* B, int ldb, int M, int N, int K, int mode,
                                const float* bias, float* outf, int ldo, void* outb, int ldob, const float* pre,
                                int ldp, int* error, cudaStream_t s)
{
    cudaError_t e = get_encode();
    if (e != cudaSuccess) return e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && !g_attr_done[dev]) {
        e = cudaFuncSetAttribute(gemm_bf16_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_tc_smem());
        if (e != cudaSuccess) return e;
        g_attr_done[dev] = true;
    }
    CUtensorMap ma, mb;
    if ((e = make_map(&ma, A, M, K, lda)) != cudaSuccess) return e;
    if ((e = make_map(&mb, B, N, K, ldb)) != cudaSuccess) return e;
    TcArgs a;
    a.M = M; a.N = N; a.K = K; a.mode = mode;
    a.bias = bias; a.outf = outf; a.ldo = ldo; a.outb = (__nv_bfloat16*)outb; a.ldob = ldob; a.pre = pre; a.ldp = ldp;
    a.error = error;
    a.max_polls = wait_limit(TC_MAX_POLLS);
    dim3 grid((N + TC_BN - 1) / TC_BN, (M + TC_BM - 1) / TC_BM);
    gemm_bf16_tc_kernel<<<grid, TC_THREADS, gemm_tc_smem(), s>>>(ma, mb, a);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace pcv

extern "C" int pcv_gemm_bf16_tc(const void* A, int lda, const void* B, int ldb, int M, int N, int K, int mode,
                                const float* bias, float* outf, int ldo, void* outb, int ldob, const float* pre,
                                int ldp, int* error, void* stream)
{
    if (!A || !B || M < 1 || N < 1 || K < 16 || K % 8 != 0) {
        pcv::set_error("gemm_bf16_tc: sizes (K must be a positive multiple of 8)");
        return PCV_EINVAL;
    }
    if (lda % 8 || ldb % 8 || lda < K || ldb < K || ((uintptr_t)A % 16) || ((uintptr_t)B % 16)) {
        pcv::set_error("gemm_bf16_tc: leading dimensions must be multiples of 8 >= K and operands 16-byte aligned");
        return PCV_EINVAL;
    }
    if (mode < 0 || mode > 3 || ((mode == 0 || mode == 2) && !outf) || ((mode == 1 || mode == 3) && !outb) ||
        ((mode == 1 || mode == 2) && !bias) || (mode == 3 && !pre)) {
        pcv::set_error("gemm_bf16_tc: epilogue arguments");
        return PCV_EINVAL;
    }
    cudaError_t e = pcv::launch_gemm_bf16_tc(A, lda, B, ldb, M, N, K, mode, bias, outf, ldo, outb, ldob, pre, ldp, error,
                                             (cudaStream_t)stream);
    if (e != cudaSuccess) {
        char buf[200];
        snprintf(buf, sizeof buf, "gemm_bf16_tc: %s", cudaGetErrorString(e));
        pcv::set_error(buf);
        return PCV_ECUDA;
    }
    return PCV_OK;
}
