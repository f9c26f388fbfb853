// Clements rectangular MZI mesh: U(phi) and the reverse-mode gradient of a
// real loss with respect to the phases, for a batch of phase sets.
//
// Components (Sec. 2, Eq. bs; the MZI of the Boson-sampling code in Sec. 4.2):
// BS = Rx(theta = pi/2) = (1/sqrt2) [[1, i], [i, 1]] and
//     MZI(phi_a, phi_b) = diag(1, e^{i phi_b}) . BS . diag(e^{i phi_a}, 1) . BS
//                       = diag(1, e^{i phi_b}) . 1/2 [[e - 1, i(e + 1)], [i(e + 1), 1 - e]],  e = e^{i phi_a}.
// Layout (Sec. 2 cites the square decomposition of Clements et al.): m
// columns; column c holds MZIs on modes (k, k+1) for k = c mod 2, c mod 2 + 2,
// ... < m-1, in that order; MZI q uses phases[2q], phases[2q+1].  Later
// components multiply on the left, so U = M_Q ... M_1.
//
// One block (one warp of column lanes) per phase set; U lives in shared memory.

#include "pcv_common.cuh"

namespace pcv {
namespace {

constexpr int kMaxMeshModes = 64;

struct Mzi { double2 t00, t01, t10, t11; };

__device__ __forceinline__ double2 cexp_i(double phi)
{
    double s, c;
    sincos(phi, &s, &c);
    return make_double2(c, s);
}

__device__ __forceinline__ double2 conj2(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 mul_i(double2 a) { return make_double2(-a.y, a.x); }
__device__ __forceinline__ double2 scale2(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

__device__ Mzi mzi(double pa, double pb)
{
    const double2 e = cexp_i(pa), f = cexp_i(pb);
    const double2 em1 = make_double2(e.x - 1.0, e.y), ep1 = make_double2(e.x + 1.0, e.y);
    Mzi t;
    t.t00 = scale2(em1, 0.5);
    t.t01 = scale2(mul_i(ep1), 0.5);
    t.t10 = cmul(f, scale2(mul_i(ep1), 0.5));
    t.t11 = cmul(f, scale2(make_double2(1.0 - e.x, -e.y), 0.5));
    return t;
}

// position k of MZI q in the Clements layout
__device__ int mzi_mode(int m, int q)
{
    for (int c = 0; c < m; ++c) {
        const int per = (c & 1) ? (m - 1) / 2 : m / 2;      // MZIs in column c
        if (q < per) return (c & 1) + 2 * q;
        q -= per;
    }
    return 0;
}

__global__ void mesh_forward_kernel(const double* __restrict__ phases, int m, int nq, double2* __restrict__ Uout)
{
    extern __shared__ double2 sU[];          // [m][m]
    const int b = blockIdx.x;
    const double* ph = phases + (size_t)b * 2 * nq;
    for (int i = threadIdx.x; i < m * m; i += blockDim.x)
        sU[i] = make_double2((i / m) == (i % m) ? 1.0 : 0.0, 0.0);
    __syncthreads();
    for (int q = 0; q < nq; ++q) {
        const Mzi t = mzi(ph[2 * q], ph[2 * q + 1]);
        const int k = mzi_mode(m, q);
        for (int j = threadIdx.x; j < m; j += blockDim.x) {
            const double2 u0 = sU[k * m + j], u1 = sU[(k + 1) * m + j];
            sU[k * m + j] = cadd(cmul(t.t00, u0), cmul(t.t01, u1));
            sU[(k + 1) * m + j] = cadd(cmul(t.t10, u0), cmul(t.t11, u1));
        }
        __syncwarp();
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m * m; i += blockDim.x) Uout[(size_t)b * m * m + i] = sU[i];
}

__device__ double2 warp_sum(double2 v)
{
    for (int off = 16; off > 0; off >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
    }
    return v;
}

// Reverse sweep: state U_q = M_q U_{q-1} is undone with M_q^H (M_q unitary);
// dL/dM_q = G_q U_{q-1}^H (2x2 block), dL/dphi = Re sum conj(dL/dM) dM/dphi,
// G_{q-1} = M_q^H G_q.  Gradients use the dL/dRe + i dL/dIm convention.
__global__ void mesh_backward_kernel(const double* __restrict__ phases, int m, int nq, const double2* __restrict__ U,
                                     const double2* __restrict__ G, double* __restrict__ gphi)
{
    extern __shared__ double2 sh[];
    double2* sU = sh;                // [m][m] current state
    double2* sG = sh + m * m;        // [m][m] current gradient
    const int b = blockIdx.x;
    const double* ph = phases + (size_t)b * 2 * nq;
    for (int i = threadIdx.x; i < m * m; i += blockDim.x) {
        sU[i] = U[(size_t)b * m * m + i];
        sG[i] = G[(size_t)b * m * m + i];
    }
    __syncthreads();
    for (int q = nq - 1; q >= 0; --q) {
        const double pa = ph[2 * q], pb = ph[2 * q + 1];
        const Mzi t = mzi(pa, pb);
        const int k = mzi_mode(m, q);
        double2 g00 = make_double2(0, 0), g01 = g00, g10 = g00, g11 = g00;
        for (int j = threadIdx.x; j < m; j += 32) {
            const double2 u0 = sU[k * m + j], u1 = sU[(k + 1) * m + j];
            // previous state rows: M^H [u0; u1]
            const double2 p0 = cadd(cmul(conj2(t.t00), u0), cmul(conj2(t.t10), u1));
            const double2 p1 = cadd(cmul(conj2(t.t01), u0), cmul(conj2(t.t11), u1));
            const double2 h0 = sG[k * m + j], h1 = sG[(k + 1) * m + j];
            g00 = cadd(g00, cmul(h0, conj2(p0)));
            g01 = cadd(g01, cmul(h0, conj2(p1)));
            g10 = cadd(g10, cmul(h1, conj2(p0)));
            g11 = cadd(g11, cmul(h1, conj2(p1)));
            sU[k * m + j] = p0;
            sU[(k + 1) * m + j] = p1;
            sG[k * m + j] = cadd(cmul(conj2(t.t00), h0), cmul(conj2(t.t10), h1));
            sG[(k + 1) * m + j] = cadd(cmul(conj2(t.t01), h0), cmul(conj2(t.t11), h1));
        }
        g00 = warp_sum(g00); g01 = warp_sum(g01); g10 = warp_sum(g10); g11 = warp_sum(g11);
        if (threadIdx.x == 0) {
            // dM/dphi_b: row 1 of M times i, row 0 zero
            const double2 d10 = mul_i(t.t10), d11 = mul_i(t.t11);
            const double db = cmul(conj2(g10), d10).x + cmul(conj2(g11), d11).x;
            // dM/dphi_a = diag(1, e^{i phi_b}) (i e / 2) [[1, i], [i, -1]]
            const double2 e = cexp_i(pa), f = cexp_i(pb);
            const double2 c = scale2(mul_i(e), 0.5);
            const double2 a00 = c, a01 = mul_i(c), a10 = cmul(f, mul_i(c)), a11 = cmul(f, scale2(c, -1.0));
            const double da = cmul(conj2(g00), a00).x + cmul(conj2(g01), a01).x +
                              cmul(conj2(g10), a10).x + cmul(conj2(g11), a11).x;
            gphi[(size_t)b * 2 * nq + 2 * q] = da;
            gphi[(size_t)b * 2 * nq + 2 * q + 1] = db;
        }
        __syncwarp();
    }
}

}  // namespace

int mesh_max_modes() { return kMaxMeshModes; }

cudaError_t launch_mesh_forward(const double* phases, int B, int m, double2* U, cudaStream_t s)
{
    const int nq = m * (m - 1) / 2;
    mesh_forward_kernel<<<B, 32, (size_t)m * m * sizeof(double2), s>>>(phases, m, nq, U);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mesh_backward(const double* phases, int B, int m, const double2* U, const double2* G,
                                 double* gphi, cudaStream_t s)
{
    const int nq = m * (m - 1) / 2;
    const size_t smem = (size_t)2 * m * m * sizeof(double2);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(mesh_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    mesh_backward_kernel<<<B, 32, smem, s>>>(phases, m, nq, U, G, gphi);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace pcv
