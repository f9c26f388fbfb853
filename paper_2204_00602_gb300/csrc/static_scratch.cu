// pcv_distribution_static: the full-distribution entry point for callers that
// cannot allocate device memory (see include/pcv.h).  Its scratch is one
// file-scope __device__ array that every GPU loading the library holds until
// the process exits; host code passes the array's device address, obtained
// once per device with cudaGetSymbolAddress, to the same kernels
// pcv_distribution runs.

#include <cmath>
#include <mutex>

#include "pcv_common.cuh"

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[PCV_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device (set up on the
// first call per device).
cudaError_t scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

int static_fail(int code, const char* msg)
{
    pcv::set_error(msg);
    return code;
}

}  // namespace

extern "C" int64_t pcv_distribution_static_max_bytes(void) { return PCV_STATIC_SCRATCH_BYTES; }

extern "C" int pcv_distribution_static(const pcv_c64* U, int m, const uint8_t* input_occ,
                                       double* prob, pcv_c64* amp, void* stream)
{
    if (m < 1 || m > PCV_MAX_MODES) return static_fail(PCV_EINVAL, "m outside [1, PCV_MAX_MODES]");
    if (!U || ((uintptr_t)U % 16) != 0) return static_fail(PCV_EINVAL, "U is NULL or not 16-byte aligned");
    if (!input_occ) return static_fail(PCV_EINVAL, "input_occ is NULL");
    if (!amp && !prob) return static_fail(PCV_EINVAL, "amp and prob are both NULL");
    if ((amp && ((uintptr_t)amp % 16) != 0) || (prob && ((uintptr_t)prob % 8) != 0))
        return static_fail(PCV_EINVAL, "amp or prob misaligned");
    pcv::Plan p;
    p.m = m;
    int n = 0;
    double f = 1.0;
    for (int j = 0; j < m; ++j) {
        n += input_occ[j];
        for (int q = 2; q <= input_occ[j]; ++q) f *= q;
    }
    if (n < 1 || n > PCV_MAX_PHOTONS) return static_fail(PCV_EINVAL, "photon number outside [1, PCV_MAX_PHOTONS]");
    p.n = n;
    int c = 0;
    for (int j = 0; j < m; ++j)
        for (int q = 0; q < input_occ[j]; ++q) p.cols[c++] = j;
    for (; c < PCV_MAX_PHOTONS; ++c) p.cols[c] = 0;
    p.norm_t = 1.0 / std::sqrt(f);

    // an output space or plan that does not fit in int64 is a range error, as
    // in pcv_distribution; only problems too big for the array are ENOMEM
    if (pcv_num_outputs(m, n) < 0) return static_fail(PCV_ERANGE, "output space C(m+n-1, n) too large");
    pcv::DistPlan dp;
    const int64_t need = pcv::dist_plan(p, 1, PCV_STATIC_SCRATCH_BYTES, amp == nullptr, &dp);
    if (need < 0) return static_fail(PCV_ERANGE, "workspace size overflows");
    if (need > PCV_STATIC_SCRATCH_BYTES)
        return static_fail(PCV_ENOMEM, "problem needs more scratch than PCV_STATIC_SCRATCH_BYTES; "
                                       "use pcv_distribution with a workspace");
    void* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) return static_fail(PCV_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
    e = pcv::launch_glynn_dist(p, dp, (const double2*)U, prob, (double2*)amp, scratch, (cudaStream_t)stream);
    return e == cudaSuccess ? PCV_OK : static_fail(PCV_ECUDA, cudaGetErrorString(e));
}
