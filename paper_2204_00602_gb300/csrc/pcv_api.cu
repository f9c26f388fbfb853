// C ABI of libpcv.so (declared in include/pcv.h): argument checks, planning
// and dispatch to the kernels.  No device memory is allocated here; scratch
// comes from the caller's workspace.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "pcv_common.cuh"

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* where)
{
    return fail(PCV_ECUDA, "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
}

int64_t binom(int a, int b)
{
    if (b < 0 || a < 0 || b > a) return 0;
    unsigned __int128 c = 1;
    for (int i = 1; i <= b; ++i) {
        c = c * (unsigned __int128)(a - b + i) / (unsigned __int128)i;
        if (c > ((unsigned __int128)1 << 62)) return -1;
    }
    return (int64_t)c;
}

int64_t msets(int w, int k) { return k == 0 ? 1 : (w <= 0 ? 0 : binom(w + k - 1, k)); }

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

int make_plan(const pcv_c64* U, int m, const uint8_t* input_occ, pcv::Plan* p)
{
    if (m < 1 || m > PCV_MAX_MODES) return fail(PCV_EINVAL, "m=%d outside [1, %d]", m, PCV_MAX_MODES);
    if (!U) return fail(PCV_EINVAL, "U is NULL");
    if (!aligned(U, 16)) return fail(PCV_EINVAL, "U is not 16-byte aligned");
    if (!input_occ) return fail(PCV_EINVAL, "input_occ is NULL");
    int n = 0;
    double f = 1.0;
    for (int j = 0; j < m; ++j) {
        n += input_occ[j];
        for (int q = 2; q <= input_occ[j]; ++q) f *= q;
    }
    if (n > PCV_MAX_PHOTONS) return fail(PCV_EINVAL, "input has %d photons, more than %d", n, PCV_MAX_PHOTONS);
    p->m = m;
    p->n = n;
    int c = 0;
    for (int j = 0; j < m; ++j)
        for (int q = 0; q < input_occ[j]; ++q) p->cols[c++] = j;
    for (; c < PCV_MAX_PHOTONS; ++c) p->cols[c] = 0;
    p->norm_t = 1.0 / std::sqrt(f);
    return PCV_OK;
}

constexpr int kSMs = 152;
// Internal choice of PCV_ALGO_AUTO for explicit outputs: the batched
// launch's per-output routing (tile kernel or Glynn's sum with
// multiplicities) applied to one circuit.
constexpr int kAlgoRouted = 100;
constexpr int kRouteMinPhotons = 13;

// Threads per permanent for the group kernel: enough threads in flight to
// cover the GPU, never more lanes than Gray steps.
int auto_group(int n, int64_t n_out)
{
    int G = 1;
    const int gmax = n >= 6 ? 32 : (1 << std::max(0, n - 1));
    while (G < gmax && n_out * G < (int64_t)kSMs * 512) G *= 2;
    return G;
}

// Blocks per permanent for the block kernel.
int auto_splits(int n, int64_t n_out)
{
    const int64_t steps = 1ll << (n - 1);
    int S = 1;
    while ((int64_t)S * 2 * pcv::glynn_block_threads() <= steps && n_out * S < (int64_t)kSMs * 8) S *= 2;
    return S;
}

struct AmpChoice { int algo, param; };

AmpChoice choose_amp(int m, int n, int64_t n_out, int algo, int param)
{
    if (algo == PCV_ALGO_AUTO) {
        // shared row sums when there are enough outputs to give every SM a tile
        if (m <= pcv::tile_max_modes() && n >= 1 && n_out >= (int64_t)kSMs * (256 / pcv::tile_splits(n)))
            return {n >= kRouteMinPhotons && n_out <= INT32_MAX ? kAlgoRouted : PCV_ALGO_TILE, 0};
        if (n <= 12 || (n <= 16 && n_out >= (int64_t)kSMs * 256)) return {PCV_ALGO_GROUP, auto_group(n, n_out)};
        return {PCV_ALGO_BLOCK, auto_splits(n, n_out)};
    }
    if (algo == PCV_ALGO_MULT && param == 0) {
        // enough warps in flight for every SM slot
        const int64_t want = (int64_t)kSMs * 16;
        const int64_t parts = n_out >= want ? 1 : (want + n_out - 1) / std::max<int64_t>(n_out, 1);
        return {algo, (int)std::min<int64_t>(parts, 1024)};
    }
    return {algo, param};
}

int check_choice(const AmpChoice& c, int n)
{
    if (c.algo == PCV_ALGO_TILE) {
        if (n < 1) return fail(PCV_EINVAL, "tile kernel needs n >= 1");
        return PCV_OK;
    }
    if (c.algo == PCV_ALGO_GROUP) {
        if (n > 16) return fail(PCV_EINVAL, "group kernel supports n <= 16 (n=%d)", n);
        const int G = c.param;
        if (G != 1 && G != 2 && G != 4 && G != 8 && G != 16 && G != 32)
            return fail(PCV_EINVAL, "threads per permanent %d not in {1,2,4,8,16,32}", G);
        if (n > 0 && (1ll << (n - 1)) < G) return fail(PCV_EINVAL, "threads per permanent %d exceed 2^(n-1)=%lld", G, 1ll << (n - 1));
        return PCV_OK;
    }
    if (c.algo == kAlgoRouted) return PCV_OK;
    if (c.algo == PCV_ALGO_MULT) {
        if (n < 1) return fail(PCV_EINVAL, "multiplicity kernel needs n >= 1");
        if (c.param < 1 || c.param > 1024) return fail(PCV_EINVAL, "warps per permanent %d outside [1, 1024]", c.param);
        return PCV_OK;
    }
    if (c.algo == PCV_ALGO_BLOCK) {
        if (n < 9 || n > PCV_MAX_PHOTONS) return fail(PCV_EINVAL, "block kernel supports 9 <= n <= 30 (n=%d)", n);
        if (c.param < 1 || (int64_t)c.param * pcv::glynn_block_threads() > (1ll << (n - 1)))
            return fail(PCV_EINVAL, "blocks per permanent %d invalid for n=%d", c.param, n);
        return PCV_OK;
    }
    return fail(PCV_EINVAL, "unknown algorithm %d", c.algo);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int64_t amp_workspace(const AmpChoice& c, int64_t n_out)
{
    if (c.algo == kAlgoRouted)
        return (int64_t)align256(sizeof(pcv_batch_desc)) + pcv::batched_workspace(1, n_out);
    if ((c.algo == PCV_ALGO_BLOCK || c.algo == PCV_ALGO_MULT) && c.param > 1)
        return (int64_t)align256((size_t)n_out * c.param * sizeof(double2));
    return 0;
}

// ------------------------------------------------------ stage timing
struct StageTimer {
    std::mutex mu;
    bool on = false;
    std::vector<cudaEvent_t> pool;
    struct Open { int stage; cudaEvent_t a; };
    struct Done { int stage; cudaEvent_t a, b; };
    std::vector<Open> open;
    std::vector<Done> done;
    double ms[pcv::kStageCount] = {};
    int64_t calls[pcv::kStageCount] = {};
    cudaEvent_t get()
    {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
};
StageTimer g_timer;
std::atomic<int64_t> g_launches{0};
std::atomic<long long> g_wait_polls{0};      // 0: each kernel's default bound

}  // namespace

namespace pcv {
void stage_begin(int stage, cudaStream_t s)
{
    std::lock_guard<std::mutex> lk(g_timer.mu);
    if (!g_timer.on) return;
    cudaEvent_t e = g_timer.get();
    cudaEventRecord(e, s);
    g_timer.open.push_back({stage, e});
}
void stage_end(int stage, cudaStream_t s)
{
    std::lock_guard<std::mutex> lk(g_timer.mu);
    if (!g_timer.on) return;
    for (size_t i = g_timer.open.size(); i-- > 0;) {
        if (g_timer.open[i].stage != stage) continue;
        cudaEvent_t b = g_timer.get();
        cudaEventRecord(b, s);
        g_timer.done.push_back({stage, g_timer.open[i].a, b});
        g_timer.open.erase(g_timer.open.begin() + (long)i);
        return;
    }
}
void note_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
void set_error(const char* msg) { g_err = msg; }
long long wait_limit(long long dflt)
{
    const long long v = g_wait_polls.load(std::memory_order_relaxed);
    return v > 0 ? v : dflt;
}
}  // namespace pcv

extern "C" {

int pcv_profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_timer.mu);
    g_timer.on = on != 0;
    return PCV_OK;
}

int pcv_profile_read(double* ms, int64_t* calls, int nstages)
{
    if (nstages < 0 || (nstages > 0 && (!ms || !calls))) return fail(PCV_EINVAL, "bad profile buffers");
    std::lock_guard<std::mutex> lk(g_timer.mu);
    for (auto& d : g_timer.done) {
        cudaError_t e = cudaEventSynchronize(d.b);
        if (e != cudaSuccess) return cuda_fail(e, "profile event");
        float t = 0.f;
        cudaEventElapsedTime(&t, d.a, d.b);
        g_timer.ms[d.stage] += t;
        g_timer.calls[d.stage] += 1;
        g_timer.pool.push_back(d.a);
        g_timer.pool.push_back(d.b);
    }
    g_timer.done.clear();
    for (int i = 0; i < nstages && i < pcv::kStageCount; ++i) {
        ms[i] = g_timer.ms[i];
        calls[i] = g_timer.calls[i];
        g_timer.ms[i] = 0;
        g_timer.calls[i] = 0;
    }
    return PCV_OK;
}

int64_t pcv_launch_count(void) { return g_launches.load(); }

int pcv_set_wait_limit(int64_t polls)
{
    if (polls < 0) return fail(PCV_EINVAL, "wait limit %lld < 0", (long long)polls);
    g_wait_polls.store((long long)polls, std::memory_order_relaxed);
    return PCV_OK;
}

int pcv_distribution_status(const void* workspace, void* stream)
{
    if (!workspace) return fail(PCV_EINVAL, "workspace is NULL");
    int code = 0;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(&code, workspace, sizeof code, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "reading the distribution status");
    if (code != 0)
        return fail(PCV_ETIMEOUT,
                    "a bounded wait of the tensor-core product kernel gave up (role %d: 1 loads, 2 MMA issue, "
                    "3 accumulator drain, 4 clean-up); the outputs of that call are not valid",
                    code);
    return PCV_OK;
}

const char* pcv_last_error(void) { return g_err.c_str(); }

const char* pcv_version(void) { return "pcv 0.1 sm_103a"; }

int64_t pcv_num_outputs(int m, int n)
{
    if (m < 1 || n < 0) return fail(PCV_EINVAL, "m=%d n=%d", m, n);
    const int64_t c = msets(m, n);
    if (c < 0) return fail(PCV_ERANGE, "C(m+n-1,n) exceeds 2^62 for m=%d n=%d", m, n);
    return c;
}

int pcv_unrank(int m, int n, int64_t idx, uint8_t* occ_out)
{
    const int64_t N = pcv_num_outputs(m, n);
    if (N < 0) return (int)N;
    if (!occ_out) return fail(PCV_EINVAL, "occ_out is NULL");
    if (idx < 0 || idx >= N) return fail(PCV_ERANGE, "index %lld outside [0, %lld)", (long long)idx, (long long)N);
    for (int r = 0; r < m; ++r) occ_out[r] = 0;
    int v = 0;
    for (int p = 0; p < n; ++p) {
        for (;;) {
            const int64_t c = msets(m - v, n - p - 1);
            if (idx < c) break;
            idx -= c;
            ++v;
        }
        occ_out[v]++;
    }
    return PCV_OK;
}

int64_t pcv_rank(int m, const uint8_t* occ)
{
    if (m < 1 || !occ) return fail(PCV_EINVAL, "bad arguments");
    int n = 0;
    for (int r = 0; r < m; ++r) n += occ[r];
    if (msets(m, n) < 0) return fail(PCV_ERANGE, "output space too large");
    int64_t rank = 0;
    int p = 0, prev = 0;
    for (int r = 0; r < m; ++r) {
        for (int q = 0; q < occ[r]; ++q) {
            for (int v = prev; v < r; ++v) rank += msets(m - v, n - p - 1);
            prev = r;
            ++p;
        }
    }
    return rank;
}

int64_t pcv_amplitudes_workspace(int m, int n, int64_t n_out)
{
    if (m < 1 || m > PCV_MAX_MODES || n < 0 || n > PCV_MAX_PHOTONS || n_out < 0) return fail(PCV_EINVAL, "bad sizes");
    return amp_workspace(choose_amp(m, n, n_out, PCV_ALGO_AUTO, 0), n_out);
}

int64_t pcv_amplitudes_ex_workspace(int m, int n, int64_t n_out, int algo, int param)
{
    if (m < 1 || m > PCV_MAX_MODES || n < 0 || n > PCV_MAX_PHOTONS || n_out < 0) return fail(PCV_EINVAL, "bad sizes");
    if (n == 0) return 0;
    const AmpChoice c = choose_amp(m, n, n_out, algo, param);
    const int rc = check_choice(c, n);
    if (rc) return rc;
    return amp_workspace(c, n_out);
}

int pcv_amplitudes_ex(const pcv_c64* U, int m, const uint8_t* input_occ,
                      const uint8_t* output_occ, int64_t n_out,
                      pcv_c64* amp, double* prob, int algo, int param,
                      void* workspace, int64_t workspace_bytes, void* stream)
{
    pcv::Plan p;
    int rc = make_plan(U, m, input_occ, &p);
    if (rc) return rc;
    if (n_out < 0) return fail(PCV_EINVAL, "n_out=%lld < 0", (long long)n_out);
    if (n_out == 0) return PCV_OK;
    if (!output_occ) return fail(PCV_EINVAL, "output_occ is NULL");
    if (!amp && !prob) return fail(PCV_EINVAL, "amp and prob are both NULL");
    if (amp && !aligned(amp, 16)) return fail(PCV_EINVAL, "amp is not 16-byte aligned");
    if (prob && !aligned(prob, 8)) return fail(PCV_EINVAL, "prob is not 8-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    if (p.n == 0) {
        cudaError_t e = pcv::launch_glynn_group(p, (const double2*)U, output_occ, nullptr, 0, n_out,
                                                (double2*)amp, prob, 1, s);
        return e == cudaSuccess ? PCV_OK : cuda_fail(e, "n0 kernel");
    }
    AmpChoice c = choose_amp(m, p.n, n_out, algo, param);
    if ((rc = check_choice(c, p.n))) return rc;
    const int64_t need = amp_workspace(c, n_out);
    if (need > 0 && (!workspace || workspace_bytes < need))
        return fail(PCV_ENOMEM, "workspace of %lld bytes needed, %lld given", (long long)need, (long long)workspace_bytes);
    if (need > 0 && !aligned(workspace, 256)) return fail(PCV_EINVAL, "workspace is not 256-byte aligned");
    if ((int64_t)n_out * ((c.algo == PCV_ALGO_BLOCK || c.algo == PCV_ALGO_MULT) ? c.param : 1) > INT32_MAX)
        return fail(PCV_ERANGE, "too many permanents for one launch");
    if (c.algo == kAlgoRouted) {
        pcv_batch_desc d;
        d.U = U;
        d.outputs = output_occ;
        d.amp = amp;
        d.prob = prob;
        d.n_out = n_out;
        d.m = m;
        d.n = p.n;
        for (int j = 0; j < PCV_MAX_PHOTONS; ++j) d.cols[j] = p.cols[j];
        int dev = 0, sms = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "device query");
        pcv_batch_desc* dd = (pcv_batch_desc*)workspace;
        void* bws = (char*)workspace + align256(sizeof(pcv_batch_desc));
        pcv::stage_begin(pcv::kStagePlain, s);
        e = pcv::launch_store_desc(d, dd, s);
        if (e == cudaSuccess) e = pcv::launch_glynn_batched(dd, 1, n_out, bws, sms, PCV_ALGO_AUTO, s);
        pcv::stage_end(pcv::kStagePlain, s);
        return e == cudaSuccess ? PCV_OK : cuda_fail(e, "routed launch");
    }
    if (c.algo == PCV_ALGO_MULT) {
        pcv_batch_desc d;
        d.U = U;
        d.outputs = output_occ;
        d.amp = amp;
        d.prob = prob;
        d.n_out = n_out;
        d.m = m;
        d.n = p.n;
        for (int j = 0; j < PCV_MAX_PHOTONS; ++j) d.cols[j] = p.cols[j];
        pcv::stage_begin(pcv::kStagePlain, s);
        cudaError_t e = pcv::launch_glynn_mult(d, c.param, 0, (double2*)workspace, s);
        pcv::stage_end(pcv::kStagePlain, s);
        return e == cudaSuccess ? PCV_OK : cuda_fail(e, "multiplicity launch");
    }
    if (c.algo == PCV_ALGO_TILE) {
        if (m > pcv::tile_max_modes()) return fail(PCV_EINVAL, "tile kernel supports m <= %d (m=%d)", pcv::tile_max_modes(), m);
        pcv_batch_desc d;
        d.U = U;
        d.outputs = output_occ;
        d.amp = amp;
        d.prob = prob;
        d.n_out = n_out;
        d.m = m;
        d.n = p.n;
        for (int j = 0; j < PCV_MAX_PHOTONS; ++j) d.cols[j] = p.cols[j];
        pcv::stage_begin(pcv::kStagePlain, s);
        cudaError_t e = pcv::launch_glynn_tile(d, s);
        pcv::stage_end(pcv::kStagePlain, s);
        return e == cudaSuccess ? PCV_OK : cuda_fail(e, "tile launch");
    }
    cudaError_t e;
    pcv::stage_begin(pcv::kStagePlain, s);
    if (c.algo == PCV_ALGO_GROUP)
        e = pcv::launch_glynn_group(p, (const double2*)U, output_occ, nullptr, 0, n_out, (double2*)amp, prob, c.param, s);
    else
        e = pcv::launch_glynn_block(p, (const double2*)U, output_occ, nullptr, 0, n_out, (double2*)amp, prob,
                                    c.param, (double2*)workspace, s);
    pcv::stage_end(pcv::kStagePlain, s);
    return e == cudaSuccess ? PCV_OK : cuda_fail(e, "glynn launch");
}

int pcv_amplitudes(const pcv_c64* U, int m, const uint8_t* input_occ,
                   const uint8_t* output_occ, int64_t n_out,
                   pcv_c64* amp, double* prob,
                   void* workspace, int64_t workspace_bytes, void* stream)
{
    return pcv_amplitudes_ex(U, m, input_occ, output_occ, n_out, amp, prob, PCV_ALGO_AUTO, 0,
                             workspace, workspace_bytes, stream);
}

int pcv_amplitudes_multi(const pcv_c64* U, int B, int m, const uint8_t* input_occ,
                         const uint8_t* output_occ, int64_t n_out, pcv_c64* amp, double* prob, void* stream)
{
    pcv::Plan p;
    int rc = make_plan(U, m, input_occ, &p);
    if (rc) return rc;
    if (B < 1 || B > 65535) return fail(PCV_EINVAL, "batch %d outside [1, 65535]", B);
    if (m > pcv::tile_max_modes()) return fail(PCV_EINVAL, "m=%d above %d", m, pcv::tile_max_modes());
    if (p.n < 1) return fail(PCV_EINVAL, "n must be >= 1");
    if (n_out < 0) return fail(PCV_EINVAL, "n_out < 0");
    if (n_out == 0) return PCV_OK;
    if (!output_occ || (!amp && !prob)) return fail(PCV_EINVAL, "bad output pointers");
    if (amp && !aligned(amp, 16)) return fail(PCV_EINVAL, "amp is not 16-byte aligned");
    pcv_batch_desc d;
    d.U = U;
    d.outputs = output_occ;
    d.amp = amp;
    d.prob = prob;
    d.n_out = n_out;
    d.m = m;
    d.n = p.n;
    for (int j = 0; j < PCV_MAX_PHOTONS; ++j) d.cols[j] = p.cols[j];
    cudaStream_t s = (cudaStream_t)stream;
    pcv::stage_begin(pcv::kStagePlain, s);
    cudaError_t e = pcv::launch_glynn_tile_multi(d, B, s);
    pcv::stage_end(pcv::kStagePlain, s);
    return e == cudaSuccess ? PCV_OK : cuda_fail(e, "tile multi launch");
}

int64_t pcv_amplitudes_batched_workspace(int n_circ, int64_t total_outputs)
{
    if (n_circ < 0 || total_outputs < 0) return fail(PCV_EINVAL, "bad sizes");
    return pcv::batched_workspace(n_circ, total_outputs);
}

int pcv_amplitudes_batched_ex(const pcv_batch_desc* descs, int n_circ, int64_t total_outputs, int algo,
                              void* workspace, int64_t workspace_bytes, void* stream)
{
    if (n_circ < 0 || total_outputs < 0) return fail(PCV_EINVAL, "n_circ=%d total_outputs=%lld", n_circ, (long long)total_outputs);
    if (algo != PCV_ALGO_AUTO && algo != PCV_ALGO_TILE && algo != PCV_ALGO_MULT)
        return fail(PCV_EINVAL, "batched routing %d is not AUTO, TILE or MULT", algo);
    if (n_circ == 0) return PCV_OK;
    if (!descs) return fail(PCV_EINVAL, "descs is NULL");
    if (total_outputs > INT32_MAX || (total_outputs / 32 + n_circ + 1) > INT32_MAX)
        return fail(PCV_ERANGE, "too many outputs for one launch");
    const int64_t need = pcv::batched_workspace(n_circ, total_outputs);
    if (!workspace || workspace_bytes < need)
        return fail(PCV_ENOMEM, "workspace of %lld bytes needed, %lld given", (long long)need, (long long)workspace_bytes);
    if (!aligned(workspace, 256)) return fail(PCV_EINVAL, "workspace is not 256-byte aligned");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    cudaStream_t s = (cudaStream_t)stream;
    pcv::stage_begin(pcv::kStagePlain, s);
    e = pcv::launch_glynn_batched(descs, n_circ, total_outputs, workspace, sms, algo, s);
    pcv::stage_end(pcv::kStagePlain, s);
    return e == cudaSuccess ? PCV_OK : cuda_fail(e, "batched launch");
}

int pcv_amplitudes_batched(const pcv_batch_desc* descs, int n_circ, int64_t total_outputs,
                           void* workspace, int64_t workspace_bytes, void* stream)
{
    return pcv_amplitudes_batched_ex(descs, n_circ, total_outputs, PCV_ALGO_AUTO, workspace, workspace_bytes, stream);
}

static int64_t dist_ws(int B, int m, int n, int algo, int param, bool need_acc, int64_t ws_bytes, pcv::DistPlan* dp)
{
    pcv::Plan p;
    p.m = m;
    p.n = n;
    if (algo == PCV_ALGO_FACTOR || algo == PCV_ALGO_AUTO) {
        if (n == 0) return 0;
        pcv::DistPlan local;
        return pcv::dist_plan(p, B, ws_bytes, need_acc, dp ? dp : &local);
    }
    const int64_t N = msets(m, n);
    int64_t bytes = (int64_t)align256((size_t)(m + 1) * (n + 1) * sizeof(int64_t));
    if (algo == PCV_ALGO_BLOCK && param > 1) bytes += (int64_t)align256((size_t)N * param * sizeof(double2));
    return bytes;
}

int64_t pcv_distribution_batched_workspace(int B, int m, int n)
{
    if (B < 1 || m < 1 || m > PCV_MAX_MODES || n < 0 || n > PCV_MAX_PHOTONS) return fail(PCV_EINVAL, "bad sizes");
    if (msets(m, n) < 0) return fail(PCV_ERANGE, "output space too large");
    const int64_t r = dist_ws(B, m, n, PCV_ALGO_FACTOR, 0, true, -1, nullptr);
    return r < 0 ? fail(PCV_ERANGE, "workspace size overflows") : r;
}

// Single-pass tensor-core plan of one distribution (no error message on
// failure): its bytes, or -1 when the path does not apply or overflows.
static int64_t tc_ws_bytes(int m, int n)
{
    if (m < 2 || m > PCV_MAX_MODES || n < 2 || n > 10 || msets(m, n) < 0) return -1;
    pcv::Plan p;
    p.m = m;
    p.n = n;
    pcv::DistPlan dp;
    return pcv::dist_plan_tc(p, true, &dp);
}

// PCV_ALGO_AUTO for one full distribution: the tensor-core products when the
// input has 2..10 photons over m >= 2 modes and the workspace holds their
// single-pass plan, else the FP64 products (which accept any workspace down to
// pcv_distribution_workspace_min).
static int auto_dist_algo(int m, int n, int64_t workspace_bytes)
{
    const int64_t tc = tc_ws_bytes(m, n);
    return (tc >= 0 && workspace_bytes >= tc) ? PCV_ALGO_FACTOR_TC : PCV_ALGO_FACTOR;
}

int64_t pcv_distribution_workspace(int m, int n)
{
    const int64_t tc = tc_ws_bytes(m, n);
    return tc >= 0 ? tc : pcv_distribution_batched_workspace(1, m, n);
}

int pcv_distribution_auto_algo(int m, int n, int64_t workspace_bytes)
{
    if (m < 1 || m > PCV_MAX_MODES || n < 0 || n > PCV_MAX_PHOTONS) return fail(PCV_EINVAL, "bad sizes");
    return auto_dist_algo(m, n, workspace_bytes);
}

int64_t pcv_distribution_workspace_min(int m, int n)
{
    if (m < 1 || m > PCV_MAX_MODES || n < 0 || n > PCV_MAX_PHOTONS) return fail(PCV_EINVAL, "bad sizes");
    if (msets(m, n) < 0) return fail(PCV_ERANGE, "output space too large");
    const int64_t r = dist_ws(1, m, n, PCV_ALGO_FACTOR, 0, true, 0, nullptr);
    return r < 0 ? fail(PCV_ERANGE, "workspace size overflows") : r;
}

// The factorised distribution with FP64 products for the outputs [lo, hi)
// (hi < 0: all) of B unitaries; arguments as pcv_distribution_batched.
static int distribution_factor(const pcv_c64* U, int B, int m, const uint8_t* input_occ, int64_t lo, int64_t hi,
                               double* prob, pcv_c64* amp, void* workspace, int64_t workspace_bytes, void* stream)
{
    pcv::Plan p;
    int rc = make_plan(U, m, input_occ, &p);
    if (rc) return rc;
    if (B < 1 || B > 65535) return fail(PCV_EINVAL, "batch %d outside [1, 65535]", B);
    if (!amp && !prob) return fail(PCV_EINVAL, "amp and prob are both NULL");
    if (amp && !aligned(amp, 16)) return fail(PCV_EINVAL, "amp is not 16-byte aligned");
    if (prob && !aligned(prob, 8)) return fail(PCV_EINVAL, "prob is not 8-byte aligned");
    if (workspace && !aligned(workspace, 256)) return fail(PCV_EINVAL, "workspace is not 256-byte aligned");
    const int64_t N = msets(m, p.n);
    if (N < 0) return fail(PCV_ERANGE, "output space C(%d,%d) too large", m + p.n - 1, p.n);
    if (hi < 0) hi = N;
    if (lo < 0 || lo > hi || hi > N)
        return fail(PCV_EINVAL, "output range [%lld, %lld) outside [0, %lld]", (long long)lo, (long long)hi, (long long)N);
    if (lo == hi) return PCV_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (p.n == 0) {                               // one output, index 0 (lo = 0, hi = 1 here)
        for (int b = 0; b < B; ++b) {
            cudaError_t e = pcv::launch_glynn_group(p, (const double2*)U, nullptr, nullptr, 0, 1,
                                                    amp ? (double2*)amp + b : nullptr, prob ? prob + b : nullptr, 1, s);
            if (e != cudaSuccess) return cuda_fail(e, "n0 kernel");
        }
        return PCV_OK;
    }
    pcv::DistPlan dp;
    const int64_t need = dist_ws(B, m, p.n, PCV_ALGO_FACTOR, 0, amp == nullptr, workspace_bytes, &dp);
    if (need < 0) return fail(PCV_ERANGE, "workspace size overflows");
    if (!workspace || need > workspace_bytes)
        return fail(PCV_ENOMEM, "workspace of at least %lld bytes needed, %lld given",
                    (long long)dist_ws(B, m, p.n, PCV_ALGO_FACTOR, 0, amp == nullptr, 0, nullptr), (long long)workspace_bytes);
    if (B > 1 && (lo != 0 || hi != N)) return fail(PCV_EINVAL, "output ranges take one unitary");
    dp.lo = lo;
    dp.hi = hi;
    cudaError_t e = pcv::launch_glynn_dist(p, dp, (const double2*)U, prob, (double2*)amp, workspace, s);
    return e == cudaSuccess ? PCV_OK : cuda_fail(e, "factorised distribution");
}

int pcv_distribution_batched(const pcv_c64* U, int B, int m, const uint8_t* input_occ,
                             double* prob, pcv_c64* amp,
                             void* workspace, int64_t workspace_bytes, void* stream)
{
    return distribution_factor(U, B, m, input_occ, 0, -1, prob, amp, workspace, workspace_bytes, stream);
}

int64_t pcv_distribution_slos_workspace(int B, int m, int n)
{
    if (B < 1 || m < 1 || m > PCV_MAX_MODES || n < 0 || n > PCV_MAX_PHOTONS) return fail(PCV_EINVAL, "bad sizes");
    if (msets(m, n) < 0) return fail(PCV_ERANGE, "output space too large");
    const int64_t r = pcv::slos_workspace(B, m, n);
    return r < 0 ? fail(PCV_ERANGE, "workspace size overflows") : r;
}

int pcv_distribution_slos(const pcv_c64* U, int B, int m, const uint8_t* input_occ,
                          double* prob, pcv_c64* amp,
                          void* workspace, int64_t workspace_bytes, void* stream)
{
    pcv::Plan p;
    int rc = make_plan(U, m, input_occ, &p);
    if (rc) return rc;
    if (B < 1 || B > 65535) return fail(PCV_EINVAL, "batch %d outside [1, 65535]", B);
    if (!amp && !prob) return fail(PCV_EINVAL, "amp and prob are both NULL");
    if (amp && !aligned(amp, 16)) return fail(PCV_EINVAL, "amp is not 16-byte aligned");
    if (prob && !aligned(prob, 8)) return fail(PCV_EINVAL, "prob is not 8-byte aligned");
    const int64_t N = msets(m, p.n);
    if (N < 0 || (N + 255) / 256 > INT32_MAX) return fail(PCV_ERANGE, "output space C(%d,%d) too large", m + p.n - 1, p.n);
    cudaStream_t s = (cudaStream_t)stream;
    if (p.n == 0) {
        for (int b = 0; b < B; ++b) {
            cudaError_t e = pcv::launch_glynn_group(p, (const double2*)U, nullptr, nullptr, 0, 1,
                                                    amp ? (double2*)amp + b : nullptr, prob ? prob + b : nullptr, 1, s);
            if (e != cudaSuccess) return cuda_fail(e, "n0 kernel");
        }
        return PCV_OK;
    }
    const int64_t need = pcv::slos_workspace(B, m, p.n);
    if (need < 0) return fail(PCV_ERANGE, "workspace size overflows");
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256))
        return fail(PCV_ENOMEM, "workspace of %lld bytes (256-byte aligned) needed, %lld given", (long long)need,
                    (long long)workspace_bytes);
    pcv::stage_begin(pcv::kStagePlain, s);
    cudaError_t e = pcv::launch_slos(p, B, (const double2*)U, prob, (double2*)amp, workspace, s);
    pcv::stage_end(pcv::kStagePlain, s);
    return e == cudaSuccess ? PCV_OK : cuda_fail(e, "state expansion");
}

int64_t pcv_distribution_tc_workspace(int m, int n)
{
    if (m < 1 || m > PCV_MAX_MODES || n < 1 || n > 10) return fail(PCV_EINVAL, "tensor-core products need 1 <= n <= 10");
    if (msets(m, n) < 0) return fail(PCV_ERANGE, "output space too large");
    pcv::Plan p;
    p.m = m;
    p.n = n;
    pcv::DistPlan dp;
    const int64_t r = pcv::dist_plan_tc(p, true, &dp);
    return r < 0 ? fail(PCV_ERANGE, "workspace size overflows") : r;
}

// The factorised distribution with tensor-core products for the outputs
// [lo, hi) (hi < 0: all), written at prob[o - lo], amp[o - lo].
static int distribution_tc(const pcv_c64* U, int m, const uint8_t* input_occ, int64_t lo, int64_t hi, double* prob,
                           pcv_c64* amp, void* workspace, int64_t workspace_bytes, void* stream)
{
    pcv::Plan p;
    int rc = make_plan(U, m, input_occ, &p);
    if (rc) return rc;
    if (p.n < 1 || p.n > 10) return fail(PCV_EINVAL, "tensor-core products need 1 <= n <= 10 (n=%d)", p.n);
    if (!amp && !prob) return fail(PCV_EINVAL, "amp and prob are both NULL");
    if (amp && !aligned(amp, 16)) return fail(PCV_EINVAL, "amp is not 16-byte aligned");
    if (prob && !aligned(prob, 8)) return fail(PCV_EINVAL, "prob is not 8-byte aligned");
    if (workspace && !aligned(workspace, 256)) return fail(PCV_EINVAL, "workspace is not 256-byte aligned");
    const int64_t N = msets(m, p.n);
    if (N < 0) return fail(PCV_ERANGE, "output space too large");
    if (hi < 0) hi = N;
    if (lo < 0 || lo > hi || hi > N)
        return fail(PCV_EINVAL, "output range [%lld, %lld) outside [0, %lld]", (long long)lo, (long long)hi, (long long)N);
    pcv::DistPlan dp;
    const int64_t need = pcv::dist_plan_tc(p, amp == nullptr, &dp);
    if (need < 0) return fail(PCV_ERANGE, "workspace size overflows");
    if (!workspace || need > workspace_bytes)
        return fail(PCV_ENOMEM, "workspace of %lld bytes needed, %lld given", (long long)need, (long long)workspace_bytes);
    if (lo == hi) return PCV_OK;
    dp.lo = lo;
    dp.hi = hi;
    cudaError_t e = pcv::launch_glynn_dist(p, dp, (const double2*)U, prob, (double2*)amp, workspace, (cudaStream_t)stream);
    return e == cudaSuccess ? PCV_OK : cuda_fail(e, "tensor-core factorised distribution");
}

int pcv_distribution_ex(const pcv_c64* U, int m, const uint8_t* input_occ,
                        double* prob, pcv_c64* amp, int algo, int param,
                        void* workspace, int64_t workspace_bytes, void* stream)
{
    if (algo == PCV_ALGO_AUTO && m >= 1 && m <= PCV_MAX_MODES && input_occ) {
        int n = 0;
        for (int i = 0; i < m; ++i) n += input_occ[i];
        algo = auto_dist_algo(m, n, workspace ? workspace_bytes : 0);
    }
    if (algo == PCV_ALGO_FACTOR_TC)
        return distribution_tc(U, m, input_occ, 0, -1, prob, amp, workspace, workspace_bytes, stream);
    if (algo == PCV_ALGO_SLOS)
        return pcv_distribution_slos(U, 1, m, input_occ, prob, amp, workspace, workspace_bytes, stream);
    if (algo == PCV_ALGO_AUTO || algo == PCV_ALGO_FACTOR)
        return pcv_distribution_batched(U, 1, m, input_occ, prob, amp, workspace, workspace_bytes, stream);
    pcv::Plan p;
    int rc = make_plan(U, m, input_occ, &p);
    if (rc) return rc;
    if (!amp && !prob) return fail(PCV_EINVAL, "amp and prob are both NULL");
    if (amp && !aligned(amp, 16)) return fail(PCV_EINVAL, "amp is not 16-byte aligned");
    if (prob && !aligned(prob, 8)) return fail(PCV_EINVAL, "prob is not 8-byte aligned");
    const int64_t N = msets(m, p.n);
    if (N < 0) return fail(PCV_ERANGE, "output space C(%d,%d) too large", m + p.n - 1, p.n);
    cudaStream_t s = (cudaStream_t)stream;
    if (p.n == 0) {
        cudaError_t e = pcv::launch_glynn_group(p, (const double2*)U, nullptr, nullptr, 0, 1, (double2*)amp, prob, 1, s);
        return e == cudaSuccess ? PCV_OK : cuda_fail(e, "n0 kernel");
    }
    if (workspace && !aligned(workspace, 256)) return fail(PCV_EINVAL, "workspace is not 256-byte aligned");
    AmpChoice c{algo, param};
    if ((rc = check_choice(c, p.n))) return rc;
    if (algo == PCV_ALGO_TILE) return fail(PCV_EINVAL, "the tile kernel takes explicit outputs");
    const int64_t need = dist_ws(1, m, p.n, algo, param, false, workspace_bytes, nullptr);
    if (!workspace || need > workspace_bytes)
        return fail(PCV_ENOMEM, "workspace of %lld bytes needed, %lld given", (long long)need, (long long)workspace_bytes);
    if (N * (algo == PCV_ALGO_BLOCK ? param : 1) > INT32_MAX) return fail(PCV_ERANGE, "too many permanents for one launch");
    int64_t* table = (int64_t*)workspace;
    double2* partial = (double2*)((char*)workspace + align256((size_t)(m + 1) * (p.n + 1) * sizeof(int64_t)));
    cudaError_t e = pcv::build_multiset_table(table, m, p.n, s);
    if (e != cudaSuccess) return cuda_fail(e, "multiset table");
    pcv::stage_begin(pcv::kStagePlain, s);
    if (algo == PCV_ALGO_GROUP)
        e = pcv::launch_glynn_group(p, (const double2*)U, nullptr, table, 0, N, (double2*)amp, prob, param, s);
    else
        e = pcv::launch_glynn_block(p, (const double2*)U, nullptr, table, 0, N, (double2*)amp, prob, param, partial, s);
    pcv::stage_end(pcv::kStagePlain, s);
    return e == cudaSuccess ? PCV_OK : cuda_fail(e, "glynn launch");
}

int pcv_distribution(const pcv_c64* U, int m, const uint8_t* input_occ,
                     double* prob, pcv_c64* amp,
                     void* workspace, int64_t workspace_bytes, void* stream)
{
    return pcv_distribution_ex(U, m, input_occ, prob, amp, PCV_ALGO_AUTO, 0, workspace, workspace_bytes, stream);
}

int pcv_distribution_range_plan(int m, int n, int64_t begin, int64_t end, int64_t* pa, int64_t* pb)
{
    if (m < 1 || m > PCV_MAX_MODES || n < 0 || n > PCV_MAX_PHOTONS || !pa || !pb) return fail(PCV_EINVAL, "bad sizes");
    const int64_t N = msets(m, n);
    if (N < 0) return fail(PCV_ERANGE, "output space too large");
    if (begin < 0 || end < begin || end > N)
        return fail(PCV_EINVAL, "output range [%lld, %lld) outside [0, %lld]", (long long)begin, (long long)end,
                    (long long)N);
    pcv::PRanges r;
    pcv::p_ranges(m, n, std::max(1, m / 2), begin, end, &r);
    for (int k = 0; k <= n; ++k) {
        pa[k] = r.pa[k];
        pb[k] = r.pb[k];
    }
    return PCV_OK;
}

int pcv_distribution_range(const pcv_c64* U, int m, const uint8_t* input_occ, int64_t begin, int64_t end,
                           double* prob, pcv_c64* amp, void* workspace, int64_t workspace_bytes, void* stream)
{
    if (begin < 0 || end < begin) return fail(PCV_EINVAL, "output range [%lld, %lld)", (long long)begin, (long long)end);
    int n = 0;
    if (m >= 1 && m <= PCV_MAX_MODES && input_occ)
        for (int i = 0; i < m; ++i) n += input_occ[i];
    if (begin == end) {                           // nothing to write; the buffers may be empty (NULL)
        pcv::Plan p;
        const int rc = make_plan(U, m, input_occ, &p);
        if (rc) return rc;
        const int64_t N = msets(m, p.n);
        if (N < 0) return fail(PCV_ERANGE, "output space too large");
        return end <= N ? PCV_OK : fail(PCV_EINVAL, "output range [%lld, %lld) outside [0, %lld]", (long long)begin,
                                        (long long)end, (long long)N);
    }
    if (auto_dist_algo(m, n, workspace ? workspace_bytes : 0) == PCV_ALGO_FACTOR_TC)
        return distribution_tc(U, m, input_occ, begin, end, prob, amp, workspace, workspace_bytes, stream);
    return distribution_factor(U, 1, m, input_occ, begin, end, prob, amp, workspace, workspace_bytes, stream);
}

int pcv_distribution_tc_blocks(int m, int n, int64_t begin, int64_t end, int64_t* out, int64_t out_len,
                               int64_t* needed)
{
    if (m < 2 || m > PCV_MAX_MODES || n < 2 || n > 10) return fail(PCV_EINVAL, "m %d, n %d outside the tensor-core plan", m, n);
    const int64_t N = msets(m, n);
    if (N < 0) return fail(PCV_ERANGE, "output space too large");
    if (end < 0) end = N;
    if (begin < 0 || begin > end || end > N) return fail(PCV_EINVAL, "range [%lld, %lld) outside [0, %lld)",
                                                         (long long)begin, (long long)end, (long long)N);
    const int64_t need = pcv::tc_block_list(m, n, begin, end, out, out_len);
    if (need < 0) return fail(PCV_ERANGE, "the plan needs more blocks than the products kernel takes");
    if (needed) *needed = need;
    if (out && out_len < need) return fail(PCV_EINVAL, "out holds %lld values, %lld needed", (long long)out_len,
                                           (long long)need);
    return PCV_OK;
}

// ------------------------------------------------------------- adjoint

// Checks shared by the backward calls; fills the plan for `count` outputs.
static int backward_common(const pcv_c64* U, int B, int m, const uint8_t* input_occ, int64_t count,
                           const pcv_c64* grad_amp, pcv_c64* grad_U, void* workspace, int64_t workspace_bytes,
                           pcv::Plan* p, pcv::AdjPlan* ap)
{
    int rc = make_plan(U, m, input_occ, p);
    if (rc) return rc;
    if (B < 1 || B > 65535) return fail(PCV_EINVAL, "batch %d outside [1, 65535]", B);
    if (count < 0) return fail(PCV_EINVAL, "n_out < 0");
    if (!grad_U || !aligned(grad_U, 16)) return fail(PCV_EINVAL, "grad_U is NULL or misaligned");
    if (count > 0 && (!grad_amp || !aligned(grad_amp, 16))) return fail(PCV_EINVAL, "bad gradient pointer");
    if (workspace && !aligned(workspace, 256)) return fail(PCV_EINVAL, "workspace is not 256-byte aligned");
    *ap = pcv::adjoint_plan(m, p->n, B, count, workspace ? workspace_bytes : 0);
    if (count > 0 && p->n > 0 && (!workspace || workspace_bytes < (int64_t)ap->min_total))
        return fail(PCV_ENOMEM, "workspace of at least %lld bytes needed, %lld given", (long long)ap->min_total,
                    (long long)workspace_bytes);
    return PCV_OK;
}

int64_t pcv_amplitudes_backward_workspace(int B, int m, int n, int64_t n_out)
{
    if (B < 1 || m < 1 || m > PCV_MAX_MODES || n < 0 || n > PCV_MAX_PHOTONS || n_out < 0)
        return fail(PCV_EINVAL, "bad sizes");
    return (int64_t)pcv::adjoint_plan(m, n, B, n_out, -1).total;
}

int pcv_amplitudes_backward(const pcv_c64* U, int m, const uint8_t* input_occ,
                            const uint8_t* output_occ, int64_t n_out, const pcv_c64* grad_amp,
                            pcv_c64* grad_U, void* workspace, int64_t workspace_bytes, void* stream)
{
    return pcv_amplitudes_backward_multi(U, 1, m, input_occ, output_occ, n_out, grad_amp, grad_U, workspace,
                                         workspace_bytes, stream);
}

int pcv_amplitudes_backward_multi(const pcv_c64* U, int B, int m, const uint8_t* input_occ,
                                  const uint8_t* output_occ, int64_t n_out, const pcv_c64* grad_amp,
                                  pcv_c64* grad_U, void* workspace, int64_t workspace_bytes, void* stream)
{
    pcv::Plan p;
    pcv::AdjPlan ap;
    int rc = backward_common(U, B, m, input_occ, n_out, grad_amp, grad_U, workspace, workspace_bytes, &p, &ap);
    if (rc) return rc;
    if (n_out > 0 && !output_occ) return fail(PCV_EINVAL, "output_occ is NULL");
    cudaError_t e = pcv::launch_adjoint(p, (const double2*)U, B, output_occ, n_out, (const double2*)grad_amp,
                                        (double2*)grad_U, workspace, ap, (cudaStream_t)stream);
    return e == cudaSuccess ? PCV_OK : cuda_fail(e, "adjoint");
}

int64_t pcv_distribution_backward_workspace(int B, int m, int n)
{
    if (B < 1 || m < 1 || m > PCV_MAX_MODES || n < 0 || n > PCV_MAX_PHOTONS) return fail(PCV_EINVAL, "bad sizes");
    const int64_t N = msets(m, n);
    if (N < 0) return fail(PCV_ERANGE, "output space too large");
    return (int64_t)pcv::adjoint_plan(m, n, B, N, -1).total;
}

int pcv_distribution_backward(const pcv_c64* U, int B, int m, const uint8_t* input_occ,
                              const pcv_c64* grad_amp, pcv_c64* grad_U,
                              void* workspace, int64_t workspace_bytes, void* stream)
{
    int n = 0;
    if (m >= 1 && m <= PCV_MAX_MODES && input_occ)
        for (int i = 0; i < m; ++i) n += input_occ[i];
    const int64_t N = msets(m, std::min(n, PCV_MAX_PHOTONS));
    if (N < 0) return fail(PCV_ERANGE, "output space too large");
    pcv::Plan p;
    pcv::AdjPlan ap;
    int rc = backward_common(U, B, m, input_occ, N, grad_amp, grad_U, workspace, workspace_bytes, &p, &ap);
    if (rc) return rc;
    cudaError_t e = pcv::launch_adjoint(p, (const double2*)U, B, nullptr, N, (const double2*)grad_amp,
                                        (double2*)grad_U, workspace, ap, (cudaStream_t)stream);
    return e == cudaSuccess ? PCV_OK : cuda_fail(e, "distribution adjoint");
}

// ----------------------------------------------------------- sampling

int pcv_sample(const pcv_c64* U, int m, const uint8_t* input_occ, const uint8_t* perm, const double* uniforms,
               int64_t count, uint8_t* samples, void* stream)
{
    pcv::Plan p;
    int rc = make_plan(U, m, input_occ, &p);
    if (rc) return rc;
    if (m > 128) return fail(PCV_EINVAL, "sampler supports m <= 128 (m=%d)", m);
    if (p.n < 1 || p.n > 16) return fail(PCV_EINVAL, "sampler supports 1 <= n <= 16 (n=%d)", p.n);
    if (count < 0) return fail(PCV_EINVAL, "count < 0");
    if (count == 0) return PCV_OK;
    if (!perm || !uniforms || !samples) return fail(PCV_EINVAL, "NULL sample buffer");
    if ((count + 3) / 4 > INT32_MAX) return fail(PCV_ERANGE, "too many samples for one launch");
    cudaStream_t s = (cudaStream_t)stream;
    pcv::stage_begin(pcv::kStagePlain, s);
    cudaError_t e = pcv::launch_sampler(p, (const double2*)U, perm, uniforms, count, samples, s);
    pcv::stage_end(pcv::kStagePlain, s);
    return e == cudaSuccess ? PCV_OK : cuda_fail(e, "sampler");
}

// --------------------------------------------------------------- mesh

int pcv_mesh_unitary(const double* phases, int B, int m, pcv_c64* U, void* stream)
{
    if (B < 1 || m < 2 || m > pcv::mesh_max_modes() || !phases || !U || !aligned(U, 16))
        return fail(PCV_EINVAL, "mesh: B=%d m=%d", B, m);
    cudaError_t e = pcv::launch_mesh_forward(phases, B, m, (double2*)U, (cudaStream_t)stream);
    return e == cudaSuccess ? PCV_OK : cuda_fail(e, "mesh forward");
}

int pcv_mesh_backward(const double* phases, int B, int m, const pcv_c64* U, const pcv_c64* grad_U,
                      double* grad_phases, void* stream)
{
    if (B < 1 || m < 2 || m > pcv::mesh_max_modes() || !phases || !U || !grad_U || !grad_phases)
        return fail(PCV_EINVAL, "mesh backward: B=%d m=%d", B, m);
    cudaError_t e = pcv::launch_mesh_backward(phases, B, m, (const double2*)U, (const double2*)grad_U, grad_phases,
                                              (cudaStream_t)stream);
    return e == cudaSuccess ? PCV_OK : cuda_fail(e, "mesh backward");
}

// ---------------------------------------------------------- reductions

int64_t pcv_dist_stats_workspace(int B)
{
    if (B < 1) return fail(PCV_EINVAL, "B < 1");
    return pcv::stats_workspace(B);
}

int pcv_dist_stats(const double* p, const double* q, int64_t N, int B, int q_batched, double* out,
                   void* workspace, int64_t workspace_bytes, void* stream)
{
    if (!p || !out || N < 1 || B < 1 || B > 65535) return fail(PCV_EINVAL, "dist_stats: bad arguments");
    if (!workspace || workspace_bytes < pcv::stats_workspace(B) || !aligned(workspace, 8))
        return fail(PCV_ENOMEM, "dist_stats: workspace of %lld bytes needed", (long long)pcv::stats_workspace(B));
    cudaError_t e = pcv::launch_stats(p, q, N, B, q_batched, out, (double*)workspace, (cudaStream_t)stream);
    return e == cudaSuccess ? PCV_OK : cuda_fail(e, "dist_stats");
}

int pcv_kl_grad(const double* p, const double* q, const pcv_c64* amp, int64_t N, int B, int q_batched,
                const double* batch_scale, double scale, pcv_c64* grad_amp, void* stream)
{
    if (!p || !q || !amp || !grad_amp || N < 1 || B < 1 || B > 65535) return fail(PCV_EINVAL, "kl_grad: bad arguments");
    cudaError_t e = pcv::launch_kl_grad(p, q, (const double2*)amp, N, B, q_batched, batch_scale, scale, (double2*)grad_amp,
                                        (cudaStream_t)stream);
    return e == cudaSuccess ? PCV_OK : cuda_fail(e, "kl_grad");
}

int pcv_prob_grad_to_amp(const double* grad_prob, const pcv_c64* amp, int64_t count, pcv_c64* grad_amp, void* stream)
{
    if (count < 0 || (count > 0 && (!grad_prob || !amp || !grad_amp))) return fail(PCV_EINVAL, "prob_grad: bad arguments");
    if (count == 0) return PCV_OK;
    cudaError_t e = pcv::launch_prob_grad(grad_prob, (const double2*)amp, count, (double2*)grad_amp, (cudaStream_t)stream);
    return e == cudaSuccess ? PCV_OK : cuda_fail(e, "prob_grad");
}

}  // extern "C"

// ------------------------------------------------------------ FP64 probe

namespace {
__global__ void fp64_probe_kernel(double* out, int iters)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double a0 = 1e-9 * t, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
    const double b = 0.9999999, c = 1e-7;
    for (int i = 0; i < iters; ++i) {
        a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
        a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
    }
    out[t] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}
}  // namespace

extern "C" int pcv_fp64_probe(double* out, int blocks, int threads, int iters, void* stream)
{
    if (!out || blocks < 1 || threads < 1 || threads > 1024 || iters < 1) return fail(PCV_EINVAL, "bad probe arguments");
    fp64_probe_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(out, iters);
    pcv::note_launches(1);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PCV_OK : cuda_fail(e, "fp64 probe");
}

// ------------------------------------------- partially distinguishable photons

namespace {

// Workspace of one class distribution of k photons: the default plan when it
// is at most 1 GiB, else the smallest plan.
int64_t class_dist_ws(int m, int k)
{
    if (k == 0) return 0;
    const int64_t full = pcv_distribution_workspace(m, k);
    if (full >= 0 && full <= (1ll << 30)) return full;
    return pcv_distribution_workspace_min(m, k);
}

int64_t tables_bytes(int m, int n) { return 2 * (int64_t)align256((size_t)(m + 1) * (n + 1) * sizeof(int64_t)); }

struct Classes {
    int m, n, G;                                  // G non-empty classes, largest first
    int size[PCV_MAX_PHOTONS];
    std::vector<uint8_t> occ;                     // G * m
};

int make_classes(int m, int G, const uint8_t* class_occ, Classes* c)
{
    if (m < 1 || m > PCV_MAX_MODES) return fail(PCV_EINVAL, "m=%d outside [1, %d]", m, PCV_MAX_MODES);
    if (G < 0 || G > 4096) return fail(PCV_EINVAL, "G=%d outside [0, 4096]", G);
    if (G > 0 && !class_occ) return fail(PCV_EINVAL, "class_occ is NULL");
    std::vector<std::pair<int, int>> order;      // (size, class)
    int n = 0;
    for (int g = 0; g < G; ++g) {
        int k = 0;
        for (int j = 0; j < m; ++j) k += class_occ[(size_t)g * m + j];
        if (k > PCV_MAX_PHOTONS) return fail(PCV_EINVAL, "class %d has %d photons", g, k);
        n += k;
        if (n > PCV_MAX_PHOTONS) return fail(PCV_EINVAL, "%d photons in all, more than %d", n, PCV_MAX_PHOTONS);
        if (k > 0) order.push_back({k, g});
    }
    std::stable_sort(order.begin(), order.end(), [](const std::pair<int, int>& a, const std::pair<int, int>& b) {
        return a.first > b.first;
    });
    if (msets(m, n) < 0) return fail(PCV_ERANGE, "output space too large");
    c->m = m;
    c->n = n;
    c->G = (int)order.size();
    c->occ.assign((size_t)c->G * m, 0);
    for (int g = 0; g < c->G; ++g) {
        c->size[g] = order[g].first;
        std::copy(class_occ + (size_t)order[g].second * m, class_occ + (size_t)(order[g].second + 1) * m,
                  c->occ.begin() + (size_t)g * m);
    }
    return PCV_OK;
}

int64_t classes_ws(const Classes& c)
{
    const int64_t N = msets(c.m, c.n);
    const int64_t NB = c.G > 1 ? msets(c.m, c.size[1]) : 0;
    int64_t dws = 0;
    for (int g = 0; g < c.G; ++g) {
        if (g > 0 && c.size[g] == 1) continue;
        const int64_t w = class_dist_ws(c.m, c.size[g]);
        if (w < 0) return w;
        dws = std::max(dws, w);
    }
    return tables_bytes(c.m, c.n) + 2 * (int64_t)align256((size_t)N * 8) + (int64_t)align256((size_t)NB * 8) + dws;
}

}  // namespace

int64_t pcv_distribution_classes_workspace(int m, int G, const uint8_t* class_occ)
{
    Classes c;
    const int rc = make_classes(m, G, class_occ, &c);
    if (rc) return rc;
    return classes_ws(c);
}

int pcv_distribution_classes(const pcv_c64* U, int m, int G, const uint8_t* class_occ, double* prob,
                             void* workspace, int64_t workspace_bytes, void* stream)
{
    Classes c;
    int rc = make_classes(m, G, class_occ, &c);
    if (rc) return rc;
    if (!U || !aligned(U, 16)) return fail(PCV_EINVAL, "U is NULL or not 16-byte aligned");
    if (!prob || !aligned(prob, 8)) return fail(PCV_EINVAL, "prob is NULL or not 8-byte aligned");
    const int64_t need = classes_ws(c);
    if (need < 0) return (int)need;
    if (!workspace || workspace_bytes < need)
        return fail(PCV_ENOMEM, "workspace of %lld bytes needed, %lld given", (long long)need, (long long)workspace_bytes);
    if (!aligned(workspace, 256)) return fail(PCV_EINVAL, "workspace is not 256-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (c.G == 0) {
        e = pcv::launch_set_one(prob, s);
        return e == cudaSuccess ? PCV_OK : cuda_fail(e, "empty input");
    }
    const int64_t N = msets(m, c.n);
    char* w = (char*)workspace;
    int64_t* mc = (int64_t*)w;               w += align256((size_t)(m + 1) * (c.n + 1) * sizeof(int64_t));
    int64_t* cum = (int64_t*)w;              w += align256((size_t)(m + 1) * (c.n + 1) * sizeof(int64_t));
    double* bufA = (double*)w;               w += align256((size_t)N * 8);
    double* bufC = (double*)w;               w += align256((size_t)N * 8);
    double* bufB = (double*)w;               w += align256((size_t)(c.G > 1 ? msets(m, c.size[1]) : 0) * 8);
    void* dws = w;
    const int64_t dws_bytes = need - (int64_t)(w - (char*)workspace);
    if ((e = pcv::build_multiset_table(mc, m, c.n, s)) != cudaSuccess) return cuda_fail(e, "multiset table");
    if ((e = pcv::build_cum_table(mc, m, c.n, cum, s)) != cudaSuccess) return cuda_fail(e, "rank table");
    double* cur = c.G == 1 ? prob : bufA;
    rc = pcv_distribution_ex(U, m, c.occ.data(), cur, nullptr, PCV_ALGO_AUTO, 0, dws, dws_bytes, stream);
    if (rc) return rc;
    int k = c.size[0];
    for (int g = 1; g < c.G; ++g) {
        double* out = g == c.G - 1 ? prob : (cur == bufA ? bufC : bufA);
        const uint8_t* t = c.occ.data() + (size_t)g * m;
        const int kn = k + c.size[g];
        if (c.size[g] == 1) {
            int mode = 0;
            while (t[mode] == 0) ++mode;
            e = pcv::launch_photon_step(mc, cum, m, c.n, kn, (const double2*)U, mode, nullptr, cur, 0.0, 1.0, out,
                                        msets(m, kn), s);
        } else {
            rc = pcv_distribution_ex(U, m, t, bufB, nullptr, PCV_ALGO_AUTO, 0, dws, dws_bytes, stream);
            if (rc) return rc;
            e = pcv::launch_class_conv(mc, cum, m, c.n, k, c.size[g], cur, bufB, out, msets(m, kn), s);
        }
        if (e != cudaSuccess) return cuda_fail(e, "class convolution");
        cur = out;
        k = kn;
    }
    return PCV_OK;
}

namespace {

constexpr int kSourceMaxPhotons = 16;

// Sum of |S_{m,k}| for k = 0..n (the photon-number-resolved output space).
int64_t graded_size(int m, int n)
{
    int64_t t = 0;
    for (int k = 0; k <= n; ++k) {
        const int64_t c = msets(m, k);
        if (c < 0 || t > INT64_MAX / 2) return -1;
        t += c;
    }
    return t;
}

int64_t source_ws(int m, int n)
{
    const int64_t T = graded_size(m, n);
    if (T < 0) return fail(PCV_ERANGE, "output space too large");
    int64_t dws = 0;
    for (int k = 1; k <= n; ++k) {
        const int64_t w = class_dist_ws(m, k);
        if (w < 0) return w;
        dws = std::max(dws, w);
    }
    return tables_bytes(m, n) + 2 * (int64_t)align256((size_t)T * 8) + dws;
}

int check_source_input(int m, const uint8_t* input_occ, int* n)
{
    if (m < 1 || m > PCV_MAX_MODES) return fail(PCV_EINVAL, "m=%d outside [1, %d]", m, PCV_MAX_MODES);
    if (!input_occ) return fail(PCV_EINVAL, "input_occ is NULL");
    int k = 0;
    for (int j = 0; j < m; ++j) k += input_occ[j];
    if (k > kSourceMaxPhotons) return fail(PCV_EINVAL, "source model supports n <= %d (n=%d)", kSourceMaxPhotons, k);
    *n = k;
    return PCV_OK;
}

}  // namespace

int64_t pcv_distribution_source_size(int m, int n)
{
    if (m < 1 || m > PCV_MAX_MODES || n < 0 || n > PCV_MAX_PHOTONS) return fail(PCV_EINVAL, "bad sizes");
    const int64_t T = graded_size(m, n);
    return T < 0 ? fail(PCV_ERANGE, "output space too large") : T;
}

int64_t pcv_distribution_source_workspace(int m, const uint8_t* input_occ)
{
    int n = 0;
    const int rc = check_source_input(m, input_occ, &n);
    if (rc) return rc;
    return source_ws(m, n);
}

int pcv_distribution_source(const pcv_c64* U, int m, const uint8_t* input_occ, double transmittance,
                            double indistinguishability, double* prob, void* workspace, int64_t workspace_bytes,
                            void* stream)
{
    int n = 0;
    int rc = check_source_input(m, input_occ, &n);
    if (rc) return rc;
    if (!(transmittance >= 0.0 && transmittance <= 1.0)) return fail(PCV_EINVAL, "transmittance outside [0, 1]");
    if (!(indistinguishability >= 0.0 && indistinguishability <= 1.0))
        return fail(PCV_EINVAL, "indistinguishability outside [0, 1]");
    if (!U || !aligned(U, 16)) return fail(PCV_EINVAL, "U is NULL or not 16-byte aligned");
    if (!prob || !aligned(prob, 8)) return fail(PCV_EINVAL, "prob is NULL or not 8-byte aligned");
    const int64_t need = source_ws(m, n);
    if (need < 0) return (int)need;
    if (!workspace || workspace_bytes < need)
        return fail(PCV_ENOMEM, "workspace of %lld bytes needed, %lld given", (long long)need, (long long)workspace_bytes);
    if (!aligned(workspace, 256)) return fail(PCV_EINVAL, "workspace is not 256-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t T = graded_size(m, n);
    int64_t off[PCV_MAX_PHOTONS + 2];
    off[0] = 0;
    for (int k = 0; k <= n; ++k) off[k + 1] = off[k] + msets(m, k);
    char* w = (char*)workspace;
    int64_t* mc = (int64_t*)w;               w += align256((size_t)(m + 1) * (n + 1) * sizeof(int64_t));
    int64_t* cum = (int64_t*)w;              w += align256((size_t)(m + 1) * (n + 1) * sizeof(int64_t));
    double* G0 = (double*)w;                 w += align256((size_t)T * 8);
    double* G1 = (double*)w;                 w += align256((size_t)T * 8);
    void* dws = w;
    const int64_t dws_bytes = need - (int64_t)(w - (char*)workspace);
    cudaError_t e = cudaMemsetAsync(prob, 0, (size_t)T * 8, s);
    if (e != cudaSuccess) return cuda_fail(e, "clear output");
    if ((e = pcv::build_multiset_table(mc, m, n, s)) != cudaSuccess) return cuda_fail(e, "multiset table");
    if ((e = pcv::build_cum_table(mc, m, n, cum, s)) != cudaSuccess) return cuda_fail(e, "rank table");
    // photon j enters mode modes[j]; a photon is absent (1 - eta), pure
    // (eta q) or noisy (eta (1 - q)), q = sqrt(indistinguishability)
    int modes[PCV_MAX_PHOTONS];
    for (int j = 0, c = 0; j < m; ++j)
        for (int r = 0; r < input_occ[j]; ++r) modes[c++] = j;
    const double eta = transmittance, q = std::sqrt(indistinguishability);
    const double alpha = 1.0 - eta, beta = eta * (1.0 - q), gamma = eta * q;
    std::vector<uint8_t> tP(m);
    for (uint32_t P = 0; P < (1u << n); ++P) {
        const int kP = __builtin_popcount(P);
        const double wP = std::pow(gamma, kP);
        if (wP == 0.0) continue;
        if (kP < n && alpha == 0.0 && beta == 0.0) continue;       // every other photon must be pure
        std::fill(tP.begin(), tP.end(), 0);
        for (int j = 0; j < n; ++j)
            if ((P >> j) & 1u) tP[modes[j]] += 1;
        double* cur = G0;
        double* nxt = G1;
        if (kP == 0) {
            if ((e = pcv::launch_set_one(cur + off[0], s)) != cudaSuccess) return cuda_fail(e, "pure set");
        } else {
            rc = pcv_distribution_ex(U, m, tP.data(), cur + off[kP], nullptr, PCV_ALGO_AUTO, 0, dws, dws_bytes, stream);
            if (rc) return rc;
        }
        int lo = kP, hi = kP;
        for (int j = 0; j < n; ++j) {
            if ((P >> j) & 1u) continue;
            const int klo = alpha == 0.0 ? hi + 1 : lo;
            for (int k = klo; k <= hi + 1; ++k) {
                const double* same = k <= hi ? cur + off[k] : nullptr;
                const double* prev = k - 1 >= lo ? cur + off[k - 1] : nullptr;
                e = pcv::launch_photon_step(mc, cum, m, n, k, (const double2*)U, modes[j], same, prev, alpha, beta,
                                            nxt + off[k], off[k + 1] - off[k], s);
                if (e != cudaSuccess) return cuda_fail(e, "photon step");
            }
            lo = klo;
            hi += 1;
            std::swap(cur, nxt);
        }
        if ((e = pcv::launch_scale_add(prob + off[lo], cur + off[lo], wP, off[hi + 1] - off[lo], s)) != cudaSuccess)
            return cuda_fail(e, "accumulate");
    }
    return PCV_OK;
}
