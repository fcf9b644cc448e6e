// Optional per-kernel timing: when enabled, every kernel launch of the
// library is bracketed by two CUDA events on its stream, and ct_profile_read
// turns the completed pairs into per-kind launch counts and device times.
#include <mutex>
#include <vector>

#include "ct_internal.cuh"

namespace ct {

static const char *const kKindNames[PROF_KINDS] = {
    "plane_copies", "joseph_A", "ramp_F", "pad_sino", "voxel_B", "mgs_pass",
    "small_fp64", "combine", "joseph_At", "voxel_Bt", "cgls_vector"};

namespace {
struct Pending {
    int kind;
    cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;
double g_ms[PROF_KINDS];
long long g_count[PROF_KINDS];

cudaEvent_t take_event()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}
}  // namespace

ProfScope::ProfScope(int kind, cudaStream_t st) : kind_(kind), st_(st), a_(nullptr)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return;
    a_ = take_event();
    if (a_) cudaEventRecord(static_cast<cudaEvent_t>(a_), st_);
}

ProfScope::~ProfScope()
{
    if (!a_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t b = take_event();
    if (!b) {
        g_pool.push_back(static_cast<cudaEvent_t>(a_));
        return;
    }
    cudaEventRecord(b, st_);
    g_pending.push_back(Pending{kind_, static_cast<cudaEvent_t>(a_), b});
}

// Load-path ceiling for the gather kernels.  Every block reads its own
// window of GP_WINDOW 16-byte words (16 KiB, resident in its SM's L1 after
// the first pass) GP_PASSES times with 128-bit read-only loads: in each pass
// a thread loads GP_UNROLL words, lanes on consecutive words, at an offset
// that moves with the pass (so no load repeats the previous pass's address
// and none can be hoisted out of the loop; the loads are volatile asm), and
// folds them into a sum that is stored only if it matches an impossible
// value.  Bytes moved per launch: blocks x GP_PASSES x GP_THREADS x
// GP_UNROLL x 16.
constexpr int GP_THREADS = 512;
constexpr int GP_WINDOW = 1024;            // words; a power of two
constexpr int GP_UNROLL = 4;
constexpr int GP_PASSES = 1024;

__device__ __forceinline__ float4 ld_nc_v4(const float4 *p)
{
    float4 v;
    asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

__global__ void __launch_bounds__(GP_THREADS) gather_peak_kernel(const float4 *__restrict__ buf, int windows,
                                                                 float *__restrict__ sink)
{
    const float4 *w = buf + size_t(blockIdx.x % windows) * GP_WINDOW;
    float4 acc[GP_UNROLL];
#pragma unroll
    for (int u = 0; u < GP_UNROLL; ++u) acc[u] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int pass = 0; pass < GP_PASSES; ++pass) {
        const int base = threadIdx.x + pass * 32;
#pragma unroll
        for (int u = 0; u < GP_UNROLL; ++u) {
            const float4 v = ld_nc_v4(w + ((base + u * (GP_WINDOW / GP_UNROLL)) & (GP_WINDOW - 1)));
            acc[u].x += v.x;
            acc[u].y += v.y;
            acc[u].z += v.z;
            acc[u].w += v.w;
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int u = 0; u < GP_UNROLL; ++u) s += acc[u].x + acc[u].y + acc[u].z + acc[u].w;
    if (s == -1.2345e30f) sink[0] = s;
}

}  // namespace ct

using namespace ct;

extern "C" {

void ct_profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = on != 0;
}

void ct_profile_reset(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &p : g_pending) {
        cudaEventSynchronize(p.b);
        g_pool.push_back(p.a);
        g_pool.push_back(p.b);
    }
    g_pending.clear();
    for (int i = 0; i < PROF_KINDS; ++i) {
        g_ms[i] = 0.0;
        g_count[i] = 0;
    }
}

int ct_profile_read(double *ms_out, long long *launches_out, int max_kinds)
{
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &p : g_pending) {
        float ms = 0.0f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            g_ms[p.kind] += ms;
            g_count[p.kind] += 1;
        } else {
            cudaGetLastError();
        }
        g_pool.push_back(p.a);
        g_pool.push_back(p.b);
    }
    g_pending.clear();
    const int n = max_kinds < PROF_KINDS ? max_kinds : PROF_KINDS;
    for (int i = 0; i < n; ++i) {
        if (ms_out) ms_out[i] = g_ms[i];
        if (launches_out) launches_out[i] = g_count[i];
    }
    return PROF_KINDS;
}

ct_status ct_measure_gather_peak(int repeats, double *gbs_out, void *stream)
{
    if (repeats < 1 || !gbs_out) return set_error(CT_EINVAL, "ct_measure_gather_peak: repeats >= 1 and gbs_out");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0, per_sm = 0;
    CT_CUDA(cudaGetDevice(&dev));
    CT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gather_peak_kernel, GP_THREADS, 0));
    if (per_sm < 1) per_sm = 1;
    const int blocks = sms * per_sm;
    const int windows = blocks;
    const size_t bytes = size_t(windows) * GP_WINDOW * sizeof(float4) + sizeof(float);
    void *buf = nullptr;
    CT_CUDA(cudaMallocAsync(&buf, bytes, st));
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaMemsetAsync(buf, 0, bytes, st);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float best = 0.0f;
    float4 *words = static_cast<float4 *>(buf);
    float *sink = reinterpret_cast<float *>(static_cast<char *>(buf) + bytes - sizeof(float));
    for (int r = 0; r <= repeats && e == cudaSuccess; ++r) {   // r = 0 warms up
        e = cudaEventRecord(a, st);
        if (e == cudaSuccess) {
            gather_peak_kernel<<<blocks, GP_THREADS, 0, st>>>(words, windows, sink);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && r > 0 && ms > 0.0f) {
            const float gbs = float(double(blocks) * GP_PASSES * GP_THREADS * GP_UNROLL * sizeof(float4) /
                                    (ms * 1e-3) / 1e9);
            if (gbs > best) best = gbs;
        }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFreeAsync(buf, st);
    if (e != cudaSuccess) return cuda_error(e, "ct_measure_gather_peak");
    CT_CUDA(cudaStreamSynchronize(st));
    *gbs_out = best;
    return CT_OK;
}

const char *ct_profile_kind_name(int kind)
{
    if (kind < 0 || kind >= PROF_KINDS) return "";
    return kKindNames[kind];
}

}  // extern "C"
