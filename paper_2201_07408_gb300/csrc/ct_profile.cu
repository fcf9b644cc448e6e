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

const char *ct_profile_kind_name(int kind)
{
    if (kind < 0 || kind >= PROF_KINDS) return "";
    return kKindNames[kind];
}

}  // extern "C"
