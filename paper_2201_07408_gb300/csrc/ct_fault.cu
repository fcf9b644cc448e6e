// Host-side fault injection for testing the solvers' failure paths without
// a GPU fault (no counterpart in the paper).  A spec, set by ct_fault_set or
// read once from the environment variable CT_FAULT when the library loads,
// is a comma-separated list of:
//   nan_at_iter:N  the solvers write a NaN into the new Krylov vector (GMRES)
//                  or into q = A p (CGLS) of iteration N (N >= 1), so the
//                  solve stops with CT_ENONFINITE after N - 1 iterations;
//   oom            allocations from the stream-ordered allocator are refused
//                  as if it had failed (CT_ENOMEM); caller workspaces still work.
// The NaN is an ordinary value written by a one-thread kernel; nothing
// faults, traps or waits.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include "ct_internal.cuh"

namespace ct {

namespace {
std::mutex g_fault_mu;
FaultSpec g_fault;
std::string g_fault_text;

bool parse_fault(const char *text, FaultSpec &out, std::string &canon, std::string &err)
{
    out = FaultSpec{};
    canon.clear();
    if (!text) return true;
    std::string s(text);
    size_t pos = 0;
    while (pos <= s.size()) {
        size_t end = s.find(',', pos);
        if (end == std::string::npos) end = s.size();
        std::string item = s.substr(pos, end - pos);
        pos = end + 1;
        if (item.empty() || item == "none") {
            if (end == s.size()) break;
            continue;
        }
        if (item == "oom") {
            out.oom = 1;
        } else if (item.compare(0, 12, "nan_at_iter:") == 0) {
            const char *num = item.c_str() + 12;
            char *stop = nullptr;
            const long v = std::strtol(num, &stop, 10);
            if (!*num || *stop || v < 1 || v > 1000000) {
                err = "nan_at_iter needs an iteration number >= 1: '" + item + "'";
                return false;
            }
            out.nan_at_iter = int(v);
        } else {
            err = "unknown fault '" + item + "' (known: nan_at_iter:N, oom, none)";
            return false;
        }
        if (end == s.size()) break;
    }
    if (out.nan_at_iter) canon = "nan_at_iter:" + std::to_string(out.nan_at_iter);
    if (out.oom) canon += std::string(canon.empty() ? "" : ",") + "oom";
    return true;
}

// CT_FAULT from the environment, once, when the library is loaded.
const bool g_env_loaded = [] {
    const char *env = std::getenv("CT_FAULT");
    if (!env) return true;
    FaultSpec f;
    std::string canon, err;
    if (parse_fault(env, f, canon, err)) {
        g_fault = f;
        g_fault_text = canon;
    } else {
        std::fprintf(stderr, "libct: ignoring CT_FAULT=%s: %s\n", env, err.c_str());
    }
    return true;
}();
}  // namespace

FaultSpec fault_spec()
{
    std::lock_guard<std::mutex> lk(g_fault_mu);
    return g_fault;
}

__global__ void poison_kernel(float *v, const int *stop)
{
    if (stop && *stop) return;
    v[0] = __int_as_float(0x7fc00000);   // quiet NaN
}

cudaError_t fault_poison(float *v, int iteration, const int *stop, cudaStream_t st)
{
    if (fault_spec().nan_at_iter != iteration) return cudaSuccess;
    poison_kernel<<<1, 1, 0, st>>>(v, stop);
    return cudaGetLastError();
}

}  // namespace ct

using namespace ct;

extern "C" {

ct_status ct_fault_set(const char *spec)
{
    FaultSpec f;
    std::string canon, err;
    if (!parse_fault(spec, f, canon, err)) return set_error(CT_EINVAL, "ct_fault_set: %s", err.c_str());
    std::lock_guard<std::mutex> lk(g_fault_mu);
    g_fault = f;
    g_fault_text = canon;
    return CT_OK;
}

const char *ct_fault_get(void)
{
    static thread_local std::string copy;
    std::lock_guard<std::mutex> lk(g_fault_mu);
    copy = g_fault_text;
    return copy.c_str();
}

int ct_bounds_checked(void)
{
#ifdef CT_CHECK_BOUNDS
    return 1;
#else
    return 0;
#endif
}

ct_status ct_bounds_take(ct_geom *geom, unsigned long long *record)
{
    if (!geom || !record) return set_error(CT_EINVAL, "ct_bounds_take: null argument");
    *record = 0;
#ifdef CT_CHECK_BOUNDS
    // on the geometry's device, whichever is current
    int prev = 0;
    cudaError_t e = cudaGetDevice(&prev);
    if (e == cudaSuccess && prev != geom->device) e = cudaSetDevice(geom->device);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaMemcpy(record, geom->g.bounds_word, sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(geom->g.bounds_word, 0, sizeof(unsigned long long));
    if (prev != geom->device) cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_error(e, "ct_bounds_take");
#endif
    return CT_OK;
}

}  // extern "C"
