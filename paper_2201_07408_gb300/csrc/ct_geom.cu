// Geometry handle, per-view tables, error reporting and scratch arenas.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "ct_internal.cuh"

namespace ct {

static thread_local char g_err[512] = "";

ct_status set_error(ct_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

ct_status cuda_error(cudaError_t e, const char *what)
{
    return set_error(e == cudaErrorMemoryAllocation ? CT_ENOMEM : CT_ECUDA, "%s: %s (%s)", what,
                     cudaGetErrorString(e), cudaGetErrorName(e));
}

ct_status arena_open(Arena &a, size_t bytes, void *workspace, size_t workspace_bytes,
                     cudaStream_t stream)
{
    a = Arena{};
    a.stream = stream;
    a.size = bytes;
    if (bytes == 0) return CT_OK;
    if (workspace) {
        if (workspace_bytes < bytes)
            return set_error(CT_ENOMEM, "workspace of %zu bytes is smaller than the %zu needed",
                             workspace_bytes, bytes);
        if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0)
            return set_error(CT_EINVAL, "workspace must be 256-byte aligned");
        a.base = static_cast<char *>(workspace);
        a.owned = false;
        return CT_OK;
    }
    if (fault_spec().oom)
        return set_error(CT_ENOMEM, "cudaMallocAsync(%zu bytes) refused: fault injected by CT_FAULT=oom", bytes);
    void *p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes, stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(CT_ENOMEM, "cudaMallocAsync(%zu bytes) failed: %s", bytes,
                         cudaGetErrorString(e));
    }
    a.base = static_cast<char *>(p);
    a.owned = true;
    return CT_OK;
}

void arena_close(Arena &a)
{
    if (a.owned && a.base) cudaFreeAsync(a.base, a.stream);
    a = Arena{};
}

size_t plane_copies_bytes(const GeomDev &g)
{
    size_t xc = size_t(g.nzp) * g.nx * g.pitchX;
    size_t yc = size_t(g.nzp) * g.ny * g.pitchY;
    return Arena::align(xc * sizeof(float)) + Arena::align(yc * sizeof(float));
}

size_t padded_sino_bytes(const GeomDev &g)
{
    return Arena::align(size_t(g.n_views) * g.nvp * g.pitchU * 4 * sizeof(float));
}

cudaError_t raise_dyn_smem(const void *func, size_t bytes)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> limit;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    size_t &cur = limit[{dev, func}];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e == cudaSuccess) cur = bytes;
    return e;
}

int num_sms()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        sms = 132;
    return sms;
}

}  // namespace ct

using namespace ct;

extern "C" {

const char *ct_last_error(void) { return ct::g_err; }

const char *ct_version(void) { return "libct 0.1 (sm_103a)"; }

void ct_solve_opts_default(ct_solve_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->b_kind = CT_B_UN;
    o->tol = 0.0;
    o->dot_mode = 0;
    o->reorth = 0;
    o->record_data_resid = 0;
    o->workspace = nullptr;
    o->workspace_bytes = 0;
}

size_t ct_geom_n(const ct_geom *geom) { return geom ? geom->n : 0; }
size_t ct_geom_m(const ct_geom *geom) { return geom ? geom->m : 0; }

ct_status ct_geom_create(const ct_geom_desc *d, ct_geom **out)
{
    if (!out) return set_error(CT_EINVAL, "ct_geom_create: out is NULL");
    *out = nullptr;
    if (!d) return set_error(CT_EINVAL, "ct_geom_create: desc is NULL");
    if (d->kind != CT_PARALLEL_2D && d->kind != CT_CONE_3D)
        return set_error(CT_EINVAL, "unknown geometry kind %d", d->kind);
    if (d->nx <= 0 || d->ny <= 0 || d->nz <= 0 || d->nu <= 0 || d->nv <= 0 || d->n_views <= 0)
        return set_error(CT_EINVAL, "all grid, detector and view counts must be positive");
    if (!(d->voxel_mm > 0) || !(d->du_mm > 0) || !(d->dv_mm > 0))
        return set_error(CT_EINVAL, "voxel and pixel sizes must be positive");
    if (!std::isfinite(d->angle_start_rad) || !std::isfinite(d->angle_span_rad))
        return set_error(CT_EINVAL, "view angles must be finite");
    if (d->projector != CT_PROJ_JOSEPH && d->projector != CT_PROJ_SIDDON)
        return set_error(CT_EINVAL, "projector must be CT_PROJ_JOSEPH or CT_PROJ_SIDDON");
    if ((d->vol_dtype != CT_F32 && d->vol_dtype != CT_BF16) || (d->sino_dtype != CT_F32 && d->sino_dtype != CT_BF16))
        return set_error(CT_EINVAL, "storage dtypes must be CT_F32 or CT_BF16");
    if (d->kind == CT_PARALLEL_2D && (d->nz != 1 || d->nv != 1))
        return set_error(CT_EINVAL, "2D parallel beam needs nz = 1 and nv = 1");
    if (d->kind == CT_CONE_3D) {
        if (!(d->sod_mm > 0) || !(d->sdd_mm > d->sod_mm))
            return set_error(CT_EINVAL, "cone beam needs sdd > sod > 0");
        double hx = 0.5 * d->nx * d->voxel_mm, hy = 0.5 * d->ny * d->voxel_mm;
        if (std::sqrt(hx * hx + hy * hy) >= d->sod_mm)
            return set_error(CT_EINVAL, "the volume must lie inside the source circle");
    }
    // back-projector row margin: a voxel at height z projects to row
    // cv + M z/dv with M <= sdd/(sod - r_max); pad so that the floor of that
    // and the row above stay inside the zero-bordered buffer, for every
    // slice the threads compute (runs of up to B_ZC_RUN_MAX slices, so up
    // to a multiple of B_ZC_RUN_MAX past nz)
    int padv = PAD_V;
    if (d->kind == CT_CONE_3D) {
        const double vx = d->voxel_mm;
        const double rmax = std::sqrt(std::pow(0.5 * (d->nx - 1) * vx, 2) + std::pow(0.5 * (d->ny - 1) * vx, 2));
        const double mmax = d->sdd_mm / (d->sod_mm - rmax);
        const int nz_run = d->nz == 1 ? 1 : (d->nz + B_ZC_RUN_MAX - 1) / B_ZC_RUN_MAX * B_ZC_RUN_MAX;
        const double zslices = std::max(0.5 * (d->nz - 1), nz_run - 1 - 0.5 * (d->nz - 1));
        const double over = zslices * vx * mmax / d->dv_mm - 0.5 * (d->nv - 1);
        padv = std::max(PAD_V, int(std::ceil(std::max(over, 0.0))) + PAD_V);
    }
#ifdef CT_CHECK_BOUNDS
    // checked builds only: a margin may be imposed to exercise the row checks
    if (const char *ev = std::getenv("CT_DEBUG_PADV")) padv = std::max(1, std::atoi(ev));
#endif
    // 32-bit indexing of rays, voxels, padded copies and the padded sinogram
    const double lim = 2147483647.0;
    double nzp = d->nz + 2.0 * PAD_A;
    if (double(d->n_views) * d->nv * d->nu >= lim ||
        double(d->nx) * d->ny * d->nz >= lim ||
        nzp * d->nx * (d->ny + 2.0 * PAD_A) >= lim || nzp * d->ny * (d->nx + 2.0 * PAD_A) >= lim ||
        double(d->n_views) * (d->nv + 2.0 * padv) * (d->nu + 2.0 * PAD_U) * 4.0 >= lim)
        return set_error(CT_EINVAL, "problem too large for 32-bit element indexing");

    ct_geom *g = new ct_geom();
    g->desc = *d;
    cudaGetDevice(&g->device);
    g->n = size_t(d->nx) * d->ny * d->nz;
    g->m = size_t(d->n_views) * d->nv * d->nu;

    GeomDev &k = g->g;
    k.kind = d->kind;
    k.nx = d->nx; k.ny = d->ny; k.nz = d->nz;
    k.n_views = d->n_views; k.nu = d->nu; k.nv = d->nv;
    k.vox = float(d->voxel_mm);
    k.inv_vox = float(1.0 / d->voxel_mm);
    k.du = float(d->du_mm); k.dv = float(d->dv_mm);
    k.inv_du = float(1.0 / d->du_mm); k.inv_dv = float(1.0 / d->dv_mm);
    k.cx = 0.5f * (d->nx - 1); k.cy = 0.5f * (d->ny - 1); k.cz = 0.5f * (d->nz - 1);
    k.cu = 0.5f * (d->nu - 1); k.cv = 0.5f * (d->nv - 1);
    const bool cone = d->kind == CT_CONE_3D;
    const double vox = d->voxel_mm;
    k.kB = float(cone ? vox * vox * vox / (d->du_mm * d->dv_mm) : vox * vox / d->du_mm);
    k.sdd = float(cone ? d->sdd_mm : 1.0);
    k.nzp = d->nz + 2 * PAD_A;
    k.pitchX = d->ny + 2 * PAD_A;
    k.pitchY = d->nx + 2 * PAD_A;
    k.padv = padv;
    k.vol_bf16 = d->vol_dtype == CT_BF16;
    k.siddon = d->projector == CT_PROJ_SIDDON;
    k.sino_bf16 = d->sino_dtype == CT_BF16;
    k.nvp = d->nv + 2 * k.padv;
    k.pitchU = d->nu + 2 * PAD_U;

    // per-view tables (computed in double, stored in float)
    std::vector<ViewA> va(d->n_views);
    std::vector<ViewB> vb(d->n_views);
    for (int s = 0; s < d->n_views; ++s) {
        double th = d->angle_start_rad + double(s) * d->angle_span_rad / double(d->n_views);
        double c = std::cos(th), sn = std::sin(th);
        if (cone) {
            double sod = d->sod_mm, sdd = d->sdd_mm;
            va[s] = ViewA{float(-sdd * c), float(-sn), float(-sdd * sn), float(c), 1.0f,
                          float(sod), float(sod * c), float(sod * sn)};
            vb[s] = ViewB{float(sod), float(-c), float(-sn), float(-sn), float(c), float(sdd), 0.f, 0.f};
        } else {
            va[s] = ViewA{float(-sn), 0.0f, float(c), 0.0f, 0.0f, 1.0f, 0.0f, 0.0f};
            vb[s] = ViewB{1.0f, 0.0f, 0.0f, float(c), float(sn), 1.0f, 0.f, 0.f};
        }
    }
    // Projector checks over every ray of the scan.  On plane c a ray of
    // detector column u and row v is at z = v (c - S_a)/d_a, so consecutive
    // rays of a column are sigma = dv (c - S_a)/(d_a vox) voxels apart in z.
    // Both are affine in c, so their extremes over a column sit at the first
    // and last plane; every column of every view is visited (the dominant
    // axis switches inside views near 45 degrees).
    //   a_window: 0 <= sigma <= 0.98, so a two-row window per column suffices;
    //   a_zsafe:  |z| stays within the grid plus one voxel, so no clamp is needed;
    //             checked over the rows the threads compute, which run up to
    //             the next multiple of the rays per thread past nv.
    k.a_window = 0;
    k.a_zsafe = 1;
    if (cone) {
        double smin = 1e300, smax = -1e300;
        const int nv_run = (d->nv + A_VR_MAX - 1) / A_VR_MAX * A_VR_MAX;
        const double vmax = std::max(0.5 * (d->nv - 1), nv_run - 1 - 0.5 * (d->nv - 1)) * d->dv_mm;
        for (int s = 0; s < d->n_views; ++s) {
            double th = d->angle_start_rad + double(s) * d->angle_span_rad / double(d->n_views);
            double c = std::cos(th), sn = std::sin(th);
            for (int iu = 0; iu < d->nu; ++iu) {
                double u = (iu - 0.5 * (d->nu - 1)) * d->du_mm;
                double dx = -d->sdd_mm * c - u * sn, dy = -d->sdd_mm * sn + u * c;
                bool xdom = std::fabs(dx) >= std::fabs(dy);
                double da = xdom ? dx : dy, Sa = d->sod_mm * (xdom ? c : sn);
                int Na = xdom ? d->nx : d->ny;
                for (int e = 0; e < 2; ++e) {
                    double cp = (e ? 0.5 : -0.5) * (Na - 1) * vox;
                    double ratio = (cp - Sa) / da;
                    double sig = d->dv_mm * ratio / vox;
                    smin = std::min(smin, sig);
                    smax = std::max(smax, sig);
                    if (vmax * std::fabs(ratio) / vox > 0.5 * (d->nz - 1) + 1.0) k.a_zsafe = 0;
                }
            }
        }
        k.a_window = (smin >= 0.0 && smax <= 0.98) ? 1 : 0;
    }
#ifdef CT_CHECK_BOUNDS
    // checked builds only: the projector may be told that no z clamp is
    // needed, to exercise its z checks
    if (std::getenv("CT_DEBUG_A_ZSAFE")) k.a_zsafe = 1;
#endif
    // Ram-Lak taps of the ramp filter with the FBP scale folded in:
    // h[0] = 1/(4 tau^2), h[odd k] = -1/(pi^2 k^2 tau^2), h[even k] = 0, times tau * c_F.
    std::vector<float> taps(d->nu);
    std::vector<double> taps64(d->nu);
    {
        const double PI = 3.14159265358979323846;
        double tau = cone ? d->du_mm * d->sod_mm / d->sdd_mm : d->du_mm;
        double cf = (PI / d->n_views) *
                    (cone ? (d->sod_mm / d->sdd_mm) * (d->sod_mm / d->sdd_mm) * d->du_mm * d->dv_mm /
                                (vox * vox * vox)
                          : d->du_mm / (vox * vox));
        double scale = cf * tau;
        for (int q = 0; q < d->nu; ++q) {
            double h = q == 0 ? 1.0 / (4.0 * tau * tau)
                              : (q % 2 ? -1.0 / (PI * PI * double(q) * q * tau * tau) : 0.0);
            taps64[q] = h * scale;
            taps[q] = float(h * scale);
        }
    }
    // the same kernel as a spectrum: circular convolution of length N with
    // the kernel wrapped (h[q] at q and N - q) equals the linear one on the
    // first nu outputs when N >= 2 nu - 1; h is even, so H is real:
    //   H[k] = h[0] + 2 sum_{q >= 1} h[q] cos(2 pi q k / N)
    int fft_n = 8;
    while (fft_n < 2 * d->nu - 1) fft_n *= 2;
    std::vector<float2> fft_tw(fft_n);
    std::vector<float> fft_h(fft_n);
    {
        const double PI = 3.14159265358979323846;
        std::vector<double> cs(fft_n);
        for (int t = 0; t < fft_n; ++t) {
            cs[t] = std::cos(2.0 * PI * t / fft_n);
            fft_tw[t] = make_float2(float(cs[t]), float(-std::sin(2.0 * PI * t / fft_n)));
        }
        for (int kk = 0; kk < fft_n; ++kk) {
            double acc = taps64[0];
            for (int q = 1; q < d->nu; ++q) acc += 2.0 * taps64[q] * cs[size_t(q) * kk % fft_n];
            fft_h[kk] = float(acc / fft_n);
        }
    }
    size_t bA = Arena::align(va.size() * sizeof(ViewA));
    size_t bB = Arena::align(vb.size() * sizeof(ViewB));
    size_t bT = Arena::align(taps.size() * sizeof(float));
    size_t bW = Arena::align(fft_tw.size() * sizeof(float2));
    size_t bH = Arena::align(fft_h.size() * sizeof(float));
    size_t bWord = 0;
#ifdef CT_CHECK_BOUNDS
    bWord = Arena::align(sizeof(unsigned long long));
#endif
    cudaError_t e = cudaMalloc(&g->d_tables, bA + bB + bT + bW + bH + bWord);
    if (e != cudaSuccess) {
        delete g;
        return cuda_error(e, "cudaMalloc(geometry tables)");
    }
    char *base = static_cast<char *>(g->d_tables);
    e = cudaMemcpy(base, va.data(), va.size() * sizeof(ViewA), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(base + bA, vb.data(), vb.size() * sizeof(ViewB), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(base + bA + bB, taps.data(), taps.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(base + bA + bB + bT, fft_tw.data(), fft_tw.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(base + bA + bB + bT + bW, fft_h.data(), fft_h.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(g->d_tables);
        delete g;
        return cuda_error(e, "cudaMemcpy(geometry tables)");
    }
    k.viewA = reinterpret_cast<const ViewA *>(base);
    k.viewB = reinterpret_cast<const ViewB *>(base + bA);
    k.ramp_taps = reinterpret_cast<const float *>(base + bA + bB);
    k.fft_n = fft_n;
    k.fft_tw = reinterpret_cast<const float2 *>(base + bA + bB + bT);
    k.fft_h = reinterpret_cast<const float *>(base + bA + bB + bT + bW);
#ifdef CT_CHECK_BOUNDS
    k.bounds_word = reinterpret_cast<unsigned long long *>(base + bA + bB + bT + bW + bH);
    e = cudaMemset(k.bounds_word, 0, sizeof(unsigned long long));
    if (e != cudaSuccess) {
        cudaFree(g->d_tables);
        delete g;
        return cuda_error(e, "cudaMemset(bounds word)");
    }
#endif
    *out = g;
    return CT_OK;
}

void ct_geom_destroy(ct_geom *geom)
{
    if (!geom) return;
    if (geom->d_tables) {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(geom->device);
        cudaFree(geom->d_tables);
        cudaSetDevice(cur);
    }
    delete geom;
}

}  // extern "C"
