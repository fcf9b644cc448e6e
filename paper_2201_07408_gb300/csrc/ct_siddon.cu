// Line-intersection projector A_S (Sec. III: the matrix element of ray i and
// voxel j is the length of the ray inside voxel j) and its exact transpose.
//
// One thread walks one ray through the grid voxel by voxel (a 3D digital
// differential analyser).  In grid units (voxel edge 1, the grid box
// [0, N_a] along each axis) the ray is o + t e with o = (S - lo)/vox and
// e = d/vox; the walk starts at the entry point p of the box and moves
// along the unit direction h = e/|e|.  Each axis keeps the distance (in
// voxel edges along h) still to go to its next boundary crossing; a step
// takes the smallest, which is the length of the ray in the current voxel,
// subtracts it from the other two and resets the crossed axis to the
// distance between its crossings, 1/|h_a|.  Every length is thus formed
// from quantities of voxel size, so FP32 resolves it to ~1e-7 of a voxel
// however long the ray; rounding only drifts the crossing points by about
// that much per step.  The walk ends when an index leaves the grid.  A
// direction component below 1e-12 counts as zero: the ray runs parallel to
// those planes, and one lying in a boundary plane belongs to the voxels on
// its positive side.  The projector reads the
// volume from the projector's zero-bordered y-major copy Yc (FP32, or bf16
// pairs whose low half is the voxel); the transpose adds into the plain
// volume with FP32 atomics.
#include "ct_internal.cuh"

namespace ct {

namespace {

struct RayWalk {
    float p[3], h[3];   // entry point (grid units), unit direction
};

// The ray of (view s, row iv, column iu); false when it misses the grid.
__device__ __forceinline__ bool ray_walk(const GeomDev &g, int s, int iv, int iu, RayWalk &w)
{
    const float4 *vp = reinterpret_cast<const float4 *>(g.viewA + s);
    const float4 a = __ldg(vp), b = __ldg(vp + 1);   // (dx0, dxu, dy0, dyu), (dzv, crossu, sx, sy)
    const float u = (float(iu) - g.cu) * g.du;
    float S[3], d[3];   // a point of the ray near the grid, and its direction
    if (g.kind == CT_CONE_3D) {
        // the ray meets the plane through the axis normal to the central ray
        // at (sod/sdd)(u e_u + v e_z), with e_u = (dxu, dyu, 0) = (a.y, a.w, 0):
        // a point of grid size, where the source point itself (sod away)
        // would lose its low bits when moved to the grid
        const float v = (float(iv) - g.cv) * g.dv;
        const float m = b.y / g.sdd;   // b.y = sod for the cone
        S[0] = m * u * a.y;
        S[1] = m * u * a.w;
        S[2] = m * v;
        d[0] = fmaf(u, a.y, a.x);
        d[1] = fmaf(u, a.w, a.z);
        d[2] = v * b.x;
    } else {   // the line u e_u + t e_d, e_u = (cos, sin), e_d = (-sin, cos) = (a.x, a.z)
        S[0] = u * a.z;
        S[1] = -u * a.x;
        S[2] = 0.0f;
        d[0] = a.x;
        d[1] = a.z;
        d[2] = 0.0f;
    }
    const float N[3] = {float(g.nx), float(g.ny), float(g.nz)};
    const float inv_dn = rsqrtf(fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2])));
    float o[3];
    float t_in = -3.0e38f, t_out = 3.0e38f;   // along h, from o
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        o[k] = S[k] * g.inv_vox + 0.5f * N[k];
        w.h[k] = d[k] * inv_dn;
        if (fabsf(w.h[k]) <= 1e-12f) {
            w.h[k] = 0.0f;
            if (!(o[k] > 0.0f && o[k] < N[k])) return false;
            continue;
        }
        const float inv = 1.0f / w.h[k];
        float t1 = -o[k] * inv, t2 = (N[k] - o[k]) * inv;
        if (t1 > t2) {
            const float t = t1;
            t1 = t2;
            t2 = t;
        }
        t_in = fmaxf(t_in, t1);
        t_out = fminf(t_out, t2);
    }
    if (!(t_out > t_in)) return false;
#pragma unroll
    for (int k = 0; k < 3; ++k) w.p[k] = fmaf(t_in, w.h[k], o[k]);
    return true;
}

// Calls visit(offset, length) for every voxel the ray crosses: offset =
// base + ix + iy ystride + iz zstride, kept up to date step by step (32-bit:
// ct_geom_create bounds every buffer below 2^31 elements), and the length
// inside the voxel in voxel units.  The per-axis state lives in scalars, so
// nothing is indexed at run time.
template <typename F>
__device__ __forceinline__ void walk(const GeomDev &g, const RayWalk &w, int base, int ystride, int zstride, F visit)
{
    // the voxel of the entry point: on the entry face the index is clamped
    // into the grid (the point lies on the boundary)
    int ix = min(max(int(floorf(w.p[0])), 0), g.nx - 1);
    int iy = min(max(int(floorf(w.p[1])), 0), g.ny - 1);
    int iz = min(max(int(floorf(w.p[2])), 0), g.nz - 1);
    const int sx = w.h[0] > 0.0f ? 1 : -1, sy = w.h[1] > 0.0f ? 1 : -1, sz = w.h[2] > 0.0f ? 1 : -1;
    int off = base + ix + iy * ystride + iz * zstride;
    const int ox = sx, oy = sy * ystride, oz = sz * zstride;
    // distance from p to the first crossing of an axis (voxel i), and between crossings
    auto first = [](float p, int i, float h) {
        return h > 0.0f ? (float(i + 1) - p) / h : (h < 0.0f ? (p - float(i)) / -h : 3.0e38f);
    };
    auto between = [](float h) { return h != 0.0f ? 1.0f / fabsf(h) : 3.0e38f; };
    float dx = first(w.p[0], ix, w.h[0]), dy = first(w.p[1], iy, w.h[1]), dz = first(w.p[2], iz, w.h[2]);
    const float tdx = between(w.h[0]), tdy = between(w.h[1]), tdz = between(w.h[2]);
    const int max_steps = g.nx + g.ny + g.nz + 3;
    for (int n = 0; n < max_steps; ++n) {
        const float dt = fminf(dx, fminf(dy, dz));
        // checked builds: the running offset is the voxel's (ix, iy, iz stay in the grid)
        if (!CT_IN_BOUNDS(g, off == base + ix + iy * ystride + iz * zstride, BS_SIDDON_VOXEL, iz, off - base))
            off = base + ix + iy * ystride + iz * zstride;
        visit(off, fmaxf(dt, 0.0f));
        // the axis crossed first steps (ties go to x, then y); the others move
        // dt closer to their next crossing.  Selects instead of branches: the
        // lanes of a warp cross different axes, and a three-way branch would
        // run all three paths one after the other.
        const bool mx = dx == dt, my = !mx && dy == dt, mz = !mx && !my;
        ix += mx ? sx : 0;
        iy += my ? sy : 0;
        iz += mz ? sz : 0;
        off += mx ? ox : (my ? oy : oz);
        dx = mx ? tdx : dx - dt;
        dy = my ? tdy : dy - dt;
        dz = mz ? tdz : dz - dt;
        if (unsigned(ix) >= unsigned(g.nx) || unsigned(iy) >= unsigned(g.ny) || unsigned(iz) >= unsigned(g.nz)) break;
    }
}

template <bool BF>
__global__ void __launch_bounds__(256) siddon_A_kernel(GeomDev g, const float *__restrict__ Yc,
                                                      float *__restrict__ y, SinoLayout lay,
                                                      const int *__restrict__ stop)
{
    if (stop && *stop) return;
    const long long ray = blockIdx.x * 256LL + threadIdx.x;
    const int per_view = g.nu * g.nv;
    if (ray >= (long long)per_view * g.n_views) return;
    const int s = int(ray / per_view);
    const int rem = int(ray - (long long)s * per_view);
    const int iv = rem / g.nu, iu = rem - iv * g.nu;
    RayWalk w;
    float acc = 0.0f;
    if (ray_walk(g, s, iv, iu, w)) {
        // Yc[zp][y][xp]: voxel (ix, iy, iz) at (iz + PAD_A) ny pitchY + iy pitchY + ix + PAD_A
        const int ystride = g.pitchY, zstride = g.ny * g.pitchY;
        walk(g, w, PAD_A * zstride + PAD_A, ystride, zstride, [&](int e, float len) {
            const float v = BF ? bf16_lo(__ldg(reinterpret_cast<const uint32_t *>(Yc) + e)) : __ldg(Yc + e);
            acc = fmaf(v, len, acc);
        });
    }
    store_sino(y, lay, s, iv, iu, acc * g.vox);
}

__global__ void __launch_bounds__(256) siddon_At_kernel(GeomDev g, const float *__restrict__ y,
                                                       float *__restrict__ x, const int *__restrict__ stop)
{
    if (stop && *stop) return;
    const long long ray = blockIdx.x * 256LL + threadIdx.x;
    const int per_view = g.nu * g.nv;
    if (ray >= (long long)per_view * g.n_views) return;
    const float yr = y[ray];
    if (yr == 0.0f) return;
    const int s = int(ray / per_view);
    const int rem = int(ray - (long long)s * per_view);
    const int iv = rem / g.nu, iu = rem - iv * g.nu;
    RayWalk w;
    if (!ray_walk(g, s, iv, iu, w)) return;
    // lengths come in voxel units: the ray's value carries the voxel size
    const float yv = yr * g.vox;
    walk(g, w, 0, g.nx, g.nx * g.ny, [&](int e, float len) {
        if (len > 0.0f) atomicAdd(x + e, yv * len);
    });
}

}  // namespace

cudaError_t launch_siddon_A(const GeomDev &g, const float *Yc, float *y, SinoLayout lay, const int *stop,
                            cudaStream_t st)
{
    const long long m = (long long)g.nu * g.nv * g.n_views;
    const unsigned blocks = unsigned((m + 255) / 256);
    if (g.vol_bf16)
        siddon_A_kernel<true><<<blocks, 256, 0, st>>>(g, Yc, y, lay, stop);
    else
        siddon_A_kernel<false><<<blocks, 256, 0, st>>>(g, Yc, y, lay, stop);
    return cudaGetLastError();
}

cudaError_t launch_siddon_At(const GeomDev &g, const float *y, float *x, const int *stop, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(x, 0, sizeof(float) * size_t(g.nx) * g.ny * g.nz, st);
    if (e != cudaSuccess) return e;
    const long long m = (long long)g.nu * g.nv * g.n_views;
    const unsigned blocks = unsigned((m + 255) / 256);
    siddon_At_kernel<<<blocks, 256, 0, st>>>(g, y, x, stop);
    return cudaGetLastError();
}

}  // namespace ct
