// Ray-driven Joseph projector A and its exact transpose A^T.
//
// A (Sec. I Eq. 1, Sec. III): every detector ray walks the voxel-centre
// planes of its dominant axis (x when |d_x| >= |d_y|, else y); on each plane
// it takes the bilinear interpolation of the four neighbouring voxels in
// that plane (neighbours outside the grid are zero), and the sum is scaled
// by the step length vox |d| / |d_a|.
//
// GPU layout.  The gathers run against two plane-major copies of the volume
// with a zero border of PAD_A voxels around the in-plane and z axes:
//   Xc[zp][x][yp]  for x-dominant rays (planes along x, in-plane axis y fastest),
//   Yc[zp][y][xp]  for y-dominant rays (planes along y, in-plane axis x fastest).
// Neighbouring rays of a detector row then read neighbouring words, and each
// ray's plane range is clipped up front so that the unrolled inner loop has no
// bounds tests.  Building the copies reads the volume once and is also where
// the Arnoldi step normalises its newest basis vector.
//
// Ray coordinates.  The sample position on plane p is affine in p:
//   f_b(p) = fbc + (p - c_a) gb,  f_z(p) = fzc + (p - c_a) gz
// with the value at the central plane computed from the cross product
// (S x d)_z rather than from S + t d, which in FP32 would cancel two terms of
// the size of the source distance; (S x d)_z = sod*u exactly for this
// geometry, so the intercept keeps full relative precision.
#include <mutex>

#include "ct_internal.cuh"

namespace ct {

struct RaySetup {
    int xdom;      // 1: planes along x
    int p0, p1;    // inclusive plane range that can hold nonzero samples
    float ca;      // (N_a - 1)/2
    float fbc, gb; // in-plane fractional index at the central plane, slope per plane
    float fzc, gz; // z fractional index at the central plane, slope per plane
    float weight;  // vox |d| / |d_a|
};

// Narrows [p0, p1] to the planes whose f(p) = fc + (p - ca) g lies in
// [lo - 0.5, hi + 0.5].  Every sample with f in [lo, hi) stays inside; every
// kept sample has floor(f) in [lo - 1, hi], inside the zero border.
__device__ __forceinline__ void clip_planes(float fc, float g, float lo, float hi, float ca, int Na,
                                            int &p0, int &p1)
{
    if (fabsf(g) < 1e-20f) {
        if (!(fc >= lo - 0.5f && fc <= hi + 0.5f)) p1 = -1;
        return;
    }
    float ig = 1.0f / g;
    float t1 = (lo - 0.5f - fc) * ig + ca;
    float t2 = (hi + 0.5f - fc) * ig + ca;
    float tl = fmaxf(fminf(t1, t2), -1.0f);
    float th = fminf(fmaxf(t1, t2), float(Na));
    p0 = max(p0, int(ceilf(tl)));
    p1 = min(p1, int(floorf(th)));
}

// Planes on which some ray of a run of rays has its coordinate f inside
// [lo, hi] (with clip_planes's half-voxel margin), the run's rays lying
// between its first ray (fc_f, g_f) and its last (fc_l, g_l) on every plane
// (f is linear in the ray's row, and the rows run in order).  On a plane the
// run covers [min(f_f, f_l), max(f_f, f_l)], so the plane is needed when one
// end ray is above lo and one end ray is below hi.  Each condition holds on a
// union of two half-lines of planes; its hull is taken (exact when one end
// ray stays above the other over the grid, as when the source lies outside
// the grid's plane range; otherwise a superset, whose extra planes add
// zeros).  Joining the two end rays' own plane ranges instead misses the far
// planes of the rays between them when the end rays leave through opposite
// faces (a short volume under a tall detector).
__device__ __forceinline__ void clip_planes_run(float fc_f, float g_f, float fc_l, float g_l, float lo, float hi,
                                                float ca, int Na, int &p0, int &p1)
{
    constexpr float BIG = 3.0e38f;
    auto hull = [](int a0, int a1, int b0, int b1, int &h0, int &h1) {
        if (a0 > a1) {
            h0 = b0;
            h1 = b1;
        } else if (b0 > b1) {
            h0 = a0;
            h1 = a1;
        } else {
            h0 = min(a0, b0);
            h1 = max(a1, b1);
        }
    };
    int a0 = 0, a1 = Na - 1, b0 = 0, b1 = Na - 1, u0, u1, w0, w1;
    clip_planes(fc_f, g_f, lo, BIG, ca, Na, a0, a1);   // first ray above lo
    clip_planes(fc_l, g_l, lo, BIG, ca, Na, b0, b1);   // last ray above lo
    hull(a0, a1, b0, b1, u0, u1);
    a0 = 0, a1 = Na - 1, b0 = 0, b1 = Na - 1;
    clip_planes(fc_f, g_f, -BIG, hi, ca, Na, a0, a1);  // first ray below hi
    clip_planes(fc_l, g_l, -BIG, hi, ca, Na, b0, b1);  // last ray below hi
    hull(a0, a1, b0, b1, w0, w1);
    p0 = max(p0, max(u0, w0));
    p1 = min(p1, min(u1, w1));
}

__device__ __forceinline__ RaySetup ray_setup(const GeomDev &g, int s, int iv, int iu)
{
    const float4 *vp = reinterpret_cast<const float4 *>(g.viewA + s);
    const float4 a = __ldg(vp), b = __ldg(vp + 1);
    // a = (dx0, dxu, dy0, dyu), b = (dzv, crossu, sx, sy)
    const float u = (float(iu) - g.cu) * g.du;
    const float v = (float(iv) - g.cv) * g.dv;
    const float dx = fmaf(u, a.y, a.x);
    const float dy = fmaf(u, a.w, a.z);
    const float dz = v * b.x;
    const float cross = u * b.y;
    RaySetup r;
    r.xdom = fabsf(dx) >= fabsf(dy);
    const float da = r.xdom ? dx : dy;
    const float db = r.xdom ? dy : dx;
    const float Sa = r.xdom ? b.z : b.w;
    const int Na = r.xdom ? g.nx : g.ny;
    const int Nb = r.xdom ? g.ny : g.nx;
    const float cb = r.xdom ? g.cy : g.cx;
    r.ca = r.xdom ? g.cx : g.cy;
    const float inv_da = 1.0f / da;
    r.gb = db * inv_da;
    // x-dominant: y(c) = (c d_y - cross)/d_x ; y-dominant: x(c) = (c d_x + cross)/d_y
    const float cterm = cross * inv_da * g.inv_vox;
    r.fbc = r.xdom ? cb - cterm : cb + cterm;
    r.gz = dz * inv_da;
    r.fzc = fmaf(-Sa * g.inv_vox, r.gz, g.cz);
    r.weight = g.vox * sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) * fabsf(inv_da);
    r.p0 = 0;
    r.p1 = Na - 1;
    clip_planes(r.fbc, r.gb, -1.0f, float(Nb), r.ca, Na, r.p0, r.p1);
    clip_planes(r.fzc, r.gz, -1.0f, float(g.nz), r.ca, Na, r.p0, r.p1);
    return r;
}

// ---------------------------------------------------------------------------
// Plane-major zero-bordered copies.  One block handles a 32x32 (x, y) tile
// of one padded z slice, read with a one-voxel halo so that bf16 pairs
// (b, b+1) can be formed; Yc rows are written straight from the tile, Xc
// rows from its transpose in shared memory.  When a basis slot is given the
// scaled volume is stored there too (each voxel by the tile that owns it).
// ---------------------------------------------------------------------------
template <bool BF>
__global__ void __launch_bounds__(256) plane_copies_kernel(GeomDev g, const float *__restrict__ vol,
                                                           const double *__restrict__ scale,
                                                           void *__restrict__ basis_out,
                                                           float *__restrict__ Xc, float *__restrict__ Yc,
                                                           const int *__restrict__ stop)
{
    if (stop && *stop) return;
    __shared__ float tile[33][33];
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    const int tid = ty * 32 + tx;
    const int xp0 = blockIdx.x * 32, yp0 = blockIdx.y * 32;  // padded tile origin
    const int zp = blockIdx.z;
    const int z = zp - PAD_A;
    const float sc = scale ? float(*scale) : 1.0f;
    const bool zin = z >= 0 && z < g.nz;
    for (int i = tid; i < 33 * 33; i += 256) {
        const int r = i / 33, c = i - r * 33;
        const int x = xp0 + c - PAD_A, y = yp0 + r - PAD_A;
        float val = 0.0f;
        if (zin && x >= 0 && x < g.nx && y >= 0 && y < g.ny) {
            const size_t idx = (size_t(z) * g.ny + y) * g.nx + x;
            val = vol[idx] * sc;
            if (basis_out && r < 32 && c < 32) {
                if (BF)
                    static_cast<__nv_bfloat16 *>(basis_out)[idx] = __float2bfloat16_rn(val);
                else
                    static_cast<float *>(basis_out)[idx] = val;
            }
        }
        tile[r][c] = val;
    }
    __syncthreads();
    // Yc[zp][y][xp] for y in the grid, xp over the padded row
    for (int r = ty; r < 32; r += 8) {
        const int y = yp0 + r - PAD_A, xp = xp0 + tx;
        if (y >= 0 && y < g.ny && xp < g.pitchY) {
            const size_t o = (size_t(zp) * g.ny + y) * g.pitchY + xp;
            if (BF)
                reinterpret_cast<uint32_t *>(Yc)[o] = pack_bf16x2(tile[r][tx], tile[r][tx + 1]);
            else
                Yc[o] = tile[r][tx];
        }
    }
    // Xc[zp][x][yp] for x in the grid, yp over the padded row
    for (int r = ty; r < 32; r += 8) {
        const int x = xp0 + r - PAD_A, yp = yp0 + tx;
        if (x >= 0 && x < g.nx && yp < g.pitchX) {
            const size_t o = (size_t(zp) * g.nx + x) * g.pitchX + yp;
            if (BF)
                reinterpret_cast<uint32_t *>(Xc)[o] = pack_bf16x2(tile[tx][r], tile[tx + 1][r]);
            else
                Xc[o] = tile[tx][r];
        }
    }
}

cudaError_t launch_plane_copies(const GeomDev &g, const float *vol, const double *scale, void *basis_out,
                                float *Xc, float *Yc, const int *stop, cudaStream_t st)
{
    ProfScope prof(PK_PLANE_COPIES, st);
    dim3 block(32, 8);
    dim3 grid((g.nx + 2 * PAD_A + 31) / 32, (g.ny + 2 * PAD_A + 31) / 32, g.nzp);
    if (g.vol_bf16)
        plane_copies_kernel<true><<<grid, block, 0, st>>>(g, vol, scale, basis_out, Xc, Yc, stop);
    else
        plane_copies_kernel<false><<<grid, block, 0, st>>>(g, vol, scale, basis_out, Xc, Yc, stop);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// y = A x.
//
// One thread walks A_VR rays of one detector column: same view and u,
// consecutive v.  On a flat detector those rays share d_x, d_y and the cross
// product, hence the dominant axis and the in-plane coordinate f_b(p) of every
// plane; only z differs, f_z(p, v) = cz + gz(v) (p - c_a - S_a/vox), with
// gz(v) = v dzv / d_a.  Per plane the thread interpolates along b once per
// z-row it needs and keeps a two-row window (rows zc, zc+1) that slides up as
// v increases (z is monotone in v along a column), so most rays cost one new
// row pair instead of two.  Lanes are consecutive u of one detector row
// segment and walk a warp-uniform plane range, so a warp's loads of one plane
// fall in a few consecutive sectors.  Samples outside a ray's own range have
// their row / column clamped into the zero border and add exactly zero.
// ---------------------------------------------------------------------------
constexpr int A_BLOCK = 128;

// b-interpolated value of one plane row: (1 - wb) V[b0] + wb V[b0+1], read as
// two floats or as one packed bf16 pair
template <bool BF>
__device__ __forceinline__ float row_lerp(const float *p, float wb)
{
    if (BF) {
        const uint32_t w = __ldg(reinterpret_cast<const uint32_t *>(p));
        const float v0 = bf16_lo(w), v1 = bf16_hi(w);
        return fmaf(wb, v1 - v0, v0);
    }
    const float v0 = __ldg(p), v1 = __ldg(p + 1);
    return fmaf(wb, v1 - v0, v0);
}

// plane-loop unroll (tuning): 2 for FP32 copies, 4 for bf16 pairs (measured
// at 256^3 with 16 rays per thread and 64 registers: 5.31 and 5.74 ms; unrolling the FP32
// loop by 1 or 4 took 8.44 and 5.63 ms, the bf16 loop by 2 8.76 ms); the
// rays per thread, A_VR, are in the shared header
#ifndef CT_A_PUNROLL
#define CT_A_PUNROLL 2
#endif
#ifndef CT_A_PUNROLL_BF
#define CT_A_PUNROLL_BF 4
#endif
constexpr int kAPlaneUnroll = CT_A_PUNROLL;
constexpr int kAPlaneUnrollBF = CT_A_PUNROLL_BF;
// resident blocks per SM that ptxas sizes the registers for (tuning): 5 for
// FP32 copies (96 registers), 4 for bf16 pairs (128).  At 256^3 these took
// 5.03 and 5.41 ms, against 5.29 and 5.73 ms with ptxas's own choice of 64
// registers (8 blocks); 6 or 7 blocks gave 5.07 / 5.04 ms (FP32), 9 blocks
// (56 registers) 8.5 ms.
constexpr int kAMinBlocks = 5;
constexpr int kAMinBlocksBF = 4;

template <int VR, bool WINDOW, bool ZCLAMP, bool BF>
__global__ void __launch_bounds__(A_BLOCK, BF ? kAMinBlocksBF : kAMinBlocks) joseph_A_kernel(GeomDev g, const float *__restrict__ Xc,
                                                           const float *__restrict__ Yc,
                                                           float *__restrict__ y, SinoLayout lay,
                                                           const int *__restrict__ stop)
{
    if (stop && *stop) return;
    const int lane_u = blockIdx.x * 32 + (threadIdx.x & 31);
    const int iv0 = (blockIdx.y * (A_BLOCK / 32) + (threadIdx.x >> 5)) * VR;
    const int s = blockIdx.z;
    const bool live = lane_u < g.nu && iv0 < g.nv;
    const int iu = min(lane_u, g.nu - 1);
    const int ivl = min(iv0 + VR - 1, g.nv - 1);

    // geometry shared by the column's rays
    const float4 *vp = reinterpret_cast<const float4 *>(g.viewA + s);
    const float4 a = __ldg(vp), b = __ldg(vp + 1);   // (dx0, dxu, dy0, dyu), (dzv, crossu, sx, sy)
    const float u = (float(iu) - g.cu) * g.du;
    const float dx = fmaf(u, a.y, a.x);
    const float dy = fmaf(u, a.w, a.z);
    const float cross = u * b.y;
    const bool xdom = fabsf(dx) >= fabsf(dy);
    const float da = xdom ? dx : dy;
    const float inv_da = 1.0f / da;
    const int Na = xdom ? g.nx : g.ny;
    const int Nb = xdom ? g.ny : g.nx;
    const float ca = xdom ? g.cx : g.cy;
    const float gb = (xdom ? dy : dx) * inv_da;
    const float cterm = cross * inv_da * g.inv_vox;
    const float fbc = xdom ? g.cy - cterm : g.cx + cterm;
    const float Sv = (xdom ? b.z : b.w) * g.inv_vox;   // source coordinate along the axis, in voxels
    const float gz_step = g.dv * b.x * inv_da;           // d gz / d iv
    const float gz0 = (float(iv0) - g.cv) * gz_step;     // gz of the first ray

    // plane range: the b range of the column met with the planes on which
    // any of its rays is inside the grid in z, then joined over the warp
    int p0 = 0, p1 = Na - 1;
    clip_planes(fbc, gb, -1.0f, float(Nb), ca, Na, p0, p1);
    {
        const float gzl = (float(ivl) - g.cv) * gz_step;
        clip_planes_run(fmaf(-Sv, gz0, g.cz), gz0, fmaf(-Sv, gzl, g.cz), gzl, -1.0f, float(g.nz), ca, Na, p0, p1);
    }
    if (!live) {  // idle lanes do not widen the warp's range
        p0 = Na;
        p1 = -1;
    }
    p0 = __reduce_min_sync(0xffffffffu, p0);
    p1 = __reduce_max_sync(0xffffffffu, p1);
    // lanes of one warp can differ in axis (views near 45 degrees); each stays
    // inside its own plane count
    p1 = min(p1, Na - 1);

    const float *__restrict__ base = xdom ? Xc : Yc;
    const int pitch = xdom ? g.pitchX : g.pitchY;
    const int zstride = Na * pitch;
    const int bmax = Nb, zmax = g.nz;

    float acc[VR];
#pragma unroll
    for (int i = 0; i < VR; ++i) acc[i] = 0.0f;

#pragma unroll (BF ? kAPlaneUnrollBF : kAPlaneUnroll)
    for (int p = p0; p <= p1; ++p) {
        const float pm = float(p) - ca;
        const float fb = fmaf(pm, gb, fbc);
        const float b0f = floorf(fb);
        const float wb = fb - b0f;
        const int b0 = min(max(int(b0f), -PAD_A), bmax);
        // element offset of (z = 0, plane p, b0) in the padded copy
        const float *rowp = base + (PAD_A * Na + p) * pitch + b0 + PAD_A;
        const float q = pm - Sv;
        const float fz0 = fmaf(gz0, q, g.cz);   // z of the first ray
        const float dzr = gz_step * q;          // z step from ray to ray
        float lo_prev = 0.0f, hi_prev = 0.0f;
        int z_prev = 0;
#pragma unroll
        for (int i = 0; i < VR; ++i) {
            const float fz = fmaf(float(i), dzr, fz0);
            const float z0f = floorf(fz);
            const float wz = fz - z0f;
            int z0 = ZCLAMP ? min(max(int(z0f), -PAD_A), zmax) : int(z0f);
            if (!ZCLAMP && !CT_IN_BOUNDS(g, z0 >= -PAD_A && z0 <= zmax + PAD_A - 2, BS_A_Z, s, z0)) z0 = -PAD_A;
            if (WINDOW && i > 0) (void)CT_IN_BOUNDS(g, z0 == z_prev || z0 == z_prev + 1, BS_A_WINDOW, s, z0 - z_prev);
            const float *r = rowp + (z0 + 1) * zstride;
            const float hi = row_lerp<BF>(r, wb);
            float lo;
            if (!WINDOW || i == 0) {
                lo = row_lerp<BF>(r - zstride, wb);
            } else {
                // z0 is z_prev or z_prev + 1: the low row is one of the previous rows
                lo = z0 == z_prev ? lo_prev : hi_prev;
            }
            acc[i] += fmaf(wz, hi - lo, lo);
            lo_prev = lo;
            hi_prev = hi;
            z_prev = z0;
        }
    }
    if (!live) return;
    const float dxy2 = fmaf(dx, dx, dy * dy);
#pragma unroll
    for (int i = 0; i < VR; ++i) {
        const int iv = iv0 + i;
        if (iv < g.nv) {
            const float v = (float(iv) - g.cv) * g.dv;
            const float dz = v * b.x;
            const float w = g.vox * sqrtf(fmaf(dz, dz, dxy2)) * fabsf(inv_da);
            store_sino(y, lay, s, iv, iu, acc[i] * w);
        }
    }
}

template <bool BF>
static void launch_joseph_A_t(const GeomDev &g, const float *Xc, const float *Yc, float *y, SinoLayout lay,
                              const int *stop, cudaStream_t st)
{
    constexpr int WPB = A_BLOCK / 32;
    if (g.nv == 1) {
        dim3 grid((g.nu + 31) / 32, (g.nv + WPB - 1) / WPB, g.n_views);
        joseph_A_kernel<1, false, true, BF><<<grid, A_BLOCK, 0, st>>>(g, Xc, Yc, y, lay, stop);
        return;
    }
    constexpr int VR = CT_A_VR;
    dim3 grid((g.nu + 31) / 32, (g.nv + WPB * VR - 1) / (WPB * VR), g.n_views);
#ifndef CT_A_FORCE_ZCLAMP
#define CT_A_FORCE_ZCLAMP 0
#endif
    if (g.a_window && g.a_zsafe && !CT_A_FORCE_ZCLAMP)
        joseph_A_kernel<VR, true, false, BF><<<grid, A_BLOCK, 0, st>>>(g, Xc, Yc, y, lay, stop);
    else if (g.a_window)
        joseph_A_kernel<VR, true, true, BF><<<grid, A_BLOCK, 0, st>>>(g, Xc, Yc, y, lay, stop);
    else
        joseph_A_kernel<VR, false, true, BF><<<grid, A_BLOCK, 0, st>>>(g, Xc, Yc, y, lay, stop);
}

cudaError_t launch_project_A(const GeomDev &g, const float *Xc, const float *Yc, float *y,
                            SinoLayout lay, const int *stop, cudaStream_t st)
{
    ProfScope prof(PK_JOSEPH_A, st);
    if (g.siddon) return launch_siddon_A(g, Yc, y, lay, stop, st);
    if (g.vol_bf16)
        launch_joseph_A_t<true>(g, Xc, Yc, y, lay, stop, st);
    else
        launch_joseph_A_t<false>(g, Xc, Yc, y, lay, stop, st);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// x = A^T y, the exact transpose of the projector above: the same column
// walk (AT_VR rays of one detector column per thread, warp-uniform plane
// range, the same sample positions and bilinear weights), scattering
// instead of gathering.  Contributions go with FP32 atomics into
// plane-major accumulators laid out like the projector's copies
// (Xa[zp][x][yp] for x-dominant rays, Ya[zp][y][xp]), so the lanes of a
// warp (consecutive u) add to neighbouring words of one row.  Within a
// thread the rays of a column add to a two-row window per plane, as the
// projector reads one: contributions to the same row are summed in
// registers and a row is flushed (two atomics: cells b0 and b0 + 1) when
// the window moves past it.  Samples on the zero border are skipped (they
// are zero entries of A).  A last pass adds the two accumulators into x.
// ---------------------------------------------------------------------------
template <int VR, bool WINDOW, bool ZCLAMP>
__global__ void __launch_bounds__(A_BLOCK) joseph_At_kernel(GeomDev g, const float *__restrict__ y,
                                                            float *__restrict__ Xa, float *__restrict__ Ya,
                                                            const int *__restrict__ stop)
{
    if (stop && *stop) return;
    const int lane_u = blockIdx.x * 32 + (threadIdx.x & 31);
    const int iv0 = (blockIdx.y * (A_BLOCK / 32) + (threadIdx.x >> 5)) * VR;
    const int s = blockIdx.z;
    const bool live = lane_u < g.nu && iv0 < g.nv;
    const int iu = min(lane_u, g.nu - 1);
    const int ivl = min(iv0 + VR - 1, g.nv - 1);

    const float4 *vp = reinterpret_cast<const float4 *>(g.viewA + s);
    const float4 a = __ldg(vp), b = __ldg(vp + 1);   // (dx0, dxu, dy0, dyu), (dzv, crossu, sx, sy)
    const float u = (float(iu) - g.cu) * g.du;
    const float dx = fmaf(u, a.y, a.x);
    const float dy = fmaf(u, a.w, a.z);
    const float cross = u * b.y;
    const bool xdom = fabsf(dx) >= fabsf(dy);
    const float da = xdom ? dx : dy;
    const float inv_da = 1.0f / da;
    const int Na = xdom ? g.nx : g.ny;
    const int Nb = xdom ? g.ny : g.nx;
    const float ca = xdom ? g.cx : g.cy;
    const float gb = (xdom ? dy : dx) * inv_da;
    const float cterm = cross * inv_da * g.inv_vox;
    const float fbc = xdom ? g.cy - cterm : g.cx + cterm;
    const float Sv = (xdom ? b.z : b.w) * g.inv_vox;
    const float gz_step = g.dv * b.x * inv_da;
    const float gz0 = (float(iv0) - g.cv) * gz_step;

    // each ray's value times its step weight (zero past nv and for idle lanes)
    float val[VR];
    bool any = false;
    {
        const float dxy2 = fmaf(dx, dx, dy * dy);
#pragma unroll
        for (int i = 0; i < VR; ++i) {
            const int iv = iv0 + i;
            val[i] = 0.0f;
            if (live && iv < g.nv) {
                const float v = (float(iv) - g.cv) * g.dv;
                const float dz = v * b.x;
                const float w = g.vox * sqrtf(fmaf(dz, dz, dxy2)) * fabsf(inv_da);
                val[i] = y[(size_t(s) * g.nv + iv) * g.nu + iu] * w;
                any = any || val[i] != 0.0f;
            }
        }
    }

    int p0 = 0, p1 = Na - 1;
    clip_planes(fbc, gb, -1.0f, float(Nb), ca, Na, p0, p1);
    {
        const float gzl = (float(ivl) - g.cv) * gz_step;
        clip_planes_run(fmaf(-Sv, gz0, g.cz), gz0, fmaf(-Sv, gzl, g.cz), gzl, -1.0f, float(g.nz), ca, Na, p0, p1);
    }
    if (!any) {   // nothing to add: this thread's rays do not widen the warp's range
        p0 = Na;
        p1 = -1;
    }
    p0 = __reduce_min_sync(0xffffffffu, p0);
    p1 = __reduce_max_sync(0xffffffffu, p1);
    p1 = min(p1, Na - 1);
    if (!any) return;   // after the warp-wide reductions

    float *__restrict__ base = xdom ? Xa : Ya;
    const int pitch = xdom ? g.pitchX : g.pitchY;
    const int zstride = Na * pitch;
    const int bmax = Nb, zmax = g.nz;

    for (int p = p0; p <= p1; ++p) {
        const float pm = float(p) - ca;
        const float fb = fmaf(pm, gb, fbc);
        const float b0f = floorf(fb);
        const float wb = fb - b0f;
        const int b0 = min(max(int(b0f), -PAD_A), bmax);
        const bool bl = b0 >= 0, bh = b0 + 1 < Nb;   // the two cells inside the grid
        if (!bl && !bh) continue;
        float *rowp = base + (PAD_A * Na + p) * pitch + b0 + PAD_A;   // (z = 0, plane p, b0)
        const float q = pm - Sv;
        const float fz0 = fmaf(gz0, q, g.cz);
        const float dzr = gz_step * q;
        // adds a row's summed contribution r to cells b0, b0 + 1 of grid row z
        auto flush = [&](int z, float r) {
            if (r == 0.0f || z < 0 || z >= zmax) return;
            float *c = rowp + z * zstride;
            if (bl) atomicAdd(c, r * (1.0f - wb));
            if (bh) atomicAdd(c + 1, r * wb);
        };
        int zc = 0;
        float acc_lo = 0.0f, acc_hi = 0.0f;   // rows zc and zc + 1
#pragma unroll
        for (int i = 0; i < VR; ++i) {
            const float fz = fmaf(float(i), dzr, fz0);
            const float z0f = floorf(fz);
            const float wz = fz - z0f;
            const int z0 = ZCLAMP ? min(max(int(z0f), -PAD_A), zmax) : int(z0f);
            const float c_lo = val[i] * (1.0f - wz), c_hi = val[i] * wz;
            if (!WINDOW) {
                flush(z0, c_lo);
                flush(z0 + 1, c_hi);
            } else if (i == 0) {
                zc = z0;
                acc_lo = c_lo;
                acc_hi = c_hi;
            } else if (z0 == zc) {
                acc_lo += c_lo;
                acc_hi += c_hi;
            } else {   // z0 == zc + 1: row zc is complete
                (void)CT_IN_BOUNDS(g, z0 == zc + 1, BS_AT_WINDOW, s, z0 - zc);
                flush(zc, acc_lo);
                zc = z0;
                acc_lo = acc_hi + c_lo;
                acc_hi = c_hi;
            }
        }
        if (WINDOW) {
            flush(zc, acc_lo);
            flush(zc + 1, acc_hi);
        }
    }
}

// x[z][y][x] = Xa[z][x][y] + Ya[z][y][x] over the grid (padded indices)
__global__ void __launch_bounds__(256) unplane_kernel(GeomDev g, const float *__restrict__ Xa,
                                                      const float *__restrict__ Ya, float *__restrict__ x,
                                                      const int *__restrict__ stop)
{
    if (stop && *stop) return;
    __shared__ float tile[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32, z = blockIdx.z;
    const size_t zp = size_t(z) + PAD_A;
    // tile[xl][yl] = Xa[zp][x0 + xl][y0 + yl + PAD_A], read along y
    for (int r = ty; r < 32; r += 8) {
        const int xx = x0 + r, yy = y0 + tx;
        tile[r][tx] = (xx < g.nx && yy < g.ny) ? Xa[(zp * g.nx + xx) * g.pitchX + yy + PAD_A] : 0.0f;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int yy = y0 + r, xx = x0 + tx;
        if (xx < g.nx && yy < g.ny)
            x[(size_t(z) * g.ny + yy) * g.nx + xx] = tile[tx][r] + Ya[(zp * g.ny + yy) * g.pitchY + xx + PAD_A];
    }
}

cudaError_t launch_project_At(const GeomDev &g, const float *y, float *x, float *Xa, float *Ya, const int *stop,
                             cudaStream_t st)
{
    ProfScope prof(PK_JOSEPH_AT, st);
    if (g.siddon) return launch_siddon_At(g, y, x, stop, st);
    cudaError_t e = cudaMemsetAsync(Xa, 0, sizeof(float) * size_t(g.nzp) * g.nx * g.pitchX, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(Ya, 0, sizeof(float) * size_t(g.nzp) * g.ny * g.pitchY, st);
    if (e != cudaSuccess) return e;
    constexpr int WPB = A_BLOCK / 32;
    if (g.nv == 1) {
        dim3 grid((g.nu + 31) / 32, (g.nv + WPB - 1) / WPB, g.n_views);
        joseph_At_kernel<1, false, true><<<grid, A_BLOCK, 0, st>>>(g, y, Xa, Ya, stop);
    } else {
        constexpr int VR = AT_VR;
        dim3 grid((g.nu + 31) / 32, (g.nv + WPB * VR - 1) / (WPB * VR), g.n_views);
        if (g.a_window && g.a_zsafe)
            joseph_At_kernel<VR, true, false><<<grid, A_BLOCK, 0, st>>>(g, y, Xa, Ya, stop);
        else if (g.a_window)
            joseph_At_kernel<VR, true, true><<<grid, A_BLOCK, 0, st>>>(g, y, Xa, Ya, stop);
        else
            joseph_At_kernel<VR, false, true><<<grid, A_BLOCK, 0, st>>>(g, y, Xa, Ya, stop);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 ublock(32, 8), ugrid((g.nx + 31) / 32, (g.ny + 31) / 32, g.nz);
    unplane_kernel<<<ugrid, ublock, 0, st>>>(g, Xa, Ya, x, stop);
    return cudaGetLastError();
}

}  // namespace ct

using namespace ct;

extern "C" ct_status ct_project_A(const ct_geom *geom, const float *x_dev, float *y_dev, void *stream)
{
    NvtxRange call_range("ct_project_A");
    if (!geom || !x_dev || !y_dev) return set_error(CT_EINVAL, "ct_project_A: NULL argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const GeomDev &g = geom->g;
    Arena ar;
    ct_status rc = arena_open(ar, plane_copies_bytes(g), nullptr, 0, st);
    if (rc != CT_OK) return rc;
    float *Xc = ar.take<float>(size_t(g.nzp) * g.nx * g.pitchX);
    float *Yc = ar.take<float>(size_t(g.nzp) * g.ny * g.pitchY);
    cudaError_t e = launch_plane_copies(g, x_dev, nullptr, nullptr, Xc, Yc, nullptr, st);
    if (e == cudaSuccess) e = launch_project_A(g, Xc, Yc, y_dev, plain_layout(g), nullptr, st);
    arena_close(ar);
    if (e != cudaSuccess) return cuda_error(e, "ct_project_A launch");
    return CT_OK;
}

extern "C" ct_status ct_adjoint_At(const ct_geom *geom, const float *y_dev, float *x_dev, void *stream)
{
    NvtxRange call_range("ct_adjoint_At");
    if (!geom || !y_dev || !x_dev) return set_error(CT_EINVAL, "ct_adjoint_At: NULL argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const GeomDev &g = geom->g;
    Arena ar;
    ct_status rc = arena_open(ar, plane_copies_bytes(g), nullptr, 0, st);
    if (rc != CT_OK) return rc;
    float *Xa = ar.take<float>(size_t(g.nzp) * g.nx * g.pitchX);
    float *Ya = ar.take<float>(size_t(g.nzp) * g.ny * g.pitchY);
    cudaError_t e = launch_project_At(g, y_dev, x_dev, Xa, Ya, nullptr, st);
    arena_close(ar);
    if (e != cudaSuccess) return cuda_error(e, "ct_adjoint_At launch");
    return CT_OK;
}

// ---------------------------------------------------------------------------
// Projector without allocation: the plane copies live in a fixed device
// array instead of stream-ordered scratch (see ct_project_A_noalloc in ct.h).
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kNoallocFloats = CT_NOALLOC_SCRATCH_BYTES / sizeof(float);
__device__ __align__(256) float g_noalloc_scratch[kNoallocFloats];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
float *g_noalloc_addr[kNoallocMaxDevices] = {};  // device address of the array, per device
}  // namespace

extern "C" ct_status ct_project_A_noalloc(const ct_geom *geom, const float *x_dev, float *y_dev,
                                          void *stream)
{
    if (!geom || !x_dev || !y_dev) return set_error(CT_EINVAL, "ct_project_A_noalloc: NULL argument");
    const GeomDev &g = geom->g;
    const size_t xc_bytes = Arena::align(size_t(g.nzp) * g.nx * g.pitchX * sizeof(float));
    const size_t yc_bytes = Arena::align(size_t(g.nzp) * g.ny * g.pitchY * sizeof(float));
    if (xc_bytes + yc_bytes > size_t(CT_NOALLOC_SCRATCH_BYTES))
        return set_error(CT_EINVAL,
                         "ct_project_A_noalloc: this volume needs %zu bytes of projector scratch, more than "
                         "the %zu-byte fixed scratch; use ct_project_A",
                         xc_bytes + yc_bytes, size_t(CT_NOALLOC_SCRATCH_BYTES));
    int dev = -1;
    CT_CUDA(cudaGetDevice(&dev));
    if (dev != geom->device)
        return set_error(CT_EINVAL, "ct_project_A_noalloc: the geometry lives on device %d but device %d is current",
                         geom->device, dev);
    if (dev < 0 || dev >= kNoallocMaxDevices)
        return set_error(CT_EINVAL, "ct_project_A_noalloc: device index %d is out of range", dev);
    float *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(projector scratch)");
            g_noalloc_addr[dev] = static_cast<float *>(p);
        }
        base = g_noalloc_addr[dev];
    }
    float *Xc = base;
    float *Yc = base + xc_bytes / sizeof(float);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_plane_copies(g, x_dev, nullptr, nullptr, Xc, Yc, nullptr, st);
    if (e == cudaSuccess) e = launch_project_A(g, Xc, Yc, y_dev, plain_layout(g), nullptr, st);
    if (e != cudaSuccess) return cuda_error(e, "ct_project_A_noalloc launch");
    return CT_OK;
}
