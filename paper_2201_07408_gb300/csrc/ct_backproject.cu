// Voxel-driven back-projector B_un, ramp filter F (B_FBP = B_un F) and the
// exact transposes B_un^T, F^T (Sec. III).
//
// B_un: for every voxel and view, the voxel centre is projected from the
// source onto the detector (depth W, magnification M = sdd/W, u = M t,
// v = M z), the detector value there is interpolated bilinearly (zero
// outside) and accumulated with weight kB M^2.
//
// GPU layout.  One thread owns a column (x, y) and a run of ZC consecutive
// z; per view it computes W, M, u and the u-interpolation weights once and
// then walks its z run with v affine in z.  The sinogram is read from a
// copy with zero borders (PAD_U pixels along u, PAD_V rows along v): a view
// whose u footprint misses the detector is skipped, and clamping the row
// index into the border makes every other gather in bounds.
#include <algorithm>

#include "ct_internal.cuh"

namespace ct {

// ---------------------------------------------------------------------------
// Plain -> padded sinogram copy (optionally scaled, optionally normalising
// the source in place).
// ---------------------------------------------------------------------------
template <bool BF>
__global__ void pad_sino_kernel(GeomDev g, const float *__restrict__ src, const double *__restrict__ scale,
                                void *__restrict__ dst, const int *__restrict__ stop)
{
    if (stop && *stop) return;
    const size_t total = size_t(g.n_views) * g.nvp * g.pitchU;
    const float sc = scale ? float(*scale) : 1.0f;
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < total;
         i += size_t(gridDim.x) * blockDim.x) {
        const int up = int(i % g.pitchU);
        const size_t t = i / g.pitchU;
        const int vp = int(t % g.nvp);
        const int s = int(t / g.nvp);
        const int u = up - PAD_U, v = vp - g.padv;
        const float *view = src + size_t(s) * g.nv * g.nu;
        const bool u0 = u >= 0 && u < g.nu, u1 = u + 1 >= 0 && u + 1 < g.nu;
        const bool v0 = v >= 0 && v < g.nv, v1 = v + 1 >= 0 && v + 1 < g.nv;
        float4 q;
        q.x = (v0 && u0) ? view[size_t(v) * g.nu + u] * sc : 0.0f;
        q.y = (v0 && u1) ? view[size_t(v) * g.nu + u + 1] * sc : 0.0f;
        q.z = (v1 && u0) ? view[size_t(v + 1) * g.nu + u] * sc : 0.0f;
        q.w = (v1 && u1) ? view[size_t(v + 1) * g.nu + u + 1] * sc : 0.0f;
        if (BF)
            static_cast<uint2 *>(dst)[i] = make_uint2(pack_bf16x2(q.x, q.y), pack_bf16x2(q.z, q.w));
        else
            static_cast<float4 *>(dst)[i] = q;
    }
}

// src *= (*scale): the Arnoldi normalisation of a data-space basis vector,
// after its padded copy has been taken from the unscaled values.
__global__ void scale_inplace_kernel(float *__restrict__ v, size_t len, const double *__restrict__ scale,
                                     const int *__restrict__ stop)
{
    if (stop && *stop) return;
    const float sc = float(*scale);
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < len; i += size_t(gridDim.x) * blockDim.x)
        v[i] *= sc;
}

cudaError_t launch_pad_sino(const GeomDev &g, float *src, const double *scale, bool normalize_inplace,
                            float *dst, const int *stop, cudaStream_t st)
{
    ProfScope prof(PK_PAD_SINO, st);
    const size_t total = size_t(g.n_views) * g.nvp * g.pitchU;
    unsigned blocks = unsigned(std::min<size_t>((total + 255) / 256, size_t(num_sms()) * 16));
    if (g.sino_bf16)
        pad_sino_kernel<true><<<blocks, 256, 0, st>>>(g, src, scale, dst, stop);
    else
        pad_sino_kernel<false><<<blocks, 256, 0, st>>>(g, src, scale, dst, stop);
    if (normalize_inplace && cudaGetLastError() == cudaSuccess)
        scale_inplace_kernel<<<blocks, 256, 0, st>>>(src, size_t(g.n_views) * g.nv * g.nu, scale, stop);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Ramp filter.  The Ram-Lak kernel is zero at even nonzero offsets, so each
// output parity only sees samples of the other parity:
//   out[2i]   = h0 E[i] + sum_m g[m] (O[i-m-1] + O[i+m])
//   out[2i+1] = h0 O[i] + sum_m g[m] (E[i-m]   + E[i+m+1])
// with E, O the even / odd samples of the (cosine-weighted) row and
// g[m] = h[2m+1].  A thread computes RAMP_R consecutive outputs of one
// parity for two detector rows at once: the two rows are interleaved in
// shared memory (float2), so each tap costs two 8-byte shared loads and
// RAMP_R packed FADD2/FFMA2 for 2*RAMP_R outputs.  The two register windows
// slide by one sample per tap as ring buffers whose slot indices are
// compile-time constants (the tap loop is unrolled by RAMP_R and the tap
// count padded with zero taps), so sliding costs no moves.  RAMP_R is odd
// so that the window loads of neighbouring threads fall in distinct banks.
// Rows sit in shared memory with zero margins, so no load is bounds-tested.
// F^T weights the output instead of the input.
// ---------------------------------------------------------------------------
constexpr int RAMP_R = 9;

struct RampShape {
    int M;       // taps g[0..M-1], M a multiple of RAMP_R (zero taps past nu/2)
    int mpad;    // floats reserved for the taps: M rounded up to 4, so the float2 rows start 16-byte aligned
    int nhE, nhO;
    int off;     // index of sample 0 inside a half-row array
    int len;     // length of one half-row array (float2 entries)
    int tpr;     // threads per row pair
    int pairs;   // row pairs per block
    int threads;
    size_t smem;
};

static RampShape ramp_shape(int nu)
{
    RampShape r;
    const int mtaps = nu / 2;
    r.M = ((mtaps + RAMP_R - 1) / RAMP_R) * RAMP_R;
    if (r.M == 0) r.M = RAMP_R;
    r.nhE = (nu + 1) / 2;
    r.nhO = nu / 2;
    r.off = r.M + 1;
    r.len = r.off + r.nhE + RAMP_R + r.M + 2;
    r.tpr = (r.nhE + RAMP_R - 1) / RAMP_R + (r.nhO + RAMP_R - 1) / RAMP_R;
    r.pairs = r.tpr >= 256 ? 1 : 256 / r.tpr;
    r.threads = ((r.tpr * r.pairs + 31) / 32) * 32;
    r.mpad = (r.M + 3) & ~3;
    r.smem = sizeof(float) * size_t(r.mpad) + sizeof(float2) * size_t(r.pairs) * 2 * r.len;
    return r;
}

__device__ __forceinline__ float cosine_weight(const GeomDev &g, int iu, int iv)
{
    if (g.kind != CT_CONE_3D) return 1.0f;
    const float u = (float(iu) - g.cu) * g.du;
    const float v = (float(iv) - g.cv) * g.dv;
    return g.sdd / sqrtf(fmaf(g.sdd, g.sdd, fmaf(u, u, v * v)));
}

__device__ __forceinline__ int ring(int x) { return ((x % RAMP_R) + RAMP_R) % RAMP_R; }

// acc[j] = h0 C[i0+j] + sum_m g[m] (L[i0+j-m-AL] + L[i0+j+m+AR]) for two rows at once
template <int AL, int AR>
__device__ __forceinline__ void ramp_conv(const float2 *__restrict__ L, const float2 *__restrict__ C,
                                          const float *__restrict__ gm, int M, int i0, float h0,
                                          float2 (&acc)[RAMP_R])
{
    // ring slots: left element q = i0 + j - m - AL sits in slot ring(q - i0),
    // right element q = i0 + j + m + AR in slot ring(q - i0)
    float2 Lw[RAMP_R], Rw[RAMP_R];
#pragma unroll
    for (int j = 0; j < RAMP_R; ++j) {   // state before tap 0 (m = -1)
        Lw[ring(j + 1 - AL)] = L[i0 + j + 1 - AL];
        Rw[ring(j - 1 + AR)] = L[i0 + j - 1 + AR];
        const float2 c = C[i0 + j];
        acc[j] = make_float2(h0 * c.x, h0 * c.y);
    }
    for (int m0 = 0; m0 < M; m0 += RAMP_R) {
#pragma unroll
        for (int t = 0; t < RAMP_R; ++t) {
            const int m = m0 + t;
            Lw[ring(-t - AL)] = L[i0 - m - AL];                 // enters at j = 0
            Rw[ring(RAMP_R - 1 + t + AR)] = L[i0 + RAMP_R - 1 + m + AR];   // enters at j = R-1
            const float gv = gm[m];
            const float2 g2 = make_float2(gv, gv);
#pragma unroll
            for (int j = 0; j < RAMP_R; ++j)
                acc[j] = __ffma2_rn(g2, __fadd2_rn(Lw[ring(j - t - AL)], Rw[ring(j + t + AR)]), acc[j]);
        }
    }
}

__global__ void ramp_kernel(GeomDev g, RampShape rs, const float *__restrict__ src, float *__restrict__ dst,
                            SinoLayout lay, int transpose, const int *__restrict__ stop)
{
    if (stop && *stop) return;
    extern __shared__ float sm[];
    const int nu = g.nu;
    const int nrows = g.n_views * g.nv;
    float *gm = sm;                                                 // taps g[m] = h[2m+1]
    float2 *half = reinterpret_cast<float2 *>(sm + rs.mpad);        // [pair][E | O][len]
    const int row_base = blockIdx.x * rs.pairs * 2;
    for (int i = threadIdx.x; i < rs.M; i += blockDim.x) gm[i] = 2 * i + 1 < nu ? g.ramp_taps[2 * i + 1] : 0.0f;
    for (int i = threadIdx.x; i < rs.pairs * 2 * rs.len; i += blockDim.x) half[i] = make_float2(0.0f, 0.0f);
    __syncthreads();
    float *halff = reinterpret_cast<float *>(half);
    for (int i = threadIdx.x; i < rs.pairs * 2 * nu; i += blockDim.x) {
        const int lr = i / nu, iu = i - lr * nu;     // lr: row within the block
        const int r = row_base + lr;
        if (r >= nrows) continue;
        const int iv = r % g.nv;
        const float w = transpose ? 1.0f : cosine_weight(g, iu, iv);
        const int pair = lr >> 1, comp = lr & 1;
        const size_t e = (size_t(pair) * 2 + (iu & 1)) * rs.len + rs.off + (iu >> 1);
        halff[2 * e + comp] = src[size_t(r) * nu + iu] * w;
    }
    __syncthreads();
    const int lp = threadIdx.x / rs.tpr;
    const int tile = threadIdx.x - lp * rs.tpr;
    const int r0 = row_base + 2 * lp;
    if (lp >= rs.pairs || r0 >= nrows) return;
    const float2 *E = half + size_t(lp) * 2 * rs.len + rs.off;
    const float2 *O = E + rs.len;
    const int tilesE = (rs.nhE + RAMP_R - 1) / RAMP_R;
    const int parity = tile < tilesE ? 0 : 1;
    const int i0 = (parity ? tile - tilesE : tile) * RAMP_R;
    const float h0 = g.ramp_taps[0];
    float2 acc[RAMP_R];
    if (parity == 0)
        ramp_conv<1, 0>(O, E, gm, rs.M, i0, h0, acc);
    else
        ramp_conv<0, 1>(E, O, gm, rs.M, i0, h0, acc);
    const int nh = parity ? rs.nhO : rs.nhE;
    const bool second = r0 + 1 < nrows;
    const int iv0 = r0 % g.nv, s0 = r0 / g.nv;
    const int iv1 = (r0 + 1) % g.nv, s1 = (r0 + 1) / g.nv;
#pragma unroll
    for (int j = 0; j < RAMP_R; ++j) {
        const int i = i0 + j;
        if (i < nh) {
            const int iu = 2 * i + parity;
            store_sino(dst, lay, s0, iv0, iu, transpose ? acc[j].x * cosine_weight(g, iu, iv0) : acc[j].x);
            if (second)
                store_sino(dst, lay, s1, iv1, iu, transpose ? acc[j].y * cosine_weight(g, iu, iv1) : acc[j].y);
        }
    }
}

cudaError_t launch_ramp(const GeomDev &g, const float *src, float *dst, SinoLayout lay, bool transpose,
                        const int *stop, cudaStream_t st)
{
    const RampShape rs = ramp_shape(g.nu);
    if (rs.smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(ramp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(rs.smem));
        if (e != cudaSuccess) return e;
    }
    const int nrows = g.n_views * g.nv;
    const unsigned blocks = unsigned((nrows + 2 * rs.pairs - 1) / (2 * rs.pairs));
    ProfScope prof(PK_RAMP, st);
    ramp_kernel<<<blocks, rs.threads, rs.smem, st>>>(g, rs, src, dst, lay, transpose ? 1 : 0, stop);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// x = B_un y.
// ---------------------------------------------------------------------------
constexpr int B_BX = 32, B_BY = 4;

struct ColumnView {
    int skip;       // the u footprint misses the detector
    int col;        // padded column of the left neighbour
    float a0, a1;   // weight * (1 - wu), weight * wu
    float fv0, gv;  // v fractional index of the first z of the run, slope per z
};

// p = (w0, wx, wy, tx), q = (ty, mnum, -, -) of one view
__device__ __forceinline__ ColumnView column_view(const GeomDev &g, float4 p, float4 q, float x, float y,
                                                  float zfirst)
{
    const float W = fmaf(x, p.y, fmaf(y, p.z, p.x));
    const float t = fmaf(x, p.w, y * q.x);
    // 1/W: hardware approximation refined by one Newton step (W is a depth of
    // hundreds of mm, or 1 in 2D, never denormal)
    float rw;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rw) : "f"(W));
    rw = fmaf(rw, fmaf(-W, rw, 1.0f), rw);
    const float M = q.y * rw;
    const float fu = fmaf(M * t, g.inv_du, g.cu);
    const float u0f = floorf(fu);
    const float wu = fu - u0f;
    ColumnView c;
    const int u0 = int(fmaxf(fminf(u0f, float(g.nu + 1)), -2.0f));
    c.skip = (u0 < -1) || (u0 > g.nu - 1);
    c.col = u0 + PAD_U;
    const float w = g.kB * M * M;
    c.a0 = w * (1.0f - wu);
    c.a1 = w * wu;
    c.gv = M * g.vox * g.inv_dv;
    c.fv0 = fmaf(M * zfirst, g.inv_dv, g.cv);
    return c;
}

__device__ __forceinline__ ColumnView column_view(const GeomDev &g, int s, float x, float y, float zfirst)
{
    const float4 *vp = reinterpret_cast<const float4 *>(g.viewB + s);
    return column_view(g, __ldg(vp), __ldg(vp + 1), x, y, zfirst);
}

// A block owns a 32 x 32 tile of (x, y) columns and B_ZC consecutive z.
// Which of x or y its lanes run along is chosen per view: the axis closer
// to the view's central ray (along x when |tx| <= |ty|, i.e. when u moves
// more slowly with x than with y).  Along the central ray the projection
// barely moves (only the magnification changes, by vox/depth per voxel), so
// a warp's gathers fall on a few neighbouring pixels of a few rows; across
// it, u moves by M vox/du pixels per lane.  The two partial sums (x-lane
// views and y-lane views) meet in shared memory.  The sinogram is read as
// quads (the 2 x 2 bilinear neighbourhood), one 16-byte load per voxel and
// view; the view table sits in shared memory.
constexpr int B_TILE = 32;

// the four bilinear neighbours of one sinogram quad entry
template <bool BF>
__device__ __forceinline__ float4 load_quad(const void *base, size_t e)
{
    if (BF) {
        const uint2 w = __ldg(static_cast<const uint2 *>(base) + e);
        return make_float4(bf16_lo(w.x), bf16_hi(w.x), bf16_lo(w.y), bf16_hi(w.y));
    }
    return __ldg(static_cast<const float4 *>(base) + e);
}

template <int ZC, bool BF>
__global__ void __launch_bounds__(B_TILE *B_TILE) voxel_B_kernel(GeomDev g, const void *__restrict__ ypad,
                                                                 float *__restrict__ x,
                                                                 const int *__restrict__ stop)
{
    if (stop && *stop) return;
    extern __shared__ float4 sviews[];   // 2 per view
    __shared__ float tile[ZC][B_TILE][B_TILE + 1];
    const int l = threadIdx.x, w = threadIdx.y;
    const int tid = w * B_TILE + l;
    const float4 *vt = reinterpret_cast<const float4 *>(g.viewB);
    for (int i = tid; i < 2 * g.n_views; i += B_TILE * B_TILE) sviews[i] = __ldg(vt + i);
    const int X0 = blockIdx.x * B_TILE, Y0 = blockIdx.y * B_TILE;
    const int iz0 = blockIdx.z * ZC;
    const float zfirst = (float(iz0) - g.cz) * g.vox;
    // column of the x-lane mapping and of the y-lane mapping (clamped into the grid;
    // columns past the edge compute throw-away values)
    const int ax = min(X0 + l, g.nx - 1), ay = min(Y0 + w, g.ny - 1);
    const int bx = min(X0 + w, g.nx - 1), by = min(Y0 + l, g.ny - 1);
    const float axc = (float(ax) - g.cx) * g.vox, ayc = (float(ay) - g.cy) * g.vox;
    const float bxc = (float(bx) - g.cx) * g.vox, byc = (float(by) - g.cy) * g.vox;
    const int view_stride = g.nvp * g.pitchU;
    const int pitch = g.pitchU;
    __syncthreads();
    float accA[ZC], accB[ZC];
#pragma unroll
    for (int k = 0; k < ZC; ++k) {
        accA[k] = 0.0f;
        accB[k] = 0.0f;
    }
    for (int s = 0; s < g.n_views; ++s) {
        const float4 p = sviews[2 * s], q = sviews[2 * s + 1];
        const bool xl = fabsf(p.w) <= fabsf(q.x);   // |tx| <= |ty|, uniform over the block
        const ColumnView c = column_view(g, p, q, xl ? axc : bxc, xl ? ayc : byc, zfirst);
        if (c.skip) continue;
        const size_t vbase = size_t(s) * view_stride + c.col;
        float r[ZC];
#pragma unroll
        for (int k = 0; k < ZC; ++k) {
            const float fv = fmaf(float(k), c.gv, c.fv0);
            const float v0f = floorf(fv);
            const float wv = fv - v0f;
            const float4 nb = load_quad<BF>(ypad, vbase + size_t((int(v0f) + g.padv) * pitch));
            const float r0 = fmaf(c.a0, nb.x, c.a1 * nb.y);
            const float r1 = fmaf(c.a0, nb.z, c.a1 * nb.w);
            r[k] = fmaf(wv, r1 - r0, r0);
        }
        if (xl) {
#pragma unroll
            for (int k = 0; k < ZC; ++k) accA[k] += r[k];
        } else {
#pragma unroll
            for (int k = 0; k < ZC; ++k) accB[k] += r[k];
        }
    }
    // x-lane sums belong to (x = X0 + l, y = Y0 + w), y-lane sums to (x = X0 + w, y = Y0 + l)
#pragma unroll
    for (int k = 0; k < ZC; ++k) tile[k][w][l] = accA[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ZC; ++k) tile[k][l][w] += accB[k];
    __syncthreads();
    const int ix = X0 + l, iy = Y0 + w;
    if (ix >= g.nx || iy >= g.ny) return;
#pragma unroll
    for (int k = 0; k < ZC; ++k) {
        const int iz = iz0 + k;
        if (iz < g.nz) x[(size_t(iz) * g.ny + iy) * g.nx + ix] = tile[k][w][l];
    }
}

template <int ZC, bool BF>
static cudaError_t launch_voxel_B_t(const GeomDev &g, const float *ypad, float *x, const int *stop, cudaStream_t st)
{
    dim3 block(B_TILE, B_TILE);
    const size_t smem = size_t(g.n_views) * 2 * sizeof(float4);
    if (smem > 8 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(voxel_B_kernel<ZC, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(smem));
        if (e != cudaSuccess) return e;
    }
    dim3 grid((g.nx + B_TILE - 1) / B_TILE, (g.ny + B_TILE - 1) / B_TILE, (g.nz + ZC - 1) / ZC);
    voxel_B_kernel<ZC, BF><<<grid, block, smem, st>>>(g, ypad, x, stop);
    return cudaGetLastError();
}

cudaError_t launch_voxel_B(const GeomDev &g, const float *ypad, float *x, const int *stop, cudaStream_t st)
{
    ProfScope prof(PK_VOXEL_B, st);
    if (g.nz == 1)
        return g.sino_bf16 ? launch_voxel_B_t<1, true>(g, ypad, x, stop, st)
                           : launch_voxel_B_t<1, false>(g, ypad, x, stop, st);
    return g.sino_bf16 ? launch_voxel_B_t<B_ZC, true>(g, ypad, x, stop, st)
                       : launch_voxel_B_t<B_ZC, false>(g, ypad, x, stop, st);
}

// ---------------------------------------------------------------------------
// y += B_un^T x: voxel splatting with the same weights (FP32 atomics into
// the plain sinogram, bounds-checked).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void splat(float *y, const GeomDev &g, int s, int iu, int iv, float val)
{
    if (iu < 0 || iu >= g.nu || iv < 0 || iv >= g.nv || val == 0.0f) return;
    atomicAdd(y + (size_t(s) * g.nv + iv) * g.nu + iu, val);
}

__global__ void __launch_bounds__(B_BX *B_BY) voxel_Bt_kernel(GeomDev g, const float *__restrict__ x,
                                                              float *__restrict__ y,
                                                              const int *__restrict__ stop)
{
    if (stop && *stop) return;
    const int ix = blockIdx.x * B_BX + threadIdx.x;
    const int iy = blockIdx.y * B_BY + threadIdx.y;
    const int iz = blockIdx.z;
    if (ix >= g.nx || iy >= g.ny) return;
    const float xv = x[(size_t(iz) * g.ny + iy) * g.nx + ix];
    if (xv == 0.0f) return;
    const float xc = (float(ix) - g.cx) * g.vox;
    const float yc = (float(iy) - g.cy) * g.vox;
    const float zc = (float(iz) - g.cz) * g.vox;
    for (int s = 0; s < g.n_views; ++s) {
        const ColumnView c = column_view(g, s, xc, yc, zc);
        if (c.skip) continue;
        const float fv = c.fv0;
        const float v0f = floorf(fv);
        const float wv = fv - v0f;
        if (v0f < -1.0f || v0f > float(g.nv - 1)) continue;
        const int v0 = int(v0f);
        const int u0 = c.col - PAD_U;
        splat(y, g, s, u0, v0, xv * c.a0 * (1.0f - wv));
        splat(y, g, s, u0 + 1, v0, xv * c.a1 * (1.0f - wv));
        splat(y, g, s, u0, v0 + 1, xv * c.a0 * wv);
        splat(y, g, s, u0 + 1, v0 + 1, xv * c.a1 * wv);
    }
}

cudaError_t launch_voxel_Bt(const GeomDev &g, const float *x, float *y, const int *stop, cudaStream_t st)
{
    dim3 block(B_BX, B_BY);
    dim3 grid((g.nx + B_BX - 1) / B_BX, (g.ny + B_BY - 1) / B_BY, g.nz);
    ProfScope prof(PK_VOXEL_BT, st);
    voxel_Bt_kernel<<<grid, block, 0, st>>>(g, x, y, stop);
    return cudaGetLastError();
}

}  // namespace ct

using namespace ct;

extern "C" ct_status ct_ramp_F(const ct_geom *geom, const float *y_dev, float *yf_dev, int transpose,
                               void *stream)
{
    if (!geom || !y_dev || !yf_dev) return set_error(CT_EINVAL, "ct_ramp_F: NULL argument");
    if (y_dev == yf_dev) return set_error(CT_EINVAL, "ct_ramp_F: input and output must differ");
    cudaError_t e = launch_ramp(geom->g, y_dev, yf_dev, plain_layout(geom->g), transpose != 0, nullptr,
                                static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_error(e, "ct_ramp_F launch");
    return CT_OK;
}

extern "C" ct_status ct_backproject_B(const ct_geom *geom, const float *y_dev, float *x_dev, int b_kind,
                                      void *stream)
{
    if (!geom || !y_dev || !x_dev) return set_error(CT_EINVAL, "ct_backproject_B: NULL argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (b_kind == CT_B_AT) return ct_adjoint_At(geom, y_dev, x_dev, stream);
    if (b_kind != CT_B_UN && b_kind != CT_B_FBP)
        return set_error(CT_EINVAL, "ct_backproject_B: unknown b_kind %d", b_kind);
    const GeomDev &g = geom->g;
    Arena ar;
    ct_status rc = arena_open(ar, padded_sino_bytes(g), nullptr, 0, st);
    if (rc != CT_OK) return rc;
    float *ypad = ar.take<float>(padded_sino_floats(g));
    cudaError_t e;
    if (b_kind == CT_B_FBP) {
        e = cudaMemsetAsync(ypad, 0, padded_sino_floats(g) * sizeof(float), st);
        if (e == cudaSuccess) e = launch_ramp(g, y_dev, ypad, padded_layout(g), false, nullptr, st);
    } else {
        e = launch_pad_sino(g, const_cast<float *>(y_dev), nullptr, false, ypad, nullptr, st);
    }
    if (e == cudaSuccess) e = launch_voxel_B(g, ypad, x_dev, nullptr, st);
    arena_close(ar);
    if (e != cudaSuccess) return cuda_error(e, "ct_backproject_B launch");
    return CT_OK;
}

extern "C" ct_status ct_adjoint_Bt(const ct_geom *geom, const float *x_dev, float *y_dev, int b_kind,
                                   void *stream)
{
    if (!geom || !x_dev || !y_dev) return set_error(CT_EINVAL, "ct_adjoint_Bt: NULL argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (b_kind == CT_B_AT) return ct_project_A(geom, x_dev, y_dev, stream);
    if (b_kind != CT_B_UN && b_kind != CT_B_FBP)
        return set_error(CT_EINVAL, "ct_adjoint_Bt: unknown b_kind %d", b_kind);
    const GeomDev &g = geom->g;
    if (b_kind == CT_B_UN) {
        CT_CUDA(cudaMemsetAsync(y_dev, 0, geom->m * sizeof(float), st));
        cudaError_t e = launch_voxel_Bt(g, x_dev, y_dev, nullptr, st);
        if (e != cudaSuccess) return cuda_error(e, "ct_adjoint_Bt launch");
        return CT_OK;
    }
    Arena ar;
    ct_status rc = arena_open(ar, Arena::align(geom->m * sizeof(float)), nullptr, 0, st);
    if (rc != CT_OK) return rc;
    float *tmp = ar.take<float>(geom->m);
    cudaError_t e = cudaMemsetAsync(tmp, 0, geom->m * sizeof(float), st);
    if (e == cudaSuccess) e = launch_voxel_Bt(g, x_dev, tmp, nullptr, st);
    if (e == cudaSuccess) e = launch_ramp(g, tmp, y_dev, plain_layout(g), true, nullptr, st);
    arena_close(ar);
    if (e != cudaSuccess) return cuda_error(e, "ct_adjoint_Bt launch");
    return CT_OK;
}
