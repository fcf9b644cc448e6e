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
// copy with zero borders (PAD_U pixels along u, padv rows along v): a view
// whose u footprint misses the detector is skipped, and the host sizes the
// row margin padv for the largest magnification over every slice computed,
// so the row index needs no clamp (the checked build tests this per sample).
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
        else   // row-difference form
            static_cast<float4 *>(dst)[i] = make_float4(q.x, q.y - q.x, q.z, q.w - q.z);
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

__device__ __forceinline__ float cosine_weight(const GeomDev &g, int iu, int iv)
{
    if (g.kind != CT_CONE_3D) return 1.0f;
    const float u = (float(iu) - g.cu) * g.du;
    const float v = (float(iv) - g.cv) * g.dv;
    return g.sdd / sqrtf(fmaf(g.sdd, g.sdd, fmaf(u, u, v * v)));
}

// ---------------------------------------------------------------------------
// Ramp filter by FFT.  Two detector rows are filtered at once as the real
// and imaginary parts of one complex row z = x1 + i x2, zero-padded to
// N = fft_n: the kernel's spectrum H is real, so the inverse transform of
// H FFT(z) is (h * x1) + i (h * x2), the two linear convolutions (N is at
// least 2 nu - 1, so the circular wrap misses the first nu outputs).  The
// inverse is taken as a forward transform of the conjugate,
// IFFT(Y) = conj(FFT(conj(Y))) / N, with 1/N folded into H.
//
// The transform is a Stockham autosort FFT in shared memory, radix 4 (a
// radix-2 stage last when N is not a power of 4), output in natural order.
// A stage of radix R after Ns points have been combined: butterfly j reads
// element j + r N/R (r < R), multiplies it by exp(-2 pi i r (j mod Ns) /
// (R Ns)), transforms the R values and writes value r to
// (j - j mod Ns) R + j mod Ns + r Ns.
//
// A group of N/4 threads owns one row pair; a block runs 256/(N/4) groups
// (one group of N/4 threads when N > 1024) and loops over row pairs.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Twiddles in shared memory, stage by stage: the radix-4 stage that follows
// Ns combined points uses exp(-2 pi i r k / (4 Ns)), r = 1..3, k < Ns, stored
// at stw[(Ns - 1) + (r - 1) Ns + k] (stages Ns = 1, 4, 16, ... take 3 Ns
// entries each, starting at Ns - 1 = 4^s - 1); the radix-2 stage's
// exp(-2 pi i k / N), k < N/2, follow.  Lanes with consecutive k read
// consecutive entries (in the full-length table they are N/(4 Ns) entries
// apart, all in one bank).
__device__ __forceinline__ int fft_stage_table(int N)
{
    int Ns = 1;
    while (Ns * 4 <= N) Ns *= 4;
    return Ns - 1;   // radix-4 entries: the sum over the stages of 3 Ns
}

// Buffer element i lives at slot fsw(i): within each aligned block of 16
// elements the low four bits are XORed with 5 ((i >> 4) mod 4).  The
// radix-4 stages after 1 and 4 combined points write elements 4t + r and
// 16 (t div 4) + (t mod 4) + 4r; unswizzled, 16 lanes of a shared-memory
// phase then hit only 4 of the 16 eight-byte banks.  The swizzle spreads
// both patterns over all 16 and keeps runs of consecutive elements (every
// other access) on distinct banks.
__device__ __forceinline__ int fsw(int i) { return i ^ (5 * ((i >> 4) & 3)); }

// One FFT of length N (= 4 T) by the T threads of a group; a holds the input
// and receives the output, b is scratch.  Every thread of the block calls it
// (it synchronises the block).
__device__ __forceinline__ void fft_group(float2 *&a, float2 *&b, const float2 *__restrict__ stw, int N, int t)
{
    const int T = N >> 2;
    int Ns = 1;
    for (; Ns * 4 <= N; Ns *= 4) {
        const int k = t & (Ns - 1);
        float2 v0 = a[fsw(t)], v1 = a[fsw(t + T)], v2 = a[fsw(t + 2 * T)], v3 = a[fsw(t + 3 * T)];
        if (Ns > 1) {
            const float2 *w = stw + (Ns - 1) + k;
            v1 = cmul(v1, w[0]);
            v2 = cmul(v2, w[Ns]);
            v3 = cmul(v3, w[2 * Ns]);
        }
        const float2 s02 = make_float2(v0.x + v2.x, v0.y + v2.y), d02 = make_float2(v0.x - v2.x, v0.y - v2.y);
        const float2 s13 = make_float2(v1.x + v3.x, v1.y + v3.y), d13 = make_float2(v1.x - v3.x, v1.y - v3.y);
        const int d = ((t - k) << 2) + k;
        b[fsw(d)] = make_float2(s02.x + s13.x, s02.y + s13.y);
        b[fsw(d + Ns)] = make_float2(d02.x + d13.y, d02.y - d13.x);       // d02 - i d13
        b[fsw(d + 2 * Ns)] = make_float2(s02.x - s13.x, s02.y - s13.y);
        b[fsw(d + 3 * Ns)] = make_float2(d02.x - d13.y, d02.y + d13.x);   // d02 + i d13
        __syncthreads();
        float2 *tmp = a;
        a = b;
        b = tmp;
    }
    if (Ns < N) {   // N = 2 Ns: one radix-2 stage, two butterflies per thread
        const float2 *w2 = stw + (Ns - 1);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = t + h * T;
            const int k = j & (Ns - 1);
            const float2 v0 = a[fsw(j)], v1 = cmul(a[fsw(j + N / 2)], w2[k]);
            const int d = ((j - k) << 1) + k;
            b[fsw(d)] = make_float2(v0.x + v1.x, v0.y + v1.y);
            b[fsw(d + Ns)] = make_float2(v0.x - v1.x, v0.y - v1.y);
        }
        __syncthreads();
        float2 *tmp = a;
        a = b;
        b = tmp;
    }
}

struct FftShape {
    int T;        // threads per group (N / 4)
    int groups;   // row pairs per block at a time
    int threads;
    size_t smem;
};

static FftShape fft_shape(int N)
{
    FftShape f;
    f.T = N / 4;
    f.groups = f.T >= 256 ? 1 : 256 / f.T;
    f.threads = f.T * f.groups;
    // staged twiddles (< 3N/2), spectrum (N floats), two buffers per group
    f.smem = sizeof(float2) * size_t(3 * N / 2) + sizeof(float) * size_t(N) + sizeof(float2) * 2 * size_t(N) * f.groups;
    return f;
}

__global__ void ramp_fft_kernel(GeomDev g, const float *__restrict__ src, float *__restrict__ dst, SinoLayout lay,
                                int transpose, const int *__restrict__ stop)
{
    if (stop && *stop) return;
    extern __shared__ float2 fsm[];
    const int N = g.fft_n, T = N >> 2;
    const int groups = blockDim.x / T;
    float2 *stw = fsm;                                              // staged twiddles, < 3N/2
    float *H = reinterpret_cast<float *>(fsm + 3 * N / 2);         // N spectrum values / N
    const int grp = threadIdx.x / T, t = threadIdx.x - grp * T;
    float2 *a = fsm + 2 * N + size_t(grp) * 2 * N;                 // this group's two buffers
    float2 *b = a + N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) H[i] = g.fft_h[i];
    for (int Ns = 1; Ns * 4 <= N; Ns *= 4)   // radix-4 entries (Ns - 1) + (r - 1) Ns + k = tw[r k N / (4 Ns)]
        for (int i = threadIdx.x; i < 3 * Ns; i += blockDim.x) {
            const int r = i / Ns + 1, k = i - (r - 1) * Ns;
            stw[(Ns - 1) + i] = g.fft_tw[r * k * (N / (4 * Ns))];
        }
    {
        const int r4 = fft_stage_table(N);
        if (r4 + 1 < N)   // a radix-2 stage (Ns = N / 2) follows: tw[k], k < N / 2
            for (int i = threadIdx.x; i < N / 2; i += blockDim.x) stw[r4 + i] = g.fft_tw[i];
    }
    const int nu = g.nu;
    const int nrows = g.n_views * g.nv;
    const int npairs = (nrows + 1) / 2;
    for (int base = blockIdx.x * groups; base < npairs; base += gridDim.x * groups) {
        const int pr = base + grp;
        const bool live = pr < npairs;
        const int r0 = 2 * pr, r1 = 2 * pr + 1;
        const bool has1 = live && r1 < nrows;
        const int s0 = r0 / g.nv, iv0 = r0 - s0 * g.nv;
        const int s1 = r1 / g.nv, iv1 = r1 - s1 * g.nv;
        __syncthreads();   // the previous pair's output reads are done (and the tables are in)
        for (int u = t; u < N; u += T) {
            float2 z = make_float2(0.0f, 0.0f);
            if (live && u < nu) {
                z.x = src[size_t(r0) * nu + u];
                if (has1) z.y = src[size_t(r1) * nu + u];
                if (!transpose) {
                    z.x *= cosine_weight(g, u, iv0);
                    z.y *= cosine_weight(g, u, iv1);
                }
            }
            a[fsw(u)] = z;
        }
        __syncthreads();
        fft_group(a, b, stw, N, t);
        for (int k = t; k < N; k += T) {   // conj(Z) H / N
            const float2 z = a[fsw(k)];
            a[fsw(k)] = make_float2(z.x * H[k], -z.y * H[k]);
        }
        __syncthreads();
        fft_group(a, b, stw, N, t);
        // conj of the transform: row 0 in .x, row 1 in -.y
        if (live && lay.quads) {
            // horizontal pairs (u, u+1) for u = -1 .. nu-1, two 8-byte stores each
            for (int u = t - 1; u < nu; u += T) {
                float l0 = 0.0f, h0 = 0.0f, l1 = 0.0f, h1 = 0.0f;
                if (u >= 0) {
                    const float2 y = a[fsw(u)];
                    l0 = transpose ? y.x * cosine_weight(g, u, iv0) : y.x;
                    l1 = transpose ? -y.y * cosine_weight(g, u, iv1) : -y.y;
                }
                if (u + 1 < nu) {
                    const float2 y = a[fsw(u + 1)];
                    h0 = transpose ? y.x * cosine_weight(g, u + 1, iv0) : y.x;
                    h1 = transpose ? -y.y * cosine_weight(g, u + 1, iv1) : -y.y;
                }
                store_sino_pair(dst, lay, s0, iv0, u, l0, h0);
                if (has1) store_sino_pair(dst, lay, s1, iv1, u, l1, h1);
            }
        } else if (live) {
            for (int u = t; u < nu; u += T) {
                const float2 y = a[fsw(u)];
                store_sino(dst, lay, s0, iv0, u, transpose ? y.x * cosine_weight(g, u, iv0) : y.x);
                if (has1) store_sino(dst, lay, s1, iv1, u, transpose ? -y.y * cosine_weight(g, u, iv1) : -y.y);
            }
        }
    }
}

static cudaError_t launch_ramp_fft(const GeomDev &g, const float *src, float *dst, SinoLayout lay, bool transpose,
                                   const int *stop, cudaStream_t st)
{
    const FftShape fs = fft_shape(g.fft_n);
    if (fs.smem > 48 * 1024) {
        cudaError_t e = raise_dyn_smem(reinterpret_cast<const void *>(ramp_fft_kernel), fs.smem);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ramp_fft_kernel, fs.threads, fs.smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int npairs = (g.n_views * g.nv + 1) / 2;
    const int want = (npairs + fs.groups - 1) / fs.groups;
    const unsigned blocks = unsigned(std::max(1, std::min(want, num_sms() * per_sm)));
    ProfScope prof(PK_RAMP, st);
    ramp_fft_kernel<<<blocks, fs.threads, fs.smem, st>>>(g, src, dst, lay, transpose ? 1 : 0, stop);
    return cudaGetLastError();
}

cudaError_t launch_ramp(const GeomDev &g, const float *src, float *dst, SinoLayout lay, bool transpose,
                        const int *stop, cudaStream_t st)
{
    return launch_ramp_fft(g, src, dst, lay, transpose, stop, st);
}

// ---------------------------------------------------------------------------
// x = B_un y.
// ---------------------------------------------------------------------------
constexpr int B_BX = 32, B_BY = 4;

struct ColumnView {
    int skip;       // the u footprint misses the detector
    int col;        // padded column of the left neighbour
    float a0, a1;   // weight * (1 - wu), weight * wu
    float w, wu;    // weight, u fraction
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
    c.w = w;
    c.wu = wu;
    c.gv = M * g.vox * g.inv_dv;
    c.fv0 = fmaf(M * zfirst, g.inv_dv, g.cv);
    return c;
}

__device__ __forceinline__ ColumnView column_view(const GeomDev &g, int s, float x, float y, float zfirst)
{
    const float4 *vp = reinterpret_cast<const float4 *>(g.viewB + s);
    return column_view(g, __ldg(vp), __ldg(vp + 1), x, y, zfirst);
}

// Lane patches.  A warp covers a patch of PA x (32/PA) columns, PA lanes
// along the axis closer to the view's central ray (chosen per view: along x
// when |tx| <= |ty|, i.e. when u moves more slowly with x than with y).
// Along the central ray the projection barely moves (only the magnification
// changes, by vox/depth per voxel); across it, u moves by M vox/du pixels per
// lane.  The load path serves a 128-bit warp load 8 lanes at a time, and its
// passes per load (ncu: data-pipe wavefronts per request) grow when those
// lanes' quads spread over several 128-byte lines: of the patches measured on
// the cone-beam scans, 4 lanes along by 2 across per group of 8 (PA = 4)
// takes fewest (at 256^3: 5.3 passes per warp load against 6.4 with all 32
// lanes along the ray).  The 3D kernel (voxel_B_slab_kernel) uses that patch.
// voxel_B_kernel serves 2D scans: a block owns a 32 x 32 tile of columns
// (ZC = 1, PA = 32: the detector is one row), and the two partial sums
// (x-lane views and y-lane views) meet in shared memory.  The sinogram is
// read as quads (the 2 x 2 bilinear neighbourhood), one 16-byte load (8 for
// bf16) per voxel and view; the view table sits in shared memory.
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

// The ZC samples of one column in one view: r[k] = B's term for z = z0 + k.
// DIFF: FP32 entries in the row-difference form, a sample is
// w (e0 + wv (e1 - e0)) with e0 = S[v][u] + wu (S[v][u+1] - S[v][u]) and e1
// likewise on row v+1 (five operations with the accumulation, against seven
// from the four values); r[k] then omits the weight w, which the caller
// folds into the accumulation.
template <int ZC, bool BF, bool DIFF>
__device__ __forceinline__ void column_samples(const GeomDev &g, const void *__restrict__ ypad, const ColumnView &c,
                                               int s, int view_stride, int pitch, float (&r)[ZC])
{
    int col = c.col;
    if (!CT_IN_BOUNDS(g, unsigned(col) < unsigned(pitch), BS_B_COL, s, col)) col = 0;
    const size_t vbase = size_t(s) * view_stride + col;
#pragma unroll
    for (int k = 0; k < ZC; ++k) {
        const float fv = fmaf(float(k), c.gv, c.fv0);
        const float v0f = floorf(fv);
        const float wv = fv - v0f;
        int row = int(v0f) + g.padv;
        if (!CT_IN_BOUNDS(g, unsigned(row) < unsigned(g.nvp), BS_B_ROW, s, row)) row = 0;
        const float4 nb = load_quad<BF>(ypad, vbase + size_t(row * pitch));
        if (DIFF) {
            const float e0 = fmaf(c.wu, nb.y, nb.x);
            const float e1 = fmaf(c.wu, nb.w, nb.z);
            r[k] = fmaf(wv, e1 - e0, e0);
        } else {
            const float r0 = fmaf(c.a0, nb.x, c.a1 * nb.y);
            const float r1 = fmaf(c.a0, nb.z, c.a1 * nb.w);
            r[k] = fmaf(wv, r1 - r0, r0);
        }
    }
}

template <int ZC, bool DIFF>
__device__ __forceinline__ void accumulate(float (&acc)[ZC], const float (&r)[ZC], float w)
{
#pragma unroll
    for (int k = 0; k < ZC; ++k) acc[k] = DIFF ? fmaf(w, r[k], acc[k]) : acc[k] + r[k];
}

template <int ZC, bool BF, bool DIFF, int PA = 32>
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
    // a warp covers a PA x (32/PA) patch of columns, PA lanes along the axis
    // nearer the central ray
    constexpr int PB = 32 / PA;
    const int along = (w % (32 / PA)) * PA + l % PA, across = (w / (32 / PA)) * PB + l / PA;
    const int tax = along, tay = across, tbx = across, tby = along;   // tile offsets of the two mappings
    // column of the x-lane mapping and of the y-lane mapping (clamped into the grid;
    // columns past the edge compute throw-away values)
    const int ax = min(X0 + tax, g.nx - 1), ay = min(Y0 + tay, g.ny - 1);
    const int bx = min(X0 + tbx, g.nx - 1), by = min(Y0 + tby, g.ny - 1);
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
        float r[ZC];
        column_samples<ZC, BF, DIFF>(g, ypad, c, s, view_stride, pitch, r);
        if (xl)
            accumulate<ZC, DIFF>(accA, r, c.w);
        else
            accumulate<ZC, DIFF>(accB, r, c.w);
    }
    // x-lane sums belong to (X0 + tax, Y0 + tay), y-lane sums to (X0 + tbx, Y0 + tby)
#pragma unroll
    for (int k = 0; k < ZC; ++k) tile[k][tay][tax] = accA[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ZC; ++k) tile[k][tby][tbx] += accB[k];
    __syncthreads();
    const int ix = X0 + l, iy = Y0 + w;
    if (ix >= g.nx || iy >= g.ny) return;
#pragma unroll
    for (int k = 0; k < ZC; ++k) {
        const int iz = iz0 + k;
        if (iz < g.nz) x[(size_t(iz) * g.ny + iy) * g.nx + ix] = tile[k][w][l];
    }
}

// The ZC samples of one column in one view from a per-view pointer: pv is
// the byte address of the column's entry in the view's first unpadded row
// (the row margin folded in), so a sample's address is one multiply-add of
// its row index and the row pitch in bytes (the entries' forms as in
// column_samples).
template <int ZC, bool BF, bool DIFF>
__device__ __forceinline__ void column_samples_at(const GeomDev &g, int s, const char *__restrict__ pv,
                                                  const ColumnView &c, int pitch_bytes, float (&r)[ZC])
{
#pragma unroll
    for (int k = 0; k < ZC; ++k) {
        const float fv = fmaf(float(k), c.gv, c.fv0);
        const float v0f = floorf(fv);
        const float wv = fv - v0f;
        int row = int(v0f);   // relative to the view's first detector row
        if (!CT_IN_BOUNDS(g, unsigned(row + g.padv) < unsigned(g.nvp), BS_B_ROW, s, row + g.padv)) row = -g.padv;
        const float4 nb = load_quad<BF>(pv + row * pitch_bytes, 0);
        if (DIFF) {
            const float e0 = fmaf(c.wu, nb.y, nb.x);
            const float e1 = fmaf(c.wu, nb.w, nb.z);
            r[k] = fmaf(wv, e1 - e0, e0);
        } else {
            const float r0 = fmaf(c.a0, nb.x, c.a1 * nb.y);
            const float r1 = fmaf(c.a0, nb.z, c.a1 * nb.w);
            r[k] = fmaf(wv, r1 - r0, r0);
        }
    }
}

// The back-projector for 3D scans (FP32 or bf16 entries).  A block of 32 x TY
// threads owns a 32 x TY tile of (x, y) columns and ZC consecutive z (ZC =
// 16: the column's projection is computed once per view for 16 samples);
// MINB blocks are resident per SM.  The view loop runs twice, once over the
// views whose lanes run along x and once over those along y, into one set of
// ZC accumulators; the tile in shared memory merges the two lane mappings.
// Warp 0 lists the views of each orientation (ballots over the view table)
// so that each pass visits only its own views.  A warp covers a 4 x 8 patch
// of columns, 4 lanes along the axis nearer the central ray (see above).
// Small blocks (256 threads, 4 per SM) keep 32 warps resident like one
// 1024-thread block, but the blocks' starts and ends (view table, tile
// merge, stores) overlap other blocks' view loops instead of idling the SM.
// At 256^3: 4.16 ms; 4.35 ms when each pass tested every view's orientation
// and addressed samples from the view index; 5.09 ms for voxel_B_kernel with
// 8-slice runs.  On bf16 entries 4.18 ms (a 1024-thread two-pass kernel took
// 4.93 ms).
template <int ZC, int TY, int MINB, bool BF, bool DIFF>
__global__ void __launch_bounds__(32 * TY, MINB) voxel_B_slab_kernel(GeomDev g, const void *__restrict__ ypad,
                                                                     float *__restrict__ x,
                                                                     const int *__restrict__ stop)
{
    static_assert(TY % 8 == 0, "a warp's 4 x 8 patch must tile the 32 x TY block both ways");
    if (stop && *stop) return;
    // 2 float4 per view, then the tile, then the views listed by orientation
    extern __shared__ float4 sviews[];
    float(*tile)[TY][B_TILE + 1] = reinterpret_cast<float(*)[TY][B_TILE + 1]>(sviews + 2 * g.n_views);
    short *order = reinterpret_cast<short *>(&tile[ZC][0][0]);
    __shared__ int n_along_x;
    const int l = threadIdx.x, w = threadIdx.y;
    const int tid = w * 32 + l;
    const float4 *vt = reinterpret_cast<const float4 *>(g.viewB);
    for (int i = tid; i < 2 * g.n_views; i += 32 * TY) sviews[i] = __ldg(vt + i);
    const int X0 = blockIdx.x * 32, Y0 = blockIdx.y * TY;
    const int iz0 = blockIdx.z * ZC;
    const float zfirst = (float(iz0) - g.cz) * g.vox;
    const int tax = (w % 8) * 4 + l % 4, tay = (w / 8) * 8 + l / 4;           // lanes along x
    const int tby = (w % (TY / 4)) * 4 + l % 4, tbx = (w / (TY / 4)) * 8 + l / 4;   // lanes along y
    const int ax = min(X0 + tax, g.nx - 1), ay = min(Y0 + tay, g.ny - 1);
    const int bx = min(X0 + tbx, g.nx - 1), by = min(Y0 + tby, g.ny - 1);
    const float axc = (float(ax) - g.cx) * g.vox, ayc = (float(ay) - g.cy) * g.vox;
    const float bxc = (float(bx) - g.cx) * g.vox, byc = (float(by) - g.cy) * g.vox;
    const int view_stride = g.nvp * g.pitchU;
    const int pitch = g.pitchU;
    __syncthreads();
    if (w == 0) {   // order[0, n_along_x): views with lanes along x; then the others
        int count = 0;
        for (int s0 = 0; s0 < g.n_views; s0 += 32) {
            const int s = s0 + l;
            const bool xl = s < g.n_views && fabsf(sviews[2 * s].w) <= fabsf(sviews[2 * s + 1].x);
            count += __popc(__ballot_sync(0xffffffffu, xl));
        }
        int a = 0, b = count;
        const unsigned below = (1u << l) - 1u;
        for (int s0 = 0; s0 < g.n_views; s0 += 32) {
            const int s = s0 + l;
            const bool in = s < g.n_views;
            const bool xl = in && fabsf(sviews[2 * s].w) <= fabsf(sviews[2 * s + 1].x);
            const unsigned mx = __ballot_sync(0xffffffffu, xl), my = __ballot_sync(0xffffffffu, in && !xl);
            if (xl)
                order[a + __popc(mx & below)] = short(s);
            else if (in)
                order[b + __popc(my & below)] = short(s);
            a += __popc(mx);
            b += __popc(my);
        }
        if (l == 0) n_along_x = count;
    }
    __syncthreads();
    float acc[ZC];
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
        for (int k = 0; k < ZC; ++k) acc[k] = 0.0f;
        const int i0 = pass == 0 ? 0 : n_along_x, i1 = pass == 0 ? n_along_x : g.n_views;
        const float cx = pass == 0 ? axc : bxc, cy = pass == 0 ? ayc : byc;
        for (int i = i0; i < i1; ++i) {
            const int s = order[i];
            const ColumnView c = column_view(g, sviews[2 * s], sviews[2 * s + 1], cx, cy, zfirst);
            if (c.skip) continue;
            constexpr int ENTRY = BF ? 8 : 16;   // bytes per quad entry
            int col = c.col;
            if (!CT_IN_BOUNDS(g, unsigned(col) < unsigned(pitch), BS_B_COL, s, col)) col = 0;
            const char *pv = static_cast<const char *>(ypad) +
                             ENTRY * (size_t(s) * view_stride + size_t(g.padv) * pitch + col);
            float r[ZC];
            column_samples_at<ZC, BF, DIFF>(g, s, pv, c, ENTRY * pitch, r);
            accumulate<ZC, DIFF>(acc, r, c.w);
        }
        // x-lane sums belong to (X0 + tax, Y0 + tay), y-lane sums to (X0 + tbx, Y0 + tby)
        if (pass == 0) {
#pragma unroll
            for (int k = 0; k < ZC; ++k) tile[k][tay][tax] = acc[k];
        } else {
#pragma unroll
            for (int k = 0; k < ZC; ++k) tile[k][tby][tbx] += acc[k];
        }
        __syncthreads();
    }
    const int ix = X0 + l, iy = Y0 + w;
    if (ix >= g.nx || iy >= g.ny) return;
#pragma unroll
    for (int k = 0; k < ZC; ++k) {
        const int iz = iz0 + k;
        if (iz < g.nz) x[(size_t(iz) * g.ny + iy) * g.nx + ix] = tile[k][w][l];
    }
}

template <int ZC, int TY, int MINB, bool BF, bool DIFF>
static cudaError_t launch_voxel_B_slab(const GeomDev &g, const float *ypad, float *x, const int *stop,
                                       cudaStream_t st)
{
    dim3 block(32, TY);
    const size_t smem = size_t(g.n_views) * 2 * sizeof(float4) + size_t(ZC) * TY * (B_TILE + 1) * sizeof(float) +
                        size_t(g.n_views) * sizeof(short);
    cudaError_t e = raise_dyn_smem(reinterpret_cast<const void *>(voxel_B_slab_kernel<ZC, TY, MINB, BF, DIFF>), smem);
    if (e != cudaSuccess) return e;
    dim3 grid((g.nx + 31) / 32, (g.ny + TY - 1) / TY, (g.nz + ZC - 1) / ZC);
    voxel_B_slab_kernel<ZC, TY, MINB, BF, DIFF><<<grid, block, smem, st>>>(g, ypad, x, stop);
    return cudaGetLastError();
}

template <int ZC, bool BF, bool DIFF, int PA = 32>
static cudaError_t launch_voxel_B_t(const GeomDev &g, const float *ypad, float *x, const int *stop, cudaStream_t st)
{
    dim3 block(B_TILE, B_TILE);
    const size_t smem = size_t(g.n_views) * 2 * sizeof(float4);
    if (smem > 8 * 1024) {
        cudaError_t e = raise_dyn_smem(reinterpret_cast<const void *>(voxel_B_kernel<ZC, BF, DIFF, PA>), smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((g.nx + B_TILE - 1) / B_TILE, (g.ny + B_TILE - 1) / B_TILE, (g.nz + ZC - 1) / ZC);
    voxel_B_kernel<ZC, BF, DIFF, PA><<<grid, block, smem, st>>>(g, ypad, x, stop);
    return cudaGetLastError();
}

template <int ZC, int PA>
static cudaError_t launch_voxel_B_z(const GeomDev &g, const float *ypad, float *x, const int *stop, cudaStream_t st,
                                    QuadForm form)
{
    if (g.sino_bf16) return launch_voxel_B_t<ZC, true, false, PA>(g, ypad, x, stop, st);
    return form == QUAD_ROWDIFF ? launch_voxel_B_t<ZC, false, true, PA>(g, ypad, x, stop, st)
                                : launch_voxel_B_t<ZC, false, false, PA>(g, ypad, x, stop, st);
}

cudaError_t launch_voxel_B(const GeomDev &g, const float *ypad, float *x, const int *stop, cudaStream_t st,
                           QuadForm form)
{
    ProfScope prof(PK_VOXEL_B, st);
    if (g.nz == 1) return launch_voxel_B_z<1, 32>(g, ypad, x, stop, st, form);
    if (g.sino_bf16) return launch_voxel_B_slab<B_ZC_SLAB, 8, 4, true, false>(g, ypad, x, stop, st);
    return form == QUAD_ROWDIFF ? launch_voxel_B_slab<B_ZC_SLAB, 8, 4, false, true>(g, ypad, x, stop, st)
                                : launch_voxel_B_slab<B_ZC_SLAB, 8, 4, false, false>(g, ypad, x, stop, st);
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

// y += B_un^T x for 3D scans by splatting voxel runs.  Per view the lanes
// run across the central ray (along x when u moves faster with x than with
// y), so a warp's atomics land on different pixels along u.  A thread's ZC
// voxels (consecutive z of one column) share the column's u and u-weights,
// and their rows increase with z: contributions to one row are summed in
// registers and added with two atomics (pixels u0, u0 + 1) when the run
// moves past the row; the flushes are predicated and the running sums
// selected, so lanes whose runs change rows at different slices share one
// copy of the atomics.  One launch per lane orientation, in 256-thread
// blocks (MINB resident per SM): XL takes the views whose lanes run along x
// on 32 x 8 column tiles, !XL those along y on 8 x 32 tiles.  Against one
// launch of 1024-thread blocks with both orientations (two value sets per
// thread): 3.23 against 4.05 ms on phantom projections at 256^3, 16.5
// against 17.0 ms dense.
template <int ZC, bool XL, int MINB>
__global__ void __launch_bounds__(256, MINB) voxel_Bt_slab_kernel(GeomDev g, const float *__restrict__ x,
                                                                  float *__restrict__ y,
                                                                  const int *__restrict__ stop)
{
    if (stop && *stop) return;
    extern __shared__ float4 bt_views[];   // 2 per view
    const int l = threadIdx.x, w = threadIdx.y;
    const int tid = w * 32 + l;
    const float4 *vt = reinterpret_cast<const float4 *>(g.viewB);
    for (int i = tid; i < 2 * g.n_views; i += 256) bt_views[i] = __ldg(vt + i);
    const int ax = XL ? blockIdx.x * 32 + l : blockIdx.x * 8 + w;
    const int ay = XL ? blockIdx.y * 8 + w : blockIdx.y * 32 + l;
    const int Z0 = blockIdx.z * ZC;
    float xa[ZC];
    bool anya = false;
#pragma unroll
    for (int k = 0; k < ZC; ++k) {
        const int z = Z0 + k;
        xa[k] = (z < g.nz && ax < g.nx && ay < g.ny) ? x[(size_t(z) * g.ny + ay) * g.nx + ax] : 0.0f;
        anya = anya || xa[k] != 0.0f;
    }
    const float axc = (float(min(ax, g.nx - 1)) - g.cx) * g.vox, ayc = (float(min(ay, g.ny - 1)) - g.cy) * g.vox;
    const float zfirst = (float(Z0) - g.cz) * g.vox;
    __syncthreads();
    if (!anya) return;
    for (int s = 0; s < g.n_views; ++s) {
        const float4 p = bt_views[2 * s], q = bt_views[2 * s + 1];
        const bool xl = fabsf(p.w) > fabsf(q.x);
        if (xl != XL) continue;
        const ColumnView c = column_view(g, p, q, axc, ayc, zfirst);
        if (c.skip) continue;
        const int u0 = c.col - PAD_U;
        auto flush = [&](int v, float r) {
            if (r == 0.0f) return;
            splat(y, g, s, u0, v, r * c.a0);
            splat(y, g, s, u0 + 1, v, r * c.a1);
        };
        int vc = 0;
        float acc_lo = 0.0f, acc_hi = 0.0f;
#pragma unroll
        for (int k = 0; k < ZC; ++k) {
            const float val = xa[k];
            const float fv = fmaf(float(k), c.gv, c.fv0);
            const float v0f = floorf(fv);
            const float wv = fv - v0f;
            const int v0 = int(fmaxf(fminf(v0f, float(g.nv + 1)), -2.0f));
            const float c_lo = val * (1.0f - wv), c_hi = val * wv;
            if (k == 0) {
                vc = v0;
                acc_lo = c_lo;
                acc_hi = c_hi;
            } else {
                const bool same = v0 == vc, next = v0 == vc + 1;
                if (!same) flush(vc, acc_lo);
                if (!same && !next) flush(vc + 1, acc_hi);
                acc_lo = same ? acc_lo + c_lo : (next ? acc_hi + c_lo : c_lo);
                acc_hi = same ? acc_hi + c_hi : c_hi;
                vc = v0;
            }
        }
        flush(vc, acc_lo);
        flush(vc + 1, acc_hi);
    }
}

template <int ZC, int MINB>
static cudaError_t launch_voxel_Bt_slab(const GeomDev &g, const float *x, float *y, const int *stop, cudaStream_t st)
{
    const size_t smem = size_t(g.n_views) * 2 * sizeof(float4);
    cudaError_t e = raise_dyn_smem(reinterpret_cast<const void *>(voxel_Bt_slab_kernel<ZC, true, MINB>), smem);
    if (e == cudaSuccess)
        e = raise_dyn_smem(reinterpret_cast<const void *>(voxel_Bt_slab_kernel<ZC, false, MINB>), smem);
    if (e != cudaSuccess) return e;
    dim3 block(32, 8);
    dim3 gx((g.nx + 31) / 32, (g.ny + 7) / 8, (g.nz + ZC - 1) / ZC);
    dim3 gy((g.nx + 7) / 8, (g.ny + 31) / 32, (g.nz + ZC - 1) / ZC);
    voxel_Bt_slab_kernel<ZC, true, MINB><<<gx, block, smem, st>>>(g, x, y, stop);
    voxel_Bt_slab_kernel<ZC, false, MINB><<<gy, block, smem, st>>>(g, x, y, stop);
    return cudaGetLastError();
}

cudaError_t launch_voxel_Bt(const GeomDev &g, const float *x, float *y, const int *stop, cudaStream_t st)
{
    ProfScope prof(PK_VOXEL_BT, st);
    if (g.nz < B_ZC) {   // 2D, or a slab thinner than a z run: one voxel per thread
        dim3 block(B_BX, B_BY);
        dim3 grid((g.nx + B_BX - 1) / B_BX, (g.ny + B_BY - 1) / B_BY, g.nz);
        voxel_Bt_kernel<<<grid, block, 0, st>>>(g, x, y, stop);
        return cudaGetLastError();
    }
    return launch_voxel_Bt_slab<B_ZC, 4>(g, x, y, stop, st);
}

}  // namespace ct

using namespace ct;

extern "C" ct_status ct_ramp_F(const ct_geom *geom, const float *y_dev, float *yf_dev, int transpose,
                               void *stream)
{
    NvtxRange call_range("ct_ramp_F");
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
    NvtxRange call_range("ct_backproject_B");
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
    if (e == cudaSuccess) e = launch_voxel_B(g, ypad, x_dev, nullptr, st, QUAD_ROWDIFF);
    arena_close(ar);
    if (e != cudaSuccess) return cuda_error(e, "ct_backproject_B launch");
    return CT_OK;
}

extern "C" ct_status ct_adjoint_Bt(const ct_geom *geom, const float *x_dev, float *y_dev, int b_kind,
                                   void *stream)
{
    NvtxRange call_range("ct_adjoint_Bt");
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
