// Internal declarations shared by the translation units of libct.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <cstddef>
#include <cstdint>

#include "ct.h"

namespace ct {

// Zero borders of the working copies the operators gather from.  With these
// borders every bilinear neighbour of a sample that lies inside the clipped
// plane range (projector) or the clamped row range (back-projector) is in
// bounds, so the inner loops carry no bounds tests.
constexpr int PAD_A = 2;   // voxels, around the in-plane and z axes of the plane-major copies
constexpr int PAD_U = 1;   // pixels, both ends of each detector row
constexpr int PAD_V = 2;   // rows, above and below each view
// rays per projector thread along a detector column (the last group of a
// column runs past nv when nv is not a multiple; those rays are discarded):
// A_VR for A, AT_VR for its exact transpose (tuning; at 256^3, 16 rays took
// A 5.31 / 5.74 ms with FP32 / bf16 copies and A^T 5.74 ms, against 5.39 /
// 6.16 ms and 6.06 ms with 8 rays, and A 8.16 / 9.01 ms with 12)
#ifndef CT_A_VR
#define CT_A_VR 16
#endif
#ifndef CT_AT_VR
#define CT_AT_VR 16
#endif
constexpr int A_VR = CT_A_VR;
constexpr int AT_VR = CT_AT_VR;
constexpr int A_VR_MAX = A_VR > AT_VR ? A_VR : AT_VR;
// consecutive z slices per thread: B_ZC_SLAB for the 3D back-projector
// (voxel_B_slab_kernel), B_ZC for its transpose.  The last run of a column
// may pass nz: those slices are computed and discarded, and the padded
// sinogram's row margin covers them too (sized for B_ZC_RUN_MAX).
#ifndef CT_B_ZC
#define CT_B_ZC 8
#endif
constexpr int B_ZC = CT_B_ZC;
constexpr int B_ZC_SLAB = 16;
constexpr int B_ZC_RUN_MAX = B_ZC > B_ZC_SLAB ? B_ZC : B_ZC_SLAB;


// Per-view constants of the projector, from which a ray's direction, its
// cross product with the source position and the source position follow:
//   d = (dx0 + u dxu, dy0 + u dyu, v dzv), (S x d)_z = u crossu, S_xy = (sx, sy).
struct ViewA {
    float dx0, dxu, dy0, dyu, dzv, crossu, sx, sy;
};

// Per-view constants of the voxel-driven back-projector: for a voxel at
// (x, y, z) the depth is W = w0 + x wx + y wy, the in-plane detector
// coordinate numerator is t = x tx + y ty, the magnification M = mnum / W,
// u = M t, v = M z and the weight kB M^2.
struct ViewB {
    float w0, wx, wy, tx, ty, mnum, pad0, pad1;
};

// Geometry as the kernels see it (passed by value).
struct GeomDev {
    int kind;
    int nx, ny, nz, n_views, nu, nv;
    float vox, inv_vox, du, dv, inv_du, inv_dv;
    float cx, cy, cz, cu, cv;   // (N-1)/2 of each axis
    float kB;                   // back-projector weight constant
    float sdd;                  // cone: source-detector distance (cosine weight)
    const ViewA *viewA;
    const ViewB *viewB;
    const float *ramp_taps;     // nu scaled Ram-Lak taps h[0..nu-1]
    // projector working copies: plane-major, zero border PAD_A
    //   Xc[zp][x][yp] (planes along x, rows along y), Yc[zp][y][xp]
    int nzp;                    // nz + 2 PAD_A
    int pitchX;                 // ny + 2 PAD_A
    int pitchY;                 // nx + 2 PAD_A
    // padded sinogram for the back-projector, quad-interleaved: entry
    //   Q[view][vp][up] = (S[v][u], S[v][u+1], S[v+1][u], S[v+1][u+1]) as float4,
    //   v = vp - padv, u = up - PAD_U, vp in [0, nv + 2 padv), up in [0, nu + 2 PAD_U),
    //   S zero outside the detector: the four bilinear neighbours of a sample in one load.
    //   FP32 entries written a row pair at a time (the pad and ramp kernels) hold row
    //   differences instead, (S[v][u], S[v][u+1] - S[v][u], S[v+1][u], S[v+1][u+1] - S[v+1][u]),
    //   which interpolate in fewer operations (QuadForm); entries written value by value
    //   (a projector's store_sino) and bf16 entries hold the four values.
    // padv (>= PAD_V) rows of zeros cover every voxel's projection, so the
    // back-projector's row index needs no clamp.
    int nvp, pitchU, padv;
    // projector: every ray of a detector column moves at most one z-row per
    // detector row on every plane (0 <= dz/dv <= 0.98 rows), so a two-row
    // window suffices (set by ct_geom_create from the geometry's extremes)
    int a_window;
    // projector: every sample of every ray lies within the zero-bordered z
    // range, so the row index needs no clamp (set by ct_geom_create)
    int a_zsafe;
    // storage precision of the working copies (arithmetic is FP32 either way):
    //   vol_bf16:  projector plane copies hold (b, b+1) bf16 pairs in 4 bytes,
    //              and the BA-GMRES Krylov basis is bf16;
    //   sino_bf16: the back-projector's quad sinogram holds 4 bf16 (8 bytes).
    int vol_bf16, sino_bf16;
    // ramp filter by FFT: the linear convolution of a row with the ramp
    // kernel is the circular one of length fft_n >= 2 nu - 1 (a power of
    // two); the kernel is even, so its spectrum is real.
    //   fft_tw[t] = exp(-2 pi i t / fft_n), t < fft_n
    //   fft_h[k]  = spectrum of the scaled kernel / fft_n, k < fft_n
    int fft_n;
    const float2 *fft_tw;
    const float *fft_h;
    // projector: 0 Joseph, 1 line intersection (Siddon)
    int siddon;
#ifdef CT_CHECK_BOUNDS
    // checked builds: the first failed index check of any kernel on this
    // geometry, as a BoundsSite record (see bounds_ok); 0 when none failed
    unsigned long long *bounds_word;
#endif
};

// Index checks of checked builds (compiled with -DCT_CHECK_BOUNDS, which
// builds libct_checked.so).  The gathers of A and B and the transposes'
// row windows rely on margins and invariants that ct_geom_create derives
// from the geometry's extremes (the row margin padv, a_zsafe, a_window); a
// checked build tests each of them where it is used.  A failed check records
// (site, view or plane, index) in the geometry's bounds word (the first
// failure wins) and the access is redirected into range, so it never leaves
// its buffer; the results are then wrong and the host reads the record with
// ct_bounds_take.  In regular builds CT_IN_BOUNDS is the constant true and
// the kernels are unchanged.
enum BoundsSite {
    BS_NONE = 0,
    BS_A_Z = 1,          // projector: a sample's two z rows inside the zero border
    BS_A_WINDOW = 2,     // projector: consecutive rays of a column move up at most one z row
    BS_AT_WINDOW = 3,    // projector transpose: the same for its row sums
    BS_B_ROW = 4,        // back-projector: a sample's quad row inside the view's padded rows
    BS_B_COL = 5,        // back-projector: a column's quad inside the padded row
    BS_SIDDON_VOXEL = 6  // line-intersection projector: a traversed voxel inside the grid
};
#ifdef CT_CHECK_BOUNDS
__device__ __forceinline__ bool bounds_ok(const GeomDev &g, bool ok, int site, int where, int index)
{
    if (!ok) {
        const unsigned long long rec = (static_cast<unsigned long long>(site) << 56) |
                                       (static_cast<unsigned long long>(where & 0xffffff) << 32) |
                                       static_cast<unsigned int>(index);
        atomicCAS(g.bounds_word, 0ull, rec);
    }
    return ok;
}
#define CT_IN_BOUNDS(g, cond, site, where, index) ::ct::bounds_ok((g), (cond), (site), (where), (index))
#else
#define CT_IN_BOUNDS(g, cond, site, where, index) true
#endif

// Layout of a sinogram buffer that an operator writes.
struct SinoLayout {
    int rows_per_view;  // nv (plain) or nv + 2 PAD_V (padded)
    int pitch;          // entries per row: nu (plain) or nu + 2 PAD_U (padded)
    int row_off;        // 0 or PAD_V
    int col_off;        // 0 or PAD_U
    int quads;          // padded quad layout: value (v, u) goes to the four entries that hold it
    int bf16;           // quad entries hold bf16 instead of float
};

inline SinoLayout plain_layout(const GeomDev &g) { return SinoLayout{g.nv, g.nu, 0, 0, 0, 0}; }
inline SinoLayout padded_layout(const GeomDev &g)
{
    return SinoLayout{g.nvp, g.pitchU, g.padv, PAD_U, 1, g.sino_bf16};
}

// Stores one sinogram value in either layout.
__device__ __forceinline__ void store_sino(float *out, const SinoLayout &lay, int s, int iv, int iu, float val)
{
    const size_t e = (size_t(s) * lay.rows_per_view + iv + lay.row_off) * lay.pitch + iu + lay.col_off;
    if (lay.quads) {
        // (v, u) is .x of entry (v, u), .y of (v, u-1), .z of (v-1, u), .w of (v-1, u-1).
        // In the last column the entry's right neighbours (.y, .w) are S[.][nu] = 0:
        // they are written here too, because a buffer that last held the
        // row-difference form has -S[v][nu-1] there.  Every other slot off the
        // detector is zero in both forms.
        const size_t up = e - lay.pitch;
        const bool last_col = iu + 1 == lay.pitch - 2 * lay.col_off;
        if (lay.bf16) {
            __nv_bfloat16 *o = reinterpret_cast<__nv_bfloat16 *>(out);
            const __nv_bfloat16 h = __float2bfloat16_rn(val);
            o[4 * e] = h;
            o[4 * (e - 1) + 1] = h;
            o[4 * up + 2] = h;
            o[4 * (up - 1) + 3] = h;
            if (last_col) {
                o[4 * e + 1] = __float2bfloat16_rn(0.0f);
                o[4 * up + 3] = __float2bfloat16_rn(0.0f);
            }
        } else {
            out[4 * e] = val;
            out[4 * (e - 1) + 1] = val;
            out[4 * up + 2] = val;
            out[4 * (up - 1) + 3] = val;
            if (last_col) {
                out[4 * e + 1] = 0.0f;
                out[4 * up + 3] = 0.0f;
            }
        }
    } else {
        out[e] = val;
    }
}

// Error reporting: thread-local message returned by ct_last_error().
ct_status set_error(ct_status st, const char *fmt, ...);
ct_status cuda_error(cudaError_t e, const char *what);

#define CT_CUDA(call)                                                        \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) return ::ct::cuda_error(e_, #call);           \
    } while (0)

#define CT_LAUNCH_CHECK(what)                                                \
    do {                                                                     \
        cudaError_t e_ = cudaGetLastError();                                 \
        if (e_ != cudaSuccess) return ::ct::cuda_error(e_, what);            \
    } while (0)

// Device memory carved out of one buffer (caller workspace or one
// stream-ordered allocation).
struct Arena {
    char *base = nullptr;
    size_t size = 0;
    size_t used = 0;
    bool owned = false;
    cudaStream_t stream = nullptr;
    static size_t align(size_t b) { return (b + 255) & ~size_t(255); }
    template <typename T>
    T *take(size_t count) {
        size_t b = align(count * sizeof(T));
        if (!base) {  // counting mode: only add up the size
            used += b;
            return nullptr;
        }
        if (used + b > size) return nullptr;
        T *p = reinterpret_cast<T *>(base + used);
        used += b;
        return p;
    }
};
// Opens an arena of `bytes`: uses the caller's workspace when given (and
// large enough), else cudaMallocAsync on `stream`.
ct_status arena_open(Arena &a, size_t bytes, void *workspace, size_t workspace_bytes,
                     cudaStream_t stream);
void arena_close(Arena &a);

// Sizes (bytes, each rounded to 256) of the operator working buffers.
size_t plane_copies_bytes(const GeomDev &g);      // Xc + Yc
size_t padded_sino_bytes(const GeomDev &g);
// 4-byte words in the quad-interleaved padded sinogram (4 floats or 4 bf16 per entry)
inline size_t padded_sino_floats(const GeomDev &g)
{
    return size_t(g.n_views) * g.nvp * g.pitchU * (g.sino_bf16 ? 2 : 4);
}

// bf16 <-> float helpers for the packed working copies
__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);   // .x in the low half
    return *reinterpret_cast<const uint32_t *>(&p);
}

// Stores the horizontal pair (S[v][u], S[v][u+1]) of a quad-layout
// sinogram: it is the first half of entry (v, u) and the second half of
// entry (v-1, u), one 8-byte (4-byte for bf16) store each.  u may be -1
// (S[v][-1] = 0): the padded layout has that column.  FP32 halves are
// stored in the row-difference form (S[v][u], S[v][u+1] - S[v][u]).
__device__ __forceinline__ void store_sino_pair(float *out, const SinoLayout &lay, int s, int iv, int iu, float lo,
                                                float hi)
{
    const size_t e = (size_t(s) * lay.rows_per_view + iv + lay.row_off) * lay.pitch + iu + lay.col_off;
    const size_t up = e - lay.pitch;
    if (lay.bf16) {
        uint32_t *o = reinterpret_cast<uint32_t *>(out);
        const uint32_t w = pack_bf16x2(lo, hi);
        o[2 * e] = w;
        o[2 * up + 1] = w;
    } else {
        float2 *o = reinterpret_cast<float2 *>(out);
        o[2 * e] = make_float2(lo, hi - lo);
        o[2 * up + 1] = make_float2(lo, hi - lo);
    }
}

// --- projector (ct_project.cu) ---------------------------------------------------
// Builds the plane-major zero-bordered copies Xc, Yc (float, or bf16 pairs
// when g.vol_bf16) of the volume `vol` scaled by (*scale) when scale !=
// nullptr; when `basis_out` is given the scaled volume is also stored there
// (the Arnoldi normalisation), as float or, when g.vol_bf16, as bf16.
cudaError_t launch_plane_copies(const GeomDev &g, const float *vol, const double *scale, void *basis_out,
                                float *Xc, float *Yc, const int *stop, cudaStream_t st);
// y = A x from the plane copies (Joseph; the line-intersection projector
// reads Yc only), written in `lay`.
cudaError_t launch_project_A(const GeomDev &g, const float *Xc, const float *Yc, float *y,
                            SinoLayout lay, const int *stop, cudaStream_t st);
// x = A^T y (overwritten); y in plain layout.  Xa, Ya: accumulators of the
// projector's copy sizes (contents overwritten).
cudaError_t launch_project_At(const GeomDev &g, const float *y, float *x, float *Xa, float *Ya, const int *stop,
                             cudaStream_t st);
// the line-intersection projector and its transpose (ct_siddon.cu); x overwritten
cudaError_t launch_siddon_A(const GeomDev &g, const float *Yc, float *y, SinoLayout lay, const int *stop,
                            cudaStream_t st);
cudaError_t launch_siddon_At(const GeomDev &g, const float *y, float *x, const int *stop, cudaStream_t st);

// --- back-projector (ct_backproject.cu) ------------------------------------------
// Copies a plain sinogram into the padded layout, scaled by (*scale) when
// given; `normalize_inplace` also writes the scaled values back to `src`.
cudaError_t launch_pad_sino(const GeomDev &g, float *src, const double *scale,
                            bool normalize_inplace, float *dst, const int *stop,
                            cudaStream_t st);
// dst = F src (or F^T src) from a plain sinogram into layout `lay`.
cudaError_t launch_ramp(const GeomDev &g, const float *src, float *dst, SinoLayout lay,
                        bool transpose, const int *stop, cudaStream_t st);
// Form of the FP32 entries of a padded quad sinogram (bf16 entries always
// hold the four values).
enum QuadForm { QUAD_ROWDIFF, QUAD_CORNERS };
// x = B_un y from the padded sinogram: QUAD_ROWDIFF after launch_pad_sino or
// launch_ramp, QUAD_CORNERS after a projector wrote it with store_sino.
cudaError_t launch_voxel_B(const GeomDev &g, const float *ypad, float *x, const int *stop,
                           cudaStream_t st, QuadForm form);
// y += B_un^T x (y plain, zeroed by the caller).
cudaError_t launch_voxel_Bt(const GeomDev &g, const float *x, float *y, const int *stop,
                            cudaStream_t st);

// --- vector kernels (ct_krylov.cu) ---------------------------------------------
int num_sms();
// Raises the dynamic shared-memory limit of kernel `func` on the current
// device to at least `bytes` (never lowers it).  The limit is process-wide per
// function, so callers on other threads with other sizes (geometries with
// other view counts) must not lower it under a launch that needs more.
cudaError_t raise_dyn_smem(const void *func, size_t bytes);

// --- host-side fault injection (ct_fault.cu; CT_FAULT, ct_fault_set) --------------
struct FaultSpec {
    int nan_at_iter = 0;   // iteration (>= 1) whose new vector gets a NaN; 0 = off
    int oom = 0;           // refuse stream-ordered allocations
};
FaultSpec fault_spec();
// Writes a NaN into v[0] when the spec names this iteration (1-based).
cudaError_t fault_poison(float *v, int iteration, const int *stop, cudaStream_t st);

// --- NVTX ranges: one per C-ABI call and per solver iteration ---------------------
// (host-side markers around the launches; free when no tool is attached)
class NvtxRange {
public:
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// --- optional per-kernel timing (ct_profile.cu) ----------------------------------
enum ProfKind {
    PK_PLANE_COPIES = 0, PK_JOSEPH_A, PK_RAMP, PK_PAD_SINO, PK_VOXEL_B, PK_MGS, PK_SMALL,
    PK_COMBINE, PK_JOSEPH_AT, PK_VOXEL_BT, PK_CGLS_VEC, PROF_KINDS
};
// Records a CUDA event pair around the launches made in its scope when
// profiling is on (ct_profile_enable); costs one mutex lock otherwise.
class ProfScope {
public:
    ProfScope(int kind, cudaStream_t st);
    ~ProfScope();
    ProfScope(const ProfScope &) = delete;
    ProfScope &operator=(const ProfScope &) = delete;
private:
    int kind_;
    cudaStream_t st_;
    void *a_;
};

}  // namespace ct

struct ct_geom {
    ct_geom_desc desc;
    int device;
    ct::GeomDev g;
    void *d_tables;
    size_t n, m;
};
