// Krylov solvers: BA-GMRES (Eq. 5), AB-GMRES (Eq. 4) and CGLS (Eqs. 2-3).
//
// Arnoldi with modified Gram-Schmidt (Sec. II): the newest Krylov vector q
// is orthogonalised against the basis one vector at a time.  Each pass is
// one streaming kernel that applies the previous projection
// (q -= h_{i-1} v_{i-1}) and forms the next inner product <q, v_i> in the
// same sweep over memory, so pass i reads q, v_{i-1}, v_i and writes q once.
// Inner products: per-thread FP32 accumulation (plain FMA, or compensated
// with an FMA two-product and a two-sum), warp-shuffle and block reductions
// in FP64, and a last-block grid reduction in a fixed order (deterministic,
// no spin-waits).  The Hessenberg column, the Givens rotations, the
// residual estimate |g_{j+1}| and the final triangular solve run in FP64 in
// one-thread kernels, so the whole solve is enqueued without host round
// trips; a device status word stops the remaining kernels on a tolerance
// stop, a lucky breakdown or a non-finite norm.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <unordered_map>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "ct_internal.cuh"

namespace ct {

constexpr int RED_BLOCK = 256;

enum : int { ST_RUN = 0, ST_TOL = 1, ST_LUCKY = 2, ST_NONFINITE = 3 };

// Device-resident solver state.
struct SolverState {
    int status;
    int iters;
    unsigned counter;
    int reorth_skip;
    double inv_norm;    // scale that normalises the newest basis vector
    double ref_sumsq;   // ||S v_j||^2 before orthogonalisation
    double sumsq;       // ||q||^2 after orthogonalisation
    double sumsq_pre2;  // ||q||^2 before the optional second sweep
    // CGLS scalars
    double gamma, gamma_new, delta, rr, data_rr;
};

// ---------------------------------------------------------------------------
// accumulators
// ---------------------------------------------------------------------------
template <int MODE>
struct Acc;

template <>
struct Acc<1> {  // FP32 FMA accumulation, FP64 reduction
    float s = 0.0f;
    __device__ __forceinline__ void add(float a, float b) { s = fmaf(a, b, s); }
    __device__ __forceinline__ double value() const { return double(s); }
};

template <>
struct Acc<0> {  // compensated: two-product (FMA) + two-sum in FP32
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float a, float b)
    {
        const float p = __fmul_rn(a, b);
        const float pe = fmaf(a, b, -p);
        const float t = __fadd_rn(s, p);
        const float bp = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
        s = t;
        c = __fadd_rn(c, __fadd_rn(e, pe));
    }
    __device__ __forceinline__ double value() const { return double(s) + double(c); }
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block sum of two values; result valid in thread 0.
__device__ __forceinline__ void block_sum2(double &a, double &b)
{
    __shared__ double sa[RED_BLOCK / 32], sb[RED_BLOCK / 32];
    a = warp_sum(a);
    b = warp_sum(b);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        sa[w] = a;
        sb[w] = b;
    }
    __syncthreads();
    if (w == 0) {
        a = lane < RED_BLOCK / 32 ? sa[lane] : 0.0;
        b = lane < RED_BLOCK / 32 ? sb[lane] : 0.0;
        a = warp_sum(a);
        b = warp_sum(b);
    }
}

// Stores the block's partial sums; the last block to finish sums all
// partials in block order and writes the outputs.
__device__ __forceinline__ void grid_finish(double a, double b, double *partials, unsigned *counter,
                                            double *out_a, double *out_b)
{
    __shared__ bool last;
    block_sum2(a, b);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = b;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double ta = 0.0, tb = 0.0;
    for (int i = threadIdx.x; i < int(gridDim.x); i += RED_BLOCK) {
        ta += __ldcg(partials + 2 * i);
        tb += __ldcg(partials + 2 * i + 1);
    }
    block_sum2(ta, tb);
    if (threadIdx.x == 0) {
        if (out_a) *out_a = ta;
        if (out_b) *out_b = tb;
        *counter = 0u;
    }
}

// ---------------------------------------------------------------------------
// One MGS pass: q -= (*hprev) vprev (if vprev), then <q, vcur> (if vcur) and
// ||q||^2 (if out_sumsq).  Stops early on *stop, or on *skip when given.
// ---------------------------------------------------------------------------
// One group of 4 elements of the FP32 pass: q -= h v_prev (stored back),
// then the dot with v_cur and the sum of squares of the new q.
template <int MODE>
__device__ __forceinline__ void mgs_group4(float4 *q4, float4 a, float4 p, float4 c, bool has_prev, bool has_cur,
                                           bool sumsq, float h, Acc<MODE> &dot, Acc<MODE> &ss)
{
    if (has_prev) {
        a.x = fmaf(-h, p.x, a.x);
        a.y = fmaf(-h, p.y, a.y);
        a.z = fmaf(-h, p.z, a.z);
        a.w = fmaf(-h, p.w, a.w);
        *q4 = a;
    }
    if (has_cur) {
        dot.add(a.x, c.x);
        dot.add(a.y, c.y);
        dot.add(a.z, c.z);
        dot.add(a.w, c.w);
    }
    if (sumsq) {
        ss.add(a.x, a.x);
        ss.add(a.y, a.y);
        ss.add(a.z, a.z);
        ss.add(a.w, a.w);
    }
}

template <int MODE>
__global__ void __launch_bounds__(RED_BLOCK) mgs_pass_kernel(
    float *__restrict__ q, const float *__restrict__ vprev, const double *__restrict__ hprev,
    const float *__restrict__ vcur, size_t len, int vec4, double *__restrict__ partials,
    unsigned *__restrict__ counter, double *__restrict__ out_dot, double *__restrict__ out_sumsq,
    const int *__restrict__ stop, const int *__restrict__ skip)
{
    if ((stop && *stop) || (skip && *skip)) return;
    const float h = vprev ? float(*hprev) : 0.0f;
    Acc<MODE> dot, ss;
    const size_t tid = blockIdx.x * size_t(RED_BLOCK) + threadIdx.x;
    const size_t nth = size_t(gridDim.x) * RED_BLOCK;
    size_t start = 0;
    if (vec4) {
        const size_t n4 = len / 4;
        float4 *q4 = reinterpret_cast<float4 *>(q);
        const float4 *p4 = reinterpret_cast<const float4 *>(vprev);
        const float4 *c4 = reinterpret_cast<const float4 *>(vcur);
        const float4 zero = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        // two groups of 4 per step: the six 16-byte loads are in flight together
        // (basis vectors stream through L2 evict-first)
        size_t i = tid;
        for (; i + nth < n4; i += 2 * nth) {
            const size_t i1 = i + nth;
            const float4 a0 = q4[i], a1 = q4[i1];
            const float4 p0 = vprev ? __ldcs(p4 + i) : zero, p1 = vprev ? __ldcs(p4 + i1) : zero;
            const float4 c0 = vcur ? __ldcs(c4 + i) : zero, c1 = vcur ? __ldcs(c4 + i1) : zero;
            mgs_group4(q4 + i, a0, p0, c0, vprev != nullptr, vcur != nullptr, out_sumsq != nullptr, h, dot, ss);
            mgs_group4(q4 + i1, a1, p1, c1, vprev != nullptr, vcur != nullptr, out_sumsq != nullptr, h, dot, ss);
        }
        if (i < n4)
            mgs_group4(q4 + i, q4[i], vprev ? __ldcs(p4 + i) : zero, vcur ? __ldcs(c4 + i) : zero, vprev != nullptr,
                       vcur != nullptr, out_sumsq != nullptr, h, dot, ss);
        start = n4 * 4;
    }
    for (size_t i = start + tid; i < len; i += nth) {
        float a = q[i];
        if (vprev) {
            a = fmaf(-h, vprev[i], a);
            q[i] = a;
        }
        if (vcur) dot.add(a, vcur[i]);
        if (out_sumsq) ss.add(a, a);
    }
    grid_finish(dot.value(), ss.value(), partials, counter, out_dot, out_sumsq);
}

// The same pass with a bf16 basis (FP32 work vector q): eight elements per
// step, the basis read as 16-byte vectors.
__device__ __forceinline__ void unpack8(const uint4 w, float (&o)[8])
{
    o[0] = bf16_lo(w.x); o[1] = bf16_hi(w.x); o[2] = bf16_lo(w.y); o[3] = bf16_hi(w.y);
    o[4] = bf16_lo(w.z); o[5] = bf16_hi(w.z); o[6] = bf16_lo(w.w); o[7] = bf16_hi(w.w);
}

// One group of 8 elements of the bf16-basis pass: q -= h v_prev (stored
// back), then the dot with v_cur and the sum of squares of the new q.
template <int MODE>
__device__ __forceinline__ void mgs_group8(float4 *q4, float4 lo, float4 hi, uint4 pw, uint4 cw, bool has_prev,
                                           bool has_cur, bool sumsq, float h, Acc<MODE> &dot, Acc<MODE> &ss)
{
    float a[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
    if (has_prev) {
        float pv[8];
        unpack8(pw, pv);
#pragma unroll
        for (int e = 0; e < 8; ++e) a[e] = fmaf(-h, pv[e], a[e]);
        q4[0] = make_float4(a[0], a[1], a[2], a[3]);
        q4[1] = make_float4(a[4], a[5], a[6], a[7]);
    }
    if (has_cur) {
        float cv[8];
        unpack8(cw, cv);
#pragma unroll
        for (int e = 0; e < 8; ++e) dot.add(a[e], cv[e]);
    }
    if (sumsq) {
#pragma unroll
        for (int e = 0; e < 8; ++e) ss.add(a[e], a[e]);
    }
}

template <int MODE>
__global__ void __launch_bounds__(RED_BLOCK) mgs_pass_bf16_kernel(
    float *__restrict__ q, const __nv_bfloat16 *__restrict__ vprev, const double *__restrict__ hprev,
    const __nv_bfloat16 *__restrict__ vcur, size_t len, int vec8, double *__restrict__ partials,
    unsigned *__restrict__ counter, double *__restrict__ out_dot, double *__restrict__ out_sumsq,
    const int *__restrict__ stop, const int *__restrict__ skip)
{
    if ((stop && *stop) || (skip && *skip)) return;
    const float h = vprev ? float(*hprev) : 0.0f;
    Acc<MODE> dot, ss;
    const size_t tid = blockIdx.x * size_t(RED_BLOCK) + threadIdx.x;
    const size_t nth = size_t(gridDim.x) * RED_BLOCK;
    size_t start = 0;
    if (vec8) {
        const size_t n8 = len / 8;
        float4 *q4 = reinterpret_cast<float4 *>(q);
        const uint4 *p8 = reinterpret_cast<const uint4 *>(vprev);
        const uint4 *c8 = reinterpret_cast<const uint4 *>(vcur);
        const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
        // two groups of 8 per step: all six 16-byte loads are in flight together
        size_t i = tid;
        for (; i + nth < n8; i += 2 * nth) {
            const size_t i1 = i + nth;
            const float4 l0 = q4[2 * i], h0 = q4[2 * i + 1], l1 = q4[2 * i1], h1 = q4[2 * i1 + 1];
            const uint4 p0 = vprev ? __ldcs(p8 + i) : zero, p1 = vprev ? __ldcs(p8 + i1) : zero;
            const uint4 c0 = vcur ? __ldcs(c8 + i) : zero, c1 = vcur ? __ldcs(c8 + i1) : zero;
            mgs_group8(q4 + 2 * i, l0, h0, p0, c0, vprev != nullptr, vcur != nullptr, out_sumsq != nullptr, h, dot, ss);
            mgs_group8(q4 + 2 * i1, l1, h1, p1, c1, vprev != nullptr, vcur != nullptr, out_sumsq != nullptr, h, dot,
                       ss);
        }
        if (i < n8)
            mgs_group8(q4 + 2 * i, q4[2 * i], q4[2 * i + 1], vprev ? __ldcs(p8 + i) : zero,
                       vcur ? __ldcs(c8 + i) : zero, vprev != nullptr, vcur != nullptr, out_sumsq != nullptr, h, dot,
                       ss);
        start = n8 * 8;
    }
    for (size_t i = start + tid; i < len; i += nth) {
        float a = q[i];
        if (vprev) {
            a = fmaf(-h, __bfloat162float(vprev[i]), a);
            q[i] = a;
        }
        if (vcur) dot.add(a, __bfloat162float(vcur[i]));
        if (out_sumsq) ss.add(a, a);
    }
    grid_finish(dot.value(), ss.value(), partials, counter, out_dot, out_sumsq);
}

// sum (a - b)^2 -> *out (recomputed data residuals)
__global__ void __launch_bounds__(RED_BLOCK) diff_sumsq_kernel(const float *__restrict__ a,
                                                               const float *__restrict__ b, size_t len,
                                                               double *__restrict__ partials,
                                                               unsigned *__restrict__ counter,
                                                               double *__restrict__ out,
                                                               const int *__restrict__ stop)
{
    if (stop && *stop) return;
    Acc<1> ss;
    for (size_t i = blockIdx.x * size_t(RED_BLOCK) + threadIdx.x; i < len;
         i += size_t(gridDim.x) * RED_BLOCK) {
        const float d = a[i] - b[i];
        ss.add(d, d);
    }
    grid_finish(0.0, ss.value(), partials, counter, nullptr, out);
}

static unsigned red_blocks(size_t len)
{
    size_t want = (len / 4 + RED_BLOCK - 1) / RED_BLOCK;
    size_t cap = size_t(num_sms()) * 8;
    return unsigned(std::max<size_t>(1, std::min(want, cap)));
}

// Blocks of a grid-stride pass over len elements (elems per thread-step):
// every SM gets as many blocks as can be resident at once (at most 8, the
// size of the partials array), so no partial second wave runs.
static unsigned resident_blocks(const void *kernel, size_t len, size_t elems)
{
    static std::mutex mu;
    static std::unordered_map<const void *, int> occ;
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = occ.find(kernel);
        if (it == occ.end()) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, RED_BLOCK, 0) != cudaSuccess) {
                cudaGetLastError();
                per_sm = 4;
            }
            occ.emplace(kernel, per_sm);
        } else {
            per_sm = it->second;
        }
    }
    per_sm = std::min(std::max(per_sm, 1), 8);
    const size_t want = (len / elems + RED_BLOCK - 1) / RED_BLOCK;
    return unsigned(std::max<size_t>(1, std::min(want, size_t(num_sms()) * per_sm)));
}

static size_t partials_count() { return size_t(num_sms()) * 8 * 2; }

static cudaError_t mgs_pass(int mode, float *q, const float *vprev, const double *hprev,
                            const float *vcur, size_t len, double *partials, unsigned *counter,
                            double *out_dot, double *out_sumsq, const int *stop, const int *skip,
                            cudaStream_t st)
{
    const int vec4 = (len % 4 == 0) && (reinterpret_cast<uintptr_t>(q) % 16 == 0) &&
                     (!vprev || reinterpret_cast<uintptr_t>(vprev) % 16 == 0) &&
                     (!vcur || reinterpret_cast<uintptr_t>(vcur) % 16 == 0);
    const unsigned blocks = resident_blocks(
        mode == 0 ? reinterpret_cast<const void *>(mgs_pass_kernel<0>)
                  : reinterpret_cast<const void *>(mgs_pass_kernel<1>), len, 4);
    ProfScope prof(PK_MGS, st);
    if (mode == 0)
        mgs_pass_kernel<0><<<blocks, RED_BLOCK, 0, st>>>(q, vprev, hprev, vcur, len, vec4, partials,
                                                         counter, out_dot, out_sumsq, stop, skip);
    else
        mgs_pass_kernel<1><<<blocks, RED_BLOCK, 0, st>>>(q, vprev, hprev, vcur, len, vec4, partials,
                                                         counter, out_dot, out_sumsq, stop, skip);
    return cudaGetLastError();
}

// MGS pass over a typed basis (float or bf16 vectors; q is always float).
static cudaError_t mgs_pass_typed(int mode, bool vbf16, float *q, const void *vprev, const double *hprev,
                                  const void *vcur, size_t len, double *partials, unsigned *counter,
                                  double *out_dot, double *out_sumsq, const int *stop, const int *skip,
                                  cudaStream_t st)
{
    if (!vbf16)
        return mgs_pass(mode, q, static_cast<const float *>(vprev), hprev, static_cast<const float *>(vcur), len,
                        partials, counter, out_dot, out_sumsq, stop, skip, st);
    const int vec8 = (len % 8 == 0) && (reinterpret_cast<uintptr_t>(q) % 16 == 0) &&
                     (!vprev || reinterpret_cast<uintptr_t>(vprev) % 16 == 0) &&
                     (!vcur || reinterpret_cast<uintptr_t>(vcur) % 16 == 0);
    const unsigned blocks = resident_blocks(
        mode == 0 ? reinterpret_cast<const void *>(mgs_pass_bf16_kernel<0>)
                  : reinterpret_cast<const void *>(mgs_pass_bf16_kernel<1>), len, 16);
    ProfScope prof(PK_MGS, st);
    const auto *p = static_cast<const __nv_bfloat16 *>(vprev);
    const auto *c = static_cast<const __nv_bfloat16 *>(vcur);
    if (mode == 0)
        mgs_pass_bf16_kernel<0><<<blocks, RED_BLOCK, 0, st>>>(q, p, hprev, c, len, vec8, partials, counter, out_dot,
                                                              out_sumsq, stop, skip);
    else
        mgs_pass_bf16_kernel<1><<<blocks, RED_BLOCK, 0, st>>>(q, p, hprev, c, len, vec8, partials, counter, out_dot,
                                                              out_sumsq, stop, skip);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Small FP64 kernels of the GMRES least-squares problem.
// H, R: (k+1) x k, column-major with leading dimension k+1.
// ---------------------------------------------------------------------------
__global__ void gmres_init_kernel(SolverState *st, double *g, double *resid, int k)
{
    const double beta = sqrt(st->sumsq);
    for (int i = 0; i <= k; ++i) {
        g[i] = 0.0;
        resid[i] = -1.0;
    }
    g[0] = beta;
    resid[0] = beta;
    st->iters = 0;
    st->status = ST_RUN;
    if (!isfinite(beta)) {
        st->status = ST_NONFINITE;
    } else if (beta == 0.0) {
        st->status = ST_LUCKY;  // b (or B b) is zero: x = 0 is exact
    } else {
        st->inv_norm = 1.0 / beta;
    }
}

__global__ void sqrt_inplace_kernel(double *p) { *p = sqrt(*p); }

__global__ void reorth_decide_kernel(SolverState *st)
{
    // second sweep only when the first removed at least half of the squared
    // norm (||q_after|| <= ||q_before|| / sqrt 2)
    st->reorth_skip = !(st->sumsq <= 0.5 * st->ref_sumsq);
    st->sumsq_pre2 = st->sumsq;
}

__global__ void givens_kernel(int j, int k, double *H, const double *H2, double *R, double *cs,
                              double *sn, double *g, double *resid, SolverState *st, double tol)
{
    if (st->status != ST_RUN) return;
    const int ld = k + 1;
    double *h = H + size_t(j) * ld;
    if (H2 && !st->reorth_skip)
        for (int i = 0; i <= j; ++i) h[i] += H2[i];
    const double hnext = sqrt(st->sumsq);
    const double ref = sqrt(st->ref_sumsq);
    h[j + 1] = hnext;
    bool bad = !isfinite(hnext) || !isfinite(ref);
    for (int i = 0; i <= j; ++i) bad = bad || !isfinite(h[i]);
    if (bad) {
        st->status = ST_NONFINITE;
        return;
    }
    const bool lucky = hnext <= 1e-14 * ref;
    double *r = R + size_t(j) * ld;
    for (int i = 0; i <= j; ++i) r[i] = h[i];
    r[j + 1] = lucky ? 0.0 : hnext;
    for (int i = 0; i < j; ++i) {
        const double t = cs[i] * r[i] + sn[i] * r[i + 1];
        r[i + 1] = -sn[i] * r[i] + cs[i] * r[i + 1];
        r[i] = t;
    }
    const double a = r[j], b = r[j + 1];
    const double rr = hypot(a, b);
    double c = 1.0, s = 0.0;
    if (rr != 0.0) {
        c = a / rr;
        s = b / rr;
    }
    cs[j] = c;
    sn[j] = s;
    r[j] = rr;
    r[j + 1] = 0.0;
    g[j + 1] = -s * g[j];
    g[j] = c * g[j];
    // a column that vanishes after the rotations (a breakdown on which the
    // operator is singular) cannot reduce g[j]: the least-squares residual
    // stays, and the back substitution gives that coefficient 0
    resid[j + 1] = rr != 0.0 ? fabs(g[j + 1]) : hypot(g[j], g[j + 1]);
    st->iters = j + 1;
    if (lucky || rr == 0.0) {
        st->status = ST_LUCKY;
    } else {
        st->inv_norm = 1.0 / hnext;
        if (tol > 0.0 && resid[j + 1] <= tol * resid[0]) st->status = ST_TOL;
    }
}

// *cnt = j when iterate j exists (j <= iterations done), else 0
__global__ void iterate_count_kernel(const SolverState *st, int j, int *cnt) { *cnt = j <= st->iters ? j : 0; }

// *cnt = min(k, iterations done): the iterate x_k, or the last one when fewer exist
__global__ void iterate_upto_kernel(const SolverState *st, int k, int *cnt) { *cnt = st->iters < k ? st->iters : k; }

// y = R_j^{-1} g_j for the first *cnt columns: the least-squares coefficients
// of iterate x_j (R's first j columns and g's first j entries are final once
// iteration j is done)
__global__ void backsolve_count_kernel(const double *R, const double *g, double *y, const int *cnt, int k)
{
    const int it = *cnt;
    const int ld = k + 1;
    for (int i = it - 1; i >= 0; --i) {
        double acc = g[i];
        for (int l = i + 1; l < it; ++l) acc -= R[size_t(l) * ld + i] * y[l];
        const double d = R[size_t(i) * ld + i];
        y[i] = d != 0.0 ? acc / d : 0.0;
    }
}

// err[j] = sqrt(err[j]) for the iterates that exist, -1 after them
__global__ void err_finish_kernel(double *err, const SolverState *st, int k)
{
    for (int j = 0; j <= k; ++j) err[j] = j <= st->iters ? sqrt(err[j]) : -1.0;
}

__global__ void backsolve_kernel(const double *R, const double *g, double *y, const SolverState *st, int k)
{
    const int it = st->iters;
    const int ld = k + 1;
    for (int i = it - 1; i >= 0; --i) {
        double acc = g[i];
        for (int l = i + 1; l < it; ++l) acc -= R[size_t(l) * ld + i] * y[l];
        const double d = R[size_t(i) * ld + i];
        y[i] = d != 0.0 ? acc / d : 0.0;
    }
}

// x = sum_{i < count} y_i V_i ; count = *count_ptr when given, else k
template <typename TB>
__global__ void __launch_bounds__(RED_BLOCK) combine_kernel(const TB *__restrict__ V, size_t ldv, int k,
                                                            size_t len, const double *__restrict__ y,
                                                            const int *__restrict__ count_ptr,
                                                            float *__restrict__ x)
{
    extern __shared__ float ys[];
    const int count = count_ptr ? min(*count_ptr, k) : k;
    for (int i = threadIdx.x; i < count; i += RED_BLOCK) ys[i] = float(y[i]);
    __syncthreads();
    for (size_t e = blockIdx.x * size_t(RED_BLOCK) + threadIdx.x; e < len;
         e += size_t(gridDim.x) * RED_BLOCK) {
        float acc = 0.0f;
        for (int i = 0; i < count; ++i) acc = fmaf(ys[i], float(V[i * ldv + e]), acc);
        x[e] = acc;
    }
}

template <typename TB>
static cudaError_t combine_t(const TB *V, size_t ldv, int k, size_t len, const double *y, const int *count_ptr,
                             float *x, cudaStream_t st)
{
    const size_t smem = std::max<size_t>(1, size_t(k)) * sizeof(float);
    if (smem > 48 * 1024) {
        cudaError_t e = raise_dyn_smem(reinterpret_cast<const void *>(combine_kernel<TB>),
                                       std::min<size_t>(smem, 200 * 1024));
        if (e != cudaSuccess) return e;
    }
    const unsigned blocks = unsigned(std::max<size_t>(1, std::min((len + RED_BLOCK - 1) / RED_BLOCK,
                                                                  size_t(num_sms()) * 8)));
    ProfScope prof(PK_COMBINE, st);
    combine_kernel<TB><<<blocks, RED_BLOCK, smem, st>>>(V, ldv, k, len, y, count_ptr, x);
    return cudaGetLastError();
}

static cudaError_t combine(const float *V, size_t ldv, int k, size_t len, const double *y, const int *count_ptr,
                           float *x, cudaStream_t st)
{
    return combine_t<float>(V, ldv, k, len, y, count_ptr, x, st);
}

// ---------------------------------------------------------------------------
// CGLS vector kernels (coefficients from device scalars).
// ---------------------------------------------------------------------------
// y += sign * (*num / *den) * x ; optionally ||y||^2
__global__ void __launch_bounds__(RED_BLOCK) axpy_ratio_kernel(float *__restrict__ y, const float *__restrict__ x,
                                                               const double *__restrict__ num,
                                                               const double *__restrict__ den, float sign,
                                                               size_t len, double *__restrict__ partials,
                                                               unsigned *__restrict__ counter,
                                                               double *__restrict__ out_sumsq,
                                                               const int *__restrict__ stop)
{
    if (stop && *stop) return;
    const float a = sign * float(*num / *den);
    Acc<1> ss;
    for (size_t i = blockIdx.x * size_t(RED_BLOCK) + threadIdx.x; i < len;
         i += size_t(gridDim.x) * RED_BLOCK) {
        const float v = fmaf(a, x[i], y[i]);
        y[i] = v;
        ss.add(v, v);
    }
    if (out_sumsq) grid_finish(0.0, ss.value(), partials, counter, nullptr, out_sumsq);
}

// p = s + (*num / *den) p
__global__ void xpby_ratio_kernel(float *__restrict__ p, const float *__restrict__ s,
                                  const double *__restrict__ num, const double *__restrict__ den,
                                  size_t len, const int *__restrict__ stop)
{
    if (stop && *stop) return;
    const float b = float(*num / *den);
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < len;
         i += size_t(gridDim.x) * blockDim.x)
        p[i] = fmaf(b, p[i], s[i]);
}

__global__ void cgls_check_kernel(SolverState *st, int phase)
{
    if (st->status != ST_RUN) return;
    if (phase == 0) {  // after delta = ||A p||^2
        if (!isfinite(st->delta) || !isfinite(st->gamma)) st->status = ST_NONFINITE;
        else if (st->delta == 0.0 || st->gamma == 0.0) st->status = ST_LUCKY;
    }
}

__global__ void cgls_record_kernel(SolverState *st, double *resid, int j, int use_data, double tol)
{
    if (st->status != ST_RUN) return;
    const double v = sqrt(use_data ? st->data_rr : st->rr);
    resid[j] = v;
    st->iters = j;
    if (!isfinite(v) || !isfinite(st->gamma_new)) {
        st->status = ST_NONFINITE;
        return;
    }
    if (tol > 0.0 && v <= tol * resid[0]) st->status = ST_TOL;
}

__global__ void cgls_shift_kernel(SolverState *st)
{
    if (st->status != ST_RUN) return;
    st->gamma = st->gamma_new;
}

__global__ void cgls_init_kernel(SolverState *st, double *resid, int k)
{
    for (int i = 0; i <= k; ++i) resid[i] = -1.0;
    resid[0] = sqrt(st->rr);
    st->iters = 0;
    st->status = ST_RUN;
    if (!isfinite(st->gamma) || !isfinite(resid[0])) st->status = ST_NONFINITE;
    else if (st->gamma == 0.0) st->status = ST_LUCKY;
}

// ---------------------------------------------------------------------------
// Operator plumbing shared by the solvers.
// ---------------------------------------------------------------------------
struct OpBufs {
    float *Xc = nullptr, *Yc = nullptr;  // plane-major volume copies
    float *ypad = nullptr;               // padded sinogram
    float *t = nullptr;                  // plain sinogram
};

static void take_op_bufs(Arena &ar, const GeomDev &g, OpBufs &b, bool need_t)
{
    b.Xc = ar.take<float>(size_t(g.nzp) * g.nx * g.pitchX);
    b.Yc = ar.take<float>(size_t(g.nzp) * g.ny * g.pitchY);
    b.ypad = ar.take<float>(padded_sino_floats(g));
    b.t = need_t ? ar.take<float>(size_t(g.n_views) * g.nv * g.nu) : nullptr;
}

// out_vol = B sino.  `sino` is a plain sinogram, scaled by (*scale) first when
// given (and normalised in place when `normalize`).
static cudaError_t apply_B(const GeomDev &g, int b_kind, float *sino, const double *scale, bool normalize,
                           OpBufs &b, float *out_vol, const int *stop, cudaStream_t st,
                           float *scratch_vec /* n floats for A^T zeroing, unused otherwise */)
{
    (void)scratch_vec;
    cudaError_t e = cudaSuccess;
    if (b_kind == CT_B_UN) {
        e = launch_pad_sino(g, sino, scale, normalize, b.ypad, stop, st);
        if (e == cudaSuccess) e = launch_voxel_B(g, b.ypad, out_vol, stop, st, QUAD_ROWDIFF);
        return e;
    }
    if (scale) {
        // normalise in place through the padded copy (values only), then filter / scatter
        e = launch_pad_sino(g, sino, scale, true, b.ypad, stop, st);
        if (e != cudaSuccess) return e;
    }
    if (b_kind == CT_B_FBP) {
        e = launch_ramp(g, sino, b.ypad, padded_layout(g), false, stop, st);
        if (e == cudaSuccess) e = launch_voxel_B(g, b.ypad, out_vol, stop, st, QUAD_ROWDIFF);
        return e;
    }
    // exact transpose A^T (the projector's copies serve as its accumulators)
    return launch_project_At(g, sino, out_vol, b.Xc, b.Yc, stop, st);
}

static ct_status check_common(const ct_geom *geom, const float *b, int k, const float *x,
                              const ct_solve_opts *o)
{
    if (!geom || !b || !x) return set_error(CT_EINVAL, "solver: NULL argument");
    if (k < 1) return set_error(CT_EINVAL, "solver: k must be >= 1 (got %d)", k);
    if (k > 4096) return set_error(CT_EINVAL, "solver: k must be <= 4096 (got %d)", k);
    if (o->b_kind != CT_B_UN && o->b_kind != CT_B_FBP && o->b_kind != CT_B_AT)
        return set_error(CT_EINVAL, "solver: unknown b_kind %d", o->b_kind);
    if (o->dot_mode != 0 && o->dot_mode != 1)
        return set_error(CT_EINVAL, "solver: dot_mode must be 0 or 1");
    if (!(o->tol >= 0.0)) return set_error(CT_EINVAL, "solver: tol must be >= 0");
    return CT_OK;
}

static size_t round_ld(size_t len) { return (len + 63) & ~size_t(63); }

// Carves the GMRES workspace; with a counting arena (base == nullptr) it
// only adds up the size.
struct GmresWs {
    void *V = nullptr;      // k+1 basis vectors, float or (BA-GMRES with vol_bf16) bf16
    bool vbf16 = false;
    size_t ldv = 0;
    float *q = nullptr;     // BA-GMRES: FP32 work vector (new Krylov vector)
    OpBufs ob;
    float *tvol = nullptr;  // AB-GMRES: B v_j
    double *H = nullptr, *H2 = nullptr, *R = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr,
           *resid = nullptr, *y = nullptr, *partials = nullptr;
    double *err = nullptr;  // squared distances of the iterates to a reference image
    int *cnt = nullptr;     // iterate count for the error history
    SolverState *st = nullptr;
    const void *vec(int i) const
    {
        return static_cast<const char *>(V) + size_t(i) * ldv * (vbf16 ? 2 : 4);
    }
    void *vec(int i) { return static_cast<char *>(V) + size_t(i) * ldv * (vbf16 ? 2 : 4); }
};

// Bytes of the k+1 basis vectors of a BA (ab = false) or AB workspace.
static size_t basis_bytes(const GeomDev &g, int k, bool ab)
{
    const size_t len = ab ? size_t(g.n_views) * g.nv * g.nu : size_t(g.nx) * g.ny * g.nz;
    return Arena::align(round_ld(len) * size_t(k + 1) * ((!ab && g.vol_bf16) ? 2 : 4));
}

// external_basis: the basis lives elsewhere (w.V is set by the caller)
static bool carve_gmres(Arena &ar, const GeomDev &g, int k, bool ab, int b_kind, GmresWs &w,
                        bool external_basis = false)
{
    const size_t n = size_t(g.nx) * g.ny * g.nz;
    const size_t m = size_t(g.n_views) * g.nv * g.nu;
    const size_t len = ab ? m : n;
    w.ldv = round_ld(len);
    w.vbf16 = !ab && g.vol_bf16;
    if (external_basis)
        w.V = nullptr;
    else if (w.vbf16)
        w.V = ar.take<__nv_bfloat16>(w.ldv * size_t(k + 1));
    else
        w.V = ar.take<float>(w.ldv * size_t(k + 1));
    if (!ab) w.q = ar.take<float>(n);
    // BA needs a plain sinogram when B reads one (F or A^T); AB never does
    take_op_bufs(ar, g, w.ob, !ab && b_kind != CT_B_UN);
    if (ab) w.tvol = ar.take<float>(n);
    const size_t ld = size_t(k) + 1;
    w.H = ar.take<double>(ld * k);
    w.H2 = ar.take<double>(ld);
    w.R = ar.take<double>(ld * k);
    w.cs = ar.take<double>(k);
    w.sn = ar.take<double>(k);
    w.g = ar.take<double>(ld);
    w.resid = ar.take<double>(ld);
    w.y = ar.take<double>(k);
    w.partials = ar.take<double>(partials_count());
    w.err = ar.take<double>(ld);
    w.cnt = ar.take<int>(1);
    w.st = ar.take<SolverState>(1);
    return w.st != nullptr;
}

static size_t gmres_bytes(const GeomDev &g, int k, bool ab, int b_kind, bool external_basis = false)
{
    Arena ar;
    ar.size = ~size_t(0) >> 1;
    ar.base = nullptr;
    GmresWs w;
    carve_gmres(ar, g, k, ab, b_kind, w, external_basis);
    return ar.used;
}

// Host-resident basis streamed through the device by the copy engine.  The
// basis vectors live in page-locked host memory; the newest one is written to
// a device buffer (vnew) and copied out on a copy stream while the operators
// run; each MGS sweep brings the older vectors back into a ring of three
// device buffers, V_i into slot i mod 3, two vectors ahead of the pass that
// reads them (the copy of V_{i+2} waits for pass i, the last reader of the
// slot's previous vector).  The kernels read only device memory, so a pass
// runs at the copy's pace instead of at the kernels' own reads over the
// host link.
struct Stager {
    cudaStream_t cs = nullptr;       // copy stream
    void *ring[3] = {};              // device slots, one basis vector each
    void *vnew = nullptr;            // device copy of the newest vector
    char *host = nullptr;            // host basis, vector i at host + i * vbytes_ld
    size_t vbytes = 0;               // bytes copied per vector
    size_t vbytes_ld = 0;            // stride of the host vectors
    cudaEvent_t ev[8] = {};
    int evi = 0;
    cudaEvent_t vnew_free = nullptr; // the last copy out of vnew has finished
    cudaEvent_t ready[3] = {};       // per slot: its current vector has arrived

    cudaEvent_t next_event() { cudaEvent_t e = ev[evi]; evi = (evi + 1) % 8; return e; }
    // copies host vector i into slot i mod 3 after the work enqueued on s so far
    cudaError_t fetch(int i, cudaStream_t s)
    {
        cudaEvent_t e = next_event();
        cudaError_t r = cudaEventRecord(e, s);
        if (r == cudaSuccess) r = cudaStreamWaitEvent(cs, e, 0);
        if (r == cudaSuccess)
            r = cudaMemcpyAsync(ring[i % 3], host + size_t(i) * vbytes_ld, vbytes, cudaMemcpyHostToDevice, cs);
        if (r == cudaSuccess) r = cudaEventRecord(ready[i % 3], cs);
        return r;
    }
    // the device copy of V_i for a sweep whose newest vector is V_j (in vnew);
    // makes s wait for its arrival
    const void *vector(int i, int j, cudaStream_t s)
    {
        if (i == j) return vnew;
        cudaStreamWaitEvent(s, ready[i % 3], 0);
        return ring[i % 3];
    }
    // copies vnew out to host vector j after the work enqueued on s so far
    cudaError_t store_new(int j, cudaStream_t s)
    {
        cudaEvent_t e = next_event();
        cudaError_t r = cudaEventRecord(e, s);
        if (r == cudaSuccess) r = cudaStreamWaitEvent(cs, e, 0);
        if (r == cudaSuccess)
            r = cudaMemcpyAsync(host + size_t(j) * vbytes_ld, vnew, vbytes, cudaMemcpyDeviceToHost, cs);
        if (r == cudaSuccess) r = cudaEventRecord(vnew_free, cs);
        return r;
    }
};

// One MGS sweep (passes i = 0..j+1) over a staged basis: V_i for i < j comes
// through the ring, V_j from vnew.
// With `prefetched`, V_0 and V_1 were fetched already (at the start of the
// iteration, so that their copies overlap the operators).
static cudaError_t staged_sweep(Stager &sg, int mode, bool vbf16, float *q, int j, double *hcol, size_t len,
                                double *partials, unsigned *ctr, double *first_ss, double *last_ss,
                                const int *stop, const int *skip, cudaStream_t s, bool prefetched)
{
    cudaError_t e = cudaSuccess;
    if (!prefetched && 0 < j) e = sg.fetch(0, s);
    if (!prefetched && e == cudaSuccess && 1 < j) e = sg.fetch(1, s);
    for (int i = 0; i <= j + 1 && e == cudaSuccess; ++i) {
        const void *vprev = i > 0 ? sg.vector(i - 1, j, s) : nullptr;
        const void *vcur = i <= j ? sg.vector(i, j, s) : nullptr;
        const double *hprev = i > 0 ? hcol + (i - 1) : nullptr;
        double *odot = i <= j ? hcol + i : nullptr;
        double *oss = i == 0 ? first_ss : (i == j + 1 ? last_ss : nullptr);
        e = mgs_pass_typed(mode, vbf16, q, vprev, hprev, vcur, len, partials, ctr, odot, oss, stop, skip, s);
        // slot (i + 2) mod 3 held V_{i-1}, whose last reader was this pass
        if (e == cudaSuccess && i + 2 < j) e = sg.fetch(i + 2, s);
    }
    return e;
}

// Enqueues the MGS sweep of iteration j (the new vector q against
// V_0..V_j) and its Givens step.
static cudaError_t arnoldi_orthogonalise(GmresWs &w, float *q, int j, int k, size_t len, const ct_solve_opts &o,
                                         cudaStream_t s, Stager *sg = nullptr)
{
    const int *stop = &w.st->status;
    unsigned *ctr = &w.st->counter;
    double *hcol = w.H + size_t(j) * (k + 1);
    cudaError_t e = fault_poison(q, j + 1, stop, s);
    if (sg) {
        if (e == cudaSuccess)
            e = staged_sweep(*sg, o.dot_mode, w.vbf16, q, j, hcol, len, w.partials, ctr, &w.st->ref_sumsq,
                             &w.st->sumsq, stop, nullptr, s, true);
        if (e != cudaSuccess) return e;
        const double *H2s = nullptr;
        if (o.reorth) {
            { ProfScope prof(PK_SMALL, s); reorth_decide_kernel<<<1, 1, 0, s>>>(w.st); }
            e = staged_sweep(*sg, o.dot_mode, w.vbf16, q, j, w.H2, len, w.partials, ctr, nullptr, &w.st->sumsq,
                             stop, &w.st->reorth_skip, s, false);
            if (e != cudaSuccess) return e;
            H2s = w.H2;
        }
        { ProfScope prof(PK_SMALL, s); givens_kernel<<<1, 1, 0, s>>>(j, k, w.H, H2s, w.R, w.cs, w.sn, w.g, w.resid, w.st, o.tol); }
        return cudaGetLastError();
    }
    for (int i = 0; i <= j + 1 && e == cudaSuccess; ++i) {
        const void *vprev = i > 0 ? w.vec(i - 1) : nullptr;
        const double *hprev = i > 0 ? hcol + (i - 1) : nullptr;
        const void *vcur = i <= j ? w.vec(i) : nullptr;
        double *odot = i <= j ? hcol + i : nullptr;
        double *oss = i == 0 ? &w.st->ref_sumsq : (i == j + 1 ? &w.st->sumsq : nullptr);
        e = mgs_pass_typed(o.dot_mode, w.vbf16, q, vprev, hprev, vcur, len, w.partials, ctr, odot, oss, stop,
                           nullptr, s);
    }
    if (e != cudaSuccess) return e;
    const double *H2 = nullptr;
    if (o.reorth) {
        { ProfScope prof(PK_SMALL, s); reorth_decide_kernel<<<1, 1, 0, s>>>(w.st); }
        const int *skip = &w.st->reorth_skip;
        for (int i = 0; i <= j + 1 && e == cudaSuccess; ++i) {
            const void *vprev = i > 0 ? w.vec(i - 1) : nullptr;
            const double *hprev = i > 0 ? w.H2 + (i - 1) : nullptr;
            const void *vcur = i <= j ? w.vec(i) : nullptr;
            double *odot = i <= j ? w.H2 + i : nullptr;
            double *oss = i == j + 1 ? &w.st->sumsq : nullptr;
            e = mgs_pass_typed(o.dot_mode, w.vbf16, q, vprev, hprev, vcur, len, w.partials, ctr, odot, oss, stop,
                               skip, s);
        }
        if (e != cudaSuccess) return e;
        H2 = w.H2;
    }
    { ProfScope prof(PK_SMALL, s); givens_kernel<<<1, 1, 0, s>>>(j, k, w.H, H2, w.R, w.cs, w.sn, w.g, w.resid, w.st, o.tol); }
    return cudaGetLastError();
}

static ct_status finish_solve(SolverState *st_dev, const double *resid_dev, int k, double *resid_hist,
                              int *iters_done, cudaStream_t s, const char *who)
{
    SolverState hst;
    std::vector<double> hres(size_t(k) + 1);
    CT_CUDA(cudaMemcpyAsync(&hst, st_dev, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
    CT_CUDA(cudaMemcpyAsync(hres.data(), resid_dev, sizeof(double) * (k + 1), cudaMemcpyDeviceToHost, s));
    CT_CUDA(cudaStreamSynchronize(s));
    if (resid_hist) std::copy(hres.begin(), hres.end(), resid_hist);
    if (iters_done) *iters_done = hst.iters;
    if (hst.status == ST_NONFINITE)
        return set_error(CT_ENONFINITE, "%s: a norm became NaN/Inf after %d iterations", who, hst.iters);
    if (hst.status == ST_LUCKY) return CT_BREAKDOWN_LUCKY;
    return CT_OK;
}

static ct_status open_ws(Arena &ar, size_t bytes, const ct_solve_opts &o, cudaStream_t s)
{
    return arena_open(ar, bytes, o.workspace, o.workspace_bytes, s);
}

// ---------------------------------------------------------------------------
// BA-GMRES
// ---------------------------------------------------------------------------
// BA-GMRES in three steps, shared by the one-call solve and the persistent
// solver state (kmax: the workspace's capacity, the leading dimension of H).
//
// Start (x0 = 0): r0 = B b into q; ||r0|| starts the residual history.
static cudaError_t ba_start(const GeomDev &g, GmresWs &w, const float *b, int kmax, size_t n,
                            const ct_solve_opts &o, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(w.st, 0, sizeof(SolverState), s);
    // zero the padded sinogram once: its border is never written afterwards
    if (e == cudaSuccess)
        e = cudaMemsetAsync(w.ob.ypad, 0, padded_sino_floats(g) * sizeof(float), s);
    if (e == cudaSuccess)
        e = apply_B(g, o.b_kind, const_cast<float *>(b), nullptr, false, w.ob, w.q, nullptr, s, nullptr);
    if (e == cudaSuccess)
        e = mgs_pass(o.dot_mode, w.q, nullptr, nullptr, nullptr, n, w.partials, &w.st->counter, nullptr,
                     &w.st->sumsq, nullptr, nullptr, s);
    if (e == cudaSuccess) {
        { ProfScope prof(PK_SMALL, s); gmres_init_kernel<<<1, 1, 0, s>>>(w.st, w.g, w.resid, kmax); }
        e = cudaGetLastError();
    }
    return e;
}

// Iteration j (0-based): v_j = q / ||q|| joins the basis, q = B A v_j is
// orthogonalised against v_0..v_j, and the Givens step updates the residual.
static cudaError_t ba_iteration(const GeomDev &g, GmresWs &w, int j, int kmax, size_t n, const ct_solve_opts &o,
                                cudaStream_t s, Stager *sg = nullptr)
{
    NvtxRange iter_range("BA-GMRES iteration");
    const int *stop = &w.st->status;
    cudaError_t e = cudaSuccess;
    // a staged basis: vnew is rewritten only after its previous copy out; the
    // first two vectors of this iteration's sweep start coming in now
    if (sg) {
        e = cudaStreamWaitEvent(s, sg->vnew_free, 0);
        if (e == cudaSuccess && 0 < j) e = sg->fetch(0, s);
        if (e == cudaSuccess && 1 < j) e = sg->fetch(1, s);
    }
    // v_j = q / ||q|| stored in the basis while the projector's plane copies are built
    if (e == cudaSuccess)
        e = launch_plane_copies(g, w.q, &w.st->inv_norm, sg ? sg->vnew : w.vec(j), w.ob.Xc, w.ob.Yc, stop, s);
    if (e == cudaSuccess && sg) e = sg->store_new(j, s);
    if (e != cudaSuccess) return e;
    // q = B A v_j
    if (o.b_kind == CT_B_UN) {
        e = launch_project_A(g, w.ob.Xc, w.ob.Yc, w.ob.ypad, padded_layout(g), stop, s);
        if (e == cudaSuccess) e = launch_voxel_B(g, w.ob.ypad, w.q, stop, s, QUAD_CORNERS);
    } else {
        e = launch_project_A(g, w.ob.Xc, w.ob.Yc, w.ob.t, plain_layout(g), stop, s);
        if (e == cudaSuccess) e = apply_B(g, o.b_kind, w.ob.t, nullptr, false, w.ob, w.q, stop, s, nullptr);
    }
    if (e == cudaSuccess) e = arnoldi_orthogonalise(w, w.q, j, kmax, n, o, s, sg);
    return e;
}

static ct_status bagmres(const ct_geom *geom, const float *b, int k, float *x, double *resid_hist,
                         const ct_solve_opts &o, int *iters_done, cudaStream_t s, const float *x_ref = nullptr,
                         double *err_hist = nullptr)
{
    const GeomDev &g = geom->g;
    const size_t n = geom->n;
    Arena ar;
    ct_status rc = open_ws(ar, gmres_bytes(g, k, false, o.b_kind), o, s);
    if (rc != CT_OK) return rc;
    GmresWs w;
    carve_gmres(ar, g, k, false, o.b_kind, w);
    cudaError_t e = ba_start(g, w, b, k, n, o, s);
    for (int j = 0; j < k && e == cudaSuccess; ++j) e = ba_iteration(g, w, j, k, n, o, s);
    // distance of every iterate x_j = V_j y_j to x_ref (x_out is the scratch
    // image; the final x_k is formed after)
    if (x_ref && e == cudaSuccess) {
        const unsigned vb = red_blocks(n);
        e = mgs_pass(1, const_cast<float *>(x_ref), nullptr, nullptr, nullptr, n, w.partials, &w.st->counter,
                     nullptr, &w.err[0], nullptr, nullptr, s);
        for (int j = 1; j <= k && e == cudaSuccess; ++j) {
            {
                ProfScope prof(PK_SMALL, s);
                iterate_count_kernel<<<1, 1, 0, s>>>(w.st, j, w.cnt);
                backsolve_count_kernel<<<1, 1, 0, s>>>(w.R, w.g, w.y, w.cnt, k);
            }
            e = w.vbf16 ? combine_t(static_cast<const __nv_bfloat16 *>(w.V), w.ldv, k, n, w.y, w.cnt, x, s)
                        : combine(static_cast<const float *>(w.V), w.ldv, k, n, w.y, w.cnt, x, s);
            if (e == cudaSuccess) {
                ProfScope prof(PK_CGLS_VEC, s);
                diff_sumsq_kernel<<<vb, RED_BLOCK, 0, s>>>(x, x_ref, n, w.partials, &w.st->counter, &w.err[j],
                                                           nullptr);
                e = cudaGetLastError();
            }
        }
        if (e == cudaSuccess) {
            { ProfScope prof(PK_SMALL, s); err_finish_kernel<<<1, 1, 0, s>>>(w.err, w.st, k); }
            e = cudaGetLastError();
        }
        if (e == cudaSuccess && err_hist)
            e = cudaMemcpyAsync(err_hist, w.err, sizeof(double) * (k + 1), cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) {
        { ProfScope prof(PK_SMALL, s); backsolve_kernel<<<1, 1, 0, s>>>(w.R, w.g, w.y, w.st, k); }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = w.vbf16 ? combine_t(static_cast<const __nv_bfloat16 *>(w.V), w.ldv, k, n, w.y, &w.st->iters, x, s)
                    : combine(static_cast<const float *>(w.V), w.ldv, k, n, w.y, &w.st->iters, x, s);
    if (e != cudaSuccess) {
        arena_close(ar);
        return cuda_error(e, "ct_bagmres_solve launch");
    }
    rc = finish_solve(w.st, w.resid, k, resid_hist, iters_done, s, "ct_bagmres_solve");
    arena_close(ar);
    return rc;
}

// ---------------------------------------------------------------------------
// Restarted BA-GMRES(m): cycles of m iterations, each on the residual
// system B A dx = B (b - A x) from dx = 0, then x += dx.
// ---------------------------------------------------------------------------
__global__ void sub_kernel(float *__restrict__ out, const float *__restrict__ a, const float *__restrict__ b,
                           size_t len)
{
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < len; i += size_t(gridDim.x) * blockDim.x)
        out[i] = a[i] - b[i];
}

__global__ void add_kernel(float *__restrict__ x, const float *__restrict__ d, size_t len)
{
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < len; i += size_t(gridDim.x) * blockDim.x)
        x[i] += d[i];
}

static ct_status bagmres_restarted(const ct_geom *geom, const float *b, int m, int cycles, float *x,
                                   double *resid_hist, const ct_solve_opts &o, int *iters_done, cudaStream_t s)
{
    const GeomDev &g = geom->g;
    const size_t n = geom->n, mm = geom->m;
    const size_t copies = size_t(g.nzp) * g.nx * g.pitchX + size_t(g.nzp) * g.ny * g.pitchY;
    float *buf = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&buf), sizeof(float) * (copies + 2 * mm + n), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(CT_ENOMEM, "ct_bagmres_restarted: %zu bytes of scratch: %s",
                         sizeof(float) * (copies + 2 * mm + n), cudaGetErrorString(e));
    }
    float *Xc = buf, *Yc = buf + size_t(g.nzp) * g.nx * g.pitchX;
    float *ax = buf + copies, *rb = ax + mm, *dx = rb + mm;
    const unsigned blocks = unsigned(std::min<size_t>((std::max(n, mm) + 255) / 256, size_t(num_sms()) * 16));
    std::vector<double> hist(size_t(m) + 1);
    int total = 0;
    ct_status rc = CT_OK;
    e = cudaMemsetAsync(x, 0, n * sizeof(float), s);
    if (resid_hist)
        for (int i = 0; i <= m * cycles; ++i) resid_hist[i] = -1.0;
    for (int c = 0; c < cycles && e == cudaSuccess; ++c) {
        const float *rhs = b;
        if (c > 0) {   // rb = b - A x
            e = launch_plane_copies(g, x, nullptr, nullptr, Xc, Yc, nullptr, s);
            if (e == cudaSuccess) e = launch_project_A(g, Xc, Yc, ax, plain_layout(g), nullptr, s);
            if (e == cudaSuccess) {
                sub_kernel<<<blocks, 256, 0, s>>>(rb, b, ax, mm);
                e = cudaGetLastError();
            }
            rhs = rb;
        }
        if (e != cudaSuccess) break;
        int it = 0;
        rc = bagmres(geom, rhs, m, dx, hist.data(), o, &it, s);
        if (rc != CT_OK && rc != CT_BREAKDOWN_LUCKY) break;
        add_kernel<<<blocks, 256, 0, s>>>(x, dx, n);
        e = cudaGetLastError();
        if (resid_hist) {
            if (c == 0) resid_hist[0] = hist[0];
            for (int j = 1; j <= it; ++j) resid_hist[total + j] = hist[j];
        }
        total += it;
        // a tolerance stop (relative to this cycle's start) or a breakdown ends the solve
        if (it < m || rc == CT_BREAKDOWN_LUCKY) break;
        if (o.tol > 0.0 && resid_hist && resid_hist[total] <= o.tol * resid_hist[0]) break;
    }
    cudaError_t e2 = cudaFreeAsync(buf, s);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (iters_done) *iters_done = total;
    if (e != cudaSuccess) return cuda_error(e, "ct_bagmres_restarted");
    return rc;
}

// ---------------------------------------------------------------------------
// AB-GMRES
// ---------------------------------------------------------------------------
static ct_status abgmres(const ct_geom *geom, const float *b, int k, float *x, double *resid_hist,
                         const ct_solve_opts &o, int *iters_done, cudaStream_t s)
{
    const GeomDev &g = geom->g;
    const size_t m = geom->m;
    Arena ar;
    ct_status rc = open_ws(ar, gmres_bytes(g, k, true, o.b_kind), o, s);
    if (rc != CT_OK) return rc;
    GmresWs w;
    carve_gmres(ar, g, k, true, o.b_kind, w);
    float *Vf = static_cast<float *>(w.V);   // data-space basis, FP32
    const int *stop = &w.st->status;
    cudaError_t e = cudaMemsetAsync(w.st, 0, sizeof(SolverState), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.ob.ypad, 0, padded_sino_floats(g) * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Vf, b, m * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = mgs_pass(o.dot_mode, Vf, nullptr, nullptr, nullptr, m, w.partials, &w.st->counter, nullptr,
                     &w.st->sumsq, nullptr, nullptr, s);
    if (e == cudaSuccess) {
        { ProfScope prof(PK_SMALL, s); gmres_init_kernel<<<1, 1, 0, s>>>(w.st, w.g, w.resid, k); }
        e = cudaGetLastError();
    }
    for (int j = 0; j < k && e == cudaSuccess; ++j) {
        NvtxRange iter_range("AB-GMRES iteration");
        float *vj = Vf + size_t(j) * w.ldv;
        float *q = Vf + size_t(j + 1) * w.ldv;
        e = apply_B(g, o.b_kind, vj, &w.st->inv_norm, true, w.ob, w.tvol, stop, s, nullptr);
        if (e == cudaSuccess) e = launch_plane_copies(g, w.tvol, nullptr, nullptr, w.ob.Xc, w.ob.Yc, stop, s);
        if (e == cudaSuccess) e = launch_project_A(g, w.ob.Xc, w.ob.Yc, q, plain_layout(g), stop, s);
        if (e == cudaSuccess) e = arnoldi_orthogonalise(w, q, j, k, m, o, s);
    }
    if (e == cudaSuccess) {
        { ProfScope prof(PK_SMALL, s); backsolve_kernel<<<1, 1, 0, s>>>(w.R, w.g, w.y, w.st, k); }
        e = cudaGetLastError();
    }
    // u = V y (data space) into the last basis slot, then x = B u
    float *u = Vf + size_t(k) * w.ldv;
    if (e == cudaSuccess) e = combine(Vf, w.ldv, k, m, w.y, &w.st->iters, u, s);
    if (e == cudaSuccess) e = apply_B(g, o.b_kind, u, nullptr, false, w.ob, x, nullptr, s, nullptr);
    if (e != cudaSuccess) {
        arena_close(ar);
        return cuda_error(e, "ct_abgmres_solve launch");
    }
    rc = finish_solve(w.st, w.resid, k, resid_hist, iters_done, s, "ct_abgmres_solve");
    arena_close(ar);
    return rc;
}

// ---------------------------------------------------------------------------
// Gradient through a converged BA-GMRES solve.  x = (BA)^{-1} B b, so for a
// scalar loss L(x) with gx = dL/dx:  dL/db = B^T (BA)^{-T} gx = B^T z with
// (A^T B^T) z = gx.  z comes from GMRES on A^T B^T (image-space basis, built
// afresh: the forward basis is not kept), each step applying B^T (voxel
// splatting, then F^T for B_FBP) and A^T (ray scatter).
// ---------------------------------------------------------------------------
struct VjpWs {
    GmresWs gm;
    float *t = nullptr, *tf = nullptr;   // sinogram-space temporaries
    float *Xa = nullptr, *Ya = nullptr;  // A^T accumulators (the projector's copy layout)
};

static void carve_vjp(Arena &ar, const GeomDev &g, int k, int b_kind, VjpWs &w)
{
    const size_t n = size_t(g.nx) * g.ny * g.nz;
    const size_t m = size_t(g.n_views) * g.nv * g.nu;
    w.gm.ldv = round_ld(n);
    w.gm.V = ar.take<float>(w.gm.ldv * size_t(k + 1));
    w.t = ar.take<float>(m);
    w.tf = b_kind == CT_B_FBP ? ar.take<float>(m) : nullptr;
    w.Xa = ar.take<float>(size_t(g.nzp) * g.nx * g.pitchX);
    w.Ya = ar.take<float>(size_t(g.nzp) * g.ny * g.pitchY);
    const size_t ld = size_t(k) + 1;
    w.gm.H = ar.take<double>(ld * k);
    w.gm.H2 = ar.take<double>(ld);
    w.gm.R = ar.take<double>(ld * k);
    w.gm.cs = ar.take<double>(k);
    w.gm.sn = ar.take<double>(k);
    w.gm.g = ar.take<double>(ld);
    w.gm.resid = ar.take<double>(ld);
    w.gm.y = ar.take<double>(k);
    w.gm.partials = ar.take<double>(partials_count());
    w.gm.st = ar.take<SolverState>(1);
}

static size_t vjp_bytes(const GeomDev &g, int k, int b_kind)
{
    Arena ar;
    ar.size = ~size_t(0) >> 1;
    VjpWs w;
    carve_vjp(ar, g, k, b_kind, w);
    return ar.used;
}

__global__ void scale_vec_kernel(float *__restrict__ v, size_t len, const double *__restrict__ scale,
                                 const int *__restrict__ stop)
{
    if (stop && *stop) return;
    const float sc = float(*scale);
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < len; i += size_t(gridDim.x) * blockDim.x)
        v[i] *= sc;
}

// out_sino = B^T vol (plain layout); b_kind B_UN or B_FBP
static cudaError_t apply_Bt(const GeomDev &g, int b_kind, const float *vol, float *t, float *tf, float *out,
                            const int *stop, cudaStream_t s)
{
    const size_t m = size_t(g.n_views) * g.nv * g.nu;
    float *dst = b_kind == CT_B_FBP ? t : out;
    cudaError_t e = cudaMemsetAsync(dst, 0, m * sizeof(float), s);
    if (e == cudaSuccess) e = launch_voxel_Bt(g, vol, dst, stop, s);
    if (e == cudaSuccess && b_kind == CT_B_FBP) e = launch_ramp(g, t, out, plain_layout(g), true, stop, s);
    (void)tf;
    return e;
}

static ct_status bagmres_vjp(const ct_geom *geom, const float *gx, int k, float *gb, double *resid_hist,
                             const ct_solve_opts &o, int *iters_done, cudaStream_t s)
{
    if (o.b_kind == CT_B_AT)
        return set_error(CT_EINVAL, "ct_bagmres_vjp: b_kind must be CT_B_UN or CT_B_FBP");
    const GeomDev &g = geom->g;
    const size_t n = geom->n;
    Arena ar;
    ct_status rc = open_ws(ar, vjp_bytes(g, k, o.b_kind), o, s);
    if (rc != CT_OK) return rc;
    VjpWs w;
    carve_vjp(ar, g, k, o.b_kind, w);
    GmresWs &gm = w.gm;
    const int *stop = &gm.st->status;
    const unsigned vb = red_blocks(n);
    float *Vf = static_cast<float *>(gm.V);   // image-space basis, FP32
    float *sino = o.b_kind == CT_B_FBP ? w.tf : w.t;   // B^T v lands here
    cudaError_t e = cudaMemsetAsync(gm.st, 0, sizeof(SolverState), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Vf, gx, n * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = mgs_pass(o.dot_mode, Vf, nullptr, nullptr, nullptr, n, gm.partials, &gm.st->counter, nullptr,
                     &gm.st->sumsq, nullptr, nullptr, s);
    if (e == cudaSuccess) {
        { ProfScope prof(PK_SMALL, s); gmres_init_kernel<<<1, 1, 0, s>>>(gm.st, gm.g, gm.resid, k); }
        e = cudaGetLastError();
    }
    for (int j = 0; j < k && e == cudaSuccess; ++j) {
        NvtxRange iter_range("adjoint GMRES iteration");
        float *vj = Vf + size_t(j) * gm.ldv;
        float *q = Vf + size_t(j + 1) * gm.ldv;
        {
            ProfScope prof(PK_CGLS_VEC, s);
            scale_vec_kernel<<<vb, RED_BLOCK, 0, s>>>(vj, n, &gm.st->inv_norm, stop);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = apply_Bt(g, o.b_kind, vj, w.t, w.tf, sino, stop, s);
        if (e == cudaSuccess) e = launch_project_At(g, sino, q, w.Xa, w.Ya, stop, s);
        if (e == cudaSuccess) e = arnoldi_orthogonalise(gm, q, j, k, n, o, s);
    }
    if (e == cudaSuccess) {
        { ProfScope prof(PK_SMALL, s); backsolve_kernel<<<1, 1, 0, s>>>(gm.R, gm.g, gm.y, gm.st, k); }
        e = cudaGetLastError();
    }
    float *z = Vf + size_t(k) * gm.ldv;
    if (e == cudaSuccess) e = combine(Vf, gm.ldv, k, n, gm.y, &gm.st->iters, z, s);
    if (e == cudaSuccess) e = apply_Bt(g, o.b_kind, z, w.t, w.tf, gb, nullptr, s);
    if (e != cudaSuccess) {
        arena_close(ar);
        return cuda_error(e, "ct_bagmres_vjp launch");
    }
    rc = finish_solve(gm.st, gm.resid, k, resid_hist, iters_done, s, "ct_bagmres_vjp");
    arena_close(ar);
    return rc;
}

// ---------------------------------------------------------------------------
// CGLS with back-projector B
// ---------------------------------------------------------------------------
struct CglsWs {
    OpBufs ob;
    float *r = nullptr, *s = nullptr, *p = nullptr, *q = nullptr, *ax = nullptr;
    double *resid = nullptr, *partials = nullptr;
    SolverState *st = nullptr;
};

static void carve_cgls(Arena &ar, const GeomDev &g, int k, bool data_resid, CglsWs &w)
{
    const size_t n = size_t(g.nx) * g.ny * g.nz;
    const size_t m = size_t(g.n_views) * g.nv * g.nu;
    take_op_bufs(ar, g, w.ob, false);
    w.r = ar.take<float>(m);
    w.q = ar.take<float>(m);
    w.s = ar.take<float>(n);
    w.p = ar.take<float>(n);
    w.ax = data_resid ? ar.take<float>(m) : nullptr;
    w.resid = ar.take<double>(size_t(k) + 1);
    w.partials = ar.take<double>(partials_count());
    w.st = ar.take<SolverState>(1);
}

static size_t cgls_ws_bytes(const GeomDev &g, int k, bool data_resid)
{
    Arena ar;
    ar.size = ~size_t(0) >> 1;
    CglsWs w;
    carve_cgls(ar, g, k, data_resid, w);
    return ar.used;
}

static ct_status cgls(const ct_geom *geom, const float *b, int k, float *x, double *resid_hist,
                      const ct_solve_opts &o, int *iters_done, cudaStream_t s)
{
    const GeomDev &g = geom->g;
    const size_t n = geom->n, m = geom->m;
    const bool data = o.record_data_resid != 0;
    Arena ar;
    ct_status rc = open_ws(ar, cgls_ws_bytes(g, k, data), o, s);
    if (rc != CT_OK) return rc;
    CglsWs w;
    carve_cgls(ar, g, k, data, w);
    SolverState *st = w.st;
    const int *stop = &st->status;
    unsigned *ctr = &st->counter;
    const unsigned vb = red_blocks(std::max(n, m));
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(SolverState), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.ob.ypad, 0, padded_sino_floats(g) * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, n * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w.r, b, m * sizeof(float), cudaMemcpyDeviceToDevice, s);
    // rr = ||r||^2, s = B r, gamma = ||s||^2, p = s
    if (e == cudaSuccess)
        e = mgs_pass(1, w.r, nullptr, nullptr, nullptr, m, w.partials, ctr, nullptr, &st->rr, nullptr, nullptr, s);
    if (e == cudaSuccess) e = apply_B(g, o.b_kind, w.r, nullptr, false, w.ob, w.s, nullptr, s, nullptr);
    if (e == cudaSuccess)
        e = mgs_pass(1, w.s, nullptr, nullptr, nullptr, n, w.partials, ctr, nullptr, &st->gamma, nullptr, nullptr, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w.p, w.s, n * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) {
        { ProfScope prof(PK_SMALL, s); cgls_init_kernel<<<1, 1, 0, s>>>(st, w.resid, k); }
        e = cudaGetLastError();
    }
    for (int j = 1; j <= k && e == cudaSuccess; ++j) {
        NvtxRange iter_range("CGLS iteration");
        // q = A p ; delta = ||q||^2
        e = launch_plane_copies(g, w.p, nullptr, nullptr, w.ob.Xc, w.ob.Yc, stop, s);
        if (e == cudaSuccess) e = launch_project_A(g, w.ob.Xc, w.ob.Yc, w.q, plain_layout(g), stop, s);
        if (e == cudaSuccess) e = fault_poison(w.q, j, stop, s);
        if (e == cudaSuccess)
            e = mgs_pass(1, w.q, nullptr, nullptr, nullptr, m, w.partials, ctr, nullptr, &st->delta, stop, nullptr, s);
        if (e == cudaSuccess) {
            { ProfScope prof(PK_SMALL, s); cgls_check_kernel<<<1, 1, 0, s>>>(st, 0); }
            e = cudaGetLastError();
        }
        // x += alpha p ; r -= alpha q (alpha = gamma / delta) ; rr = ||r||^2
        if (e == cudaSuccess) {
            ProfScope prof(PK_CGLS_VEC, s);
            axpy_ratio_kernel<<<vb, RED_BLOCK, 0, s>>>(x, w.p, &st->gamma, &st->delta, 1.0f, n, w.partials,
                                                       ctr, nullptr, stop);
            axpy_ratio_kernel<<<vb, RED_BLOCK, 0, s>>>(w.r, w.q, &st->gamma, &st->delta, -1.0f, m, w.partials,
                                                       ctr, &st->rr, stop);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess && data) {
            e = launch_plane_copies(g, x, nullptr, nullptr, w.ob.Xc, w.ob.Yc, stop, s);
            if (e == cudaSuccess) e = launch_project_A(g, w.ob.Xc, w.ob.Yc, w.ax, plain_layout(g), stop, s);
            if (e == cudaSuccess) {
                { ProfScope prof(PK_CGLS_VEC, s); diff_sumsq_kernel<<<vb, RED_BLOCK, 0, s>>>(b, w.ax, m, w.partials, ctr, &st->data_rr, stop); }
                e = cudaGetLastError();
            }
        }
        // s = B r ; gamma_new = ||s||^2 ; p = s + (gamma_new/gamma) p ; gamma = gamma_new
        if (e == cudaSuccess) e = apply_B(g, o.b_kind, w.r, nullptr, false, w.ob, w.s, stop, s, nullptr);
        if (e == cudaSuccess)
            e = mgs_pass(1, w.s, nullptr, nullptr, nullptr, n, w.partials, ctr, nullptr, &st->gamma_new, stop,
                         nullptr, s);
        if (e == cudaSuccess) {
            { ProfScope prof(PK_SMALL, s); cgls_record_kernel<<<1, 1, 0, s>>>(st, w.resid, j, data ? 1 : 0, o.tol); }
            { ProfScope prof(PK_CGLS_VEC, s); xpby_ratio_kernel<<<vb, RED_BLOCK, 0, s>>>(w.p, w.s, &st->gamma_new, &st->gamma, n, stop); }
            { ProfScope prof(PK_SMALL, s); cgls_shift_kernel<<<1, 1, 0, s>>>(st); }
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) {
        arena_close(ar);
        return cuda_error(e, "ct_cgls_solve launch");
    }
    rc = finish_solve(st, w.resid, k, resid_hist, iters_done, s, "ct_cgls_solve");
    arena_close(ar);
    return rc;
}

// ---------------------------------------------------------------------------
// Persistent BA-GMRES state: the workspace of one solve kept between calls,
// so a finished solve can be extended by more iterations, saved to a file
// and restored (the paper keeps its growing Krylov basis on disk, Sec. II).
// The basis lives in device memory or in page-locked host memory that the
// kernels read and write in place (on Grace-Blackwell over NVLink-C2C).
// ---------------------------------------------------------------------------
struct StateFileHeader {
    char magic[8];            // "CTGMRS01"
    int version;              // 1
    int vbf16;                // basis storage: 1 = bf16, 0 = float
    ct_geom_desc desc;        // the geometry the state belongs to
    int b_kind, dot_mode, reorth;
    int k_done;               // iterations done
    unsigned long long n;     // basis vector length
    SolverState st;           // device solver state at the save
};

}  // namespace ct

struct ct_gmres_state {
    const ct_geom *geom = nullptr;
    ct_solve_opts o{};
    int kmax = 0;
    int basis = CT_BASIS_DEVICE;
    void *dev_mem = nullptr;      // cudaMalloc'ed workspace (all but a host basis)
    void *host_basis = nullptr;   // cudaHostAlloc'ed basis (CT_BASIS_HOST)
    void *stage_mem = nullptr;    // cudaMalloc'ed ring and newest-vector buffers (CT_BASIS_HOST)
    ct::Stager stager;            // streams a host basis through stage_mem (CT_BASIS_HOST)
    ct::GmresWs w;
    int started = 0;
    int k_done = 0;               // iterations done, as of the last synchronising call
    int status = 0;               // device status word, as of the last synchronising call
};

namespace ct {

static void state_free(ct_gmres_state *st)
{
    if (!st) return;
    Stager &sg = st->stager;
    if (sg.cs) cudaStreamSynchronize(sg.cs);
    for (cudaEvent_t e : sg.ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : sg.ready)
        if (e) cudaEventDestroy(e);
    if (sg.vnew_free) cudaEventDestroy(sg.vnew_free);
    if (sg.cs) cudaStreamDestroy(sg.cs);
    if (st->dev_mem) cudaFree(st->dev_mem);
    if (st->stage_mem) cudaFree(st->stage_mem);
    if (st->host_basis) cudaFreeHost(st->host_basis);
    delete st;
}

// The copy stream, events and device buffers of a staged host basis.
static cudaError_t stager_init(ct_gmres_state *st)
{
    Stager &sg = st->stager;
    const GmresWs &w = st->w;
    const size_t esz = w.vbf16 ? 2 : 4;
    sg.vbytes = st->geom->n * esz;
    sg.vbytes_ld = w.ldv * esz;
    const size_t slot = Arena::align(sg.vbytes);
    cudaError_t e = cudaMalloc(&st->stage_mem, 4 * slot);
    if (e != cudaSuccess) return e;
    char *base = static_cast<char *>(st->stage_mem);
    for (int i = 0; i < 3; ++i) sg.ring[i] = base + i * slot;
    sg.vnew = base + 3 * slot;
    sg.host = static_cast<char *>(st->host_basis);
    e = cudaStreamCreateWithFlags(&sg.cs, cudaStreamNonBlocking);
    for (int i = 0; i < 8 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&sg.ev[i], cudaEventDisableTiming);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&sg.ready[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sg.vnew_free, cudaEventDisableTiming);
    return e;
}

__global__ void __launch_bounds__(RED_BLOCK) basis_axpy_kernel_f32(float *__restrict__ x, const float *__restrict__ v,
                                                                   const double *__restrict__ y, int i, size_t len)
{
    const float yi = float(y[i]);
    for (size_t e = blockIdx.x * size_t(RED_BLOCK) + threadIdx.x; e < len; e += size_t(gridDim.x) * RED_BLOCK)
        x[e] = fmaf(yi, v[e], i == 0 ? 0.0f : x[e]);
}

__global__ void __launch_bounds__(RED_BLOCK) basis_axpy_kernel_bf16(float *__restrict__ x,
                                                                    const __nv_bfloat16 *__restrict__ v,
                                                                    const double *__restrict__ y, int i, size_t len)
{
    const float yi = float(y[i]);
    for (size_t e = blockIdx.x * size_t(RED_BLOCK) + threadIdx.x; e < len; e += size_t(gridDim.x) * RED_BLOCK)
        x[e] = fmaf(yi, __bfloat162float(v[e]), i == 0 ? 0.0f : x[e]);
}

// x = sum_{i < count} y_i V_i over a staged basis, one vector at a time in
// the order (and with the FMA rounding) of combine_kernel, so the result is
// the same bits.
static cudaError_t staged_combine(Stager &sg, bool vbf16, int count, const double *y, size_t len, float *x,
                                  cudaStream_t s)
{
    if (count <= 0) return cudaMemsetAsync(x, 0, len * sizeof(float), s);
    cudaError_t e = sg.fetch(0, s);
    if (e == cudaSuccess && 1 < count) e = sg.fetch(1, s);
    const unsigned blocks = unsigned(std::max<size_t>(1, std::min((len + RED_BLOCK - 1) / RED_BLOCK,
                                                                  size_t(num_sms()) * 8)));
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
        const void *v = sg.vector(i, -1, s);
        {
            ProfScope prof(PK_COMBINE, s);
            if (vbf16)
                basis_axpy_kernel_bf16<<<blocks, RED_BLOCK, 0, s>>>(x, static_cast<const __nv_bfloat16 *>(v), y, i,
                                                                      len);
            else
                basis_axpy_kernel_f32<<<blocks, RED_BLOCK, 0, s>>>(x, static_cast<const float *>(v), y, i, len);
        }
        e = cudaGetLastError();
        if (e == cudaSuccess && i + 2 < count) e = sg.fetch(i + 2, s);
    }
    return e;
}

static ct_status state_alloc(const ct_geom *geom, int kmax, int basis, const ct_solve_opts &o, ct_gmres_state **out)
{
    const GeomDev &g = geom->g;
    const bool host = basis == CT_BASIS_HOST;
    ct_gmres_state *st = new (std::nothrow) ct_gmres_state;
    if (!st) return set_error(CT_ENOMEM, "ct_bagmres_state: out of host memory");
    st->geom = geom;
    st->o = o;
    st->o.tol = 0.0;   // the state runs exactly the iterations asked for
    st->o.workspace = nullptr;
    st->o.workspace_bytes = 0;
    st->kmax = kmax;
    st->basis = basis;
    const size_t bytes = gmres_bytes(g, kmax, false, o.b_kind, host);
    cudaError_t e = cudaMalloc(&st->dev_mem, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        st->dev_mem = nullptr;
        state_free(st);
        return set_error(CT_ENOMEM, "ct_bagmres_state: cudaMalloc(%zu bytes) failed", bytes);
    }
    Arena ar;
    ar.base = static_cast<char *>(st->dev_mem);
    ar.size = bytes;
    carve_gmres(ar, g, kmax, false, o.b_kind, st->w, host);
    if (host) {
        const size_t vb = basis_bytes(g, kmax, false);
        e = cudaHostAlloc(&st->host_basis, vb, cudaHostAllocMapped | cudaHostAllocPortable);
        if (e != cudaSuccess) {
            cudaGetLastError();
            st->host_basis = nullptr;
            state_free(st);
            return set_error(CT_ENOMEM, "ct_bagmres_state: cudaHostAlloc(%zu bytes) for the basis failed", vb);
        }
        // the kernels see only the device staging buffers; the host pointer
        // serves the copies (and save/load)
        st->w.V = st->host_basis;
        e = stager_init(st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            state_free(st);
            return set_error(CT_ENOMEM, "ct_bagmres_state: the device staging buffers of a host basis failed");
        }
    }
    *out = st;
    return CT_OK;
}

static ct_status state_check_device(const ct_geom *geom, const char *who)
{
    int dev = -1;
    CT_CUDA(cudaGetDevice(&dev));
    if (dev != geom->device)
        return set_error(CT_EINVAL, "%s: the geometry lives on device %d but device %d is current", who,
                         geom->device, dev);
    return CT_OK;
}

static bool same_desc(const ct_geom_desc &a, const ct_geom_desc &b)
{
    return a.kind == b.kind && a.nx == b.nx && a.ny == b.ny && a.nz == b.nz && a.voxel_mm == b.voxel_mm &&
           a.n_views == b.n_views && a.angle_start_rad == b.angle_start_rad &&
           a.angle_span_rad == b.angle_span_rad && a.nu == b.nu && a.nv == b.nv && a.du_mm == b.du_mm &&
           a.dv_mm == b.dv_mm && a.sod_mm == b.sod_mm && a.sdd_mm == b.sdd_mm && a.vol_dtype == b.vol_dtype &&
           a.sino_dtype == b.sino_dtype && a.projector == b.projector;
}

}  // namespace ct

using namespace ct;

static ct_solve_opts resolve_opts(const ct_solve_opts *opts)
{
    ct_solve_opts o;
    ct_solve_opts_default(&o);
    if (opts) o = *opts;
    return o;
}

extern "C" {

size_t ct_workspace_bytes(const ct_geom *geom, int k, int solver, const ct_solve_opts *opts)
{
    if (!geom || k < 1) return 0;
    ct_solve_opts o = resolve_opts(opts);
    switch (solver) {
    case CT_SOLVER_BA: return gmres_bytes(geom->g, k, false, o.b_kind);
    case CT_SOLVER_AB: return gmres_bytes(geom->g, k, true, o.b_kind);
    case CT_SOLVER_CGLS: return cgls_ws_bytes(geom->g, k, o.record_data_resid != 0);
    case CT_SOLVER_BA_VJP: return vjp_bytes(geom->g, k, o.b_kind);
    default: return 0;
    }
}

ct_status ct_bagmres_solve(const ct_geom *geom, const float *b_dev, int k, float *x_out_dev,
                           double *resid_hist, const ct_solve_opts *opts, int *iters_done, void *stream)
{
    NvtxRange call_range("ct_bagmres_solve");
    ct_solve_opts o = resolve_opts(opts);
    ct_status rc = check_common(geom, b_dev, k, x_out_dev, &o);
    if (rc != CT_OK) return rc;
    return bagmres(geom, b_dev, k, x_out_dev, resid_hist, o, iters_done, static_cast<cudaStream_t>(stream));
}

ct_status ct_bagmres_solve_host(const ct_geom *geom, const float *b_host, int k, float *x_out_host,
                                double *resid_hist, const ct_solve_opts *opts, int *iters_done, void *stream)
{
    NvtxRange call_range("ct_bagmres_solve_host");
    ct_solve_opts o = resolve_opts(opts);
    ct_status rc = check_common(geom, b_host, k, x_out_host, &o);
    if (rc != CT_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t mb = geom->m * sizeof(float), nb = geom->n * sizeof(float);
    void *bd = nullptr, *xd = nullptr;
    cudaError_t e = cudaMallocAsync(&bd, mb, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&xd, nb, s);
    if (e != cudaSuccess) {
        if (bd) cudaFreeAsync(bd, s);
        cudaGetLastError();
        return set_error(CT_ENOMEM, "ct_bagmres_solve_host: device buffers of %zu + %zu bytes: %s", mb, nb,
                         cudaGetErrorString(e));
    }
    e = cudaMemcpyAsync(bd, b_host, mb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        rc = bagmres(geom, static_cast<const float *>(bd), k, static_cast<float *>(xd), resid_hist, o, iters_done, s);
        if (rc == CT_OK || rc == CT_BREAKDOWN_LUCKY) {
            e = cudaMemcpyAsync(x_out_host, xd, nb, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        }
    }
    cudaFreeAsync(xd, s);
    cudaFreeAsync(bd, s);
    if (e != cudaSuccess) return cuda_error(e, "ct_bagmres_solve_host copy");
    return rc;
}

ct_status ct_bagmres_solve_err(const ct_geom *geom, const float *b_dev, int k, float *x_out_dev,
                               const float *x_ref_dev, double *resid_hist, double *err_hist,
                               const ct_solve_opts *opts, int *iters_done, void *stream)
{
    NvtxRange call_range("ct_bagmres_solve_err");
    ct_solve_opts o = resolve_opts(opts);
    ct_status rc = check_common(geom, b_dev, k, x_out_dev, &o);
    if (rc != CT_OK) return rc;
    if (!x_ref_dev || !err_hist) return set_error(CT_EINVAL, "ct_bagmres_solve_err: NULL x_ref or err_hist");
    return bagmres(geom, b_dev, k, x_out_dev, resid_hist, o, iters_done, static_cast<cudaStream_t>(stream),
                   x_ref_dev, err_hist);
}

ct_status ct_bagmres_restarted(const ct_geom *geom, const float *b_dev, int m, int cycles, float *x_out_dev,
                               double *resid_hist, const ct_solve_opts *opts, int *iters_done, void *stream)
{
    NvtxRange call_range("ct_bagmres_restarted");
    ct_solve_opts o = resolve_opts(opts);
    ct_status rc = check_common(geom, b_dev, m, x_out_dev, &o);
    if (rc != CT_OK) return rc;
    if (cycles < 1 || size_t(m) * cycles > 1u << 20)
        return set_error(CT_EINVAL, "ct_bagmres_restarted: cycles must be >= 1 and m * cycles <= 2^20");
    return bagmres_restarted(geom, b_dev, m, cycles, x_out_dev, resid_hist, o, iters_done,
                             static_cast<cudaStream_t>(stream));
}

ct_status ct_abgmres_solve(const ct_geom *geom, const float *b_dev, int k, float *x_out_dev,
                           double *resid_hist, const ct_solve_opts *opts, int *iters_done, void *stream)
{
    NvtxRange call_range("ct_abgmres_solve");
    ct_solve_opts o = resolve_opts(opts);
    ct_status rc = check_common(geom, b_dev, k, x_out_dev, &o);
    if (rc != CT_OK) return rc;
    return abgmres(geom, b_dev, k, x_out_dev, resid_hist, o, iters_done, static_cast<cudaStream_t>(stream));
}

ct_status ct_cgls_solve(const ct_geom *geom, const float *b_dev, int k, float *x_out_dev,
                        double *resid_hist, const ct_solve_opts *opts, int *iters_done, void *stream)
{
    NvtxRange call_range("ct_cgls_solve");
    ct_solve_opts o = resolve_opts(opts);
    ct_status rc = check_common(geom, b_dev, k, x_out_dev, &o);
    if (rc != CT_OK) return rc;
    return cgls(geom, b_dev, k, x_out_dev, resid_hist, o, iters_done, static_cast<cudaStream_t>(stream));
}

ct_status ct_bagmres_vjp(const ct_geom *geom, const float *gx_dev, int k, float *gb_dev, double *resid_hist,
                         const ct_solve_opts *opts, int *iters_done, void *stream)
{
    NvtxRange call_range("ct_bagmres_vjp");
    ct_solve_opts o = resolve_opts(opts);
    if (!geom || !gx_dev || !gb_dev) return set_error(CT_EINVAL, "ct_bagmres_vjp: NULL argument");
    if (k < 1 || k > 4096) return set_error(CT_EINVAL, "ct_bagmres_vjp: k must be in [1, 4096] (got %d)", k);
    if (o.dot_mode != 0 && o.dot_mode != 1) return set_error(CT_EINVAL, "ct_bagmres_vjp: dot_mode must be 0 or 1");
    if (!(o.tol >= 0.0)) return set_error(CT_EINVAL, "ct_bagmres_vjp: tol must be >= 0");
    return bagmres_vjp(geom, gx_dev, k, gb_dev, resid_hist, o, iters_done, static_cast<cudaStream_t>(stream));
}

ct_status ct_bagmres_state_create(const ct_geom *geom, int kmax, int basis, const ct_solve_opts *opts,
                                  ct_gmres_state **out)
{
    NvtxRange call_range("ct_bagmres_state_create");
    if (out) *out = nullptr;
    if (!geom || !out) return set_error(CT_EINVAL, "ct_bagmres_state_create: NULL argument");
    if (kmax < 1 || kmax > 4096)
        return set_error(CT_EINVAL, "ct_bagmres_state_create: kmax must be in 1..4096 (got %d)", kmax);
    if (basis != CT_BASIS_DEVICE && basis != CT_BASIS_HOST)
        return set_error(CT_EINVAL, "ct_bagmres_state_create: unknown basis location %d", basis);
    ct_solve_opts o = resolve_opts(opts);
    if (o.b_kind != CT_B_UN && o.b_kind != CT_B_FBP && o.b_kind != CT_B_AT)
        return set_error(CT_EINVAL, "ct_bagmres_state_create: unknown b_kind %d", o.b_kind);
    if (o.dot_mode != 0 && o.dot_mode != 1)
        return set_error(CT_EINVAL, "ct_bagmres_state_create: dot_mode must be 0 or 1");
    ct_status rc = state_check_device(geom, "ct_bagmres_state_create");
    if (rc != CT_OK) return rc;
    return state_alloc(geom, kmax, basis, o, out);
}

void ct_gmres_state_destroy(ct_gmres_state *state)
{
    if (!state) return;
    cudaDeviceSynchronize();   // no kernel of the state may still run
    state_free(state);
}

int ct_gmres_state_iters(const ct_gmres_state *state) { return state ? state->k_done : -1; }

size_t ct_gmres_state_basis_bytes(const ct_geom *geom, int kmax)
{
    if (!geom || kmax < 1) return 0;
    return basis_bytes(geom->g, kmax, false);
}

ct_status ct_bagmres_state_start(ct_gmres_state *state, const float *b_dev, void *stream)
{
    NvtxRange call_range("ct_bagmres_state_start");
    if (!state || !b_dev) return set_error(CT_EINVAL, "ct_bagmres_state_start: NULL argument");
    ct_status rc = state_check_device(state->geom, "ct_bagmres_state_start");
    if (rc != CT_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = ba_start(state->geom->g, state->w, b_dev, state->kmax, state->geom->n, state->o, s);
    if (e != cudaSuccess) return cuda_error(e, "ct_bagmres_state_start launch");
    state->started = 1;
    state->k_done = 0;
    state->status = ST_RUN;
    return CT_OK;
}

ct_status ct_bagmres_state_extend(ct_gmres_state *state, int k, float *x_out_dev, double *resid_hist,
                                  int *iters_done, void *stream)
{
    NvtxRange call_range("ct_bagmres_state_extend");
    if (!state || !x_out_dev) return set_error(CT_EINVAL, "ct_bagmres_state_extend: NULL argument");
    if (!state->started) return set_error(CT_EINVAL, "ct_bagmres_state_extend: the state has not been started");
    if (k < 1 || k > state->kmax)
        return set_error(CT_EINVAL, "ct_bagmres_state_extend: k must be in 1..%d (the state's kmax), got %d",
                         state->kmax, k);
    ct_status rc = state_check_device(state->geom, "ct_bagmres_state_extend");
    if (rc != CT_OK) return rc;
    const GeomDev &g = state->geom->g;
    const size_t n = state->geom->n;
    GmresWs &w = state->w;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    Stager *sg = state->basis == CT_BASIS_HOST ? &state->stager : nullptr;
    if (state->status == ST_RUN)
        for (int j = state->k_done; j < k && e == cudaSuccess; ++j)
            e = ba_iteration(g, w, j, state->kmax, n, state->o, s, sg);
    // x = V_c y_c with c = min(k, iterations done)
    if (e == cudaSuccess) {
        ProfScope prof(PK_SMALL, s);
        iterate_upto_kernel<<<1, 1, 0, s>>>(w.st, k, w.cnt);
        backsolve_count_kernel<<<1, 1, 0, s>>>(w.R, w.g, w.y, w.cnt, state->kmax);
        e = cudaGetLastError();
    }
    SolverState hst;
    std::vector<double> hres(size_t(k) + 1);
    if (e == cudaSuccess && sg) {
        // a staged basis streams exactly the vectors the iterate needs: learn
        // how many first
        e = cudaMemcpyAsync(&hst, w.st, sizeof(SolverState), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = staged_combine(*sg, w.vbf16, hst.iters < k ? hst.iters : k, w.y, n, x_out_dev, s);
    } else if (e == cudaSuccess) {
        e = w.vbf16 ? combine_t(static_cast<const __nv_bfloat16 *>(w.V), w.ldv, state->kmax, n, w.y, w.cnt,
                                x_out_dev, s)
                    : combine(static_cast<const float *>(w.V), w.ldv, state->kmax, n, w.y, w.cnt, x_out_dev, s);
    }
    if (e != cudaSuccess) return cuda_error(e, "ct_bagmres_state_extend launch");
    CT_CUDA(cudaMemcpyAsync(&hst, w.st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
    CT_CUDA(cudaMemcpyAsync(hres.data(), w.resid, sizeof(double) * (k + 1), cudaMemcpyDeviceToHost, s));
    CT_CUDA(cudaStreamSynchronize(s));
    if (sg) CT_CUDA(cudaStreamSynchronize(sg->cs));   // the host basis holds every vector on return
    state->k_done = hst.iters;
    state->status = hst.status;
    if (resid_hist) std::copy(hres.begin(), hres.end(), resid_hist);
    if (iters_done) *iters_done = hst.iters < k ? hst.iters : k;
    if (hst.status == ST_NONFINITE)
        return set_error(CT_ENONFINITE, "ct_bagmres_state_extend: a norm became NaN/Inf after %d iterations",
                         hst.iters);
    if (hst.status == ST_LUCKY) return CT_BREAKDOWN_LUCKY;
    return CT_OK;
}

ct_status ct_gmres_state_save(const ct_gmres_state *state, const char *path, void *stream)
{
    NvtxRange call_range("ct_gmres_state_save");
    if (!state || !path) return set_error(CT_EINVAL, "ct_gmres_state_save: NULL argument");
    if (!state->started) return set_error(CT_EINVAL, "ct_gmres_state_save: the state has not been started");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const GmresWs &w = state->w;
    const size_t n = state->geom->n;
    const int kd = state->k_done;
    const size_t ld = size_t(state->kmax) + 1;
    StateFileHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, "CTGMRS01", 8);
    h.version = 1;
    h.vbf16 = w.vbf16 ? 1 : 0;
    h.desc = state->geom->desc;
    h.b_kind = state->o.b_kind;
    h.dot_mode = state->o.dot_mode;
    h.reorth = state->o.reorth;
    h.k_done = kd;
    h.n = n;
    CT_CUDA(cudaStreamSynchronize(s));
    if (state->stager.cs) CT_CUDA(cudaStreamSynchronize(state->stager.cs));
    CT_CUDA(cudaMemcpy(&h.st, w.st, sizeof(SolverState), cudaMemcpyDeviceToHost));
    if (h.st.iters != kd) return set_error(CT_EINVAL, "ct_gmres_state_save: the state changed since its last call");
    // the first kd columns of H and R (rows 0..kd), cs, sn, g and resid (kd + 1)
    const size_t rows = size_t(kd) + 1;
    std::vector<double> H(rows * kd), R(rows * kd), cs(kd), sn(kd), gv(rows), res(rows);
    for (int j = 0; j < kd; ++j) {
        CT_CUDA(cudaMemcpy(H.data() + j * rows, w.H + j * ld, rows * sizeof(double), cudaMemcpyDeviceToHost));
        CT_CUDA(cudaMemcpy(R.data() + j * rows, w.R + j * ld, rows * sizeof(double), cudaMemcpyDeviceToHost));
    }
    if (kd > 0) {
        CT_CUDA(cudaMemcpy(cs.data(), w.cs, kd * sizeof(double), cudaMemcpyDeviceToHost));
        CT_CUDA(cudaMemcpy(sn.data(), w.sn, kd * sizeof(double), cudaMemcpyDeviceToHost));
    }
    CT_CUDA(cudaMemcpy(gv.data(), w.g, rows * sizeof(double), cudaMemcpyDeviceToHost));
    CT_CUDA(cudaMemcpy(res.data(), w.resid, rows * sizeof(double), cudaMemcpyDeviceToHost));
    std::vector<float> q(n);
    CT_CUDA(cudaMemcpy(q.data(), w.q, n * sizeof(float), cudaMemcpyDeviceToHost));
    FILE *f = std::fopen(path, "wb");
    if (!f) return set_error(CT_EINVAL, "ct_gmres_state_save: cannot open %s for writing", path);
    bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1;
    auto put = [&](const void *p, size_t bytes) { ok = ok && (bytes == 0 || std::fwrite(p, bytes, 1, f) == 1); };
    put(H.data(), H.size() * sizeof(double));
    put(R.data(), R.size() * sizeof(double));
    put(cs.data(), cs.size() * sizeof(double));
    put(sn.data(), sn.size() * sizeof(double));
    put(gv.data(), gv.size() * sizeof(double));
    put(res.data(), res.size() * sizeof(double));
    put(q.data(), n * sizeof(float));
    // the kd basis vectors, one at a time
    const size_t esz = w.vbf16 ? 2 : 4;
    std::vector<char> vbuf(n * esz);
    for (int i = 0; i < kd && ok; ++i) {
        cudaError_t e = cudaMemcpy(vbuf.data(), w.vec(i), n * esz, cudaMemcpyDefault);
        if (e != cudaSuccess) {
            std::fclose(f);
            return cuda_error(e, "ct_gmres_state_save: basis copy");
        }
        put(vbuf.data(), n * esz);
    }
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return set_error(CT_EINVAL, "ct_gmres_state_save: writing %s failed", path);
    return CT_OK;
}

ct_status ct_gmres_state_load(const ct_geom *geom, const char *path, int kmax, int basis, ct_gmres_state **out,
                              void *stream)
{
    NvtxRange call_range("ct_gmres_state_load");
    if (out) *out = nullptr;
    if (!geom || !path || !out) return set_error(CT_EINVAL, "ct_gmres_state_load: NULL argument");
    if (basis != CT_BASIS_DEVICE && basis != CT_BASIS_HOST)
        return set_error(CT_EINVAL, "ct_gmres_state_load: unknown basis location %d", basis);
    ct_status rc = state_check_device(geom, "ct_gmres_state_load");
    if (rc != CT_OK) return rc;
    FILE *f = std::fopen(path, "rb");
    if (!f) return set_error(CT_EINVAL, "ct_gmres_state_load: cannot open %s", path);
    StateFileHeader h;
    bool ok = std::fread(&h, sizeof(h), 1, f) == 1;
    const size_t n = geom->n;
    if (!ok || std::memcmp(h.magic, "CTGMRS01", 8) != 0 || h.version != 1) {
        std::fclose(f);
        return set_error(CT_EINVAL, "ct_gmres_state_load: %s is not a saved solver state", path);
    }
    if (!same_desc(h.desc, geom->desc) || h.n != n || h.vbf16 != (geom->g.vol_bf16 ? 1 : 0)) {
        std::fclose(f);
        return set_error(CT_EINVAL, "ct_gmres_state_load: %s belongs to another geometry", path);
    }
    const int kd = h.k_done;
    if (kd < 0 || kd > 4096 || kmax < kd || kmax < 1 || kmax > 4096) {
        std::fclose(f);
        return set_error(CT_EINVAL, "ct_gmres_state_load: kmax %d must be in %d..4096 (the iterations saved)",
                         kmax, kd > 1 ? kd : 1);
    }
    ct_solve_opts o;
    ct_solve_opts_default(&o);
    o.b_kind = h.b_kind;
    o.dot_mode = h.dot_mode;
    o.reorth = h.reorth;
    ct_gmres_state *st = nullptr;
    rc = state_alloc(geom, kmax, basis, o, &st);
    if (rc != CT_OK) {
        std::fclose(f);
        return rc;
    }
    const size_t rows = size_t(kd) + 1, ld = size_t(kmax) + 1;
    std::vector<double> H(rows * kd), R(rows * kd), cs(kd), sn(kd), gv(rows), res(rows);
    auto get = [&](void *p, size_t bytes) { ok = ok && (bytes == 0 || std::fread(p, bytes, 1, f) == 1); };
    get(H.data(), H.size() * sizeof(double));
    get(R.data(), R.size() * sizeof(double));
    get(cs.data(), cs.size() * sizeof(double));
    get(sn.data(), sn.size() * sizeof(double));
    get(gv.data(), gv.size() * sizeof(double));
    get(res.data(), res.size() * sizeof(double));
    std::vector<float> q(n);
    get(q.data(), n * sizeof(float));
    GmresWs &w = st->w;
    cudaError_t e = cudaSuccess;
    // H, R, g zero beyond what was saved; resid -1 after the iterations done
    std::vector<double> res_full(ld, -1.0);
    std::copy(res.begin(), res.end(), res_full.begin());
    e = cudaMemset(w.H, 0, sizeof(double) * ld * kmax);
    if (e == cudaSuccess) e = cudaMemset(w.R, 0, sizeof(double) * ld * kmax);
    if (e == cudaSuccess) e = cudaMemset(w.g, 0, sizeof(double) * ld);
    if (e == cudaSuccess) e = cudaMemset(w.ob.ypad, 0, padded_sino_floats(geom->g) * sizeof(float));
    for (int j = 0; j < kd && e == cudaSuccess; ++j) {
        e = cudaMemcpy(w.H + j * ld, H.data() + j * rows, rows * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(w.R + j * ld, R.data() + j * rows, rows * sizeof(double), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && kd > 0) e = cudaMemcpy(w.cs, cs.data(), kd * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && kd > 0) e = cudaMemcpy(w.sn, sn.data(), kd * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w.g, gv.data(), rows * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w.resid, res_full.data(), ld * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w.q, q.data(), n * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w.st, &h.st, sizeof(SolverState), cudaMemcpyHostToDevice);
    const size_t esz = w.vbf16 ? 2 : 4;
    std::vector<char> vbuf(n * esz);
    for (int i = 0; i < kd && ok && e == cudaSuccess; ++i) {
        get(vbuf.data(), n * esz);
        if (ok) e = cudaMemcpy(w.vec(i), vbuf.data(), n * esz, cudaMemcpyDefault);
    }
    std::fclose(f);
    if (e == cudaSuccess) e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (!ok || e != cudaSuccess) {
        state_free(st);
        if (e != cudaSuccess) return cuda_error(e, "ct_gmres_state_load: upload");
        return set_error(CT_EINVAL, "ct_gmres_state_load: %s is truncated", path);
    }
    st->started = 1;
    st->k_done = kd;
    st->status = h.st.status;
    *out = st;
    return CT_OK;
}

ct_status ct_mgs_sweep(const float *V_dev, size_t ldv, int j, size_t len, float *q_dev, double *h_dev,
                       int dot_mode, void *stream)
{
    NvtxRange call_range("ct_mgs_sweep");
    if (!q_dev || !h_dev || (j > 0 && !V_dev)) return set_error(CT_EINVAL, "ct_mgs_sweep: NULL argument");
    if (j < 0 || len == 0 || (j > 0 && ldv < len))
        return set_error(CT_EINVAL, "ct_mgs_sweep: bad sizes (j=%d len=%zu ldv=%zu)", j, len, ldv);
    if (dot_mode != 0 && dot_mode != 1) return set_error(CT_EINVAL, "ct_mgs_sweep: dot_mode must be 0 or 1");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Arena ar;
    const size_t bytes = Arena::align(partials_count() * sizeof(double)) + Arena::align(sizeof(unsigned));
    ct_status rc = arena_open(ar, bytes, nullptr, 0, s);
    if (rc != CT_OK) return rc;
    double *partials = ar.take<double>(partials_count());
    unsigned *ctr = ar.take<unsigned>(1);
    cudaError_t e = cudaMemsetAsync(ctr, 0, sizeof(unsigned), s);
    for (int i = 0; i <= j && e == cudaSuccess; ++i) {
        const float *vprev = i > 0 ? V_dev + size_t(i - 1) * ldv : nullptr;
        const double *hprev = i > 0 ? h_dev + (i - 1) : nullptr;
        const float *vcur = i < j ? V_dev + size_t(i) * ldv : nullptr;
        double *odot = i < j ? h_dev + i : nullptr;
        double *oss = i == j ? h_dev + j : nullptr;
        e = mgs_pass(dot_mode, q_dev, vprev, hprev, vcur, len, partials, ctr, odot, oss, nullptr, nullptr, s);
    }
    // h[j] = sqrt(||q||^2)
    if (e == cudaSuccess) {
        { ProfScope prof(PK_SMALL, s); sqrt_inplace_kernel<<<1, 1, 0, s>>>(h_dev + j); }
        e = cudaGetLastError();
    }
    arena_close(ar);
    if (e != cudaSuccess) return cuda_error(e, "ct_mgs_sweep launch");
    return CT_OK;
}

ct_status ct_basis_combine(const float *V_dev, size_t ldv, int k, size_t len, const double *y_dev,
                           float *x_dev, void *stream)
{
    NvtxRange call_range("ct_basis_combine");
    if (!V_dev || !y_dev || !x_dev) return set_error(CT_EINVAL, "ct_basis_combine: NULL argument");
    if (k < 1 || len == 0 || ldv < len) return set_error(CT_EINVAL, "ct_basis_combine: bad sizes");
    if (k > 4096) return set_error(CT_EINVAL, "ct_basis_combine: k must be <= 4096");
    cudaError_t e = combine(V_dev, ldv, k, len, y_dev, nullptr, x_dev, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_error(e, "ct_basis_combine launch");
    return CT_OK;
}

}  // extern "C"
