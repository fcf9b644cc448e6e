/*
 * ct.h -- C-ABI of libct, the GB300 (sm_103a) CUDA library for CT
 * reconstruction with an unmatched projector/back-projector pair by
 * BA-GMRES and AB-GMRES (Sidky, Hansen, Jorgensen & Pan, arXiv 2201.07408).
 *
 * Model (Sec. I, Eq. 1): A x = b, A is m x n (m detector readings, n voxels).
 * Square systems solved by GMRES (Sec. II): B A x = B b (Eq. 5, BA-GMRES) and
 * A B y = b, x = B y (Eq. 4, AB-GMRES), from a zero initial vector; CGLS
 * (Eqs. 2-3) for comparison.
 *
 * Conventions shared by every entry point
 *   - Vectors are caller-owned, contiguous DEVICE buffers on the device that
 *     was current when the geometry was created.  Volumes are vol[z][y][x]
 *     (x fastest, n = nx*ny*nz elements); sinograms are sino[view][v][u]
 *     (u fastest, m = n_views*nv*nu elements).  Element type: float (FP32).
 *     A buffer may not alias another buffer of the same call.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Operator
 *     calls are asynchronous and stream-ordered; solver calls return after
 *     their result and residual history are complete (they synchronise the
 *     stream once at the end).
 *   - Scratch memory: operator calls and solvers take their temporary device
 *     memory from the stream-ordered allocator (cudaMallocAsync on `stream`)
 *     and release it before returning, unless the solver options supply a
 *     workspace.
 *   - Errors: every call returns a ct_status; on failure the outputs are
 *     unspecified (except CT_BREAKDOWN_LUCKY, whose outputs are valid) and
 *     ct_last_error() gives a message for the calling thread.  No call
 *     aborts the process.
 *
 * Geometry (lengths in mm, angles in radians): voxel (i,j,k) centre is
 * ((i-(nx-1)/2) vox, (j-(ny-1)/2) vox, (k-(nz-1)/2) vox); view s is at angle
 * theta_s = angle_start + s*angle_span/n_views.  Cone beam: source at
 * sod (cos, sin, 0), flat detector at distance sdd from the source with
 * axes e_u = (-sin, cos, 0), e_v = (0, 0, 1); pixel (iu, iv) centre at
 * u = (iu-(nu-1)/2) du, v = (iv-(nv-1)/2) dv.  2D parallel beam (nz = nv = 1):
 * ray iu is the line u e_u + t e_d, e_u = (cos, sin), e_d = (-sin, cos).
 */
#ifndef CT_H
#define CT_H

#include <stddef.h>

#if defined(__GNUC__)
#define CT_API __attribute__((visibility("default")))
#else
#define CT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CT_OK = 0,
    CT_EINVAL = 1,          /* invalid argument (sizes, pointers, options) */
    CT_ENOMEM = 2,          /* device allocation or workspace too small */
    CT_ECUDA = 3,           /* a CUDA runtime call failed */
    CT_ENONFINITE = 4,      /* a norm became NaN/Inf during a solve */
    CT_ETIMEOUT = 5,        /* a bounded device wait gave up */
    CT_BREAKDOWN_LUCKY = 6  /* informational: the Krylov space became invariant;
                               the returned iterate is valid: it minimises
                               the residual over that space, which solves the
                               system exactly unless the operator is singular
                               on it (then resid_hist[iters_done] > 0 shows
                               the residual that remains) */
} ct_status;

typedef enum { CT_PARALLEL_2D = 0, CT_CONE_3D = 1 } ct_geom_kind;

typedef enum { CT_F32 = 0, CT_BF16 = 1 } ct_dtype;

/* Which discretisation the projector A uses (Sec. III). */
typedef enum {
    CT_PROJ_JOSEPH = 0,  /* Joseph: one bilinear sample per voxel-centre plane (default) */
    CT_PROJ_SIDDON = 1   /* line intersection: the length of the ray inside each voxel */
} ct_projector;

/* Which back-projector B a call uses (Sec. III). */
typedef enum {
    CT_B_UN = 0,   /* B_un: voxel-driven back-projection, bilinear detector interpolation */
    CT_B_FBP = 1,  /* B_FBP = B_un F: ramp-filtered (FDK-weighted) back-projection */
    CT_B_AT = 2    /* the exact transpose A^T (matched pair; CGLS reference) */
} ct_b_kind;

typedef enum { CT_SOLVER_BA = 0, CT_SOLVER_AB = 1, CT_SOLVER_CGLS = 2, CT_SOLVER_BA_VJP = 3 } ct_solver;

typedef struct {
    int kind;                  /* ct_geom_kind */
    int nx, ny, nz;            /* voxels; 2D parallel beam needs nz = 1 */
    double voxel_mm;           /* voxel edge */
    int n_views;
    double angle_start_rad;    /* theta_0 */
    double angle_span_rad;     /* views at theta_0 + s*span/n_views */
    int nu, nv;                /* detector pixels; 2D parallel beam needs nv = 1 */
    double du_mm, dv_mm;       /* pixel pitch */
    double sod_mm, sdd_mm;     /* source-axis and source-detector distances (cone only) */
    int vol_dtype;             /* storage of the projector's working copies of the volume and of
                                  the BA-GMRES Krylov basis: CT_F32 or CT_BF16 */
    int sino_dtype;            /* storage of the back-projector's working sinogram: CT_F32 or
                                  CT_BF16.  Arithmetic is FP32 (FP64 for the least squares) and
                                  caller buffers are FP32 whatever the storage. */
    int projector;             /* ct_projector: the A (and A^T) of every call on this geometry */
} ct_geom_desc;

typedef struct ct_geom ct_geom;

typedef struct {
    int b_kind;              /* ct_b_kind; default CT_B_UN */
    double tol;              /* stop when resid[j] <= tol*resid[0]; 0 = run all k */
    int dot_mode;            /* Arnoldi inner products: 0 = compensated FP32 accumulation (FMA
                                two-product + two-sum) then FP64 reduction (default),
                                1 = plain FP32 FMA accumulation then FP64 reduction */
    int reorth;              /* 0 = one MGS sweep (default), 1 = a second sweep when the
                                norm drops below 1/sqrt(2) of its value before the sweep */
    int record_data_resid;   /* CGLS only: resid holds the recomputed ||b - A x_j|| */
    void *workspace;         /* optional caller device buffer (NULL = library allocates) */
    size_t workspace_bytes;  /* its size; must be >= ct_workspace_bytes(...) */
} ct_solve_opts;

/* Fills `opts` with the defaults listed above. */
CT_API void ct_solve_opts_default(ct_solve_opts *opts);

/* Creates a geometry handle on the current device: validates the
 * description (positive sizes, 2D needs nz = nv = 1, cone needs
 * sdd > sod > 0 and the volume inside the source circle) and
 * uploads per-view tables; storage dtypes CT_F32 or CT_BF16.  The library owns the handle; free it with
 * ct_geom_destroy.  Returns CT_EINVAL or CT_ECUDA on failure (*out = NULL). */
CT_API ct_status ct_geom_create(const ct_geom_desc *desc, ct_geom **out);

/* Frees the handle and its device tables (NULL is a no-op). */
CT_API void ct_geom_destroy(ct_geom *geom);

/* Number of voxels n and of detector readings m of a geometry. */
CT_API size_t ct_geom_n(const ct_geom *geom);
CT_API size_t ct_geom_m(const ct_geom *geom);

/* y = A x: ray-driven projector (Sec. I Eq. 1; Sec. III "ray-driven
 * cone-beam projector").  CT_PROJ_JOSEPH: for each ray, one bilinear
 * sample on every voxel-centre plane of the ray's dominant axis (x when
 * |d_x| >= |d_y|), neighbours outside the grid count as zero, sum times the
 * step vox*|d|/|d_a|.  CT_PROJ_SIDDON: the sum over the voxels the ray
 * crosses of the voxel value times the length of the ray inside the voxel
 * (voxel (i,j,k) is the cube of edge vox around its centre), the
 * line-intersection method the paper names.  x: n floats, y: m floats
 * (overwritten). */
CT_API ct_status ct_project_A(const ct_geom *geom, const float *x_dev, float *y_dev, void *stream);

/* x = B y: back-projection (Sec. III).  b_kind CT_B_UN: voxel-driven
 * back-projection with bilinear detector interpolation, weight
 * vox^3 M^2/(du dv) (M = sdd/depth; 2D: vox^2/du).  CT_B_FBP: B_un F, F the
 * ramp filter (cosine weight, Ram-Lak row convolution, FBP scaling).
 * CT_B_AT: the exact transpose A^T.  y: m floats, x: n floats (overwritten). */
CT_API ct_status ct_backproject_B(const ct_geom *geom, const float *y_dev, float *x_dev, int b_kind,
                           void *stream);

/* x = A^T y: exact transpose of ct_project_A (normal equations, Sec. I
 * Eq. 3).  Scatter with FP32 atomics: the summation order varies between
 * runs.  y: m floats, x: n floats (overwritten). */
CT_API ct_status ct_adjoint_At(const ct_geom *geom, const float *y_dev, float *x_dev, void *stream);

/* y = B^T x: exact transpose of ct_backproject_B for b_kind CT_B_UN
 * (voxel splatting with the same bilinear weights) and CT_B_FBP
 * (F^T B_un^T); CT_B_AT gives A x.  FP32 atomics.  x: n, y: m (overwritten). */
CT_API ct_status ct_adjoint_Bt(const ct_geom *geom, const float *x_dev, float *y_dev, int b_kind,
                        void *stream);

/* yf = F y (transpose = 0) or yf = F^T y (transpose = 1): the ramp filter
 * of B_FBP = B_un F (Sec. III) on its own.  y, yf: m floats, distinct. */
CT_API ct_status ct_ramp_F(const ct_geom *geom, const float *y_dev, float *yf_dev, int transpose,
                    void *stream);

/* BA-GMRES (Sec. II, Eq. 5): k iterations on B A x = B b from x0 = 0, with
 * the Krylov basis (k+1 image-space vectors, FP32) held on the device,
 * modified Gram-Schmidt Arnoldi, FP64 Givens least squares.
 *   b_dev:      m floats (data).
 *   k:          iteration count >= 1 (the method's only parameter, Sec. I).
 *   x_out_dev:  n floats, the iterate x_j after the last iteration done.
 *   resid_hist: HOST array of k+1 doubles: resid[0] = ||B b||,
 *               resid[j] = ||B b - B A x_j|| (non-increasing); entries after
 *               the last iteration done are set to -1.  May be NULL.
 *   opts:       NULL = defaults.
 *   iters_done: iterations performed (< k after a tolerance stop or a lucky
 *               breakdown).  May be NULL.
 * Returns CT_BREAKDOWN_LUCKY (solution valid, see ct_status) when the Krylov
 * space became invariant, CT_ENONFINITE when a norm was NaN/Inf. */
CT_API ct_status ct_bagmres_solve(const ct_geom *geom, const float *b_dev, int k, float *x_out_dev,
                           double *resid_hist, const ct_solve_opts *opts, int *iters_done,
                           void *stream);

/* ct_bagmres_solve with the data and the image in HOST memory: b_host (m
 * floats) is copied to the device, the solve runs as ct_bagmres_solve, and
 * x_k is copied back into x_out_host (n floats) before the call returns.
 * The two device vectors are taken from the stream-ordered allocator
 * (cudaMallocAsync) on `stream` and freed before return; the workspace is
 * as for ct_bagmres_solve.  Page-locked host buffers give asynchronous
 * copies; pageable ones work too.  Synchronous: on return x_out_host and
 * resid_hist hold the result.  Returns CT_ENOMEM when the device vectors
 * cannot be allocated; other codes as ct_bagmres_solve. */
CT_API ct_status ct_bagmres_solve_host(const ct_geom *geom, const float *b_host, int k, float *x_out_host,
                                       double *resid_hist, const ct_solve_opts *opts, int *iters_done,
                                       void *stream);

/* ct_bagmres_solve that also measures the image error of every iterate:
 * err_hist[j] = ||x_j - x_ref|| for j = 0..k (err_hist[0] = ||x_ref||,
 * since x_0 = 0); entries after the last iteration done are -1.  The
 * paper's semi-convergence curves (Sec. III, Fig. 4: the image error falls,
 * reaches a minimum and rises again as the iterates fit the noise) are this
 * history against the true image.  After the solve each x_j = V_j y_j is
 * formed in x_out_dev from the first j basis vectors (one pass over them),
 * so the call costs about k(k+1)/2 extra basis-vector reads; x_out_dev
 * holds x_k on return.
 *   x_ref_dev: n floats (device).  err_hist: HOST array of k+1 doubles.
 * Other arguments and return codes as ct_bagmres_solve. */
CT_API ct_status ct_bagmres_solve_err(const ct_geom *geom, const float *b_dev, int k, float *x_out_dev,
                                      const float *x_ref_dev, double *resid_hist, double *err_hist,
                                      const ct_solve_opts *opts, int *iters_done, void *stream);

/* Restarted BA-GMRES(m) (Sec. II discusses restarting GMRES to bound the
 * basis): `cycles` cycles of m iterations.  Cycle c solves
 * B A dx = B (b - A x_c) from dx = 0 with m BA-GMRES iterations (the basis
 * holds m+1 vectors) and sets x_{c+1} = x_c + dx; x_0 = 0.
 *   resid_hist: HOST array of m*cycles + 1 doubles: resid[0] = ||B b||,
 *               then the m residuals ||B (b - A x)|| of each cycle in turn;
 *               -1 after the last iteration done.  May be NULL.
 *   iters_done: total iterations over all cycles.
 * opts->tol stops a cycle at tol times that cycle's starting residual and
 * stops the solve when the residual reaches tol times resid[0].  Scratch
 * (the projector's copies, two sinograms and one volume) comes from the
 * stream-ordered allocator; the workspace, when given, is as for
 * ct_bagmres_solve with k = m.  Synchronous.  Return codes as
 * ct_bagmres_solve; CT_EINVAL for cycles < 1. */
CT_API ct_status ct_bagmres_restarted(const ct_geom *geom, const float *b_dev, int m, int cycles,
                                      float *x_out_dev, double *resid_hist, const ct_solve_opts *opts,
                                      int *iters_done, void *stream);

/* AB-GMRES (Sec. II, Eq. 4): k iterations on A B y = b from y0 = 0 with the
 * basis in data space (k+1 sinogram-size vectors), x = B y.
 * resid[0] = ||b||, resid[j] = ||b - A x_j||.  Arguments as ct_bagmres_solve. */
CT_API ct_status ct_abgmres_solve(const ct_geom *geom, const float *b_dev, int k, float *x_out_dev,
                           double *resid_hist, const ct_solve_opts *opts, int *iters_done,
                           void *stream);

/* CGLS (Sec. I, Eqs. 2-3) with back-projector opts->b_kind in place of A^T
 * (CT_B_AT gives the textbook method; CT_B_UN shows the divergence of
 * Sec. III).  resid[j] = ||r_j|| of the recursively updated residual, or the
 * recomputed ||b - A x_j|| when opts->record_data_resid is set (one more A
 * per iteration).  Arguments as ct_bagmres_solve. */
CT_API ct_status ct_cgls_solve(const ct_geom *geom, const float *b_dev, int k, float *x_out_dev,
                        double *resid_hist, const ct_solve_opts *opts, int *iters_done,
                        void *stream);

/* Gradient through a converged BA-GMRES solve (Sec. II, Eq. 5):
 * x = (BA)^{-1} B b, so for a scalar loss L(x) with gx = dL/dx,
 * dL/db = B^T (BA)^{-T} gx = B^T z where (A^T B^T) z = gx.  z is found by k
 * iterations of GMRES on A^T B^T from z0 = 0 (or fewer, with opts->tol),
 * with a new image-space Krylov basis: the forward solve's basis is not
 * needed, so it need not be kept.  Each iteration applies B^T (voxel
 * splatting; F^T after it for CT_B_FBP) and A^T (ray scatter).
 *   gx_dev: n floats; gb_dev: m floats (output, dL/db).
 *   resid_hist: HOST k+1 doubles, ||gx - A^T B^T z_j|| (resid[0] = ||gx||).
 *   opts->b_kind: CT_B_UN or CT_B_FBP (the B of the forward solve).
 * Other arguments and return codes as ct_bagmres_solve. */
CT_API ct_status ct_bagmres_vjp(const ct_geom *geom, const float *gx_dev, int k, float *gb_dev,
                                double *resid_hist, const ct_solve_opts *opts, int *iters_done,
                                void *stream);

/* Device workspace in bytes that a solve with these arguments needs when
 * the caller supplies it through ct_solve_opts (solver: ct_solver). */
CT_API size_t ct_workspace_bytes(const ct_geom *geom, int k, int solver, const ct_solve_opts *opts);

/* One modified Gram-Schmidt sweep of the Arnoldi process (Sec. II: the
 * new Krylov vector is orthonormalised against the basis).  For
 * i = 0..j-1: h[i] = <q, V_i>; q -= h[i] V_i; then h[j] = ||q||.
 *   V_dev: j vectors of len floats, vector i at V_dev + i*ldv (ldv >= len).
 *   q_dev: len floats, updated in place (not normalised).
 *   h_dev: DEVICE array of j+1 doubles (output).
 * dot_mode as in ct_solve_opts.  Stream-ordered, asynchronous. */
CT_API ct_status ct_mgs_sweep(const float *V_dev, size_t ldv, int j, size_t len, float *q_dev,
                       double *h_dev, int dot_mode, void *stream);

/* x = sum_i y[i] V_i for i < k (the GMRES update x_k = V_k y_k, Sec. II).
 * y_dev: DEVICE array of k doubles.  Stream-ordered, asynchronous. */
CT_API ct_status ct_basis_combine(const float *V_dev, size_t ldv, int k, size_t len,
                           const double *y_dev, float *x_dev, void *stream);

/* Persistent BA-GMRES state: a solve whose workspace outlives the call, so
 * that it can be extended by more iterations, saved to a file and restored
 * later.  The paper stores the growing Krylov basis on disk and adds one
 * vector per iteration (Sec. II); here the basis stays in device memory, or
 * in page-locked host memory (CT_BASIS_HOST) for bases larger than the
 * device memory left free: the newest vector is copied out by the copy
 * engine while the operators run, and every Gram-Schmidt sweep streams the
 * older ones back through a ring of three device buffers (four basis vectors
 * of device memory in all).  Iterating a state k times gives bit for bit the
 * image and residual history of ct_bagmres_solve with k iterations and the
 * same options, however the k iterations are split over calls, saved and
 * restored.  opts->tol is ignored (a state runs the iterations it is asked
 * for); opts->workspace is ignored (the state allocates its own memory with
 * cudaMalloc, and cudaHostAlloc for a host basis).  A state belongs to its
 * geometry (which must outlive it) and to the device that was current when
 * it was made; it is not safe for concurrent use. */
typedef struct ct_gmres_state ct_gmres_state;
typedef enum { CT_BASIS_DEVICE = 0, CT_BASIS_HOST = 1 } ct_basis_location;

/* Allocates a state for up to kmax iterations (1..4096) of BA-GMRES on
 * `geom` with opts->b_kind, dot_mode and reorth (NULL = defaults), its basis
 * of kmax+1 image vectors at `basis`.  CT_ENOMEM when an allocation fails. */
CT_API ct_status ct_bagmres_state_create(const ct_geom *geom, int kmax, int basis, const ct_solve_opts *opts,
                                         ct_gmres_state **out);

/* Starts (or restarts) the solve from x0 = 0 with data b_dev (m floats):
 * r0 = B b, resid[0] = ||B b||.  Stream-ordered, asynchronous. */
CT_API ct_status ct_bagmres_state_start(ct_gmres_state *state, const float *b_dev, void *stream);

/* Runs the iterations from the state's current count up to k (1 <= k <=
 * kmax; none when k is not above the count) and writes x_k = V_k y_k to
 * x_out_dev (n floats); with k below the count it forms the earlier iterate
 * x_k from the first k basis vectors.  resid_hist: HOST array of k+1
 * doubles, as in ct_bagmres_solve (may be NULL).  iters_done: the index of
 * the iterate written (k, or fewer after a lucky breakdown).  Synchronous.
 * Return codes as ct_bagmres_solve. */
CT_API ct_status ct_bagmres_state_extend(ct_gmres_state *state, int k, float *x_out_dev, double *resid_hist,
                                         int *iters_done, void *stream);

/* Iterations done by the state as of its last synchronous call (-1 for NULL). */
CT_API int ct_gmres_state_iters(const ct_gmres_state *state);

/* Bytes of the basis of a state with capacity kmax on `geom`. */
CT_API size_t ct_gmres_state_basis_bytes(const ct_geom *geom, int kmax);

/* Writes the state (the basis vectors of the iterations done, the Hessenberg
 * and rotated columns, the rotations, g, the residual history, the pending
 * Krylov vector, the device status and the geometry description) to `path`
 * in a binary file that ct_gmres_state_load reads on any machine of the same
 * byte order.  Waits for `stream` first.  CT_EINVAL when the file cannot be
 * written or the state was never started. */
CT_API ct_status ct_gmres_state_save(const ct_gmres_state *state, const char *path, void *stream);

/* Restores a saved state into a new one of capacity kmax (>= the iterations
 * saved) with its basis at `basis`.  The geometry must equal the saved one
 * (CT_EINVAL otherwise).  Synchronous. */
CT_API ct_status ct_gmres_state_load(const ct_geom *geom, const char *path, int kmax, int basis,
                                     ct_gmres_state **out, void *stream);

/* Frees the state (waits for the device first).  NULL is a no-op. */
CT_API void ct_gmres_state_destroy(ct_gmres_state *state);

/* Size in bytes of the fixed device scratch of ct_project_A_noalloc. */
#define CT_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* y = A x exactly as ct_project_A, for callers that cannot allocate device
 * memory while they run: a TensorRT plugin inside enqueue(), a framework
 * that has reserved the whole device memory for its own pool, or a
 * real-time loop that must not pay for, or fail on, an allocation.  The
 * paper has no counterpart; this is a deployment variant of the projector.
 *   - Scratch: the projector's two zero-bordered plane-major copies of x
 *     live in a CT_NOALLOC_SCRATCH_BYTES (32 MiB) array that the library
 *     defines in device memory; every GPU that loads the library holds it
 *     until the process exits.  No cudaMalloc, cudaFree or other allocating
 *     call is made.
 *   - Limit: volumes whose copies need more than the array, about 155^3
 *     voxels for a cubic grid, are refused with CT_EINVAL and a message
 *     giving the bytes needed.
 *   - Set-up: the first call on a device looks up the array's device
 *     address (cudaGetSymbolAddress) with that device current; make that
 *     first call before any stream capture.  The geometry's device must be
 *     the current device.
 *   - Sharing: all calls use the same array.  Calls that can overlap on the
 *     GPU (other streams, other host threads) race on it; order them on one
 *     stream.  Each call rewrites all of the scratch it reads, so nothing
 *     carries over from the previous call.
 * Arguments and layouts as ct_project_A. */
CT_API ct_status ct_project_A_noalloc(const ct_geom *geom, const float *x_dev, float *y_dev,
                                      void *stream);

/* Per-kernel timing (no counterpart in the paper; instrumentation for
 * measurement).  ct_profile_enable(1) makes every kernel launch of the
 * library record a CUDA event pair on its stream; ct_profile_read waits for
 * the recorded pairs and writes, per kernel kind (index < the returned
 * count, names from ct_profile_kind_name), the accumulated device
 * milliseconds and launch counts since the last ct_profile_reset.  Either
 * output may be NULL.  Process-wide, thread-safe. */
CT_API void ct_profile_enable(int on);
CT_API void ct_profile_reset(void);
CT_API int ct_profile_read(double *ms_out, long long *launches_out, int max_kinds);
CT_API const char *ct_profile_kind_name(int kind);

/* Ceiling of the SM load path that the gather kernels (A, B) use: the best
 * of `repeats` timed launches (after one warm-up) of a kernel in which every
 * block reads its own 16 KiB window, resident in its SM's L1 after the
 * first pass, with 128-bit read-only loads (lanes on consecutive words),
 * over and over.  *gbs_out receives the bytes loaded per second / 1e9.
 * Instrumentation for the roofline (no counterpart in the paper).  Takes a
 * few MiB from the stream-ordered allocator on `stream`; synchronous.
 * CT_EINVAL for repeats < 1 or gbs_out NULL; CT_ECUDA on a CUDA failure. */
CT_API ct_status ct_measure_gather_peak(int repeats, double *gbs_out, void *stream);

/* Host-side fault injection, for testing the failure paths of a caller
 * without a GPU fault (no counterpart in the paper).  `spec` is a
 * comma-separated list of
 *   "nan_at_iter:N"  every later solve writes a NaN (an ordinary value, by a
 *                    one-thread kernel) into the new Krylov vector of
 *                    iteration N >= 1 (GMRES), or into q = A p (CGLS), so it
 *                    returns CT_ENONFINITE with iters_done = N - 1, the
 *                    residual history valid up to N - 1 and -1 after;
 *   "oom"            every later request to the stream-ordered allocator is
 *                    refused as if it had failed (CT_ENOMEM); calls given a
 *                    workspace, and ct_project_A_noalloc, still run;
 *   "none" or ""     (or spec NULL) clears the injection.
 * The environment variable CT_FAULT, read once when the library is loaded,
 * sets the initial spec (a malformed value is reported on stderr and
 * ignored).  Process-wide.  Returns CT_EINVAL, leaving the active spec
 * unchanged, for a malformed spec. */
CT_API ct_status ct_fault_set(const char *spec);

/* The active fault spec in canonical form ("" when none), valid until the
 * calling thread's next call. */
CT_API const char *ct_fault_get(void);

/* Index checks (checked builds).  The library built with -DCT_CHECK_BOUNDS
 * (libct_checked.so; libct.so is the regular build) tests, where each is
 * used, the margins and invariants that ct_geom_create derives from the
 * geometry and on which the gathers of A and B rely (no counterpart in the
 * paper; they guard the layouts of Sec. III's operators):
 *   site 1  A: a sample's two z rows lie inside the volume copy's zero border;
 *   site 2  A: the rays of a detector column move up at most one z row from
 *           ray to ray (the two-row window);
 *   site 3  A^T: the same for its row sums;
 *   site 4  B: a sample's quad row lies inside its view's padded rows (the
 *           row margin padv);
 *   site 5  B: a column's quad lies inside the padded row;
 *   site 6  A_S, A_S^T: the running voxel offset is the traversed voxel's.
 * A failed check redirects the access into range (it never leaves its
 * buffer), so the call's results are wrong, and records the first failure on
 * the geometry.  ct_bounds_checked() returns 1 in a checked build, 0 in the
 * regular one, where the checks are compiled out. */
CT_API int ct_bounds_checked(void);

/* Takes the geometry's first failed-check record and clears it, after the
 * geometry's device has finished all work (cudaDeviceSynchronize on it; the
 * current device is left as it was).  *record is 0 when
 * no check failed (always in the regular build); otherwise
 *   bits 56..63  the site (1..6 above),
 *   bits 32..55  the view (sites 1-5) or z slice (site 6),
 *   bits  0..31  the offending value as a signed 32-bit integer: the z row
 *                (1), the row step (2, 3), the padded row (4) or column (5),
 *                the offset from the ray's base (6).
 * The record is per geometry, shared by all streams using it.  Returns
 * CT_EINVAL for null arguments, CT_ECUDA when the copy fails. */
CT_API ct_status ct_bounds_take(ct_geom *geom, unsigned long long *record);

/* Message describing the last failure on the calling thread ("" if none). */
CT_API const char *ct_last_error(void);

/* Library version string. */
CT_API const char *ct_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CT_H */
