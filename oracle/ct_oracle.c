/*
 * FP64 CPU oracle for the linear CT model of Sidky, Hansen, Jorgensen & Pan,
 * "Iterative image reconstruction for CT with unmatched projection matrices
 * using the generalized minimal residual algorithm" (arXiv 2201.07408).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA library is checked against.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark load it; the library never does, and
 * it shares no code, header or table with the library.
 *
 * What it defines (Sec. I Eq. 1 and Sec. III):
 *   A      m x n   ray-driven projector.  The paper names a line-intersection
 *                  projector; this build reads it as the Joseph projector:
 *                  one bilinear sample per voxel-centre plane of the ray's
 *                  dominant axis, times the step length.
 *   B_un   n x m   voxel-driven back-projector with linear (bilinear in 3D)
 *                  interpolation on the detector; B_un ~ A^T but not equal.
 *   F      m x m   ramp filter per detector row (cosine weight, Ram-Lak,
 *                  linear convolution), so that B_FBP = B_un F.
 *   A^T, B_un^T, F^T  exact transposes.
 *   A_S    m x n   the line-intersection projector itself (the length of
 *                  the ray inside each voxel), and its transpose.
 *
 * A and A^T are both built from one enumerator of the nonzeros of a row of A
 * (a_row), and B_un and B_un^T from one enumerator of a row of B_un (b_row),
 * so each transpose is exact by construction; the tests pin the enumerators
 * themselves against closed forms.
 *
 * Geometry conventions (lengths in mm):
 *   voxel (i,j,k) centre = ((i-(nx-1)/2) vox, (j-(ny-1)/2) vox, (k-(nz-1)/2) vox),
 *   flat index (k*ny + j)*nx + i.
 *   view s: theta = ang0 + s*span/n_views, c = cos theta, s = sin theta.
 *   cone beam: source S = sod (c, s, 0); detector centre D = -(sdd-sod)(c, s, 0);
 *     axes e_u = (-s, c, 0), e_v = (0, 0, 1); pixel (iu, iv) centre
 *     P = D + u e_u + v e_v, u = (iu-(nu-1)/2) du, v = (iv-(nv-1)/2) dv.
 *   2D parallel beam (nz = nv = 1): ray iu is the line u e_u + t e_d with
 *     e_u = (c, s), e_d = (-s, c).
 *   sinogram flat index (s*nv + iv)*nu + iu.
 *
 * Compiled with -ffp-contract=off so that x86 and Arm hosts round alike.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PARALLEL_2D 0
#define OR_CONE_3D 1

typedef struct {
    int kind;
    int nx, ny, nz;
    double vox;
    int n_views;
    double ang0, span;
    int nu, nv;
    double du, dv;
    double sod, sdd;
} or_geom;

static double view_angle(const or_geom *g, long s)
{
    return g->ang0 + (double)s * g->span / (double)g->n_views;
}

static int max_i(int a, int b) { return a > b ? a : b; }

/* Upper bound on the nonzeros of one row of A / of B_un. */
int or_a_row_capacity(const or_geom *g) { return 4 * max_i(g->nx, g->ny); }
int or_b_row_capacity(const or_geom *g) { return 4 * g->n_views; }

/* Source point S and direction d of ray `ray` (unnormalised for the cone). */
static void ray_of(const or_geom *g, long ray, double S[3], double d[3])
{
    long per_view = (long)g->nu * g->nv;
    long s = ray / per_view;
    long rem = ray % per_view;
    long iv = rem / g->nu, iu = rem % g->nu;
    double th = view_angle(g, s);
    double c = cos(th), sn = sin(th);
    double u = ((double)iu - (g->nu - 1) / 2.0) * g->du;
    if (g->kind == OR_CONE_3D) {
        double v = ((double)iv - (g->nv - 1) / 2.0) * g->dv;
        double P[3];
        S[0] = g->sod * c; S[1] = g->sod * sn; S[2] = 0.0;
        P[0] = -(g->sdd - g->sod) * c - u * sn;
        P[1] = -(g->sdd - g->sod) * sn + u * c;
        P[2] = v;
        d[0] = P[0] - S[0]; d[1] = P[1] - S[1]; d[2] = P[2] - S[2];
    } else {
        S[0] = u * c; S[1] = u * sn; S[2] = 0.0;
        d[0] = -sn; d[1] = c; d[2] = 0.0;
    }
}

/*
 * Nonzeros of row `ray` of A (Joseph).  The dominant axis a is x when
 * |d_x| >= |d_y|, else y.  For every voxel-centre plane p = 0..N_a-1 of that
 * axis the ray point r = S + t d with r_a = c_a(p) is converted to fractional
 * grid indices f = r/vox + (N-1)/2 along the two other axes; the sample is
 * the bilinear interpolation of the four neighbours floor(f), floor(f)+1
 * (neighbours outside the grid count as zero).  The row is the sum of the
 * samples times the step length vox*|d|/|d_a|.
 */
int or_a_row(const or_geom *g, long ray, long *idx, double *w)
{
    double S[3], d[3];
    ray_of(g, ray, S, d);
    int a = fabs(d[0]) >= fabs(d[1]) ? 0 : 1;
    int b = 1 - a;
    int Na = a == 0 ? g->nx : g->ny;
    int Nb = a == 0 ? g->ny : g->nx;
    double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double step = g->vox * dn / fabs(d[a]);
    int cnt = 0;
    for (int p = 0; p < Na; ++p) {
        double ca = ((double)p - (Na - 1) / 2.0) * g->vox;
        double t = (ca - S[a]) / d[a];
        double rb = S[b] + t * d[b];
        double rz = S[2] + t * d[2];
        double fb = rb / g->vox + (Nb - 1) / 2.0;
        double fz = rz / g->vox + (g->nz - 1) / 2.0;
        double b0f = floor(fb), z0f = floor(fz);
        double wb = fb - b0f, wz = fz - z0f;
        long b0 = (long)b0f, z0 = (long)z0f;
        for (int dz = 0; dz < 2; ++dz) {
            for (int db = 0; db < 2; ++db) {
                double wt = (db ? wb : 1.0 - wb) * (dz ? wz : 1.0 - wz);
                long ib = b0 + db, iz = z0 + dz;
                if (wt == 0.0 || ib < 0 || ib >= Nb || iz < 0 || iz >= g->nz)
                    continue;
                long ix = a == 0 ? p : ib;
                long iy = a == 0 ? ib : p;
                idx[cnt] = (iz * g->ny + iy) * (long)g->nx + ix;
                w[cnt] = step * wt;
                ++cnt;
            }
        }
    }
    return cnt;
}

/*
 * Nonzeros of row `voxel` of B_un (voxel-driven back-projection, Sec. III).
 * For each view the voxel centre r is projected along the ray from the
 * source: depth L = sod - r.(c, s, 0), magnification M = sdd/L, detector
 * coordinates u = M r.e_u, v = M r_z; the detector value is interpolated
 * bilinearly (zero outside) and weighted by vox^3 M^2/(du dv).  2D parallel
 * beam: u = r.e_u, linear interpolation, weight vox^2/du.  The weight makes
 * B_un ~ A^T in scale (each voxel collects about (M vox/du)(M vox/dv) rays
 * per view in A^T); A^T also carries the obliquity factor |d|/|d_a| that this
 * back-projector omits.
 */
int or_b_row(const or_geom *g, long voxel, long *idx, double *w)
{
    long ix = voxel % g->nx;
    long iy = (voxel / g->nx) % g->ny;
    long iz = voxel / ((long)g->nx * g->ny);
    double rx = ((double)ix - (g->nx - 1) / 2.0) * g->vox;
    double ry = ((double)iy - (g->ny - 1) / 2.0) * g->vox;
    double rz = ((double)iz - (g->nz - 1) / 2.0) * g->vox;
    int cnt = 0;
    for (long s = 0; s < g->n_views; ++s) {
        double th = view_angle(g, s);
        double c = cos(th), sn = sin(th);
        double u, v, wgt;
        if (g->kind == OR_CONE_3D) {
            double L = g->sod - (rx * c + ry * sn);
            double M = g->sdd / L;
            u = M * (-rx * sn + ry * c);
            v = M * rz;
            wgt = g->vox * g->vox * g->vox * M * M / (g->du * g->dv);
        } else {
            u = rx * c + ry * sn;
            v = 0.0;
            wgt = g->vox * g->vox / g->du;
        }
        double fu = u / g->du + (g->nu - 1) / 2.0;
        double fv = v / g->dv + (g->nv - 1) / 2.0;
        double u0f = floor(fu), v0f = floor(fv);
        double wu = fu - u0f, wv = fv - v0f;
        long u0 = (long)u0f, v0 = (long)v0f;
        for (int dv_ = 0; dv_ < 2; ++dv_) {
            for (int du_ = 0; du_ < 2; ++du_) {
                double wt = (du_ ? wu : 1.0 - wu) * (dv_ ? wv : 1.0 - wv);
                long iu = u0 + du_, iv = v0 + dv_;
                if (wt == 0.0 || iu < 0 || iu >= g->nu || iv < 0 || iv >= g->nv)
                    continue;
                idx[cnt] = (s * g->nv + iv) * (long)g->nu + iu;
                w[cnt] = wgt * wt;
                ++cnt;
            }
        }
    }
    return cnt;
}

/*
 * Nonzeros of row `ray` of the line-intersection projector A_S (Sec. III:
 * the paper's matrix elements are the lengths of the ray inside each
 * voxel).  Voxel (i,j,k) is the box of side vox around its centre; the grid
 * is the box [-N vox/2, N vox/2] along each axis (2D: the ray lies in z = 0,
 * inside the single slice).  The ray point is S + alpha d.  The values of
 * alpha where the ray crosses a voxel boundary plane, together with its
 * entry and exit of the grid box, are sorted; each interval between
 * consecutive values lies in one voxel (the one containing the interval's
 * midpoint), and its length is the interval times |d|.  Zero-length
 * intervals (simultaneous crossings) are skipped.  A direction component
 * below 1e-12 |d| counts as zero: such a ray runs parallel to those
 * boundary planes, and one lying in a plane belongs to the voxels on its
 * positive side (a measure-zero case that the method leaves open; the
 * rounded cosine of a 90-degree view would otherwise split the ray between
 * the two sides at an arbitrary point).
 */
static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

int or_s_row_capacity(const or_geom *g) { return g->nx + g->ny + g->nz + 4; }

int or_s_row(const or_geom *g, long ray, long *idx, double *w)
{
    double S[3], d[3];
    ray_of(g, ray, S, d);
    const int N[3] = {g->nx, g->ny, g->nz};
    double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int a = 0; a < 3; ++a)
        if (fabs(d[a]) <= 1e-12 * dn) d[a] = 0.0;
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        hi[a] = 0.5 * N[a] * g->vox;
        lo[a] = -hi[a];
    }
    /* entry and exit of the grid box */
    double a_in = -INFINITY, a_out = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (!(S[a] > lo[a] && S[a] < hi[a])) return 0;
            continue;
        }
        double t1 = (lo[a] - S[a]) / d[a], t2 = (hi[a] - S[a]) / d[a];
        if (t1 > t2) { double t = t1; t1 = t2; t2 = t; }
        if (t1 > a_in) a_in = t1;
        if (t2 < a_out) a_out = t2;
    }
    if (!(a_out > a_in)) return 0;
    int cap = g->nx + g->ny + g->nz + 3;
    double *al = malloc(sizeof(double) * (size_t)(cap + 2));
    int na = 0;
    al[na++] = a_in;
    al[na++] = a_out;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) continue;
        for (int k = 0; k <= N[a]; ++k) {
            double t = (lo[a] + k * g->vox - S[a]) / d[a];
            if (t > a_in && t < a_out) al[na++] = t;
        }
    }
    qsort(al, (size_t)na, sizeof(double), cmp_double);
    int cnt = 0;
    for (int m = 0; m + 1 < na; ++m) {
        double len = (al[m + 1] - al[m]) * dn;
        if (len <= 0.0) continue;
        double am = 0.5 * (al[m] + al[m + 1]);
        long id[3];
        for (int a = 0; a < 3; ++a) {
            /* grid units measured from the centre: exact for a point at the
             * centre (S = 0 on an axis the ray runs parallel to), so that a ray
             * in the central plane of an even grid lies on the plane and goes
             * to its positive side; (S - lo)/vox can round below the plane */
            double f = (S[a] + am * d[a]) / g->vox + 0.5 * N[a];
            long i = (long)floor(f);
            if (i < 0) i = 0;
            if (i >= N[a]) i = N[a] - 1;
            id[a] = i;
        }
        idx[cnt] = (id[2] * g->ny + id[1]) * (long)g->nx + id[0];
        w[cnt] = len;
        ++cnt;
    }
    free(al);
    return cnt;
}

/* y = A_S x, and x = A_S^T y, with the line-intersection projector. */
void or_project_S(const or_geom *g, const double *x, double *y)
{
    long m = (long)g->n_views * g->nv * g->nu;
    int cap = or_s_row_capacity(g);
#pragma omp parallel
    {
        long *idx = malloc(sizeof(long) * cap);
        double *w = malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 256)
        for (long r = 0; r < m; ++r) {
            int cnt = or_s_row(g, r, idx, w);
            double acc = 0.0;
            for (int e = 0; e < cnt; ++e)
                acc += w[e] * x[idx[e]];
            y[r] = acc;
        }
        free(idx);
        free(w);
    }
}

void or_project_S_rays(const or_geom *g, const double *x, const long *rays, long count, double *out)
{
    int cap = or_s_row_capacity(g);
#pragma omp parallel
    {
        long *idx = malloc(sizeof(long) * cap);
        double *w = malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 16)
        for (long e = 0; e < count; ++e) {
            int cnt = or_s_row(g, rays[e], idx, w);
            double acc = 0.0;
            for (int q = 0; q < cnt; ++q)
                acc += w[q] * x[idx[q]];
            out[e] = acc;
        }
        free(idx);
        free(w);
    }
}

void or_adjoint_St(const or_geom *g, const double *y, double *x)
{
    long n = (long)g->nx * g->ny * g->nz;
    long m = (long)g->n_views * g->nv * g->nu;
    int cap = or_s_row_capacity(g);
    memset(x, 0, sizeof(double) * n);
#pragma omp parallel
    {
        long *idx = malloc(sizeof(long) * cap);
        double *w = malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 256)
        for (long r = 0; r < m; ++r) {
            int cnt = or_s_row(g, r, idx, w);
            for (int e = 0; e < cnt; ++e) {
                double val = w[e] * y[r];
#pragma omp atomic
                x[idx[e]] += val;
            }
        }
        free(idx);
        free(w);
    }
}

/* y = A x  (x: n, y: m). */
void or_project_A(const or_geom *g, const double *x, double *y)
{
    long m = (long)g->n_views * g->nv * g->nu;
    int cap = or_a_row_capacity(g);
#pragma omp parallel
    {
        long *idx = malloc(sizeof(long) * cap);
        double *w = malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 256)
        for (long r = 0; r < m; ++r) {
            int cnt = or_a_row(g, r, idx, w);
            double acc = 0.0;
            for (int e = 0; e < cnt; ++e)
                acc += w[e] * x[idx[e]];
            y[r] = acc;
        }
        free(idx);
        free(w);
    }
}

/* out[e] = (A x)[rays[e]] for a list of rays (full-size spot checks). */
void or_project_A_rays(const or_geom *g, const double *x, const long *rays, long count,
                       double *out)
{
    int cap = or_a_row_capacity(g);
#pragma omp parallel
    {
        long *idx = malloc(sizeof(long) * cap);
        double *w = malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 16)
        for (long e = 0; e < count; ++e) {
            int cnt = or_a_row(g, rays[e], idx, w);
            double acc = 0.0;
            for (int q = 0; q < cnt; ++q)
                acc += w[q] * x[idx[q]];
            out[e] = acc;
        }
        free(idx);
        free(w);
    }
}

/* x = A^T y  (y: m, x: n); scatter of the rows of A. */
void or_adjoint_At(const or_geom *g, const double *y, double *x)
{
    long n = (long)g->nx * g->ny * g->nz;
    long m = (long)g->n_views * g->nv * g->nu;
    int cap = or_a_row_capacity(g);
    memset(x, 0, sizeof(double) * n);
#pragma omp parallel
    {
        long *idx = malloc(sizeof(long) * cap);
        double *w = malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 256)
        for (long r = 0; r < m; ++r) {
            int cnt = or_a_row(g, r, idx, w);
            for (int e = 0; e < cnt; ++e) {
                double val = w[e] * y[r];
#pragma omp atomic
                x[idx[e]] += val;
            }
        }
        free(idx);
        free(w);
    }
}

/* x = B_un y  (y: m, x: n). */
void or_backproject_B(const or_geom *g, const double *y, double *x)
{
    long n = (long)g->nx * g->ny * g->nz;
    int cap = or_b_row_capacity(g);
#pragma omp parallel
    {
        long *idx = malloc(sizeof(long) * cap);
        double *w = malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 256)
        for (long j = 0; j < n; ++j) {
            int cnt = or_b_row(g, j, idx, w);
            double acc = 0.0;
            for (int e = 0; e < cnt; ++e)
                acc += w[e] * y[idx[e]];
            x[j] = acc;
        }
        free(idx);
        free(w);
    }
}

/* out[e] = (B_un y)[voxels[e]] for a list of voxels. */
void or_backproject_B_voxels(const or_geom *g, const double *y, const long *voxels,
                             long count, double *out)
{
    int cap = or_b_row_capacity(g);
#pragma omp parallel
    {
        long *idx = malloc(sizeof(long) * cap);
        double *w = malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 16)
        for (long e = 0; e < count; ++e) {
            int cnt = or_b_row(g, voxels[e], idx, w);
            double acc = 0.0;
            for (int q = 0; q < cnt; ++q)
                acc += w[q] * y[idx[q]];
            out[e] = acc;
        }
        free(idx);
        free(w);
    }
}

/* y = B_un^T x  (x: n, y: m); scatter of the rows of B_un. */
void or_adjoint_Bt(const or_geom *g, const double *x, double *y)
{
    long n = (long)g->nx * g->ny * g->nz;
    long m = (long)g->n_views * g->nv * g->nu;
    int cap = or_b_row_capacity(g);
    memset(y, 0, sizeof(double) * m);
#pragma omp parallel
    {
        long *idx = malloc(sizeof(long) * cap);
        double *w = malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 256)
        for (long j = 0; j < n; ++j) {
            int cnt = or_b_row(g, j, idx, w);
            for (int e = 0; e < cnt; ++e) {
                double val = w[e] * x[j];
#pragma omp atomic
                y[idx[e]] += val;
            }
        }
        free(idx);
        free(w);
    }
}

/*
 * Ramp filter F (Sec. III, B_FBP = B_un F).  The paper names only "the ramp
 * filter"; this build reads it as the FDK filtering step: each detector row
 * is multiplied by the cosine weight sdd/sqrt(sdd^2+u^2+v^2) (1 for parallel
 * beam), then linearly convolved (zero outside the row) with the Ram-Lak
 * kernel h[0] = 1/(4 tau^2), h[k odd] = -1/(pi^2 k^2 tau^2), h[k even] = 0,
 * tau = detector spacing at the rotation axis (du*sod/sdd, or du), and scaled
 * by tau * c_F.  c_F = (pi/n_views) * (sod/sdd)^2 du dv / vox^3 (cone) or
 * (pi/n_views) du / vox^2 (parallel) turns B_un F into an FBP reconstruction
 * in density units.
 */
static double ramlak(long k, double tau)
{
    if (k == 0)
        return 1.0 / (4.0 * tau * tau);
    if (k % 2 == 0)
        return 0.0;
    return -1.0 / (M_PI * M_PI * (double)k * (double)k * tau * tau);
}

static double ramp_tau(const or_geom *g)
{
    return g->kind == OR_CONE_3D ? g->du * g->sod / g->sdd : g->du;
}

double or_ramp_scale(const or_geom *g)
{
    double base = M_PI / (double)g->n_views;
    double cf;
    if (g->kind == OR_CONE_3D)
        cf = base * (g->sod / g->sdd) * (g->sod / g->sdd) * g->du * g->dv /
             (g->vox * g->vox * g->vox);
    else
        cf = base * g->du / (g->vox * g->vox);
    return cf * ramp_tau(g);
}

static double cos_weight(const or_geom *g, long iu, long iv)
{
    if (g->kind != OR_CONE_3D)
        return 1.0;
    double u = ((double)iu - (g->nu - 1) / 2.0) * g->du;
    double v = ((double)iv - (g->nv - 1) / 2.0) * g->dv;
    return g->sdd / sqrt(g->sdd * g->sdd + u * u + v * v);
}

/* Filter the detector rows listed in `rows` (row r = s*nv + iv). */
static void ramp_rows(const or_geom *g, const double *y, double *out, const long *rows,
                      long count, int transpose)
{
    double tau = ramp_tau(g);
    double scale = or_ramp_scale(g);
    long nu = g->nu;
#pragma omp parallel
    {
        double *wrow = malloc(sizeof(double) * nu);
#pragma omp for schedule(dynamic, 4)
        for (long e = 0; e < count; ++e) {
            long r = rows ? rows[e] : e;
            long iv = r % g->nv;
            const double *in = y + r * nu;
            double *o = out + (rows ? e : r) * nu;
            /* F = scale * H * diag(cw); F^T = diag(cw) * H^T * scale, H symmetric */
            for (long k = 0; k < nu; ++k)
                wrow[k] = transpose ? in[k] : in[k] * cos_weight(g, k, iv);
            for (long i = 0; i < nu; ++i) {
                double acc = 0.0;
                for (long k = 0; k < nu; ++k)
                    acc += ramlak(i - k, tau) * wrow[k];
                o[i] = scale * acc * (transpose ? cos_weight(g, i, iv) : 1.0);
            }
        }
        free(wrow);
    }
}

/* yf = F y over the whole sinogram. */
void or_ramp_F(const or_geom *g, const double *y, double *yf)
{
    ramp_rows(g, y, yf, NULL, (long)g->n_views * g->nv, 0);
}

/* y = F^T z. */
void or_ramp_Ft(const or_geom *g, const double *z, double *y)
{
    ramp_rows(g, z, y, NULL, (long)g->n_views * g->nv, 1);
}

/* out[e*nu + i] = (F y)[row rows[e], i] for a list of detector rows. */
void or_ramp_F_rows(const or_geom *g, const double *y, const long *rows, long count,
                    double *out)
{
    ramp_rows(g, y, out, rows, count, 0);
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
