/*
 * FP64 CPU oracle for voxel-driven circular cone-beam back-projection.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the bench's CPU
 * baseline leg use it. It shares no code, header, table or helper with the
 * CUDA library; both sides only see the same seeded input arrays.
 *
 * Every routine is the plain definition, in double precision, with no
 * blocking or fusion. Citations name the paper's sections and listings
 * (Chen et al., "Performance Portable Back-projection Algorithms on CPUs",
 * ICS '21).
 *
 * Readings where the paper is silent (the paper skips the derivation of the
 * projection matrix, Section 2.1.1, and assumes already-filtered input,
 * Section 2.1.2):
 *   - voxel (i,j,k) sits at x=(i-(nx-1)/2)sx+ox, same for y and z;
 *   - view s: source at sid*e_r, e_r=(cos t, sin t, 0), e_u=(-sin t, cos t, 0),
 *     e_v=(0,0,1); flat detector normal to e_r at distance sdd from the source;
 *   - homogeneous depth w=(sid - X.e_r)/sid (1 at the isocenter), so the
 *     Listing 1 weight f^2 = 1/w^2 is the FDK distance weight;
 *   - pixel centres at integer indices; the detector centre is at
 *     ((nu-1)/2+u_off, (nv-1)/2+v_off);
 *   - bilinear sampling uses floor (not truncation) and a zero-padded
 *     detector: every tap outside [0,nu-1]x[0,nv-1] contributes 0;
 *   - Ram-Lak: isocenter pitch dp=du*sid/sdd, h[0]=1/(4dp^2),
 *     h[odd n]=-1/(pi^2 n^2 dp^2), h[even n!=0]=0, cosine weight
 *     sdd/sqrt(sdd^2+u^2+v^2), linear (zero-padded) convolution along u,
 *     Q = dp * (h conv g_w); FDK scale pi/np (Feldkamp; the paper cites it
 *     but prints no formula).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ */
/* Geometry: 3x4 projection matrix per view (pinhole model, Sec. 2.1.1) */
/* ------------------------------------------------------------------ */

/* P is [np][3][4], row-major, acting on the voxel index vector (i,j,k,1).
 * Row 2 gives w, rows 0 and 1 give u*w and v*w (homogeneous detector
 * coordinates in pixels). */
void orc_matrices(double sid, double sdd, int np, const double *angles,
                  int nu, int nv, double du, double dv, double u_off,
                  double v_off, int nx, int ny, int nz, double sx, double sy,
                  double sz, double ox, double oy, double oz, double *P)
{
    const double cu = 0.5 * (nu - 1) + u_off;
    const double cv = 0.5 * (nv - 1) + v_off;
    const double x0 = ox - 0.5 * (nx - 1) * sx;
    const double y0 = oy - 0.5 * (ny - 1) * sy;
    const double z0 = oz - 0.5 * (nz - 1) * sz;
    for (int s = 0; s < np; ++s) {
        const double t = angles[s];
        const double c = cos(t), sn = sin(t);
        /* rows in world coordinates (x, y, z, 1) */
        double r2[4] = {-c / sid, -sn / sid, 0.0, 1.0};
        double mu = sdd / (sid * du), mv = sdd / (sid * dv);
        double r0[4] = {-sn * mu + cu * r2[0], c * mu + cu * r2[1], 0.0, cu};
        double r1[4] = {cv * r2[0], cv * r2[1], mv, cv};
        const double *rows[3] = {r0, r1, r2};
        for (int r = 0; r < 3; ++r) {
            const double *w = rows[r];
            double *o = P + 12 * s + 4 * r;
            /* compose with index -> world: (x0+sx*i, y0+sy*j, z0+sz*k, 1) */
            o[0] = w[0] * sx;
            o[1] = w[1] * sy;
            o[2] = w[2] * sz;
            o[3] = w[0] * x0 + w[1] * y0 + w[2] * z0 + w[3];
        }
    }
}

/* dot4 of Listing 2: inner product with the homogeneous 1 in slot 3. */
static double dot4(const double *row, double i, double j, double k)
{
    return row[0] * i + row[1] * j + row[2] * k + row[3];
}

/* mix of Listing 2: x*(1-a) + y*a. */
static double mix(double x, double y, double a) { return x * (1.0 - a) + y * a; }

static double tap(const double *img, int nu, int nv, long r, long c)
{
    if (r < 0 || r >= nv || c < 0 || c >= nu) return 0.0;
    return img[r * (long)nu + c];
}

/* Bilinear_Interpolate of Listing 2: horizontal mix on two rows, then a
 * vertical mix. x is the detector column (u), y the row (v). */
static double bilinear(const double *img, int nu, int nv, double x, double y)
{
    if (!(x > -2.0 && x < nu + 1.0 && y > -2.0 && y < nv + 1.0)) return 0.0;
    double fx = floor(x), fy = floor(y);
    long n = (long)fx, m = (long)fy;
    double a = x - fx, b = y - fy;
    double s0 = mix(tap(img, nu, nv, m, n), tap(img, nu, nv, m, n + 1), a);
    double s1 = mix(tap(img, nu, nv, m + 1, n), tap(img, nu, nv, m + 1, n + 1), a);
    return mix(s0, s1, b);
}

/* Back-projection, Listing 1 in double: for every view s and voxel (i,j,k),
 * z = dot4(P2,v); f = 1/z; x = dot4(P0,v) f; y = dot4(P1,v) f;
 * vol += Bilinear(img_s, x, y) * f^2. The sum is then multiplied by scale.
 * img: [np][nv][nu]; vol: [nz][ny][nx] (overwritten). */
void orc_backproject(const double *P, int np, const double *img, int nu,
                     int nv, int nx, int ny, int nz, double scale, double *vol)
{
    const long nvox = (long)nx * ny * nz;
    for (long t = 0; t < nvox; ++t) vol[t] = 0.0;
    for (int s = 0; s < np; ++s) {
        const double *Ps = P + 12 * s;
        const double *im = img + (long)s * nu * nv;
#pragma omp parallel for collapse(2) schedule(static)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    double z = dot4(Ps + 8, i, j, k);
                    double f = 1.0 / z;
                    double x = dot4(Ps + 0, i, j, k) * f;
                    double y = dot4(Ps + 4, i, j, k) * f;
                    double val = bilinear(im, nu, nv, x, y);
                    double w = f * f;
                    vol[((long)k * ny + j) * nx + i] += val * w;
                }
    }
    for (long t = 0; t < nvox; ++t) vol[t] *= scale;
}

/* The same sum as orc_backproject, for a list of voxels only (used to check
 * sampled outputs of volumes too large for the full loop). ijk: [n][3]. */
void orc_backproject_points(const double *P, int np, const double *img,
                            int nu, int nv, long n, const int *ijk,
                            double scale, double *out)
{
#pragma omp parallel for schedule(static)
    for (long t = 0; t < n; ++t) {
        double i = ijk[3 * t], j = ijk[3 * t + 1], k = ijk[3 * t + 2];
        double acc = 0.0;
        for (int s = 0; s < np; ++s) {
            const double *Ps = P + 12 * s;
            double z = dot4(Ps + 8, i, j, k);
            double f = 1.0 / z;
            double x = dot4(Ps + 0, i, j, k) * f;
            double y = dot4(Ps + 4, i, j, k) * f;
            acc += bilinear(img + (long)s * nu * nv, nu, nv, x, y) * f * f;
        }
        out[t] = acc * scale;
    }
}

/* Back-projection restricted to slices k0..k0+nks-1 (a z-slab); vol holds
 * [nks][ny][nx]. Same loop order and arithmetic as orc_backproject. */
void orc_backproject_slab(const double *P, int np, const double *img, int nu,
                          int nv, int nx, int ny, int k0, int nks,
                          double scale, double *vol)
{
    const long nvox = (long)nx * ny * nks;
    for (long t = 0; t < nvox; ++t) vol[t] = 0.0;
    for (int s = 0; s < np; ++s) {
        const double *Ps = P + 12 * s;
        const double *im = img + (long)s * nu * nv;
        /* threads share the (slice, row) pairs, so a thin slab keeps every
         * core busy; each voxel's arithmetic is the same as above */
#pragma omp parallel for collapse(2) schedule(static)
        for (int kk = 0; kk < nks; ++kk) {
            for (int j = 0; j < ny; ++j) {
                const int k = k0 + kk;
                for (int i = 0; i < nx; ++i) {
                    double z = dot4(Ps + 8, i, j, k);
                    double f = 1.0 / z;
                    double x = dot4(Ps + 0, i, j, k) * f;
                    double y = dot4(Ps + 4, i, j, k) * f;
                    vol[((long)kk * ny + j) * nx + i] +=
                        bilinear(im, nu, nv, x, y) * f * f;
                }
            }
        }
    }
    for (long t = 0; t < nvox; ++t) vol[t] *= scale;
}

/* Matched forward projector: the exact transpose of orc_backproject. Each
 * voxel value, times scale*f^2, is scattered to the same four taps with the
 * bilinear weights (1-a)(1-b), a(1-b), (1-a)b, ab. proj: [np][nv][nu]
 * (overwritten). */
void orc_forward_project(const double *P, int np, const double *vol, int nx,
                         int ny, int nz, double scale, int nu, int nv,
                         double *proj)
{
#pragma omp parallel for schedule(dynamic)
    for (int s = 0; s < np; ++s) {
        const double *Ps = P + 12 * s;
        double *q = proj + (long)s * nu * nv;
        for (long t = 0; t < (long)nu * nv; ++t) q[t] = 0.0;
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    double z = dot4(Ps + 8, i, j, k);
                    double f = 1.0 / z;
                    double x = dot4(Ps + 0, i, j, k) * f;
                    double y = dot4(Ps + 4, i, j, k) * f;
                    if (!(x > -2.0 && x < nu + 1.0 && y > -2.0 && y < nv + 1.0))
                        continue;
                    double fx = floor(x), fy = floor(y);
                    long n = (long)fx, m = (long)fy;
                    double a = x - fx, b = y - fy;
                    double val = vol[((long)k * ny + j) * nx + i] * f * f * scale;
                    long rr[4] = {m, m, m + 1, m + 1};
                    long cc[4] = {n, n + 1, n, n + 1};
                    double ww[4] = {(1 - a) * (1 - b), a * (1 - b), (1 - a) * b, a * b};
                    for (int q4 = 0; q4 < 4; ++q4) {
                        if (rr[q4] < 0 || rr[q4] >= nv || cc[q4] < 0 || cc[q4] >= nu) continue;
                        q[rr[q4] * nu + cc[q4]] += ww[q4] * val;
                    }
                }
    }
}

/* ------------------------------------------------------------------ */
/* Filtering before back-projection (FDK, Sec. 2.1; formula is our reading) */
/* ------------------------------------------------------------------ */

/* Cosine weight then a direct linear convolution along u with the discrete
 * Ram-Lak kernel on the isocenter grid. in/out: [nrows_total = np*nv][nu]. */
void orc_filter_rows(int np, int nu, int nv, int r0, int nr, double du,
                     double dv, double u_off, double v_off, double sid,
                     double sdd, const double *in, double *out);

void orc_filter(int np, int nu, int nv, double du, double dv, double u_off,
                double v_off, double sid, double sdd, const double *in,
                double *out)
{
    orc_filter_rows(np, nu, nv, 0, nv, du, dv, u_off, v_off, sid, sdd, in, out);
}

/* The same filter for detector rows r0..r0+nr-1 only: in/out are
 * [np][nr][nu] and row t of view s is detector row r0+t (its cosine weight
 * uses that row's v). */
void orc_filter_rows(int np, int nu, int nv, int r0, int nr, double du,
                     double dv, double u_off, double v_off, double sid,
                     double sdd, const double *in, double *out)
{
    const double cu = 0.5 * (nu - 1) + u_off;
    const double cv = 0.5 * (nv - 1) + v_off;
    const double dp = du * sid / sdd;
    double *h = (double *)malloc(sizeof(double) * (2 * nu - 1));
    for (int n = -(nu - 1); n <= nu - 1; ++n) {
        double v;
        if (n == 0) v = 1.0 / (4.0 * dp * dp);
        else if (n % 2 == 0) v = 0.0;
        else v = -1.0 / (M_PI * M_PI * (double)n * (double)n * dp * dp);
        h[n + nu - 1] = v;
    }
#pragma omp parallel
    {
        double *g = (double *)malloc(sizeof(double) * nu);
#pragma omp for schedule(static)
        for (long row = 0; row < (long)np * nr; ++row) {
            int r = r0 + (int)(row % nr);
            double vm = (r - cv) * dv;
            const double *src = in + row * nu;
            double *dst = out + row * nu;
            for (int m = 0; m < nu; ++m) {
                double um = (m - cu) * du;
                g[m] = src[m] * sdd / sqrt(sdd * sdd + um * um + vm * vm);
            }
            for (int n = 0; n < nu; ++n) {
                double acc = 0.0;
                for (int m = 0; m < nu; ++m) acc += h[n - m + nu - 1] * g[m];
                dst[n] = dp * acc;
            }
        }
        free(g);
    }
    free(h);
}

/* ------------------------------------------------------------------ */
/* Input data: analytic line integrals of an ellipsoid phantom          */
/* ------------------------------------------------------------------ */

/* ell: [ne][16] = cx, cy, cz, ax, ay, az, R (3x3 row-major, body->world),
 * rho. Overlapping ellipsoids add. Ray from the source to each pixel
 * centre; the line integral of one ellipsoid is rho * chord length.
 * out: [np][nv][nu]. */
void orc_phantom_project_rows(double sid, double sdd, int np,
                              const double *angles, int nu, int nv, int r0,
                              int nr, double du, double dv, double u_off,
                              double v_off, int ne, const double *ell,
                              double *out);

void orc_phantom_project(double sid, double sdd, int np, const double *angles,
                         int nu, int nv, double du, double dv, double u_off,
                         double v_off, int ne, const double *ell, double *out)
{
    orc_phantom_project_rows(sid, sdd, np, angles, nu, nv, 0, nv, du, dv, u_off,
                             v_off, ne, ell, out);
}

/* Detector rows r0..r0+nr-1 only; out is [np][nr][nu]. */
void orc_phantom_project_rows(double sid, double sdd, int np,
                              const double *angles, int nu, int nv, int r0,
                              int nr, double du, double dv, double u_off,
                              double v_off, int ne, const double *ell,
                              double *out)
{
    const double cu = 0.5 * (nu - 1) + u_off;
    const double cv = 0.5 * (nv - 1) + v_off;
#pragma omp parallel for schedule(dynamic)
    for (long row = 0; row < (long)np * nr; ++row) {
        int s = (int)(row / nr), r = r0 + (int)(row % nr);
        double c = cos(angles[s]), sn = sin(angles[s]);
        double er[3] = {c, sn, 0.0}, eu[3] = {-sn, c, 0.0};
        double S[3] = {sid * er[0], sid * er[1], 0.0};
        double V = (r - cv) * dv;
        for (int col = 0; col < nu; ++col) {
            double U = (col - cu) * du;
            double pix[3] = {(sid - sdd) * er[0] + U * eu[0],
                             (sid - sdd) * er[1] + U * eu[1], V};
            double dir[3] = {pix[0] - S[0], pix[1] - S[1], pix[2] - S[2]};
            double L = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
            double sum = 0.0;
            for (int e = 0; e < ne; ++e) {
                const double *E = ell + 16 * e;
                const double *R = E + 6;
                double p[3] = {S[0] - E[0], S[1] - E[1], S[2] - E[2]};
                double pb[3], db[3];
                for (int a = 0; a < 3; ++a) {
                    /* body coordinates: R^T times, then divide by the semi-axis */
                    pb[a] = (R[0 * 3 + a] * p[0] + R[1 * 3 + a] * p[1] + R[2 * 3 + a] * p[2]) / E[3 + a];
                    db[a] = (R[0 * 3 + a] * dir[0] + R[1 * 3 + a] * dir[1] + R[2 * 3 + a] * dir[2]) / E[3 + a];
                }
                double A = db[0] * db[0] + db[1] * db[1] + db[2] * db[2];
                double B = 2.0 * (pb[0] * db[0] + pb[1] * db[1] + pb[2] * db[2]);
                double C = pb[0] * pb[0] + pb[1] * pb[1] + pb[2] * pb[2] - 1.0;
                double disc = B * B - 4.0 * A * C;
                if (disc > 0.0) sum += E[15] * sqrt(disc) / A * L;
            }
            out[row * nu + col] = sum;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Ray-driven (Siddon) line integrals through a voxel grid              */
/* ------------------------------------------------------------------ */

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Line integral from the source to each pixel centre through the piecewise
 * constant voxel volume vol [nz][ny][nx] (voxel (i,j,k) fills the box of
 * half-size (sx,sy,sz)/2 around its centre). All plane crossings are
 * collected and sorted; each segment adds length * value of the voxel that
 * holds its midpoint. out: [np][nv][nu]. */
void orc_siddon(double sid, double sdd, int np, const double *angles, int nu,
                int nv, double du, double dv, double u_off, double v_off,
                int nx, int ny, int nz, double sx, double sy, double sz,
                double ox, double oy, double oz, const double *vol, double *out)
{
    const double cu = 0.5 * (nu - 1) + u_off;
    const double cv = 0.5 * (nv - 1) + v_off;
    const double bx = ox - 0.5 * nx * sx, by = oy - 0.5 * ny * sy, bz = oz - 0.5 * nz * sz;
#pragma omp parallel
    {
        double *al = (double *)malloc(sizeof(double) * (nx + ny + nz + 8));
#pragma omp for schedule(dynamic)
        for (long row = 0; row < (long)np * nv; ++row) {
            int s = (int)(row / nv), r = (int)(row % nv);
            double c = cos(angles[s]), sn = sin(angles[s]);
            double S[3] = {sid * c, sid * sn, 0.0};
            double V = (r - cv) * dv;
            for (int col = 0; col < nu; ++col) {
                double U = (col - cu) * du;
                double pix[3] = {(sid - sdd) * c - U * sn, (sid - sdd) * sn + U * c, V};
                double d[3] = {pix[0] - S[0], pix[1] - S[1], pix[2] - S[2]};
                double L = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                int na = 0;
                al[na++] = 0.0;
                al[na++] = 1.0;
                const double base[3] = {bx, by, bz};
                const double step[3] = {sx, sy, sz};
                const int cnt[3] = {nx, ny, nz};
                for (int a = 0; a < 3; ++a) {
                    if (fabs(d[a]) < 1e-300) continue;
                    for (int p = 0; p <= cnt[a]; ++p) {
                        double t = (base[a] + p * step[a] - S[a]) / d[a];
                        if (t > 0.0 && t < 1.0) al[na++] = t;
                    }
                }
                qsort(al, na, sizeof(double), cmp_double);
                double sum = 0.0;
                for (int m = 0; m + 1 < na; ++m) {
                    double t0 = al[m], t1 = al[m + 1];
                    if (t1 <= t0) continue;
                    double tm = 0.5 * (t0 + t1);
                    double X[3] = {S[0] + tm * d[0], S[1] + tm * d[1], S[2] + tm * d[2]};
                    long ii = (long)floor((X[0] - bx) / sx);
                    long jj = (long)floor((X[1] - by) / sy);
                    long kk = (long)floor((X[2] - bz) / sz);
                    if (ii < 0 || ii >= nx || jj < 0 || jj >= ny || kk < 0 || kk >= nz) continue;
                    sum += (t1 - t0) * L * vol[(kk * ny + jj) * nx + ii];
                }
                out[row * nu + col] = sum;
            }
        }
        free(al);
    }
}

/* Number of OpenMP threads the routines above use (1 without OpenMP). */
/* ------------------------------------------------------------------ */
/* Iterative reconstruction on the projector pair (Section 1 names     */
/* MLEM and SART as the methods that call back-projection repeatedly)   */
/* ------------------------------------------------------------------ */

/* Views of subset t (of nsub): s = t, t + nsub, t + 2 nsub, ... Their
 * matrices and projections are gathered into compact arrays. */
static int subset_views(int np, int nsub, int t, const double *P, const double *proj,
                        long plane, double *Pt, double *pt)
{
    int n = 0;
    for (int s = t; s < np; s += nsub, ++n) {
        memcpy(Pt + 12 * n, P + 12 * s, 12 * sizeof(double));
        if (proj) memcpy(pt + plane * n, proj + plane * s, plane * sizeof(double));
    }
    return n;
}

/* MLEM (Shepp and Vardi) with ordered subsets of views (Hudson and Larkin;
 * nsub = 1 is plain MLEM). A is the voxel-driven forward projector with
 * scale 1, A^T the back-projector. Per subset t:
 *   y = A_t x;  r_i = p_i / y_i where y_i > eps, else 0;
 *   x_j <- x_j (A_t^T r)_j / (A_t^T 1)_j where (A_t^T 1)_j > eps, else x_j.
 * iters passes over all subsets; x holds the start value on entry. */
void orc_mlem(const double *P, int np, const double *proj, int nu, int nv, int nx,
              int ny, int nz, int nsub, int iters, double eps, double *x)
{
    const long plane = (long)nu * nv, nvox = (long)nx * ny * nz;
    const int nmax = (np + nsub - 1) / nsub;
    double *Pt = malloc(sizeof(double) * 12 * nmax);
    double *pt = malloc(sizeof(double) * plane * nmax);
    double *y = malloc(sizeof(double) * plane * nmax);
    double *ones = malloc(sizeof(double) * plane * nmax);
    double *b = malloc(sizeof(double) * nvox);
    double *sens = malloc(sizeof(double) * nvox);
    for (long i = 0; i < plane * nmax; ++i) ones[i] = 1.0;
    for (int it = 0; it < iters; ++it) {
        for (int t = 0; t < nsub; ++t) {
            const int n = subset_views(np, nsub, t, P, proj, plane, Pt, pt);
            orc_backproject(Pt, n, ones, nu, nv, nx, ny, nz, 1.0, sens);
            orc_forward_project(Pt, n, x, nx, ny, nz, 1.0, nu, nv, y);
            for (long i = 0; i < plane * n; ++i) y[i] = (y[i] > eps) ? pt[i] / y[i] : 0.0;
            orc_backproject(Pt, n, y, nu, nv, nx, ny, nz, 1.0, b);
            for (long j = 0; j < nvox; ++j)
                if (sens[j] > eps) x[j] = x[j] * b[j] / sens[j];
        }
    }
    free(Pt); free(pt); free(y); free(ones); free(b); free(sens);
}

/* SART (Andersen and Kak) in block form over the same view subsets (nsub = 1
 * is the simultaneous version, SIRT). Per subset t:
 *   y = A_t x;  r_i = (p_i - y_i) / (A_t 1)_i where (A_t 1)_i > eps, else 0;
 *   x_j <- x_j + lambda (A_t^T r)_j / (A_t^T 1)_j where (A_t^T 1)_j > eps;
 *   then x_j <- max(x_j, 0) when nonneg. */
void orc_sart(const double *P, int np, const double *proj, int nu, int nv, int nx,
              int ny, int nz, int nsub, int iters, double lambda, int nonneg,
              double eps, double *x)
{
    const long plane = (long)nu * nv, nvox = (long)nx * ny * nz;
    const int nmax = (np + nsub - 1) / nsub;
    double *Pt = malloc(sizeof(double) * 12 * nmax);
    double *pt = malloc(sizeof(double) * plane * nmax);
    double *y = malloc(sizeof(double) * plane * nmax);
    double *ray = malloc(sizeof(double) * plane * nmax);
    double *ones_p = malloc(sizeof(double) * plane * nmax);
    double *ones_v = malloc(sizeof(double) * nvox);
    double *b = malloc(sizeof(double) * nvox);
    double *sens = malloc(sizeof(double) * nvox);
    for (long i = 0; i < plane * nmax; ++i) ones_p[i] = 1.0;
    for (long j = 0; j < nvox; ++j) ones_v[j] = 1.0;
    for (int it = 0; it < iters; ++it) {
        for (int t = 0; t < nsub; ++t) {
            const int n = subset_views(np, nsub, t, P, proj, plane, Pt, pt);
            orc_backproject(Pt, n, ones_p, nu, nv, nx, ny, nz, 1.0, sens);
            orc_forward_project(Pt, n, ones_v, nx, ny, nz, 1.0, nu, nv, ray);
            orc_forward_project(Pt, n, x, nx, ny, nz, 1.0, nu, nv, y);
            for (long i = 0; i < plane * n; ++i) y[i] = (ray[i] > eps) ? (pt[i] - y[i]) / ray[i] : 0.0;
            orc_backproject(Pt, n, y, nu, nv, nx, ny, nz, 1.0, b);
            for (long j = 0; j < nvox; ++j) {
                if (sens[j] > eps) x[j] += lambda * b[j] / sens[j];
                if (nonneg && x[j] < 0.0) x[j] = 0.0;
            }
        }
    }
    free(Pt); free(pt); free(y); free(ray); free(ones_p); free(ones_v); free(b); free(sens);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads the routines above use from now on (n >= 1; timing only: the
 * arithmetic of every voxel is the same at any count). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------ */
/* 3x3x3 convolution of the few-view correction network (no paper      */
/* counterpart): plain definitions in double, channels-last tensors.   */
/* ------------------------------------------------------------------ */

/* y[n][z][y][x][co] = b[co] + sum_{dz,dy,dx,ci} w[co][(dz*3+dy)*3+dx][ci]
 *                     * x[n][z+dz-1][y+dy-1][x+dx-1][ci], zero outside. */
void orc_conv3d(const double *x, int N, int D, int H, int W, int cin, const double *w,
                const double *b, int cout, double *y)
{
#pragma omp parallel for collapse(2) schedule(static)
    for (int n = 0; n < N; ++n)
        for (int z = 0; z < D; ++z)
            for (int yy = 0; yy < H; ++yy)
                for (int xx = 0; xx < W; ++xx)
                    for (int co = 0; co < cout; ++co) {
                        double acc = b ? b[co] : 0.0;
                        for (int t = 0; t < 27; ++t) {
                            int zi = z + t / 9 - 1, yi = yy + (t / 3) % 3 - 1, xi = xx + t % 3 - 1;
                            if (zi < 0 || zi >= D || yi < 0 || yi >= H || xi < 0 || xi >= W) continue;
                            const double *xp = x + ((((long)n * D + zi) * H + yi) * W + xi) * cin;
                            const double *wp = w + ((long)co * 27 + t) * cin;
                            for (int ci = 0; ci < cin; ++ci) acc += wp[ci] * xp[ci];
                        }
                        y[((((long)n * D + z) * H + yy) * W + xx) * cout + co] = acc;
                    }
}

/* Input gradient: dx[v][ci] = sum_{t,co} w[co][t][ci] dy[v - off(t)][co]. */
void orc_conv3d_dgrad(const double *dy, int N, int D, int H, int W, int cout, const double *w,
                      int cin, double *dx)
{
#pragma omp parallel for collapse(2) schedule(static)
    for (int n = 0; n < N; ++n)
        for (int z = 0; z < D; ++z)
            for (int yy = 0; yy < H; ++yy)
                for (int xx = 0; xx < W; ++xx)
                    for (int ci = 0; ci < cin; ++ci) {
                        double acc = 0.0;
                        for (int t = 0; t < 27; ++t) {
                            int zo = z - (t / 9 - 1), yo = yy - ((t / 3) % 3 - 1), xo = xx - (t % 3 - 1);
                            if (zo < 0 || zo >= D || yo < 0 || yo >= H || xo < 0 || xo >= W) continue;
                            const double *gp = dy + ((((long)n * D + zo) * H + yo) * W + xo) * cout;
                            for (int co = 0; co < cout; ++co) acc += w[((long)co * 27 + t) * cin + ci] * gp[co];
                        }
                        dx[((((long)n * D + z) * H + yy) * W + xx) * cin + ci] = acc;
                    }
}

/* Weight and bias gradients: dw[co][t][ci] = sum_v dy[v][co] x[v + off(t)][ci],
 * db[co] = sum_v dy[v][co] (overwritten). */
void orc_conv3d_wgrad(const double *x, const double *dy, int N, int D, int H, int W, int cin,
                      int cout, double *dw, double *db)
{
#pragma omp parallel for schedule(static)
    for (int co = 0; co < cout; ++co) {
        double bsum = 0.0;
        for (long v = 0; v < (long)N * D * H * W; ++v) bsum += dy[v * cout + co];
        db[co] = bsum;
        for (int t = 0; t < 27; ++t)
            for (int ci = 0; ci < cin; ++ci) {
                double acc = 0.0;
                for (int n = 0; n < N; ++n)
                    for (int z = 0; z < D; ++z)
                        for (int yy = 0; yy < H; ++yy)
                            for (int xx = 0; xx < W; ++xx) {
                                int zi = z + t / 9 - 1, yi = yy + (t / 3) % 3 - 1, xi = xx + t % 3 - 1;
                                if (zi < 0 || zi >= D || yi < 0 || yi >= H || xi < 0 || xi >= W) continue;
                                acc += dy[((((long)n * D + z) * H + yy) * W + xx) * cout + co] *
                                       x[((((long)n * D + zi) * H + yi) * W + xi) * cin + ci];
                            }
                dw[((long)co * 27 + t) * cin + ci] = acc;
            }
    }
}
