/*
 * FP64 CPU oracle for 3D degridding (arXiv:2102.12739) -- TEST INFRASTRUCTURE.
 *
 * This file is the plain, slow, obviously correct statement of what the
 * degridding path computes.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load it; the library never does.  It shares
 * no code, header, table or constant with the CUDA implementation.
 *
 * Every function follows the paper's Section "Implementation":
 *   - inputs: oversampled GCF tables G_uv (support 8x8, separable here as
 *     g(a) g(b)) and G_w (support 4), a stack of S subgrids and, per subgrid,
 *     a list of visibility coordinates [u, v, w];
 *   - per visibility two sets of coordinates: the subgrid point g = [x, y, z]
 *     where the footprint starts, and the row of each GCF table;
 *   - the degridded visibility is the sum of the subgrid samples of the
 *     footprint weighted by G_uv times G_w.
 * The paper leaves the rounding and orientation details open; the readings
 * taken here are:
 *   - coordinates are in subgrid pixels, origin at element (0,0,0);
 *   - p = rint(q * O) (nearest, ties to even) with O a power of two, so q*O
 *     is exact; i = floor(p / O); f = p - i*O; start = i - W/2 + 1;
 *   - table row f, column k holds the kernel at offset (k - W/2 + 1) - f/O;
 *   - subgrid layout is C-order [S][ny][nx][nz] with y <-> v, x <-> u,
 *     z <-> w, complex values stored as (re, im) pairs;
 *   - a visibility is valid when q is finite, |q*O| < 2^62 and
 *     0 <= start <= n - W on all three axes; an invalid visibility yields 0
 *     and is counted;
 *   - no conjugation and no phase term: V is a real-weighted sum.
 * All arithmetic is double precision; compile without -ffast-math and with
 * -ffp-contract=off so that x86-64 and AArch64 builds agree bit for bit.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* One axis: snap coordinate q to the oversampled grid (Section
 * "Implementation": the start point of the footprint and the location of
 * the GCF weights).  Returns 1 and sets *start, *frac when the footprint of
 * support W lies inside [0, n); returns 0 otherwise. */
static int snap_axis(double q, int W, int O, int n, long long *start, long long *frac)
{
    if (!isfinite(q))
        return 0;
    double qo = q * (double)O;               /* exact: O = 2^k */
    if (fabs(qo) >= 0x1p62)
        return 0;
    long long p = llrint(qo);                /* nearest, ties to even */
    long long i = p / O;                     /* C truncates toward zero ... */
    if (p % O != 0 && p < 0)
        i -= 1;                              /* ... so fix up to floor */
    long long f = p - i * O;
    long long s = i - W / 2 + 1;
    *start = s;
    *frac = f;
    return s >= 0 && s <= (long long)n - W;
}

typedef struct {
    long long x0, y0, z0, fu, fv, fw;
} coords_t;

static int visibility_coords(const double *q, int nx, int ny, int nz,
                             int uv_support, int uv_oversample,
                             int w_support, int w_oversample, coords_t *c)
{
    int ok_u = snap_axis(q[0], uv_support, uv_oversample, nx, &c->x0, &c->fu);
    int ok_v = snap_axis(q[1], uv_support, uv_oversample, ny, &c->y0, &c->fv);
    int ok_w = snap_axis(q[2], w_support, w_oversample, nz, &c->z0, &c->fw);
    return ok_u && ok_v && ok_w;
}

static int offsets_ok(int n_subgrids, const int64_t *vis_offsets, int64_t n_vis)
{
    if (vis_offsets[0] != 0 || vis_offsets[n_subgrids] != n_vis)
        return 0;
    for (int s = 0; s < n_subgrids; ++s)
        if (vis_offsets[s + 1] < vis_offsets[s])
            return 0;
    return 1;
}

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Per-visibility coordinates (x0, y0, z0, fu, fv, fw) as int32 [n][6];
 * invalid visibilities get all six set to -1.  Returns the invalid count. */
int64_t oracle_coords(int nx, int ny, int nz, int uv_support, int uv_oversample,
                      int w_support, int w_oversample, const double *uvw,
                      int64_t n_vis, int32_t *coords_out)
{
    int64_t bad = 0;
#pragma omp parallel for reduction(+ : bad) schedule(static)
    for (int64_t i = 0; i < n_vis; ++i) {
        coords_t c;
        int32_t *o = coords_out + 6 * i;
        if (visibility_coords(uvw + 3 * i, nx, ny, nz, uv_support, uv_oversample,
                              w_support, w_oversample, &c)) {
            o[0] = (int32_t)c.x0; o[1] = (int32_t)c.y0; o[2] = (int32_t)c.z0;
            o[3] = (int32_t)c.fu; o[4] = (int32_t)c.fv; o[5] = (int32_t)c.fw;
        } else {
            for (int k = 0; k < 6; ++k)
                o[k] = -1;
            bad += 1;
        }
    }
    return bad;
}

/* Degridding: vis_out[i] = sum_b sum_a sum_c g_uv[fv][b] g_uv[fu][a]
 * g_w[fw][c] * s[y0+b][x0+a][z0+c] for every visibility i of subgrid s.
 * subgrids: double [S][ny][nx][nz][2]; vis_out: double [n][2].
 * Returns the number of invalid visibilities, or -1 for bad offsets. */
int64_t oracle_degrid(int nx, int ny, int nz,
                      const double *g_uv, int uv_support, int uv_oversample,
                      const double *g_w, int w_support, int w_oversample,
                      int n_subgrids, const double *subgrids,
                      const double *uvw, const int64_t *vis_offsets,
                      int64_t n_vis, double *vis_out)
{
    if (!offsets_ok(n_subgrids, vis_offsets, n_vis))
        return -1;
    const int64_t plane = (int64_t)ny * nx * nz;
    int64_t bad = 0;
    for (int s = 0; s < n_subgrids; ++s) {
        const double *sg = subgrids + 2 * plane * s;
        const int64_t lo = vis_offsets[s], hi = vis_offsets[s + 1];
#pragma omp parallel for reduction(+ : bad) schedule(static)
        for (int64_t i = lo; i < hi; ++i) {
            coords_t c;
            double re = 0.0, im = 0.0;
            if (visibility_coords(uvw + 3 * i, nx, ny, nz, uv_support, uv_oversample,
                                  w_support, w_oversample, &c)) {
                const double *gu = g_uv + c.fu * uv_support;
                const double *gv = g_uv + c.fv * uv_support;
                const double *gw = g_w + c.fw * w_support;
                for (int b = 0; b < uv_support; ++b)
                    for (int a = 0; a < uv_support; ++a)
                        for (int k = 0; k < w_support; ++k) {
                            double w = gv[b] * gu[a] * gw[k];
                            int64_t e = ((c.y0 + b) * nx + (c.x0 + a)) * nz + (c.z0 + k);
                            re += w * sg[2 * e];
                            im += w * sg[2 * e + 1];
                        }
            } else {
                bad += 1;
            }
            vis_out[2 * i] = re;
            vis_out[2 * i + 1] = im;
        }
    }
    return bad;
}

/* Degridding with a non-separable G_uv.  The paper states G_uv as a kernel of
 * support 8 x 8 (Section "Implementation"); the separable table above is the
 * special case G_uv(a, b) = g(a) g(b).  Here the oversampled table holds one
 * W x W weight block per pair of oversampled offsets:
 *   vis_out[i] = sum_b sum_a sum_c G[fv][fu][b][a] g_w[fw][c] s[y0+b][x0+a][z0+c]
 * with g_uv2: double [O][O][W][W] indexed [fv][fu][b][a] (b along v / y, a
 * along u / x), O = uv_oversample.  Coordinates, validity and the w table are
 * exactly those of oracle_degrid.  Returns the invalid count, -1 for bad
 * offsets. */
int64_t oracle_degrid_2d(int nx, int ny, int nz,
                         const double *g_uv2, int uv_support, int uv_oversample,
                         const double *g_w, int w_support, int w_oversample,
                         int n_subgrids, const double *subgrids,
                         const double *uvw, const int64_t *vis_offsets,
                         int64_t n_vis, double *vis_out)
{
    if (!offsets_ok(n_subgrids, vis_offsets, n_vis))
        return -1;
    const int64_t plane = (int64_t)ny * nx * nz;
    const int64_t block = (int64_t)uv_support * uv_support;
    int64_t bad = 0;
    for (int s = 0; s < n_subgrids; ++s) {
        const double *sg = subgrids + 2 * plane * s;
        const int64_t lo = vis_offsets[s], hi = vis_offsets[s + 1];
#pragma omp parallel for reduction(+ : bad) schedule(static)
        for (int64_t i = lo; i < hi; ++i) {
            coords_t c;
            double re = 0.0, im = 0.0;
            if (visibility_coords(uvw + 3 * i, nx, ny, nz, uv_support, uv_oversample,
                                  w_support, w_oversample, &c)) {
                const double *G = g_uv2 + ((int64_t)c.fv * uv_oversample + c.fu) * block;
                const double *gw = g_w + c.fw * w_support;
                for (int b = 0; b < uv_support; ++b)
                    for (int a = 0; a < uv_support; ++a)
                        for (int k = 0; k < w_support; ++k) {
                            double w = G[b * uv_support + a] * gw[k];
                            int64_t e = ((c.y0 + b) * nx + (c.x0 + a)) * nz + (c.z0 + k);
                            re += w * sg[2 * e];
                            im += w * sg[2 * e + 1];
                        }
            } else {
                bad += 1;
            }
            vis_out[2 * i] = re;
            vis_out[2 * i + 1] = im;
        }
    }
    return bad;
}

/* Adjoint (gridding): grid_out[s][y0+b][x0+a][z0+c] += weight * vis_in[i],
 * the transpose of oracle_degrid (real weights, so no conjugation).
 * grid_out: double [S][ny][nx][nz][2], zeroed first unless accumulate.
 * Visibilities of one subgrid are added serially in list order; subgrids
 * are independent.  Returns the invalid count, or -1 for bad offsets. */
int64_t oracle_grid(int nx, int ny, int nz,
                    const double *g_uv, int uv_support, int uv_oversample,
                    const double *g_w, int w_support, int w_oversample,
                    int n_subgrids, const double *uvw, const int64_t *vis_offsets,
                    int64_t n_vis, const double *vis_in, double *grid_out,
                    int accumulate)
{
    if (!offsets_ok(n_subgrids, vis_offsets, n_vis))
        return -1;
    const int64_t plane = (int64_t)ny * nx * nz;
    if (!accumulate)
        memset(grid_out, 0, sizeof(double) * 2 * plane * n_subgrids);
    int64_t bad = 0;
#pragma omp parallel for reduction(+ : bad) schedule(dynamic, 1)
    for (int s = 0; s < n_subgrids; ++s) {
        double *sg = grid_out + 2 * plane * s;
        for (int64_t i = vis_offsets[s]; i < vis_offsets[s + 1]; ++i) {
            coords_t c;
            if (!visibility_coords(uvw + 3 * i, nx, ny, nz, uv_support, uv_oversample,
                                   w_support, w_oversample, &c)) {
                bad += 1;
                continue;
            }
            const double *gu = g_uv + c.fu * uv_support;
            const double *gv = g_uv + c.fv * uv_support;
            const double *gw = g_w + c.fw * w_support;
            const double yre = vis_in[2 * i], yim = vis_in[2 * i + 1];
            for (int b = 0; b < uv_support; ++b)
                for (int a = 0; a < uv_support; ++a)
                    for (int k = 0; k < w_support; ++k) {
                        double w = gv[b] * gu[a] * gw[k];
                        int64_t e = ((c.y0 + b) * nx + (c.x0 + a)) * nz + (c.z0 + k);
                        sg[2 * e] += w * yre;
                        sg[2 * e + 1] += w * yim;
                    }
        }
    }
    return bad;
}

/* Adjoint of oracle_degrid_2d (gridding with a non-separable G_uv):
 * grid_out[s][y0+b][x0+a][z0+c] += G[fv][fu][b][a] g_w[fw][c] vis_in[i], with
 * g_uv2 [O][O][W][W] indexed [fv][fu][b][a] as in oracle_degrid_2d. */
int64_t oracle_grid_2d(int nx, int ny, int nz,
                       const double *g_uv2, int uv_support, int uv_oversample,
                       const double *g_w, int w_support, int w_oversample,
                       int n_subgrids, const double *uvw, const int64_t *vis_offsets,
                       int64_t n_vis, const double *vis_in, double *grid_out,
                       int accumulate)
{
    if (!offsets_ok(n_subgrids, vis_offsets, n_vis))
        return -1;
    const int64_t plane = (int64_t)ny * nx * nz;
    const int64_t block = (int64_t)uv_support * uv_support;
    if (!accumulate)
        memset(grid_out, 0, sizeof(double) * 2 * plane * n_subgrids);
    int64_t bad = 0;
#pragma omp parallel for reduction(+ : bad) schedule(dynamic, 1)
    for (int s = 0; s < n_subgrids; ++s) {
        double *sg = grid_out + 2 * plane * s;
        for (int64_t i = vis_offsets[s]; i < vis_offsets[s + 1]; ++i) {
            coords_t c;
            if (!visibility_coords(uvw + 3 * i, nx, ny, nz, uv_support, uv_oversample,
                                   w_support, w_oversample, &c)) {
                bad += 1;
                continue;
            }
            const double *G = g_uv2 + ((int64_t)c.fv * uv_oversample + c.fu) * block;
            const double *gw = g_w + c.fw * w_support;
            const double yre = vis_in[2 * i], yim = vis_in[2 * i + 1];
            for (int b = 0; b < uv_support; ++b)
                for (int a = 0; a < uv_support; ++a)
                    for (int k = 0; k < w_support; ++k) {
                        double w = G[b * uv_support + a] * gw[k];
                        int64_t e = ((c.y0 + b) * nx + (c.x0 + a)) * nz + (c.z0 + k);
                        sg[2 * e] += w * yre;
                        sg[2 * e + 1] += w * yim;
                    }
        }
    }
    return bad;
}

/* Number of distinct subgrid elements touched by the footprints of each
 * subgrid's valid visibilities (the compulsory subgrid bytes of a
 * degridding pass are this count times the element size). */
int64_t oracle_touched(int nx, int ny, int nz, int uv_support, int uv_oversample,
                       int w_support, int w_oversample, int n_subgrids,
                       const double *uvw, const int64_t *vis_offsets, int64_t n_vis,
                       int64_t *touched_out)
{
    if (!offsets_ok(n_subgrids, vis_offsets, n_vis))
        return -1;
    const int64_t plane = (int64_t)ny * nx * nz;
    int64_t total = 0;
#pragma omp parallel for reduction(+ : total) schedule(dynamic, 1)
    for (int s = 0; s < n_subgrids; ++s) {
        unsigned char *mark = (unsigned char *)calloc((size_t)plane, 1);
        int64_t count = 0;
        for (int64_t i = vis_offsets[s]; mark && i < vis_offsets[s + 1]; ++i) {
            coords_t c;
            if (!visibility_coords(uvw + 3 * i, nx, ny, nz, uv_support, uv_oversample,
                                   w_support, w_oversample, &c))
                continue;
            for (int b = 0; b < uv_support; ++b)
                for (int a = 0; a < uv_support; ++a)
                    for (int k = 0; k < w_support; ++k) {
                        int64_t e = ((c.y0 + b) * nx + (c.x0 + a)) * nz + (c.z0 + k);
                        count += !mark[e];
                        mark[e] = 1;
                    }
        }
        free(mark);
        touched_out[s] = count;
        total += count;
    }
    return total;
}
