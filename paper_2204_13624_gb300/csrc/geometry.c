/*
 * geometry.c -- host helper for the synthetic microstructure generator
 * (paper_2204_13624_gb300/microstructure.py).  Input data only: it classifies
 * voxels against periodic balls and integrates each cut voxel's inclusion
 * volume fraction; it holds none of the homogenization method.
 *
 * Volume of a ball |x| < R inside a box: integral over x of the area of the
 * disc of radius rho(x) = sqrt(R^2 - x^2) clipped to the (y, z) rectangle.
 * The clipped area has a closed form (inclusion-exclusion of "disc below and
 * left of a point" areas); it is smooth between the x where rho(x) equals the
 * distance to an edge or a corner, so each such piece is integrated with
 * Gauss-Legendre after the substitution x = a + (b - a)(3t^2 - 2t^3), which
 * flattens the (x - x*)^{1/2, 3/2} behaviour at the piece ends.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static double S_anti(double Y, double rho)
{
    if (rho <= 0.0) return 0.0;
    if (Y < -rho) Y = -rho;
    if (Y > rho) Y = rho;
    double s = sqrt(fmax(rho * rho - Y * Y, 0.0));
    double t = Y / rho;
    if (t > 1.0) t = 1.0;
    if (t < -1.0) t = -1.0;
    return 0.5 * (Y * s + rho * rho * asin(t));
}

/* area of the disc |(Y,Z)| < rho intersected with {Y <= y, Z <= z} */
static double quad_area(double y, double z, double rho)
{
    if (rho <= 0.0 || z <= -rho || y <= -rho) return 0.0;
    double yp = y > rho ? rho : y;
    double S0 = S_anti(-rho, rho);
    if (z >= rho) return 2.0 * (S_anti(yp, rho) - S0);
    double w = sqrt(fmax(rho * rho - z * z, 0.0));
    double out = 0.0;
    if (z >= 0.0) {
        double b1 = yp < -w ? yp : -w;
        if (b1 > -rho) out += 2.0 * (S_anti(b1, rho) - S0);
    }
    double b2 = yp < w ? yp : w;
    if (b2 > -w) out += z * (b2 + w) + S_anti(b2, rho) - S_anti(-w, rho);
    if (z >= 0.0 && yp > w) out += 2.0 * (S_anti(yp, rho) - S_anti(w, rho));
    return out;
}

double geo_disc_rect_area(double rho, double y0, double y1, double z0, double z1)
{
    return quad_area(y1, z1, rho) - quad_area(y0, z1, rho) - quad_area(y1, z0, rho) + quad_area(y0, z0, rho);
}

static int cmp_d(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

double geo_ball_box_volume(double R, double x0, double x1, double y0, double y1, double z0, double z1, int ng,
                           const double* gx, const double* gw)
{
    double ds[8] = {fabs(y0), fabs(y1), fabs(z0), fabs(z1), hypot(y0, z0), hypot(y0, z1), hypot(y1, z0),
                    hypot(y1, z1)};
    double bp[20];
    int nb = 0;
    bp[nb++] = x0;
    bp[nb++] = x1;
    if (-R > x0 && -R < x1) bp[nb++] = -R;
    if (R > x0 && R < x1) bp[nb++] = R;
    for (int q = 0; q < 8; q++) {
        if (ds[q] >= R) continue;
        double h = sqrt(R * R - ds[q] * ds[q]);
        if (h > x0 && h < x1) bp[nb++] = h;
        if (-h > x0 && -h < x1) bp[nb++] = -h;
    }
    qsort(bp, (size_t)nb, sizeof(double), cmp_d);
    double vol = 0.0;
    for (int p = 0; p + 1 < nb; p++) {
        double a = bp[p], b = bp[p + 1];
        if (!(b > a)) continue;
        for (int g = 0; g < ng; g++) {
            double t = 0.5 * (gx[g] + 1.0), wt = 0.5 * gw[g];
            double u = 3 * t * t - 2 * t * t * t, du = 6 * t - 6 * t * t;
            double x = a + (b - a) * u;
            double rho = sqrt(fmax(R * R - x * x, 0.0));
            vol += geo_disc_rect_area(rho, y0, y1, z0, z1) * (b - a) * du * wt;
        }
    }
    return vol;
}

/* Voxel index range [i0, i1] per axis that can meet a ball of radius R at
 * centre c (coordinates in [-l/2, l/2)). */
static void ball_range(const int n[3], const double l[3], const double* c, double R, int lo[3], int hi[3])
{
    for (int ax = 0; ax < 3; ax++) {
        double h = l[ax] / n[ax];
        lo[ax] = (int)floor((c[ax] - R + 0.5 * l[ax]) / h) - 1;
        hi[ax] = (int)floor((c[ax] + R + 0.5 * l[ax]) / h) + 1;
    }
}

static int classify(const int n[3], const double l[3], const double* c, double R, int i, int j, int k, double lo[3],
                    double hi[3])
{
    int ijk[3] = {i, j, k};
    double near2 = 0.0, far2 = 0.0;
    for (int ax = 0; ax < 3; ax++) {
        double h = l[ax] / n[ax];
        lo[ax] = -0.5 * l[ax] + h * ijk[ax] - c[ax];
        hi[ax] = lo[ax] + h;
        double nr = lo[ax] > 0 ? lo[ax] : (hi[ax] < 0 ? hi[ax] : 0.0);
        double fr = fmax(fabs(lo[ax]), fabs(hi[ax]));
        near2 += nr * nr;
        far2 += fr * fr;
    }
    if (far2 <= R * R) return 1; /* inside */
    if (near2 < R * R) return 2; /* cut */
    return 0;
}

static int64_t lin(const int n[3], int i, int j, int k)
{
    i = ((i % n[0]) + n[0]) % n[0];
    j = ((j % n[1]) + n[1]) % n[1];
    k = ((k % n[2]) + n[2]) % n[2];
    return (int64_t)i + (int64_t)n[0] * ((int64_t)j + (int64_t)n[1] * k);
}

/* Count cut voxels per ball (counts[b]); mark inside voxels in phase (=1). */
void geo_balls_count(const int n[3], const double l[3], int nballs, const double* cen, double R, uint8_t* phase,
                     int64_t* counts)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < nballs; b++) {
        int lo[3], hi[3];
        ball_range(n, l, cen + 3 * b, R, lo, hi);
        int64_t cnt = 0;
        double blo[3], bhi[3];
        for (int k = lo[2]; k <= hi[2]; k++)
            for (int j = lo[1]; j <= hi[1]; j++)
                for (int i = lo[0]; i <= hi[0]; i++) {
                    int cl = classify(n, l, cen + 3 * b, R, i, j, k, blo, bhi);
                    if (cl == 1) phase[lin(n, i, j, k)] = 1;
                    else if (cl == 2) cnt++;
                }
        counts[b] = cnt;
    }
}

/* Fill cut voxels of every ball at offsets[b]: index, volume fraction, normal
 * (unit vector from the ball centre to the voxel centre). */
void geo_balls_fill(const int n[3], const double l[3], int nballs, const double* cen, double R,
                    const int64_t* offsets, int ng, const double* gx, const double* gw, int64_t* idx, double* frac,
                    double* nrm)
{
    double hv = (l[0] / n[0]) * (l[1] / n[1]) * (l[2] / n[2]);
#pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < nballs; b++) {
        int lo[3], hi[3];
        ball_range(n, l, cen + 3 * b, R, lo, hi);
        int64_t o = offsets[b];
        double blo[3], bhi[3];
        for (int k = lo[2]; k <= hi[2]; k++)
            for (int j = lo[1]; j <= hi[1]; j++)
                for (int i = lo[0]; i <= hi[0]; i++) {
                    if (classify(n, l, cen + 3 * b, R, i, j, k, blo, bhi) != 2) continue;
                    idx[o] = lin(n, i, j, k);
                    frac[o] = geo_ball_box_volume(R, blo[0], bhi[0], blo[1], bhi[1], blo[2], bhi[2], ng, gx, gw) / hv;
                    double cx = 0.5 * (blo[0] + bhi[0]), cy = 0.5 * (blo[1] + bhi[1]), cz = 0.5 * (blo[2] + bhi[2]);
                    double nn = sqrt(cx * cx + cy * cy + cz * cz);
                    nrm[3 * o] = cx / nn;
                    nrm[3 * o + 1] = cy / nn;
                    nrm[3 * o + 2] = cz / nn;
                    o++;
                }
    }
}
