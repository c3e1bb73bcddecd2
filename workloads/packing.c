/*
 * packing.c -- seeded synthetic sphere packings: geometric overlap removal.
 *
 * Input generation only.  Spheres start at seeded random positions in a
 * periodic cube; their radii are scaled up in stages from `scale0` to 1 and,
 * at each stage, overlapping pairs are pushed apart along their centre line by
 * half of their overlap each (Jacobi sweeps over a cell list) until the
 * largest overlap falls below the stage tolerance.  The displacement of each
 * sphere is gathered from its neighbours in a fixed order, so the result is
 * independent of the number of threads.  This is a geometric projection, not
 * a force model.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline double wrap1(double v, double L) {
  while (v >= L) v -= L;
  while (v < 0.0) v += L;
  return v;
}

static inline double min_img(double d, double L) {
  return d - L * floor(d / L + 0.5);
}

/* Returns the number of sweeps done; stats = {max overlap / a_min, sweeps}. */
int64_t wl_relax(int64_t N, const double* radii, const double* L, double* x,
                 double scale0, int32_t nstages, int32_t max_sweeps,
                 double tol, double* stats) {
  if (N <= 0) return 0;
  double amin = radii[0], amax = radii[0];
  for (int64_t i = 0; i < N; ++i) {
    if (radii[i] < amin) amin = radii[i];
    if (radii[i] > amax) amax = radii[i];
  }
  int32_t nc[3];
  for (int d = 0; d < 3; ++d) {
    nc[d] = (int32_t)floor(L[d] / (2.0 * amax * 1.0000001));
    if (nc[d] < 3) nc[d] = 1; /* small boxes: a single cell, brute force */
  }
  int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
  int64_t* start = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
  int64_t* cell = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
  double* disp = (double*)malloc(sizeof(double) * 3 * (size_t)N);
  double* ovl = (double*)malloc(sizeof(double) * (size_t)N);
  if (!start || !order || !cell || !disp || !ovl) {
    free(start); free(order); free(cell); free(disp); free(ovl);
    return -1;
  }
  int64_t sweeps = 0;
  double worst = 0.0;
  for (int32_t stage = 0; stage <= nstages; ++stage) {
    double scale = nstages > 0
                       ? scale0 + (1.0 - scale0) * (double)stage / (double)nstages
                       : 1.0;
    double stage_tol = stage == nstages ? tol : 1e-2;
    int32_t limit = stage == nstages ? max_sweeps : max_sweeps / 4 + 1;
    for (int32_t it = 0; it < limit; ++it) {
      /* counting sort of spheres into cells */
      memset(start, 0, sizeof(int64_t) * ((size_t)ncell + 1));
      for (int64_t i = 0; i < N; ++i) {
        int64_t c[3];
        for (int d = 0; d < 3; ++d) {
          c[d] = (int64_t)floor(x[3 * i + d] / L[d] * nc[d]);
          if (c[d] >= nc[d]) c[d] = nc[d] - 1;
          if (c[d] < 0) c[d] = 0;
        }
        cell[i] = (c[2] * nc[1] + c[1]) * nc[0] + c[0];
        start[cell[i] + 1] += 1;
      }
      for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
      {
        int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
        memcpy(fill, start, sizeof(int64_t) * (size_t)ncell);
        for (int64_t i = 0; i < N; ++i) order[fill[cell[i]]++] = i;
        free(fill);
      }
      /* gather displacements */
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < N; ++i) {
        double xi0 = x[3 * i], xi1 = x[3 * i + 1], xi2 = x[3 * i + 2];
        double ai = radii[i] * scale;
        double dx0 = 0.0, dx1 = 0.0, dx2 = 0.0, mo = 0.0;
        int64_t ci = cell[i];
        int64_t cx = ci % nc[0], cy = (ci / nc[0]) % nc[1], cz = ci / ((int64_t)nc[0] * nc[1]);
        int32_t rx = nc[0] >= 3 ? 1 : 0, ry = nc[1] >= 3 ? 1 : 0, rz = nc[2] >= 3 ? 1 : 0;
        for (int32_t oz = -rz; oz <= rz; ++oz)
          for (int32_t oy = -ry; oy <= ry; ++oy)
            for (int32_t ox = -rx; ox <= rx; ++ox) {
              int64_t qx = (cx + ox + nc[0]) % nc[0];
              int64_t qy = (cy + oy + nc[1]) % nc[1];
              int64_t qz = (cz + oz + nc[2]) % nc[2];
              int64_t q = (qz * nc[1] + qy) * nc[0] + qx;
              for (int64_t s = start[q]; s < start[q + 1]; ++s) {
                int64_t j = order[s];
                if (j == i) continue;
                double r0 = min_img(x[3 * j] - xi0, L[0]);
                double r1 = min_img(x[3 * j + 1] - xi1, L[1]);
                double r2 = min_img(x[3 * j + 2] - xi2, L[2]);
                double d2 = r0 * r0 + r1 * r1 + r2 * r2;
                double S = ai + radii[j] * scale;
                if (d2 >= S * S) continue;
                double d = sqrt(d2);
                double ov = S - d;
                if (ov > mo) mo = ov;
                if (d > 0.0) {
                  double f = 0.5 * ov / d;
                  dx0 -= f * r0; dx1 -= f * r1; dx2 -= f * r2;
                } else {
                  dx0 -= 0.5 * ov; /* coincident centres: separate along x */
                }
              }
            }
        disp[3 * i] = dx0; disp[3 * i + 1] = dx1; disp[3 * i + 2] = dx2;
        ovl[i] = mo;
      }
      worst = 0.0;
      for (int64_t i = 0; i < N; ++i) if (ovl[i] > worst) worst = ovl[i];
      sweeps++;
      if (worst <= stage_tol * amin) break;
      for (int64_t i = 0; i < N; ++i)
        for (int d = 0; d < 3; ++d)
          x[3 * i + d] = wrap1(x[3 * i + d] + disp[3 * i + d], L[d]);
    }
  }
  if (stats) { stats[0] = worst / amin; stats[1] = (double)sweeps; }
  free(start); free(order); free(cell); free(disp); free(ovl);
  return sweeps;
}
