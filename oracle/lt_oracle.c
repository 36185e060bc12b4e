/*
 * CPU ORACLE — test infrastructure only.
 *
 * Plain, slow, obviously correct loops that evaluate the definitions the
 * method rests on. Only the tests, the smoke check and the benchmark's CPU
 * baseline may load this code; the library path never does. It shares no
 * code, header, table or helper with the CUDA sources.
 *
 * Definitions (Sec. 1 and Sec. 4 of the paper: local thickness is the radius
 * of the largest inscribed circle/sphere containing a point):
 *   foreground  F = {p : mask(p) != 0}; every point outside the array counts
 *               as background (the array is padded by one background layer).
 *   DT2(p)      = min over background b of |p - b|^2 (0 on background).
 *   LT2(x)      = max { DT2(c) : label(c) = label(x) != 0, |x - c|^2 <= DT2(c) }
 *               for labelled x, 0 elsewhere.
 * The radius of the largest ball centred at c inside the object is sqrt(DT2(c));
 * a ball is inclusive (|x - c|^2 <= r^2).
 *
 * Layout: C order [z][y][x], x fastest. ndim == 2 uses nz == 1 and no z axis.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int64_t sq(int64_t v) { return v * v; }

static int64_t isqrt64(int64_t v) {
  if (v <= 0) return 0;
  int64_t r = (int64_t)sqrt((double)v);
  while (r * r > v) --r;
  while ((r + 1) * (r + 1) <= v) ++r;
  return r;
}

/* DT2 at one voxel: min over the padding layer and over in-array background
 * voxels, visited in Chebyshev shells of growing radius k; a background voxel
 * at Chebyshev distance >= k is at squared distance >= k^2, so the search
 * stops once k^2 reaches the best value found. */
static uint32_t dt2_point(const uint8_t* mask, int64_t nx, int64_t ny, int64_t nz, int ndim,
                          int64_t x, int64_t y, int64_t z) {
  if (!mask[(z * ny + y) * nx + x]) return 0;
  int64_t best = sq(x + 1);
  if (sq(nx - x) < best) best = sq(nx - x);
  if (sq(y + 1) < best) best = sq(y + 1);
  if (sq(ny - y) < best) best = sq(ny - y);
  if (ndim == 3) {
    if (sq(z + 1) < best) best = sq(z + 1);
    if (sq(nz - z) < best) best = sq(nz - z);
  }
  for (int64_t k = 1; k * k < best; ++k) {
    int64_t zr = ndim == 3 ? k : 0;
    for (int64_t dz = -zr; dz <= zr; ++dz) {
      int64_t zz = z + dz;
      if (zz < 0 || zz >= nz) continue;
      for (int64_t dy = -k; dy <= k; ++dy) {
        int64_t yy = y + dy;
        if (yy < 0 || yy >= ny) continue;
        int full = (dz == k || dz == -k) || (dy == k || dy == -k);
        for (int64_t dx = -k; dx <= k; dx += full ? 1 : 2 * k) {
          int64_t xx = x + dx;
          if (xx < 0 || xx >= nx) continue;
          if (!mask[(zz * ny + yy) * nx + xx]) {
            int64_t d = dz * dz + dy * dy + dx * dx;
            if (d < best) best = d;
          }
        }
      }
    }
  }
  return (uint32_t)best;
}

/* Squared Euclidean distance transform of the whole array. */
void oracle_dt2(const uint8_t* mask, int64_t nx, int64_t ny, int64_t nz, int ndim, uint32_t* out) {
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
  for (int64_t z = 0; z < nz; ++z)
    for (int64_t y = 0; y < ny; ++y)
      for (int64_t x = 0; x < nx; ++x) out[(z * ny + y) * nx + x] = dt2_point(mask, nx, ny, nz, ndim, x, y, z);
}

/* DT2 at a list of voxels (linear indices). */
void oracle_dt2_at(const uint8_t* mask, int64_t nx, int64_t ny, int64_t nz, int ndim,
                   const int64_t* idx, int64_t n, uint32_t* out) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) {
    int64_t v = idx[i], x = v % nx, y = (v / nx) % ny, z = v / (nx * ny);
    out[i] = dt2_point(mask, nx, ny, nz, ndim, x, y, z);
  }
}

/* Local thickness by its definition: every labelled foreground voxel c is a
 * centre and raises LT2 to DT2(c) on every same-label voxel of its ball. No
 * centre is skipped. Threads own disjoint slabs of the output (along z in 3D,
 * along y in 2D), so there are no write races. */
void oracle_lt2(const uint32_t* dt2, const uint32_t* labels, int64_t nx, int64_t ny, int64_t nz,
                int ndim, uint32_t* out) {
  int64_t n = nx * ny * nz;
  memset(out, 0, (size_t)n * sizeof(uint32_t));
  uint32_t maxr2 = 0;
  for (int64_t i = 0; i < n; ++i)
    if (labels[i] && dt2[i] > maxr2) maxr2 = dt2[i];
  const int64_t Rmax = isqrt64(maxr2);
  const int64_t nslab = ndim == 3 ? nz : ny; /* slab axis */
  const int64_t chunk = 4;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t s0 = 0; s0 < nslab; s0 += chunk) {
    int64_t s1 = s0 + chunk < nslab ? s0 + chunk : nslab;
    int64_t c0 = s0 - Rmax < 0 ? 0 : s0 - Rmax, c1 = s1 + Rmax > nslab ? nslab : s1 + Rmax;
    /* centres whose slab coordinate lies in [c0, c1) */
    int64_t first = ndim == 3 ? c0 * nx * ny : c0 * nx, last = ndim == 3 ? c1 * nx * ny : c1 * nx;
    for (int64_t c = first; c < last; ++c) {
      uint32_t l = labels[c];
      if (!l || !dt2[c]) continue;
      int64_t r2 = dt2[c], R = isqrt64(r2);
      int64_t cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
      int64_t zlo = ndim == 3 ? cz - R : 0, zhi = ndim == 3 ? cz + R : 0;
      int64_t ylo = cy - R, yhi = cy + R;
      if (ndim == 3) { if (zlo < s0) zlo = s0; if (zhi > s1 - 1) zhi = s1 - 1; }
      else { if (ylo < s0) ylo = s0; if (yhi > s1 - 1) yhi = s1 - 1; }
      if (zlo < 0) zlo = 0;
      if (zhi > nz - 1) zhi = nz - 1;
      if (ylo < 0) ylo = 0;
      if (yhi > ny - 1) yhi = ny - 1;
      for (int64_t z = zlo; z <= zhi; ++z)
        for (int64_t y = ylo; y <= yhi; ++y) {
          int64_t rem = r2 - sq(z - cz) - sq(y - cy);
          if (rem < 0) continue;
          for (int64_t x = cx - R; x <= cx + R; ++x) {
            if (x < 0 || x >= nx) continue;
            if (sq(x - cx) > rem) continue;
            int64_t i = (z * ny + y) * nx + x;
            if (labels[i] == l && out[i] < (uint32_t)r2) out[i] = (uint32_t)r2;
          }
        }
    }
  }
}

/* Distance transform and local thickness of selected objects only, for
 * checking full-size volumes one object at a time. Object k is the list of
 * its voxels idx[off[k] .. off[k+1]) (all with the same label). Writes DT2 and
 * LT2 of those voxels in the same order. Uses the whole mask for DT2 and the
 * object's own voxels as centres and targets (same label). */
void oracle_objects(const uint8_t* mask, int64_t nx, int64_t ny, int64_t nz, int ndim,
                    const int64_t* idx, const int64_t* off, int64_t nobj, uint32_t* dt2_out,
                    uint32_t* lt2_out) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t k = 0; k < nobj; ++k) {
    int64_t b = off[k], e = off[k + 1];
    if (e <= b) continue;
    int64_t lo[3] = {INT64_MAX, INT64_MAX, INT64_MAX}, hi[3] = {-1, -1, -1};
    for (int64_t i = b; i < e; ++i) {
      int64_t v = idx[i], p[3] = {v % nx, (v / nx) % ny, v / (nx * ny)};
      dt2_out[i] = dt2_point(mask, nx, ny, nz, ndim, p[0], p[1], p[2]);
      for (int a = 0; a < 3; ++a) {
        if (p[a] < lo[a]) lo[a] = p[a];
        if (p[a] > hi[a]) hi[a] = p[a];
      }
    }
    int64_t bx = hi[0] - lo[0] + 1, by = hi[1] - lo[1] + 1, bz = hi[2] - lo[2] + 1;
    uint8_t* in = (uint8_t*)calloc((size_t)(bx * by * bz), 1);
    uint32_t* lt = (uint32_t*)calloc((size_t)(bx * by * bz), sizeof(uint32_t));
    for (int64_t i = b; i < e; ++i) {
      int64_t v = idx[i];
      int64_t x = v % nx - lo[0], y = (v / nx) % ny - lo[1], z = v / (nx * ny) - lo[2];
      in[(z * by + y) * bx + x] = 1;
    }
    for (int64_t i = b; i < e; ++i) {
      int64_t v = idx[i], r2 = dt2_out[i], R = isqrt64(r2);
      int64_t cx = v % nx - lo[0], cy = (v / nx) % ny - lo[1], cz = v / (nx * ny) - lo[2];
      for (int64_t z = cz - R; z <= cz + R; ++z) {
        if (z < 0 || z >= bz) continue;
        for (int64_t y = cy - R; y <= cy + R; ++y) {
          if (y < 0 || y >= by) continue;
          int64_t rem = r2 - sq(z - cz) - sq(y - cy);
          if (rem < 0) continue;
          for (int64_t x = cx - R; x <= cx + R; ++x) {
            if (x < 0 || x >= bx || sq(x - cx) > rem) continue;
            int64_t j = (z * by + y) * bx + x;
            if (in[j] && lt[j] < (uint32_t)r2) lt[j] = (uint32_t)r2;
          }
        }
      }
    }
    for (int64_t i = b; i < e; ++i) {
      int64_t v = idx[i];
      int64_t x = v % nx - lo[0], y = (v / nx) % ny - lo[1], z = v / (nx * ny) - lo[2];
      lt2_out[i] = lt[(z * by + y) * bx + x];
    }
    free(in);
    free(lt);
  }
}

/* ---------------------------------------------------------------- meshes
 * Surface area of an object's marching-tetrahedra isosurface, the "strict"
 * sphericity's area (Eq. 1 with a mesh area in place of S; the paper's
 * baseline meshes the mask with marching cubes, Sec. 5.2). The field is the
 * object's indicator (1 on its voxels, 0 elsewhere and outside the array)
 * sampled at voxel centres, optionally smoothed by a separable Gaussian of
 * standard deviation sigma voxels (truncated at 3 sigma; sigma = 0 keeps the
 * binary field). Every unit cube of the dual grid is split into the six
 * tetrahedra of the Kuhn subdivision (vertices 0, e_a, e_a + e_b,
 * e_a + e_b + e_c for each ordering (a, b, c) of the axes), which tile
 * space consistently across cubes. The level-0.5 surface crosses an edge
 * whose ends lie on either side at the linear-interpolation point; a
 * tetrahedron with one vertex apart contributes a triangle, one with two and
 * two a quadrilateral (two triangles). Object k is the voxel list
 * idx[off[k] .. off[k+1]). Output in FP64. */
/* adds triangle (a, b, c) to the totals, oriented with its normal pointing
 * away from `in` (a point on the inside): area, and the signed volume
 * a . (b x c) / 6 of the divergence theorem (global coordinates) */
static void add_tri(const double a[3], const double b[3], const double c[3], const double in[3],
                    double* area, double* vol) {
  double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
  double w[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
  *area += 0.5 * sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  double s = w[0] * (a[0] - in[0]) + w[1] * (a[1] - in[1]) + w[2] * (a[2] - in[2]);
  double det = a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
               a[2] * (b[0] * c[1] - b[1] * c[0]);
  *vol += (s >= 0.0 ? det : -det) / 6.0;
}

/* point where the field crosses 0.5 on the edge p-q (fp, fq on either side) */
static void crossing(const double p[3], const double q[3], double fp, double fq, double m[3]) {
  double t = (0.5 - fp) / (fq - fp);
  m[0] = p[0] + t * (q[0] - p[0]);
  m[1] = p[1] + t * (q[1] - p[1]);
  m[2] = p[2] + t * (q[2] - p[2]);
}

static void tet_surface(const double P[4][3], const double f[4], double* area, double* vol) {
  int inside[4], n_in = 0;
  for (int i = 0; i < 4; ++i) {
    inside[i] = f[i] > 0.5;
    n_in += inside[i];
  }
  if (n_in == 0 || n_in == 4) return;
  double cin[3] = {0.0, 0.0, 0.0};  /* centroid of the inside vertices */
  for (int i = 0; i < 4; ++i)
    if (inside[i])
      for (int a = 0; a < 3; ++a) cin[a] += P[i][a] / n_in;
  if (n_in == 1 || n_in == 3) {
    int odd = 0;
    for (int i = 0; i < 4; ++i)
      if (inside[i] == (n_in == 1)) odd = i;
    double m[3][3];
    int k = 0;
    for (int i = 0; i < 4; ++i)
      if (i != odd) crossing(P[odd], P[i], f[odd], f[i], m[k++]);
    add_tri(m[0], m[1], m[2], cin, area, vol);
    return;
  }
  int in[2], out[2], a = 0, b = 0;
  for (int i = 0; i < 4; ++i) {
    if (inside[i]) in[a++] = i;
    else out[b++] = i;
  }
  /* quadrilateral with corners on edges in0-out0, in0-out1, in1-out1, in1-out0 */
  double m00[3], m01[3], m11[3], m10[3];
  crossing(P[in[0]], P[out[0]], f[in[0]], f[out[0]], m00);
  crossing(P[in[0]], P[out[1]], f[in[0]], f[out[1]], m01);
  crossing(P[in[1]], P[out[1]], f[in[1]], f[out[1]], m11);
  crossing(P[in[1]], P[out[0]], f[in[1]], f[out[0]], m10);
  add_tri(m00, m01, m11, cin, area, vol);
  add_tri(m00, m11, m10, cin, area, vol);
}

/* separable Gaussian blur of a bx*by*bz field along one axis (in place) */
static void blur_axis(double* f, int64_t bx, int64_t by, int64_t bz, int axis, const double* w, int r,
                      double* tmp) {
  int64_t n[3] = {bx, by, bz}, st[3] = {1, bx, bx * by};
  int64_t len = n[axis], s = st[axis];
  int64_t o1 = axis == 0 ? 1 : 0, o2 = axis == 2 ? 1 : 2;
  for (int64_t i2 = 0; i2 < n[o2]; ++i2)
    for (int64_t i1 = 0; i1 < n[o1]; ++i1) {
      int64_t base = i1 * st[o1] + i2 * st[o2];
      for (int64_t i = 0; i < len; ++i) {
        double acc = 0.0;
        for (int k = -r; k <= r; ++k) {
          int64_t j = i + k;
          if (j >= 0 && j < len) acc += w[k + r] * f[base + j * s];
        }
        tmp[i] = acc;
      }
      for (int64_t i = 0; i < len; ++i) f[base + i * s] = tmp[i];
    }
}

void oracle_mesh_area(int64_t nx, int64_t ny, int64_t nz, const int64_t* idx, const int64_t* off,
                      int64_t nobj, double sigma, double* area_out, double* vol_out) {
  static const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  const int r = sigma > 0.0 ? (int)ceil(3.0 * sigma) : 0;
  double w[64];
  if (r > 0) {
    double z = 0.0;
    for (int k = -r; k <= r; ++k) z += (w[k + r] = exp(-0.5 * (double)(k * k) / (sigma * sigma)));
    for (int k = 0; k <= 2 * r; ++k) w[k] /= z;
  }
  (void)nz;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t k = 0; k < nobj; ++k) {
    int64_t b = off[k], e = off[k + 1];
    area_out[k] = 0.0;
    vol_out[k] = 0.0;
    if (e <= b) continue;
    int64_t lo[3] = {INT64_MAX, INT64_MAX, INT64_MAX}, hi[3] = {-1, -1, -1};
    for (int64_t i = b; i < e; ++i) {
      int64_t v = idx[i], p[3] = {v % nx, (v / nx) % ny, v / (nx * ny)};
      for (int a = 0; a < 3; ++a) {
        if (p[a] < lo[a]) lo[a] = p[a];
        if (p[a] > hi[a]) hi[a] = p[a];
      }
    }
    /* local field with r + 1 layers of zeros on every side */
    const int64_t pad = r + 1;
    int64_t bx = hi[0] - lo[0] + 1 + 2 * pad, by = hi[1] - lo[1] + 1 + 2 * pad, bz = hi[2] - lo[2] + 1 + 2 * pad;
    double* f = (double*)calloc((size_t)(bx * by * bz), sizeof(double));
    int64_t mx = bx > by ? bx : by;
    if (bz > mx) mx = bz;
    double* tmp = (double*)malloc(sizeof(double) * (size_t)mx);
    for (int64_t i = b; i < e; ++i) {
      int64_t v = idx[i];
      int64_t x = v % nx - lo[0] + pad, y = (v / nx) % ny - lo[1] + pad, z = v / (nx * ny) - lo[2] + pad;
      f[(z * by + y) * bx + x] = 1.0;
    }
    if (r > 0)
      for (int a = 0; a < 3; ++a) blur_axis(f, bx, by, bz, a, w, r, tmp);
    double total = 0.0, volume = 0.0;
    for (int64_t z = 0; z + 1 < bz; ++z)
      for (int64_t y = 0; y + 1 < by; ++y)
        for (int64_t x = 0; x + 1 < bx; ++x) {
          double c[8];
          int above = 0;
          for (int q = 0; q < 8; ++q) {
            int dx = q & 1, dy = (q >> 1) & 1, dz = (q >> 2) & 1;
            c[q] = f[((z + dz) * by + (y + dy)) * bx + (x + dx)];
            above += c[q] > 0.5;
          }
          if (above == 0 || above == 8) continue;
          for (int t = 0; t < 6; ++t) {
            double P[4][3], val[4];
            int cur[3] = {0, 0, 0};
            for (int j = 0; j < 4; ++j) {
              if (j > 0) cur[perm[t][j - 1]] = 1;
              P[j][0] = (double)(x + cur[0]);
              P[j][1] = (double)(y + cur[1]);
              P[j][2] = (double)(z + cur[2]);
              val[j] = c[cur[0] | (cur[1] << 1) | (cur[2] << 2)];
            }
            tet_surface(P, val, &total, &volume);
          }
        }
    area_out[k] = total;
    vol_out[k] = volume;
    free(f);
    free(tmp);
  }
}
