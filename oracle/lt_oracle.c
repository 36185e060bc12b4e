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
