/*
 * Seeded synthetic inputs: labelled 2D/3D masks of non-touching particles.
 *
 * This module only draws shapes and rasterises them. It contains none of the
 * measurement method (no distance transform, no local thickness, no shape
 * formula), so both the CPU oracle and the CUDA path can consume its output.
 *
 * Determinism: every random number comes from PCG32 (O'Neill 2014, the
 * XSH-RR 64->32 output function, written from its published definition).
 * The only floating-point library call is sqrt (IEEE correctly rounded), and
 * the file must be compiled with -ffp-contract=off so that x86-64 and AArch64
 * produce identical volumes.
 *
 * Layout of every volume: C order [z][y][x], x fastest; 2D uses nz = 1.
 * mask is 1 on particle voxels, 0 elsewhere; labels holds 1..n on particle
 * voxels and 0 elsewhere. Any two particles are separated by at least one
 * background voxel in every direction (no 26-adjacency, 8-adjacency in 2D).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ PCG32 */
typedef struct { uint64_t state, inc; } pcg32_t;

static uint32_t pcg32_next(pcg32_t* r) {
  uint64_t old = r->state;
  r->state = old * 6364136223846793005ULL + r->inc;
  uint32_t xs = (uint32_t)(((old >> 18u) ^ old) >> 27u);
  uint32_t rot = (uint32_t)(old >> 59u);
  return (xs >> rot) | (xs << ((32u - rot) & 31u));
}

static void pcg32_seed(pcg32_t* r, uint64_t seed, uint64_t stream) {
  r->state = 0u;
  r->inc = (stream << 1u) | 1u;
  pcg32_next(r);
  r->state += seed;
  pcg32_next(r);
}

/* uniform double in [0, 1) with 53 random bits */
static double u01(pcg32_t* r) {
  uint64_t a = pcg32_next(r) >> 5, b = pcg32_next(r) >> 6;
  return ((double)a * 67108864.0 + (double)b) * (1.0 / 9007199254740992.0);
}
static double unif(pcg32_t* r, double lo, double hi) { return lo + (hi - lo) * u01(r); }
static int uint_range(pcg32_t* r, int lo, int hi) { /* inclusive */
  return lo + (int)(u01(r) * (double)(hi - lo + 1));
}

/* uniform unit vector in d dimensions by rejection from the cube */
static void unit_vec(pcg32_t* r, int d, double* v) {
  for (;;) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) { v[i] = unif(r, -1.0, 1.0); s += v[i] * v[i]; }
    if (s > 1e-4 && s <= 1.0) {
      double inv = 1.0 / sqrt(s);
      for (int i = 0; i < d; ++i) v[i] *= inv;
      return;
    }
  }
}

/* uniform random rotation: a unit quaternion uniform on S^3, as a matrix */
static void random_rotation(pcg32_t* r, double m[3][3]) {
  double q[4];
  unit_vec(r, 4, q);
  double w = q[0], x = q[1], y = q[2], z = q[3];
  m[0][0] = 1 - 2 * (y * y + z * z); m[0][1] = 2 * (x * y - z * w);     m[0][2] = 2 * (x * z + y * w);
  m[1][0] = 2 * (x * y + z * w);     m[1][1] = 1 - 2 * (x * x + z * z); m[1][2] = 2 * (y * z - x * w);
  m[2][0] = 2 * (x * z - y * w);     m[2][1] = 2 * (y * z + x * w);     m[2][2] = 1 - 2 * (x * x + y * y);
}

/* a signed axis permutation (random, or want[i] = the local axis to put on
 * world axis i) followed by a tilt of at most 25 degrees
 * about a uniform random axis (quaternion (1, t u) normalised, t <= tan 12.5deg) */
static void near_aligned_rotation(pcg32_t* r, double m[3][3], const int* want) {
  int perm[3] = {0, 1, 2};
  for (int i = 2; i > 0; --i) {
    int j = (int)(u01(r) * (double)(i + 1));
    int t = perm[i]; perm[i] = perm[j]; perm[j] = t;
  }
  if (want) for (int i = 0; i < 3; ++i) perm[i] = want[i];
  double sgn[3];
  for (int i = 0; i < 3; ++i) sgn[i] = u01(r) < 0.5 ? -1.0 : 1.0;
  double P[3][3] = {{0}};
  for (int i = 0; i < 3; ++i) P[i][perm[i]] = sgn[i];
  double u[3];
  unit_vec(r, 3, u);
  double t = unif(r, 0.0, 0.2216946626415899);
  double q[4] = {1.0, t * u[0], t * u[1], t * u[2]};
  double inv = 1.0 / sqrt(1.0 + t * t);
  for (int i = 0; i < 4; ++i) q[i] *= inv;
  double w = q[0], x = q[1], y = q[2], z = q[3], T[3][3];
  T[0][0] = 1 - 2 * (y * y + z * z); T[0][1] = 2 * (x * y - z * w);     T[0][2] = 2 * (x * z + y * w);
  T[1][0] = 2 * (x * y + z * w);     T[1][1] = 1 - 2 * (x * x + z * z); T[1][2] = 2 * (y * z - x * w);
  T[2][0] = 2 * (x * z - y * w);     T[2][1] = 2 * (y * z + x * w);     T[2][2] = 1 - 2 * (x * x + y * y);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += T[i][k] * P[k][j];
      m[i][j] = acc;
    }
}

/* ----------------------------------------------------------------- shapes */
enum { SH_ELLIPSOID = 0, SH_SUPER = 1, SH_POLY = 2, SH_BUMPY = 3, SH_ELLIPSE2D = 4 };
#define MAX_PLANES 20
#define MAX_BUMPS 32

typedef struct {
  int type;
  double a[3];          /* semi-axes (local frame), scaled by s */
  int ehalf;            /* superellipsoid exponent = ehalf / 2 */
  int nplanes;
  double pn[MAX_PLANES][3], pd[MAX_PLANES]; /* unit normal, distance (fraction of a[0]) */
  int nbumps;
  double bdir[MAX_BUMPS][3], bamp[MAX_BUMPS];
  double rot[3][3];     /* local = rot^T * (p - c) */
  double s;             /* scale applied to a[] and plane distances */
} shape_t;

/* |t|^(k/2) using only multiplication and sqrt */
static double pow_half(double t, int k) {
  double at = fabs(t), out = 1.0;
  for (int i = 0; i < k / 2; ++i) out *= at;
  if (k & 1) out *= sqrt(at);
  return out;
}

/* smooth bump profile on the unit sphere: zero outside a cap of cosine t0 */
static double bump_profile(double cosang) {
  const double t0 = 0.9393727128473789; /* cos(0.35 rad) */
  if (cosang <= t0) return 0.0;
  double u = (cosang - t0) / (1.0 - t0);
  return u * u;
}

/* point p in the shape's local frame (unscaled coordinates) */
static int inside_local(const shape_t* sh, const double p[3]) {
  const double s = sh->s;
  switch (sh->type) {
    case SH_ELLIPSOID: {
      double q = 0.0;
      for (int i = 0; i < 3; ++i) { double t = p[i] / (sh->a[i] * s); q += t * t; }
      return q <= 1.0;
    }
    case SH_ELLIPSE2D: {
      double t0 = p[0] / (sh->a[0] * s), t1 = p[1] / (sh->a[1] * s);
      return t0 * t0 + t1 * t1 <= 1.0;
    }
    case SH_SUPER: {
      double q = 0.0;
      for (int i = 0; i < 3; ++i) q += pow_half(p[i] / (sh->a[i] * s), sh->ehalf);
      return q <= 1.0;
    }
    case SH_POLY: {
      double R = sh->a[0] * s;
      if (p[0] * p[0] + p[1] * p[1] + p[2] * p[2] > R * R) return 0;
      for (int j = 0; j < sh->nplanes; ++j) {
        double d = sh->pn[j][0] * p[0] + sh->pn[j][1] * p[1] + sh->pn[j][2] * p[2];
        if (d > sh->pd[j] * R) return 0;
      }
      return 1;
    }
    case SH_BUMPY: {
      double q = 0.0;
      for (int i = 0; i < 3; ++i) { double t = p[i] / (sh->a[i] * s); q += t * t; }
      if (q <= 1.0) return 1;
      double n2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
      if (n2 <= 0.0) return 1;
      double inv = 1.0 / sqrt(n2), bump = 0.0;
      for (int k = 0; k < sh->nbumps; ++k) {
        double c = (sh->bdir[k][0] * p[0] + sh->bdir[k][1] * p[1] + sh->bdir[k][2] * p[2]) * inv;
        bump += sh->bamp[k] * bump_profile(c);
      }
      double lim = 1.0 + bump;
      return q <= lim * lim;
    }
  }
  return 0;
}

static int inside_world(const shape_t* sh, const double c[3], double x, double y, double z) {
  double d[3] = {x - c[0], y - c[1], z - c[2]}, p[3];
  for (int i = 0; i < 3; ++i) p[i] = sh->rot[0][i] * d[0] + sh->rot[1][i] * d[1] + sh->rot[2][i] * d[2];
  return inside_local(sh, p);
}

/* conservative world half-extent along each axis, for scale s */
static void world_extent(const shape_t* sh, double s, double ext[3]) {
  double a[3];
  double grow = 1.0;
  if (sh->type == SH_BUMPY) {
    for (int k = 0; k < sh->nbumps; ++k) grow += sh->bamp[k];
  }
  for (int i = 0; i < 3; ++i) a[i] = sh->a[i] * s * grow;
  for (int i = 0; i < 3; ++i) {
    double e = 0.0;
    if (sh->type == SH_POLY) {
      e = a[0];
    } else if (sh->type == SH_SUPER) {
      for (int j = 0; j < 3; ++j) e += fabs(sh->rot[i][j]) * a[j];
    } else {
      for (int j = 0; j < 3; ++j) e += (sh->rot[i][j] * a[j]) * (sh->rot[i][j] * a[j]);
      e = sqrt(e);
    }
    ext[i] = e;
  }
}

/* --------------------------------------------------- 2D / 3D rasterising */
typedef struct {
  uint8_t* mask;
  uint32_t* labels;
  int64_t nx, ny, nz;
  int ndim;
} vol_t;

static int64_t vidx(const vol_t* v, int64_t x, int64_t y, int64_t z) {
  return (z * v->ny + y) * v->nx + x;
}

/* voxel box [lo, hi) per axis covering the shape at centre c */
static void shape_box(const vol_t* v, const shape_t* sh, const double c[3], int64_t lo[3], int64_t hi[3]) {
  double ext[3];
  world_extent(sh, sh->s, ext);
  int64_t n[3] = {v->nx, v->ny, v->nz};
  for (int i = 0; i < 3; ++i) {
    if (i == 2 && v->ndim == 2) { lo[2] = 0; hi[2] = 1; continue; }
    lo[i] = (int64_t)floor(c[i] - ext[i]) - 1;
    hi[i] = (int64_t)ceil(c[i] + ext[i]) + 2;
    if (lo[i] < 0) lo[i] = 0;
    if (hi[i] > n[i]) hi[i] = n[i];
  }
}

/* Random sequential addition test: the shape lies strictly inside the volume
 * (not touching its faces) and none of its voxels is blocked, where blocked
 * marks every voxel within one voxel (Chebyshev) of an existing particle.
 * On commit, writes the particle and extends the blocked map.
 * Returns the voxel count, 0 if rejected. */
static int64_t rsa_try(const vol_t* v, uint8_t* blocked, const shape_t* sh, const double c[3],
                       int commit, uint32_t label) {
  int64_t lo[3], hi[3];
  shape_box(v, sh, c, lo, hi);
  if (!commit) {
    int64_t cx = (int64_t)floor(c[0] + 0.5), cy = (int64_t)floor(c[1] + 0.5);
    int64_t cz = v->ndim == 3 ? (int64_t)floor(c[2] + 0.5) : 0;
    if (blocked[vidx(v, cx, cy, cz)]) return 0; /* cheap early rejection */
  }
  int64_t count = 0;
  for (int pass = commit ? 1 : 0; pass < 2; ++pass) {
    /* pass 0 probes every second voxel per axis, pass 1 visits all */
    int64_t st = pass == 0 ? 2 : 1;
    for (int64_t z = lo[2]; z < hi[2]; z += (v->ndim == 3 ? st : 1))
      for (int64_t y = lo[1]; y < hi[1]; y += st)
        for (int64_t x = lo[0]; x < hi[0]; x += st) {
          if (!inside_world(sh, c, (double)x, (double)y, (double)z)) continue;
          if (x == 0 || y == 0 || x == v->nx - 1 || y == v->ny - 1) return 0;
          if (v->ndim == 3 && (z == 0 || z == v->nz - 1)) return 0;
          int64_t i = vidx(v, x, y, z);
          if (!commit) {
            if (blocked[i]) return 0;
          } else {
            v->mask[i] = 1;
            v->labels[i] = label;
            int64_t z0 = v->ndim == 3 ? z - 1 : z, z1 = v->ndim == 3 ? z + 1 : z;
            for (int64_t zz = z0; zz <= z1; ++zz)
              for (int64_t yy = y - 1; yy <= y + 1; ++yy)
                for (int64_t xx = x - 1; xx <= x + 1; ++xx) blocked[vidx(v, xx, yy, zz)] = 1;
          }
          if (pass == 1) ++count;
        }
  }
  return count;
}

static void draw_rsa_shape(pcg32_t* r, int ndim, double amin, double amax, double bump_frac,
                           int bmin, int bmax, double amp_lo, double amp_hi, shape_t* sh) {
  memset(sh, 0, sizeof(*sh));
  sh->s = 1.0;
  if (ndim == 2) {
    sh->type = SH_ELLIPSE2D;
    sh->a[0] = unif(r, amin, amax);
    sh->a[1] = unif(r, amin, amax);
    sh->a[2] = 1.0;
    double u[2];
    unit_vec(r, 2, u);
    /* rotation in the (x, y) plane; columns are the local axes in world */
    sh->rot[0][0] = u[0]; sh->rot[0][1] = -u[1]; sh->rot[0][2] = 0;
    sh->rot[1][0] = u[1]; sh->rot[1][1] = u[0];  sh->rot[1][2] = 0;
    sh->rot[2][0] = 0;    sh->rot[2][1] = 0;     sh->rot[2][2] = 1;
    return;
  }
  for (int i = 0; i < 3; ++i) sh->a[i] = unif(r, amin, amax);
  random_rotation(r, sh->rot);
  sh->type = SH_ELLIPSOID;
  if (u01(r) < bump_frac) {
    sh->type = SH_BUMPY;
    sh->nbumps = uint_range(r, bmin, bmax);
    if (sh->nbumps > MAX_BUMPS) sh->nbumps = MAX_BUMPS;
    for (int k = 0; k < sh->nbumps; ++k) {
      unit_vec(r, 3, sh->bdir[k]);
      sh->bamp[k] = unif(r, amp_lo, amp_hi);
    }
  }
}

/*
 * Random sequential addition of n_obj ellipses (2D, nz = 1) or ellipsoids (3D)
 * with semi-axes uniform in [amin, amax] and uniform random orientation. In
 * 3D a fraction bump_frac of them carry between bmin and bmax radial bumps of
 * relative amplitude uniform in [amp_lo, amp_hi].
 * Returns the number of particles placed (labels 1..count).
 */
int64_t synth_rsa(uint8_t* mask, uint32_t* labels, int64_t nx, int64_t ny, int64_t nz, int ndim,
                  int64_t n_obj, double amin, double amax, double bump_frac, int bmin, int bmax,
                  double amp_lo, double amp_hi, uint64_t seed) {
  vol_t v = {mask, labels, nx, ny, nz, ndim};
  int64_t n = nx * ny * nz;
  memset(mask, 0, (size_t)n);
  memset(labels, 0, (size_t)n * sizeof(uint32_t));
  uint8_t* blocked = (uint8_t*)calloc((size_t)n, 1);
  if (!blocked) return -1;
  pcg32_t r;
  pcg32_seed(&r, seed, 0x5eedULL);
  int64_t placed = 0;
  for (int64_t k = 0; k < n_obj; ++k) {
    int ok = 0;
    for (int redraw = 0; redraw < 200 && !ok; ++redraw) {
      shape_t sh;
      draw_rsa_shape(&r, ndim, amin, amax, bump_frac, bmin, bmax, amp_lo, amp_hi, &sh);
      double ext[3];
      world_extent(&sh, 1.0, ext);
      for (int attempt = 0; attempt < 100 && !ok; ++attempt) {
        double c[3];
        c[0] = unif(&r, ext[0] + 1.0, (double)nx - 2.0 - ext[0]);
        c[1] = unif(&r, ext[1] + 1.0, (double)ny - 2.0 - ext[1]);
        c[2] = ndim == 3 ? unif(&r, ext[2] + 1.0, (double)nz - 2.0 - ext[2]) : 0.0;
        if (rsa_try(&v, blocked, &sh, c, 0, 0) > 0) {
          rsa_try(&v, blocked, &sh, c, 1, (uint32_t)(placed + 1));
          ++placed;
          ok = 1;
        }
      }
    }
    if (!ok) break;
  }
  free(blocked);
  return placed;
}

/* ----------------------------------------------- packed (partition) mode */
typedef struct { double lo[3], hi[3]; int64_t first, count; } cell_t;

typedef struct {
  double* w;      /* weights (target volumes) in a shuffled order */
  int64_t* id;    /* particle ids in the same order */
  cell_t* cells;  /* leaf cells, one per particle */
  int64_t ncells;
  int ndim;
} part_t;

static void partition(part_t* P, double lo[3], double hi[3], int64_t first, int64_t count) {
  if (count == 1) {
    cell_t* c = &P->cells[P->ncells++];
    memcpy(c->lo, lo, sizeof(double) * 3);
    memcpy(c->hi, hi, sizeof(double) * 3);
    c->first = first;
    c->count = 1;
    return;
  }
  int axis = 0;
  for (int i = 1; i < P->ndim; ++i)
    if (hi[i] - lo[i] > hi[axis] - lo[axis]) axis = i;
  int64_t k = count / 2;
  double w1 = 0.0, w = 0.0;
  for (int64_t i = 0; i < count; ++i) {
    w += P->w[first + i];
    if (i < k) w1 += P->w[first + i];
  }
  double cut = lo[axis] + (hi[axis] - lo[axis]) * (w1 / w);
  double hi1[3], lo2[3];
  memcpy(hi1, hi, sizeof(hi1));
  memcpy(lo2, lo, sizeof(lo2));
  hi1[axis] = cut;
  lo2[axis] = cut;
  partition(P, lo, hi1, first, k);
  partition(P, lo2, hi, first + k, count - k);
}

static void draw_packed_shape(pcg32_t* r, int ndim, double f_ell, double f_super, shape_t* sh) {
  memset(sh, 0, sizeof(*sh));
  sh->s = 1.0;
  if (ndim == 2) {
    sh->type = SH_ELLIPSE2D;
    double ratio = unif(r, 1.0, 3.0);
    sh->a[0] = 1.0;
    sh->a[1] = 1.0 / ratio;
    sh->a[2] = 1.0;
    double u[2];
    unit_vec(r, 2, u);
    sh->rot[0][0] = u[0]; sh->rot[0][1] = -u[1];
    sh->rot[1][0] = u[1]; sh->rot[1][1] = u[0];
    sh->rot[2][2] = 1.0;
    return;
  }
  random_rotation(r, sh->rot);
  double t = u01(r);
  if (t < f_ell) {
    sh->type = SH_ELLIPSOID;
    /* axis ratios uniform in [1, 4] relative to the longest axis */
    /* longest / shortest axis uniform in [1, 4], middle axis in between */
    double q = unif(r, 1.0, 4.0);
    sh->a[0] = 1.0;
    sh->a[2] = 1.0 / q;
    sh->a[1] = 1.0 / unif(r, 1.0, q);
  } else if (t < f_ell + f_super) {
    sh->type = SH_SUPER;
    sh->ehalf = uint_range(r, 4, 12); /* exponent 2.0, 2.5, ..., 6.0 */
    sh->a[0] = 1.0;
    sh->a[1] = 1.0 / unif(r, 1.0, 2.0);
    sh->a[2] = 1.0 / unif(r, 1.0, 2.0);
  } else {
    sh->type = SH_POLY;
    sh->a[0] = sh->a[1] = sh->a[2] = 1.0;
    sh->nplanes = uint_range(r, 6, 20);
    for (int j = 0; j < sh->nplanes; ++j) {
      unit_vec(r, 3, sh->pn[j]);
      sh->pd[j] = unif(r, 0.5, 0.95);
    }
  }
}

/* Does the shape at scale s, centred at c, stay inside the voxel box
 * [lo, hi) per axis? Counts its voxels into *nvox when it does. */
static int fits_cell(const vol_t* v, shape_t* sh, double s, const double c[3],
                     const int64_t lo[3], const int64_t hi[3], int64_t* nvox) {
  sh->s = s;
  int64_t blo[3], bhi[3];
  shape_box(v, sh, c, blo, bhi);
  int64_t cnt = 0;
  for (int64_t z = blo[2]; z < bhi[2]; ++z)
    for (int64_t y = blo[1]; y < bhi[1]; ++y)
      for (int64_t x = blo[0]; x < bhi[0]; ++x) {
        if (!inside_world(sh, c, (double)x, (double)y, (double)z)) continue;
        if (x < lo[0] || x >= hi[0] || y < lo[1] || y >= hi[1] || z < lo[2] || z >= hi[2]) return 0;
        ++cnt;
      }
  *nvox = cnt;
  return 1;
}

/* Does the particle (shape sh at scale s, centre c, label lab) fit where it
 * stands: every voxel of its rasterisation off the volume faces and with no
 * other label in its 26-neighbourhood (the one-voxel gap)? */
static int grow_fits(const vol_t* v, shape_t* sh, double s, const double c[3], uint32_t lab) {
  sh->s = s;
  int64_t blo[3], bhi[3];
  shape_box(v, sh, c, blo, bhi);
  const int64_t n[3] = {v->nx, v->ny, v->nz};
  const int nd = v->ndim;
  for (int64_t z = blo[2]; z < bhi[2]; ++z)
    for (int64_t y = blo[1]; y < bhi[1]; ++y)
      for (int64_t x = blo[0]; x < bhi[0]; ++x) {
        if (!inside_world(sh, c, (double)x, (double)y, (double)z)) continue;
        const int64_t q[3] = {x, y, z};
        for (int i = 0; i < nd; ++i)
          if (q[i] < 1 || q[i] > n[i] - 2) return 0;
        const int64_t z0 = nd == 3 ? z - 1 : z, z1 = nd == 3 ? z + 1 : z;
        for (int64_t zz = z0; zz <= z1; ++zz)
          for (int64_t yy = y - 1; yy <= y + 1; ++yy)
            for (int64_t xx = x - 1; xx <= x + 1; ++xx) {
              uint32_t o = v->labels[vidx(v, xx, yy, zz)];
              if (o != 0u && o != lab) return 0;
            }
      }
  return 1;
}

/* Voxel box of the particle at scale s widened by one voxel, unclamped. */
static void grow_box(const shape_t* sh, double s, const double c[3], int ndim, int64_t lo[3],
                     int64_t hi[3]) {
  double ext[3];
  world_extent(sh, s, ext);
  for (int i = 0; i < 3; ++i) {
    lo[i] = (int64_t)floor(c[i] - ext[i]) - 2;
    hi[i] = (int64_t)ceil(c[i] + ext[i]) + 3;
  }
  if (ndim == 2) { lo[2] = 0; hi[2] = 1; }
}

/*
 * Growth into free space, after the packing: each particle is scaled about
 * its centre by the largest factor in [1, grow_max] (bisection, 8 steps) at
 * which it still fits (grow_fits). The shapes are convex and contain their
 * centre, so a grown particle covers its old voxels. Particles whose widened
 * boxes at grow_max overlap never grow at the same time: a greedy colouring
 * in label order splits them into rounds, and the particles of one round grow
 * in parallel. The result depends on neither the thread count nor the
 * schedule.
 */
static void grow_particles(vol_t* v, shape_t* shs, double (*cs)[3], const uint8_t* placed,
                           int64_t ncells, double grow_max) {
  int64_t (*box)[6] = (int64_t(*)[6])malloc(sizeof(int64_t[6]) * (size_t)ncells);
  int32_t* colour = (int32_t*)malloc(sizeof(int32_t) * (size_t)ncells);
  if (!box || !colour) { free(box); free(colour); return; }
  int32_t ncol = 0;
  for (int64_t i = 0; i < ncells; ++i) {
    colour[i] = -1;
    if (!placed[i]) continue;
    grow_box(&shs[i], shs[i].s * grow_max, cs[i], v->ndim, &box[i][0], &box[i][3]);
  }
  uint64_t used[64];
  for (int64_t i = 0; i < ncells; ++i) {
    if (!placed[i]) continue;
    memset(used, 0, sizeof(used));
    for (int64_t j = 0; j < i; ++j) {
      if (colour[j] < 0) continue;
      int apart = 0;
      for (int k = 0; k < 3; ++k)
        if (box[i][k] >= box[j][k + 3] || box[j][k] >= box[i][k + 3]) { apart = 1; break; }
      if (!apart && colour[j] < 4096) used[colour[j] >> 6] |= 1ull << (colour[j] & 63);
    }
    int32_t c = 0;
    while (c < 4096 && (used[c >> 6] >> (c & 63) & 1ull)) ++c;
    if (c >= 4096) continue; /* crowded beyond any real packing: leave it as placed */
    colour[i] = c;
    if (c + 1 > ncol) ncol = c + 1;
  }
  for (int32_t round = 0; round < ncol; ++round) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < ncells; ++i) {
      if (colour[i] != round) continue;
      shape_t sh = shs[i];
      const uint32_t lab = (uint32_t)(i + 1);
      const double s0 = sh.s;
      double lo = 1.0, hi = grow_max;
      if (grow_fits(v, &sh, s0 * hi, cs[i], lab)) {
        lo = hi;
      } else {
        for (int it = 0; it < 8; ++it) {
          double mid = 0.5 * (lo + hi);
          if (grow_fits(v, &sh, s0 * mid, cs[i], lab)) lo = mid; else hi = mid;
        }
      }
      if (lo <= 1.0) continue;
      sh.s = s0 * lo;
      int64_t blo[3], bhi[3];
      shape_box(v, &sh, cs[i], blo, bhi);
      for (int64_t z = blo[2]; z < bhi[2]; ++z)
        for (int64_t y = blo[1]; y < bhi[1]; ++y)
          for (int64_t x = blo[0]; x < bhi[0]; ++x)
            if (inside_world(&sh, cs[i], (double)x, (double)y, (double)z)) {
              int64_t q = vidx(v, x, y, z);
              v->mask[q] = 1;
              v->labels[q] = lab;
            }
    }
  }
  free(box);
  free(colour);
}

/*
 * Dense packing of n_obj particles: the volume is split by weighted recursive
 * bisection into one cell per particle (cell volume proportional to a drawn
 * equivalent radius cubed, radius uniform in [rmin, rmax]); each cell
 * receives one randomly oriented particle, grown to the largest scale that
 * keeps it inside the cell minus its last voxel layer (the one-voxel gap).
 * 3D mix: f_ell ellipsoids (axis ratios 1-4), f_super superellipsoids
 * (exponent 2-6 in steps of 0.5), the rest convex polyhedra (a ball cut by
 * 6-20 random half-spaces at 0.5-0.95 of its radius). 2D: ellipses with axis
 * ratio 1-3. Each particle's final scale is multiplied by a factor uniform
 * in [shrink_lo, shrink_hi] (1, 1 for the densest packing). Orientation: the
 * best of twelve candidates (uniform random rotations and tilted axis-aligned
 * ones in 3D, uniform in 2D). Cells are processed in parallel, each from its own PCG32 stream,
 * so the result does not depend on the thread count. grow_max > 1 then
 * grows every particle into the free space around it (grow_particles).
 * Returns the number of particles (labels 1..count; a particle too small to
 * hold a voxel leaves its label unused).
 */
int64_t synth_packed(uint8_t* mask, uint32_t* labels, int64_t nx, int64_t ny, int64_t nz, int ndim,
                     int64_t n_obj, double rmin, double rmax, double f_ell, double f_super,
                     double shrink_lo, double shrink_hi, double grow_max, uint64_t seed) {
  vol_t v = {mask, labels, nx, ny, nz, ndim};
  int64_t n = nx * ny * nz;
  memset(mask, 0, (size_t)n);
  memset(labels, 0, (size_t)n * sizeof(uint32_t));
  if (n_obj <= 0) return 0;
  part_t P;
  P.w = (double*)malloc(sizeof(double) * (size_t)n_obj);
  P.id = (int64_t*)malloc(sizeof(int64_t) * (size_t)n_obj);
  P.cells = (cell_t*)malloc(sizeof(cell_t) * (size_t)n_obj);
  P.ncells = 0;
  P.ndim = ndim;
  if (!P.w || !P.id || !P.cells) { free(P.w); free(P.id); free(P.cells); return -1; }
  pcg32_t r;
  pcg32_seed(&r, seed, 0xce11ULL);
  for (int64_t i = 0; i < n_obj; ++i) {
    double rad = unif(&r, rmin, rmax);
    P.w[i] = ndim == 3 ? rad * rad * rad : rad * rad;
    P.id[i] = i;
  }
  for (int64_t i = n_obj - 1; i > 0; --i) { /* Fisher-Yates */
    int64_t j = (int64_t)(u01(&r) * (double)(i + 1));
    double tw = P.w[i]; P.w[i] = P.w[j]; P.w[j] = tw;
    int64_t ti = P.id[i]; P.id[i] = P.id[j]; P.id[j] = ti;
  }
  double lo[3] = {0, 0, 0}, hi[3] = {(double)nx, (double)ny, (double)(ndim == 3 ? nz : 1)};
  partition(&P, lo, hi, 0, n_obj);
  const int grow = grow_max > 1.0;
  shape_t* shs = NULL;
  double (*cs)[3] = NULL;
  uint8_t* placed = NULL;
  if (grow) {
    shs = (shape_t*)malloc(sizeof(shape_t) * (size_t)P.ncells);
    cs = (double(*)[3])malloc(sizeof(double[3]) * (size_t)P.ncells);
    placed = (uint8_t*)calloc((size_t)P.ncells, 1);
    if (!shs || !cs || !placed) {
      free(shs); free(cs); free(placed); free(P.w); free(P.id); free(P.cells);
      return -1;
    }
  }

#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t ci = 0; ci < P.ncells; ++ci) {
    const cell_t* cell = &P.cells[ci];
    pcg32_t rr;
    pcg32_seed(&rr, seed ^ 0x9e3779b97f4a7c15ULL, (uint64_t)ci + 1u);
    int64_t clo[3], chi[3];
    double c[3];
    for (int i = 0; i < 3; ++i) {
      clo[i] = (int64_t)floor(cell->lo[i] + 0.5);
      if (clo[i] == 0) clo[i] = 1; /* keep particles off the volume faces */
      chi[i] = (int64_t)floor(cell->hi[i] + 0.5) - 1; /* last layer is the gap */
      c[i] = 0.5 * (double)(clo[i] + chi[i] - 1);
    }
    if (ndim == 2) { clo[2] = 0; chi[2] = 1; c[2] = 0.0; }
    int empty = 0;
    for (int i = 0; i < ndim; ++i) if (chi[i] - clo[i] < 1) empty = 1;
    if (empty) continue;
    shape_t sh, best;
    draw_packed_shape(&rr, ndim, f_ell, f_super, &sh);
    /* keep the best of a few random orientations: the one that reaches the
     * largest voxel count inside the cell */
    double s = 0.0;
    int64_t nv = 0;
    for (int trial = 0; trial < 12; ++trial) {
      if (trial > 0) {
        if (ndim == 3) {
          if (trial % 3 == 1) {
            random_rotation(&rr, sh.rot);
          } else if (trial % 3 == 2) {
            near_aligned_rotation(&rr, sh.rot, NULL);
          } else {
            /* longest local axis on the longest cell axis, and so on */
            int wa[3] = {0, 1, 2}, la[3] = {0, 1, 2}, want[3];
            for (int i = 0; i < 3; ++i)
              for (int j = i + 1; j < 3; ++j) {
                if (chi[wa[j]] - clo[wa[j]] > chi[wa[i]] - clo[wa[i]]) { int t = wa[i]; wa[i] = wa[j]; wa[j] = t; }
                if (sh.a[la[j]] > sh.a[la[i]]) { int t = la[i]; la[i] = la[j]; la[j] = t; }
              }
            for (int i = 0; i < 3; ++i) want[wa[i]] = la[i];
            near_aligned_rotation(&rr, sh.rot, want);
          }
        } else {
          double u[2];
          unit_vec(&rr, 2, u);
          sh.rot[0][0] = u[0]; sh.rot[0][1] = -u[1];
          sh.rot[1][0] = u[1]; sh.rot[1][1] = u[0];
        }
      }
      /* conservative scale from the analytic extent, then grow while it fits */
      double ext[3];
      world_extent(&sh, 1.0, ext);
      double st = 1e30;
      for (int i = 0; i < ndim; ++i) {
        double half = 0.5 * (double)(chi[i] - clo[i]) - 0.5;
        double si = half / ext[i];
        if (si < st) st = si;
      }
      int64_t nvt = 0;
      if (st <= 0.0 || !fits_cell(&v, &sh, st, c, clo, chi, &nvt)) continue;
      double step = 0.5;
      for (int it = 0; it < 6; ++it) {
        int64_t nv2 = 0;
        if (fits_cell(&v, &sh, st * (1.0 + step), c, clo, chi, &nv2)) { st *= 1.0 + step; nvt = nv2; }
        step *= 0.5;
      }
      if (nvt > nv) { nv = nvt; s = st; best = sh; }
    }
    if (nv == 0) continue;
    sh = best;
    s *= unif(&rr, shrink_lo, shrink_hi);
    sh.s = s;
    uint32_t label = (uint32_t)(ci + 1);
    if (grow) {
      shs[ci] = sh;
      for (int i = 0; i < 3; ++i) cs[ci][i] = c[i];
      placed[ci] = 1;
    }
    for (int64_t z = clo[2]; z < chi[2]; ++z)
      for (int64_t y = clo[1]; y < chi[1]; ++y)
        for (int64_t x = clo[0]; x < chi[0]; ++x)
          if (inside_world(&sh, c, (double)x, (double)y, (double)z)) {
            int64_t i = vidx(&v, x, y, z);
            mask[i] = 1;
            labels[i] = label;
          }
  }
  if (grow) grow_particles(&v, shs, cs, placed, P.ncells, grow_max);
  free(shs);
  free(cs);
  free(placed);
  int64_t out = P.ncells;
  free(P.w);
  free(P.id);
  free(P.cells);
  return out;
}
