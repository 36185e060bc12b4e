// Exact local thickness on sm_103a.
//
// LT2(x) = max { DT2(c) : label(c) = label(x) != 0, |x - c|^2 <= DT2(c) }:
// the squared radius of the largest inscribed ball of x's object that holds
// x (local thickness, Sec. 1 and Sec. 4 of the paper). Computed by painting
// balls with atomic max, with two reductions that keep the result exact.
//
// Ball of c: B(c) = lattice points y with |y - c|^2 <= r_c^2, r_c^2 = DT2(c),
// restricted to voxels of c's object. Rank: c' > c when r_c'^2 > r_c^2, or
// equal radii and a larger linear index (a strict total order).
//
// 1. Containment (ridge) test. For a neighbour offset d (|d|_inf = 1) let
//    M(d, r^2) = max { |y - d|^2 : |y|^2 <= r^2 } over lattice points y. Then
//    B(c) is a subset of B(c + d) exactly when r_{c+d}^2 >= M(d, r_c^2); such a
//    c (same label as c + d) is dropped. M > r^2, so the container ranks
//    higher. M depends only on the class of d (1, 2 or 3 nonzero
//    coordinates) by the symmetry of the lattice ball, and is tabulated on
//    the device for r^2 up to 2^18; larger centres are never dropped.
// 2. Crescent painting. A kept centre c picks one higher-ranked same-label
//    neighbour D (the one whose ball reaches farthest past c's, if any) and
//    raises LT2 only on voxels of B(c) outside B(D).
// Exactness, by induction down the rank order: every object voxel x in any
// B(c) ends with LT2(x) >= r_c^2. If c was dropped, x lies in a higher-ranked
// ball of radius >= r_c. If c is kept, x is either painted by c or lies in
// B(D) with r_D >= r_c. The highest-ranked centre paints its whole ball.
// Since only true ball radii are painted, LT2 is exactly the maximum.
//
// Voxels strictly inside B(c) are foreground (DT2(c) is the distance to the
// nearest background), so only points with |y - c|^2 == r_c^2 may be
// background; they are checked against DT2. Each ball voxel is joined to c by
// a face-connected path of strictly inner voxels, so when no two
// face-adjacent foreground voxels carry different labels (checked by the
// ridge kernel, flag `touch`) every foreground ball voxel has c's label and
// the label test is skipped.
#include <algorithm>
#include <climits>

#include "lt_internal.cuh"

namespace ltk {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kTableCap = 1u << 18;
constexpr uint32_t kNoDominant = 31u;

// raw[cls][n] = max over sorted lattice points (y1 >= y2 >= y3 >= 0) with
// |y|^2 = n of |y|^2 + 2 (sum of the cls largest |y_i|) + cls: the largest
// |y - d|^2 among the signed permutations of y for d of class cls.
__global__ void mtable_points_kernel(uint32_t* __restrict__ raw, uint32_t cap, int R, int ndim) {
  const size_t total = (size_t)(R + 1) * (R + 1);
  const size_t stride = (size_t)(cap + 1);
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const uint32_t y1 = (uint32_t)(t / (R + 1)), y2 = (uint32_t)(t % (R + 1));
    if (y2 > y1) continue;
    const uint32_t n12 = y1 * y1 + y2 * y2;
    if (n12 > cap) continue;
    if (ndim == 2) {
      atomicMax(&raw[n12], n12 + 2 * y1 + 1);
      atomicMax(&raw[stride + n12], n12 + 2 * (y1 + y2) + 2);
    } else {
      for (uint32_t y3 = 0; y3 <= y2; ++y3) {
        const uint32_t n = n12 + y3 * y3;
        if (n > cap) break;
        atomicMax(&raw[n], n + 2 * y1 + 1);
        atomicMax(&raw[stride + n], n + 2 * (y1 + y2) + 2);
        atomicMax(&raw[2 * stride + n], n + 2 * (y1 + y2 + y3) + 3);
      }
    }
  }
}

// In-place prefix maximum over n of one table row (one 1024-thread block per
// class): M(d, r^2) = max over n <= r^2 of raw[n].
__global__ void __launch_bounds__(1024) mtable_prefix_kernel(uint32_t* __restrict__ tab, uint32_t cap) {
  __shared__ uint32_t part[1024];
  uint32_t* row = tab + (size_t)blockIdx.x * (cap + 1);
  const uint32_t n = cap + 1;
  const uint32_t chunk = (n + 1023) / 1024;
  const uint32_t lo = threadIdx.x * chunk, hi = min(n, lo + chunk);
  uint32_t m = 0;
  for (uint32_t i = lo; i < hi; ++i) m = max(m, row[i]);
  part[threadIdx.x] = m;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const uint32_t t = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0u;
    __syncthreads();
    part[threadIdx.x] = max(part[threadIdx.x], t);
    __syncthreads();
  }
  uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
  for (uint32_t i = lo; i < hi; ++i) {
    run = max(run, row[i]);
    row[i] = run;
  }
}

// One thread per voxel: clears LT2, validates labels against the mask, sets
// the `touch` flag, applies the containment test and appends kept centres.
// A CTA covers 256 x-positions of kRidgeRows rows; kept centres collect in
// shared memory and leave with one global atomic per CTA.
// Record: x = linear index, y = r^2 | dominant neighbour code << 25 (code =
// (dz+1)*9 + (dy+1)*3 + (dx+1), or 31 for none).
constexpr int kRidgeRows = 8;

template <int NDIM>
__global__ void __launch_bounds__(256) lt_ridge_kernel(const uint32_t* __restrict__ dt2,
                                                       const uint32_t* __restrict__ labels,
                                                       uint32_t* __restrict__ lt2,
                                                       const uint32_t* __restrict__ mtab,
                                                       uint32_t cap, Dims d, uint2* __restrict__ surv,
                                                       WsHeader* __restrict__ hdr) {
  __shared__ uint2 buf[256 * kRidgeRows];
  __shared__ uint32_t cnt, base, flags;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    cnt = 0;
    flags = 0;
  }
  __syncthreads();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int z = blockIdx.z;
  const bool in = x < d.nx;
  const size_t sy = (size_t)d.nx, sz = (size_t)d.nx * d.ny;
  for (int r = 0; r < kRidgeRows; ++r) {
    const int y = blockIdx.y * kRidgeRows + r;
    if (y >= d.ny) break;  // uniform across the CTA
    const uint32_t v = in ? (uint32_t)(z * sz + y * sy + x) : 0u;
    bool keep = false, touch = false, bad = false;
    uint32_t r2 = 0, code = kNoDominant;
    if (in) {
      r2 = dt2[v];
      const uint32_t l = labels[v];
      lt2[v] = 0u;
      if (r2 == 0) {
        bad = l != 0;
      } else {
        if (x + 1 < d.nx && dt2[v + 1] && labels[v + 1] != l) touch = true;
        if (y + 1 < d.ny && dt2[v + sy] && labels[v + sy] != l) touch = true;
        if (NDIM == 3 && z + 1 < d.nz && dt2[v + sz] && labels[v + sz] != l) touch = true;
        if (l != 0) {
          keep = true;
          uint32_t m1 = UINT_MAX, m2 = UINT_MAX, m3 = UINT_MAX;
          if (r2 <= cap) {
            m1 = __ldg(mtab + r2);
            m2 = __ldg(mtab + (cap + 1) + r2);
            if (NDIM == 3) m3 = __ldg(mtab + 2 * (size_t)(cap + 1) + r2);
          }
          float best_reach = -1e30f;
          const int zlo = NDIM == 3 ? -1 : 0, zhi = NDIM == 3 ? 1 : 0;
          for (int dz = zlo; dz <= zhi && keep; ++dz) {
            if (z + dz < 0 || z + dz >= d.nz) continue;
            for (int dy = -1; dy <= 1 && keep; ++dy) {
              if (y + dy < 0 || y + dy >= d.ny) continue;
              for (int dx = -1; dx <= 1; ++dx) {
                if ((dx | dy | dz) == 0 || x + dx < 0 || x + dx >= d.nx) continue;
                const uint32_t u = (uint32_t)((int64_t)v + dz * (int64_t)sz + dy * (int64_t)sy + dx);
                if (labels[u] != l) continue;
                const uint32_t rn = dt2[u];
                const int cls = abs(dx) + abs(dy) + abs(dz);
                const uint32_t mm = cls == 1 ? m1 : (cls == 2 ? m2 : m3);
                if (rn >= mm) {
                  keep = false;
                  break;
                }
                if (rn > r2 || (rn == r2 && u > v)) {
                  const float reach =
                      sqrtf((float)rn) - (cls == 1 ? 1.0f : (cls == 2 ? 1.41421356f : 1.73205081f));
                  if (reach > best_reach) {
                    best_reach = reach;
                    code = (uint32_t)((dz + 1) * 9 + (dy + 1) * 3 + (dx + 1));
                  }
                }
              }
            }
          }
        }
      }
    }
    if (__any_sync(kFull, bad) && lane == 0) atomicOr(&flags, 1u);
    if (__any_sync(kFull, touch) && lane == 0) atomicOr(&flags, 2u);
    const unsigned bal = __ballot_sync(kFull, keep);
    if (bal) {
      uint32_t wb = 0;
      if (lane == 0) wb = atomicAdd(&cnt, (uint32_t)__popc(bal));
      wb = __shfl_sync(kFull, wb, 0);
      if (keep) buf[wb + __popc(bal & ((1u << lane) - 1u))] = make_uint2(v, r2 | (code << 25));
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    base = cnt ? atomicAdd(&hdr->n_surv, cnt) : 0u;
    if (flags & 1u) atomicOr(&hdr->error, ERR_LABEL_OUTSIDE_MASK);
    if (flags & 2u) atomicOr(&hdr->touch, 1u);
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) surv[base + i] = buf[i];
}

struct Centre {
  int cx, cy, cz, R;
  uint32_t r2, label;
  int ddx, ddy, ddz, r2d;  // dominant neighbour offset and its r^2 (-1: none)
  int start, pad;
};

// Paints the part of one ball row (offsets dz, dy from the centre, squared
// half-width h) that lies outside the dominant neighbour's ball.
__device__ __forceinline__ void paint_row(const Centre& c, int dz, int dy, int h, size_t rowbase,
                                          int nx, bool touch, const uint32_t* __restrict__ dt2,
                                          const uint32_t* __restrict__ labels,
                                          uint32_t* __restrict__ lt2) {
  const int w = (int)isqrt24((uint32_t)h);
  int hd = -1;
  if (c.r2d >= 0) hd = c.r2d - (dz - c.ddz) * (dz - c.ddz) - (dy - c.ddy) * (dy - c.ddy);
  auto vox = [&](int dx) {
    const int x = c.cx + dx;
    if (x < 0 || x >= nx) return;
    const size_t i = rowbase + x;
    if (dx * dx == h && dt2[i] == 0) return;  // ball boundary point may be background
    if (touch && labels[i] != c.label) return;
    atomicMax(lt2 + i, c.r2);
  };
  int xl = -w;
  while (xl <= w && (hd < 0 || (xl - c.ddx) * (xl - c.ddx) > hd)) vox(xl++);
  int xr = w;
  while (xr >= xl && (hd < 0 || (xr - c.ddx) * (xr - c.ddx) > hd)) vox(xr--);
}

// Warps take chunks of 32 kept centres from a global counter. Each centre
// contributes 2R+1 items (one per z offset in 3D, one per row in 2D); the 32
// lanes share the items of the chunk, so big and small balls balance.
template <int NDIM>
__global__ void __launch_bounds__(256) lt_paint_kernel(const uint2* __restrict__ surv,
                                                       const uint32_t* __restrict__ dt2,
                                                       const uint32_t* __restrict__ labels,
                                                       uint32_t* __restrict__ lt2, Dims d,
                                                       WsHeader* __restrict__ hdr) {
  __shared__ Centre cs[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t n = *(volatile uint32_t*)&hdr->n_surv;
  const bool touch = *(volatile uint32_t*)&hdr->touch != 0;
  const uint32_t nchunks = (n + 31) / 32;
  const size_t sy = (size_t)d.nx, sz = (size_t)d.nx * d.ny;
  uint32_t* counter = &hdr->reserved[0];
  for (;;) {
    uint32_t ch = 0;
    if (lane == 0) ch = atomicAdd(counter, 1u);
    ch = __shfl_sync(kFull, ch, 0);
    if (ch >= nchunks) break;
    const uint32_t i = ch * 32 + lane;
    int cnt = 0;
    if (i < n) {
      const uint2 rec = surv[i];
      const uint32_t idx = rec.x, code = rec.y >> 25;
      Centre c;
      c.r2 = rec.y & 0x1FFFFFFu;
      c.cx = (int)(idx % (uint32_t)d.nx);
      const uint32_t t = idx / (uint32_t)d.nx;
      c.cy = (int)(t % (uint32_t)d.ny);
      c.cz = (int)(t / (uint32_t)d.ny);
      c.R = (int)isqrt24(c.r2);
      c.label = touch ? labels[idx] : 0u;
      if (code != kNoDominant) {
        c.ddz = (int)(code / 9) - 1;
        c.ddy = (int)(code / 3 % 3) - 1;
        c.ddx = (int)(code % 3) - 1;
        c.r2d = (int)dt2[(int64_t)idx + c.ddz * (int64_t)sz + c.ddy * (int64_t)sy + c.ddx];
      } else {
        c.ddx = c.ddy = c.ddz = 0;
        c.r2d = -1;
      }
      c.start = 0;
      c.pad = 0;
      cs[w][lane] = c;
      cnt = 2 * c.R + 1;
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += t;
    }
    const int start = incl - cnt;
    if (i < n) cs[w][lane].start = start;
    const int total = __shfl_sync(kFull, incl, 31);
    __syncwarp();
    for (int kb = 0; kb < total; kb += 32) {
      const int k = kb + lane;
      int j = 0;  // owner: the last lane whose start <= k
#pragma unroll
      for (int step = 16; step; step >>= 1) {
        const int s = __shfl_sync(kFull, start, j + step);
        if (s <= k) j += step;
      }
      if (k < total) {
        const Centre c = cs[w][j];
        const int u = k - c.start - c.R;
        if (NDIM == 3) {
          const int z = c.cz + u;
          if (z >= 0 && z < d.nz) {
            const int hz2 = (int)c.r2 - u * u;
            const int hz = (int)isqrt24((uint32_t)hz2);
            for (int dy = -hz; dy <= hz; ++dy) {
              const int y = c.cy + dy;
              if (y < 0 || y >= d.ny) continue;
              paint_row(c, u, dy, hz2 - dy * dy, (size_t)z * sz + (size_t)y * sy, d.nx, touch, dt2,
                        labels, lt2);
            }
          }
        } else {
          const int y = c.cy + u;
          if (y >= 0 && y < d.ny)
            paint_row(c, 0, u, (int)c.r2 - u * u, (size_t)y * sy, d.nx, touch, dt2, labels, lt2);
        }
      }
    }
    __syncwarp();
  }
}

}  // namespace

uint32_t lt_table_r2cap(const Dims& d) {
  int m = std::min((d.nx + 1) / 2, (d.ny + 1) / 2);
  if (d.ndim == 3) m = std::min(m, (d.nz + 1) / 2);
  const uint64_t bound = (uint64_t)m * (uint64_t)m;
  return (uint32_t)(bound < kTableCap ? bound : kTableCap);
}

static size_t table_bytes(const Dims& d) {
  const int ncls = d.ndim == 3 ? 3 : 2;
  return align_up((size_t)ncls * (lt_table_r2cap(d) + 1) * sizeof(uint32_t));
}

size_t lt_workspace_bytes(const Dims& d) { return table_bytes(d) + align_up((size_t)d.n * sizeof(uint2)); }

cudaError_t lt_launch(const uint32_t* dt2, const uint32_t* labels, uint32_t* lt2, const Dims& d,
                      WsHeader* hdr, void* body, cudaStream_t s) {
  const uint32_t cap = lt_table_r2cap(d);
  const int ncls = d.ndim == 3 ? 3 : 2;
  uint32_t* tab = reinterpret_cast<uint32_t*>(body);
  uint2* surv = reinterpret_cast<uint2*>(reinterpret_cast<char*>(body) + table_bytes(d));
  cudaError_t e = cudaMemsetAsync(tab, 0, (size_t)ncls * (cap + 1) * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  int R = 0;
  while ((uint32_t)(R + 1) * (uint32_t)(R + 1) <= cap) ++R;
  const size_t pairs = (size_t)(R + 1) * (R + 1);
  const size_t want = (pairs + 255) / 256, cap_blocks = (size_t)sm_count() * 8;
  const unsigned tblocks = (unsigned)(want < cap_blocks ? want : cap_blocks);
  {
    TraceScope t("lt_table_points", s);
    mtable_points_kernel<<<tblocks, 256, 0, s>>>(tab, cap, R, d.ndim);
  }
  {
    TraceScope t("lt_table_prefix", s);
    mtable_prefix_kernel<<<ncls, 1024, 0, s>>>(tab, cap);
  }
  dim3 grid((d.nx + 255) / 256, (d.ny + kRidgeRows - 1) / kRidgeRows, d.nz);
  {
    TraceScope t("lt_ridge", s);
    if (d.ndim == 3)
      lt_ridge_kernel<3><<<grid, 256, 0, s>>>(dt2, labels, lt2, tab, cap, d, surv, hdr);
    else
      lt_ridge_kernel<2><<<grid, 256, 0, s>>>(dt2, labels, lt2, tab, cap, d, surv, hdr);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const unsigned pblocks = (unsigned)sm_count() * 8;
  {
    TraceScope t("lt_paint", s);
    if (d.ndim == 3)
      lt_paint_kernel<3><<<pblocks, 256, 0, s>>>(surv, dt2, labels, lt2, d, hdr);
    else
      lt_paint_kernel<2><<<pblocks, 256, 0, s>>>(surv, dt2, labels, lt2, d, hdr);
  }
  return cudaGetLastError();
}

}  // namespace ltk
