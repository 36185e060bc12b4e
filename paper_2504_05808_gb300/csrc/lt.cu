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
//    coordinates) by the symmetry of the lattice ball. It is tabulated for
//    r^2 <= 2^18; larger centres are never dropped.
// 2. Crescent painting. A kept centre c picks one higher-ranked same-label
//    neighbour D and raises LT2 only on voxels of B(c) outside B(D).
// Exactness, by induction down the rank order: every object voxel x in any
// B(c) ends with LT2(x) >= r_c^2. If c was dropped, x lies in a higher-ranked
// ball of radius >= r_c. If c is kept, x is either painted by c or lies in
// B(D) with r_D >= r_c. The highest-ranked centre paints its whole ball.
// Since only true ball radii are painted, LT2 is exactly the maximum.
//
// Crescent tables. B(c) \ B(c + d) depends only on (r_c^2, d, r_D^2), and a
// signed permutation of the axes maps it onto the crescent of the canonical
// offset of d's class, (1,0,0), (1,1,0) or (1,1,1). A kept centre has
// r_c^2 <= r_D^2 < M(d, r_c^2), about 2 |d| r_c values of r_D^2, so for
// r_c^2 <= 324 every crescent fits a table of 10.4 M voxel offsets. Such a
// centre paints its tabulated crescent voxel by voxel (lanes of a warp share
// the voxels of 32 centres). The dominant neighbour D is the one whose
// crescent is smallest (for larger radii: the one whose ball comes closest to
// containing c's). Centres with r^2 > 324, without a higher-ranked neighbour,
// or in 2D paint row by row instead.
//
// Voxels strictly inside B(c) are foreground (DT2(c) is the distance to the
// nearest background), so only points with |y - c|^2 == r_c^2 may be
// background; they are checked against DT2. Each ball voxel is joined to c by
// a face-connected path of strictly inner voxels, so when no two
// face-adjacent foreground voxels carry different labels (checked by the
// ridge kernel, flag `touch`) every foreground ball voxel has c's label and
// the label test is skipped.
//
// The tables are built once per process on the host and copied once per
// device into the arrays below (about 26 MiB of device memory).
#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>
#include <vector>

#include "lt_internal.cuh"
#include "tma.cuh"

#include <cudaTypedefs.h>

namespace ltk {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kMCap = 1u << 18;  // containment table covers r^2 <= 2^18
constexpr int kCresT = 324;           // crescent tables cover r^2 <= 324
constexpr int kCresMaxCombos = 1 << 15;
constexpr int kCresMaxVoxels = 16 * 1024 * 1024;  // both orderings (about 15.6 M voxels)
constexpr uint32_t kNoDominant = 31u;
constexpr uint32_t kTableRecord = 1u << 31;  // record z flag: painted from a crescent table
constexpr int kChunkCres = 64;  // largest crescent painted in shared chunks
constexpr int kChunkR2D = 64;   // 2D: largest r^2 painted in shared chunks (bigger discs: a warp each)
constexpr uint32_t kParts = 4096;      // warps sharing one big row-mode centre, at most
constexpr uint32_t kPartWork = 1024;  // row-mode work (voxels) per sharing warp, at least

// Centre records: at most one per voxel, plus the extra part records of the
// shared row-mode centres (at most n/8). The front list starts at 0, the
// back list at the last slot.
__host__ __device__ __forceinline__ size_t record_capacity(uint32_t n) { return (size_t)n + n / 8 + 4; }
constexpr int kNoTable = 0x3FFFFFFF;  // "never contained" beyond the table

__device__ uint32_t g_m3[3 * (kMCap + 1)];  // M for offset classes 1..3 (3D)
__device__ uint32_t g_m2[2 * (kMCap + 1)];  // M for offset classes 1..2 (2D)
__device__ uint32_t g_cres_base[3 * (kCresT + 1)];  // first combination of (class, r^2)
// per combination: x = first voxel | (size & 255) << 24, y = first voxel of
// the same crescent in the alternative order below | (size >> 8) << 24
__device__ uint2 g_cres_combo[kCresMaxCombos];
// (the same crescents with another canonical axis innermost: y for class 1,
// z for class 2; class 3 has one order)
// canonical crescent voxels: (x+128) | (y+128) << 8 | (z+128) << 16 |
// (on the sphere |y|^2 == r^2) << 24
__device__ uint32_t g_cres_vox[kCresMaxVoxels];

// ------------------------------------------------------------ host tables
struct HostTables {
  std::vector<uint32_t> m3, m2, base, start, start_alt, vox;
  std::vector<uint2> combo;
  bool ok = false;
};

int isqrt_host(int64_t v) {
  int64_t r = 0;
  while ((r + 1) * (r + 1) <= v) ++r;
  return (int)r;
}

HostTables* build_host_tables() {
  HostTables* t = new HostTables();
  const uint32_t cap = kMCap;
  t->m3.assign(3 * (size_t)(cap + 1), 0u);
  t->m2.assign(2 * (size_t)(cap + 1), 0u);
  const int R = isqrt_host(cap);
  // sorted lattice points y1 >= y2 (>= y3) >= 0: the largest |y - d|^2 over
  // the signed permutations of y is |y|^2 + 2 (sum of the cls largest |y_i|) + cls
  for (uint32_t y1 = 0; y1 <= (uint32_t)R; ++y1)
    for (uint32_t y2 = 0; y2 <= y1; ++y2) {
      const uint32_t n12 = y1 * y1 + y2 * y2;
      if (n12 > cap) break;
      t->m2[n12] = std::max(t->m2[n12], n12 + 2 * y1 + 1);
      t->m2[(cap + 1) + n12] = std::max(t->m2[(cap + 1) + n12], n12 + 2 * (y1 + y2) + 2);
      for (uint32_t y3 = 0; y3 <= y2; ++y3) {
        const uint32_t n = n12 + y3 * y3;
        if (n > cap) break;
        t->m3[n] = std::max(t->m3[n], n + 2 * y1 + 1);
        t->m3[(cap + 1) + n] = std::max(t->m3[(cap + 1) + n], n + 2 * (y1 + y2) + 2);
        t->m3[2 * (size_t)(cap + 1) + n] = std::max(t->m3[2 * (size_t)(cap + 1) + n], n + 2 * (y1 + y2 + y3) + 3);
      }
    }
  // prefix maximum over n: M(d, r^2) = max over |y|^2 <= r^2
  for (int k = 0; k < 3; ++k)
    for (uint32_t n = 1; n <= cap; ++n)
      t->m3[k * (size_t)(cap + 1) + n] = std::max(t->m3[k * (size_t)(cap + 1) + n], t->m3[k * (size_t)(cap + 1) + n - 1]);
  for (int k = 0; k < 2; ++k)
    for (uint32_t n = 1; n <= cap; ++n)
      t->m2[k * (size_t)(cap + 1) + n] = std::max(t->m2[k * (size_t)(cap + 1) + n], t->m2[k * (size_t)(cap + 1) + n - 1]);
  // crescents B(0, r^2) \ B(d, rd^2) for the canonical offsets, canonical
  // x innermost; then classes 1 and 2 again with canonical y (class 1) or z
  // (class 2) innermost, the axis that is world x when the offset has no x
  // component, so that consecutive voxels run along memory rows
  const int dl[3][3] = {{1, 0, 0}, {1, 1, 0}, {1, 1, 1}};
  // the lattice points of B(0, r^2) in the order with axis `inner` running
  // fastest, each with its squared distance to the class-k offset; a
  // crescent is the ordered subsequence with that distance above rd^2
  std::vector<std::pair<uint32_t, int>> pts;
  auto ball = [&](int k, int r2, int inner) {
    pts.clear();
    const int Rr = isqrt_host(r2);
    for (int u = -Rr; u <= Rr; ++u)
      for (int v = -Rr; v <= Rr; ++v)
        for (int w = -Rr; w <= Rr; ++w) {
          int c[3];  // canonical x, y, z; w runs along axis `inner`
          c[inner] = w;
          c[inner == 0 ? 1 : 0] = v;
          c[inner == 2 ? 1 : 2] = u;
          const int n = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
          if (n > r2) continue;
          const int e = (c[0] - dl[k][0]) * (c[0] - dl[k][0]) + (c[1] - dl[k][1]) * (c[1] - dl[k][1]) +
                        (c[2] - dl[k][2]) * (c[2] - dl[k][2]);
          pts.emplace_back((uint32_t)(c[0] + 128) | ((uint32_t)(c[1] + 128) << 8) |
                               ((uint32_t)(c[2] + 128) << 16) | ((n == r2 ? 1u : 0u) << 24),
                           e);
        }
  };
  auto crescent = [&](uint32_t rd2) {
    for (const auto& p : pts)
      if (p.second > (int)rd2) t->vox.push_back(p.first);
  };
  t->base.assign(3 * (kCresT + 1), 0u);
  for (int k = 0; k < 3; ++k)
    for (int r2 = 0; r2 <= kCresT; ++r2) {
      t->base[k * (kCresT + 1) + r2] = (uint32_t)t->start.size();
      const uint32_t mlim = t->m3[k * (size_t)(cap + 1) + r2];
      ball(k, r2, 0);
      for (uint32_t rd2 = (uint32_t)r2; rd2 < mlim; ++rd2) {
        t->start.push_back((uint32_t)t->vox.size());
        crescent(rd2);
      }
    }
  t->start.push_back((uint32_t)t->vox.size());  // end of the last crescent
  t->start_alt.assign(t->start.begin(), t->start.end() - 1);
  for (int k = 0; k < 2; ++k)
    for (int r2 = 0; r2 <= kCresT; ++r2) {
      const uint32_t mlim = t->m3[k * (size_t)(cap + 1) + r2];
      ball(k, r2, k == 0 ? 1 : 2);
      for (uint32_t rd2 = (uint32_t)r2; rd2 < mlim; ++rd2) {
        t->start_alt[t->base[k * (kCresT + 1) + r2] + (rd2 - r2)] = (uint32_t)t->vox.size();
        crescent(rd2);
      }
    }
  t->ok = t->start.size() <= (size_t)kCresMaxCombos + 1 && t->vox.size() <= (size_t)kCresMaxVoxels;
  // table records hold a crescent's size in 11 bits; the ridge kernel keeps
  // the first combination of each (class, r^2) in 16 bits
  for (size_t i = 0; i + 1 < t->start.size(); ++i) t->ok = t->ok && t->start[i + 1] - t->start[i] < 2048u;
  t->ok = t->ok && t->start.size() < (1u << 16) && t->vox.size() < (1u << 24);
  for (size_t i = 0; i + 1 < t->start.size(); ++i) {
    const uint32_t size = t->start[i + 1] - t->start[i];
    t->combo.push_back(make_uint2(t->start[i] | ((size & 255u) << 24), t->start_alt[i] | ((size >> 8) << 24)));
  }
  return t;
}

std::mutex g_tables_mu;
HostTables* g_host_tables = nullptr;
bool g_tables_on[64] = {false};

// Copies the tables to the current device on its first use.
cudaError_t ensure_tables() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_tables_mu);
  if (g_tables_on[dev]) return cudaSuccess;
  if (!g_host_tables) g_host_tables = build_host_tables();
  const HostTables& h = *g_host_tables;
  if (!h.ok) return cudaErrorInvalidValue;
  e = cudaMemcpyToSymbol(g_m3, h.m3.data(), h.m3.size() * 4);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_m2, h.m2.data(), h.m2.size() * 4);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_cres_base, h.base.data(), h.base.size() * 4);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_cres_combo, h.combo.data(), h.combo.size() * sizeof(uint2));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_cres_vox, h.vox.data(), h.vox.size() * 4);
  if (e == cudaSuccess) g_tables_on[dev] = true;
  return e;
}

__device__ __forceinline__ uint32_t cres_combo(const uint16_t* base, int cls, uint32_t r2, uint32_t rd2) {
  return base[cls * (kCresT + 1) + r2] + (rd2 - r2);
}

// ---------------------------------------------------------- ridge kernel
// Clears LT2, validates labels against the mask, sets the `touch` flag,
// applies the containment test, appends kept centres and (optionally) takes
// the largest DT2 of every object (the largest DT2 of an object is that of
// its highest-ranked voxel, which no neighbour's ball can hold, so the
// maximum over kept centres is the maximum over the object).
//
// A CTA owns a 64 x 8 (x, y) column tile and marches along z through RZ
// planes; warp w takes row y0 + w, lane j the voxels x0 + j and x0 + 32 + j.
// Halo planes of DT2 and labels (x0-4 .. x0+67 so that the TMA x coordinate
// stays 16-byte aligned; y0-1 .. y0+8) sit in a ring of four shared-memory
// slots. With TMA (row pitch a multiple of 16 bytes) one thread issues a
// tiled bulk copy per plane and array, completing on the slot's mbarrier;
// otherwise all threads load planes with plain loads. Outside the array the
// halo holds (0, 0), which never matches an object label.
// Three stages, software-pipelined so that one CTA barrier per plane
// separates them (iteration z runs stage 1 of plane z, stage 2 of plane
// z - 1 and stage 3 of plane z - 2, on planes z - 2 .. z of the ring; the
// lists between stages alternate by plane parity):
//   stage 1  every voxel: clear LT2, check the label against the mask,
//            compact the labelled foreground voxels;
//   stage 2  the compacted voxels, full warps: per neighbour class (1, 2 or
//            3 nonzero offset coordinates) the largest key (r'^2 << 6 | rank
//            bit << 5 | offset code) over same-label neighbours; r'^2 against
//            M(class, r^2) decides containment; a face neighbour in the
//            foreground with another label sets `touch` (every such pair has
//            a labelled side, so looking from labelled voxels finds them
//            all); kept voxels are compacted again with their keys (up to
//            kKeptQ per plane; a voxel beyond that builds its record here);
//   stage 3  the kept voxels, full warps: dominant and extra neighbours (a
//            key ranking above the centre) and the record.
// Kept centres collect in one shared buffer (front list from its front,
// back list from its back) and leave with one global atomic per list
// whenever another plane might not fit (the two list counters are hot, one
// atomic per flush keeps them from serialising the CTAs). The front of
// `surv` gets the centres painted in shared chunks: 3D centres with r^2 <=
// kCresT, a dominant neighbour and a crescent of at most kChunkCres voxels,
// and every 2D centre. The back gets those a warp paints alone: bigger
// crescents and the centres painted row by row.
// Records (uint4). Offset codes: (dz+1)*9 + (dy+1)*3 + (dx+1), 31 for none.
//   Table centres (3D): x = linear index; y = first crescent voxel; z = r^2 |
//   dominant code << 9 | codes of up to two more higher-ranked same-label
//   neighbours << 14 (5 bits each) | ball inside the array << 24 |
//   kTableRecord; w = those two neighbours' r^2 (9 bits each, 0x1FF none) |
//   crescent size << 18.
//   Painting needs no other lookup.
//   Row centres and 2D: x = linear index, y = r^2 | dominant code << 25,
//   z = the two extra codes; w = part | parts << 16 (row-mode centres go to
//   the back list directly; a big one as up to kParts records, one per
//   part, while the extra records stay within n/8).
constexpr int kTX = 64, kTY = 8;
constexpr int kTile = kTX * kTY;                   // voxels per tile plane (2 per thread)
constexpr int kOX = 4;                             // halo column of x0 (keeps TMA x 16-byte aligned)
constexpr int kBX = kTX + 2 * kOX, kBY = kTY + 2;  // TMA box: 72 x 10 words
constexpr int kSlotPitch = 736;                    // words per slot: 72 x 10 rounded up to 128 bytes
constexpr int kSlots = 4;                          // planes z-2 .. z in use, z+1 in flight
constexpr int kListBuf = 832;  // kept centres buffered per CTA (a plane adds at most kTile)
constexpr int kKeptQ = 128;    // kept voxels per plane handed from stage 2 to stage 3
constexpr uint32_t kPlaneBytes = kBX * kBY * 4;
static_assert(kSlotPitch * 4 % 128 == 0 && kSlotPitch >= kBX * kBY, "slot layout");
static_assert(kListBuf >= kTile && kSlots == 4 && kKeptQ <= 256, "buffer, ring and list sizes");

// Wait: the time limit of each plane wait. extra_tx: bytes each plane's
// barrier expects beyond its two copies, 0 except in the timeout self-test,
// where it makes every wait reach its limit.
struct RidgeWait {
  uint64_t limit_ns = kWaitNs;
  uint32_t extra_tx = 0;
  uint32_t chunk_cres = kChunkCres;  // largest crescent of the front list (shared chunks)
};

// The record of kept centre at tile position (tx, ty) of plane zc from its
// three class keys (see the ridge kernel); also decides which list takes
// it. Row-mode centres shared by several warps are written to the back of
// `surv` at once (keepA = keepB = false).
template <int NDIM>
__device__ __forceinline__ uint4 make_record(uint32_t r2, const uint32_t kmax[3], int tx, int ty, int zc, int x0,
                                             int y0, const Dims& d, const uint32_t* mt, const uint16_t* sbase,
                                             uint4* __restrict__ surv, WsHeader* __restrict__ hdr,
                                             uint32_t chunk_cres, bool& keepA, bool& keepB) {
  // candidates: per class the largest key when it ranks above c (2 r'^2 +
  // bit > 2 r^2)
  int brn[3] = {-1, -1, -1};
  uint32_t bcode[3] = {kNoDominant, kNoDominant, kNoDominant};
#pragma unroll
  for (int k = 0; k < (NDIM == 3 ? 3 : 2); ++k)
    if ((kmax[k] >> 5) > 2 * r2) {
      brn[k] = (int)(kmax[k] >> 6);
      bcode[k] = kmax[k] & 31u;
    }
  uint32_t code = kNoDominant, vstart = 0, best = UINT_MAX;
  int kd = -1;
  if (NDIM == 3 && r2 <= (uint32_t)kCresT) {
    // the candidate whose crescent has the fewest voxels; its voxels in the
    // order with world x innermost (the alternative order when the offset
    // has no x component)
    uint2 ce[3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
      ce[k] = brn[k] >= 0 ? g_cres_combo[cres_combo(sbase, k, r2, (uint32_t)brn[k])] : make_uint2(0u, 0u);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const uint32_t sz = (ce[k].x >> 24) | ((ce[k].y >> 24) << 8);
      if (brn[k] >= 0 && sz < best) {
        best = sz;
        vstart = (bcode[k] % 3 == 1 ? ce[k].y : ce[k].x) & 0xFFFFFFu;
        code = bcode[k];
        kd = k;
      }
    }
  } else {
    // the candidate whose ball comes closest to containing c's
    int m[3] = {kNoTable, kNoTable, kNoTable};
    if (r2 <= kMCap) {
      m[0] = (int)mt[r2];
      m[1] = (int)mt[(kMCap + 1) + r2];
      if (NDIM == 3) m[2] = (int)mt[2 * (kMCap + 1) + r2];
    }
    int bestm = INT_MIN;
#pragma unroll
    for (int k = 0; k < (NDIM == 3 ? 3 : 2); ++k)
      if (brn[k] >= 0 && brn[k] - m[k] > bestm) {
        bestm = brn[k] - m[k];
        code = bcode[k];
        kd = k;
      }
  }
  const int x = x0 + tx, y = y0 + ty;
  const uint32_t v = (uint32_t)(((size_t)zc * d.ny + (size_t)y) * d.nx + (size_t)x);
  // the other classes' candidates: extra balls a crescent voxel may lie in,
  // with their r^2 (below M(d, r^2) < 400 for table centres; 9 bits each)
  uint32_t extra = kNoDominant | (kNoDominant << 5), er = 0x3FFFFu, ne = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k)
    if (NDIM == 3 && k != kd && brn[k] >= 0 && ne < 2) {
      extra = (extra & ~(31u << (5 * ne))) | (bcode[k] << (5 * ne));
      er = (er & ~(0x1FFu << (9 * ne))) | ((uint32_t)min(brn[k], 0x1FE) << (9 * ne));
      ++ne;
    }
  const bool tab = NDIM == 2 || (r2 <= (uint32_t)kCresT && code != kNoDominant);
  uint4 rec;
  if (NDIM == 3 && tab) {
    // the ball inside the array: R <= x, x + R < nx per axis, R =
    // floor(sqrt(r^2)); R <= k exactly when r^2 < (k + 1)^2
    auto fits = [&](int vv, int nv) {
      return (int64_t)r2 < (int64_t)(vv + 1) * (vv + 1) && (int64_t)r2 < (int64_t)(nv - vv) * (nv - vv);
    };
    const uint32_t inside = fits(x, d.nx) && fits(y, d.ny) && fits(zc, d.nz);
    rec = make_uint4(v, vstart, r2 | (code << 9) | (extra << 14) | (inside << 24) | kTableRecord, er | (best << 18));
  } else {
    rec = make_uint4(v, r2 | (code << 25), extra, 0u);
  }
  // small crescents are shared out in chunks; a big one takes a warp
  keepA = tab && (NDIM == 2 ? r2 <= (uint32_t)kChunkR2D : best <= chunk_cres);
  keepB = !keepA;
  if (keepB && (NDIM == 2 || !tab)) {
    // painted row by row. Work: without a dominant the whole ball, else
    // about 4 voxels' worth per row that can meet the crescent's cap (see
    // cap_rows: depth along d about R + T / (2 |d|), T = |d|^2 - (rD^2 -
    // r^2); the rows through a cap of depth t and base radius a number about
    // pi a^2 + 2 a (t + 3)). A centre with more than kPartWork of it per
    // warp (8 kPartWork with a dominant) is written at once as up to kParts
    // records, one per warp sharing it (w = part | parts << 16), while the
    // extra records fit their budget of n/8; the others go to the back list
    // like big table crescents.
    const int R = (int)isqrt24(r2), side = 2 * R + 1;
    float work;
    if (code == kNoDominant) {
      work = NDIM == 3 ? 4.19f * (float)R * (float)R * (float)R : 3.1416f * (float)R * (float)R;
    } else {
      float rows = (float)(NDIM == 3 ? side * side : side);
      if (NDIM == 3 && kd >= 0) {
        const float dn = sqrtf((float)(kd + 1));
        const float t = fminf(fmaxf((float)R + (float)(kd + 1 - (brn[kd] - (int)r2)) / (2.0f * dn), 0.0f), (float)side);
        const float a = sqrtf(fmaxf(t * ((float)side - t), 0.0f));
        rows = fminf(rows, 3.1416f * a * a + 2.0f * a * (t + 3.0f) + 2.0f * t + 16.0f);
      }
      work = 4.0f * rows;
    }
    // (a cap's rows are mostly cut further by the extra balls, so a centre
    // with a dominant is split only when its cap is very large)
    const float per_part = code == kNoDominant ? (float)kPartWork : 8.0f * (float)kPartWork;
    uint32_t parts = min(kParts, max(1u, (uint32_t)(work / per_part)));
    if (parts > 1 && atomicAdd(&hdr->n_extra, parts - 1) + (parts - 1) > d.n / 8) parts = 1;
    if (parts > 1) {
      keepB = false;
      const uint32_t bb = atomicAdd(&hdr->n_big, parts);
      for (uint32_t q = 0; q < parts; ++q)
        surv[record_capacity(d.n) - 1 - (bb + q)] = make_uint4(rec.x, rec.y, rec.z, q | (parts << 16));
    }
  }
  return rec;
}

// Shared memory of one ridge CTA (declared by the kernels, so that a kernel
// that picks the TMA or the plain-load body at run time holds it once).
template <int NDIM>
struct RidgeSmem {
  __align__(128) uint32_t sD[kSlots][kSlotPitch];
  __align__(128) uint32_t sL[kSlots][kSlotPitch];
  uint4 buf[kListBuf];
  uint4 keptq[2][kKeptQ];   // stage 2 -> stage 3: (tile position, class keys), by plane parity
  uint16_t work[2][kTile];  // stage 1 -> stage 2, by plane parity
  __align__(8) uint64_t bar[kSlots];
  uint32_t cntA, cntB, baseA, baseB, flags;
  // list counts by plane mod 3: filled in one iteration, read in the next,
  // cleared in the one after
  uint32_t nwork_s[3], nkept_s[3];
  // records each warp appended since the last flush, published before the
  // barrier of plane z in slot z & 1 (untouched until the next barrier), so
  // that every thread reads the same total after it
  uint32_t wrec[2][8];
  uint16_t sbase[NDIM == 3 ? 3 * (kCresT + 1) : 2];  // copy of g_cres_base
};

// One CTA of the ridge pass: column tile (blk.x, blk.y), z chunk blk.z.
template <int NDIM, int RZ, bool TMA>
__device__ __forceinline__ void ridge_body(RidgeSmem<NDIM>& sm, const CUtensorMap* map_dt2,
                                           const CUtensorMap* map_lab, const uint32_t* __restrict__ dt2,
                                           const uint32_t* __restrict__ labels, uint32_t* __restrict__ lt2,
                                           const Dims& d, uint4* __restrict__ surv, WsHeader* __restrict__ hdr,
                                           const RidgeWait& wt, int z_base, uint32_t* __restrict__ max_dt2,
                                           uint32_t n_labels, uint3 blk) {
  auto& sD = sm.sD;
  auto& sL = sm.sL;
  auto& buf = sm.buf;
  auto& keptq = sm.keptq;
  auto& work = sm.work;
  auto& bar = sm.bar;
  auto& cntA = sm.cntA;
  auto& cntB = sm.cntB;
  auto& baseA = sm.baseA;
  auto& baseB = sm.baseB;
  auto& flags = sm.flags;
  auto& nwork_s = sm.nwork_s;
  auto& nkept_s = sm.nkept_s;
  auto& wrec = sm.wrec;
  auto& sbase = sm.sbase;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int x0 = (int)blk.x * kTX, y0 = (int)blk.y * kTY;
  const int z0 = NDIM == 3 ? (int)blk.z * RZ + z_base : 0;
  const int z1 = NDIM == 3 ? min(d.nz, z0 + RZ) : 1;
  const size_t plane = (size_t)d.nx * d.ny;
  const uint32_t* mt = NDIM == 3 ? g_m3 : g_m2;
  const unsigned below = (1u << lane) - 1u;
  // plane p lives in slot (p - z0 + 1) mod kSlots; its copy is the k-th into
  // that slot, k = (p - z0 + 1) / kSlots, completing the barrier phase of
  // parity k & 1
  auto slot_of = [&](int p) { return (int)((uint32_t)(p - z0 + 1) % kSlots); };
  auto parity_of = [&](int p) { return ((uint32_t)(p - z0 + 1) / kSlots) & 1u; };
  auto issue = [&](int p) {
    const int s = slot_of(p);
    mbar_expect_tx(&bar[s], 2 * kPlaneBytes + wt.extra_tx);
    tma_load_3d(sD[s], map_dt2, x0 - kOX, y0 - 1, p, &bar[s]);
    tma_load_3d(sL[s], map_lab, x0 - kOX, y0 - 1, p, &bar[s]);
  };
  // without TMA: asynchronous 4-byte copies of the halo plane (zeros outside
  // the array), one commit group per plane
  // (a thread's halo positions i = tid + 256 k are the same in every plane:
  // their shared-memory index and in-plane offset, -1 outside the array, are
  // worked out once)
  constexpr int kHalo = (kTX + 2) * kBY, kPerThread = (kHalo + 255) / 256;
  int hoff[kPerThread];
  uint32_t hdst = 0;  // shared-memory indices, 10 bits each
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    const int i = tid + 256 * k;
    const int hx = i % (kTX + 2), hy = i / (kTX + 2);
    const int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
    hoff[k] = i < kHalo && gx >= 0 && gx < d.nx && gy >= 0 && gy < d.ny ? gy * d.nx + gx : -1;
    hdst |= (uint32_t)(i < kHalo ? hy * kBX + hx + kOX - 1 : 0) << (10 * k);
  }
  static_assert(kPerThread <= 3 && kBX * kBY <= 1024, "halo positions per thread, index bits");
  auto load_plane = [&](int z) {
    const int s = slot_of(z);
    const bool zin = z >= 0 && z < d.nz;
#pragma unroll
    for (int k = 0; k < kPerThread; ++k)
      if (tid + 256 * k < kHalo) {
        const bool in = zin && hoff[k] >= 0;
        const size_t g = in ? (size_t)z * plane + (size_t)hoff[k] : 0;
        const int dst = (int)((hdst >> (10 * k)) & 1023u);
        cp_async4(&sD[s][dst], dt2 + g, in);
        cp_async4(&sL[s][dst], labels + g, in);
      }
    cp_async_commit();
  };
  // appends records to the shared buffer: list A from its front, list B
  // from its back (all lanes of the warp call it)
  uint32_t appended = 0;  // records this warp appended since the last flush
  auto append = [&](bool keepA, bool keepB, const uint4& rec) {
    const unsigned ba = __ballot_sync(kFull, keepA), bb = __ballot_sync(kFull, keepB);
    appended += (uint32_t)(__popc(ba) + __popc(bb));
    if (ba) {
      uint32_t wb = 0;
      if (lane == 0) wb = atomicAdd(&cntA, (uint32_t)__popc(ba));
      wb = __shfl_sync(kFull, wb, 0);
      if (keepA) buf[wb + __popc(ba & below)] = rec;
    }
    if (bb) {
      uint32_t wb = 0;
      if (lane == 0) wb = atomicAdd(&cntB, (uint32_t)__popc(bb));
      wb = __shfl_sync(kFull, wb, 0);
      if (keepB) buf[kListBuf - 1 - (wb + __popc(bb & below))] = rec;
    }
  };
  if (NDIM == 3)
    for (int i = tid; i < 3 * (kCresT + 1); i += 256) sbase[i] = (uint16_t)g_cres_base[i];
  if (tid == 0) {
    cntA = cntB = 0;
    // after a timeout anywhere in this launch, the remaining CTAs stop at once
    flags = TMA && (*(volatile uint32_t*)&hdr->error & ERR_TIMEOUT) ? 4u : 0u;
    for (int k = 0; k < 3; ++k) nwork_s[k] = nkept_s[k] = 0;
    if (TMA) {
      for (int s = 0; s < kSlots; ++s) mbar_init(&bar[s], 1);
      fence_barrier_init();
    }
  }
  __syncthreads();
  if (flags & 4u) return;
  if (TMA) {
    if (tid == 0)
      for (int p = z0 - 1; p <= min(z1, z0 + 1); ++p) issue(p);
  } else {
    load_plane(z0 - 1);
    load_plane(z0);
    cp_async_wait_none();
    __syncthreads();
  }
  bool touch = false;  // this thread saw two face-adjacent foreground voxels with different labels
  for (int z = z0; z <= z1 + 1; ++z) {
    // plane z (and at the start plane z0 - 1) must have arrived
    bool ok = true;
    if (z <= z1) {
      if (TMA) {
        if (z == z0) ok = mbar_wait(&bar[slot_of(z - 1)], parity_of(z - 1), wt.limit_ns);
        ok = ok && mbar_wait(&bar[slot_of(z)], parity_of(z), wt.limit_ns);
      } else if (z + 1 <= z1) {
        // plane z + 1 (into the slot plane z - 3 left in the last iteration)
        // flies while this plane is worked on; each thread waits for its
        // copies before the plane barrier below, which shows them all
        load_plane(z + 1);
      }
    }
    // stage 1, every voxel of plane z: clear LT2, label check, compaction.
    // (After a timed-out wait the stages read stale shared memory; they only
    // write LT2 voxels and records of this tile, and the CTA stops below.)
    if (z < z1) {
      const int y = y0 + warp;
      const uint32_t* D0 = sD[slot_of(z)];
      const uint32_t* L0 = sL[slot_of(z)];
      uint16_t* wl = work[z & 1];
      bool bad = false;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int tx = lane + 32 * j, x = x0 + tx;
        const bool in = x < d.nx && y < d.ny;
        const int c = (warp + 1) * kBX + (tx + kOX);
        const uint32_t md = D0[c], ml = L0[c];
        if (in) lt2[(size_t)z * plane + (size_t)y * d.nx + x] = 0u;
        bad = bad || (in && md == 0 && ml != 0);
        const bool isw = in && md != 0 && ml != 0;
        const unsigned bal = __ballot_sync(kFull, isw);
        uint32_t off = 0;
        if (lane == 0 && bal) off = atomicAdd(&nwork_s[z % 3], (uint32_t)__popc(bal));
        off = __shfl_sync(kFull, off, 0);
        if (isw) wl[off + __popc(bal & below)] = (uint16_t)(warp * kTX + tx);
      }
      if (__any_sync(kFull, bad) && lane == 0) atomicOr(&flags, 1u);
    }
    // stage 2, the labelled voxels of plane zc = z - 1: containment test
    if (z > z0 && z <= z1) {
      const int zc = z - 1;
      const uint32_t nwork = nwork_s[zc % 3];  // complete: filled before the last barrier
      const uint32_t* Dm = sD[slot_of(zc - 1)];
      const uint32_t* D0 = sD[slot_of(zc)];
      const uint32_t* Dp = sD[slot_of(zc + 1)];
      const uint32_t* Lm = sL[slot_of(zc - 1)];
      const uint32_t* L0 = sL[slot_of(zc)];
      const uint32_t* Lp = sL[slot_of(zc + 1)];
      const uint16_t* wl = work[zc & 1];
      uint4* kq = keptq[zc & 1];
      for (uint32_t base = 0; base < nwork; base += 256) {  // uniform
        const uint32_t i = base + (uint32_t)tid;
        bool kept = false;
        uint32_t r2 = 0, l = 0, t = 0;
        uint32_t kmax[3] = {0u, 0u, 0u};
        if (i < nwork) {
          t = wl[i];
          const int c = (int)(t / kTX + 1) * kBX + (int)(t % kTX) + kOX;
          r2 = D0[c];
          l = L0[c];
          int m[3] = {kNoTable, kNoTable, kNoTable};
          if (r2 <= kMCap) {
            m[0] = (int)mt[r2];
            m[1] = (int)mt[(kMCap + 1) + r2];
            if (NDIM == 3) m[2] = (int)mt[2 * (kMCap + 1) + r2];
          }
#pragma unroll
          for (int dz = (NDIM == 3 ? -1 : 0); dz <= (NDIM == 3 ? 1 : 0); ++dz) {
            const uint32_t* Dz = dz < 0 ? Dm : (dz == 0 ? D0 : Dp);
            const uint32_t* Lz = dz < 0 ? Lm : (dz == 0 ? L0 : Lp);
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
              for (int dx = -1; dx <= 1; ++dx) {
                if (dx == 0 && dy == 0 && dz == 0) continue;
                const int h = c + dy * kBX + dx;
                const uint32_t nd = Dz[h], nl = Lz[h];
                const int k = (dx != 0) + (dy != 0) + (dz != 0) - 1;
                const uint32_t pos = dz > 0 || (dz == 0 && (dy > 0 || (dy == 0 && dx > 0)));
                const uint32_t key = (nd << 6) | (pos << 5) | (uint32_t)((dz + 1) * 9 + (dy + 1) * 3 + (dx + 1));
                kmax[k] = max(kmax[k], nl == l ? key : 0u);
                if (k == 0) touch = touch || (nd != 0 && nl != l);
              }
            }
          }
          bool pruned = false;
#pragma unroll
          for (int k = 0; k < (NDIM == 3 ? 3 : 2); ++k) pruned = pruned || (int)(kmax[k] >> 6) >= m[k];
          kept = !pruned;
        }
        // largest DT2 per object: one atomic per group of equal labels in the warp
        if (max_dt2) {
          const bool has = kept && l < n_labels;
          const unsigned act = __ballot_sync(kFull, has);
          if (has) {
            const unsigned grp = __match_any_sync(act, l);
            const uint32_t mx = __reduce_max_sync(grp, r2);
            if (lane == __ffs(grp) - 1) atomicMax(max_dt2 + l, mx);
          }
        }
        // kept voxels to stage 3; those beyond its list build their record now
        const unsigned bk = __ballot_sync(kFull, kept);
        uint32_t off = 0;
        if (lane == 0 && bk) off = atomicAdd(&nkept_s[zc % 3], (uint32_t)__popc(bk));
        off = __shfl_sync(kFull, off, 0) + __popc(bk & below);
        const bool late = kept && off >= (uint32_t)kKeptQ;
        if (kept && !late) kq[off] = make_uint4(t, kmax[0], kmax[1], kmax[2]);
        if (__any_sync(kFull, late)) {
          bool keepA = false, keepB = false;
          uint4 rec = make_uint4(0u, 0u, 0u, 0u);
          if (late)
            rec = make_record<NDIM>(r2, kmax, (int)(t % kTX), (int)(t / kTX), zc, x0, y0, d, mt, sbase, surv, hdr,
                                    wt.chunk_cres, keepA, keepB);
          append(keepA, keepB, rec);
        }
      }
    }
    // stage 3, the kept voxels of plane zr = z - 2: records
    if (z > z0 + 1) {
      const int zr = z - 2;
      const uint32_t nkept = min(nkept_s[zr % 3], (uint32_t)kKeptQ);
      const uint32_t* D0 = sD[slot_of(zr)];
      const uint4* kq = keptq[zr & 1];
      if ((uint32_t)(255 - tid) < ((nkept + 31u) & ~31u)) {  // the last warps, whole warps
        const uint32_t i = (uint32_t)(255 - tid);
        bool keepA = false, keepB = false;
        uint4 rec = make_uint4(0u, 0u, 0u, 0u);
        if (i < nkept) {
          const uint4 q = kq[i];
          const int tx = (int)(q.x % kTX), ty = (int)(q.x / kTX);
          const uint32_t r2 = D0[(ty + 1) * kBX + tx + kOX];
          const uint32_t kmax[3] = {q.y, q.z, q.w};
          rec = make_record<NDIM>(r2, kmax, tx, ty, zr, x0, y0, d, mt, sbase, surv, hdr, wt.chunk_cres, keepA, keepB);
        }
        append(keepA, keepB, rec);
      }
    }
    if (tid == 0) {
      nwork_s[(z + 1) % 3] = 0;  // plane z - 2's count: read in iteration z - 1, refilled in z + 1
      nkept_s[z % 3] = 0;        // plane z - 3's count: read in iteration z - 1, refilled in z + 1
    }
    if (lane == 0) wrec[z & 1][warp] = appended;
    if (!TMA) cp_async_wait_none();  // plane z + 1 has landed (this thread's part)
    // the one barrier of the plane; it also agrees on a timed-out wait
    if (__syncthreads_or(!ok)) {
      // record the timeout, wait (again bounded) for the copies this CTA
      // still has in flight, and stop
      if (tid == 0) {
        atomicOr(&hdr->error, ERR_TIMEOUT);
        for (int p = z; p <= min(z1, z + 1); ++p) mbar_wait(&bar[slot_of(p)], parity_of(p), wt.limit_ns);
      }
      return;
    }
    // plane z - 2 is free again: its slot takes plane z + 2
    if (TMA && tid == 0 && z + 2 <= z1) {
      fence_proxy_async();
      issue(z + 2);
    }
    // buffered records: the same sum for every thread (fast warps already
    // append the next plane's records, to cntA/cntB and to the other slot)
    uint32_t held = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) held += wrec[z & 1][w];
    if (held > (uint32_t)(kListBuf - kTile) || z == z1 + 1) {  // uniform
      // nobody appends until the second barrier below: the counts are final
      const uint32_t nA = cntA, nB = cntB;
      // the two list atomics from two warps, so that their latencies overlap
      if (tid == 0) baseA = nA ? atomicAdd(&hdr->n_surv, nA) : 0u;
      if (tid == 32) baseB = nB ? atomicAdd(&hdr->n_big, nB) : 0u;
      __syncthreads();
      if (tid == 0) cntA = cntB = 0;
      for (uint32_t i = tid; i < nA; i += 256) surv[baseA + i] = buf[i];
      for (uint32_t i = tid; i < nB; i += 256) surv[record_capacity(d.n) - 1 - (baseB + i)] = buf[kListBuf - 1 - i];
      appended = 0;
      __syncthreads();
    }
  }
  if (__syncthreads_or(touch) && tid == 0) atomicOr(&hdr->touch, 1u);
  if (tid == 0 && (flags & 1u)) atomicOr(&hdr->error, ERR_LABEL_OUTSIDE_MASK);
}

template <int NDIM, int RZ, bool TMA>
__global__ void __launch_bounds__(256) lt_ridge_kernel(const __grid_constant__ CUtensorMap map_dt2,
                                                       const __grid_constant__ CUtensorMap map_lab,
                                                       const uint32_t* __restrict__ dt2,
                                                       const uint32_t* __restrict__ labels,
                                                       uint32_t* __restrict__ lt2, Dims d,
                                                       uint4* __restrict__ surv,
                                                       WsHeader* __restrict__ hdr, RidgeWait wt, int z_base,
                                                       uint32_t* __restrict__ max_dt2, uint32_t n_labels) {
  __shared__ RidgeSmem<NDIM> sm;
  ridge_body<NDIM, RZ, TMA>(sm, &map_dt2, &map_lab, dt2, labels, lt2, d, surv, hdr, wt, z_base, max_dt2, n_labels,
                            make_uint3(blockIdx.x, blockIdx.y, blockIdx.z));
}

// The ridge pass over many volumes (each with its own workspace: header and
// centre records); with TMA every volume of the launch has tensor maps.
template <int NDIM, int RZ, bool TMA>
__global__ void __launch_bounds__(256, 5) lt_ridge_multi_kernel(MultiArgs m, RidgeWait wt) {
  __shared__ RidgeSmem<NDIM> sm;
  uint3 blk;
  const VolParams& p = m.vols[find_volume(m, blockIdx.x, blk)];
  ridge_body<NDIM, RZ, TMA>(sm, reinterpret_cast<const CUtensorMap*>(p.map_dt2),
                            reinterpret_cast<const CUtensorMap*>(p.map_lab), p.dt2, p.labels, p.lt2, p.d,
                            reinterpret_cast<uint4*>(p.body), p.hdr, wt, 0, nullptr, 0u, blk);
}

// ---------------------------------------------------------- paint kernel
struct Centre {
  int cx, cy, cz, R;
  uint32_t r2, label, idx;
  int ddx, ddy, ddz, r2d;  // dominant neighbour offset and its r^2 (-1: none)
  int start, nseg;         // first item of this centre in the chunk; dy segments
  float inv_nseg;
  int eoff[2], er2[2];     // 3D row mode: two more higher-ranked balls, offset code and r^2 (-1: none)
};
constexpr int kRowSeg = 8;  // rows per row-mode work item

// Raises LT2 to c.r2 on row voxels dx in [a, b] (already clamped to the
// array). Only the two ends of an exact row (w^2 == h) can be background.
__device__ __forceinline__ void paint_span(const Centre& c, int a, int b, int w, bool exact,
                                           size_t rowbase, bool touch,
                                           const uint32_t* __restrict__ dt2,
                                           const uint32_t* __restrict__ labels,
                                           uint32_t* __restrict__ lt2, uint32_t& nupd) {
  for (int dx = a; dx <= b; ++dx) {
    const size_t i = rowbase + (size_t)(c.cx + dx);
    if (exact && (dx == w || dx == -w) && dt2[i] == 0) continue;
    if (touch && labels[i] != c.label) continue;
    atomicMax(lt2 + i, c.r2);
    ++nupd;
  }
}

// Row mode: rows dy0..dy0+7 of the disc at height dz, minus the dominant
// neighbour's rows; half-widths are updated incrementally along the segment.
__device__ __forceinline__ void paint_rows(const Centre& c, int dz, int seg, const Dims& d, size_t sy,
                                           size_t sz, bool touch, const uint32_t* __restrict__ dt2,
                                           const uint32_t* __restrict__ labels,
                                           uint32_t* __restrict__ lt2, uint32_t& nupd) {
  const int z = c.cz + dz;
  if (z < 0 || z >= d.nz) return;
  const int hz2 = (int)c.r2 - dz * dz;
  const int dy0 = -c.R + seg * kRowSeg, dy1 = min(c.R, dy0 + kRowSeg - 1);
  const int xmin = -c.cx, xmax = d.nx - 1 - c.cx;
  int wr = -1, wd = -1;
  for (int dy = dy0; dy <= dy1; ++dy) {
    const int h = hz2 - dy * dy;
    const int y = c.cy + dy;
    if (h < 0 || y < 0 || y >= d.ny) continue;
    if (wr < 0) wr = (int)isqrt24((uint32_t)h);
    while (wr * wr > h) --wr;
    while ((wr + 1) * (wr + 1) <= h) ++wr;
    int hi1 = wr, lo2 = 1, hi2 = 0;  // pieces [-wr, hi1] and [lo2, hi2]
    if (c.r2d >= 0) {
      const int hd = c.r2d - (dz - c.ddz) * (dz - c.ddz) - (dy - c.ddy) * (dy - c.ddy);
      if (hd >= 0) {
        if (wd < 0) wd = (int)isqrt24((uint32_t)hd);
        while (wd * wd > hd) --wd;
        while ((wd + 1) * (wd + 1) <= hd) ++wd;
        hi1 = min(wr, c.ddx - wd - 1);
        lo2 = max(-wr, c.ddx + wd + 1);
        hi2 = wr;
      }
    }
    const bool exact = wr * wr == h;
    const size_t rowbase = (size_t)z * sz + (size_t)y * sy;
    paint_span(c, max(-wr, xmin), min(hi1, xmax), wr, exact, rowbase, touch, dt2, labels, lt2, nupd);
    paint_span(c, max(lo2, xmin), min(hi2, xmax), wr, exact, rowbase, touch, dt2, labels, lt2, nupd);
  }
}

// Decodes a row-mode record (3D row centres, every 2D centre); returns its
// number of work items: (2R+1) * ceil((2R+1)/8) row segments in 3D,
// ceil((2R+1)/8) in 2D.
template <int NDIM>
__device__ __forceinline__ int make_centre(uint4 rec, const Dims& d, size_t sy, size_t sz, bool touch,
                                           const uint32_t* __restrict__ dt2,
                                           const uint32_t* __restrict__ labels, Centre& c) {
  const uint32_t idx = rec.x, code = rec.y >> 25;
  c.idx = idx;
  c.r2 = rec.y & 0x1FFFFFFu;
  c.cx = (int)(idx % (uint32_t)d.nx);
  const uint32_t t = idx / (uint32_t)d.nx;
  c.cy = (int)(t % (uint32_t)d.ny);
  c.cz = (int)(t / (uint32_t)d.ny);
  c.R = (int)isqrt24(c.r2);
  c.label = touch ? labels[idx] : 0u;
  c.start = 0;
  if (code != kNoDominant) {
    c.ddz = (int)(code / 9) - 1;
    c.ddy = (int)(code / 3 % 3) - 1;
    c.ddx = (int)(code % 3) - 1;
    c.r2d = (int)dt2[(int64_t)idx + c.ddz * (int64_t)sz + c.ddy * (int64_t)sy + c.ddx];
  } else {
    c.ddx = c.ddy = c.ddz = 0;
    c.r2d = -1;
  }
  c.nseg = (2 * c.R + kRowSeg) / kRowSeg;
  c.inv_nseg = 1.0f / (float)c.nseg;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const uint32_t ec = (rec.z >> (5 * q)) & 31u;
    c.eoff[q] = (int)ec;
    c.er2[q] = -1;
    if (NDIM == 3 && ec != kNoDominant) {
      const int ez = (int)(ec / 9) - 1, ey = (int)(ec / 3 % 3) - 1, ex = (int)(ec % 3) - 1;
      c.er2[q] = (int)dt2[(int64_t)idx + ez * (int64_t)sz + ey * (int64_t)sy + ex];
    }
  }
  return (NDIM == 3 ? 2 * c.R + 1 : 1) * c.nseg;
}

// Per-CTA lookup tables of the paint kernel (shared memory, built at launch):
// integer square roots of small values, and for every dominant offset code
// the canonical axis order and signs of its crescent, and the canonical
// offset of every other neighbour under that order.
constexpr int kSqrtLut = 4096;
struct PaintLut {
  uint8_t sq[kSqrtLut];  // floor(sqrt(v)), v < kSqrtLut
  uint16_t perm[27];     // world axis of canonical x, y, z (2 bits each) | their sign bits << 6
  uint8_t eo[27 * 27];   // [dominant code][neighbour code]: canonical offset, (o + 1) in 2 bits per axis
};

// Canonical x, y, z of a crescent: the nonzero axes of the dominant offset
// first (in x, y, z order), then the zero axes; signs make the offset
// (1,0,0), (1,1,0) or (1,1,1).
__device__ void init_paint_lut(PaintLut& L) {
  for (int i = threadIdx.x; i < kSqrtLut; i += blockDim.x) L.sq[i] = (uint8_t)isqrt24((uint32_t)i);
  for (int i = threadIdx.x; i < 27 * 28; i += blockDim.x) {
    const int code = i / 28, e = i % 28;  // e == 27: the permutation itself
    const int ddz = code / 9 - 1, ddy = code / 3 % 3 - 1, ddx = code % 3 - 1;
    const int cls = (ddx != 0) + (ddy != 0) + (ddz != 0);
    int a0 = 0, a1 = 1, a2 = 2;
    if (cls == 2) {
      if (ddx == 0) { a0 = 1; a1 = 2; a2 = 0; }
      else if (ddy == 0) { a0 = 0; a1 = 2; a2 = 1; }
    } else if (cls == 1) {
      if (ddy != 0) { a0 = 1; a1 = 0; a2 = 2; }
      else if (ddz != 0) { a0 = 2; a1 = 0; a2 = 1; }
    }
    auto comp = [](int a, int vx, int vy, int vz) { return a == 0 ? vx : (a == 1 ? vy : vz); };
    const int g0 = comp(a0, ddx, ddy, ddz) < 0, g1 = comp(a1, ddx, ddy, ddz) < 0, g2 = comp(a2, ddx, ddy, ddz) < 0;
    if (e == 27) {
      L.perm[code] = (uint16_t)(a0 | (a1 << 2) | (a2 << 4) | (g0 << 6) | (g1 << 7) | (g2 << 8));
    } else {
      const int ez = e / 9 - 1, ey = e / 3 % 3 - 1, ex = e % 3 - 1;
      const int q0 = g0 ? -comp(a0, ex, ey, ez) : comp(a0, ex, ey, ez);
      const int q1 = g1 ? -comp(a1, ex, ey, ez) : comp(a1, ex, ey, ez);
      const int q2 = g2 ? -comp(a2, ex, ey, ez) : comp(a2, ex, ey, ez);
      L.eo[code * 27 + e] = (uint8_t)((q0 + 1) | ((q1 + 1) << 2) | ((q2 + 1) << 4));
    }
  }
}

__device__ __forceinline__ int isqrt_lut(const PaintLut& L, int v) {
  return v < kSqrtLut ? (int)L.sq[v] : (int)isqrt24((uint32_t)v);
}

// Table mode: a 3D centre with r^2 <= kCresT and a dominant neighbour,
// decoded from its record alone. In the shared chunks of phase 2 it is kept
// as two 16-byte words (idx, vstart, start, r2ax) and (S, ex), plus the label.
struct TabCentre {
  uint32_t idx, vstart, start;
  uint32_t r2ax;  // r^2 | world axis (2 bits each) and sign bit (<< 6..8) of canonical x, y, z << 9 | inside << 18
  int S[3];       // signed linear strides of the canonical axes x, y, z
  uint32_t ex;    // extra balls: r^2 (9 bits each, 0x1FF none) | canonical offsets << 18 (6 bits each)
  uint32_t label;
};

// Returns the crescent size.
__device__ __forceinline__ int make_tab_centre(uint4 rec, size_t sy, size_t sz, bool touch,
                                               const uint32_t* __restrict__ labels, const PaintLut& L,
                                               TabCentre& c) {
  c.idx = rec.x;
  c.vstart = rec.y;
  c.start = 0;
  const uint32_t code = (rec.z >> 9) & 31u;
  const uint32_t pm = L.perm[code];
  c.r2ax = (rec.z & 0x1FFu) | (pm << 9) | (((rec.z >> 24) & 1u) << 18);
  const int sy_ = (int)sy, sz_ = (int)sz;
  auto stride = [&](uint32_t a, uint32_t g) {
    const int t = a == 0 ? 1 : (a == 1 ? sy_ : sz_);
    return g ? -t : t;
  };
  c.S[0] = stride(pm & 3u, (pm >> 6) & 1u);
  c.S[1] = stride((pm >> 2) & 3u, (pm >> 7) & 1u);
  c.S[2] = stride((pm >> 4) & 3u, (pm >> 8) & 1u);
  uint32_t ex = 0;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const uint32_t ec = (rec.z >> (14 + 5 * q)) & 31u;
    uint32_t er = (rec.w >> (9 * q)) & 0x1FFu, eo = 0;
    if (ec == kNoDominant)
      er = 0x1FFu;
    else
      eo = L.eo[code * 27 + ec];
    ex |= (er << (9 * q)) | (eo << (18 + 6 * q));
  }
  c.ex = ex;
  c.label = touch ? labels[c.idx] : 0u;
  return (int)((rec.w >> 18) & 0x7FFu);
}

// Linear index of canonical crescent voxel p of c; false when the voxel lies
// in one of c's extra higher-ranked balls (it is covered there) or outside
// the array.
__device__ __forceinline__ bool tab_voxel_index(const TabCentre& c, uint32_t p, const Dims& d, uint32_t& i) {
  const int o0 = (int)(p & 0xFFu) - 128, o1 = (int)((p >> 8) & 0xFFu) - 128,
            o2 = (int)((p >> 16) & 0xFFu) - 128;
  const uint32_t ex = c.ex;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int er = (int)((ex >> (9 * q)) & 0x1FFu);
    const uint32_t eo = (ex >> (18 + 6 * q)) & 63u;
    const int e0 = (int)(eo & 3u) - 1, e1 = (int)((eo >> 2) & 3u) - 1, e2 = (int)((eo >> 4) & 3u) - 1;
    if (er != 0x1FF && (o0 - e0) * (o0 - e0) + (o1 - e1) * (o1 - e1) + (o2 - e2) * (o2 - e2) <= er) return false;
  }
  const uint32_t axes = c.r2ax >> 9;
  if (!(axes & 512u)) {  // the ball may leave the array: check each coordinate
    const int cx = (int)(c.idx % (uint32_t)d.nx);
    const uint32_t t = c.idx / (uint32_t)d.nx;
    const int cy = (int)(t % (uint32_t)d.ny), cz = (int)(t / (uint32_t)d.ny);
    const int a0 = axes & 3, a1 = (axes >> 2) & 3, a2 = (axes >> 4) & 3;
    const int v0 = (axes >> 6) & 1 ? -o0 : o0, v1 = (axes >> 7) & 1 ? -o1 : o1, v2 = (axes >> 8) & 1 ? -o2 : o2;
    const int x = cx + (a0 == 0 ? v0 : 0) + (a1 == 0 ? v1 : 0) + (a2 == 0 ? v2 : 0);
    const int y = cy + (a0 == 1 ? v0 : 0) + (a1 == 1 ? v1 : 0) + (a2 == 1 ? v2 : 0);
    const int z = cz + (a0 == 2 ? v0 : 0) + (a1 == 2 ? v1 : 0) + (a2 == 2 ? v2 : 0);
    if (x < 0 || x >= d.nx || y < 0 || y >= d.ny || z < 0 || z >= d.nz) return false;
  }
  i = c.idx + (uint32_t)(o0 * c.S[0] + o1 * c.S[1] + o2 * c.S[2]);  // modulo 2^32: the sum is in range
  return true;
}

// Row-mode item `local` of a centre: the z offset and the group of 8 rows.
template <int NDIM>
__device__ __forceinline__ void paint_row_item(const Centre& c, int local, const Dims& d, size_t sy,
                                               size_t sz, bool touch, const uint32_t* __restrict__ dt2,
                                               const uint32_t* __restrict__ labels,
                                               uint32_t* __restrict__ lt2, uint32_t& nupd) {
  if (NDIM == 3) {
    int q = (int)((float)local * c.inv_nseg);
    if (q * c.nseg > local) --q;
    else if ((q + 1) * c.nseg <= local) ++q;
    paint_rows(c, q - c.R, local - q * c.nseg, d, sy, sz, touch, dt2, labels, lt2, nupd);
  } else {
    paint_rows(c, 0, local, d, sy, sz, touch, dt2, labels, lt2, nupd);
  }
}

// Lane-parallel exclusive prefix sum of cnt over the warp; returns the
// lane's start, the warp's total in *total.
__device__ __forceinline__ int warp_starts(int cnt, int lane, int* total) {
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += t;
  }
  *total = __shfl_sync(kFull, incl, 31);
  return incl - cnt;
}

// Owner of work item k: the last lane whose start <= k.
__device__ __forceinline__ int owner_lane(int start, int k) {
  int j = 0;
#pragma unroll
  for (int step = 16; step; step >>= 1) {
    const int s = __shfl_sync(kFull, start, j + step);
    if (s <= k) j += step;
  }
  return j;
}

// Rows of a row-mode centre that can hold crescent voxels. A voxel u (offset
// from c) inside B(c) but outside the ball of a neighbour X = c + d has
// |u|^2 <= r^2 and |u - d|^2 > rX^2, so 2 u.d < |d|^2 - (rX^2 - r^2) =: T:
// every voxel of B(c) outside that half-space lies in B(X). For the dominant
// (the neighbour whose ball comes closest to containing c's) the half-space
// leaves a small cap at the far side of B(c); the extra balls cut it
// further. Row (oy, oz) holds voxels |ox| <= w = isqrt(r^2 - oy^2 - oz^2),
// so it can meet the half-space only when 2 (ddy oy + ddz oz) - 2 |ddx| w
// <= T - 1. cap_clip narrows [lo, hi], the candidate oy at height oz (H =
// r^2 - oz^2), to the rows that can (a superset: each row's spans are still
// computed exactly).
__device__ __forceinline__ void cap_clip(int r2, int H, int ddx, int ddy, int ddz, int r2x, int oz, int& lo,
                                         int& hi) {
  const int T = ddx * ddx + ddy * ddy + ddz * ddz - (r2x - r2);
  if (ddx == 0) {
    // 2 ddy oy <= T - 1 - 2 ddz oz
    const int q = (T - 1 - 2 * ddz * oz) >> 1;  // floor
    if (ddy == 0) {
      if (q < 0) hi = lo - 1;
    } else if (ddy > 0) {
      hi = min(hi, q);
    } else {
      lo = max(lo, -q);
    }
    return;
  }
  // |ddx| = 1: w >= s - K with s = ddy oy + ddz oz, K = floor((T - 1) / 2);
  // rows with s <= K qualify, the others need oy^2 + (s - K)^2 <= H
  const int e = ddz * oz - ((T - 1) >> 1);  // s - K = ddy oy + e
  if (ddy == 0) {
    if (e <= 0) return;
    const int H2 = H - e * e;
    if (H2 < 0) {
      hi = lo - 1;
      return;
    }
    const int w2 = (int)isqrt24((uint32_t)H2);
    lo = max(lo, -w2);
    hi = min(hi, w2);
    return;
  }
  // t = ddy oy: t <= -e, or 2 t^2 + 2 e t + e^2 - H <= 0; the two sets join
  // into t <= max(-e, (-e + sqrt(2H - e^2)) / 2) within the disc (bound
  // rounded up by one)
  int tmax = -e;
  const int disc = 2 * H - e * e;
  if (disc >= 0) tmax = max(tmax, (int)floorf((sqrtf((float)disc) - (float)e) * 0.5f) + 1);
  if (ddy > 0) hi = min(hi, tmax);
  else lo = max(lo, -tmax);
}

// The candidate rows at height oz: the disc's rows within [ylo, yhi], cut by
// the half-spaces of the higher-ranked balls (hr[k] < 0: none).
__device__ __forceinline__ void cap_rows(const Centre& c, const int hr[3], const int hx[3], const int hy[3],
                                         const int hz[3], int oz, int ylo, int yhi, int& lo, int& hi) {
  const int H = (int)c.r2 - oz * oz;
  const int wy = (int)isqrt24((uint32_t)H);
  lo = max(-wy, ylo);
  hi = min(wy, yhi);
#pragma unroll
  for (int k = 0; k < 3; ++k)
    if (hr[k] >= 0) cap_clip((int)c.r2, H, hx[k], hy[k], hz[k], hr[k], oz, lo, hi);
}

// One row-mode centre, one warp. The heights oz go 32 at a time, each lane
// one height and its interval of candidate rows (cap_rows); a warp scan
// numbers the rows, which are then taken 32 at a time, lane k the k-th row,
// and each row's crescent spans are computed (the row of the ball minus the
// higher-ranked neighbours' rows, clamped to the array); then the spans'
// voxels are shared out in order, so consecutive lanes update consecutive
// x. Part p of `parts` takes the row groups q (rows 32q .. 32q + 31 in the
// numbering over all heights) with q = p mod parts.
template <int NDIM>
__device__ __forceinline__ void paint_centre_rows(const Centre& c, int part, int parts, const Dims& d, size_t sy,
                                                  size_t sz, bool touch, const uint32_t* __restrict__ dt2,
                                                  const uint32_t* __restrict__ labels,
                                                  uint32_t* __restrict__ lt2, const PaintLut& L, uint32_t& nupd) {
  const int lane = threadIdx.x & 31;
  const int xmin = -c.cx, xmax = d.nx - 1 - c.cx;
  // the higher-ranked balls: dominant first, then the two extras (r^2 -1: none)
  int hr[3], hx[3], hy[3], hz[3];
  hr[0] = c.r2d, hx[0] = c.ddx, hy[0] = c.ddy, hz[0] = c.ddz;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int ec = c.eoff[q];
    hr[q + 1] = c.er2[q], hx[q + 1] = ec % 3 - 1, hy[q + 1] = ec / 3 % 3 - 1, hz[q + 1] = ec / 9 - 1;
  }
  const int oz_lo = NDIM == 3 ? max(-c.R, -c.cz) : 0, oz_hi = NDIM == 3 ? min(c.R, d.nz - 1 - c.cz) : 0;
  int row0 = 0;  // number of the first row of this batch of heights
  for (int oz0 = oz_lo; oz0 <= oz_hi; oz0 += 32) {
    const int oz = oz0 + lane;
    int lo = 0, hi = -1;
    if (oz <= oz_hi) cap_rows(c, hr, hx, hy, hz, oz, -c.cy, d.ny - 1 - c.cy, lo, hi);
    int nrows;
    const int rstart = warp_starts(max(0, hi - lo + 1), lane, &nrows);
    // this part's row groups among rows row0 .. row0 + nrows - 1
    const int qa = row0 >> 5, qb = (row0 + nrows - 1) >> 5;
    int q = qa + ((part - qa) % parts + parts) % parts;
    for (; nrows > 0 && q <= qb; q += parts) {
      const int k = 32 * q + lane - row0;  // row of this batch taken by the lane
      int a1 = 0, n1 = 0, a2 = 0, n2 = 0, w = -1;  // spans [a1, a1 + n1), [a2, a2 + n2) of dx
      uint32_t rowbase = 0;                        // linear index of (cx, y, z)
      const int j = owner_lane(rstart, max(0, min(k, nrows - 1)));
      const int dz = __shfl_sync(kFull, oz, j);
      const int dy = __shfl_sync(kFull, lo, j) + (k - __shfl_sync(kFull, rstart, j));
      if (k >= 0 && k < nrows) {
        const int z = c.cz + dz, y = c.cy + dy;
        const int h = (int)c.r2 - dz * dz - dy * dy;
        w = isqrt_lut(L, h);
        // this row of the higher-ranked balls as one interval [elo, ehi] of
        // dx: an extra's row joins only when it touches the interval so far
        // (skipping one excludes less, which only paints more true-ball
        // voxels)
        int elo = 1, ehi = 0;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          if (hr[e] < 0) continue;
          const int hd = hr[e] - (dz - hz[e]) * (dz - hz[e]) - (dy - hy[e]) * (dy - hy[e]);
          if (hd < 0) continue;
          const int wd = isqrt_lut(L, hd);
          const int elo2 = hx[e] - wd, ehi2 = hx[e] + wd;
          if (elo > ehi) {
            elo = elo2;
            ehi = ehi2;
          } else if (elo2 <= ehi + 1 && ehi2 >= elo - 1) {
            elo = min(elo, elo2);
            ehi = max(ehi, ehi2);
          }
        }
        int hi1 = w, lo2 = 1, hi2 = 0;
        if (elo <= ehi) {
          hi1 = min(w, elo - 1);
          lo2 = max(-w, ehi + 1);
          hi2 = w;
        }
        a1 = max(-w, xmin);
        n1 = max(0, min(hi1, xmax) - a1 + 1);
        a2 = max(lo2, xmin);
        n2 = max(0, min(hi2, xmax) - a2 + 1);
        if (w * w != h) w = -1;  // only the ends of an exact row can be background
        rowbase = (uint32_t)((size_t)z * sz + (size_t)y * sy + (size_t)c.cx);
      }
      int total;
      const int start = warp_starts(n1 + n2, lane, &total);
      for (int kb = 0; kb < total; kb += 32) {
        const int kk = kb + lane;
        const int jj = owner_lane(start, kk);
        const int o = kk - __shfl_sync(kFull, start, jj);
        const int a1j = __shfl_sync(kFull, a1, jj), n1j = __shfl_sync(kFull, n1, jj);
        const int a2j = __shfl_sync(kFull, a2, jj), wj = __shfl_sync(kFull, w, jj);
        const uint32_t rb = __shfl_sync(kFull, rowbase, jj);
        if (kk >= total) continue;
        const int dx = o < n1j ? a1j + o : a2j + (o - n1j);
        const uint32_t i = rb + (uint32_t)dx;  // modulo 2^32: the sum is in range
        if (wj >= 0 && (dx == wj || dx == -wj) && dt2[i] == 0) continue;
        if (touch && labels[i] != c.label) continue;
        atomicMax(lt2 + i, c.r2);
        ++nupd;
      }
    }
    row0 += nrows;
  }
}

// Up to two crescent voxels k0, k1 of table centres c0, c1: each is painted
// unless it lies outside the array or in an extra ball, or on the sphere
// and in the background, or (touch) carries another label.
__device__ __forceinline__ void paint_tab_pair(const TabCentre& c0, int k0, bool v0, const TabCentre& c1, int k1,
                                               bool v1, const Dims& d, bool touch,
                                               const uint32_t* __restrict__ dt2,
                                               const uint32_t* __restrict__ labels,
                                               uint32_t* __restrict__ lt2, uint32_t& ntab) {
  const uint32_t p0 = v0 ? g_cres_vox[c0.vstart + (uint32_t)k0] : 0u;
  const uint32_t p1 = v1 ? g_cres_vox[c1.vstart + (uint32_t)k1] : 0u;
  uint32_t i0 = 0, i1 = 0;
  bool w0 = v0 && tab_voxel_index(c0, p0, d, i0);
  bool w1 = v1 && tab_voxel_index(c1, p1, d, i1);
  // inside the ball only the sphere |y|^2 == r^2 can be background
  const uint32_t b0 = w0 && (p0 >> 24) ? dt2[i0] : 1u;
  const uint32_t b1 = w1 && (p1 >> 24) ? dt2[i1] : 1u;
  if (touch) {
    w0 = w0 && labels[i0] == c0.label;
    w1 = w1 && labels[i1] == c1.label;
  }
  if (w0 && b0) {
    atomicMax(lt2 + i0, c0.r2ax & 0x1FFu);
    ++ntab;
  }
  if (w1 && b1) {
    atomicMax(lt2 + i1, c1.r2ax & 0x1FFu);
    ++ntab;
  }
}

// Work items from one device counter by guided self-scheduling: a warp takes
// about 1/(2 * warps) of the items not yet taken (at most `cap`), so the hot
// counter sees few atomics while much work is left, and the last items still
// spread over all warps one at a time.
struct WorkGrab {
  uint32_t next = 0, end = 0, first = 0;  // [first, end): the warp's current range
  __device__ __forceinline__ bool take(unsigned int* ctr, uint32_t items, uint32_t cap, uint32_t& item) {
    if (next == end) {
      const uint32_t warps = gridDim.x * (blockDim.x / 32);
      const uint32_t left = items > end ? items - end : 0u;  // end: the counter after this warp's last take
      const uint32_t g = max(1u, min(cap, left / (2u * warps)));
      uint32_t b = 0;
      if ((threadIdx.x & 31) == 0) b = atomicAdd(ctr, g);
      next = __shfl_sync(kFull, b, 0);
      first = next;
      end = next + g;
    }
    if (next >= items) return false;
    item = next++;
    return true;
  }
};
constexpr uint32_t kChunkGrab = 8;  // phase 2 chunks per counter update, at most
constexpr uint32_t kBigGrab = 8;    // phase 1 centres per counter update, at most (<= 32)

// The record of phase-1 item b, from `held` (lane j holds the record of
// item first + j of the warp's range, loaded when the range was taken: one
// load for all instead of one dependent load per item).
__device__ __forceinline__ uint4 held_record(const uint4& held, uint32_t b, uint32_t first) {
  const int j = (int)(b - first);
  return make_uint4(__shfl_sync(kFull, held.x, j), __shfl_sync(kFull, held.y, j), __shfl_sync(kFull, held.z, j),
                    __shfl_sync(kFull, held.w, j));
}

// Phase 2 in 3D: chunk ch of 32 table centres (of n in the front list),
// lane j holding the record of centre 32 ch + j in `rec`; the lanes share
// the chunk's crescent voxels, two per lane in flight.
__device__ __forceinline__ void paint_table_chunk(const uint4& rec, uint32_t n, uint32_t ch, const Dims& d,
                                                  size_t sy, size_t sz, bool touch,
                                                  const uint32_t* __restrict__ dt2,
                                                  const uint32_t* __restrict__ labels, uint32_t* __restrict__ lt2,
                                                  const PaintLut& L, uint32_t& ntab) {
  __shared__ uint4 csA[8][32], csB[8][32];  // (idx, vstart, start, r2ax), (S, ex) of the chunk's centres
  __shared__ uint32_t csL[8][32];            // their labels (touch only)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t i = ch * 32 + lane;
  int cnt = 0;
  TabCentre mine;
  if (i < n) cnt = make_tab_centre(rec, sy, sz, touch, labels, L, mine);
  int total;
  const int start = warp_starts(cnt, lane, &total);
  if (i < n) {
    csA[w][lane] = make_uint4(mine.idx, mine.vstart, (uint32_t)start, mine.r2ax);
    csB[w][lane] = make_uint4((uint32_t)mine.S[0], (uint32_t)mine.S[1], (uint32_t)mine.S[2], mine.ex);
    csL[w][lane] = mine.label;
  }
  __syncwarp();
  auto load = [&](int j) {
    TabCentre c;
    const uint4 A = csA[w][j], B = csB[w][j];
    c.idx = A.x, c.vstart = A.y, c.start = A.z, c.r2ax = A.w;
    c.S[0] = (int)B.x, c.S[1] = (int)B.y, c.S[2] = (int)B.z, c.ex = B.w;
    c.label = touch ? csL[w][j] : 0u;
    return c;
  };
  for (int kb = 0; kb < total; kb += 64) {
    const int k0 = kb + lane, k1 = k0 + 32;
    const TabCentre c0 = load(owner_lane(start, k0)), c1 = load(owner_lane(start, k1));
    paint_tab_pair(c0, k0 - (int)c0.start, k0 < total, c1, k1 - (int)c1.start, k1 < total, d, touch, dt2, labels,
                   lt2, ntab);
  }
  __syncwarp();
}

// Phase 2 in 2D: chunk ch of 32 centres; the lanes share the chunk's row
// segments.
__device__ __forceinline__ void paint_row_chunk(const uint4* __restrict__ surv, uint32_t n, uint32_t ch,
                                                const Dims& d, size_t sy, size_t sz, bool touch,
                                                const uint32_t* __restrict__ dt2, const uint32_t* __restrict__ labels,
                                                uint32_t* __restrict__ lt2, uint32_t& nupd) {
  __shared__ Centre cs[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t i = ch * 32 + lane;
  int cnt = 0;
  if (i < n) cnt = make_centre<2>(surv[i], d, sy, sz, touch, dt2, labels, cs[w][lane]);
  int total;
  const int start = warp_starts(cnt, lane, &total);
  if (i < n) cs[w][lane].start = start;
  __syncwarp();
  for (int kb = 0; kb < total; kb += 32) {
    const int k = kb + lane;
    const int j = owner_lane(start, k);
    if (k < total) {
      const Centre& c = cs[w][j];
      paint_row_item<2>(c, k - c.start, d, sy, sz, touch, dt2, labels, lt2, nupd);
    }
  }
  __syncwarp();
}

// Phase 1: one back-list record, one warp (big table crescent, or a part of
// a centre painted row by row).
template <int NDIM>
__device__ __forceinline__ void paint_big(const uint4& rec, const Dims& d, size_t sy, size_t sz, bool touch,
                                          const uint32_t* __restrict__ dt2, const uint32_t* __restrict__ labels,
                                          uint32_t* __restrict__ lt2, const PaintLut& lut, uint32_t& nupd,
                                          uint32_t& ntab) {
  const int lane = threadIdx.x & 31;
  if (NDIM == 3 && (rec.z & kTableRecord)) {
    TabCentre c;
    const int items = make_tab_centre(rec, sy, sz, touch, labels, lut, c);
    for (int k = lane; k < items; k += 64)
      paint_tab_pair(c, k, true, c, k + 32, k + 32 < items, d, touch, dt2, labels, lt2, ntab);
  } else {
    Centre c;
    make_centre<NDIM>(rec, d, sy, sz, touch, dt2, labels, c);
    paint_centre_rows<NDIM>(c, (int)(rec.w & 0xFFFFu), max(1, (int)(rec.w >> 16)), d, sy, sz, touch, dt2, labels, lt2,
                            lut, nupd);
  }
}

// Two phases, each fed by a global work counter.
// 1. Centres from the back of the list, one per warp: the lanes share its
//    crescent voxels (big 3D table crescents) or take its rows 32 at a time
//    (row mode: 3D centres without a table, 2D discs with r^2 > 64). These
//    are the biggest pieces of work, so they go first.
// 2. Chunks of 32 centres from the front of the list: the 32 lanes share the
//    chunk's work items (crescent voxels in 3D, row segments in 2D), so big
//    and small crescents balance.
template <int NDIM>
__global__ void __launch_bounds__(256) lt_paint_kernel(const uint4* __restrict__ surv,
                                                       const uint32_t* __restrict__ dt2,
                                                       const uint32_t* __restrict__ labels,
                                                       uint32_t* __restrict__ lt2, Dims d,
                                                       WsHeader* __restrict__ hdr) {
  const int lane = threadIdx.x & 31;
  const uint32_t n = *(volatile uint32_t*)&hdr->n_surv;
  const uint32_t nbig = *(volatile uint32_t*)&hdr->n_big;
  const bool touch = *(volatile uint32_t*)&hdr->touch != 0;
  const size_t sy = (size_t)d.nx, sz = (size_t)d.nx * d.ny;
  uint32_t nupd = 0, ntab = 0;  // updates this thread issued: row by row, from tables
  __shared__ PaintLut lut;
  init_paint_lut(lut);
  __syncthreads();
  {
    WorkGrab grab;
    uint32_t b = 0;
    uint4 held = make_uint4(0u, 0u, 0u, 0u);
    while (grab.take(&hdr->ctr_big, nbig, kBigGrab, b)) {
      if (b == grab.first) {  // a new range (uniform in the warp): its records in one go
        const uint32_t k = b + (uint32_t)lane;
        if (k < grab.end && k < nbig) held = surv[record_capacity(d.n) - 1 - k];
      }
      paint_big<NDIM>(held_record(held, b, grab.first), d, sy, sz, touch, dt2, labels, lt2, lut, nupd, ntab);
    }
  }
  {
    const uint32_t nchunks = (n + 31) / 32;
    WorkGrab grab;
    uint32_t ch = 0;
    uint4 next = make_uint4(0u, 0u, 0u, 0u);  // lane j: record j of chunk ch + 1 (3D), loaded ahead
    // 2D chunks vary most in cost: one at a time
    while (grab.take(&hdr->ctr_small, nchunks, NDIM == 3 ? kChunkGrab : 1u, ch)) {
      if (NDIM == 3) {
        uint4 rec = next;
        if (ch == grab.first) {  // a new range (uniform in the warp)
          const uint32_t i = ch * 32 + (uint32_t)lane;
          rec = i < n ? surv[i] : make_uint4(0u, 0u, 0u, 0u);
        }
        if (ch + 1 < grab.end) {  // the next chunk's records fly while this one is painted
          const uint32_t i = (ch + 1) * 32 + (uint32_t)lane;
          next = i < n ? surv[i] : make_uint4(0u, 0u, 0u, 0u);
        }
        paint_table_chunk(rec, n, ch, d, sy, sz, touch, dt2, labels, lt2, lut, ntab);
      } else {
        paint_row_chunk(surv, n, ch, d, sy, sz, touch, dt2, labels, lt2, nupd);
      }
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    nupd += __shfl_xor_sync(kFull, nupd, o);
    ntab += __shfl_xor_sync(kFull, ntab, o);
  }
  if (lane == 0 && nupd + ntab) {
    atomicAdd(&hdr->n_updates, (unsigned long long)(nupd + ntab));
    atomicAdd(&hdr->n_table_updates, (unsigned long long)ntab);
  }
}

// Painting of many volumes in one persistent grid: the back lists of all
// volumes, then the front lists' chunks, each from one counter of `ctr`
// (ctr[0] back items, ctr[1] chunks; zero before the launch). Every CTA
// first takes the volumes' list lengths (from their headers, after the
// ridge pass) and their prefix sums, so that an item maps to its volume.
template <int NDIM>
__global__ void __launch_bounds__(256) lt_paint_multi_kernel(MultiArgs m, uint32_t* __restrict__ ctr) {
  __shared__ uint32_t big0[kMaxBatchVols + 1], chunk0[kMaxBatchVols + 1];
  __shared__ uint32_t wsum[2][8];
  __shared__ PaintLut lut;
  init_paint_lut(lut);
  // block-wide exclusive scans of the per-volume item counts (nvol <= 256)
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  uint32_t nb = 0, nc = 0;
  if (tid < m.nvol) {
    const WsHeader* h = m.vols[tid].hdr;
    nb = *(volatile const uint32_t*)&h->n_big;
    nc = (*(volatile const uint32_t*)&h->n_surv + 31u) / 32u;
  }
  uint32_t ib = nb, ic = nc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t tb = __shfl_up_sync(kFull, ib, o), tc = __shfl_up_sync(kFull, ic, o);
    if (lane >= o) {
      ib += tb;
      ic += tc;
    }
  }
  if (lane == 31) {
    wsum[0][w] = ib;
    wsum[1][w] = ic;
  }
  __syncthreads();
  uint32_t ob = 0, oc = 0;
  for (int k = 0; k < w; ++k) {
    ob += wsum[0][k];
    oc += wsum[1][k];
  }
  if (tid < m.nvol) {
    big0[tid] = ob + ib - nb;
    chunk0[tid] = oc + ic - nc;
  }
  if (tid == 0) {
    uint32_t tb = 0, tc = 0;
    for (int k = 0; k < 8; ++k) {
      tb += wsum[0][k];
      tc += wsum[1][k];
    }
    big0[m.nvol] = tb;
    chunk0[m.nvol] = tc;
  }
  __syncthreads();
  auto vol_of = [&](const uint32_t* start, uint32_t item) {
    int lo = 0, hi = m.nvol;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (start[mid] <= item) lo = mid;
      else hi = mid;
    }
    return lo;
  };
  uint32_t nupd = 0, ntab = 0;
  {
    WorkGrab grab;
    uint32_t b = 0;
    uint4 held = make_uint4(0u, 0u, 0u, 0u);
    while (grab.take(&ctr[0], big0[m.nvol], kBigGrab, b)) {
      if (b == grab.first) {  // a new range (uniform in the warp): its records in one go
        const uint32_t k = b + (uint32_t)lane;
        if (k < grab.end && k < big0[m.nvol]) {
          const int vk = vol_of(big0, k);
          const VolParams& pk = m.vols[vk];
          held = reinterpret_cast<const uint4*>(pk.body)[record_capacity(pk.d.n) - 1 - (k - big0[vk])];
        }
      }
      const uint4 rec = held_record(held, b, grab.first);
      const int v = vol_of(big0, b);
      const VolParams& p = m.vols[v];
      const bool touch = *(volatile const uint32_t*)&p.hdr->touch != 0;
      paint_big<NDIM>(rec, p.d, (size_t)p.d.nx, (size_t)p.d.nx * p.d.ny, touch, p.dt2, p.labels, p.lt2, lut, nupd,
                      ntab);
    }
  }
  {
    WorkGrab grab;
    uint32_t ch = 0;
    while (grab.take(&ctr[1], chunk0[m.nvol], NDIM == 3 ? kChunkGrab : 1u, ch)) {
      const int v = vol_of(chunk0, ch);
      const VolParams& p = m.vols[v];
      const bool touch = *(volatile const uint32_t*)&p.hdr->touch != 0;
      const uint4* surv = reinterpret_cast<const uint4*>(p.body);
      const uint32_t n = *(volatile const uint32_t*)&p.hdr->n_surv;
      const size_t sy = (size_t)p.d.nx, sz = (size_t)p.d.nx * p.d.ny;
      if (NDIM == 3) {
        const uint32_t i = (ch - chunk0[v]) * 32 + (uint32_t)lane;
        const uint4 rec = i < n ? surv[i] : make_uint4(0u, 0u, 0u, 0u);
        paint_table_chunk(rec, n, ch - chunk0[v], p.d, sy, sz, touch, p.dt2, p.labels, p.lt2, lut, ntab);
      }
      else
        paint_row_chunk(surv, n, ch - chunk0[v], p.d, sy, sz, touch, p.dt2, p.labels, p.lt2, nupd);
    }
  }
}

template <int NDIM, int RZ>
void launch_ridge(bool tma, dim3 grid, cudaStream_t s, const CUtensorMap& md, const CUtensorMap& ml,
                  const uint32_t* dt2, const uint32_t* labels, uint32_t* lt2, const Dims& d, uint4* surv,
                  WsHeader* hdr, RidgeWait wt = RidgeWait(), int z_base = 0, uint32_t* max_dt2 = nullptr,
                  uint32_t n_labels = 0) {
  if (tma)
    lt_ridge_kernel<NDIM, RZ, true><<<grid, 256, 0, s>>>(md, ml, dt2, labels, lt2, d, surv, hdr, wt, z_base,
                                                          max_dt2, n_labels);
  else
    lt_ridge_kernel<NDIM, RZ, false><<<grid, 256, 0, s>>>(md, ml, dt2, labels, lt2, d, surv, hdr, wt, z_base,
                                                           max_dt2, n_labels);
}

}  // namespace

bool make_tensor_map_u32_3d(CUtensorMap* map, const void* base, int nx, int ny, int nz, int bx, int by) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  if (!encode || (reinterpret_cast<uintptr_t>(base) & 15u) || (nx * 4) % 16) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, const_cast<void*>(base), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t lt_workspace_bytes(const Dims& d) { return align_up(record_capacity(d.n) * sizeof(uint4)); }

int paint_fit(int ndim);

cudaError_t lt_prepare_device() {
  paint_fit(3);
  return ensure_tables();
}

// Timeout self-test: the TMA ridge kernel on a 32 x 8 x 8 all-background
// volume carved from `ws`, with every plane barrier expecting 16 bytes more
// than its copies deliver, so each wait gives up after 1 ms; the kernel must
// record ERR_TIMEOUT in the header and return.
size_t ridge_selftest_bytes() { return sizeof(WsHeader) + 2048 * (3 * 4 + 16); }

cudaError_t ridge_selftest_launch(void* ws, cudaStream_t s) {
  cudaError_t e = ensure_tables();
  if (e != cudaSuccess) return e;
  Dims d;
  d.ndim = 3;
  d.nx = 32;
  d.ny = 8;
  d.nz = 8;
  d.n = 2048;
  char* p = reinterpret_cast<char*>(ws);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(p);
  uint32_t* dt2 = reinterpret_cast<uint32_t*>(p + sizeof(WsHeader));
  uint32_t* labels = dt2 + d.n;
  uint32_t* lt2 = labels + d.n;
  uint4* surv = reinterpret_cast<uint4*>(lt2 + d.n);
  e = cudaMemsetAsync(ws, 0, sizeof(WsHeader) + 3 * 4 * (size_t)d.n, s);
  if (e != cudaSuccess) return e;
  CUtensorMap md, ml;
  if (!make_tensor_map_u32_3d(&md, dt2, d.nx, d.ny, d.nz, kBX, kBY) ||
      !make_tensor_map_u32_3d(&ml, labels, d.nx, d.ny, d.nz, kBX, kBY))
    return cudaErrorInvalidValue;
  RidgeWait wt;
  wt.limit_ns = 1000000ull;
  wt.extra_tx = 16;
  launch_ridge<3, 32>(true, dim3(1, 1, 1), s, md, ml, dt2, labels, lt2, d, surv, hdr, wt);
  return cudaGetLastError();
}

int ridge_chunk(const Tuning& tu) { return tu.ridge_z == 8 || tu.ridge_z == 32 ? tu.ridge_z : 16; }

cudaError_t lt_ridge_launch(const uint32_t* dt2, const uint32_t* labels, uint32_t* lt2, const Dims& d,
                            WsHeader* hdr, void* body, cudaStream_t s, const Tuning& tu, int z_lo, int z_hi,
                            uint32_t* max_dt2, uint32_t n_labels) {
  cudaError_t e = ensure_tables();
  if (e != cudaSuccess) return e;
  uint4* surv = reinterpret_cast<uint4*>(body);
  const int rz = ridge_chunk(tu);
  if (d.ndim == 2) {
    z_lo = 0;
    z_hi = 1;
  } else if (z_hi < 0 || z_hi > d.nz) {
    z_hi = d.nz;
  }
  const int c_lo = z_lo / rz, c_hi = (z_hi + rz - 1) / rz;  // z_lo is a multiple of rz
  if (c_hi <= c_lo) return cudaSuccess;
  dim3 grid((d.nx + kTX - 1) / kTX, (d.ny + kTY - 1) / kTY, d.ndim == 3 ? c_hi - c_lo : 1);
  // TMA needs a row pitch that is a multiple of 16 bytes
  CUtensorMap md, ml;
  std::memset(&md, 0, sizeof(md));
  std::memset(&ml, 0, sizeof(ml));
  const bool tma = d.nx % 4 == 0 && make_tensor_map_u32_3d(&md, dt2, d.nx, d.ny, d.nz, kBX, kBY) &&
                   make_tensor_map_u32_3d(&ml, labels, d.nx, d.ny, d.nz, kBX, kBY);
  const int zb = c_lo * rz;
  {
    TraceScope t("lt_ridge", s);
    RidgeWait wt;
    wt.chunk_cres = (uint32_t)std::max(1, std::min(1024, tu.chunk_cres));
    if (d.ndim == 2)
      launch_ridge<2, 16>(tma, grid, s, md, ml, dt2, labels, lt2, d, surv, hdr, wt, 0, max_dt2, n_labels);
    else if (rz == 8)
      launch_ridge<3, 8>(tma, grid, s, md, ml, dt2, labels, lt2, d, surv, hdr, wt, zb, max_dt2, n_labels);
    else if (rz == 32)
      launch_ridge<3, 32>(tma, grid, s, md, ml, dt2, labels, lt2, d, surv, hdr, wt, zb, max_dt2, n_labels);
    else
      launch_ridge<3, 16>(tma, grid, s, md, ml, dt2, labels, lt2, d, surv, hdr, wt, zb, max_dt2, n_labels);
  }
  return cudaGetLastError();
}

// CTAs of the paint kernel that fit on one SM (queried once; callers that
// capture graphs query it first through lt_prepare_device)
int paint_fit(int ndim) {
  static const int fit[2] = {[] {
                               int v = 0;
                               if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, lt_paint_kernel<2>, 256, 0) !=
                                       cudaSuccess || v < 1)
                                 v = 1;
                               return v;
                             }(),
                             [] {
                               int v = 0;
                               if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, lt_paint_kernel<3>, 256, 0) !=
                                       cudaSuccess || v < 1)
                                 v = 1;
                               return v;
                             }()};
  return fit[ndim == 3];
}

cudaError_t lt_paint_launch(const uint32_t* dt2, const uint32_t* labels, uint32_t* lt2, const Dims& d,
                            WsHeader* hdr, void* body, cudaStream_t s, const Tuning& tu) {
  const uint4* surv = reinterpret_cast<const uint4*>(body);
  // the persistent grid: the tuned CTAs per SM, at most as many as fit
  const int bps = std::min(tu.paint_blocks_per_sm > 0 ? tu.paint_blocks_per_sm : 8, paint_fit(d.ndim));
  const unsigned pblocks = (unsigned)(sm_count() * bps);
  {
    TraceScope t("lt_paint", s);
    if (d.ndim == 3)
      lt_paint_kernel<3><<<pblocks, 256, 0, s>>>(surv, dt2, labels, lt2, d, hdr);
    else
      lt_paint_kernel<2><<<pblocks, 256, 0, s>>>(surv, dt2, labels, lt2, d, hdr);
  }
  return cudaGetLastError();
}

// ---- batched ridge and paint (see StagePlan)
dim3 lt_ridge_grid(const Dims& d, const Tuning& tu) {
  const int rz = ridge_chunk(tu);
  return dim3((d.nx + kTX - 1) / kTX, (d.ny + kTY - 1) / kTY, d.ndim == 3 ? (d.nz + rz - 1) / rz : 1);
}

bool lt_ridge_tensor_maps(void* map_dt2, void* map_lab, const uint32_t* dt2, const uint32_t* labels, const Dims& d) {
  return d.nx % 4 == 0 &&
         make_tensor_map_u32_3d(reinterpret_cast<CUtensorMap*>(map_dt2), dt2, d.nx, d.ny, d.nz, kBX, kBY) &&
         make_tensor_map_u32_3d(reinterpret_cast<CUtensorMap*>(map_lab), labels, d.nx, d.ny, d.nz, kBX, kBY);
}

template <bool TMA>
static void ridge_multi(const MultiArgs& m, uint32_t blocks, int ndim, int rz, const RidgeWait& wt, cudaStream_t s) {
  if (ndim == 2)
    lt_ridge_multi_kernel<2, 16, TMA><<<blocks, 256, 0, s>>>(m, wt);
  else if (rz == 8)
    lt_ridge_multi_kernel<3, 8, TMA><<<blocks, 256, 0, s>>>(m, wt);
  else if (rz == 32)
    lt_ridge_multi_kernel<3, 32, TMA><<<blocks, 256, 0, s>>>(m, wt);
  else
    lt_ridge_multi_kernel<3, 16, TMA><<<blocks, 256, 0, s>>>(m, wt);
}

cudaError_t lt_ridge_multi_launch(const MultiArgs& m, uint32_t blocks, int ndim, bool tma, const Tuning& tu,
                                  cudaStream_t s) {
  cudaError_t e = ensure_tables();
  if (e != cudaSuccess || blocks == 0) return e;
  RidgeWait wt;
  wt.chunk_cres = (uint32_t)std::max(1, std::min(1024, tu.chunk_cres));
  {
    TraceScope t("lt_ridge", s);
    if (tma)
      ridge_multi<true>(m, blocks, ndim, ridge_chunk(tu), wt, s);
    else
      ridge_multi<false>(m, blocks, ndim, ridge_chunk(tu), wt, s);
  }
  return cudaGetLastError();
}

cudaError_t lt_paint_multi_launch(const MultiArgs& m, int ndim, uint32_t* ctr, const Tuning& tu, cudaStream_t s) {
  static const int fit[2] = {[] {
                               int v = 0;
                               if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, lt_paint_multi_kernel<2>, 256,
                                                                                 0) != cudaSuccess || v < 1)
                                 v = 1;
                               return v;
                             }(),
                             [] {
                               int v = 0;
                               if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, lt_paint_multi_kernel<3>, 256,
                                                                                 0) != cudaSuccess || v < 1)
                                 v = 1;
                               return v;
                             }()};
  const int bps = std::min(tu.paint_blocks_per_sm > 0 ? tu.paint_blocks_per_sm : 8, fit[ndim == 3]);
  const unsigned blocks = (unsigned)(sm_count() * bps);
  {
    TraceScope t("lt_paint", s);
    if (ndim == 3)
      lt_paint_multi_kernel<3><<<blocks, 256, 0, s>>>(m, ctr);
    else
      lt_paint_multi_kernel<2><<<blocks, 256, 0, s>>>(m, ctr);
  }
  return cudaGetLastError();
}

cudaError_t lt_launch(const uint32_t* dt2, const uint32_t* labels, uint32_t* lt2, const Dims& d,
                      WsHeader* hdr, void* body, cudaStream_t s, const Tuning& tu) {
  cudaError_t e = lt_ridge_launch(dt2, labels, lt2, d, hdr, body, s, tu, 0, d.nz);
  if (e == cudaSuccess) e = lt_paint_launch(dt2, labels, lt2, d, hdr, body, s, tu);
  return e;
}

}  // namespace ltk
