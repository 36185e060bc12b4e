// Per-object sphericity and roundness on sm_103a (Sec. 4.1 and 4.2 of the
// paper).
//
// shape_reduce: one thread per voxel. An object voxel contributes 1 to its
// volume, round(sqrt(LT2) * 2^20) to the fixed-point LT sum, LT2 to the
// maximum, and, when one of its face neighbours (4 in 2D, 6 in 3D) is outside
// its object (other label, background or outside the array), the same to the
// shell count and shell sum. Lanes of a warp cover 32 consecutive voxels of a
// row; equal labels form runs, which are combined by a segmented warp scan so
// that one lane per run issues the atomics. Integer sums make the result
// independent of the order of the atomics.
//
// shape_finalize: one thread per label, FP64:
//   3D  a = mean LT, c = 3V / (4 pi a^2)                          (Eq. 8)
//       area = 2 pi a^2 (1 + (1 - e^2)/e artanh e), e = sqrt(1 - c^2/a^2)  c < a
//       area = 2 pi a^2 (1 + c/(a e) arcsin e),     e = sqrt(1 - a^2/c^2)  c > a
//       area = 4 pi a^2                                            c = a
//       (Eqs. 6-7; the printed eccentricity lacks its square root)
//       S = pi^(1/3) (6V)^(2/3) / area                             (Eq. 1)
//   2D  b = A / (pi a); P_o = pi (3(a+b) - sqrt((3a+b)(a+3b)));  (Eqs. 9-10)
//       P_c = 2 sqrt(pi A); S = P_c / P_o                          (Eqs. 2, 11)
//   R = (shell LT sum / shell count) / sqrt(max LT2)               (Sec. 4.2)
#include "lt_internal.cuh"

namespace ltk {

// Accumulator bytes for n labels: three uint32 and two uint64 arrays, each
// starting on a kAlign boundary (the layout of acc_layout below).
__host__ __device__ constexpr size_t acc_bytes(uint32_t n) {
  return 3 * align_up((size_t)n * 4) + 2 * align_up((size_t)n * 8);
}

// Per-object accumulators at the start of a shape workspace body: volume,
// n_shell, max LT2 (uint32), sum LT, sum shell LT (uint64), each array
// starting on a kAlign boundary.
__host__ __device__ inline ShapeAcc acc_layout(void* body, uint32_t n_labels) {
  char* p = reinterpret_cast<char*>(body);
  ShapeAcc acc;
  acc.volume = reinterpret_cast<uint32_t*>(p);
  p += align_up((size_t)n_labels * 4);
  acc.n_shell = reinterpret_cast<uint32_t*>(p);
  p += align_up((size_t)n_labels * 4);
  acc.max_lt2 = reinterpret_cast<uint32_t*>(p);
  p += align_up((size_t)n_labels * 4);
  acc.sum_lt = reinterpret_cast<unsigned long long*>(p);
  p += align_up((size_t)n_labels * 8);
  acc.sum_shell_lt = reinterpret_cast<unsigned long long*>(p);
  return acc;
}

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kFixScale = 1048576.0f;  // 2^LT_FIXED_POINT_SHIFT

// Object label of voxel v as the reduction sees it: with FILTER, voxels
// whose LT2 is below min_lt2 are outside every object (the object is the
// union of its inscribed balls with r^2 >= min_lt2).
template <bool FILTER>
__device__ __forceinline__ uint32_t obj_label(const uint32_t* __restrict__ labels,
                                              const uint32_t* __restrict__ lt2, size_t v, uint32_t min_lt2) {
  const uint32_t l = labels[v];
  return FILTER && l && lt2[v] < min_lt2 ? 0u : l;
}

template <int NDIM, bool FILTER>
__device__ __forceinline__ void shape_reduce_body(const uint32_t* __restrict__ labels,
                                                  const uint32_t* __restrict__ lt2, const Dims& d, uint32_t n_labels,
                                                  const ShapeAcc& acc, WsHeader* __restrict__ hdr, uint32_t min_lt2,
                                                  int z_lo, uint3 blk) {
  const int lane = threadIdx.x & 31;
  const int x = (int)blk.x * blockDim.x + threadIdx.x;
  const int y = (int)blk.y, z = (int)blk.z + z_lo;
  const bool in = x < d.nx;
  const size_t sy = (size_t)d.nx, sz = (size_t)d.nx * d.ny;
  const size_t v = in ? (size_t)z * sz + (size_t)y * sy + x : 0;
  uint32_t l = in ? labels[v] : 0u;
  if (__ballot_sync(kFull, l != 0) == 0) return;  // uniform per warp
  const bool bad = l >= n_labels;
  if (__any_sync(kFull, bad) && lane == 0) atomicOr(&hdr->error, ERR_LABEL_RANGE);
  if (bad) l = 0;
  if (FILTER && l && lt2[v] < min_lt2) l = 0;

  uint32_t pk = 0, mx = 0;  // pk = count | shell count << 16
  unsigned long long q = 0, qs = 0;
  if (l) {
    const uint32_t t = lt2[v];
    const uint32_t qq = __float2uint_rn(sqrtf((float)t) * kFixScale);
    auto nb = [&](size_t u) { return obj_label<FILTER>(labels, lt2, u, min_lt2); };
    bool s = x == 0 || nb(v - 1) != l || x == d.nx - 1 || nb(v + 1) != l || y == 0 || nb(v - sy) != l ||
             y == d.ny - 1 || nb(v + sy) != l;
    if (NDIM == 3) s = s || z == 0 || nb(v - sz) != l || z == d.nz - 1 || nb(v + sz) != l;
    pk = 1u | (s ? 1u << 16 : 0u);
    mx = t;
    q = qq;
    qs = s ? qq : 0ull;
  }
  // segmented inclusive scan over runs of equal labels
  const uint32_t lprev = __shfl_up_sync(kFull, l, 1);
  int seg = (lane == 0 || lprev != l) ? lane : 0;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(kFull, seg, o);
    if (lane >= o) seg = max(seg, t);
  }
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t a = __shfl_up_sync(kFull, pk, o);
    const unsigned long long b = __shfl_up_sync(kFull, q, o);
    const unsigned long long c = __shfl_up_sync(kFull, qs, o);
    const uint32_t m = __shfl_up_sync(kFull, mx, o);
    if (lane - o >= seg) {
      pk += a;
      q += b;
      qs += c;
      mx = max(mx, m);
    }
  }
  const uint32_t lnext = __shfl_down_sync(kFull, l, 1);
  if (l && (lane == 31 || lnext != l)) {
    atomicAdd(acc.volume + l, pk & 0xFFFFu);
    atomicAdd(acc.n_shell + l, pk >> 16);
    atomicAdd(acc.sum_lt + l, q);
    atomicAdd(acc.sum_shell_lt + l, qs);
    atomicMax(acc.max_lt2 + l, mx);
  }
}

// Vector form for nx % 4 == 0: a thread covers 4 consecutive voxels of a
// row (16-byte loads of labels, LT2 and the neighbouring rows), adds the
// voxels of its first nonzero label locally (voxels of another nonzero label
// in the same 4, which needs touching objects, go straight to the atomics),
// then runs of equal labels across the warp are combined as above.
__device__ __forceinline__ uint32_t comp(const uint4& v, int k) {
  return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

// Four labels of a row with those whose LT2 is below min_lt2 set to 0.
__device__ __forceinline__ uint4 filter4(uint4 L, const uint32_t* __restrict__ lt2, size_t v, uint32_t min_lt2) {
  if ((L.x | L.y | L.z | L.w) == 0u) return L;
  const uint4 T = *reinterpret_cast<const uint4*>(lt2 + v);
  return make_uint4(T.x < min_lt2 ? 0u : L.x, T.y < min_lt2 ? 0u : L.y, T.z < min_lt2 ? 0u : L.z,
                    T.w < min_lt2 ? 0u : L.w);
}

// Bin of LT2 t in an object whose largest LT2 is mx (t <= mx): the largest
// b in 0..15 with b^2 mx <= 256 t, from a float estimate fixed in integers.
__device__ __forceinline__ uint32_t lt_bin16(uint32_t t, uint32_t mx) {
  int b = min(15, (int)(16.0f * sqrtf((float)t / (float)max(mx, 1u))));
  const unsigned long long T = 256ull * t, M = mx;
  while (b < 15 && (unsigned long long)((b + 1) * (b + 1)) * M <= T) ++b;
  while (b > 0 && (unsigned long long)(b * b) * M > T) --b;
  return (uint32_t)b;
}

// The same bin from a float estimate e of 16 sqrt(t / mx) that is within
// one of it (from sqrt(t * 256 / mx), or from sqrtf(t) times 16 / sqrtf(mx)):
// two integer checks then make it exact, in 32 bits (b^2 <= 256, mx < 2^24,
// 256 t < 2^32).
__device__ __forceinline__ uint32_t lt_bin16_e(uint32_t t, uint32_t mx, float e) {
  uint32_t b = min(15u, (uint32_t)e);
  const uint32_t T = 256u * t;
  if (b < 15u && (b + 1) * (b + 1) * mx <= T) ++b;
  if (b > 0u && b * b * mx > T) --b;
  return b;
}
__device__ __forceinline__ uint32_t lt_bin16_r(uint32_t t, uint32_t mx, float rmx) {
  uint32_t b = min(15u, (uint32_t)sqrtf((float)t * rmx));
  const uint32_t T = 256u * t;
  if (b < 15u && (b + 1) * (b + 1) * mx <= T) ++b;
  if (b > 0u && b * b * mx > T) --b;
  return b;
}

// Sums of one warp's 32 per-thread partials that all belong to one label
// (or to none), by warp reductions: counts, max and the two fixed-point
// sums (each split into 16-bit halves whose warp sums fit 32 bits: a
// thread's partial is at most 4 * 2^32).
__device__ __forceinline__ void warp_uniform_sums(uint32_t& pk, uint32_t& mx, unsigned long long& q,
                                                  unsigned long long& qs) {
  pk = __reduce_add_sync(kFull, pk);
  mx = __reduce_max_sync(kFull, mx);
  const uint32_t qh = __reduce_add_sync(kFull, (uint32_t)(q >> 16)), ql = __reduce_add_sync(kFull, (uint32_t)q & 0xFFFFu);
  const uint32_t sh = __reduce_add_sync(kFull, (uint32_t)(qs >> 16)), sl = __reduce_add_sync(kFull, (uint32_t)qs & 0xFFFFu);
  q = ((unsigned long long)qh << 16) + ql;
  qs = ((unsigned long long)sh << 16) + sl;
}

template <int NDIM, bool FILTER>
__global__ void __launch_bounds__(256) shape_reduce_kernel(const uint32_t* __restrict__ labels,
                                                           const uint32_t* __restrict__ lt2, Dims d,
                                                           uint32_t n_labels, ShapeAcc acc,
                                                           WsHeader* __restrict__ hdr, uint32_t min_lt2,
                                                           int z_lo) {
  shape_reduce_body<NDIM, FILTER>(labels, lt2, d, n_labels, acc, hdr, min_lt2, z_lo,
                                  make_uint3(blockIdx.x, blockIdx.y, blockIdx.z));
}

// Vector form for nx % 4 == 0: a thread covers 4 consecutive voxels of a
// row (16-byte loads of labels, LT2 and the neighbouring rows), adds the
// voxels of its first nonzero label locally (voxels of another nonzero label
// in the same 4, which needs touching objects, go straight to the atomics).
// A warp whose voxels carry one label (the common case) sums its partials
// by warp reductions; otherwise runs of equal labels across the warp are
// combined by a segmented scan as above. With HIST, the voxels are also
// counted into hist[label][32]: bin b (interior) or 16 + b (shell), b the
// LT/M bin of lt_bin16 with M^2 = ref_max[label] (the object's largest
// LT2); equal (label, shell, bin) keys of consecutive voxels are counted
// together, then runs of equal keys across the warp.
template <int NDIM, bool FILTER, bool HIST>
__device__ __forceinline__ void shape_reduce4_body(const uint32_t* __restrict__ labels,
                                                   const uint32_t* __restrict__ lt2, const Dims& d, uint32_t n_labels,
                                                   const ShapeAcc& acc, WsHeader* __restrict__ hdr, uint32_t min_lt2,
                                                   int z_lo, const uint32_t* __restrict__ ref_max,
                                                   uint32_t* __restrict__ hist, uint3 blk) {
  const int lane = threadIdx.x & 31;
  const int x0 = 4 * ((int)blk.x * blockDim.x + threadIdx.x);
  const int y = (int)blk.y * blockDim.y + threadIdx.y, z = (int)blk.z + z_lo;
  const bool in = x0 < d.nx && y < d.ny;
  const size_t sy = (size_t)d.nx, sz = (size_t)d.nx * d.ny;
  const size_t v = in ? (size_t)z * sz + (size_t)y * sy + x0 : 0;
  uint4 L = make_uint4(0u, 0u, 0u, 0u);
  if (in) L = *reinterpret_cast<const uint4*>(labels + v);
  const bool any = (L.x | L.y | L.z | L.w) != 0u;
  if (__ballot_sync(kFull, any) == 0) return;  // uniform per warp
  uint32_t lab = 0, pk = 0, mx = 0;
  unsigned long long q = 0, qs = 0;
  uint32_t hkey = 0xFFFFFFFFu, hcnt = 0;  // HIST: this thread's first key and its count
  bool bad = false;
  if (any) {
    const uint4 T = *reinterpret_cast<const uint4*>(lt2 + v);
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    uint4 Ym = y > 0 ? *reinterpret_cast<const uint4*>(labels + v - sy) : zero;
    uint4 Yp = y + 1 < d.ny ? *reinterpret_cast<const uint4*>(labels + v + sy) : zero;
    uint4 Zm = zero, Zp = zero;
    if (NDIM == 3) {
      if (z > 0) Zm = *reinterpret_cast<const uint4*>(labels + v - sz);
      if (z + 1 < d.nz) Zp = *reinterpret_cast<const uint4*>(labels + v + sz);
    }
    uint32_t xl = x0 > 0 ? labels[v - 1] : 0u;
    uint32_t xr = x0 + 4 < d.nx ? labels[v + 4] : 0u;
    if (FILTER) {  // neighbours below the threshold are outside their object
      if (y > 0) Ym = filter4(Ym, lt2, v - sy, min_lt2);
      if (y + 1 < d.ny) Yp = filter4(Yp, lt2, v + sy, min_lt2);
      if (NDIM == 3 && z > 0) Zm = filter4(Zm, lt2, v - sz, min_lt2);
      if (NDIM == 3 && z + 1 < d.nz) Zp = filter4(Zp, lt2, v + sz, min_lt2);
      if (xl && lt2[v - 1] < min_lt2) xl = 0u;
      if (xr && lt2[v + 4] < min_lt2) xr = 0u;
    }
    uint4 Lf = L;  // labels as objects: range-checked raw labels, filtered
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t l = comp(L, k);
      if (l >= n_labels) bad = true;
      const uint32_t lf = l >= n_labels || (FILTER && comp(T, k) < min_lt2) ? 0u : l;
      Lf = make_uint4(k == 0 ? lf : Lf.x, k == 1 ? lf : Lf.y, k == 2 ? lf : Lf.z, k == 3 ? lf : Lf.w);
    }
    if (FILTER) L = Lf;
    uint32_t hprev = 0xFFFFFFFFu, hrun = 0, lref = 0, mref = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      uint32_t l = comp(L, k);
      uint32_t hk = 0xFFFFFFFFu;
      if (l != 0 && l < n_labels) {
        const uint32_t left = k == 0 ? xl : comp(L, k - 1), right = k == 3 ? xr : comp(L, k + 1);
        bool s = left != l || right != l || comp(Ym, k) != l || comp(Yp, k) != l;
        if (NDIM == 3) s = s || comp(Zm, k) != l || comp(Zp, k) != l;
        const uint32_t t = comp(T, k);
        const uint32_t qq = __float2uint_rn(sqrtf((float)t) * kFixScale);
        if (lab == 0) lab = l;
        if (l == lab) {
          pk += 1u | (s ? 1u << 16 : 0u);
          mx = max(mx, t);
          q += qq;
          qs += s ? qq : 0ull;
        } else {  // a second object within the same four voxels
          atomicAdd(acc.volume + l, 1u);
          if (s) atomicAdd(acc.n_shell + l, 1u);
          atomicAdd(acc.sum_lt + l, (unsigned long long)qq);
          if (s) atomicAdd(acc.sum_shell_lt + l, (unsigned long long)qq);
          atomicMax(acc.max_lt2 + l, t);
        }
        if (HIST) {
          if (l != lref) {
            lref = l;
            mref = ref_max[l];
          }
          hk = l * 32u + (s ? 16u : 0u) + lt_bin16(t, mref);
        }
      }
      if (HIST && hk != hprev) {  // close the previous run of keys
        if (hprev != 0xFFFFFFFFu) {
          if (hkey == 0xFFFFFFFFu) {
            hkey = hprev;
            hcnt = hrun;
          } else {
            atomicAdd(hist + hprev, hrun);
          }
        }
        hprev = hk;
        hrun = 0;
      }
      ++hrun;
    }
    if (HIST && hprev != 0xFFFFFFFFu) {
      if (hkey == 0xFFFFFFFFu) {
        hkey = hprev;
        hcnt = hrun;
      } else if (hprev == hkey) {
        hcnt += hrun;
      } else {
        atomicAdd(hist + hprev, hrun);
      }
    }
  }
  if (__any_sync(kFull, bad) && lane == 0) atomicOr(&hdr->error, ERR_LABEL_RANGE);
  const unsigned has = __ballot_sync(kFull, lab != 0);
  const uint32_t l0 = has ? __shfl_sync(kFull, lab, __ffs(has) - 1) : 0u;
  if (__all_sync(kFull, lab == 0 || lab == l0)) {
    if (has) {
      warp_uniform_sums(pk, mx, q, qs);
      if (lane == 0) {
        atomicAdd(acc.volume + l0, pk & 0xFFFFu);
        atomicAdd(acc.n_shell + l0, pk >> 16);
        atomicAdd(acc.sum_lt + l0, q);
        atomicAdd(acc.sum_shell_lt + l0, qs);
        atomicMax(acc.max_lt2 + l0, mx);
      }
    }
  } else {
    // segmented inclusive scan over runs of equal labels
    const uint32_t lprev = __shfl_up_sync(kFull, lab, 1);
    int seg = (lane == 0 || lprev != lab) ? lane : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(kFull, seg, o);
      if (lane >= o) seg = max(seg, t);
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t a = __shfl_up_sync(kFull, pk, o);
      const unsigned long long b = __shfl_up_sync(kFull, q, o);
      const unsigned long long c = __shfl_up_sync(kFull, qs, o);
      const uint32_t m = __shfl_up_sync(kFull, mx, o);
      if (lane - o >= seg) {
        pk += a;
        q += b;
        qs += c;
        mx = max(mx, m);
      }
    }
    const uint32_t lnext = __shfl_down_sync(kFull, lab, 1);
    if (lab && (lane == 31 || lnext != lab)) {
      atomicAdd(acc.volume + lab, pk & 0xFFFFu);
      atomicAdd(acc.n_shell + lab, pk >> 16);
      atomicAdd(acc.sum_lt + lab, q);
      atomicAdd(acc.sum_shell_lt + lab, qs);
      atomicMax(acc.max_lt2 + lab, mx);
    }
  }
  if (HIST) {
    // segmented inclusive scan of the counts over runs of equal first keys
    const uint32_t kprev = __shfl_up_sync(kFull, hkey, 1);
    int seg = (lane == 0 || kprev != hkey) ? lane : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(kFull, seg, o);
      if (lane >= o) seg = max(seg, t);
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t a = __shfl_up_sync(kFull, hcnt, o);
      if (lane - o >= seg) hcnt += a;
    }
    const uint32_t knext = __shfl_down_sync(kFull, hkey, 1);
    if (hkey != 0xFFFFFFFFu && (lane == 31 || knext != hkey)) atomicAdd(hist + hkey, hcnt);
  }
}

template <int NDIM, bool FILTER, bool HIST>
__global__ void __launch_bounds__(256) shape_reduce4_kernel(const uint32_t* __restrict__ labels,
                                                            const uint32_t* __restrict__ lt2, Dims d,
                                                            uint32_t n_labels, ShapeAcc acc,
                                                            WsHeader* __restrict__ hdr, uint32_t min_lt2,
                                                            int z_lo, const uint32_t* __restrict__ ref_max,
                                                            uint32_t* __restrict__ hist) {
  shape_reduce4_body<NDIM, FILTER, HIST>(labels, lt2, d, n_labels, acc, hdr, min_lt2, z_lo, ref_max, hist,
                                         make_uint3(blockIdx.x, blockIdx.y, blockIdx.z));
}

// z-marching form for 3D volumes with nx % 4 == 0: a thread owns 4
// consecutive voxels of one row (x0 .. x0+3, y) and walks kZChunk planes of
// z; the labels of the planes below and above stay in registers (the z
// neighbours of the shell test), and the sums of the thread's current object
// accumulate in registers until the object changes, when they go out as one
// set of atomics (a column meets a new object every ~2R planes, so this is
// far fewer atomics than one per warp and plane). A voxel of a second object
// within the same four voxels flushes and switches too (touching objects).
// With HIST the thread also counts its current object's voxels per (shell,
// LT/M bin) in shared memory (counter b of thread t at b * 256 + t, so the
// threads of a warp hit distinct banks), flushed with the sums.
constexpr int kZChunk = 32;

// Four consecutive uint32 at p (voxels x0 .. x0+3 of a row): one 16-byte load
// when rows are 16-byte aligned (VEC), else scalar loads, zero past nx.
template <bool VEC>
__device__ __forceinline__ uint4 load_quad(const uint32_t* __restrict__ p, int x0, int nx) {
  if (VEC) return *reinterpret_cast<const uint4*>(p);
  return make_uint4(p[0], x0 + 1 < nx ? p[1] : 0u, x0 + 2 < nx ? p[2] : 0u, x0 + 3 < nx ? p[3] : 0u);
}

template <bool HIST, bool VEC>
__device__ __forceinline__ void shape_reduce_z_body(const uint32_t* __restrict__ labels,
                                                    const uint32_t* __restrict__ lt2, const Dims& d,
                                                    uint32_t n_labels, const ShapeAcc& acc,
                                                    WsHeader* __restrict__ hdr, int z_lo, int z_hi,
                                                    const uint32_t* __restrict__ ref_max,
                                                    uint32_t* __restrict__ hist, uint32_t* __restrict__ hs,
                                                    uint3 blk) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int x0 = 4 * ((int)blk.x * blockDim.x + threadIdx.x);
  const int y = (int)blk.y * blockDim.y + threadIdx.y;
  const int zb = z_lo + (int)blk.z * kZChunk, ze = min(z_hi, zb + kZChunk);
  if (x0 >= d.nx || y >= d.ny || zb >= ze) return;
  const size_t sy = (size_t)d.nx, sz = (size_t)d.nx * d.ny;
  const uint32_t* col = labels + (size_t)y * sy + x0;  // this thread's labels at z = 0
  const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
  auto lab4 = [&](int z) { return load_quad<VEC>(col + (size_t)z * sz, x0, d.nx); };
  uint4 Lm = zb > 0 ? lab4(zb - 1) : zero, L = lab4(zb);
  uint32_t cl = 0, mref = 0, cnt = 0, shc = 0, mx = 0, used = 0;  // used: bins counted since the last flush
  float rref = 0.f;
  unsigned long long q = 0, qs = 0;
  bool bad = false;
  auto flush = [&]() {
    if (cl == 0) return;
    atomicAdd(acc.volume + cl, cnt);
    if (shc) atomicAdd(acc.n_shell + cl, shc);
    atomicAdd(acc.sum_lt + cl, q);
    if (shc) atomicAdd(acc.sum_shell_lt + cl, qs);
    atomicMax(acc.max_lt2 + cl, mx);
    if (HIST)
      while (used) {
        const int b = __ffs(used) - 1;
        used &= used - 1;
        atomicAdd(hist + cl * 32u + b, hs[b * 256 + tid]);
        hs[b * 256 + tid] = 0u;
      }
    cnt = shc = mx = 0;
    q = qs = 0;
  };
  for (int z = zb; z < ze; ++z) {
    const uint4 Lp = z + 1 < d.nz ? lab4(z + 1) : zero;
    if ((L.x | L.y | L.z | L.w) != 0u) {
      const size_t v = (size_t)z * sz + (size_t)y * sy + x0;
      const uint4 T = load_quad<VEC>(lt2 + v, x0, d.nx);
      const uint4 Ym = y > 0 ? load_quad<VEC>(labels + v - sy, x0, d.nx) : zero;
      const uint4 Yp = y + 1 < d.ny ? load_quad<VEC>(labels + v + sy, x0, d.nx) : zero;
      const uint32_t xl = x0 > 0 ? labels[v - 1] : 0u;
      const uint32_t xr = x0 + 4 < d.nx ? labels[v + 4] : 0u;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t l = comp(L, k);
        if (l == 0) continue;
        if (l >= n_labels) {
          bad = true;
          continue;
        }
        const uint32_t left = k == 0 ? xl : comp(L, k - 1), right = k == 3 ? xr : comp(L, k + 1);
        const bool s = left != l || right != l || comp(Ym, k) != l || comp(Yp, k) != l || comp(Lm, k) != l ||
                       comp(Lp, k) != l;
        const uint32_t t = comp(T, k);
        const float st = sqrtf((float)t);
        const uint32_t qq = __float2uint_rn(st * kFixScale);
        if (l != cl) {
          flush();
          cl = l;
          if (HIST) {
            mref = max(ref_max[l], 1u);
            rref = 16.0f / sqrtf((float)mref);
          }
        }
        ++cnt;
        shc += s ? 1u : 0u;
        mx = max(mx, t);
        q += qq;
        qs += s ? qq : 0ull;
        if (HIST) {
          const uint32_t b = (s ? 16u : 0u) + lt_bin16_e(t, mref, st * rref);
          atomicAdd(&hs[b * 256 + tid], 1u);  // the thread's own counter: no conflicts
          used |= 1u << b;
        }
      }
    }
    Lm = L;
    L = Lp;
  }
  flush();
  if (bad) atomicOr(&hdr->error, ERR_LABEL_RANGE);
}

template <bool HIST, bool VEC>
__global__ void __launch_bounds__(256) shape_reduce_z_kernel(const uint32_t* __restrict__ labels,
                                                             const uint32_t* __restrict__ lt2, Dims d,
                                                             uint32_t n_labels, ShapeAcc acc,
                                                             WsHeader* __restrict__ hdr, int z_lo, int z_hi,
                                                             const uint32_t* __restrict__ ref_max,
                                                             uint32_t* __restrict__ hist) {
  __shared__ uint32_t hs[HIST ? 32 * 256 : 1];
  if (HIST) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int b = 0; b < 32; ++b) hs[b * 256 + tid] = 0u;  // each thread clears its own counters
  }
  shape_reduce_z_body<HIST, VEC>(labels, lt2, d, n_labels, acc, hdr, z_lo, z_hi, ref_max, hist, hs,
                                 make_uint3(blockIdx.x, blockIdx.y, blockIdx.z));
}

// grid of the z-marching form over planes [z_lo, z_hi)
inline dim3 z_grid(const Dims& d, int z_lo, int z_hi) {
  return dim3(((d.nx + 3) / 4 + 63) / 64, (d.ny + 3) / 4, (z_hi - z_lo + kZChunk - 1) / kZChunk);
}

// The shape reduction over many volumes (each volume's accumulators at the
// start of its workspace body): VEC4 with the 64 x 4 blocks of the vector
// form (rows of a multiple of 4 voxels), else the one-voxel form.
template <int NDIM, bool VEC4>
__global__ void __launch_bounds__(256) shape_reduce_multi_kernel(MultiArgs m) {
  uint3 blk;
  const VolParams& p = m.vols[find_volume(m, blockIdx.x, blk)];
  const ShapeAcc acc = acc_layout(p.body, p.n_labels);
  if (NDIM == 3)
    shape_reduce_z_body<false, VEC4>(p.labels, p.lt2, p.d, p.n_labels, acc, p.hdr, 0, p.d.nz, nullptr, nullptr,
                                     nullptr, blk);
  else if (VEC4)
    shape_reduce4_body<NDIM, false, false>(p.labels, p.lt2, p.d, p.n_labels, acc, p.hdr, 0u, 0, nullptr, nullptr,
                                           blk);
  else
    shape_reduce_body<NDIM, false>(p.labels, p.lt2, p.d, p.n_labels, acc, p.hdr, 0u, 0, blk);
}

__device__ double spheroid_area(double a, double c) {
  const double pi = 3.141592653589793;
  if (c == a) return 4.0 * pi * a * a;
  if (c < a) {
    const double e = sqrt(1.0 - (c * c) / (a * a));
    return 2.0 * pi * a * a * (1.0 + (1.0 - e * e) / e * atanh(e));
  }
  const double e = sqrt(1.0 - (a * a) / (c * c));
  return 2.0 * pi * a * a * (1.0 + c / (a * e) * asin(e));
}

template <int NDIM>
__device__ __forceinline__ void shape_finalize_body(const ShapeAcc& acc, uint32_t n_labels, float* __restrict__ S,
                                                    float* __restrict__ R, const lt_object_stats& st,
                                                    const uint32_t* __restrict__ hist, float* __restrict__ F,
                                                    uint32_t l) {
  if (l >= n_labels) return;
  const uint32_t V = l ? acc.volume[l] : 0u;
  const uint32_t ns = l ? acc.n_shell[l] : 0u;
  const uint32_t mx = l ? acc.max_lt2[l] : 0u;
  const unsigned long long sl = l ? acc.sum_lt[l] : 0ull, ss = l ? acc.sum_shell_lt[l] : 0ull;
  if (st.volume) st.volume[l] = V;
  if (st.n_shell) st.n_shell[l] = ns;
  if (st.max_lt2) st.max_lt2[l] = mx;
  if (st.sum_lt) st.sum_lt[l] = sl;
  if (st.sum_shell_lt) st.sum_shell_lt[l] = ss;
  double sph = nan(""), rnd = nan("");
  if (V > 0) {
    const double pi = 3.141592653589793;
    const double inv = 1.0 / 1048576.0;
    const double Vd = (double)V;
    const double a = (double)sl * inv / Vd;
    if (NDIM == 3) {
      const double c = 3.0 * Vd / (4.0 * pi * a * a);
      const double k = cbrt(6.0 * Vd);
      sph = cbrt(pi) * k * k / spheroid_area(a, c);
    } else {
      const double b = Vd / (pi * a);
      const double po = pi * (3.0 * (a + b) - sqrt((3.0 * a + b) * (a + 3.0 * b)));
      sph = 2.0 * sqrt(pi * Vd) / po;
    }
    rnd = ((double)ss * inv / (double)ns) / sqrt((double)mx);
  }
  if (S) S[l] = (float)sph;
  if (R) R[l] = (float)rnd;

}

template <int NDIM>
__global__ void shape_finalize_kernel(ShapeAcc acc, uint32_t n_labels, float* __restrict__ S,
                                      float* __restrict__ R, lt_object_stats st,
                                      const uint32_t* __restrict__ hist, float* __restrict__ F) {
  shape_finalize_body<NDIM>(acc, n_labels, S, R, st, hist, F, blockIdx.x * blockDim.x + threadIdx.x);
}

template <int NDIM>
__global__ void shape_finalize_multi_kernel(MultiArgs m) {
  uint3 blk;
  const VolParams& p = m.vols[find_volume(m, blockIdx.x, blk)];
  const lt_object_stats st = {nullptr, nullptr, nullptr, nullptr, nullptr};
  shape_finalize_body<NDIM>(acc_layout(p.body, p.n_labels), p.n_labels, p.S, p.R, st, nullptr, nullptr,
                            blk.x * blockDim.x + threadIdx.x);
}

// Zeroes every volume's workspace header (WHAT 0) or shape accumulators
// (WHAT 1), 16 bytes per thread.
template <int WHAT>
__global__ void __launch_bounds__(256) clear_multi_kernel(MultiArgs m) {
  uint3 blk;
  const VolParams& p = m.vols[find_volume(m, blockIdx.x, blk)];
  char* base = WHAT == 0 ? reinterpret_cast<char*>(p.hdr) : p.body;
  const size_t bytes = WHAT == 0 ? sizeof(WsHeader) : acc_bytes(p.n_labels);
  const size_t i = ((size_t)blk.x * blockDim.x + threadIdx.x) * 16;
  if (i < bytes) *reinterpret_cast<uint4*>(base + i) = make_uint4(0u, 0u, 0u, 0u);
}

// Roundness mapped to 0-1 with the reported minimum (Sec. 6.1). Step 1:
// the smallest finite R over [0, n) by warp minima and one atomic per warp
// (R > 0, so the float bits order like the values). Step 2: the map.
__global__ void min_finite_kernel(const float* __restrict__ R, uint32_t n, uint32_t* __restrict__ out_bits) {
  uint32_t m = 0x7F800000u;  // +inf (out_bits starts at 0xFFFFFFFF: no finite value)
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float r = R[i];
    if (isfinite(r) && r >= 0.f) m = min(m, __float_as_uint(r));
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) m = min(m, __shfl_xor_sync(kFull, m, o));
  if ((threadIdx.x & 31) == 0 && m != 0x7F800000u) atomicMin(out_bits, m);
}

__global__ void rescale_kernel(const float* __restrict__ R, uint32_t n, const uint32_t* __restrict__ min_bits,
                               float r_min, float* __restrict__ out) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float r = R[i];
  const double m = r_min >= 0.f ? (double)r_min : (double)__uint_as_float(*min_bits);
  float v = nanf("");
  if (isfinite(r)) v = m >= 1.0 ? 1.f : (float)fmax(((double)r - m) / (1.0 - m), 0.0);
  out[i] = v;
}

}  // namespace

cudaError_t rescale_launch(const float* R, uint32_t n, float r_min, uint32_t* scratch, float* out,
                           cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (r_min < 0.f) {
    cudaError_t e = cudaMemsetAsync(scratch, 0xFF, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)std::min<uint32_t>((n + 255) / 256, (uint32_t)sm_count() * 4u);
    TraceScope t("roundness_min", s);
    min_finite_kernel<<<blocks, 256, 0, s>>>(R, n, scratch);
  }
  {
    TraceScope t("roundness_rescale", s);
    rescale_kernel<<<(n + 255) / 256, 256, 0, s>>>(R, n, scratch, r_min, out);
  }
  return cudaGetLastError();
}


size_t shape_workspace_bytes(uint32_t n_labels) { return acc_bytes(n_labels); }

template <int NDIM, bool FILTER>
void launch_reduce(const uint32_t* labels, const uint32_t* lt2, uint32_t n_labels, const Dims& d,
                   const ShapeAcc& acc, WsHeader* hdr, uint32_t min_lt2, int z_lo, int z_hi, cudaStream_t s) {
  TraceScope t("shape_reduce", s);
  if (NDIM == 3 && !FILTER) {
    // 64 x 4 threads (256 x 4 voxels of a plane), kZChunk planes each
    const dim3 block(64, 4), grid = z_grid(d, z_lo, z_hi);
    if (d.nx % 4 == 0)
      shape_reduce_z_kernel<false, true>
          <<<grid, block, 0, s>>>(labels, lt2, d, n_labels, acc, hdr, z_lo, z_hi, nullptr, nullptr);
    else
      shape_reduce_z_kernel<false, false>
          <<<grid, block, 0, s>>>(labels, lt2, d, n_labels, acc, hdr, z_lo, z_hi, nullptr, nullptr);
  } else if (d.nx % 4 == 0) {
    // 64 threads (256 voxels) per row, 4 rows per CTA
    dim3 block(64, 4), grid((d.nx / 4 + 63) / 64, (d.ny + 3) / 4, z_hi - z_lo);
    shape_reduce4_kernel<NDIM, FILTER, false>
        <<<grid, block, 0, s>>>(labels, lt2, d, n_labels, acc, hdr, min_lt2, z_lo, nullptr, nullptr);
  } else {
    dim3 grid((d.nx + 255) / 256, d.ny, z_hi - z_lo);
    shape_reduce_kernel<NDIM, FILTER><<<grid, 256, 0, s>>>(labels, lt2, d, n_labels, acc, hdr, min_lt2, z_lo);
  }
}


cudaError_t shape_clear(void* body, uint32_t n_labels, cudaStream_t s) {
  return cudaMemsetAsync(body, 0, acc_bytes(n_labels), s);
}

cudaError_t shape_accumulate(const uint32_t* labels, const uint32_t* lt2, uint32_t n_labels, const Dims& d,
                             WsHeader* hdr, void* body, int z_lo, int z_hi, cudaStream_t s, uint32_t min_lt2) {
  const ShapeAcc acc = acc_layout(body, n_labels);
  if (z_hi <= z_lo) return cudaSuccess;
  if (min_lt2 > 1) {  // (every object voxel has LT2 >= 1: thresholds 0 and 1 filter nothing)
    if (d.ndim == 3)
      launch_reduce<3, true>(labels, lt2, n_labels, d, acc, hdr, min_lt2, z_lo, z_hi, s);
    else
      launch_reduce<2, true>(labels, lt2, n_labels, d, acc, hdr, min_lt2, z_lo, z_hi, s);
  } else if (d.ndim == 3) {
    launch_reduce<3, false>(labels, lt2, n_labels, d, acc, hdr, 0u, z_lo, z_hi, s);
  } else {
    launch_reduce<2, false>(labels, lt2, n_labels, d, acc, hdr, 0u, z_lo, z_hi, s);
  }
  return cudaGetLastError();
}

cudaError_t shape_finalize(int ndim, uint32_t n_labels, void* body, float* S, float* R,
                           const lt_object_stats* stats, cudaStream_t s) {
  const ShapeAcc acc = acc_layout(body, n_labels);
  lt_object_stats st = {nullptr, nullptr, nullptr, nullptr, nullptr};
  if (stats) st = *stats;
  const unsigned blocks = (n_labels + 255) / 256;
  {
    TraceScope t("shape_finalize", s);
    if (ndim == 3)
      shape_finalize_kernel<3><<<blocks, 256, 0, s>>>(acc, n_labels, S, R, st, nullptr, nullptr);
    else
      shape_finalize_kernel<2><<<blocks, 256, 0, s>>>(acc, n_labels, S, R, st, nullptr, nullptr);
  }
  return cudaGetLastError();
}

cudaError_t shape_launch(const uint32_t* labels, const uint32_t* lt2, uint32_t n_labels,
                         const Dims& d, WsHeader* hdr, void* body, float* S, float* R,
                         const lt_object_stats* stats, cudaStream_t s, uint32_t min_lt2) {
  cudaError_t e = shape_clear(body, n_labels, s);
  if (e == cudaSuccess) e = shape_accumulate(labels, lt2, n_labels, d, hdr, body, 0, d.nz, s, min_lt2);
  if (e == cudaSuccess) e = shape_finalize(d.ndim, n_labels, body, S, R, stats, s);
  return e;
}

// ---- batched shape stage (see StagePlan). Kinds: 0 reduction with
// 4-voxel vectors, 1 one-voxel reduction, 2 finalize, 3 clear headers, 4
// clear accumulators.
dim3 shape_multi_grid(const Dims& d, uint32_t n_labels, int kind) {
  switch (kind) {
    case 0: return d.ndim == 3 ? z_grid(d, 0, d.nz) : dim3((d.nx / 4 + 63) / 64, (d.ny + 3) / 4, d.nz);
    case 1: return d.ndim == 3 ? z_grid(d, 0, d.nz) : dim3((d.nx + 255) / 256, d.ny, d.nz);
    case 2: return dim3((n_labels + 255) / 256, 1, 1);
    case 3: return dim3(1, 1, 1);
    default: return dim3((unsigned)((acc_bytes(n_labels) + 4095) / 4096), 1, 1);
  }
}

cudaError_t shape_multi_launch(const MultiArgs& m, uint32_t blocks, int kind, int ndim, cudaStream_t s) {
  if (blocks == 0) return cudaSuccess;
  if (kind == 0) {
    TraceScope t("shape_reduce", s);
    if (ndim == 3)
      shape_reduce_multi_kernel<3, true><<<blocks, dim3(64, 4), 0, s>>>(m);
    else
      shape_reduce_multi_kernel<2, true><<<blocks, dim3(64, 4), 0, s>>>(m);
  } else if (kind == 1) {
    TraceScope t("shape_reduce", s);
    if (ndim == 3)
      shape_reduce_multi_kernel<3, false><<<blocks, dim3(64, 4), 0, s>>>(m);
    else
      shape_reduce_multi_kernel<2, false><<<blocks, 256, 0, s>>>(m);
  } else if (kind == 2) {
    TraceScope t("shape_finalize", s);
    if (ndim == 3)
      shape_finalize_multi_kernel<3><<<blocks, 256, 0, s>>>(m);
    else
      shape_finalize_multi_kernel<2><<<blocks, 256, 0, s>>>(m);
  } else if (kind == 3) {
    clear_multi_kernel<0><<<blocks, 256, 0, s>>>(m);
  } else {
    clear_multi_kernel<1><<<blocks, 256, 0, s>>>(m);
  }
  return cudaGetLastError();
}

size_t shape_features_bytes(uint32_t n_labels) { return acc_bytes(n_labels) + align_up((size_t)n_labels * 32 * 4); }

cudaError_t shape_features_launch(const uint32_t* labels, const uint32_t* lt2, uint32_t n_labels, const Dims& d,
                                  WsHeader* hdr, void* body, const uint32_t* ref_max, float* S, float* R, float* F,
                                  const lt_object_stats* stats, cudaStream_t s) {
  const ShapeAcc acc = acc_layout(body, n_labels);
  uint32_t* hist = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(body) + acc_bytes(n_labels));
  cudaError_t e = cudaMemsetAsync(body, 0, shape_features_bytes(n_labels), s);
  if (e != cudaSuccess) return e;
  if (d.ndim == 3 || d.nx % 4 == 0) {
    TraceScope t("shape_reduce_features", s);
    if (d.ndim == 3) {
      const dim3 block(64, 4), grid = z_grid(d, 0, d.nz);
      if (d.nx % 4 == 0)
        shape_reduce_z_kernel<true, true>
            <<<grid, block, 0, s>>>(labels, lt2, d, n_labels, acc, hdr, 0, d.nz, ref_max, hist);
      else
        shape_reduce_z_kernel<true, false>
            <<<grid, block, 0, s>>>(labels, lt2, d, n_labels, acc, hdr, 0, d.nz, ref_max, hist);
    } else {
      dim3 block(64, 4), grid((d.nx / 4 + 63) / 64, (d.ny + 3) / 4, d.nz);
      shape_reduce4_kernel<2, false, true>
          <<<grid, block, 0, s>>>(labels, lt2, d, n_labels, acc, hdr, 0u, 0, ref_max, hist);
    }
    e = cudaGetLastError();
  } else {  // rows not a multiple of 4 voxels: the histograms in a pass of their own
    e = shape_accumulate(labels, lt2, n_labels, d, hdr, body, 0, d.nz, s, 0u);
    if (e == cudaSuccess) e = features_hist_launch(labels, lt2, n_labels, d, ref_max, hist, s);
  }
  if (e != cudaSuccess) return e;
  e = shape_finalize(d.ndim, n_labels, body, S, R, stats, s);
  if (e != cudaSuccess) return e;
  const lt_object_stats sums = {acc.volume, acc.n_shell, acc.max_lt2, reinterpret_cast<uint64_t*>(acc.sum_lt),
                                reinterpret_cast<uint64_t*>(acc.sum_shell_lt)};
  return features_final_launch(n_labels, sums, S, R, hist, F, s);
}

}  // namespace ltk

// ------------------------------------------------------------------------
// lt_shape_measures_static: the shape measures with library-owned scratch,
// for callers that cannot allocate device memory. The scratch (workspace
// header + per-label accumulators for LT_STATIC_MAX_LABELS labels) is one
// file-scope device array; host code never dereferences its name, it asks the
// runtime for the array's device address once per device and passes that
// address to the same launch sequence as lt_shape_measures.
#include <mutex>

namespace {

// Header followed by the accumulators of LT_STATIC_MAX_LABELS labels, the
// same layout a caller-owned shape workspace has.
constexpr size_t kStaticScratchBytes = sizeof(ltk::WsHeader) + ltk::acc_bytes(LT_STATIC_MAX_LABELS);
static_assert(kStaticScratchBytes % ltk::kAlign == 0, "scratch ends on an alignment boundary");

static __device__ __align__(256) unsigned char g_shape_scratch[kStaticScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_addr[64] = {nullptr};

// Device address of g_shape_scratch on the current device (looked up on the
// first call per device), or nullptr on failure.
void* static_scratch() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> g(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_shape_scratch) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    g_scratch_addr[dev] = p;
  }
  return g_scratch_addr[dev];
}

}  // namespace

extern "C" lt_status lt_shape_measures_static(const uint32_t* labels, const uint32_t* lt2,
                                              uint32_t n_labels, int ndim, int64_t nx, int64_t ny,
                                              int64_t nz, float* sphericity, float* roundness,
                                              const lt_object_stats* stats, void* stream) {
  ltk::Dims d;
  lt_status st = ltk::make_dims_checked(ndim, nx, ny, nz, &d);
  if (st != LT_OK) return st;
  if (n_labels == 0) return LT_ERR_INVALID_ARG;
  if (n_labels > LT_STATIC_MAX_LABELS) return LT_ERR_WORKSPACE;
  static_assert(sizeof(ltk::WsHeader) + ltk::acc_bytes(LT_STATIC_MAX_LABELS) <= kStaticScratchBytes,
                "the scratch array holds the accumulators of the largest label count");
  if ((st = ltk::device_ptr_ok(labels)) != LT_OK || (st = ltk::device_ptr_ok(lt2)) != LT_OK) return st;
  if (sphericity && (st = ltk::device_ptr_ok(sphericity)) != LT_OK) return st;
  if (roundness && (st = ltk::device_ptr_ok(roundness)) != LT_OK) return st;
  if (stats) {
    const void* arr[5] = {stats->volume, stats->n_shell, stats->max_lt2, stats->sum_lt, stats->sum_shell_lt};
    for (const void* p : arr)
      if (p && (st = ltk::device_ptr_ok(p)) != LT_OK) return st;
  }
  if ((st = ltk::stream_on_current_device(stream)) != LT_OK) return st;
  void* scratch = static_scratch();
  if (!scratch) return LT_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  ltk::WsHeader* hdr = reinterpret_cast<ltk::WsHeader*>(scratch);
  // the array keeps the previous call's contents: clear the header here; the
  // accumulators are cleared by shape_launch
  cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(ltk::WsHeader), s);
  if (e == cudaSuccess)
    e = ltk::shape_launch(labels, lt2, n_labels, d, hdr, hdr + 1, sphericity, roundness, stats, s);
  return e == cudaSuccess ? LT_OK : LT_ERR_CUDA;
}
