// Exact squared Euclidean distance transform on sm_103a.
//
// Separable form of DT2(p) = min over background b of |p - b|^2 with the
// array padded by one background layer:
//   pass x:  g(p)  = distance along the row to the nearest background voxel
//                    (positions -1 and nx count as background); written as
//                    16-bit g (<= 8193) to scratch, squared on loading.
//   pass y:  f(p)  = min_q g^2(x, q, z) + (y - q)^2, plus the two padding
//                    rows at y = -1 and y = ny (height 0).
//   pass z:  same along z on f, giving DT2.
// Every value is an exact integer below 2^24 (axis lengths <= 8192).
//
// The strided passes compute the lower envelope of the parabolas
// q -> f(q) + (p - q)^2 at every p by scanning outwards from p and stopping
// once k^2 reaches the best value found (no parabola at distance >= k can be
// lower). Each CTA holds a full column tile (TX adjacent columns times the
// whole axis) in shared memory, so the pass runs in place and is exact.
#include "lt_internal.cuh"

namespace ltk {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSeg = 512;       // voxels of a row handled by one warp step
constexpr int kBig = 1 << 30;

// Bit j set when voxel x0 + j (0 <= j < 16, x0 + j < nx) is background.
template <bool VEC>
__device__ __forceinline__ uint32_t zero_bits(const uint8_t* __restrict__ row, int x0, int nx) {
  uint32_t bits = 0;
  if (VEC && x0 + 16 <= nx) {
    const uint4 q = __ldg(reinterpret_cast<const uint4*>(row + x0));
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t m = __vcmpeq4(w[k], 0u) & 0x01010101u;
      const uint32_t b = (m & 1u) | ((m >> 7) & 2u) | ((m >> 14) & 4u) | ((m >> 21) & 8u);
      bits |= b << (4 * k);
    }
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (x0 + j < nx && row[x0 + j] == 0) bits |= 1u << j;
  }
  return bits;
}

// Rows whose length is not a multiple of 16 start at any byte: a warp copies
// its 512-voxel segment of the mask into shared memory with coalesced byte
// loads (voxels past the row read as foreground) and each lane takes its 16
// bytes from there as one aligned vector.
__device__ __forceinline__ uint32_t zero_bits_staged(const uint8_t* __restrict__ row, int seg0, int nx,
                                                     uint8_t* buf) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
#pragma unroll 4
  for (int k = lane; k < kSeg; k += 32) buf[k] = seg0 + k < nx ? row[seg0 + k] : (uint8_t)1;
  __syncwarp();
  const uint4 q = *reinterpret_cast<const uint4*>(buf + lane * 16);
  const uint32_t w[4] = {q.x, q.y, q.z, q.w};
  uint32_t bits = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t m = __vcmpeq4(w[k], 0u) & 0x01010101u;
    bits |= ((m & 1u) | ((m >> 7) & 2u) | ((m >> 14) & 4u) | ((m >> 21) & 8u)) << (4 * k);
  }
  return bits;
}

// One warp per row (8 rows per CTA, block rb). Output: g per voxel (0 on
// background), 16 bits. VEC: rows of a multiple of 16 voxels, read and
// written with 16-byte vectors; otherwise through a per-warp staging buffer
// in shared memory with coalesced scalar accesses.
template <bool VEC>
__device__ __forceinline__ void edt_rows_body(const uint8_t* __restrict__ mask, uint16_t* __restrict__ out,
                                              int nx, uint32_t nrows, uint32_t rb) {
  __shared__ __align__(16) uint8_t stage_m[VEC ? 1 : 8][VEC ? 16 : kSeg];
  __shared__ __align__(16) uint16_t stage_g[VEC ? 1 : 8][VEC ? 8 : kSeg];
  const int lane = threadIdx.x & 31, wid = VEC ? 0 : (int)(threadIdx.x >> 5);
  const uint32_t row = rb * 8u + (threadIdx.x >> 5);
  if (row >= nrows) return;  // uniform per warp
  const uint8_t* mrow = mask + (size_t)row * nx;
  uint16_t* orow = out + (size_t)row * nx;
  const int nseg = (nx + kSeg - 1) / kSeg;  // <= 16

  // First background position of each segment, held by lane == segment, and
  // the inclusive suffix minimum over segments (lane i: min over segments
  // >= i); a row of one segment needs neither.
  int suf = kBig;
  if (nseg > 1) {  // uniform per warp
    int segfirst = kBig;
    for (int s = 0; s < nseg; ++s) {
      const int x0 = s * kSeg + lane * 16;
      const uint32_t z = VEC ? zero_bits<true>(mrow, x0, nx) : zero_bits_staged(mrow, s * kSeg, nx, stage_m[wid]);
      int f = z ? x0 + __ffs(z) - 1 : kBig;
#pragma unroll
      for (int o = 16; o; o >>= 1) f = min(f, __shfl_xor_sync(kFull, f, o));
      if (lane == s) segfirst = f;
    }
    suf = segfirst;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_down_sync(kFull, suf, o);
      if (lane + o < 32) suf = min(suf, t);
    }
  }

  int carry_left = -1;  // last background before the segment (virtual at -1)
  for (int s = 0; s < nseg; ++s) {
    const int x0 = s * kSeg + lane * 16;
    int after = __shfl_sync(kFull, suf, (s + 1) & 31);
    if (s + 1 >= nseg) after = kBig;
    after = min(after, nx);  // virtual background at nx
    const uint32_t z = VEC ? zero_bits<true>(mrow, x0, nx) : zero_bits_staged(mrow, s * kSeg, nx, stage_m[wid]);
    const int lastz = z ? x0 + 31 - __clz(z) : -1;
    const int firstz = z ? x0 + __ffs(z) - 1 : kBig;
    int incl = lastz;  // inclusive prefix max over lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl = max(incl, t);
    }
    int left = __shfl_up_sync(kFull, incl, 1);
    if (lane == 0) left = -1;
    left = max(left, carry_left);
    int inclr = firstz;  // inclusive suffix min over lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_down_sync(kFull, inclr, o);
      if (lane + o < 32) inclr = min(inclr, t);
    }
    int right = __shfl_down_sync(kFull, inclr, 1);
    if (lane == 31) right = kBig;
    right = min(right, after);
    carry_left = max(carry_left, __shfl_sync(kFull, incl, 31));

    int lpos[16];
    int L = left;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if ((z >> j) & 1u) L = x0 + j;
      lpos[j] = L;
    }
    uint32_t g[16];
    int R = right;
#pragma unroll
    for (int j = 15; j >= 0; --j) {
      if ((z >> j) & 1u) R = x0 + j;
      const int x = x0 + j;
      g[j] = (uint32_t)min(x - lpos[j], R - x);
    }
    const uint4 o0 = make_uint4(g[0] | (g[1] << 16), g[2] | (g[3] << 16), g[4] | (g[5] << 16), g[6] | (g[7] << 16));
    const uint4 o1 =
        make_uint4(g[8] | (g[9] << 16), g[10] | (g[11] << 16), g[12] | (g[13] << 16), g[14] | (g[15] << 16));
    if (VEC && x0 + 16 <= nx) {
      uint4* o4 = reinterpret_cast<uint4*>(orow + x0);
      o4[0] = o0;
      o4[1] = o1;
    } else if (VEC) {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (x0 + j < nx) orow[x0 + j] = (uint16_t)g[j];
    } else {  // through the staging buffer, then coalesced 2-byte stores
      uint16_t* sg = stage_g[wid];
      reinterpret_cast<uint4*>(sg + lane * 16)[0] = o0;
      reinterpret_cast<uint4*>(sg + lane * 16)[1] = o1;
      __syncwarp();
      const int sx = s * kSeg;
#pragma unroll 4
      for (int k = lane; k < kSeg; k += 32)
        if (sx + k < nx) orow[sx + k] = sg[k];
      __syncwarp();
    }
  }
}

template <bool VEC>
__global__ void __launch_bounds__(256) edt_rows_kernel(const uint8_t* __restrict__ mask,
                                                       uint16_t* __restrict__ out, int nx, uint32_t nrows) {
  edt_rows_body<VEC>(mask, out, nx, nrows, blockIdx.x);
}

// The row pass over many volumes (the 16-bit distances go to each volume's
// workspace body).
__global__ void __launch_bounds__(256) edt_rows_multi_kernel(MultiArgs m) {
  uint3 blk;
  const VolParams& p = m.vols[find_volume(m, blockIdx.x, blk)];
  const uint32_t nrows = (uint32_t)p.d.ny * (uint32_t)p.d.nz;
  uint16_t* g = reinterpret_cast<uint16_t*>(p.body);
  if (p.d.nx % 16 == 0)
    edt_rows_body<true>(p.mask, g, p.d.nx, nrows, blk.x);
  else
    edt_rows_body<false>(p.mask, g, p.d.nx, nrows, blk.x);
}

// Lower envelope at p. best starts at min(f(p), (p+1)^2, (L-p)^2), the last
// two being the padding parabolas; the scan only visits k with k^2 < best,
// hence k <= p and p + k < L: no bounds checks are needed. Two distances per
// step, the second only when its k^2 is still below best.
__device__ __forceinline__ uint32_t envelope_at(const uint32_t* __restrict__ col, int stride, int p,
                                                int L) {
  uint32_t best = col[p * stride];
  if (best == 0) return 0;
  const uint32_t b1 = (uint32_t)(p + 1) * (uint32_t)(p + 1);
  const uint32_t b2 = (uint32_t)(L - p) * (uint32_t)(L - p);
  best = min(best, min(b1, b2));
  const uint32_t* lo = col + p * stride;
  const uint32_t* hi = lo;
  uint32_t k2 = 1, dk = 3;  // k^2 and (k+1)^2 - k^2
  while (k2 < best) {
    best = min(best, min(lo[-stride], hi[stride]) + k2);
    const uint32_t k2b = k2 + dk;
    if (k2b >= best) break;
    best = min(best, min(lo[-2 * stride], hi[2 * stride]) + k2b);
    lo -= 2 * stride;
    hi += 2 * stride;
    k2 = k2b + dk + 2;
    dk += 4;
  }
  return best;
}

// Loads four consecutive elements of a column tile row as uint32 values:
// 16-bit row-pass distances are squared, 32-bit values copied.
__device__ __forceinline__ uint4 load4(const uint16_t* src, bool vec, int n) {
  uint32_t v[4];
  if (vec) {
    const uint2 q = *reinterpret_cast<const uint2*>(src);
    v[0] = q.x & 0xFFFFu; v[1] = q.x >> 16; v[2] = q.y & 0xFFFFu; v[3] = q.y >> 16;
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = j < n ? src[j] : 0u;
  }
  return make_uint4(v[0] * v[0], v[1] * v[1], v[2] * v[2], v[3] * v[3]);
}
__device__ __forceinline__ uint4 load4(const uint32_t* src, bool vec, int n) {
  if (vec) return *reinterpret_cast<const uint4*>(src);
  return make_uint4(0 < n ? src[0] : 0u, 1 < n ? src[1] : 0u, 2 < n ? src[2] : 0u, 3 < n ? src[3] : 0u);
}
__device__ __forceinline__ uint32_t load1(const uint16_t* src) { return (uint32_t)*src * (uint32_t)*src; }
__device__ __forceinline__ uint32_t load1(const uint32_t* src) { return *src; }

// Column pass in shared memory. Tile: TX adjacent columns x the whole axis
// (length L, stride sp between elements); blockIdx.y picks the other
// coordinate (stride so). `in` and `out` have the same layout and may be the
// same array (the tile is read completely before anything is written).
// Threads per CTA of a column tile of width TX: 512 for 32-column tiles
// (their rows are whole 128-byte lines; three such CTAs fit an SM), else 256.
template <int TX>
__host__ __device__ constexpr int cols_threads() { return TX == 32 ? 512 : 256; }

template <int TX, typename In>
__device__ __forceinline__ void edt_cols_body(const In* in, uint32_t* out, int L, size_t sp, int nx, size_t so,
                                              int vec, uint32_t bx, uint32_t by) {
  extern __shared__ uint4 smem_raw[];
  uint32_t* tile = reinterpret_cast<uint32_t*>(smem_raw);
  constexpr int NT = cols_threads<TX>();
  constexpr int Q = TX / 4;          // 4-element pieces per tile row
  constexpr int kRows = NT / Q;      // tile rows loaded per sweep of the CTA
  constexpr int kOutRows = NT / TX;  // tile rows computed per sweep
  const int x0 = (int)bx * TX;
  const size_t off = (size_t)by * so + x0;
  const int ncol = min(TX, nx - x0);
  {
    const int qd = threadIdx.x % Q;
    const bool v = vec && qd * 4 + 4 <= ncol;
    const In* src = in + off + (size_t)(threadIdx.x / Q) * sp + qd * 4;
    uint32_t* dst = tile + (threadIdx.x / Q) * TX + qd * 4;
    for (int p = threadIdx.x / Q; p < L; p += kRows) {
      *reinterpret_cast<uint4*>(dst) = load4(src, v, ncol - qd * 4);
      src += kRows * sp;
      dst += kRows * TX;
    }
  }
  __syncthreads();
  const int c = threadIdx.x % TX;
  if (c < ncol) {
    uint32_t* o = out + off + (size_t)(threadIdx.x / TX) * sp + c;
    for (int p = threadIdx.x / TX; p < L; p += kOutRows) {
      *o = envelope_at(tile + c, TX, p, L);
      o += kOutRows * sp;
    }
  }
}

template <int TX, typename In>
__global__ void __launch_bounds__(cols_threads<TX>()) edt_cols_kernel(const In* in, uint32_t* out, int L,
                                                                      size_t sp, int nx, size_t so, int vec) {
  edt_cols_body<TX, In>(in, out, L, sp, nx, so, vec, blockIdx.x, blockIdx.y);
}

// The y (AXIS 1: the 16-bit row distances of the workspace into dt2) or z
// (AXIS 2: dt2 in place) column pass over many volumes; the dynamic shared
// memory holds the longest column of the launch.
template <int TX, int AXIS>
__global__ void __launch_bounds__(cols_threads<TX>()) edt_cols_multi_kernel(MultiArgs m) {
  uint3 blk;
  const VolParams& p = m.vols[find_volume(m, blockIdx.x, blk)];
  const Dims& d = p.d;
  const size_t plane = (size_t)d.nx * d.ny;
  const int vec = d.nx % 4 == 0;
  if (AXIS == 1)
    edt_cols_body<TX, uint16_t>(reinterpret_cast<const uint16_t*>(p.body), p.dt2, d.ny, (size_t)d.nx, d.nx, plane,
                                vec, blk.x, blk.y);
  else
    edt_cols_body<TX, uint32_t>(p.dt2, p.dt2, d.nz, plane, d.nx, (size_t)d.nx, vec, blk.x, blk.y);
}

// Column pass reading `in` and writing `out` directly (axes longer than the
// shared-memory tile allows); `in` and `out` must differ.
template <typename In>
__device__ __forceinline__ void edt_cols_global_body(const In* __restrict__ in, uint32_t* __restrict__ out, int L,
                                                     size_t sp, int nx, size_t so, int rows_per_block, uint32_t bx,
                                                     uint32_t by, uint32_t bz) {
  const int c = (int)bx * 32 + (threadIdx.x & 31);
  if (c >= nx) return;
  const size_t off = (size_t)by * so + c;
  const In* col = in + off;
  const int p0 = (int)bz * rows_per_block;
  const int p1 = min(L, p0 + rows_per_block);
  for (int p = p0 + (threadIdx.x >> 5); p < p1; p += blockDim.x >> 5) {
    uint32_t best = load1(col + (size_t)p * sp);
    if (best) {
      const uint32_t b1 = (uint32_t)(p + 1) * (uint32_t)(p + 1);
      const uint32_t b2 = (uint32_t)(L - p) * (uint32_t)(L - p);
      best = min(best, min(b1, b2));
      for (uint32_t k = 1; k * k < best; ++k) {
        if ((uint32_t)p >= k) best = min(best, load1(col + (size_t)(p - (int)k) * sp) + k * k);
        if (p + (int)k < L) best = min(best, load1(col + (size_t)(p + (int)k) * sp) + k * k);
      }
    }
    out[off + (size_t)p * sp] = best;
  }
}

template <typename In>
__global__ void __launch_bounds__(256) edt_cols_global_kernel(const In* __restrict__ in,
                                                              uint32_t* __restrict__ out, int L,
                                                              size_t sp, int nx, size_t so,
                                                              int rows_per_block) {
  edt_cols_global_body<In>(in, out, L, sp, nx, so, rows_per_block, blockIdx.x, blockIdx.y, blockIdx.z);
}

// The y pass of 2D images whose columns are longer than the shared-memory
// tiles allow, over many images (16-bit row distances into dt2).
constexpr int kGlobalRows = 64;  // column positions per CTA of the global-memory pass
__global__ void __launch_bounds__(256) edt_cols_global_multi_kernel(MultiArgs m) {
  uint3 blk;
  const VolParams& p = m.vols[find_volume(m, blockIdx.x, blk)];
  const Dims& d = p.d;
  edt_cols_global_body<uint16_t>(reinterpret_cast<const uint16_t*>(p.body), p.dt2, d.ny, (size_t)d.nx, d.nx,
                                 (size_t)d.nx * d.ny, kGlobalRows, blk.x, blk.y, blk.z);
}

template <int TX, typename In>
cudaError_t launch_cols(const char* name, const In* in, uint32_t* out, int L, size_t sp, int nx, size_t so,
                        int nother, bool vec, cudaStream_t s) {
  const int smem = L * TX * 4;
  cudaError_t e = allow_smem((const void*)edt_cols_kernel<TX, In>, smem);
  if (e != cudaSuccess) return e;
  dim3 grid((nx + TX - 1) / TX, nother);
  {
    TraceScope t(name, s);
    edt_cols_kernel<TX, In><<<grid, cols_threads<TX>(), smem, s>>>(in, out, L, sp, nx, so, vec ? 1 : 0);
  }
  return cudaGetLastError();
}

// One strided pass from `in` into `out` (the same array is allowed except for
// axes over 2048, which go through `tmp`, n uint32 values).
template <typename In>
cudaError_t col_pass(const char* name, const In* in, uint32_t* out, int L, size_t sp, int nx, size_t so,
                     int nother, uint32_t* tmp, size_t n, cudaStream_t s, int tx_small) {
  const bool vec = (nx % 4) == 0;
  if (L <= 512 && tx_small == 8) return launch_cols<8>(name, in, out, L, sp, nx, so, nother, vec, s);
  if (L <= 512 && tx_small == 16) return launch_cols<16>(name, in, out, L, sp, nx, so, nother, vec, s);
  if (L <= 512) return launch_cols<32>(name, in, out, L, sp, nx, so, nother, vec, s);
  if (L <= 1024) return launch_cols<16>(name, in, out, L, sp, nx, so, nother, vec, s);
  if (L <= 2048) return launch_cols<8>(name, in, out, L, sp, nx, so, nother, vec, s);
  const bool inplace = (const void*)in == (const void*)out;
  const int rpb = 64;
  dim3 grid((nx + 31) / 32, nother, (L + rpb - 1) / rpb);
  {
    TraceScope t(name, s);
    edt_cols_global_kernel<In><<<grid, 256, 0, s>>>(in, inplace ? tmp : out, L, sp, nx, so, rpb);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !inplace) return e;
  return cudaMemcpyAsync(out, tmp, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
}

}  // namespace

// ---- batched passes (see StagePlan). Column tile width for a launch whose
// longest column is max_L: the tuned width up to 512, then 16 up to 1024, 8
// up to 2048; 0 = the global-memory pass (2D y pass only).
int edt_multi_tx(int max_L, int tx_small) {
  if (max_L <= 512) return tx_small == 8 || tx_small == 16 ? tx_small : 32;
  if (max_L <= 1024) return 16;
  if (max_L <= 2048) return 8;
  return 0;
}

// A volume's grid of pass 0 (rows), 1 (y columns), 2 (z columns) with tile
// width tx (0: the global-memory y pass).
dim3 edt_multi_grid(const Dims& d, int pass, int tx) {
  if (pass == 0) return dim3(((uint32_t)d.ny * (uint32_t)d.nz + 7) / 8, 1, 1);
  if (pass == 1 && tx == 0) return dim3((d.nx + 31) / 32, d.nz, (d.ny + kGlobalRows - 1) / kGlobalRows);
  return dim3((d.nx + tx - 1) / tx, pass == 1 ? d.nz : d.ny, 1);
}

template <int TX, int AXIS>
static cudaError_t launch_cols_multi(const MultiArgs& m, uint32_t blocks, int max_L, cudaStream_t s) {
  const int smem = max_L * TX * 4;
  cudaError_t e = allow_smem((const void*)edt_cols_multi_kernel<TX, AXIS>, smem);
  if (e != cudaSuccess) return e;
  {
    TraceScope t(AXIS == 1 ? "edt_cols_y" : "edt_cols_z", s);
    edt_cols_multi_kernel<TX, AXIS><<<blocks, cols_threads<TX>(), smem, s>>>(m);
  }
  return cudaGetLastError();
}

cudaError_t edt_multi_launch(const MultiArgs& m, uint32_t blocks, int pass, int tx, int max_L, cudaStream_t s) {
  if (blocks == 0) return cudaSuccess;
  if (pass == 0) {
    {
      TraceScope t("edt_rows_x", s);
      edt_rows_multi_kernel<<<blocks, 256, 0, s>>>(m);
    }
    return cudaGetLastError();
  }
  if (pass == 1 && tx == 0) {
    {
      TraceScope t("edt_cols_y", s);
      edt_cols_global_multi_kernel<<<blocks, 256, 0, s>>>(m);
    }
    return cudaGetLastError();
  }
  if (pass == 1) {
    if (tx == 8) return launch_cols_multi<8, 1>(m, blocks, max_L, s);
    if (tx == 16) return launch_cols_multi<16, 1>(m, blocks, max_L, s);
    return launch_cols_multi<32, 1>(m, blocks, max_L, s);
  }
  if (tx == 8) return launch_cols_multi<8, 2>(m, blocks, max_L, s);
  if (tx == 16) return launch_cols_multi<16, 2>(m, blocks, max_L, s);
  return launch_cols_multi<32, 2>(m, blocks, max_L, s);
}

cudaError_t edt_prepare_device() {
  cudaError_t e = cudaSuccess;
  e = allow_smem((const void*)edt_cols_kernel<32, uint16_t>, 64 * 1024);
  if (e == cudaSuccess) e = allow_smem((const void*)edt_cols_kernel<16, uint16_t>, 64 * 1024);
  if (e == cudaSuccess) e = allow_smem((const void*)edt_cols_kernel<8, uint16_t>, 64 * 1024);
  if (e == cudaSuccess) e = allow_smem((const void*)edt_cols_kernel<32, uint32_t>, 64 * 1024);
  if (e == cudaSuccess) e = allow_smem((const void*)edt_cols_kernel<16, uint32_t>, 64 * 1024);
  if (e == cudaSuccess) e = allow_smem((const void*)edt_cols_kernel<8, uint32_t>, 64 * 1024);
  return e;
}

// Scratch: the row pass's 16-bit distances, then (z axes over 2048) one
// uint32 per voxel for the out-of-place z pass.
size_t edt_workspace_bytes(const Dims& d) {
  const size_t g = align_up((size_t)d.n * sizeof(uint16_t));
  return d.ndim == 3 && d.nz > 2048 ? g + (size_t)d.n * sizeof(uint32_t) : g;
}

cudaError_t edt_launch(const uint8_t* mask, uint32_t* dt2, const Dims& d, void* ws, cudaStream_t s,
                       const Tuning& tu, int passes) {
  uint16_t* g = reinterpret_cast<uint16_t*>(ws);
  uint32_t* tmp = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(ws) + align_up((size_t)d.n * sizeof(uint16_t)));
  const size_t plane = (size_t)d.nx * d.ny;
  if (!(passes & 1)) {  // z pass only, on the y pass's output already in dt2
    if (d.ndim == 2) return cudaSuccess;
    return col_pass<uint32_t>("edt_cols_z", dt2, dt2, d.nz, plane, d.nx, (size_t)d.nx, d.ny, tmp, d.n, s,
                              tu.edt_tx_z);
  }
  const uint32_t nrows = (uint32_t)d.ny * (uint32_t)d.nz;
  const unsigned blocks = (nrows + 7) / 8;
  {
    TraceScope t("edt_rows_x", s);
    if (d.nx % 16 == 0)
      edt_rows_kernel<true><<<blocks, 256, 0, s>>>(mask, g, d.nx, nrows);
    else
      edt_rows_kernel<false><<<blocks, 256, 0, s>>>(mask, g, d.nx, nrows);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // y: columns of length ny, stride nx; one tile row per z; g -> dt2.
  e = col_pass<uint16_t>("edt_cols_y", g, dt2, d.ny, (size_t)d.nx, d.nx, plane, d.nz, tmp, d.n, s,
                         tu.edt_tx_y);
  if (e != cudaSuccess || d.ndim == 2 || !(passes & 2)) return e;
  // z: columns of length nz, stride nx*ny; one tile row per y; in place.
  return col_pass<uint32_t>("edt_cols_z", dt2, dt2, d.nz, plane, d.nx, (size_t)d.nx, d.ny, tmp, d.n, s,
                            tu.edt_tx_z);
}

}  // namespace ltk
