// The pipeline over a volume held in host memory, a few z planes at a time,
// for volumes whose working set does not fit the device (or a memory budget
// on it). Every result equals lt_measure's bit for bit:
//
//   1. x and y EDT passes, slab by slab of P planes: the mask goes up, the
//      y pass's output f comes back into the caller's host DT2 buffer.
//   2. z pass, y-slab by y-slab: all z of a band of rows (one 2D copy each
//      way, in place in the host buffer), which is now DT2; the largest DT2
//      of the volume is kept on the device.
//   3. local thickness and shape sums, core slab by core slab: a ball that
//      holds a voxel of the core has its centre within H = ceil(sqrt(max
//      DT2)) planes of it, so each core slab goes up with H + 1 planes on
//      either side (the extra plane for the containment test) and is
//      solved as a volume of its own: centres at its cut faces see fewer
//      neighbours and may be kept where the whole volume drops them, which
//      only paints true balls again, so the core's LT2 is exact. The
//      shape sums add the core planes (their neighbour planes are present
//      for the shell test); integer sums make the order irrelevant.
//   4. the formulas, once.
#include <cstddef>

#include "lt_internal.cuh"

namespace ltk {
namespace {

__global__ void max_kernel(const uint32_t* __restrict__ a, size_t n, uint32_t* __restrict__ out) {
  uint32_t m = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    m = max(m, a[i]);
#pragma unroll
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

Dims sub_dims(int nx, int ny, int nz) {
  Dims d;
  d.ndim = 3;
  d.nx = nx;
  d.ny = ny;
  d.nz = nz;
  d.n = (uint32_t)((size_t)nx * ny * nz);
  return d;
}

size_t acc_region(uint32_t n_labels) {
  // shape accumulators (as lt_shape_measures lays them out) + S and R
  return shape_workspace_bytes(n_labels) + 2 * align_up((size_t)n_labels * 4);
}

}  // namespace

// Region for a slab of P planes: phase 3 needs DT2, labels, LT2 and the
// local-thickness scratch (30 bytes per voxel); phases 1 and 2 fit in it.
size_t slabs_ws_bytes(uint32_t n_labels, int nx, int ny, int P) {
  const size_t n = (size_t)P * nx * ny;
  return sizeof(WsHeader) + acc_region(n_labels) + 3 * align_up(n * 4) + lt_workspace_bytes(sub_dims(nx, ny, P)) +
         4 * kAlign;
}

lt_status slabs_run(const uint8_t* mask_h, const uint32_t* labels_h, uint32_t n_labels, int nx, int ny, int nz,
                    int P, uint32_t* dt2_h, uint32_t* lt2_h, float* S_h, float* R_h, void* ws, size_t ws_bytes,
                    cudaStream_t s) {
  const size_t plane = (size_t)nx * ny;
  WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
  char* acc = reinterpret_cast<char*>(ws) + sizeof(WsHeader);
  float* S = reinterpret_cast<float*>(acc + shape_workspace_bytes(n_labels));
  float* R = S + align_up((size_t)n_labels * 4) / 4;
  char* region = acc + acc_region(n_labels);
  const size_t region_bytes = ws_bytes - (size_t)(region - reinterpret_cast<char*>(ws));
  auto ok = [](cudaError_t e) { return e == cudaSuccess; };
  if (!ok(cudaMemsetAsync(hdr, 0, sizeof(WsHeader), s)) || !ok(shape_clear(acc, n_labels, s))) return LT_ERR_CUDA;

  // 1. x and y passes per slab of P planes
  for (int z0 = 0; z0 < nz; z0 += P) {
    const int p = z0 + P <= nz ? P : nz - z0;
    const Dims d = sub_dims(nx, ny, p);
    char* q = region;
    uint8_t* mask = reinterpret_cast<uint8_t*>(q);
    q += align_up((size_t)d.n);
    uint32_t* f = reinterpret_cast<uint32_t*>(q);
    q += align_up((size_t)d.n * 4);
    if (!ok(cudaMemcpyAsync(mask, mask_h + (size_t)z0 * plane, (size_t)d.n, cudaMemcpyHostToDevice, s)) ||
        !ok(edt_launch(mask, f, d, q, s, Tuning(), 1)) ||
        !ok(cudaMemcpyAsync(dt2_h + (size_t)z0 * plane, f, (size_t)d.n * 4, cudaMemcpyDeviceToHost, s)))
      return LT_ERR_CUDA;
  }
  // 2. z pass per band of rows (all z), in place in dt2_h
  const size_t row_bytes = (size_t)nz * nx * (nz > 2048 ? 10 : 6);  // data + EDT scratch per row
  int ys = (int)std::min<size_t>((size_t)ny, (region_bytes - 4 * kAlign) / row_bytes);
  while (ys > 1 && (size_t)nz * nx * ys >= (1ull << 32)) --ys;
  if (ys < 1) return LT_ERR_WORKSPACE;
  for (int y0 = 0; y0 < ny; y0 += ys) {
    const int r = y0 + ys <= ny ? ys : ny - y0;
    const Dims d = sub_dims(nx, r, nz);
    uint32_t* f = reinterpret_cast<uint32_t*>(region);
    char* q = region + align_up((size_t)d.n * 4);
    const size_t w = (size_t)r * nx * 4;
    if (!ok(cudaMemcpy2DAsync(f, w, dt2_h + (size_t)y0 * nx, plane * 4, w, nz, cudaMemcpyHostToDevice, s)) ||
        !ok(edt_launch(nullptr, f, d, q, s, Tuning(), 2)))
      return LT_ERR_CUDA;
    max_kernel<<<(unsigned)sm_count() * 4, 256, 0, s>>>(f, d.n, &hdr->max_dt2);
    if (!ok(cudaGetLastError()) ||
        !ok(cudaMemcpy2DAsync(dt2_h + (size_t)y0 * nx, plane * 4, f, w, w, nz, cudaMemcpyDeviceToHost, s)))
      return LT_ERR_CUDA;
  }
  uint32_t maxd = 0;
  if (!ok(cudaMemcpyAsync(&maxd, &hdr->max_dt2, 4, cudaMemcpyDeviceToHost, s)) || !ok(cudaStreamSynchronize(s)))
    return LT_ERR_CUDA;
  int H = 0;
  while ((uint64_t)H * H < maxd) ++H;
  // 3. local thickness and shape sums per core slab, with H + 1 planes of halo
  const int core = P - 2 * (H + 1);
  if (core < 1) return LT_ERR_WORKSPACE;
  for (int z0 = 0; z0 < nz; z0 += core) {
    const int c = z0 + core <= nz ? core : nz - z0;
    const int e0 = z0 - (H + 1) > 0 ? z0 - (H + 1) : 0;
    const int e1 = z0 + c + H + 1 < nz ? z0 + c + H + 1 : nz;
    const Dims d = sub_dims(nx, ny, e1 - e0);
    char* q = region;
    uint32_t* dt2 = reinterpret_cast<uint32_t*>(q);
    q += align_up((size_t)d.n * 4);
    uint32_t* lab = reinterpret_cast<uint32_t*>(q);
    q += align_up((size_t)d.n * 4);
    uint32_t* lt2 = reinterpret_cast<uint32_t*>(q);
    q += align_up((size_t)d.n * 4);
    // per-slab painting counters start from zero; error bits and `touch` accumulate
    if (!ok(cudaMemcpyAsync(dt2, dt2_h + (size_t)e0 * plane, (size_t)d.n * 4, cudaMemcpyHostToDevice, s)) ||
        !ok(cudaMemcpyAsync(lab, labels_h + (size_t)e0 * plane, (size_t)d.n * 4, cudaMemcpyHostToDevice, s)) ||
        !ok(cudaMemsetAsync(&hdr->n_surv, 0, offsetof(WsHeader, n_updates) - offsetof(WsHeader, n_surv), s)) ||
        !ok(cudaMemsetAsync(&hdr->n_extra, 0, sizeof(uint32_t), s)) ||
        !ok(lt_launch(dt2, lab, lt2, d, hdr, q, s)) ||
        !ok(shape_accumulate(lab, lt2, n_labels, d, hdr, acc, z0 - e0, z0 - e0 + c, s)))
      return LT_ERR_CUDA;
    if (lt2_h && !ok(cudaMemcpyAsync(lt2_h + (size_t)z0 * plane, lt2 + (size_t)(z0 - e0) * plane,
                                     (size_t)c * plane * 4, cudaMemcpyDeviceToHost, s)))
      return LT_ERR_CUDA;
  }
  // 4. formulas
  if (!ok(shape_finalize(3, n_labels, acc, S, R, nullptr, s)) ||
      !ok(cudaMemcpyAsync(S_h, S, (size_t)n_labels * 4, cudaMemcpyDeviceToHost, s)) ||
      !ok(cudaMemcpyAsync(R_h, R, (size_t)n_labels * 4, cudaMemcpyDeviceToHost, s)))
    return LT_ERR_CUDA;
  return LT_OK;
}

}  // namespace ltk
