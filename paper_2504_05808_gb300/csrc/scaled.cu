// Scaled local thickness: the reduced-resolution option of the fast
// local-thickness work the paper builds on (Sec. 1, Sec. 4): exact LT on the
// volume sampled every s voxels, brought back to full resolution.
//
//   sample:   low-res voxel B takes mask and label of the full-res voxel
//             c(B) = min(s*B + s/2, n - 1) per axis (the block's centre).
//   exact:    DT2 and LT2 of the low-res volume (the kernels of edt.cu and
//             lt.cu, unchanged).
//   upsample: an object voxel x of label l in block B = x / s gets
//             s^2 * LT2_low(B) when B carries label l; otherwise the largest
//             s^2 * LT2_low over the (up to 27) blocks B + d, |d|_inf <= 1,
//             that carry l; otherwise 1 (every object voxel has LT2 >= 1).
//             Voxels of no object get 0.
// Every step is integer arithmetic, so the result is exact for this
// definition (the oracle's lt2_scaled); its distance to the exact LT is the
// price of the speed-up, measured by the scaled-LT protocol of bench.py.
#include "lt_internal.cuh"

namespace ltk {
namespace {

__global__ void sample_kernel(const uint8_t* __restrict__ mask, const uint32_t* __restrict__ labels, Dims d,
                              int s, uint8_t* __restrict__ mask_low, uint32_t* __restrict__ labels_low,
                              Dims dl) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= dl.n) return;
  const uint32_t X = i % (uint32_t)dl.nx, t = i / (uint32_t)dl.nx;
  const uint32_t Y = t % (uint32_t)dl.ny, Z = t / (uint32_t)dl.ny;
  const uint32_t h = (uint32_t)s / 2;
  const uint32_t x = min(X * s + h, (uint32_t)d.nx - 1), y = min(Y * s + h, (uint32_t)d.ny - 1),
                 z = min(Z * s + h, (uint32_t)d.nz - 1);
  const size_t v = ((size_t)z * d.ny + y) * d.nx + x;
  mask_low[i] = mask[v];
  labels_low[i] = labels[v];
}

__global__ void upsample_kernel(const uint32_t* __restrict__ labels, Dims d, int s,
                                const uint32_t* __restrict__ labels_low, const uint32_t* __restrict__ lt2_low,
                                Dims dl, uint32_t* __restrict__ lt2) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  const uint32_t l = labels[i];
  uint32_t out = 0;
  if (l) {
    const uint32_t x = (uint32_t)(i % (uint32_t)d.nx), t = (uint32_t)(i / (uint32_t)d.nx);
    const uint32_t y = t % (uint32_t)d.ny, z = t / (uint32_t)d.ny;
    const int X = (int)(x / s), Y = (int)(y / s), Z = (int)(z / s);
    const uint32_t b = ((uint32_t)Z * dl.ny + Y) * dl.nx + X;
    const uint32_t s2 = (uint32_t)(s * s);
    if (labels_low[b] == l) {
      out = s2 * lt2_low[b];
    } else {
      uint32_t best = 0;
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            const int bx = X + dx, by = Y + dy, bz = Z + dz;
            if (bx < 0 || bx >= dl.nx || by < 0 || by >= dl.ny || bz < 0 || bz >= dl.nz) continue;
            const uint32_t q = ((uint32_t)bz * dl.ny + by) * dl.nx + bx;
            if (labels_low[q] == l) best = max(best, lt2_low[q]);
          }
      out = best ? s2 * best : 1u;
    }
  }
  lt2[i] = out;
}

}  // namespace

Dims scaled_dims(const Dims& d, int s) {
  Dims dl;
  dl.ndim = d.ndim;
  dl.nx = (d.nx + s - 1) / s;
  dl.ny = (d.ny + s - 1) / s;
  dl.nz = d.ndim == 3 ? (d.nz + s - 1) / s : 1;
  dl.n = (uint32_t)dl.nx * (uint32_t)dl.ny * (uint32_t)dl.nz;
  return dl;
}

// Workspace after the header: low-res mask, labels, DT2, LT2, then the
// low-res EDT / local-thickness scratch. The header is shared with the
// low-res pass (its counters and device-detected errors).
size_t scaled_body_bytes(const Dims& d, int s) {
  const Dims dl = scaled_dims(d, s);
  const size_t b = align_up(dl.n) + 3 * align_up((size_t)dl.n * 4);
  const size_t l = lt_workspace_bytes(dl), e = edt_workspace_bytes(dl);
  return b + (l > e ? l : e);
}

cudaError_t scaled_launch(const uint8_t* mask, const uint32_t* labels, const Dims& d, int s, WsHeader* hdr,
                          void* body, uint32_t* lt2, cudaStream_t st) {
  const Dims dl = scaled_dims(d, s);
  char* p = reinterpret_cast<char*>(body);
  uint8_t* mask_low = reinterpret_cast<uint8_t*>(p);
  p += align_up(dl.n);
  uint32_t* labels_low = reinterpret_cast<uint32_t*>(p);
  p += align_up((size_t)dl.n * 4);
  uint32_t* dt2_low = reinterpret_cast<uint32_t*>(p);
  p += align_up((size_t)dl.n * 4);
  uint32_t* lt2_low = reinterpret_cast<uint32_t*>(p);
  p += align_up((size_t)dl.n * 4);
  void* inner_body = p;
  {
    TraceScope t("scaled_sample", st);
    sample_kernel<<<(dl.n + 255) / 256, 256, 0, st>>>(mask, labels, d, s, mask_low, labels_low, dl);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = edt_launch(mask_low, dt2_low, dl, inner_body, st);
  if (e == cudaSuccess) e = lt_launch(dt2_low, labels_low, lt2_low, dl, hdr, inner_body, st);
  if (e != cudaSuccess) return e;
  {
    TraceScope t("scaled_upsample", st);
    upsample_kernel<<<(unsigned)((d.n + 255) / 256), 256, 0, st>>>(labels, d, s, labels_low, lt2_low, dl, lt2);
  }
  return cudaGetLastError();
}

}  // namespace ltk
