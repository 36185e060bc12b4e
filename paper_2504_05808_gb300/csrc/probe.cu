// Calibration probe: the rate of 32-bit atomic-max updates to global memory
// on this GPU, the ceiling the painting step of local thickness is compared
// against (painting is nothing but such updates).
//
// Pattern 0: the 32 lanes of a warp update the 32 words of one 128-byte line,
//            so each warp instruction is one line-sized request.
// Pattern 1: every lane updates one word of its own line, 32 lines per
//            instruction.
// Lines are chosen by an integer hash of (warp, iteration[, lane]) over the
// whole buffer.
#include "lt_internal.cuh"

namespace ltk {
namespace {

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

template <int PATTERN>
__global__ void __launch_bounds__(256) update_probe_kernel(uint32_t* __restrict__ buf, uint32_t line_mask,
                                                           uint32_t iters) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (uint32_t i = 0; i < iters; ++i) {
    const uint32_t key = warp * iters + i;
    const uint32_t line = (PATTERN == 0 ? mix32(key) : mix32(key * 32u + lane)) & line_mask;
    atomicMax(buf + (size_t)line * 32u + lane, i + 1u);
  }
}

constexpr uint32_t kProbeIters = 256;
constexpr int kProbeBlocksPerSm = 8;

}  // namespace
}  // namespace ltk

using namespace ltk;

extern "C" lt_status lt_probe_update_rate(uint32_t* buf, size_t words, int pattern, int reps, void* stream,
                                          double* rate) {
  if (!rate || reps < 1 || (pattern != 0 && pattern != 1)) return LT_ERR_INVALID_ARG;
  if (words < (1u << 20) || (words & (words - 1)) != 0 || words > (1ull << 36)) return LT_ERR_INVALID_ARG;
  lt_status st = device_ptr_ok(buf);
  if (st != LT_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const uint32_t line_mask = (uint32_t)(words / 32 - 1);
  const unsigned blocks = (unsigned)(sm_count() * kProbeBlocksPerSm);
  auto launch = [&]() {
    if (pattern == 0)
      update_probe_kernel<0><<<blocks, 256, 0, s>>>(buf, line_mask, kProbeIters);
    else
      update_probe_kernel<1><<<blocks, 256, 0, s>>>(buf, line_mask, kProbeIters);
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return LT_ERR_CUDA;
  }
  launch();
  cudaEventRecord(e0, s);
  for (int r = 0; r < reps; ++r) launch();
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || ms <= 0.f) return LT_ERR_CUDA;
  const double updates = (double)blocks * 256.0 * kProbeIters * reps;
  *rate = updates / (ms * 1e-3);
  return LT_OK;
}
