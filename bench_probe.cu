// Calibration probe for the benchmark (not part of the library): the rate of
// 32-bit atomic-max updates to global memory on this GPU, the ceiling the
// painting step of local thickness is compared against (painting is nothing
// but such updates). Built by __graft_entry__.build() into _bench_probe.so,
// loaded by bench.py only.
//
// Pattern 0: the 32 lanes of a warp update the 32 words of one 128-byte line,
//            so each warp instruction is one line-sized request.
// Pattern 1: every lane updates one word of its own line, 32 lines per
//            instruction.
// Lines are chosen by an integer hash of (warp, iteration[, lane]) over the
// whole buffer.
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace {

// 32-bit integer mixer ("lowbias32" from C. Wellons' hash-prospector, a
// public-domain xorshift-multiply hash).

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

// Updates per second written to *rate; returns 0 on success, 1 for bad
// arguments (buf not device memory of the current device, words not a power
// of two >= 2^20), 2 for a CUDA error. Synchronous.
extern "C" int probe_update_rate(uint32_t* buf, size_t words, int pattern, int reps, void* stream, double* rate) {
  if (!rate || !buf || reps < 1 || (pattern != 0 && pattern != 1)) return 1;
  if (words < (1u << 20) || (words & (words - 1)) != 0 || words > (1ull << 36)) return 1;
  cudaPointerAttributes a;
  int cur = -1;
  if (cudaPointerGetAttributes(&a, buf) != cudaSuccess || a.type != cudaMemoryTypeDevice ||
      cudaGetDevice(&cur) != cudaSuccess || a.device != cur) {
    cudaGetLastError();
    return 1;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cur) != cudaSuccess) return 2;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const uint32_t line_mask = (uint32_t)(words / 32 - 1);
  const unsigned blocks = (unsigned)(sms * kProbeBlocksPerSm);
  auto launch = [&]() {
    if (pattern == 0)
      update_probe_kernel<0><<<blocks, 256, 0, s>>>(buf, line_mask, kProbeIters);
    else
      update_probe_kernel<1><<<blocks, 256, 0, s>>>(buf, line_mask, kProbeIters);
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return 2;
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
  if (e != cudaSuccess || ms <= 0.f) return 2;
  const double updates = (double)blocks * 256.0 * kProbeIters * reps;
  *rate = updates / (ms * 1e-3);
  return 0;
}
