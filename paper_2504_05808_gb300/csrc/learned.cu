// Learned sphericity correction on sm_103a: per-object features, a
// 48-64-64-1 ReLU network with BF16 weights and activations and FP32
// accumulation, its inference, gradients and Adam update. The paper has no
// learned component; the network corrects the spheroid sphericity S_LT
// (Sec. 4.1) toward the strict mesh sphericity of Eq. 1.
//
// Features of an object (V voxels, n_s shell voxels, M = sqrt(max LT2),
// mean LT m), index: value
//   0: log(V)/10   1: log(n_s)/10   2: log(M)/4   3: m/M   4: R_LT   5: S_LT
//   6-21: fraction of interior (non-shell) voxels with LT/M in bin b,
//   22-37: the same over the shell voxels, 38-47: 0.
// Bin b of a voxel: the largest b in 0..15 with b^2 * maxLT2 <= 256 * LT2
// (decided in integers).
//
// Network (parameters in one FP32 vector, layout W1[48][64], b1[64],
// W2[64][64], b2[64], w3[64], b3): x = bf16(features); h1 =
// bf16(relu(x W1q + b1)); h2 = bf16(relu(h1 W2q + b2)); out = h2 . w3q + b3,
// with Wq = bf16(W); sums in FP32. Corrected sphericity: clamp(S_LT + out,
// 0, 1). Training minimises the mean of (S_LT + out - target)^2 over a batch;
// gradients pass straight through the BF16 roundings.
#include <cuda_bf16.h>

#include "lt_internal.cuh"

namespace ltk {
namespace {

constexpr int kF = LT_MLP_FEATURES, kH = LT_MLP_HIDDEN;
constexpr int kOffB1 = kF * kH, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH, kOffW3 = kOffB2 + kH,
              kOffB3 = kOffW3 + kH;
static_assert(kOffB3 + 1 == LT_MLP_PARAMS, "parameter layout");

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// ---------------------------------------------------------------- features
// One thread per voxel: labelled voxels add 1 to hist[label][bin] (interior)
// or hist[label][16 + bin] (shell); equal keys within a warp are combined.
template <int NDIM>
__global__ void __launch_bounds__(256) features_hist_kernel(const uint32_t* __restrict__ labels,
                                                            const uint32_t* __restrict__ lt2, Dims d,
                                                            uint32_t n_labels,
                                                            const uint32_t* __restrict__ max_lt2,
                                                            uint32_t* __restrict__ hist) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  const bool in = x < d.nx;
  const size_t sy = (size_t)d.nx, sz = (size_t)d.nx * d.ny;
  const size_t v = in ? (size_t)z * sz + (size_t)y * sy + x : 0;
  const uint32_t l = in ? labels[v] : 0u;
  if (__ballot_sync(0xffffffffu, l != 0 && l < n_labels) == 0) return;
  uint32_t key = 0xffffffffu;
  if (l != 0 && l < n_labels) {
    const bool s = x == 0 || labels[v - 1] != l || x == d.nx - 1 || labels[v + 1] != l || y == 0 ||
                   labels[v - sy] != l || y == d.ny - 1 || labels[v + sy] != l ||
                   (NDIM == 3 && (z == 0 || labels[v - sz] != l || z == d.nz - 1 || labels[v + sz] != l));
    const unsigned long long t = 256ull * lt2[v], mx = max_lt2[l];
    uint32_t b = 0;
    for (uint32_t k = 1; k < 16; ++k)
      if ((unsigned long long)(k * k) * mx <= t) b = k;
    key = l * 32u + (s ? 16u : 0u) + b;
  }
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int lane = threadIdx.x & 31;
  if (key != 0xffffffffu && lane == __ffs(peers) - 1) atomicAdd(hist + key, (uint32_t)__popc(peers));
}

// Bin of LT2 t in an object with largest LT2 mx (t <= mx): the largest b in
// 0..15 with b^2 mx <= 256 t, from a float estimate fixed in integers.
__device__ __forceinline__ uint32_t lt_bin(uint32_t t, uint32_t mx) {
  int b = min(15, (int)(16.0f * sqrtf((float)t / (float)max(mx, 1u))));
  const unsigned long long T = 256ull * t, M = mx;
  while (b < 15 && (unsigned long long)((b + 1) * (b + 1)) * M <= T) ++b;
  while (b > 0 && (unsigned long long)(b * b) * M > T) --b;
  return (uint32_t)b;
}

// Vector form for nx % 4 == 0: a thread bins 4 consecutive voxels of a row
// (16-byte loads of labels, LT2 and the neighbouring rows); equal keys
// (label, shell, bin) of consecutive voxels are counted together, and runs of
// equal first keys across the warp are combined by a segmented scan so that
// one lane per run issues the atomic.
__device__ __forceinline__ uint32_t c4(const uint4& v, int k) {
  return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

template <int NDIM>
__global__ void __launch_bounds__(256) features_hist4_kernel(const uint32_t* __restrict__ labels,
                                                             const uint32_t* __restrict__ lt2, Dims d,
                                                             uint32_t n_labels,
                                                             const uint32_t* __restrict__ max_lt2,
                                                             uint32_t* __restrict__ hist) {
  const int lane = threadIdx.x & 31;
  const int x0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
  const bool in = x0 < d.nx && y < d.ny;
  const size_t sy = (size_t)d.nx, sz = (size_t)d.nx * d.ny;
  const size_t v = in ? (size_t)z * sz + (size_t)y * sy + x0 : 0;
  uint4 L = make_uint4(0u, 0u, 0u, 0u);
  if (in) L = *reinterpret_cast<const uint4*>(labels + v);
  const bool any = (L.x | L.y | L.z | L.w) != 0u;
  if (__ballot_sync(0xffffffffu, any) == 0) return;  // uniform per warp
  uint32_t key = 0xffffffffu, cnt = 0;  // this thread's first key and its count
  if (any) {
    const uint4 T = *reinterpret_cast<const uint4*>(lt2 + v);
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    const uint4 Ym = y > 0 ? *reinterpret_cast<const uint4*>(labels + v - sy) : zero;
    const uint4 Yp = y + 1 < d.ny ? *reinterpret_cast<const uint4*>(labels + v + sy) : zero;
    uint4 Zm = zero, Zp = zero;
    if (NDIM == 3) {
      if (z > 0) Zm = *reinterpret_cast<const uint4*>(labels + v - sz);
      if (z + 1 < d.nz) Zp = *reinterpret_cast<const uint4*>(labels + v + sz);
    }
    const uint32_t xl = x0 > 0 ? labels[v - 1] : 0u;
    const uint32_t xr = x0 + 4 < d.nx ? labels[v + 4] : 0u;
    uint32_t prev = 0xffffffffu, run = 0, lm = 0, mx = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t l = c4(L, k);
      uint32_t kk = 0xffffffffu;
      if (l != 0 && l < n_labels) {
        const uint32_t left = k == 0 ? xl : c4(L, k - 1), right = k == 3 ? xr : c4(L, k + 1);
        bool s = left != l || right != l || c4(Ym, k) != l || c4(Yp, k) != l;
        if (NDIM == 3) s = s || c4(Zm, k) != l || c4(Zp, k) != l;
        if (l != lm) {
          lm = l;
          mx = max_lt2[l];
        }
        kk = l * 32u + (s ? 16u : 0u) + lt_bin(c4(T, k), mx);
      }
      if (kk != prev) {  // close the previous run
        if (prev != 0xffffffffu) {
          if (key == 0xffffffffu) {
            key = prev;
            cnt = run;
          } else {
            atomicAdd(hist + prev, run);
          }
        }
        prev = kk;
        run = 0;
      }
      ++run;
    }
    if (prev != 0xffffffffu) {
      if (key == 0xffffffffu) {
        key = prev;
        cnt = run;
      } else if (prev == key) {
        cnt += run;
      } else {
        atomicAdd(hist + prev, run);
      }
    }
  }
  // segmented inclusive scan of the counts over runs of equal keys
  const uint32_t kprev = __shfl_up_sync(0xffffffffu, key, 1);
  int seg = (lane == 0 || kprev != key) ? lane : 0;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, seg, o);
    if (lane >= o) seg = max(seg, t);
  }
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t a = __shfl_up_sync(0xffffffffu, cnt, o);
    if (lane - o >= seg) cnt += a;
  }
  const uint32_t knext = __shfl_down_sync(0xffffffffu, key, 1);
  if (key != 0xffffffffu && (lane == 31 || knext != key)) atomicAdd(hist + key, cnt);
}

// One thread per (label, feature index), so that consecutive threads write
// consecutive floats of the [n_labels][48] matrix.
__global__ void __launch_bounds__(256) features_final_kernel(uint32_t n_labels, lt_object_stats st,
                                                             const float* __restrict__ S,
                                                             const float* __restrict__ R,
                                                             const uint32_t* __restrict__ hist,
                                                             float* __restrict__ F) {
  const size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (size_t)n_labels * kF) return;
  const uint32_t l = (uint32_t)(g / kF);
  const int i = (int)(g % kF);
  const uint32_t V = l ? st.volume[l] : 0u;
  float f = 0.0f;
  // FP32 throughout (FP64 is slow on this GPU): each value within ~3e-7
  // relative of its exact value
  if (V != 0 && i < 38) {
    const uint32_t ns = st.n_shell[l];
    if (i == 0) {
      f = logf((float)V) / 10.0f;
    } else if (i == 1) {
      f = logf((float)ns) / 10.0f;
    } else if (i == 2) {
      f = 0.5f * logf((float)st.max_lt2[l]) / 4.0f;
    } else if (i == 3) {
      f = (float)st.sum_lt[l] * (1.0f / 1048576.0f) / (float)V / sqrtf((float)st.max_lt2[l]);
    } else if (i == 4) {
      f = R[l];
    } else if (i == 5) {
      f = S[l];
    } else if (i < 22) {
      f = (float)hist[(size_t)l * 32 + (i - 6)] / (float)max(1u, V - ns);
    } else {
      f = (float)hist[(size_t)l * 32 + 16 + (i - 22)] / (float)max(1u, ns);
    }
  }
  F[g] = f;
}

}  // namespace

cudaError_t features_final_launch(uint32_t n_labels, const lt_object_stats& st, const float* S, const float* R,
                                  const uint32_t* hist, float* F, cudaStream_t s) {
  const size_t n = (size_t)n_labels * kF;
  {
    TraceScope t("features_final", s);
    features_final_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n_labels, st, S, R, hist, F);
  }
  return cudaGetLastError();
}

namespace {

// --------------------------------------------------------------- network
// BF16-rounded weights staged in shared memory as floats.
struct SmemNet {
  float W1[kF * kH], b1[kH], W2[kH * kH], b2[kH], w3[kH], b3;
};

__device__ void stage_net(const float* __restrict__ p, SmemNet& n) {
  for (int i = threadIdx.x; i < kF * kH; i += blockDim.x) n.W1[i] = bf(p[i]);
  for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) n.W2[i] = bf(p[kOffW2 + i]);
  for (int i = threadIdx.x; i < kH; i += blockDim.x) {
    n.b1[i] = p[kOffB1 + i];
    n.b2[i] = p[kOffB2 + i];
    n.w3[i] = bf(p[kOffW3 + i]);
  }
  if (threadIdx.x == 0) n.b3 = p[kOffB3];
}

// Forward pass of one feature row; fills x, pre1, h1, pre2, h2 when given.
__device__ float net_forward(const SmemNet& n, const float* __restrict__ frow, float* x, float* pre1,
                             float* h1, float* pre2, float* h2) {
  float xv[kF];
#pragma unroll
  for (int i = 0; i < kF; ++i) xv[i] = bf(frow[i]);
  float a1[kH];
#pragma unroll 4
  for (int j = 0; j < kH; ++j) {
    float acc = n.b1[j];
#pragma unroll
    for (int i = 0; i < kF; ++i) acc = fmaf(xv[i], n.W1[i * kH + j], acc);
    if (pre1) pre1[j] = acc;
    a1[j] = bf(fmaxf(acc, 0.0f));
  }
  float out = n.b3;
#pragma unroll 4
  for (int j = 0; j < kH; ++j) {
    float acc = n.b2[j];
#pragma unroll
    for (int i = 0; i < kH; ++i) acc = fmaf(a1[i], n.W2[i * kH + j], acc);
    if (pre2) pre2[j] = acc;
    const float h = bf(fmaxf(acc, 0.0f));
    if (h2) h2[j] = h;
    out = fmaf(h, n.w3[j], out);
  }
  if (x)
    for (int i = 0; i < kF; ++i) x[i] = xv[i];
  if (h1)
    for (int j = 0; j < kH; ++j) h1[j] = a1[j];
  return out;
}

__global__ void __launch_bounds__(128) mlp_infer_kernel(const float* __restrict__ params,
                                                        const float* __restrict__ F,
                                                        const float* __restrict__ S, uint32_t n,
                                                        float* __restrict__ out) {
  __shared__ SmemNet net;
  stage_net(params, net);
  __syncthreads();
  for (uint32_t o = blockIdx.x * blockDim.x + threadIdx.x; o < n; o += gridDim.x * blockDim.x) {
    const float s = S[o];
    if (isnan(s)) {
      out[o] = s;
      continue;
    }
    const float corr = net_forward(net, F + (size_t)o * kF, nullptr, nullptr, nullptr, nullptr, nullptr);
    out[o] = fminf(fmaxf(s + corr, 0.0f), 1.0f);
  }
}

// Per-sample forward and backward vectors of a batch. Scratch per sample
// (kSampleStride floats): x[48], h1[64], h2[64], g1[64] (d loss / d pre1),
// g2[64] (d loss / d pre2), g_out, 3 unused.
constexpr int kSampleStride = kF + 4 * kH + 4;

__global__ void __launch_bounds__(128) mlp_backprop_kernel(const float* __restrict__ params,
                                                           const float* __restrict__ F,
                                                           const float* __restrict__ S,
                                                           const float* __restrict__ target,
                                                           const uint32_t* __restrict__ idx,
                                                           uint32_t batch, float* __restrict__ scratch,
                                                           float* __restrict__ sq) {
  __shared__ SmemNet net;
  stage_net(params, net);
  __syncthreads();
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const uint32_t o = idx[b];
  float* sc = scratch + (size_t)b * kSampleStride;
  float* x = sc;
  float* h1 = x + kF;
  float* h2 = h1 + kH;
  float* g1 = h2 + kH;
  float* g2 = g1 + kH;
  float pre1[kH], pre2[kH];
  const float out = net_forward(net, F + (size_t)o * kF, x, pre1, h1, pre2, h2);
  const float r = S[o] + out - target[o];
  const float g_out = 2.0f * r / (float)batch;
  sq[b] = r * r;
  g2[kH] = g_out;  // the slot after g2 (offset kF + 4 kH of the sample)
#pragma unroll 4
  for (int j = 0; j < kH; ++j) g2[j] = pre2[j] > 0.0f ? g_out * net.w3[j] : 0.0f;
#pragma unroll 4
  for (int i = 0; i < kH; ++i) {
    float acc = 0.0f;
#pragma unroll
    for (int j = 0; j < kH; ++j) acc = fmaf(g2[j], net.W2[i * kH + j], acc);
    g1[i] = pre1[i] > 0.0f ? acc : 0.0f;
  }
}

// One thread per parameter: its gradient summed over the batch in a fixed
// order (deterministic); thread LT_MLP_PARAMS sums the loss.
__global__ void __launch_bounds__(256) mlp_grad_kernel(const float* __restrict__ scratch, uint32_t batch,
                                                       const float* __restrict__ sq,
                                                       float* __restrict__ grad, float* __restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > LT_MLP_PARAMS) return;
  if (p == LT_MLP_PARAMS) {
    if (loss) {
      float acc = 0.0f;
      for (uint32_t b = 0; b < batch; ++b) acc += sq[b];
      *loss = acc / (float)batch;
    }
    return;
  }
  float acc = 0.0f;
  for (uint32_t b = 0; b < batch; ++b) {
    const float* sc = scratch + (size_t)b * kSampleStride;
    const float* x = sc;
    const float* h1 = x + kF;
    const float* h2 = h1 + kH;
    const float* g1 = h2 + kH;
    const float* g2 = g1 + kH;
    const float g_out = g2[kH];
    float t;
    if (p < kOffB1) t = x[p / kH] * g1[p % kH];
    else if (p < kOffW2) t = g1[p - kOffB1];
    else if (p < kOffB2) t = h1[(p - kOffW2) / kH] * g2[(p - kOffW2) % kH];
    else if (p < kOffW3) t = g2[p - kOffB2];
    else if (p < kOffB3) t = h2[p - kOffW3] * g_out;
    else t = g_out;
    acc += t;
  }
  grad[p] = acc;
}

__global__ void mlp_adam_kernel(float* __restrict__ params, float* __restrict__ m, float* __restrict__ v,
                                const float* __restrict__ grad, float lr, float bc1, float bc2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= LT_MLP_PARAMS) return;
  const float g = grad[p];
  const float mm = 0.9f * m[p] + 0.1f * g;
  const float vv = 0.999f * v[p] + 0.001f * g * g;
  m[p] = mm;
  v[p] = vv;
  params[p] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + 1e-8f);
}

}  // namespace

size_t features_workspace_bytes(uint32_t n_labels) { return align_up((size_t)n_labels * 32 * 4); }

cudaError_t features_hist_launch(const uint32_t* labels, const uint32_t* lt2, uint32_t n_labels, const Dims& d,
                                 const uint32_t* max_lt2, uint32_t* hist, cudaStream_t s) {
  TraceScope t("features_hist", s);
  if (d.nx % 4 == 0) {
    // 64 threads (256 voxels) per row, 4 rows per CTA
    dim3 block(64, 4), grid((d.nx / 4 + 63) / 64, (d.ny + 3) / 4, d.nz);
    if (d.ndim == 3)
      features_hist4_kernel<3><<<grid, block, 0, s>>>(labels, lt2, d, n_labels, max_lt2, hist);
    else
      features_hist4_kernel<2><<<grid, block, 0, s>>>(labels, lt2, d, n_labels, max_lt2, hist);
  } else {
    dim3 grid((d.nx + 255) / 256, d.ny, d.nz);
    if (d.ndim == 3)
      features_hist_kernel<3><<<grid, 256, 0, s>>>(labels, lt2, d, n_labels, max_lt2, hist);
    else
      features_hist_kernel<2><<<grid, 256, 0, s>>>(labels, lt2, d, n_labels, max_lt2, hist);
  }
  return cudaGetLastError();
}

cudaError_t features_launch(const uint32_t* labels, const uint32_t* lt2, uint32_t n_labels, const Dims& d,
                            const lt_object_stats& st, const float* S, const float* R, void* body, float* F,
                            cudaStream_t s) {
  uint32_t* hist = reinterpret_cast<uint32_t*>(body);
  cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)n_labels * 32 * 4, s);
  if (e == cudaSuccess) e = features_hist_launch(labels, lt2, n_labels, d, st.max_lt2, hist, s);
  if (e != cudaSuccess) return e;
  return features_final_launch(n_labels, st, S, R, hist, F, s);
}

cudaError_t mlp_infer_launch(const float* params, const float* F, const float* S, uint32_t n, float* out,
                             cudaStream_t s) {
  const unsigned blocks = (unsigned)std::min<size_t>((n + 127) / 128, (size_t)sm_count() * 8);
  {
    TraceScope t("mlp_infer", s);
    mlp_infer_kernel<<<blocks ? blocks : 1, 128, 0, s>>>(params, F, S, n, out);
  }
  return cudaGetLastError();
}

size_t mlp_train_workspace_bytes(uint32_t batch) {
  return align_up((size_t)batch * kSampleStride * 4) + align_up((size_t)batch * 4);
}

cudaError_t mlp_grad_launch(const float* params, const float* F, const float* S, const float* target,
                            const uint32_t* idx, uint32_t batch, void* ws, float* grad, float* loss,
                            cudaStream_t s) {
  float* scratch = reinterpret_cast<float*>(ws);
  float* sq = reinterpret_cast<float*>(reinterpret_cast<char*>(ws) + align_up((size_t)batch * kSampleStride * 4));
  {
    TraceScope t("mlp_backprop", s);
    mlp_backprop_kernel<<<(batch + 127) / 128, 128, 0, s>>>(params, F, S, target, idx, batch, scratch, sq);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  {
    TraceScope t("mlp_grad", s);
    mlp_grad_kernel<<<(LT_MLP_PARAMS + 1 + 255) / 256, 256, 0, s>>>(scratch, batch, sq, grad, loss);
  }
  return cudaGetLastError();
}

cudaError_t mlp_adam_launch(float* params, float* m, float* v, const float* grad, uint32_t step, float lr,
                            cudaStream_t s) {
  const float bc1 = 1.0f - powf(0.9f, (float)step), bc2 = 1.0f - powf(0.999f, (float)step);
  {
    TraceScope t("mlp_adam", s);
    mlp_adam_kernel<<<(LT_MLP_PARAMS + 255) / 256, 256, 0, s>>>(params, m, v, grad, lr, bc1, bc2);
  }
  return cudaGetLastError();
}

}  // namespace ltk
