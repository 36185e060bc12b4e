// Internal declarations shared by the CUDA translation units of the library.
#pragma once

#include <cstddef>
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "lt.h"

namespace ltk {

// Array shape. nx, ny, nz <= 8192 and n = nx * ny * nz < 2^32.
struct Dims {
  int ndim;
  int nx, ny, nz;
  uint32_t n;
};

// First 256 bytes of every workspace.
struct WsHeader {
  uint32_t error;   // bit set of ERR_* found on the device
  uint32_t touch;   // nonzero: two face-adjacent foreground voxels differ in label
  uint32_t n_surv;  // kept centres painted in shared chunks (list from the front)
  uint32_t n_big;   // kept centres painted by one warp each (list from the back)
  uint32_t ctr_small, ctr_big;  // work counters of the paint kernel
  unsigned long long n_updates;        // LT2 updates (atomic max) the paint kernel issued
  unsigned long long n_table_updates;  // of which from crescent tables
  uint32_t max_dt2;                    // slab pipeline: largest DT2 of the volume
  uint32_t n_extra;                    // extra part records of shared row-mode centres
  uint32_t reserved[52];
};
static_assert(sizeof(WsHeader) == 256, "header is 256 bytes");

enum : uint32_t { ERR_LABEL_RANGE = 1u, ERR_LABEL_OUTSIDE_MASK = 2u, ERR_TIMEOUT = 4u };

constexpr size_t kAlign = 256;
__host__ __device__ constexpr size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Floor square root of v < 2^24: IEEE-rounded single-precision square root
// of an exactly representable integer is within one of the floor; fix it.
__device__ __forceinline__ uint32_t isqrt24(uint32_t v) {
  uint32_t r = (uint32_t)sqrtf((float)v);
  if (r * r > v) --r;
  else if ((r + 1) * (r + 1) <= v) ++r;
  return r;
}

// Per-object accumulators (structure of arrays in the workspace).
struct ShapeAcc {
  uint32_t* volume;
  uint32_t* n_shell;
  uint32_t* max_lt2;
  unsigned long long* sum_lt;
  unsigned long long* sum_shell_lt;
};

// ---- stage-major batches: one launch of a stage covers many volumes ----
// Per volume, its parameters in device memory; per stage, the first CTA of
// every volume in the launch's one-dimensional grid and the volume's own
// grid extents, so that a CTA finds its volume by binary search and its
// block coordinates within that volume's grid.
constexpr int kMaxBatchVols = 256;
struct VolParams {
  Dims d;
  uint32_t n_labels;
  const uint8_t* mask;
  const uint32_t* labels;
  uint32_t* dt2;
  uint32_t* lt2;
  float* S;
  float* R;
  WsHeader* hdr;        // the volume's workspace header
  char* body;           // and the scratch after it
  const void* map_dt2;  // TMA tensor maps (CUtensorMap, global memory), null without TMA
  const void* map_lab;
};
struct StagePlan {
  uint32_t start[kMaxBatchVols + 1];  // first CTA of volume v; start[n] = the launch's CTAs
  uint32_t gx[kMaxBatchVols], gy[kMaxBatchVols];
};
struct MultiArgs {
  const VolParams* vols;
  const StagePlan* plan;
  int nvol;
};
// The volume of CTA b and its block coordinates within that volume's grid.
__device__ __forceinline__ int find_volume(const MultiArgs& m, uint32_t b, uint3& blk) {
  int lo = 0, hi = m.nvol;  // start[lo] <= b < start[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(&m.plan->start[mid]) <= b) lo = mid;
    else hi = mid;
  }
  const uint32_t local = b - __ldg(&m.plan->start[lo]);
  const uint32_t gx = __ldg(&m.plan->gx[lo]), gy = __ldg(&m.plan->gy[lo]);
  blk = make_uint3(local % gx, local / gx % gy, local / (gx * gy));
  return lo;
}

// Launch parameters the batch autotuner may change (defaults: single calls).
// Defaults: the autotuner's choice for the 512^3 particle volume on GB300.
struct Tuning {
  int edt_tx_y = 8;             // EDT column-tile width of the y pass for axes <= 512 (32, 16 or 8)
  int edt_tx_z = 32;            // and of the z pass (32: whole 128-byte tile rows, 512 threads)
  int ridge_z = 32;             // z planes per ridge CTA (8, 16 or 32)
  int paint_blocks_per_sm = 6;  // persistent paint grid, CTAs per SM
  int chunk_cres = 64;          // largest crescent painted in shared chunks (bigger: a warp each)
};

// ---- host launchers (each returns cudaSuccess or the launch error) ----
// edt.cu
size_t edt_workspace_bytes(const Dims& d);
cudaError_t edt_prepare_device();  // kernel attributes; call before capture
// passes: 1 = x and y, 2 = z (on dt2 in place), 3 = all
cudaError_t edt_launch(const uint8_t* mask, uint32_t* dt2, const Dims& d, void* ws, cudaStream_t s,
                       const Tuning& tu = Tuning(), int passes = 3);
// batched EDT passes (pass 0 rows, 1 y columns, 2 z columns; tx 0 = the
// global-memory y pass of long 2D columns)
int edt_multi_tx(int max_L, int tx_small);
dim3 edt_multi_grid(const Dims& d, int pass, int tx);
cudaError_t edt_multi_launch(const MultiArgs& m, uint32_t blocks, int pass, int tx, int max_L, cudaStream_t s);
// lt.cu
size_t lt_workspace_bytes(const Dims& d);
cudaError_t lt_launch(const uint32_t* dt2, const uint32_t* labels, uint32_t* lt2, const Dims& d,
                      WsHeader* hdr, void* body, cudaStream_t s, const Tuning& tu = Tuning());
// the two stages of lt_launch: the ridge pass over planes [z_lo, z_hi)
// (z_lo a multiple of ridge_chunk(tu); its planes and the one on either side
// must hold final DT2 and labels), then the painting of every kept centre
int ridge_chunk(const Tuning& tu);
// max_dt2 (n_labels entries, may be null): raised (atomic max) to the
// largest DT2 of each object's voxels in the planes processed
cudaError_t lt_ridge_launch(const uint32_t* dt2, const uint32_t* labels, uint32_t* lt2, const Dims& d,
                            WsHeader* hdr, void* body, cudaStream_t s, const Tuning& tu, int z_lo, int z_hi,
                            uint32_t* max_dt2 = nullptr, uint32_t n_labels = 0);
cudaError_t lt_paint_launch(const uint32_t* dt2, const uint32_t* labels, uint32_t* lt2, const Dims& d,
                            WsHeader* hdr, void* body, cudaStream_t s, const Tuning& tu);
// batched ridge and paint: a volume's ridge grid; its two TMA tensor maps
// (CUtensorMap, 128 bytes each, written to host memory; false without TMA);
// the launches (ctr: two zeroed work counters of the persistent paint grid)
dim3 lt_ridge_grid(const Dims& d, const Tuning& tu);
bool lt_ridge_tensor_maps(void* map_dt2, void* map_lab, const uint32_t* dt2, const uint32_t* labels, const Dims& d);
cudaError_t lt_ridge_multi_launch(const MultiArgs& m, uint32_t blocks, int ndim, bool tma, const Tuning& tu,
                                  cudaStream_t s);
cudaError_t lt_paint_multi_launch(const MultiArgs& m, int ndim, uint32_t* ctr, const Tuning& tu, cudaStream_t s);
// timeout self-test of the ridge kernel's bounded waits (see lt.h)
size_t ridge_selftest_bytes();
cudaError_t ridge_selftest_launch(void* ws, cudaStream_t s);
// copies the lookup tables to the current device (first use); call before capture
cudaError_t lt_prepare_device();
// shape.cu
size_t shape_workspace_bytes(uint32_t n_labels);
// slabs.cu: the pipeline over a host-resident volume, z-slab by z-slab
size_t slabs_ws_bytes(uint32_t n_labels, int nx, int ny, int P);
lt_status slabs_run(const uint8_t* mask_h, const uint32_t* labels_h, uint32_t n_labels, int nx, int ny, int nz,
                    int P, uint32_t* dt2_h, uint32_t* lt2_h, float* S_h, float* R_h, void* ws, size_t ws_bytes,
                    cudaStream_t s);
// scaled.cu: local thickness at 1/s resolution, upsampled (header shared with the low-res pass)
Dims scaled_dims(const Dims& d, int s);
size_t scaled_body_bytes(const Dims& d, int s);
cudaError_t scaled_launch(const uint8_t* mask, const uint32_t* labels, const Dims& d, int s, WsHeader* hdr,
                          void* body, uint32_t* lt2, cudaStream_t st);
// roundness mapped to 0-1; r_min < 0: the smallest finite value (scratch: 4 bytes)
cudaError_t rescale_launch(const float* R, uint32_t n, float r_min, uint32_t* scratch, float* out,
                           cudaStream_t s);
// the shape stage in three steps (shape_launch runs all three): clear the
// accumulators, add planes [z_lo, z_hi) of a (sub-)volume (the planes
// around them are read for the shell test), and the formulas
cudaError_t shape_clear(void* body, uint32_t n_labels, cudaStream_t s);
cudaError_t shape_accumulate(const uint32_t* labels, const uint32_t* lt2, uint32_t n_labels, const Dims& d,
                             WsHeader* hdr, void* body, int z_lo, int z_hi, cudaStream_t s, uint32_t min_lt2 = 0);
cudaError_t shape_finalize(int ndim, uint32_t n_labels, void* body, float* S, float* R,
                           const lt_object_stats* stats, cudaStream_t s);
// min_lt2 > 1: the objects are reduced to their voxels with LT2 >= min_lt2
cudaError_t shape_launch(const uint32_t* labels, const uint32_t* lt2, uint32_t n_labels,
                         const Dims& d, WsHeader* hdr, void* body, float* S, float* R,
                         const lt_object_stats* stats, cudaStream_t s, uint32_t min_lt2 = 0);

// batched shape stage: a volume's grid for kind 0 (reduction, 4-voxel
// vectors: rows of a multiple of 4 voxels), 1 (one-voxel reduction), 2
// (finalize), 3 (clear the workspace header), 4 (clear the accumulators)
dim3 shape_multi_grid(const Dims& d, uint32_t n_labels, int kind);
cudaError_t shape_multi_launch(const MultiArgs& m, uint32_t blocks, int kind, int ndim, cudaStream_t s);
// the shape stage with the learned features in the same pass over the
// volume: per-object histograms of LT / M (M^2 = ref_max[label], the
// object's largest LT2) next to the sums, then S, R, features [n][48]
size_t shape_features_bytes(uint32_t n_labels);
cudaError_t shape_features_launch(const uint32_t* labels, const uint32_t* lt2, uint32_t n_labels, const Dims& d,
                                  WsHeader* hdr, void* body, const uint32_t* ref_max, float* S, float* R, float* F,
                                  const lt_object_stats* stats, cudaStream_t s);
// measure_launch plus the features; ref_max: n_labels uint32 scratch that
// lives through the whole sequence (the ridge pass fills it)
cudaError_t measure_features_launch(const uint8_t* mask, const uint32_t* labels, uint32_t n_labels, const Dims& d,
                                    void* ws, uint32_t* ref_max, uint32_t* dt2, uint32_t* lt2, float* S, float* R,
                                    float* F, const lt_object_stats* stats, cudaStream_t s, const Tuning& tu);

// learned.cu
// histogram pass of the features (a separate pass over labels and LT2)
cudaError_t features_hist_launch(const uint32_t* labels, const uint32_t* lt2, uint32_t n_labels, const Dims& d,
                                 const uint32_t* max_lt2, uint32_t* hist, cudaStream_t s);
// the [n_labels][48] feature matrix from the per-object sums (volume,
// n_shell, max_lt2, sum_lt of st), S, R and the histograms hist[n][32]
cudaError_t features_final_launch(uint32_t n_labels, const lt_object_stats& st, const float* S, const float* R,
                                  const uint32_t* hist, float* F, cudaStream_t s);
size_t features_workspace_bytes(uint32_t n_labels);
cudaError_t features_launch(const uint32_t* labels, const uint32_t* lt2, uint32_t n_labels, const Dims& d,
                            const lt_object_stats& st, const float* S, const float* R, void* body, float* F,
                            cudaStream_t s);
cudaError_t mlp_infer_launch(const float* params, const float* F, const float* S, uint32_t n, float* out,
                             cudaStream_t s);
size_t mlp_train_workspace_bytes(uint32_t batch);
cudaError_t mlp_grad_launch(const float* params, const float* F, const float* S, const float* target,
                            const uint32_t* idx, uint32_t batch, void* ws, float* grad, float* loss,
                            cudaStream_t s);
cudaError_t mlp_adam_launch(float* params, float* m, float* v, const float* grad, uint32_t step, float lr,
                            cudaStream_t s);

// Brackets one kernel launch with trace events when tracing is enabled
// (see lt_trace_enable). Construct right before the launch; the destructor
// records the end event after it.
class TraceScope {
 public:
  TraceScope(const char* name, cudaStream_t s);
  ~TraceScope();

 private:
  int slot_;
  cudaStream_t s_;
};

// api.cu: checked dimensions, workspace of one lt_measure, and its launch
lt_status make_dims_checked(int ndim, int64_t nx, int64_t ny, int64_t nz, Dims* d);
size_t measure_ws_bytes(const Dims& d, uint32_t n_labels);
cudaError_t measure_launch(const uint8_t* mask, const uint32_t* labels, uint32_t n_labels, const Dims& d,
                           void* ws, uint32_t* dt2, uint32_t* lt2, float* S, float* R, cudaStream_t s,
                           const Tuning& tu);
// 16-byte aligned device memory of the current device (the library never
// changes the current device), and a stream of the current device
lt_status device_ptr_ok(const void* p);
lt_status stream_on_current_device(void* s);

// Number of SMs of the current device (cached per device).
int sm_count();
// Raise the dynamic shared-memory limit of a kernel once per device.
cudaError_t allow_smem(const void* func, int bytes);

}  // namespace ltk
