// Host side of the C ABI declared in include/lt.h: argument checks, workspace
// layout, device selection and the launch sequence. All compute is in the
// kernels of edt.cu, lt.cu and shape.cu.
#include <cstring>
#include <mutex>

#include "lt_internal.cuh"

using namespace ltk;

namespace ltk {

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (!cached[dev]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    cached[dev] = v;
  }
  return cached[dev];
}

cudaError_t allow_smem(const void* func, int bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  // Cheap and idempotent; called before each launch that needs more than
  // the default 48 KiB.
  return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace ltk

namespace {

constexpr int kMaxAxis = 8192;

lt_status make_dims(int ndim, int64_t nx, int64_t ny, int64_t nz, Dims* d) {
  if (ndim != 2 && ndim != 3) return LT_ERR_INVALID_ARG;
  if (nx < 1 || ny < 1 || nz < 1 || nx > kMaxAxis || ny > kMaxAxis || nz > kMaxAxis) return LT_ERR_DIMS;
  if (ndim == 2 && nz != 1) return LT_ERR_DIMS;
  const uint64_t n = (uint64_t)nx * (uint64_t)ny * (uint64_t)nz;
  if (n >= (1ull << 32)) return LT_ERR_DIMS;
  d->ndim = ndim;
  d->nx = (int)nx;
  d->ny = (int)ny;
  d->nz = (int)nz;
  d->n = (uint32_t)n;
  return LT_OK;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Accepts device (or managed) memory of the calling thread's current device
// only. The library never changes the current device: a pointer that
// belongs to another device is an argument error, returned before anything
// is enqueued.
lt_status on_current_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return LT_ERR_INVALID_ARG;
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return LT_ERR_INVALID_ARG;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return LT_ERR_CUDA;
  return a.device == cur ? LT_OK : LT_ERR_INVALID_ARG;
}

lt_status dev_ptr(const void* p) {
  if (!p || !aligned(p, 16)) return LT_ERR_INVALID_ARG;
  return on_current_device(p);
}

lt_status cuda_status(cudaError_t e) { return e == cudaSuccess ? LT_OK : LT_ERR_CUDA; }

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// The stream must belong to the current device as well (NULL: the legacy
// default stream, which always does).
lt_status stream_ok(void* s) {
  if (!s) return LT_OK;
  int dev = -1, cur = -1;
  if (cudaStreamGetDevice(as_stream(s), &dev) != cudaSuccess) {
    cudaGetLastError();
    return LT_ERR_INVALID_ARG;
  }
  if (cudaGetDevice(&cur) != cudaSuccess) return LT_ERR_CUDA;
  return dev == cur ? LT_OK : LT_ERR_INVALID_ARG;
}

lt_status check_ws(void* ws, size_t ws_bytes, size_t need) {
  if (need == 0) return LT_OK;
  if (!ws || !aligned(ws, kAlign) || ws_bytes < need) return LT_ERR_WORKSPACE;
  return on_current_device(ws);
}

size_t measure_body_bytes(const Dims& d, uint32_t n_labels) {
  size_t b = edt_workspace_bytes(d);
  b = b > lt_workspace_bytes(d) ? b : lt_workspace_bytes(d);
  const size_t sb = shape_workspace_bytes(n_labels);
  return b > sb ? b : sb;
}

lt_status run_measure(const uint8_t* mask, const uint32_t* labels, uint32_t n_labels, const Dims& d,
                      void* ws, uint32_t* dt2, uint32_t* lt2, float* S, float* R, cudaStream_t s) {
  return cuda_status(ltk::measure_launch(mask, labels, n_labels, d, ws, dt2, lt2, S, R, s, Tuning()));
}

}  // namespace

namespace ltk {

lt_status make_dims_checked(int ndim, int64_t nx, int64_t ny, int64_t nz, Dims* d) {
  return make_dims(ndim, nx, ny, nz, d);
}

size_t measure_ws_bytes(const Dims& d, uint32_t n_labels) {
  return sizeof(WsHeader) + measure_body_bytes(d, n_labels);
}

cudaError_t measure_launch(const uint8_t* mask, const uint32_t* labels, uint32_t n_labels, const Dims& d,
                           void* ws, uint32_t* dt2, uint32_t* lt2, float* S, float* R, cudaStream_t s,
                           const Tuning& tu) {
  WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
  void* body = reinterpret_cast<char*>(ws) + sizeof(WsHeader);
  cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), s);
  if (e == cudaSuccess) e = edt_launch(mask, dt2, d, body, s, tu);
  if (e == cudaSuccess) e = lt_launch(dt2, labels, lt2, d, hdr, body, s, tu);
  if (e == cudaSuccess) e = shape_launch(labels, lt2, n_labels, d, hdr, body, S, R, nullptr, s);
  return e;
}

cudaError_t measure_features_launch(const uint8_t* mask, const uint32_t* labels, uint32_t n_labels, const Dims& d,
                                    void* ws, uint32_t* ref_max, uint32_t* dt2, uint32_t* lt2, float* S, float* R,
                                    float* F, const lt_object_stats* stats, cudaStream_t s, const Tuning& tu) {
  WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
  void* body = reinterpret_cast<char*>(ws) + sizeof(WsHeader);
  cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ref_max, 0, (size_t)n_labels * 4, s);
  if (e == cudaSuccess) e = edt_launch(mask, dt2, d, body, s, tu);
  if (e == cudaSuccess) e = lt_ridge_launch(dt2, labels, lt2, d, hdr, body, s, tu, 0, d.nz, ref_max, n_labels);
  if (e == cudaSuccess) e = lt_paint_launch(dt2, labels, lt2, d, hdr, body, s, tu);
  if (e == cudaSuccess) e = shape_features_launch(labels, lt2, n_labels, d, hdr, body, ref_max, S, R, F, stats, s);
  return e;
}

lt_status device_ptr_ok(const void* p) { return dev_ptr(p); }
lt_status stream_on_current_device(void* s) { return stream_ok(s); }

}  // namespace ltk

extern "C" {

const char* lt_status_string(lt_status status) {
  switch (status) {
    case LT_OK: return "ok";
    case LT_ERR_INVALID_ARG: return "invalid argument (null, misaligned or non-device pointer, or bad ndim)";
    case LT_ERR_DIMS: return "dimensions outside the supported range";
    case LT_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case LT_ERR_LABEL_RANGE: return "a label is >= n_labels";
    case LT_ERR_LABEL_OUTSIDE_MASK: return "a voxel outside the mask carries a nonzero label";
    case LT_ERR_CUDA: return "CUDA error";
    case LT_ERR_NO_DEVICE: return "no usable CUDA device";
    case LT_ERR_TIMEOUT: return "a kernel's wait for an asynchronous copy reached its limit";
    case LT_ERR_CHECKPOINT: return "checkpoint unreadable, of another format or network shape, or corrupt";
  }
  return "unknown status";
}

uint32_t lt_version(void) { return 0x000100u; }

size_t lt_edt_workspace_size(int ndim, int64_t nx, int64_t ny, int64_t nz) {
  Dims d;
  if (make_dims(ndim, nx, ny, nz, &d) != LT_OK) return 0;
  return edt_workspace_bytes(d);
}

lt_status lt_edt(const uint8_t* mask, uint32_t* dt2, int ndim, int64_t nx, int64_t ny, int64_t nz,
                 void* ws, size_t ws_bytes, void* stream) {
  Dims d;
  lt_status st = make_dims(ndim, nx, ny, nz, &d);
  if (st != LT_OK) return st;
  if ((st = stream_ok(stream)) != LT_OK) return st;
  if ((st = dev_ptr(mask)) != LT_OK || (st = dev_ptr(dt2)) != LT_OK) return st;
  const size_t need = edt_workspace_bytes(d);
  if ((st = check_ws(ws, ws_bytes, need)) != LT_OK) return st;
  return cuda_status(edt_launch(mask, dt2, d, ws, as_stream(stream)));
}

size_t lt_local_thickness_workspace_size(int ndim, int64_t nx, int64_t ny, int64_t nz) {
  Dims d;
  if (make_dims(ndim, nx, ny, nz, &d) != LT_OK) return 0;
  return sizeof(WsHeader) + lt_workspace_bytes(d);
}

lt_status lt_local_thickness(const uint32_t* dt2, const uint32_t* labels, uint32_t* lt2, int ndim,
                             int64_t nx, int64_t ny, int64_t nz, void* ws, size_t ws_bytes,
                             void* stream) {
  Dims d;
  lt_status st = make_dims(ndim, nx, ny, nz, &d);
  if (st != LT_OK) return st;
  if ((st = stream_ok(stream)) != LT_OK) return st;
  if ((st = dev_ptr(dt2)) != LT_OK || (st = dev_ptr(labels)) != LT_OK || (st = dev_ptr(lt2)) != LT_OK)
    return st;
  if ((st = check_ws(ws, ws_bytes, sizeof(WsHeader) + lt_workspace_bytes(d))) != LT_OK) return st;
  cudaStream_t s = as_stream(stream);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
  cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), s);
  if (e == cudaSuccess) e = lt_launch(dt2, labels, lt2, d, hdr, hdr + 1, s);
  return cuda_status(e);
}

static constexpr int kMaxScale = 8;

size_t lt_local_thickness_scaled_workspace_size(int scale, int ndim, int64_t nx, int64_t ny, int64_t nz) {
  Dims d;
  if (scale < 1 || scale > kMaxScale || make_dims(ndim, nx, ny, nz, &d) != LT_OK) return 0;
  return sizeof(WsHeader) + scaled_body_bytes(d, scale);
}

lt_status lt_local_thickness_scaled(const uint8_t* mask, const uint32_t* labels, int scale, uint32_t* lt2,
                                    int ndim, int64_t nx, int64_t ny, int64_t nz, void* ws, size_t ws_bytes,
                                    void* stream) {
  Dims d;
  lt_status st = make_dims(ndim, nx, ny, nz, &d);
  if (st != LT_OK) return st;
  if ((st = stream_ok(stream)) != LT_OK) return st;
  if (scale < 1 || scale > kMaxScale) return LT_ERR_INVALID_ARG;
  if ((st = dev_ptr(mask)) != LT_OK || (st = dev_ptr(labels)) != LT_OK || (st = dev_ptr(lt2)) != LT_OK)
    return st;
  if ((st = check_ws(ws, ws_bytes, sizeof(WsHeader) + scaled_body_bytes(d, scale))) != LT_OK) return st;
  cudaStream_t s = as_stream(stream);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
  cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), s);
  if (e == cudaSuccess) e = scaled_launch(mask, labels, d, scale, hdr, hdr + 1, lt2, s);
  return cuda_status(e);
}

size_t lt_shape_workspace_size(uint32_t n_labels) {
  return sizeof(WsHeader) + shape_workspace_bytes(n_labels);
}

lt_status lt_shape_measures(const uint32_t* labels, const uint32_t* lt2, uint32_t n_labels, int ndim,
                            int64_t nx, int64_t ny, int64_t nz, void* ws, size_t ws_bytes,
                            float* sphericity, float* roundness, const lt_object_stats* stats,
                            void* stream) {
  return lt_shape_measures_filtered(labels, lt2, n_labels, 0u, ndim, nx, ny, nz, ws, ws_bytes, sphericity,
                                    roundness, stats, stream);
}

lt_status lt_shape_measures_filtered(const uint32_t* labels, const uint32_t* lt2, uint32_t n_labels,
                                     uint32_t min_lt2, int ndim, int64_t nx, int64_t ny, int64_t nz, void* ws,
                                     size_t ws_bytes, float* sphericity, float* roundness,
                                     const lt_object_stats* stats, void* stream) {
  Dims d;
  lt_status st = make_dims(ndim, nx, ny, nz, &d);
  if (st != LT_OK) return st;
  if ((st = stream_ok(stream)) != LT_OK) return st;
  if (n_labels == 0) return LT_ERR_INVALID_ARG;
  if ((st = dev_ptr(labels)) != LT_OK || (st = dev_ptr(lt2)) != LT_OK) return st;
  if (sphericity && (st = dev_ptr(sphericity)) != LT_OK) return st;
  if (roundness && (st = dev_ptr(roundness)) != LT_OK) return st;
  if (stats) {
    const void* arr[5] = {stats->volume, stats->n_shell, stats->max_lt2, stats->sum_lt, stats->sum_shell_lt};
    for (const void* p : arr)
      if (p && (st = dev_ptr(p)) != LT_OK) return st;
  }
  if ((st = check_ws(ws, ws_bytes, lt_shape_workspace_size(n_labels))) != LT_OK) return st;
  cudaStream_t s = as_stream(stream);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
  cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), s);
  if (e == cudaSuccess)
    e = shape_launch(labels, lt2, n_labels, d, hdr, hdr + 1, sphericity, roundness, stats, s, min_lt2);
  return cuda_status(e);
}

size_t lt_measure_workspace_size(uint32_t n_labels, int ndim, int64_t nx, int64_t ny, int64_t nz) {
  Dims d;
  if (make_dims(ndim, nx, ny, nz, &d) != LT_OK) return 0;
  return sizeof(WsHeader) + measure_body_bytes(d, n_labels);
}

lt_status lt_measure(const uint8_t* mask, const uint32_t* labels, uint32_t n_labels, int ndim,
                     int64_t nx, int64_t ny, int64_t nz, void* ws, size_t ws_bytes, uint32_t* dt2,
                     uint32_t* lt2, float* sphericity, float* roundness, void* stream) {
  Dims d;
  lt_status st = make_dims(ndim, nx, ny, nz, &d);
  if (st != LT_OK) return st;
  if ((st = stream_ok(stream)) != LT_OK) return st;
  if (n_labels == 0) return LT_ERR_INVALID_ARG;
  if ((st = dev_ptr(mask)) != LT_OK || (st = dev_ptr(labels)) != LT_OK || (st = dev_ptr(dt2)) != LT_OK ||
      (st = dev_ptr(lt2)) != LT_OK)
    return st;
  if (sphericity && (st = dev_ptr(sphericity)) != LT_OK) return st;
  if (roundness && (st = dev_ptr(roundness)) != LT_OK) return st;
  if ((st = check_ws(ws, ws_bytes, sizeof(WsHeader) + measure_body_bytes(d, n_labels))) != LT_OK) return st;
  return run_measure(mask, labels, n_labels, d, ws, dt2, lt2, sphericity, roundness, as_stream(stream));
}

// lt_measure_features: header, the stages' scratch, then the per-object
// largest DT2 that the ridge pass writes and the shape pass reads.
static size_t features_body_bytes(const Dims& d, uint32_t n_labels) {
  const size_t b = measure_body_bytes(d, n_labels), f = shape_features_bytes(n_labels);
  return align_up(b > f ? b : f);
}

size_t lt_measure_features_workspace_size(uint32_t n_labels, int ndim, int64_t nx, int64_t ny, int64_t nz) {
  Dims d;
  if (n_labels == 0 || make_dims(ndim, nx, ny, nz, &d) != LT_OK) return 0;
  return sizeof(WsHeader) + features_body_bytes(d, n_labels) + align_up((size_t)n_labels * 4);
}

lt_status lt_measure_features(const uint8_t* mask, const uint32_t* labels, uint32_t n_labels, int ndim, int64_t nx,
                              int64_t ny, int64_t nz, void* ws, size_t ws_bytes, uint32_t* dt2, uint32_t* lt2,
                              float* sphericity, float* roundness, float* features, const lt_object_stats* stats,
                              void* stream) {
  Dims d;
  lt_status st = make_dims(ndim, nx, ny, nz, &d);
  if (st != LT_OK) return st;
  if ((st = stream_ok(stream)) != LT_OK) return st;
  if (n_labels == 0) return LT_ERR_INVALID_ARG;
  const void* ptrs[5] = {mask, labels, dt2, lt2, features};
  for (const void* p : ptrs)
    if ((st = dev_ptr(p)) != LT_OK) return st;
  if (sphericity && (st = dev_ptr(sphericity)) != LT_OK) return st;
  if (roundness && (st = dev_ptr(roundness)) != LT_OK) return st;
  if (stats) {
    const void* arr[5] = {stats->volume, stats->n_shell, stats->max_lt2, stats->sum_lt, stats->sum_shell_lt};
    for (const void* p : arr)
      if (p && (st = dev_ptr(p)) != LT_OK) return st;
  }
  const size_t need = lt_measure_features_workspace_size(n_labels, ndim, nx, ny, nz);
  if ((st = check_ws(ws, ws_bytes, need)) != LT_OK) return st;
  uint32_t* ref_max =
      reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(ws) + sizeof(WsHeader) + features_body_bytes(d, n_labels));
  return cuda_status(measure_features_launch(mask, labels, n_labels, d, ws, ref_max, dt2, lt2, sphericity,
                                             roundness, features, stats, as_stream(stream), Tuning()));
}

static size_t host_layout(const Dims& d, uint32_t n_labels, size_t off[6]) {
  size_t p = sizeof(WsHeader) + measure_body_bytes(d, n_labels);
  p = align_up(p);
  off[0] = p; p += align_up((size_t)d.n);                  // mask
  off[1] = p; p += align_up((size_t)d.n * 4);              // labels
  off[2] = p; p += align_up((size_t)d.n * 4);              // dt2
  off[3] = p; p += align_up((size_t)d.n * 4);              // lt2
  off[4] = p; p += align_up((size_t)n_labels * 4);         // sphericity
  off[5] = p; p += align_up((size_t)n_labels * 4);         // roundness
  return p;
}

constexpr int kHostSlabs = 8;  // z-slabs of the mask copy in lt_measure_host

// Non-blocking helper streams per device, created on first use and kept:
// which = 0 the copy stream, 1 a second work stream.
static cudaStream_t helper_stream(int which) {
  static std::mutex mu;
  static cudaStream_t streams[2][64] = {{nullptr}};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> g(mu);
  cudaStream_t& st = streams[which][dev];
  if (!st && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
  return st;
}

size_t lt_measure_host_workspace_size(uint32_t n_labels, int ndim, int64_t nx, int64_t ny, int64_t nz) {
  Dims d;
  if (make_dims(ndim, nx, ny, nz, &d) != LT_OK) return 0;
  size_t off[6];
  return host_layout(d, n_labels, off);
}

lt_status lt_measure_host(const uint8_t* mask_host, const uint32_t* labels_host, uint32_t n_labels,
                          int ndim, int64_t nx, int64_t ny, int64_t nz, void* ws, size_t ws_bytes,
                          float* sphericity_host, float* roundness_host, void* stream) {
  Dims d;
  lt_status st = make_dims(ndim, nx, ny, nz, &d);
  if (st != LT_OK) return st;
  if ((st = stream_ok(stream)) != LT_OK) return st;
  if (n_labels == 0 || !mask_host || !labels_host || !sphericity_host || !roundness_host)
    return LT_ERR_INVALID_ARG;
  size_t off[6];
  const size_t need = host_layout(d, n_labels, off);
  if ((st = check_ws(ws, ws_bytes, need)) != LT_OK) return st;
  char* base = reinterpret_cast<char*>(ws);
  uint8_t* mask = reinterpret_cast<uint8_t*>(base + off[0]);
  uint32_t* labels = reinterpret_cast<uint32_t*>(base + off[1]);
  uint32_t* dt2 = reinterpret_cast<uint32_t*>(base + off[2]);
  uint32_t* lt2 = reinterpret_cast<uint32_t*>(base + off[3]);
  float* S = reinterpret_cast<float*>(base + off[4]);
  float* R = reinterpret_cast<float*>(base + off[5]);
  cudaStream_t s = as_stream(stream);
  // The copies run on a second stream and overlap the work: the mask
  // arrives in z-slabs, each slab's x and y EDT passes start as soon as it
  // is there; the labels arrive in z-slabs during the EDT, and the ridge
  // pass runs slab by slab as they land (a slab also needs the next slab's
  // first plane), alternating between `stream` and a second work stream:
  // slabs are independent (their own LT2 planes, records appended by
  // atomics), and one slab's launch is too small to fill the GPU alone. The
  // last two slabs are one ridge chunk each, since they run after the last
  // copy. Painting needs every centre (and the `touch` flag of the whole
  // volume), so it starts after the last ridge slab on both streams.
  cudaStream_t c = helper_stream(0), s2 = helper_stream(1);
  if (!c || !s2) return LT_ERR_CUDA;
  const Tuning tu;
  const int K = d.ndim == 3 ? std::min(d.nz, kHostSlabs) : 1;
  const int rz = ridge_chunk(tu), nch = (d.nz + rz - 1) / rz;
  const int KL = d.ndim == 3 ? std::min(nch, kHostSlabs) : 1;  // label slabs: whole ridge chunks
  cudaEvent_t ev[2 * kHostSlabs + 3];
  const int nev = K + KL + 3;
  for (int k = 0; k < nev; ++k)
    if (cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming) != cudaSuccess) {
      for (int j = 0; j < k; ++j) cudaEventDestroy(ev[j]);
      return LT_ERR_CUDA;
    }
  cudaEvent_t* ev_mask = ev;
  cudaEvent_t* ev_lab = ev + K;
  cudaEvent_t ev_start = ev[K + KL], ev_edt = ev[K + KL + 1], ev_s2 = ev[K + KL + 2];
  const size_t plane = (size_t)d.nx * d.ny;
  // label slab k starts at ridge chunk c0[k]: the last two slabs one chunk
  // each, the others shared out evenly
  int c0[kHostSlabs + 1];
  for (int k = 0; k <= KL; ++k) {
    const int tail = std::min(KL - 1, 2), head = KL - tail;
    c0[k] = k <= head ? (int)((int64_t)(nch - tail) * k / head) : (nch - tail) + (k - head);
  }
  auto lab_z = [&](int k) { return d.ndim == 3 ? std::min(d.nz, c0[k] * rz) : 0; };
  WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
  void* body = reinterpret_cast<char*>(ws) + sizeof(WsHeader);
  cudaError_t e = cudaEventRecord(ev_start, s);  // the copies start after earlier work on `stream`
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c, ev_start, 0);
  if (e == cudaSuccess) e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), s);
  for (int k = 0; k < K && e == cudaSuccess; ++k) {
    const int z0 = (int)((int64_t)d.nz * k / K), z1 = (int)((int64_t)d.nz * (k + 1) / K);
    e = cudaMemcpyAsync(mask + z0 * plane, mask_host + z0 * plane, (size_t)(z1 - z0) * plane,
                        cudaMemcpyHostToDevice, c);
    if (e == cudaSuccess) e = cudaEventRecord(ev_mask[k], c);
  }
  for (int k = 0; k < KL && e == cudaSuccess; ++k) {
    const int z0 = lab_z(k), z1 = d.ndim == 3 ? lab_z(k + 1) : 1;
    const size_t pl = d.ndim == 3 ? plane : (size_t)d.n;
    e = cudaMemcpyAsync(labels + z0 * pl, labels_host + z0 * pl, (size_t)(z1 - z0) * pl * 4,
                        cudaMemcpyHostToDevice, c);
    if (e == cudaSuccess) e = cudaEventRecord(ev_lab[k], c);
  }
  for (int k = 0; k < K && e == cudaSuccess; ++k) {
    const int z0 = (int)((int64_t)d.nz * k / K), z1 = (int)((int64_t)d.nz * (k + 1) / K);
    Dims dk = d;
    dk.nz = z1 - z0;
    dk.n = (uint32_t)((size_t)dk.nz * plane);
    e = cudaStreamWaitEvent(s, ev_mask[k], 0);
    if (e == cudaSuccess) e = edt_launch(mask + z0 * plane, dt2 + z0 * plane, dk, body, s, tu, 1);
  }
  if (e == cudaSuccess) e = edt_launch(nullptr, dt2, d, body, s, tu, 2);
  if (e == cudaSuccess) e = cudaEventRecord(ev_edt, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s2, ev_edt, 0);
  for (int k = 0; k < KL && e == cudaSuccess; ++k) {
    cudaStream_t w = (k & 1) ? s2 : s;
    e = cudaStreamWaitEvent(w, ev_lab[std::min(k + 1, KL - 1)], 0);  // (copies land in order)
    if (e == cudaSuccess) e = lt_ridge_launch(dt2, labels, lt2, d, hdr, body, w, tu, lab_z(k), d.ndim == 3 ? lab_z(k + 1) : 1);
  }
  if (e == cudaSuccess) e = cudaEventRecord(ev_s2, s2);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_s2, 0);
  if (e == cudaSuccess) e = lt_paint_launch(dt2, labels, lt2, d, hdr, body, s, tu);
  if (e == cudaSuccess) e = shape_launch(labels, lt2, n_labels, d, hdr, body, S, R, nullptr, s);
  for (int k = 0; k < nev; ++k) cudaEventDestroy(ev[k]);  // (released once the streams are past them)
  if (e != cudaSuccess) return LT_ERR_CUDA;
  e = cudaMemcpyAsync(sphericity_host, S, (size_t)n_labels * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(roundness_host, R, (size_t)n_labels * 4, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return LT_ERR_CUDA;
  return lt_workspace_status(ws, ws_bytes, stream);
}

lt_status lt_workspace_status(const void* ws, size_t ws_bytes, void* stream) {
  if (!ws || ws_bytes < sizeof(WsHeader) || !aligned(ws, kAlign)) return LT_ERR_WORKSPACE;
  lt_status st = on_current_device(ws);
  if (st == LT_OK) st = stream_ok(stream);
  if (st != LT_OK) return st;
  if (cudaStreamSynchronize(as_stream(stream)) != cudaSuccess) return LT_ERR_CUDA;
  uint32_t err = 0;
  if (cudaMemcpy(&err, ws, sizeof(err), cudaMemcpyDeviceToHost) != cudaSuccess) return LT_ERR_CUDA;
  if (err & ERR_TIMEOUT) return LT_ERR_TIMEOUT;
  if (err & ERR_LABEL_OUTSIDE_MASK) return LT_ERR_LABEL_OUTSIDE_MASK;
  if (err & ERR_LABEL_RANGE) return LT_ERR_LABEL_RANGE;
  return LT_OK;
}

static bool slab_dims_ok(int64_t nx, int64_t ny, int64_t nz, int slab_planes) {
  if (nx < 1 || ny < 1 || nz < 1 || nx > kMaxAxis || ny > kMaxAxis || nz > kMaxAxis) return false;
  const int64_t mn = std::min(nx, std::min(ny, nz));
  if ((mn + 1) / 2 * ((mn + 1) / 2) >= (1 << 24)) return false;  // DT2 < 2^24
  return slab_planes >= 1 && (uint64_t)slab_planes * (uint64_t)(nx * ny) < (1ull << 32);
}

size_t lt_measure_slabs_workspace_size(uint32_t n_labels, int64_t nx, int64_t ny, int64_t nz, int slab_planes) {
  if (n_labels == 0 || !slab_dims_ok(nx, ny, nz, slab_planes)) return 0;
  return slabs_ws_bytes(n_labels, (int)nx, (int)ny, slab_planes);
}

lt_status lt_measure_slabs(const uint8_t* mask_host, const uint32_t* labels_host, uint32_t n_labels, int64_t nx,
                           int64_t ny, int64_t nz, int slab_planes, uint32_t* dt2_host, uint32_t* lt2_host,
                           float* sphericity_host, float* roundness_host, void* ws, size_t ws_bytes,
                           void* stream) {
  if (!mask_host || !labels_host || !dt2_host || !sphericity_host || !roundness_host || n_labels == 0)
    return LT_ERR_INVALID_ARG;
  if (!slab_dims_ok(nx, ny, nz, slab_planes)) return LT_ERR_DIMS;
  lt_status st = check_ws(ws, ws_bytes, slabs_ws_bytes(n_labels, (int)nx, (int)ny, slab_planes));
  if (st == LT_OK) st = stream_ok(stream);
  if (st != LT_OK) return st;
  cudaStream_t s = as_stream(stream);
  st = slabs_run(mask_host, labels_host, n_labels, (int)nx, (int)ny, (int)nz, slab_planes, dt2_host, lt2_host,
                 sphericity_host, roundness_host, ws, ws_bytes, s);
  if (st != LT_OK) {
    cudaStreamSynchronize(s);
    return st;
  }
  return lt_workspace_status(ws, ws_bytes, stream);
}

size_t lt_roundness_rescale_workspace_size(void) { return kAlign; }

lt_status lt_roundness_rescale(const float* roundness, uint32_t n, float r_min, float* out, void* ws,
                               size_t ws_bytes, void* stream) {
  if (n == 0) return LT_OK;
  lt_status st;
  if ((st = dev_ptr(roundness)) != LT_OK || (st = dev_ptr(out)) != LT_OK) return st;
  if (!(r_min < 1.f) && !(r_min >= 1.f)) return LT_ERR_INVALID_ARG;  // NaN
  if ((st = check_ws(ws, ws_bytes, kAlign)) != LT_OK || (st = stream_ok(stream)) != LT_OK) return st;
  return cuda_status(rescale_launch(roundness, n, r_min, reinterpret_cast<uint32_t*>(ws), out, as_stream(stream)));
}

size_t lt_selftest_workspace_size(void) { return ridge_selftest_bytes(); }

lt_status lt_selftest_wait_timeout(void* ws, size_t ws_bytes, void* stream) {
  lt_status st = check_ws(ws, ws_bytes, ridge_selftest_bytes());
  if (st == LT_OK) st = stream_ok(stream);
  if (st != LT_OK) return st;
  if (ridge_selftest_launch(ws, as_stream(stream)) != cudaSuccess) return LT_ERR_CUDA;
  return lt_workspace_status(ws, ws_bytes, stream);
}

lt_status lt_workspace_counters(const void* ws, size_t ws_bytes, void* stream, lt_lt_counters* out) {
  if (!ws || ws_bytes < sizeof(WsHeader) || !aligned(ws, kAlign)) return LT_ERR_WORKSPACE;
  if (!out) return LT_ERR_INVALID_ARG;
  lt_status st = on_current_device(ws);
  if (st == LT_OK) st = stream_ok(stream);
  if (st != LT_OK) return st;
  if (cudaStreamSynchronize(as_stream(stream)) != cudaSuccess) return LT_ERR_CUDA;
  WsHeader h;
  if (cudaMemcpy(&h, ws, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return LT_ERR_CUDA;
  out->chunk_centres = h.n_surv;
  out->warp_centres = h.n_big;
  out->updates = h.n_updates;
  out->table_updates = h.n_table_updates;
  return LT_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ tracing
#include <mutex>
#include <string>
#include <vector>

namespace {

struct TraceRecord {
  std::string name;
  cudaEvent_t start, stop;
  int device;
};

struct TraceState {
  std::mutex mu;
  bool enabled = false;
  std::vector<TraceRecord> pending;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pool;  // free event pairs
  std::vector<std::pair<std::string, std::pair<uint32_t, double>>> totals;
};

TraceState& trace() {
  static TraceState* t = new TraceState();  // never destroyed: events may outlive static teardown
  return *t;
}

}  // namespace

namespace ltk {

TraceScope::TraceScope(const char* name, cudaStream_t s) : slot_(-1), s_(s) {
  TraceState& t = trace();
  std::lock_guard<std::mutex> g(t.mu);
  if (!t.enabled) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;  // no event timing inside graph capture
  }
  std::pair<cudaEvent_t, cudaEvent_t> ev;
  if (!t.pool.empty()) {
    ev = t.pool.back();
    t.pool.pop_back();
  } else if (cudaEventCreate(&ev.first) != cudaSuccess || cudaEventCreate(&ev.second) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaEventRecord(ev.first, s);
  t.pending.push_back({name, ev.first, ev.second, dev});
  slot_ = (int)t.pending.size() - 1;
}

TraceScope::~TraceScope() {
  if (slot_ < 0) return;
  TraceState& t = trace();
  std::lock_guard<std::mutex> g(t.mu);
  if (slot_ < (int)t.pending.size()) cudaEventRecord(t.pending[slot_].stop, s_);
}

}  // namespace ltk

extern "C" {

lt_status lt_trace_enable(int enable) {
  TraceState& t = trace();
  std::lock_guard<std::mutex> g(t.mu);
  if (enable) {
    for (auto& r : t.pending) t.pool.push_back({r.start, r.stop});
    t.pending.clear();
    t.totals.clear();
  }
  t.enabled = enable != 0;
  return LT_OK;
}

int lt_trace_summary(lt_trace_entry* out, int max_entries) {
  TraceState& t = trace();
  std::lock_guard<std::mutex> g(t.mu);
  int bad = 0;
  for (auto& r : t.pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.stop) != cudaSuccess || cudaEventElapsedTime(&ms, r.start, r.stop) != cudaSuccess) {
      cudaGetLastError();
      bad = 1;
    }
    bool found = false;
    for (auto& e : t.totals)
      if (e.first == r.name) {
        e.second.first += 1;
        e.second.second += ms;
        found = true;
        break;
      }
    if (!found) t.totals.push_back({r.name, {1u, (double)ms}});
    t.pool.push_back({r.start, r.stop});
  }
  t.pending.clear();
  if (bad) return -1;
  const int n = (int)t.totals.size();
  for (int i = 0; i < n && i < max_entries && out; ++i) {
    std::memset(out[i].name, 0, sizeof(out[i].name));
    std::strncpy(out[i].name, t.totals[i].first.c_str(), sizeof(out[i].name) - 1);
    out[i].launches = t.totals[i].second.first;
    out[i].total_ms = t.totals[i].second.second;
  }
  return n;
}

}  // extern "C"

// ---------------------------------------------------------- learned part
extern "C" {

size_t lt_features_workspace_size(uint32_t n_labels) { return features_workspace_bytes(n_labels); }

lt_status lt_object_features(const uint32_t* labels, const uint32_t* lt2, uint32_t n_labels, int ndim,
                             int64_t nx, int64_t ny, int64_t nz, const lt_object_stats* stats,
                             const float* sphericity, const float* roundness, void* ws, size_t ws_bytes,
                             float* features, void* stream) {
  Dims d;
  lt_status st = make_dims(ndim, nx, ny, nz, &d);
  if (st != LT_OK) return st;
  if ((st = stream_ok(stream)) != LT_OK) return st;
  if (n_labels == 0 || !stats) return LT_ERR_INVALID_ARG;
  const void* ptrs[9] = {labels, lt2, stats->volume, stats->n_shell, stats->max_lt2, stats->sum_lt,
                         sphericity, roundness, features};
  for (const void* p : ptrs)
    if ((st = dev_ptr(p)) != LT_OK) return st;
  if (!ws || !aligned(ws, kAlign) || ws_bytes < features_workspace_bytes(n_labels)) return LT_ERR_WORKSPACE;
  if ((st = on_current_device(ws)) != LT_OK) return st;
  return cuda_status(features_launch(labels, lt2, n_labels, d, *stats, sphericity, roundness, ws, features,
                                     as_stream(stream)));
}

lt_status lt_mlp_infer(const float* params, const float* features, const float* sphericity, uint32_t n,
                       float* s_learned, void* stream) {
  lt_status st;
  if (n == 0) return LT_OK;
  const void* ptrs[4] = {params, features, sphericity, s_learned};
  for (const void* p : ptrs)
    if ((st = dev_ptr(p)) != LT_OK) return st;
  if ((st = stream_ok(stream)) != LT_OK) return st;
  return cuda_status(mlp_infer_launch(params, features, sphericity, n, s_learned, as_stream(stream)));
}

size_t lt_mlp_train_workspace_size(uint32_t batch) { return mlp_train_workspace_bytes(batch); }

lt_status lt_mlp_gradients(const float* params, const float* features, const float* sphericity,
                           const float* target, const uint32_t* batch_idx, uint32_t batch, void* ws,
                           size_t ws_bytes, float* grad, float* loss, void* stream) {
  lt_status st;
  if (batch == 0) return LT_ERR_INVALID_ARG;
  const void* ptrs[6] = {params, features, sphericity, target, batch_idx, grad};
  for (const void* p : ptrs)
    if ((st = dev_ptr(p)) != LT_OK) return st;
  if (loss && (st = dev_ptr(loss)) != LT_OK) return st;
  if ((st = stream_ok(stream)) != LT_OK) return st;
  if (!ws || !aligned(ws, kAlign) || ws_bytes < mlp_train_workspace_bytes(batch)) return LT_ERR_WORKSPACE;
  if ((st = on_current_device(ws)) != LT_OK) return st;
  return cuda_status(mlp_grad_launch(params, features, sphericity, target, batch_idx, batch, ws, grad, loss,
                                     as_stream(stream)));
}

lt_status lt_mlp_adam(float* params, float* m, float* v, const float* grad, uint32_t step, float lr,
                      void* stream) {
  lt_status st;
  if (step == 0) return LT_ERR_INVALID_ARG;
  const void* ptrs[4] = {params, m, v, grad};
  for (const void* p : ptrs)
    if ((st = dev_ptr(p)) != LT_OK) return st;
  if ((st = stream_ok(stream)) != LT_OK) return st;
  return cuda_status(mlp_adam_launch(params, m, v, grad, step, lr, as_stream(stream)));
}

lt_status lt_mlp_train_step(float* params, float* m, float* v, float* grad, uint32_t step, float lr,
                            const float* features, const float* sphericity, const float* target,
                            const uint32_t* batch_idx, uint32_t batch, void* ws, size_t ws_bytes,
                            float* loss, void* stream) {
  lt_status st = lt_mlp_gradients(params, features, sphericity, target, batch_idx, batch, ws, ws_bytes,
                                  grad, loss, stream);
  if (st != LT_OK) return st;
  return lt_mlp_adam(params, m, v, grad, step, lr, stream);
}

}  // extern "C"

// ------------------------------------------------------- MLP checkpoints
// Layout (little-endian): "LTMLPCK1", then uint32 version, n_features,
// hidden, n_params, step, flags (bit 0: Adam moments stored), then float32
// params[n_params], m[n_params], v[n_params] (zeros when no moments), then
// the CRC-32 (IEEE 802.3, reflected, polynomial 0xEDB88320) of every byte
// before it.
#include <cstdio>

namespace {

constexpr char kCkptMagic[8] = {'L', 'T', 'M', 'L', 'P', 'C', 'K', '1'};
constexpr uint32_t kCkptVersion = 1;
constexpr size_t kCkptHeader = 8 + 6 * 4;
constexpr size_t kCkptBytes = kCkptHeader + 3 * (size_t)LT_MLP_PARAMS * 4 + 4;

// CRC-32 bit by bit from its definition: the remainder of the message
// polynomial (bits reflected, register preset to all ones, result inverted)
// modulo x^32 + x^26 + x^23 + ... + 1.
uint32_t crc32_ieee(const unsigned char* p, size_t n) {
  uint32_t c = 0xFFFFFFFFu;
  for (size_t i = 0; i < n; ++i) {
    c ^= p[i];
    for (int k = 0; k < 8; ++k) c = (c >> 1) ^ (0xEDB88320u & (0u - (c & 1u)));
  }
  return ~c;
}

void put_u32(unsigned char* p, uint32_t v) {
  for (int k = 0; k < 4; ++k) p[k] = (unsigned char)(v >> (8 * k));
}
uint32_t get_u32(const unsigned char* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
void put_floats(unsigned char* p, const float* v) {
  for (size_t i = 0; i < (size_t)LT_MLP_PARAMS; ++i) {
    uint32_t u = 0;
    if (v) std::memcpy(&u, v + i, 4);
    put_u32(p + 4 * i, u);
  }
}
void get_floats(const unsigned char* p, float* v) {
  for (size_t i = 0; i < (size_t)LT_MLP_PARAMS; ++i) {
    const uint32_t u = get_u32(p + 4 * i);
    std::memcpy(v + i, &u, 4);
  }
}

}  // namespace

extern "C" {

size_t lt_mlp_checkpoint_size(void) { return kCkptBytes; }

lt_status lt_mlp_checkpoint_pack(const float* params_host, const float* m_host, const float* v_host,
                                 uint32_t step, void* out_host, size_t out_bytes) {
  if (!params_host || !out_host || (!m_host != !v_host)) return LT_ERR_INVALID_ARG;
  if (out_bytes < kCkptBytes) return LT_ERR_WORKSPACE;
  unsigned char* p = reinterpret_cast<unsigned char*>(out_host);
  std::memcpy(p, kCkptMagic, 8);
  const uint32_t head[6] = {kCkptVersion, LT_MLP_FEATURES, LT_MLP_HIDDEN, LT_MLP_PARAMS, step,
                            m_host ? 1u : 0u};
  for (int k = 0; k < 6; ++k) put_u32(p + 8 + 4 * k, head[k]);
  unsigned char* body = p + kCkptHeader;
  put_floats(body, params_host);
  put_floats(body + 4 * (size_t)LT_MLP_PARAMS, m_host);
  put_floats(body + 8 * (size_t)LT_MLP_PARAMS, v_host);
  put_u32(p + kCkptBytes - 4, crc32_ieee(p, kCkptBytes - 4));
  return LT_OK;
}

lt_status lt_mlp_checkpoint_unpack(const void* in_host, size_t in_bytes, float* params_host, float* m_host,
                                   float* v_host, uint32_t* step) {
  if (!in_host || (!m_host != !v_host)) return LT_ERR_INVALID_ARG;
  const unsigned char* p = reinterpret_cast<const unsigned char*>(in_host);
  if (in_bytes != kCkptBytes || std::memcmp(p, kCkptMagic, 8) != 0) return LT_ERR_CHECKPOINT;
  if (get_u32(p + kCkptBytes - 4) != crc32_ieee(p, kCkptBytes - 4)) return LT_ERR_CHECKPOINT;
  if (get_u32(p + 8) != kCkptVersion || get_u32(p + 12) != LT_MLP_FEATURES || get_u32(p + 16) != LT_MLP_HIDDEN ||
      get_u32(p + 20) != LT_MLP_PARAMS)
    return LT_ERR_CHECKPOINT;
  const bool moments = (get_u32(p + 28) & 1u) != 0;
  if (m_host && !moments) return LT_ERR_CHECKPOINT;
  const unsigned char* body = p + kCkptHeader;
  if (params_host) get_floats(body, params_host);
  if (m_host) {
    get_floats(body + 4 * (size_t)LT_MLP_PARAMS, m_host);
    get_floats(body + 8 * (size_t)LT_MLP_PARAMS, v_host);
  }
  if (step) *step = get_u32(p + 24);
  return LT_OK;
}

lt_status lt_mlp_save(const char* path, const float* params, const float* m, const float* v, uint32_t step,
                      void* stream) {
  if (!path || (!m != !v)) return LT_ERR_INVALID_ARG;
  lt_status st;
  const float* ptrs[3] = {params, m, v};
  for (int k = 0; k < 3; ++k)
    if ((k == 0 || ptrs[k]) && (st = dev_ptr(ptrs[k])) != LT_OK) return st;
  if ((st = stream_ok(stream)) != LT_OK) return st;
  std::vector<float> h(3 * (size_t)LT_MLP_PARAMS);
  cudaStream_t s = as_stream(stream);
  for (int k = 0; k < 3; ++k)
    if (ptrs[k] && cudaMemcpyAsync(h.data() + k * (size_t)LT_MLP_PARAMS, ptrs[k], 4 * (size_t)LT_MLP_PARAMS,
                                   cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return LT_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return LT_ERR_CUDA;
  std::vector<unsigned char> buf(kCkptBytes);
  st = lt_mlp_checkpoint_pack(h.data(), m ? h.data() + LT_MLP_PARAMS : nullptr,
                              v ? h.data() + 2 * (size_t)LT_MLP_PARAMS : nullptr, step, buf.data(), buf.size());
  if (st != LT_OK) return st;
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return LT_ERR_CHECKPOINT;
  const bool ok = std::fwrite(buf.data(), 1, buf.size(), f) == buf.size();
  if (std::fclose(f) != 0 || !ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return LT_ERR_CHECKPOINT;
  }
  return LT_OK;
}

lt_status lt_mlp_load(const char* path, float* params, float* m, float* v, uint32_t* step, void* stream) {
  if (!path || (!m != !v)) return LT_ERR_INVALID_ARG;
  lt_status st;
  float* ptrs[3] = {params, m, v};
  for (int k = 0; k < 3; ++k)
    if ((k == 0 || ptrs[k]) && (st = dev_ptr(ptrs[k])) != LT_OK) return st;
  if ((st = stream_ok(stream)) != LT_OK) return st;
  std::vector<unsigned char> buf(kCkptBytes + 1);
  FILE* f = std::fopen(path, "rb");
  if (!f) return LT_ERR_CHECKPOINT;
  const size_t got = std::fread(buf.data(), 1, buf.size(), f);
  std::fclose(f);
  std::vector<float> h(3 * (size_t)LT_MLP_PARAMS);
  st = lt_mlp_checkpoint_unpack(buf.data(), got, h.data(), m ? h.data() + LT_MLP_PARAMS : nullptr,
                                v ? h.data() + 2 * (size_t)LT_MLP_PARAMS : nullptr, step);
  if (st != LT_OK) return st;
  cudaStream_t s = as_stream(stream);
  for (int k = 0; k < 3; ++k)
    if (ptrs[k] && cudaMemcpyAsync(ptrs[k], h.data() + k * (size_t)LT_MLP_PARAMS, 4 * (size_t)LT_MLP_PARAMS,
                                   cudaMemcpyHostToDevice, s) != cudaSuccess)
      return LT_ERR_CUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? LT_OK : LT_ERR_CUDA;
}

}  // extern "C"
