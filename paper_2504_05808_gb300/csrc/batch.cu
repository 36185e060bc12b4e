// Batched form: many volumes as one CUDA graph launch, and its autotuner.
//
// Each volume runs the kernels of lt_measure in its own workspace slice.
// At creation the batch is recorded into a graph: a fork event fans out to
// `branches` capture streams, volumes are assigned largest first to the
// least loaded branch, and a join brings the branches back. Volumes on
// different branches have no dependency, so the GPU overlaps them; small
// volumes that cannot fill the GPU alone run side by side.
//
// The autotuner changes one setting at a time (branch count, EDT column-tile
// width, ridge z-chunk, paint CTAs per SM), re-records the graph for each
// candidate and times a few launches with CUDA events; the fastest setting of
// each pass is kept. Results go to a small JSON file keyed by GPU name and
// the batch's shape class (2D/3D counts and the median volume size).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lt_internal.cuh"

using namespace ltk;

struct lt_batch {
  std::vector<lt_volume> vols;
  std::vector<Dims> dims;
  std::vector<size_t> off;  // workspace slice of each volume
  char* ws = nullptr;
  int device = 0;
  int branches = 1;
  Tuning tu;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

constexpr int kMaxBranches = 32;

size_t slice_bytes(const Dims& d, uint32_t n_labels) { return align_up(measure_ws_bytes(d, n_labels)); }

lt_status check_volume(const lt_volume& v, Dims* d) {
  lt_status st = make_dims_checked(v.ndim, v.nx, v.ny, v.nz, d);
  if (st != LT_OK) return st;
  if (v.n_labels == 0) return LT_ERR_INVALID_ARG;
  const void* ptrs[6] = {v.mask, v.labels, v.dt2, v.lt2, v.sphericity, v.roundness};
  for (const void* p : ptrs)
    if ((st = device_ptr_ok(p)) != LT_OK) return st;
  return LT_OK;
}

void destroy_graph(lt_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// Records the batch into a graph with b->branches branches and b->tu.
lt_status record(lt_batch* b) {
  destroy_graph(b);
  const int nb = b->branches;
  while ((int)b->streams.size() < nb + 1) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return LT_ERR_CUDA;
    b->streams.push_back(s);
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return LT_ERR_CUDA;
    b->join.push_back(e);
  }
  if (!b->fork && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) return LT_ERR_CUDA;
  // largest volumes first, each to the least loaded branch
  std::vector<int> order(b->vols.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return b->dims[x].n > b->dims[y].n; });
  std::vector<double> load(nb, 0.0);
  std::vector<int> branch(b->vols.size(), 0);
  for (int i : order) {
    const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    branch[i] = k;
    load[k] += (double)b->dims[i].n;
  }
  cudaStream_t cap = b->streams[nb];
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return LT_ERR_CUDA;
  cudaError_t e = cudaEventRecord(b->fork, cap);
  for (int k = 0; k < nb && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->streams[k], b->fork, 0);
  for (int i : order) {
    if (e != cudaSuccess) break;
    const lt_volume& v = b->vols[i];
    e = measure_launch(v.mask, v.labels, v.n_labels, b->dims[i], b->ws + b->off[i], v.dt2, v.lt2,
                       v.sphericity, v.roundness, b->streams[branch[i]], b->tu);
  }
  for (int k = 0; k < nb && e == cudaSuccess; ++k) {
    e = cudaEventRecord(b->join[k], b->streams[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, b->join[k], 0);
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(cap, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return LT_ERR_CUDA;
  }
  b->graph = g;
  if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
    cudaGetLastError();
    destroy_graph(b);
    return LT_ERR_CUDA;
  }
  return LT_OK;
}

std::string shape_class(const lt_batch* b) {
  std::vector<double> n;
  int n2 = 0, n3 = 0;
  for (const Dims& d : b->dims) {
    n.push_back((double)d.n);
    (d.ndim == 3 ? n3 : n2)++;
  }
  std::sort(n.begin(), n.end());
  const double med = n.empty() ? 1.0 : n[n.size() / 2];
  char buf[96];
  std::snprintf(buf, sizeof(buf), "2d%d-3d%d-med2^%d", n2, n3, (int)std::lround(std::log2(med)));
  return buf;
}

// ---- minimal JSON cache: {"key": {"branches": 4, "edt_tx_y": 8, ...}, ...}
constexpr int kSettings = 5;  // branches, EDT y and z tile widths, ridge z-chunk, paint CTAs/SM
struct CacheEntry {
  std::string key;
  int v[kSettings];
  double ms;
};

std::vector<CacheEntry> read_cache(const char* path) {
  std::vector<CacheEntry> out;
  if (!path) return out;
  FILE* f = std::fopen(path, "rb");
  if (!f) return out;
  std::string text;
  char buf[4096];
  size_t k;
  while ((k = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, k);
  std::fclose(f);
  static const char* names[kSettings] = {"\"branches\"", "\"edt_tx_y\"", "\"edt_tx_z\"", "\"ridge_z\"",
                                         "\"paint_bpsm\""};
  size_t pos = 0;
  while (true) {
    const size_t q0 = text.find('"', pos);
    if (q0 == std::string::npos) break;
    const size_t q1 = text.find('"', q0 + 1);
    const size_t ob = text.find('{', q1 == std::string::npos ? text.size() : q1);
    const size_t cb = text.find('}', ob == std::string::npos ? text.size() : ob);
    if (q1 == std::string::npos || ob == std::string::npos || cb == std::string::npos) break;
    CacheEntry e;
    e.key = text.substr(q0 + 1, q1 - q0 - 1);
    const std::string body = text.substr(ob, cb - ob);
    bool ok = true;
    for (int i = 0; i < kSettings; ++i) {
      const size_t p = body.find(names[i]);
      if (p == std::string::npos) {
        ok = false;
        break;
      }
      e.v[i] = std::atoi(body.c_str() + body.find(':', p) + 1);
    }
    const size_t pm = body.find("\"ms\"");
    e.ms = pm == std::string::npos ? 0.0 : std::atof(body.c_str() + body.find(':', pm) + 1);
    if (ok) out.push_back(e);
    pos = cb + 1;
  }
  return out;
}

bool write_cache(const char* path, const std::vector<CacheEntry>& entries) {
  if (!path) return true;
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return false;
  std::fprintf(f, "{\n");
  for (size_t i = 0; i < entries.size(); ++i) {
    const CacheEntry& e = entries[i];
    std::fprintf(f,
                 "  \"%s\": {\"branches\": %d, \"edt_tx_y\": %d, \"edt_tx_z\": %d, \"ridge_z\": %d, "
                 "\"paint_bpsm\": %d, \"ms\": %.4f}%s\n",
                 e.key.c_str(), e.v[0], e.v[1], e.v[2], e.v[3], e.v[4], e.ms, i + 1 < entries.size() ? "," : "");
  }
  std::fprintf(f, "}\n");
  std::fclose(f);
  return std::rename(tmp.c_str(), path) == 0;
}

void apply(lt_batch* b, const int v[kSettings]) {
  b->branches = std::max(1, std::min(kMaxBranches, v[0]));
  b->tu.edt_tx_y = v[1] == 8 || v[1] == 16 ? v[1] : 32;
  b->tu.edt_tx_z = v[2] == 8 || v[2] == 16 ? v[2] : 32;
  b->tu.ridge_z = v[3] == 8 || v[3] == 32 ? v[3] : 16;
  b->tu.paint_blocks_per_sm = std::max(1, std::min(32, v[4]));
}

void current(const lt_batch* b, int v[kSettings]) {
  v[0] = b->branches;
  v[1] = b->tu.edt_tx_y;
  v[2] = b->tu.edt_tx_z;
  v[3] = b->tu.ridge_z;
  v[4] = b->tu.paint_blocks_per_sm;
}

// mean ms of `reps` graph launches (after one warm-up launch)
lt_status time_graph(lt_batch* b, cudaStream_t s, int reps, double* ms) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return LT_ERR_CUDA;
  cudaError_t e = cudaGraphLaunch(b->exec, s);
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  for (int i = 0; i < reps && e == cudaSuccess; ++i) e = cudaGraphLaunch(b->exec, s);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = t / reps;
  return e == cudaSuccess ? LT_OK : LT_ERR_CUDA;
}

// A batch runs on the device it was created on, which must be the current
// device (the library never changes it), with a stream of that device.
lt_status batch_device_ok(const lt_batch* b, void* stream) {
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return LT_ERR_CUDA;
  if (cur != b->device) return LT_ERR_INVALID_ARG;
  return stream_on_current_device(stream);
}

}  // namespace

extern "C" {

size_t lt_batch_workspace_size(const lt_volume* vols, int n_vols) {
  if (!vols || n_vols <= 0) return 0;
  size_t total = 0;
  for (int i = 0; i < n_vols; ++i) {
    Dims d;
    if (make_dims_checked(vols[i].ndim, vols[i].nx, vols[i].ny, vols[i].nz, &d) != LT_OK) return 0;
    total += slice_bytes(d, vols[i].n_labels);
  }
  return total;
}

lt_status lt_batch_create(const lt_volume* vols, int n_vols, void* ws, size_t ws_bytes, int branches,
                          lt_batch** out) {
  if (!out || !vols || n_vols <= 0 || branches < 1) return LT_ERR_INVALID_ARG;
  *out = nullptr;
  lt_batch* b = new lt_batch();
  b->vols.assign(vols, vols + n_vols);
  size_t total = 0;
  for (int i = 0; i < n_vols; ++i) {
    Dims d;
    const lt_status st = check_volume(vols[i], &d);
    if (st != LT_OK) {
      delete b;
      return st;
    }
    b->dims.push_back(d);
    b->off.push_back(total);
    total += slice_bytes(d, vols[i].n_labels);
  }
  if (!ws || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0 || ws_bytes < total ||
      device_ptr_ok(ws) != LT_OK) {
    delete b;
    return LT_ERR_WORKSPACE;
  }
  b->ws = reinterpret_cast<char*>(ws);
  cudaGetDevice(&b->device);
  b->branches = std::min(branches, kMaxBranches);
  if (lt_prepare_device() != cudaSuccess || edt_prepare_device() != cudaSuccess) {
    delete b;
    return LT_ERR_CUDA;
  }
  const lt_status st = record(b);
  if (st != LT_OK) {
    lt_batch_destroy(b);
    return st;
  }
  *out = b;
  return LT_OK;
}

lt_status lt_batch_run(lt_batch* b, void* stream) {
  if (!b || !b->exec) return LT_ERR_INVALID_ARG;
  const lt_status st = batch_device_ok(b, stream);
  if (st != LT_OK) return st;
  return cudaGraphLaunch(b->exec, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? LT_OK : LT_ERR_CUDA;
}

lt_status lt_batch_run_eager(lt_batch* b, void* stream) {
  if (!b) return LT_ERR_INVALID_ARG;
  if (const lt_status dst = batch_device_ok(b, stream)) return dst;
  for (size_t i = 0; i < b->vols.size(); ++i) {
    const lt_volume& v = b->vols[i];
    if (measure_launch(v.mask, v.labels, v.n_labels, b->dims[i], b->ws + b->off[i], v.dt2, v.lt2,
                       v.sphericity, v.roundness, reinterpret_cast<cudaStream_t>(stream), b->tu) != cudaSuccess)
      return LT_ERR_CUDA;
  }
  return LT_OK;
}

lt_status lt_batch_status(lt_batch* b, void* stream) {
  if (!b) return LT_ERR_INVALID_ARG;
  if (const lt_status dst = batch_device_ok(b, stream)) return dst;
  lt_status first = LT_OK;
  for (size_t i = 0; i < b->vols.size() && first == LT_OK; ++i) {
    const size_t bytes = measure_ws_bytes(b->dims[i], b->vols[i].n_labels);
    first = lt_workspace_status(b->ws + b->off[i], bytes, stream);
  }
  return first;
}

lt_status lt_batch_autotune(lt_batch* b, void* stream, const char* cache_path) {
  if (!b) return LT_ERR_INVALID_ARG;
  if (const lt_status dst = batch_device_ok(b, stream)) return dst;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, b->device) != cudaSuccess) return LT_ERR_CUDA;
  const std::string key = std::string(prop.name) + "|" + shape_class(b);
  std::vector<CacheEntry> cache = read_cache(cache_path);
  for (const CacheEntry& e : cache)
    if (e.key == key) {
      apply(b, e.v);
      return record(b);
    }
  int best[kSettings];
  current(b, best);
  double best_ms = 0.0;
  lt_status st = time_graph(b, s, 3, &best_ms);
  if (st != LT_OK) return st;
  const std::vector<int> cand[kSettings] = {{1, 2, 4, 8, 16}, {32, 16, 8}, {32, 16, 8}, {8, 16, 32}, {4, 6, 8, 12}};
  for (int axis = 0; axis < kSettings; ++axis) {
    for (int c : cand[axis]) {
      int v[kSettings];
      std::memcpy(v, best, sizeof(v));
      if (v[axis] == c) continue;
      v[axis] = c;
      apply(b, v);
      if ((st = record(b)) != LT_OK) return st;
      double ms = 0.0;
      if ((st = time_graph(b, s, 3, &ms)) != LT_OK) return st;
      if (ms < best_ms) {
        best_ms = ms;
        std::memcpy(best, v, sizeof(best));
      }
    }
  }
  apply(b, best);
  if ((st = record(b)) != LT_OK) return st;
  if (cache_path) {
    CacheEntry e;
    e.key = key;
    std::memcpy(e.v, best, sizeof(best));
    e.ms = best_ms;
    cache.push_back(e);
    write_cache(cache_path, cache);
  }
  return LT_OK;
}

lt_status lt_batch_settings(const lt_batch* b, int32_t out[5]) {
  if (!b || !out) return LT_ERR_INVALID_ARG;
  int v[kSettings];
  current(b, v);
  for (int i = 0; i < kSettings; ++i) out[i] = v[i];
  return LT_OK;
}

void lt_batch_destroy(lt_batch* b) {
  if (!b) return;
  destroy_graph(b);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

}  // extern "C"
