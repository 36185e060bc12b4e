// Batched form: many volumes of uneven size as one CUDA graph launch whose
// stages each run as one kernel launch over all volumes, and its autotuner.
//
// Volumes are grouped by the kernels they need: 3D volumes, and 2D images
// (different templates and, for long 2D columns, a global-memory y pass).
// Volumes whose axes exceed what the shared-memory column tiles hold (over
// 2048) run as single lt_measure chains on extra graph branches. For each
// group a table in device memory (carved from the batch workspace after the
// volumes' own workspaces) holds every volume's parameters, its TMA tensor
// maps, and, per stage, each volume's first CTA in the launch's grid (see
// StagePlan in lt_internal.cuh). The graph then runs, per group on its own
// branch, one launch per stage: clear the headers, EDT rows, y columns, z
// columns, the ridge pass (TMA volumes and plain-load volumes as two
// launches), painting (one persistent grid fed by the union of all volumes'
// centre lists), clear the accumulators, the shape reduction (4-voxel and
// one-voxel forms), the formulas. A stage's kernels see the whole batch, so
// small volumes no longer leave the GPU idle; kernel boundaries are the only
// barriers between stages.
//
// The autotuner changes one setting at a time (EDT column-tile widths, ridge
// z-chunk, paint CTAs per SM, the largest crescent painted in shared
// chunks), re-records the graph for each candidate and takes the median of
// several timed launches; the fastest setting of each pass is kept. Results
// go to a small JSON file keyed by GPU name and the batch's shape class
// (2D/3D counts and the median volume size).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lt_internal.cuh"

using namespace ltk;

namespace {

constexpr int kMaxBranches = 32;
constexpr int kMaxColumn = 2048;  // longest column of the shared-memory EDT tiles
enum Stage {
  kClearHdr,
  kRows,
  kColsY,
  kColsZ,
  kRidgeTma,
  kRidgePlain,
  kClearAcc,
  kReduce4,
  kReduce1,
  kFinalize,
  kStages
};

// Device-table layout of one group: VolParams[n], StagePlan[kStages],
// tensor maps (2 per volume, 128 bytes each), two paint work counters.
struct Group {
  int ndim = 3;
  std::vector<int> vols;  // indices into lt_batch::vols
  size_t off = 0;         // table offset in the batch workspace
  uint32_t blocks[kStages] = {};
  int tx_y = 0, tx_z = 0, max_ny = 0, max_nz = 0;
};

size_t table_bytes(size_t n) {
  return align_up(n * sizeof(VolParams)) + align_up(kStages * sizeof(StagePlan)) + align_up(n * 2 * 128) + kAlign;
}

}  // namespace

struct lt_batch {
  std::vector<lt_volume> vols;
  std::vector<Dims> dims;
  std::vector<size_t> off;  // workspace slice of each volume
  char* ws = nullptr;
  int device = 0;
  int branches = 1;  // branches of the single-chain volumes
  Tuning tu;
  std::vector<Group> groups;
  std::vector<int> single;  // volumes run as lt_measure chains
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

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

// Volumes of the groups (3D volumes whose y and z axes fit the shared-memory
// column tiles; 2D images), the rest run alone.
void plan_groups(const std::vector<Dims>& dims, std::vector<Group>* groups, std::vector<int>* single) {
  groups->clear();
  single->clear();
  Group g3, g2;
  g3.ndim = 3;
  g2.ndim = 2;
  for (int i = 0; i < (int)dims.size(); ++i) {
    const Dims& d = dims[i];
    if (d.ndim == 3 && d.ny <= kMaxColumn && d.nz <= kMaxColumn)
      g3.vols.push_back(i);
    else if (d.ndim == 2)
      g2.vols.push_back(i);
    else
      single->push_back(i);
  }
  // a group's table holds at most kMaxBatchVols volumes: more of one kind
  // are split into that many groups of near-equal size (each on a branch)
  for (Group* g : {&g3, &g2}) {
    const int n = (int)g->vols.size();
    if (n == 0) continue;
    const int parts = (n + kMaxBatchVols - 1) / kMaxBatchVols;
    for (int k = 0; k < parts; ++k) {
      Group part;
      part.ndim = g->ndim;
      part.vols.assign(g->vols.begin() + (int64_t)n * k / parts, g->vols.begin() + (int64_t)n * (k + 1) / parts);
      groups->push_back(part);
    }
  }
}

size_t volumes_bytes(const std::vector<lt_volume>& vols, const std::vector<Dims>& dims) {
  size_t total = 0;
  for (size_t i = 0; i < vols.size(); ++i) total += slice_bytes(dims[i], vols[i].n_labels);
  return total;
}

size_t tables_bytes(const std::vector<Group>& groups) {
  size_t t = 0;
  for (const Group& g : groups) t += table_bytes(g.vols.size());
  return t;
}

VolParams* table_vols(char* ws, const Group& g) { return reinterpret_cast<VolParams*>(ws + g.off); }
StagePlan* table_plans(char* ws, const Group& g) {
  return reinterpret_cast<StagePlan*>(ws + g.off + align_up(g.vols.size() * sizeof(VolParams)));
}
char* table_maps(char* ws, const Group& g) {
  return ws + g.off + align_up(g.vols.size() * sizeof(VolParams)) + align_up(kStages * sizeof(StagePlan));
}
uint32_t* table_ctr(char* ws, const Group& g) {
  return reinterpret_cast<uint32_t*>(table_maps(ws, g) + align_up(g.vols.size() * 2 * 128));
}

// Fills a group's device table for the current tuning (synchronous).
lt_status write_table(lt_batch* b, Group& g) {
  const int n = (int)g.vols.size();
  std::vector<VolParams> vp(n);
  std::vector<StagePlan> plans(kStages);
  std::vector<unsigned char> maps((size_t)n * 2 * 128, 0);
  g.max_ny = g.max_nz = 0;
  for (int k = 0; k < n; ++k) {
    const Dims& d = b->dims[g.vols[k]];
    g.max_ny = std::max(g.max_ny, d.ny);
    g.max_nz = std::max(g.max_nz, d.nz);
  }
  g.tx_y = edt_multi_tx(g.max_ny, b->tu.edt_tx_y);
  g.tx_z = edt_multi_tx(g.max_nz, b->tu.edt_tx_z);
  char* maps_dev = table_maps(b->ws, g);
  for (int k = 0; k < n; ++k) {
    const int i = g.vols[k];
    const lt_volume& v = b->vols[i];
    const Dims& d = b->dims[i];
    VolParams& p = vp[k];
    p.d = d;
    p.n_labels = v.n_labels;
    p.mask = v.mask;
    p.labels = v.labels;
    p.dt2 = v.dt2;
    p.lt2 = v.lt2;
    p.S = v.sphericity;
    p.R = v.roundness;
    p.hdr = reinterpret_cast<WsHeader*>(b->ws + b->off[i]);
    p.body = b->ws + b->off[i] + sizeof(WsHeader);
    const bool tma = lt_ridge_tensor_maps(maps.data() + (size_t)k * 256, maps.data() + (size_t)k * 256 + 128, v.dt2,
                                          v.labels, d);
    p.map_dt2 = tma ? maps_dev + (size_t)k * 256 : nullptr;
    p.map_lab = tma ? maps_dev + (size_t)k * 256 + 128 : nullptr;
    auto count = [](dim3 g3) { return g3.x * g3.y * g3.z; };
    dim3 grid[kStages];
    grid[kClearHdr] = shape_multi_grid(d, v.n_labels, 3);
    grid[kRows] = edt_multi_grid(d, 0, 0);
    grid[kColsY] = edt_multi_grid(d, 1, g.tx_y);
    grid[kColsZ] = d.ndim == 3 ? edt_multi_grid(d, 2, g.tx_z) : dim3(0, 1, 1);
    const dim3 rg = lt_ridge_grid(d, b->tu);
    grid[kRidgeTma] = tma ? rg : dim3(0, 1, 1);
    grid[kRidgePlain] = tma ? dim3(0, 1, 1) : rg;
    grid[kClearAcc] = shape_multi_grid(d, v.n_labels, 4);
    grid[kReduce4] = d.nx % 4 == 0 ? shape_multi_grid(d, v.n_labels, 0) : dim3(0, 1, 1);
    grid[kReduce1] = d.nx % 4 == 0 ? dim3(0, 1, 1) : shape_multi_grid(d, v.n_labels, 1);
    grid[kFinalize] = shape_multi_grid(d, v.n_labels, 2);
    for (int s = 0; s < kStages; ++s) {
      StagePlan& pl = plans[s];
      if (k == 0) pl.start[0] = 0;
      pl.gx[k] = std::max(1u, grid[s].x);
      pl.gy[k] = std::max(1u, grid[s].y);
      pl.start[k + 1] = pl.start[k] + count(grid[s]);
    }
  }
  for (int s = 0; s < kStages; ++s) {
    g.blocks[s] = plans[s].start[n];
    if (g.blocks[s] > 0x7FFFFFFFu) return LT_ERR_DIMS;
  }
  if (cudaMemcpy(table_vols(b->ws, g), vp.data(), n * sizeof(VolParams), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(table_plans(b->ws, g), plans.data(), kStages * sizeof(StagePlan), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(maps_dev, maps.data(), maps.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return LT_ERR_CUDA;
  return LT_OK;
}

// The stage launches of one group on stream s.
cudaError_t launch_group(lt_batch* b, const Group& g, cudaStream_t s) {
  MultiArgs m[kStages];
  for (int k = 0; k < kStages; ++k) m[k] = MultiArgs{table_vols(b->ws, g), table_plans(b->ws, g) + k, (int)g.vols.size()};
  const int nd = g.ndim;
  cudaError_t e = cudaMemsetAsync(table_ctr(b->ws, g), 0, 2 * sizeof(uint32_t), s);
  if (e == cudaSuccess) e = shape_multi_launch(m[kClearHdr], g.blocks[kClearHdr], 3, nd, s);
  if (e == cudaSuccess) e = edt_multi_launch(m[kRows], g.blocks[kRows], 0, 0, 0, s);
  if (e == cudaSuccess) e = edt_multi_launch(m[kColsY], g.blocks[kColsY], 1, g.tx_y, g.max_ny, s);
  if (e == cudaSuccess && nd == 3) e = edt_multi_launch(m[kColsZ], g.blocks[kColsZ], 2, g.tx_z, g.max_nz, s);
  if (e == cudaSuccess) e = lt_ridge_multi_launch(m[kRidgeTma], g.blocks[kRidgeTma], nd, true, b->tu, s);
  if (e == cudaSuccess) e = lt_ridge_multi_launch(m[kRidgePlain], g.blocks[kRidgePlain], nd, false, b->tu, s);
  if (e == cudaSuccess) e = lt_paint_multi_launch(m[kRidgeTma], nd, table_ctr(b->ws, g), b->tu, s);
  if (e == cudaSuccess) e = shape_multi_launch(m[kClearAcc], g.blocks[kClearAcc], 4, nd, s);
  if (e == cudaSuccess) e = shape_multi_launch(m[kReduce4], g.blocks[kReduce4], 0, nd, s);
  if (e == cudaSuccess) e = shape_multi_launch(m[kReduce1], g.blocks[kReduce1], 1, nd, s);
  if (e == cudaSuccess) e = shape_multi_launch(m[kFinalize], g.blocks[kFinalize], 2, nd, s);
  return e;
}

void destroy_graph(lt_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// Records the batch into a graph: each group on a branch of its own, the
// single-chain volumes on b->branches more (largest first to the least
// loaded).
lt_status record(lt_batch* b) {
  // earlier launches of the old graph read the tables rewritten below
  if (cudaDeviceSynchronize() != cudaSuccess) return LT_ERR_CUDA;
  destroy_graph(b);
  for (Group& g : b->groups) {
    const lt_status st = write_table(b, g);
    if (st != LT_OK) return st;
  }
  const int ng = (int)b->groups.size();
  const int nb = b->single.empty() ? 0 : std::min(b->branches, (int)b->single.size());
  while ((int)b->streams.size() < ng + nb + 1) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return LT_ERR_CUDA;
    b->streams.push_back(s);
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return LT_ERR_CUDA;
    b->join.push_back(e);
  }
  if (!b->fork && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) return LT_ERR_CUDA;
  std::vector<int> order = b->single;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return b->dims[x].n > b->dims[y].n; });
  std::vector<double> load(nb, 0.0);
  std::vector<int> branch(b->vols.size(), 0);
  for (int i : order) {
    const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    branch[i] = k;
    load[k] += (double)b->dims[i].n;
  }
  cudaStream_t cap = b->streams[ng + nb];
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return LT_ERR_CUDA;
  cudaError_t e = cudaEventRecord(b->fork, cap);
  for (int k = 0; k < ng + nb && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->streams[k], b->fork, 0);
  for (int k = 0; k < ng && e == cudaSuccess; ++k) e = launch_group(b, b->groups[k], b->streams[k]);
  for (int i : order) {
    if (e != cudaSuccess) break;
    const lt_volume& v = b->vols[i];
    e = measure_launch(v.mask, v.labels, v.n_labels, b->dims[i], b->ws + b->off[i], v.dt2, v.lt2, v.sphericity,
                       v.roundness, b->streams[ng + branch[i]], b->tu);
  }
  for (int k = 0; k < ng + nb && e == cudaSuccess; ++k) {
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

// ---- minimal JSON cache: {"key": {"edt_tx_y": 8, ...}, ...}
constexpr int kSettings = 5;  // EDT y and z tile widths, ridge z-chunk, paint CTAs/SM, chunk crescent bound
const char* const kSettingNames[kSettings] = {"\"edt_tx_y\"", "\"edt_tx_z\"", "\"ridge_z\"", "\"paint_bpsm\"",
                                              "\"chunk_cres\""};
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
      const size_t p = body.find(kSettingNames[i]);
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
    std::fprintf(f, "  \"%s\": {", e.key.c_str());
    for (int k = 0; k < kSettings; ++k) std::fprintf(f, "%s: %d, ", kSettingNames[k], e.v[k]);
    std::fprintf(f, "\"ms\": %.4f}%s\n", e.ms, i + 1 < entries.size() ? "," : "");
  }
  std::fprintf(f, "}\n");
  std::fclose(f);
  return std::rename(tmp.c_str(), path) == 0;
}

void apply(lt_batch* b, const int v[kSettings]) {
  b->tu.edt_tx_y = v[0] == 8 || v[0] == 16 ? v[0] : 32;
  b->tu.edt_tx_z = v[1] == 8 || v[1] == 16 ? v[1] : 32;
  b->tu.ridge_z = v[2] == 8 || v[2] == 32 ? v[2] : 16;
  b->tu.paint_blocks_per_sm = std::max(1, std::min(32, v[3]));
  b->tu.chunk_cres = std::max(8, std::min(1024, v[4]));
}

void current(const lt_batch* b, int v[kSettings]) {
  v[0] = b->tu.edt_tx_y;
  v[1] = b->tu.edt_tx_z;
  v[2] = b->tu.ridge_z;
  v[3] = b->tu.paint_blocks_per_sm;
  v[4] = b->tu.chunk_cres;
}

// median ms of `reps` graph launches, each timed alone (after one warm-up)
lt_status time_graph(lt_batch* b, cudaStream_t s, int reps, double* ms) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return LT_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return LT_ERR_CUDA;
  }
  cudaError_t e = cudaGraphLaunch(b->exec, s);
  std::vector<double> t;
  for (int i = 0; i < reps && e == cudaSuccess; ++i) {
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float x = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&x, e0, e1);
    t.push_back(x);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || t.empty()) return LT_ERR_CUDA;
  std::sort(t.begin(), t.end());
  *ms = t[t.size() / 2];
  return LT_OK;
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
  std::vector<lt_volume> v(vols, vols + n_vols);
  std::vector<Dims> dims;
  for (int i = 0; i < n_vols; ++i) {
    Dims d;
    if (make_dims_checked(vols[i].ndim, vols[i].nx, vols[i].ny, vols[i].nz, &d) != LT_OK) return 0;
    dims.push_back(d);
  }
  std::vector<Group> groups;
  std::vector<int> single;
  plan_groups(dims, &groups, &single);
  return volumes_bytes(v, dims) + tables_bytes(groups);
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
  plan_groups(b->dims, &b->groups, &b->single);
  for (Group& g : b->groups) {
    g.off = total;
    total += table_bytes(g.vols.size());
  }
  if (!ws || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0 || ws_bytes < total || device_ptr_ok(ws) != LT_OK) {
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
                       v.sphericity, v.roundness, reinterpret_cast<cudaStream_t>(stream), Tuning()) != cudaSuccess)
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
  constexpr int kReps = 5;
  int best[kSettings];
  current(b, best);
  double best_ms = 0.0;
  lt_status st = time_graph(b, s, kReps, &best_ms);
  if (st != LT_OK) return st;
  const std::vector<int> cand[kSettings] = {{32, 16, 8}, {32, 16, 8}, {8, 16, 32}, {4, 6, 8}, {32, 48, 64, 96, 128}};
  for (int axis = 0; axis < kSettings; ++axis) {
    for (int c : cand[axis]) {
      int v[kSettings];
      std::memcpy(v, best, sizeof(v));
      if (v[axis] == c) continue;
      v[axis] = c;
      apply(b, v);
      if ((st = record(b)) != LT_OK) return st;
      double ms = 0.0;
      if ((st = time_graph(b, s, kReps, &ms)) != LT_OK) return st;
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
