/*
 * lt.h — C ABI of the GB300 (sm_103a) local-thickness shape library.
 *
 * Method: "Fast Sphericity and Roundness approximation in 2D and 3D using
 * Local Thickness" (Pieta, Rasmussen, Dahl, Christensen). A labelled mask
 * goes through
 *     lt_edt              exact squared Euclidean distance transform,
 *     lt_local_thickness  exact local thickness (squared radius),
 *     lt_shape_measures   per-object sphericity S_LT and roundness R_LT,
 * each a sequence of hand-written CUDA kernels. lt_measure runs all three.
 *
 * Conventions shared by every call
 *   Layout      C order [z][y][x], x fastest. ndim = 2 requires nz = 1 and
 *               treats the array as an (ny, nx) image; ndim = 3 is a volume.
 *   Limits      1 <= nx, ny, nz <= 8192 and nx * ny * nz < 2^32, so that
 *               every squared distance is below 2^24 and every voxel index
 *               fits in 32 bits. Violations return LT_ERR_DIMS.
 *   Pointers    Device pointers unless the name ends in _host. Device buffers
 *               are owned by the caller and must be 16-byte aligned.
 *   Device      Every device pointer, the workspace and the stream must
 *               belong to the calling thread's current device. The library
 *               never changes the current device; a pointer or stream of
 *               another device returns LT_ERR_INVALID_ARG before anything is
 *               enqueued.
 *   Workspace   Scratch memory is always passed in by the caller (`ws`,
 *               `ws_bytes`, 256-byte aligned); the library allocates nothing.
 *               Size it with the matching *_workspace_size function. A
 *               workspace may be reused across calls on the same stream;
 *               concurrent calls need distinct workspaces.
 *   Streams     `stream` is a cudaStream_t (NULL = the legacy default
 *               stream). Device-pointer calls only enqueue work and return;
 *               argument errors are returned immediately and nothing is
 *               enqueued. Errors that only the device can see (a label out of
 *               range, a labelled voxel outside the mask, a wait limit
 *               reached) are recorded in the workspace; read them with
 *               lt_workspace_status.
 *   Threads     Calls are thread-safe as long as they use distinct
 *               workspaces and outputs.
 *
 * Definitions (the paper's Sec. 1 and Sec. 4)
 *   Foreground  mask != 0. Everything outside the array counts as background
 *               (the array is padded by one background layer).
 *   DT2(p)      min |p - b|^2 over background b; 0 on background.
 *   Object l    the voxels with label l != 0. Labels must be 0 wherever the
 *               mask is 0 (checked on the device). Foreground voxels with
 *               label 0 shape the distance transform but belong to no object.
 *   LT2(x)      the local thickness squared: the largest DT2(c) over centres
 *               c of x's object whose inclusive ball |x - c|^2 <= DT2(c)
 *               holds x (local thickness = radius of the largest inscribed
 *               ball containing x); 0 outside every object.
 *   Shell       object voxels with a face neighbour (4 in 2D, 6 in 3D)
 *               outside the object: another label, background, or outside
 *               the array (Sec. 4.2).
 */
#ifndef LT_H
#define LT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lt_status {
  LT_OK = 0,
  LT_ERR_INVALID_ARG = 1,         /* null, misaligned or other-device pointer, bad ndim */
  LT_ERR_DIMS = 2,                /* dimensions outside the limits above */
  LT_ERR_WORKSPACE = 3,           /* workspace missing, too small or misaligned */
  LT_ERR_LABEL_RANGE = 4,         /* device-detected: a label >= n_labels */
  LT_ERR_LABEL_OUTSIDE_MASK = 5,  /* device-detected: label != 0 where mask == 0 */
  LT_ERR_CUDA = 6,                /* a CUDA call or kernel launch failed */
  LT_ERR_NO_DEVICE = 7,           /* no usable sm_103 device */
  LT_ERR_TIMEOUT = 8,             /* device-detected: an asynchronous copy did not arrive
                                     within a kernel's wait limit (the kernel stopped early;
                                     outputs are invalid) */
  LT_ERR_CHECKPOINT = 9           /* checkpoint file unreadable, of another format or
                                     network shape, or corrupt (CRC mismatch) */
} lt_status;

/* Per-object sums, one entry per label (structure of arrays, device memory).
 * sum_lt and sum_shell_lt are fixed point: the sum over voxels of
 * round(sqrtf(LT2) * 2^20), sqrtf the IEEE single-precision square root (so
 * each term is within 2^-24 relative plus 2^-21 absolute of the exact LT
 * times 2^20; the sums are exact integers, independent of summation order). */
typedef struct lt_object_stats {
  uint32_t* volume;        /* voxel (pixel) count V (area A in 2D) */
  uint32_t* n_shell;       /* shell voxel count */
  uint32_t* max_lt2;       /* largest LT2 of the object (= largest DT2) */
  uint64_t* sum_lt;        /* fixed point, scale 2^20 */
  uint64_t* sum_shell_lt;  /* fixed point, scale 2^20 */
} lt_object_stats;

#define LT_FIXED_POINT_SHIFT 20

/* Short English name of a status code (static storage). */
const char* lt_status_string(lt_status status);

/* Library version, e.g. 0x000100 for 0.1.0. */
uint32_t lt_version(void);

/* ------------------------------------------------------------------ EDT --
 * Exact squared Euclidean distance transform of `mask` (uint8, nonzero =
 * foreground) into `dt2` (uint32, DT2 as defined above; 0 on background).
 * Three separable passes: a row pass along x (distance to the nearest
 * background in the row, exact integer), then the lower envelope of the
 * parabolas f(q) + (p - q)^2 along y and (3D) along z, with the padding
 * layer entering as two zero-height parabolas at -1 and n. All arithmetic is
 * exact integer arithmetic, so the result is bit-exact.
 * Workspace: lt_edt_workspace_size bytes: 2 bytes per voxel (the row pass
 * leaves 16-bit distances there for the y pass), plus 4 bytes per voxel in
 * 3D when nz > 2048 (columns longer than 2048 do not fit in shared memory;
 * that z pass goes out of place). */
size_t lt_edt_workspace_size(int ndim, int64_t nx, int64_t ny, int64_t nz);
lt_status lt_edt(const uint8_t* mask, uint32_t* dt2, int ndim, int64_t nx, int64_t ny, int64_t nz,
                 void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------- local thickness --
 * Exact local thickness squared, LT2 as defined above, from `dt2` (output of
 * lt_edt) and `labels` (uint32) into `lt2` (uint32). Bit-exact.
 * Centres whose ball lies inside a same-label neighbour's ball of larger
 * radius are dropped (an exact digital-ball containment test by lookup
 * table); every other centre raises LT2 (atomic max) only on the voxels of
 * its ball that one chosen higher-ranked neighbour's ball does not hold.
 * Neither step changes the maximum (proof in the kernel source).
 * Device-detected error: LT_ERR_LABEL_OUTSIDE_MASK.
 * Workspace: lt_local_thickness_workspace_size bytes (18 bytes per voxel for
 * the centre list: up to one 16-byte record per voxel, plus part records of
 * big balls that several warps share). The first call on a device also copies lookup tables
 * (about 26 MiB, built once per process on the host) into device memory
 * owned by the library; make that first call before any stream capture. */
size_t lt_local_thickness_workspace_size(int ndim, int64_t nx, int64_t ny, int64_t nz);
lt_status lt_local_thickness(const uint32_t* dt2, const uint32_t* labels, uint32_t* lt2, int ndim,
                             int64_t nx, int64_t ny, int64_t nz, void* ws, size_t ws_bytes,
                             void* stream);

/* ------------------------------------------------ scaled local thickness --
 * Approximate LT2 at 1/scale resolution: the reduced-resolution option of
 * the fast local-thickness work the paper builds on (Sec. 1, Sec. 4),
 * trading accuracy for speed. From `mask` and `labels` (full resolution):
 *   sample   low-res voxel B (ceil(n/scale) per axis) takes mask and label of
 *            the full-res voxel min(scale*B + scale/2, n-1) per axis;
 *   exact    DT2 and LT2 of the low-res volume (as lt_edt and
 *            lt_local_thickness compute them);
 *   upsample object voxel x of label l, block B = x / scale:
 *            scale^2 * LT2_low(B) when B has label l, else the largest
 *            scale^2 * LT2_low over the blocks B + d (|d|_inf <= 1) with
 *            label l, else 1; 0 outside every object.
 * into `lt2` (full resolution, usable by lt_shape_measures). scale 1 gives
 * the exact LT2. 1 <= scale <= 8. Device-detected error:
 * LT_ERR_LABEL_OUTSIDE_MASK. Workspace: lt_local_thickness_scaled_workspace_size
 * bytes (about 29/scale^ndim bytes per voxel). */
size_t lt_local_thickness_scaled_workspace_size(int scale, int ndim, int64_t nx, int64_t ny, int64_t nz);
lt_status lt_local_thickness_scaled(const uint8_t* mask, const uint32_t* labels, int scale, uint32_t* lt2,
                                    int ndim, int64_t nx, int64_t ny, int64_t nz, void* ws, size_t ws_bytes,
                                    void* stream);

/* --------------------------------------------------------- shape measures --
 * Per-object sphericity and roundness from `labels` and `lt2` (as produced by
 * lt_local_thickness) for labels 0 .. n_labels-1.
 *   3D (Eqs. 1, 6-8): a = mean LT over the object, c = 3V / (4 pi a^2);
 *      spheroid area with e = sqrt(1 - c^2/a^2) (c < a) or
 *      e = sqrt(1 - a^2/c^2) (c > a), 4 pi a^2 at c = a;
 *      S = pi^(1/3) (6V)^(2/3) / area.
 *   2D (Eqs. 2, 9-11): a = mean LT, b = A / (pi a), Ramanujan's
 *      P_o = pi (3(a + b) - sqrt((3a + b)(a + 3b))), P_c = 2 sqrt(pi A),
 *      S = P_c / P_o.
 *   R (Sec. 4.2) = (mean LT over the shell) / sqrt(max LT2).
 * Outputs `sphericity[n_labels]`, `roundness[n_labels]` (float, device; NaN
 * for label 0 and for labels with no voxel); either may be NULL. `stats` may
 * be NULL; when given, its arrays (device, n_labels entries each) receive the
 * per-object sums. The sums are exact integers and the formulas run in FP64;
 * the result is within 1e-6 relative of an FP64 evaluation with exact sums.
 * Device-detected error: LT_ERR_LABEL_RANGE (such voxels are skipped).
 * Workspace: lt_shape_workspace_size bytes (28 bytes per label + 256). */
size_t lt_shape_workspace_size(uint32_t n_labels);
lt_status lt_shape_measures(const uint32_t* labels, const uint32_t* lt2, uint32_t n_labels, int ndim,
                            int64_t nx, int64_t ny, int64_t nz, void* ws, size_t ws_bytes,
                            float* sphericity, float* roundness, const lt_object_stats* stats,
                            void* stream);

/* ---------------------------------------------- post-processing of R, S --
 * lt_shape_measures_filtered: lt_shape_measures after roughness filtering.
 *   The paper expects surface roughness to be controllable by filtering
 *   the contour/surface (Sec. 7) and names no filter; this library's filter
 *   keeps, of every object, the voxels whose local thickness is at least
 *   sqrt(min_lt2), i.e. the union of its inscribed balls of squared radius
 *   >= min_lt2 (an opening of the object by a ball), and measures S, R and
 *   the sums on what remains: voxels below the threshold count as outside
 *   their object (also for the shell test). Features thinner than the
 *   threshold radius disappear; objects entirely below it give NaN.
 *   min_lt2 <= 1 filters nothing (every object voxel has LT2 >= 1), so the
 *   result equals lt_shape_measures. Same arguments, workspace and errors.
 * lt_roundness_rescale: R_LT never exceeds 1 and stays above 0 (Sec. 6.1);
 *   with its minimum m it maps onto 0-1: out = max(0, (R - m) / (1 - m)).
 *   m = r_min when r_min >= 0 (a reference minimum, e.g. from another
 *   population; values below it map to 0), else the smallest finite value
 *   of roundness[0..n). NaN stays NaN; m >= 1 gives 1. Device arrays of n
 *   floats (out may alias roundness); workspace:
 *   lt_roundness_rescale_workspace_size() bytes. r_min NaN is rejected. */
lt_status lt_shape_measures_filtered(const uint32_t* labels, const uint32_t* lt2, uint32_t n_labels,
                                     uint32_t min_lt2, int ndim, int64_t nx, int64_t ny, int64_t nz, void* ws,
                                     size_t ws_bytes, float* sphericity, float* roundness,
                                     const lt_object_stats* stats, void* stream);
size_t lt_roundness_rescale_workspace_size(void);
lt_status lt_roundness_rescale(const float* roundness, uint32_t n, float r_min, float* out, void* ws,
                               size_t ws_bytes, void* stream);

/* ---------------------------------------------------------- batched form --
 * Many volumes (2D and 3D, uneven sizes) measured as one unit of work. The
 * batch owns no device memory: `ws` (lt_batch_workspace_size bytes) holds
 * every volume's workspace and the batch's device tables. lt_batch_create
 * checks the volumes, copies the lookup tables to the device if needed and
 * records the batch into a CUDA graph in which every stage of lt_measure is
 * one kernel launch over all volumes of a group (3D volumes; 2D images):
 * per-volume parameters and each volume's first CTA of every stage sit in a
 * device table, and painting is one persistent grid fed by the union of all
 * volumes' centre lists. The groups run on parallel branches; volumes with an
 * axis over 2048 (beyond the shared-memory column tiles) run as single
 * lt_measure chains on `branches` further branches. Results equal single
 * lt_measure calls bit for bit. lt_batch_run launches the graph on `stream`
 * (one launch per batch); lt_batch_run_eager issues lt_measure volume after
 * volume on `stream`, the per-volume baseline. lt_batch_status waits for
 * `stream` and returns the first device-detected error of any volume.
 * lt_batch_autotune times candidate settings on the batch itself (the median
 * of five graph launches each), one setting at a time from the defaults,
 * keeps the fastest and re-records the graph (this waits for the device);
 * results are cached in the JSON file `cache_path` (NULL: no cache) under the
 * GPU name and the batch's shape class, and a cached entry is reused without
 * timing. The batch and its graph are host objects: lt_batch_destroy
 * releases them. Host-side calls (create, autotune, destroy) are not
 * thread-safe for the same batch. */
typedef struct lt_volume {
  int32_t ndim;
  uint32_t n_labels;
  int64_t nx, ny, nz;
  const uint8_t* mask;
  const uint32_t* labels;
  uint32_t* dt2;
  uint32_t* lt2;
  float* sphericity;
  float* roundness;
} lt_volume;
typedef struct lt_batch lt_batch;
size_t lt_batch_workspace_size(const lt_volume* vols, int n_vols);
lt_status lt_batch_create(const lt_volume* vols, int n_vols, void* ws, size_t ws_bytes, int branches,
                          lt_batch** batch);
lt_status lt_batch_run(lt_batch* batch, void* stream);
lt_status lt_batch_run_eager(lt_batch* batch, void* stream);
lt_status lt_batch_status(lt_batch* batch, void* stream);
lt_status lt_batch_autotune(lt_batch* batch, void* stream, const char* cache_path);
/* current settings: EDT y and z column-tile widths, ridge z-chunk, paint CTAs
 * per SM, largest crescent (voxels) painted in shared chunks of 32 centres */
lt_status lt_batch_settings(const lt_batch* batch, int32_t out[5]);
void lt_batch_destroy(lt_batch* batch);

/* ------------------------------------------------ learned sphericity --
 * A correction of S_LT toward the strict (mesh) sphericity of Eq. 1 by a
 * small network; the paper has none, so its definition is this library's:
 *
 * lt_object_features: 48 features per object into `features`
 *   ([n_labels][48] float, device), from labels, lt2, the per-object sums of
 *   lt_shape_measures (`stats`, all five arrays required) and its outputs
 *   S_LT and R_LT. Index: 0 log(V)/10, 1 log(n_shell)/10, 2 log(M)/4 with
 *   M = sqrt(max LT2), 3 (mean LT)/M, 4 R_LT, 5 S_LT, 6-21 the fraction of
 *   interior (non-shell) voxels whose LT/M falls in bin b (the largest b in
 *   0..15 with b^2 * max LT2 <= 256 * LT2), 22-37 the same over the shell,
 *   38-47 zero. Rows of empty labels (and label 0) are zero. One extra pass
 *   over the volume. Workspace: lt_features_workspace_size (128 bytes per
 *   label + 256).
 * Network: 48 -> 64 -> 64 -> 1 with ReLU, parameters in one FP32 vector of
 *   LT_MLP_PARAMS floats laid out W1[48][64], b1[64], W2[64][64], b2[64],
 *   w3[64], b3 (W[i][j]: input i to output j). Inputs, weights and hidden
 *   activations are rounded to BF16; sums run in FP32.
 * lt_mlp_infer: s_learned[o] = clamp(sphericity[o] + net(features[o]), 0, 1)
 *   for o < n (NaN where sphericity is NaN). Device pointers.
 * lt_mlp_gradients: for the batch batch_idx[0..batch), the gradient (device,
 *   LT_MLP_PARAMS floats) of the mean over the batch of
 *   (sphericity + net(features) - target)^2 with respect to the FP32
 *   parameters (straight through the BF16 roundings), and the loss (device
 *   float, may be NULL). The sum over the batch runs in a fixed order, so
 *   the result is deterministic. Workspace: lt_mlp_train_workspace_size.
 * lt_mlp_adam: one Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias
 *   corrected; `step` counts from 1) on params with moments m and v.
 * lt_mlp_train_step: lt_mlp_gradients then lt_mlp_adam; `grad` is scratch
 *   of LT_MLP_PARAMS floats. */
#define LT_MLP_FEATURES 48
#define LT_MLP_HIDDEN 64
#define LT_MLP_PARAMS 7361
/* Checkpoints of the network and its optimiser (no handle: the network is
 * the caller's parameter vector, the optimiser state its two moment vectors
 * and the step count). A checkpoint is lt_mlp_checkpoint_size() bytes,
 * little-endian: the 8 bytes "LTMLPCK1"; uint32 format version (1),
 * LT_MLP_FEATURES, LT_MLP_HIDDEN, LT_MLP_PARAMS, the Adam step, flags (bit
 * 0: moments stored); float32 params, m, v (LT_MLP_PARAMS each, zeros when
 * no moments are stored); the CRC-32 (IEEE 802.3, as zlib's crc32) of all
 * bytes before it. Restoring all three vectors and the step and continuing
 * with the same batches reproduces an uninterrupted run bit for bit.
 * lt_mlp_checkpoint_pack / _unpack: host buffers only (no GPU needed); m and
 *   v are given together or both NULL (pack: no moments stored; unpack: not
 *   read). unpack returns LT_ERR_CHECKPOINT for a wrong size, magic,
 *   version or network shape, a CRC mismatch, or moments requested from a
 *   checkpoint that has none; params and step may be NULL.
 * lt_mlp_save / lt_mlp_load: the same with device vectors (LT_MLP_PARAMS
 *   floats each) and a file: save copies them to the host on `stream`,
 *   waits, and writes `path` (through a temporary file renamed into
 *   place); load reads and checks `path`, then copies to the device on
 *   `stream` and waits. File errors return LT_ERR_CHECKPOINT. */
size_t lt_mlp_checkpoint_size(void);
lt_status lt_mlp_checkpoint_pack(const float* params_host, const float* m_host, const float* v_host,
                                 uint32_t step, void* out_host, size_t out_bytes);
lt_status lt_mlp_checkpoint_unpack(const void* in_host, size_t in_bytes, float* params_host, float* m_host,
                                   float* v_host, uint32_t* step);
lt_status lt_mlp_save(const char* path, const float* params, const float* m, const float* v, uint32_t step,
                      void* stream);
lt_status lt_mlp_load(const char* path, float* params, float* m, float* v, uint32_t* step, void* stream);

size_t lt_features_workspace_size(uint32_t n_labels);
lt_status lt_object_features(const uint32_t* labels, const uint32_t* lt2, uint32_t n_labels, int ndim,
                             int64_t nx, int64_t ny, int64_t nz, const lt_object_stats* stats,
                             const float* sphericity, const float* roundness, void* ws, size_t ws_bytes,
                             float* features, void* stream);
lt_status lt_mlp_infer(const float* params, const float* features, const float* sphericity, uint32_t n,
                       float* s_learned, void* stream);
size_t lt_mlp_train_workspace_size(uint32_t batch);
lt_status lt_mlp_gradients(const float* params, const float* features, const float* sphericity,
                           const float* target, const uint32_t* batch_idx, uint32_t batch, void* ws,
                           size_t ws_bytes, float* grad, float* loss, void* stream);
lt_status lt_mlp_adam(float* params, float* m, float* v, const float* grad, uint32_t step, float lr,
                      void* stream);
lt_status lt_mlp_train_step(float* params, float* m, float* v, float* grad, uint32_t step, float lr,
                            const float* features, const float* sphericity, const float* target,
                            const uint32_t* batch_idx, uint32_t batch, void* ws, size_t ws_bytes,
                            float* loss, void* stream);

/* ------------------------------------------- shape measures, no allocation --
 * Same computation and outputs as lt_shape_measures, for callers that cannot
 * allocate device memory: code that receives device buffers from another
 * framework but has no allocator of its own (plugins, callbacks inside
 * someone else's pipeline), and latency-critical loops that must not call
 * cudaMalloc after start-up because it can synchronise the whole device.
 * The paper has no counterpart; this is a deployment convenience.
 * Scratch: a fixed array in device memory that belongs to the library (every
 * GPU that loads the library holds it until the process exits), large enough
 * for LT_STATIC_MAX_LABELS labels. n_labels above that returns
 * LT_ERR_WORKSPACE without enqueuing anything.
 * The first call on each device looks up the array's device address (a
 * one-time set-up); make that first call before any stream capture.
 * All calls share the one array: calls that may overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * Labels >= n_labels are skipped but, unlike lt_shape_measures, not reported. */
#define LT_STATIC_MAX_LABELS 131072u
lt_status lt_shape_measures_static(const uint32_t* labels, const uint32_t* lt2, uint32_t n_labels,
                                   int ndim, int64_t nx, int64_t ny, int64_t nz, float* sphericity,
                                   float* roundness, const lt_object_stats* stats, void* stream);

/* ------------------------------------------------------------- pipeline --
 * lt_edt, lt_local_thickness and lt_shape_measures in sequence on one
 * workspace. dt2 and lt2 are outputs (device, one uint32 per voxel each). */
size_t lt_measure_workspace_size(uint32_t n_labels, int ndim, int64_t nx, int64_t ny, int64_t nz);
lt_status lt_measure(const uint8_t* mask, const uint32_t* labels, uint32_t n_labels, int ndim,
                     int64_t nx, int64_t ny, int64_t nz, void* ws, size_t ws_bytes, uint32_t* dt2,
                     uint32_t* lt2, float* sphericity, float* roundness, void* stream);

/* lt_measure plus the learned correction's features (see lt_object_features
 * for their definition) in the same shape pass: the ridge pass of local
 * thickness also takes every object's largest DT2 (which equals its largest
 * LT2), so the shape pass bins the LT / max-LT histograms next to the sums
 * instead of a second pass over labels and LT2. Outputs as lt_measure plus
 * `features` ([n_labels][48] float, device, required) and, when `stats` is
 * given, the per-object sums. Feed features and sphericity to lt_mlp_infer.
 * Workspace: lt_measure_features_workspace_size bytes (lt_measure's plus
 * 132 bytes per label). */
size_t lt_measure_features_workspace_size(uint32_t n_labels, int ndim, int64_t nx, int64_t ny, int64_t nz);
lt_status lt_measure_features(const uint8_t* mask, const uint32_t* labels, uint32_t n_labels, int ndim, int64_t nx,
                              int64_t ny, int64_t nz, void* ws, size_t ws_bytes, uint32_t* dt2, uint32_t* lt2,
                              float* sphericity, float* roundness, float* features, const lt_object_stats* stats,
                              void* stream);

/* Slab form of lt_measure for volumes held in host memory whose working set
 * does not fit the device (or a budget on it): the device works on
 * `slab_planes` z planes at a time (workspace ~30 bytes per voxel of a slab,
 * lt_measure_slabs_workspace_size). Results equal lt_measure's bit for bit.
 * Phases: x/y EDT passes per slab (the y pass's output goes to dt2_host);
 * the z pass per band of rows over all z (2D copies, in place in dt2_host,
 * which then holds DT2); local thickness and the shape sums per core slab,
 * uploaded with H + 1 planes on each side, H = ceil(sqrt(max DT2)) (a ball
 * holding a core voxel has its centre within H planes); the formulas once.
 * 3D only. Host buffers: mask_host, labels_host (inputs, n voxels),
 * dt2_host (n uint32, required: scratch, then DT2), lt2_host (n uint32 or
 * NULL), sphericity_host and roundness_host (n_labels floats); pinned memory
 * copies fastest. Axes up to 8192, the smallest at most 8190 (DT2 < 2^24);
 * n itself may exceed 2^32; slab_planes * nx * ny < 2^32. Waits for the
 * stream. LT_ERR_WORKSPACE also when the objects are too thick for the slab
 * (2 H + 3 > slab_planes): use more planes. */
size_t lt_measure_slabs_workspace_size(uint32_t n_labels, int64_t nx, int64_t ny, int64_t nz, int slab_planes);
lt_status lt_measure_slabs(const uint8_t* mask_host, const uint32_t* labels_host, uint32_t n_labels, int64_t nx,
                           int64_t ny, int64_t nz, int slab_planes, uint32_t* dt2_host, uint32_t* lt2_host,
                           float* sphericity_host, float* roundness_host, void* ws, size_t ws_bytes,
                           void* stream);

/* Host-buffer form of lt_measure for callers whose data lives in host memory:
 * copies mask_host and labels_host to the device, runs the pipeline, copies
 * sphericity_host and roundness_host (n_labels floats each) back and waits
 * for the stream. Host buffers should be pinned for full copy speed. The
 * device copies of the inputs, DT2 and LT2 live in `ws` (device memory,
 * lt_measure_host_workspace_size bytes). Returns device-detected errors too. */
size_t lt_measure_host_workspace_size(uint32_t n_labels, int ndim, int64_t nx, int64_t ny, int64_t nz);
lt_status lt_measure_host(const uint8_t* mask_host, const uint32_t* labels_host, uint32_t n_labels,
                          int ndim, int64_t nx, int64_t ny, int64_t nz, void* ws, size_t ws_bytes,
                          float* sphericity_host, float* roundness_host, void* stream);

/* ------------------------------------------------------------- tracing --
 * Kernel timing for profiling. While tracing is enabled, the library records
 * a CUDA event on the launch stream before and after every kernel it
 * launches (events come from a pool created on first use, so tracing can
 * stay on inside timed loops). lt_trace_enable(1) clears earlier records;
 * lt_trace_enable(0) stops recording. lt_trace_summary waits for the
 * recorded events, then writes up to max_entries per-kernel totals (name,
 * launches, summed event time in ms) and returns the number of distinct
 * kernels seen (negative on a CUDA error). Not meant for use while a stream
 * is being captured into a CUDA graph. */
typedef struct lt_trace_entry {
  char name[40];
  uint32_t launches;
  double total_ms;
} lt_trace_entry;
lt_status lt_trace_enable(int enable);
int lt_trace_summary(lt_trace_entry* out, int max_entries);

/* Waits for `stream`, then returns the first device-detected error recorded
 * in `ws` since the last call that used it (LT_OK if none). */
lt_status lt_workspace_status(const void* ws, size_t ws_bytes, void* stream);

/* Work counters of the last lt_local_thickness (or lt_measure) that used
 * `ws`, after waiting for `stream`: centres kept by the containment test,
 * painted by warps sharing chunks of 32 centres (chunk_centres) or by one
 * warp each (warp_centres: big crescents and balls painted row by row), and
 * the LT2 updates (32-bit atomic max) the painting issued, in total and from
 * crescent tables. */
typedef struct lt_lt_counters {
  uint32_t chunk_centres;
  uint32_t warp_centres;
  uint64_t updates;
  uint64_t table_updates;
} lt_lt_counters;
lt_status lt_workspace_counters(const void* ws, size_t ws_bytes, void* stream, lt_lt_counters* out);

/* Self-test of failure detection: runs the local-thickness ridge kernel
 * (the one kernel that waits, on its shared-memory copies) on a 32 x 8 x 8
 * all-background volume carved from `ws`, with every copy barrier expecting
 * 16 bytes more than its copies deliver, so that each wait reaches its limit
 * (1 ms here). The kernel records the timeout in `ws` and returns; this
 * function waits for `stream` and returns what lt_workspace_status reads:
 * LT_ERR_TIMEOUT when the limit works. No copy is left in flight and the
 * context stays usable. Workspace: lt_selftest_workspace_size() bytes. */
size_t lt_selftest_workspace_size(void);
lt_status lt_selftest_wait_timeout(void* ws, size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LT_H */
