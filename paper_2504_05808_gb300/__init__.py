"""Python binding of the GB300 local-thickness shape library (include/lt.h).

Argument marshalling only: every step runs in the CUDA kernels of _lt.so.
PyTorch provides device memory and streams. There is no CPU fallback: if the
library has not been built (python -c "import __graft_entry__ as g; g.build()")
importing this package raises ImportError.

Tensors: mask uint8; labels, dt2, lt2 int32 or uint32 (bit patterns are
reinterpreted as uint32); shape (ny, nx) for 2D or (nz, ny, nx) for 3D,
contiguous, on a CUDA device. Calls run on torch's current stream unless a
stream is given.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lt.so")

LT_OK = 0
STATUS_NAMES = {0: "LT_OK", 1: "LT_ERR_INVALID_ARG", 2: "LT_ERR_DIMS", 3: "LT_ERR_WORKSPACE",
                4: "LT_ERR_LABEL_RANGE", 5: "LT_ERR_LABEL_OUTSIDE_MASK", 6: "LT_ERR_CUDA",
                7: "LT_ERR_NO_DEVICE", 8: "LT_ERR_TIMEOUT", 9: "LT_ERR_CHECKPOINT"}
FIXED_POINT_SHIFT = 20
MLP_FEATURES = 48
MLP_PARAMS = 7361

# exported symbol -> (restype, argtypes)
_vp, _sz, _i32, _i64, _u32 = (ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int64,
                             ctypes.c_uint32)
_DIMS = [_i32, _i64, _i64, _i64]
SIGNATURES = {
    "lt_status_string": (ctypes.c_char_p, [_i32]),
    "lt_version": (_u32, []),
    "lt_edt_workspace_size": (_sz, _DIMS),
    "lt_edt": (_i32, [_vp, _vp] + _DIMS + [_vp, _sz, _vp]),
    "lt_local_thickness_workspace_size": (_sz, _DIMS),
    "lt_local_thickness": (_i32, [_vp, _vp, _vp] + _DIMS + [_vp, _sz, _vp]),
    "lt_local_thickness_scaled_workspace_size": (_sz, [_i32] + _DIMS),
    "lt_local_thickness_scaled": (_i32, [_vp, _vp, _i32, _vp] + _DIMS + [_vp, _sz, _vp]),
    "lt_shape_workspace_size": (_sz, [_u32]),
    "lt_shape_measures": (_i32, [_vp, _vp, _u32] + _DIMS + [_vp, _sz, _vp, _vp, _vp, _vp]),
    "lt_shape_measures_filtered": (_i32, [_vp, _vp, _u32, _u32] + _DIMS + [_vp, _sz, _vp, _vp, _vp, _vp]),
    "lt_roundness_rescale_workspace_size": (_sz, []),
    "lt_roundness_rescale": (_i32, [_vp, _u32, ctypes.c_float, _vp, _vp, _sz, _vp]),
    "lt_measure_workspace_size": (_sz, [_u32] + _DIMS),
    "lt_measure": (_i32, [_vp, _vp, _u32] + _DIMS + [_vp, _sz, _vp, _vp, _vp, _vp, _vp]),
    "lt_measure_features_workspace_size": (_sz, [_u32] + _DIMS),
    "lt_measure_features": (_i32, [_vp, _vp, _u32] + _DIMS + [_vp, _sz, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "lt_measure_slabs_workspace_size": (_sz, [_u32, _i64, _i64, _i64, _i32]),
    "lt_measure_slabs": (_i32, [_vp, _vp, _u32, _i64, _i64, _i64, _i32, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "lt_measure_host_workspace_size": (_sz, [_u32] + _DIMS),
    "lt_measure_host": (_i32, [_vp, _vp, _u32] + _DIMS + [_vp, _sz, _vp, _vp, _vp]),
    "lt_workspace_status": (_i32, [_vp, _sz, _vp]),
    "lt_workspace_counters": (_i32, [_vp, _sz, _vp, _vp]),
    "lt_selftest_workspace_size": (_sz, []),
    "lt_selftest_wait_timeout": (_i32, [_vp, _sz, _vp]),
    "lt_shape_measures_static": (_i32, [_vp, _vp, _u32] + _DIMS + [_vp, _vp, _vp, _vp]),
    "lt_features_workspace_size": (_sz, [_u32]),
    "lt_object_features": (_i32, [_vp, _vp, _u32] + _DIMS + [_vp, _vp, _vp, _vp, _sz, _vp, _vp]),
    "lt_mlp_infer": (_i32, [_vp, _vp, _vp, _u32, _vp, _vp]),
    "lt_mlp_train_workspace_size": (_sz, [_u32]),
    "lt_mlp_gradients": (_i32, [_vp, _vp, _vp, _vp, _vp, _u32, _vp, _sz, _vp, _vp, _vp]),
    "lt_mlp_adam": (_i32, [_vp, _vp, _vp, _vp, _u32, ctypes.c_float, _vp]),
    "lt_mlp_train_step": (_i32, [_vp, _vp, _vp, _vp, _u32, ctypes.c_float, _vp, _vp, _vp, _vp,
                                 _u32, _vp, _sz, _vp, _vp]),
    "lt_mlp_checkpoint_size": (_sz, []),
    "lt_mlp_checkpoint_pack": (_i32, [_vp, _vp, _vp, _u32, _vp, _sz]),
    "lt_mlp_checkpoint_unpack": (_i32, [_vp, _sz, _vp, _vp, _vp, _vp]),
    "lt_mlp_save": (_i32, [ctypes.c_char_p, _vp, _vp, _vp, _u32, _vp]),
    "lt_mlp_load": (_i32, [ctypes.c_char_p, _vp, _vp, _vp, _vp, _vp]),
    "lt_batch_workspace_size": (_sz, [_vp, _i32]),
    "lt_batch_create": (_i32, [_vp, _i32, _vp, _sz, _i32, _vp]),
    "lt_batch_run": (_i32, [_vp, _vp]),
    "lt_batch_run_eager": (_i32, [_vp, _vp]),
    "lt_batch_status": (_i32, [_vp, _vp]),
    "lt_batch_autotune": (_i32, [_vp, _vp, ctypes.c_char_p]),
    "lt_batch_settings": (_i32, [_vp, _vp]),
    "lt_batch_destroy": (None, [_vp]),
    "lt_trace_enable": (_i32, [_i32]),
    "lt_trace_summary": (_i32, [_vp, _i32]),
}


class LTError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}")
        self.status = status


class LTCounters(ctypes.Structure):
    _fields_ = [("chunk_centres", ctypes.c_uint32), ("warp_centres", ctypes.c_uint32),
                ("updates", ctypes.c_uint64), ("table_updates", ctypes.c_uint64)]


class ObjectStats(ctypes.Structure):
    _fields_ = [("volume", _vp), ("n_shell", _vp), ("max_lt2", _vp), ("sum_lt", _vp),
                ("sum_shell_lt", _vp)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library {LIB_PATH} is missing; build it with "
                          "python paper_2504_05808_gb300/build.py")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def _check(status: int, where: str):
    if status != LT_OK:
        raise LTError(status, where)


def _dims(t):
    if t.dim() == 2:
        return 2, t.shape[1], t.shape[0], 1
    if t.dim() == 3:
        return 3, t.shape[2], t.shape[1], t.shape[0]
    raise ValueError("expected a 2D or 3D tensor")


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def workspace(nbytes: int, device):
    """Device workspace (uint8 tensor; torch's allocator aligns to 512 bytes)."""
    import torch
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def lt_edt(mask, dt2, ws=None, stream=None):
    nd, nx, ny, nz = _dims(mask)
    need = lib.lt_edt_workspace_size(nd, nx, ny, nz)
    if need and ws is None:
        ws = workspace(need, mask.device)
    _check(lib.lt_edt(_ptr(mask), _ptr(dt2), nd, nx, ny, nz, _ptr(ws) if need else None,
                      ws.numel() if need else 0, _stream(stream)), "lt_edt")


def lt_local_thickness(dt2, labels, lt2, ws=None, stream=None):
    nd, nx, ny, nz = _dims(dt2)
    if ws is None:
        ws = workspace(lib.lt_local_thickness_workspace_size(nd, nx, ny, nz), dt2.device)
    _check(lib.lt_local_thickness(_ptr(dt2), _ptr(labels), _ptr(lt2), nd, nx, ny, nz, _ptr(ws),
                                  ws.numel(), _stream(stream)), "lt_local_thickness")
    return ws


def lt_local_thickness_scaled(mask, labels, scale, lt2, ws=None, stream=None):
    """Approximate LT2 computed at 1/scale resolution (see include/lt.h)."""
    nd, nx, ny, nz = _dims(mask)
    if ws is None:
        ws = workspace(lib.lt_local_thickness_scaled_workspace_size(scale, nd, nx, ny, nz), mask.device)
    _check(lib.lt_local_thickness_scaled(_ptr(mask), _ptr(labels), int(scale), _ptr(lt2), nd, nx, ny, nz,
                                         _ptr(ws), ws.numel(), _stream(stream)), "lt_local_thickness_scaled")
    return ws


def lt_shape_measures(labels, lt2, n_labels, sphericity=None, roundness=None, stats=None,
                      ws=None, stream=None):
    """stats: optional dict of device tensors volume, n_shell, max_lt2 (int32,
    n_labels) and sum_lt, sum_shell_lt (int64, n_labels)."""
    nd, nx, ny, nz = _dims(labels)
    if ws is None:
        ws = workspace(lib.lt_shape_workspace_size(n_labels), labels.device)
    st = None
    if stats is not None:
        st = ObjectStats(*[stats[k].data_ptr() if k in stats else None
                           for k in ("volume", "n_shell", "max_lt2", "sum_lt", "sum_shell_lt")])
    _check(lib.lt_shape_measures(_ptr(labels), _ptr(lt2), n_labels, nd, nx, ny, nz, _ptr(ws),
                                 ws.numel(), _ptr(sphericity), _ptr(roundness),
                                 ctypes.byref(st) if st is not None else None, _stream(stream)),
           "lt_shape_measures")
    return ws


def lt_shape_measures_filtered(labels, lt2, n_labels, min_lt2, sphericity=None, roundness=None,
                               stats=None, ws=None, stream=None):
    """lt_shape_measures on the objects reduced to their voxels with
    LT2 >= min_lt2 (roughness filtering; see include/lt.h)."""
    nd, nx, ny, nz = _dims(labels)
    if ws is None:
        ws = workspace(lib.lt_shape_workspace_size(n_labels), labels.device)
    st = None
    if stats is not None:
        st = ObjectStats(*[stats[k].data_ptr() if k in stats else None
                           for k in ("volume", "n_shell", "max_lt2", "sum_lt", "sum_shell_lt")])
    _check(lib.lt_shape_measures_filtered(_ptr(labels), _ptr(lt2), n_labels, int(min_lt2), nd, nx, ny, nz,
                                          _ptr(ws), ws.numel(), _ptr(sphericity), _ptr(roundness),
                                          ctypes.byref(st) if st is not None else None, _stream(stream)),
           "lt_shape_measures_filtered")
    return ws


def lt_roundness_rescale(roundness, out, r_min=None, stream=None):
    """out = max(0, (R - m) / (1 - m)), m = r_min or the smallest finite R."""
    ws = workspace(lib.lt_roundness_rescale_workspace_size(), roundness.device)
    _check(lib.lt_roundness_rescale(_ptr(roundness), roundness.numel(), -1.0 if r_min is None else float(r_min),
                                    _ptr(out), _ptr(ws), ws.numel(), _stream(stream)), "lt_roundness_rescale")


def lt_measure(mask, labels, n_labels, dt2, lt2, sphericity, roundness, ws=None, stream=None):
    nd, nx, ny, nz = _dims(mask)
    if ws is None:
        ws = workspace(lib.lt_measure_workspace_size(n_labels, nd, nx, ny, nz), mask.device)
    _check(lib.lt_measure(_ptr(mask), _ptr(labels), n_labels, nd, nx, ny, nz, _ptr(ws), ws.numel(),
                          _ptr(dt2), _ptr(lt2), _ptr(sphericity), _ptr(roundness),
                          _stream(stream)), "lt_measure")
    return ws


def lt_measure_features(mask, labels, n_labels, dt2, lt2, sphericity, roundness, features, stats=None, ws=None,
                        stream=None):
    """lt_measure plus the learned correction's features ([n_labels, 48]
    float32) from the same shape pass; stats (dict of five tensors) optional."""
    nd, nx, ny, nz = _dims(mask)
    if ws is None:
        ws = workspace(lib.lt_measure_features_workspace_size(n_labels, nd, nx, ny, nz), mask.device)
    st = ctypes.byref(_stats_struct(stats)) if stats is not None else None
    _check(lib.lt_measure_features(_ptr(mask), _ptr(labels), n_labels, nd, nx, ny, nz, _ptr(ws), ws.numel(),
                                   _ptr(dt2), _ptr(lt2), _ptr(sphericity), _ptr(roundness), _ptr(features), st,
                                   _stream(stream)), "lt_measure_features")
    return ws


def lt_measure_host(mask_host, labels_host, n_labels, sphericity_host, roundness_host, ws,
                    stream=None):
    """Host tensors (ideally pinned) in and out; ws is a device workspace of
    lt_measure_host_workspace_size bytes. Synchronises the stream."""
    nd, nx, ny, nz = _dims(mask_host)
    for t in (mask_host, labels_host, sphericity_host, roundness_host):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError("expected contiguous host tensors")
    _check(lib.lt_measure_host(ctypes.c_void_p(mask_host.data_ptr()),
                               ctypes.c_void_p(labels_host.data_ptr()), n_labels, nd, nx, ny, nz,
                               _ptr(ws), ws.numel(), ctypes.c_void_p(sphericity_host.data_ptr()),
                               ctypes.c_void_p(roundness_host.data_ptr()), _stream(stream)),
           "lt_measure_host")


def lt_measure_slabs(mask_host, labels_host, n_labels, slab_planes, dt2_host, lt2_host, sphericity_host,
                     roundness_host, ws=None, device="cuda", stream=None):
    """Slab form of lt_measure over host tensors (3D; see include/lt.h);
    lt2_host may be None. Waits for the stream; returns the workspace."""
    nz, ny, nx = mask_host.shape
    for t in (mask_host, labels_host, dt2_host, sphericity_host, roundness_host):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError("expected contiguous host tensors")
    if ws is None:
        ws = workspace(lib.lt_measure_slabs_workspace_size(n_labels, nx, ny, nz, slab_planes), device)
    hp = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    _check(lib.lt_measure_slabs(hp(mask_host), hp(labels_host), n_labels, nx, ny, nz, int(slab_planes),
                                hp(dt2_host), hp(lt2_host), hp(sphericity_host), hp(roundness_host), _ptr(ws),
                                ws.numel(), _stream(stream)), "lt_measure_slabs")
    return ws


def lt_measure_host_workspace_size(n_labels, shape):
    nd = len(shape)
    nz, ny, nx = (1,) + tuple(shape) if nd == 2 else tuple(shape)
    return lib.lt_measure_host_workspace_size(n_labels, nd, nx, ny, nz)


class TraceEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", _u32), ("total_ms", ctypes.c_double)]


def lt_trace_enable(enable: bool = True):
    _check(lib.lt_trace_enable(1 if enable else 0), "lt_trace_enable")


def lt_trace_summary():
    """{kernel name: (launches, total ms)} of the kernels launched while
    tracing was enabled (waits for their events)."""
    buf = (TraceEntry * 64)()
    n = lib.lt_trace_summary(buf, 64)
    if n < 0:
        raise LTError(6, "lt_trace_summary")
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms))
            for i in range(min(n, 64))}


def lt_workspace_status(ws, stream=None):
    _check(lib.lt_workspace_status(_ptr(ws), ws.numel(), _stream(stream)), "device status")


def lt_workspace_counters(ws, stream=None):
    """Work counters of the last local-thickness run on `ws`: dict with
    chunk_centres, warp_centres (kept centres painted in shared chunks or
    one warp each), updates (LT2 atomic-max updates) and table_updates
    (those from crescent tables)."""
    c = LTCounters()
    _check(lib.lt_workspace_counters(_ptr(ws), ws.numel(), _stream(stream), ctypes.byref(c)),
           "workspace counters")
    return {"chunk_centres": c.chunk_centres, "warp_centres": c.warp_centres, "updates": c.updates,
            "table_updates": c.table_updates}


def lt_selftest_wait_timeout(device="cuda", stream=None):
    """Runs the bounded-wait self-test (see include/lt.h) and returns the
    device status it produced: LT_ERR_TIMEOUT (8) when the wait limit works."""
    ws = workspace(lib.lt_selftest_workspace_size(), device)
    return lib.lt_selftest_wait_timeout(_ptr(ws), ws.numel(), _stream(stream))


def _stats_struct(stats):
    return ObjectStats(*[stats[k].data_ptr() for k in ("volume", "n_shell", "max_lt2", "sum_lt",
                                                       "sum_shell_lt")])


def lt_object_features(labels, lt2, n_labels, stats, sphericity, roundness, features, ws=None,
                       stream=None):
    """features: float32 CUDA tensor [n_labels, 48]; stats as for
    lt_shape_measures (all five arrays)."""
    nd, nx, ny, nz = _dims(labels)
    if ws is None:
        ws = workspace(lib.lt_features_workspace_size(n_labels), labels.device)
    st = _stats_struct(stats)
    _check(lib.lt_object_features(_ptr(labels), _ptr(lt2), n_labels, nd, nx, ny, nz, ctypes.byref(st),
                                  _ptr(sphericity), _ptr(roundness), _ptr(ws), ws.numel(),
                                  _ptr(features), _stream(stream)), "lt_object_features")
    return ws


def lt_mlp_infer(params, features, sphericity, s_learned, stream=None):
    _check(lib.lt_mlp_infer(_ptr(params), _ptr(features), _ptr(sphericity), sphericity.numel(),
                            _ptr(s_learned), _stream(stream)), "lt_mlp_infer")


def lt_mlp_gradients(params, features, sphericity, target, batch_idx, grad, loss=None, ws=None,
                     stream=None):
    b = batch_idx.numel()
    if ws is None:
        ws = workspace(lib.lt_mlp_train_workspace_size(b), params.device)
    _check(lib.lt_mlp_gradients(_ptr(params), _ptr(features), _ptr(sphericity), _ptr(target),
                                _ptr(batch_idx), b, _ptr(ws), ws.numel(), _ptr(grad), _ptr(loss),
                                _stream(stream)), "lt_mlp_gradients")
    return ws


def lt_mlp_adam(params, m, v, grad, step, lr, stream=None):
    _check(lib.lt_mlp_adam(_ptr(params), _ptr(m), _ptr(v), _ptr(grad), int(step), float(lr),
                           _stream(stream)), "lt_mlp_adam")


def lt_mlp_train_step(params, m, v, grad, step, lr, features, sphericity, target, batch_idx,
                      loss=None, ws=None, stream=None):
    b = batch_idx.numel()
    if ws is None:
        ws = workspace(lib.lt_mlp_train_workspace_size(b), params.device)
    _check(lib.lt_mlp_train_step(_ptr(params), _ptr(m), _ptr(v), _ptr(grad), int(step), float(lr),
                                 _ptr(features), _ptr(sphericity), _ptr(target), _ptr(batch_idx), b,
                                 _ptr(ws), ws.numel(), _ptr(loss), _stream(stream)),
           "lt_mlp_train_step")
    return ws


def lt_mlp_save(path, params, m=None, v=None, step=0, stream=None):
    """Writes a checkpoint file of the network (and Adam state) held in
    device tensors."""
    _check(lib.lt_mlp_save(os.fsencode(path), _ptr(params), _ptr(m), _ptr(v), int(step), _stream(stream)),
           "lt_mlp_save")


def lt_mlp_load(path, params, m=None, v=None, stream=None):
    """Reads a checkpoint file into device tensors; returns the Adam step."""
    step = ctypes.c_uint32(0)
    _check(lib.lt_mlp_load(os.fsencode(path), _ptr(params), _ptr(m), _ptr(v), ctypes.byref(step),
                           _stream(stream)), "lt_mlp_load")
    return int(step.value)


def train_mlp(params, features, sphericity, target, train_idx, epochs, batch, lr, order_seed=0):
    """Adam training on the GPU with lt_mlp_train_step. params (FP32 CUDA
    tensor of MLP_PARAMS) is updated in place; train_idx lists the objects
    to train on; batches follow a seeded shuffle per epoch. Returns the
    per-epoch mean loss (host floats)."""
    import numpy as np
    import torch
    dev = params.device
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    grad = torch.empty_like(params)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    ws = workspace(lib.lt_mlp_train_workspace_size(batch), dev)
    rng = np.random.default_rng(order_seed)
    idx = np.asarray(train_idx, dtype=np.int64)
    step, history = 0, []
    for _ in range(epochs):
        perm = idx[rng.permutation(idx.size)]
        perm_dev = torch.from_numpy(perm.astype(np.int32)).to(dev)  # one upload per epoch
        losses = []
        for s0 in range(0, perm.size - batch + 1, batch):
            b = perm_dev[s0:s0 + batch]
            step += 1
            lt_mlp_train_step(params, m, v, grad, step, lr, features, sphericity, target, b, loss,
                              ws=ws)
            losses.append(loss.clone())
        history.append(float(torch.stack(losses).mean().item()) if losses else float("nan"))
    return history


# ------------------------------------------------------------- batched form
class Volume(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("n_labels", ctypes.c_uint32), ("nx", _i64), ("ny", _i64),
                ("nz", _i64), ("mask", _vp), ("labels", _vp), ("dt2", _vp), ("lt2", _vp),
                ("sphericity", _vp), ("roundness", _vp)]


class Batch:
    """Many volumes measured by one CUDA graph launch (lt_batch_*).

    items: list of dicts with CUDA tensors mask, labels, dt2, lt2,
    sphericity, roundness and the int n_labels. The tensors must stay alive
    and in place while the batch exists (the graph holds their addresses).
    """

    def __init__(self, items, branches=4, device=None):
        import torch
        self.items = items
        arr = (Volume * len(items))()
        for a, it in zip(arr, items):
            nd, nx, ny, nz = _dims(it["mask"])
            a.ndim, a.n_labels, a.nx, a.ny, a.nz = nd, int(it["n_labels"]), nx, ny, nz
            for k in ("mask", "labels", "dt2", "lt2", "sphericity", "roundness"):
                setattr(a, k, it[k].data_ptr())
        self._vols = arr
        dev = device if device is not None else items[0]["mask"].device
        self.ws = workspace(lib.lt_batch_workspace_size(arr, len(items)), dev)
        h = ctypes.c_void_p()
        _check(lib.lt_batch_create(arr, len(items), _ptr(self.ws), self.ws.numel(), int(branches),
                                   ctypes.byref(h)), "lt_batch_create")
        self.handle = h

    def run(self, stream=None):
        _check(lib.lt_batch_run(self.handle, _stream(stream)), "lt_batch_run")

    def run_eager(self, stream=None):
        _check(lib.lt_batch_run_eager(self.handle, _stream(stream)), "lt_batch_run_eager")

    def status(self, stream=None):
        _check(lib.lt_batch_status(self.handle, _stream(stream)), "lt_batch_status")

    def autotune(self, cache_path=None, stream=None):
        p = cache_path.encode() if cache_path else None
        _check(lib.lt_batch_autotune(self.handle, _stream(stream), p), "lt_batch_autotune")

    def settings(self):
        out = (ctypes.c_int32 * 5)()
        _check(lib.lt_batch_settings(self.handle, out), "lt_batch_settings")
        return {"edt_tx_y": out[0], "edt_tx_z": out[1], "ridge_z": out[2], "paint_bpsm": out[3],
                "chunk_cres": out[4]}

    def close(self):
        if getattr(self, "handle", None):
            lib.lt_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

