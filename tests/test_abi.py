"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/lt.h declares, and rejects bad arguments before any
CUDA call is made."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lt.h")


@pytest.fixture(scope="module")
def lt():
    import __graft_entry__
    __graft_entry__._cuda_builder().build()
    import paper_2504_05808_gb300 as mod
    return mod


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(lt_[a-z0-9_]+)\s*\(", text,
                       flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lt):
    names = declared_functions()
    assert len(names) >= 13
    lib = ctypes.CDLL(lt.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(lt.SIGNATURES)


def test_status_strings_and_version(lt):
    for code in range(10):
        s = lt.lib.lt_status_string(code)
        assert s and s != b"unknown status"
    assert lt.lib.lt_status_string(99) == b"unknown status"
    assert lt.lib.lt_version() == 0x000100


def test_workspace_sizes(lt):
    L = lt.lib
    n = 512 ** 3
    # local thickness: header + 18 bytes per voxel (centre records, up to one
    # per voxel plus n/8 part records of shared big centres)
    ws = L.lt_local_thickness_workspace_size(3, 512, 512, 512)
    assert 18 * n <= ws < 18 * n + 4096
    # EDT: 16-bit row distances, plus uint32 per voxel for z axes over 2048
    assert L.lt_edt_workspace_size(3, 512, 512, 512) == 2 * n
    assert L.lt_edt_workspace_size(2, 100, 3000, 1) == -(-2 * 300000 // 256) * 256  # 256-byte aligned
    assert L.lt_edt_workspace_size(3, 16, 16, 3000) == 2 * 768000 + 4 * 768000
    assert L.lt_shape_workspace_size(1000) >= 28 * 1000
    assert L.lt_measure_workspace_size(100, 3, 512, 512, 512) >= ws
    host = L.lt_measure_host_workspace_size(100, 3, 64, 64, 64)
    assert host >= L.lt_measure_workspace_size(100, 3, 64, 64, 64) + 13 * 64 ** 3
    # invalid dimensions give 0
    assert L.lt_local_thickness_workspace_size(2, 10, 10, 2) == 0
    assert L.lt_local_thickness_workspace_size(3, 8193, 1, 1) == 0
    assert L.lt_local_thickness_workspace_size(4, 1, 1, 1) == 0


def test_argument_errors_need_no_gpu(lt):
    L = lt.lib
    E = {v: k for k, v in lt.STATUS_NAMES.items()}
    assert L.lt_edt(None, None, 3, 0, 4, 4, None, 0, None) == E["LT_ERR_DIMS"]
    assert L.lt_edt(None, None, 2, 4, 4, 3, None, 0, None) == E["LT_ERR_DIMS"]
    assert L.lt_edt(None, None, 5, 4, 4, 4, None, 0, None) == E["LT_ERR_INVALID_ARG"]
    assert L.lt_edt(None, None, 3, 4096, 4096, 4096, None, 0, None) == E["LT_ERR_DIMS"]
    assert L.lt_edt(None, None, 3, 4, 4, 4, None, 0, None) == E["LT_ERR_INVALID_ARG"]
    assert L.lt_local_thickness(None, None, None, 3, 4, 4, 4, None, 0, None) == E["LT_ERR_INVALID_ARG"]
    assert L.lt_shape_measures(None, None, 0, 3, 4, 4, 4, None, 0, None, None, None, None) == \
        E["LT_ERR_INVALID_ARG"]
    # misaligned pointers are rejected before use
    assert L.lt_edt(ctypes.c_void_p(17), ctypes.c_void_p(32), 3, 4, 4, 4, None, 0, None) == \
        E["LT_ERR_INVALID_ARG"]
    assert L.lt_measure_host(None, None, 3, 3, 4, 4, 4, None, 0, None, None, None) == \
        E["LT_ERR_INVALID_ARG"]
    assert L.lt_workspace_status(None, 0, None) == E["LT_ERR_WORKSPACE"]


def test_product_path_does_not_touch_the_oracle():
    """The library package neither imports nor links the CPU oracle."""
    pkg = os.path.join(ROOT, "paper_2504_05808_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "lt_oracle" not in text, f


def test_batch_argument_errors_need_no_gpu(lt):
    L = lt.lib
    E = {v: k for k, v in lt.STATUS_NAMES.items()}
    assert L.lt_batch_workspace_size(None, 0) == 0
    h = ctypes.c_void_p()
    assert L.lt_batch_create(None, 0, None, 0, 1, ctypes.byref(h)) == E["LT_ERR_INVALID_ARG"]
    vols = (lt.Volume * 2)()
    vols[0].ndim, vols[0].n_labels, vols[0].nx, vols[0].ny, vols[0].nz = 3, 5, 64, 64, 64
    vols[1].ndim, vols[1].n_labels, vols[1].nx, vols[1].ny, vols[1].nz = 2, 3, 100, 50, 1
    one = L.lt_measure_workspace_size(5, 3, 64, 64, 64)
    two = L.lt_measure_workspace_size(3, 2, 100, 50, 1)
    assert L.lt_batch_workspace_size(vols, 2) >= one + two
    vols[1].nz = 2  # 2D with nz != 1
    assert L.lt_batch_workspace_size(vols, 2) == 0
    # null device pointers are rejected before anything is recorded
    vols[1].nz = 1
    assert L.lt_batch_create(vols, 2, None, 0, 2, ctypes.byref(h)) == E["LT_ERR_INVALID_ARG"]
    assert L.lt_batch_run(None, None) == E["LT_ERR_INVALID_ARG"]


def test_mlp_checkpoint_format_needs_no_gpu(lt, tmp_path):
    """The checkpoint layout through the C ABI on host buffers: the header
    fields, the float32 vectors in place, the CRC-32 equal to zlib's over the
    bytes before it, a round trip, and rejection of damaged or foreign data."""
    import struct
    import zlib
    import numpy as np
    L = lt.lib
    E = {v: k for k, v in lt.STATUS_NAMES.items()}
    n = lt.MLP_PARAMS
    size = L.lt_mlp_checkpoint_size()
    assert size == 8 + 6 * 4 + 3 * 4 * n + 4
    rng = np.random.default_rng(0)
    p, m, v = (rng.normal(size=n).astype(np.float32) for _ in range(3))
    buf = np.zeros(size, np.uint8)
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data)
    assert L.lt_mlp_checkpoint_pack(ptr(p), ptr(m), ptr(v), 1234, ptr(buf), size) == 0
    raw = buf.tobytes()
    assert raw[:8] == b"LTMLPCK1"
    assert struct.unpack("<6I", raw[8:32]) == (1, 48, 64, n, 1234, 1)
    body = np.frombuffer(raw[32:-4], dtype="<f4")
    assert np.array_equal(body[:n], p) and np.array_equal(body[n:2 * n], m) and np.array_equal(body[2 * n:], v)
    assert struct.unpack("<I", raw[-4:])[0] == zlib.crc32(raw[:-4])
    out = [np.zeros(n, np.float32) for _ in range(3)]
    step = ctypes.c_uint32(0)
    assert L.lt_mlp_checkpoint_unpack(ptr(buf), size, *[ptr(a) for a in out], ctypes.byref(step)) == 0
    assert step.value == 1234 and all(np.array_equal(a, b) for a, b in zip(out, (p, m, v)))
    for k in (0, 20, 40, size - 1):  # magic, network shape, a weight, the CRC itself
        bad = buf.copy()
        bad[k] ^= 1
        assert L.lt_mlp_checkpoint_unpack(ptr(bad), size, ptr(out[0]), None, None, None) == E["LT_ERR_CHECKPOINT"]
    assert L.lt_mlp_checkpoint_unpack(ptr(buf), size - 1, ptr(out[0]), None, None, None) == E["LT_ERR_CHECKPOINT"]
    # without moments: stored as zeros, flag clear, and not readable as moments
    assert L.lt_mlp_checkpoint_pack(ptr(p), None, None, 7, ptr(buf), size) == 0
    assert struct.unpack("<I", buf.tobytes()[28:32])[0] == 0
    assert L.lt_mlp_checkpoint_unpack(ptr(buf), size, ptr(out[0]), ptr(out[1]), ptr(out[2]), None) == \
        E["LT_ERR_CHECKPOINT"]
    assert L.lt_mlp_checkpoint_unpack(ptr(buf), size, ptr(out[0]), None, None, None) == 0
    assert L.lt_mlp_checkpoint_pack(ptr(p), ptr(m), None, 7, ptr(buf), size) == E["LT_ERR_INVALID_ARG"]
    assert L.lt_mlp_checkpoint_pack(ptr(p), None, None, 7, ptr(buf), size - 1) == E["LT_ERR_WORKSPACE"]
    assert L.lt_mlp_load(str(tmp_path / "missing").encode(), None, None, None, None, None) == E["LT_ERR_INVALID_ARG"]
