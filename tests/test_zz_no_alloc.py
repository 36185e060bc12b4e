"""The no-allocation shape-measures entry point, lt_shape_measures_static.

It serves callers that cannot allocate device memory (code handed device
buffers by another framework without an allocator of its own, and loops that
must not call cudaMalloc after start-up). Its scratch is an array that the
library keeps in device memory, so this test checks, through the C ABI, that
two calls in a row (the array keeps the previous call's contents) give the
same sphericity and roundness as lt_shape_measures with a caller workspace,
and that label counts beyond the array's capacity are refused.

The file name makes pytest collect it last; it also runs alone in a fresh
process (the first call on the device performs the one-time set-up).
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

REL_TOL = 1e-5
MAX_LABELS = 131072  # LT_STATIC_MAX_LABELS in include/lt.h


@pytest.fixture(scope="module")
def lt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_05808_gb300 as mod
    return mod


def _dims(shape):
    return (2, shape[1], shape[0], 1) if len(shape) == 2 else (3, shape[2], shape[1], shape[0])


def _lt2_on_device(lt, mask, labels):
    import torch
    m = torch.from_numpy(mask).cuda()
    lab = torch.from_numpy(labels.view(np.int32)).cuda()
    dt2 = torch.empty(mask.shape, dtype=torch.int32, device="cuda")
    lt2 = torch.empty_like(dt2)
    lt.lt_edt(m, dt2)
    ws = lt.lt_local_thickness(dt2, lab, lt2)
    lt.lt_workspace_status(ws)
    return lab, lt2


def _close(got, ref):
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    f = ~np.isnan(ref)
    err = np.abs(got[f].astype(np.float64) - ref[f]) / np.abs(ref[f].astype(np.float64))
    assert err.size == 0 or err.max() <= REL_TOL


def test_static_scratch_matches_workspace_entry(lt):
    import torch
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for name, seed in (("ellipsoids_3d_128", 5), ("ellipses_2d_256", 6)):
        mask, labels, n = synth.workload(name, seed)
        lab, lt2 = _lt2_on_device(lt, mask, labels)
        nd, nx, ny, nz = _dims(mask.shape)
        S_ref = torch.empty(n, dtype=torch.float32, device="cuda")
        R_ref = torch.empty_like(S_ref)
        ws = lt.workspace(lt.lib.lt_shape_workspace_size(n), "cuda")
        assert lt.lib.lt_shape_measures(
            ctypes.c_void_p(lab.data_ptr()), ctypes.c_void_p(lt2.data_ptr()), n, nd, nx, ny, nz,
            ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.c_void_p(S_ref.data_ptr()),
            ctypes.c_void_p(R_ref.data_ptr()), None, stream) == 0
        for _ in range(2):  # two calls in a row share the library's array
            S = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
            R = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
            st = lt.lib.lt_shape_measures_static(
                ctypes.c_void_p(lab.data_ptr()), ctypes.c_void_p(lt2.data_ptr()), n, nd, nx, ny,
                nz, ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(R.data_ptr()), None, stream)
            assert st == 0, lt.lib.lt_status_string(st)
            torch.cuda.synchronize()
            _close(S.cpu().numpy(), S_ref.cpu().numpy())
            _close(R.cpu().numpy(), R_ref.cpu().numpy())


def test_static_scratch_refuses_too_many_labels(lt):
    import torch
    lab = torch.zeros((8, 8), dtype=torch.int32, device="cuda")
    lt2 = torch.zeros_like(lab)
    S = torch.empty(MAX_LABELS + 1, dtype=torch.float32, device="cuda")
    st = lt.lib.lt_shape_measures_static(ctypes.c_void_p(lab.data_ptr()),
                                         ctypes.c_void_p(lt2.data_ptr()), MAX_LABELS + 1, 2, 8, 8,
                                         1, ctypes.c_void_p(S.data_ptr()), None, None, None)
    assert st == 3  # LT_ERR_WORKSPACE
