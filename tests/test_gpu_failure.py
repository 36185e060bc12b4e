"""Failure detection on the GPU without a fault.

The ridge kernel is the one kernel that waits (on the mbarriers of its
shared-memory copies). Its self-test makes every wait run out (a barrier that
expects more bytes than its copies deliver, 1 ms limit): the kernel must
record LT_ERR_TIMEOUT and return, leaving the context usable, which a normal
run afterwards (bit-exact against the oracle) shows. Device-detected input
errors are reported the same way, through the workspace.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("built_cpu_parts")]

LT_ERR_LABEL_OUTSIDE_MASK = 5
LT_ERR_TIMEOUT = 8


@pytest.fixture(scope="module")
def lt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_05808_gb300 as mod
    return mod


def run(lt, mask, labels, n):
    import torch
    m = torch.from_numpy(mask).cuda()
    l = torch.from_numpy(labels.view(np.int32)).cuda()
    dt2 = torch.empty(mask.shape, dtype=torch.int32, device="cuda")
    lt2 = torch.empty_like(dt2)
    S = torch.empty(n, dtype=torch.float32, device="cuda")
    R = torch.empty_like(S)
    ws = lt.lt_measure(m, l, n, dt2, lt2, S, R)
    return ws, dt2, lt2


def test_wait_limit_reports_timeout_and_context_survives(lt):
    import torch
    assert lt.lt_selftest_wait_timeout() == LT_ERR_TIMEOUT
    assert lt.lt_selftest_wait_timeout() == LT_ERR_TIMEOUT  # repeatable
    torch.cuda.synchronize()
    mask, labels, n = synth.workload("particles_3d_64", 2)
    ws, dt2, lt2 = run(lt, mask, labels, n)
    lt.lt_workspace_status(ws)
    d_ref, l_ref, _, _ = oracle.pipeline(mask, labels, n)
    assert np.array_equal(dt2.cpu().numpy().view(np.uint32), d_ref)
    assert np.array_equal(lt2.cpu().numpy().view(np.uint32), l_ref)


def test_device_input_error_is_reported_then_cleared(lt):
    mask, labels, n = synth.workload("particles_3d_64", 3)
    bad = labels.copy()
    z, y, x = np.argwhere(mask == 0)[0]
    bad[z, y, x] = 1  # a labelled voxel outside the mask
    ws, _, _ = run(lt, mask, bad, n)
    with pytest.raises(lt.LTError) as e:
        lt.lt_workspace_status(ws)
    assert e.value.status == LT_ERR_LABEL_OUTSIDE_MASK
    ws, _, _ = run(lt, mask, labels, n)  # a fresh call starts from a clean header
    lt.lt_workspace_status(ws)
