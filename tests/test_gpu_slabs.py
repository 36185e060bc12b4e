"""The slab form of the pipeline (host-resident volume, a few z planes on
the device at a time) gives lt_measure's results bit for bit: DT2, LT2,
sphericity and roundness, with several slabs in every phase, halos that
reach the array's faces, and ragged sizes."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("built_cpu_parts")]


@pytest.fixture(scope="module")
def lt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_05808_gb300 as mod
    return mod


def in_core(lt, mask, labels, n):
    import torch
    m = torch.from_numpy(mask).cuda()
    l = torch.from_numpy(labels.view(np.int32)).cuda()
    dt2 = torch.empty(mask.shape, dtype=torch.int32, device="cuda")
    lt2 = torch.empty_like(dt2)
    S = torch.empty(n, dtype=torch.float32, device="cuda")
    R = torch.empty_like(S)
    lt.lt_workspace_status(lt.lt_measure(m, l, n, dt2, lt2, S, R))
    return dt2.cpu().numpy(), lt2.cpu().numpy(), S.cpu().numpy(), R.cpu().numpy()


def slabs(lt, mask, labels, n, planes):
    import torch
    mh = torch.from_numpy(mask).pin_memory()
    lh = torch.from_numpy(labels.view(np.int32)).pin_memory()
    dt2 = torch.empty(mask.shape, dtype=torch.int32).pin_memory()
    lt2 = torch.empty(mask.shape, dtype=torch.int32).pin_memory()
    S = torch.empty(n, dtype=torch.float32).pin_memory()
    R = torch.empty(n, dtype=torch.float32).pin_memory()
    lt.lt_measure_slabs(mh, lh, n, planes, dt2, lt2, S, R)
    return dt2.numpy(), lt2.numpy(), S.numpy(), R.numpy()


def same(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(x, y, equal_nan=True)


@pytest.mark.parametrize("name,planes", [("particles_3d_96", 48), ("ellipsoids_3d_128", 60)])
def test_slabs_equal_in_core(lt, name, planes):
    mask, labels, n = synth.workload(name, 3)
    same(slabs(lt, mask, labels, n, planes), in_core(lt, mask, labels, n))


def test_ragged_and_touching(lt):
    import scipy.ndimage as ndi
    rng = np.random.default_rng(5)
    shape = (41, 29, 37)
    f = ndi.gaussian_filter(rng.random(shape), 1.5)
    mask = (f > np.quantile(f, 0.45)).astype(np.uint8)
    labels = ndi.label(mask)[0].astype(np.uint32)
    labels[labels % 3 == 0] = 0  # unlabelled foreground too
    n = int(labels.max()) + 1
    got = slabs(lt, mask, labels, n, 16)
    same(got, in_core(lt, mask, labels, n))
    d, l2, _, _ = oracle.pipeline(mask, labels, n)
    assert np.array_equal(got[0].view(np.uint32), d) and np.array_equal(got[1].view(np.uint32), l2)


def test_too_few_planes_for_the_objects(lt):
    mask, labels, n = synth.workload("particles_3d_96", 3)
    with pytest.raises(lt.LTError) as e:
        slabs(lt, mask, labels, n, 8)
    assert e.value.status == 3  # LT_ERR_WORKSPACE
