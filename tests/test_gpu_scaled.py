"""GPU parity of the scaled local thickness (LT at 1/s resolution, upsampled)
with the oracle's definition: bit-exact for every scale, ragged sizes and
the synthetic workloads; scale 1 equals the exact LT."""
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


def gpu_scaled(lt, mask, labels, s):
    import torch
    m = torch.from_numpy(np.ascontiguousarray(mask, np.uint8)).cuda()
    l = torch.from_numpy(np.ascontiguousarray(labels, np.uint32).view(np.int32)).cuda()
    out = torch.full(mask.shape, -1, dtype=torch.int32, device="cuda")
    ws = lt.lt_local_thickness_scaled(m, l, s, out)
    lt.lt_workspace_status(ws)
    return out.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("shape", [(37, 45), (130, 66), (21, 34, 29), (40, 9, 70)])
def test_scaled_matches_oracle_on_random_masks(lt, shape):
    import scipy.ndimage as ndi
    rng = np.random.default_rng(sum(shape))
    f = ndi.gaussian_filter(rng.random(shape), 2.0)
    mask = (f > np.quantile(f, 0.4)).astype(np.uint8)
    labels = ndi.label(mask)[0].astype(np.uint32)
    for s in (1, 2, 3, 4):
        assert np.array_equal(gpu_scaled(lt, mask, labels, s), oracle.lt2_scaled(mask, labels, s)), s
    exact = oracle.lt2(oracle.dt2(mask), labels)
    assert np.array_equal(gpu_scaled(lt, mask, labels, 1), exact)


@pytest.mark.parametrize("name", ["ellipses_2d_256", "particles_3d_64"])
def test_scaled_matches_oracle_on_workloads(lt, name):
    mask, labels, n = synth.workload(name, 2)
    for s in (2, 3):
        assert np.array_equal(gpu_scaled(lt, mask, labels, s), oracle.lt2_scaled(mask, labels, s)), s
