"""Objects measured one at a time equal objects measured all at once.

The object-count protocol (Sec. 5.3) times three ways of measuring a subset
of objects: one call over the volume holding only them, a graph batch of
per-object crops, and per-object launches. With a one-voxel gap between
objects, a bounding-box crop (outside the array counts as background) gives
the same DT, LT and measures as the whole volume, so all three must agree bit
for bit; the oracle checks one of them.
"""
import numpy as np
import pytest
import scipy.ndimage as ndi

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


def test_crops_batch_and_subset_volume_agree(lt):
    import torch
    mask, labels, n = synth.workload("particles_3d_96", 11)
    boxes = ndi.find_objects(labels.astype(np.int64))
    rng = np.random.default_rng(0)
    pick = sorted(rng.choice([l for l in range(1, n) if boxes[l - 1] is not None], 12, replace=False))
    items = []
    for l in pick:
        lab = labels[boxes[l - 1]] == l
        items.append({"mask": torch.from_numpy(lab.astype(np.uint8)).cuda(),
                      "labels": torch.from_numpy(lab.astype(np.int32)).cuda(),
                      "dt2": torch.empty(lab.shape, dtype=torch.int32, device="cuda"),
                      "lt2": torch.empty(lab.shape, dtype=torch.int32, device="cuda"),
                      "sphericity": torch.empty(2, dtype=torch.float32, device="cuda"),
                      "roundness": torch.empty(2, dtype=torch.float32, device="cuda"), "n_labels": 2})
    # the volume holding only the selected objects, measured in one call
    keep = np.isin(labels, pick)
    sub_lab = np.where(keep, labels, 0).astype(np.uint32)
    m = torch.from_numpy(keep.astype(np.uint8)).cuda()
    l = torch.from_numpy(sub_lab.view(np.int32)).cuda()
    dt2 = torch.empty(labels.shape, dtype=torch.int32, device="cuda")
    lt2 = torch.empty_like(dt2)
    S = torch.empty(n, dtype=torch.float32, device="cuda")
    R = torch.empty_like(S)
    lt.lt_workspace_status(lt.lt_measure(m, l, n, dt2, lt2, S, R))
    S, R = S.cpu().numpy(), R.cpu().numpy()
    # per-object launches and one graph launch over the crops
    batch = lt.Batch(items, branches=4)
    for run in (batch.run_eager, batch.run):
        for it in items:
            it["sphericity"].fill_(-1)
        run()
        batch.status()
        for it, lab_id in zip(items, pick):
            assert it["sphericity"][1].item() == S[lab_id]
            assert it["roundness"][1].item() == R[lab_id]
    batch.close()
    # crops against the oracle (bit-exact LT, measures within 1e-5)
    for it, lab_id in zip(items[:4], pick[:4]):
        cm = it["mask"].cpu().numpy()
        d, l2, So, Ro = oracle.pipeline(cm, cm.astype(np.uint32), 2)
        assert np.array_equal(it["lt2"].cpu().numpy().view(np.uint32), l2)
        assert abs(it["sphericity"][1].item() - So[1]) <= 1e-5 * So[1]
        assert abs(it["roundness"][1].item() - Ro[1]) <= 1e-5 * Ro[1]
