"""The batched form: one CUDA graph launch over many uneven 2D/3D volumes.

Every volume of a batch must come out bit-identical to a single lt_measure
call (same kernels), for the graph, the eager per-volume path, replays, and
after autotuning; small volumes are also checked against the oracle.
"""
import os

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


def make_item(mask, labels, n):
    import torch
    dev = "cuda"
    return {"mask": torch.from_numpy(mask).to(dev),
            "labels": torch.from_numpy(labels.view(np.int32)).to(dev),
            "dt2": torch.full(mask.shape, -1, dtype=torch.int32, device=dev),
            "lt2": torch.full(mask.shape, -1, dtype=torch.int32, device=dev),
            "sphericity": torch.full((n,), -1.0, dtype=torch.float32, device=dev),
            "roundness": torch.full((n,), -1.0, dtype=torch.float32, device=dev),
            "n_labels": n}


def _blobs(shape, seed):
    import scipy.ndimage as ndi
    rng = np.random.default_rng(seed)
    f = ndi.gaussian_filter(rng.random(shape), 1.5)
    m = (f > np.quantile(f, 0.6)).astype(np.uint8)
    lab = ndi.label(m)[0].astype(np.uint32)
    return m, lab, int(lab.max()) + 1


def volumes():
    """3D volumes of several sizes (rows of a multiple of 4 voxels and not,
    TMA and plain-load ridge passes), 2D images (one with columns longer than
    the shared-memory tiles: the global-memory y pass), and a 3D volume with
    an axis over 2048 (run as a single chain inside the graph)."""
    out = []
    for seed, edge in enumerate((40, 64, 33, 96, 72)):
        out.append(synth.workload(f"particles_3d_{edge}", seed))
    out.append(synth.workload("ellipses_2d_256", 3))
    out.append(synth.workload("ellipses_2d_300", 4))
    out.append(synth.workload("ellipsoids_3d_128", 5))
    out.append(synth.packed((2100, 90), 180, 8.0, 18.0, 6, shrink=(0.72, 0.86))[:2] + (181,))
    out.append(_blobs((2050, 6, 9), 7))
    return out


def single(lt, mask, labels, n):
    it = make_item(mask, labels, n)
    lt.lt_measure(it["mask"], it["labels"], n, it["dt2"], it["lt2"], it["sphericity"], it["roundness"])
    return it


def same(a, b):
    import torch
    for k in ("dt2", "lt2"):
        assert torch.equal(a[k], b[k]), k
    for k in ("sphericity", "roundness"):
        assert np.array_equal(a[k].cpu().numpy(), b[k].cpu().numpy(), equal_nan=True), k


def test_graph_batch_equals_single_calls(lt, tmp_path):
    import torch
    vols = volumes()
    ref = [single(lt, *v) for v in vols]
    items = [make_item(*v) for v in vols]
    batch = lt.Batch(items, branches=3)
    batch.run()
    batch.status()
    torch.cuda.synchronize()
    for a, b in zip(items, ref):
        same(a, b)
    # replay and the eager per-volume path give the same bits
    for it in items:
        it["lt2"].fill_(-1)
        it["sphericity"].fill_(-1)
    batch.run()
    batch.run()
    batch.status()
    for a, b in zip(items, ref):
        same(a, b)
    batch.run_eager()
    batch.status()
    for a, b in zip(items, ref):
        same(a, b)
    # autotuning writes a cache entry, a new batch reuses it, results unchanged
    cache = str(tmp_path / "autotune.json")
    batch.autotune(cache)
    s1 = batch.settings()
    assert os.path.exists(cache)
    batch.run()
    batch.status()
    for a, b in zip(items, ref):
        same(a, b)
    batch.close()
    items2 = [make_item(*v) for v in vols]
    b2 = lt.Batch(items2, branches=1)
    b2.autotune(cache)
    assert b2.settings() == s1
    b2.run()
    b2.status()
    for a, b in zip(items2, ref):
        same(a, b)
    b2.close()


def test_batch_matches_oracle_on_small_volumes(lt):
    vols = [synth.workload("particles_3d_48", 7), synth.workload("ellipses_2d_256", 8)]
    items = [make_item(*v) for v in vols]
    batch = lt.Batch(items, branches=2)
    batch.run()
    batch.status()
    for it, (m, lab, n) in zip(items, vols):
        d, l2, S, R = oracle.pipeline(m, lab, n)
        assert np.array_equal(it["dt2"].cpu().numpy().view(np.uint32), d)
        assert np.array_equal(it["lt2"].cpu().numpy().view(np.uint32), l2)
        got = it["sphericity"].cpu().numpy()
        f = ~np.isnan(S)
        assert np.array_equal(np.isnan(got), ~f)
        assert np.all(np.abs(got[f] - S[f]) <= 1e-5 * np.abs(S[f]))
    batch.close()


def test_batch_reports_device_errors(lt):
    m, lab, n = synth.workload("ellipses_2d_256", 9)
    bad = lab.copy()
    bad[0, 0] = 1  # labelled voxel outside the mask
    items = [make_item(m, lab, n), make_item(m, bad, n)]
    batch = lt.Batch(items, branches=2)
    batch.run()
    with pytest.raises(lt.LTError) as e:
        batch.status()
    assert e.value.status == 5
    batch.close()


def test_more_volumes_than_one_group_holds(lt):
    """300 small 3D volumes and 260 small 2D images: more of each kind than one
    group's table holds (256), so each kind is split into several groups on
    their own branches; every volume still equals a single call bit for bit."""
    import torch
    rng = np.random.default_rng(11)
    vols = [_blobs(tuple(int(e) for e in rng.integers(6, 20, 3)), 100 + i) for i in range(300)]
    vols += [_blobs(tuple(int(e) for e in rng.integers(8, 40, 2)), 500 + i) for i in range(260)]
    ref = [single(lt, *v) for v in vols]
    items = [make_item(*v) for v in vols]
    batch = lt.Batch(items, branches=2)
    batch.run()
    batch.status()
    torch.cuda.synchronize()
    for a, b in zip(items, ref):
        same(a, b)
    batch.close()
