"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bar: DT2 and LT2 bit-exact; sphericity and roundness within 1e-5 relative
(float32 outputs of FP64 formulas on fixed-point sums; each LT value enters
the sums as round(sqrtf(LT2) * 2^20), off by at most 2^-24 relative plus
2^-21 absolute); integer per-object counts exact.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("built_cpu_parts")]

REL_TOL = 1e-5


@pytest.fixture(scope="module")
def lt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_05808_gb300 as mod
    return mod


def dev_u32(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def host_u32(t):
    return t.cpu().numpy().view(np.uint32)


def gpu_pipeline(lt, mask, labels, n_labels, separate=False):
    import torch
    m = torch.from_numpy(np.ascontiguousarray(mask, dtype=np.uint8)).cuda()
    l = dev_u32(labels)
    dt2 = torch.empty(mask.shape, dtype=torch.int32, device="cuda")
    lt2 = torch.empty_like(dt2)
    S = torch.empty(n_labels, dtype=torch.float32, device="cuda")
    R = torch.empty_like(S)
    stats = {k: torch.empty(n_labels, dtype=torch.int32, device="cuda")
             for k in ("volume", "n_shell", "max_lt2")}
    stats.update({k: torch.empty(n_labels, dtype=torch.int64, device="cuda")
                  for k in ("sum_lt", "sum_shell_lt")})
    if separate:
        lt.lt_edt(m, dt2)
        ws = lt.lt_local_thickness(dt2, l, lt2)
        lt.lt_workspace_status(ws)
        ws = lt.lt_shape_measures(l, lt2, n_labels, S, R, stats)
    else:
        ws = lt.lt_measure(m, l, n_labels, dt2, lt2, S, R)
    lt.lt_workspace_status(ws)
    torch.cuda.synchronize()
    st = {k: v.cpu().numpy() for k, v in stats.items()}
    return host_u32(dt2), host_u32(lt2), S.cpu().numpy(), R.cpu().numpy(), st


def assert_close(got, ref, what):
    ref = np.asarray(ref, dtype=np.float64)
    got = np.asarray(got, dtype=np.float64)
    assert np.array_equal(np.isnan(got), np.isnan(ref)), what + ": NaN pattern"
    f = ~np.isnan(ref)
    err = np.abs(got[f] - ref[f]) / np.maximum(np.abs(ref[f]), 1e-30)
    assert err.size == 0 or err.max() <= REL_TOL, f"{what}: max rel err {err.max():.3g}"


def check_full(lt, mask, labels, n_labels, separate=False):
    d, l2, S, R, st = gpu_pipeline(lt, mask, labels, n_labels, separate)
    d_ref, l_ref, S_ref, R_ref = oracle.pipeline(mask, labels, n_labels)
    assert np.array_equal(d, d_ref), "DT2"
    assert np.array_equal(l2, l_ref), "LT2"
    assert_close(S, S_ref, "sphericity")
    assert_close(R, R_ref, "roundness")
    if separate:
        ost = oracle.object_stats(labels, l_ref, n_labels)
        for k in ("volume", "n_shell", "max_lt2"):
            assert np.array_equal(st[k].astype(np.int64) & 0xFFFFFFFF, ost[k]), k
        for k in ("sum_lt", "sum_shell_lt"):
            got = st[k].astype(np.float64) / 2.0 ** 20
            n = ost["volume"] if k == "sum_lt" else ost["n_shell"]
            # per voxel: single-precision sqrt (<= 2^-24 relative) then rounding
            # to 2^-20 (<= 2^-21 absolute)
            assert np.all(np.abs(got - ost[k]) <= n * 2.0 ** -21 + ost[k] * 2.0 ** -23), k
    return d, l2


@pytest.mark.parametrize("ndim", [2, 3])
def test_random_small_masks(lt, ndim):
    """Ragged sizes (not multiples of any tile), random density, labelled by
    connected component; every third case splits components so that
    different labels touch."""
    import scipy.ndimage as ndi
    rng = np.random.default_rng(40 + ndim)
    for t in range(25):
        if ndim == 2:
            shape = (int(rng.integers(1, 90)), int(rng.integers(1, 90)))
        else:
            shape = tuple(int(v) for v in rng.integers(1, 30, size=3))
        f = ndi.gaussian_filter(rng.random(shape), rng.uniform(0.5, 2.5))
        mask = (f > np.quantile(f, rng.uniform(0.2, 0.8))).astype(np.uint8)
        labels = ndi.label(mask)[0].astype(np.uint32)
        if t % 3 == 0 and labels.max() > 0:
            labels[(labels > 0) & (rng.random(shape) < 0.2)] = labels.max() + 1
        if t % 4 == 1:  # unlabelled foreground
            labels[(labels > 0) & (rng.random(shape) < 0.1)] = 0
        check_full(lt, mask, labels, int(labels.max()) + 2, separate=(t % 2 == 0))


def test_ellipses_2d_256(lt):
    m, l, n = synth.workload("ellipses_2d_256", 0)
    check_full(lt, m, l, n, separate=True)


def test_ellipsoids_3d_128(lt):
    m, l, n = synth.workload("ellipsoids_3d_128", 0)
    check_full(lt, m, l, n, separate=True)
    check_full(lt, m, l, n)


def test_long_axes_use_every_column_path(lt):
    """Axis lengths that select the 32-, 16- and 8-column shared-memory tiles
    and the global-memory column pass."""
    import scipy.ndimage as ndi
    rng = np.random.default_rng(3)
    for shape in [(700, 37), (1500, 21), (2500, 9), (600, 20, 24), (1100, 9, 17), (2100, 6, 8)]:
        f = ndi.gaussian_filter(rng.random(shape), 4.0)
        mask = (f > np.quantile(f, 0.3)).astype(np.uint8)
        labels = ndi.label(mask)[0].astype(np.uint32)
        check_full(lt, mask, labels, int(labels.max()) + 1)


def test_degenerate_inputs(lt):
    cases = []
    cases.append((np.zeros((17, 33), np.uint8), None))
    cases.append((np.ones((9, 10, 11), np.uint8), None))
    one = np.zeros((5, 6, 7), np.uint8)
    one[2, 3, 4] = 1
    cases.append((one, None))
    cases.append((np.ones((1, 1), np.uint8), None))
    cases.append((np.ones((1, 64), np.uint8), None))
    cases.append((np.ones((64, 1), np.uint8), None))
    cases.append((np.ones((40, 1, 1), np.uint8), None))
    line = np.zeros((8, 8, 8), np.uint8)
    line[4, 4, :] = 1
    cases.append((line, None))
    for mask, labels in cases:
        labels = mask.astype(np.uint32) if labels is None else labels
        check_full(lt, mask, labels, 3)


def test_digital_balls(lt):
    for r in (5, 10, 20):
        n = 2 * r + 5
        g = np.indices((n, n, n)) - n // 2
        ball = ((g ** 2).sum(0) <= r * r).astype(np.uint8)
        _, l2, S, R, _ = gpu_pipeline(lt, ball, ball.astype(np.uint32), 2)
        assert np.all(l2[ball > 0] == l2.max())
        assert abs(R[1] - 1.0) <= 1e-6 and S[1] < 1.0


def test_full_size_particles_512_whole_volume(lt):
    """The 512^3 particle volume (5,000 objects) in the benchmark's launch
    configuration (lt_measure on the whole volume), against the oracle on
    the whole volume: DT2 and LT2 of every voxel bit for bit, S and R of
    every object within 1e-5, plus properties that hold at any size."""
    mask, labels, n = synth.workload("particles_3d_512", 0)
    d, l2, S, R, _ = gpu_pipeline(lt, mask, labels, n)
    d_ref = oracle.dt2(mask)
    assert np.array_equal(d, d_ref), "DT2"
    del d_ref
    l_ref = oracle.lt2(d, labels)
    assert np.array_equal(l2, l_ref), "LT2"
    S_ref, R_ref, _ = oracle.measures(labels, l_ref, n)
    assert_close(S, S_ref, "sphericity")
    assert_close(R, R_ref, "roundness")
    on = labels != 0
    assert np.array_equal(d == 0, mask == 0)
    assert np.all(l2[on] >= d[on]) and np.all(l2[~on] == 0)
    vols = np.bincount(labels.reshape(-1), minlength=n)
    f = ~np.isnan(S)
    assert np.all(S[f] <= 1 + 1e-6) and np.all(R[f] <= 1 + 1e-6) and np.all(R[f] > 0)
    assert np.isnan(S[0]) and np.array_equal(np.isnan(S[1:]), vols[1:] == 0)


def test_large_thick_objects_whole_volume(lt):
    """Forty big ellipsoids and superellipsoids in 256^3 (equivalent radii
    ~20-50 voxels, volumes up to ~5e5 voxels, 33% foreground): long EDT scans
    and many kept centres with r^2 > 200, painted row by row. Whole volume
    against the oracle."""
    mask, labels, n = synth.workload("large_3d_256", 0)
    vols = np.bincount(labels.reshape(-1))[1:]
    assert vols.max() > 1.5e5 and mask.mean() > 0.32
    d, l2 = check_full(lt, mask, labels, n)
    assert np.count_nonzero(d > 400) > 10000  # radii above 20 voxels


def test_solid_ball_radius_100(lt):
    """One digital ball of radius 100 (47% of a 208^3 volume): DT2 against
    scipy's exact EDT of the padded mask; LT2 by the closed form (every
    voxel of a digital ball lies in the centre's ball, so LT2 is DT2 at the
    centre everywhere, the least sum of three squares above r^2 = 10^4, i.e.
    10001); S and R against the oracle's formulas on that LT2 (R = 1)."""
    import scipy.ndimage as ndi
    mask, labels, n = synth.workload("solid_ball_3d_208", 0)
    d, l2, S, R, _ = gpu_pipeline(lt, mask, labels, n)
    e = ndi.distance_transform_edt(np.pad(mask, 1))[1:-1, 1:-1, 1:-1]
    assert np.array_equal(d, np.rint(e * e).astype(np.uint32)), "DT2"
    c = tuple(s // 2 for s in mask.shape)
    assert d[c] == 10001
    want = np.where(mask > 0, np.uint32(10001), np.uint32(0))
    assert np.array_equal(l2, want), "LT2"
    S_ref, R_ref, _ = oracle.measures(labels, want, n)
    assert abs(R_ref[1] - 1.0) < 1e-9  # exactly 1 up to the FP64 sums
    assert_close(S, S_ref, "sphericity")
    assert_close(R, R_ref, "roundness")


def test_device_detected_errors(lt):
    import torch
    m, l, n = synth.workload("ellipses_2d_256", 2)
    bad = l.copy()
    bad[0, 0] = 1  # a labelled voxel outside the mask
    mt = torch.from_numpy(m).cuda()
    dt2 = torch.empty(m.shape, dtype=torch.int32, device="cuda")
    lt2 = torch.empty_like(dt2)
    lt.lt_edt(mt, dt2)
    ws = lt.lt_local_thickness(dt2, dev_u32(bad), lt2)
    with pytest.raises(lt.LTError) as e:
        lt.lt_workspace_status(ws)
    assert e.value.status == 5
    # labels beyond n_labels are reported and skipped
    ws = lt.lt_local_thickness(dt2, dev_u32(l), lt2)
    lt.lt_workspace_status(ws)
    S = torch.empty(5, dtype=torch.float32, device="cuda")
    ws = lt.lt_shape_measures(dev_u32(l), lt2, 5, S, None)
    with pytest.raises(lt.LTError) as e:
        lt.lt_workspace_status(ws)
    assert e.value.status == 4
    _, l_ref, S_ref, _ = oracle.pipeline(m, np.where(l < 5, l, 0).astype(np.uint32), 5)
    assert_close(S.cpu().numpy(), S_ref, "S with out-of-range labels skipped")


def test_host_buffer_entry_matches_device_path(lt):
    """The host-buffer entry copies in z-slabs and runs the ridge pass slab by
    slab as the labels land; it must give the device path's bits: for slab
    counts that do not divide the volume, in 2D, with touching labels
    (painting then tests labels), and with a ball thicker than the thinnest
    slab."""
    import torch
    import scipy.ndimage as ndi
    rng = np.random.default_rng(8)
    f = ndi.gaussian_filter(rng.random((70, 45, 36)), 2.0)
    rag = (f > np.quantile(f, 0.5)).astype(np.uint8)
    rag_l = ndi.label(rag)[0].astype(np.uint32)
    m2, l2, n2 = synth.workload("ellipsoids_3d_128", 2)
    touch = l2.copy()
    half = (np.indices(l2.shape)[2] >= 64) & (l2 > 0)
    touch[half] += np.uint32(n2)  # halves of objects cut at x = 64 touch their other half
    g = np.indices((100, 40, 40)) - np.array([50, 20, 20]).reshape(3, 1, 1, 1)
    big = ((g ** 2).sum(0) <= 12 ** 2).astype(np.uint8)  # radius 12 > the 4-plane last slab
    big[5:9, 3:7, 3:7] = 1
    big_l = ndi.label(big)[0].astype(np.uint32)
    cases = [synth.workload("ellipsoids_3d_128", 1), synth.workload("ellipses_2d_256", 2),
             (rag, rag_l, int(rag_l.max()) + 1), (m2, touch, 2 * n2), (big, big_l, int(big_l.max()) + 1)]
    for m, l, n in cases:
        _, _, S_dev, R_dev, _ = gpu_pipeline(lt, m, l, n)
        mh = torch.from_numpy(m).pin_memory()
        lh = torch.from_numpy(l.view(np.int32)).pin_memory()
        Sh = torch.empty(n, dtype=torch.float32).pin_memory()
        Rh = torch.empty(n, dtype=torch.float32).pin_memory()
        ws = lt.workspace(lt.lt_measure_host_workspace_size(n, m.shape), "cuda")
        lt.lt_measure_host(mh, lh, n, Sh, Rh, ws)
        assert np.array_equal(Sh.numpy(), S_dev, equal_nan=True)
        assert np.array_equal(Rh.numpy(), R_dev, equal_nan=True)


def test_repeated_calls_reuse_workspace(lt):
    """Same workspace, different volumes: results do not leak across calls."""
    import torch
    ws = None
    for seed in (3, 4, 3):
        m, l, n = synth.workload("ellipses_2d_256", seed)
        mt, lt_ = torch.from_numpy(m).cuda(), dev_u32(l)
        dt2 = torch.empty(m.shape, dtype=torch.int32, device="cuda")
        lt2 = torch.empty_like(dt2)
        S = torch.empty(64, dtype=torch.float32, device="cuda")
        R = torch.empty_like(S)
        if ws is None:
            ws = lt.workspace(lt.lib.lt_measure_workspace_size(64, 2, 256, 256, 1), "cuda")
        lt.lt_measure(mt, lt_, 64, dt2, lt2, S, R, ws=ws)
        lt.lt_workspace_status(ws)
        _, _, S_ref, R_ref = oracle.pipeline(m, l, 64)
        assert_close(S.cpu().numpy(), S_ref, "S")
        assert_close(R.cpu().numpy(), R_ref, "R")


@pytest.mark.parametrize("bound", [200, 324])
def test_crescent_table_bounds(lt, bound):
    """Rotated ellipsoids whose inscribed-ball radii run up to and across the
    edge of the tabulated crescents (r^2 = 324; 200 was the edge of an
    earlier, smaller table): kept centres on both sides of it, painted from
    tables and row by row, next to each other in one object."""
    rng = np.random.default_rng(7)
    sets = {200: [(14.5, 17.0, 18.0), (14.3, 16.5, 22.0), (14.9, 14.9, 25.0)],
            324: [(18.5, 21.0, 22.0), (18.3, 20.5, 26.0), (18.9, 18.9, 30.0)]}
    lo = {200: 144, 324: 256}[bound]
    for axes in sets[bound]:
        n = int(2 * max(axes)) + 5
        g = np.indices((n, n, n)).reshape(3, -1).T - (n - 1) / 2.0
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        w, x, y, z = q
        rot = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
        u = g @ rot
        mask = (((u / np.array(axes)) ** 2).sum(1) <= 1.0).reshape(n, n, n).astype(np.uint8)
        d, _ = check_full(lt, mask, mask.astype(np.uint32), 2)
        r2 = d[mask > 0]
        assert r2.max() > bound and np.count_nonzero((r2 > lo) & (r2 <= bound)) > 0


@pytest.mark.parametrize("shape", [(64, 80), (64, 81), (4, 16, 80)])
def test_fixed_point_lt_of_every_small_value(lt, shape):
    """Each voxel its own object with LT2 = 1, 2, ...: the per-object LT sum
    is exactly round(sqrtf(LT2) * 2^20) (float32 square root, rounding half
    to even), for the tabulated small values and the computed larger ones,
    in the four-voxel (nx % 4 == 0) and the one-voxel reduction."""
    import torch
    n = int(np.prod(shape))
    t = np.arange(1, n + 1, dtype=np.uint32).reshape(shape)
    labels = t.copy()
    S = torch.empty(n + 1, dtype=torch.float32, device="cuda")
    R = torch.empty_like(S)
    stats = {k: torch.empty(n + 1, dtype=torch.int32, device="cuda") for k in ("volume", "n_shell", "max_lt2")}
    stats.update({k: torch.empty(n + 1, dtype=torch.int64, device="cuda") for k in ("sum_lt", "sum_shell_lt")})
    ws = lt.lt_shape_measures(dev_u32(labels), dev_u32(t), n + 1, S, R, stats)
    lt.lt_workspace_status(ws)
    want = np.rint(np.sqrt(np.arange(1, n + 1, dtype=np.float32)) * np.float32(2.0 ** 20)).astype(np.int64)
    got = stats["sum_lt"].cpu().numpy()[1:]
    assert np.array_equal(got, want)
    assert np.array_equal(stats["sum_shell_lt"].cpu().numpy()[1:], want)  # every one-voxel object is shell
    assert np.array_equal(stats["max_lt2"].cpu().numpy()[1:], np.arange(1, n + 1))


def test_pointers_of_another_device_are_rejected(lt):
    """The library never changes the caller's current device: a host
    pointer, or (with two GPUs) a buffer or stream of another device, is an
    argument error returned before anything is enqueued, and the current
    device stays what it was."""
    import ctypes
    import torch
    E = {v: k for k, v in lt.STATUS_NAMES.items()}
    m = torch.zeros((8, 8, 8), dtype=torch.uint8, device="cuda")
    dt2 = torch.empty((8, 8, 8), dtype=torch.int32, device="cuda")
    host = torch.zeros((8, 8, 8), dtype=torch.uint8).pin_memory()
    ws = lt.workspace(lt.lib.lt_edt_workspace_size(3, 8, 8, 8), "cuda")
    args = (3, 8, 8, 8, ctypes.c_void_p(ws.data_ptr()), ws.numel(), None)
    assert lt.lib.lt_edt(ctypes.c_void_p(host.data_ptr()), ctypes.c_void_p(dt2.data_ptr()), *args) == \
        E["LT_ERR_INVALID_ARG"]
    assert lt.lib.lt_edt(ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(dt2.data_ptr()), *args) == 0
    if torch.cuda.device_count() < 2:
        return
    dev0 = torch.cuda.current_device()
    other = (dev0 + 1) % torch.cuda.device_count()
    dt2_other = torch.empty((8, 8, 8), dtype=torch.int32, device=f"cuda:{other}")
    assert lt.lib.lt_edt(ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(dt2_other.data_ptr()), *args) == \
        E["LT_ERR_INVALID_ARG"]
    assert torch.cuda.current_device() == dev0
    s_other = torch.cuda.Stream(device=other)
    assert lt.lib.lt_edt(ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(dt2.data_ptr()), 3, 8, 8, 8,
                         ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.c_void_p(s_other.cuda_stream)) == \
        E["LT_ERR_INVALID_ARG"]
    assert torch.cuda.current_device() == dev0
