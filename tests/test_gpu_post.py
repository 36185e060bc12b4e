"""GPU parity of the post-processing entry points with the oracle:
roughness-filtered shape measures (objects reduced to their voxels with
LT2 >= min_lt2) and roundness mapped to 0-1 (Sec. 6.1, Sec. 7)."""
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


def gpu_filtered(lt, labels, l2, n, min_lt2):
    import torch
    lab = torch.from_numpy(np.ascontiguousarray(labels, np.uint32).view(np.int32)).cuda()
    t2 = torch.from_numpy(np.ascontiguousarray(l2, np.uint32).view(np.int32)).cuda()
    S = torch.empty(n, dtype=torch.float32, device="cuda")
    R = torch.empty_like(S)
    stats = {k: torch.empty(n, dtype=torch.int32, device="cuda") for k in ("volume", "n_shell", "max_lt2")}
    stats.update({k: torch.empty(n, dtype=torch.int64, device="cuda") for k in ("sum_lt", "sum_shell_lt")})
    ws = lt.lt_shape_measures_filtered(lab, t2, n, min_lt2, S, R, stats)
    lt.lt_workspace_status(ws)
    return S.cpu().numpy(), R.cpu().numpy(), {k: v.cpu().numpy() for k, v in stats.items()}


def close(got, want):
    assert np.array_equal(np.isnan(got), np.isnan(want))
    ok = np.isfinite(want)
    assert np.all(np.abs(got[ok] - want[ok]) <= REL_TOL * np.abs(want[ok]))


@pytest.mark.parametrize("name", ["ellipsoids_3d_128", "ellipses_2d_256", "particles_3d_48"])
def test_filtered_measures_match_oracle(lt, name):
    mask, labels, n = synth.workload(name, 5)
    _, l2, S0, R0 = oracle.pipeline(mask, labels, n)
    for min_lt2 in (0, 1, 2, 5, 17, 50):
        S, R, st = gpu_filtered(lt, labels, l2, n, min_lt2)
        S_ref, R_ref, st_ref = oracle.measures_filtered(labels, l2, n, min_lt2)
        assert np.array_equal(st["volume"], st_ref["volume"].astype(np.int32))
        assert np.array_equal(st["n_shell"], st_ref["n_shell"].astype(np.int32))
        close(S, S_ref)
        close(R, R_ref)
        if min_lt2 <= 1:  # nothing is filtered
            close(S, S0)
            close(R, R0)


def test_filter_removes_a_spike(lt):
    n = 21
    g = np.indices((n, n, n)) - n // 2
    ball = ((g ** 2).sum(0) <= 36).astype(np.uint32)
    c = n // 2
    spiky = ball.copy()
    spiky[c, c, c + 7:c + 11] = 1
    l2s = oracle.lt2(oracle.dt2(spiky), spiky)
    l2b = oracle.lt2(oracle.dt2(ball), ball)
    Sf, Rf, _ = gpu_filtered(lt, spiky, l2s, 2, 2)
    Sb, Rb, _ = gpu_filtered(lt, ball, l2b, 2, 0)
    assert Sf[1] == Sb[1] and Rf[1] == Rb[1]
    Su, Ru, _ = gpu_filtered(lt, spiky, l2s, 2, 0)
    assert Ru[1] < Rf[1] - 1e-3


def test_roundness_rescale_matches_oracle(lt):
    import torch
    mask, labels, n = synth.workload("ellipsoids_3d_128", 6)
    _, _, _, R = oracle.pipeline(mask, labels, n)
    Rf = torch.from_numpy(R.astype(np.float32)).cuda()
    out = torch.empty_like(Rf)
    lt.lt_roundness_rescale(Rf, out)
    want = oracle.roundness_rescaled(R.astype(np.float32).astype(np.float64))
    got = out.cpu().numpy()
    assert np.array_equal(np.isnan(got), np.isnan(want))
    ok = np.isfinite(want)
    assert np.abs(got[ok] - want[ok]).max() <= 1e-6
    assert got[ok].min() == 0.0
    # a given minimum, in place
    lt.lt_roundness_rescale(Rf, Rf, r_min=0.7)
    want = oracle.roundness_rescaled(R.astype(np.float32).astype(np.float64), 0.7)
    got = Rf.cpu().numpy()
    assert np.abs(got[ok] - want[ok]).max() <= 1e-6
