"""Pins for the oracle's post-processing of the measures: roughness filtering
(objects reduced to the union of their inscribed balls of squared radius >=
min_lt2; the paper leaves the filter open, Sec. 7) and roundness mapped to
0-1 with the reported minimum (Sec. 6.1).

Independent references: all-pairs brute force of the ball union from the
definition, a digital ball with a one-voxel spike (the filter must give back
exactly the plain ball), and closed forms for the rescaling.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.usefixtures("built_cpu_parts")


def _ball(r, n):
    g = np.indices((n, n, n)) - n // 2
    return ((g ** 2).sum(0) <= r * r).astype(np.uint32)


def test_spike_is_filtered_away_exactly():
    """A digital ball of radius 6 with a 4-voxel spike along +x. The spike's
    voxels lie only in balls of r^2 = 1; every ball voxel lies in the
    centre's ball (r^2 = 37). Filtering at r^2 >= 2 must give the plain
    ball's S and R bit for bit; unfiltered, the spike lowers R."""
    n = 21
    ball = _ball(6, n)
    c = n // 2
    spiky = ball.copy()
    spiky[c, c, c + 7:c + 11] = 1
    d = oracle.dt2(spiky)
    l2 = oracle.lt2(d, spiky)
    assert np.all(l2[c, c, c + 7:c + 11] == 1)
    S0, R0, _ = oracle.measures(ball, oracle.lt2(oracle.dt2(ball), ball), 2)
    Sf, Rf, st = oracle.measures_filtered(spiky, l2, 2, 2)
    assert st["volume"][1] == ball.sum()
    assert Sf[1] == S0[1] and Rf[1] == R0[1] == pytest.approx(1.0, abs=1e-13)
    Su, Ru, _ = oracle.measures(spiky, l2, 2)
    assert Ru[1] < Rf[1] - 1e-3
    # thresholds at or below 1 remove nothing
    S1, R1, _ = oracle.measures_filtered(spiky, l2, 2, 1)
    assert S1[1] == Su[1] and R1[1] == Ru[1]
    # above the largest radius everything goes: NaN
    Se, Re, _ = oracle.measures_filtered(spiky, l2, 2, 38)
    assert np.isnan(Se[1]) and np.isnan(Re[1])


def _union_of_big_balls(mask, labels, min_lt2):
    """Brute force: x stays when some same-label centre c with
    DT2(c) >= min_lt2 has |x - c|^2 <= DT2(c) (DT2 by all pairs too)."""
    d = oracle.dt2_brute(mask)
    coords = np.argwhere(np.ones(mask.shape, bool))
    flat_l = labels.reshape(-1)
    flat_d = d.reshape(-1)
    keep = np.zeros(mask.size, bool)
    cent = np.flatnonzero((flat_l != 0) & (flat_d.astype(np.int64) >= min_lt2))
    for i in np.flatnonzero(flat_l != 0):
        x = coords[i]
        for j in cent:
            if flat_l[j] == flat_l[i] and ((coords[j] - x) ** 2).sum() <= flat_d[j]:
                keep[i] = True
                break
    return np.where(keep.reshape(mask.shape), labels, 0)


@pytest.mark.parametrize("seed", range(6))
def test_filter_matches_brute_force_union(seed):
    rng = np.random.default_rng(seed)
    shape = (9, 10, 11) if seed % 2 else (17, 19)
    mask = (rng.random(shape) < 0.8).astype(np.uint8)
    labels = mask.astype(np.uint32) * (1 + (np.indices(shape)[0] >= shape[0] // 2)).astype(np.uint32)
    l2 = oracle.lt2(oracle.dt2(mask), labels)
    for min_lt2 in (2, 3, 5):
        kept = _union_of_big_balls(mask, labels, min_lt2)
        S, R, st = oracle.measures_filtered(labels, l2, 3, min_lt2)
        S_ref, R_ref, st_ref = oracle.measures(kept, l2, 3)
        assert np.array_equal(st["volume"], st_ref["volume"])
        assert np.array_equal(st["n_shell"], st_ref["n_shell"])
        assert np.array_equal(np.isnan(S), np.isnan(S_ref))
        ok = np.isfinite(S_ref)
        assert np.array_equal(S[ok], S_ref[ok]) and np.array_equal(R[ok], R_ref[ok])


def test_rescale_closed_forms():
    R = np.array([np.nan, 0.5, 0.75, 1.0, 0.625])
    out = oracle.roundness_rescaled(R)
    assert np.isnan(out[0])
    assert np.allclose(out[1:], [0.0, 0.5, 1.0, 0.25], rtol=0, atol=1e-15)
    out = oracle.roundness_rescaled(R, 0.6)  # a given minimum; values below it clamp to 0
    assert np.allclose(out[1:], [0.0, 0.375, 1.0, 0.0625], rtol=0, atol=1e-15)
    assert np.all(oracle.roundness_rescaled(np.array([np.nan, 1.0, 1.0]))[1:] == 1.0)
    # order preserving, minimum to 0, 1 to 1
    rng = np.random.default_rng(0)
    R = rng.uniform(0.3, 1.0, 100)
    out = oracle.roundness_rescaled(R)
    assert np.array_equal(np.argsort(out, kind="stable"), np.argsort(R, kind="stable"))
    assert out.min() == 0.0 and out.max() <= 1.0
