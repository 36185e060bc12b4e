"""Pins for the oracle's distance transform and local thickness.

Each check ties the oracle to something other than itself: brute force over
all point pairs, scipy's exact Euclidean feature transform, lattice-point
counts of digital balls and discs (OEIS A000605, A000328), Legendre's
three-square theorem, and a small case worked by hand.
"""
import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle

pytestmark = pytest.mark.usefixtures("built_cpu_parts")


def _random_mask(rng, shape):
    return (rng.random(shape) < rng.uniform(0.3, 0.97)).astype(np.uint8)


@pytest.mark.parametrize("ndim", [2, 3])
def test_dt2_equals_all_pairs_brute_force(ndim):
    rng = np.random.default_rng(100 + ndim)
    for _ in range(150):
        shape = tuple(int(v) for v in rng.integers(1, 14 if ndim == 2 else 9, size=ndim))
        m = _random_mask(rng, shape)
        assert np.array_equal(oracle.dt2(m), oracle.dt2_brute(m)), shape


def _scipy_dt2(mask):
    """Exact squared distances from scipy's feature transform on the padded mask."""
    pm = np.pad(mask != 0, 1)
    ind = ndi.distance_transform_edt(pm, return_distances=False, return_indices=True)
    g = np.indices(pm.shape)
    d = ((ind - g) ** 2).sum(0)
    return d[tuple(slice(1, -1) for _ in range(mask.ndim))].astype(np.uint32)


@pytest.mark.parametrize("shape", [(97, 131), (40, 45, 50)])
def test_dt2_equals_scipy_exact_edt(shape):
    rng = np.random.default_rng(7)
    # smooth blobs so that distances grow well beyond 1
    f = ndi.gaussian_filter(rng.random(shape), 3.0)
    m = (f > np.quantile(f, 0.4)).astype(np.uint8)
    assert np.array_equal(oracle.dt2(m), _scipy_dt2(m))


def test_dt2_solid_box_is_distance_to_the_padding():
    shape = (6, 9, 11)
    m = np.ones(shape, np.uint8)
    g = np.indices(shape)
    want = np.min([np.minimum(g[a] + 1, shape[a] - g[a]) for a in range(3)], axis=0) ** 2
    assert np.array_equal(oracle.dt2(m), want.astype(np.uint32))


def test_dt2_edge_cases():
    assert oracle.dt2(np.zeros((4, 5), np.uint8)).max() == 0
    one = np.zeros((3, 3, 3), np.uint8)
    one[1, 1, 1] = 1
    d = oracle.dt2(one)
    assert d[1, 1, 1] == 1 and d.sum() == 1
    assert oracle.dt2(np.ones((1, 1), np.uint8))[0, 0] == 1
    assert np.array_equal(oracle.dt2(np.ones((1, 7), np.uint8)), np.ones((1, 7), np.uint32))


def _next_sum_of_three_squares(n):
    """Smallest integer > n that is a sum of three squares: by Legendre's
    theorem, every integer not of the form 4^a (8b + 7)."""
    k = n + 1
    while True:
        m = k
        while m % 4 == 0:
            m //= 4
        if m % 8 != 7:
            return k
        k += 1


def _ball(r, ndim):
    n = 2 * r + 5
    g = np.indices((n,) * ndim) - n // 2
    return ((g ** 2).sum(0) <= r * r).astype(np.uint8), n // 2


# lattice points in a ball / disc of radius r (OEIS A000605 and A000328)
BALL_COUNT = {5: 515, 10: 4169, 20: 33401}
DISC_COUNT = {5: 81, 10: 317, 20: 1257}


@pytest.mark.parametrize("r", [5, 10, 20])
def test_digital_ball_and_disc(r):
    for ndim, counts in ((3, BALL_COUNT), (2, DISC_COUNT)):
        m, c = _ball(r, ndim)
        assert int(m.sum()) == counts[r]
        d = oracle.dt2(m)
        centre = (c,) * ndim
        # nearest lattice point outside the ball; in 2D it is (r, 1) or
        # (r+1, 0): for these radii r^2 + 1 is always a sum of two squares
        want = _next_sum_of_three_squares(r * r) if ndim == 3 else r * r + 1
        assert int(d[centre]) == want
        lt = oracle.lt2(d, m.astype(np.uint32))
        # every ball voxel lies in the centre's ball, which has the largest radius
        assert np.all(lt[m > 0] == want)
        assert np.all(lt[m == 0] == 0)


def test_lt2_equals_all_pairs_brute_force():
    rng = np.random.default_rng(5)
    for t in range(120):
        ndim = 2 + (t % 2)
        shape = tuple(int(v) for v in rng.integers(2, 13 if ndim == 2 else 8, size=ndim))
        m = _random_mask(rng, shape)
        lab = ndi.label(m)[0].astype(np.uint32)
        if t % 3 == 0:  # touching objects: split one component by a second label
            lab[(lab > 0) & (rng.random(shape) < 0.3)] = lab.max() + 1
        d = oracle.dt2(m)
        assert np.array_equal(oracle.lt2(d, lab), oracle.lt2_brute(d, lab)), shape


def test_lt2_bounds_and_object_maximum():
    rng = np.random.default_rng(11)
    f = ndi.gaussian_filter(rng.random((40, 44, 48)), 2.5)
    m = (f > np.quantile(f, 0.55)).astype(np.uint8)
    lab = ndi.label(m)[0].astype(np.uint32)
    d = oracle.dt2(m)
    lt = oracle.lt2(d, lab)
    on = lab > 0
    assert np.all(lt[on] >= d[on]) and np.all(lt[~on] == 0)
    for l in range(1, int(lab.max()) + 1):
        sel = lab == l
        assert lt[sel].max() == d[sel].max()


def test_worked_rectangle_2d():
    """A 3x5 rectangle in a 5x7 image, worked by hand.

    DT2: the 12 rim pixels touch background (1); the three inner pixels of
    the middle row are two steps from background above, below and beside (4).
    LT2: the radius-2 balls of the inner pixels reach every rectangle pixel
    (the farthest, a corner, is at squared distance 2 from the nearest inner
    pixel), so LT2 = 4 everywhere on the rectangle.
    """
    m = np.zeros((5, 7), np.uint8)
    m[1:4, 1:6] = 1
    d = oracle.dt2(m)
    want_d = np.zeros((5, 7), np.uint32)
    want_d[1:4, 1:6] = 1
    want_d[2, 2:5] = 4
    assert np.array_equal(d, want_d)
    lt = oracle.lt2(d, m.astype(np.uint32))
    assert np.array_equal(lt, 4 * m.astype(np.uint32))


def test_objects_match_full_volume():
    import synth
    m, lab, n = synth.workload("ellipsoids_3d_128", 3)
    d = oracle.dt2(m)
    lt = oracle.lt2(d, lab)
    got = oracle.objects_dt2_lt2(m, lab, [1, 9, 25, n - 1])
    for l, (idx, dd, ll) in got.items():
        assert np.array_equal(np.sort(idx), np.flatnonzero(lab.reshape(-1) == l))
        assert np.array_equal(dd, d.reshape(-1)[idx])
        assert np.array_equal(ll, lt.reshape(-1)[idx])
