"""Pins for the oracle's shape statistics and formulas (Sec. 4.1, 4.2).

Independent references: numeric quadrature of a spheroid's surface of
revolution, the complete elliptic integral of the second kind for an
ellipse perimeter, the sphere/circle limits, scipy's binary erosion for the
shell, and per-object Python loops for the sums.
"""
import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.ndimage as ndi
import scipy.special as sp

import oracle

pytestmark = pytest.mark.usefixtures("built_cpu_parts")


def _quad_area(a, c):
    """Surface of revolution of x(z) = a sqrt(1 - z^2/c^2), |z| <= c:
    2 pi * integral of sqrt(x^2 + (x x')^2) dz, with x x' = -a^2 z / c^2."""
    f = lambda z: math.sqrt(a * a * (1 - z * z / (c * c)) + (a * a * z / (c * c)) ** 2)
    val, _ = si.quad(f, -c, c, epsabs=0, epsrel=1e-13, limit=200)
    return 2 * math.pi * val


@pytest.mark.parametrize("a,c", [(1, 2), (2, 1), (3.7, 0.4), (0.5, 9.0), (5, 5.001), (5, 4.999),
                                 (1.0, 1.0 + 1e-7), (7.3, 2.2)])
def test_spheroid_area_matches_quadrature(a, c):
    assert oracle.spheroid_area(a, c) == pytest.approx(_quad_area(a, c), rel=1e-11)


def test_spheroid_area_printed_reading_values():
    # the eccentricity with its square root; without it these would be 20.49
    # and 39.40
    assert oracle.spheroid_area(1, 2) == pytest.approx(21.4784, abs=5e-5)
    assert oracle.spheroid_area(2, 1) == pytest.approx(34.6875, abs=5e-5)
    assert oracle.spheroid_area(3, 3) == pytest.approx(4 * math.pi * 9, rel=1e-15)


def test_ramanujan_against_elliptic_integral():
    # circle: 2 pi r exactly
    assert oracle.ramanujan_perimeter(2.5, 2.5) == pytest.approx(5 * math.pi, rel=1e-15)
    for ratio in np.linspace(0.02, 1.0, 50):
        a, b = 3.0, 3.0 * ratio
        exact = 4 * a * sp.ellipe(1 - (b / a) ** 2)
        r1 = oracle.ramanujan_perimeter(a, b)
        assert r1 <= exact * (1 + 1e-14)  # the first approximation underestimates
        assert abs(r1 / exact - 1) < (1e-5 if ratio >= 0.5 else 5e-3)
        assert oracle.ramanujan_perimeter(b, a) == pytest.approx(r1, rel=1e-15)


def test_sphericity_3d_of_true_spheroids():
    """For a spheroid with semi-axes (a, a, c), V = 4/3 pi a^2 c and mean
    width a must give Wadell's sphericity with the true surface area."""
    for a, c in [(2.0, 2.0), (2.0, 5.0), (4.0, 1.0), (1.3, 1.31)]:
        V = 4.0 / 3.0 * math.pi * a * a * c
        wadell = math.pi ** (1 / 3) * (6 * V) ** (2 / 3) / _quad_area(a, c)
        assert oracle.sphericity_3d(V, a) == pytest.approx(wadell, rel=1e-10)
    assert oracle.sphericity_3d(4 / 3 * math.pi * 8.0, 2.0) == pytest.approx(1.0, abs=1e-14)


def test_sphericity_is_at_most_one():
    rng = np.random.default_rng(0)
    for _ in range(500):
        a = rng.uniform(0.5, 20)
        V = rng.uniform(0.1, 50) * a ** 3
        assert oracle.sphericity_3d(V, a) <= 1 + 1e-12
        A = rng.uniform(0.1, 50) * a ** 2
        assert oracle.sphericity_2d(A, a) <= 1 + 1e-12


def test_sphericity_2d_of_true_ellipses():
    for a, b in [(3.0, 3.0), (3.0, 1.5), (1.0, 4.0)]:
        A = math.pi * a * b
        exact_perim = 4 * max(a, b) * sp.ellipe(1 - (min(a, b) / max(a, b)) ** 2)
        want = 2 * math.sqrt(math.pi * A) / exact_perim
        tol = 2e-5 if min(a, b) / max(a, b) >= 0.5 else 5e-3  # Ramanujan's own error
        assert oracle.sphericity_2d(A, a) == pytest.approx(want, rel=tol)
    assert oracle.sphericity_2d(math.pi * 4.0, 2.0) == pytest.approx(1.0, abs=1e-14)


def test_shell_matches_binary_erosion():
    rng = np.random.default_rng(3)
    for ndim in (2, 3):
        shape = (60, 70) if ndim == 2 else (30, 34, 38)
        f = ndi.gaussian_filter(rng.random(shape), 2.0)
        lab = ndi.label(f > np.quantile(f, 0.5))[0].astype(np.uint32)
        shell = oracle.shell_mask(lab)
        cross = ndi.generate_binary_structure(ndim, 1)
        want = np.zeros(shape, bool)
        for l in range(1, lab.max() + 1):
            obj = lab == l
            want |= obj & ~ndi.binary_erosion(obj, cross, border_value=0)
        assert np.array_equal(shell, want)


def test_object_stats_against_loops():
    rng = np.random.default_rng(9)
    lab = rng.integers(0, 4, size=(6, 7, 8)).astype(np.uint32)
    lt2 = np.where(lab > 0, rng.integers(1, 50, size=lab.shape), 0).astype(np.uint32)
    st = oracle.object_stats(lab, lt2, 5)
    sh = oracle.shell_mask(lab)
    for l in range(1, 5):
        V = ns = 0
        s1 = s2 = 0.0
        mx = 0
        for p in zip(*np.nonzero(lab == l)):
            V += 1
            v = math.sqrt(int(lt2[p]))
            s1 += v
            mx = max(mx, int(lt2[p]))
            if sh[p]:
                ns += 1
                s2 += v
        assert st["volume"][l] == V and st["n_shell"][l] == ns and st["max_lt2"][l] == mx
        assert st["sum_lt"][l] == pytest.approx(s1, rel=1e-14)
        assert st["sum_shell_lt"][l] == pytest.approx(s2, rel=1e-14)
        # assembly of S and R from the loop sums (mean over the object, mean
        # over the shell, largest LT)
        S, R, _ = oracle.measures(lab, lt2, 5)
        if V == 0:
            assert np.isnan(S[l]) and np.isnan(R[l])
            continue
        assert S[l] == pytest.approx(oracle.sphericity_3d(V, s1 / V), rel=1e-13)
        assert R[l] == pytest.approx((s2 / ns) / math.sqrt(mx), rel=1e-13)
    assert st["volume"][4] == 0


def test_digital_balls_round_and_near_spherical():
    """Digital balls of radius 5, 10, 20: LT is constant (see the DT/LT pins),
    so R = 1; S tends to 1 from below as the ball gets finer."""
    prev = 0.0
    for r in (5, 10, 20):
        n = 2 * r + 5
        g = np.indices((n, n, n)) - n // 2
        ball = ((g ** 2).sum(0) <= r * r).astype(np.uint32)
        d = oracle.dt2(ball)
        S, R, _ = oracle.measures(ball, oracle.lt2(d, ball), 2)
        assert R[1] == pytest.approx(1.0, abs=1e-13)
        assert prev < S[1] < 1.0
        prev = S[1]
    assert prev == pytest.approx(0.999991, abs=1e-6)


def test_worked_rectangle_measures():
    """3x5 rectangle (LT = 2 everywhere, worked in the DT/LT pins).
    A = 15, a = 2, b = 15 / (2 pi); Ramanujan P_o = 13.810054, P_c =
    2 sqrt(15 pi) = 13.729368, S = 0.994157. Shell: 12 rim pixels, R = 2/2."""
    m = np.zeros((5, 7), np.uint32)
    m[1:4, 1:6] = 1
    S, R, st = oracle.measures(m, 4 * m, 2)
    assert st["n_shell"][1] == 12 and st["volume"][1] == 15
    assert S[1] == pytest.approx(0.994157, abs=1e-6)
    assert R[1] == pytest.approx(1.0, abs=1e-15)


def test_absent_labels_are_nan():
    lab = np.zeros((4, 4), np.uint32)
    lab[1:3, 1:3] = 2
    S, R, _ = oracle.measures(lab, lab * 2, 4)
    assert np.isnan(S[0]) and np.isnan(S[1]) and np.isnan(S[3]) and np.isfinite(S[2])
    assert np.isnan(R[1]) and np.isfinite(R[2])
