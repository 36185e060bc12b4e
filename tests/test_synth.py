"""The seeded generators: deterministic, labels inside the mask, particles
separated by background (no two labels 26-adjacent, 8-adjacent in 2D)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.usefixtures("built_cpu_parts")


def _touching(lab):
    p = np.pad(lab, 1)
    core = tuple(slice(1, -1) for _ in range(lab.ndim))
    bad = False
    for off in np.ndindex(*(3,) * lab.ndim):
        sl = tuple(slice(1 + o - 1, p.shape[a] - 1 + o - 1) for a, o in enumerate(off))
        nb = p[sl]
        bad |= bool(np.any((lab != 0) & (nb != 0) & (nb != lab)))
    return bad


@pytest.mark.parametrize("name", ["ellipses_2d_256", "ellipsoids_3d_128", "particles_3d_96",
                                  "ellipses_2d_300"])
def test_workloads(name):
    m, lab, n = synth.workload(name, 1)
    m2, lab2, n2 = synth.workload(name, 1)
    assert np.array_equal(m, m2) and np.array_equal(lab, lab2) and n == n2
    assert np.array_equal(m != 0, lab != 0)
    assert lab.max() <= n - 1
    assert not _touching(lab)
    assert m.mean() > 0.1
    m3, _, _ = synth.workload(name, 2)
    assert not np.array_equal(m, m3)
