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


def _labels_digest(threads):
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import hashlib, synth; m, l, n = synth.workload('particles_3d_96', 4); "
            "print(hashlib.sha256(l.tobytes()).hexdigest(), n)")
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=root,
                       env=env, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout.strip()


def test_packed_growth_is_thread_independent():
    """The growth pass runs its rounds in parallel; one thread and several
    must give the same volume."""
    assert _labels_digest(1) == _labels_digest(4)


def test_packed_growth_fills_free_space():
    """Growth adds foreground, keeps every particle's old voxels, keeps the
    one-voxel gap and the faces clear."""
    shape = (128, 128, 128)
    n = synth.particles_per_volume(128)
    m0, lab0, _ = synth.packed(shape, n, 8.0, 18.0, 3)
    m1, lab1, _ = synth.packed(shape, n, 8.0, 18.0, 3, grow=2.0)
    assert m1.mean() > m0.mean() + 0.02
    keep = lab0 != 0
    assert np.array_equal(lab1[keep], lab0[keep])
    assert not _touching(lab1)
    for a in range(3):
        assert not np.take(m1, [0, shape[a] - 1], axis=a).any()
