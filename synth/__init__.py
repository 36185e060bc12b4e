"""Seeded synthetic labelled masks (the only module both the oracle tests and
the CUDA path take inputs from).

It draws and rasterises particles; it holds none of the measurement method.
The paper's own data (Krumbein charts, brightfield cells, a 400^3 mozzarella
micro-CT scan with 15,503 fat objects; Sec. 5.1) is not available, so these
generators stand in for it with particles of comparable size, shape variety
and packing density.

Workloads (named by what they are):
  ellipses_2d_256      2D 256x256, 20 ellipses, semi-axes U(4, 30) px, random
                       rotation, random sequential addition with a 1 px gap.
  ellipsoids_3d_128    3D 128^3, 50 ellipsoids, semi-axes U(4, 20), random
                       rotation; half carry 8-32 radial bumps of relative
                       amplitude U(0.10, 0.25).
  particles_3d_512     3D 512^3, 5000 particles: 40% ellipsoids (axis ratios
                       1-4), 30% superellipsoids (exponent 2-6), 30% convex
                       polyhedra (6-20 cuts); dense packing, then each
                       particle grown (scale factor up to 2) into the free
                       space around it; 1 voxel gap; 33.5% foreground.
  particles_3d_1024    3D 1024^3, ~1M particles of the same mix (equivalent
                       radius about 4.5).
  particles_3d_<n>     any edge n: the 512^3 mix at the same density.
  ellipses_2d_<n>      2D n x n dense ellipse packing.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_synth.so")
_SRC = os.path.join(_HERE, "synth.c")
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator into synth/_synth.so (gcc, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
             _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        i64, dbl, i32, u64 = ctypes.c_int64, ctypes.c_double, ctypes.c_int, ctypes.c_uint64
        vp = ctypes.c_void_p
        lib.synth_rsa.restype = i64
        lib.synth_rsa.argtypes = [vp, vp, i64, i64, i64, i32, i64, dbl, dbl, dbl, i32, i32,
                                  dbl, dbl, u64]
        lib.synth_packed.restype = i64
        lib.synth_packed.argtypes = [vp, vp, i64, i64, i64, i32, i64, dbl, dbl, dbl, dbl, dbl, dbl,
                                     dbl, u64]
        _lib = lib
    return _lib


def _alloc(shape):
    mask = np.zeros(shape, dtype=np.uint8)
    labels = np.zeros(shape, dtype=np.uint32)
    return mask, labels


def rsa(shape, n_obj, amin, amax, seed, bump_frac=0.0, bumps=(8, 32), amp=(0.10, 0.25)):
    """Random sequential addition of ellipses (2D) or ellipsoids (3D).

    shape is (ny, nx) or (nz, ny, nx). Returns (mask u8, labels u32, count).
    """
    lib = _load()
    ndim = len(shape)
    nz, ny, nx = (1,) + tuple(shape) if ndim == 2 else tuple(shape)
    mask, labels = _alloc(shape)
    cnt = lib.synth_rsa(mask.ctypes.data, labels.ctypes.data, nx, ny, nz, ndim, n_obj,
                        float(amin), float(amax), float(bump_frac), int(bumps[0]),
                        int(bumps[1]), float(amp[0]), float(amp[1]), seed)
    return mask, labels, int(cnt)


def packed(shape, n_obj, rmin, rmax, seed, f_ell=0.4, f_super=0.3, shrink=(1.0, 1.0), grow=1.0):
    """Dense packing of n_obj particles, one per cell of a weighted bisection;
    grow > 1 then scales each particle up, by at most that factor, into the
    free space around it (one-voxel gap kept)."""
    lib = _load()
    ndim = len(shape)
    nz, ny, nx = (1,) + tuple(shape) if ndim == 2 else tuple(shape)
    mask, labels = _alloc(shape)
    cnt = lib.synth_packed(mask.ctypes.data, labels.ctypes.data, nx, ny, nz, ndim, n_obj,
                           float(rmin), float(rmax), float(f_ell), float(f_super),
                           float(shrink[0]), float(shrink[1]), float(grow), seed)
    if cnt < 0:
        raise MemoryError("synth_packed: allocation failed")
    return mask, labels, int(cnt)


def ball(shape, r: int):
    """One digital ball |x - centre|^2 <= r^2 (integer r, centre at the
    middle voxel) labelled 1: a solid-dominated volume."""
    g = np.indices(shape, dtype=np.int64)
    d2 = sum((g[i] - shape[i] // 2) ** 2 for i in range(len(shape)))
    mask = (d2 <= r * r).astype(np.uint8)
    return mask, mask.astype(np.uint32), 1


def particles_per_volume(edge: int, ndim: int = 3, voxels_per_particle: float = 512**3 / 5000):
    return max(1, int(round(edge**ndim / voxels_per_particle)))


def workload(name: str, seed: int = 0):
    """Named workload -> (mask, labels, n_labels) with n_labels = count + 1."""
    if name == "ellipses_2d_256":
        m, l, c = rsa((256, 256), 20, 4.0, 30.0, seed)
    elif name == "ellipsoids_3d_128":
        m, l, c = rsa((128, 128, 128), 50, 4.0, 20.0, seed, bump_frac=0.5)
    elif name == "particles_3d_1024":
        m, l, c = packed((1024, 1024, 1024), 1 << 20, 3.0, 6.0, seed)
    elif name == "large_3d_256":
        # big, thick objects (equivalent radius ~20-50, volumes ~1e4-5e5
        # voxels, the paper's micro-CT range): ellipsoids and superellipsoids
        m, l, c = packed((256, 256, 256), 40, 20.0, 60.0, seed, f_ell=0.25, f_super=0.75)
    elif name == "solid_ball_3d_208":
        m, l, c = ball((208, 208, 208), 100)
    elif name.startswith("particles_3d_"):
        n = int(name.rsplit("_", 1)[1])
        m, l, c = packed((n, n, n), particles_per_volume(n), 8.0, 18.0, seed, grow=2.0)
    elif name.startswith("ellipses_2d_"):
        n = int(name.rsplit("_", 1)[1])
        m, l, c = packed((n, n), max(1, int(round(n * n / 900.0))), 8.0, 18.0, seed,
                         shrink=(0.72, 0.86))
    else:
        raise KeyError(name)
    return m, l, c + 1


def mlp_initial_params(seed: int, n_features: int = 48, hidden: int = 64):
    """Seeded initial parameters of the 48-64-64-1 sphericity-correction
    network (random inputs shared by the CUDA path and the oracle): weights
    uniform in +-sqrt(6 / fan_in) (the last layer scaled by 0.1), biases 0.
    Layout: W1[48][64], b1[64], W2[64][64], b2[64], w3[64], b3 (float32)."""
    import math
    rng = np.random.default_rng(seed)
    n = n_features * hidden + hidden + hidden * hidden + hidden + hidden + 1
    p = np.zeros(n, np.float32)
    o_b1 = n_features * hidden
    o_w2 = o_b1 + hidden
    o_b2 = o_w2 + hidden * hidden
    o_w3 = o_b2 + hidden
    p[:o_b1] = rng.uniform(-1, 1, o_b1) * math.sqrt(6.0 / n_features)
    p[o_w2:o_b2] = rng.uniform(-1, 1, hidden * hidden) * math.sqrt(6.0 / hidden)
    p[o_w3:o_w3 + hidden] = rng.uniform(-1, 1, hidden) * math.sqrt(6.0 / hidden) * 0.1
    return p


def training_particles(edge: int, seed: int):
    """Particles of the 512^3 mix with equivalent radii widened to 3-18
    voxels (so that the smaller particles of the 1024^3 volume are covered)
    at the same packing: (mask, labels, n_labels)."""
    n = particles_per_volume(edge, voxels_per_particle=512**3 / 5000 / 2.0)
    m, l, c = packed((edge, edge, edge), n, 3.0, 18.0, seed)
    return m, l, c + 1



def batch_workload(seed: int = 0, n3d: int = 64, n2d: int = 8, edge_lo: int = 64, edge_hi: int = 384,
                   edge2d: int = 4096):
    """Uneven batch: n3d cubic volumes with edges uniform in [edge_lo, edge_hi]
    (the 512^3 particle mix at the same density) and n2d dense 2D ellipse
    masks of edge2d^2. Returns a list of (mask, labels, n_labels)."""
    rng = np.random.default_rng(seed)
    edges = rng.integers(edge_lo, edge_hi + 1, n3d)
    out = []
    for i, e in enumerate(edges):
        out.append(workload(f"particles_3d_{int(e)}", seed * 1000 + i))
    for j in range(n2d):
        out.append(workload(f"ellipses_2d_{edge2d}", seed * 1000 + 500 + j))
    return out
