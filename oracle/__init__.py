"""CPU ORACLE — test infrastructure only.

A plain, slow, obviously correct CPU implementation of what the method
computes, in FP64 where floating point is involved. Only tests/, the smoke
check in __graft_entry__ and bench.py's CPU-baseline leg may import it; the
library (paper_2504_05808_gb300) never does, and the two share no code.

What it computes (paper: "Fast Sphericity and Roundness approximation in 2D
and 3D using Local Thickness"):

  dt2(mask)            squared Euclidean distance from each foreground voxel to
                       the nearest background voxel; outside the array counts
                       as background. Plain definition (C loops, lt_oracle.c).
  lt2(dt2, labels)     local thickness, squared: the largest DT2(c) over all
                       same-label centres c whose inclusive ball
                       |x - c|^2 <= DT2(c) holds x (Sec. 1; Sec. 4, first
                       paragraph). Painting from every centre, no pruning.
  object_stats(...)    per label: V (voxel count, Sec. 4.1 after Eq. 7),
                       shell voxels (a 4-/6-neighbour outside the object,
                       Sec. 4.2), sum of LT, sum of LT on the shell, max LT2.
  sphericity_3d        Eqs. 1, 6-8: spheroid with a = mean LT, c = 3V/(4 pi a^2).
  sphericity_2d        Eqs. 2, 9-11: ellipse with a = mean LT, b = A/(pi a);
                       Ramanujan's perimeter P_o and P_c = 2 sqrt(pi A).
  roundness            Sec. 4.2: mean LT on the shell / max LT.
  lt2_scaled           LT2 at 1/s resolution, upsampled (fast-LT scale option).
  measures_filtered    roughness filtering (Sec. 7: filter left open; read
                       as keeping each object's voxels with LT >= rho).
  roundness_rescaled   R mapped to 0-1 with the reported minimum (Sec. 6.1).

Readings where the paper is garbled or silent:
  * Eqs. 6-7 print e = 1 - c^2/a^2 without a square root; the spheroid's
    eccentricity is e = sqrt(1 - c^2/a^2) (oblate) and sqrt(1 - a^2/c^2)
    (prolate). At c = a both give the sphere, 4 pi a^2.
  * Eq. 8 writes a where a_s is meant. The text after Eq. 9 names P_o where
    Eq. 11 defines P_c.
  * LT is a radius (Sec. 1), so a_s, a_e are the mean LT radius.
  * Mean LT is over all voxels of the object; the shell uses face neighbours
    (4 in 2D, 6 in 3D); a neighbour outside the array or with another label
    counts as outside the object.
  * Objects are the voxels of one nonzero label; labels must be zero outside
    the mask.

Parity pins (tests/test_oracle_*.py): brute force on tiny inputs, scipy's
exact EDT, digital balls and discs (known lattice counts), numeric
quadrature of the spheroid surface, the complete elliptic integral for the
ellipse perimeter, and the sphere/circle limits S = 1, R = 1.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lt_oracle.c")
_SO = os.path.join(_HERE, "_lt_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C loops into oracle/_lt_oracle.so."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.oracle_dt2.argtypes = [vp, i64, i64, i64, i32, vp]
        lib.oracle_dt2.restype = None
        lib.oracle_dt2_at.argtypes = [vp, i64, i64, i64, i32, vp, i64, vp]
        lib.oracle_dt2_at.restype = None
        lib.oracle_lt2.argtypes = [vp, vp, i64, i64, i64, i32, vp]
        lib.oracle_lt2.restype = None
        lib.oracle_objects.argtypes = [vp, i64, i64, i64, i32, vp, vp, i64, vp, vp]
        lib.oracle_objects.restype = None
        _lib = lib
    return _lib


def _dims(a: np.ndarray):
    if a.ndim == 2:
        return 2, a.shape[1], a.shape[0], 1
    if a.ndim == 3:
        return 3, a.shape[2], a.shape[1], a.shape[0]
    raise ValueError("2D or 3D arrays only")


# ----------------------------------------------------------------- DT and LT
def dt2(mask: np.ndarray) -> np.ndarray:
    """Squared EDT by the definition (nearest background, padded array)."""
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    ndim, nx, ny, nz = _dims(mask)
    out = np.empty(mask.shape, np.uint32)
    _load().oracle_dt2(mask.ctypes.data, nx, ny, nz, ndim, out.ctypes.data)
    return out


def dt2_at(mask: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """DT2 at the given linear voxel indices."""
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    ndim, nx, ny, nz = _dims(mask)
    out = np.empty(idx.shape, np.uint32)
    _load().oracle_dt2_at(mask.ctypes.data, nx, ny, nz, ndim, idx.ctypes.data, idx.size,
                          out.ctypes.data)
    return out


def lt2(dt2_arr: np.ndarray, labels: np.ndarray) -> np.ndarray:
    """Squared local thickness by painting from every labelled centre."""
    d = np.ascontiguousarray(dt2_arr, dtype=np.uint32)
    lab = np.ascontiguousarray(labels, dtype=np.uint32)
    ndim, nx, ny, nz = _dims(d)
    out = np.empty(d.shape, np.uint32)
    _load().oracle_lt2(d.ctypes.data, lab.ctypes.data, nx, ny, nz, ndim, out.ctypes.data)
    return out


def objects_dt2_lt2(mask: np.ndarray, labels: np.ndarray, which):
    """DT2 and LT2 of the voxels of selected labels, one object at a time.

    Returns {label: (linear_indices, dt2, lt2)}.
    """
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    ndim, nx, ny, nz = _dims(mask)
    flat = labels.reshape(-1)
    which = [int(w) for w in which]
    sel = np.isin(flat, np.asarray(which, dtype=flat.dtype))
    idx_all = np.flatnonzero(sel)
    lab_all = flat[idx_all]
    order = np.argsort(lab_all, kind="stable")
    idx_all, lab_all = idx_all[order], lab_all[order]
    bounds = np.searchsorted(lab_all, np.asarray(which, dtype=lab_all.dtype), side="left")
    ends = np.searchsorted(lab_all, np.asarray(which, dtype=lab_all.dtype), side="right")
    idx_list = [idx_all[b:e] for b, e in zip(bounds, ends)]
    off = np.zeros(len(which) + 1, np.int64)
    off[1:] = np.cumsum([len(x) for x in idx_list])
    idx = np.ascontiguousarray(np.concatenate(idx_list) if idx_list else np.zeros(0, np.int64),
                               dtype=np.int64)
    d_out = np.empty(idx.shape, np.uint32)
    l_out = np.empty(idx.shape, np.uint32)
    _load().oracle_objects(mask.ctypes.data, nx, ny, nz, ndim, idx.ctypes.data, off.ctypes.data,
                           len(which), d_out.ctypes.data, l_out.ctypes.data)
    return {w: (idx[off[k]:off[k + 1]], d_out[off[k]:off[k + 1]], l_out[off[k]:off[k + 1]])
            for k, w in enumerate(which)}


def dt2_brute(mask: np.ndarray) -> np.ndarray:
    """All-pairs DT2 for tiny arrays: every voxel against every background
    voxel of the array padded by one background layer."""
    m = np.pad(np.asarray(mask) != 0, 1, constant_values=False)
    bg = np.argwhere(~m).astype(np.int64)
    fg = np.argwhere(m).astype(np.int64)
    out = np.zeros(m.shape, np.int64)
    if len(fg):
        d = ((fg[:, None, :] - bg[None, :, :]) ** 2).sum(-1).min(1)
        out[tuple(fg.T)] = d
    sl = tuple(slice(1, -1) for _ in range(m.ndim))
    return out[sl].astype(np.uint32)


def lt2_brute(dt2_arr: np.ndarray, labels: np.ndarray) -> np.ndarray:
    """All-pairs local thickness for tiny arrays."""
    d = np.asarray(dt2_arr).astype(np.int64)
    lab = np.asarray(labels)
    pts = np.argwhere(lab != 0).astype(np.int64)
    out = np.zeros(d.shape, np.int64)
    if len(pts):
        r2 = d[tuple(pts.T)]
        pl = lab[tuple(pts.T)]
        dist2 = ((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1)  # [target, centre]
        ok = (dist2 <= r2[None, :]) & (pl[:, None] == pl[None, :])
        out[tuple(pts.T)] = np.where(ok, r2[None, :], 0).max(1)
    return out.astype(np.uint32)


# ----------------------------------------------------------- per-object sums
def shell_mask(labels: np.ndarray) -> np.ndarray:
    """Object voxels with a face neighbour (4 in 2D, 6 in 3D) outside the
    object: another label, background, or outside the array (Sec. 4.2)."""
    lab = np.asarray(labels)
    p = np.pad(lab, 1, constant_values=0)
    core = tuple(slice(1, -1) for _ in range(lab.ndim))
    shell = np.zeros(lab.shape, bool)
    for ax in range(lab.ndim):
        for s in (-1, 1):
            sl = list(core)
            sl[ax] = slice(1 + s, p.shape[ax] - 1 + s)
            shell |= p[tuple(sl)] != lab
    return shell & (lab != 0)


def object_stats(labels: np.ndarray, lt2_arr: np.ndarray, n_labels: int) -> dict:
    """FP64 per-label sums (label 0 is background and is reported as empty)."""
    lab = np.asarray(labels).reshape(-1).astype(np.int64)
    if lab.size and lab.max() >= n_labels:
        raise ValueError("label >= n_labels")
    lt = np.sqrt(np.asarray(lt2_arr).reshape(-1).astype(np.float64))
    sh = shell_mask(labels).reshape(-1)
    obj = lab != 0
    V = np.bincount(lab[obj], minlength=n_labels).astype(np.int64)
    ns = np.bincount(lab[sh], minlength=n_labels).astype(np.int64)
    s_lt = np.bincount(lab[obj], weights=lt[obj], minlength=n_labels)
    s_sh = np.bincount(lab[sh], weights=lt[sh], minlength=n_labels)
    mx = np.zeros(n_labels, np.int64)
    np.maximum.at(mx, lab[obj], np.asarray(lt2_arr).reshape(-1)[obj].astype(np.int64))
    V[0] = ns[0] = mx[0] = 0
    s_lt[0] = s_sh[0] = 0.0
    return {"volume": V, "n_shell": ns, "sum_lt": s_lt, "sum_shell_lt": s_sh, "max_lt2": mx}


# --------------------------------------------------------- shape formulas
def spheroid_area(a: float, c: float) -> float:
    """Surface area of a spheroid with equal semi-axes a and third semi-axis c
    (Eqs. 6-7, with e the eccentricity, read with its square root)."""
    if c == a:
        return 4.0 * math.pi * a * a
    if c < a:
        e = math.sqrt(1.0 - (c * c) / (a * a))
        return 2.0 * math.pi * a * a * (1.0 + (1.0 - e * e) / e * math.atanh(e))
    e = math.sqrt(1.0 - (a * a) / (c * c))
    return 2.0 * math.pi * a * a * (1.0 + c / (a * e) * math.asin(e))


def ramanujan_perimeter(a: float, b: float) -> float:
    """Ramanujan's first approximation of an ellipse perimeter (Eq. 9)."""
    return math.pi * (3.0 * (a + b) - math.sqrt((3.0 * a + b) * (a + 3.0 * b)))


def sphericity_3d(V: float, mean_lt: float) -> float:
    """S_LT in 3D: Eq. 1 with the spheroid area of Eqs. 6-8."""
    a = mean_lt
    c = 3.0 * V / (4.0 * math.pi * a * a)
    return math.pi ** (1.0 / 3.0) * (6.0 * V) ** (2.0 / 3.0) / spheroid_area(a, c)


def sphericity_2d(A: float, mean_lt: float) -> float:
    """S_LT in 2D: Eq. 2 with P_o from Eqs. 9-10 and P_c from Eq. 11."""
    a = mean_lt
    b = A / (math.pi * a)
    return 2.0 * math.sqrt(math.pi * A) / ramanujan_perimeter(a, b)


def roundness(sum_shell_lt: float, n_shell: int, max_lt2: int) -> float:
    """R_LT: mean LT over the contour/surface divided by the largest LT (Sec. 4.2)."""
    return (sum_shell_lt / n_shell) / math.sqrt(max_lt2)


def measures(labels: np.ndarray, lt2_arr: np.ndarray, n_labels: int):
    """(sphericity, roundness, stats) in FP64; NaN for labels with no voxel."""
    st = object_stats(labels, lt2_arr, n_labels)
    nd = np.asarray(labels).ndim
    S = np.full(n_labels, np.nan)
    R = np.full(n_labels, np.nan)
    for l in range(1, n_labels):
        V = int(st["volume"][l])
        if V == 0:
            continue
        mean_lt = st["sum_lt"][l] / V
        S[l] = sphericity_3d(V, mean_lt) if nd == 3 else sphericity_2d(V, mean_lt)
        R[l] = roundness(st["sum_shell_lt"][l], int(st["n_shell"][l]), int(st["max_lt2"][l]))
    return S, R, st


def object_measures_from_voxels(labels: np.ndarray, idx: np.ndarray, lt2_vals: np.ndarray):
    """S and R of one object given its voxels (linear indices into labels)
    and their LT2, for objects of arrays too large to process whole. The
    shell test looks at the object's face neighbours in `labels`."""
    lab = np.asarray(labels)
    shape = lab.shape
    flat = lab.reshape(-1)
    l = flat[idx[0]]
    coords = np.unravel_index(idx, shape)
    shell = np.zeros(idx.shape, bool)
    for ax in range(lab.ndim):
        for s in (-1, 1):
            c = list(coords)
            c[ax] = c[ax] + s
            out = (c[ax] < 0) | (c[ax] >= shape[ax])
            c[ax] = np.clip(c[ax], 0, shape[ax] - 1)
            shell |= out | (flat[np.ravel_multi_index(tuple(c), shape)] != l)
    lt = np.sqrt(np.asarray(lt2_vals).astype(np.float64))
    V = idx.size
    mean_lt = lt.sum() / V
    S = sphericity_3d(V, mean_lt) if lab.ndim == 3 else sphericity_2d(V, mean_lt)
    R = roundness(lt[shell].sum(), int(shell.sum()), int(np.max(lt2_vals)))
    return S, R


def lt2_scaled(mask: np.ndarray, labels: np.ndarray, s: int) -> np.ndarray:
    """Local thickness at 1/s resolution brought back to full resolution
    (the reduced-resolution option of the fast local-thickness work the
    paper cites, Sec. 1 and Sec. 4), this library's definition: sample mask
    and labels at the voxels min(s*B + s//2, n-1) per axis; exact LT2 of the
    sampled volume; an object voxel of label l in block x//s gets s^2 times
    the block's LT2 when the block has label l, else the largest s^2*LT2 of
    the neighbouring blocks (|d|_inf <= 1) with label l, else 1; 0 outside
    objects."""
    mask = np.asarray(mask)
    lab = np.asarray(labels).astype(np.uint32)
    idx = [np.minimum(np.arange(-(-n // s)) * s + s // 2, n - 1) for n in lab.shape]
    m_low = mask[np.ix_(*idx)]
    l_low = lab[np.ix_(*idx)]
    t_low = lt2(dt2(m_low), l_low).astype(np.int64)
    blk = [np.arange(n) // s for n in lab.shape]
    own_l = l_low[np.ix_(*blk)]
    own_t = t_low[np.ix_(*blk)]
    best = np.zeros(lab.shape, np.int64)
    nd = lab.ndim
    for d in np.ndindex(*(3,) * nd):
        off = [int(v) - 1 for v in d]
        sel = [np.clip(b + o, 0, n - 1) for b, o, n in zip(blk, off, l_low.shape)]
        valid = np.ones(lab.shape, bool)
        for ax, (b, o, n) in enumerate(zip(blk, off, l_low.shape)):
            ok = (b + o >= 0) & (b + o < n)
            shape = [1] * nd
            shape[ax] = -1
            valid &= ok.reshape(shape)
        nl = l_low[np.ix_(*sel)]
        nt = t_low[np.ix_(*sel)]
        best = np.where(valid & (nl == lab), np.maximum(best, nt), best)
    out = np.where(own_l == lab, s * s * own_t, np.where(best > 0, s * s * best, 1))
    return np.where(lab != 0, out, 0).astype(np.uint32)


def measures_filtered(labels: np.ndarray, lt2_arr: np.ndarray, n_labels: int, min_lt2: int):
    """S and R after roughness filtering (Sec. 7 leaves the filter open; this
    is the reading used): each object is reduced to its voxels whose local
    thickness is at least sqrt(min_lt2), i.e. to the union of its inscribed
    balls of squared radius >= min_lt2, and S, R are measured on what
    remains (shell and sums by the same definitions). Empty objects give NaN."""
    lab = np.asarray(labels)
    kept = np.where(np.asarray(lt2_arr).astype(np.int64) >= int(min_lt2), lab, 0)
    return measures(kept, lt2_arr, n_labels)


def roundness_rescaled(R: np.ndarray, r_min: float | None = None) -> np.ndarray:
    """Roundness mapped to the 0-1 range with the reported minimum (Sec. 6.1
    remarks that R_LT never exceeds 1 and never reaches 0, and that the
    minimum can map it onto 0-1): R' = (R - m) / (1 - m), m = r_min or the
    smallest finite R; clamped below at 0; NaN stays NaN; 1 when m >= 1."""
    R = np.asarray(R, dtype=np.float64)
    fin = np.isfinite(R)
    m = float(np.min(R[fin])) if r_min is None else float(r_min)
    out = np.full(R.shape, np.nan)
    if m >= 1.0:
        out[fin] = 1.0
    else:
        out[fin] = np.maximum((R[fin] - m) / (1.0 - m), 0.0)
    return out


def pipeline(mask: np.ndarray, labels: np.ndarray, n_labels: int):
    """mask, labels -> (dt2, lt2, sphericity, roundness) by the oracle."""
    lab = np.asarray(labels)
    if np.any((lab != 0) & (np.asarray(mask) == 0)):
        raise ValueError("labels must be zero outside the mask")
    d = dt2(mask)
    l2 = lt2(d, lab)
    S, R, _ = measures(lab, l2, n_labels)
    return d, l2, S, R
