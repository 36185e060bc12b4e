"""CPU ORACLE for the learned sphericity correction — test infrastructure only.

The paper models sphericity with a spheroid of mean-local-thickness width
(Sec. 4.1, Eqs. 6-8) and compares it with the "strict" mesh-area
sphericity of Eq. 1 (marching cubes in the paper's baseline, Sec. 5.2).
The learned part maps per-object local-thickness features to a correction
of S_LT toward the strict value; the paper has no learned component, so
everything here is this project's own definition, written plainly in FP64:

  strict_sphericity   pi^(1/3) (6V)^(2/3) / A with A and V the area and the
                      enclosed volume of the marching-tetrahedra surface of
                      the object's indicator smoothed by a Gaussian of one
                      voxel (lt_oracle.c). The binary indicator's mesh
                      follows the voxel staircase and overstates a sphere's
                      area by about 27%; volume from the same mesh keeps
                      S <= 1 (isoperimetric inequality).
  strict_sphericity_binary
                      the same with the binary indicator's mesh (no
                      smoothing) and V the voxel count.
  object_features     48 features per object (layout below).
  bf16                round-to-nearest-even to bfloat16.
  mlp_forward /       the 48-64-64-1 ReLU network with BF16 weights and
  mlp_loss_grad       activations, evaluated in FP64 on the BF16-rounded
                      values at the same points as the CUDA kernels.
  adam_step           the Adam update in FP64.

Feature layout (index: value), for an object with V voxels, n_s shell
voxels, largest local thickness M = sqrt(max LT2), mean LT m:
  0: log(V) / 10        1: log(n_s) / 10      2: log(M) / 4
  3: m / M              4: R_LT               5: S_LT
  6-21: interior voxels (not shell) with LT / M in bin b, as a fraction of
        the interior count (bin b = largest b in 0..15 with b / 16 <= LT / M,
        decided in integers: b^2 * maxLT2 <= 256 * LT2)
  22-37: the same over the shell voxels      38-47: 0
Parameter vector (7361 floats): W1[48][64], b1[64], W2[64][64], b2[64],
w3[64], b3.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import _load, object_stats, shell_mask

N_FEATURES = 48
HIDDEN = 64
N_PARAMS = N_FEATURES * HIDDEN + HIDDEN + HIDDEN * HIDDEN + HIDDEN + HIDDEN + 1
OFF_W1, OFF_B1 = 0, N_FEATURES * HIDDEN
OFF_W2 = OFF_B1 + HIDDEN
OFF_B2 = OFF_W2 + HIDDEN * HIDDEN
OFF_W3 = OFF_B2 + HIDDEN
OFF_B3 = OFF_W3 + HIDDEN


# ---------------------------------------------------------------- targets
STRICT_SIGMA = 1.0  # Gaussian smoothing (voxels) of the indicator before meshing


def mesh_area(labels: np.ndarray, which, sigma: float = STRICT_SIGMA):
    """Marching-tetrahedra surface (area, enclosed volume), FP64, of the
    objects `which`, on the indicator smoothed by a Gaussian of `sigma`
    voxels (0: binary)."""
    lab = np.asarray(labels)
    if lab.ndim != 3:
        raise ValueError("3D volumes only")
    nz, ny, nx = lab.shape
    flat = lab.reshape(-1)
    which = np.asarray(list(which), dtype=flat.dtype)
    order = np.argsort(flat, kind="stable")
    srt = flat[order]
    b = np.searchsorted(srt, which, side="left")
    e = np.searchsorted(srt, which, side="right")
    idx = np.ascontiguousarray(np.concatenate([order[i:j] for i, j in zip(b, e)]) if len(which)
                               else np.zeros(0, np.int64), dtype=np.int64)
    off = np.zeros(len(which) + 1, np.int64)
    off[1:] = np.cumsum(e - b)
    out = np.zeros(len(which), np.float64)
    vol = np.zeros(len(which), np.float64)
    lib = _load()
    fn = lib.oracle_mesh_area
    fn.argtypes = ([ctypes.c_int64] * 3 + [ctypes.c_void_p] * 2 +
                   [ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p])
    fn.restype = None
    fn(nx, ny, nz, idx.ctypes.data, off.ctypes.data, len(which), float(sigma), out.ctypes.data,
       vol.ctypes.data)
    return out, vol


def strict_sphericity(labels: np.ndarray, n_labels: int) -> np.ndarray:
    """Eq. 1 on the object's mesh: area and enclosed volume both from the
    marching-tetrahedra surface (so S <= 1 for every object by the
    isoperimetric inequality); NaN for absent labels."""
    V = np.bincount(np.asarray(labels).reshape(-1), minlength=n_labels)
    which = [l for l in range(1, n_labels) if V[l] > 0]
    out = np.full(n_labels, np.nan)
    if which:
        A, Vm = mesh_area(labels, which)
        w = np.asarray(which)
        ok = A > 0  # objects too thin to cross the level after smoothing have no surface
        out[w[ok]] = math.pi ** (1.0 / 3.0) * (6.0 * Vm[ok]) ** (2.0 / 3.0) / A[ok]
    return out


def strict_sphericity_binary(labels: np.ndarray, n_labels: int) -> np.ndarray:
    """Eq. 1 with the area of the marching-tetrahedra surface of the
    object's binary indicator (level 0.5, no smoothing) and V its voxel
    count (the volume the paper's Sec. 4.1 uses). The surface follows the
    voxel staircase, so a sphere scores about 0.8, not 1; NaN for absent
    labels."""
    V = np.bincount(np.asarray(labels).reshape(-1), minlength=n_labels)
    which = [l for l in range(1, n_labels) if V[l] > 0]
    out = np.full(n_labels, np.nan)
    if which:
        A, _ = mesh_area(labels, which, 0.0)
        w = np.asarray(which)
        ok = A > 0
        out[w[ok]] = math.pi ** (1.0 / 3.0) * (6.0 * V[w[ok]]) ** (2.0 / 3.0) / A[ok]
    return out


# --------------------------------------------------------------- features
def lt_bins(lt2: np.ndarray, max_lt2: np.ndarray) -> np.ndarray:
    """Largest b in 0..15 with b^2 * max_lt2 <= 256 * lt2 (integers)."""
    lt2 = np.asarray(lt2, np.int64)
    mx = np.asarray(max_lt2, np.int64)
    b = np.zeros(lt2.shape, np.int64)
    for k in range(1, 16):
        b = np.where(k * k * mx <= 256 * lt2, k, b)
    return b


def object_features(labels: np.ndarray, lt2: np.ndarray, n_labels: int, S: np.ndarray,
                    R: np.ndarray) -> np.ndarray:
    """Feature matrix [n_labels, 48] in FP64 (zeros for empty labels)."""
    st = object_stats(labels, lt2, n_labels)
    lab = np.asarray(labels).reshape(-1).astype(np.int64)
    l2 = np.asarray(lt2).reshape(-1).astype(np.int64)
    sh = shell_mask(labels).reshape(-1)
    obj = lab != 0
    F = np.zeros((n_labels, N_FEATURES))
    mx = st["max_lt2"]
    bins = lt_bins(l2[obj], mx[lab[obj]])
    shell = sh[obj]
    hist_in = np.zeros((n_labels, 16))
    hist_sh = np.zeros((n_labels, 16))
    np.add.at(hist_in, (lab[obj][~shell], bins[~shell]), 1.0)
    np.add.at(hist_sh, (lab[obj][shell], bins[shell]), 1.0)
    for l in range(1, n_labels):
        V = int(st["volume"][l])
        if V == 0:
            continue
        ns = int(st["n_shell"][l])
        M = math.sqrt(int(mx[l]))
        F[l, 0] = math.log(V) / 10.0
        F[l, 1] = math.log(ns) / 10.0
        F[l, 2] = math.log(M) / 4.0
        F[l, 3] = (st["sum_lt"][l] / V) / M
        F[l, 4] = R[l]
        F[l, 5] = S[l]
        F[l, 6:22] = hist_in[l] / max(1, V - ns)
        F[l, 22:38] = hist_sh[l] / max(1, ns)
    return F


# -------------------------------------------------------------------- MLP
def bf16(x) -> np.ndarray:
    """Round FP32 values to bfloat16 (nearest, ties to even), as float64."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params: np.ndarray):
    p = np.asarray(params, np.float64)
    W1 = p[OFF_W1:OFF_B1].reshape(N_FEATURES, HIDDEN)
    b1 = p[OFF_B1:OFF_W2]
    W2 = p[OFF_W2:OFF_B2].reshape(HIDDEN, HIDDEN)
    b2 = p[OFF_B2:OFF_W3]
    w3 = p[OFF_W3:OFF_B3]
    b3 = p[OFF_B3]
    return W1, b1, W2, b2, w3, b3


def mlp_forward(params: np.ndarray, X: np.ndarray, quantize: bool = True):
    """Correction `out` for feature rows X; returns (out, cache). With
    quantize=False the BF16 roundings are skipped (plain FP64 network)."""
    q = bf16 if quantize else (lambda a: np.asarray(a, np.float64))
    W1, b1, W2, b2, w3, b3 = unpack(params)
    W1q, W2q, w3q = q(W1), q(W2), q(w3)
    x = q(X)
    pre1 = x @ W1q + b1
    h1 = q(np.maximum(pre1, 0.0))
    pre2 = h1 @ W2q + b2
    h2 = q(np.maximum(pre2, 0.0))
    out = h2 @ w3q + b3
    return out, (x, pre1, h1, pre2, h2, W2q, w3q)


def mlp_loss_grad(params: np.ndarray, X: np.ndarray, s_lt: np.ndarray, target: np.ndarray,
                  quantize: bool = True):
    """Mean squared error of S_LT + out against the target, and its
    gradient with respect to the FP32 parameters (straight through the BF16
    rounding)."""
    out, (x, pre1, h1, pre2, h2, W2q, w3q) = mlp_forward(params, X, quantize)
    B = X.shape[0]
    r = s_lt + out - target
    loss = float(np.mean(r * r))
    g_out = 2.0 * r / B
    g = np.zeros(N_PARAMS)
    g[OFF_W3:OFF_B3] = h2.T @ g_out
    g[OFF_B3] = g_out.sum()
    g_pre2 = np.outer(g_out, w3q) * (pre2 > 0)
    g[OFF_W2:OFF_B2] = (h1.T @ g_pre2).reshape(-1)
    g[OFF_B2:OFF_W3] = g_pre2.sum(0)
    g_pre1 = (g_pre2 @ W2q.T) * (pre1 > 0)
    g[OFF_W1:OFF_B1] = (x.T @ g_pre1).reshape(-1)
    g[OFF_B1:OFF_W2] = g_pre1.sum(0)
    return loss, g


def adam_step(params, m, v, grad, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected, step counted from 1); returns new
    (params, m, v) in FP64."""
    m = beta1 * np.asarray(m, np.float64) + (1 - beta1) * grad
    v = beta2 * np.asarray(v, np.float64) + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return np.asarray(params, np.float64) - lr * mh / (np.sqrt(vh) + eps), m, v


# ------------------------------------------------- bound of an FP32 forward
_U32 = 2.0 ** -24  # unit roundoff of binary32
_U64 = 2.0 ** -53  # unit roundoff of binary64


def _gamma(k: int, u: float) -> float:
    """Higham's gamma_k = k u / (1 - k u): a sum of k + 1 terms evaluated
    with k roundings of relative size <= u differs from the exact sum by at
    most gamma_k times the sum of the terms' magnitudes (any order)."""
    return k * u / (1.0 - k * u)


def _interval_dot(lo: np.ndarray, hi: np.ndarray, W: np.ndarray):
    """Range of sum_j a_j W[j, k] over a_j in [lo_j, hi_j] (rows of samples),
    and the largest sum of magnitudes sum_j |a_j W[j, k]|."""
    Wp, Wn = np.maximum(W, 0.0), np.minimum(W, 0.0)
    low = lo @ Wp + hi @ Wn
    high = hi @ Wp + lo @ Wn
    mag = np.maximum(np.abs(lo), np.abs(hi)) @ np.abs(W)
    return low, high, mag


def mlp_infer_bounds(params: np.ndarray, X: np.ndarray, s_lt: np.ndarray):
    """Interval [lo, hi] that holds clamp(S_LT + net(x), 0, 1) for any
    evaluation with this network's rounding points: inputs, weights and both
    hidden layers rounded to BF16 (nearest even), every dot product plus its
    bias summed in FP32 in any order (each addition, or fused multiply-add
    of exact BF16 products, rounded once), S_LT + net rounded to FP32, then
    clamped. Derived by interval arithmetic: each layer's FP64 sum of the
    interval ends, widened by gamma_k (FP32) plus gamma_k (FP64) times the
    sum of magnitudes; bf16(max(t, 0)) is monotone in t, so a layer's
    activation lies between the roundings of its interval's ends. A sample
    whose sums all stay clear of a BF16 rounding boundary gets an interval
    of width ~1e-7; one whose FP32 sum may round either way gets both
    outcomes. NaN S_LT gives NaN bounds."""
    W1, b1, W2, b2, w3, b3 = unpack(params)
    W1q, W2q, w3q = bf16(W1), bf16(W2), bf16(w3)
    x = bf16(X)
    # layer 1: exact products of BF16 values, 48 additions onto the bias
    pre1 = x @ W1q + b1
    mag1 = np.abs(x) @ np.abs(W1q) + np.abs(b1)
    e1 = (_gamma(N_FEATURES, _U32) + _gamma(N_FEATURES + 1, _U64)) * mag1
    h1lo, h1hi = bf16(np.maximum(pre1 - e1, 0.0)), bf16(np.maximum(pre1 + e1, 0.0))
    # layer 2
    lo2, hi2, mag2 = _interval_dot(h1lo, h1hi, W2q)
    e2 = (_gamma(HIDDEN, _U32) + _gamma(HIDDEN + 1, _U64)) * (mag2 + np.abs(b2))
    h2lo, h2hi = bf16(np.maximum(lo2 + b2 - e2, 0.0)), bf16(np.maximum(hi2 + b2 + e2, 0.0))
    # output unit
    lo3, hi3, mag3 = _interval_dot(h2lo, h2hi, w3q.reshape(-1, 1))
    lo3, hi3, mag3 = lo3[:, 0] + b3, hi3[:, 0] + b3, mag3[:, 0] + abs(b3)
    e3 = (_gamma(HIDDEN, _U32) + _gamma(HIDDEN + 1, _U64)) * mag3
    s = np.asarray(s_lt, np.float64)
    ylo, yhi = s + lo3 - e3, s + hi3 + e3
    ylo = ylo - (_U32 + _U64) * np.abs(ylo)  # the FP32 rounding of S_LT + net
    yhi = yhi + (_U32 + _U64) * np.abs(yhi)
    lo, hi = np.clip(ylo, 0.0, 1.0), np.clip(yhi, 0.0, 1.0)
    bad = np.isnan(s)
    lo[bad] = np.nan
    hi[bad] = np.nan
    return lo, hi
