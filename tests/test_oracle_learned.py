"""Pins for the oracle of the learned sphericity correction.

Independent references: exact polynomial growth of the mesh of cubes, axis
permutation symmetry of the Kuhn subdivision, the isoperimetric bound,
spheres, torch's bfloat16 conversion and Adam optimiser, and central finite
differences of the loss.
"""
import math

import numpy as np
import pytest

import oracle
import oracle.learned as L
import synth

pytestmark = pytest.mark.usefixtures("built_cpu_parts")


def _cube(n, pad=6):
    lab = np.zeros((n + 2 * pad,) * 3, np.uint32)
    lab[pad:pad + n, pad:pad + n, pad:pad + n] = 1
    return lab


@pytest.mark.parametrize("sigma,sizes", [(0.0, range(1, 9)), (1.0, range(7, 13))])
def test_mesh_of_cubes_is_polynomial(sigma, sizes):
    """Flat faces sit on the level set exactly, so the area of an n-cube is a
    quadratic 6n^2 + an + b (second difference 12) and the enclosed volume a
    cubic with leading coefficient 1 (third difference 6)."""
    A, V = zip(*[tuple(x[0] for x in L.mesh_area(_cube(n), [1], sigma)) for n in sizes])
    assert np.allclose(np.diff(A, 2), 12.0, atol=1e-6)
    assert np.allclose(np.diff(V, 3), 6.0, atol=1e-6)


@pytest.mark.parametrize("sigma", [0.0, 1.0])
def test_mesh_is_symmetric_under_axis_permutations(sigma):
    import scipy.ndimage as ndi
    rng = np.random.default_rng(2)
    f = ndi.gaussian_filter(rng.random((22, 25, 28)), 2.0)
    obj = (f > np.quantile(f, 0.7)).astype(np.uint32)
    lab = ndi.label(obj)[0].astype(np.uint32)
    big = np.argmax(np.bincount(lab.reshape(-1))[1:]) + 1
    lab = (lab == big).astype(np.uint32)
    ref = L.mesh_area(lab, [1], sigma)
    for perm in [(0, 2, 1), (1, 0, 2), (2, 1, 0), (1, 2, 0)]:
        got = L.mesh_area(np.ascontiguousarray(lab.transpose(perm)), [1], sigma)
        assert got[0][0] == pytest.approx(ref[0][0], rel=1e-12)
        assert got[1][0] == pytest.approx(ref[1][0], rel=1e-12)


def test_strict_sphericity_spheres_and_bound():
    for r in (5, 10, 20):
        n = 2 * r + 9
        g = np.indices((n, n, n)) - n // 2
        ball = ((g ** 2).sum(0) <= r * r).astype(np.uint32)
        s = L.strict_sphericity(ball, 2)[1]
        assert 0.98 < s <= 1.0
        A, V = L.mesh_area(ball, [1])
        assert V[0] / (4 / 3 * math.pi * r ** 3) == pytest.approx(1.0, abs=0.16)
    m, lab, n = synth.training_particles(96, 3)
    S = L.strict_sphericity(lab, n)
    f = np.isfinite(S)
    assert f.sum() > 20 and np.all(S[f] <= 1.0 + 1e-12) and np.all(S[f] > 0.2)


def test_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.normal(size=5000).astype(np.float32),
                        np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.5, 0.0, 1e-30], np.float32)])
    # exact ties: mantissa patterns ...x1000...0 in the dropped half
    ties = (np.arange(100, dtype=np.uint32) << 16 | 0x8000).view(np.float32)
    x = np.concatenate([x, ties])
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(L.bf16(x), want)


def test_backward_equals_finite_differences():
    rng = np.random.default_rng(5)
    p = synth.mlp_initial_params(1).astype(np.float64)
    p[L.OFF_B1:L.OFF_W2] = rng.normal(0, 0.1, L.HIDDEN)
    p[L.OFF_B2:L.OFF_W3] = rng.normal(0, 0.1, L.HIDDEN)
    X = rng.random((12, L.N_FEATURES))
    s = rng.random(12)
    t = rng.random(12)
    _, g = L.mlp_loss_grad(p, X, s, t, quantize=False)
    h = 1e-6
    for i in list(range(0, L.N_PARAMS, 37)) + [L.N_PARAMS - 1, L.OFF_B1 + 3, L.OFF_B2 + 5]:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        num = (L.mlp_loss_grad(pp, X, s, t, quantize=False)[0] -
               L.mlp_loss_grad(pm, X, s, t, quantize=False)[0]) / (2 * h)
        assert g[i] == pytest.approx(num, rel=1e-5, abs=1e-9), i


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    p0 = rng.normal(size=50)
    grads = rng.normal(size=(7, 50))
    w = torch.tensor(p0.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([w], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for k, g in enumerate(grads, start=1):
        opt.zero_grad()
        w.grad = torch.tensor(g)
        opt.step()
        p, m, v = L.adam_step(p, m, v, g, k, 1e-2)
    assert np.allclose(p, w.detach().numpy(), rtol=0, atol=1e-12)


def test_features_of_a_ball():
    r = 6
    n = 2 * r + 5
    g = np.indices((n, n, n)) - n // 2
    ball = ((g ** 2).sum(0) <= r * r).astype(np.uint32)
    lt2 = oracle.lt2(oracle.dt2(ball), ball)
    S, R, st = oracle.measures(ball, lt2, 2)
    F = L.object_features(ball, lt2, 2, S, R)
    assert np.all(F[0] == 0)
    assert F[1, 3] == pytest.approx(1.0) and F[1, 4] == pytest.approx(1.0)
    assert F[1, 6 + 15] == pytest.approx(1.0) and F[1, 22 + 15] == pytest.approx(1.0)
    assert F[1, 0] == pytest.approx(math.log(int(st["volume"][1])) / 10)


def test_feature_histograms_are_fractions():
    m, lab, n = synth.workload("ellipsoids_3d_128", 2)
    d, l2, S, R = oracle.pipeline(m, lab, n)
    F = L.object_features(lab, l2, n, S, R)
    V = np.bincount(lab.reshape(-1), minlength=n)
    for l in range(1, n):
        if V[l] == 0:
            continue
        assert F[l, 6:22].sum() == pytest.approx(1.0) and F[l, 22:38].sum() == pytest.approx(1.0)
        assert 0 < F[l, 3] <= 1 and np.all(F[l, 38:] == 0)


def test_bins_agree_with_real_ratio():
    rng = np.random.default_rng(7)
    mx = rng.integers(1, 5000, 20000)
    lt = (rng.random(20000) * mx).astype(np.int64) + 1
    lt = np.minimum(lt, mx)
    b = L.lt_bins(lt, mx)
    ratio = np.sqrt(lt / mx)
    want = np.minimum(15, np.floor(16 * ratio)).astype(np.int64)
    exact_edge = np.isclose(16 * ratio, np.round(16 * ratio), rtol=0, atol=1e-9)
    assert np.array_equal(b[~exact_edge], want[~exact_edge])


def _random_net(seed, n):
    rng = np.random.default_rng(seed)
    p = synth.mlp_initial_params(seed).astype(np.float32)
    p[L.OFF_B1:L.OFF_W2] = rng.normal(size=L.HIDDEN).astype(np.float32) * 0.1
    p[L.OFF_B2:L.OFF_W3] = rng.normal(size=L.HIDDEN).astype(np.float32) * 0.1
    p[L.OFF_B3] = np.float32(0.05)
    X = rng.normal(size=(n, L.N_FEATURES)).astype(np.float32)
    S = rng.random(n).astype(np.float32)
    return p, X, S


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bf16_forward_matches_torch_reference(seed):
    """The oracle's BF16 forward against one written with torch's own
    bfloat16 conversion and torch.nn.functional.linear in FP64: inputs and
    weights rounded to BF16, each hidden layer's FP64 pre-activation rounded
    to FP32 (the precision the sums are taken in) and then to BF16 after the
    ReLU. The rounded activations agree exactly, the output to FP64 order."""
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    p, X, _ = _random_net(seed, 3000)
    t = torch.from_numpy(p).double()
    W1 = t[L.OFF_W1:L.OFF_B1].reshape(L.N_FEATURES, L.HIDDEN)
    b1, b2, b3 = t[L.OFF_B1:L.OFF_W2], t[L.OFF_B2:L.OFF_W3], t[L.OFF_B3]
    W2 = t[L.OFF_W2:L.OFF_B2].reshape(L.HIDDEN, L.HIDDEN)
    w3 = t[L.OFF_W3:L.OFF_B3]
    q = lambda a: a.float().to(torch.bfloat16).double()
    x = q(torch.from_numpy(X).double())
    h1 = q(torch.relu(F.linear(x, q(W1).T, b1)))
    h2 = q(torch.relu(F.linear(h1, q(W2).T, b2)))
    out = F.linear(h2, q(w3).reshape(1, -1), b3.reshape(1)).reshape(-1)
    got, cache = L.mlp_forward(p, X.astype(np.float64))
    assert np.array_equal(cache[2], h1.numpy())
    assert np.array_equal(cache[4], h2.numpy())
    assert np.allclose(got, out.numpy(), rtol=0, atol=1e-12)
    assert np.count_nonzero(h1.numpy()) > 0.2 * h1.numel()  # the ReLUs are not all off


def _fp32_forward(p, X, S, reverse):
    """The network in plain float32 numpy, one multiply-add at a time in the
    given order (forward or reversed), rounding as the network specifies."""
    b = lambda a: L.bf16(a).astype(np.float32)
    W1, b1, W2, b2, w3, b3 = [np.asarray(a, np.float32) for a in L.unpack(p)]
    W1q, W2q, w3q = b(W1), b(W2), b(w3)
    x = b(X)

    def layer(a, W, bias):
        acc = np.broadcast_to(np.asarray(bias, np.float32), (a.shape[0], W.shape[1])).copy()
        rng = range(W.shape[0] - 1, -1, -1) if reverse else range(W.shape[0])
        for i in rng:
            acc = (acc + a[:, i:i + 1] * W[i]).astype(np.float32)  # exact product, one rounding
        return acc

    h1 = b(np.maximum(layer(x, W1q, b1), 0))
    h2 = b(np.maximum(layer(h1, W2q, b2), 0))
    out = layer(h2, w3q.reshape(-1, 1), np.float32(b3))[:, 0]
    return np.clip((S.astype(np.float32) + out).astype(np.float32), 0, 1)


@pytest.mark.parametrize("seed", [0, 3])
def test_inference_bounds_hold_float32_evaluations(seed):
    """mlp_infer_bounds against independent FP32 evaluations in two
    summation orders: both lie inside; so does the FP64 evaluation. The
    interval's width is the worst-case FP32 summation error (~1e-5 here),
    plus a BF16 step wherever a hidden unit's sum may round either way."""
    p, X, S = _random_net(seed, 4000)
    S[11] = np.nan
    lo, hi = L.mlp_infer_bounds(p, X.astype(np.float64), S)
    assert np.isnan(lo[11]) and np.isnan(hi[11])
    ok = ~np.isnan(S)
    for rev in (False, True):
        y = _fp32_forward(p, X, S, rev)
        assert np.all((y[ok] >= lo[ok]) & (y[ok] <= hi[ok]))
    out, _ = L.mlp_forward(p, X.astype(np.float64))
    y64 = np.clip(S.astype(np.float64) + out, 0, 1)
    assert np.all((y64[ok] >= lo[ok]) & (y64[ok] <= hi[ok]))
    width = (hi - lo)[ok]
    assert np.median(width) <= 5e-5 and width.max() <= 0.05
    # a mistake in the network (an output bias off by 1e-3) leaves the
    # interval for most samples
    bad = p.copy()
    bad[L.OFF_B3] += np.float32(1e-3)
    yb = _fp32_forward(bad, X, S, False)
    inside = (yb[ok] >= lo[ok]) & (yb[ok] <= hi[ok])
    clamped = (yb[ok] == 0) | (yb[ok] == 1)
    assert np.count_nonzero(~inside & ~clamped) > 0.8 * np.count_nonzero(~clamped)


def test_binary_strict_sphericity_of_cubes_and_balls():
    """Binary-indicator target: the mesh of an n-cube is a quadratic in n with
    leading term 6 n^2 (pinned above), so with V = n^3 voxels the value tends
    to the cube's sphericity (pi/6)^(1/3) = 0.806 with an O(1/n) error. For
    digital balls the staircase surface is a fixed fraction larger than the
    sphere's whatever the radius, so the value settles near 0.79 instead of
    approaching 1."""
    lim = (math.pi / 6.0) ** (1.0 / 3.0)
    errs = []
    for n in (8, 16, 32):
        s = L.strict_sphericity_binary(_cube(n), 2)[1]
        errs.append(abs(s - lim))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.01
    assert errs[1] / errs[2] == pytest.approx(2.0, rel=0.2)  # first order in 1/n
    vals = []
    for r in (8, 16):
        n = 2 * r + 9
        g = np.indices((n, n, n)) - n // 2
        ball = ((g ** 2).sum(0) <= r * r).astype(np.uint32)
        vals.append(L.strict_sphericity_binary(ball, 2)[1])
    assert all(0.75 < v < 0.85 for v in vals) and abs(vals[0] - vals[1]) < 0.01
