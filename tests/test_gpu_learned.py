"""GPU tests of the learned sphericity correction against the CPU oracle.

Features: within 1e-5 (histograms exact; logs and ratios from the
fixed-point sums). Gradients: the kernels sum in FP32, the oracle in FP64 on
the same BF16-rounded forward values; a hidden activation whose FP32 and FP64
pre-activations straddle a BF16 rounding boundary may differ by one BF16 step,
so the gradient is compared by its largest error relative to its largest
component (<= 2e-3). Ablation: trained on the GPU, the network beats the
plain spheroid formula's MAE against strict sphericity on held-out particles.
"""
import numpy as np
import pytest

import oracle
import oracle.learned as L
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("built_cpu_parts")]


@pytest.fixture(scope="module")
def lt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_05808_gb300 as mod
    return mod


def gpu_objects(lt, mask, labels, n):
    """GPU pipeline + features: (S, R, features) as numpy."""
    import torch
    m = torch.from_numpy(mask).cuda()
    lab = torch.from_numpy(labels.view(np.int32)).cuda()
    dt2 = torch.empty(mask.shape, dtype=torch.int32, device="cuda")
    lt2 = torch.empty_like(dt2)
    S = torch.empty(n, dtype=torch.float32, device="cuda")
    R = torch.empty_like(S)
    stats = {k: torch.empty(n, dtype=torch.int32, device="cuda") for k in ("volume", "n_shell", "max_lt2")}
    stats.update({k: torch.empty(n, dtype=torch.int64, device="cuda") for k in ("sum_lt", "sum_shell_lt")})
    lt.lt_edt(m, dt2)
    ws = lt.lt_local_thickness(dt2, lab, lt2)
    lt.lt_workspace_status(ws)
    ws = lt.lt_shape_measures(lab, lt2, n, S, R, stats)
    lt.lt_workspace_status(ws)
    F = torch.empty((n, lt.MLP_FEATURES), dtype=torch.float32, device="cuda")
    lt.lt_object_features(lab, lt2, n, stats, S, R, F)
    torch.cuda.synchronize()
    return S, R, F


@pytest.mark.parametrize("name", ["ellipsoids_3d_128", "ellipses_2d_256"])
def test_features_match_oracle(lt, name):
    m, lab, n = synth.workload(name, 4)
    S, R, F = gpu_objects(lt, m, lab, n)
    d_ref, l_ref, S_ref, R_ref = oracle.pipeline(m, lab, n)
    F_ref = L.object_features(lab, l_ref, n, S_ref, R_ref)
    assert np.abs(F.cpu().numpy() - F_ref).max() <= 1e-5


def _fused(lt, mask, labels, n):
    """lt_measure_features: (S, R, features, stats) as numpy."""
    import torch
    m = torch.from_numpy(mask).cuda()
    lab = torch.from_numpy(labels.view(np.int32)).cuda()
    dt2 = torch.empty(mask.shape, dtype=torch.int32, device="cuda")
    lt2 = torch.empty_like(dt2)
    S = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
    R = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
    F = torch.full((n, lt.MLP_FEATURES), -1.0, dtype=torch.float32, device="cuda")
    stats = {k: torch.empty(n, dtype=torch.int32, device="cuda") for k in ("volume", "n_shell", "max_lt2")}
    stats.update({k: torch.empty(n, dtype=torch.int64, device="cuda") for k in ("sum_lt", "sum_shell_lt")})
    ws = lt.lt_measure_features(m, lab, n, dt2, lt2, S, R, F, stats)
    lt.lt_workspace_status(ws)
    torch.cuda.synchronize()
    return S.cpu().numpy(), R.cpu().numpy(), F.cpu().numpy(), {k: v.cpu().numpy() for k, v in stats.items()}


@pytest.mark.parametrize("case", ["ellipsoids_3d_128", "ellipses_2d_256", "particles_3d_160", "ragged_3d"])
def test_fused_features_equal_two_pass_features(lt, case):
    """lt_measure_features bins the histograms inside the shape pass, with
    the per-object maximum taken by the ridge pass: the same bits as
    lt_measure (S, R) and as the separate features pass (features, sums),
    and the oracle's features within 1e-5. ragged_3d has rows of 75 voxels
    (the pass without 4-voxel vectors)."""
    import scipy.ndimage as ndi
    if case == "ragged_3d":
        rng = np.random.default_rng(5)
        f = ndi.gaussian_filter(rng.random((40, 37, 75)), 2.0)
        m = (f > np.quantile(f, 0.55)).astype(np.uint8)
        lab = ndi.label(m)[0].astype(np.uint32)
        n = int(lab.max()) + 1
    elif case == "particles_3d_160":
        m, lab, n = synth.training_particles(160, 7)
    else:
        m, lab, n = synth.workload(case, 4)
    S, R, F, st = _fused(lt, m, lab, n)
    S2, R2, F2 = gpu_objects(lt, m, lab, n)
    assert np.array_equal(S.view(np.uint32), S2.cpu().numpy().view(np.uint32))
    assert np.array_equal(R.view(np.uint32), R2.cpu().numpy().view(np.uint32))
    assert np.array_equal(F.view(np.uint32), F2.cpu().numpy().view(np.uint32))
    _, l_ref, S_ref, R_ref = oracle.pipeline(m, lab, n)
    F_ref = L.object_features(lab, l_ref, n, S_ref, R_ref)
    assert np.abs(F - F_ref).max() <= 1e-5
    ost = oracle.object_stats(lab, l_ref, n)
    for k in ("volume", "n_shell", "max_lt2"):
        assert np.array_equal(st[k].astype(np.int64) & 0xFFFFFFFF, ost[k]), k


def _random_problem(seed, n=3000):
    rng = np.random.default_rng(seed)
    F = rng.random((n, L.N_FEATURES)).astype(np.float32)
    F[:, 38:] = 0
    S = rng.uniform(0.5, 1.0, n).astype(np.float32)
    T = np.clip(S + rng.normal(0, 0.05, n), 0, 1).astype(np.float32)
    p = synth.mlp_initial_params(seed)
    p[L.OFF_B1:L.OFF_W2] = rng.normal(0, 0.1, L.HIDDEN)
    p[L.OFF_B2:L.OFF_W3] = rng.normal(0, 0.1, L.HIDDEN)
    return F, S, T, p


def test_gradients_match_oracle(lt):
    import torch
    F, S, T, p = _random_problem(11)
    idx = np.random.default_rng(1).choice(len(S), 512, replace=False).astype(np.int32)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    grad = torch.empty(lt.MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    lt.lt_mlp_gradients(d(p), d(F), d(S), d(T), d(idx), grad, loss)
    torch.cuda.synchronize()
    ref_loss, ref = L.mlp_loss_grad(p, F[idx].astype(np.float64), S[idx].astype(np.float64),
                                    T[idx].astype(np.float64))
    g = grad.cpu().numpy().astype(np.float64)
    assert np.abs(g - ref).max() <= 2e-3 * np.abs(ref).max()
    assert float(loss.item()) == pytest.approx(ref_loss, rel=2e-3)
    # deterministic: the same call gives the same bits
    grad2 = torch.empty_like(grad)
    lt.lt_mlp_gradients(d(p), d(F), d(S), d(T), d(idx), grad2)
    assert torch.equal(grad, grad2)


def test_inference_and_adam_match_oracle(lt):
    import torch
    F, S, T, p = _random_problem(12, 4000)
    S[7] = np.nan
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = torch.empty(len(S), dtype=torch.float32, device="cuda")
    lt.lt_mlp_infer(d(p), d(F), d(S), out)
    corr, _ = L.mlp_forward(p, F.astype(np.float64))
    want = np.clip(S.astype(np.float64) + corr, 0, 1)
    got = out.cpu().numpy()
    assert np.isnan(got[7])
    ok = ~np.isnan(want)
    # every output inside the interval that BF16 roundings at the network's
    # rounding points and FP32 sums in any order allow (oracle-derived)
    lo, hi = L.mlp_infer_bounds(p, F.astype(np.float64), S)
    assert np.all((got[ok] >= lo[ok]) & (got[ok] <= hi[ok]))
    err = np.abs(got[ok] - want[ok])
    assert np.quantile(err, 0.99) <= 1e-5
    # one Adam step
    rng = np.random.default_rng(3)
    g = rng.normal(size=lt.MLP_PARAMS).astype(np.float32)
    m0 = rng.normal(size=lt.MLP_PARAMS).astype(np.float32) * 0.1
    v0 = rng.random(lt.MLP_PARAMS).astype(np.float32) * 0.1
    pt, mt, vt = d(p.copy()), d(m0.copy()), d(v0.copy())
    lt.lt_mlp_adam(pt, mt, vt, d(g), 5, 1e-3)
    pr, mr, vr = L.adam_step(p, m0, v0, g.astype(np.float64), 5, 1e-3)
    assert np.allclose(pt.cpu().numpy(), pr, rtol=0, atol=1e-6)
    assert np.allclose(mt.cpu().numpy(), mr, rtol=1e-5, atol=1e-7)
    assert np.allclose(vt.cpu().numpy(), vr, rtol=1e-5, atol=1e-7)


def test_trained_network_beats_plain_formula(lt):
    """Train on particles of five volumes, evaluate on a sixth (held out)."""
    import torch
    feats, S_all, T_all = [], [], []
    for seed in range(6):
        m, lab, n = synth.training_particles(160, 100 + seed)
        S, R, F = gpu_objects(lt, m, lab, n)
        T = L.strict_sphericity(lab, n)
        S = S.cpu().numpy()
        ok = np.isfinite(T) & np.isfinite(S)
        ok[0] = False
        feats.append(F.cpu().numpy()[ok])
        S_all.append(S[ok])
        T_all.append(T[ok].astype(np.float32))
    ntr = sum(len(x) for x in S_all[:5])
    F = torch.from_numpy(np.concatenate(feats)).cuda()
    S = torch.from_numpy(np.concatenate(S_all)).cuda()
    T = torch.from_numpy(np.concatenate(T_all)).cuda()
    p = torch.from_numpy(synth.mlp_initial_params(0)).cuda()
    hist = lt.train_mlp(p, F, S, T, np.arange(ntr), epochs=150, batch=256, lr=1e-3)
    assert hist[-1] < 0.25 * hist[0]
    out = torch.empty(len(S_all[5]), dtype=torch.float32, device="cuda")
    lt.lt_mlp_infer(p, F[ntr:].contiguous(), S[ntr:].contiguous(), out)
    held_T = T_all[5].astype(np.float64)
    mae_plain = np.abs(S_all[5] - held_T).mean()
    mae_learned = np.abs(out.cpu().numpy() - held_T).mean()
    assert mae_learned < 0.5 * mae_plain, (mae_learned, mae_plain)


def test_checkpoint_resume_matches_continuous_run(lt, tmp_path):
    """Eight Adam steps in one go against four steps, a checkpoint written
    and read back into fresh device tensors, and four more steps: the same
    bits in the parameters and both moments."""
    import torch
    F, S, T, p = _random_problem(5, 2000)
    rng = np.random.default_rng(9)
    batches = [torch.from_numpy(rng.choice(len(S), 256, replace=False).astype(np.int32)).cuda()
               for _ in range(8)]
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    Fd, Sd, Td = d(F), d(S), d(T)

    def run(params, m, v, first, last):
        grad = torch.empty_like(params)
        for k in range(first, last):
            lt.lt_mlp_train_step(params, m, v, grad, k + 1, 1e-3, Fd, Sd, Td, batches[k])

    ref = [d(p.astype(np.float32)), torch.zeros(lt.MLP_PARAMS, device="cuda"),
           torch.zeros(lt.MLP_PARAMS, device="cuda")]
    run(*ref, 0, 8)
    part = [d(p.astype(np.float32)), torch.zeros(lt.MLP_PARAMS, device="cuda"),
            torch.zeros(lt.MLP_PARAMS, device="cuda")]
    run(*part, 0, 4)
    path = str(tmp_path / "net.ckpt")
    lt.lt_mlp_save(path, *part, step=4)
    fresh = [torch.full((lt.MLP_PARAMS,), float("nan"), device="cuda") for _ in range(3)]
    assert lt.lt_mlp_load(path, *fresh) == 4
    for a, b in zip(fresh, part):
        assert torch.equal(a, b)
    run(*fresh, 4, 8)
    for a, b in zip(fresh, ref):
        assert torch.equal(a, b)
    # a damaged file is refused and leaves the tensors alone
    raw = bytearray(open(path, "rb").read())
    raw[100] ^= 0xFF
    open(path, "wb").write(bytes(raw))
    keep = fresh[0].clone()
    with pytest.raises(lt.LTError) as e:
        lt.lt_mlp_load(path, *fresh)
    assert e.value.status == 9 and torch.equal(fresh[0], keep)
