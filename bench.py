"""Benchmark: Mvoxels/s of the whole path (exact EDT -> exact local thickness
-> per-object sphericity and roundness) on the 512^3 particle volume.

One step = lt_measure over the resident volume (every kernel of the path).
Prints one JSON line (rank 0). Under torchrun (N > 1) every rank processes
its own volume (replicas, weak scaling); value = voxels of all ranks / max
time over ranks.

--impl reference times the CPU oracle (plain definition-level C loops) on a
bounded slab of the same workload, on this machine's host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mvoxels/s EDT+LT+shape at 512^3"
UNIT = "Mvoxels/s"


def max_over_ranks(x, dist, device):
    """The largest of every rank's x (x itself with one rank): the job's time
    is its slowest rank's."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, voxels_per_rank, seconds):
    """Mvoxels/s of the whole job: every rank's voxels over the slowest
    rank's time (weak scaling: each rank measures a volume of its own)."""
    return world * voxels_per_rank / seconds / 1e6


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="particles_3d_512")
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=10)
    p.add_argument("--no-batch", action="store_true", help="skip the batched-form measurement")
    p.add_argument("--no-learned", action="store_true", help="skip the learned-sphericity evaluation")
    p.add_argument("--batch-steps", type=int, default=10)
    p.add_argument("--targets", default=None,
                   help="learned-c4 protocol: targets file of tests/golden/make_strict_targets.py c4")
    p.add_argument("--epochs", type=int, default=40, help="learned-c4 protocol: training epochs")
    p.add_argument("--planes", type=int, default=64, help="slabs protocol: z planes per slab")
    p.add_argument("--protocol", choices=["object-count", "scaled-lt", "learned-c4", "slabs"], default=None,
                   help="run a timing protocol instead of the bench line (prints its own JSON)")
    p.add_argument("--draws", type=int, default=40, help="object-count protocol: selections per count")
    return p.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"lt_bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.gpu)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def algorithmic_bytes(name, n, n_surv):
    """Bytes a kernel must move per launch by its definition: the inputs it
    must read and the outputs it must write, once each."""
    table = {
        "edt_rows_x": 5 * n,          # mask in, g^2 out
        "edt_cols_y": 8 * n,          # u32 in, u32 out
        "edt_cols_z": 8 * n,
        "lt_ridge": 12 * n + 16 * n_surv,  # DT2, labels in; LT2 cleared; centre records out
        "shape_reduce": 8 * n,        # labels, LT2 in
    }
    return table.get(name)


# DRAM bytes (read + write) per launch from one ncu capture (dram__bytes_read
# and _write, one pass) of the current kernels on the 512^3 particle volume;
# valid for that workload only.
TRAFFIC = {"particles_3d_512": {"edt_rows_x": 341698304, "edt_cols_y": 752080384, "edt_cols_z": 1009333333, "lt_ridge": 1817653589, "lt_paint": 1923266389, "shape_reduce": 896663893}}


def _probe_lib():
    """The benchmark's calibration probe (bench_probe.cu, built next to this
    file by __graft_entry__.build(); not part of the library)."""
    import ctypes
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_bench_probe.so")
    lib = ctypes.CDLL(path)
    lib.probe_update_rate.restype = ctypes.c_int
    lib.probe_update_rate.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_void_p, ctypes.c_void_p]
    return lib


def update_rate_probe(dev):
    """Atomic-max update ceilings (G updates/s): one line per warp instruction
    or one line per lane, on a 32 MiB (L2-resident) and a 512 MiB buffer."""
    import ctypes
    import torch
    lib = _probe_lib()
    out = {}
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    for words, tag in ((1 << 23, "l2"), (1 << 27, "hbm")):
        buf = torch.zeros(words, dtype=torch.int32, device=dev)
        for pat, pname in ((0, "line_per_warp"), (1, "line_per_lane")):
            rate = ctypes.c_double(0.0)
            st = lib.probe_update_rate(ctypes.c_void_p(buf.data_ptr()), words, pat, 5, stream,
                                       ctypes.byref(rate))
            if st != 0:
                raise RuntimeError(f"update-rate probe failed ({st})")
            out[f"{pname}_{tag}"] = rate.value / 1e9
        del buf
    return out


def cpu_oracle_rate(mask, labels, n_labels, target_s=15.0):
    """The oracle as it stands on a z-slab of the workload; slab grown until
    one run takes about target_s seconds (bounded)."""
    import oracle
    oracle.build()
    nz = mask.shape[0]
    t = 8
    while True:
        sl = slice(0, min(t, nz))
        m, l = np.ascontiguousarray(mask[sl]), np.ascontiguousarray(labels[sl])
        t0 = time.perf_counter()
        oracle.pipeline(m, l, n_labels)
        dt = time.perf_counter() - t0
        if dt >= target_s / 3 or t >= nz:
            break
        t = min(nz, max(t * 2, int(t * target_s / max(dt, 1e-3) / 2)))
    what = "x".join(str(v) for v in m.shape)
    return m.size / dt / 1e6, f"{'rows' if m.ndim == 2 else 'z-slab'} {what} of the workload", dt


def measure_batch(lt, args, dev):
    """Batched form: 64 uneven 3D volumes + 8 2D 4096^2 masks as one graph
    launch (autotuned), against the same kernels issued volume by volume."""
    import tempfile
    import torch
    import synth
    t0 = time.perf_counter()
    vols = synth.batch_workload(args.seed)
    gen_s = time.perf_counter() - t0
    items = []
    for m, l, n in vols:
        items.append({"mask": torch.from_numpy(m).to(dev),
                      "labels": torch.from_numpy(l.view(np.int32)).to(dev),
                      "dt2": torch.empty(m.shape, dtype=torch.int32, device=dev),
                      "lt2": torch.empty(m.shape, dtype=torch.int32, device=dev),
                      "sphericity": torch.empty(n, dtype=torch.float32, device=dev),
                      "roundness": torch.empty(n, dtype=torch.float32, device=dev), "n_labels": n})
    nvox = sum(m.size for m, _, _ in vols)
    # algorithmic bytes of the whole batch: per voxel the EDT passes (x 5, y
    # 8, z 8 in 3D), the ridge pass's 12 and the shape reduction's 8 (the
    # 16 B per kept centre left out: the batch reports no centre counts)
    abytes = sum((41 if m.ndim == 3 else 33) * m.size for m, _, _ in vols)
    del vols
    batch = lt.Batch(items, branches=4)
    cache = os.environ.get("LT_AUTOTUNE_CACHE") or os.path.join(tempfile.mkdtemp(), "autotune.json")
    batch.autotune(cache)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_graph = timed(batch.run, args.batch_steps)
    ms_eager = timed(batch.run_eager, max(3, args.batch_steps // 2))
    # where an eager run's time goes, per kernel name (launches on parallel
    # branches overlap, so the sum can exceed the run)
    lt.lt_trace_enable(True)
    batch.run_eager()
    torch.cuda.synchronize()
    stages = {k: round(v[1], 4) for k, v in lt.lt_trace_summary().items()}
    lt.lt_trace_enable(False)
    batch.status()
    peak, peak_kind = peaks()
    out = {"value": nvox / (ms_graph * 1e-3) / 1e6, "unit": UNIT, "ms_per_batch": ms_graph,
           "algorithmic_bytes": abytes, "achieved_gbs": abytes / (ms_graph * 1e-3) / 1e9,
           "frac_hbm": abytes / (ms_graph * 1e-3) / 1e9 / peak, "peak_source": peak_kind,
           "eager_value": nvox / (ms_eager * 1e-3) / 1e6, "eager_ms_per_batch": ms_eager,
           "volumes": len(items), "voxels": nvox, "settings": batch.settings(), "eager_stage_ms": stages,
           "workload": "64 cubic volumes, edge U{64..384}, 512^3 mix; 8 x 2D 4096^2 ellipses",
           "generate_s": gen_s}
    batch.close()
    return out


GOLDEN_TARGETS = os.path.join(ROOT, "tests", "golden", "strict_sphericity_bench.txt")


def read_golden_targets(path=GOLDEN_TARGETS):
    """{seed: (n_labels, crc32, smoothed targets, binary targets)} from the
    text file tests/golden/make_strict_targets.py writes (only oracle code
    computes the targets; this reads numbers)."""
    out = {}
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            seed = int(p[1])
            if p[0] == "volume":
                out[seed] = [int(p[2]), int(p[3]), None, None]
            else:
                T = np.full(out[seed][0], np.nan)
                T[1:] = np.array(p[2:], dtype=np.float64)
                out[seed][2 if p[0] == "smooth" else 3] = T
    return {k: tuple(v) for k, v in out.items()}


def labels_crc(lab):
    import zlib
    return zlib.crc32(np.ascontiguousarray(lab, np.uint32).tobytes()) & 0xFFFFFFFF


LEARNED_TRAIN = 10  # the first volumes of the golden file train; the rest are held out


def learned_eval(lt, args, dev, mask, labels, n_labels):
    """The learned correction at scale: features of every particle of the
    golden file's volumes (synth.training_particles(320, seed)) from
    lt_measure_features, one network per strict-sphericity definition
    trained on the GPU on the first volumes (~20 k particles) and evaluated
    on the held-out rest (~100 k), MAE against each definition beside the
    plain S_LT. Per-object cost on the benchmark volume: lt_measure_features
    minus lt_measure (the histograms binned in the shape pass) plus
    lt_mlp_infer, against the plain path's own finalize step."""
    import torch
    import synth
    golden = read_golden_targets()
    seeds = sorted(golden)
    feats, S_all, T_all, vol_of = [], [], {"smooth": [], "binary": []}, []
    dt2 = lt2 = F = ws = None
    for i, seed in enumerate(seeds):
        m, lab, n = synth.training_particles(320, seed)
        gn, gcrc, Ts, Tb = golden[seed]
        if gn != n or gcrc != labels_crc(lab):
            raise RuntimeError("training volume differs from the one the golden targets were written for")
        mt = torch.from_numpy(m).to(dev)
        labt = torch.from_numpy(lab.view(np.int32)).to(dev)
        if dt2 is None or dt2.shape != m.shape:
            dt2 = torch.empty(m.shape, dtype=torch.int32, device=dev)
            lt2 = torch.empty_like(dt2)
        S = torch.empty(n, dtype=torch.float32, device=dev)
        R = torch.empty_like(S)
        F = torch.empty((n, lt.MLP_FEATURES), dtype=torch.float32, device=dev)
        ws = lt.lt_measure_features(mt, labt, n, dt2, lt2, S, R, F, ws=ws if ws is not None and
                                    ws.numel() >= lt.lib.lt_measure_features_workspace_size(n, 3, *m.shape[::-1]) else None)
        lt.lt_workspace_status(ws)
        Sn = S.cpu().numpy()
        ok = np.isfinite(Sn) & np.isfinite(Ts) & np.isfinite(Tb)
        ok[0] = False
        feats.append(F.cpu().numpy()[ok])
        S_all.append(Sn[ok])
        T_all["smooth"].append(Ts[ok].astype(np.float32))
        T_all["binary"].append(Tb[ok].astype(np.float32))
        vol_of.append(np.full(int(ok.sum()), i))
    ntr = sum(len(x) for x in S_all[:LEARNED_TRAIN])
    Fd = torch.from_numpy(np.concatenate(feats)).to(dev)
    Sd = torch.from_numpy(np.concatenate(S_all)).to(dev)
    S_held = np.concatenate(S_all[LEARNED_TRAIN:]).astype(np.float64)
    res = {"volumes": len(seeds), "objects_train": int(ntr), "objects_held_out": int(len(S_held)),
           "features": "lt_measure_features (histograms binned in the shape pass)"}
    out = torch.empty(len(S_held), dtype=torch.float32, device=dev)
    for name, desc in (("smooth", "smoothed-indicator mesh, mesh volume"),
                       ("binary", "binary-indicator mesh, voxel count")):
        Td = torch.from_numpy(np.concatenate(T_all[name])).to(dev)
        p = torch.from_numpy(synth.mlp_initial_params(0)).to(dev)
        t0 = time.perf_counter()
        hist = lt.train_mlp(p, Fd, Sd, Td, np.arange(ntr), epochs=60, batch=256, lr=1e-3)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        lt.lt_mlp_infer(p, Fd[ntr:].contiguous(), Sd[ntr:].contiguous(), out)
        held_T = np.concatenate(T_all[name][LEARNED_TRAIN:]).astype(np.float64)
        res[name] = {"target": desc, "mae_plain": float(np.abs(S_held - held_T).mean()),
                     "mae_learned": float(np.abs(out.cpu().numpy().astype(np.float64) - held_T).mean()),
                     "train_s": train_s, "final_train_loss": hist[-1]}
    # per-object cost on the benchmark volume
    m = torch.from_numpy(mask).to(dev)
    lab = torch.from_numpy(labels.view(np.int32)).to(dev)
    dt2 = torch.empty(mask.shape, dtype=torch.int32, device=dev)
    lt2 = torch.empty_like(dt2)
    S = torch.empty(n_labels, dtype=torch.float32, device=dev)
    R = torch.empty_like(S)
    F = torch.empty((n_labels, lt.MLP_FEATURES), dtype=torch.float32, device=dev)
    sl = torch.empty(n_labels, dtype=torch.float32, device=dev)
    wsp = lt.lt_measure(m, lab, n_labels, dt2, lt2, S, R)
    wsf = lt.lt_measure_features(m, lab, n_labels, dt2, lt2, S, R, F)
    p = torch.from_numpy(synth.mlp_initial_params(0)).to(dev)

    def timed(fn, reps=20):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    t_plain = timed(lambda: lt.lt_measure(m, lab, n_labels, dt2, lt2, S, R, ws=wsp))
    t_feat = timed(lambda: lt.lt_measure_features(m, lab, n_labels, dt2, lt2, S, R, F, ws=wsf))
    t_inf = timed(lambda: lt.lt_mlp_infer(p, F, S, sl))
    lt.lt_trace_enable(True)
    for _ in range(10):
        lt.lt_measure(m, lab, n_labels, dt2, lt2, S, R, ws=wsp)
        lt.lt_measure_features(m, lab, n_labels, dt2, lt2, S, R, F, ws=wsf)
    torch.cuda.synchronize()
    lt.lt_trace_enable(False)
    tr = {k: v[1] / max(1, v[0]) for k, v in lt.lt_trace_summary().items()}
    objs = n_labels - 1
    res["cost_512"] = {
        "objects": objs, "plain_ms": t_plain, "with_features_ms": t_feat, "infer_ms": t_inf,
        "features_ns_per_object": (t_feat - t_plain) * 1e6 / objs,
        "infer_ns_per_object": t_inf * 1e6 / objs,
        "learned_ns_per_object": (t_feat - t_plain + t_inf) * 1e6 / objs,
        "plain_finalize_ns_per_object": tr.get("shape_finalize", 0.0) * 1e6 / objs,
        "plain_ns_per_object": t_plain * 1e6 / objs,
        "shape_reduce_ms": tr.get("shape_reduce"), "shape_reduce_features_ms": tr.get("shape_reduce_features"),
        "features_final_ms": tr.get("features_final")}
    return res


def object_count_protocol(lt, args, dev):
    """The paper's second speed protocol (Sec. 5.3) on the synthetic
    particles: 10 object counts log-spaced in [1, 2000]; for each, `draws`
    random selections without replacement; for each selection the mean time
    (CUDA events, ms) to measure the selected objects
      whole_volume: one lt_measure over the volume holding only them (the
                    paper's all-objects-at-once use),
      graph:        one graph launch over per-object crops (lt_batch),
      per_object:   the same crops launched object after object.
    Crops are the objects' bounding boxes (outside the array is background,
    so no margin is needed; particles keep a one-voxel gap, so a crop gives
    the same DT, LT, S and R as the whole volume: `identical` checks it)."""
    import torch
    import scipy.ndimage as ndi
    import synth
    mask, labels, n = synth.workload(args.workload, args.seed)
    boxes = ndi.find_objects(labels.astype(np.int64))
    objs = []
    for l, sl in enumerate(boxes, start=1):
        if sl is None:
            continue
        lab = (labels[sl] == l)
        objs.append({"mask": torch.from_numpy(lab.astype(np.uint8)).to(dev),
                     "labels": torch.from_numpy(lab.astype(np.int32)).to(dev),
                     "dt2": torch.empty(lab.shape, dtype=torch.int32, device=dev),
                     "lt2": torch.empty(lab.shape, dtype=torch.int32, device=dev),
                     "sphericity": torch.empty(2, dtype=torch.float32, device=dev),
                     "roundness": torch.empty(2, dtype=torch.float32, device=dev),
                     "n_labels": 2, "label": l})
    lab_d = torch.from_numpy(labels.view(np.int32)).to(dev)
    shape = labels.shape
    dt2 = torch.empty(shape, dtype=torch.int32, device=dev)
    lt2 = torch.empty_like(dt2)
    S = torch.empty(n, dtype=torch.float32, device=dev)
    R = torch.empty_like(S)
    nz, ny, nx = shape
    ws = lt.workspace(lt.lib.lt_measure_workspace_size(n, 3, nx, ny, nz), dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    counts = sorted(set(int(round(c)) for c in np.logspace(0, np.log10(2000), 10)))
    rng = np.random.default_rng(args.seed)
    rows = []
    for k in counts:
        t_whole, t_graph, t_each, same = [], [], [], True
        for _ in range(args.draws):
            pick = rng.choice(len(objs), size=min(k, len(objs)), replace=False)
            sel = [objs[i] for i in pick]
            keep = torch.isin(lab_d, torch.tensor([o["label"] for o in sel], dtype=torch.int32, device=dev))
            m_sel = keep.to(torch.uint8)
            l_sel = torch.where(keep, lab_d, torch.zeros_like(lab_d))
            t_whole.append(timed(lambda: lt.lt_measure(m_sel, l_sel, n, dt2, lt2, S, R, ws=ws)))
            b = lt.Batch(sel, branches=8)
            t_graph.append(timed(b.run))
            t_each.append(timed(b.run_eager))
            b.status()
            got = torch.stack([torch.stack([o["sphericity"][1], o["roundness"][1]]) for o in sel]).cpu()
            idx = torch.tensor([o["label"] for o in sel], dtype=torch.long, device=dev)
            want = torch.stack([S[idx], R[idx]], 1).cpu()
            same = same and torch.equal(got, want)
            b.close()
            del keep, m_sel, l_sel
        rows.append({"objects": k, "whole_volume_ms": float(np.mean(t_whole)),
                     "graph_ms": float(np.mean(t_graph)), "per_object_ms": float(np.mean(t_each)),
                     "identical": bool(same)})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    return {"protocol": "object-count", "workload": args.workload, "objects_available": len(objs),
            "draws": args.draws, "volume": list(shape), "rows": rows}


def scaled_lt_protocol(lt, args, dev):
    """Accuracy against speed of the scaled local thickness (LT at 1/s
    resolution, upsampled; the fast-LT scale option) on the bench workload:
    per scale s, the time of lt_local_thickness_scaled + lt_shape_measures
    (full resolution) against the exact lt_measure, and the errors of S, R
    and LT against the exact values (objects with both finite)."""
    import torch
    import synth
    mask, labels, n = synth.workload(args.workload, args.seed)
    shape = labels.shape
    nd = labels.ndim
    nz, ny, nx = (1,) + shape if nd == 2 else shape
    m = torch.from_numpy(mask).to(dev)
    l = torch.from_numpy(labels.view(np.int32)).to(dev)
    dt2 = torch.empty(shape, dtype=torch.int32, device=dev)
    lt2 = torch.empty_like(dt2)
    S = torch.empty(n, dtype=torch.float32, device=dev)
    R = torch.empty_like(S)
    ws = lt.workspace(lt.lib.lt_measure_workspace_size(n, nd, nx, ny, nz), dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps=20):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_exact = timed(lambda: lt.lt_measure(m, l, n, dt2, lt2, S, R, ws=ws))
    lt.lt_workspace_status(ws)
    S0, R0, lt_exact = S.cpu().numpy().astype(np.float64), R.cpu().numpy().astype(np.float64), lt2.clone()
    obj = l != 0
    rows = [{"scale": 1, "ms": ms_exact, "speedup": 1.0}]
    for sc in (2, 3, 4):
        l2s = torch.empty_like(dt2)
        Ss, Rs = torch.empty_like(S), torch.empty_like(R)
        sws = lt.workspace(lt.lib.lt_local_thickness_scaled_workspace_size(sc, nd, nx, ny, nz), dev)
        shws = lt.workspace(lt.lib.lt_shape_workspace_size(n), dev)

        def step():
            lt.lt_local_thickness_scaled(m, l, sc, l2s, ws=sws)
            lt.lt_shape_measures(l, l2s, n, Ss, Rs, ws=shws)

        ms = timed(step)
        lt.lt_workspace_status(sws)
        a, b = Ss.cpu().numpy().astype(np.float64), Rs.cpu().numpy().astype(np.float64)
        ok = np.isfinite(a) & np.isfinite(S0)
        dS, dR = np.abs(a[ok] - S0[ok]), np.abs(b[ok] - R0[ok])
        dlt = (l2s[obj].double().sqrt() - lt_exact[obj].double().sqrt()).abs()
        rows.append({"scale": sc, "ms": ms, "speedup": ms_exact / ms,
                     "S_mae": float(dS.mean()), "S_p95": float(np.quantile(dS, 0.95)), "S_max": float(dS.max()),
                     "R_mae": float(dR.mean()), "R_p95": float(np.quantile(dR, 0.95)), "R_max": float(dR.max()),
                     "LT_mae_vox": float(dlt.mean()), "LT_rel_mae": float((dlt / lt_exact[obj].double().sqrt()).mean())})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
        del sws, shws
    return {"protocol": "scaled-lt", "workload": args.workload, "objects": n - 1, "rows": rows}


def _object_features(lt, dev, m, lab, n):
    """GPU pipeline with the learned features of one volume: (S, R, features)
    as numpy, the device time (ms) of lt_measure_features and of the plain
    lt_measure on the same volume."""
    import torch
    mt = torch.from_numpy(m).to(dev)
    labt = torch.from_numpy(lab.view(np.int32)).to(dev)
    dt2 = torch.empty(m.shape, dtype=torch.int32, device=dev)
    lt2 = torch.empty_like(dt2)
    S = torch.empty(n, dtype=torch.float32, device=dev)
    R = torch.empty_like(S)
    F = torch.empty((n, lt.MLP_FEATURES), dtype=torch.float32, device=dev)
    wsf = lt.lt_measure_features(mt, labt, n, dt2, lt2, S, R, F)
    wsp = lt.lt_measure(mt, labt, n, dt2, lt2, S, R)
    for _ in range(2):  # warm: the timed calls below do not pay first-use costs
        lt.lt_measure(mt, labt, n, dt2, lt2, S, R, ws=wsp)
        lt.lt_measure_features(mt, labt, n, dt2, lt2, S, R, F, ws=wsf)
    reps = 3
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    for _ in range(reps):
        lt.lt_measure(mt, labt, n, dt2, lt2, S, R, ws=wsp)
    ev[1].record()
    for _ in range(reps):
        lt.lt_measure_features(mt, labt, n, dt2, lt2, S, R, F, ws=wsf)
    ev[2].record()
    torch.cuda.synchronize()
    lt.lt_workspace_status(wsf)
    return (S.cpu().numpy(), R.cpu().numpy(), F.cpu().numpy(), ev[1].elapsed_time(ev[2]) / reps,
            ev[0].elapsed_time(ev[1]) / reps)


def learned_c4_protocol(lt, args, dev):
    """The learned-sphericity configuration at scale: train the correction on
    the GPU on the particles of N volumes of the widened 512^3 mix (~200 k
    particles for N = 82 at 320^3) and evaluate it on the 1024^3 volume of
    ~1 M particles: MAE of the plain S_LT and of the learned S against strict
    sphericity, and per-object costs. Targets (the FP64 oracle's strict
    sphericity) are read from --targets, written for the same seeded volumes
    by tests/golden/make_strict_targets.py c4."""
    import concurrent.futures as cf
    import torch
    import synth
    with np.load(args.targets) as z:  # read everything here: NpzFile is not thread-safe
        d = {k: z[k] for k in z.files}
    n_train = int(d["n_train"])
    feats, S_all, T_all = [], [], []

    def gen(i):
        crc_, n_, edge = (int(v) for v in d[f"train_{i}_crc"])
        m, lab, n = synth.training_particles(edge, 1000 + i)
        if n != n_ or labels_crc(lab) != crc_:
            raise RuntimeError(f"training volume {i} differs from the one its targets were written for")
        return m, lab, n, d[f"train_{i}"]

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=max(1, (os.cpu_count() or 4) // 2)) as ex:
        for m, lab, n, T in ex.map(gen, range(n_train)):
            S, R, F, _, _ = _object_features(lt, dev, m, lab, n)
            ok = np.isfinite(T) & np.isfinite(S)
            ok[0] = False
            feats.append(F[ok])
            S_all.append(S[ok])
            T_all.append(T[ok].astype(np.float32))
    prep_s = time.perf_counter() - t0
    F = torch.from_numpy(np.concatenate(feats)).to(dev)
    S = torch.from_numpy(np.concatenate(S_all)).to(dev)
    T = torch.from_numpy(np.concatenate(T_all)).to(dev)
    p = torch.from_numpy(synth.mlp_initial_params(0)).to(dev)
    t0 = time.perf_counter()
    hist = lt.train_mlp(p, F, S, T, np.arange(len(S)), epochs=args.epochs, batch=256, lr=1e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del F, S, T, feats
    # evaluation on the 1024^3 volume
    crc_, n_, _ = (int(v) for v in d["eval_crc"])
    m, lab, n = synth.workload("particles_3d_1024", 0)
    if n != n_ or labels_crc(lab) != crc_:
        raise RuntimeError("1024^3 volume differs from the one its targets were written for")
    Te = d["eval"]
    Sg, Rg, Fg, ms_with, ms_plain = _object_features(lt, dev, m, lab, n)
    Ft = torch.from_numpy(Fg).to(dev)
    St = torch.from_numpy(Sg).to(dev)
    og = torch.empty(n, dtype=torch.float32, device=dev)
    lt.lt_mlp_infer(p, Ft, St, og)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    lt.lt_mlp_infer(p, Ft, St, og)
    e1.record()
    torch.cuda.synchronize()
    ms_inf = e0.elapsed_time(e1)
    On = og.cpu().numpy()
    ok = np.isfinite(Te) & np.isfinite(Sg)
    ok[0] = False
    n_obj = int(ok.sum())
    return {"protocol": "learned-c4", "train_volumes": n_train, "train_objects": int(sum(len(x) for x in S_all)),
            "epochs": args.epochs, "train_loss_first_last": [hist[0], hist[-1]], "train_s": train_s,
            "prep_s": prep_s, "eval_volume": "particles_3d_1024", "eval_objects": n_obj,
            "mae_plain": float(np.abs(Sg[ok] - Te[ok]).mean()),
            "mae_learned": float(np.abs(On[ok] - Te[ok]).mean()),
            "per_object_ns": {"plain_pipeline": ms_plain * 1e6 / max(1, n - 1),
                              "features": (ms_with - ms_plain) * 1e6 / max(1, n - 1),
                              "inference": ms_inf * 1e6 / max(1, n - 1)},
            "target": "strict sphericity, FP64 oracle (smoothed marching tetrahedra), precomputed"}


def slabs_protocol(lt, args, dev):
    """The slab form (host-resident volume, --planes z planes on the device at
    a time) against the in-core host-buffer entry point on the same pinned
    host buffers: device memory used, Mvoxels/s end to end, identical S, R."""
    import torch
    import synth
    mask, labels, n = synth.workload(args.workload, args.seed)
    nz, ny, nx = mask.shape
    mh = torch.from_numpy(mask).pin_memory()
    lh = torch.from_numpy(labels.view(np.int32)).pin_memory()
    dt2 = torch.empty(mask.shape, dtype=torch.int32).pin_memory()
    S1, R1 = torch.empty(n).pin_memory(), torch.empty(n).pin_memory()
    S2, R2 = torch.empty(n).pin_memory(), torch.empty(n).pin_memory()
    wss = lt.workspace(lt.lib.lt_measure_slabs_workspace_size(n, nx, ny, nz, args.planes), dev)
    lt.lt_measure_slabs(mh, lh, n, args.planes, dt2, None, S1, R1, ws=wss)
    t0 = time.perf_counter()
    for _ in range(3):
        lt.lt_measure_slabs(mh, lh, n, args.planes, dt2, None, S1, R1, ws=wss)
    t_slabs = (time.perf_counter() - t0) / 3
    slab_bytes = wss.numel()
    del wss
    torch.cuda.empty_cache()
    wsh = lt.workspace(lt.lt_measure_host_workspace_size(n, mask.shape), dev)
    lt.lt_measure_host(mh, lh, n, S2, R2, wsh)
    t0 = time.perf_counter()
    for _ in range(3):
        lt.lt_measure_host(mh, lh, n, S2, R2, wsh)
    t_core = (time.perf_counter() - t0) / 3
    same = bool(np.array_equal(S1.numpy(), S2.numpy(), equal_nan=True) and
                np.array_equal(R1.numpy(), R2.numpy(), equal_nan=True))
    return {"protocol": "slabs", "workload": args.workload, "planes": args.planes,
            "device_bytes_slabs": int(slab_bytes), "device_bytes_in_core": int(wsh.numel()),
            "slabs_ms": t_slabs * 1e3, "in_core_ms": t_core * 1e3,
            "slabs_mvox_s": mask.size / t_slabs / 1e6, "in_core_mvox_s": mask.size / t_core / 1e6,
            "identical": same}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synth
    mask, labels, n = synth.workload(args.workload, args.seed)
    import oracle
    oracle.build()
    # size each step so that warmup + steps stay within about two minutes
    per_step = max(0.5, min(5.0, 120.0 / max(1, args.steps + args.warmup)))
    rate, sample, _ = cpu_oracle_rate(mask, labels, n, target_s=per_step * 3)
    t = int(sample.split()[1].split("x")[0])
    m, l = np.ascontiguousarray(mask[:t]), np.ascontiguousarray(labels[:t])
    for _ in range(args.warmup):
        oracle.pipeline(m, l, n)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.pipeline(m, l, n)
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    value = m.size / dt / 1e6
    cores = os.cpu_count()
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/f64",
           "data": "synthetic", "config": {"workload": args.workload, "seed": args.seed,
                                           "sample": sample},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import synth
    import paper_2504_05808_gb300 as lt

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    if args.protocol is not None:
        fn = {"object-count": object_count_protocol, "scaled-lt": scaled_lt_protocol,
              "learned-c4": learned_c4_protocol, "slabs": slabs_protocol}[args.protocol]
        if rank == 0:
            print(json.dumps(fn(lt, args, torch.device("cuda", local))), flush=True)
        return
    mask, labels, n_labels = synth.workload(args.workload, args.seed + rank)
    nd = mask.ndim
    shape = mask.shape
    nvox = mask.size
    dev = torch.device("cuda", local)
    m = torch.from_numpy(mask).to(dev)
    l = torch.from_numpy(labels.view(np.int32)).to(dev)
    dt2 = torch.empty(shape, dtype=torch.int32, device=dev)
    lt2 = torch.empty_like(dt2)
    S = torch.empty(n_labels, dtype=torch.float32, device=dev)
    R = torch.empty_like(S)
    nz, ny, nx = (1,) + shape if nd == 2 else shape
    ws = lt.workspace(lt.lib.lt_measure_workspace_size(n_labels, nd, nx, ny, nz), dev)
    stream = torch.cuda.current_stream(dev)

    for _ in range(max(3, args.warmup)):
        lt.lt_measure(m, l, n_labels, dt2, lt2, S, R, ws=ws)
    lt.lt_workspace_status(ws)
    counters = lt.lt_workspace_counters(ws)
    n_surv = counters["chunk_centres"] + counters["warp_centres"]

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    lt.lt_trace_enable(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        lt.lt_measure(m, l, n_labels, dt2, lt2, S, R, ws=ws)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    lt.lt_trace_enable(False)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    trace = lt.lt_trace_summary()
    lt.lt_workspace_status(ws)
    ms = max_over_ranks(ms, dist, dev)
    value = whole_job_rate(world, nvox, ms * 1e-3)

    # end to end through the host-buffer entry point (pinned host memory)
    mh = torch.from_numpy(mask).pin_memory()
    lh = torch.from_numpy(labels.view(np.int32)).pin_memory()
    Sh = torch.empty(n_labels, dtype=torch.float32).pin_memory()
    Rh = torch.empty(n_labels, dtype=torch.float32).pin_memory()
    del ws
    wsh = lt.workspace(lt.lt_measure_host_workspace_size(n_labels, shape), dev)
    for _ in range(2):
        lt.lt_measure_host(mh, lh, n_labels, Sh, Rh, wsh)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        lt.lt_measure_host(mh, lh, n_labels, Sh, Rh, wsh)
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    e2e_s = max_over_ranks(e2e_s, dist, dev)
    # the copy rate alone: the same pinned host bytes into device buffers,
    # one cudaMemcpyAsync each, no kernels (bounds what the host path can reach)
    dm = torch.empty(mh.shape, dtype=mh.dtype, device=dev)
    dl = torch.empty(lh.shape, dtype=lh.dtype, device=dev)
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dm.copy_(mh, non_blocking=True)
    dl.copy_(lh, non_blocking=True)
    h0.record(stream)
    for _ in range(3):
        dm.copy_(mh, non_blocking=True)
        dl.copy_(lh, non_blocking=True)
    h1.record(stream)
    torch.cuda.synchronize()
    h2d_gbs = 3 * (mask.nbytes + labels.nbytes) / (h0.elapsed_time(h1) * 1e-3) / 1e9
    del dm, dl
    e2e = {"value": whole_job_rate(world, nvox, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": int(mask.nbytes + labels.nbytes),
           "d2h_bytes_per_step": int(2 * 4 * n_labels),
           "ms_per_step": e2e_s * 1e3, "h2d_copy_gbs": h2d_gbs}

    # per-kernel roofline: HBM kernels by algorithmic bytes, painting by
    # updates per second against the probed atomic-update ceiling
    peak, peak_kind = peaks()
    probe = update_rate_probe(dev) if rank == 0 else None
    total_ms = sum(x[1] for x in trace.values())
    kernels = {}
    for k, v in trace.items():
        avg = v[1] / max(1, v[0])
        e = {"launches": v[0], "avg_ms": avg, "share": v[1] / max(1e-9, total_ms)}
        ab = algorithmic_bytes(k, nvox, n_surv)
        if ab is not None:
            e.update({"algorithmic_bytes": ab, "achieved_gbs": ab / (avg * 1e-3) / 1e9})
            e["frac_hbm"] = e["achieved_gbs"] / peak
        tr = TRAFFIC.get(args.workload, {}).get(k)
        if tr is not None:
            e["traffic"] = tr
        if k == "lt_paint":
            e.update({"updates": counters["updates"],
                      "achieved_gupd": counters["updates"] / (avg * 1e-3) / 1e9})
        kernels[k] = e
    dom = max(trace, key=lambda k: trace[k][1])
    kd = kernels[dom]
    if dom == "lt_paint" and probe:
        upeak = max(probe.values())
        roof = {"kernel": dom, "bound": "atomic", "achieved": kd["achieved_gupd"], "peak": upeak,
                "unit": "Gupdates/s", "frac": kd["achieved_gupd"] / upeak,
                "traffic": TRAFFIC.get(args.workload, {}).get(dom), "avg_ms": kd["avg_ms"], "updates": counters["updates"],
                "peak_source": "measured in this run by the atomic-max rate probe (best of its patterns)",
                "probe_gupd": probe}
    else:
        roof = {"kernel": dom, "bound": "hbm", "achieved": kd.get("achieved_gbs"), "peak": peak,
                "unit": "GB/s", "frac": kd.get("frac_hbm"), "traffic": TRAFFIC.get(args.workload, {}).get(dom),
                "avg_ms": kd["avg_ms"], "algorithmic_bytes": kd.get("algorithmic_bytes"),
                "peak_source": peak_kind}
    gpu_launches = sum(v[0] for v in trace.values())
    # the whole step against HBM by the same per-kernel algorithmic bytes
    # (painting, counted in updates, adds none)
    step_ab = sum(algorithmic_bytes(k, nvox, n_surv) or 0 for k in trace)
    step_roof = {"algorithmic_bytes": step_ab, "achieved_gbs": step_ab / (ms * 1e-3) / 1e9,
                 "frac_hbm": step_ab / (ms * 1e-3) / 1e9 / peak, "peak_source": peak_kind}

    batched = None
    if not args.no_batch:
        del wsh
        torch.cuda.empty_cache()
        batched = measure_batch(lt, args, dev)
    learned = None
    if not args.no_learned and rank == 0:
        learned = learned_eval(lt, args, dev, mask, labels, n_labels)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, sample, _ = cpu_oracle_rate(mask, labels, n_labels)
        cpu = {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": sample}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "u32",
               "data": "synthetic",
               "config": {"workload": args.workload, "voxels": nvox, "objects": n_labels - 1,
                          "foreground": float(mask.mean()), "centres_kept": n_surv,
                          "counters": counters,
                          "seed": args.seed, "parallelism": f"replicas{world}",
                          "l2": "inputs larger than L2 (no flush needed)"},
               "roofline": roof, "kernels": kernels, "step_roofline": step_roof, "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": gpu_launches, "clocks": clk, "batched": batched, "learned": learned}
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
