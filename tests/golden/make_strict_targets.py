"""Writes strict-sphericity targets for seeded synthetic particle volumes.

The targets of the learned sphericity correction are the FP64 oracle's
strict sphericity (Eq. 1 on a marching-tetrahedra mesh of the object's
indicator smoothed by a Gaussian of one voxel; oracle.learned). This script
is the only place that computes them outside the tests: it calls only
oracle/ and the seeded generators in synth/, and writes plain numbers that
bench.py reads, so the measurement never runs the oracle itself.

  python tests/golden/make_strict_targets.py bench
      the learned leg of bench.py: BENCH_VOLUMES volumes of
      synth.training_particles(320, seed), seeds from BENCH_SEED0 (the first
      BENCH_TRAIN for training, ~20 k particles; the rest held out, ~100 k),
      both target definitions (smoothed mesh with its enclosed volume, and
      binary-indicator mesh with the voxel count)
      -> tests/golden/strict_sphericity_bench.txt
  python tests/golden/make_strict_targets.py c4 --out FILE.npz [--train-volumes N] [--edge E]
      N training volumes of edge E (about 2,440 particles each at E = 320;
      82 volumes give ~200 k particles) and the 1024^3 volume of ~1 M
      particles -> FILE.npz (crc32 of each volume's labels, targets with NaN
      for absent labels)

Each volume is identified by the generator call and the crc32 of its labels,
which the reader checks before using the targets.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import sys
import zlib

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import oracle.learned as L  # noqa: E402
import synth  # noqa: E402

BENCH_FILE = os.path.join(HERE, "strict_sphericity_bench.txt")
BENCH_EDGE, BENCH_SEED0, BENCH_VOLUMES, BENCH_TRAIN = 320, 2000, 62, 10


def crc(labels: np.ndarray) -> int:
    return zlib.crc32(np.ascontiguousarray(labels, np.uint32).tobytes()) & 0xFFFFFFFF


def targets(labels: np.ndarray, n: int) -> np.ndarray:
    return L.strict_sphericity(labels, n)


def _fmt(T: np.ndarray) -> str:
    return " ".join("nan" if not np.isfinite(t) else f"{t:.7g}" for t in T[1:])


def write_bench() -> None:
    lines = ["# strict sphericity targets (FP64 oracle, Eq. 1 on marching-tetrahedra meshes) of",
             f"# synth.training_particles({BENCH_EDGE}, seed); written by make_strict_targets.py",
             f"# train: the first {BENCH_TRAIN} volumes; held out: the rest",
             "# 'volume seed n_labels crc32', then 'smooth seed t_1 .. t_{n-1}' (smoothed indicator, mesh volume)",
             "# and 'binary seed t_1 .. t_{n-1}' (binary indicator, voxel count); nan: no voxel or no surface"]
    for seed in range(BENCH_SEED0, BENCH_SEED0 + BENCH_VOLUMES):
        _, lab, n = synth.training_particles(BENCH_EDGE, seed)
        lines.append(f"volume {seed} {n} {crc(lab)}")
        lines.append(f"smooth {seed} " + _fmt(targets(lab, n)))
        lines.append(f"binary {seed} " + _fmt(L.strict_sphericity_binary(lab, n)))
        print(f"volume {seed}: {n - 1} labels", file=sys.stderr, flush=True)
    with open(BENCH_FILE, "w") as f:
        f.write("\n".join(lines) + "\n")


def read_bench(path: str = BENCH_FILE):
    """{seed: (n_labels, crc32, smoothed targets, binary targets)}, targets
    as float64 arrays of n_labels with NaN where absent (label 0 NaN)."""
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
                T[1:] = np.array([float(v) for v in p[2:]], np.float64)
                out[seed][2 if p[0] == "smooth" else 3] = T
    return {k: tuple(v) for k, v in out.items()}


def write_c4(path: str, n_train: int, edge: int, threads: int) -> None:
    res = {}

    def one(i):
        _, lab, n = synth.training_particles(edge, 1000 + i)
        return i, n, crc(lab), lab

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        for i, n, c, lab in ex.map(one, range(n_train)):
            res[f"train_{i}_crc"] = np.array([c, n, edge], np.int64)
            res[f"train_{i}"] = targets(lab, n)
            del lab
            print(f"train volume {i}: {n - 1} labels", file=sys.stderr, flush=True)
    _, lab, n = synth.workload("particles_3d_1024", 0)
    res["eval_crc"] = np.array([crc(lab), n, 1024], np.int64)
    res["eval"] = targets(lab, n)
    np.savez(path, n_train=np.array(n_train), **res)


def main():
    p = argparse.ArgumentParser()
    p.add_argument("set", choices=["bench", "c4"])
    p.add_argument("--out")
    p.add_argument("--train-volumes", type=int, default=82)
    p.add_argument("--edge", type=int, default=320)
    p.add_argument("--threads", type=int, default=os.cpu_count() or 4)
    a = p.parse_args()
    oracle.build()
    if a.set == "bench":
        write_bench()
    else:
        write_c4(a.out, a.train_volumes, a.edge, a.threads)


if __name__ == "__main__":
    main()
