"""Training and held-out data of the MLP surrogate: seeded points of the
sweep box, each solved by the batched CUDA solver (``bte_batch_run``) under
the surrogate run protocol (``workloads.surrogate_params``).

Usage: python -m paper_1401_6047_gb300.surrogate_data OUT.npz N SEED [CHUNK [MAX_SECONDS]]

Writes y [N, 2] (absorption, time-averaged drift velocity, float64) and a
per-point status for the N seeded points x = workloads.sweep_matrix(N, SEED)
(E_dc, E_omega, omega, B, mu), which load() regenerates from N and SEED.
The file is rewritten after every chunk, so an interrupted run keeps its
work and a later run with the same N and SEED continues it; MAX_SECONDS
stops after the chunk that passes that time.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

from . import bte
from . import workloads as W

DATA_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")
FILES = {"train": "surrogate_train.npz", "heldout": "surrogate_heldout.npz"}

# training schedule of the shipped ensemble (Adam, cosine decay of lr)
TRAINING = dict(epochs=200, batch=1024, lr=2e-3, lr_min=2e-5, seed=0)


def load(name: str):
    """(x, y) of a data file, points the solver reported OK only; None when
    the file is absent."""
    path = os.path.join(DATA_DIR, FILES[name])
    if not os.path.exists(path):
        return None
    d = np.load(path)
    x = d["x"] if "x" in d else W.sweep_matrix(int(d["n"]), int(d["seed"]))
    ok = (d["status"] == bte.OK) & np.all(np.isfinite(d["y"]), axis=1)
    return x[ok], d["y"][ok]


def generate(path: str, n: int, seed: int, chunk: int = 4096, precision: int = W.FP32_MIXED,
             max_seconds: float = 0.0):
    X = W.sweep_matrix(n, seed)
    Y = np.full((n, 2), np.nan)
    S = np.full(n, -99, dtype=np.int8)
    done = 0
    if os.path.exists(path):
        d = np.load(path)
        if int(d["seed"]) == seed and d["y"].shape == Y.shape:
            Y, S, done = d["y"].copy(), d["status"].astype(np.int8), int(d["done"])
    t0 = time.time()
    while done < n:
        hi = min(n, done + chunk)
        pts = [W.surrogate_params(x, precision) for x in X[done:hi]]
        res = bte.batch_run(pts, check=False)
        Y[done:hi, 0] = [o.absorption for o in res]
        Y[done:hi, 1] = [o.v_dc_avg for o in res]
        S[done:hi] = [o.status for o in res]
        done = hi
        np.savez(path, y=Y, status=S, done=done, seed=seed, n=n)
        print(f"{done}/{n} points, {time.time() - t0:.1f} s", flush=True)
        if max_seconds and time.time() - t0 > max_seconds:
            break
    return X, Y, S


if __name__ == "__main__":
    out, n, seed = sys.argv[1], int(sys.argv[2]), int(sys.argv[3])
    chunk = int(sys.argv[4]) if len(sys.argv) > 4 else 4096
    limit = float(sys.argv[5]) if len(sys.argv) > 5 else 0.0
    generate(out, n, seed, chunk, max_seconds=limit)
