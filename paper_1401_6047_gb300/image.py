"""Headless image dump of a distribution f(phi_x, phi_y): an 8-bit grayscale
PGM file (no graphics library involved), f scaled linearly from its minimum
(black) to its maximum (white), phi_y along the rows from top to bottom,
phi_x along the columns."""
from __future__ import annotations

import numpy as np


def write_pgm(path: str, f: np.ndarray) -> None:
    """f [nphix][m_points] as returned by ``Solver.pdf``."""
    img = np.asarray(f, dtype=np.float64).T  # rows: phi_y, columns: phi_x
    lo, hi = float(np.min(img)), float(np.max(img))
    scale = 255.0 / (hi - lo) if hi > lo else 0.0
    px = np.clip(np.rint((img - lo) * scale), 0, 255).astype(np.uint8)
    with open(path, "wb") as fh:
        fh.write(f"P5\n{px.shape[1]} {px.shape[0]}\n255\n".encode("ascii"))
        fh.write(px.tobytes())


def read_pgm(path: str) -> np.ndarray:
    with open(path, "rb") as fh:
        data = fh.read()
    parts = data.split(b"\n", 3)
    assert parts[0] == b"P5"
    w, h = (int(v) for v in parts[1].split())
    return np.frombuffer(parts[3], dtype=np.uint8).reshape(h, w)
