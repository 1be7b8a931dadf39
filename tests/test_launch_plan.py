"""Host-side checks of the launch plan the library picks: every TMA bulk copy
of the fused step kernel starts on a 16-byte boundary, copies a multiple of
16 bytes and stays inside its row; the grid covers every cell."""
import pytest

from paper_1401_6047_gb300 import bte
from paper_1401_6047_gb300 import workloads as W

SHAPES = [(9, 37, 32, 4), (23, 131, 32, 8), (40, 301, 64, 12), (17, 250, 128, 5), (1, 3, 32, 4),
          (64, 1000, 256, 16), (30, 401, 0, 0), (33, 157, 64, 8), (25, 301, 0, 0),
          (12, 121, 32, 4), (5, 21, 0, 0), (20, 201, 0, 0), (12, 101, 0, 0), (20, 161, 0, 0)]


def _plans():
    for prec in (W.FP64, W.FP32_MIXED):
        for n_max, m_points, tile, chunk in SHAPES:
            yield W.Params(n_max=n_max, m_points=m_points, precision=prec), tile, chunk
        for p in (W.c1_fp64(), W.c2(), W.c3(), W.paper_table1()):
            yield p.replace(precision=prec), 0, 0
        for tile in (32, 64, 128, 256, 512, 1024):
            yield W.c2(prec), tile, 0


@pytest.mark.parametrize("case", list(_plans()), ids=lambda c: f"{c[0].n_max}x{c[0].m_points}p{c[0].precision}t{c[1]}c{c[2]}")
def test_bulk_copies_aligned_and_in_bounds(case):
    p, tile, chunk = case
    elem = 8 if p.precision == W.FP64 else 4
    H = 16 // elem     # halo columns streamed per side (one TMA granule)
    G = 128 // elem    # zero ghost columns before m = 0
    try:
        s = bte.launch_shape(p, tile, chunk)
    except bte.BteError as e:
        # only shapes whose shared memory or block does not fit may be refused
        assert e.code == bte.EINVAL and ("shared memory" in str(e) or "for this precision" in str(e))
        return
    Wt, pitch, ntx, nty, cn = s["tile_m"], s["pitch"], s["grid_x"], s["grid_y"], s["chunk_n"]
    M1, N1 = p.m_points, p.n_max + 1
    assert ntx * Wt >= M1 and (ntx - 1) * Wt < M1
    assert nty * cn >= N1 and (nty - 1) * cn < N1
    assert Wt <= 1024 and Wt % 4 == 0
    assert (pitch * elem) % 16 == 0
    LW = Wt + 2 * H
    assert (LW * elem) % 16 == 0
    for tx in range(ntx):
        p0 = G + tx * Wt
        first = p0 - H
        assert first >= 0 and (first * elem) % 16 == 0
        assert first + LW <= pitch
        assert (p0 * elem) % 16 == 0  # vector stores of a thread's columns
    # ghost columns: interior columns G..G+M, zero ghosts on both sides
    assert H >= 2 and G + M1 + 1 <= pitch
