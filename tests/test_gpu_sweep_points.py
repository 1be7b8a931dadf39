"""Real points of the 4096-point parameter sweep, at their full grid sizes,
against the FP64 oracle.

The sweep's per-point grids (up to 103 harmonics and 1847 phi_y points under
the grid rule) are far larger than the small random points of the other
batched-run tests.  Six points are taken from the seeded sweep itself: the
two largest of those run by 16-CTA clusters and two run by 8-CTA clusters
in FP32, the point with the most phi_y points and the one with the most
harmonics.  Their runs are shortened to two drive periods (the last one
averaged) so that the oracle finishes in seconds; the grids, the drive and
the time step are the sweep's.  FP32 on chip and streamed: 1e-5 absolute on
absorption and drift velocity; FP64 (streamed at these sizes): 1e-10
relative.
"""
import numpy as np
import pytest

import oracle
from paper_1401_6047_gb300 import bte
from paper_1401_6047_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# indices into W.sweep_points(4096) (seed 1401) and the cluster size the
# FP32 on-chip tier gives each
PICK = {1974: 16, 534: 16, 2168: 8, 1735: 8, 3886: 16, 2398: 16}
ATOL32 = 1e-5
RTOL64 = 1e-10


@pytest.fixture(scope="module")
def cases():
    sweep = W.sweep_points(4096)
    pts = [sweep[i].replace(periods=2.0, avg_window=1.0) for i in PICK]
    refs = [oracle.solve(p.replace(precision=W.FP64)) for p in pts]
    return pts, refs


def test_points_are_the_large_sweep_grids(cases):
    pts, _ = cases
    assert list(bte.batch_plan(pts)) == list(PICK.values())
    assert max(p.m_points for p in pts) == 1847 and max(p.n_max for p in pts) == 102
    # in FP64 these grids do not fit on chip: they take the streamed tier
    assert not bte.batch_plan([p.replace(precision=W.FP64) for p in pts]).any()


@pytest.mark.parametrize("resident", [2, 1])
def test_fp32_sweep_points_match_oracle(cases, resident):
    """resident = 2: every point on chip (clusters of 16 and 8 CTAs);
    resident = 1: every point streamed."""
    pts, refs = cases
    res = bte.batch_run(pts, resident=resident)
    for p, o, r in zip(pts, res, refs):
        assert o.status == bte.OK and o.steps_total == r.K and o.window_steps == r.Kw
        assert abs(o.absorption - r.A) <= ATOL32, (p, o.absorption, r.A)
        assert abs(o.v_dc_avg - r.v_dc) <= ATOL32, (p, o.v_dc_avg, r.v_dc)
        assert abs(o.v_dr - r.v[-1]) <= ATOL32


def test_fp64_sweep_points_match_oracle(cases):
    pts, refs = cases
    res = bte.batch_run([p.replace(precision=W.FP64) for p in pts])
    for p, o, r in zip(pts, res, refs):
        assert o.status == bte.OK
        assert abs(o.absorption - r.A) <= RTOL64 * abs(r.A), (p, o.absorption, r.A)
        assert abs(o.v_dc_avg - r.v_dc) <= RTOL64 * abs(r.v_dc), (p, o.v_dc_avg, r.v_dc)
        assert abs(o.v_dr - r.v[-1]) <= RTOL64 * abs(r.v[-1]) + 1e-15
        assert abs(o.norm_max_abs_err - r.norm_err) <= 1e-12
