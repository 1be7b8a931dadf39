"""Persistent mode of the single-instance solver (bte_tuning.resident = 2):
one cooperative launch per call (per 8192 steps) whose CTAs run the fused
step for every step, with a grid barrier between steps and the state in
global memory (L2-resident when it fits there).

The per-cell arithmetic, the launch shape and the order of the per-step
sums are those of the one-launch-per-step mode, so both modes must agree
bit for bit: trace and final state, FP64 and FP32.  Against the oracle the
usual bars hold (FP64 1e-10 relative on the full 31 x 201 run).
"""
import numpy as np
import pytest

import oracle
from paper_1401_6047_gb300 import bte
from paper_1401_6047_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _params(n_max, m_points, prec, periods=3.0):
    return W.Params(E_dc=1.4, E_omega=0.7, omega=2.2, B=2.6, mu=1.7, n_max=n_max,
                    m_points=m_points, phiy_min=-7.0, phiy_max=7.0, dt=4e-3, periods=periods,
                    avg_window=1.0, precision=prec)


def _run(p, resident, steps, state=None, **kw):
    with bte.Solver(p, resident=resident, **kw) as s:
        if state is not None:
            s.set_state(0, state[0], state[1])
            s.set_state(1, state[2], state[3])
        for n in steps:
            s.step(n)
        v, nr = s.trace()
        return v, nr, s.get_state(0), s.get_state(1), s.observables(check=False)


SHAPES = [(9, 37, 32, 4), (40, 301, 64, 12), (64, 1000, 256, 16), (1, 3, 32, 4)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec,vec", [(W.FP64, 2), (W.FP32_MIXED, 4), (W.FP32_MIXED, 2)])
def test_persistent_equals_one_launch_per_step(shape, prec, vec):
    n_max, m_points, tile_m, chunk_n = shape
    p = _params(n_max, m_points, prec)
    st = W.random_state(p, seed=3 + n_max)
    kw = dict(tile_m=tile_m, chunk_n=chunk_n, vec=vec)
    ref = _run(p, 0, [57], st, **kw)
    got = _run(p, 2, [20, 1, 36], st, **kw)  # split over calls: one launch each
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    for g, r in zip(got[2] + got[3], ref[2] + ref[3]):
        assert np.array_equal(g, r)


@pytest.mark.parametrize("prec", [W.FP64, W.FP32_MIXED])
def test_persistent_c2_grid_equals_streamed(prec):
    """401 x 4001 grid (the L2-resident configuration) with its default
    launch shape, 40 steps from the equilibrium start."""
    p = W.c2(prec)
    ref = _run(p, 0, [40])
    got = _run(p, 2, [40])
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    for g, r in zip(got[2] + got[3], ref[2] + ref[3]):
        assert np.array_equal(g, r)


def test_persistent_c1_full_run_matches_oracle():
    """31 x 201, 125,660 steps: 16 launches of up to 8192 steps."""
    p = W.c1_fp64()
    ref = oracle.solve(p, want_state=True)
    with bte.Solver(p, resident=2) as s:
        s.run()
        o = s.observables()
        v, _ = s.trace()
        aw, bw = s.get_state(0)
    assert o.status == bte.OK
    assert abs(o.absorption - ref.A) <= 1e-10 * abs(ref.A)
    assert abs(o.v_dc_avg - ref.v_dc) <= 1e-10 * abs(ref.v_dc)
    assert np.max(np.abs(v - ref.v)) <= 1e-10 * np.max(np.abs(ref.v))
    sc = np.max(np.abs(ref.state.aw))
    assert np.max(np.abs(aw - ref.state.aw)) <= 1e-10 * sc
    assert np.max(np.abs(bw - ref.state.bw)) <= 1e-10 * sc


def test_persistent_reset_and_timeout_report():
    p = _params(12, 97, W.FP64, periods=1.0)
    with bte.Solver(p, resident=2) as s:
        s.run()
        a = s.observables()
        s.wait_probe(20_000)
        assert s.observables(check=False).status == bte.ETIMEOUT
        s.reset()
        s.run()
        b = s.observables()
    assert a.status == b.status == bte.OK
    assert a.absorption == b.absorption and a.v_dc_avg == b.v_dc_avg
