"""The single-instance solver's on-chip mode (tuning.resident = 1): the grid
is held in the shared memory of one thread-block cluster and each step/run
call is one persistent launch of the batched run's on-chip kernel, which
writes the per-step trace of the single-instance API.

Against the streamed single-instance solver: the state bit for bit (both
kernels perform the per-cell update as the same sequence of roundings);
the per-step phi_y sums are added in another order, so FP64 observables
and trace agree to 1e-12 relative and FP32 ones to 2e-6 absolute.  Against
the FP64 oracle: 1e-10 relative.
A run split over several calls equals one call bit for bit (the state is
stored and reloaded exactly, the drive phase continues from the step
index)."""
import numpy as np
import pytest

import oracle
from paper_1401_6047_gb300 import bte
from paper_1401_6047_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _params(prec=W.FP64, **kw):
    base = dict(E_dc=1.1, E_omega=0.7, omega=2.2, B=1.3, B_omega=0.4, B_phase=0.3, mu=2.0,
                n_max=23, m_points=161, phiy_min=-8.0, phiy_max=8.0, dt=4e-3, periods=3.0,
                avg_window=1.0, precision=prec)
    base.update(kw)
    return W.Params(**base)


def _run(p, **kw):
    with bte.Solver(p, **kw) as s:
        s.run()
        o = s.observables()
        v, nr = s.trace()
        st = [np.array(x) for x in s.get_state(0) + s.get_state(1)]
    return o, v, nr, st


@pytest.mark.parametrize("prec", [W.FP64, W.FP32_MIXED])
def test_on_chip_equals_streamed(prec):
    p = _params(prec)
    o1, v1, n1, s1 = _run(p, resident=1)
    o0, v0, n0, s0 = _run(p)
    assert o1.status == bte.OK and o1.steps_total == o0.steps_total and o1.step == o0.step
    assert all(np.array_equal(x, y) for x, y in zip(s1, s0))
    if prec == W.FP64:
        for k in ("absorption", "v_dc_avg", "v_dr", "norm"):
            a, b = getattr(o1, k), getattr(o0, k)
            assert abs(a - b) <= 1e-12 * abs(b) + 1e-15, (k, a, b)
        assert np.max(np.abs(v1 - v0)) <= 1e-12 * np.max(np.abs(v0))
        assert np.max(np.abs(n1 - n0)) <= 1e-13
        scale = max(np.max(np.abs(x)) for x in s0)
        assert max(np.max(np.abs(x - y)) for x, y in zip(s1, s0)) <= 1e-12 * scale
    else:
        assert abs(o1.absorption - o0.absorption) <= 2e-6
        assert abs(o1.v_dc_avg - o0.v_dc_avg) <= 2e-6
        assert np.max(np.abs(n1 - n0)) <= 1e-7


def test_on_chip_fp64_matches_oracle():
    p = W.c1_fp64()  # 31 x 201, 125,660 steps: a 16-CTA cluster of two rows each
    ref = oracle.solve(p)
    with bte.Solver(p, resident=1) as s:
        s.run()
        o = s.observables()
    assert o.status == bte.OK
    assert abs(o.absorption - ref.A) <= 1e-10 * abs(ref.A)
    assert abs(o.v_dc_avg - ref.v_dc) <= 1e-10 * abs(ref.v_dc)
    assert abs(o.norm_max_abs_err - ref.norm_err) <= 1e-13


@pytest.mark.parametrize("prec", [W.FP64, W.FP32_MIXED])
def test_split_run_equals_one_call(prec):
    p = _params(prec, periods=1.0)
    o1, v1, n1, s1 = _run(p, resident=1)
    with bte.Solver(p, resident=1) as s:
        for n in (1, 7, 130):
            s.step(n)
        s.run()
        o2 = s.observables()
        v2, n2 = s.trace()
        s2 = [np.array(x) for x in s.get_state(0) + s.get_state(1)]
    assert o2.absorption == o1.absorption and o2.v_dc_avg == o1.v_dc_avg
    assert np.array_equal(v2, v1) and np.array_equal(n2, n1)
    assert all(np.array_equal(x, y) for x, y in zip(s2, s1))


def test_reset_and_rerun_on_chip():
    p = _params(periods=1.0)
    with bte.Solver(p, resident=1) as s:
        s.run()
        a = s.observables()
        s.reset()
        s.run()
        b = s.observables()
    assert a.absorption == b.absorption and a.v_dc_avg == b.v_dc_avg
