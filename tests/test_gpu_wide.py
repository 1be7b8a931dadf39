"""On-chip mode over several clusters (bte_tuning.resident = 3): the grid
cut into column blocks, one thread-block cluster each, CTAs holding their
part of the four arrays in shared memory for a whole call and exchanging
edge columns through global memory as words tagged with their half-step.

Per cell the kernel performs the operations of the one-launch-per-step
mode in the same order: FP64 states come out bit for bit the same, FP32
ones to 2e-6 of their scale (as in the one-cluster on-chip mode, the two
kernels' FP32 arithmetic is compiled to differently rounded code); the
per-step drift velocity and norm add the same terms in another order (per
cluster, then over clusters).  Against the oracle the usual bars hold:
FP64 1e-10 relative on the full 31 x 201 run, FP32 1e-5 absolute on
absorption and drift velocity.
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


def _run(p, steps, state=None, **kw):
    with bte.Solver(p, **kw) as s:
        if state is not None:
            s.set_state(0, state[0], state[1])
            s.set_state(1, state[2], state[3])
        for n in steps:
            s.step(n)
        v, nr = s.trace()
        o = s.observables(check=False)
        return v, nr, s.get_state(0), s.get_state(1), o


# (n_max, m_points, wide_cols): several clusters with a ragged last block,
# one column per cluster, one cluster, rows ragged over the cluster's CTAs,
# one CTA per cluster (two harmonics)
SHAPES = [
    (30, 201, 0),
    (30, 201, 29),
    (9, 37, 8),
    (40, 301, 64),
    (17, 250, 240),
    (1, 13, 3),
    (4, 21, 1),
    (64, 600, 96),
]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec", [W.FP64, W.FP32_MIXED])
def test_wide_equals_one_launch_per_step(shape, prec):
    n_max, m_points, cols = shape
    p = _params(n_max, m_points, prec)
    st = W.random_state(p, seed=11 + n_max)
    ref = _run(p, [57], st)
    got = _run(p, [20, 1, 36], st, resident=3, wide_cols=cols)  # three calls
    assert got[4].status == ref[4].status  # random states: |norm - 1| is large
    for g, r in zip(got[2] + got[3], ref[2] + ref[3]):
        if prec == W.FP64:
            assert np.array_equal(g, r)
        else:
            assert np.max(np.abs(g - r)) <= 2e-6 * max(1.0, np.max(np.abs(r)))
    tol = 1e-12 if prec == W.FP64 else 2e-6
    for g, r in zip(got[:2], ref[:2]):
        assert np.max(np.abs(g - r)) <= tol * max(1.0, np.max(np.abs(r)))


@pytest.mark.parametrize("prec", [W.FP64, W.FP32_MIXED])
def test_wide_c1_full_run_matches_oracle(prec):
    """31 x 201, 125,660 steps (16 launches of up to 8192 steps) against the
    FP64 oracle: FP64 1e-10 relative, FP32 1e-5 absolute."""
    p = W.c1_fp64().replace(precision=prec)
    ref = oracle.solve(W.c1_fp64(), want_state=True)
    with bte.Solver(p, resident=3) as s:
        s.run()
        o = s.observables()
        v, _ = s.trace()
        aw, bw = s.get_state(0)
    assert o.status == bte.OK
    if prec == W.FP64:
        assert abs(o.absorption - ref.A) <= 1e-10 * abs(ref.A)
        assert abs(o.v_dc_avg - ref.v_dc) <= 1e-10 * abs(ref.v_dc)
        assert np.max(np.abs(v - ref.v)) <= 1e-10 * np.max(np.abs(ref.v))
        sc = np.max(np.abs(ref.state.aw))
        assert np.max(np.abs(aw - ref.state.aw)) <= 1e-10 * sc
        assert np.max(np.abs(bw - ref.state.bw)) <= 1e-10 * sc
    else:
        assert abs(o.absorption - ref.A) <= 1e-5
        assert abs(o.v_dc_avg - ref.v_dc) <= 1e-5
        assert np.max(np.abs(v - ref.v)) <= 1e-5


def test_wide_matches_single_cluster_on_chip_mode():
    """Mode 3 and the one-cluster on-chip mode (1) on the 31 x 201 grid, 2000
    steps from equilibrium: the same final state to FP64 rounding."""
    p = W.c1_fp64()
    a = _run(p, [2000], resident=1)
    b = _run(p, [2000], resident=3)
    sc = np.max(np.abs(a[2][0]))
    for g, r in zip(b[2] + b[3], a[2] + a[3]):
        assert np.max(np.abs(g - r)) <= 1e-12 * sc
    assert np.max(np.abs(b[0] - a[0])) <= 1e-12 * np.max(np.abs(a[0]))


def test_wide_abort_after_recorded_error_and_reset():
    """With an error already recorded (a bounded wait that ran out), a poll
    of an exchange word that has to wait gives up at once, its CTA skips
    the rest of its work while still passing each cluster barrier, and the
    CTAs that poll its words give up in turn: the launch ends, the call
    reports BTE_ETIMEOUT, and a reset gives the same results as a fresh
    run."""
    p = _params(30, 201, W.FP64, periods=1.0)
    with bte.Solver(p, resident=3, wide_cols=32) as s:
        s.run()
        a = s.observables()
        s.reset()
        s.wait_probe(20_000)
        s.step(100)
        assert s.observables(check=False).status == bte.ETIMEOUT
        s.reset()
        s.run()
        b = s.observables()
    assert a.status == b.status == bte.OK
    assert a.absorption == b.absorption and a.v_dc_avg == b.v_dc_avg
