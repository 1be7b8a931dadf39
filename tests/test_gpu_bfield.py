"""A time-dependent field B(t) = B + B_omega cos(omega t + B_phase) through
the C ABI, against the FP64 oracle (reading R13: B sampled where E is, the
stencil coefficient at the time of the grid that supplies the stencil).

Bars as for a constant field: FP64 1e-10 relative (observables, trace and
state), FP32-mixed 1e-5 absolute on absorption and drift velocity; both
tiers of the batched run against the oracle.  With omega = 0 the field is
the constant B + B_omega cos(B_phase), and the library must give the same
bits as a constant-field run with that B."""
import math

import numpy as np
import pytest

import oracle
from paper_1401_6047_gb300 import bte
from paper_1401_6047_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL64 = 1e-10


def _params(prec=W.FP64, **kw):
    base = dict(E_dc=1.2, E_omega=0.6, omega=2.5, B=1.1, B_omega=0.7, B_phase=0.4, mu=2.0,
                n_max=28, m_points=257, phiy_min=-8.0, phiy_max=8.0, dt=4e-3, periods=3.0,
                avg_window=1.0, precision=prec)
    base.update(kw)
    return W.Params(**base)


def _rel_state(sol, st):
    aw, bw = sol.get_state(0)
    af, bf = sol.get_state(1)
    sw = max(np.max(np.abs(st.aw)), np.max(np.abs(st.bw)))
    sf = max(np.max(np.abs(st.af)), np.max(np.abs(st.bf)))
    return max(np.max(np.abs(aw - st.aw)) / sw, np.max(np.abs(bw - st.bw)) / sw,
               np.max(np.abs(af - st.af)) / sf, np.max(np.abs(bf - st.bf)) / sf)


def test_fp64_single_instance_matches_oracle():
    """Several tiles and row chunks (tile_m 64, chunk_n 8) with a ragged last
    tile (257 columns): observables, the drift-velocity trace and both final
    grids within 1e-10 relative."""
    p = _params()
    ref = oracle.solve(p, want_state=True)
    with bte.Solver(p, tile_m=64, chunk_n=8) as s:
        s.run()
        o = s.observables()
        v, nr = s.trace()
        assert o.status == bte.OK
        assert abs(o.absorption - ref.A) <= RTOL64 * abs(ref.A)
        assert abs(o.v_dc_avg - ref.v_dc) <= RTOL64 * abs(ref.v_dc)
        assert abs(o.norm_max_abs_err - ref.norm_err) <= 1e-13
        assert np.max(np.abs(v - ref.v)) <= RTOL64 * np.max(np.abs(ref.v))
        assert _rel_state(s, ref.state) <= RTOL64


def test_fp32_single_instance_within_1e5():
    p = _params(W.FP32_MIXED)
    ref = oracle.solve(p.replace(precision=W.FP64))
    with bte.Solver(p) as s:
        s.run()
        o = s.observables()
    assert abs(o.absorption - ref.A) <= 1e-5
    assert abs(o.v_dc_avg - ref.v_dc) <= 1e-5


def test_field_oscillation_changes_the_result():
    """The oscillating part is not ignored: B_omega = 0.7 moves the drift
    and the absorption far beyond the parity bars."""
    with bte.Solver(_params()) as s:
        s.run()
        o1 = s.observables()
    with bte.Solver(_params(B_omega=0.0)) as s:
        s.run()
        o0 = s.observables()
    assert abs(o1.v_dc_avg - o0.v_dc_avg) > 1e-4
    assert abs(o1.absorption - o0.absorption) > 1e-4


@pytest.mark.parametrize("resident", [2, 1])
@pytest.mark.parametrize("prec", [W.FP64, W.FP32_MIXED])
def test_batched_tiers_match_oracle(resident, prec):
    """On chip (resident=2, shrunk shared memory so that clusters of several
    CTAs are used) and streamed (resident=1): every point against the
    oracle."""
    rng = np.random.default_rng(71)
    pts = []
    for _ in range(4):
        pts.append(_params(prec, E_dc=float(rng.uniform(0.0, 3.0)),
                           omega=float(rng.uniform(1.0, 4.0)), B=float(rng.uniform(0.0, 2.0)),
                           B_omega=float(rng.uniform(0.1, 1.0)),
                           B_phase=float(rng.uniform(-math.pi, math.pi)),
                           n_max=int(rng.integers(10, 36)), m_points=int(rng.integers(60, 240)),
                           periods=1.5))
    smem = 30000 if prec == W.FP32_MIXED else 60000
    res = bte.batch_run(pts, resident=resident,
                        resident_smem=smem if resident == 2 else 0)
    for p, o in zip(pts, res):
        ref = oracle.solve(p.replace(precision=W.FP64))
        assert o.status == bte.OK
        if prec == W.FP64:
            assert abs(o.absorption - ref.A) <= RTOL64 * abs(ref.A) + 1e-15
            assert abs(o.v_dc_avg - ref.v_dc) <= RTOL64 * abs(ref.v_dc) + 1e-15
        else:
            assert abs(o.absorption - ref.A) <= 1e-5
            assert abs(o.v_dc_avg - ref.v_dc) <= 1e-5


def test_zero_frequency_is_a_constant_field_bit_for_bit():
    q = W.Params(E_dc=1.3, E_omega=0.0, omega=0.0, B=0.8, mu=2.0, n_max=16, m_points=121,
                 phiy_min=-8, phiy_max=8, dt=5e-3, t_max=2.0, avg_window=1.0)
    a = q.replace(B_omega=0.5, B_phase=0.9)
    b = q.replace(B=0.8 + 0.5 * math.cos(0.9))
    for kw in (dict(), dict(precision=W.FP32_MIXED)):
        out = []
        for p in (a, b):
            with bte.Solver(p.replace(**kw)) as s:
                s.run()
                o = s.observables()
                out.append((o.v_dc_avg, o.norm_max_abs_err, s.get_state(0)[0].copy()))
        assert out[0][0] == out[1][0] and out[0][1] == out[1][1]
        assert np.array_equal(out[0][2], out[1][2])
