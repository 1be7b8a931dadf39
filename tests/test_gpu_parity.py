"""Parity of the CUDA solver (through the C ABI) with the FP64 CPU oracle.

Tolerances: the FP64 path must match the oracle to 1e-10 relative (state
arrays relative to their largest entry, observables relative to their
value); the FP32-mixed path to 1e-5 absolute on absorption and drift
velocity.  Run lengths are cut where the oracle would take more than a few
seconds; grids are the full configured sizes where stated.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1401_6047_gb300 import bte
from paper_1401_6047_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL64 = 1e-10


def _rel_arr(x, ref):
    s = np.max(np.abs(ref))
    return np.max(np.abs(x - ref)) / (s if s > 0 else 1.0)


def _cmp_state(sol, st, rtol, what=""):
    """Largest error of each array relative to the largest |a| of its grid
    (the state's scale: b starts at zero and its FP32 rounding error is set
    by the a-sized terms of the update)."""
    aw, bw = sol.get_state(0)
    af, bf = sol.get_state(1)
    sw = max(np.max(np.abs(st.aw)), np.max(np.abs(st.bw)))
    sf = max(np.max(np.abs(st.af)), np.max(np.abs(st.bf)))
    errs = {"aw": np.max(np.abs(aw - st.aw)) / sw, "bw": np.max(np.abs(bw - st.bw)) / sw,
            "af": np.max(np.abs(af - st.af)) / sf, "bf": np.max(np.abs(bf - st.bf)) / sf}
    worst = max(errs.values())
    assert worst <= rtol, (what, errs)
    return worst


def test_c1_fp64_full_run_matches_oracle():
    """31 x 201 grid, 125,660 steps (20 drive periods): every observable,
    the whole trace and the final state within 1e-10 relative."""
    p = W.c1_fp64()
    ref = oracle.solve(p, want_state=True)
    with bte.Solver(p) as s:
        s.run()
        o = s.observables()
        v, nr = s.trace()
        assert o.step == ref.K and o.steps_total == ref.K and o.window_steps == ref.Kw
        assert abs(o.dt_eff - ref.dt_eff) <= 1e-18
        assert abs(o.absorption - ref.A) <= RTOL64 * abs(ref.A)
        assert abs(o.v_dc_avg - ref.v_dc) <= RTOL64 * abs(ref.v_dc)
        assert abs(o.norm_max_abs_err - ref.norm_err) <= 1e-13
        assert _rel_arr(v, ref.v) <= RTOL64
        assert np.max(np.abs(nr - ref.norm)) <= 1e-13
        _cmp_state(s, ref.state, RTOL64, "c1 final state")
        assert o.status == bte.OK


SHAPES = [
    # (n_max, m_points, tile_m, chunk_n): several tiles, ragged column tail,
    # several row chunks, ragged row tail
    (9, 37, 32, 4),
    (23, 131, 32, 8),
    (40, 301, 64, 12),
    (17, 250, 128, 5),
    (1, 3, 32, 4),       # smallest grid
    (64, 1000, 256, 16),
]


def _rand_params(n_max, m_points, prec, omega=1.3):
    return W.Params(E_dc=0.9, E_omega=0.6, omega=omega, B=2.1, mu=1.4, n_max=n_max,
                    m_points=m_points, phiy_min=-6.0, phiy_max=6.0, dt=4e-3, periods=4.0,
                    avg_window=1.0, precision=prec)


def test_low_temperature_fp64_matches_oracle():
    """The paper's low-temperature point (mu = 116, B = 4, E_omega = 0.1,
    E_dc = 6, alpha = 0.9496, omega = 3; 61 harmonics, 1201 phi_y points,
    12 drive periods): the regime of high harmonics and a narrow f0, where
    the oracle is pinned by the characteristics integral."""
    p = W.Params(E_dc=6.0, E_omega=0.1, omega=3.0, B=4.0, mu=116.0, alpha=0.9496, n_max=60,
                 m_points=1201, phiy_min=-6.0, phiy_max=6.0, dt=2e-3, periods=12.0,
                 avg_window=1.0)
    ref = oracle.solve(p, want_state=True)
    with bte.Solver(p) as s:
        s.run()
        o = s.observables()
        assert o.status == bte.OK
        assert abs(o.absorption - ref.A) <= RTOL64 * abs(ref.A)
        assert abs(o.v_dc_avg - ref.v_dc) <= RTOL64 * abs(ref.v_dc)
        assert abs(o.norm_max_abs_err - ref.norm_err) <= 1e-13
        # every harmonic of both grids, not only the rows the observables read
        _cmp_state(s, ref.state, RTOL64, "low temperature final state")
        v, _ = s.trace()
        assert _rel_arr(v, ref.v) <= RTOL64


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec,vec", [(W.FP64, 2), (W.FP32_MIXED, 2), (W.FP32_MIXED, 4)])
def test_random_state_parity(shape, prec, vec):
    """Arbitrary (random) state on both grids, 40 steps at B != 0 and
    E_omega != 0, several launch shapes: element-wise parity of all four
    arrays and of the drift-velocity / norm trace."""
    n_max, m_points, tile_m, chunk_n = shape
    p = _rand_params(n_max, m_points, prec)
    aw, bw, af, bf = W.random_state(p, seed=11 + n_max)
    st = oracle.State(aw.copy(), bw.copy(), af.copy(), bf.copy())
    v_ref, n_ref = oracle.advance(p, st, 0, 40)
    with bte.Solver(p, tile_m=tile_m, chunk_n=chunk_n, graph_steps=16, vec=vec) as s:
        s.set_state(0, aw, bw)
        s.set_state(1, af, bf)
        s.step(40)
        v, nr = s.trace(1, 40)
        tol = RTOL64 if prec == W.FP64 else 2e-5
        _cmp_state(s, st, tol, f"shape {shape}")
        assert _rel_arr(v, v_ref) <= tol
        assert _rel_arr(nr, n_ref) <= tol


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec,vec", [(W.FP64, 2), (W.FP32_MIXED, 2), (W.FP32_MIXED, 4)])
def test_alternating_row_walk_parity(shape, prec, vec):
    """The downward row walk (odd one-step launches with walk = 2; the
    default for states larger than L2) against the oracle on a random state
    of every launch shape, and equal bit for bit to walking upward every
    step (walk = 1): the same per-cell arithmetic in another order.  Graphs
    of 6 launches plus direct launches for the remaining 5 steps, so both
    directions run in both launch forms."""
    n_max, m_points, tile_m, chunk_n = shape
    p = _rand_params(n_max, m_points, prec)
    aw, bw, af, bf = W.random_state(p, seed=29 + n_max)
    st = oracle.State(aw.copy(), bw.copy(), af.copy(), bf.copy())
    v_ref, n_ref = oracle.advance(p, st, 0, 17)
    got = {}
    for walk in (1, 2):
        with bte.Solver(p, tile_m=tile_m, chunk_n=chunk_n, graph_steps=6, vec=vec, walk=walk) as s:
            s.set_state(0, aw, bw)
            s.set_state(1, af, bf)
            s.step(17)
            got[walk] = (*s.get_state(0), *s.get_state(1), *s.trace(1, 17))
            if walk == 2:
                tol = RTOL64 if prec == W.FP64 else 2e-5
                _cmp_state(s, st, tol, f"shape {shape}, alternating walk")
                assert _rel_arr(got[2][4], v_ref) <= tol
                assert _rel_arr(got[2][5], n_ref) <= tol
    for x, y in zip(got[1], got[2]):
        assert np.array_equal(x, y)


def test_alternating_row_walk_batched_is_bitwise():
    """The batched streamed tier with both walk orders: identical bits."""
    pts = [_rand_params(20 + 3 * i, 161 + 40 * i, W.FP32_MIXED).replace(periods=0.3, avg_window=0.1)
           for i in range(3)]
    r1 = bte.batch_run(pts, resident=1, walk=1)
    r2 = bte.batch_run(pts, resident=1, walk=2)
    for a, b in zip(r1, r2):
        assert a.status == bte.OK and b.status == bte.OK
        assert a.absorption == b.absorption and a.v_dc_avg == b.v_dc_avg
        assert a.norm_max_abs_err == b.norm_max_abs_err


@pytest.mark.parametrize("prec", [W.FP64, W.FP32_MIXED])
def test_c2_full_grid_short_run(prec):
    """401 x 4001 grid in the launch shape the benchmark times, 24 steps from
    the equilibrium start, full state against the oracle."""
    p = W.c2(prec)
    st = oracle.init(p)
    v_ref, n_ref = oracle.advance(p, st, 0, 24)
    with bte.Solver(p) as s:
        s.step(24)
        tol = RTOL64 if prec == W.FP64 else 1e-6
        _cmp_state(s, st, tol, "c2")
        v, nr = s.trace(1, 24)
        assert np.max(np.abs(v - v_ref)) <= (1e-12 if prec == W.FP64 else 1e-6)
        assert np.max(np.abs(nr - n_ref)) <= (1e-12 if prec == W.FP64 else 1e-6)


def test_c3_full_grid_short_run_fp32():
    """2049 x 8193 grid (16.8 M cells), FP32-mixed, 3 steps, full state."""
    p = W.c3(W.FP32_MIXED)
    st = oracle.init(p)
    v_ref, n_ref = oracle.advance(p, st, 0, 3)
    with bte.Solver(p) as s:
        s.step(3)
        _cmp_state(s, st, 1e-6, "c3")
        v, nr = s.trace(1, 3)
        assert np.max(np.abs(v - v_ref)) <= 1e-6
        assert np.max(np.abs(nr - n_ref)) <= 1e-6


def test_fp32_mixed_matches_fp64_on_observables():
    """Per-result error of the FP32-mixed path against FP64 on the 401 x 4001
    configuration (run shortened to 6 periods, 2 averaged): <= 1e-5 absolute
    on absorption and time-averaged drift velocity."""
    p = W.c2().replace(periods=6.0, avg_window=2.0)
    o64 = bte.solve(p.replace(precision=W.FP64))
    o32 = bte.solve(p.replace(precision=W.FP32_MIXED))
    assert abs(o32.absorption - o64.absorption) <= 1e-5
    assert abs(o32.v_dc_avg - o64.v_dc_avg) <= 1e-5
    assert o32.norm_max_abs_err <= 1e-4 and o64.norm_max_abs_err <= 1e-10


def test_graph_replay_equals_direct_launches():
    """CUDA-graph replay and one launch per step give identical bits."""
    p = _rand_params(30, 401, W.FP64)
    outs = []
    for g in (1, 50):
        with bte.Solver(p, graph_steps=g) as s:
            s.step(173)
            outs.append((s.get_state(0), s.get_state(1), s.trace()))
    for x, y in zip(outs[0], outs[1]):
        for a, b in zip(x, y):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", [W.FP64, W.FP32_MIXED])
def test_checkpoint_resume_is_bitwise(prec):
    """A run split at step k, saved and resumed in a new handle, equals the
    uninterrupted run bit for bit."""
    p = _rand_params(25, 301, prec, omega=2.0).replace(periods=3.0)
    with bte.Solver(p) as s:
        s.run()
        full = (s.get_state(0), s.get_state(1), s.trace(), s.observables())
    k = 1001
    with bte.Solver(p) as s:
        s.step(k)
        ck = (s.get_state(0), s.get_state(1), s.trace())
    with bte.Solver(p) as s:
        s.set_state(0, *ck[0])
        s.set_state(1, *ck[1])
        s.set_step(k, *ck[2])
        s.run()
        res = (s.get_state(0), s.get_state(1), s.trace(), s.observables())
    for x, y in zip(full[:3], res[:3]):
        for a, b in zip(x, y):
            assert np.array_equal(a, b)
    assert full[3].absorption == res[3].absorption
    assert full[3].v_dc_avg == res[3].v_dc_avg


def test_sublattice_decoupling_on_gpu():
    """Two runs that differ only on the n+m-even sublattice agree exactly on
    the odd one (the stencil reads (n+-1, m+-1) only)."""
    p = _rand_params(33, 157, W.FP64)
    base = W.random_state(p, seed=5)
    pert = W.random_state(p, seed=6, parity=0)
    res = []
    for st in (base, [x + y for x, y in zip(base, pert)]):
        with bte.Solver(p, tile_m=64, chunk_n=8) as s:
            s.set_state(0, st[0], st[1])
            s.set_state(1, st[2], st[3])
            s.step(37)
            res.append(s.get_state(0) + s.get_state(1))
    n, m = np.indices(base[0].shape)
    odd = ((n + m) % 2) == 1
    for x, y in zip(res[0], res[1]):
        assert np.array_equal(x[odd], y[odd])


def test_step_past_end_and_bad_state_rejected():
    p = _rand_params(5, 21, W.FP64).replace(periods=1.0)
    with bte.Solver(p) as s:
        K = s.observables().steps_total
        with pytest.raises(bte.BteError) as e:
            s.step(K + 1)
        assert e.value.code == bte.ESTATE
        a, b = s.get_state(0)
        b[0, 3] = 1.0
        with pytest.raises(bte.BteError) as e:
            s.set_state(0, a, b)
        assert e.value.code == bte.EINVAL
        s.run()
        assert s.observables().step == K


def test_instability_reported():
    """A time step far beyond the stencil's stability limit produces
    non-finite values or a drifting norm, reported as BTE_EUNSTABLE."""
    p = W.Params(E_dc=1.0, E_omega=0.0, omega=0.0, B=40.0, mu=1.0, n_max=12, m_points=101,
                 phiy_min=-5, phiy_max=5, dt=0.05, t_max=20.0, avg_window=1.0)
    with bte.Solver(p) as s:
        s.run()
        o = s.observables(check=False)
        assert o.status == bte.EUNSTABLE
        with pytest.raises(bte.BteError) as e:
            s.observables()
        assert e.value.code == bte.EUNSTABLE


def test_zero_omega_run():
    """omega = 0: constant drive, absorption undefined (NaN), drift velocity
    averaged over the final time window; parity with the oracle."""
    p = W.Params(E_dc=1.7, E_omega=0.0, omega=0.0, B=1.5, mu=2.0, n_max=20, m_points=161,
                 phiy_min=-8, phiy_max=8, dt=5e-3, t_max=6.0, avg_window=1.0)
    ref = oracle.solve(p)
    o = bte.solve(p)
    assert math.isnan(o.absorption)
    assert abs(o.v_dc_avg - ref.v_dc) <= RTOL64 * abs(ref.v_dc)


def test_caller_workspace_and_stream():
    """Device memory and the stream can come from PyTorch (the caller)."""
    torch = pytest.importorskip("torch")
    p = _rand_params(20, 201, W.FP64).replace(periods=1.0)
    n = bte.workspace_size(p)
    buf = torch.empty(n, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    with bte.Solver(p, stream=stream.cuda_stream, workspace=buf.data_ptr(),
                    workspace_bytes=n) as s:
        s.run()
        o1 = s.observables()
    o2 = bte.solve(p)
    assert o1.absorption == o2.absorption and o1.v_dc_avg == o2.v_dc_avg
