"""Batched sweep (bte_batch_run): many independent parameter points with
different grids, drives and run lengths advance in lock-step, one fused
launch per step over every point's tiles.

Each point must give what the single-instance solver gives with the same
tile shape (the per-step drift velocity and norm bit for bit, the window
averages up to summation order), and what the FP64 oracle gives (1e-10
relative in FP64, 1e-5 absolute on absorption and drift velocity in FP32).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1401_6047_gb300 import bte
from paper_1401_6047_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL64 = 1e-10


def _mixed_points(prec, seed=7, n=7):
    """Small heterogeneous points: harmonic counts, grids, B, mu, omega (so
    run lengths) all differ; one point at B = 0 and one at E_omega = 0."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        n_max = int(rng.integers(6, 30))
        m_points = int(rng.integers(40, 260))
        L = float(rng.uniform(4.0, 9.0))
        out.append(W.Params(E_dc=float(rng.uniform(0.0, 4.0)), E_omega=float(rng.uniform(0.05, 1.0)),
                            omega=float(rng.uniform(0.8, 4.0)), B=float(rng.uniform(0.0, 3.0)),
                            mu=float(rng.uniform(0.5, 4.0)), n_max=n_max, m_points=m_points,
                            phiy_min=-L, phiy_max=L, dt=float(rng.choice([2e-3, 4e-3, 5e-3])),
                            periods=float(rng.choice([1.5, 2.0, 3.0])), avg_window=1.0,
                            precision=prec))
    if n > 2:
        out[1] = out[1].replace(B=0.0)
        out[2] = out[2].replace(E_omega=0.0)
    return out


def _same_obs(o, r, exact_window=False):
    assert o.step == r.step and o.steps_total == r.steps_total
    assert o.window_steps == r.window_steps and o.steps_per_period == r.steps_per_period
    assert o.dt_eff == r.dt_eff
    assert o.v_dr == r.v_dr and o.norm == r.norm
    assert o.norm_max_abs_err == r.norm_max_abs_err
    assert o.status == r.status
    for x, y in ((o.absorption, r.absorption), (o.v_dc_avg, r.v_dc_avg)):
        if math.isnan(y):
            assert math.isnan(x)
        elif exact_window:
            assert x == y
        else:
            assert abs(x - y) <= 1e-12 * max(abs(y), 1e-3)


@pytest.mark.parametrize("prec,vec", [(W.FP64, 2), (W.FP32_MIXED, 2), (W.FP32_MIXED, 4)])
def test_batch_equals_single_instance(prec, vec):
    pts = _mixed_points(prec)
    tile, chunk = 32 * vec, 8
    res = bte.batch_run(pts, tile_m=tile, chunk_n=chunk, vec=vec, resident=1)
    for p, o in zip(pts, res):
        r = bte.solve(p, tile_m=tile, chunk_n=chunk, vec=vec)
        _same_obs(o, r)


def test_batch_fp64_matches_oracle():
    pts = _mixed_points(W.FP64, seed=11)
    res = bte.batch_run(pts)
    for p, o in zip(pts, res):
        ref = oracle.solve(p)
        assert o.steps_total == ref.K and o.window_steps == ref.Kw
        assert abs(o.v_dc_avg - ref.v_dc) <= RTOL64 * abs(ref.v_dc) + 1e-15
        if p.E_omega > 0:
            assert abs(o.absorption - ref.A) <= RTOL64 * abs(ref.A) + 1e-15
        assert abs(o.v_dr - ref.v[-1]) <= RTOL64 * abs(ref.v[-1]) + 1e-15
        assert abs(o.norm - ref.norm[-1]) <= 1e-13
        assert abs(o.norm_max_abs_err - ref.norm_err) <= 1e-13
        assert o.status == bte.OK


@pytest.mark.parametrize("vec", [2, 4])
def test_batch_fp32_within_1e5_of_oracle(vec):
    pts = _mixed_points(W.FP32_MIXED, seed=13)
    res = bte.batch_run(pts, vec=vec)
    for p, o in zip(pts, res):
        ref = oracle.solve(p)
        assert abs(o.absorption - ref.A) <= 1e-5 or (p.E_omega == 0 and math.isnan(ref.A))
        assert abs(o.v_dc_avg - ref.v_dc) <= 1e-5
        assert o.status == bte.OK


def test_batch_split_into_several_batches_is_bitwise():
    """Batch composition changes which CTA runs which tile, never the bits."""
    pts = _mixed_points(W.FP32_MIXED, seed=17, n=9)
    whole = bte.batch_run(pts)
    split = bte.batch_run(pts, max_batch=2)
    tiny = bte.batch_run(pts, max_batch_bytes=1)
    for a, b, c in zip(whole, split, tiny):
        _same_obs(a, b, exact_window=True)
        _same_obs(a, c, exact_window=True)


def test_batch_graph_and_direct_launches_agree():
    pts = _mixed_points(W.FP64, seed=19, n=4)
    g = bte.batch_run(pts, graph_steps=256, resident=1)
    d = bte.batch_run(pts, graph_steps=1, resident=1)
    for a, b in zip(g, d):
        _same_obs(a, b, exact_window=True)


def test_batch_reports_unstable_point_and_keeps_the_rest():
    good = _mixed_points(W.FP64, seed=23, n=3)
    bad = W.Params(E_dc=1.0, E_omega=0.0, omega=0.0, B=40.0, mu=1.0, n_max=12, m_points=101,
                   phiy_min=-5, phiy_max=5, dt=0.05, t_max=20.0, avg_window=1.0)
    pts = good[:1] + [bad] + good[1:]
    with pytest.raises(bte.BteError) as e:
        bte.batch_run(pts, resident=1)
    assert e.value.code == bte.EUNSTABLE
    res = bte.batch_run(pts, check=False, resident=1)
    assert res[1].status == bte.EUNSTABLE
    for p, o in zip(pts[:1] + pts[2:], res[:1] + res[2:]):
        r = bte.solve(p, tile_m=128, chunk_n=16)
        _same_obs(o, r)


def test_batch_zero_omega_point():
    p = W.Params(E_dc=1.7, E_omega=0.0, omega=0.0, B=1.5, mu=2.0, n_max=20, m_points=161,
                 phiy_min=-8, phiy_max=8, dt=5e-3, t_max=6.0, avg_window=1.0)
    q = _mixed_points(W.FP64, seed=29, n=2)
    res = bte.batch_run([p] + q)
    ref = oracle.solve(p)
    assert math.isnan(res[0].absorption)
    assert abs(res[0].v_dc_avg - ref.v_dc) <= RTOL64 * abs(ref.v_dc)


def test_batch_sweep_points_fp32_vs_fp64():
    """Points of the 4096-point sweep (its grid rule, shortened to two
    periods, one averaged): FP32 batched within 1e-5 absolute of the FP64
    single-instance solver on absorption and drift velocity."""
    pts = W.sweep_points(n=4096, periods=2.0, avg_window=1.0)[:: 512]
    res = bte.batch_run(pts)
    for p, o in zip(pts, res):
        r = bte.solve(p.replace(precision=W.FP64))
        assert abs(o.absorption - r.absorption) <= 1e-5
        assert abs(o.v_dc_avg - r.v_dc_avg) <= 1e-5
        assert o.status == bte.OK and r.status == bte.OK
