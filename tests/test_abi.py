"""CPU-side checks of the C ABI library: it loads without a GPU, exports every
symbol the headers declare, and its host-only helpers (Miller Bessel ratios,
time grid, parameter validation) are right."""
import ctypes
import glob
import math
import os
import re

import numpy as np
import pytest

from paper_1401_6047_gb300 import bte
from paper_1401_6047_gb300 import workloads as W
from tests import analytic as an

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        names += re.findall(r"^BTE_API\s+[\w\s\*]+?\b(bte\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("bte_create", "bte_step", "bte_run", "bte_observables", "bte_destroy",
                     "bte_get_state", "bte_set_state", "bte_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    L = bte.lib()
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing
    assert "sm_103a" in bte.version()


def test_miller_bessel_ratio_matches_scipy():
    """The library's I_n/I_0 (Miller recurrence) against scipy.special.ive."""
    for mu, nmax in [(0.5, 200), (1.0, 30), (2.0, 400), (20.0, 2048), (116.0, 119), (10.0, 4000)]:
        r = bte.bessel_ratio(mu, nmax)
        ref = an.bessel_ratio(mu, np.arange(nmax + 1))
        big = ref > 1e-280
        assert np.all(np.abs(r[big] - ref[big]) <= 1e-12 * ref[big] + 1e-300), (mu, nmax)
        assert np.max(np.abs(r - ref)) < 1e-14
        assert r[0] == 1.0


def test_time_grid_closed_form():
    p = W.c2()
    dt, P, K, Kw = bte.time_grid(p)
    assert P == round(2 * math.pi / (p.omega * p.dt)) == 6283
    assert abs(dt - 2 * math.pi / (p.omega * P)) < 1e-18
    assert K == 50 * P and Kw == 10 * P
    q = W.Params(omega=0.0, E_omega=0.0, t_max=3.0, dt=1e-2, avg_window=1.0)
    dt, P, K, Kw = bte.time_grid(q)
    assert (dt, P, K, Kw) == (1e-2, 0, 300, 100)


@pytest.mark.parametrize("bad", [dict(n_max=0), dict(m_points=2), dict(dt=0.0), dict(mu=0.0),
                                 dict(alpha=-1.0), dict(omega=-2.0), dict(E_dc=float("inf")),
                                 dict(phiy_max=-20.0), dict(avg_window=25.0), dict(precision=7),
                                 dict(B_omega=float("nan")), dict(B_phase=float("inf"))])
def test_invalid_parameters_rejected_on_host(bad):
    """Validation happens before any CUDA call, so it needs no GPU."""
    with pytest.raises(bte.BteError) as e:
        bte.workspace_size(W.c1_fp64().replace(**bad))
    assert e.value.code == bte.EINVAL


def test_on_chip_single_instance_mode_is_planned_on_host():
    """resident=1 (one cluster holds the grid): a grid that fits plans with
    the same device layout as the streamed mode; one that does not fit any
    16-CTA cluster, or a bad flag, is rejected before any CUDA call.
    resident=2 (persistent launches) plans the streamed layout, plus its
    dependency counters, for any grid."""
    p = W.c1_fp64()
    assert bte.workspace_size(p, resident=1) == bte.workspace_size(p)
    with pytest.raises(bte.BteError) as e:
        bte.workspace_size(W.c2(), resident=1)  # 401 x 4001: about 26 MB of state
    assert e.value.code == bte.EINVAL
    # resident=2 (persistent launches): the streamed layout plus the per-item
    # completion counters and ntx + 1 slots of row-0 partial sums, any grid
    ws0, ws2 = bte.workspace_size(W.c2()), bte.workspace_size(W.c2(), resident=2)
    shape = bte.launch_shape(W.c2())
    assert ws0 < ws2 <= ws0 + 4096 * (shape["grid_x"] + 1) + 4 * shape["grid_x"] * shape["grid_y"] + 1024
    for bad in (dict(resident=4), dict(resident=-1), dict(walk=3), dict(walk=-1)):
        t = bte._tuning()
        for k, v in bad.items():
            setattr(t, k, v)
        n = ctypes.c_size_t()
        rc = bte.lib().bte_workspace_size(ctypes.byref(bte.to_params(p)), ctypes.byref(t), ctypes.byref(n))
        assert rc == bte.EINVAL


def test_workspace_size_covers_state():
    p = W.c2()
    n = bte.workspace_size(p)
    assert n >= 8 * p.cells * 4
    n64 = bte.workspace_size(p.replace(precision=W.FP64))
    assert n64 >= 8 * p.cells * 8
    with pytest.raises(bte.BteError):
        bte.workspace_size(p, tile_m=30)


@pytest.mark.parametrize("case", ["mixed_precision", "vec3", "fp64_vec4", "tile", "chunk",
                                  "bad_point", "smem"])
def test_batch_run_rejects_bad_input_on_host(case):
    """bte_batch_run validates every point and option before any CUDA call."""
    pts = [W.c1_fp64(), W.c1_fp64().replace(omega=2.0)]
    kw = {}
    if case == "mixed_precision":
        pts[1] = pts[1].replace(precision=W.FP32_MIXED)
    elif case == "vec3":
        kw = dict(vec=3)
    elif case == "fp64_vec4":
        kw = dict(vec=4)
    elif case == "tile":
        kw = dict(tile_m=30)
    elif case == "chunk":
        kw = dict(chunk_n=2)
    elif case == "bad_point":
        pts[1] = pts[1].replace(m_points=2)
    elif case == "smem":
        kw = dict(tile_m=1024, chunk_n=4096)
    with pytest.raises(bte.BteError) as e:
        bte.batch_run(pts, **kw)
    assert e.value.code == bte.EINVAL


def test_batch_run_of_nothing_is_ok():
    assert bte.batch_run([]) == []


def test_batch_plan_assigns_tiers_on_host():
    """bte_batch_plan: on-chip cluster sizes grow as the per-CTA budget
    shrinks, streamed (0) when told so or when nothing fits."""
    pts = [W.Params(n_max=40, m_points=401, precision=W.FP32_MIXED),
           W.Params(n_max=200, m_points=2001, precision=W.FP32_MIXED),
           W.Params(n_max=400, m_points=4001, precision=W.FP32_MIXED)]
    big = bte.batch_plan(pts)
    small = bte.batch_plan(pts, resident_smem=40000)
    assert list(bte.batch_plan(pts, resident=1)) == [0, 0, 0]
    assert big[0] >= 1 and big[2] == 0            # 401 x 4001 never fits on chip
    assert small[0] >= big[0]
    assert all(t in (0, 1, 2, 4, 8, 16) for t in list(big) + list(small))
    with pytest.raises(bte.BteError) as e:
        bte.batch_plan(pts, resident=2)
    assert e.value.code == bte.EINVAL


def test_batch_tune_rejects_bad_arguments_on_host():
    pts = [W.c1_fp64()]
    for kw in (dict(sample=0), dict(steps=1)):
        with pytest.raises(bte.BteError) as e:
            bte.batch_tune(pts, **kw)
        assert e.value.code == bte.EINVAL
    with pytest.raises(bte.BteError) as e:
        bte.batch_tune([W.c1_fp64().replace(m_points=2)])
    assert e.value.code == bte.EINVAL
