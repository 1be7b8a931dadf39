"""CPU-side checks of the surrogate ABI: the library's run protocol for a
surrogate point equals the workload definition, and bad configurations are
rejected before any CUDA call."""
import math

import numpy as np
import pytest

from paper_1401_6047_gb300 import bte
from paper_1401_6047_gb300 import surrogate as S
from paper_1401_6047_gb300 import workloads as W


def test_protocol_matches_workload_definition():
    X = W.sweep_matrix(2000, 99)
    X[0] = [0.0, 0.01, 0.5, 0.0, 0.5]   # box corners
    X[1] = [6.0, 1.0, 6.0, 6.0, 10.0]
    for x in X:
        c = S.protocol(x)
        p = W.surrogate_params(x)
        for k in ("E_dc", "E_omega", "omega", "B", "mu", "alpha", "phiy_min", "phiy_max", "dt",
                  "periods", "t_max", "avg_window", "n_max", "m_points", "precision"):
            assert getattr(c, k) == getattr(p, k), k
        assert c.reserved == 0


def test_protocol_run_length_reaches_the_steady_state():
    """At least 16 time units before a one-period window."""
    for x in W.sweep_matrix(200, 5):
        p = W.surrogate_params(x)
        dt, P, K, Kw = bte.time_grid(p)
        assert Kw == P
        assert (K - Kw) * dt >= 16.0 - 1e-9


@pytest.mark.parametrize("bad", ["omega", "mu", "nan"])
def test_protocol_rejects_bad_points(bad):
    x = np.array([1.0, 0.5, 2.0, 1.0, 2.0])
    if bad == "omega":
        x[2] = 0.0
    elif bad == "mu":
        x[4] = -1.0
    else:
        x[0] = math.nan
    with pytest.raises(bte.BteError) as e:
        S.protocol(x)
    assert e.value.code == bte.EINVAL


@pytest.mark.parametrize("bad", [dict(members=65), dict(width=128), dict(batch_capacity=100),
                                 dict(y_std=(0.0, 1.0)), dict(x_hi=(0, 0, 0, 0, 0))])
def test_bad_configuration_rejected_on_host(bad):
    kw = dict(y_mean=(0.0, 0.0), y_std=(1.0, 1.0))
    members = bad.pop("members", 8)
    cap = bad.pop("batch_capacity", 16384)
    kw.update(bad)
    width = kw.pop("width", 256)
    cfg = S.bte_sur_config()
    lo, hi = S.box_bounds()
    cfg.members, cfg.width, cfg.batch_capacity, cfg.reserved = members, width, cap, 0
    cfg.x_lo[:] = list(lo)
    cfg.x_hi[:] = list(kw.get("x_hi", hi))
    cfg.y_mean[:] = list(kw["y_mean"])
    cfg.y_std[:] = list(kw["y_std"])
    import ctypes
    h = ctypes.c_void_p()
    rc = S._lib().bte_sur_create(ctypes.byref(cfg), ctypes.byref(h))
    assert rc == bte.EINVAL and not h.value


def test_init_params_layout():
    p = S.init_params(3, seed=4)
    assert p.shape == (3, 133_634) and p.dtype == np.float32
    # biases are zero, weights bounded by sqrt(3 / fan_in)
    b1 = p[:, 1280:1536]
    assert np.all(b1 == 0)
    W2 = p[:, 1536:1536 + 65536]
    assert np.max(np.abs(W2)) <= math.sqrt(3 / 256) + 1e-7
    assert not np.array_equal(p[0], p[1])
