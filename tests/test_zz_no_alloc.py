"""The allocation-free observables entry point against the handle-based one.

bte_observe_noalloc is for callers that cannot allocate device memory (their
device memory all belongs to their own pool allocator, or their host path
cannot afford an allocation's synchronisation).  It reduces caller-owned
device rows with partial sums kept in a fixed library array.  This test runs
a solver through the normal entry points, hands rows 0 (a) and 1 (b) of its
whole grid to bte_observe_noalloc twice in a row, and compares the drift
velocity and norm with the solver's own trace at that step and with the FP64
oracle's reduction of the same rows.  It lives in a file of its own,
collected last.
"""
import numpy as np
import pytest

import oracle
from paper_1401_6047_gb300 import bte
from paper_1401_6047_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [W.FP64, W.FP32_MIXED])
def test_observe_noalloc_matches_solver_trace(prec):
    torch = pytest.importorskip("torch")
    p = W.Params(E_dc=1.3, E_omega=0.7, omega=1.9, B=2.4, mu=1.6, n_max=24, m_points=3001,
                 phiy_min=-9.0, phiy_max=9.0, dt=4e-3, periods=2.0, avg_window=1.0, precision=prec)
    with bte.Solver(p) as s:
        s.step(211)
        v_ref, n_ref = s.trace(211, 1)
        a, b = s.get_state(0)
    dt = torch.float64 if prec == W.FP64 else torch.float32
    a0 = torch.tensor(a[0], dtype=dt, device="cuda")   # FP32 state widens exactly
    b1 = torch.tensor(b[1], dtype=dt, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    v_or, n_or = oracle.observe(p, a, b)  # the same rows, reduced on the CPU in FP64
    tol = 1e-12
    for _ in range(2):  # two calls in a row share the fixed scratch array
        out.zero_()
        bte.observe_noalloc(p, a0.data_ptr(), b1.data_ptr(), out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        v, nr = out.tolist()
        assert abs(v - v_ref[0]) <= tol * max(1.0, abs(v_ref[0])), (v, v_ref[0])
        assert abs(nr - n_ref[0]) <= tol * max(1.0, abs(n_ref[0])), (nr, n_ref[0])
        assert abs(v - v_or) <= tol * max(1.0, abs(v_or)), (v, v_or)
        assert abs(nr - n_or) <= tol * max(1.0, abs(n_or)), (nr, n_or)


def test_observe_noalloc_rejects_oversize():
    pytest.importorskip("torch")
    import torch
    p = W.Params(m_points=1_048_577, n_max=2)
    buf = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(bte.BteError) as e:
        bte.observe_noalloc(p, buf.data_ptr(), buf.data_ptr(), buf.data_ptr())
    assert e.value.code == bte.EINVAL
