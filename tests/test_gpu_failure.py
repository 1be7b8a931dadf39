"""Failure detection of the bounded in-kernel waits, exercised without a GPU
fault.

Every wait of the library's kernels on an mbarrier is bounded by the GPU's
%globaltimer; a wait that gives up records an error word that the host
reports as BTE_ETIMEOUT.  bte_wait_probe runs one such wait on an mbarrier
that nothing completes (no copy in flight, no other thread), with a short
limit, so the timeout path runs end to end: kernel -> error word ->
bte_observables status, and the handle and context stay usable after it.
"""
import math

import pytest

from paper_1401_6047_gb300 import bte
from paper_1401_6047_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _params(prec):
    return W.Params(E_dc=1.1, E_omega=0.4, omega=2.5, B=1.2, mu=1.3, n_max=14, m_points=161,
                    phiy_min=-7.0, phiy_max=7.0, dt=5e-3, periods=1.0, avg_window=1.0,
                    precision=prec)


@pytest.mark.parametrize("prec", [W.FP64, W.FP32_MIXED])
def test_timed_out_wait_is_reported_and_cleared_by_reset(prec):
    p = _params(prec)
    with bte.Solver(p) as s:
        s.run()
        good = s.observables()
        assert good.status == bte.OK
        s.wait_probe(50_000)  # 50 us: the wait runs out
        with pytest.raises(bte.BteError) as e:
            s.observables()
        assert e.value.code == bte.ETIMEOUT
        assert s.observables(check=False).status == bte.ETIMEOUT
        # the context and the handle still work; reset clears the error word
        s.reset()
        s.run()
        again = s.observables()
    assert again.status == bte.OK
    assert again.absorption == good.absorption and again.v_dc_avg == good.v_dc_avg
    assert not math.isnan(again.absorption)


def test_wait_probe_rejects_limits_out_of_range():
    with bte.Solver(_params(W.FP64)) as s:
        for bad in (0, -5, 2_000_000_001):
            with pytest.raises(bte.BteError) as e:
                s.wait_probe(bad)
            assert e.value.code == bte.EINVAL
        assert s.observables(check=False).status == bte.OK
