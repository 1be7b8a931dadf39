"""The distribution itself (bte_pdf): the GPU's Fourier sum of the device
state equals the same sum taken on the host from bte_get_state, its
integrals are the norm and the drift velocity, and it agrees pointwise with
backward characteristics from the closed-form equilibrium."""
import math

import numpy as np
import pytest

from paper_1401_6047_gb300 import bte
from paper_1401_6047_gb300 import image
from paper_1401_6047_gb300 import workloads as W
from tests import analytic as an

pytestmark = pytest.mark.gpu


def _host_pdf(a, b, nphix):
    x = -math.pi + 2 * math.pi * np.arange(nphix) / nphix
    n = np.arange(a.shape[0])
    return np.cos(np.outer(x, n)) @ a + np.sin(np.outer(x, n)) @ b


@pytest.mark.parametrize("prec", [W.FP64, W.FP32_MIXED])
def test_pdf_equals_host_sum_and_integrates_to_observables(prec):
    p = W.Params(E_dc=1.0, E_omega=0.5, omega=2.0, B=1.0, mu=3.0, alpha=0.9496, n_max=24,
                 m_points=321, phiy_min=-8, phiy_max=8, dt=2e-3, periods=2.0, avg_window=1.0,
                 precision=prec)
    with bte.Solver(p) as s:
        s.step(300)
        for grid in (0, 1):
            f = s.pdf(grid, 96)
            a, b = s.get_state(grid)
            ref = _host_pdf(a, b, 96)
            assert np.max(np.abs(f - ref)) <= 1e-12 * np.max(np.abs(ref))
        o = s.observables(check=False)
        f = s.pdf(0, 64)
    dphi = (p.phiy_max - p.phiy_min) / (p.m_points - 1)
    dx = 2 * math.pi / 64
    x = -math.pi + dx * np.arange(64)
    # the trapezoid rule in phi_x is exact for trigonometric polynomials of degree < 64
    norm = math.sqrt(p.alpha) * dx * dphi * f.sum()
    v = math.sqrt(p.alpha) * dx * dphi * (np.sin(x)[:, None] * f).sum()
    assert abs(norm - o.norm) <= 1e-12
    assert abs(v - o.v_dr) <= 1e-12


def test_pdf_pointwise_against_characteristics():
    """t ~ 1 from the equilibrium, B != 0 and a time-dependent drive: the GPU
    distribution on the 641-point grid within 5e-5 of its maximum of
    backward characteristics at 16 random points (the error is O(dphi^2))."""
    p = W.Params(E_dc=1.0, E_omega=0.5, omega=2.0, B=1.0, mu=3.0, alpha=0.9496, n_max=24,
                 m_points=641, phiy_min=-8, phiy_max=8, dt=2e-3, periods=1.0, avg_window=1.0,
                 precision=W.FP64)
    dt, P, K, Kw = bte.time_grid(p)
    k = int(round(1.0 / dt))
    nphix = 48
    with bte.Solver(p) as s:
        s.step(k)
        f = s.pdf(0, nphix)
    rng = np.random.default_rng(5)
    i = rng.integers(0, nphix, 16)
    m = rng.integers(160, 480, 16)
    x = -math.pi + 2 * math.pi * i / nphix
    y = p.phiy_min + m * (p.phiy_max - p.phiy_min) / (p.m_points - 1)
    ref = an.characteristics_pdf(1.0, 0.5, 2.0, 1.0, 3.0, k * dt, x, y, alpha=0.9496)
    assert np.max(np.abs(f[i, m] - ref)) <= 5e-5 * np.max(np.abs(f))


def test_pdf_dump_is_a_readable_image(tmp_path):
    p = W.c1_fp64().replace(periods=0.2, avg_window=0.1)
    with bte.Solver(p) as s:
        s.step(10)  # t = 0.01: the peak has moved by E t = 0.01 rad, a third of a pixel
        f = s.pdf(0, 200)
    path = tmp_path / "f.pgm"
    image.write_pgm(str(path), f)
    img = image.read_pgm(str(path))
    assert img.shape == (p.m_points, 200)
    assert img.max() == 255 and img.min() == 0
    # the peak of f0-like state sits at phi_x ~ 0, phi_y ~ 0 (image centre)
    r, c = np.unravel_index(np.argmax(img), img.shape)
    assert abs(r - p.m_points // 2) <= 2 and abs(c - 100) <= 2


def test_pdf_rejects_bad_arguments():
    p = W.c1_fp64()
    with bte.Solver(p) as s:
        for grid, n in ((2, 10), (0, 0), (0, 70000)):
            with pytest.raises(bte.BteError) as e:
                s.pdf(grid, n)
            assert e.value.code == bte.EINVAL
