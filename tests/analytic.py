"""Closed forms and independent integrators used to pin the oracle.

Nothing here shares arithmetic with the oracle or the CUDA library.  Each
function is derived from the continuum equation of the paper (Sec. 2,
Eq. boltzmann_final) by a route other than the finite-difference scheme.
"""
from __future__ import annotations

import numpy as np
import scipy.special as sp


def xi(x):
    """Esaki-Tsu shape x/(1+x^2) (Sec. 4, Eq. xi_def)."""
    return x / (1.0 + x * x)


def bessel_ratio(mu: float, n: int | np.ndarray):
    """I_n(mu)/I_0(mu) from scipy's exponentially scaled I_n."""
    return sp.ive(n, mu) / sp.ive(0, mu)


def esaki_tsu(E: float, mu: float) -> float:
    """Stationary drift velocity at B = 0 and constant E:
    v = (I_1/I_0) E/(1+E^2).  At B = 0 each harmonic obeys
    da/dt = a0 - a - nE b, db/dt = -b + nE a, whose fixed point for n = 1
    integrated over phi_y gives this."""
    return float(bessel_ratio(mu, 1) * xi(E))


def tucker_absorption(E_dc: float, E_omega: float, omega: float, nterms: int = 80) -> float:
    """Absorption A = <2 I_0 v cos(omega t)/I_1> at B = 0 (Eq. absorption_def).

    Solving the n = 1 harmonic equation at B = 0 with the Jacobi-Anger
    expansion of exp(i (E_omega/omega) sin(omega t)) gives
        A = sum_k J_k(a) [J_{k+1}(a) + J_{k-1}(a)] xi(E_dc + k omega),
    a = E_omega/omega.  (The printed Eq. absorption_tacker carries an extra
    factor 2 I_1/I_0 that is inconsistent with Eq. absorption_def; the
    definition is followed here.)"""
    a = E_omega / omega
    k = np.arange(-nterms, nterms + 1)
    return float(np.sum(sp.jv(k, a) * (sp.jv(k + 1, a) + sp.jv(k - 1, a)) *
                        xi(E_dc + k * omega)))


def tucker_vdc(E_dc: float, E_omega: float, omega: float, mu: float, nterms: int = 80) -> float:
    """Time-averaged drift velocity at B = 0: (I_1/I_0) sum_k J_k(a)^2 xi(E_dc + k omega)."""
    a = E_omega / omega
    k = np.arange(-nterms, nterms + 1)
    return float(bessel_ratio(mu, 1) * np.sum(sp.jv(k, a) ** 2 * xi(E_dc + k * omega)))


def ktitorov_absorption(E_dc: float, E_omega: float, omega: float) -> float:
    """Small-signal limit of the Tucker form: A ~ (a/2)[xi(E_dc+omega) - xi(E_dc-omega)]
    to first order in a = E_omega/omega."""
    a = E_omega / omega
    return 0.5 * a * (xi(E_dc + omega) - xi(E_dc - omega))


def characteristics_vdc(E: float, B: float, mu: float, nx: int = 128, ny: int = 200,
                        ds: float = 0.01, smax: float = 25.0, ysig: float = 7.0) -> float:
    """Stationary drift velocity for constant E and B by the method of
    characteristics (Sec. 4, Eqs. pendulum_phi_x, pendulum_phi_y and
    pendulum_drift_velocity, extended to finite temperature).

    The streaming field (E + B phi_y, -B sin phi_x) is divergence free, so the
    relaxation-time equation is solved exactly by
        v = int_0^inf e^{-s} < sin Phi_x(s; phi0) >_{f0} ds,
    Phi(s; phi0) the pendulum trajectory started at phi0 drawn from f0
    (von Mises(mu) in phi_x, normal with variance 1/mu in phi_y).
    Midpoint quadrature over phi0, RK4 in s, Simpson in s."""
    x = 2 * np.pi * (np.arange(nx) + 0.5) / nx - np.pi
    wx = np.exp(mu * (np.cos(x) - 1.0))
    wx /= wx.sum()
    L = ysig / np.sqrt(mu)
    y = -L + 2 * L * (np.arange(ny) + 0.5) / ny
    wy = np.exp(-mu * y * y / 2.0)
    wy /= wy.sum()
    px, py = np.meshgrid(x, y, indexing="ij")
    w = np.outer(wx, wy)

    def f(px, py):
        return E + B * py, -B * np.sin(px)

    ns = int(round(smax / ds))
    ns += ns % 2
    vals = np.empty(ns + 1)
    vals[0] = np.sum(w * np.sin(px))
    for i in range(ns):
        k1 = f(px, py)
        k2 = f(px + 0.5 * ds * k1[0], py + 0.5 * ds * k1[1])
        k3 = f(px + 0.5 * ds * k2[0], py + 0.5 * ds * k2[1])
        k4 = f(px + ds * k3[0], py + ds * k3[1])
        px = px + ds / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
        py = py + ds / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
        vals[i + 1] = np.sum(w * np.sin(px))
    g = np.exp(-ds * np.arange(ns + 1)) * vals
    return float(ds / 3 * (g[0] + g[-1] + 4 * g[1:-1:2].sum() + 2 * g[2:-1:2].sum()))


def f0_fourier(mu: float, alpha: float, nmax: int, phiy: np.ndarray, nx: int = 1024) -> np.ndarray:
    """Fourier cosine coefficients a0_n(phi_y) of the closed-form equilibrium
    f0 = exp(mu cos phi_x - mu phi_y^2/2) sqrt(mu/(2 pi alpha)) / (2 pi I_0(mu))
    (Eq. Bolzmann_initial_pdf), by FFT of f0 sampled in phi_x: the series
    f0 = sum_n a0_n cos(n phi_x) of Eq. f0_fourier."""
    x = 2 * np.pi * np.arange(nx) / nx
    # exp(mu cos x)/I_0(mu) = exp(mu (cos x - 1)) / ive(0, mu)
    fx = np.exp(mu * (np.cos(x) - 1.0)) / sp.ive(0, mu)
    c = np.fft.rfft(fx).real / nx       # c_k with fx = c_0 + 2 sum_k c_k cos(kx)
    coef = np.concatenate([[c[0]], 2 * c[1:nmax + 1]])
    gy = np.sqrt(mu / (2 * np.pi * alpha)) * np.exp(-mu * phiy ** 2 / 2) / (2 * np.pi)
    return np.outer(coef, gy)


def characteristics_ac(E_dc: float, E_omega: float, omega: float, B: float, mu: float,
                       nphase: int = 12, nx: int = 64, ny: int = 96, ds: float = 0.01,
                       smax: float = 25.0, ysig: float = 7.0, B_omega: float = 0.0,
                       B_phase: float = 0.0, xsig: float = 0.0):
    """Periodic-state absorption and time-averaged drift velocity for the
    drive E(t) = E_dc + E_omega cos(omega t) and the field
    B(t) = B + B_omega cos(omega t + B_phase) (constant for B_omega = 0), by
    the method of characteristics (the exact solution of the relaxation-time
    equation for the streaming field (E(t) + B(t) phi_y, -B(t) sin phi_x),
    divergence free at every t):
        v(t) = int_0^inf e^{-u} < sin Phi_x(t; t - u, phi0) >_{f0} du.
    With tau = t - u and the period T = 2 pi/omega, the time averages become
    averages over start phases tau in [0, T):
        <v cos(omega t)> = (1/T) int_0^T dtau int_0^inf du e^{-u} cos(omega (tau + u)) G(tau, u)
        <v>              = (1/T) int_0^T dtau int_0^inf du e^{-u} G(tau, u),
    G(tau, u) = < sin Phi_x(tau + u; tau, phi0) >_{f0}.  Midpoint rule in tau
    (periodic integrand), midpoint quadrature over phi0 (von Mises(mu) x
    normal(0, 1/mu)), RK4 in u, Simpson in u.  At low temperature (large
    mu) the start points can be confined to |phi_x| < xsig/sqrt(mu) (xsig > 0),
    where the von Mises weight is not negligible.  Returns (A, v_dc) with
    A = (2 I_0/I_1) <v cos(omega t)> (Eq. absorption_def)."""
    T = 2 * np.pi / omega
    tau = T * (np.arange(nphase) + 0.5) / nphase
    if xsig > 0:
        Lx = min(np.pi, xsig / np.sqrt(mu))
        x = -Lx + 2 * Lx * (np.arange(nx) + 0.5) / nx
    else:
        x = 2 * np.pi * (np.arange(nx) + 0.5) / nx - np.pi
    wx = np.exp(mu * (np.cos(x) - 1.0))
    wx /= wx.sum()
    L = ysig / np.sqrt(mu)
    y = -L + 2 * L * (np.arange(ny) + 0.5) / ny
    wy = np.exp(-mu * y * y / 2.0)
    wy /= wy.sum()
    w = np.outer(wx, wy)[None, :, :] / nphase
    px = np.broadcast_to(x[None, :, None], (nphase, nx, ny)).copy()
    py = np.broadcast_to(y[None, None, :], (nphase, nx, ny)).copy()
    t0 = tau[:, None, None]

    def f(px, py, u):
        Bt = B + B_omega * np.cos(omega * (t0 + u) + B_phase)
        return E_dc + E_omega * np.cos(omega * (t0 + u)) + Bt * py, -Bt * np.sin(px)

    ns = int(round(smax / ds))
    ns += ns % 2
    G = np.empty((ns + 1, nphase))
    G[0] = np.sum(w * np.sin(px), axis=(1, 2))
    for i in range(ns):
        u = i * ds
        k1 = f(px, py, u)
        k2 = f(px + 0.5 * ds * k1[0], py + 0.5 * ds * k1[1], u + 0.5 * ds)
        k3 = f(px + 0.5 * ds * k2[0], py + 0.5 * ds * k2[1], u + 0.5 * ds)
        k4 = f(px + ds * k3[0], py + ds * k3[1], u + ds)
        px = px + ds / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
        py = py + ds / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
        G[i + 1] = np.sum(w * np.sin(px), axis=(1, 2))
    u = ds * np.arange(ns + 1)
    simpson = np.full(ns + 1, 2.0)
    simpson[1::2] = 4.0
    simpson[0] = simpson[-1] = 1.0
    simpson *= ds / 3
    decay = np.exp(-u)[:, None]
    vc = np.sum(simpson[:, None] * decay * np.cos(omega * (tau[None, :] + u[:, None])) * G)
    vb = np.sum(simpson[:, None] * decay * G)
    return float(2.0 / bessel_ratio(mu, 1) * vc), float(vb)


def f0_closed(phix, phiy, mu: float, alpha: float = 1.0):
    """The equilibrium distribution (Eq. Bolzmann_initial_pdf):
    f0 = sqrt(mu / (2 pi alpha)) exp(mu cos phi_x - mu phi_y^2 / 2) / (2 pi I_0(mu)),
    written with exp(mu (cos - 1)) / ive(0, mu) to stay finite."""
    return (np.sqrt(mu / (2 * np.pi * alpha)) * np.exp(mu * (np.cos(phix) - 1.0) - mu * phiy ** 2 / 2)
            / (2 * np.pi * sp.ive(0, mu)))


def characteristics_pdf(E_dc: float, E_omega: float, omega: float, B: float, mu: float,
                        t: float, phix, phiy, alpha: float = 1.0, ds: float = 1e-3):
    """The distribution f(phi_x, phi_y, t) of the relaxation-time equation
    started from f0 at t = 0, by backward characteristics: with Phi(t'; t,
    phi) the trajectory of the streaming field (E(t') + B phi_y, -B sin
    phi_x) through phi at time t,
        f(phi, t) = e^{-t} f0(Phi(0)) + int_0^t e^{-s} f0(Phi(t - s)) ds.
    RK4 backward in time, Simpson in s (t / ds even)."""
    px = np.array(phix, dtype=np.float64)
    py = np.array(phiy, dtype=np.float64)
    ns = int(round(t / ds))
    ns += ns % 2
    ds = t / ns

    def f(px, py, tt):  # d phi / d t' (the backward step uses -ds)
        return E_dc + E_omega * np.cos(omega * tt) + B * py, -B * np.sin(px)

    vals = [f0_closed(px, py, mu, alpha)]
    tt = t
    for i in range(ns):
        h = -ds
        k1 = f(px, py, tt)
        k2 = f(px + 0.5 * h * k1[0], py + 0.5 * h * k1[1], tt + 0.5 * h)
        k3 = f(px + 0.5 * h * k2[0], py + 0.5 * h * k2[1], tt + 0.5 * h)
        k4 = f(px + h * k3[0], py + h * k3[1], tt + h)
        px = px + h / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
        py = py + h / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
        tt += h
        vals.append(f0_closed(px, py, mu, alpha))
    vals = np.array(vals)  # vals[i]: f0 at Phi(t - i ds)
    s = ds * np.arange(ns + 1)
    wts = np.full(ns + 1, 2.0)
    wts[1::2] = 4.0
    wts[0] = wts[-1] = 1.0
    integral = ds / 3 * np.tensordot(wts * np.exp(-s), vals, axes=1)
    return np.exp(-t) * vals[-1] + integral
