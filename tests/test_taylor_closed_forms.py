"""The Taylor-dispersion analysis against what fixes it independently: the
paper's Eq. taylordiff at second order in U, and a direct time integration of
the passive-scalar advection-diffusion equation in the cosine flow."""
import math

import numpy as np

from paper_1105_3634_gb300 import taylor as T


def test_no_flow_is_plain_diffusion():
    assert abs(T.passive_scalar_rate(0.3, 0.0, 0.05, 0.2) - 0.3) < 1e-12


def test_second_order_is_eq_taylordiff_for_any_kx():
    D, ky, Ly = 0.3, 2 * math.pi / 32, 32.0
    for kx in (2 * math.pi / 512, 2 * math.pi / 128, 2 * math.pi / 40):
        for U in (1e-3, 2e-3):
            exact = T.passive_scalar_rate(D, U, kx, ky)
            second = T.taylor_formula(D, U, Ly)
            assert abs(exact - second) < 1e-6 * D, (kx, U, exact, second)
    # the next order is O(U^4): halving U divides the remainder by ~16
    kx = 2 * math.pi / 128
    r1 = T.passive_scalar_rate(D, 0.08, kx, ky) - T.taylor_formula(D, 0.08, Ly)
    r2 = T.passive_scalar_rate(D, 0.04, kx, ky) - T.taylor_formula(D, 0.04, Ly)
    assert 14.0 < r1 / r2 < 18.0


def test_peclet_form():
    D, U, Ly = 0.25, 0.05, 32.0
    Pe = T.peclet(D, U, Ly)
    assert abs(T.taylor_formula(D, U, Ly) - D * (1 + Pe * Pe / (2 * math.pi ** 2))) < 1e-14


def test_eigenvalue_equals_time_integration():
    """c(x, y, t) = Re[a(y, t) e^{i kx x}]: a_t = -i kx U cos(ky y) a + D (a_yy - kx^2 a)
    on 64 points in y (advection pointwise on the grid, a_yy by FFT), RK4;
    the late decay rate of the y-mean of a equals the slowest eigenvalue."""
    D, U, Ly, Lx = 0.3, 0.06, 32.0, 128.0
    kx, ky = 2 * math.pi / Lx, 2 * math.pi / Ly
    M = 64
    y = np.arange(M) * Ly / M
    kk = 2 * math.pi * np.fft.fftfreq(M, d=Ly / M)
    adv = -1j * kx * U * np.cos(ky * y)

    def rhs(a):
        return adv * a + D * (np.fft.ifft(-(kk * kk) * np.fft.fft(a)) - kx * kx * a)

    a = np.ones(M, complex)
    dt = 0.2
    ts, means = [], []
    for n in range(1, 15001):
        k1 = rhs(a)
        k2 = rhs(a + 0.5 * dt * k1)
        k3 = rhs(a + 0.5 * dt * k2)
        k4 = rhs(a + dt * k3)
        a = a + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        if n % 500 == 0 and n * dt >= 1000:
            ts.append(n * dt)
            means.append(abs(a.mean()))
    rate = -np.polyfit(ts, np.log(means), 1)[0]
    expect = T.passive_scalar_rate(D, U, kx, ky)
    assert abs(rate / (kx * kx) - expect) < 1e-5 * expect, (rate / (kx * kx), expect)


def test_channel_operator_tends_to_taylor_aris():
    """The finite-volume channel operator with the plane Couette profile: at
    small kx h its D_eff is the Taylor-Aris coefficient D + U^2 h^2 / (30 D)."""
    D, U, h = 0.25, 0.03, 64
    y = np.arange(h) + 0.5
    u = U * (2 * y / h - 1)
    Deff = T.passive_scalar_rate_channel(D, u, 2 * math.pi / (400 * h))
    assert abs(Deff - T.taylor_aris_couette(D, U, h)) < 2e-3 * Deff
    assert abs(T.passive_scalar_rate_channel(D, np.zeros(h), 0.1) - D) < 1e-12
