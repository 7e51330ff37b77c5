"""Oscillatory decay of short concentration waves (Sec. IV, the critical wave
number above which the concentration pair of modes turns complex): on the
lattice the slowest concentration eigenvalue of the one-step operator L(q)
is real for long waves and complex for short ones at low packing, and the
oracle's concentration amplitude then changes sign as the wave decays,
exactly as L(q) predicts; at higher packing the same wave decays
monotonically."""
import math

import numpy as np
import pytest

import linear_model as LM
from paper_1105_3634_gb300 import workloads as W
from test_gpu_physics import concentration_mode


def _lattice(L):
    return W.Lattice(shape=(L, 2, 2), sigma=[1.0, 1.5], tau=1.0)


def _concentration_series(orc, lat, n0, amp, steps):
    """w(t) = n0_B dn_A(q) - n0_A dn_B(q), q = 2 pi / L_x, for a cos wave of
    relative amplitude +amp / -amp, from the oracle and from L(q)."""
    L = lat.shape[0]
    q = np.array([2 * math.pi / L, 0.0, 0.0])
    x = W.coordinate(lat, 0)
    cosf = np.cos(q[0] * x)
    n = np.stack([n0[0] * (1 + amp * cosf), n0[1] * (1 - amp * cosf)])
    f = orc.init(lat, n)
    Lm, Dn, _ = LM.operator(lat, n0, q)
    s = LM.initial_state(lat, n0, 0.5 * n0 * np.array([amp, -amp]), np.zeros((2, 3)))
    ph = np.exp(-1j * q[0] * x) / lat.nsites
    w_orc, w_lin = [], []
    for _ in range(steps):
        nn, _ = orc.moments(lat, f)
        a = (nn - n0[:, None]) @ ph
        w_orc.append((n0[1] * a[0] - n0[0] * a[1]).real)
        b = Dn @ s
        w_lin.append((n0[1] * b[0] - n0[0] * b[1]).real)
        orc.step(lat, f, 1)
        s = Lm @ s
    return np.array(w_orc), np.array(w_lin)


def test_concentration_eigenvalue_turns_complex_for_short_waves_at_low_packing():
    low = W.densities_from_packing(0.05, [1.0, 1.5], [0.5, 0.5])
    high = W.densities_from_packing(0.2, [1.0, 1.5], [0.5, 0.5])
    lam64, _ = concentration_mode(_lattice(64), low, 2 * math.pi / 64)
    lam8, _ = concentration_mode(_lattice(8), low, 2 * math.pi / 8)
    lam8h, _ = concentration_mode(_lattice(8), high, 2 * math.pi / 8)
    assert abs(lam64.imag) < 1e-12 and abs(lam8h.imag) < 1e-12
    assert abs(np.angle(lam8)) > 0.3                       # about a quarter turn per 4 steps


def test_oracle_concentration_amplitude_changes_sign(orc):
    lat = _lattice(8)
    n0 = W.densities_from_packing(0.05, lat.sigma, [0.5, 0.5])
    w_orc, w_lin = _concentration_series(orc, lat, n0, 1e-6, 30)
    scale = abs(w_orc[0])
    assert np.abs(w_orc - w_lin).max() < 1e-7 * scale
    flips = np.count_nonzero(np.diff(np.sign(w_orc)) != 0)
    assert flips >= 3
    assert np.array_equal(np.sign(w_orc), np.sign(w_lin))


def test_denser_mixture_decays_monotonically(orc):
    lat = _lattice(8)
    n0 = W.densities_from_packing(0.2, lat.sigma, [0.5, 0.5])
    w_orc, _ = _concentration_series(orc, lat, n0, 1e-6, 30)
    assert np.all(w_orc > 0) and np.all(np.diff(w_orc) < 0)
