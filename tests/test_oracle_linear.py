"""Pin of the oracle's full time step in the linear regime.

A small plane-wave perturbation of a uniform mixture is advanced by the
oracle and by the independently written linear operator L(q)
(tests/linear_model.py); the Fourier amplitude of every species' density
and momentum must agree.  This pins moments, contact values, the smoothing
ball, all three force terms, the collision and the streaming direction.
"""
import math

import numpy as np
import pytest

import linear_model as LM
from paper_1105_3634_gb300 import workloads as W


def _coords(lat):
    nx, ny, nz = lat.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], 1).astype(float)


def _run_case(orc, lat, n0, q, dn_rel, du, steps):
    S = lat.nspecies
    N = lat.nsites
    r = _coords(lat)
    phase = r @ q
    cosf = np.cos(phase)
    n = n0[:, None] * (1 + np.asarray(dn_rel)[:, None] * cosf[None, :])
    u = np.asarray(du)[:, :, None] * cosf[None, None, :]
    f = orc.init(lat, n, u)
    L, Dn, Dj = LM.operator(lat, n0, q)
    # e^{i q r} amplitude of A cos(q r) is A/2
    x = LM.initial_state(lat, n0, 0.5 * n0 * np.asarray(dn_rel), 0.5 * np.asarray(du))
    ph = np.exp(-1j * phase) / N
    t = 0
    worst = 0.0
    scale = np.abs(n0 * np.asarray(dn_rel)).max() + np.abs(n0[:, None] * du).max()
    for target in steps:
        orc.step(lat, f, target - t)
        for _ in range(target - t):
            x = L @ x
        t = target
        nn, jj = orc.moments(lat, f)
        an = (nn - n0[:, None]) @ ph
        aj = jj @ ph
        worst = max(worst, np.abs(an - Dn @ x).max() / scale, np.abs(aj - Dj @ x).max() / scale)
    return worst, x


def test_linear_config1_wave_along_x(orc):
    lat = W.Lattice(shape=(32, 2, 3), sigma=[1.0, 1.5], tau=1.0)
    n0 = W.densities_from_packing(0.2, lat.sigma, [0.5, 0.5])
    q = np.array([2 * math.pi / 32, 0, 0])
    worst, _ = _run_case(orc, lat, n0, q, [1e-6, -1e-6], np.zeros((2, 3)), [1, 10, 80])
    assert worst < 1e-7


def test_linear_attraction_oblique_wave(orc):
    lat, _ = W.binary_attraction((12, 12, 2))
    lat.tau = 0.8
    n0 = W.densities_from_packing(0.3, lat.sigma, [0.5, 0.5])
    q = np.array([2 * math.pi / 12, 2 * math.pi / 12, 0])
    worst, _ = _run_case(orc, lat, n0, q, [1e-6, -0.5e-6], np.zeros((2, 3)), [1, 7, 40])
    assert worst < 1e-7


def test_linear_shear_wave_three_species_drag_only(orc):
    lat = W.Lattice(shape=(2, 3, 16), sigma=[1.0, 1.5, 2.0], tau=1.3, drag_only=True)
    n0 = W.densities_from_packing(0.25, lat.sigma, [0.3, 0.3, 0.4])
    q = np.array([0, 0, 2 * math.pi / 16])
    du = np.array([[1e-6, 0, 0], [-2e-6, 1e-6, 0], [0, 0, 1e-6]])
    worst, _ = _run_case(orc, lat, n0, q, [0.5e-6, 1e-6, -1e-6], du, [1, 9, 50])
    assert worst < 1e-7


def test_linear_shear_and_sound_three_species_with_attraction(orc):
    lat = W.Lattice(shape=(10, 2, 2), sigma=[1.0, 2.0, 1.5], tau=0.7,
                    eps=[[0.1, 0.05, 0.08], [0.05, 0.2, 0.1], [0.08, 0.1, 0.15]],
                    lambda_c=[[2.5, 2.0, 2.2], [2.0, 2.5, 2.1], [2.2, 2.1, 2.0]])
    n0 = W.densities_from_packing(0.2, lat.sigma, [0.5, 0.2, 0.3])
    q = np.array([2 * math.pi / 10, 0, 0])
    du = np.array([[1e-6, 1e-6, 0], [0, -1e-6, 1e-6], [-1e-6, 0, 0]])
    worst, _ = _run_case(orc, lat, n0, q, [1e-6, -1e-6, 0.5e-6], du, [1, 6, 30])
    assert worst < 1e-7


def test_linear_forward_euler_scheme_low_packing(orc):
    """The forward-Euler forcing (flag) on a state where it is stable."""
    lat = W.Lattice(shape=(24, 2, 2), sigma=[2.0, 2.5], tau=1.0, force_scheme="explicit")
    n0 = W.densities_from_packing(0.15, lat.sigma, [0.5, 0.5])
    q = np.array([2 * math.pi / 24, 0, 0])
    du = np.array([[0, 1e-6, 0], [0, 0, -1e-6]])
    worst, _ = _run_case(orc, lat, n0, q, [1e-6, -1e-6], du, [1, 10, 60])
    assert worst < 1e-7


def test_forward_euler_is_unstable_at_config1(orc):
    """Why the semi-implicit shift is the default: with forward-Euler forcing
    the grid-scale velocity modes of sigma = (1, 1.5) at packing 0.2 and
    tau = 1 grow (the velocity-exchange rate there exceeds 2 per step)."""
    lat = W.Lattice(shape=(8, 8, 8), sigma=[1.0, 1.5], tau=1.0, force_scheme="explicit")
    n0 = W.densities_from_packing(0.2, lat.sigma, [0.5, 0.5])
    L, _, _ = LM.operator(lat, n0, np.array([math.pi, 0, 0]))
    assert np.abs(np.linalg.eigvals(L)).max() > 1.5
    lat.force_scheme = "semi_implicit"
    worst = 0.0
    for k in range(5):
        for l in range(k + 1):
            for m in range(l + 1):
                L, _, _ = LM.operator(lat, n0, 2 * math.pi * np.array([k, l, m]) / 8)
                worst = max(worst, np.abs(np.linalg.eigvals(L)).max())
    assert worst < 1 + 1e-9


def test_linear_three_predictor_sweeps(orc):
    """The oracle's predictor with three Jacobi sweeps (the partners' u* of the
    previous sweep) against L(q) with the same sweeps."""
    lat = W.Lattice(shape=(16, 3, 2), sigma=[1.0, 1.5], tau=1.0, predictor_sweeps=3)
    n0 = W.densities_from_packing(0.2, lat.sigma, [0.5, 0.5])
    q = np.array([2 * math.pi / 16, 2 * math.pi / 3, 0])
    worst, _ = _run_case(orc, lat, n0, q, [1e-6, -2e-6], np.array([[1e-6, 0, 0], [0, -1e-6, 0]]), [1, 7, 40])
    assert worst < 1e-7


def test_three_sweeps_keep_a_denser_mixture_stable(orc):
    """Packing 0.3, sigma 1/1.5, 1 % noise: one predictor sweep blows up,
    three sweeps stay bounded (the linearised step's growth factors)."""
    def run(sweeps, steps):
        lat = W.Lattice(shape=(12, 6, 5), sigma=[1.0, 1.5], tau=1.0, predictor_sweeps=sweeps)
        n0 = W.densities_from_packing(0.3, lat.sigma, [0.5, 0.5])
        f = orc.init(lat, W.noise(lat, n0, 0.01, seed=17))
        status = orc.step(lat, f, steps)
        n, _ = orc.moments(lat, f)
        ok = status == 0 and np.isfinite(n).all()
        return ok, (float(np.abs(n - n0[:, None]).max() / n0.max()) if ok else np.inf)
    ok1, dev1 = run(1, 120)
    ok3, dev3 = run(3, 300)
    assert not ok1 or dev1 > 1.0
    assert ok3 and dev3 < 0.05
