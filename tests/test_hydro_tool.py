"""The linear hydrodynamic analysis of Sec. IV (paper_1105_3634_gb300/hydro.py)
against the exact linearised lattice step L(q) (tests/linear_model.py, equal
to the oracle's evolution to 1e-7) and against the paper's closed forms."""
import math

import numpy as np
import pytest

import linear_model as LM
from test_physics_pins import lattice_D_long
from paper_1105_3634_gb300 import hydro as H
from paper_1105_3634_gb300 import workloads as W


def _berthelot(w_AA):
    w_BB = w_AA / 2
    w_AB = math.sqrt(w_AA * w_BB)
    return [[w_AA, w_AB], [w_AB, w_BB]]


@pytest.mark.parametrize("sigma,packing,eps", [
    ([2.0, 2.0], 0.2, None),
    ([2.0, 2.0], 0.2, _berthelot(H.KT)),              # tails, equal diameters
])
def test_D0_is_the_lattice_diffusion_equal_diameters(sigma, packing, eps):
    lam = [[2.5] * 2] * 2 if eps else None
    lat = W.Lattice(shape=(8, 8, 8), sigma=sigma, tau=1.0, eps=eps, lambda_c=lam)
    n0 = W.densities_from_packing(packing, sigma, [0.5, 0.5])
    m = H.Mixture(sigma, n0, eps=eps, lambda_c=lam)
    D = lattice_D_long(lat, n0)
    assert abs(m.D0() - D) < 1e-6 * D, (m.D0(), D)
    if eps is None:
        assert abs(m.thermodynamic_factor() - 1.0) < 1e-12


@pytest.mark.parametrize("sigma,packing,eps", [
    ([1.0, 1.5], 0.2, None),
    ([2.0, 3.0], 0.3, [[H.KT / 2] * 2] * 2),          # the attraction workload's mixture
])
def test_D0_unequal_diameters(sigma, packing, eps):
    """Unequal diameters: D_0 with the thermodynamic factor of the model's own
    forces (0.96 and 0.97 here) is the lattice's long-wavelength diffusion
    coefficient when the half step u* = u + a(u*)/2 is solved exactly (to
    1e-6; Eq. dab alone is 3.3 % and 2.0 % off).  The method's one Jacobi
    sweep, with the partner species' velocity held at u, diffuses faster by
    0.6 % and 1.1 %: the whole gap between the tool and the lattice."""
    lam = [[2.5] * 2] * 2 if eps else None
    n0 = W.densities_from_packing(packing, sigma, [0.5, 0.5])
    m = H.Mixture(sigma, n0, eps=eps, lambda_c=lam)
    D = {}
    for scheme in ("implicit_coupled", "semi_implicit"):
        lat = W.Lattice(shape=(8, 8, 8), sigma=sigma, tau=1.0, eps=eps, lambda_c=lam, force_scheme=scheme)
        D[scheme] = lattice_D_long(lat, n0)
    print(f"sigma={sigma}: D_0 {m.D0():.6f}, lattice exact half step {D['implicit_coupled']:.6f}, "
          f"one Jacobi sweep {D['semi_implicit']:.6f}, Eq. dab {m.D_AB():.6f}")
    assert abs(m.D0() - D["implicit_coupled"]) < 1e-6 * m.D0()
    assert 0.003 < (D["semi_implicit"] - m.D0()) / m.D0() < 0.015


def test_one_jacobi_sweep_is_exact_for_equal_diameters():
    n0 = W.densities_from_packing(0.2, [2.0, 2.0], [0.5, 0.5])
    Ds = [lattice_D_long(W.Lattice(shape=(8, 8, 8), sigma=[2.0, 2.0], force_scheme=s), n0)
          for s in ("implicit_coupled", "semi_implicit")]
    assert abs(Ds[0] - Ds[1]) < 1e-8 * Ds[0]


def test_force_matrix_and_friction_are_the_oracles():
    """The long-wavelength force matrix and friction of the tool equal the
    oracle's hard-core force on a small wave (to the wave's own sin(k)/k
    factor) and its exchange force on a uniform relative velocity."""
    import oracle as orc
    orc.build()
    sigma, packing, L = [1.0, 1.5], 0.2, 128
    lat = W.Lattice(shape=(L, 4, 4), sigma=sigma, tau=1.0)
    n0 = W.densities_from_packing(packing, sigma, [0.5, 0.5])
    m = H.Mixture(sigma, n0)
    M = m.jacobian() - np.diag(H.KT / np.asarray(n0))
    x = W.coordinate(lat, 0)
    k = 2 * math.pi / L
    for c in range(2):
        n = np.array([np.full(lat.nsites, v) for v in n0])
        n[c] *= 1 + 1e-4 * np.sin(k * x)
        _, hc, _, _ = orc.forces(lat, n, np.zeros((2, 3, lat.nsites)))
        for a in range(2):
            Mac = -2 * np.mean(hc[a, 0] * np.cos(k * x)) / (n0[c] * 1e-4 * math.sin(k))
            assert abs(Mac - M[a, c]) < 2e-4 * abs(M[a, c]), (a, c, Mac, M[a, c])
    n = np.array([np.full(lat.nsites, v) for v in n0])
    j = np.zeros((2, 3, lat.nsites))
    j[0, 0] = n0[0] * 1e-4
    _, _, vx, _ = orc.forces(lat, n, j)
    gamma = (-vx[0, 0, 0] + vx[1, 0, 0]) / 1e-4
    assert abs(gamma - m.gamma()) < 1e-9 * m.gamma()


def test_sound_speed_is_the_lattice_acoustic_mode():
    sigma, packing = [1.0, 1.5], 0.2
    lat = W.Lattice(shape=(8, 8, 8), sigma=sigma, tau=1.0)
    n0 = W.densities_from_packing(packing, sigma, [0.5, 0.5])
    q = np.array([2 * math.pi / 512, 0.0, 0.0])
    Lm, _, _ = LM.operator(lat, n0, q)
    ev = np.linalg.eigvals(Lm).astype(complex)
    z = np.log(ev[np.abs(ev) > 0.99])              # the hydrodynamic (weakly damped) modes
    cs = np.max(np.abs(z.imag)) / q[0]
    assert abs(cs - H.Mixture(sigma, n0).sound_speed()) < 1e-5 * cs


def test_roots_of_the_hydrodynamic_matrix():
    """The 4 x 4 matrix of Sec. IV: slow root -D_0 q^2, acoustic roots
    +- i c_s q - Gamma q^2 with Gamma of the closed form, to O(q^4)."""
    n0 = W.densities_from_packing(0.3, [2.0, 3.0], [0.5, 0.5])
    m = H.Mixture([2.0, 3.0], n0, eps=[[H.KT / 2] * 2] * 2, lambda_c=[[2.5] * 2] * 2)
    nu_l = 0.7
    q = 2e-3
    r = m.roots(q, nu_l)
    slow = r[np.argmin(np.abs(r))]
    assert abs(-slow.real / q ** 2 - m.D0()) < 1e-5 * m.D0()
    ac = r[np.argmax(r.imag)]
    assert abs(ac.imag / q - m.sound_speed()) < 1e-5 * m.sound_speed()
    assert abs(-ac.real / q ** 2 - m.sound_damping(nu_l)) < 1e-4 * m.sound_damping(nu_l)


def test_oscillatory_crossover_and_knudsen_number():
    """Above q_c the decoupled concentration pair zeta^2 + gamma zeta + Delta q^2 = 0
    (Sec. IV) turns complex; at low density Kn = lambda_mf q_c / (2 pi) tends
    to (4/3) / (2 pi)^{3/2} = 0.0847 (Eq. critical)."""
    n0 = W.densities_from_packing(1e-4, [1.0, 1.0], [0.5, 0.5])
    m = H.Mixture([1.0, 1.0], n0, lattice=False)
    qc = m.q_c()
    g = m.gamma()
    Delta = 0.25 * m.derivatives()[0]
    for q, cplx in ((0.99 * qc, False), (1.01 * qc, True)):
        disc = g * g / 4 - Delta * q * q
        assert (disc < 0) == cplx
    lam_mf = 1.0 / (math.sqrt(2) * math.pi * m.g(0, 1) * sum(n0))
    Kn = lam_mf * qc / (2 * math.pi)
    assert abs(Kn - H.knudsen_crossover_low_density()) < 1e-3
    assert abs(H.knudsen_crossover_low_density() - 0.08467) < 1e-4


def test_attraction_ratio_fig1_trend():
    """Fig. 1 setting (equisized spheres, w_AA = 5 kT, w_BB = w_AA/2, Berthelot):
    the tails lower D at every concentration, most at c = 1/2, and more at
    higher packing."""
    for packing in (0.1, 0.2, 0.3):
        rs = [H.attraction_ratio(c, packing) for c in (0.1, 0.3, 0.5, 0.7, 0.9)]
        assert all(r < 1.0 for r in rs)
        assert min(rs) == rs[2]
    assert H.attraction_ratio(0.5, 0.3) < H.attraction_ratio(0.5, 0.2) < H.attraction_ratio(0.5, 0.1)


@pytest.mark.parametrize("sigma,packing,eps,bounds", [
    # (one sweep, two sweeps, three sweeps): bounds on the relative D excess
    ([1.0, 1.5], 0.2, None, ((0.005, 0.007), (0.0, 5e-4), (0.0, 2e-4))),
    ([2.0, 3.0], 0.3, [[H.KT / 2] * 2] * 2, ((0.010, 0.013), (0.0, 0.003), (0.0, 0.0015))),
])
def test_predictor_sweeps_approach_the_exact_half_step(sigma, packing, eps, bounds):
    """The lattice mutual diffusion coefficient with 1, 2 and 3 Jacobi sweeps
    of u* = u + a(u*)/2 (the half-force shift of Eq. evolution), against the
    half step solved exactly: one sweep diffuses faster by 0.63 % (sigma
    1/1.5) and 1.16 % (2/3 with tails); two sweeps leave 0.02 % and 0.27 %,
    three 0.01 % and 0.11 %."""
    lam = [[2.5] * 2] * 2 if eps else None
    n0 = W.densities_from_packing(packing, sigma, [0.5, 0.5])
    mk = lambda **kw: W.Lattice(shape=(8, 8, 8), sigma=sigma, tau=1.0, eps=eps, lambda_c=lam, **kw)
    D_exact = lattice_D_long(mk(force_scheme="implicit_coupled"), n0)
    for k, (lo, hi) in zip((1, 2, 3), bounds):
        excess = (lattice_D_long(mk(predictor_sweeps=k), n0) - D_exact) / D_exact
        print(f"sigma={sigma}: {k} sweeps, D excess {excess * 100:+.3f} %")
        assert lo <= excess <= hi, (k, excess)
