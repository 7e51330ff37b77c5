"""The scheme against closed forms the paper prints (Secs. III-IV).

Computed through the linear one-step operator L(q) of tests/linear_model.py,
which the oracle reproduces to 1e-7 (tests/test_oracle_linear.py): the
slowest concentration mode and the shear mode of L(q) at long wavelength give
the lattice mutual-diffusion coefficient and kinematic viscosity.

* Eq. dab: D^AB = (3/8n) sqrt(kT/(2 pi mu_AB)) / (sigma_AB^2 g_AB).  For equal
  diameters the mixture is thermodynamically ideal in the concentration, so
  the diffusive eigenvalue -D_0 q^2 of Sec. IV has D_0 = D^AB exactly.
* Shear mode: nu = eta/rho with eta = eta^K + eta^C; the collisional part is
  eta^C = (4/15) sum_ab sqrt(2 pi mu_ab kT) sigma_ab^4 g_ab n_a n_b (Sec. III);
  the lattice kinetic part is c_s^2 (tau - 1/2).  The lattice contact shell
  reproduces the fourth radial moment of the sphere only for sigma >~ 3
  (asserted at sigma = 4).
"""
import math

import numpy as np
import pytest

import linear_model as LM
from paper_1105_3634_gb300 import workloads as W

KT = 1.0 / 3.0


def _slow_mode(lat, n0, L, pick):
    q = np.array([2 * math.pi / L, 0.0, 0.0])
    Lm, Dn, Dj = LM.operator(lat, n0, q)
    ev, V = np.linalg.eig(Lm)
    best = None
    for i in range(len(ev)):
        w = pick(V[:, i], Dn, Dj) / np.linalg.norm(V[:, i])
        if abs(ev[i]) > 0.5 and (best is None or w > best[0]):
            best = (w, ev[i])
    return -math.log(abs(best[1])) / q[0] ** 2


def lattice_D(lat, n0, L):
    return _slow_mode(lat, n0, L, lambda v, Dn, Dj: abs((Dn @ v)[0] * n0[1] - (Dn @ v)[1] * n0[0]))


def lattice_D_long(lat, n0):
    """Long-wavelength limit: the q^2 correction removed by Richardson
    extrapolation from wavelengths 128 and 256."""
    return (4.0 * lattice_D(lat, n0, 256) - lattice_D(lat, n0, 128)) / 3.0


def lattice_nu(lat, n0, L):
    return _slow_mode(lat, n0, L, lambda v, Dn, Dj: abs((Dj[:, 1, :] @ v).sum()))


def eq_dab(sigma, n0):
    xi2 = math.pi / 6 * float(np.dot(n0, np.array(sigma) ** 2))
    xi3 = math.pi / 6 * float(np.dot(n0, np.array(sigma) ** 3))
    s = 0.5 * (sigma[0] + sigma[1])
    g = LM.bmcsl(sigma[0], sigma[1], xi2, xi3)
    mu = 0.5
    return 3.0 / (8.0 * n0.sum()) * math.sqrt(KT / (2 * math.pi * mu)) / (s * s * g)


@pytest.mark.parametrize("sigma,packing", [([2.0, 2.0], 0.2), ([4.0, 4.0], 0.1), ([4.0, 4.0], 0.3)])
def test_mutual_diffusion_equal_diameters_is_eq_dab(sigma, packing):
    lat = W.Lattice(shape=(8, 8, 8), sigma=sigma, tau=1.0)
    n0 = W.densities_from_packing(packing, sigma, [0.5, 0.5])
    D = lattice_D_long(lat, n0)
    ref = eq_dab(sigma, n0)
    assert abs(D - ref) < 1e-3 * ref, (D, ref)


def test_mutual_diffusion_unequal_diameters_reported():
    """Unequal diameters: D_0 = D^AB times the thermodynamic factor of the
    mixture (Sec. IV), not computed here; the lattice value is reported and
    only required to lie within 40 % of Eq. dab (it is +3 % ... +30 %)."""
    for sigma, packing in [([1.0, 1.5], 0.2), ([2.0, 3.0], 0.3)]:
        lat = W.Lattice(shape=(8, 8, 8), sigma=sigma, tau=1.0)
        n0 = W.densities_from_packing(packing, sigma, [0.5, 0.5])
        D, ref = lattice_D_long(lat, n0), eq_dab(sigma, n0)
        print(f"sigma={sigma} packing={packing}: D_lattice={D:.4f}  Eq. dab={ref:.4f}  ratio={D / ref:.3f}")
        assert 0.6 < D / ref < 1.4


@pytest.mark.parametrize("packing,tau", [(0.1, 1.0), (0.3, 1.0), (0.2, 0.8)])
def test_shear_viscosity_eta_C(packing, tau):
    sigma = [4.0, 4.0]
    lat = W.Lattice(shape=(8, 8, 8), sigma=sigma, tau=tau)
    n0 = W.densities_from_packing(packing, sigma, [0.5, 0.5])
    xi2 = math.pi / 6 * float(np.dot(n0, np.array(sigma) ** 2))
    xi3 = math.pi / 6 * float(np.dot(n0, np.array(sigma) ** 3))
    etaC = 0.0
    for a in range(2):
        for b in range(2):
            s = 0.5 * (sigma[a] + sigma[b])
            etaC += 4.0 / 15.0 * math.sqrt(2 * math.pi * 0.5 * KT) * s ** 4 * LM.bmcsl(sigma[a], sigma[b], xi2, xi3) * n0[a] * n0[b]
    nu_theory = KT * (tau - 0.5) + etaC / n0.sum()
    nu = lattice_nu(lat, n0, 256)
    assert abs(nu - nu_theory) < 0.025 * nu_theory, (nu, nu_theory)
