"""Linear hydrodynamics of the multispecies model (Sec. IV, "Hydrodynamic
analysis"), evaluated for the lattice the library solves.

From the linearised equations (Eqs. cc1-cc4) around a uniform binary state:
* the friction of the relative velocity w = u^A - u^B, gamma (Eq.
  gammasymmetrized1), and the mutual diffusion coefficient D^AB = kT / (gamma m)
  (Eqs. mutualdiffusion, dab);
* the diffusive root zeta = -D_0 q^2 with D_0 = c (1 - c) (d mu_D / d c)_P / gamma,
  mu_D = mu^A - mu^B (Eq. mudif, equal unit masses), the thermodynamic
  factor (d mu_D / d c)_P c (1 - c) / kT multiplying D^AB;
* the acoustic roots zeta = +- i c_s q - Gamma q^2 (Eq. damping) and the
  crossover q_c = sqrt(gamma^2 / (4 Delta)), Delta = c (1 - c) (d mu_D / d c)_rho,
  above which a concentration fluctuation decays oscillating; at low density
  the Knudsen number of the crossover is 4 / (3 (2 pi)^{3/2}) (Eq. critical).

The chemical-potential derivatives are those the model's forces imply
(mechanical route): at long wavelength the hard-core term of Eq.
potmeanforce on a lattice shell S_ab of weight 4 pi / |S_ab| is
F^a = -kT (4 pi / 3) sum_b sigma_ab^2 m1_ab [g_ab grad n^b + n^b grad g_ab / 2],
m1_ab = 3 <d_x^2 / |d|>_S (sigma_ab for the continuous sphere), and the RPA
tail -eps_ab (sigma_ab / r)^6 on sigma_ab <= r <= lambda_c sigma_ab adds
+sum_b A_ab eps_ab grad n^b with A_ab = (1/3) sum_d |d| |U'(|d|)| / eps
over the lattice region (continuum: (8 pi / 3) sigma^3 (1 - lambda_c^-3)).
g_ab is the BMCSL contact value (reading R2); masses are 1 and kT = 1/3 in
lattice units.  Host-side closed forms only (numpy).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

KT = 1.0 / 3.0


# ------------------------------------------------------------------ BMCSL contact values
def bmcsl(sa: float, sb: float, xi2: float, xi3: float) -> float:
    """g_ab = 1/(1-xi3) + 3 h xi2/(1-xi3)^2 + 2 h^2 xi2^2/(1-xi3)^3, h = sa sb/(sa+sb)."""
    h, o = sa * sb / (sa + sb), 1.0 - xi3
    return 1.0 / o + 3.0 * h * xi2 / o ** 2 + 2.0 * h * h * xi2 * xi2 / o ** 3


def bmcsl_grad(sa: float, sb: float, xi2: float, xi3: float):
    """(dg/dxi2, dg/dxi3) of the BMCSL contact value."""
    h, o = sa * sb / (sa + sb), 1.0 - xi3
    d2 = 3.0 * h / o ** 2 + 4.0 * h * h * xi2 / o ** 3
    d3 = 1.0 / o ** 2 + 6.0 * h * xi2 / o ** 3 + 6.0 * h * h * xi2 * xi2 / o ** 4
    return d2, d3


# ------------------------------------------------------------------ lattice moments
def shell_points(s: float):
    """Offsets of the lattice contact shell s - 1/2 <= |d| < s + 1/2 (reading R3)."""
    R = int(math.ceil(s + 0.5)) + 1
    r = np.arange(-R, R + 1)
    d = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    q = (d * d).sum(1)
    lo = max(s - 0.5, 0.0)
    return d[(q > 0) & (q >= lo * lo) & (q < (s + 0.5) ** 2)]


def shell_moment(s: float, lattice: bool = True) -> float:
    """m1 = 3 <d_x^2 / |d|> over the shell (s for the continuous sphere)."""
    if not lattice:
        return s
    d = shell_points(s)
    r = np.sqrt((d * d).sum(1))
    return float(3.0 * np.mean(d[:, 0] ** 2 / r))


def attraction_moment(s: float, lam: float, lattice: bool = True) -> float:
    """A = (1/3) sum_d |d| |U'(|d|)| / eps for U = -eps (s/r)^6 on s <= |d| <= lam s,
    i.e. 2 s^6 sum_d |d|^-6 (continuum: (8 pi / 3) s^3 (1 - lam^-3))."""
    if not lattice:
        return 8.0 * math.pi / 3.0 * s ** 3 * (1.0 - lam ** -3)
    rc = lam * s
    R = int(math.ceil(rc)) + 1
    r = np.arange(-R, R + 1)
    d = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    q = (d * d).sum(1).astype(float)
    sel = (q > 0) & (q >= s * s) & (q <= rc * rc)
    return float(2.0 * s ** 6 * np.sum(q[sel] ** -3))


# ------------------------------------------------------------------ the mixture
@dataclass
class Mixture:
    sigma: Sequence[float]                 # diameters sigma_aa
    n: Sequence[float]                     # number densities n^a
    eps: Optional[Sequence[Sequence[float]]] = None       # tail strengths eps_ab (symmetric)
    lambda_c: Optional[Sequence[Sequence[float]]] = None  # cutoff / sigma_ab
    kT: float = KT
    lattice: bool = True                   # lattice shell and tail sums, else continuum integrals

    def __post_init__(self):
        self.sigma = np.asarray(self.sigma, float)
        self.n = np.asarray(self.n, float)
        S = len(self.sigma)
        self.eps = np.zeros((S, S)) if self.eps is None else np.asarray(self.eps, float)
        self.lambda_c = np.full((S, S), 2.5) if self.lambda_c is None else np.asarray(self.lambda_c, float)

    @property
    def S(self) -> int:
        return len(self.sigma)

    def sab(self, a: int, b: int) -> float:
        return 0.5 * (self.sigma[a] + self.sigma[b])

    def xi(self, k: int) -> float:
        return math.pi / 6.0 * float(np.dot(self.n, self.sigma ** k))

    def g(self, a: int, b: int) -> float:
        return bmcsl(self.sigma[a], self.sigma[b], self.xi(2), self.xi(3))

    def dg_dn(self, a: int, b: int, c: int) -> float:
        d2, d3 = bmcsl_grad(self.sigma[a], self.sigma[b], self.xi(2), self.xi(3))
        return (d2 * self.sigma[c] ** 2 + d3 * self.sigma[c] ** 3) * math.pi / 6.0

    # d mu_a / d n_c: ideal part plus the hard-core and tail forces (mechanical route)
    def jacobian(self) -> np.ndarray:
        S, kT = self.S, self.kT
        J = np.zeros((S, S))
        for a in range(S):
            for c in range(S):
                s = self.sab(a, c)
                v = s * s * shell_moment(s, self.lattice) * self.g(a, c)
                for b in range(S):
                    sb = self.sab(a, b)
                    v += 0.5 * self.n[b] * sb * sb * shell_moment(sb, self.lattice) * self.dg_dn(a, b, c)
                J[a, c] = kT * 4.0 * math.pi / 3.0 * v
                if self.eps[a, c] != 0.0:
                    J[a, c] -= self.eps[a, c] * attraction_moment(s, self.lambda_c[a, c], self.lattice)
                if a == c:
                    J[a, c] += kT / self.n[a]
        return J

    def dP_dn(self) -> np.ndarray:
        """Mechanical pressure: grad P = sum_a n^a grad mu_a."""
        return self.n @ self.jacobian()

    # binary mixtures, equal unit masses: rho = n_A + n_B, c = n_A / rho
    def _binary(self):
        if self.S != 2:
            raise ValueError("the hydrodynamic matrix of Sec. IV is binary")
        rho = float(self.n.sum())
        return rho, float(self.n[0] / rho)

    def derivatives(self):
        """((d mu_D/d c)_rho, (d mu_D/d rho)_c, (dP/d c)_rho, (dP/d rho)_c)."""
        rho, c = self._binary()
        J, Pn = self.jacobian(), self.dP_dn()
        muD_n = J[0] - J[1]                           # d mu_D / d n_k
        dc = np.array([rho, -rho])                    # (dn_A, dn_B) per unit dc at fixed rho
        dr = np.array([c, 1.0 - c])                   # per unit drho at fixed c
        return float(muD_n @ dc), float(muD_n @ dr), float(Pn @ dc), float(Pn @ dr)

    def gamma(self) -> float:
        """Eq. gammasymmetrized1 (unit masses): (8/3) rho sqrt(2 pi mu_AB kT) g_AB sigma_AB^2."""
        rho, _ = self._binary()
        s = self.sab(0, 1)
        return 8.0 / 3.0 * rho * math.sqrt(2.0 * math.pi * 0.5 * self.kT) * self.g(0, 1) * s * s

    def D_AB(self) -> float:
        """Eq. dab (= kT / gamma for unit masses)."""
        return self.kT / self.gamma()

    def thermodynamic_factor(self, at: str = "P") -> float:
        """c (1 - c) (d mu_D / d c)_X / kT at constant pressure (X = P: the slow
        root of the hydrodynamic matrix) or constant total density (X = rho)."""
        rho, c = self._binary()
        mc, mr, pc, pr = self.derivatives()
        if at == "rho":
            return c * (1.0 - c) * mc / self.kT
        if pr <= 0.0:
            raise ValueError("(dP/drho)_c <= 0: the uniform state is mechanically unstable (spinodal)")
        return c * (1.0 - c) * (mc - mr * pc / pr) / self.kT

    def D0(self, at: str = "P") -> float:
        """The diffusive root -D_0 q^2: D_0 = D^AB times the thermodynamic factor."""
        return self.D_AB() * self.thermodynamic_factor(at)

    def sound_speed(self) -> float:
        return math.sqrt(self.derivatives()[3])

    def roots(self, q: float, nu_l: float) -> np.ndarray:
        """Roots zeta of the 4 x 4 determinant of Sec. IV (variables drho, u, w, dc)
        for wavenumber q and longitudinal kinematic viscosity nu_l."""
        rho, c = self._binary()
        mc, mr, pc, pr = self.derivatives()
        g = self.gamma()
        A = np.array([[0.0, -1j * q * rho, 0.0, 0.0],
                      [-1j * q / rho * pr, -nu_l * q * q, 0.0, -1j * q / rho * pc],
                      [-1j * q * mr, 0.0, -g, -1j * q * mc],
                      [0.0, 0.0, -1j * q * c * (1.0 - c), 0.0]])
        return np.linalg.eigvals(A)

    def sound_damping(self, nu_l: float) -> float:
        """Gamma of zeta = +- i c_s q - Gamma q^2 to order q^2: sound damped by the
        longitudinal viscosity and by interdiffusion,
        Gamma = [nu_l + c (1 - c) (d mu_D/d rho)_c (dP/dc)_rho / (gamma (dP/d rho)_c)] / 2."""
        rho, c = self._binary()
        mc, mr, pc, pr = self.derivatives()
        return 0.5 * (nu_l + c * (1.0 - c) * mr * pc / (self.gamma() * pr))

    def q_c(self) -> float:
        """Crossover q_c = sqrt(gamma^2 / (4 Delta)), Delta = c (1 - c) (d mu_D / d c)_rho."""
        rho, c = self._binary()
        Delta = c * (1.0 - c) * self.derivatives()[0]
        return math.sqrt(self.gamma() ** 2 / (4.0 * Delta))


def knudsen_crossover_low_density() -> float:
    """Eq. critical: Kn = lambda_mf / L_c = (4/3) / (2 pi)^{3/2}."""
    return 4.0 / 3.0 / (2.0 * math.pi) ** 1.5


def attraction_ratio(c: float, packing: float, sigma: float = 1.0, w_AA: float = 5.0 * KT,
                     lam: float = 2.5, lattice: bool = False, at: str = "rho") -> float:
    """D_0 with tails / D_0 without, for equisized spheres at concentration c
    and packing fraction packing, w_BB = w_AA / 2, w_AB = sqrt(w_AA w_BB)
    (Eq. berthelot; the setting of Fig. 1).  The default takes d mu_D / d c at
    constant total density, the form in which the figure's trend (a reduction,
    largest at c = 1/2) appears; at w_AA = 5 kT the uniform state lies inside
    the spinodal ((dP/drho)_c < 0), where the constant-pressure root has no
    meaning."""
    n = packing / (math.pi / 6.0 * sigma ** 3)
    dens = [c * n, (1.0 - c) * n]
    w_BB = w_AA / 2.0
    eps = [[w_AA, math.sqrt(w_AA * w_BB)], [math.sqrt(w_AA * w_BB), w_BB]]
    with_tails = Mixture([sigma, sigma], dens, eps=eps, lambda_c=[[lam] * 2] * 2, lattice=lattice)
    without = Mixture([sigma, sigma], dens, lattice=lattice)
    return with_tails.D0(at) / without.D0(at)
