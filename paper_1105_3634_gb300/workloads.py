"""Lattice descriptions and seeded synthetic inputs.

This module is shared by the CUDA path's callers and by the oracle's callers.
It holds parameters and input generators only: no step of the lattice
Boltzmann method is computed here.  Random numbers come from one SplitMix64
stream per seed (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), implemented below from its published definition.

Workloads follow the paper's numerical section (Sec. V): binary hard-sphere
mixtures of equal masses in lattice units (lattice spacing = time step = 1,
m = 1, kT = c_s^2 = 1/3), a small concentration sine wave (Eq. perturba),
seeded uniform density noise, and a Taylor-dispersion channel with moving
walls.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

KT_LATTICE = 1.0 / 3.0


@dataclasses.dataclass
class Lattice:
    shape: Tuple[int, int, int]                # (nx, ny, nz), x fastest
    sigma: List[float]                         # hard-sphere diameters sigma_aa
    mass: List[float] = None                   # equal masses (lattice units: 1)
    eps: List[List[float]] = None              # attraction strengths eps_ab (symmetric)
    lambda_c: List[List[float]] = None         # cutoff radius / sigma_ab
    tau: float = 1.0
    kT: float = KT_LATTICE
    kappa: float = 0.5                         # smoothing-ball radius / sigma
    wall_axis: int = -1                        # -1 periodic; 0/1/2 walls normal to that axis
    wall_u_lo: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    wall_u_hi: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    drag_only: bool = False
    force_scheme: str = "semi_implicit"        # or "explicit" (forward Euler forcing)
    predictor_sweeps: int = 1                  # Jacobi sweeps of the half step u* = u + a(u*)/2
    meanfield: str = "fp32"                    # attraction on the GPU: "fp32" column sums, "bf16"
                                               # compensated tensor-core product, "bf16_1pass" hi*hi only

    def __post_init__(self):
        S = len(self.sigma)
        if self.mass is None:
            self.mass = [1.0] * S
        if self.eps is None:
            self.eps = [[0.0] * S for _ in range(S)]
        if self.lambda_c is None:
            self.lambda_c = [[2.5] * S for _ in range(S)]

    @property
    def nspecies(self) -> int:
        return len(self.sigma)

    @property
    def nsites(self) -> int:
        nx, ny, nz = self.shape
        return nx * ny * nz


# ---------------------------------------------------------------- SplitMix64
_M64 = (1 << 64) - 1


def splitmix64(seed: int, count: int) -> np.ndarray:
    """`count` successive outputs of SplitMix64 started at `seed` (uint64)."""
    with np.errstate(over="ignore"):
        state = np.uint64(seed & _M64)
        gamma = np.uint64(0x9E3779B97F4A7C15)
        k = np.arange(1, count + 1, dtype=np.uint64)
        z = state + gamma * k
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


# ---------------------------------------------------------------- densities
def densities_from_packing(xi3: float, sigma: Sequence[float], mole_fractions: Sequence[float]) -> np.ndarray:
    """Uniform number densities with packing fraction xi3 = (pi/6) sum n_a sigma_a^3
    (the packing definition of the Fig. 1 caption) at the given mole fractions."""
    x = np.asarray(mole_fractions, np.float64)
    s3 = np.asarray(sigma, np.float64) ** 3
    ntot = xi3 / (math.pi / 6.0 * float(np.dot(x, s3)))
    return ntot * x


def coordinate(lat: Lattice, axis: int) -> np.ndarray:
    """Coordinate along `axis` of every site, flattened x-fastest."""
    nx, ny, nz = lat.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return [x, y, z][axis].reshape(-1).astype(np.float64)


def sine_wave(lat: Lattice, n0: Sequence[float], rel_amp: float, axis: int = 0,
              wavelength: float = None) -> np.ndarray:
    """Eq. perturba: n^A = n0^A (1 + amp sin(q x)), n^B = n0^B (1 - amp sin(q x));
    further species (if any) stay uniform.  Returns n [S][N]."""
    L = lat.shape[axis]
    lam = float(L if wavelength is None else wavelength)
    s = np.sin(2.0 * math.pi * coordinate(lat, axis) / lam)
    S = lat.nspecies
    n = np.empty((S, lat.nsites))
    for a in range(S):
        sign = 1.0 if a == 0 else (-1.0 if a == 1 else 0.0)
        n[a] = n0[a] * (1.0 + sign * rel_amp * s)
    return n


def noise(lat: Lattice, n0: Sequence[float], rel: float, seed: int) -> np.ndarray:
    """n^a = n0^a (1 + rel U(-1, 1)), one SplitMix64 stream for all species."""
    S, N = lat.nspecies, lat.nsites
    u = uniform01(seed, S * N).reshape(S, N)
    return np.asarray(n0, np.float64)[:, None] * (1.0 + rel * (2.0 * u - 1.0))


def random_velocities(lat: Lattice, scale: float, seed: int) -> np.ndarray:
    """Species velocities uniform in [-scale, scale): u [S][3][N]."""
    S, N = lat.nspecies, lat.nsites
    u = uniform01(seed, S * 3 * N).reshape(S, 3, N)
    return scale * (2.0 * u - 1.0)


def gaussian_pulse(lat: Lattice, n_bg: Sequence[float], solute: int, solute_fraction: float,
                   width: float, axis: int = 0) -> np.ndarray:
    """Solvent species uniform at n_bg; the solute is a Gaussian pulse of
    standard deviation `width` along `axis`, centred in the box, whose peak
    is `solute_fraction` of the total solvent density."""
    S, N = lat.nspecies, lat.nsites
    L = lat.shape[axis]
    xc = coordinate(lat, axis)
    prof = np.exp(-0.5 * ((xc - 0.5 * (L - 1)) / width) ** 2)
    n = np.empty((S, N))
    tot = sum(n_bg[a] for a in range(S) if a != solute)
    for a in range(S):
        n[a] = n_bg[a] if a != solute else solute_fraction * tot * prof
    return n


# ---------------------------------------------------------------- named workloads
def binary_config1(shape=(64, 8, 8)) -> Tuple[Lattice, np.ndarray]:
    """Binary hard spheres sigma = (1, 1.5), packing 0.2, equal mole
    fractions, no attraction, tau = 1, relative sine amplitude 0.05 along x
    with wavelength = box length.  Returns (lattice, n [S][N])."""
    lat = Lattice(shape=tuple(shape), sigma=[1.0, 1.5], tau=1.0)
    n0 = densities_from_packing(0.2, lat.sigma, [0.5, 0.5])
    return lat, sine_wave(lat, n0, 0.05, axis=0)


def binary_attraction(shape=(128, 128, 128), seed: int = 20110518) -> Tuple[Lattice, np.ndarray]:
    """Binary sigma = (2, 3) with tail -eps (sigma_ab/r)^6 cut at 2.5 sigma_ab,
    eps = 0.5 kT, packing 0.3, equal mole fractions, 1% uniform noise."""
    S = 2
    eps = 0.5 * KT_LATTICE
    lat = Lattice(shape=tuple(shape), sigma=[2.0, 3.0],
                  eps=[[eps] * S for _ in range(S)], lambda_c=[[2.5] * S for _ in range(S)])
    n0 = densities_from_packing(0.3, lat.sigma, [0.5, 0.5])
    return lat, noise(lat, n0, 0.01, seed)


def taylor_channel(shape=(512, 64, 64), U: float = 0.05) -> Tuple[Lattice, np.ndarray]:
    """Two solvents sigma = 2, 2.5 (packing 0.211, equal mole fractions) and a
    dilute solute sigma = 3 at mole fraction 1e-3 in a Gaussian pulse of
    width 8 along x; walls normal to y moving at -U and +U along x."""
    lat = Lattice(shape=tuple(shape), sigma=[2.0, 2.5, 3.0], wall_axis=1,
                  wall_u_lo=(-U, 0.0, 0.0), wall_u_hi=(U, 0.0, 0.0))
    n_solv = densities_from_packing(0.211, lat.sigma[:2], [0.5, 0.5])
    n = gaussian_pulse(lat, [n_solv[0], n_solv[1], 0.0], solute=2, solute_fraction=1e-3, width=8.0)
    return lat, n


def ensemble_attraction(count: int = 64, seed: int = 1106, meanfield: str = "bf16") -> List[Tuple[Lattice, np.ndarray]]:
    """Independent binary systems with the attractive tails of the attraction
    workload (sigma = (2, 3), -eps (sigma_ab / r)^6 cut at 2.5 sigma_ab, eps =
    kT/2; the mean field on the tensor cores by default): cubes of side L in
    {32, 40, ..., 128}, packing 0.05 .. 0.30 (equal mole fractions, tau = 1),
    a 5% concentration wave along x, shear U in 0 .. 0.05 as in ensemble()."""
    r = uniform01(seed, 3 * count).reshape(count, 3)
    eps = 0.5 * KT_LATTICE
    tails = dict(eps=[[eps] * 2 for _ in range(2)], lambda_c=[[2.5] * 2 for _ in range(2)])
    out = []
    for k in range(count):
        L = 32 + 8 * int(r[k, 0] * 13)
        packing = 0.05 + 0.25 * r[k, 1]
        U = 0.05 * r[k, 2]
        if U > 0.005:
            lat = Lattice(shape=(L, L, L), sigma=[2.0, 3.0], wall_axis=1, wall_u_lo=(-U, 0.0, 0.0),
                          wall_u_hi=(U, 0.0, 0.0), meanfield=meanfield, **tails)
        else:
            lat = Lattice(shape=(L, L, L), sigma=[2.0, 3.0], meanfield=meanfield, **tails)
        n0 = densities_from_packing(packing, lat.sigma, [0.5, 0.5])
        out.append((lat, sine_wave(lat, n0, 0.05)))
    return out


def ensemble(count: int = 64, seed: int = 1105) -> List[Tuple[Lattice, np.ndarray]]:
    """Independent binary systems of uneven sizes for batched runs: cubes of
    side L in {32, 40, ..., 128}, packing 0.05 .. 0.20 (equal mole fractions,
    sigma = (1, 1.5), tau = 1), a 5% concentration wave along x, and shear
    U in 0 .. 0.05: U > 0.005 gives a channel between walls normal to y
    moving at -U and +U along x (Couette), else a periodic box.  With these
    one-site spheres the scheme stays stable to packing 0.20 between moving
    walls (the contact layer at a wall raises the local packing to ~0.34);
    at 0.22 with walls and at 0.25 without it does not."""
    r = uniform01(seed, 3 * count).reshape(count, 3)
    out = []
    for k in range(count):
        L = 32 + 8 * int(r[k, 0] * 13)
        packing = 0.05 + 0.15 * r[k, 1]
        U = 0.05 * r[k, 2]
        if U > 0.005:
            lat = Lattice(shape=(L, L, L), sigma=[1.0, 1.5], wall_axis=1, wall_u_lo=(-U, 0.0, 0.0),
                          wall_u_hi=(U, 0.0, 0.0))
        else:
            lat = Lattice(shape=(L, L, L), sigma=[1.0, 1.5])
        n0 = densities_from_packing(packing, lat.sigma, [0.5, 0.5])
        out.append((lat, sine_wave(lat, n0, 0.05)))
    return out
