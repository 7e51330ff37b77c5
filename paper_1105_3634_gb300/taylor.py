"""Taylor dispersion in a periodically modulated flow (Sec. V, Eqs. ushape,
c99, taylordiff), run through the library on the GPU.

A binary mixture in a box periodic in every direction carries the steady
shear flow u_x(y) = U cos(2 pi y / L_y), held by a body force on every
particle, and a small concentration wave along x (Eq. perturba).  The
section-averaged concentration C(x, t) decays as exp(-D_eff k_x^2 t) with,
to second order in U, D_eff = D (1 + U^2 L_y^2 / (8 pi^2 D^2)) (Eq.
taylordiff; Pe = U L_y / (2 D)).  The measurement here uses:

* D: the decay rate of the same wave without flow (the lattice's own mutual
  diffusion coefficient);
* nu: the decay rate of a free shear wave u_x ~ cos(k_y y) (the mixture's
  kinematic viscosity, kinetic plus collisional), which sets the force
  F = nu k_y^2 U cos(k_y y) that holds the flow;
* U: the cos(k_y y) amplitude of the barycentric velocity actually reached.

`passive_scalar_rate` gives the exact slowest rate of the advection-diffusion
operator for a passive scalar in this flow (all orders in U), against which
the kinetic model's D_eff is compared; `taylor_formula` is Eq. taylordiff.
Host-side analysis (fits, Fourier projections) only: every time step runs in
the library's kernels.
"""
from __future__ import annotations

import math
from typing import Dict, Sequence, Tuple

import numpy as np

from . import workloads as W


# ------------------------------------------------------------------ closed forms
def taylor_formula(D: float, U: float, Ly: float) -> float:
    """Eq. taylordiff: D_eff = D (1 + U^2 L_y^2 / (8 pi^2 D^2))."""
    return D * (1.0 + U * U * Ly * Ly / (8.0 * math.pi ** 2 * D * D))


def peclet(D: float, U: float, Ly: float) -> float:
    """Pe = U L_y / (2 D) (Sec. V)."""
    return U * Ly / (2.0 * D)


def passive_scalar_rate(D: float, U: float, kx: float, ky: float, modes: int = 24) -> float:
    """Slowest decay rate of c(x, y) = Re[sum_n a_n e^{i n ky y} e^{i kx x}]
    under dc/dt = -u_x(y) dc/dx + D lap c with u_x = U cos(ky y): the
    eigenvalue of the tridiagonal matrix a_n' = -D (kx^2 + n^2 ky^2) a_n
    - i kx U (a_{n-1} + a_{n+1}) / 2, n = -modes..modes, closest to zero.
    Returns D_eff = -rate / kx^2."""
    n = np.arange(-modes, modes + 1)
    A = np.diag(-D * (kx * kx + (n * ky) ** 2)).astype(complex)
    off = -0.5j * kx * U
    A += np.diag(np.full(2 * modes, off), 1) + np.diag(np.full(2 * modes, off), -1)
    ev = np.linalg.eigvals(A)
    lam = ev[np.argmax(ev.real)]
    return float(-lam.real / (kx * kx))


def passive_scalar_rate_channel(D: float, u_profile, kx: float) -> float:
    """Slowest decay of c = C(y) e^{i kx x} under dc/dt = -u_x(y) dc/dx + D lap c
    in a channel of cells y = 0 .. ny-1 (unit spacing) with no-flux walls at
    -1/2 and ny - 1/2, u_x(y) given per cell: the eigenvalue closest to zero of
    the finite-volume operator.  Returns D_eff = -rate / kx^2.  For the plane
    Couette profile u = U (2 (y + 1/2) / h - 1) and kx h -> 0 it tends to the
    Taylor-Aris value D + U^2 h^2 / (30 D)."""
    u = np.asarray(u_profile, float)
    ny = len(u)
    A = np.diag(-1j * kx * u - D * kx * kx).astype(complex)
    for i in range(ny - 1):
        A[i, i + 1] += D
        A[i + 1, i] += D
        A[i, i] -= D
        A[i + 1, i + 1] -= D
    ev = np.linalg.eigvals(A)
    return float(-ev[np.argmax(ev.real)].real / (kx * kx))


def taylor_aris_couette(D: float, U: float, h: float) -> float:
    """Plane Couette flow between walls moving at -U and +U, gap h: the
    long-wave Taylor-Aris coefficient D + U^2 h^2 / (30 D)."""
    return D + U * U * h * h / (30.0 * D)


# ------------------------------------------------------------------ fields
def cosine_flow(lat: W.Lattice, U: float) -> np.ndarray:
    """u_x(y) = U cos(2 pi y / L_y) = -U cos(2 pi y / L_y + pi) (Eq. ushape), every species."""
    y = W.coordinate(lat, 1)
    u = np.zeros((lat.nspecies, 3, lat.nsites))
    u[:, 0, :] = U * np.cos(2.0 * math.pi * y / lat.shape[1])[None, :]
    return u


def _mode(lat: W.Lattice, field: np.ndarray, axis: int) -> complex:
    """Fourier amplitude of `field` [N] at the longest wavelength along `axis`
    (all other directions averaged)."""
    q = 2.0 * math.pi * W.coordinate(lat, axis) / lat.shape[axis]
    return complex(np.mean(field * np.exp(-1j * q)))


def _fit_rate(t: np.ndarray, amp: np.ndarray) -> float:
    """Least-squares slope of -log|amp| against t."""
    return float(-np.polyfit(t, np.log(np.abs(amp)), 1)[0])


def _concentration(n: np.ndarray) -> np.ndarray:
    return n[0] / (n[0] + n[1])


# ------------------------------------------------------------------ runs on the GPU
def _sim(mlb, lat, n, u=None, fext=None):
    sim = mlb.Simulation(lat)
    sim.set_fields(n, u)
    if fext is not None:
        sim.set_external_force(fext)
    return sim


def measure_viscosity(mlb, lat: W.Lattice, n0: Sequence[float], U: float = 1e-3,
                      t0: int = 20, t1: int = 220, every: int = 20) -> float:
    """Kinematic viscosity from the decay of a free shear wave u_x ~ cos(k_y y)
    in the uniform mixture: nu = rate / k_y^2."""
    n = np.array([np.full(lat.nsites, v) for v in n0])
    sim = _sim(mlb, lat, n, cosine_flow(lat, U))
    ts, amps = [], []
    t = 0
    for target in range(t0, t1 + 1, every):
        sim.step(target - t)
        t = target
        nn, uu = sim.moments()
        ub = (nn[:, None, :] * uu).sum(0) / nn.sum(0)
        ts.append(t)
        amps.append(_mode(lat, ub[0], 1))
    sim.close()
    ky = 2.0 * math.pi / lat.shape[1]
    return _fit_rate(np.array(ts), np.array(amps)) / (ky * ky)


def measure_dispersion(mlb, lat: W.Lattice, n0: Sequence[float], U: float, nu: float, delta: float = 0.01,
                       t0: int = 400, t1: int = 2400, every: int = 100) -> Tuple[float, float]:
    """(D_eff, U reached): the concentration wave n^{A,B} = n0 (1 +- delta sin(k_x x))
    in the cosine flow held by F_x = nu k_y^2 U cos(k_y y) per particle."""
    n = W.sine_wave(lat, n0, delta)
    ky = 2.0 * math.pi / lat.shape[1]
    fext = None
    u = None
    if U != 0.0:
        u = cosine_flow(lat, U)
        fext = np.zeros((lat.nspecies, 3, lat.nsites))
        fext[:, 0, :] = nu * ky * ky * u[:, 0, :]
    sim = _sim(mlb, lat, n, u, fext)
    ts, amps, flows = [], [], []
    t = 0
    for target in range(t0, t1 + 1, every):
        sim.step(target - t)
        t = target
        nn, uu = sim.moments()
        ts.append(t)
        amps.append(_mode(lat, _concentration(nn), 0))
        ub = (nn[:, None, :] * uu).sum(0) / nn.sum(0)
        flows.append(2.0 * abs(_mode(lat, ub[0], 1)))
    sim.close()
    kx = 2.0 * math.pi / lat.shape[0]
    return _fit_rate(np.array(ts), np.array(amps)) / (kx * kx), float(np.mean(flows))


def couette_flow(lat: W.Lattice) -> np.ndarray:
    """The steady profile between the walls normal to y (halfway bounce-back at
    -1/2 and ny - 1/2): u_x linear from the lower wall's velocity to the upper's,
    every species."""
    ny = lat.shape[1]
    y = W.coordinate(lat, 1)
    lo, hi = lat.wall_u_lo[0], lat.wall_u_hi[0]
    u = np.zeros((lat.nspecies, 3, lat.nsites))
    u[:, 0, :] = (lo + (hi - lo) * (y + 0.5) / ny)[None, :]
    return u


def measure_channel_dispersion(mlb, lat: W.Lattice, n0: Sequence[float], species: int, delta: float = 0.5,
                               t0: int = 100, t1: int = 600, every: int = 50) -> float:
    """D_eff of one species between moving walls normal to y (the Taylor
    channel): n^s = n0_s (1 + delta sin(k_x x)) with the other species uniform,
    the flow started from the Couette profile of the walls; the decay rate of
    the k_x mode of n^s (averaged over y, z) divided by k_x^2.  For a dilute
    solute delta may be large (its own density barely acts on the solvents)."""
    n = np.array([np.full(lat.nsites, v) for v in n0])
    x = W.coordinate(lat, 0)
    kx = 2.0 * math.pi / lat.shape[0]
    n[species] = n0[species] * (1.0 + delta * np.sin(kx * x))
    sim = _sim(mlb, lat, n, couette_flow(lat))
    ts, amps = [], []
    t = 0
    for target in range(t0, t1 + 1, every):
        sim.step(target - t)
        t = target
        nn, _ = sim.moments()
        ts.append(t)
        amps.append(_mode(lat, nn[species], 0))
    sim.close()
    return _fit_rate(np.array(ts), np.array(amps)) / (kx * kx)


def dispersion_curve(mlb, lat: W.Lattice, n0: Sequence[float], Us: Sequence[float], **kw) -> Dict:
    """D(0), nu, and for every U: the measured D_eff, the flow reached, Pe, the
    exact passive-scalar D_eff and Eq. taylordiff."""
    D0, _ = measure_dispersion(mlb, lat, n0, 0.0, 0.0, **kw)
    nu = measure_viscosity(mlb, lat, n0)
    kx = 2.0 * math.pi / lat.shape[0]
    ky = 2.0 * math.pi / lat.shape[1]
    rows = []
    for U in Us:
        Deff, Ur = measure_dispersion(mlb, lat, n0, U, nu, **kw)
        rows.append({"U": U, "U_reached": Ur, "Pe": peclet(D0, Ur, lat.shape[1]), "D_eff": Deff,
                     "D_eff_passive_scalar": passive_scalar_rate(D0, Ur, kx, ky),
                     "D_eff_eq_taylordiff": taylor_formula(D0, Ur, lat.shape[1])})
    return {"D0": D0, "nu": nu, "rows": rows}


# ------------------------------------------------------------------ the paper's experiment (Sec. V, Figs. 3-5)
def paper_lattice(packing: float, Lx: int, Ly: int = 40, Lz: int = 40, tau: float = 1.0, sweeps: int = 1):
    """The mixture of Figs. 3-5: sigma_AA = 8, sigma_BB = 4 (contact shells of
    762 points for A-A), equal mole fractions c_0 = 0.5, total packing xi_3
    (0.211 or 0.332), box L_x x 40 x 40, periodic; tau is not stated (1).
    sweeps: Jacobi sweeps of the half step (1 = the library's default)."""
    lat = W.Lattice(shape=(Lx, Ly, Lz), sigma=[8.0, 4.0], tau=tau)
    lat.predictor_sweeps = sweeps
    return lat, W.densities_from_packing(packing, lat.sigma, [0.5, 0.5])


def paper_curve(mlb, packing: float, Lx: int, pes: Sequence[float], Ly: int = 40, Lz: int = 40,
                sweeps: int = 1) -> Dict:
    """Fig. 5: D_eff against Pe = U L_y / (2 D) for the Fig. 3 mixture.  D(0)
    is measured first (no flow), the flow amplitude for each target Pe is
    U = 2 D(0) Pe / L_y, and every fit spans 0.3 to 2.5 decay times of the
    wave; rows give the Pe reached, D_eff / D(0), the exact passive-scalar
    ratio for the flow reached and Eq. taylordiff's 1 + Pe^2 / (2 pi^2)."""
    lat, n0 = paper_lattice(packing, Lx, Ly, Lz, sweeps=sweeps)
    kx = 2.0 * math.pi / Lx
    ky = 2.0 * math.pi / Ly

    def window(D):
        rate = D * kx * kx
        t0, t1 = max(5, int(0.3 / rate)), max(40, int(2.5 / rate))
        return dict(t0=t0, t1=t1, every=max(1, (t1 - t0) // 12))

    D_guess, _ = measure_dispersion(mlb, lat, n0, 0.0, 0.0, t0=10, t1=60, every=5)
    D0, _ = measure_dispersion(mlb, lat, n0, 0.0, 0.0, **window(D_guess))
    nu = measure_viscosity(mlb, lat, n0)
    rows = []
    for pe in pes:
        U = 2.0 * D0 * pe / Ly
        Deff, Ur = measure_dispersion(mlb, lat, n0, U, nu, **window(D0 * (1.0 + pe * pe / (2 * math.pi ** 2))))
        pe_r = peclet(D0, Ur, Ly)
        rows.append({"Pe_target": pe, "U": U, "Pe": pe_r, "D_eff": Deff, "ratio": Deff / D0,
                     "ratio_passive_scalar": passive_scalar_rate(D0, Ur, kx, ky) / D0,
                     "ratio_eq_taylordiff": 1.0 + pe_r * pe_r / (2.0 * math.pi ** 2)})
    return {"packing": packing, "Lx": Lx, "Ly": Ly, "Lz": Lz, "sweeps": sweeps, "D0": D0, "nu": nu, "rows": rows}


if __name__ == "__main__":  # pragma: no cover
    # python -m paper_1105_3634_gb300.taylor [--packings 0.211 0.332] [--lx 40 80] [--pe 0.5 1 1.5 2] [--sweeps 1]
    import argparse
    import json
    ap = argparse.ArgumentParser(description="Taylor dispersion of Sec. V (Figs. 3-5) on the GPU")
    ap.add_argument("--packings", type=float, nargs="+", default=[0.211, 0.332])
    ap.add_argument("--lx", type=int, nargs="+", default=[40, 80])
    ap.add_argument("--pe", type=float, nargs="+", default=[0.5, 1.0, 1.5, 2.0])
    ap.add_argument("--sweeps", type=int, default=1, help="Jacobi sweeps of the half step (1..8)")
    args = ap.parse_args()
    from . import mlb as _mlb
    for packing in args.packings:
        for Lx in args.lx:
            print(json.dumps(paper_curve(_mlb, packing, Lx, args.pe, sweeps=args.sweeps)), flush=True)
