"""FP64 CPU oracle of the multispecies Enskog/RPA lattice Boltzmann step.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg (and ``--impl reference`` arm) of ``bench.py`` may import
this package.  The product path (``paper_1105_3634_gb300``) never imports it.

The arithmetic lives in ``mlb_oracle.c`` (plain C, FP64, OpenMP over sites);
this module only builds it with gcc and marshals numpy arrays through ctypes.
Array layouts (x fastest, site = x + nx*(y + ny*z)):

    f    [S][19][N]   populations in the oracle's own velocity order
    n    [S][N]       number densities
    j    [S][3][N]    momentum densities n^a u^a
    g    [S][S][N]    pair contact values
    phi  [S][3][N]    effective field Phi^a
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mlb_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liborc.so")
MAXS = 8
Q = 19


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, -O2, no -march flags)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("nspecies", ctypes.c_int32),
        ("wall_axis", ctypes.c_int32), ("drag_only", ctypes.c_int32),
        ("explicit_force", ctypes.c_int32), ("predictor_sweeps", ctypes.c_int32),
        ("wall_u_lo", ctypes.c_double * 3), ("wall_u_hi", ctypes.c_double * 3),
        ("tau", ctypes.c_double), ("kT", ctypes.c_double), ("kappa", ctypes.c_double),
        ("sigma", ctypes.c_double * MAXS), ("mass", ctypes.c_double * MAXS),
        ("eps", ctypes.c_double * (MAXS * MAXS)),
        ("lambda_c", ctypes.c_double * (MAXS * MAXS)),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER(OrcParams)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        lp = ctypes.POINTER(ctypes.c_int64)
        L.orc_velocities.argtypes = [ip, dp]
        L.orc_shell.argtypes = [ctypes.c_double, ip, ctypes.c_int]
        L.orc_attraction_set.argtypes = [ctypes.c_double, ctypes.c_double, ip, ctypes.c_int]
        L.orc_bmcsl.argtypes = [ctypes.c_double] * 4
        L.orc_bmcsl.restype = ctypes.c_double
        L.orc_moments.argtypes = [P, dp, dp, dp]
        L.orc_gfield.argtypes = [P, dp, dp, dp]
        L.orc_forces.argtypes = [P, dp, dp, dp, dp, dp, dp, dp]
        L.orc_forces_sites.argtypes = [P, dp, dp, dp, ctypes.c_long, lp, dp, dp, dp, dp]
        L.orc_collide_local.argtypes = [P, ctypes.c_long, dp, dp, dp, dp, dp]
        L.orc_accel_sites.argtypes = [P, dp, dp, dp, dp, ctypes.c_long, lp, dp, dp]
        L.orc_init.argtypes = [P, dp, dp, dp]
        L.orc_step.argtypes = [P, dp, dp, ctypes.c_int]
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_set_num_threads.argtypes = [ctypes.c_int]
        L.orc_set_num_threads.restype = None
        _lib = L
    return _lib


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def params(lat) -> OrcParams:
    """Oracle parameter block from a ``workloads.Lattice``."""
    S = len(lat.sigma)
    if S > MAXS:
        raise ValueError("too many species")
    p = OrcParams()
    p.nx, p.ny, p.nz = lat.shape
    p.nspecies = S
    p.wall_axis = lat.wall_axis
    p.drag_only = 1 if lat.drag_only else 0
    if lat.force_scheme not in ("semi_implicit", "explicit"):
        raise ValueError(f"unknown force scheme {lat.force_scheme!r}")
    p.explicit_force = 1 if lat.force_scheme == "explicit" else 0
    p.predictor_sweeps = int(getattr(lat, "predictor_sweeps", 1))
    for k in range(3):
        p.wall_u_lo[k] = lat.wall_u_lo[k]
        p.wall_u_hi[k] = lat.wall_u_hi[k]
    p.tau, p.kT, p.kappa = lat.tau, lat.kT, lat.kappa
    for a in range(S):
        p.sigma[a] = lat.sigma[a]
        p.mass[a] = lat.mass[a]
        for b in range(S):
            p.eps[a * S + b] = lat.eps[a][b]
            p.lambda_c[a * S + b] = lat.lambda_c[a][b]
    return p


def velocities():
    c = np.zeros((Q, 3), np.int32)
    w = np.zeros(Q, np.float64)
    lib().orc_velocities(c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(w))
    return c, w


def shell(sab: float) -> np.ndarray:
    cap = 20000
    out = np.zeros((cap, 3), np.int32)
    n = lib().orc_shell(sab, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), cap)
    return out[:n].copy()


def attraction_set(sab: float, lc: float) -> np.ndarray:
    cap = 200000
    out = np.zeros((cap, 3), np.int32)
    n = lib().orc_attraction_set(sab, lc, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), cap)
    return out[:n].copy()


def bmcsl(sa, sb, xi2, xi3) -> float:
    return lib().orc_bmcsl(sa, sb, xi2, xi3)


def _N(lat):
    nx, ny, nz = lat.shape
    return nx * ny * nz


def init(lat, n, u=None):
    """f := psi_perp(n, u) (R10).  n: [S][N]; u: [S][3][N] or None."""
    S, N = len(lat.sigma), _N(lat)
    n = np.ascontiguousarray(n, np.float64).reshape(S, N)
    uu = None if u is None else np.ascontiguousarray(u, np.float64).reshape(S, 3, N)
    f = np.zeros((S, Q, N), np.float64)
    p = params(lat)
    rc = lib().orc_init(ctypes.byref(p), _dp(n), _dp(uu), _dp(f))
    if rc != 0:
        raise RuntimeError("orc_init failed")
    return f


def step(lat, f, nsteps: int, fext=None):
    """Advance f in place by nsteps.  Returns the oracle status (0 ok, 1 xi3 >= 1)."""
    S, N = len(lat.sigma), _N(lat)
    assert f.shape == (S, Q, N) and f.dtype == np.float64 and f.flags.c_contiguous
    fe = None if fext is None else np.ascontiguousarray(fext, np.float64).reshape(S, 3, N)
    p = params(lat)
    return lib().orc_step(ctypes.byref(p), _dp(f), _dp(fe), int(nsteps))


def moments(lat, f):
    S, N = len(lat.sigma), _N(lat)
    n = np.zeros((S, N))
    j = np.zeros((S, 3, N))
    p = params(lat)
    lib().orc_moments(ctypes.byref(p), _dp(np.ascontiguousarray(f)), _dp(n), _dp(j))
    return n, j


def gfield(lat, n):
    S, N = len(lat.sigma), _N(lat)
    g = np.zeros((S, S, N))
    xi = np.zeros((2, N))
    p = params(lat)
    bad = lib().orc_gfield(ctypes.byref(p), _dp(np.ascontiguousarray(n, np.float64)), _dp(g), _dp(xi))
    return g, xi, bool(bad)


def forces(lat, n, j, g=None):
    """Phi and its parts (hard core, velocity exchange, attraction): each [S][3][N]."""
    S, N = len(lat.sigma), _N(lat)
    n = np.ascontiguousarray(n, np.float64).reshape(S, N)
    j = np.ascontiguousarray(j, np.float64).reshape(S, 3, N)
    if g is None:
        g, _, _ = gfield(lat, n)
    phi, hc, vx, at = (np.zeros((S, 3, N)) for _ in range(4))
    p = params(lat)
    lib().orc_forces(ctypes.byref(p), _dp(n), _dp(j), _dp(np.ascontiguousarray(g)),
                     _dp(phi), _dp(hc), _dp(vx), _dp(at))
    return phi, hc, vx, at


def forces_sites(lat, n, j, g, sites):
    """Phi at the listed sites only: returns [S][3][len(sites)]."""
    S, N = len(lat.sigma), _N(lat)
    sites = np.ascontiguousarray(sites, np.int64)
    M = len(sites)
    phi = np.zeros((S, 3, M))
    p = params(lat)
    lib().orc_forces_sites(ctypes.byref(p), _dp(np.ascontiguousarray(n, np.float64)),
                           _dp(np.ascontiguousarray(j, np.float64)), _dp(np.ascontiguousarray(g, np.float64)),
                           M, sites.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                           _dp(phi), None, None, None)
    return phi


def accel(lat, n, j, g=None, fext=None, sites=None, want_ustar=False):
    """Acceleration (Phi + F_ext)/m that one step applies (R8'): [S][3][M].

    sites=None: every site (M = N); otherwise only the listed sites."""
    S, N = len(lat.sigma), _N(lat)
    n = np.ascontiguousarray(n, np.float64).reshape(S, N)
    j = np.ascontiguousarray(j, np.float64).reshape(S, 3, N)
    if g is None:
        g, _, _ = gfield(lat, n)
    fe = None if fext is None else np.ascontiguousarray(fext, np.float64).reshape(S, 3, N)
    if sites is None:
        M, sp = N, None
    else:
        sites = np.ascontiguousarray(sites, np.int64)
        M, sp = len(sites), sites.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    acc = np.zeros((S, 3, M))
    ust = np.zeros((S, 3, N)) if want_ustar else None
    p = params(lat)
    lib().orc_accel_sites(ctypes.byref(p), _dp(n), _dp(j), _dp(np.ascontiguousarray(g)), _dp(fe),
                          M if sites is not None else 0, sp, _dp(acc), _dp(ust))
    return (acc, ust) if want_ustar else acc


def collide_local(lat, f, n, j, acc):
    """Post-collision populations from site-local data.

    f [M][S][19], n [M][S], j [M][S][3], acc [M][S][3] accelerations.
    """
    S = len(lat.sigma)
    f = np.ascontiguousarray(f, np.float64)
    M = f.shape[0]
    out = np.zeros((M, S, Q))
    p = params(lat)
    lib().orc_collide_local(ctypes.byref(p), M, _dp(f), _dp(np.ascontiguousarray(n, np.float64)),
                            _dp(np.ascontiguousarray(j, np.float64)),
                            _dp(np.ascontiguousarray(acc, np.float64)), _dp(out))
    return out


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops from now on."""
    lib().orc_set_num_threads(int(n))


def velocity_fields(lat, n, j):
    """Species velocities (R1): u^a = j^a / n^a, and the barycentric velocity
    u = sum_a m^a j^a / sum_a m^a n^a where n^a vanishes.  [S][3][N]."""
    m = np.asarray(lat.mass, np.float64)
    rho = np.einsum("a,an->n", m, n)
    with np.errstate(divide="ignore", invalid="ignore"):
        ub = np.where(rho > 0, np.einsum("a,akn->kn", m, j) / rho, 0.0)
        u = np.where(n[:, None, :] > 1e-300, j / n[:, None, :], ub[None, :, :])
    return u


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
