"""Linearised one-step operator of the lattice method about a uniform rest state.

Written from the paper's equations, independently of the oracle, as a pin for
it.  About the state n^a = n0^a, u = 0, a plane-wave perturbation
delta f^a_i(r) = x^a_i exp(i q.r) evolves by x -> L(q) x with

  moments      dn^a = sum_i x^a_i,   dj^a = sum_i c_i x^a_i             (Eq. colonna)
  contact g    dg_ab = sum_c dg_ab/dn-bar^c  B_c(q) dn^c                 (smoothing ball B_c)
  hard core    -kT s_ab^2 w_ab V_ab(q) [ n0^b dg_ab / 2 + g_ab dn^b ]    (Eq. potmeanforce)
  velocities   K_ab w_ab g_ab n0^b [ T_ab(q) du^b - T_ab(0) du^a ]       (Eqs. gammaab, viscousforce)
  attraction   A_ab(q) dn^b                                              (G term of Eq. potmeanforce)
  collision    (1 - omega) x + omega w_i (dn + c_i.dj/cs2) + w_i n0 c_i.dPhi/(m cs2)
  streaming    x_i -> exp(-i q.c_i) x_i

With the semi-implicit half-force shift (the default time integration) the
acceleration is instead a = F_rest + gain(u*) - Gamma u* with
u* = (u + (F_rest + gain(u))/2)/(1 + Gamma/2), and the collision relaxes to
psi_perp at u + a/2 with the forcing scaled by (1 - omega/2); Gamma is the
local friction sum_b K_ab w_ab g_ab n0^b T_ab(0) and gain the neighbour part.

where V(q) = sum_d s_d e^{i q.d}, T(q) = sum_d s_d s_d^T e^{i q.d} over the
contact shell, A(q) = sum_d (-grad U)(d)... e^{i q.d} over the attraction region,
B_c(q) the mean of e^{i q.d} over the smoothing ball, w_ab = 4 pi/|S_ab| and
K_ab = 2 s_ab^2 sqrt(2 mu_ab kT / pi).
"""
import math

import numpy as np

CS2 = 1.0 / 3.0


def d3q19():
    """D3Q19 velocities listed by speed shell, with their weights."""
    c = [(0, 0, 0)]
    c += [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    c += [(1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
          (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
          (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]
    w = [1 / 3] + [1 / 18] * 6 + [1 / 36] * 12
    return np.array(c, float), np.array(w)


def _points(r_lo2, r_hi2, lo_incl=True, hi_incl=True, zero=False):
    R = int(math.ceil(math.sqrt(r_hi2))) + 1
    g = np.arange(-R, R + 1)
    d = np.array(np.meshgrid(g, g, g, indexing="ij")).reshape(3, -1).T
    q = (d ** 2).sum(1)
    keep = (q >= r_lo2) if lo_incl else (q > r_lo2)
    keep &= (q <= r_hi2) if hi_incl else (q < r_hi2)
    if not zero:
        keep &= q > 0
    return d[keep].astype(float)


def bmcsl(sa, sb, xi2, xi3):
    h = sa * sb / (sa + sb)
    o = 1 - xi3
    return 1 / o + 3 * h * xi2 / o ** 2 + 2 * h * h * xi2 ** 2 / o ** 3


def bmcsl_grad(sa, sb, xi2, xi3):
    """(dg/dxi2, dg/dxi3) of the BMCSL contact value."""
    h = sa * sb / (sa + sb)
    o = 1 - xi3
    return (3 * h / o ** 2 + 4 * h * h * xi2 / o ** 3,
            1 / o ** 2 + 6 * h * xi2 / o ** 3 + 6 * h * h * xi2 ** 2 / o ** 4)


def operator(lat, n0, q, scheme=None, sweeps=None):
    """L(q) as a (19 S) x (19 S) complex matrix, index a*19 + i.

    scheme: 'explicit' or 'semi_implicit' (default: lat.force_scheme), or
    'implicit_coupled': the half-force shift with u* = u + a(u*)/2 solved
    exactly, every species' u* and the partners' together (the method's
    semi-implicit scheme takes one Jacobi sweep of it, partners held at u;
    sweeps > 1 repeats the sweep with the partners' u* of the previous one).
    """
    if scheme is None:
        scheme = lat.force_scheme
    if sweeps is None:
        sweeps = getattr(lat, "predictor_sweeps", 1)
    c, w = d3q19()
    S = lat.nspecies
    Qn = 19
    q = np.asarray(q, float)
    sig = np.asarray(lat.sigma, float)
    m = np.asarray(lat.mass, float)
    kT = lat.kT
    omega = 1.0 / lat.tau
    n0 = np.asarray(n0, float)
    rho0 = float(np.dot(m, n0))
    xi2 = math.pi / 6 * float(np.dot(n0, sig ** 2))
    xi3 = math.pi / 6 * float(np.dot(n0, sig ** 3))
    dim = S * Qn

    # linear maps from the state to moment perturbations
    Dn = np.zeros((S, dim), complex)
    Dj = np.zeros((S, 3, dim), complex)
    for a in range(S):
        Dn[a, a * Qn:(a + 1) * Qn] = 1.0
        Dj[a, :, a * Qn:(a + 1) * Qn] = c.T
    Du = Dj / n0[:, None, None]                       # species velocity perturbations

    # smoothed densities and contact values
    B = np.zeros(S, complex)
    for cc in range(S):
        d = _points(0, (lat.kappa * sig[cc]) ** 2, zero=True)
        B[cc] = np.exp(1j * d @ q).mean()
    Dg = np.zeros((S, S, dim), complex)
    g0 = np.zeros((S, S))
    for a in range(S):
        for b in range(S):
            g0[a, b] = bmcsl(sig[a], sig[b], xi2, xi3)
            d2, d3 = bmcsl_grad(sig[a], sig[b], xi2, xi3)
            for cc in range(S):
                coef = d2 * math.pi / 6 * sig[cc] ** 2 + d3 * math.pi / 6 * sig[cc] ** 3
                Dg[a, b] += coef * B[cc] * Dn[cc]

    # effective field perturbation, per species
    Dphi = np.zeros((S, 3, dim), complex)
    vex = []          # velocity-exchange pieces (a, b, pre, T(q), T(0))
    for a in range(S):
        for b in range(S):
            sab = 0.5 * (sig[a] + sig[b])
            lo = sab - 0.5
            d = _points(lo * lo if lo > 0 else 0.0, (sab + 0.5) ** 2, hi_incl=False)
            s = d / np.linalg.norm(d, axis=1)[:, None]
            wS = 4 * math.pi / len(d)
            ph = np.exp(1j * d @ q)
            V = (s * ph[:, None]).sum(0)
            T = np.einsum("k,ka,kb->ab", ph, s, s)
            T0 = np.einsum("ka,kb->ab", s, s)
            # hard core
            Dphi[a] += -kT * sab ** 2 * wS * V[:, None] * (0.5 * n0[b] * Dg[a, b] + g0[a, b] * Dn[b])[None, :]
            # drag + viscous (or drag only)
            mu = m[a] * m[b] / (m[a] + m[b])
            K = 2 * sab ** 2 * math.sqrt(2 * mu * kT / math.pi)
            pre = K * wS * g0[a, b] * n0[b]
            vex.append((a, b, pre, T, T0))
            if lat.drag_only:
                Dphi[a] += pre * np.einsum("ab,bk->ak", T0, Du[b] - Du[a])
            else:
                Dphi[a] += pre * (np.einsum("ab,bk->ak", T, Du[b]) - np.einsum("ab,bk->ak", T0, Du[a]))
            # attraction: -grad U(r - r') with U = -eps (sab/|x|)^6 at r' = r + d
            e = lat.eps[a][b]
            if e != 0.0:
                rc = lat.lambda_c[a][b] * sab
                dd = _points(sab * sab, rc * rc)
                r = np.linalg.norm(dd, axis=1)
                Kd = 6 * e * sab ** 6 * dd / r[:, None] ** 8
                A = (Kd * np.exp(1j * dd @ q)[:, None]).sum(0)
                Dphi[a] += A[:, None] * Dn[b][None, :]

    acc = Dphi / m[:, None, None]
    implicit = scheme in ("semi_implicit", "implicit_coupled")
    if implicit:
        # rest of the field (hard core + attraction) = Dphi minus the velocity part at u
        def vel_part(x):
            out = np.zeros_like(acc)
            for a, b, pre, T, T0 in vex:
                if lat.drag_only:
                    out[a] += pre * np.einsum("ab,bk->ak", T0, x[b] - x[a])
                else:
                    out[a] += pre * (np.einsum("ab,bk->ak", T, x[b]) - np.einsum("ab,bk->ak", T0, x[a]))
            return out
        def gain(x):
            out = np.zeros_like(acc)
            for a, b, pre, T, T0 in vex:
                out[a] += pre * np.einsum("ab,bk->ak", T0 if lat.drag_only else T, x[b])
            return out
        Gam = np.zeros(S)
        for a, b, pre, T, T0 in vex:
            Gam[a] += pre * T0[0, 0]
        Frest = Dphi - vel_part(Du)
        if scheme == "implicit_coupled":
            # (I - V / 2m) u* = u + Frest / 2m with V the velocity part as a 3S x 3S matrix
            Vm = np.zeros((3 * S, 3 * S), complex)
            for a, b, pre, T, T0 in vex:
                Vm[3 * a:3 * a + 3, 3 * b:3 * b + 3] += pre * (T0 if lat.drag_only else T)
                Vm[3 * a:3 * a + 3, 3 * a:3 * a + 3] -= pre * T0
            A = np.eye(3 * S) - Vm / (2 * np.repeat(m, 3))[:, None]
            rhs = (Du + Frest / (2 * m[:, None, None])).reshape(3 * S, dim)
            ustar = np.linalg.solve(A, rhs).reshape(S, 3, dim)
        else:
            ustar = Du
            for _ in range(sweeps):
                ustar = (Du + (Frest + gain(ustar)) / (2 * m[:, None, None])) / (1 + Gam / (2 * m))[:, None, None]
        acc = (Frest + vel_part(ustar)) / m[:, None, None]

    # collision and streaming
    L = np.zeros((dim, dim), complex)
    for a in range(S):
        for i in range(Qn):
            row = np.zeros(dim, complex)
            row[a * Qn + i] += 1 - omega
            if implicit:
                ueq = Du[a] + 0.5 * acc[a]
                row += omega * w[i] * (Dn[a] + n0[a] * (c[i] @ ueq) / CS2)
                row += (1 - 0.5 * omega) * w[i] * n0[a] * (c[i] @ acc[a]) / CS2
            else:
                row += omega * w[i] * (Dn[a] + (c[i] @ Dj[a]) / CS2)
                row += w[i] * n0[a] * (c[i] @ acc[a]) / CS2
            L[a * Qn + i] = np.exp(-1j * q @ c[i]) * row
    return L, Dn, Dj


def initial_state(lat, n0, dn_hat, du_hat):
    """Plane-wave amplitudes of f = psi_perp(n0 + dn, u = du) at first order."""
    c, w = d3q19()
    S = lat.nspecies
    x = np.zeros(S * 19, complex)
    for a in range(S):
        for i in range(19):
            x[a * 19 + i] = w[i] * (dn_hat[a] + n0[a] * (c[i] @ du_hat[a]) / CS2)
    return x
