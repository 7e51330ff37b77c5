"""Taylor dispersion between moving walls (the channel of the Taylor
workload, binary benchmark physics) on the FP64 oracle.  Hard spheres layer
at the bounce-back walls (first layer ~1.44 x the bulk density, the interior
depleted), so the channel has its own D(0) and the flow next to the walls
lags them (u_x ~ 0.64 U in the first layer, not the ideal Couette 0.94 U).
With that D(0) and the measured section-averaged u_x(y), the decay rate of a
long concentration wave is the exact passive-scalar rate of the channel to a
fraction of a percent; the ideal Taylor-Aris value D + U^2 h^2 / (30 D) is
reported, not asserted."""
import math

import numpy as np

from paper_1105_3634_gb300 import taylor as T
from paper_1105_3634_gb300 import workloads as W

H, L = 16, 128


def _run(orc, U):
    lat = W.Lattice(shape=(L, H, 2), sigma=[1.0, 1.5], tau=1.0, wall_axis=1, wall_u_lo=(-U, 0.0, 0.0),
                    wall_u_hi=(U, 0.0, 0.0))
    n0 = W.densities_from_packing(0.2, lat.sigma, [0.5, 0.5])
    y = W.coordinate(lat, 1)
    u = np.zeros((2, 3, lat.nsites))
    u[:, 0, :] = (U * (2 * (y + 0.5) / H - 1))[None, :]
    f = orc.init(lat, W.sine_wave(lat, n0, 0.01), u)
    ts, amps, profiles = [], [], []
    t = 0
    for target in range(600, 3001, 200):
        orc.step(lat, f, target - t)
        t = target
        n, j = orc.moments(lat, f)
        ts.append(t)
        amps.append(abs(T._mode(lat, n[0] / n.sum(0), 0)))
        profiles.append((j.sum(0)[0] / n.sum(0)).reshape(2, H, L).mean((0, 2)))
    kx = 2 * math.pi / L
    return float(-np.polyfit(ts, np.log(amps), 1)[0]) / kx ** 2, np.mean(profiles, 0)


def test_couette_channel_dispersion_is_the_passive_scalar_rate_of_its_own_flow(orc):
    D0, _ = _run(orc, 0.0)
    U = 0.03
    Deff, uy = _run(orc, U)
    kx = 2 * math.pi / L
    ideal = U * (2 * (np.arange(H) + 0.5) / H - 1)
    exact = T.passive_scalar_rate_channel(D0, uy, kx)
    print(f"channel D(0) {D0:.5f}; U {U}: D_eff {Deff:.5f}, passive scalar with the measured u_x(y) {exact:.5f} "
          f"({(Deff - exact) / exact:+.2e}); first layer u_x / U {uy[-1] / U:.3f}; ideal Couette "
          f"{T.passive_scalar_rate_channel(D0, ideal, kx):.5f}; Taylor-Aris {T.taylor_aris_couette(D0, U, H):.5f}")
    assert abs(Deff - exact) < 5e-3 * exact
    assert Deff > D0 * 1.02                                   # the flow does disperse
    assert 0.5 < uy[-1] / U < 0.8                             # the wall layer lags the wall
