"""The seeded ensemble workloads: sizes, packing and shear ranges, and the
linear stability of their densest uniform members (the linearised lattice
step of tests/linear_model.py, one predictor sweep as the library runs)."""
import math

import numpy as np
import pytest

import linear_model as LM
from paper_1105_3634_gb300 import workloads as W


def _ranges(systems):
    L = [lat.shape[0] for lat, _ in systems]
    shear = [lat.wall_u_hi[0] if lat.wall_axis == 1 else 0.0 for lat, _ in systems]
    return L, shear


def test_ensembles_span_the_stated_ranges():
    for systems, sig, pk_max in ((W.ensemble(64), [1.0, 1.5], 0.20),
                                 (W.ensemble_attraction(64), [2.0, 3.0], 0.30)):
        assert len(systems) == 64
        L, shear = _ranges(systems)
        assert set(L) <= set(range(32, 129, 8)) and min(L) <= 40 and max(L) >= 120
        assert all(lat.shape == (l, l, l) for (lat, _), l in zip(systems, L))
        assert max(shear) <= 0.05 and sum(1 for u in shear if u > 0) > 32
        for lat, n in systems:
            assert lat.sigma == sig
            xi3 = math.pi / 6 * sum(n[a].mean() * s ** 3 for a, s in enumerate(sig))
            assert 0.05 - 1e-9 <= xi3 <= pk_max + 1e-9
    att = W.ensemble_attraction(4, meanfield="fp32")
    assert all(lat.meanfield == "fp32" and lat.eps is not None for lat, _ in att)


@pytest.mark.parametrize("sweeps", [1])
def test_densest_attraction_member_is_linearly_stable(sweeps):
    """sigma = 2/3 with the tails at packing 0.30 (the range's top): no wave
    vector grows under the linearised step."""
    lat = W.ensemble_attraction(1)[0][0]
    lat = W.Lattice(shape=(32, 32, 32), sigma=lat.sigma, eps=lat.eps, lambda_c=lat.lambda_c)
    n0 = W.densities_from_packing(0.30, lat.sigma, [0.5, 0.5])
    worst = 0.0
    for q in ([0.3, 0, 0], [math.pi / 2, 0, 0], [math.pi, 0, 0], [math.pi, math.pi, 0], [1.0, 0.5, 0.25]):
        Lm, _, _ = LM.operator(lat, n0, np.array(q, float), sweeps=sweeps)
        worst = max(worst, float(np.abs(np.linalg.eigvals(Lm)).max()))
    assert worst < 1.0 + 1e-9, worst
