"""Linear stability of the half-force shift's predictor (reading R8') on the
benchmark spheres sigma = 1/1.5: the largest one-step growth factor of the
linearised lattice step over wave vectors, with one Jacobi sweep of
u* = u + a(u*)/2 (the method), with three, and with the half step solved
exactly.  One sweep limits the uniform mixture to packing ~0.2; three sweeps
reach the exact half step's limit, which lies between 0.3 and 0.35."""
import math

import numpy as np
import pytest

import linear_model as LM
from paper_1105_3634_gb300 import workloads as W


def _max_growth(packing, scheme, sweeps=1, sigma=(1.0, 1.5)):
    lat = W.Lattice(shape=(8, 8, 8), sigma=list(sigma), tau=1.0, force_scheme=scheme)
    n0 = W.densities_from_packing(packing, list(sigma), [0.5, 0.5])
    worst = 0.0
    for qx in np.linspace(0.0, math.pi, 5):
        for qy in (0.0, math.pi / 2, math.pi):
            for qz in (0.0, math.pi):
                Lm, _, _ = LM.operator(lat, n0, np.array([qx, qy, qz]), sweeps=sweeps)
                worst = max(worst, float(np.abs(np.linalg.eigvals(Lm)).max()))
    return worst


def test_one_sweep_is_stable_at_the_benchmark_packing():
    assert _max_growth(0.2, "semi_implicit") < 1.0 + 1e-9


@pytest.mark.parametrize("packing", [0.25, 0.3])
def test_three_sweeps_or_the_exact_half_step_stabilise_denser_mixtures(packing):
    assert _max_growth(packing, "semi_implicit", sweeps=1) > 1.01
    assert _max_growth(packing, "semi_implicit", sweeps=3) < 1.0 + 1e-9
    assert _max_growth(packing, "implicit_coupled") < 1.0 + 1e-9


def test_the_exact_half_step_is_unstable_at_packing_035():
    assert _max_growth(0.35, "implicit_coupled") > 1.05
