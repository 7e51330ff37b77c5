"""The FP64 reference network's hand-written gradient against central
finite differences (it is what the GPU training kernels are checked against)."""
import numpy as np

import net_reference as R


def test_param_count_matches_the_abi_layout():
    assert R.NPARAM == 27 * 32 * 2 + 32 + 27 * 32 * 32 + 32 + 6 * 32 + 6


def test_gradient_is_finite_differences():
    rng = np.random.default_rng(3)
    p = R.random_params(5)
    x = rng.normal(0, 1, (4, 5, 6, 2))
    t = rng.normal(0, 1, (4, 5, 6, 6))
    loss, g = R.loss_and_grad(p, x, t)
    idx = np.concatenate([rng.choice(R.NPARAM, 60, replace=False), [0, 1727, 1759, 29439, 29471, R.NPARAM - 1]])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (R.loss_and_grad(pp, x, t)[0] - R.loss_and_grad(pm, x, t)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 * max(1.0, abs(fd)) + 1e-8, (i, fd, g[i])


def test_taps_read_the_periodic_neighbour():
    X = np.arange(4 * 5 * 6, dtype=float).reshape(4, 5, 6, 1)
    # tap (dz, dy, dx) = (1, -1, 1): value at (z+1, y-1, x+1)
    t = R.TAPS.index((1, -1, 1))
    S = R.shifted(X, R.TAPS[t])
    assert S[0, 0, 0, 0] == X[1, 4, 1, 0]
    assert S[3, 2, 5, 0] == X[0, 1, 0, 0]


def test_forward_at_sampled_sites_equals_the_whole_field():
    rng = np.random.default_rng(8)
    p = R.random_params(9)
    x = rng.normal(0, 1, (5, 6, 7, 2))
    full, _ = R.forward(p, x)
    sites = [(0, 0, 0), (4, 5, 6), (2, 3, 1), (1, 5, 0)]
    at = R.forward_at(p, x, sites)
    for k, (z, y, xx) in enumerate(sites):
        assert np.allclose(at[k], full[z, y, xx], rtol=1e-12, atol=1e-12)
