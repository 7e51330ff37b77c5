"""Host logic of the surrogate's training recipe: the least-squares linear
stencil recovers a stencil that generated the frames, and the parameters
built from a stencil reproduce it through the FP64 reference network."""
import numpy as np

import net_reference as R
from paper_1105_3634_gb300 import surrogate as SG

SHAPE = (6, 5, 4)                    # (nx, ny, nz)
N = SHAPE[0] * SHAPE[1] * SHAPE[2]


def _apply(S, x):
    """t [6][N] = sum_tap S[tap] x(r + tap), x [2][N], straight from the definition."""
    nx, ny, nz = SHAPE
    X = x.reshape(2, nz, ny, nx)
    t = np.zeros((6, nz, ny, nx))
    for tap, (dz, dy, dx) in enumerate(R.TAPS):
        for z in range(nz):
            for y in range(ny):
                for xx in range(nx):
                    v = X[:, (z + dz) % nz, (y + dy) % ny, (xx + dx) % nx]
                    t[:, z, y, xx] += S[tap] @ v
    return t.reshape(6, N)


def test_taps_order_matches_the_network_layout():
    x = np.arange(2 * N, dtype=float).reshape(2, N)
    A = SG._taps(x, SHAPE)
    X = x.reshape(2, SHAPE[2], SHAPE[1], SHAPE[0])
    for tap, (dz, dy, dx) in enumerate(R.TAPS):
        for c in range(2):
            assert A[0, 2 * tap + c] == X[c, dz % SHAPE[2], dy % SHAPE[1], dx % SHAPE[0]]


def test_linear_stencil_recovers_the_generating_stencil():
    rng = np.random.default_rng(4)
    S = rng.normal(0, 1, (27, 6, 2))
    ins, outs = [3.0, 0.5], [2.0, 7.0]
    data = []
    for k in range(6):
        dn = rng.normal(0, 1, (2, N))
        t = _apply(S, dn * np.array(ins)[:, None])
        F = t.reshape(2, 3, N) / np.array(outs)[:, None, None]
        data.append((dn, F))
    got = SG.linear_stencil(data, SHAPE, ins, outs)
    assert np.allclose(got, S, rtol=0, atol=1e-8)


def test_stencil_parameters_reproduce_the_stencil():
    rng = np.random.default_rng(5)
    S = rng.normal(0, 1, (27, 6, 2))
    x = rng.normal(0, 0.3, (2, N))
    t = _apply(S, x)
    t_max = float(np.abs(t).max())
    p = SG.stencil_params(S, t_max, pre_max=0.01).astype(np.float64)
    X = np.stack([x[c].reshape(SHAPE[2], SHAPE[1], SHAPE[0]) for c in range(2)], -1)
    out, _ = R.forward(p, X)
    got = np.stack([out[..., o].reshape(-1) for o in range(6)])
    # tanh(v) = v (1 - v^2/3 + ...) with |v| <= 0.01 on each of two layers
    assert np.linalg.norm(got - t) / np.linalg.norm(t) < 1e-4
    P = R.unpack(p)
    assert not P["b1"].any() and not P["b2"].any() and not P["b3"].any()


def test_smooth_training_fields():
    """The training frames' random fields: unit rms, zero mean, the same for
    the same seed, and a spectrum falling off as exp(-q^2 corr^2 / 2)."""
    shape = (32, 8, 8)
    f = SG.smooth_field(shape, 3, 3.0)
    assert f.shape == (32 * 8 * 8,)
    assert abs(np.sqrt(np.mean(f * f)) - 1.0) < 1e-12 and abs(f.mean()) < 1e-12
    assert np.array_equal(f, SG.smooth_field(shape, 3, 3.0))
    assert not np.array_equal(f, SG.smooth_field(shape, 4, 3.0))
    # power at the lattice scale against the longest waves, for a long and a short correlation
    def ratio(corr):
        p = np.zeros(2)
        for seed in range(20):
            F = np.abs(np.fft.fftn(SG.smooth_field(shape, seed, corr).reshape(8, 8, 32))) ** 2
            p += [F[0, 0, 1:3].sum(), F[4, 4, 12:20].sum()]
        return p[1] / p[0]
    assert ratio(3.0) < 1e-6 < ratio(0.5)
