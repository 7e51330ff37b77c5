"""Host logic of the surrogate's training recipe: the least-squares linear
stencil recovers a stencil that generated the frames, and the parameters
built from a stencil reproduce it through the FP64 reference network."""
import numpy as np

import net_reference as R
from paper_1105_3634_gb300 import surrogate as SG
from paper_1105_3634_gb300 import workloads as W

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


def test_stencil_start_reproduces_the_oracles_hard_core_force(orc):
    """The surrogate's physics target is Eq. potmeanforce's hard-core term.
    Frames of the benchmark mixture built here, with the FP64 oracle's F^hc,
    give the least-squares stencil; the network started from it (evaluated
    by the FP64 reference network) reproduces the oracle's F^hc on held-out
    frames to 0.2 % at amplitude 0.2 % and 0.7 % at 1 %: the remainder grows
    with the amplitude (the force's quadratic part, left to the training)."""
    shape = (12, 6, 6)
    lat = W.Lattice(shape=shape, sigma=[1.0, 1.5], tau=1.0)
    n0 = W.densities_from_packing(0.2, lat.sigma, [0.5, 0.5])
    N = lat.nsites

    def frame(seed, amp):
        wc = SG.smooth_field(shape, seed, 2.0)
        wt = SG.smooth_field(shape, seed + 1, 3.0)
        n = np.stack([n0[0] * (1 + amp * (wc + 0.5 * wt)), n0[1] * (1 + amp * (-wc + 0.5 * wt))])
        _, hc, _, _ = orc.forces(lat, n, np.zeros((2, 3, N)))
        return n - n.mean(1, keepdims=True), hc

    train = [frame(100 + 3 * k, 0.002 + 0.004 * (k % 5)) for k in range(30)]
    ins, outs = SG.scales(train)
    p = SG.stencil_params(SG.linear_stencil(train, shape, ins, outs), SG.max_scaled_force(train, outs))

    def worst(amp):
        errs = []
        for k in range(5):
            dn, F = frame(500 + 3 * k, amp)
            x, _ = R.fields(shape, dn, F, ins, outs)
            o, _ = R.forward(p.astype(np.float64), x)
            got = np.stack([o[..., c].reshape(-1) for c in range(6)]).reshape(2, 3, N) / np.array(outs)[:, None, None]
            errs.append(np.linalg.norm(got - F) / np.linalg.norm(F))
        return max(errs)

    e_small, e_large = worst(0.002), worst(0.01)
    print(f"held-out relative error against the oracle's F^hc: {e_small:.2e} at amplitude 0.2 %, "
          f"{e_large:.2e} at 1 % (the force's quadratic part, which a linear stencil leaves out)")
    assert e_small < 2e-3 and e_large < 1.5e-2
    assert e_large > 2 * e_small
