"""Training and checking the learned hard-core force (mlb_net) on frames the
exact method generates.

A frame is a state of the benchmark mixture (sigma = 1/1.5, packing 0.2) on a
periodic lattice: a smooth Gaussian random concentration field (Fourier
modes with a Gaussian envelope of random correlation length), an independent
total-density field of random relative weight, in some frames lattice-scale
noise, with an rms amplitude drawn log-uniformly over a decade, then evolved a
random number of exact steps (biased to the early, out-of-mechanical-
equilibrium transient, where the force is largest).  Its input is n - n_ref (the context's own
reference densities, exactly what the step feeds the network) and its target
the exact hard-core force (mlb_get_rest_force; no tails, no external force).
Training runs Adam on the relative squared force error on the GPU through
mlb_net_train, so that every amplitude weighs the same; everything here is
host-side orchestration.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np

from . import workloads as W

Frame = Tuple[np.ndarray, np.ndarray]        # (dn [2][N], F [2][3][N])


def benchmark_lattice(shape) -> W.Lattice:
    return W.Lattice(shape=tuple(shape), sigma=[1.0, 1.5], tau=1.0)


def smooth_field(shape, seed: int, corr: float) -> np.ndarray:
    """Gaussian random field of unit rms on the periodic lattice `shape`
    (x fastest, flattened), spectrum exp(-|q|^2 corr^2 / 2), q = 2 pi m / L."""
    nx, ny, nz = shape
    q2 = sum(np.meshgrid(*[(2.0 * math.pi * np.fft.fftfreq(n)) ** 2 for n in (nz, ny, nx)], indexing="ij"))
    env = np.exp(-0.25 * q2 * corr * corr)           # amplitude: the square root of the power spectrum
    env[0, 0, 0] = 0.0
    u = W.uniform01(seed, 2 * env.size).reshape(2, *env.shape)
    c = env * np.sqrt(-2.0 * np.log(np.maximum(u[0], 1e-300))) * np.exp(2j * math.pi * u[1])
    f = np.real(np.fft.ifftn(c)).reshape(-1)
    return f / max(float(np.sqrt(np.mean(f * f))), 1e-300)


def frames(mlb, shape, count: int, seed: int, amp_min: float = 0.003, amp_max: float = 0.05,
           steps_max: int = 300, noisy: float = 0.25, noise_max: float = 0.1) -> List[Frame]:
    lat = benchmark_lattice(shape)
    n0 = W.densities_from_packing(0.2, lat.sigma, [0.5, 0.5])
    r = W.uniform01(seed, count * 8).reshape(count, 8)
    sim = mlb.Simulation(lat)
    out = []
    for k in range(count):
        amp = amp_min * (amp_max / amp_min) ** r[k, 0]
        wc = smooth_field(lat.shape, seed * 100003 + 3 * k, 1.0 + 5.0 * r[k, 1])
        wt = smooth_field(lat.shape, seed * 100003 + 3 * k + 1, 1.0 + 5.0 * r[k, 2])
        rel = np.zeros((2, lat.nsites))
        if r[k, 3] < noisy:
            rel = W.noise(lat, [1.0, 1.0], math.sqrt(3.0) * noise_max * r[k, 4], seed=seed * 100003 + 3 * k + 2) - 1.0
        n = np.empty((2, lat.nsites))
        t = r[k, 5]
        n[0] = n0[0] * (1.0 + amp * (wc + t * wt + rel[0]))
        n[1] = n0[1] * (1.0 + amp * (-wc + t * wt + rel[1]))
        sim.set_fields(n)
        sim.step(int(r[k, 6] ** 2 * steps_max))     # half the frames within the first quarter
        nn, _ = sim.moments()
        _, nref, _ = sim.populations()
        out.append((nn - nref[:, None], sim.rest_force()))
    sim.close()
    return out


def scales(data: Sequence[Frame], in_gain: float = 0.3):
    """in_scale_a = in_gain / rms(n^a - n_ref^a), out_scale_a = 1 / rms(F^a)
    over the frames.  A gain below one keeps the hidden units near the linear
    part of tanh, where the force (linear in dn at small amplitude) lives."""
    dn = np.stack([f[0] for f in data])
    F = np.stack([f[1] for f in data])
    ins = [in_gain / float(np.sqrt(np.mean(dn[:, a] ** 2))) for a in range(2)]
    outs = [1.0 / float(np.sqrt(np.mean(F[:, a] ** 2))) for a in range(2)]
    return ins, outs


def train(net, data: Sequence[Frame], epochs: int = 200, lr0: float = 1e-3, lr_min: float = 1e-5,
          iters: int = 1) -> List[float]:
    """Cosine-decayed Adam over the frames; returns the mean loss (squared
    relative force error) per epoch."""
    hist = []
    for e in range(epochs):
        lr = lr_min + 0.5 * (lr0 - lr_min) * (1.0 + math.cos(math.pi * e / max(1, epochs - 1)))
        hist.append(float(np.mean([net.train(dn, F, iters, lr) for dn, F in data])))
    return hist


def force_error(net, data: Sequence[Frame]) -> float:
    """Relative 2-norm error of the network's force over all the frames together."""
    num = den = 0.0
    for dn, F in data:
        d = net.forward(dn) - F
        num += float(np.sum(d * d))
        den += float(np.sum(F * F))
    return math.sqrt(num / den)


def frame_errors(net, data: Sequence[Frame]) -> np.ndarray:
    """Relative 2-norm error of the network's force, frame by frame."""
    return np.array([float(np.linalg.norm(net.forward(dn) - F) / np.linalg.norm(F)) for dn, F in data])


def initial_params(seed: int = 7) -> np.ndarray:
    """He-type initial weights (zero biases) in the mlb_net parameter layout."""
    r = W.uniform01(seed, 29638)
    u = 2.0 * r - 1.0                                   # uniform (-1, 1): variance 1/3
    p = np.zeros(29638)
    for off, n, fan_in in _WEIGHTS:
        p[off:off + n] = u[off:off + n] * math.sqrt(3.0 * 2.0 / fan_in)
    return p.astype(np.float32)


# (offset, size, fan-in) of W1, W2, W3 in the parameter layout
# W1[27][32][2] b1[32] W2[27][32][32] b2[32] W3[6][32] b3[6]
_OFF_W1, _OFF_W2, _OFF_W3 = 0, 27 * 32 * 2 + 32, 27 * 32 * 2 + 32 + 27 * 32 * 32 + 32
_WEIGHTS = [(_OFF_W1, 27 * 32 * 2, 27 * 2), (_OFF_W2, 27 * 32 * 32, 27 * 32), (_OFF_W3, 6 * 32, 32)]


def _taps(x: np.ndarray, shape) -> np.ndarray:
    """[2][N] -> [N][27 * 2]: the 3^3 periodic neighbourhood of every site,
    tap = (dz+1)*9 + (dy+1)*3 + (dx+1) reading (x+dx, y+dy, z+dz), channel fastest."""
    nx, ny, nz = shape
    X = x.reshape(2, nz, ny, nx)
    cols = []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                v = np.roll(X, (-dz, -dy, -dx), axis=(1, 2, 3)).reshape(2, -1)
                cols.extend([v[0], v[1]])
    return np.stack(cols, 1)


def max_scaled_force(data: Sequence[Frame], out_scale) -> float:
    return max(float(np.max(np.abs(F * np.asarray(out_scale)[:, None, None]))) for _, F in data)


def linear_stencil(data: Sequence[Frame], shape, in_scale, out_scale) -> np.ndarray:
    """Least-squares 3^3 linear stencil S[27][6][2] from the scaled input
    x = dn in_scale to the scaled force t = F out_scale, every frame weighted
    by 1/|F|^2 (the relative error, as in training): the linear response of
    the hard-core force, which the frames' small amplitudes make dominant."""
    AtA = np.zeros((54, 54))
    AtB = np.zeros((54, 6))
    for dn, F in data:
        A = _taps(dn * np.asarray(in_scale)[:, None], shape)
        B = (F * np.asarray(out_scale)[:, None, None]).reshape(6, -1).T
        w = 1.0 / float(np.sum(B * B))
        AtA += w * (A.T @ A)
        AtB += w * (A.T @ B)
    sol = np.linalg.solve(AtA + 1e-12 * np.trace(AtA) / 54 * np.eye(54), AtB)   # [27*2][6]
    return sol.reshape(27, 2, 6).transpose(0, 2, 1)


def stencil_params(S: np.ndarray, t_max: float, pre_max: float = 0.1, noise: float = 0.01,
                   seed: int = 7) -> np.ndarray:
    """Parameters whose response is the stencil S[27][6][2] up to tanh's
    curvature: hidden unit o < 6 of layer 1 is eps (S x)_o (the stencil in
    FP32, on the input), passed through layer 2 by its centre tap and read out
    by layer 3 with 1/eps^2, where eps = pre_max / t_max keeps every
    pre-activation below pre_max for scaled forces up to t_max
    (tanh(v) = v (1 - v^2/3 + ...): a relative error below pre_max^2 / 3 per
    layer).  The other 26 hidden units start as small random weights (the
    room for the nonlinear correction); biases are zero."""
    eps = pre_max / t_max
    p = initial_params(seed).astype(np.float64)
    W1 = p[_OFF_W1:_OFF_W1 + 27 * 32 * 2].reshape(27, 32, 2) * noise
    W2 = p[_OFF_W2:_OFF_W2 + 27 * 32 * 32].reshape(27, 32, 32) * noise
    W3 = np.zeros((6, 32))
    W1[:, :6, :] = eps * S
    W2[:, :6, :] = 0.0
    W2[:, :, :6] = 0.0
    W2[13, np.arange(6), np.arange(6)] = eps
    W3[np.arange(6), np.arange(6)] = 1.0 / (eps * eps)
    p[:] = 0.0
    p[_OFF_W1:_OFF_W1 + W1.size] = W1.reshape(-1)
    p[_OFF_W2:_OFF_W2 + W2.size] = W2.reshape(-1)
    p[_OFF_W3:_OFF_W3 + W3.size] = W3.reshape(-1)
    return p.astype(np.float32)


def recipe(mlb, shape=(64, 8, 8), count: int = 240, seed: int = 21, epochs: int = 100, lr0: float = 1e-6):
    """The production recipe: frames on `shape`, scales, the least-squares
    linear-response stencil as the start, `epochs` of GPU fine-tuning.
    Returns (params, in_scale, out_scale, frames).  The parameters serve any
    lattice size (the network is a convolution)."""
    data = frames(mlb, shape, count, seed)
    ins, outs = scales(data)
    p0 = stencil_params(linear_stencil(data, shape, ins, outs), max_scaled_force(data, outs))
    net = mlb.Net(shape)
    net.set_params(p0)
    net.set_scales(ins, outs)
    train(net, data, epochs=epochs, lr0=lr0, lr_min=lr0 / 100, iters=1)
    p = net.params()
    net.close()
    return p, ins, outs, data


def time_forward(mlb, shape, reps: int = 3, seed: int = 13) -> float:
    """Milliseconds per network forward (host input staged, force read back)
    on a lattice of `shape` with He-type random weights and a random input:
    the kernels' cost does not depend on the values."""
    import time
    net = mlb.Net(shape)
    net.set_params(initial_params(seed))
    net.set_scales([100.0, 100.0], [100.0, 100.0])
    N = shape[0] * shape[1] * shape[2]
    dn = (W.uniform01(seed, 2 * N).reshape(2, N) - 0.5) * 0.01
    net.forward(dn)
    t0 = time.perf_counter()
    for _ in range(reps):
        net.forward(dn)
    dt = (time.perf_counter() - t0) / reps
    net.close()
    return dt * 1e3


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser(description="time the surrogate network's forward on an n^3 lattice")
    ap.add_argument("--size", type=int, default=128)
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args()
    from . import build as _build
    _build.build()
    from . import mlb as _mlb
    print(f"forward {a.size}^3: {time_forward(_mlb, (a.size,) * 3, a.reps):.3f} ms (host staging included)")
