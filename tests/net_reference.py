"""FP64 reference of the learned hard-core force network (test
infrastructure): the same layers, parameter layout and periodic taps as the
library's mlb_net, written plainly with numpy.

Parameters: W1[27][32][2] b1[32] W2[27][32][32] b2[32] W3[6][32] b3[6];
W[tap][out][in], tap = (dz+1)*9 + (dy+1)*3 + (dx+1) reads the input at
(x+dx, y+dy, z+dz) with periodic wrap.  Fields are site-major arrays of
shape (nz, ny, nx, C)."""
import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
SIZES = [("W1", (27, 32, 2)), ("b1", (32,)), ("W2", (27, 32, 32)), ("b2", (32,)), ("W3", (6, 32)), ("b3", (6,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    out, k = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(p[k:k + n], np.float64).reshape(shape)
        k += n
    return out


def pack(d):
    return np.concatenate([d[name].reshape(-1) for name, _ in SIZES])


def shifted(X, tap):
    dz, dy, dx = tap
    return np.roll(X, shift=(-dz, -dy, -dx), axis=(0, 1, 2))


def unshift(X, tap):
    dz, dy, dx = tap
    return np.roll(X, shift=(dz, dy, dx), axis=(0, 1, 2))


def act(v):
    return np.tanh(v)


def act_grad(v):
    return 1.0 - np.tanh(v) ** 2


def conv(X, W, b):
    out = np.zeros(X.shape[:3] + (W.shape[1],)) + b
    for t, tap in enumerate(TAPS):
        out += shifted(X, tap) @ W[t].T
    return out


def forward(p, x):
    P = unpack(p)
    pre1 = conv(x, P["W1"], P["b1"])
    a1 = act(pre1)
    pre2 = conv(a1, P["W2"], P["b2"])
    a2 = act(pre2)
    out = a2 @ P["W3"].T + P["b3"]
    return out, (x, pre1, a1, pre2, a2)


def forward_at(p, x, sites):
    """The network's output at the listed sites (z, y, x) only: each from
    its 5^3 periodic patch of x (shape (nz, ny, nx, C)), by valid
    convolutions of the same taps.  Returns (len(sites), 6)."""
    P = unpack(p)
    nz, ny, nx = x.shape[:3]
    out = []
    for z, y, xx in sites:
        patch = x[np.ix_([(z + k) % nz for k in range(-2, 3)], [(y + k) % ny for k in range(-2, 3)],
                         [(xx + k) % nx for k in range(-2, 3)])]          # (5, 5, 5, C), centre (2, 2, 2)
        pre1 = np.zeros((3, 3, 3, P["W1"].shape[1])) + P["b1"]
        for t, (dz, dy, dx) in enumerate(TAPS):
            pre1 += patch[1 + dz:4 + dz, 1 + dy:4 + dy, 1 + dx:4 + dx] @ P["W1"][t].T
        a1 = act(pre1)
        pre2 = P["b2"].copy()
        for t, (dz, dy, dx) in enumerate(TAPS):
            pre2 += a1[1 + dz, 1 + dy, 1 + dx] @ P["W2"][t].T
        out.append(act(pre2) @ P["W3"].T + P["b3"])
    return np.array(out)


def loss_and_grad(p, x, target):
    """Relative squared error sum (out - target)^2 / sum target^2 and its gradient."""
    P = unpack(p)
    out, (x, pre1, a1, pre2, a2) = forward(p, x)
    tn = float(np.sum(target ** 2))
    loss = float(np.sum((out - target) ** 2)) / tn
    dout = 2.0 * (out - target) / tn
    G = {"W3": np.einsum("zyxo,zyxc->oc", dout, a2), "b3": dout.sum((0, 1, 2))}
    dpre2 = (dout @ P["W3"]) * act_grad(pre2)
    G["W2"] = np.stack([np.einsum("zyxo,zyxc->oc", dpre2, shifted(a1, tap)) for tap in TAPS])
    G["b2"] = dpre2.sum((0, 1, 2))
    da1 = np.zeros_like(a1)
    for t, tap in enumerate(TAPS):
        da1 += unshift(dpre2 @ P["W2"][t], tap)
    dpre1 = da1 * act_grad(pre1)
    G["W1"] = np.stack([np.einsum("zyxo,zyxc->oc", dpre1, shifted(x, tap)) for tap in TAPS])
    G["b1"] = dpre1.sum((0, 1, 2))
    return loss, pack(G)


def fields(shape, dn, F, in_scale, out_scale):
    """Library arrays (dn [2][N], F [2][3][N], x fastest) -> the network's
    input (nz, ny, nx, 2) and target (nz, ny, nx, 6)."""
    nx, ny, nz = shape
    x = np.stack([dn[a].reshape(nz, ny, nx) * in_scale[a] for a in range(2)], -1)
    t = None
    if F is not None:
        t = np.stack([F[a, i].reshape(nz, ny, nx) * out_scale[a] for a in range(2) for i in range(3)], -1)
    return x, t


def zero_biases(p):
    d = unpack(p)
    for name in ("b1", "b2", "b3"):
        d[name][:] = 0.0
    return pack(d)


def random_params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    d = {}
    for name, shape in SIZES:
        fan_in = shape[-1] * (27 if name in ("W1", "W2") else 1) if name.startswith("W") else 1
        d[name] = rng.normal(0.0, scale / np.sqrt(fan_in), shape) if name.startswith("W") else rng.normal(0, 0.05, shape)
    return pack(d)
