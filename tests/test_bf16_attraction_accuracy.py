"""Why the mean field stays on the FP32 pipes: a BF16 tensor-core form of
the attraction G^a = sum_b sum_d K_ab(d) n^b(r + d) (Eq. potmeanforce's tail
term), emulated here with BF16-rounded densities and kernel weights and exact
sums, misses the 1e-5 parity bar by two orders of magnitude; only the
compensated three-pass form (hi x hi + lo x hi + hi x lo of the BF16 hi/lo
splits) reaches it, and three passes cost more than the FP32 column kernel."""
import numpy as np

from paper_1105_3634_gb300 import workloads as W


def _bf16(a):
    a32 = np.asarray(a, np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16        # round to nearest even, 8-bit significand
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def test_one_bf16_pass_misses_the_parity_bar_the_compensated_form_meets_it(orc):
    lat, n = W.binary_attraction((20, 20, 20), seed=3)
    shape = lat.shape[::-1]
    dn = n - n.mean(1, keepdims=True)
    kernels = {}
    for a in range(2):
        for b in range(2):
            sab = 0.5 * (lat.sigma[a] + lat.sigma[b])
            d = orc.attraction_set(sab, lat.lambda_c[a][b]).astype(int)
            r = np.linalg.norm(d, axis=1)
            kernels[a, b] = (d, 6 * lat.eps[a][b] * sab ** 6 * d / r[:, None] ** 8)

    def G(field, kmap):
        out = np.zeros((2, 3) + shape)
        for (a, b), (d, K) in kernels.items():
            X = np.fft.fftn(field[b].reshape(shape))
            Kq = kmap(K)
            for k in range(3):
                ker = np.zeros(shape)
                np.add.at(ker, (d[:, 2] % shape[0], d[:, 1] % shape[1], d[:, 0] % shape[2]), Kq[:, k])
                out[a, k] += np.real(np.fft.ifftn(np.conj(np.fft.fftn(ker)) * X))
        return out

    ref = G(dn, lambda K: K)
    hi = _bf16(dn)
    lo = _bf16(dn - hi)
    one = G(hi, _bf16)
    comp = G(hi, _bf16) + G(lo, _bf16) + G(hi, lambda K: _bf16(K - _bf16(K)))
    e1 = np.linalg.norm(one - ref) / np.linalg.norm(ref)
    e3 = np.linalg.norm(comp - ref) / np.linalg.norm(ref)
    print(f"relative error of G: one BF16 pass {e1:.2e}, compensated three passes {e3:.2e}")
    assert e1 > 1e-3
    assert e3 < 1e-5
