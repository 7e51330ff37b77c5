"""The learned hard-core force: GPU forward and gradients against the FP64
reference network, training on frames of the exact method, and its use in the
step (mutual diffusion within 1 % of the exact method; rejection and fallback
by the periodic exact recheck)."""
import math

import numpy as np
import pytest

import net_reference as R
from paper_1105_3634_gb300 import surrogate as SG
from paper_1105_3634_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_3634_gb300 import build
    build.build()
    from paper_1105_3634_gb300 import mlb
    return mlb


def _random_frame(shape, seed):
    rng = np.random.default_rng(seed)
    N = shape[0] * shape[1] * shape[2]
    return rng.normal(0, 0.01, (2, N)), rng.normal(0, 0.002, (2, 3, N))


def test_forward_and_gradient_match_the_fp64_reference(gpu):
    shape = (16, 12, 10)
    net = gpu.Net(shape)
    p = R.random_params(11).astype(np.float32)
    net.set_params(p)
    ins, outs = [80.0, 90.0], [400.0, 300.0]
    net.set_scales(ins, outs)
    dn, F = _random_frame(shape, 1)
    x, t = R.fields(shape, dn, F, ins, outs)
    out_ref, _ = R.forward(p.astype(np.float64), x)
    f_gpu = net.forward(dn)
    f_ref = np.stack([out_ref[..., 3 * a + i].reshape(-1) / outs[a] for a in range(2) for i in range(3)])
    f_ref = f_ref.reshape(2, 3, -1)
    err = np.linalg.norm(f_gpu - f_ref) / np.linalg.norm(f_ref)
    print("forward rel error (BF16 activations)", err)
    assert err < 2e-2
    loss_gpu, g_gpu = net.gradient(dn, F)
    loss_ref, g_ref = R.loss_and_grad(p.astype(np.float64), x, t)
    gerr = np.linalg.norm(g_gpu - g_ref) / np.linalg.norm(g_ref)
    print("loss", loss_gpu, loss_ref, "gradient rel error", gerr)
    assert abs(loss_gpu - loss_ref) < 2e-2 * loss_ref
    assert gerr < 3e-2
    # per block: each layer's weights and biases
    k = 0
    for name, shp in R.SIZES:
        n = int(np.prod(shp))
        e = np.linalg.norm(g_gpu[k:k + n] - g_ref[k:k + n]) / np.linalg.norm(g_ref[k:k + n])
        assert e < 5e-2, (name, e)
        k += n
    net.close()


@pytest.mark.parametrize("shape", [(128, 6, 4), (256, 3, 5)])
def test_tensor_core_inference_matches_the_fp64_reference(gpu, shape):
    """Lattices with nx % 128 == 0 run layers 2 and 3 as one tcgen05 kernel
    (128-site row tiles, FP32 act2); the tiles' x halos wrap periodically."""
    net = gpu.Net(shape)
    p = R.random_params(13).astype(np.float32)
    net.set_params(p)
    ins, outs = [80.0, 90.0], [400.0, 300.0]
    net.set_scales(ins, outs)
    dn, F = _random_frame(shape, 2)
    x, _ = R.fields(shape, dn, F, ins, outs)
    out_ref, _ = R.forward(p.astype(np.float64), x)
    f_ref = np.stack([out_ref[..., o].reshape(-1) for o in range(6)]).reshape(2, 3, -1)
    f_ref /= np.array(outs)[:, None, None]
    f_gpu = net.forward(dn)
    err = np.linalg.norm(f_gpu - f_ref) / np.linalg.norm(f_ref)
    worst = np.abs(f_gpu - f_ref).max() / np.abs(f_ref).max()
    print("tcgen05 forward rel error", err, "worst", worst)
    assert err < 1e-2 and worst < 3e-2
    net.close()


def test_tensor_core_inference_at_256_cubed_on_sampled_sites(gpu):
    """The bench's lattice, 256^3 (131072 row tiles of the persistent
    tcgen05 launch bench.py times): 516 sampled sites, the lattice corners
    among them, against the FP64 reference evaluated on their 5^3 patches."""
    shape = (256, 256, 256)
    N = shape[0] * shape[1] * shape[2]
    net = gpu.Net(shape)
    p = R.random_params(21).astype(np.float32)
    net.set_params(p)
    ins, outs = [80.0, 90.0], [400.0, 300.0]
    net.set_scales(ins, outs)
    dn = (W.uniform01(77, 2 * N).reshape(2, N) - 0.5) * 0.02
    f_gpu = net.forward(dn)
    x = np.stack([(dn[a] * ins[a]).astype(np.float32).astype(np.float64).reshape(shape[::-1]) for a in range(2)], -1)
    r = W.uniform01(78, 3 * 512).reshape(512, 3)
    sites = [(int(a * shape[2]), int(b * shape[1]), int(c * shape[0])) for a, b, c in r]
    sites += [(0, 0, 0), (255, 255, 255), (0, 255, 127), (255, 0, 128)]    # every wrap
    ref = R.forward_at(p.astype(np.float64), x, sites)
    got = np.stack([f_gpu[a, i, [s_[0] * shape[1] * shape[0] + s_[1] * shape[0] + s_[2] for s_ in sites]] * outs[a]
                    for a in range(2) for i in range(3)], 1)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    worst = np.abs(got - ref).max() / np.abs(ref).max()
    print("256^3 tcgen05 sampled rel error", err, "worst", worst)
    assert err < 1e-2 and worst < 3e-2
    net.close()


@pytest.fixture(scope="module")
def frame_sets(gpu):
    shape = (64, 8, 8)
    return shape, SG.frames(gpu, shape, 240, seed=21), SG.frames(gpu, shape, 40, seed=99)


def test_training_from_random_weights_learns_the_force(gpu, frame_sets):
    """The GPU forward/backward/Adam kernels alone, from He-type random
    weights: the relative loss falls by more than 100x and the typical
    held-out frame is within 3 %."""
    shape, train, held = frame_sets
    net = gpu.Net(shape)
    net.set_params(SG.initial_params())
    net.set_scales(*SG.scales(train))
    hist = SG.train(net, train, epochs=300, lr0=1e-3, lr_min=1e-5, iters=1)
    errs = SG.frame_errors(net, held)
    print("from random weights: loss", hist[0], "->", hist[-1], "held-out median", np.median(errs), "max", errs.max())
    assert hist[-1] < 0.01 * hist[0]
    assert np.median(errs) < 0.03
    net.close()


@pytest.fixture(scope="module")
def trained(gpu, frame_sets):
    """The production recipe: start from the least-squares linear-response
    stencil, fine-tune every weight on the GPU."""
    shape, train, held = frame_sets
    ins, outs = SG.scales(train)
    p0 = SG.stencil_params(SG.linear_stencil(train, shape, ins, outs), SG.max_scaled_force(train, outs))
    net = gpu.Net(shape)
    net.set_params(p0)
    net.set_scales(ins, outs)
    before = SG.frame_errors(net, held)
    hist = SG.train(net, train, epochs=100, lr0=1e-6, lr_min=1e-8, iters=1)
    errs = SG.frame_errors(net, held)
    print("stencil start: held-out median", np.median(before), "max", before.max(), "| fine-tuned: loss", hist[-1],
          "held-out median", np.median(errs), "90th percentile", np.percentile(errs, 90), "max", errs.max())
    return shape, net, errs, before


def test_the_fine_tuned_network_is_within_a_percent(trained):
    shape, net, errs, before = trained
    assert np.median(errs) < 0.01 and np.percentile(errs, 90) < 0.03 and errs.max() < 0.06
    assert np.median(errs) <= 1.05 * np.median(before)       # the training does not undo the start


def test_the_network_is_odd_in_its_input(gpu, trained):
    shape, net, _, _ = trained
    dn = SG.frames(gpu, shape, 1, seed=5)[0][0]
    assert np.array_equal(net.forward(-dn), -net.forward(dn))


def _decay_rate(sim, lat, t0, t1, every):
    x = W.coordinate(lat, 0)
    q = 2 * math.pi / lat.shape[0]
    ts, amps = [], []
    t = 0
    for target in range(t0, t1 + 1, every):
        sim.step(target - t)
        t = target
        n, _ = sim.moments()
        c = n[0] / n.sum(0)
        ts.append(t)
        amps.append(abs(np.mean(c * np.exp(-1j * q * x))))
    return -np.polyfit(ts, np.log(amps), 1)[0] / q ** 2


def test_mutual_diffusion_with_the_surrogate(gpu, trained):
    """D_mutual from the decay of a 2 % concentration wave (wavelength 64),
    exact force against the trained surrogate (exact recheck every 50 steps,
    bound 5 % relative force error) and against the method without the
    hard-core force (an all-zero network that is never rejected): the network
    gains the hard-core contribution to D at a fraction of a percent."""
    shape, net, _, _ = trained
    lat = SG.benchmark_lattice(shape)
    n0 = W.densities_from_packing(0.2, lat.sigma, [0.5, 0.5])
    n = W.sine_wave(lat, n0, 0.02)
    exact = gpu.Simulation(lat)
    exact.set_fields(n)
    D_x = _decay_rate(exact, lat, 100, 1100, 100)
    surr = gpu.Simulation(lat)
    surr.set_fields(n)
    surr.attach_surrogate(net, recheck_every=50, bound=0.05)
    D_s = _decay_rate(surr, lat, 100, 1100, 100)
    active, last, rechecks, rejections = surr.surrogate_status()
    zero = gpu.Net(shape)
    zero.set_scales([1.0, 1.0], [1.0, 1.0])
    bare = gpu.Simulation(lat)
    bare.set_fields(n)
    bare.attach_surrogate(zero, recheck_every=2 ** 31 - 1, bound=1e300)
    D_0 = _decay_rate(bare, lat, 100, 1100, 100)
    print(f"D exact {D_x:.6f}, with the surrogate {D_s:.6f} ({(D_s - D_x) / D_x:+.2e}), without the hard-core "
          f"force {D_0:.6f} ({(D_0 - D_x) / D_x:+.2e}); last recheck error {last:.4f}, rechecks {rechecks}, "
          f"rejections {rejections}")
    assert active and rejections == 0 and rechecks >= 20 and last < 0.05
    assert abs(D_s - D_x) < 0.01 * D_x
    assert abs(D_0 - D_x) > 10 * abs(D_s - D_x)
    for o in (exact, surr, bare, zero):
        o.close()


def test_a_bad_surrogate_is_rejected_and_the_exact_force_takes_over(gpu):
    shape = (32, 8, 8)
    lat = SG.benchmark_lattice(shape)
    n0 = W.densities_from_packing(0.2, lat.sigma, [0.5, 0.5])
    n = W.sine_wave(lat, n0, 0.03)
    net = gpu.Net(shape)                        # all parameters zero: predicts no force
    net.set_scales([1.0, 1.0], [1.0, 1.0])
    a = gpu.Simulation(lat)
    a.set_fields(n)
    a.attach_surrogate(net, recheck_every=10, bound=0.05)
    a.step(30)
    active, last, rechecks, rejections = a.surrogate_status()
    assert not active and rejections == 1 and rechecks == 1 and last > 0.9
    b = gpu.Simulation(lat)
    b.set_fields(n)
    b.step(30)
    # step 0 was the recheck (exact force), then the surrogate was off: bit for bit the exact run
    assert np.array_equal(a.populations()[0].view(np.uint32), b.populations()[0].view(np.uint32))
    with pytest.raises(gpu.MLBError, match="lattice size"):
        a.attach_surrogate(gpu.Net((16, 8, 8)))
    a.close()
    b.close()
    net.close()
