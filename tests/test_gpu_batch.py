"""Batched ensembles (one captured CUDA graph for many independent contexts)
and the work-decomposition tuner: neither may change a single bit of the
populations compared with stepping each context alone with the defaults."""
import math

import numpy as np
import pytest

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


def members():
    """Uneven lattices and settings: the benchmark physics (fused launch),
    a sheared channel, attraction (reach-3 tiles, split launch), three species."""
    out = []
    lat, n = W.binary_config1((24, 16, 12))
    out.append((lat, n))
    lat = W.Lattice(shape=(40, 12, 16), sigma=[1.0, 1.5], wall_axis=1, wall_u_lo=(-0.03, 0.0, 0.0),
                    wall_u_hi=(0.03, 0.0, 0.0))
    out.append((lat, W.noise(lat, W.densities_from_packing(0.25, lat.sigma, [0.5, 0.5]), 0.02, seed=3)))
    out.append(W.binary_attraction((18, 16, 17), seed=4))
    lat, n = W.taylor_channel((40, 16, 10), U=0.05)
    n[2] = n[2] * 1e3 / 8
    out.append((lat, n))
    return out


def make(gpu, torch, lat, n):
    sim = gpu.Simulation(lat, stream=torch.cuda.Stream())
    sim.set_fields(n, W.random_velocities(lat, 0.005, seed=11))
    return sim


@pytest.mark.parametrize("nsteps", [7, 10])
def test_batch_equals_members_alone(gpu, nsteps):
    import torch
    cases = members()
    alone = []
    for lat, n in cases:
        sim = make(gpu, torch, lat, n)
        sim.step(nsteps)
        alone.append(sim.populations()[0])
        sim.close()
    sims = [make(gpu, torch, lat, n) for lat, n in cases]
    batch = gpu.Batch(sims)
    batch.step(nsteps)
    batch.synchronize()
    for k, sim in enumerate(sims):
        f, _, step = sim.populations()
        assert step == nsteps
        assert np.array_equal(f.view(np.uint32), alone[k].view(np.uint32)), k
    batch.close()
    for sim in sims:
        sim.close()


def test_batch_recaptures_after_a_settings_change(gpu):
    """Steps 4 in the batch, then an external force on one member (its kernel
    parameters change, so the graph must be captured again), then 4 more."""
    import torch
    cases = members()[:2]
    lat0 = cases[0][0]
    y = np.arange(lat0.nsites) // lat0.shape[0] % lat0.shape[1]
    fext = np.zeros((lat0.nspecies, 3, lat0.nsites))
    fext[:, 0, :] = 1e-5 * np.sin(2 * math.pi * y / lat0.shape[1])[None, :]

    ref = [make(gpu, torch, lat, n) for lat, n in cases]
    for sim in ref:
        sim.step(4)
    ref[0].set_external_force(fext)
    for sim in ref:
        sim.step(4)
    expect = [sim.populations()[0] for sim in ref]

    sims = [make(gpu, torch, lat, n) for lat, n in cases]
    batch = gpu.Batch(sims)
    batch.step(4)
    batch.synchronize()
    sims[0].set_external_force(fext)
    batch.step(4)
    batch.synchronize()
    for k, sim in enumerate(sims):
        assert np.array_equal(sim.populations()[0].view(np.uint32), expect[k].view(np.uint32)), k
    batch.close()
    for sim in sims + ref:
        sim.close()


def test_autotune_keeps_state_and_results(gpu):
    import torch
    for lat, n in members()[:3]:
        a = make(gpu, torch, lat, n)
        b = make(gpu, torch, lat, n)
        f0 = a.populations()[0]
        zchunk, fused = a.autotune(trials=2)
        assert zchunk in (4, 8, 12, 16, 32) or zchunk == lat.shape[2]
        assert np.array_equal(a.populations()[0].view(np.uint32), f0.view(np.uint32))
        a.step(6)
        b.step(6)
        assert np.array_equal(a.populations()[0].view(np.uint32), b.populations()[0].view(np.uint32))
        a.close()
        b.close()


def test_batch_rejects_bad_members(gpu):
    import torch
    lat, n = members()[0]
    sim = make(gpu, torch, lat, n)
    with pytest.raises(gpu.MLBError):
        gpu.Batch([sim, sim])                  # the same context twice
    fresh = gpu.Simulation(lat, stream=torch.cuda.Stream())
    batch = gpu.Batch([sim, fresh])          # fresh has no fields yet
    with pytest.raises(gpu.MLBError, match="member 1"):
        batch.step(2)
    batch.close()
    sim.close()
    fresh.close()


def grouped_members():
    """Members for the grouped launches: the benchmark spheres periodic and in
    a sheared channel, with attractive tails (the FP32 column kernel and the
    tensor-core mean field), walls normal to z and to x, two drag-only
    members (a second group), one species with shells of reach 1 and of
    reach 2 (two more groups), and three that step by their own launches: nx not a multiple of 4 (no bulk
    tensor copies), two predictor sweeps, reach-3 shells."""
    eps = 0.5 * W.KT_LATTICE
    tails = dict(eps=[[eps] * 2 for _ in range(2)], lambda_c=[[2.5] * 2 for _ in range(2)])
    sig = [1.0, 1.5]
    n0 = W.densities_from_packing(0.2, sig, [0.5, 0.5])
    out = []
    lat = W.Lattice(shape=(32, 16, 12), sigma=sig)
    out.append((lat, W.sine_wave(lat, n0, 0.05)))
    lat = W.Lattice(shape=(40, 12, 16), sigma=sig, wall_axis=1, wall_u_lo=(-0.03, 0.0, 0.0),
                    wall_u_hi=(0.03, 0.0, 0.0))
    out.append((lat, W.noise(lat, n0, 0.02, seed=3)))
    lat = W.Lattice(shape=(24, 16, 16), sigma=sig, **tails)
    out.append((lat, W.noise(lat, n0, 0.02, seed=5)))
    lat = W.Lattice(shape=(36, 20, 16), sigma=sig, meanfield="bf16", **tails)
    out.append((lat, W.noise(lat, n0, 0.02, seed=6)))
    for shape, seed in (((28, 12, 8), 7), ((20, 8, 8), 8)):
        lat = W.Lattice(shape=shape, sigma=sig, drag_only=True)
        out.append((lat, W.noise(lat, n0, 0.02, seed=seed)))
    lat = W.Lattice(shape=(24, 12, 10), sigma=sig, wall_axis=2, wall_u_lo=(0.0, -0.02, 0.0),
                    wall_u_hi=(0.02, 0.0, 0.0))
    out.append((lat, W.noise(lat, n0, 0.02, seed=11)))
    lat = W.Lattice(shape=(20, 12, 12), sigma=sig, wall_axis=0, wall_u_lo=(0.0, 0.0, 0.01),
                    wall_u_hi=(0.0, -0.01, 0.0))
    out.append((lat, W.noise(lat, n0, 0.02, seed=12)))
    for sig1, shape, seed in (([1.0], (24, 8, 8), 13), ([1.0], (16, 12, 8), 14),
                              ([1.75], (24, 12, 12), 15), ([1.75], (32, 8, 12), 16)):
        lat = W.Lattice(shape=shape, sigma=sig1)
        out.append((lat, W.noise(lat, W.densities_from_packing(0.2, sig1, [1.0]), 0.03, seed=seed)))
    lat = W.Lattice(shape=(18, 12, 8), sigma=sig)
    out.append((lat, W.noise(lat, n0, 0.02, seed=9)))
    lat = W.Lattice(shape=(24, 12, 8), sigma=sig)
    lat.predictor_sweeps = 2
    out.append((lat, W.noise(lat, n0, 0.02, seed=10)))
    out.append(W.binary_attraction((18, 16, 16), seed=4))
    return out


@pytest.mark.parametrize("nsteps", [6, 9])
def test_grouped_launches_equal_members_alone(gpu, nsteps):
    """Twelve members step by grouped launches (four groups: two species with
    and without the drag-only flag, one species at reach 1 and 2; in one lane
    per group, in two lanes, or not grouped),
    three by their own; every member's populations equal those of
    the member stepped alone bit for bit."""
    import torch
    cases = grouped_members()
    alone = []
    for lat, n in cases:
        sim = make(gpu, torch, lat, n)
        sim.step(nsteps)
        alone.append(sim.populations()[0])
        sim.close()
    for lanes in (1, 2, 0):
        sims = [make(gpu, torch, lat, n) for lat, n in cases]
        batch = gpu.Batch(sims, lanes=lanes)
        batch.step(nsteps)
        batch.synchronize()
        assert batch.grouped_members() == (12 if lanes else 0)
        for k, sim in enumerate(sims):
            f, _, step = sim.populations()
            assert step == nsteps
            assert np.array_equal(f.view(np.uint32), alone[k].view(np.uint32)), (lanes, k)
        batch.close()
        for sim in sims:
            sim.close()


def test_grouping_settings(gpu):
    """Only members of at most max_sites sites are grouped; bad settings are refused."""
    import torch
    cases = grouped_members()[:2]                  # 6144 and 7680 sites, both groupable
    sims = [make(gpu, torch, lat, n) for lat, n in cases]
    batch = gpu.Batch(sims, max_sites=7000)        # only the first fits: a group of one is not formed
    batch.step(2)
    batch.synchronize()
    assert batch.grouped_members() == 0
    batch.close()
    batch = gpu.Batch(sims, max_sites=8000)
    batch.step(2)
    batch.synchronize()
    assert batch.grouped_members() == 2
    for bad in ((65, 1 << 17), (-1, 1 << 17), (1, 0)):
        with pytest.raises(gpu.MLBError, match="lanes|max_sites"):
            batch._check(gpu.lib.mlb_batch_set_grouping(batch.b, *bad))
    batch.close()
    for sim in sims:
        sim.close()
