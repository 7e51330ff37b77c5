"""The multi-rank step: the oracle's slab decomposition along x (moment halos
of depth H, outgoing face populations) reproduces the monolithic oracle bit
for bit, with ranks as threads and with two gloo processes; a halo one plane
shallower does not."""
import os
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from oracle import slabs
from paper_1105_3634_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    oracle.build()


def _case(kind):
    """(lattice, initial populations, external force) of a small seeded state."""
    if kind == "config1":
        lat = W.Lattice(shape=(12, 6, 5), sigma=[1.0, 1.5], tau=1.0)
    elif kind == "attraction":
        lat = W.Lattice(shape=(15, 6, 6), sigma=[1.0, 1.5], tau=0.8,
                        eps=[[0.1, 0.12], [0.12, 0.15]], lambda_c=[[1.6, 1.6], [1.6, 1.6]])
    elif kind == "walls_y":
        lat = W.Lattice(shape=(10, 7, 4), sigma=[1.0, 1.25, 1.5], tau=1.2, wall_axis=1,
                        wall_u_lo=(-0.02, 0.0, 0.01), wall_u_hi=(0.03, 0.0, -0.01))
    elif kind == "three_sweeps":
        lat = W.Lattice(shape=(16, 6, 5), sigma=[1.0, 1.5], tau=1.0, predictor_sweeps=3)
    elif kind == "explicit_drag":
        lat = W.Lattice(shape=(9, 5, 5), sigma=[1.0, 1.5], tau=0.9, drag_only=True, force_scheme="explicit")
    else:
        raise ValueError(kind)
    S = lat.nspecies
    n0 = W.densities_from_packing(0.2, lat.sigma, [1.0 / S] * S)
    n = W.noise(lat, n0, 0.05, seed=11)
    u = W.random_velocities(lat, 0.02, seed=12)
    if lat.wall_axis >= 0:
        u[:, lat.wall_axis, :] = 0.0
    f = oracle.init(lat, n, u)
    fext = None
    if kind == "attraction":
        fext = 1e-4 * (W.uniform01(13, S * 3 * lat.nsites).reshape(S, 3, lat.nsites) - 0.5)
    return lat, f, fext


def test_halo_depth_of_the_benchmark_physics():
    # contact shells of sigma_ab <= 1.5 reach one plane, smoothing balls none
    assert slabs.halo_depth(W.Lattice(shape=(8, 8, 8), sigma=[1.0, 1.5])) == 2
    # an attraction region to 1.6 x 1.5 = 2.4 reaches two planes
    lat = W.Lattice(shape=(8, 8, 8), sigma=[1.0, 1.5], eps=[[0.1, 0.1], [0.1, 0.1]],
                    lambda_c=[[1.6, 1.6], [1.6, 1.6]])
    assert slabs.halo_depth(lat) == 1 + 2
    # sigma = 2 smoothing balls (radius 1) add one plane
    assert slabs.halo_depth(W.Lattice(shape=(8, 8, 8), sigma=[2.0, 3.0])) == 3 + 3 + 1
    # every further predictor sweep reads one more shell
    assert slabs.halo_depth(W.Lattice(shape=(8, 8, 8), sigma=[1.0, 1.5], predictor_sweeps=3)) == 2 + 2


@pytest.mark.parametrize("kind,P", [("config1", 2), ("config1", 3), ("attraction", 3), ("walls_y", 2),
                                    ("explicit_drag", 2), ("three_sweeps", 2)])
def test_slabs_equal_the_monolithic_oracle_bitwise(kind, P):
    lat, f, fext = _case(kind)
    ref = f.copy()
    oracle.step(lat, ref, 5, fext)
    out = slabs.run_threads(lat, f, 5, P, fext=fext)
    assert np.array_equal(out, ref)


def test_a_halo_one_plane_short_is_wrong():
    lat, f, fext = _case("config1")
    ref = f.copy()
    oracle.step(lat, ref, 3)
    out = slabs.run_threads(lat, f, 3, 2, depth=slabs.halo_depth(lat) - 1)
    assert not np.array_equal(out, ref)
    assert np.abs(out - ref).max() > 1e-9


def test_slab_thinner_than_the_halo_is_refused():
    lat, f, _ = _case("config1")
    with pytest.raises(ValueError, match="thinner"):
        slabs.run_threads(lat, f, 1, 12)


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import oracle as O
    from oracle import slabs as SL
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        lat, f, fext = _case("config1")
        rk = SL.SlabRank(lat, rank, world, f, SL.TorchComm(dist), fext)
        for _ in range(4):
            rk.step()
        comm = SL.TorchComm(dist)
        if rank == 0:
            parts = [rk.f] + comm.exchange(0, [], [(r, 99, rk.f.shape[:-1] + (SL.slab_bounds(lat.shape[0], world)[r][1]
                                                                                - SL.slab_bounds(lat.shape[0], world)[r][0],))
                                                   for r in range(1, world)])
            got = SL.gather(lat, parts)
            ref = f.copy()
            O.step(lat, ref, 4, fext)
            out.put(("equal", bool(np.array_equal(got, ref))))
        else:
            comm.exchange(rank, [(0, 99, rk.f)], [])
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_equal_the_monolithic_oracle():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29517
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    tag, equal = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert tag == "equal" and equal
