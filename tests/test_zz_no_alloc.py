"""The allocation-free conservation entry point.

mlb_conservation_noalloc serves callers that cannot let the library
allocate device memory: their own memory manager owns every device byte
(a framework pool, a stream-ordered allocator), or they must not allocate
once a run is under way.  It runs the same kernels as the context's
mlb_conservation, so on the same populations it must give the same sums bit
for bit, call after call, using only its fixed scratch array and taking no
device memory.  This file is collected last so that a failure here leaves
every other test already run.
"""
import ctypes

import numpy as np
import pytest

from paper_1105_3634_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_3634_gb300 import build
    build.build()
    from paper_1105_3634_gb300 import mlb
    return torch, mlb


def _noalloc(mlb, torch, fdev, nref, S, N, out):
    stream = torch.cuda.current_stream()
    return mlb.lib.mlb_conservation_noalloc(
        ctypes.c_void_p(fdev.data_ptr()), mlb._dp(np.ascontiguousarray(nref, dtype=np.float64)), S, N,
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("shape", [(20, 18, 16), (64, 64, 40)])
def test_noalloc_conservation_matches_context_twice(env, shape):
    """Two calls in a row on different states equal mlb_conservation bit for
    bit; the larger box (163840 sites) runs the kernel's grid-stride loop
    beyond its 512 x 256 threads."""
    torch, mlb = env
    lat, n = W.binary_attraction(shape, seed=5)
    S, N = lat.nspecies, lat.nsites
    sim = mlb.Simulation(lat)
    sim.set_fields(n, W.random_velocities(lat, 0.01, seed=3))
    out = torch.full((S + 3,), float("nan"), dtype=torch.float64, device="cuda")
    for steps in (0, 37):
        sim.step(steps)
        mass, mom = sim.conservation()
        f, nref, _ = sim.populations()
        fdev = torch.from_numpy(f).cuda()
        torch.cuda.synchronize()
        assert _noalloc(mlb, torch, fdev, nref, S, N, out) == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.array_equal(got[:S], mass), (got[:S], mass)
        assert np.array_equal(got[S:], mom), (got[S:], mom)
    sim.close()


def test_noalloc_takes_no_device_memory_and_refuses_oversize(env):
    torch, mlb = env
    lat, n = W.binary_config1((32, 16, 16))
    S, N = lat.nspecies, lat.nsites
    sim = mlb.Simulation(lat)
    sim.set_fields(n)
    f, nref, _ = sim.populations()
    sim.close()
    fdev = torch.from_numpy(f).cuda()
    out = torch.zeros(S + 3, dtype=torch.float64, device="cuda")
    assert _noalloc(mlb, torch, fdev, nref, S, N, out) == 0     # first call: the kernels load
    torch.cuda.synchronize()
    first = out.cpu().numpy().copy()
    free0, _ = torch.cuda.mem_get_info()
    assert _noalloc(mlb, torch, fdev, nref, S, N, out) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert np.array_equal(out.cpu().numpy(), first)
    # more species than the fixed array holds: refused without a launch
    assert _noalloc(mlb, torch, fdev, np.zeros(8), 8, N, out) == 1
