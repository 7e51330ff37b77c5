"""The allocation-free conservation entry point.

mlb_conservation_noalloc serves callers that cannot let the library
allocate device memory (their own memory manager owns it, or they must not
allocate mid-run).  It must give the same sums as the context's
mlb_conservation, call after call, while using only its fixed scratch array.
This file is collected last so that a failure here leaves every other test
already run.
"""
import ctypes

import numpy as np
import pytest

from paper_1105_3634_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-6     # relative, as for the context's conservation sums


def test_noalloc_conservation_matches_context_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_3634_gb300 import build
    build.build()
    from paper_1105_3634_gb300 import mlb

    lat, n = W.binary_attraction((20, 18, 16), seed=5)
    S, N = lat.nspecies, lat.nsites
    sim = mlb.Simulation(lat)
    sim.set_fields(n, W.random_velocities(lat, 0.01, seed=3))
    stream = torch.cuda.current_stream()
    out = torch.full((S + 3,), float("nan"), dtype=torch.float64, device="cuda")
    for steps in (0, 37):                 # two calls in a row, on different states
        sim.step(steps)
        mass, mom = sim.conservation()
        f, nref, _ = sim.populations()
        fdev = torch.from_numpy(f).cuda()
        torch.cuda.synchronize()
        st = mlb.lib.mlb_conservation_noalloc(
            ctypes.c_void_p(fdev.data_ptr()), mlb._dp(np.ascontiguousarray(nref)), S, N,
            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert st == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.abs(got[:S] - mass) <= TOL * mass)
        assert np.all(np.abs(got[S:] - mom) <= TOL * n.sum() * np.sqrt(1 / 3))
    sim.close()
    # sizes beyond the fixed scratch are refused without a launch
    st = mlb.lib.mlb_conservation_noalloc(ctypes.c_void_p(fdev.data_ptr()), mlb._dp(np.zeros(8)), 8, N,
                                          ctypes.c_void_p(out.data_ptr()), None)
    assert st == 1
