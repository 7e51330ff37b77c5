"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Element-wise comparison of densities, velocities and accelerations on the
same seeded inputs.  Tolerance: 1e-5 on densities and velocities after 500
steps (FP32 populations), both as the relative error of the field in the
2-norm over the lattice, ||x_gpu - x_oracle|| / ||x_oracle||, and at the
worst single site, max|x_gpu - x_oracle| / max|x_oracle|.  FP32 storage of
the populations (f - w_i n_ref, rounding ~ ulp(w_i dn)) puts the velocity
error of a 5% concentration wave at a few 1e-6.
"""
import math

import numpy as np
import pytest

from paper_1105_3634_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_STATE = 1e-5      # densities, velocities (FP32 vs FP64), 2-norm over the lattice
TOL_SITE = 1e-5       # the same, worst single site
TOL_ACC = 1e-4        # accelerations from one FP32 force evaluation


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_3634_gb300 import build
    build.build()
    from paper_1105_3634_gb300 import mlb
    return mlb


U_FLOOR = 1e-9        # velocity scale below which a field counts as at rest


def rel(a, b, floor=0.0):
    """max|a - b| / max(max|b|, floor): the worst site."""
    scale = max(float(np.abs(b).max()), floor)
    return float(np.abs(a - b).max() / scale) if scale > 0 else float(np.abs(a - b).max())


def rel2(a, b, floor=0.0):
    """||a - b|| / max(||b||, floor sqrt(size)): relative error of the field in the 2-norm."""
    scale = max(float(np.linalg.norm(b)), floor * math.sqrt(b.size))
    return float(np.linalg.norm(a - b) / scale) if scale > 0 else float(np.linalg.norm(a - b))


def run_pair(mlbmod, orc, lat, n, u=None, checkpoints=(0, 1, 50), fext=None, report=None):
    """Advance GPU and oracle side by side; return the worst relative errors."""
    sim = mlbmod.Simulation(lat)
    sim.set_fields(n, u)
    if fext is not None:
        sim.set_external_force(fext)
    f = orc.init(lat, n, u)
    t = 0
    worst = {"n": 0.0, "u": 0.0, "acc": 0.0, "n_site": 0.0, "u_site": 0.0}
    for cp in checkpoints:
        sim.step(cp - t)
        orc.step(lat, f, cp - t, fext)
        t = cp
        gn, gu = sim.moments()
        on, oj = orc.moments(lat, f)
        ou = orc.velocity_fields(lat, on, oj)
        e = {"n": rel2(gn, on), "u": rel2(gu, ou, U_FLOOR), "n_site": rel(gn, on), "u_site": rel(gu, ou, U_FLOOR)}
        ga = sim.acceleration()
        oa = orc.accel(lat, on, oj, fext=fext)
        e["acc"] = rel(ga, oa, U_FLOOR)
        for k in worst:
            worst[k] = max(worst[k], e[k])
        if report is not None:
            report.append((cp, e))
    sim.close()
    return worst


def ok(w):
    return (w["n"] < TOL_STATE and w["u"] < TOL_STATE and w["n_site"] < TOL_SITE and w["u_site"] < TOL_SITE
            and w["acc"] < TOL_ACC)


def test_config1_500_steps(gpu, orc):
    """Binary sigma = (1, 1.5), packing 0.2, tau = 1, 5% sine wave, 64x8x8, 500 steps."""
    lat, n = W.binary_config1()
    rep = []
    w = run_pair(gpu, orc, lat, n, checkpoints=(0, 1, 10, 100, 500), report=rep)
    print("config1", rep)
    assert ok(w), w


def test_attraction_ragged_box(gpu, orc):
    """sigma = (2, 3), eps = kT/2 tails cut at 2.5 sigma, packing 0.3, 1% noise,
    on a ragged 18x16x17 box (every stencil wraps), 60 steps."""
    lat, n = W.binary_attraction((18, 16, 17), seed=11)
    rep = []
    w = run_pair(gpu, orc, lat, n, checkpoints=(0, 1, 20, 60), report=rep)
    print("attraction", rep)
    assert ok(w), w


# attraction in isolation: the acceleration is linear in the mean field G^a at
# fixed densities and velocities, so a(eps) - a(eps = 0) is the attraction's
# share on both sides; cases span every species-group shape of the column
# kernel (S = 1..4), the reach tiers 3, 5, 7, 8, walls on x and z, ragged tiles
ATTRACTION_CASES = {
    "S1_reach3": dict(shape=(20, 12, 11), sigma=[2.0], lam=1.5, wall=-1),
    "S2_reach7_zwalls": dict(shape=(36, 10, 19), sigma=[2.0, 3.0], lam=2.5, wall=2),
    "S3_reach5_xwalls": dict(shape=(22, 13, 12), sigma=[1.5, 2.0, 2.5], lam=2.0, wall=0, zero=(0, 2)),
    "S4_reach8": dict(shape=(19, 18, 17), sigma=[1.0, 1.5, 2.0, 2.5], lam=3.4, wall=-1),
}


def attraction_lattices(case):
    S = len(case["sigma"])
    eps = [[0.3 * W.KT_LATTICE * (1.0 + 0.1 * (a + b)) for b in range(S)] for a in range(S)]
    if "zero" in case:
        a, b = case["zero"]
        eps[a][b] = eps[b][a] = 0.0
    lam = [[case["lam"]] * S for _ in range(S)]
    mk = lambda e: W.Lattice(shape=case["shape"], sigma=case["sigma"], eps=e, lambda_c=lam,
                             wall_axis=case["wall"])
    return mk(eps), mk(None)


@pytest.mark.parametrize("name", sorted(ATTRACTION_CASES))
def test_attraction_field_isolated(gpu, orc, name):
    lat, lat0 = attraction_lattices(ATTRACTION_CASES[name])
    n0 = W.densities_from_packing(0.25, lat.sigma, [1.0 / lat.nspecies] * lat.nspecies)
    n = W.noise(lat, n0, 0.05, seed=31)
    u = W.random_velocities(lat, 0.01, seed=32)
    j = n[:, None, :] * u
    got = []
    for L in (lat, lat0):
        sim = gpu.Simulation(L)
        sim.set_fields(n, u)
        got.append(sim.acceleration())
        sim.close()
    g_gpu = got[0] - got[1]
    g_orc = orc.accel(lat, n, j) - orc.accel(lat0, n, j)
    assert np.abs(g_orc).max() > 1e-6
    # FP32 accumulation over ~1e3 - 1e4 region points of 5% deviations
    assert rel(g_gpu, g_orc) < 2e-4, (name, rel(g_gpu, g_orc))
    assert rel2(g_gpu, g_orc) < 5e-5, (name, rel2(g_gpu, g_orc))


def test_taylor_channel_three_species_walls(gpu, orc):
    """Two solvents sigma = 2, 2.5 and a dilute solute sigma = 3 between
    walls moving at -U, +U (halfway bounce-back), 40x16x10, 150 steps."""
    lat, n = W.taylor_channel((40, 16, 10), U=0.05)
    n[2] = n[2] * 1e3 / 8            # a visible solute pulse on this small box
    rep = []
    w = run_pair(gpu, orc, lat, n, checkpoints=(0, 1, 30, 150), report=rep)
    print("taylor", rep)
    assert ok(w), w


def test_global_memory_passes_reach4(gpu, orc):
    """sigma = (4, 3): contact shells of reach 4, beyond the shared-memory
    tiles, so both passes read neighbours from global memory; 40 steps."""
    lat = W.Lattice(shape=(20, 16, 14), sigma=[4.0, 3.0], tau=0.9)
    n0 = W.densities_from_packing(0.2, lat.sigma, [0.5, 0.5])
    n = W.noise(lat, n0, 0.02, seed=41)
    u = W.random_velocities(lat, 0.005, seed=42)
    w = run_pair(gpu, orc, lat, n, u, checkpoints=(0, 1, 40))
    assert ok(w), w


@pytest.mark.parametrize("drag_only,scheme", [(True, "semi_implicit"), (False, "explicit"), (True, "explicit")])
def test_flags_drag_only_and_forward_euler(gpu, orc, drag_only, scheme):
    lat = W.Lattice(shape=(24, 9, 8), sigma=[1.0, 2.0], tau=0.8, drag_only=drag_only, force_scheme=scheme)
    n0 = W.densities_from_packing(0.1, lat.sigma, [0.5, 0.5])
    n = W.noise(lat, n0, 0.05, seed=4)
    u = W.random_velocities(lat, 0.01, seed=9)
    w = run_pair(gpu, orc, lat, n, u, checkpoints=(0, 1, 40))
    assert ok(w), w


def test_external_force_and_initial_velocities(gpu, orc):
    """A Kolmogorov-type body force F_x = F0 sin(2 pi y / L) on both species."""
    lat = W.Lattice(shape=(10, 20, 9), sigma=[1.0, 1.5], tau=1.0)
    n0 = W.densities_from_packing(0.15, lat.sigma, [0.5, 0.5])
    n = W.noise(lat, n0, 0.02, seed=21)
    y = W.coordinate(lat, 1)
    fext = np.zeros((2, 3, lat.nsites))
    fext[:, 0, :] = 1e-5 * np.sin(2 * math.pi * y / 20)[None, :]
    u = W.random_velocities(lat, 0.005, seed=2)
    w = run_pair(gpu, orc, lat, n, u, checkpoints=(0, 1, 80), fext=fext)
    assert ok(w), w


def _fused_case(case):
    if case == "cube":
        lat, n = W.binary_config1((40, 12, 10))
    elif case == "tile2_walls":
        lat = W.Lattice(shape=(36, 10, 12), sigma=[2.0, 1.5], wall_axis=2, wall_u_lo=(-0.02, 0.0, 0.0),
                        wall_u_hi=(0.02, 0.0, 0.0))
        n = W.noise(lat, W.densities_from_packing(0.2, lat.sigma, [0.5, 0.5]), 0.03, seed=7)
    elif case == "global_attraction":
        lat, n = W.binary_attraction((18, 16, 17), seed=3)
    else:
        lat = W.Lattice(shape=(24, 9, 8), sigma=[1.0, 2.0], tau=0.8, drag_only=True)
        n = W.noise(lat, W.densities_from_packing(0.1, lat.sigma, [0.5, 0.5]), 0.05, seed=4)
    return lat, n


@pytest.mark.parametrize("case", ["cube", "tile2_walls", "global_attraction", "drag"])
def test_fused_pass2_collide_is_bitwise_split(gpu, case):
    """The fused pass-2 + collision launch and the split pair (acceleration
    stored, then collided) give the same populations bit for bit (shells of
    reach 3 always run split)."""
    lat, n = _fused_case(case)
    u = W.random_velocities(lat, 0.01, seed=5)
    out = []
    for split in (False, True):
        sim = gpu.Simulation(lat, split_collide=split)
        local_g = case == "cube"                 # every smoothing ball is the single site
        untiled = case == "global_attraction"     # shell reach 3: never fused
        assert sim.launches_per_step() == (1 if local_g else 2) + (3 if split or untiled else 2) + (
            1 if case == "global_attraction" else 0)
        sim.set_fields(n, u)
        sim.step(25)
        out.append(sim.populations()[0])
        sim.close()
    assert np.array_equal(out[0].view(np.uint32), out[1].view(np.uint32))


def test_conservation_sums(gpu):
    lat, n = W.binary_attraction((20, 18, 16), seed=5)
    sim = gpu.Simulation(lat)
    sim.set_fields(n, W.random_velocities(lat, 0.01, seed=1))
    m0, p0 = sim.conservation()
    assert np.allclose(m0, n.sum(1), rtol=1e-7)
    sim.step(200)
    m1, p1 = sim.conservation()
    assert np.abs(m1 - m0).max() < 1e-6 * m0.max()
    assert np.abs(p1 - p0).max() < 1e-6 * n.sum() * math.sqrt(1 / 3)
    sim.close()


def test_checkpoint_resume_is_bitwise(gpu):
    lat, n = W.binary_attraction((16, 16, 16), seed=8)
    sim = gpu.Simulation(lat)
    sim.set_fields(n)
    sim.step(20)
    f20, nref, step = sim.populations()
    assert step == 20
    sim.step(15)
    fa, _, _ = sim.populations()
    sim2 = gpu.Simulation(lat)
    sim2.set_populations(f20, nref, step)
    sim2.step(15)
    fb, _, stepb = sim2.populations()
    assert stepb == 35
    assert np.array_equal(fa.view(np.uint32), fb.view(np.uint32))
    sim.close()
    sim2.close()


def test_zero_steps_and_rerun_determinism(gpu):
    lat, n = W.binary_config1((32, 8, 8))
    a = gpu.Simulation(lat)
    a.set_fields(n)
    f0, _, _ = a.populations()
    a.step(0)
    assert np.array_equal(a.populations()[0], f0)
    a.step(7)
    b = gpu.Simulation(lat)
    b.set_fields(n)
    b.step(7)
    assert np.array_equal(a.populations()[0].view(np.uint32), b.populations()[0].view(np.uint32))
    # fields set again on a used context: the same reference densities and state
    a.set_fields(n)
    c = gpu.Simulation(lat)
    c.set_fields(n)
    fa, nref_a, _ = a.populations()
    fc, nref_c, _ = c.populations()
    assert np.array_equal(nref_a, nref_c)
    assert np.array_equal(fa.view(np.uint32), fc.view(np.uint32))


def test_invalid_inputs_are_rejected(gpu):
    lat, n = W.binary_config1((16, 8, 8))
    sim = gpu.Simulation(lat)
    with pytest.raises(gpu.MLBError, match="EINVAL"):
        bad = n.copy(); bad[0, 3] = -1.0
        sim.set_fields(bad)
    with pytest.raises(gpu.MLBError, match=r"n\[1\]\[5\] = nan"):
        bad = n.copy(); bad[1, 5] = np.nan; bad[1, 9] = -1.0
        sim.set_fields(bad)
    with pytest.raises(gpu.MLBError, match="xi3 = .* at site 0"):
        sim.set_fields(n * 10)
    with pytest.raises(gpu.MLBError, match=f"velocity entry {4 * n.shape[1] + 7} = 1"):
        u = np.zeros((2, 3, n.shape[1])); u[1, 1, 7] = 1.0; u[1, 2, 3] = np.inf
        sim.set_fields(n, u)
    with pytest.raises(gpu.MLBError, match="ESTATE"):
        sim.step(1)                     # no state yet
    sim.set_fields(n)
    sim.step(2)
    with pytest.raises(gpu.MLBError, match="symmetric"):
        sim._check(gpu.lib.mlb_set_interactions(sim.ctx, gpu._dp(np.array([[0.1, 0.2], [0.0, 0.1]])),
                                                 gpu._dp(np.full((2, 2), 2.0))))
    sim.close()
    lat2 = W.Lattice(shape=(3, 8, 8), sigma=[2.0, 3.0])
    with pytest.raises(gpu.MLBError, match="periodic extent"):
        gpu.Simulation(lat2)
    lat3 = W.Lattice(shape=(16, 16, 16), sigma=[1.0, 1.5], mass=[1.0, 2.0])
    with pytest.raises(gpu.MLBError, match="mass"):
        gpu.Simulation(lat3)


def test_empty_species(gpu, orc):
    """A species with zero density everywhere stays empty and exerts no force."""
    lat = W.Lattice(shape=(16, 8, 8), sigma=[1.0, 1.5, 2.0])
    n0 = W.densities_from_packing(0.15, lat.sigma[:2], [0.5, 0.5])
    n = np.zeros((3, lat.nsites))
    n[:2] = W.sine_wave(W.Lattice(shape=(16, 8, 8), sigma=[1.0, 1.5]), n0, 0.05)
    w = run_pair(gpu, orc, lat, n, checkpoints=(0, 1, 30))
    assert ok(w), w


def test_full_size_sampled(gpu, orc):
    """256^3 binary (the benchmark workload, same launch sequence): after 3
    steps the accelerations and the next populations at 48 sampled sites
    equal the oracle's evaluated one by one from the GPU's own state."""
    lat, n = W.binary_config1((256, 256, 256))
    sim = gpu.Simulation(lat)
    sim.set_fields(n)
    sim.step(3)
    gn, gu = sim.moments()
    gj = gn[:, None, :] * gu
    ga = sim.acceleration()
    f_t, nref, _ = sim.populations()
    sim.step(1)
    f_t1, _, _ = sim.populations()
    sim.close()
    rng = np.random.default_rng(0)
    N = lat.nsites
    sites = np.sort(rng.choice(N, 48, replace=False))
    sites[0] = 0                                  # a corner: every stencil wraps
    g, _, _ = orc.gfield(lat, gn)
    oa = orc.accel(lat, gn, gj, g=g, sites=sites)
    assert rel(ga[:, :, sites], oa) < TOL_ACC
    # populations at t+1 on the sampled sites: pull from the 19 source sites
    cg, wg = gpu.velocity_set()
    co, _ = orc.velocities()
    perm = [int(np.where((co == v).all(1))[0][0]) for v in cg]        # gpu index -> oracle index
    nx, ny, nz = lat.shape
    x, y, z = sites % nx, (sites // nx) % ny, sites // (nx * ny)
    src = np.stack([((x - cg[i, 0]) % nx) + nx * (((y - cg[i, 1]) % ny) + ny * ((z - cg[i, 2]) % nz))
                    for i in range(19)], 1)                            # [M][19]
    flat = src.reshape(-1)
    oacc = orc.accel(lat, gn, gj, g=g, sites=flat)                    # [S][3][M*19]
    ff = np.empty((flat.size, 2, 19))
    for a in range(2):
        for i in range(19):
            ff[:, a, perm[i]] = f_t[a, i, flat].astype(np.float64) + wg[i] * nref[a]
    post = orc.collide_local(lat, ff, gn[:, flat].T.copy(), np.transpose(gj[:, :, flat], (2, 0, 1)).copy(),
                             np.transpose(oacc, (2, 0, 1)).copy())
    post = post.reshape(len(sites), 19, 2, 19)
    expect = np.empty((2, 19, len(sites)))
    got = np.empty((2, 19, len(sites)))
    for a in range(2):
        for i in range(19):
            expect[a, i] = post[:, i, a, perm[i]] - wg[i] * nref[a]
            got[a, i] = f_t1[a, i, sites]
    assert rel(got, expect) < TOL_STATE


@pytest.mark.parametrize("sigma,shape,wall_axis", [
    ([1.0, 1.5], (37, 9, 19), 1),      # shell reach 1: 2 x-tiles (one partial), 3 y-tiles, 2 z-chunks
    ([1.0, 2.0], (45, 11, 35), 2),     # shell reach 2, walls normal to z
    ([1.25, 1.5, 2.0], (33, 7, 18), -1),
])
def test_tiled_kernels_ragged_boxes(gpu, orc, sigma, shape, wall_axis):
    """The shared-memory tiled force passes on boxes that leave partial tiles
    and partial z-chunks, periodic and with walls on different axes."""
    S = len(sigma)
    lat = W.Lattice(shape=shape, sigma=sigma, tau=0.9, wall_axis=wall_axis,
                    wall_u_lo=tuple(0.0 if k == wall_axis else (0.01 if k == 0 else 0.0) for k in range(3)) if wall_axis >= 0 else (0, 0, 0),
                    wall_u_hi=tuple(0.0 if k == wall_axis else (-0.02 if k == 0 else 0.0) for k in range(3)) if wall_axis >= 0 else (0, 0, 0))
    n0 = W.densities_from_packing(0.15, sigma, [1.0 / S] * S)
    n = W.noise(lat, n0, 0.05, seed=31)
    u = W.random_velocities(lat, 0.005, seed=32)
    w = run_pair(gpu, orc, lat, n, u, checkpoints=(0, 1, 25))
    assert ok(w), w


def test_conservation_is_the_fp64_sum_of_the_populations(gpu):
    """mlb_conservation (Eqs. continuity, momentcomponent) equals the FP64
    host sum of the stored populations plus w_i n_ref to 1e-12, on a 128^3
    state with flow."""
    lat, n = W.binary_config1((128, 128, 128))
    sim = gpu.Simulation(lat)
    sim.set_fields(n, W.random_velocities(lat, 0.01, seed=6))
    sim.step(3)
    mass, mom = sim.conservation()
    f, nref, _ = sim.populations()
    sim.close()
    c, w = gpu.velocity_set()
    S = lat.nspecies
    hm = np.array([(f[a].astype(np.float64) + (w * nref[a])[:, None]).sum() for a in range(S)])
    hp = np.zeros(3)
    for a in range(S):
        fa = f[a].astype(np.float64) + (w * nref[a])[:, None]
        hp += c.T.astype(np.float64) @ fa.sum(1)
    assert np.all(np.abs(mass - hm) <= 1e-12 * hm), (mass, hm)
    assert np.all(np.abs(mom - hp) <= 1e-12 * hm.sum() * math.sqrt(1 / 3)), (mom, hp)


def test_monitored_steps_report_the_conservation_sums(gpu):
    """mlb_step_monitored: the same populations as mlb_step, and per step the
    FP64 sums of the state the step starts from, within the stated bound of
    mlb_conservation's (FP32 site moments summed in 8-site FP32 groups:
    8 x 2^-24 x sum|dn| for a mass, 8 x 2^-24 x sum|j| per momentum
    component)."""
    import torch
    lat, n = W.binary_config1((40, 12, 10))
    u = W.random_velocities(lat, 0.01, seed=3)
    a = gpu.Simulation(lat)
    b = gpu.Simulation(lat)
    a.set_fields(n, u)
    b.set_fields(n, u)
    S = lat.nspecies
    bufs = [torch.empty(S + 3, dtype=torch.float64, pin_memory=True).numpy() for _ in range(6)]
    for k in range(6):
        a.step_monitored(bufs[k])
    a.synchronize()
    for k in range(6):
        m, p = b.conservation()
        gn, gu = b.moments()
        nref = b.populations()[1]
        bound_m = 8 * 2.0 ** -24 * np.abs(gn - nref[:, None]).sum(1) + 1e-12 * m
        bound_p = 8 * 2.0 ** -24 * np.abs(gn[:, None, :] * gu).sum((0, 2)) + 1e-12 * m.sum()
        assert np.all(np.abs(bufs[k][:S] - m) <= bound_m), (bufs[k][:S], m)
        assert np.all(np.abs(bufs[k][S:S + 3] - p) <= bound_p), (bufs[k][S:S + 3], p)
        b.step(1)
    assert np.array_equal(a.populations()[0].view(np.uint32), b.populations()[0].view(np.uint32))
    a.close()
    b.close()


@pytest.mark.parametrize("case,sweeps", [
    ("config1", 2),              # the benchmark physics, cube tiles, 500 steps
    ("attraction", 3),           # sigma = 2/3 with tails: reach-3 tiles, the column attraction kernel
    ("drag_walls", 2),           # drag only (partner u* at the site), reach-2 tiles, walls normal to z
    ("reach4", 2),               # the global-memory passes
    ("channel3", 2),             # three species between moving walls (sigma 2, 2.5, 3; contact-value balls)
])
def test_predictor_sweeps_match_the_oracle(gpu, orc, case, sweeps):
    """Further Jacobi sweeps of the half step on the GPU against the oracle
    with the same sweeps (partners at the previous sweep's u*)."""
    if case == "config1":
        lat, n = W.binary_config1()
        u, cps = None, (0, 1, 100, 500)
    elif case == "attraction":
        lat, n = W.binary_attraction((18, 16, 17), seed=11)
        u, cps = None, (0, 1, 20, 60)
    elif case == "drag_walls":
        lat = W.Lattice(shape=(36, 10, 12), sigma=[2.0, 1.5], drag_only=True, wall_axis=2,
                        wall_u_lo=(-0.02, 0.0, 0.0), wall_u_hi=(0.02, 0.0, 0.0))
        n = W.noise(lat, W.densities_from_packing(0.2, lat.sigma, [0.5, 0.5]), 0.03, seed=7)
        u, cps = W.random_velocities(lat, 0.01, seed=5), (0, 1, 40)
    elif case == "channel3":
        lat, n = W.taylor_channel((40, 16, 10), U=0.05)
        n[2] = n[2] * 1e3 / 8
        u, cps = None, (0, 1, 40)
    else:
        lat = W.Lattice(shape=(20, 16, 14), sigma=[4.0, 3.0], tau=0.9)
        n = W.noise(lat, W.densities_from_packing(0.2, lat.sigma, [0.5, 0.5]), 0.02, seed=41)
        u, cps = W.random_velocities(lat, 0.005, seed=42), (0, 1, 40)
    lat.predictor_sweeps = sweeps
    rep = []
    w = run_pair(gpu, orc, lat, n, u, checkpoints=cps, report=rep)
    print(case, sweeps, rep)
    assert ok(w), w


def test_measured_peaks_are_plausible(gpu):
    """The project's peak probes: the FP32 FMA kernel reaches most of the
    nominal rate (152 SMs x 128 lanes x 2 flops at up to 2.07 GHz = 80.5
    TFLOP/s), and the copy kernel most of the HBM3e bandwidth."""
    tf = gpu.fma_throughput(1 << 12, 3)
    assert 40.0 < tf < 82.0, tf
    gbs = gpu.copy_bandwidth(1 << 30, 3)
    assert 3000.0 < gbs < 8500.0, gbs
    with pytest.raises(gpu.MLBError):
        gpu.fma_throughput(0, 1)
