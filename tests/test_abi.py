"""CPU checks of the C-ABI library: it builds, loads, and exports every
function include/mlb.h declares; host-side validation that needs no GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mlbmod():
    from paper_1105_3634_gb300 import build
    build.build()
    from paper_1105_3634_gb300 import mlb
    return mlb


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "mlb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mlb_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ["mlb_create", "mlb_set_species", "mlb_set_interactions", "mlb_set_fields", "mlb_step",
                 "mlb_get_moments", "mlb_get_acceleration", "mlb_conservation", "mlb_get_populations",
                 "mlb_set_populations", "mlb_last_error", "mlb_destroy"]:
        assert must in names


def test_library_exports_every_declared_symbol(mlbmod):
    lib = ctypes.CDLL(mlbmod.LIB_PATH)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_velocity_set_is_d3q19(mlbmod):
    c, w = mlbmod.velocity_set()
    assert len(w) == 19 and abs(w.sum() - 1) < 1e-15
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(3) / 3, atol=1e-15)
    assert {tuple(v) for v in c} == {tuple(-v) for v in c}
    assert np.abs(np.einsum("i,ia->a", w, c)).max() < 1e-16


def _desc(mlbmod, **kw):
    d = mlbmod.mlb_lattice_desc()
    d.nx, d.ny, d.nz, d.nspecies = 8, 8, 8, 2
    d.wall_axis = -1
    d.tau, d.kT, d.kappa = 1.0, 1.0 / 3.0, 0.5
    for k, v in kw.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("field,value,word", [
    ("nspecies", 0, "nspecies"), ("nspecies", 5, "nspecies"), ("nx", 0, "extents"),
    ("tau", 0.5, "tau"), ("kT", 0.3, "kT"), ("wall_axis", 3, "wall_axis"), ("flags", 64, "flag"),
])
def test_create_rejects_bad_descriptors_before_touching_the_gpu(mlbmod, field, value, word):
    d = _desc(mlbmod, **{field: value})
    ctx = ctypes.c_void_p()
    st = mlbmod.lib.mlb_create(ctypes.byref(d), ctypes.byref(ctx))
    assert st == 1
    assert word in mlbmod.lib.mlb_last_error(ctx).decode()
    mlbmod.lib.mlb_destroy(ctx)


def test_normal_wall_velocity_rejected(mlbmod):
    d = _desc(mlbmod, wall_axis=1)
    d.wall_u_hi[1] = 0.01
    ctx = ctypes.c_void_p()
    assert mlbmod.lib.mlb_create(ctypes.byref(d), ctypes.byref(ctx)) == 1
    assert "tangential" in mlbmod.lib.mlb_last_error(ctx).decode()
    mlbmod.lib.mlb_destroy(ctx)


def test_null_arguments(mlbmod):
    assert mlbmod.lib.mlb_create(None, None) == 1
    assert mlbmod.lib.mlb_step(None, 1) == 1
    assert mlbmod.lib.mlb_last_error(None) == b"null context"
    for s in range(7):
        assert mlbmod.lib.mlb_status_string(s)


def test_new_entry_points_validate_before_touching_the_gpu(mlbmod):
    """Host-side argument checks of the surrogate network, the monitored step
    and the copy-bandwidth and FMA probes: refused with MLB_EINVAL, no device call."""
    L = mlbmod.lib
    assert L.mlb_net_param_count() == 27 * 32 * 2 + 32 + 27 * 32 * 32 + 32 + 6 * 32 + 6
    net = ctypes.c_void_p()
    dims = (ctypes.c_int32 * 3)(2, 8, 8)                  # every extent must be >= 3
    assert L.mlb_net_create(dims, ctypes.byref(net)) == 1 and not net.value
    assert L.mlb_net_create(None, ctypes.byref(net)) == 1
    out = ctypes.c_double(-1.0)
    assert L.mlb_copy_bandwidth(1 << 19, 5, ctypes.byref(out)) == 1          # below 1 MiB
    assert L.mlb_copy_bandwidth(1 << 24, 0, ctypes.byref(out)) == 1          # no repetition
    assert L.mlb_copy_bandwidth(1 << 24, 5, None) == 1
    assert L.mlb_fma_throughput(0, 5, ctypes.byref(out)) == 1                 # no iteration
    assert L.mlb_fma_throughput(64, 0, ctypes.byref(out)) == 1                # no repetition
    assert L.mlb_fma_throughput(64, 5, None) == 1
    sums = np.zeros(8)
    assert L.mlb_step_monitored(None, sums.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == 1
    assert L.mlb_attach_surrogate(None, None, 50, 0.05) == 1
