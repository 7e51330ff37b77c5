"""Taylor dispersion in the cosine flow (Sec. V, Eqs. ushape, taylordiff) on
the GPU: the kinetic model's effective diffusion of a concentration wave
across the held shear flow equals the passive-scalar result for the lattice's
own D and the flow amplitude reached, and follows Eq. taylordiff."""
import math

import pytest

from paper_1105_3634_gb300 import taylor as T
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


def test_cosine_flow_taylor_dispersion(gpu):
    lat = W.Lattice(shape=(128, 32, 4), sigma=[1.0, 1.5], tau=1.0)
    n0 = W.densities_from_packing(0.2, lat.sigma, [0.5, 0.5])
    res = T.dispersion_curve(gpu, lat, n0, [0.02, 0.04, 0.06])
    print(f"D0={res['D0']:.5f} nu={res['nu']:.5f}")
    for r in res["rows"]:
        print({k: round(v, 5) for k, v in r.items()})
    assert res["D0"] > 0 and res["nu"] > 0
    enh = []
    for r in res["rows"]:
        assert abs(r["U_reached"] - r["U"]) < 0.05 * r["U"]           # the force holds the flow
        assert abs(r["D_eff"] - r["D_eff_passive_scalar"]) < 0.03 * r["D_eff_passive_scalar"]
        enh.append(r["D_eff"] / res["D0"] - 1.0)
    # the enhancement grows as Pe^2
    assert enh[0] < enh[1] < enh[2]
    assert 3.0 < enh[1] / enh[0] < 5.0
