"""The FP64 oracle behind the Simulation interface the measurement drivers
(paper_1105_3634_gb300.taylor) use: set_fields, set_external_force, step,
moments, close.  Test infrastructure: lets one measurement routine run the
same experiment on the GPU and on the oracle with identical inputs."""
import types

import oracle


class OracleSim:
    def __init__(self, lat, **_):
        self.lat = lat
        self.f = None
        self.fext = None

    def set_fields(self, n, u=None):
        self.f = oracle.init(self.lat, n, u)

    def set_external_force(self, fext):
        self.fext = fext

    def step(self, nsteps):
        if nsteps > 0:
            oracle.step(self.lat, self.f, int(nsteps), self.fext)

    def moments(self):
        n, j = oracle.moments(self.lat, self.f)
        return n, oracle.velocity_fields(self.lat, n, j)

    def close(self):
        self.f = None


def module():
    """A stand-in for the binding module: module().Simulation(lat) runs on the oracle."""
    oracle.build()
    return types.SimpleNamespace(Simulation=OracleSim)
