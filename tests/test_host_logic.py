"""Host-side harness rules shared by the benchmark and the tests (CPU)."""
import numpy as np
import pytest

from oracle import dg, rk
from paper_2003_08831_gb300 import inputs
from paper_2003_08831_gb300.solver import stable_dt


@pytest.mark.parametrize("mu", [0.0, 1.0 / 1600.0, 0.05])
def test_stable_dt_matches_the_oracle_rule(mu):
    """The package's fixed-time-step rule (used by the benchmark on host arrays) and the
    oracle's agree: the same reading of the unstated CFL condition."""
    mesh = dg.Mesh(3, (4, 3, 5), (0.0, 0.0, 0.0), (2 * np.pi, 2.0, 3.0))
    x, y, z = mesh.coords()
    U = inputs.tgv_state(x, y, z, mach=0.3)
    phys = dg.Physics(1.4, mu=mu, Pr=0.72)
    ref = rk.stable_dt(mesh, U, phys, 0.5)
    got = stable_dt(mesh.flat(U), 3, list(mesh.h), 0.5, mu=mu, Pr=0.72)
    assert abs(got - ref) <= 1e-15 * ref
