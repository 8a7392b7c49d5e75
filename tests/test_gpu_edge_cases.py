"""Edge cases of the CUDA path, against the FP64 oracle and against itself.

* The smallest meshes: one element, periodic in all three directions (every face joins
  the element to itself, so each interface flux is taken between the element's own
  opposite faces), and meshes one element thick in one or two directions -- the
  right-hand side at the FP64 bars of test_gpu_parity, and the tile variants of the
  mixed modes bit-identical to one another on them.
* Zero steps: es_advance with nsteps = 0 leaves the state and t untouched.
* A free stream (uniform state): no change, so every element's relative change
  delta_kappa is at the rounding level, below the degenerate-element floor; every
  element is unconstrained (gamma_kappa = +inf), gamma = 1 and t advances by dt per step,
  as in the oracle (Section 2: gamma_kappa solves the estimate equation only where the
  element's state changes).
* A batch of one- and two-element instances of every degree: bit-identical to each
  instance advanced alone, and each such instance at the oracle's bars.
"""
import numpy as np
import pytest

from oracle import dg, rk
from paper_2003_08831_gb300 import inputs
from test_gpu_parity import assert_rhs_close, compare_advance, random_state

pytestmark = pytest.mark.gpu
G = 1.4


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def solver(p, n, lo, hi, **kw):
    from paper_2003_08831_gb300.solver import Solver
    return Solver(p, n, lo, hi, **kw)


SMALL = [
    (2, (1, 1, 1), 0.0, 1),
    (5, (1, 1, 1), 0.0, 1),
    (3, (1, 2, 1), 0.02, 1),
    (4, (2, 1, 1), 0.0, 2),
    (2, (1, 1, 3), 0.05, 0),
]


@pytest.mark.parametrize("p,n,mu,diss", SMALL)
def test_rhs_smallest_meshes(p, n, mu, diss):
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.5, 2.0)
    mesh = dg.Mesh(p, n, lo, hi)
    U = random_state(mesh, seed=31 + p)
    phys = dg.Physics(G, mu=mu, Pr=0.72, diss=diss)
    ref = dg.rhs(mesh, U, phys)
    s = solver(p, n, lo, hi, mu=mu, interface_diss=diss)
    dq, _ = s.rhs(s.to_device(U), want_E=True)
    assert s.status() == 0
    assert_rhs_close(dq.cpu().numpy(), ref, dg.rhs_term_magnitude(mesh, U, phys))
    s.close()


@pytest.mark.parametrize("p,n", [(2, (1, 1, 1)), (3, (1, 1, 2)), (5, (1, 2, 1))])
@pytest.mark.parametrize("precision", [1, 3])
def test_tile_variants_bit_identical_on_smallest_meshes(p, n, precision):
    """Every volume tile variant (those forming the interface fluxes in the kernel too:
    FP32 fluxes, periodic Euler) gives the same bits on meshes smaller than one tile."""
    import torch
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.5, 2.0)
    mesh = dg.Mesh(p, n, lo, hi)
    U = random_state(mesh, seed=5 + p)
    s = solver(p, n, lo, hi, precision=precision)
    q = s.to_device(U)
    out = []
    for v in range(6):
        s.set_volume_variant(v)
        out.append(s.rhs(q).clone())
    torch.cuda.synchronize()
    assert s.status() == 0
    for v in range(1, 6):
        assert torch.equal(out[v], out[0]), v
    s.close()


def test_zero_steps_leave_state_and_time():
    import torch
    mesh = dg.Mesh(3, (3, 2, 2), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    U = random_state(mesh, seed=2)
    s = solver(3, (3, 2, 2), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    q = s.to_device(U)
    q0 = q.clone()
    t = torch.full((1,), 0.25, dtype=torch.float64, device="cuda")
    s.advance(q, 0, 1e-3, t=t, want_hist=False, want_gamma_elem=False)
    torch.cuda.synchronize()
    assert s.status() == 0
    assert torch.equal(q, q0)
    assert t.item() == 0.25
    s.close()


def free_stream(mesh):
    x, _, _ = mesh.coords()
    def f(c):
        return np.full(x.shape, c)
    return inputs.conserved(f(1.0), f(0.3), f(-0.2), f(0.1), f(1.0), G)


@pytest.mark.parametrize("p,n,mu", [(3, (2, 3, 1), 0.0), (4, (1, 2, 2), 0.01)])
def test_free_stream_every_element_unconstrained(p, n, mu):
    import torch
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.5, 2.0)
    mesh = dg.Mesh(p, n, lo, hi)
    U = free_stream(mesh)
    phys = dg.Physics(G, mu=mu, Pr=0.72, diss=1)
    g = compare_advance(mesh, U, lo, hi, phys, "BS3", 3)
    assert np.all(g == 1.0)
    # the same run once more for gamma_kappa, t and the state
    dt = rk.stable_dt(mesh, U, phys, 0.5)
    s = solver(p, n, lo, hi, mu=mu)
    q = s.to_device(U)
    t, hist, gk = s.advance(q, 3, dt)
    assert s.status() == 0
    assert np.all(np.isposinf(gk.cpu().numpy()))
    assert np.all(hist.cpu().numpy() == 1.0)
    assert t.item() == 3 * dt or abs(t.item() - 3 * dt) <= 4 * np.finfo(float).eps * 3 * dt
    U0 = torch.as_tensor(U.reshape(5, -1))
    err = (q.cpu().reshape(5, -1) - U0).abs().max(dim=1).values / U0.abs().max(dim=1).values
    assert torch.all(err < 1e-13), err
    s.close()


def smooth_state(x, y, z, L):
    c = lambda a, k, v: np.cos(2 * np.pi * v / L[k] + a)
    return inputs.conserved(1.0 + 0.1 * c(0.3, 0, x), 0.3 + 0.05 * c(1.1, 1, y), -0.2 + 0.05 * c(2.0, 2, z),
                            0.1 + 0.05 * c(0.7, 0, y), 1.0 + 0.1 * c(1.9, 1, z), G)


TINY = [dict(p=2, n=(1, 1, 1)), dict(p=5, n=(1, 1, 1)), dict(p=3, n=(2, 1, 1)), dict(p=4, n=(1, 2, 1)),
        dict(p=2, n=(1, 1, 3)), dict(p=3, n=(1, 1, 1))]


def test_batch_of_tiny_instances():
    """One captured graph over instances of one and two elements (several instances
    inside one tile of the flux kernel): bit-identical to each instance alone."""
    from paper_2003_08831_gb300.solver import BatchSolver, Solver
    insts = [dict(d, lo=(0.0, 0.0, 0.0), hi=(1.0 + 0.1 * i, 1.5, 2.0)) for i, d in enumerate(TINY)]
    b = BatchSolver(insts)
    dts, q0s = [], []
    for i, inst in enumerate(insts):
        xyz = b.coords(i)
        q0 = smooth_state(xyz[0], xyz[1], xyz[2], np.array(inst["hi"]) - np.array(inst["lo"]))
        b.set_state(i, q0)
        mesh = dg.Mesh(inst["p"], inst["n"], inst["lo"], inst["hi"])
        dts.append(rk.stable_dt(mesh, mesh.unflat(q0), dg.Physics(G, diss=1), 0.5))
        q0s.append(q0)
    b.set_dt(dts)
    nsteps = 3
    b.advance(nsteps)
    assert b.status() == 0
    for i, inst in enumerate(insts):
        s = Solver(inst["p"], inst["n"], inst["lo"], inst["hi"])
        q = s.to_device(q0s[i])
        s.advance(q, nsteps, dts[i])
        assert s.status() == 0
        assert np.array_equal(q.cpu().numpy(), b.get_state(i)), i
        s.close()
    b.close()


@pytest.mark.parametrize("p,n", [(5, (1, 1, 1)), (2, (1, 1, 3))])
def test_tiny_instance_advance_against_oracle(p, n):
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.5, 2.0)
    mesh = dg.Mesh(p, n, lo, hi)
    x, y, z = mesh.coords()
    U = smooth_state(x, y, z, np.array(hi) - np.array(lo))
    compare_advance(mesh, U, lo, hi, dg.Physics(G, diss=1), "BS3", 4)
