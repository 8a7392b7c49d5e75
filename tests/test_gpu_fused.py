"""The volume kernel with on-chip interface fluxes (tile variants 3..5: k_volume
evaluates the interface flux at both ends of each line from the neighbours' parameter
vectors, and k_face is not launched; FP32 fluxes on periodic Euler meshes) against
k_prep + k_face + k_volume (variants 0..2): bit-identical right-hand sides, element
sums, relaxed advances and batches, on ragged meshes that span several tiles with a
ragged last one (p = 2..5; both mixed modes; entropy-conservative, Rusanov and matrix
interface dissipation).  The mixed modes' parity with the oracle is covered by the
tests of test_gpu_parity.py, test_gpu_batch.py and test_gpu_fullsize.py on the
default variant 0, which these tests tie to 3..5 bit for bit."""
import numpy as np
import pytest

from oracle import dg
from paper_2003_08831_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def state(p, n, lo, hi, seed):
    mesh = dg.Mesh(p, n, lo, hi)
    x, y, z = mesh.coords()
    rng = np.random.default_rng(seed)
    U = inputs.tgv_state(x + 0.1, y, z, mach=0.3)
    return U * (1 + 1e-3 * rng.uniform(-1, 1, U.shape))


CASES = [(2, (5, 3, 4), 1), (3, (7, 3, 5), 1), (3, (4, 4, 4), 0), (4, (3, 5, 3), 2), (5, (3, 2, 3), 1)]


@pytest.mark.parametrize("precision", [1, 3])
@pytest.mark.parametrize("p,n,diss", CASES)
def test_fused_rhs_bit_identical(p, n, diss, precision):
    from paper_2003_08831_gb300.solver import Solver
    lo, hi = (0.0, 0.0, 0.0), (2 * np.pi,) * 3
    U = state(p, n, lo, hi, seed=p)
    s = Solver(p, n, lo, hi, precision=precision, interface_diss=diss)
    assert s.volume_variant() == 0
    q = s.to_device(U)
    out = {}
    for v in range(6):
        s.set_volume_variant(v)
        dq, E = s.rhs(q, want_E=True)
        assert s.status() == 0
        out[v] = (dq.cpu().numpy(), E.cpu().numpy())
    s.close()
    for v in range(1, 6):
        assert np.array_equal(out[v][0], out[0][0]), v
        assert np.array_equal(out[v][1], out[0][1]), v


@pytest.mark.parametrize("precision", [1, 3])
@pytest.mark.parametrize("p,n,diss", CASES)
def test_fused_advance_bit_identical(p, n, diss, precision):
    from paper_2003_08831_gb300.solver import Solver, stable_dt
    lo, hi = (0.0, 0.0, 0.0), (2 * np.pi,) * 3
    U = state(p, n, lo, hi, seed=10 + p)
    s = Solver(p, n, lo, hi, precision=precision, interface_diss=diss)
    dt = stable_dt(U, p, [(hi[m] - lo[m]) / n[m] for m in range(3)], 0.5)
    res = {}
    for v in (0, 3, 4, 5):
        s.set_volume_variant(v)
        q = s.to_device(U)
        t, gh, gk = s.advance(q, 4, dt)
        assert s.status() == 0
        res[v] = (q.cpu().numpy(), t.item(), gh.cpu().numpy(), gk.cpu().numpy())
    s.close()
    for v in (3, 4, 5):
        assert np.array_equal(res[v][0], res[0][0]), v
        assert res[v][1] == res[0][1]
        assert np.array_equal(res[v][2], res[0][2]) and np.array_equal(res[v][3], res[0][3])


def test_fused_variant_availability():
    """The on-chip interface fluxes serve FP32 fluxes on periodic Euler meshes only: FP64,
    FP64X and Navier--Stokes contexts reject the variants, boundaries fall back to the
    same tile with k_face."""
    from paper_2003_08831_gb300 import _binding as B
    from paper_2003_08831_gb300.solver import Solver
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    for kw in (dict(precision=0), dict(precision=2), dict(precision=1, mu=0.01)):
        s = Solver(3, (2, 2, 2), lo, hi, **kw)
        assert s.volume_variant() < 3
        with pytest.raises(B.ESError):
            s.set_volume_variant(3)
        s.close()
    s = Solver(3, (4, 2, 2), lo, hi, precision=1)
    s.set_volume_variant(4)
    s.set_boundary(0, B.ES_BC_STATE, [1.0, 0.0, 0.0, 0.0, 2.5] * 2)
    assert s.volume_variant() == 1
    with pytest.raises(B.ESError):
        s.set_volume_variant(7)
    s.close()


@pytest.mark.parametrize("precision", [1, 3])
def test_fused_batch_equals_unfused_contexts(precision):
    """A mixed batch (degrees 2..5, autotuned over all six variants) against each
    instance in its own context on tile 0 with k_face: bit-identical states after 3
    steps."""
    from paper_2003_08831_gb300.solver import BatchSolver, Solver, stable_dt
    params = inputs.batch_instances(8, seed=5, nmin=2, nmax=4)
    insts = [dict(p=d["p"], n=(d["n"],) * 3, lo=(0.0, 0.0, 0.0), hi=(d["box"],) * 3) for d in params]
    b = BatchSolver(insts, precision=precision)
    q0s, dts = [], []
    for i, d in enumerate(params):
        xyz = b.coords(i)
        q0 = inputs.vortex_state(xyz[0], xyz[1], 0.0, eps=d["eps"], mach=d["mach"], centre=d["centre"],
                                 period=d["box"])
        b.set_state(i, q0)
        q0s.append(q0)
        dts.append(stable_dt(q0, d["p"], [d["box"] / d["n"]] * 3, 0.5))
    b.set_dt(dts)
    b.autotune()
    b.advance(3)
    assert b.status() in (0, -4)
    for i, d in enumerate(insts):
        s = Solver(d["p"], d["n"], d["lo"], d["hi"], precision=precision)
        s.set_volume_variant(0)
        q = s.to_device(q0s[i])
        s.advance(q, 3, dts[i])
        assert np.array_equal(q.cpu().numpy(), b.get_state(i).reshape(q.shape)), i
        s.close()
    b.close()


@pytest.mark.parametrize("precision", [2, 3])
def test_eight_stage_tableau_float_float(precision):
    """A loaded 8-stage tableau (a_ij = 1/8 below the diagonal, b_i = 1/8, c_i = i/8): the
    last stage forms d from seven earlier stages' values in float-float (ES_FP64X,
    ES_MIXED_FF) -- more than the built-in tableaux need -- against the oracle with the
    same tableau: state within 1e-12 per variable (FP64X) or 1e-5 relative L2 (mixed)."""
    from oracle import rk
    from paper_2003_08831_gb300.solver import Solver
    s_ = 8
    A = np.tril(np.full((s_, s_), 1.0 / s_), -1)
    b = np.full(s_, 1.0 / s_)
    c = A.sum(axis=1)
    tab = {"name": "EU8", "A": A, "b": b, "c": c, "order": 1}
    lo, hi = (0.0, 0.0, 0.0), (10.0, 10.0, 10.0)
    mesh = dg.Mesh(2, (3, 3, 3), lo, hi)
    x, y, _ = mesh.coords()
    U = inputs.vortex_state(x, y, 0.0, centre=(5.0, 5.0))
    phys = dg.Physics(1.4, diss=1)
    dt = rk.stable_dt(mesh, U, phys, 0.5)
    Uo, to, _ = rk.advance(mesh, U, dt, 3, phys, tab)
    s = Solver(2, (3, 3, 3), lo, hi, precision=precision)
    s.set_tableau(A, b, c)
    q = s.to_device(U)
    t, gh, gk = s.advance(q, 3, dt)
    assert s.status() == 0
    a, r = q.cpu().numpy().reshape(5, -1), Uo.reshape(5, -1)
    if precision == 2:
        scale = np.maximum(np.max(np.abs(r), axis=1), 1e-3 * np.max(np.abs(r)))
        assert np.all(np.max(np.abs(a - r), axis=1) <= 1e-12 * scale)
    else:
        nr = np.sqrt(np.sum(r * r, axis=1))
        nr = np.maximum(nr, 1e-3 * nr.max())
        assert np.all(np.sqrt(np.sum((a - r) ** 2, axis=1)) <= 1e-5 * nr)
    s.close()
