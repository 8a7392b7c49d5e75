"""Dirichlet-penalty boundaries and the viscous-shock study (Section 4.1.2) on the GPU.

Parity with the oracle (same bars as test_gpu_parity): es_rhs with prescribed
boundary states in each direction, es_advance of the moving viscous shock (stage
times t + c_i dt enter the boundary states), FP64 and FP64X; then the convergence
study of Table 2 at the paper's sizes on N x 1 x 1 meshes (the solution varies
only along x1, so the periodic x2, x3 directions are exact).
"""
import numpy as np
import pytest

from oracle import dg, rk
from paper_2003_08831_gb300 import inputs
from test_gpu_parity import G, TOL, EPS, assert_rhs_close, rel_err_per_var, solver

pytestmark = pytest.mark.gpu
EPS_FF = 2.0 ** -47
SHOCK = (2.5, 10.0, 0.75)   # Mach, Reynolds, Prandtl of Section 4.1.2


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _B():
    from paper_2003_08831_gb300 import _binding as B
    return B


def _rk(tab):
    B = _B()
    return {"BS3": B.ES_RK_BS3, "RK4": B.ES_RK_RK4, "RK65": B.ES_RK_RK65}[tab]


def shock_setup(p, n, speed=-1.0, nyz=(1, 1)):
    prm = inputs.viscous_shock_parameters(*SHOCK)
    h = 1.0 / n
    lo = (-0.5, -0.5 * h * nyz[0], -0.5 * h * nyz[1])
    hi = (0.5, 0.5 * h * nyz[0], 0.5 * h * nyz[1])

    def left(t):
        return inputs.viscous_shock_state(np.array(lo[0]), t, prm, speed)

    def right(t):
        return inputs.viscous_shock_state(np.array(hi[0]), t, prm, speed)
    mesh = dg.Mesh(p, (n, nyz[0], nyz[1]), lo, hi, bc={0: (left, right)})
    phys = dg.Physics(G, mu=prm["mu"], Pr=prm["prandtl"], diss=1)
    return mesh, phys, prm, lo, hi


def gpu_shock_solver(mesh, phys, lo, hi, speed=-1.0, **kw):
    B = _B()
    s = solver(mesh.p, mesh.n, lo, hi, mu=phys.mu, Pr=phys.Pr, interface_diss=phys.diss, **kw)
    s.set_boundary(0, B.ES_BC_VISCOUS_SHOCK, list(SHOCK) + [speed])
    return s


@pytest.mark.parametrize("p,n,nyz,t,prec", [(2, 5, (1, 1), 0.0, 0), (3, 4, (2, 3), 0.13, 0), (4, 3, (1, 2), 0.31, 0),
                                           (3, 4, (2, 1), 0.13, 2)])
def test_shock_rhs_parity(p, n, nyz, t, prec):
    mesh, phys, prm, lo, hi = shock_setup(p, n, nyz=nyz)
    x, _, _ = mesh.coords()
    # a state near the profile, perturbed so that the boundary jumps are not zero
    U = inputs.viscous_shock_state(x + 0.03, t, prm)
    U = U * (1.0 + 0.01 * np.sin(7.0 * x))
    ref = dg.rhs(mesh, U, phys, t)
    s = gpu_shock_solver(mesh, phys, lo, hi, precision=prec)
    s.set_time(t)
    dq = s.rhs(s.to_device(U)).cpu().numpy()
    assert s.status() == 0
    assert_rhs_close(dq, ref, dg.rhs_term_magnitude(mesh, U, phys, t), eps=EPS if prec == 0 else EPS_FF)
    s.close()


@pytest.mark.parametrize("direction", [1, 2])
def test_state_boundary_rhs_parity(direction):
    """Constant prescribed states on the faces of x2 or x3 (Euler and Navier--Stokes)."""
    B = _B()
    rng = np.random.default_rng(direction)
    qL = inputs.conserved(np.array(1.1), np.array(0.2), np.array(-0.3), np.array(0.1), np.array(0.9), G)
    qR = inputs.conserved(np.array(0.8), np.array(-0.1), np.array(0.25), np.array(0.3), np.array(1.2), G)
    for p, n, mu in [(2, (3, 4, 5), 0.0), (3, (2, 3, 4), 0.02)]:
        lo, hi = (0.0, 0.0, 0.0), (0.8, 1.0, 1.3)
        mesh = dg.Mesh(p, n, lo, hi, bc={direction: (lambda t: qL, lambda t: qR)})
        x, y, z = mesh.coords()
        U = inputs.conserved(1.0 + 0.1 * np.sin(3 * x + y), 0.1 * np.cos(2 * z), 0.2 * np.sin(y), -0.1 + 0.05 * x,
                             1.0 + 0.1 * np.cos(x * y), G)
        U = U * (1.0 + 0.01 * rng.uniform(-1, 1, U.shape))
        phys = dg.Physics(G, mu=mu, Pr=0.72, diss=1)
        ref = dg.rhs(mesh, U, phys, 0.0)
        s = solver(p, n, lo, hi, mu=mu, Pr=0.72, interface_diss=1)
        s.set_boundary(direction, B.ES_BC_STATE, list(qL) + list(qR))
        dq = s.rhs(s.to_device(U)).cpu().numpy()
        assert s.status() == 0
        assert_rhs_close(dq, ref, dg.rhs_term_magnitude(mesh, U, phys, 0.0))
        s.close()


@pytest.mark.parametrize("p,n,nyz,t,alpha,prec", [(3, 4, (2, 1), 0.13, 1.0, 0), (2, 5, (1, 2), 0.21, 0.5, 0),
                                                  (3, 4, (2, 1), 0.13, 1.0, 2)])
def test_shock_rhs_parity_viscous_interface_dissipation(p, n, nyz, t, alpha, prec):
    """diss^V with Dirichlet-penalty boundaries: the penalty also acts between the
    interior and the prescribed exterior state on the boundary faces."""
    mesh, phys, prm, lo, hi = shock_setup(p, n, nyz=nyz)
    phys = dg.Physics(G, mu=prm["mu"], Pr=prm["prandtl"], diss=1, visc_diss=alpha)
    x, _, _ = mesh.coords()
    U = inputs.viscous_shock_state(x + 0.03, t, prm)
    U = U * (1.0 + 0.01 * np.sin(7.0 * x))
    ref = dg.rhs(mesh, U, phys, t)
    s = gpu_shock_solver(mesh, phys, lo, hi, precision=prec, visc_diss=alpha)
    s.set_time(t)
    dq = s.rhs(s.to_device(U)).cpu().numpy()
    assert s.status() == 0
    assert_rhs_close(dq, ref, dg.rhs_term_magnitude(mesh, U, phys, t), eps=EPS if prec == 0 else EPS_FF)
    s.close()


@pytest.mark.parametrize("prec,tab", [(0, "BS3"), (0, "RK4"), (2, "RK4")])
def test_shock_advance_parity(prec, tab):
    """Relaxed steps of the moving shock: state 1e-12 per variable against the oracle."""
    B = _B()
    p, n = 3, 4
    mesh, phys, prm, lo, hi = shock_setup(p, n, nyz=(1, 2))
    x, _, _ = mesh.coords()
    U = inputs.viscous_shock_state(x, 0.0, prm)
    dt = 0.03 / n ** 2
    nsteps = 12
    Uo, to, hist = rk.advance(mesh, U, dt, nsteps, phys, rk.TABLEAUX[tab])
    s = gpu_shock_solver(mesh, phys, lo, hi, precision=prec, rk=_rk(tab))
    q = s.to_device(U)
    t, gh, gk = s.advance(q, nsteps, dt)
    assert s.status() == 0
    err = rel_err_per_var(q.cpu().numpy(), Uo)
    assert np.all(err < TOL), err
    assert abs(t.item() - to) <= 1e-12 * to
    s.close()


@pytest.mark.parametrize("p,tab,rate_min,diss,alpha", [(2, "BS3", 2.5, 1, 0.0), (3, "RK4", 3.5, 1, 0.0),
                                                       (2, "BS3", 2.75, 2, 0.0), (3, "RK4", 3.5, 1, 0.25),
                                                       (4, "RK65", 4.5, 1, 0.0)])
def test_viscous_shock_convergence(p, tab, rate_min, diss, alpha):
    """Table 2's study at N = 10, 15, 20 to t = 0.5 with U dt/dx^2 fixed: least-squares L2
    density rate above p + 1/2 (the paper observes 3.1 for p = 2, 3.4-4.0 for p = 3; at
    N = 5 both are pre-asymptotic).  The errors are of the size Table 2 lists (p = 3,
    N = 20: 1.8e-5 here, 1.05e-5 there).  With the matrix interface dissipation
    (diss = 2) the p = 2 rate is the paper's (2.9-3.0 here, 3.1 there; 2.6 with Rusanov).
    The diss^V penalty (alpha = 0.25) leaves the p = 3 errors within 7 % and the rate at 4.4.
    p = 4 with the fifth-order RK(6,5) (Table 2 pairs p = 4 with a fifth-order method):
    rate 4.8 over N = 10..20."""
    B = _B()
    errs = []
    Ns = (10, 15, 20)
    for n in Ns:
        mesh, phys, prm, lo, hi = shock_setup(p, n)
        phys = dg.Physics(G, mu=prm["mu"], Pr=prm["prandtl"], diss=diss)
        x, _, _ = mesh.coords()
        U = inputs.viscous_shock_state(x, 0.0, prm)
        dt = 0.03 / n ** 2
        nsteps = int(np.ceil(0.5 / dt))
        s = gpu_shock_solver(mesh, phys, lo, hi, rk=_rk(tab), visc_diss=alpha)
        q = s.to_device(U)
        t, gh, _ = s.advance(q, nsteps, dt)
        assert s.status() == 0
        g = gh.cpu().numpy()
        assert np.all(np.abs(g - 1.0) < 1e-2)
        exact = inputs.viscous_shock_state(x, t.item(), prm)
        err = q.cpu().numpy().reshape(mesh.shape)[0] - exact[0]
        errs.append(np.sqrt(np.sum(mesh.mass() * err * err) / (1.0 / n) ** 2))
        s.close()
    rate = -np.polyfit(np.log2(np.array(Ns, dtype=float)), np.log2(errs), 1)[0]
    assert rate > rate_min, (errs, rate)


def _table2():
    rows, tol = [], None
    import os
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "viscous_shock_table2.txt")):
        line = line.split("#")[0].split()
        if not line:
            continue
        if line[0] == "tolerance":
            tol = float(line[1])
        else:
            rows.append((int(line[0]), line[1], int(line[2]), float(line[3])))
    return rows, tol


def test_viscous_shock_table2_errors():
    """The N = 5 density errors of Table 2 (L2 over the domain, t = 0.5) within the stated band."""
    B = _B()
    rows, tol = _table2()
    for p, tab, n, ref in rows:
        mesh, phys, prm, lo, hi = shock_setup(p, n)
        x, _, _ = mesh.coords()
        U = inputs.viscous_shock_state(x, 0.0, prm)
        dt = 0.03 / n ** 2
        s = gpu_shock_solver(mesh, phys, lo, hi, rk=_rk(tab))
        q = s.to_device(U)
        t, _, _ = s.advance(q, int(np.ceil(0.5 / dt)), dt)
        assert s.status() == 0
        e = q.cpu().numpy().reshape(mesh.shape)[0] - inputs.viscous_shock_state(x, t.item(), prm)[0]
        l2 = np.sqrt(np.sum(mesh.mass() * e * e) / (1.0 / n) ** 2)
        s.close()
        assert abs(l2 - ref) <= tol * ref, (p, l2, ref)
