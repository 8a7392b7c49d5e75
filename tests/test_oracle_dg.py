"""Pins for oracle.dg: SBP-SAT identities of Section 3.1 that hold exactly.

Free-stream preservation (D 1 = 0), conservation of mass, momentum and energy
on periodic meshes, semidiscrete entropy conservation with the EC interface
flux and dissipation with Rusanov / BR1 (Eq. (estimate-no-slip-bc-2) with
BT = 0 on a periodic mesh), the BR1 identity, direction symmetry and
consistency with the exact time derivative of the isentropic vortex.
"""
import numpy as np
import pytest

from oracle import dg, gas
from paper_2003_08831_gb300 import inputs

G = 1.4


def smooth_state(mesh, seed=0, amp=0.2, noise=0.0):
    """Random periodic state: a few low Fourier modes per field, plus optional
    nodal noise (which makes the state jump across element interfaces)."""
    rng = np.random.default_rng(seed)
    x, y, z = mesh.coords()
    L = mesh.hi - mesh.lo
    def field(base, a):
        f = np.full(x.shape, base)
        for _ in range(3):
            k = rng.integers(0, 3, size=3)
            ph = rng.uniform(0, 2 * np.pi)
            f = f + a * rng.uniform(-1, 1) * np.cos(2 * np.pi * (k[0] * x / L[0] + k[1] * y / L[1] + k[2] * z / L[2]) + ph)
        return f
    rho = field(1.0, amp)
    v = np.stack([field(0.3, amp), field(-0.2, amp), field(0.1, amp)])
    p = field(1.0, amp)
    if noise:
        rho = rho * (1 + noise * rng.uniform(-1, 1, rho.shape))
        v = v + noise * rng.uniform(-1, 1, v.shape)
        p = p * (1 + noise * rng.uniform(-1, 1, p.shape))
    return gas.conserved(rho, v, p, G)


MESHES = [(2, (3, 2, 2)), (3, (2, 3, 2)), (4, (2, 2, 3))]


@pytest.mark.parametrize("p,n", MESHES)
@pytest.mark.parametrize("mu,diss", [(0.0, 0), (0.0, 1), (0.01, 1), (0.0, 2)])
def test_free_stream(p, n, mu, diss):
    mesh = dg.Mesh(p, n, (0, 0, 0), (1.0, 2.0, 1.5))
    U = np.empty(mesh.shape)
    q0 = gas.conserved(np.array(1.3), np.array([0.4, -0.7, 0.2]), np.array(0.8), G)
    U[:] = q0.reshape(5, 1, 1, 1, 1, 1, 1)
    R = dg.rhs(mesh, U, dg.Physics(G, mu=mu, diss=diss))
    assert np.max(np.abs(R)) < 1e-12


@pytest.mark.parametrize("p,n", MESHES)
@pytest.mark.parametrize("mu,diss", [(0.0, 0), (0.0, 1), (0.02, 1), (0.02, 2)])
def test_conservation(p, n, mu, diss):
    mesh = dg.Mesh(p, n, (0, 0, 0), (1.0, 2.0, 1.5))
    U = smooth_state(mesh, seed=p, noise=0.05)
    R = dg.rhs(mesh, U, dg.Physics(G, mu=mu, diss=diss))
    tot = [np.sum(mesh.element_sum(R[v])) for v in range(5)]
    scale = np.sum(mesh.element_sum(np.abs(R)))
    assert max(abs(t) for t in tot) < 1e-13 * scale


@pytest.mark.parametrize("p,n", MESHES)
def test_entropy_conservation_ec(p, n):
    mesh = dg.Mesh(p, n, (0, 0, 0), (1.0, 2.0, 1.5))
    U = smooth_state(mesh, seed=10 + p, noise=0.05)
    R = dg.rhs(mesh, U, dg.Physics(G, diss=0))
    W = gas.entropy_variables(U, G)
    prod = mesh.element_sum(np.sum(W * R, axis=0))
    scale = np.sum(mesh.element_sum(np.sum(np.abs(W * R), axis=0)))
    assert abs(np.sum(prod)) < 1e-13 * scale
    # with Rusanov interface dissipation the total entropy decreases
    R1 = dg.rhs(mesh, U, dg.Physics(G, diss=1))
    assert np.sum(mesh.element_sum(np.sum(W * R1, axis=0))) < -1e-6 * scale
    # matrix interface dissipation: decreases too, by less than the scalar Rusanov term
    R2 = dg.rhs(mesh, U, dg.Physics(G, diss=2))
    d2 = np.sum(mesh.element_sum(np.sum(W * R2, axis=0)))
    assert -np.sum(mesh.element_sum(np.sum(W * R1, axis=0))) > -d2 > 1e-8 * scale


@pytest.mark.parametrize("p,n", MESHES)
def test_br1_identity(p, n):
    """sum P w.(viscous part) = -sum P sum_m theta_m.F^V_m <= 0 on a periodic mesh."""
    mesh = dg.Mesh(p, n, (0, 0, 0), (1.0, 2.0, 1.5))
    U = smooth_state(mesh, seed=20 + p, noise=0.05)
    phys = dg.Physics(G, mu=0.05, Pr=0.72, diss=1)
    V, theta, fv = dg.viscous_term(mesh, U, phys, return_parts=True)
    W = gas.entropy_variables(U, G)
    lhs = np.sum(mesh.element_sum(np.sum(W * V, axis=0)))
    diss = np.sum(mesh.element_sum(np.sum(theta * fv, axis=(0, 1))))
    scale = np.sum(mesh.element_sum(np.sum(np.abs(W * V), axis=0)))
    assert diss > 0
    assert abs(lhs + diss) < 1e-12 * scale


@pytest.mark.parametrize("mu", [0.0, 0.03])
def test_direction_symmetry(mu):
    """A state varying along one axis gives the same RHS along x, y and z."""
    p, N = 3, 4
    phys = dg.Physics(G, mu=mu, diss=1)
    outs = []
    for m in range(3):
        n = [1, 1, 1]
        n[m] = N
        mesh = dg.Mesh(p, tuple(n), (0, 0, 0), (2.0, 2.0, 2.0))
        c = mesh.coords()[m]
        rho = 1 + 0.2 * np.sin(np.pi * c)
        vel = [0.1 + 0.3 * np.cos(np.pi * c), 0.2 * np.sin(np.pi * c), -0.1 + 0 * c]
        vel[0], vel[m] = vel[m], vel[0]      # the normal velocity follows the axis
        v = np.stack(vel)
        U = gas.conserved(rho, v, 1 + 0.1 * np.cos(np.pi * c), G)
        R = dg.rhs(mesh, U, phys)
        # bring direction m to x: swap momentum components 0 and m, node/element axes
        R = R[[0, 1 + m if m else 1, 2 if m != 1 else 1, 3 if m != 2 else 1, 4]]
        ax_e, ax_n = {0: (3, 6), 1: (2, 5), 2: (1, 4)}[m]
        R = np.swapaxes(np.swapaxes(R, ax_e, 3), ax_n, 6)
        outs.append(R)
    assert np.max(np.abs(outs[1] - outs[0])) < 1e-12 * np.max(np.abs(outs[0]))
    assert np.max(np.abs(outs[2] - outs[0])) < 1e-12 * np.max(np.abs(outs[0]))


def test_vortex_rhs_consistency():
    """dq/dt of the vortex's closed form = -U_inf . grad q; the RHS converges to it."""
    errs = []
    for N in (8, 16):
        mesh = dg.Mesh(3, (N, N, 1), (-5, -5, -5), (5, 5, 5))
        x, y, _ = mesh.coords()
        U = inputs.vortex_state(x, y, 0.0)
        R = dg.rhs(mesh, U, dg.Physics(G, diss=1))
        dt = 1e-4
        exact = (inputs.vortex_state(x, y, dt) - inputs.vortex_state(x, y, -dt)) / (2 * dt)
        errs.append(np.sqrt(np.sum(mesh.element_sum((R[0] - exact[0]) ** 2))))
    rate = np.log2(errs[0] / errs[1])
    assert rate > 2.5, (errs, rate)


@pytest.mark.parametrize("mu,radius", [(0.0, 1), (0.02, 2)])
def test_element_block_matches_full_mesh(mu, radius):
    mesh = dg.Mesh(2, (6, 5, 7), (0, 0, 0), (1.0, 1.0, 1.0))
    U = smooth_state(mesh, seed=30, noise=0.05)
    phys = dg.Physics(G, mu=mu, diss=1)
    R = dg.rhs(mesh, U, phys)
    for centre in [(0, 0, 0), (5, 2, 3), (3, 4, 6)]:
        B = dg.element_block(U, centre, radius)
        nb = 2 * radius + 1
        bm = dg.Mesh(2, (nb, nb, nb), (0, 0, 0), tuple(nb * h for h in mesh.h))
        RB = dg.rhs(bm, B, phys)
        ex, ey, ez = centre
        got = RB[:, radius, radius, radius]
        ref = R[:, ez, ey, ex]
        assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_viscous_term_consistency():
    """Shear wave v_y = A sin(2 pi x), rho = p = 1: the BR1 term converges to the exact
    d/dx of the viscous flux, mu v_y'' (y momentum) and mu (v_y v_y')' (energy)."""
    mu, A = 0.05, 0.3
    phys = dg.Physics(G, mu=mu, Pr=0.72, diss=1)
    errs = []
    for N in (4, 8):
        mesh = dg.Mesh(3, (N, 1, 1), (0, 0, 0), (1.0, 1.0 / N, 1.0 / N))
        x, _, _ = mesh.coords()
        k = 2 * np.pi
        vy = A * np.sin(k * x)
        one = np.ones_like(x)
        U = gas.conserved(one, np.stack([0 * x, vy, 0 * x]), one, G)
        V = dg.viscous_term(mesh, U, phys)
        ex_my = -mu * k * k * A * np.sin(k * x)
        ex_E = mu * A * A * k * k * np.cos(2 * k * x)
        err = np.sqrt(np.sum(mesh.element_sum((V[2] - ex_my) ** 2 + (V[4] - ex_E) ** 2)))
        errs.append(err)
        assert np.max(np.abs(V[0])) < 1e-14
    assert errs[1] < errs[0] / 4, errs
    assert errs[1] < 1e-3 * mu * k * k * A


@pytest.mark.parametrize("p,n", MESHES)
def test_viscous_interface_dissipation(p, n):
    """diss^V: zero on a uniform state and (to rounding) on data continuous across the
    faces, conservative, and strictly entropy-dissipative on data that jumps."""
    mesh = dg.Mesh(p, n, (0, 0, 0), (1.0, 2.0, 1.5))
    phys = dg.Physics(G, mu=0.02, Pr=0.72, diss=1, visc_diss=1.0)
    U = np.empty(mesh.shape)
    U[:] = gas.conserved(np.array(1.3), np.array([0.4, -0.7, 0.2]), np.array(0.8), G).reshape(5, 1, 1, 1, 1, 1, 1)
    assert np.max(np.abs(dg.viscous_interface_dissipation(mesh, U, phys))) == 0.0
    Us = smooth_state(mesh, seed=40 + p)
    ref = np.max(np.abs(dg.viscous_term(mesh, Us, phys)))
    assert np.max(np.abs(dg.viscous_interface_dissipation(mesh, Us, phys))) < 1e-11 * ref
    U = smooth_state(mesh, seed=50 + p, noise=0.05)
    V = dg.viscous_interface_dissipation(mesh, U, phys)
    scale = np.sum(mesh.element_sum(np.abs(V)))
    assert max(abs(np.sum(mesh.element_sum(V[v]))) for v in range(5)) < 1e-13 * scale
    W = gas.entropy_variables(U, G)
    dS = np.sum(mesh.element_sum(np.sum(W * V, axis=0)))
    assert dS < -1e-3 * np.sum(mesh.element_sum(np.sum(np.abs(W * V), axis=0)))
    # and it enters rhs() only with a viscosity and a positive coefficient
    R1 = dg.rhs(mesh, U, phys)
    R0 = dg.rhs(mesh, U, dg.Physics(G, mu=0.02, Pr=0.72, diss=1))
    assert np.max(np.abs(R1 - R0 - V)) < 1e-12 * np.max(np.abs(R0))
