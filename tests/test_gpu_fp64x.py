"""Float-float precision mode (ES_FP64X) against the FP64 oracle.

The flux, SAT and viscous kernels compute in float-float arithmetic on the FP32
pipe (hi + lo pairs of floats); state, entropy sums and the relaxation solve
stay in FP64.  The bars are the FP64 ones of test_gpu_parity with the
arithmetic's rounding unit in place of FP64's: eps_ff = 2^-47 (twice the
2^-48 unit of a float-float value, as eps = 2^-52 is twice FP64's unit):
* right-hand side: 1e-12 max |oracle| per variable, or 256 eps_ff times the
  magnitude of the summed terms where the SBP sums cancel;
* state after the stated steps: 1e-12 max |oracle| per variable;
* gamma, gamma_kappa: 1e-12 relative or 8x their response to right-hand-side
  changes of 2 eps_ff times the term magnitude.
"""
import numpy as np
import pytest

from oracle import dg, gas, rk
from test_gpu_parity import (G, RHS_CASES, SAMPLES, TOL, assert_rhs_close, compare_advance, gamma_sensitivity,
                             random_state, solver, tgv_full, vortex_setup)

pytestmark = pytest.mark.gpu
EPS_FF = 2.0 ** -47


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _fp64x():
    from paper_2003_08831_gb300 import _binding as B
    return B.ES_FP64X


@pytest.mark.parametrize("p,n,mu,diss", RHS_CASES)
def test_fp64x_rhs_and_entropy_rate(p, n, mu, diss):
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.5, 2.0)
    mesh = dg.Mesh(p, n, lo, hi)
    U = random_state(mesh, seed=p * 10 + n[0])
    phys = dg.Physics(G, mu=mu, Pr=0.72, diss=diss)
    ref = dg.rhs(mesh, U, phys)
    Eref = dg.entropy_rate(mesh, U, ref, phys).reshape(-1)
    s = solver(p, n, lo, hi, mu=mu, interface_diss=diss, precision=_fp64x())
    dq, E = s.rhs(s.to_device(U), want_E=True)
    assert s.status() == 0
    assert_rhs_close(dq.cpu().numpy(), ref, dg.rhs_term_magnitude(mesh, U, phys), eps=EPS_FF)
    W = gas.entropy_variables(U, G)
    Escale = mesh.element_sum(np.sum(np.abs(W * ref), axis=0)).reshape(-1)
    assert np.max(np.abs(E.cpu().numpy() - Eref) / Escale) < TOL
    s.close()


def test_fp64x_advance_vortex_4cubed_p3():
    """4^3 elements, p = 3, [0,10]^3, BS3, CFL 0.5, 20 locally relaxed steps."""
    mesh, U, lo, hi = vortex_setup()
    g = compare_advance(mesh, U, lo, hi, dg.Physics(G, diss=1), "BS3", 20, eps=EPS_FF, precision=_fp64x())
    assert np.all(np.abs(g - 1) < 0.1)


def test_fp64x_root_rtol_below_float_float_resolution():
    """A root_rtol far below the float-float resolution (the oracle's 4 * 2^-52) is
    clamped to 2^-40 in the float-float solve: it ends and meets the FP64X bars."""
    mesh, U, lo, hi = vortex_setup()
    compare_advance(mesh, U, lo, hi, dg.Physics(G, diss=1), "BS3", 6, eps=EPS_FF, precision=_fp64x(),
                    root_rtol=4 * 2.0 ** -52)


def test_fp64x_advance_rk4_ec_ragged():
    mesh, U, lo, hi = vortex_setup(N=5, p=2, nz=3)
    compare_advance(mesh, U, lo, hi, dg.Physics(G, diss=0), "RK4", 6, eps=EPS_FF, precision=_fp64x())


def test_fp64x_advance_rk65():
    """Six stages: the float-float stage preparation with a run-time count of earlier stages."""
    mesh, U, lo, hi = vortex_setup(N=4, p=3, nz=1)
    compare_advance(mesh, U, lo, hi, dg.Physics(G, diss=1), "RK65", 6, eps=EPS_FF, precision=_fp64x())


def test_fp64x_advance_navier_stokes():
    mesh, U, lo, hi = vortex_setup(N=3, p=4, nz=2)
    compare_advance(mesh, U, lo, hi, dg.Physics(G, mu=0.005, Pr=0.72, diss=1), "BS3", 5, eps=EPS_FF,
                    precision=_fp64x())


@pytest.mark.parametrize("p,mu", [(3, 0.0), (4, 1.0 / 1600.0)])
def test_fp64x_full_size_rhs_sampled(p, mu):
    """32^3 TGV at Mach 0.1 (strong cancellation of the pressure terms) in float-float."""
    mesh, U, lo, hi = tgv_full(p)
    phys = dg.Physics(G, mu=mu, Pr=0.72, diss=1)
    s = solver(p, mesh.n, lo, hi, mu=mu, precision=_fp64x())
    dq = s.rhs(s.to_device(U)).cpu().numpy().reshape(mesh.shape)
    assert s.status() == 0
    s.close()
    radius = 2 if mu > 0 else 1
    nb = 2 * radius + 1
    bm = dg.Mesh(p, (nb, nb, nb), (0, 0, 0), tuple(nb * h for h in mesh.h))
    for c in SAMPLES:
        B = dg.element_block(U, c, radius)
        ref = dg.rhs(bm, B, phys)[:, radius, radius, radius]
        terms = dg.rhs_term_magnitude(bm, B, phys)[:, radius, radius, radius]
        assert_rhs_close(dq[:, c[2], c[1], c[0]], ref, terms, eps=EPS_FF)


def test_fp64x_full_size_step_sampled():
    """One relaxed BS3 step of the 32^3 p = 3 Euler TGV: gamma_kappa of sampled elements."""
    p = 3
    mesh, U, lo, hi = tgv_full(p)
    phys = dg.Physics(G, diss=1)
    dt = rk.stable_dt(mesh, U, phys, 0.5)
    s = solver(p, mesh.n, lo, hi, precision=_fp64x())
    q = s.to_device(U)
    t, gh, gk = s.advance(q, 1, dt)
    assert s.status() == 0
    gk = gk.cpu().numpy().reshape(mesh.n[2], mesh.n[1], mesh.n[0])
    gamma = gh.cpu().numpy()[0]
    s.close()
    assert gamma == np.min(gk)
    radius = 3
    nb = 2 * radius + 1
    bm = dg.Mesh(p, (nb, nb, nb), (0, 0, 0), tuple(nb * h for h in mesh.h))
    for c in SAMPLES[:3]:
        B = dg.element_block(U, c, radius)
        r = rk.rk_step(bm, B, dt, phys, rk.BS3)
        g_ref = r.gamma_kappa[radius, radius, radius]
        _, sens = gamma_sensitivity(bm, B, dt, 1, phys, rk.BS3, "local", [r], seeds=2, eps=EPS_FF)
        tol = max(TOL, 8 * sens.reshape(nb, nb, nb)[radius, radius, radius])
        g_got = gk[c[2], c[1], c[0]]
        assert abs(g_got - g_ref) <= tol * g_ref, (c, g_got, g_ref, tol)
