"""Section 4.1.1 on the GPU path: design-order convergence of the locally relaxed
scheme on the isentropic vortex (closed form, Eq. (vortex-solution)), compared at
the relaxed time t_gamma, at resolutions the CPU oracle cannot reach quickly.

Setup: entropy-stable (Rusanov) interfaces, a 2D vortex extruded over one element
in x3, periodic box [-5, 5]^2, t_end = 1, CFL 0.5 (the time step shrinks with h),
N = 16, 32, 64 elements per direction (h = 0.625 to 0.156; Table 1 spans h = 1 to
0.125).  The paper pairs p = 2 with BSRK(4,3) and p = 3 with RK(4,4) (Table 1) and
observes L2 density rates of 3.2 and 4.5; this setup (BS3, which advances as BSRK(4,3) with
fixed steps: its fourth stage feeds only the embedded pair) gives
2.6 and 4.0 with Rusanov interfaces and 2.9 for p = 2 with the matrix interface
dissipation (interface_diss = 2).
"""
import numpy as np
import pytest

from paper_2003_08831_gb300 import inputs

pytestmark = pytest.mark.gpu


def l2_density_error(p, N, rk, diss=1):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2003_08831_gb300.solver import Solver, stable_dt
    lo, hi = (-5.0, -5.0, 0.0), (5.0, 5.0, 10.0 / N)
    s = Solver(p, (N, N, 1), lo, hi, rk=rk, interface_diss=diss)
    xyz = s.coords()
    q0 = inputs.vortex_state(xyz[0], xyz[1], 0.0, period=10.0)
    h = 10.0 / N
    dt = stable_dt(q0, p, [h, h, h], 0.5)
    nsteps = int(np.ceil(1.0 / dt))
    q = s.to_device(q0)
    t, gh, _ = s.advance(q, nsteps, dt)
    assert s.status() == 0
    exact = inputs.vortex_state(xyz[0], xyz[1], t.item(), period=10.0)
    from oracle import sbp
    _, w, _ = sbp.sbp_operator(p)
    W = (w[:, None, None] * w[None, :, None] * w[None, None, :]).reshape(-1) * (h / 2) ** 3
    err = q.cpu().numpy()[0] - exact[0]
    l2 = np.sqrt(np.sum(W[None, :] * err * err) / (100.0 * h))
    s.close()
    return l2, gh.cpu().numpy()


@pytest.mark.parametrize("p,rk,diss", [(2, 0, 1), (3, 1, 1), (2, 0, 2)])
def test_vortex_design_order(p, rk, diss):
    """Least-squares rate over N = 16, 32, 64 above p + 1/2, the general a-priori rate of
    DG schemes for hyperbolic problems (the design order p + 1 is the paper's observation;
    a dropped or mis-signed term falls to first or second order)."""
    errs = []
    Ns = (16, 32, 64)
    for N in Ns:
        e, g = l2_density_error(p, N, rk, diss)
        assert np.all(np.abs(g - 1.0) < 0.05)
        errs.append(e)
    rate = np.polyfit(np.log2(10.0 / np.array(Ns)), np.log2(errs), 1)[0]
    print("p=%d diss=%d errors %s rate %.3f" % (p, diss, " ".join("%.3e" % e for e in errs), rate))
    assert rate > p + 0.5, (errs, rate)
    if diss == 2:
        # with the matrix dissipation the even degree comes within a quarter of design order
        # (2.86 measured; the coarsest mesh, 16 elements over the vortex, is still
        # under-resolved)
        assert rate > p + 0.75, (errs, rate)
