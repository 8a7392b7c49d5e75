"""Entropy histories on the GPU path (Section 2, Theorem 2.3; the eta(t) observable of Fig. 1).

* Entropy-conservative interfaces (diss = 0) make the semidiscretisation conserve the total
  entropy; relaxation with one global gamma then conserves it in the fully discrete scheme
  (Eq. (u-n-gamma): eta(u^n) = eta(u^{n-1}) + gamma (eta_new - eta_old), the estimate being
  exact), while the plain RK step drifts.
* With local relaxation every element satisfies eta_kappa(u^n) <= eta_kappa(u^{n-1}) +
  gamma Delta eta_kappa (Theorem 2.3), and the element estimates of an entropy-conservative
  semidiscretisation sum to zero: the total entropy does not increase.
* Entropy-stable interfaces (diss = 1) with local relaxation: the total entropy decreases.
"""
import numpy as np
import pytest

from test_gpu_parity import G, solver, vortex_setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def entropy_history(diss, relax, nsteps=30):
    import torch
    from oracle import dg, rk
    mesh, U, lo, hi = vortex_setup(N=4, p=3, nz=2)
    phys = dg.Physics(G, diss=diss)
    dt = rk.stable_dt(mesh, U, phys, 0.5)
    s = solver(mesh.p, mesh.n, lo, hi, interface_diss=diss, relax=relax)
    q = s.to_device(U)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    etas = [float(s.entropy(q).sum().item())]
    for _ in range(nsteps):
        s.advance(q, 1, dt, t)
        etas.append(float(s.entropy(q).sum().item()))
    assert s.status() == 0
    s.close()
    return np.array(etas)


def test_global_relaxation_conserves_entropy():
    from paper_2003_08831_gb300 import _binding as B
    eta = entropy_history(0, B.ES_RELAX_GLOBAL)
    scale = np.abs(eta[0])
    assert np.max(np.abs(eta - eta[0])) <= 1e-13 * scale
    base = entropy_history(0, B.ES_RELAX_NONE)
    assert np.max(np.abs(base - base[0])) > 100 * np.max(np.abs(eta - eta[0]))


def test_local_relaxation_entropy_does_not_increase():
    from paper_2003_08831_gb300 import _binding as B
    eta = entropy_history(0, B.ES_RELAX_LOCAL)
    assert np.all(np.diff(eta) <= 1e-13 * np.abs(eta[0]))


def test_entropy_stable_interfaces_dissipate():
    from paper_2003_08831_gb300 import _binding as B
    eta = entropy_history(1, B.ES_RELAX_LOCAL)
    assert np.all(np.diff(eta) <= 1e-13 * np.abs(eta[0]))
    assert eta[-1] < eta[0]
