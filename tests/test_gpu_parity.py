"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bars (FP64), on the same seeded inputs:
* state after the stated steps: max |gpu - oracle| <= 1e-12 max |oracle| per
  conserved variable;
* right-hand side: |gpu - oracle| <= 1e-12 max |oracle| per variable, or, where
  the SBP sums cancel (low Mach number), 256 eps times the magnitude of the
  summed terms (oracle.dg.rhs_term_magnitude), the rounding bound of any FP64
  evaluation;
* gamma and gamma_kappa: 1e-12 relative, or 8x their response to rounding-level
  changes of the right-hand side where that is larger (gamma_kappa is the root
  of a second-order quantity).
Meshes span several CTA tiles with a ragged last tile (element counts that are
not multiples of the elements-per-CTA of any degree).
"""
import numpy as np
import pytest

from oracle import dg, gas, relax, rk
from oracle_jobs import gamma_sensitivity  # noqa: F401  (also imported from here by other test modules)
from paper_2003_08831_gb300 import inputs

pytestmark = pytest.mark.gpu
G = 1.4
TOL = 1e-12
EPS = 2.0 ** -52


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def solver(p, n, lo, hi, **kw):
    from paper_2003_08831_gb300.solver import Solver
    return Solver(p, n, lo, hi, **kw)


def random_state(mesh, seed, amp=0.2, noise=0.02):
    """Seeded smooth periodic state plus nodal noise (jumps across interfaces)."""
    rng = np.random.default_rng(seed)
    x, y, z = mesh.coords()
    L = mesh.hi - mesh.lo

    def field(base, a):
        f = np.full(x.shape, base)
        for _ in range(3):
            k = rng.integers(0, 3, size=3)
            f = f + a * rng.uniform(-1, 1) * np.cos(
                2 * np.pi * (k[0] * x / L[0] + k[1] * y / L[1] + k[2] * z / L[2]) + rng.uniform(0, 6.3))
        return f * (1 + noise * rng.uniform(-1, 1, x.shape))
    return inputs.conserved(field(1.0, amp), field(0.3, amp), field(-0.2, amp), field(0.1, amp), field(1.0, amp), G)


def assert_rhs_close(got, ref, terms, eps=EPS):
    got = np.asarray(got).reshape(5, -1)
    ref = np.asarray(ref).reshape(5, -1)
    terms = np.asarray(terms).reshape(5, -1)
    scale = np.maximum(np.max(np.abs(ref), axis=1), 1e-3 * np.max(np.abs(ref)))[:, None]
    bound = np.maximum(TOL * scale, 256 * eps * terms)
    bad = np.abs(got - ref) > bound
    assert not bad.any(), (np.argwhere(bad)[:5], np.max(np.abs(got - ref) / bound))


def rel_err_per_var(a, b):
    a = np.asarray(a).reshape(5, -1)
    b = np.asarray(b).reshape(5, -1)
    scale = np.maximum(np.max(np.abs(b), axis=1), 1e-3 * np.max(np.abs(b)))
    return np.max(np.abs(a - b), axis=1) / scale


RHS_CASES = [
    (2, (3, 5, 7), 0.0, 0),
    (3, (3, 5, 7), 0.0, 1),
    (4, (4, 3, 5), 0.0, 1),
    (5, (2, 3, 3), 0.0, 1),
    (2, (5, 3, 2), 0.05, 1),
    (3, (3, 5, 7), 0.02, 1),
    (4, (3, 2, 4), 0.01, 1),
    (5, (2, 2, 3), 0.02, 0),
]


@pytest.mark.parametrize("p,n,mu,diss", RHS_CASES)
def test_rhs_and_entropy_rate(p, n, mu, diss):
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.5, 2.0)
    mesh = dg.Mesh(p, n, lo, hi)
    U = random_state(mesh, seed=p * 10 + n[0])
    phys = dg.Physics(G, mu=mu, Pr=0.72, diss=diss)
    ref = dg.rhs(mesh, U, phys)
    Eref = dg.entropy_rate(mesh, U, ref, phys).reshape(-1)
    s = solver(p, n, lo, hi, mu=mu, interface_diss=diss)
    q = s.to_device(U)
    dq, E = s.rhs(q, want_E=True)
    assert s.status() == 0
    assert_rhs_close(dq.cpu().numpy(), ref, dg.rhs_term_magnitude(mesh, U, phys))
    W = gas.entropy_variables(U, G)
    Escale = mesh.element_sum(np.sum(np.abs(W * ref), axis=0)).reshape(-1)
    assert np.max(np.abs(E.cpu().numpy() - Eref) / Escale) < TOL
    s.close()


@pytest.mark.parametrize("p,n", [(3, (3, 5, 7)), (5, (2, 3, 2))])
def test_local_entropies(p, n):
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    mesh = dg.Mesh(p, n, lo, hi)
    U = random_state(mesh, seed=3)
    ref = dg.local_entropies(mesh, U, dg.Physics(G)).reshape(-1)
    s = solver(p, n, lo, hi)
    eta = s.entropy(s.to_device(U)).cpu().numpy()
    assert np.max(np.abs(eta - ref) / np.abs(ref)) < 1e-13
    s.close()


def vortex_setup(N=4, p=3, nz=None):
    nz = N if nz is None else nz
    lo, hi = (0.0, 0.0, 0.0), (10.0, 10.0, 10.0 * nz / N)
    mesh = dg.Mesh(p, (N, N, nz), lo, hi)
    x, y, _ = mesh.coords()
    U = inputs.vortex_state(x, y, 0.0, centre=(5.0, 5.0))
    return mesh, U, lo, hi


def compare_advance(mesh, U, lo, hi, phys, tabname, nsteps, mode="local", cfl=0.5, eps=EPS, **kw):
    """FP64 parity of es_advance: state at 1e-12 per variable; gamma and gamma_kappa at
    1e-12 or, where larger, 8x their measured sensitivity to last-bit RHS changes."""
    from paper_2003_08831_gb300 import _binding as B
    dt = rk.stable_dt(mesh, U, phys, cfl)
    Uo, to, hist = rk.advance(mesh, U, dt, nsteps, phys, rk.TABLEAUX[tabname], mode=mode)
    sens_g, sens_gk = gamma_sensitivity(mesh, U, dt, nsteps, phys, rk.TABLEAUX[tabname], mode, hist, eps=eps)
    relax_mode = {"local": B.ES_RELAX_LOCAL, "global": B.ES_RELAX_GLOBAL, "none": B.ES_RELAX_NONE}[mode]
    s = solver(mesh.p, mesh.n, lo, hi, mu=phys.mu, Pr=phys.Pr, interface_diss=phys.diss,
               rk={"BS3": B.ES_RK_BS3, "RK4": B.ES_RK_RK4, "RK65": B.ES_RK_RK65}[tabname], relax=relax_mode,
               visc_diss=phys.visc_diss, **kw)
    q = s.to_device(U)
    t, gh, gk = s.advance(q, nsteps, dt)
    assert s.status() == 0
    err = rel_err_per_var(q.cpu().numpy(), Uo)
    assert np.all(err < TOL), err
    gref = np.array([h.gamma for h in hist])
    gh = gh.cpu().numpy()
    tol_g = np.maximum(TOL, 8 * sens_g)
    assert np.all(np.abs(gh - gref) / gref <= tol_g), (gh, gref, tol_g)
    # t = t0 + sum_n gamma_n dt (Eq. (t-n-gamma)): its bound is the sum of the gamma bounds
    assert abs(t.item() - to) <= max(TOL * to, dt * np.sum(tol_g * gref))
    gko = hist[-1].gamma_kappa.reshape(-1)
    gkg = gk.cpu().numpy()
    fin = np.isfinite(gko)
    assert np.array_equal(fin, np.isfinite(gkg))
    tol_gk = np.maximum(TOL, 8 * sens_gk)
    assert np.all(np.abs(gkg[fin] - gko[fin]) / gko[fin] <= tol_gk[fin])
    s.close()
    return gref


def test_advance_vortex_4cubed_p3():
    """4^3 elements, p = 3, [0,10]^3, BS3, CFL 0.5, 20 steps, local relaxation (FP64)."""
    mesh, U, lo, hi = vortex_setup()
    g = compare_advance(mesh, U, lo, hi, dg.Physics(G, diss=1), "BS3", 20)
    assert np.all(np.abs(g - 1) < 0.1)


def test_advance_root_rtol_at_oracle_tolerance():
    """es_config.root_rtol = 4 * 2^-52, the oracle's own stop: the CUDA solve then stops
    on the same rule as the oracle's and meets the same bars (FP64); the float-float
    solve clamps the request to 2^-40 and meets its bars too (test_gpu_fp64x)."""
    mesh, U, lo, hi = vortex_setup()
    g = compare_advance(mesh, U, lo, hi, dg.Physics(G, diss=1), "BS3", 8, root_rtol=4 * EPS)
    assert np.all(np.abs(g - 1) < 0.1)


def test_advance_rk4_ec_ragged():
    mesh, U, lo, hi = vortex_setup(N=5, p=2, nz=3)
    compare_advance(mesh, U, lo, hi, dg.Physics(G, diss=0), "RK4", 6)


def test_advance_navier_stokes():
    mesh, U, lo, hi = vortex_setup(N=3, p=4, nz=2)
    compare_advance(mesh, U, lo, hi, dg.Physics(G, mu=0.005, Pr=0.72, diss=1), "BS3", 5)


def test_advance_global_relaxation():
    """Global relaxation (one gamma for eta = sum eta_kappa), the paper's comparison mode."""
    mesh, U, lo, hi = vortex_setup(N=4, p=3, nz=2)
    g = compare_advance(mesh, U, lo, hi, dg.Physics(G, diss=1), "BS3", 6, mode="global")
    assert np.all(np.abs(g - 1) < 0.05)


def test_advance_baseline_no_relaxation():
    mesh, U, lo, hi = vortex_setup(N=3, p=3, nz=2)
    g = compare_advance(mesh, U, lo, hi, dg.Physics(G, diss=1), "BS3", 4, mode="none")
    assert np.all(g == 1.0)


def test_relax_step_interface():
    """es_relax_step(u_old, u_new, d_eta) against the oracle's root of the same equation."""
    mesh, U, lo, hi = vortex_setup(N=4, p=3, nz=2)
    phys = dg.Physics(G, diss=1)
    dt = rk.stable_dt(mesh, U, phys, 0.5)
    res = rk.rk_step(mesh, U, dt, phys, rk.BS3, mode="none")
    u_new = U + res.d
    deta = res.deta.reshape(-1)
    uf, df = mesh.flat(U), mesh.flat(u_new) - mesh.flat(U)
    P = np.broadcast_to(mesh.mass().reshape(1, -1), (mesh.K, mesh.Np))
    A = np.sum(P * np.sum(gas.entropy_variables(uf, G) * df, axis=0), axis=-1) - deta
    gko, flags = relax.solve_gamma(uf, df, A, P, G)
    s = solver(mesh.p, mesh.n, lo, hi)
    import torch
    gk, g, out = s.relax_step(s.to_device(U), s.to_device(u_new), torch.from_numpy(deta.copy()).cuda())
    assert s.status() == 0
    gk = gk.cpu().numpy()
    fin = np.isfinite(gko)
    assert np.array_equal(fin, np.isfinite(gk))
    # gamma_kappa here is conditioned by sum P w.d - d_eta (a difference of O(dt) sums):
    # the bound is the rounding of those sums relative to the root's curvature term
    a = 0.5 * np.sum(P * relax.hessian_form(uf, df, G), axis=-1)
    X = np.sum(P * np.sum(np.abs(gas.entropy_variables(uf, G) * df), axis=0), axis=-1)
    tol = TOL + 64 * 2.2e-16 * X / a
    assert np.all(np.abs(gk[fin] - gko[fin]) / gko[fin] <= tol[fin])
    gmin = relax.global_gamma(gko)
    assert abs(g.item() - gmin) <= tol[np.argmin(gko)] * gmin
    ref_out = uf + g.item() * df
    assert np.all(rel_err_per_var(out.cpu().numpy(), ref_out) < TOL)
    s.close()


def test_nonphysical_state_flag():
    mesh, U, lo, hi = vortex_setup(N=2, p=2, nz=1)
    U = U.copy()
    U[0].reshape(-1)[5] = -1.0
    s = solver(mesh.p, mesh.n, lo, hi)
    s.rhs(s.to_device(U))
    from paper_2003_08831_gb300 import _binding as B
    assert s.status() == B.ES_ERR_NONPHYSICAL
    assert s.status() == 0  # sticky bits are cleared once read
    s.close()


def test_no_root_flag():
    """An estimate Delta eta far below the linearised change leaves r'(0) > 0."""
    mesh, U, lo, hi = vortex_setup(N=2, p=3, nz=1)
    phys = dg.Physics(G, diss=1)
    dt = rk.stable_dt(mesh, U, phys, 0.5)
    res = rk.rk_step(mesh, U, dt, phys, rk.BS3, mode="none")
    import torch
    s = solver(mesh.p, mesh.n, lo, hi)
    deta = torch.full((mesh.K,), -1e3, dtype=torch.float64, device="cuda")
    gk, g, out = s.relax_step(s.to_device(U), s.to_device(U + res.d), deta)
    from paper_2003_08831_gb300 import _binding as B
    assert s.status() == B.ES_ERR_NO_ROOT
    assert np.all(np.isinf(gk.cpu().numpy()))
    assert g.item() == 1.0
    s.close()


# ---------------------------------------------------------------------------------------
# full-size workloads: sampled elements against oracle element blocks

def tgv_full(p, N=32, noise=False):
    lo, hi = (0.0, 0.0, 0.0), (2 * np.pi,) * 3
    mesh = dg.Mesh(p, (N, N, N), lo, hi)
    x, y, z = mesh.coords()
    if noise:
        U = inputs.perturbed_tgv_state(x.reshape(-1), y.reshape(-1), z.reshape(-1)).reshape(mesh.shape)
    else:
        U = inputs.tgv_state(x, y, z)
    return mesh, U, lo, hi


SAMPLES = [(0, 0, 0), (31, 31, 31), (5, 17, 30), (16, 0, 9), (23, 11, 4)]


@pytest.mark.parametrize("p,mu", [(3, 0.0), (4, 1.0 / 1600.0)])
def test_full_size_rhs_sampled(p, mu):
    """32^3 TGV (p = 3 Euler, p = 4 Navier--Stokes Re 1600): es_rhs at full size vs the
    oracle's RHS of the centre element of a periodic block around sampled elements."""
    mesh, U, lo, hi = tgv_full(p)
    phys = dg.Physics(G, mu=mu, Pr=0.72, diss=1)
    s = solver(p, mesh.n, lo, hi, mu=mu)
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
        got = dq[:, c[2], c[1], c[0]]
        assert_rhs_close(got, ref, terms)


def test_full_size_step_sampled():
    """One relaxed BS3 step of the 32^3 p = 3 Euler TGV: gamma_kappa of sampled elements vs
    the oracle on radius-3 blocks (three stages each widen the stencil by one element), and
    q_new - q_old = gamma d there."""
    p = 3
    mesh, U, lo, hi = tgv_full(p)
    phys = dg.Physics(G, diss=1)
    dt = rk.stable_dt(mesh, U, phys, 0.5)
    s = solver(p, mesh.n, lo, hi)
    q = s.to_device(U)
    t, gh, gk = s.advance(q, 1, dt)
    assert s.status() == 0
    qn = q.cpu().numpy().reshape(mesh.shape)
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
        _, sens = gamma_sensitivity(bm, B, dt, 1, phys, rk.BS3, "local", [r], seeds=2)
        tol = max(TOL, 8 * sens.reshape(nb, nb, nb)[radius, radius, radius])
        g_got = gk[c[2], c[1], c[0]]
        assert abs(g_got - g_ref) <= tol * g_ref, (c, g_got, g_ref, tol)
        # the state moved by gamma d (the GPU's own gamma): compare with the oracle's d at
        # the rounding level of the stage sums (dt times the RHS bound) plus the rounding
        # of q_new - q_old divided by gamma
        d_ref = r.d[:, radius, radius, radius]
        d_got = (qn[:, c[2], c[1], c[0]] - U[:, c[2], c[1], c[0]]) / gamma
        terms = dg.rhs_term_magnitude(bm, B, phys)[:, radius, radius, radius]
        bound = dt * 256 * EPS * terms + 4 * EPS * np.abs(U[:, c[2], c[1], c[0]]) / gamma
        assert np.all(np.abs(d_got - d_ref) <= bound), np.max(np.abs(d_got - d_ref) / bound)


# ---------------------------------------------------------------------------------------
# mixed precision: FP32 fluxes, SATs and viscous terms; FP64 state, entropy sums and gamma

def rel_l2(a, b):
    a = np.asarray(a).reshape(5, -1)
    b = np.asarray(b).reshape(5, -1)
    nb = np.sqrt(np.sum(b * b, axis=1))
    nb = np.maximum(nb, 1e-3 * nb.max())
    return np.sqrt(np.sum((a - b) ** 2, axis=1)) / nb


@pytest.mark.parametrize("p,n,mu", [(3, (3, 5, 4), 0.0), (4, (3, 3, 4), 0.02)])
def test_mixed_rhs_error(p, n, mu):
    """The FP32 right-hand side against the FP64 oracle: relative L2 error per variable
    bounded by 64 eps_32 times the flux-to-result cancellation of the SBP sums."""
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.5, 2.0)
    mesh = dg.Mesh(p, n, lo, hi)
    U = random_state(mesh, seed=7 + p, noise=0.0)
    phys = dg.Physics(G, mu=mu, Pr=0.72, diss=1)
    ref = dg.rhs(mesh, U, phys)
    # cancellation: size of the individual terms sum_j |2 D_ij f*_ij| against the result
    terms = np.zeros_like(U)
    for m in range(3):
        A = np.moveaxis(U, {0: 6, 1: 5, 2: 4}[m], -1)
        F = gas.ec_flux(A[..., :, None], A[..., None, :], G, m)
        terms += (2.0 / mesh.h[m]) * np.moveaxis(np.einsum("ij,...ij->...i", np.abs(2 * mesh.D), np.abs(F)),
                                                 -1, {0: 6, 1: 5, 2: 4}[m])
    kappa = np.sqrt(np.sum(terms.reshape(5, -1) ** 2, axis=1)) / np.maximum(
        np.sqrt(np.sum(ref.reshape(5, -1) ** 2, axis=1)), 1e-300)
    from paper_2003_08831_gb300 import _binding as B
    s = solver(p, n, lo, hi, mu=mu, precision=B.ES_MIXED)
    dq = s.rhs(s.to_device(U)).cpu().numpy()
    assert s.status() == 0
    s.close()
    err = rel_l2(dq, ref)
    bound = 64 * 6e-8 * kappa
    assert np.all(err <= np.maximum(bound, 1e-6)), (err, bound)


@pytest.mark.parametrize("prec", [1, 3])
@pytest.mark.parametrize("case", ["vortex", "tgv_noise_ns", "vortex_rk65"])
def test_mixed_advance_error(case, prec):
    """Mixed-precision relaxed steps against the FP64 oracle, with FP64 (ES_MIXED) and
    float-float (ES_MIXED_FF) estimates: state relative L2 <= 1e-5."""
    from paper_2003_08831_gb300 import _binding as B
    tab, rkc = rk.BS3, B.ES_RK_BS3
    if case == "vortex":
        mesh, U, lo, hi = vortex_setup()
        phys = dg.Physics(G, diss=1)
        nsteps = 20
    elif case == "vortex_rk65":
        mesh, U, lo, hi = vortex_setup()
        phys = dg.Physics(G, diss=1)
        nsteps = 8
        tab, rkc = rk.RK65, B.ES_RK_RK65
    else:
        lo, hi = (0.0, 0.0, 0.0), (2 * np.pi,) * 3
        mesh = dg.Mesh(4, (4, 4, 4), lo, hi)
        x, y, z = mesh.coords()
        U = inputs.perturbed_tgv_state(x.reshape(-1), y.reshape(-1), z.reshape(-1)).reshape(mesh.shape)
        phys = dg.Physics(G, mu=1.0 / 1600.0, Pr=0.72, diss=1)
        nsteps = 10
    dt = rk.stable_dt(mesh, U, phys, 0.5)
    Uo, to, hist = rk.advance(mesh, U, dt, nsteps, phys, tab)
    s = solver(mesh.p, mesh.n, lo, hi, mu=phys.mu, precision=prec, rk=rkc)
    q = s.to_device(U)
    t, gh, gk = s.advance(q, nsteps, dt)
    assert s.status() == 0
    err = rel_l2(q.cpu().numpy(), Uo)
    assert np.all(err < 1e-5), err
    s.close()


# ---------------------------------------------------------------------------------------
# Section 4.4 (Eq. visu_of_local_gamma): the 1D smooth + discontinuous case as a
# 200 x 1 x 1 periodic mesh, RK(4,4), dt = 1e-4.

def x6_state(mesh):
    x, _, _ = mesh.coords()
    left = x < 0
    rho = np.where(left, 1 + 0.5 * np.cos(2 * np.pi * x), 0.5 + 0.25 * np.cos(2 * np.pi * x))
    u = np.full_like(x, 0.5)
    pr = np.where(left, 1.0, 0.8)
    return inputs.conserved(rho, u, 0 * u, 0 * u, pr, G)


def test_local_gamma_variation_x6():
    """Parity with the oracle over the first 20 steps, then the paper's printed bound
    |gamma_kappa - 1| < 2e-5 at t = 0.1 (tests/golden/local_gamma_variation.txt)."""
    import os
    from paper_2003_08831_gb300 import _binding as B
    gold = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "local_gamma_variation.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                gold[k.strip()] = float(v)
    K = int(gold["elements"])
    lo, hi = (-2.0, 0.0, 0.0), (2.0, 4.0 / K, 4.0 / K)
    mesh = dg.Mesh(int(gold["p"]), (K, 1, 1), lo, hi)
    U = x6_state(mesh)
    phys = dg.Physics(G, diss=1)
    dt = gold["dt"]
    Uo, to, hist = rk.advance(mesh, U, dt, 20, phys, rk.RK4)
    s = solver(mesh.p, mesh.n, lo, hi, rk=B.ES_RK_RK4)
    q = s.to_device(U)
    t, gh, gk = s.advance(q, 20, dt)
    assert s.status() == 0
    err = rel_err_per_var(q.cpu().numpy(), Uo)
    assert np.all(err < TOL), err
    steps = int(round(gold["t_final"] / dt))
    t, gh, gk = s.advance(q, steps - 20, dt, t)
    assert s.status() == 0
    g = gk.cpu().numpy()
    g = g[np.isfinite(g)]
    assert g.size > 0
    assert np.max(np.abs(g - 1.0)) < gold["bound"], np.max(np.abs(g - 1.0))
    s.close()


def test_reciprocal_matches_ieee_division():
    """The kernels' FP64 reciprocal (hardware approximation + one third-order step) against
    IEEE 1/x over random mantissas and exponents 2^-300 .. 2^300: within one ulp."""
    import torch
    from paper_2003_08831_gb300 import _binding as B
    rng = np.random.default_rng(7)
    x = np.ldexp(rng.uniform(1.0, 2.0, 1 << 20), rng.integers(-300, 300, 1 << 20))
    x[::2] *= -1.0
    xd = torch.from_numpy(x).cuda()
    out = torch.empty_like(xd)
    B.es_reciprocal(xd, out)
    torch.cuda.synchronize()
    ref = 1.0 / x
    ulp = np.abs(out.cpu().numpy().view(np.int64) - ref.view(np.int64))
    assert ulp.max() <= 1, ulp.max()


# ---------------------------------------------------------------------------------------
# matrix interface dissipation in entropy variables (interface_diss = 2)

@pytest.mark.parametrize("p,n,mu,prec", [(2, (3, 5, 4), 0.0, 0), (3, (3, 4, 5), 0.02, 0), (4, (2, 3, 3), 0.0, 0),
                                        (5, (2, 2, 3), 0.01, 0), (3, (3, 4, 5), 0.02, 2)])
def test_rhs_matrix_dissipation(p, n, mu, prec):
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.5, 2.0)
    mesh = dg.Mesh(p, n, lo, hi)
    U = random_state(mesh, seed=p * 7 + n[0])
    phys = dg.Physics(G, mu=mu, Pr=0.72, diss=2)
    ref = dg.rhs(mesh, U, phys)
    s = solver(p, n, lo, hi, mu=mu, interface_diss=2, precision=prec)
    dq = s.rhs(s.to_device(U)).cpu().numpy()
    assert s.status() == 0
    assert_rhs_close(dq, ref, dg.rhs_term_magnitude(mesh, U, phys), eps=EPS if prec == 0 else 2.0 ** -47)
    s.close()


def test_advance_matrix_dissipation():
    mesh, U, lo, hi = vortex_setup(N=4, p=3, nz=2)
    compare_advance(mesh, U, lo, hi, dg.Physics(G, diss=2), "BS3", 10)


# ---------------------------------------------------------------------------------------
# diss^V: interior penalty on the entropy-variable jump (visc_diss = alpha)

@pytest.mark.parametrize("p,n,mu,alpha,diss,prec", [(2, (3, 5, 4), 0.02, 1.0, 1, 0), (3, (4, 3, 5), 0.01, 0.5, 2, 0),
                                                    (4, (2, 3, 3), 0.05, 1.0, 1, 0), (5, (2, 2, 3), 0.02, 2.0, 0, 0),
                                                    (3, (4, 3, 5), 0.01, 1.0, 1, 2)])
def test_rhs_viscous_interface_dissipation(p, n, mu, alpha, diss, prec):
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.5, 2.0)
    mesh = dg.Mesh(p, n, lo, hi)
    U = random_state(mesh, seed=p * 11 + n[1])
    phys = dg.Physics(G, mu=mu, Pr=0.72, diss=diss, visc_diss=alpha)
    ref = dg.rhs(mesh, U, phys)
    s = solver(p, n, lo, hi, mu=mu, interface_diss=diss, precision=prec, visc_diss=alpha)
    dq = s.rhs(s.to_device(U)).cpu().numpy()
    assert s.status() == 0
    s.close()
    assert_rhs_close(dq, ref, dg.rhs_term_magnitude(mesh, U, phys), eps=EPS if prec == 0 else 2.0 ** -47)
    # the penalty is really there: without it the right-hand side differs by far more than the bar
    ref0 = dg.rhs(mesh, U, dg.Physics(G, mu=mu, Pr=0.72, diss=diss))
    assert np.max(rel_err_per_var(ref0, ref)) > 1e-6


def test_advance_viscous_interface_dissipation():
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    mesh = dg.Mesh(3, (3, 3, 3), lo, hi)
    U = random_state(mesh, seed=77, noise=0.01)
    compare_advance(mesh, U, lo, hi, dg.Physics(G, mu=0.01, Pr=0.72, diss=1, visc_diss=1.0), "BS3", 5)


# ---------------------------------------------------------------------------------------
# fifth-order tableau (RK(6,5), b >= 0) and caller-supplied tableaux (es_set_tableau)

@pytest.mark.parametrize("mode", ["local", "global"])
def test_advance_rk65(mode):
    mesh, U, lo, hi = vortex_setup(N=4, p=4, nz=1)
    g = compare_advance(mesh, U, lo, hi, dg.Physics(G, diss=1), "RK65", 8, mode=mode)
    assert np.all(np.abs(g - 1) < 0.1)


def test_advance_rk65_navier_stokes():
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    mesh = dg.Mesh(3, (3, 3, 3), lo, hi)
    U = random_state(mesh, seed=91, noise=0.01)
    compare_advance(mesh, U, lo, hi, dg.Physics(G, mu=0.01, Pr=0.72, diss=1), "RK65", 4)


def _run(p, n, lo, hi, U, dt, nsteps, rkc, tab=None):
    s = solver(p, n, lo, hi, rk=rkc)
    if tab is not None:
        s.set_tableau(tab["A"], tab["b"], tab["c"])
    q = s.to_device(U)
    t, gh, gk = s.advance(q, nsteps, dt)
    assert s.status() == 0
    out = (q.cpu().numpy(), t.item(), gh.cpu().numpy(), gk.cpu().numpy())
    s.close()
    return out


def test_set_tableau_reproduces_builtin_and_oracle():
    """A tableau loaded through es_set_tableau runs the same kernels as the built-in one
    (bit-identical states, gamma and t); a 7-stage tableau with a trailing zero weight
    (RK65 with an unused last stage) is identical too; a 3-stage method loaded into a
    context created with RK(4,4) matches the oracle."""
    from paper_2003_08831_gb300 import _binding as B
    mesh, U, lo, hi = vortex_setup(N=4, p=3, nz=1)
    phys = dg.Physics(G, diss=1)
    dt = rk.stable_dt(mesh, U, phys, 0.5)
    ref = _run(3, mesh.n, lo, hi, U, dt, 5, B.ES_RK_RK65)
    got = _run(3, mesh.n, lo, hi, U, dt, 5, B.ES_RK_BS3, rk.RK65)
    for a, b in zip(ref, got):
        assert np.array_equal(np.asarray(a), np.asarray(b))
    t7 = {"A": np.zeros((7, 7)), "b": np.zeros(7), "c": np.zeros(7)}
    t7["A"][:6, :6] = rk.RK65["A"]
    t7["A"][6, :6] = rk.RK65["b"]
    t7["b"][:6] = rk.RK65["b"]
    t7["c"][:6] = rk.RK65["c"]
    t7["c"][6] = 1.0
    got7 = _run(3, mesh.n, lo, hi, U, dt, 5, B.ES_RK_RK4, t7)
    for a, b in zip(ref, got7):
        assert np.array_equal(np.asarray(a), np.asarray(b))
    Uo, to, hist = rk.advance(mesh, U, dt, 5, phys, rk.BS3)
    q, t, gh, _ = _run(3, mesh.n, lo, hi, U, dt, 5, B.ES_RK_RK4, rk.BS3)
    assert np.all(rel_err_per_var(q, Uo) < TOL)
    assert abs(t - to) < 1e-12 * to


def test_set_tableau_rejects_invalid():
    from paper_2003_08831_gb300 import _binding as B
    s = solver(3, (2, 2, 2), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    A, b, c = rk.RK4["A"].copy(), rk.RK4["b"].copy(), rk.RK4["c"].copy()
    bad = []
    A1 = A.copy()
    A1[1, 2] = 0.1                                    # implicit entry
    bad.append((A1, b, c))
    bad.append((A, b * 1.01, c))                      # sum b != 1
    c1 = c.copy()
    c1[2] = 0.6                                       # row sum != c
    bad.append((A, b, c1))
    b1 = np.array([0.25, 0.5, 0.5, -0.25])            # negative weight with relaxation on
    bad.append((A, b1, c))
    bad.append((np.zeros((11, 11)), np.full(11, 1.0 / 11), np.zeros(11)))   # more than 10 stages
    for A_, b_, c_ in bad:
        with pytest.raises(B.ESError):
            s.set_tableau(A_, b_, c_)
    s.set_tableau(A, b, c)                            # still usable
    assert s.status() == 0
    s.close()


# ---------------------------------------------------------------------------------------
# mixed modes at full size (32^3 TGV): sampled elements against oracle element blocks,
# bars in the FP32 rounding unit

EPS32 = 2.0 ** -23


@pytest.mark.parametrize("prec", [1, 3])
@pytest.mark.parametrize("p,mu,noise", [(3, 0.0, False), (4, 1.0 / 1600.0, True)])
def test_mixed_full_size_rhs_sampled(p, mu, noise, prec):
    """Euler TGV 32^3 p = 3 and the noisy Navier--Stokes TGV 32^3 p = 4 with FP32 fluxes:
    es_rhs per node within 256 eps_32 of the summed term magnitudes of the oracle."""
    mesh, U, lo, hi = tgv_full(p, noise=noise)
    phys = dg.Physics(G, mu=mu, Pr=0.72, diss=1)
    s = solver(p, mesh.n, lo, hi, mu=mu, precision=prec)
    dq = s.rhs(s.to_device(U)).cpu().numpy().reshape(mesh.shape)
    assert s.status() == 0
    s.close()
    radius = 2 if mu > 0 else 1
    nb = 2 * radius + 1
    bm = dg.Mesh(p, (nb, nb, nb), (0, 0, 0), tuple(nb * h for h in mesh.h))
    for c in SAMPLES[:3]:
        B = dg.element_block(U, c, radius)
        ref = dg.rhs(bm, B, phys)[:, radius, radius, radius]
        terms = dg.rhs_term_magnitude(bm, B, phys)[:, radius, radius, radius]
        assert_rhs_close(dq[:, c[2], c[1], c[0]], ref, terms, eps=EPS32)


@pytest.mark.parametrize("prec", [1, 3])
def test_mixed_full_size_step_sampled(prec):
    """One relaxed BS3 step of the 32^3 p = 3 Euler TGV with FP32 fluxes: gamma_kappa of
    sampled elements within 8x its response to FP32-level changes of the right-hand
    side, and q_new - q_old = gamma d within the FP32 rounding of the stage sums."""
    p = 3
    mesh, U, lo, hi = tgv_full(p)
    phys = dg.Physics(G, diss=1)
    dt = rk.stable_dt(mesh, U, phys, 0.5)
    s = solver(p, mesh.n, lo, hi, precision=prec)
    q = s.to_device(U)
    t, gh, gk = s.advance(q, 1, dt)
    assert s.status() == 0
    qn = q.cpu().numpy().reshape(mesh.shape)
    gk = gk.cpu().numpy().reshape(mesh.n[2], mesh.n[1], mesh.n[0])
    gamma = gh.cpu().numpy()[0]
    s.close()
    assert gamma == np.min(gk)
    radius = 3
    nb = 2 * radius + 1
    bm = dg.Mesh(p, (nb, nb, nb), (0, 0, 0), tuple(nb * h for h in mesh.h))
    for c in SAMPLES[:3]:
        B = dg.element_block(U, c, radius)
        r = rk.rk_step(bm, B, dt, phys, rk.BS3, delta_floor=4e-6)
        g_ref = r.gamma_kappa[radius, radius, radius]
        _, sens = gamma_sensitivity(bm, B, dt, 1, phys, rk.BS3, "local", [r], seeds=2, eps=EPS32)
        tol = max(1e-6, 8 * sens.reshape(nb, nb, nb)[radius, radius, radius])
        g_got = gk[c[2], c[1], c[0]]
        if np.isinf(g_ref):        # change below the floor: unconstrained on both sides
            assert np.isinf(g_got), (c, g_got)
        else:
            assert abs(g_got - g_ref) <= tol * g_ref, (c, g_got, g_ref, tol)
        d_ref = r.d[:, radius, radius, radius]
        d_got = (qn[:, c[2], c[1], c[0]] - U[:, c[2], c[1], c[0]]) / gamma
        terms = dg.rhs_term_magnitude(bm, B, phys)[:, radius, radius, radius]
        bound = 1e-6 * np.max(np.abs(d_ref)) + dt * 256 * EPS32 * terms + 4 * EPS * np.abs(U[:, c[2], c[1], c[0]])
        assert np.all(np.abs(d_got - d_ref) <= bound)

