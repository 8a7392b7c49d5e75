"""Explicit Runge--Kutta step with the local relaxation of Section 2 (FP64).

Eq. (RK-step): y^i = u + dt sum_j a_ij f(y^j), u_new = u + dt sum_i b_i f(y^i).
Eq. (eta-est-1-RK): eta_kappa_new = eta_kappa(u) + dt sum_i b_i (eta_kappa' f)(y^i),
valid for b_i >= 0; m = 1 (u_old = u^{n-1}).
Eq. (relaxation-local-gamma) + Theorem 2.3: gamma = min_kappa gamma_kappa,
u^n = u + gamma (u_new - u), t^n = t + gamma dt.

Tableaux (Section 4 names them; the paper prints no coefficients):
* BS3  -- Bogacki & Shampine (1989) 3(2) pair, c = (0, 1/2, 3/4, 1),
          a21 = 1/2, a32 = 3/4, a4 = (2/9, 1/3, 4/9), b = (2/9, 1/3, 4/9, 0).
          b_4 = 0, so only three stages enter u_new and the estimate.
* RK4  -- the classical four-stage method, b = (1/6, 1/3, 1/3, 1/6).
* RK65 -- Butcher's (1964) six-stage fifth-order method, c = (0, 1/4, 1/4, 1/2, 3/4, 1),
          b = (7, 0, 32, 12, 32, 7)/90 >= 0: a fifth-order method for p = 4 in place of
          the BSRK(8,5) that Section 4 names without printing it.

Relaxation modes: 'local' (this paper), 'global' (one gamma for the sum of the
local entropies, Eqs. (u-n-gamma), (t-n-gamma)), 'none' (gamma = 1, the baseline).
"""
import numpy as np

from . import dg, gas, relax

BS3 = {
    "name": "BS3",
    "A": np.array([[0.0, 0.0, 0.0, 0.0],
                   [0.5, 0.0, 0.0, 0.0],
                   [0.0, 0.75, 0.0, 0.0],
                   [2.0 / 9.0, 1.0 / 3.0, 4.0 / 9.0, 0.0]]),
    "b": np.array([2.0 / 9.0, 1.0 / 3.0, 4.0 / 9.0, 0.0]),
    "c": np.array([0.0, 0.5, 0.75, 1.0]),
    "order": 3,
}

RK4 = {
    "name": "RK4",
    "A": np.array([[0.0, 0.0, 0.0, 0.0],
                   [0.5, 0.0, 0.0, 0.0],
                   [0.0, 0.5, 0.0, 0.0],
                   [0.0, 0.0, 1.0, 0.0]]),
    "b": np.array([1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0]),
    "c": np.array([0.0, 0.5, 0.5, 1.0]),
    "order": 4,
}

RK65 = {
    "name": "RK65",
    "A": np.array([[0.0, 0.0, 0.0, 0.0, 0.0, 0.0],
                   [1.0 / 4.0, 0.0, 0.0, 0.0, 0.0, 0.0],
                   [1.0 / 8.0, 1.0 / 8.0, 0.0, 0.0, 0.0, 0.0],
                   [0.0, -1.0 / 2.0, 1.0, 0.0, 0.0, 0.0],
                   [3.0 / 16.0, 0.0, 0.0, 9.0 / 16.0, 0.0, 0.0],
                   [-3.0 / 7.0, 2.0 / 7.0, 12.0 / 7.0, -12.0 / 7.0, 8.0 / 7.0, 0.0]]),
    "b": np.array([7.0, 0.0, 32.0, 12.0, 32.0, 7.0]) / 90.0,
    "c": np.array([0.0, 1.0 / 4.0, 1.0 / 4.0, 1.0 / 2.0, 3.0 / 4.0, 1.0]),
    "order": 5,
}

TABLEAUX = {"BS3": BS3, "RK4": RK4, "RK65": RK65}


def used_stages(tab):
    """Stages whose f(y^i) enter u_new (trailing zero weights dropped)."""
    b = tab["b"]
    s = len(b)
    while s > 0 and b[s - 1] == 0.0:
        s -= 1
    return s


class StepResult:
    pass


def rk_step(mesh, U, dt, phys, tab, mode="local", delta_floor=relax.DELTA_FLOOR, rhs=None, t=0.0):
    """One relaxed RK step from U (shape mesh.shape) at time t.  Returns a StepResult.

    rhs(mesh, U, phys, t=...) defaults to dg.rhs; tests pass a perturbed one to
    measure how the relaxation parameters respond to last-bit changes of f.  Stage i
    is evaluated at t + c_i dt (prescribed boundary states depend on it)."""
    rhs = dg.rhs if rhs is None else rhs
    g = phys.gamma
    A_tab, b = tab["A"], tab["b"]
    s = used_stages(tab)
    P = mesh.mass()
    ks = []
    E = []                       # (eta_kappa' f)(y^i)
    Acc = np.zeros(U.shape[1:4])  # -dt sum_i b_i sum_n P (w(y^i) - w(u)).k_i
    for i in range(s):
        Y = U.copy()
        for j in range(i):
            if A_tab[i, j] != 0.0:
                Y = Y + dt * A_tab[i, j] * ks[j]
        k = rhs(mesh, Y, phys, t=t + tab["c"][i] * dt)
        ks.append(k)
        E.append(dg.entropy_rate(mesh, Y, k, phys))
        if i > 0 and b[i] != 0.0:
            dW = relax.entropy_variables_difference(U, Y - U, g)
            Acc -= dt * b[i] * mesh.element_sum(np.sum(dW * k, axis=0))
    d = np.zeros_like(U)
    for i in range(s):
        d = d + dt * b[i] * ks[i]
    res = StepResult()
    res.d = d
    res.ks = ks
    res.E = np.stack(E)
    res.deta = dt * np.tensordot(b[:s], res.E, axes=1)          # eta_new - eta_old
    res.A = Acc
    if mode == "none":
        gam_k = np.full(mesh.K, np.inf)       # no element constrains the step
        flags = np.ones(mesh.K, dtype=np.int64)
        gam = 1.0
    else:
        uf = mesh.flat(U)
        df = mesh.flat(d)
        Pf = np.broadcast_to(P.reshape(1, -1), (mesh.K, mesh.Np))
        Af = Acc.reshape(-1)
        if mode == "local":
            gam_k, flags = relax.solve_gamma(uf, df, Af, Pf, g, delta_floor=delta_floor)
            gam = relax.global_gamma(gam_k)
        elif mode == "global":
            gk, flags = relax.solve_gamma(uf.reshape(5, 1, -1), df.reshape(5, 1, -1),
                                          np.array([Af.sum()]), Pf.reshape(1, -1), g,
                                          delta_floor=delta_floor)
            gam = relax.global_gamma(gk)
            gam_k = np.full(mesh.K, gam)
        else:
            raise ValueError(mode)
    res.gamma_kappa = np.asarray(gam_k).reshape(U.shape[1:4]) if np.ndim(gam_k) else gam_k
    res.flags = np.asarray(flags).reshape(-1)
    res.gamma = gam
    res.U = U + gam * d
    return res


def advance(mesh, U, dt, nsteps, phys, tab, mode="local", t0=0.0, delta_floor=relax.DELTA_FLOOR, rhs=None):
    """nsteps relaxed steps; returns (U, t, list of StepResult)."""
    t = t0
    hist = []
    for _ in range(nsteps):
        r = rk_step(mesh, U, dt, phys, tab, mode=mode, delta_floor=delta_floor, rhs=rhs, t=t)
        U = r.U
        t = t + r.gamma * dt
        hist.append(r)
    return U, t, hist


def stable_dt(mesh, U, phys, cfl):
    """Fixed time step from the initial state (the paper states none; Section 4.1.1
    only fixes U dt/dx).  Reading: the sum of the directional Courant numbers,
    dt = cfl / ((2p+1) max_n sum_m (|v_m| + c)/h_m), and for mu > 0 also
    dt <= cfl rho_min / (mu max(4/3, gamma/Pr) sum_m ((2p+1)/h_m)^2)."""
    g = phys.gamma
    rho, v, p = gas.primitives(U, g)
    c = np.sqrt(g * p / rho)
    lam = np.max(sum((np.abs(v[m]) + c) / mesh.h[m] for m in range(3)))
    dt = cfl / ((2 * mesh.p + 1) * lam)
    if phys.mu > 0.0:
        k2 = sum(((2 * mesh.p + 1) / mesh.h[m]) ** 2 for m in range(3))
        dt = min(dt, cfl * float(np.min(rho)) / (phys.mu * max(4.0 / 3.0, g / phys.Pr) * k2))
    return dt
