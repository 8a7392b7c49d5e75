"""Local relaxation: Eq. (relaxation-local-gamma), Lemma 2.1, Theorem 2.3 (FP64).

For every element kappa the last row of Eq. (relaxation-local-gamma) is the
scalar equation

    r_kappa(gamma) = eta_kappa(u_old + gamma d) - eta_kappa_old - gamma Delta eta_kappa = 0,

d = u_new - u_old, Delta eta_kappa = eta_kappa_new - eta_kappa_old.  Lemma 2.1
gives a unique root gamma_kappa > 0; Theorem 2.3 takes gamma = min_kappa
gamma_kappa, u = u_old + gamma d, t = t_old + gamma dt.

Reading (the paper prints only the equation).  r_kappa is evaluated in a
form that is algebraically identical but free of the cancellation between the
O(1) entropies and the O(dt^2) root condition:

    r_kappa(gamma) = sum_n P_n Dbreg_n(gamma) + gamma A_kappa,
    Dbreg_n(gamma) = S(u_n + gamma d_n) - S(u_n) - gamma w(u_n).d_n   (>= 0),
    A_kappa        = sum_n P_n w(u_n).d_n - Delta eta_kappa.

With x = gamma d_rho/rho, dv = gamma (d_m - v d_rho)/rho', y = (p' - p)/p
(primes at u + gamma d) the Bregman term of S = -rho s/(gamma_g - 1) is

    Dbreg = rho [gamma_g phi(x) + psi(y) - x log1p(y)]/(gamma_g - 1)
            + rho rho' |dv|^2 / (2 p),
    phi(x) = (1+x) log1p(x) - x,   psi(y) = y - log1p(y),

in which the s terms cancel exactly.  Inside a Runge--Kutta step A_kappa is
accumulated as -dt sum_i b_i sum_n P_n (w(y^i_n) - w(u_n)).k_i,n with the
differences of w evaluated from the stage increments (``entropy_variables_
difference``); that equals sum P w(u).d - dt sum_i b_i (eta' f)(y^i) of
Eq. (eta-est-1-RK).

Root (Section 4 allows any robust scalar solver): Newton's method started at
the root of the quadratic model a gamma^2 + A gamma, a = (1/2) sum P d^T S'' d,
safeguarded by bisection on a bracket [lo, hi] with r(lo) <= 0 < r(hi) inside
(0, GAMMA_MAX]; it stops when the Newton step is below 4 * 2^-52 max(1, gamma)
or the bracket is that narrow.

Degenerate elements (the paper needs eta''(f, f) != 0, Lemma 2.1): with
s_kappa = sum_n P_n rho_n and delta_kappa = sqrt(2 a / s_kappa), the RMS relative
change of the element's state over the step, an element with
delta_kappa <= delta_floor is unconstrained (gamma_kappa = +inf).  If r'(0) =
A_kappa >= 0 on a non-degenerate element no positive root exists: the element
is flagged and left unconstrained.  If r(GAMMA_MAX) <= 0, gamma_kappa =
GAMMA_MAX.  gamma = min_kappa gamma_kappa, or 1 when every element is
unconstrained.
"""
import numpy as np

from . import gas

GAMMA_MAX = 8.0
DELTA_FLOOR = 1.0e-8
TOL = 4.0 * 2.0 ** -52


def log1pmx(z):
    """log(1 + z) - z without cancellation: Taylor series for |z| < 1/2."""
    z = np.asarray(z, dtype=np.float64)
    small = np.abs(z) < 0.5
    zs = np.where(small, z, 0.0)
    acc = np.zeros_like(zs)
    term = zs * zs
    # sum_{k>=2} (-1)^(k+1) z^k / k ; 0.5^60 / 60 < 1e-19
    for k in range(2, 62):
        acc += (-1.0) ** (k + 1) * term / k
        term = term * zs
    with np.errstate(invalid="ignore", divide="ignore"):
        direct = np.log1p(z) - z
    return np.where(small, acc, direct)


def _increment_parts(u, e, g):
    """x, dv, y and rho' for the state change u -> u + e (see module docstring)."""
    rho, v, p = gas.primitives(u, g)
    x = e[0] / rho
    rho1 = rho + e[0]
    dv = (e[1:4] - v * e[0]) / rho1
    dv2 = np.sum(dv * dv, axis=0)
    # p' - p = (g-1) [e_E - v.e_m + |v|^2 e_rho / 2] - (g-1) rho' |dv|^2 / 2
    dp = (g - 1.0) * (e[4] - np.sum(v * e[1:4], axis=0) + 0.5 * np.sum(v * v, axis=0) * e[0]) \
        - 0.5 * (g - 1.0) * rho1 * dv2
    y = dp / p
    return rho, v, p, x, rho1, dv, dv2, y


def bregman_entropy(u, e, g):
    """S(u + e) - S(u) - w(u).e, cancellation-free; nan where u + e is not physical."""
    rho, v, p, x, rho1, dv, dv2, y = _increment_parts(u, e, g)
    ok = (x > -1.0) & (y > -1.0)
    xs = np.where(ok, x, 0.0)
    ys = np.where(ok, y, 0.0)
    Lx = log1pmx(xs)
    Ly = log1pmx(ys)
    phi = (1.0 + xs) * Lx + xs * xs          # (1+x) log1p(x) - x
    psi = -Ly                                # y - log1p(y)
    cross = xs * (ys + Ly)                   # x log1p(y)
    D = rho * (g * phi + psi - cross) / (g - 1.0) + rho * rho1 * dv2 / (2.0 * p)
    return np.where(ok, D, np.nan)


def entropy_variables_difference(u, e, g):
    """w(u + e) - w(u) from the increment e without cancellation."""
    rho, v, p, x, rho1, dv, dv2, y = _increment_parts(u, e, g)
    beta = rho / p
    ds = np.log1p(y) - g * np.log1p(x)                # s(u+e) - s(u)
    v2 = np.sum(v * v, axis=0)
    # beta' |v'|^2/2 - beta |v|^2/2 with beta' = beta (1+x)/(1+y), v' = v + dv
    dkin = 0.5 * beta * ((x - y) * v2 + (1.0 + x) * (2.0 * np.sum(v * dv, axis=0) + dv2)) / (1.0 + y)
    dw1 = -ds / (g - 1.0) - dkin
    dwv = beta * ((x - y) * v + (1.0 + x) * dv) / (1.0 + y)
    dw5 = -beta * (x - y) / (1.0 + y)
    return np.stack([dw1, dwv[0], dwv[1], dwv[2], dw5])


def hessian_form(u, d, g):
    """d^T S''(u) d = rho X^2 + rho (X - Y)^2/(g-1) + rho^2 |dv|^2/p (X = d_rho/rho, Y = dp_lin/p)."""
    rho, v, p = gas.primitives(u, g)
    X = d[0] / rho
    dvl = (d[1:4] - v * d[0]) / rho
    Y = (g - 1.0) * (d[4] - np.sum(v * d[1:4], axis=0) + 0.5 * np.sum(v * v, axis=0) * d[0]) / p
    return rho * X * X + rho * (X - Y) ** 2 / (g - 1.0) + rho * rho * np.sum(dvl * dvl, axis=0) / p


class ElementProblem:
    """r(gamma) for a set of elements; u, d of shape (5, ne, Np), weights P (ne, Np)."""

    def __init__(self, u, d, A, P, g):
        self.u, self.d, self.A, self.P, self.g = u, d, np.asarray(A, dtype=np.float64), P, g

    def r(self, gam):
        gam = np.asarray(gam, dtype=np.float64)
        D = bregman_entropy(self.u, gam[:, None] * self.d, self.g)
        return np.sum(self.P * D, axis=-1) + gam * self.A

    def dr(self, gam):
        gam = np.asarray(gam, dtype=np.float64)
        dw = entropy_variables_difference(self.u, gam[:, None] * self.d, self.g)
        return np.sum(self.P * np.sum(dw * self.d, axis=0), axis=-1) + self.A


def solve_gamma(u, d, A, P, g, delta_floor=DELTA_FLOOR, gamma_max=GAMMA_MAX, max_iter=200):
    """gamma_kappa for each element.

    u, d: (5, ne, Np); A: (ne,); P: (ne, Np) mass weights.
    Returns (gamma_kappa, flags) with flags 0 = solved, 1 = unconstrained
    (degenerate), 2 = no positive root (r'(0) >= 0), 3 = capped at gamma_max.
    """
    ne = u.shape[1]
    rho = u[0]
    a = 0.5 * np.sum(P * hessian_form(u, d, g), axis=-1)
    s = np.sum(P * rho, axis=-1)
    delta = np.sqrt(2.0 * a / s)
    gam_k = np.full(ne, np.inf)
    flags = np.zeros(ne, dtype=np.int64)
    degenerate = delta <= delta_floor
    flags[degenerate] = 1
    noroot = (~degenerate) & (A >= 0.0)
    flags[noroot] = 2
    act = np.nonzero(~degenerate & ~noroot)[0]
    if act.size == 0:
        return gam_k, flags
    prob = ElementProblem(u[:, act], d[:, act], A[act], P[act], g)
    g0 = np.clip(-A[act] / a[act], 1e-3, gamma_max)
    # bracket: lo with r(lo) <= 0 (r(0) = 0), hi with r(hi) > 0 or gamma_max
    lo = np.zeros(act.size)
    hi = np.full(act.size, gamma_max)
    r_hi = prob.r(hi)
    capped = ~(r_hi > 0.0)     # includes nan (non-physical at gamma_max): treated as r > 0 below
    capped &= ~np.isnan(r_hi)
    gam = g0.copy()
    done = capped.copy()
    for _ in range(max_iter):
        if np.all(done):
            break
        idx = np.nonzero(~done)[0]
        sub = ElementProblem(prob.u[:, idx], prob.d[:, idx], prob.A[idx], prob.P[idx], g)
        gi = gam[idx]
        ri = sub.r(gi)
        nonphys = np.isnan(ri)
        pos = nonphys | (ri > 0.0)
        lo[idx] = np.where(pos, lo[idx], gi)
        hi[idx] = np.where(pos, gi, hi[idx])
        di = sub.dr(gi)
        with np.errstate(divide="ignore", invalid="ignore"):
            step_n = ri / di
            newton = gi - step_n
        tol = TOL * np.maximum(1.0, gi)
        # a Newton step below the tolerance has converged even when rounding puts the
        # iterate on an end of the bracket
        newton_conv = (~nonphys) & (di > 0.0) & np.isfinite(newton) & (np.abs(step_n) <= tol)
        ok = (~nonphys) & np.isfinite(newton) & (newton > lo[idx]) & (newton < hi[idx])
        nxt = np.where(ok, newton, 0.5 * (lo[idx] + hi[idx]))
        conv = newton_conv | ((hi[idx] - lo[idx]) <= tol) | (ri == 0.0)
        gam[idx] = np.where(newton_conv, np.clip(newton, lo[idx], hi[idx]), np.where(conv, gi, nxt))
        done[idx] = conv
    gam = np.where(capped, gamma_max, gam)
    gam_k[act] = gam
    flags[act[capped]] = 3
    return gam_k, flags


def global_gamma(gamma_kappa):
    """gamma = min_kappa gamma_kappa (Theorem 2.3); 1 when nothing constrains the step."""
    gmin = np.min(gamma_kappa)
    return 1.0 if not np.isfinite(gmin) else float(gmin)
