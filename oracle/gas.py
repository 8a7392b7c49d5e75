"""Ideal-gas thermodynamics, entropy and two-point fluxes (FP64, Section 3.1).

Conserved variables q = (rho, rho U1, rho U2, rho U3, rho E) with P = rho R T
(Section 3.1, first equations).  Arrays carry the 5 components on axis 0 and
broadcast over the remaining axes.

Readings where the paper is silent (it cites the references but prints none of
these formulas):

* Entropy.  S = -rho s with s the thermodynamic entropy (Section 3.1).  The
  specific entropy is taken as s = ln p - gamma ln rho and S = -rho s/(gamma-1)
  (Harten's scaling).  The relaxation parameter is invariant under
  S -> a S + b.q with a > 0, so the scaling cannot change any gamma_kappa.
  Entropy variables w = dS/dq = ((gamma - s)/(gamma-1) - rho|v|^2/(2p),
  rho v/p, -rho/p).
* Entropy-conservative two-point flux: the Ismail--Roe flux in the
  parameter-vector form z = sqrt(rho/p) (1, v1, v2, v3, p).
* Logarithmic mean: the Ismail--Roe series, zeta = aL/aR, f = (zeta-1)/(zeta+1),
  u = f^2, F = 1 + u/3 + u^2/5 + u^3/7 when u < eps_s else ln(zeta)/(2f), and
  a_ln = (aL + aR)/(2F).  eps_s = 1e-4 in FP64 (truncation below 1.2e-17).
* Interface dissipation diss^I: scalar Rusanov (local Lax--Friedrichs) in
  conserved variables with lambda = max over both sides of |v.n| + c (diss = 1),
  or the matrix dissipation in entropy variables of the references the paper cites
  for diss^I (diss = 2): (1/2) R |Lambda| T R^T [[w]] with the eigenvectors R of
  the flux Jacobian along the face normal and Barth's scaling T (R T R^T = dq/dw),
  evaluated at the mean state rho = zb1 zb5, u = zb_v/zb1, p = zb5/zb1 of the
  parameter-vector averages (any positive mean state keeps the term dissipative;
  this one needs no logarithmic mean).
* Viscous flux: Stokes stress with constant mu, Fourier heat flux with
  kappa = mu c_p / Pr, c_p = gamma R / (gamma - 1).  The flux is evaluated from
  the entropy-variable gradients theta_j = dw/dx_j through the chain rule
  v = -w_{2..4}/w_5, T = -1/(R w_5), which is the product C_mj theta_j of
  Eq. (compressible_ns_diss) without forming C.
"""
import numpy as np

LOGMEAN_EPS_FP64 = 1.0e-4


def primitives(q, g):
    rho = q[0]
    v = q[1:4] / rho
    p = (g - 1.0) * (q[4] - 0.5 * rho * np.sum(v * v, axis=0))
    return rho, v, p


def conserved(rho, v, p, g):
    v = np.asarray(v)
    return np.stack([rho, rho * v[0], rho * v[1], rho * v[2],
                     p / (g - 1.0) + 0.5 * rho * np.sum(v * v, axis=0)])


def specific_entropy(rho, p, g):
    return np.log(p) - g * np.log(rho)


def entropy(q, g):
    """S(q) = -rho s / (gamma - 1)."""
    rho, _, p = primitives(q, g)
    return -rho * specific_entropy(rho, p, g) / (g - 1.0)


def entropy_variables(q, g):
    """w = dS/dq."""
    rho, v, p = primitives(q, g)
    s = specific_entropy(rho, p, g)
    beta = rho / p
    w1 = (g - s) / (g - 1.0) - 0.5 * beta * np.sum(v * v, axis=0)
    return np.stack([w1, beta * v[0], beta * v[1], beta * v[2], -beta])


def euler_flux(q, g, m):
    """Inviscid flux F^I_m(q) in coordinate direction m (0, 1, 2)."""
    rho, v, p = primitives(q, g)
    vm = v[m]
    f = np.stack([q[0] * vm, q[1] * vm, q[2] * vm, q[3] * vm, (q[4] + p) * vm])
    f[1 + m] = f[1 + m] + p
    return f


def entropy_potential(q, g, m):
    """psi_m = w.F_m - S v_m, which equals rho v_m for this entropy scaling."""
    rho, v, _ = primitives(q, g)
    return rho * v[m]


def sound_speed(q, g):
    rho, _, p = primitives(q, g)
    return np.sqrt(g * p / rho)


def log_mean(aL, aR, eps=LOGMEAN_EPS_FP64):
    """Logarithmic mean (aR - aL)/(ln aR - ln aL) by the Ismail--Roe series."""
    aL = np.asarray(aL, dtype=np.float64)
    aR = np.asarray(aR, dtype=np.float64)
    zeta = aL / aR
    f = (zeta - 1.0) / (zeta + 1.0)
    u = f * f
    small = u < eps
    F_series = 1.0 + u / 3.0 + u * u / 5.0 + u * u * u / 7.0
    with np.errstate(divide="ignore", invalid="ignore"):
        F_log = np.log(zeta) / (2.0 * f)
    F = np.where(small, F_series, F_log)
    return (aL + aR) / (2.0 * F)


def parameter_vector(q, g):
    rho, v, p = primitives(q, g)
    z1 = np.sqrt(rho / p)
    return np.stack([z1, z1 * v[0], z1 * v[1], z1 * v[2], np.sqrt(rho * p)])


def ec_flux(qL, qR, g, m):
    """Ismail--Roe entropy-conservative two-point flux in direction m."""
    zL = parameter_vector(qL, g)
    zR = parameter_vector(qR, g)
    zb = 0.5 * (zL + zR)
    z1ln = log_mean(zL[0], zR[0])
    z5ln = log_mean(zL[4], zR[4])
    rho_hat = zb[0] * z5ln
    u_hat = zb[1:4] / zb[0]
    p1_hat = zb[4] / zb[0]
    p2_hat = (g + 1.0) / (2.0 * g) * z5ln / z1ln + (g - 1.0) / (2.0 * g) * zb[4] / zb[0]
    h_hat = g * p2_hat / ((g - 1.0) * rho_hat) + 0.5 * np.sum(u_hat * u_hat, axis=0)
    um = u_hat[m]
    f = np.stack([rho_hat * um,
                  rho_hat * um * u_hat[0],
                  rho_hat * um * u_hat[1],
                  rho_hat * um * u_hat[2],
                  rho_hat * um * h_hat])
    f[1 + m] = f[1 + m] + p1_hat
    return f


def matrix_dissipation_parts(zL, zR, g, m):
    """Eigenvectors R (5 x 5 x ...: R[:, k] the k-th), eigenvalues lam and Barth's
    scaling T along direction m at the mean state of the parameter-vector averages."""
    zb = 0.5 * (zL + zR)
    rho = zb[0] * zb[4]
    u = zb[1:4] / zb[0]
    p = zb[4] / zb[0]
    a = np.sqrt(g * p / rho)
    h = a * a / (g - 1.0) + 0.5 * np.sum(u * u, axis=0)
    un = u[m]
    e = np.zeros((3,) + np.shape(un))
    e[m] = 1.0
    t1, t2 = [k for k in range(3) if k != m]
    one, zero = np.ones_like(un), np.zeros_like(un)
    R = np.empty((5, 5) + np.shape(un))
    R[:, 0] = np.concatenate([[one], u - a * e, [h - un * a]])
    R[:, 1] = np.concatenate([[one], u, [0.5 * np.sum(u * u, axis=0)]])
    for col, t in ((2, t1), (3, t2)):
        et = np.zeros((3,) + np.shape(un))
        et[t] = 1.0
        R[:, col] = np.concatenate([[zero], et, [u[t]]])
    R[:, 4] = np.concatenate([[one], u + a * e, [h + un * a]])
    lam = np.stack([un - a, un, un, un, un + a])
    T = np.stack([rho / (2.0 * g), rho * (g - 1.0) / g, p, p, rho / (2.0 * g)])
    return R, lam, T


def interface_flux(qL, qR, g, m, diss):
    """Numerical interface flux f_num(qL, qR) (qL on the -x_m side, qR on the +x_m side).

    diss = 0: the entropy-conservative flux; diss = 1: minus the Rusanov term
    lambda/2 (qR - qL); diss = 2: minus the matrix term (1/2) R |Lambda| T R^T [[w]].
    """
    f = ec_flux(qL, qR, g, m)
    if diss == 2:
        R, lam, T = matrix_dissipation_parts(parameter_vector(qL, g), parameter_vector(qR, g), g, m)
        jw = entropy_variables(qR, g) - entropy_variables(qL, g)
        alpha = np.einsum("ik...,i...->k...", R, jw) * np.abs(lam) * T
        return f - 0.5 * np.einsum("ik...,k...->i...", R, alpha)
    if diss:
        _, vL, _ = primitives(qL, g)
        _, vR, _ = primitives(qR, g)
        lam = np.maximum(np.abs(vL[m]) + sound_speed(qL, g),
                         np.abs(vR[m]) + sound_speed(qR, g))
        f = f - diss * 0.5 * lam * (qR - qL)
    return f


def viscous_flux(q, theta, g, mu, Pr, R):
    """Viscous fluxes F^V_m, m = 0, 1, 2, from theta[m] = dw/dx_m.

    Returns an array of shape (3, 5, ...).
    """
    rho, v, p = primitives(q, g)
    w5 = -rho / p
    # velocity and temperature gradients via the chain rule
    # v_k = -w_{k+1}/w_5  ->  d v_k = -(d w_{k+1} + v_k d w_5)/w_5
    # T = -1/(R w_5)       ->  d T = d w_5 / (R w_5^2)
    grad_v = np.empty((3, 3) + rho.shape)        # grad_v[j, k] = d v_k / d x_j
    grad_T = np.empty((3,) + rho.shape)
    for j in range(3):
        for k in range(3):
            grad_v[j, k] = -(theta[j][1 + k] + v[k] * theta[j][4]) / w5
        grad_T[j] = theta[j][4] / (R * w5 * w5)
    div_v = grad_v[0, 0] + grad_v[1, 1] + grad_v[2, 2]
    kappa = mu * g * R / ((g - 1.0) * Pr)
    fv = np.zeros((3, 5) + rho.shape)
    for m in range(3):
        for k in range(3):
            tau_mk = mu * (grad_v[m, k] + grad_v[k, m])
            if k == m:
                tau_mk = tau_mk - mu * (2.0 / 3.0) * div_v
            fv[m, 1 + k] = tau_mk
            fv[m, 4] = fv[m, 4] + tau_mk * v[k]
        fv[m, 4] = fv[m, 4] + kappa * grad_T[m]
    return fv


def viscous_jacobian(q, g, mu, Pr, R, m):
    """C_mm(q), the block of F^V_m = sum_j C_mj dw/dx_j that multiplies dw/dx_m, written
    out as a 5 x 5 matrix per node (shape (5, 5, ...)); Section 3.1 cites the C_mj.

    With RT = p/rho, the velocity part of a w-gradient g is b = M g, M = [0 | I_3 | v]
    (d v = RT (d w_{2..4} + v d w_5)), and d T = R T^2 d w_5, so
        C_mm = mu RT M^T (I + e_m e_m^T / 3) M + kappa R T^2 e_5 e_5^T,
    symmetric positive semidefinite.
    """
    rho, v, p = primitives(q, g)
    RT = p / rho
    kappa = mu * g * R / ((g - 1.0) * Pr)
    M = np.zeros((3, 5) + rho.shape)
    for k in range(3):
        M[k, 1 + k] = 1.0
        M[k, 4] = v[k]
    N = np.eye(3)
    N[m, m] += 1.0 / 3.0
    C = mu * RT * np.einsum("ki...,kl,lj...->ij...", M, N, M)
    C[4, 4] = C[4, 4] + kappa * RT * RT / R
    return C
