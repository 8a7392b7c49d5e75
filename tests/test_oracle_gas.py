"""Pins for oracle.gas and the pointwise parts of oracle.relax.

Each check is fixed by mathematics independent of the oracle's formulas:
high-precision evaluations of the defining expressions (mpmath, 40 digits),
Tadmor's entropy-conservation condition, Eq. (compat), closed-form values.
"""
import numpy as np
import pytest

from oracle import gas, relax

mp = pytest.importorskip("mpmath")
mp.mp.dps = 40
G = 1.4


def rand_states(n, seed, spread=0.3):
    rng = np.random.default_rng(seed)
    rho = 1.0 + spread * (2 * rng.random(n) - 1)
    v = rng.normal(size=(3, n)) * 0.8
    p = 1.0 + spread * (2 * rng.random(n) - 1)
    return gas.conserved(rho, v, p, G)


def _mpf(a):
    return a if isinstance(a, mp.mpf) else mp.mpf(float(a))


def mp_S(q):
    rho, m1, m2, m3, E = [_mpf(a) for a in q]
    p = (mp.mpf(G) - 1) * (E - (m1 * m1 + m2 * m2 + m3 * m3) / (2 * rho))
    s = mp.log(p) - mp.mpf(G) * mp.log(rho)
    return -rho * s / (mp.mpf(G) - 1)


def mp_S_at(q, e, gam=1):
    qq = [mp.mpf(float(a)) + mp.mpf(gam) * mp.mpf(float(b)) for a, b in zip(q, e)]
    rho, m1, m2, m3, E = qq
    p = (mp.mpf(G) - 1) * (E - (m1 * m1 + m2 * m2 + m3 * m3) / (2 * rho))
    s = mp.log(p) - mp.mpf(G) * mp.log(rho)
    return -rho * s / (mp.mpf(G) - 1)


def mp_w(q):
    return [mp.diff(lambda t, i=i: mp_S(list(q[:i]) + [t] + list(q[i + 1:])), _mpf(q[i])) for i in range(5)]


def test_euler_flux_closed_form():
    q = gas.conserved(np.array(1.0), np.array([1.0, 0.0, 0.0]), np.array(1.0), G)
    f = gas.euler_flux(q, G, 0)
    # rho = 1, v = (1,0,0), p = 1: E = 1/0.4 + 1/2 = 3, flux (1, 1 + 1, 0, 0, (3 + 1) * 1)
    assert np.allclose(f, [1.0, 2.0, 0.0, 0.0, 4.0], rtol=0, atol=1e-15)
    fy = gas.euler_flux(q, G, 1)
    assert np.allclose(fy, [0.0, 0.0, 1.0, 0.0, 0.0], rtol=0, atol=1e-15)


def test_entropy_variables_are_gradient_of_S():
    q = rand_states(6, 1)
    w = gas.entropy_variables(q, G)
    for n in range(6):
        ref = mp_w(q[:, n])
        for i in range(5):
            assert abs(w[i, n] - float(ref[i])) <= 1e-13 * max(1.0, abs(float(ref[i])))


def test_entropy_potential():
    q = rand_states(6, 2)
    w = gas.entropy_variables(q, G)
    S = gas.entropy(q, G)
    for m in range(3):
        f = gas.euler_flux(q, G, m)
        rho, v, p = gas.primitives(q, G)
        psi = np.sum(w * f, axis=0) - S * v[m]
        assert np.max(np.abs(psi - rho * v[m])) < 1e-12


def test_log_mean_against_exact():
    rng = np.random.default_rng(3)
    a = np.exp(rng.normal(size=200))
    rel = np.concatenate([10.0 ** rng.uniform(-12, 0, 150), rng.uniform(0.5, 3, 50)])
    b = a * (1 + rel * np.sign(rng.normal(size=200)))
    b = np.abs(b)
    lm = gas.log_mean(a, b)
    for ai, bi, li in zip(a, b, lm):
        A, B = mp.mpf(float(ai)), mp.mpf(float(bi))
        ref = A if A == B else (B - A) / (mp.log(B) - mp.log(A))
        assert abs(li - float(ref)) <= 4e-16 * float(ref) * 8
    assert gas.log_mean(np.array(2.5), np.array(2.5)) == 2.5


def test_ec_flux_consistency_symmetry_tadmor():
    qL = rand_states(500, 4)
    rng = np.random.default_rng(5)
    scale = 10.0 ** rng.uniform(-8, -0.5, 500)
    qR = gas.conserved(*(lambda r, v, p: (r * (1 + scale * rng.normal(size=500) * 0.3),
                                          v + scale * rng.normal(size=(3, 500)),
                                          p * (1 + scale * rng.normal(size=500) * 0.3)))(*gas.primitives(qL, G)), G)
    for m in range(3):
        fLL = gas.ec_flux(qL, qL, G, m)
        assert np.max(np.abs(fLL - gas.euler_flux(qL, G, m))) < 1e-14 * np.max(np.abs(fLL))
        fLR = gas.ec_flux(qL, qR, G, m)
        fRL = gas.ec_flux(qR, qL, G, m)
        assert np.max(np.abs(fLR - fRL)) < 1e-14 * np.max(np.abs(fLR))
        # Tadmor: (w_R - w_L).f* = psi_R - psi_L, Eq. (compat) in discrete form
        dw = gas.entropy_variables(qR, G) - gas.entropy_variables(qL, G)
        lhs = np.sum(dw * fLR, axis=0)
        rhs_ = gas.entropy_potential(qR, G, m) - gas.entropy_potential(qL, G, m)
        # round-off scale of the two sides: the w's and psi's themselves are O(1)
        wabs = np.abs(gas.entropy_variables(qR, G)) + np.abs(gas.entropy_variables(qL, G))
        sc = np.sum(wabs * np.abs(fLR), axis=0) + np.abs(gas.entropy_potential(qR, G, m)) \
            + np.abs(gas.entropy_potential(qL, G, m))
        assert np.max(np.abs(lhs - rhs_) / sc) < 1e-14


def test_rusanov_dissipates_entropy():
    qL = rand_states(300, 6)
    qR = rand_states(300, 7)
    for m in range(3):
        f_ec = gas.interface_flux(qL, qR, G, m, 0)
        f_es = gas.interface_flux(qL, qR, G, m, 1)
        dw = gas.entropy_variables(qR, G) - gas.entropy_variables(qL, G)
        # entropy production of the interface: (w_R - w_L).(f_es - f_ec) <= 0
        assert np.all(np.sum(dw * (f_es - f_ec), axis=0) <= 1e-14)


def test_sound_speed_closed_form():
    """c = sqrt(gamma p / rho): rho = 1, p = 1 gives sqrt(1.4); rho = 2, p = 3 gives sqrt(2.1)."""
    q = gas.conserved(np.array([1.0, 2.0]), np.array([[0.5, -1.0], [-0.2, 0.3], [0.1, 0.0]]),
                      np.array([1.0, 3.0]), G)
    assert np.allclose(gas.sound_speed(q, G), [np.sqrt(1.4), np.sqrt(2.1)], rtol=1e-15, atol=0)


@pytest.mark.parametrize("m,lam", [(0, 1.0 + np.sqrt(2.1)),          # right side: |-1.0| + sqrt(2.1)
                                   (1, 0.3 + np.sqrt(2.1)),          # right side: |0.3| + sqrt(2.1)
                                   (2, 0.4 + np.sqrt(1.4))])         # left side: |0.4| + sqrt(1.4) > sqrt(2.1)
def test_rusanov_lambda_closed_form(m, lam):
    """Rusanov term of the interface flux: f_num = f_ec - (lambda/2)(qR - qL) with
    lambda = max(|vL.n| + cL, |vR.n| + cR) along the face normal e_m, for the two states
    rho = 1, v = (0.5, -0.2, 0.4), p = 1 (c = sqrt(1.4)) and rho = 2, v = (-1, 0.3, 0),
    p = 3 (c = sqrt(2.1)); in x3 the left side gives the larger speed.  A wrong factor on
    c, a wrong velocity component or a min in place of the max changes lambda."""
    qL = gas.conserved(np.array(1.0), np.array([0.5, -0.2, 0.4]), np.array(1.0), G)
    qR = gas.conserved(np.array(2.0), np.array([-1.0, 0.3, 0.0]), np.array(3.0), G)
    f_ec = gas.interface_flux(qL, qR, G, m, 0)
    f_rus = gas.interface_flux(qL, qR, G, m, 1)
    jump = qR - qL
    assert np.all(np.abs(jump) > 0.05)
    assert np.allclose((f_ec - f_rus) / (0.5 * jump), lam, rtol=1e-13, atol=0)


def _jacobian(fun, x, h=1e-6):
    """Central-difference Jacobian of a vector function of a 5-vector."""
    J = np.empty((5, 5))
    for j in range(5):
        dx = np.zeros(5)
        dx[j] = h * max(1.0, abs(x[j]))
        J[:, j] = (fun(x + dx) - fun(x - dx)) / (2 * dx[j])
    return J


@pytest.mark.parametrize("m", [0, 1, 2])
def test_matrix_dissipation_eigensystem(m):
    """At a single state the mean state is that state: R diag(lam) R^-1 is the flux
    Jacobian df_m/dq and R T R^T = dq/dw (Barth's scaling for S = -rho s/(gamma-1));
    a wrong eigenvector, eigenvalue or scale fails one of the two."""
    q = rand_states(3, 21 + m)[:, 1]
    z = gas.parameter_vector(q, G)
    R, lam, T = gas.matrix_dissipation_parts(z, z, G, m)
    A = _jacobian(lambda x: gas.euler_flux(x, G, m), q)
    assert np.allclose(R @ np.diag(lam) @ np.linalg.inv(R), A, rtol=1e-7, atol=1e-7 * np.max(np.abs(A)))
    dwdq = _jacobian(lambda x: gas.entropy_variables(x, G), q)
    dqdw = np.linalg.inv(dwdq)
    assert np.allclose(R @ np.diag(T) @ R.T, dqdw, rtol=1e-6, atol=1e-7 * np.max(np.abs(dqdw)))


def test_matrix_dissipation_consistent_and_dissipative():
    qL = rand_states(300, 16)
    qR = rand_states(300, 17)
    for m in range(3):
        f_ec = gas.interface_flux(qL, qR, G, m, 0)
        f_md = gas.interface_flux(qL, qR, G, m, 2)
        dw = gas.entropy_variables(qR, G) - gas.entropy_variables(qL, G)
        assert np.all(np.sum(dw * (f_md - f_ec), axis=0) <= 1e-14)
        assert np.allclose(gas.interface_flux(qL, qL, G, m, 2), gas.euler_flux(qL, G, m), rtol=1e-13, atol=1e-13)
        # the matrix form dissipates no more than the scalar one on each wave family:
        # |lambda_k| <= lambda_max, so its entropy production is smaller in size
        f_rs = gas.interface_flux(qL, qR, G, m, 1)
        assert np.all(np.sum(dw * (f_md - f_ec), axis=0) >= np.sum(dw * (f_rs - f_ec), axis=0) - 1e-12)


def test_viscous_flux_shear_and_positivity():
    # linear shear u = a y: tau_xy = mu a; heat flux from a temperature gradient
    rho, p = 1.2, 0.9
    v = np.array([0.3, -0.2, 0.1])
    q = gas.conserved(np.array(rho), v, np.array(p), G)
    R, mu, Pr = 1.0, 0.01, 0.72
    w = gas.entropy_variables(q, G)
    a, bT = 0.7, 0.4
    # d/dy of w for u_x' = a at fixed rho, p: d w_2 / dy = rho a / p
    theta = np.zeros((3, 5))
    theta[1, 1] = rho * a / p
    fv = gas.viscous_flux(q, theta, G, mu, Pr, R)
    assert abs(fv[1, 1] - mu * a) < 1e-15 and abs(fv[0, 2] - mu * a) < 1e-15
    assert abs(fv[1, 4] - mu * a * v[0]) < 1e-15
    # temperature gradient along z: T = p/(rho R), dT/dz = bT via w_5 = -1/(R T)
    T = p / (rho * R)
    theta = np.zeros((3, 5))
    theta[2, 4] = bT / (R * T * T)
    theta[2, 1:4] = -v * theta[2, 4] * (-w[4]) / (-w[4])  # keep velocity gradient zero: dw_v = -v dw_5
    theta[2, 1:4] = -v * theta[2, 4]
    fv = gas.viscous_flux(q, theta, G, mu, Pr, R)
    kappa = mu * G * R / ((G - 1) * Pr)
    assert abs(fv[2, 4] - kappa * bT) < 1e-14
    assert np.max(np.abs(fv[2, 1:4])) < 1e-15
    # pure dilatation u_x = a x at fixed rho, p: tau_xx = (4/3) mu a, tau_yy = tau_zz = -(2/3) mu a
    theta = np.zeros((3, 5))
    theta[0, 1] = rho * a / p
    fv = gas.viscous_flux(q, theta, G, mu, Pr, R)
    assert abs(fv[0, 1] - 4.0 / 3.0 * mu * a) < 1e-15
    assert abs(fv[1, 2] + 2.0 / 3.0 * mu * a) < 1e-15 and abs(fv[2, 3] + 2.0 / 3.0 * mu * a) < 1e-15
    # theta . F^V >= 0 for random gradients (C_mj positive semidefinite)
    rng = np.random.default_rng(8)
    qs = rand_states(100, 9)
    th = rng.normal(size=(3, 5, 100))
    fv = gas.viscous_flux(qs, th, G, mu, Pr, R)
    assert np.all(np.sum(th * fv, axis=(0, 1)) >= -1e-15)


def test_log1pmx():
    for z in [1e-12, -3e-9, 1e-5, -0.01, 0.2, -0.45, 0.49, 0.51, -0.7, 2.0]:
        ref = mp.log1p(mp.mpf(z)) - mp.mpf(z)
        assert abs(float(relax.log1pmx(np.array(z))) - float(ref)) <= 4e-16 * abs(float(ref)) * 4


@pytest.mark.parametrize("scale", [1e-9, 1e-6, 1e-3, 5e-2])
def test_bregman_entropy_against_definition(scale):
    """S(u+e) - S(u) - w(u).e in 40-digit arithmetic vs the cancellation-free oracle form."""
    u = rand_states(8, 10)
    rng = np.random.default_rng(11)
    e = scale * rng.normal(size=u.shape) * np.abs(u)
    D = relax.bregman_entropy(u, e, G)
    for n in range(8):
        w = mp_w(u[:, n])
        ref = mp_S_at(u[:, n], e[:, n]) - mp_S(u[:, n]) - sum(w[i] * mp.mpf(float(e[i, n])) for i in range(5))
        assert float(ref) > 0
        assert abs(D[n] - float(ref)) <= 1e-13 * float(ref)


@pytest.mark.parametrize("scale", [1e-9, 1e-5, 1e-2])
def test_entropy_variable_difference_against_definition(scale):
    u = rand_states(6, 12)
    rng = np.random.default_rng(13)
    e = scale * rng.normal(size=u.shape) * np.abs(u)
    dw = relax.entropy_variables_difference(u, e, G)
    for n in range(6):
        w0 = mp_w(u[:, n])
        w1 = mp_w(u[:, n] + e[:, n])
        for i in range(5):
            ref = float(w1[i] - w0[i])
            # mp_w at u + e uses the rounded sum; compare within the rounding of that sum
            # mp_w(u + e) sees the fp64-rounded sum u + e; allow for that rounding
            tol = 1e-12 * abs(ref) + 1e-14 * float(abs(w0[i]))
            assert abs(dw[i, n] - ref) <= tol


def test_hessian_form_against_second_derivative():
    u = rand_states(5, 14)
    rng = np.random.default_rng(15)
    d = rng.normal(size=u.shape) * 0.1
    H = relax.hessian_form(u, d, G)
    for n in range(5):
        f = lambda t, n=n: mp_S_at(u[:, n], d[:, n], t)
        ref = mp.diff(f, 0, 2)
        assert abs(H[n] - float(ref)) <= 1e-12 * abs(float(ref))


@pytest.mark.parametrize("m", [0, 1, 2])
def test_viscous_jacobian_against_definition(m):
    """C_mm g against the viscous flux of its definition: the velocity and temperature
    derivatives along x_m that the w-gradient g implies (v = -w_{2..4}/w_5 and
    T = -1/(R w_5), differentiated in 40 digits), Stokes' stress and Fourier's law.
    C_mm is symmetric positive semidefinite and has no first row or column."""
    mu, Pr, R = 0.03, 0.72, 1.3
    qs = rand_states(6, 20 + m)
    rng = np.random.default_rng(30 + m)
    gs = rng.normal(size=(5, 6))
    C = gas.viscous_jacobian(qs, G, mu, Pr, R, m)
    assert C.shape == (5, 5, 6)
    scale = np.max(np.abs(C))
    assert np.max(np.abs(C - np.swapaxes(C, 0, 1))) <= 1e-15 * scale
    assert np.max(np.abs(C[0])) == 0.0 and np.max(np.abs(C[:, 0])) == 0.0
    kappa = mu * G * R / ((G - 1) * Pr)
    for i in range(6):
        assert np.min(np.linalg.eigvalsh(C[:, :, i])) >= -1e-14 * scale
        rho, m1, m2, m3, E = [mp.mpf(float(a)) for a in qs[:, i]]
        p = (mp.mpf(G) - 1) * (E - (m1 * m1 + m2 * m2 + m3 * m3) / (2 * rho))
        w = [m1 / p, m2 / p, m3 / p, -rho / p]              # rho v/p and -rho/p
        g = [mp.mpf(float(a)) for a in gs[1:, i]]

        def vel(eps, k):
            return -(w[k] + eps * g[k]) / (w[3] + eps * g[3])

        def temp(eps):
            return -1 / (mp.mpf(R) * (w[3] + eps * g[3]))
        dv = [mp.diff(lambda e, k=k: vel(e, k), 0) for k in range(3)]
        dT = mp.diff(temp, 0)
        v = [m1 / rho, m2 / rho, m3 / rho]
        tau = [mu * (dv[k] + (dv[m] if k == m else 0) - (mp.mpf(2) / 3 * dv[m] if k == m else 0))
               for k in range(3)]
        f = [0, tau[0], tau[1], tau[2], sum(tau[k] * v[k] for k in range(3)) + kappa * dT]
        got = C[:, :, i] @ gs[:, i]
        ref = np.array([float(a) for a in f])
        assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref)), (i, got, ref)
