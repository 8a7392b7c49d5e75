"""Semidiscretisation of Eq. (compressible_ns_diss) on a periodic Cartesian mesh.

Section 3.1: on element kappa

    dq_k/dt + sum_m 2 D^I_{x_m} o F_{x_m}(q_k, q_k) 1
        = sum_{m,j} D^V_{x_m} [C_mj] theta_j + SAT^I + SAT^V + diss^I + diss^V

with diagonal-norm SBP operators on LGL nodes.  The paper defers the SAT,
dissipation and viscous details to its references; the readings taken here:

* Volume term: 2 D o F 1 with F_ij = f*_m(q_i, q_j), the Ismail--Roe flux;
  the diagonal uses f*(q, q) = f(q) through the same flux formula.
* SAT^I + diss^I: at a face node with outward normal n = +-e_m,
  -(2/h_m)(1/omega_face) [f_num(q-, q+) - f_m(q)] . n with f_num the
  entropy-conservative flux minus diss * Rusanov dissipation.
* Viscous terms: BR1 in entropy variables.  theta_m = (2/h_m)[D w + lifting
  toward the face average of w], viscous flux F^V_m(q, theta), divergence
  (2/h_m)[D F^V_m + lifting toward the face average of F^V_m].
* diss^V (its construction is deferred to the references; off unless
  Physics.visc_diss = alpha > 0): an interior penalty on the jump of the entropy
  variables, g = sigma_m Chat (w - w+) added to the interface flux like diss^I,
  Chat = (C_mm(q) + C_mm(q+))/2, sigma_m = alpha (2/h_m)/omega_0.  Chat is symmetric
  positive semidefinite, so each face removes sigma [[w]]^T Chat [[w]] >= 0 of entropy
  and the two sides' terms cancel in the conservation sums.
* Mesh: n_x x n_y x n_z elements of size h_x x h_y x h_z, periodic in every
  direction unless a Dirichlet-penalty boundary is given for it; metric 2/h_m per
  direction, Jacobian h_x h_y h_z / 8.
* Dirichlet-penalty boundaries (Section 4.1.2 penalises the solution against the
  analytic one; the form is not printed).  Reading: at a boundary face the exterior
  state is the prescribed state q_b(t); the inviscid SAT uses the interface flux
  f_num(q, q_b) (left boundary: f_num(q_b, q)); the BR1 gradient lifts toward
  (w + w(q_b))/2; the viscous boundary flux is the interior one (no viscous penalty).

Array layout: U has shape (5, nz, ny, nx, P1, P1, P1) with node axes (k, j, i)
running in (z, y, x).  Flattened in C order this is the SoA layout
[var][element][node] with element = ex + nx (ey + ny ez) and
node = i + P1 (j + P1 k).
"""
import numpy as np

from . import gas, sbp

# (element axis, node axis) of U for the directions x, y, z
_AXES = {0: (3, 6), 1: (2, 5), 2: (1, 4)}


class Physics:
    def __init__(self, gamma=1.4, mu=0.0, Pr=0.72, R=1.0, diss=0, visc_diss=0.0):
        self.gamma = float(gamma)
        self.mu = float(mu)
        self.Pr = float(Pr)
        self.R = float(R)
        self.diss = diss
        self.visc_diss = float(visc_diss)


class Mesh:
    def __init__(self, p, n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), bc=None):
        """bc: {direction m: (left(t), right(t))} prescribed exterior states (5,) at the
        faces x_m = lo_m and x_m = hi_m; directions not listed are periodic."""
        self.bc = dict(bc or {})
        self.p = int(p)
        self.P1 = self.p + 1
        self.n = tuple(int(a) for a in n)             # (nx, ny, nz)
        self.lo = np.asarray(lo, dtype=np.float64)
        self.hi = np.asarray(hi, dtype=np.float64)
        self.h = (self.hi - self.lo) / np.asarray(self.n, dtype=np.float64)
        self.xi, self.omega, self.D = sbp.sbp_operator(self.p)
        self.K = self.n[0] * self.n[1] * self.n[2]
        self.Np = self.P1 ** 3

    @property
    def shape(self):
        nx, ny, nz = self.n
        P1 = self.P1
        return (5, nz, ny, nx, P1, P1, P1)

    def coords(self):
        """Node coordinates x, y, z, each of shape (nz, ny, nx, P1, P1, P1)."""
        nx, ny, nz = self.n
        P1 = self.P1
        out = []
        for m, (ne, nax) in enumerate([(nx, 5), (ny, 4), (nz, 3)]):
            e = np.arange(ne, dtype=np.float64)
            # physical coordinate of node a in element e along direction m
            x1 = self.lo[m] + self.h[m] * (e[:, None] + 0.5 * (1.0 + self.xi[None, :]))
            shape = [1] * 6
            shape[2 - m] = ne
            shape[nax] = P1
            out.append(np.broadcast_to(x1.reshape(shape), (nz, ny, nx, P1, P1, P1)).copy())
        return out

    def mass(self):
        """Diagonal of P-hat: J omega_i omega_j omega_k, shape (P1, P1, P1) as (k, j, i)."""
        J = np.prod(self.h) / 8.0
        w = self.omega
        return J * w[:, None, None] * w[None, :, None] * w[None, None, :]

    def element_sum(self, nodal):
        """sum_n P_n nodal_n for each element: (..., nz, ny, nx, P1, P1, P1) -> (..., nz, ny, nx)."""
        return np.sum(nodal * self.mass(), axis=(-3, -2, -1))

    def flat(self, U):
        return np.ascontiguousarray(U).reshape(5, self.K, self.Np)

    def unflat(self, q):
        return np.asarray(q, dtype=np.float64).reshape(self.shape)


def _next_trace(mesh, A_left, m, eax, t, fn=None):
    """Trace of the +x_m neighbour at each element's +x_m face: its -x_m face values,
    or the prescribed right boundary state (through fn) on the last element."""
    out = np.roll(A_left, -1, axis=eax)
    if m in mesh.bc:
        qb = np.asarray(mesh.bc[m][1](t), dtype=np.float64)
        val = qb if fn is None else fn(qb)
        idx = [slice(None)] * out.ndim
        idx[eax] = -1
        out[tuple(idx)] = np.asarray(val).reshape((-1,) + (1,) * (out.ndim - 2))
    return out


def _prev_trace(mesh, A_right, m, eax, t, fn=None):
    """Trace of the -x_m neighbour at each element's -x_m face (left boundary state
    on the first element)."""
    out = np.roll(A_right, 1, axis=eax)
    if m in mesh.bc:
        qb = np.asarray(mesh.bc[m][0](t), dtype=np.float64)
        val = qb if fn is None else fn(qb)
        idx = [slice(None)] * out.ndim
        idx[eax] = 0
        out[tuple(idx)] = np.asarray(val).reshape((-1,) + (1,) * (out.ndim - 2))
    return out


def _apply_D(D, A, axis):
    """(D A) along one node axis."""
    A = np.moveaxis(A, axis, -1)
    out = np.einsum("ij,...j->...i", D, A)
    return np.moveaxis(out, -1, axis)


def _face(A, index, axis):
    return np.take(A, index, axis=axis)


def _add_face(A, index, axis, val):
    idx = [slice(None)] * A.ndim
    idx[axis] = index
    A[tuple(idx)] += val


def volume_term(mesh, U, phys):
    """-sum_m (2/h_m) 2 D_m o F_m(q, q) 1 for every node."""
    g = phys.gamma
    out = np.zeros_like(U)
    for m in range(3):
        _, nax = _AXES[m]
        A = np.moveaxis(U, nax, -1)
        F = gas.ec_flux(A[..., :, None], A[..., None, :], g, m)   # F[..., i, j]
        vol = np.einsum("ij,...ij->...i", 2.0 * mesh.D, F)
        out -= (2.0 / mesh.h[m]) * np.moveaxis(vol, -1, nax)
    return out


def _boundary_fluxes(mesh, U, phys, m, t):
    """Interface fluxes on the +x_m and -x_m faces of every element (Dirichlet-penalty
    exterior states on boundary faces)."""
    g = phys.gamma
    eax, nax = _AXES[m]
    q_right = _face(U, mesh.p, nax)                   # this element, face +x_m
    q_left = _face(U, 0, nax)                         # this element, face -x_m
    q_next = _next_trace(mesh, q_left, m, eax, t)     # +x_m neighbour's -x_m face
    f_right = gas.interface_flux(q_right, q_next, g, m, phys.diss)
    f_left = np.roll(f_right, 1, axis=eax)            # flux on this element's -x_m face
    if m in mesh.bc:
        q_prev = _prev_trace(mesh, q_right, m, eax, t)
        fb = gas.interface_flux(q_prev, q_left, g, m, phys.diss)
        idx = [slice(None)] * f_left.ndim
        idx[eax] = 0
        f_left[tuple(idx)] = fb[tuple(idx)]
    return q_right, q_left, f_right, f_left


def inviscid_surface_term(mesh, U, phys, t=0.0):
    """SAT^I + diss^I on all six faces of every element."""
    g = phys.gamma
    p = mesh.p
    out = np.zeros_like(U)
    for m in range(3):
        eax, nax = _AXES[m]
        q_right, q_left, f_right, f_left = _boundary_fluxes(mesh, U, phys, m, t)
        s = 2.0 / mesh.h[m]
        _add_face(out, p, nax, -s / mesh.omega[p] * (f_right - gas.euler_flux(q_right, g, m)))
        _add_face(out, 0, nax, s / mesh.omega[0] * (f_left - gas.euler_flux(q_left, g, m)))
    return out


def entropy_gradients(mesh, U, phys, t=0.0):
    """BR1 theta_m = dw/dx_m, m = 0, 1, 2 (shape (3, 5, ...))."""
    W = gas.entropy_variables(U, phys.gamma)
    p = mesh.p
    theta = np.zeros((3,) + U.shape)

    def wfun(q):
        return gas.entropy_variables(q, phys.gamma)
    for m in range(3):
        eax, nax = _AXES[m]
        dw = _apply_D(mesh.D, W, nax)
        w_right = _face(W, p, nax)
        w_left = _face(W, 0, nax)
        w_next = _next_trace(mesh, w_left, m, eax, t, wfun)
        w_prev = _prev_trace(mesh, w_right, m, eax, t, wfun)
        _add_face(dw, p, nax, (0.5 * (w_right + w_next) - w_right) / mesh.omega[p])
        _add_face(dw, 0, nax, -(0.5 * (w_prev + w_left) - w_left) / mesh.omega[0])
        theta[m] = (2.0 / mesh.h[m]) * dw
    return theta


def viscous_term(mesh, U, phys, return_parts=False, t=0.0):
    """BR1 divergence of the viscous fluxes, with central interface SAT^V (the interior
    flux on boundary faces)."""
    p = mesh.p
    theta = entropy_gradients(mesh, U, phys, t)
    fv = gas.viscous_flux(U, theta, phys.gamma, phys.mu, phys.Pr, phys.R)
    out = np.zeros_like(U)
    for m in range(3):
        eax, nax = _AXES[m]
        F = fv[m]
        dF = _apply_D(mesh.D, F, nax)
        f_right = _face(F, p, nax)
        f_left = _face(F, 0, nax)
        f_next = np.roll(f_left, -1, axis=eax)
        f_prev = np.roll(f_right, 1, axis=eax)
        if m in mesh.bc:
            last = [slice(None)] * f_next.ndim
            last[eax] = -1
            first = [slice(None)] * f_prev.ndim
            first[eax] = 0
            f_next[tuple(last)] = f_right[tuple(last)]
            f_prev[tuple(first)] = f_left[tuple(first)]
        _add_face(dF, p, nax, (0.5 * (f_right + f_next) - f_right) / mesh.omega[p])
        _add_face(dF, 0, nax, -(0.5 * (f_prev + f_left) - f_left) / mesh.omega[0])
        out += (2.0 / mesh.h[m]) * dF
    if return_parts:
        return out, theta, fv
    return out


def _penalty_fluxes(mesh, U, phys, m, t):
    """diss^V penalty fluxes sigma_m Chat (w_minus - w_plus) on the +x_m and -x_m faces of
    every element, oriented along +x_m (exterior states on boundary faces)."""
    g = phys.gamma
    p = mesh.p
    eax, nax = _AXES[m]
    sig = phys.visc_diss * (2.0 / mesh.h[m]) / mesh.omega[p]

    def flux(qa, qb):
        C = 0.5 * (gas.viscous_jacobian(qa, g, phys.mu, phys.Pr, phys.R, m)
                   + gas.viscous_jacobian(qb, g, phys.mu, phys.Pr, phys.R, m))
        jump = gas.entropy_variables(qa, g) - gas.entropy_variables(qb, g)
        return sig * np.einsum("ij...,j...->i...", C, jump)
    q_right = _face(U, p, nax)
    q_left = _face(U, 0, nax)
    g_right = flux(q_right, _next_trace(mesh, q_left, m, eax, t))
    g_left = np.roll(g_right, 1, axis=eax)
    if m in mesh.bc:
        gb = flux(_prev_trace(mesh, q_right, m, eax, t), q_left)
        idx = [slice(None)] * g_left.ndim
        idx[eax] = 0
        g_left[tuple(idx)] = gb[tuple(idx)]
    return g_right, g_left


def viscous_interface_dissipation(mesh, U, phys, t=0.0):
    """diss^V at the faces of every element: -(2/h_m)(1/omega) g on the +x_m face,
    +(2/h_m)(1/omega) g on the -x_m face, with g the penalty flux through that face."""
    p = mesh.p
    out = np.zeros_like(U)
    for m in range(3):
        _, nax = _AXES[m]
        s = 2.0 / mesh.h[m]
        g_right, g_left = _penalty_fluxes(mesh, U, phys, m, t)
        _add_face(out, p, nax, -s / mesh.omega[p] * g_right)
        _add_face(out, 0, nax, s / mesh.omega[0] * g_left)
    return out


def rhs(mesh, U, phys, t=0.0):
    """f(u) of Eq. (ode): the right-hand side dq/dt of Eq. (compressible_ns_diss) at time
    t (t only enters through prescribed boundary states)."""
    out = volume_term(mesh, U, phys) + inviscid_surface_term(mesh, U, phys, t)
    if phys.mu != 0.0:
        out = out + viscous_term(mesh, U, phys, t=t)
        if phys.visc_diss > 0.0:
            out = out + viscous_interface_dissipation(mesh, U, phys, t)
    return out


def rhs_term_magnitude(mesh, U, phys, t=0.0):
    """Sum of the absolute values of the terms that rhs() adds at every node.

    Test infrastructure: the rounding error of any FP64 evaluation of the
    right-hand side is a small multiple of eps times this magnitude, which can
    exceed |rhs| by orders of magnitude where the fluxes nearly cancel (low Mach
    number: the pressure part of the momentum flux).
    """
    g = phys.gamma
    p = mesh.p
    T = np.zeros_like(U)
    for m in range(3):
        eax, nax = _AXES[m]
        s = 2.0 / mesh.h[m]
        A = np.moveaxis(U, nax, -1)
        F = gas.ec_flux(A[..., :, None], A[..., None, :], g, m)
        T += s * np.moveaxis(np.einsum("ij,...ij->...i", np.abs(2.0 * mesh.D), np.abs(F)), -1, nax)
        q_right, q_left, f_right, f_left = _boundary_fluxes(mesh, U, phys, m, t)
        _add_face(T, p, nax, s / mesh.omega[p] * (np.abs(f_right) + np.abs(gas.euler_flux(q_right, g, m))))
        _add_face(T, 0, nax, s / mesh.omega[0] * (np.abs(f_left) + np.abs(gas.euler_flux(q_left, g, m))))
    if phys.mu != 0.0:
        _, theta, fv = viscous_term(mesh, U, phys, return_parts=True, t=t)
        for m in range(3):
            eax, nax = _AXES[m]
            T += (2.0 / mesh.h[m]) * _apply_D(np.abs(mesh.D), np.abs(fv[m]), nax)
            if phys.visc_diss > 0.0:
                s = 2.0 / mesh.h[m]
                g_right, g_left = _penalty_fluxes(mesh, U, phys, m, t)
                _add_face(T, p, nax, s / mesh.omega[p] * np.abs(g_right))
                _add_face(T, 0, nax, s / mesh.omega[0] * np.abs(g_left))
    return T


def local_entropies(mesh, U, phys):
    """eta_kappa(u) = 1^T P S_kappa (Section 3.2)."""
    return mesh.element_sum(gas.entropy(U, phys.gamma))


def entropy_rate(mesh, U, dU, phys):
    """(eta_kappa' f)(u) = sum_n P_n w(u_n) . f(u)_n for every element."""
    W = gas.entropy_variables(U, phys.gamma)
    return mesh.element_sum(np.sum(W * dU, axis=0))


def element_block(U, centre, radius):
    """Periodic block of (2 radius + 1)^3 elements centred on element (ex, ey, ez).

    The right-hand side on the centre element of the block, taken as its own
    periodic mesh, equals the right-hand side of that element on the full mesh
    whenever radius covers the stencil (1 for Euler, 2 for BR1 viscous terms).
    """
    ex, ey, ez = centre
    r = np.arange(-radius, radius + 1)
    nz, ny, nx = U.shape[1:4]
    B = U[:, ((ez + r) % nz)[:, None, None], ((ey + r) % ny)[None, :, None],
          ((ex + r) % nx)[None, None, :]]
    return B
