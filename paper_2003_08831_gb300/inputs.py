"""Seeded synthetic inputs: closed-form initial states and counter-based noise.

This module only evaluates workload definitions at given points; it holds none
of the scheme's arithmetic (no fluxes, no SBP operators, no entropy).  Both the
CUDA path and the CPU oracle receive states built here.

* Isentropic vortex, Eq. (vortex-solution) of Section 4.1.1.  Readings:
  U_inf = 1, rho_inf = T_inf = 1, c_inf = 1/M_inf, p = rho T/(gamma M_inf^2)
  (then the formula is an exact Euler solution), and the sign of the
  x_1-term of U_2 is +, the rotational vortex (the printed - sign gives a
  strain field that is not a solution).  The vortex is two-dimensional,
  extruded in x_3 (U_3 = 0).
* Taylor--Green vortex (not in the paper; the standard Euler/Navier--Stokes
  benchmark): V_0 = L = rho_0 = 1, u = sin x cos y cos z, v = -cos x sin y cos z,
  w = 0, p = p_0 + (cos 2x + cos 2y)(cos 2z + 2)/16, p_0 = 1/(gamma M^2),
  rho = p/p_0 (isothermal start).
* Viscous shock, Section 4.1.2 (Pr = 3/4, where the total enthalpy is constant
  across the shock and the momentum and energy equations reduce to one ODE for
  V = u/u_L).  Readings: the shock-frame upstream state (x -> -inf) is rho = u = 1,
  p = 1/(gamma M^2); mu = 1/Re (unit length); V_f = u_R/u_L from the
  Rankine--Hugoniot relations, (2 + (gamma-1) M^2)/((gamma+1) M^2); the implicit
  solution is x = (alpha/2) [log|(V-1)(V-V_f)| + (1+V_f)/(1-V_f) log|(V-1)/(V-V_f)|]
  (the printed form lacks the bracket; differentiating this one gives the ODE
  alpha V V' = (V-1)(V-V_f)); the "uniform translation" moves the frame with the
  upstream gas at rest: lab velocity u - 1, shock at x = -t.
* Noise: SplitMix64 (Steele, Lea & Flood 2014) keyed by (seed, counter).
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

SEED = 20030831


def splitmix64(seed, counter):
    """SplitMix64 output for state = seed + (counter + 1) * golden gamma."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(counter, dtype=np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed, counter):
    """Uniform doubles in [0, 1) from the top 53 bits."""
    return (splitmix64(seed, counter) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def conserved(rho, vx, vy, vz, p, gamma):
    """Stack (rho, rho v, p/(gamma-1) + rho |v|^2/2) on a new axis 0."""
    return np.stack([rho, rho * vx, rho * vy, rho * vz,
                     p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz)])


def vortex_primitives(x, y, t=0.0, eps=5.0, mach=0.5, gamma=1.4, alpha=np.pi / 4, centre=(0.0, 0.0),
                      period=None):
    """(rho, u1, u2, u3, p) of the isentropic vortex at time t.

    With period = L the offsets from the (moving) centre are taken to the nearest
    periodic image (minimum-image convention), so a vortex placed anywhere in a
    periodic box of side L is continuous up to its tail at distance L/2."""
    uinf = 1.0
    dx = (x - centre[0]) - uinf * np.cos(alpha) * t
    dy = (y - centre[1]) - uinf * np.sin(alpha) * t
    if period is not None:
        dx = np.mod(dx + 0.5 * period, period) - 0.5 * period
        dy = np.mod(dy + 0.5 * period, period) - 0.5 * period
    G = 1.0 - (dx * dx + dy * dy)
    T = 1.0 - eps * eps * mach * mach * (gamma - 1.0) / (8.0 * np.pi ** 2) * np.exp(G)
    rho = T ** (1.0 / (gamma - 1.0))
    e = eps / (2.0 * np.pi) * np.exp(0.5 * G)
    u1 = uinf * np.cos(alpha) - e * dy
    u2 = uinf * np.sin(alpha) + e * dx
    p = rho * T / (gamma * mach * mach)
    return rho, u1, u2, np.zeros_like(rho), p


def vortex_state(x, y, t=0.0, eps=5.0, mach=0.5, gamma=1.4, alpha=np.pi / 4, centre=(0.0, 0.0), period=None):
    rho, u1, u2, u3, p = vortex_primitives(x, y, t, eps, mach, gamma, alpha, centre, period)
    return conserved(rho, u1, u2, u3, p, gamma)


def tgv_primitives(x, y, z, mach=0.1, gamma=1.4):
    p0 = 1.0 / (gamma * mach * mach)
    u = np.sin(x) * np.cos(y) * np.cos(z)
    v = -np.cos(x) * np.sin(y) * np.cos(z)
    w = np.zeros_like(u)
    p = p0 + (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0) / 16.0
    rho = p / p0
    return rho, u, v, w, p


def tgv_state(x, y, z, mach=0.1, gamma=1.4):
    return conserved(*tgv_primitives(x, y, z, mach, gamma), gamma)


def perturbed_tgv_state(x, y, z, mach=0.1, gamma=1.4, amp=1e-3, seed=SEED):
    """TGV with rho <- rho (1 + amp U[-1,1]) and v_k <- v_k + amp U[-1,1].

    x, y, z are flat arrays in the global node order [element][node]; node
    index n draws counters 4n (density) and 4n + 1..3 (velocity components).
    """
    rho, u, v, w, p = tgv_primitives(x, y, z, mach, gamma)
    n = np.arange(rho.size, dtype=np.uint64).reshape(rho.shape)
    r = [2.0 * uniform(seed, np.uint64(4) * n + np.uint64(c)) - 1.0 for c in range(4)]
    rho = rho * (1.0 + amp * r[0])
    return conserved(rho, u + amp * r[1], v + amp * r[2], w + amp * r[3], p, gamma)


def batch_instances(count=256, seed=SEED, nmin=4, nmax=12, pmin=2, pmax=5, box=10.0):
    """Per-instance parameters of the batched vortex workload.

    Each instance i draws, from counters 8 i + 0..5: n in {nmin..nmax} (n^3
    elements), p in {pmin..pmax}, vortex centre in [0, box]^2, strength in
    [3, 6] and background Mach number in [0.1, 0.5].  The instance's initial
    state is vortex_state(..., period=box): the centre can be anywhere.
    """
    out = []
    for i in range(count):
        u = [float(uniform(seed ^ 0x5A5A5A5A, 8 * i + c)) for c in range(6)]
        out.append({
            "n": nmin + int(u[0] * (nmax - nmin + 1)),
            "p": pmin + int(u[1] * (pmax - pmin + 1)),
            "centre": (box * u[2], box * u[3]),
            "eps": 3.0 + 3.0 * u[4],
            "mach": 0.1 + 0.4 * u[5],
            "box": box,
        })
    return out


def viscous_shock_parameters(mach=2.5, reynolds=10.0, prandtl=0.75, gamma=1.4):
    """Constants of the viscous-shock solution: upstream p, mu, V_f, alpha, total enthalpy."""
    p_up = 1.0 / (gamma * mach * mach)
    mu = 1.0 / reynolds
    v_f = (2.0 + (gamma - 1.0) * mach * mach) / ((gamma + 1.0) * mach * mach)
    alpha = 2.0 * gamma / (gamma + 1.0) * mu / prandtl          # mass flux rho u = 1
    enthalpy = gamma / (gamma - 1.0) * p_up + 0.5
    return {"p_up": p_up, "mu": mu, "v_f": v_f, "alpha": alpha, "H": enthalpy, "gamma": gamma,
            "mach": mach, "reynolds": reynolds, "prandtl": prandtl}


def viscous_shock_velocity(xi, prm):
    """V(xi) in (V_f, 1) from the implicit solution by bisection to the last bit."""
    xi = np.asarray(xi, dtype=np.float64)
    vf, alpha = prm["v_f"], prm["alpha"]
    c = (1.0 + vf) / (1.0 - vf)
    lo = np.full(xi.shape, vf)
    hi = np.ones(xi.shape)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        with np.errstate(divide="ignore"):
            x_mid = 0.5 * alpha * (np.log((1.0 - mid) * (mid - vf)) + c * np.log((1.0 - mid) / (mid - vf)))
        # x(V) decreases with V: x(mid) > xi means the root lies above mid
        above = x_mid > xi
        lo = np.where(above, mid, lo)
        hi = np.where(above, hi, mid)
    return 0.5 * (lo + hi)


def viscous_shock_primitives(x, t, prm, speed=-1.0):
    """(rho, u, v, w, p) of the viscous shock at lab position x and time t: the shock-frame
    profile at xi = x - speed t, lab velocity u_shock + speed."""
    v = viscous_shock_velocity(np.asarray(x, dtype=np.float64) - speed * t, prm)
    g = prm["gamma"]
    u = v                     # u_L = 1
    rho = 1.0 / u             # mass flux 1
    p = (g - 1.0) / g * rho * (prm["H"] - 0.5 * u * u)
    z = np.zeros_like(rho)
    return rho, u + speed, z, z.copy(), p


def viscous_shock_state(x, t, prm, speed=-1.0):
    rho, u, v, w, p = viscous_shock_primitives(x, t, prm, speed)
    return conserved(rho, u, v, w, p, prm["gamma"])
