"""Legendre--Gauss--Lobatto nodes, weights and the SBP derivative matrix.

Section 3.1 (text after Eq. (compressible_ns_diss)): the scheme uses
diagonal-norm SBP operators on the LGL nodes, i.e. a collocated discontinuous
spectral element method.  The paper prints no formulas for these operators; the
textbook definitions are used:

* nodes   xi_0 = -1 < xi_1 < ... < xi_p = 1, the interior ones the roots of P_p',
* weights omega_i = 2 / (p (p+1) P_p(xi_i)^2),
* D_ij    = P_p(xi_i) / (P_p(xi_j) (xi_i - xi_j))  (i != j),
  D_00 = -p(p+1)/4, D_pp = p(p+1)/4, other diagonal entries 0,

so that P = diag(omega), Q = P D and Q + Q^T = B = diag(-1, 0, ..., 0, 1).
"""
import numpy as np


def legendre(p, x):
    """P_p(x) and P_p'(x) by the three-term recurrence (fp64)."""
    x = np.asarray(x, dtype=np.float64)
    p0 = np.ones_like(x)
    if p == 0:
        return p0, np.zeros_like(x)
    p1 = x.copy()
    for n in range(1, p):
        p0, p1 = p1, ((2 * n + 1) * x * p1 - n * p0) / (n + 1)
    # derivative from (1 - x^2) P_p' = p (P_{p-1} - x P_p), valid off x = +-1
    with np.errstate(divide="ignore", invalid="ignore"):
        dp = p * (p0 - x * p1) / (1.0 - x * x)
    end = np.abs(np.abs(x) - 1.0) == 0.0
    dp = np.where(end, np.sign(x) ** (p + 1) * p * (p + 1) / 2.0, dp)
    return p1, dp


def lgl_nodes(p):
    """LGL nodes: +-1 and the p-1 roots of P_p' (Newton from Chebyshev points)."""
    if p < 1:
        raise ValueError("p >= 1 required")
    x = -np.cos(np.pi * np.arange(p + 1) / p)
    for _ in range(100):
        # Newton on (1 - x^2) P_p'(x) = p (P_{p-1}(x) - x P_p(x)) for interior nodes
        pp, _ = legendre(p, x)
        pm, _ = legendre(p - 1, x)
        g = p * (pm - x * pp)
        # g'(x) = -p (p+1) P_p(x)   (Legendre ODE)
        dg = -p * (p + 1) * pp
        step = np.zeros_like(x)
        step[1:-1] = g[1:-1] / dg[1:-1]
        x = x - step
        if np.max(np.abs(step)) < 1e-16:
            break
    x[0], x[-1] = -1.0, 1.0
    # enforce the exact symmetry of the node set
    x = 0.5 * (x - x[::-1])
    return x


def lgl_weights(p, x=None):
    if x is None:
        x = lgl_nodes(p)
    pp, _ = legendre(p, x)
    return 2.0 / (p * (p + 1) * pp * pp)


def lgl_diff_matrix(p, x=None):
    if x is None:
        x = lgl_nodes(p)
    pp, _ = legendre(p, x)
    n = p + 1
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = pp[i] / (pp[j] * (x[i] - x[j]))
    D[0, 0] = -p * (p + 1) / 4.0
    D[p, p] = p * (p + 1) / 4.0
    return D


def sbp_operator(p):
    """(xi, omega, D) for degree p."""
    x = lgl_nodes(p)
    return x, lgl_weights(p, x), lgl_diff_matrix(p, x)
