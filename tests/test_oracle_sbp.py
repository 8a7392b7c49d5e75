"""Pins for oracle.sbp: textbook LGL closed forms and the SBP identities.

Section 3.1 uses diagonal-norm SBP operators on LGL nodes; the node/weight
closed forms are the textbook ones (e.g. Abramowitz & Stegun 25.4.32).
"""
import math

import numpy as np
import pytest

from oracle import sbp

CLOSED = {
    2: ([-1.0, 0.0, 1.0], [1 / 3, 4 / 3, 1 / 3]),
    3: ([-1.0, -math.sqrt(1 / 5), math.sqrt(1 / 5), 1.0], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
    4: ([-1.0, -math.sqrt(3 / 7), 0.0, math.sqrt(3 / 7), 1.0], [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
    5: ([-1.0, -math.sqrt(1 / 3 + 2 * math.sqrt(7) / 21), -math.sqrt(1 / 3 - 2 * math.sqrt(7) / 21),
         math.sqrt(1 / 3 - 2 * math.sqrt(7) / 21), math.sqrt(1 / 3 + 2 * math.sqrt(7) / 21), 1.0],
        [1 / 15, (14 - math.sqrt(7)) / 30, (14 + math.sqrt(7)) / 30,
         (14 + math.sqrt(7)) / 30, (14 - math.sqrt(7)) / 30, 1 / 15]),
}


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_closed_form_nodes_weights(p):
    x, w, _ = sbp.sbp_operator(p)
    xe, we = CLOSED[p]
    assert np.max(np.abs(x - np.array(xe))) < 4e-16
    assert np.max(np.abs(w - np.array(we))) < 4e-16


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7])
def test_quadrature_degree(p):
    x, w, _ = sbp.sbp_operator(p)
    assert abs(np.sum(w) - 2.0) < 1e-15
    for k in range(2 * p):            # exact up to degree 2p - 1
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 2e-15
    # and not exact at degree 2p (Lobatto rule)
    assert abs(np.dot(w, x ** (2 * p)) - 2.0 / (2 * p + 1)) > 1e-6


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7])
def test_sbp_property_and_exactness(p):
    x, w, D = sbp.sbp_operator(p)
    Q = np.diag(w) @ D
    B = np.zeros_like(Q)
    B[0, 0], B[-1, -1] = -1.0, 1.0
    assert np.max(np.abs(Q + Q.T - B)) < 1e-14
    assert np.max(np.abs(D @ np.ones(p + 1))) < 1e-13
    for k in range(1, p + 1):
        assert np.max(np.abs(D @ x ** k - k * x ** (k - 1))) < 1e-12 * k * p * p
