"""Finite-field stencils of Eqs. 19-20.  TEST INFRASTRUCTURE ONLY.

``mu1 = (8[mu(A) - mu(-A)] - [mu(2A) - mu(-2A)]) / (12 A)``
``mu2 = (16[mu(A) + mu(-A)] - [mu(2A) + mu(-2A)] - 30 mu(0)) / (24 A^2)``
"""
import numpy as np


def first_order(mu_p1, mu_m1, mu_p2, mu_m2, A):
    return (8.0 * (np.asarray(mu_p1) - mu_m1) - (np.asarray(mu_p2) - mu_m2)) / (12.0 * A)


def second_order(mu_0, mu_p1, mu_m1, mu_p2, mu_m2, A):
    return (16.0 * (np.asarray(mu_p1) + mu_m1) - (np.asarray(mu_p2) + mu_m2)
            - 30.0 * np.asarray(mu_0)) / (24.0 * A * A)
