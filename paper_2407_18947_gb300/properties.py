"""Optical properties from real-time dipole trajectories (host post-processing).

The propagations themselves run on the GPU (``RTCC3.propagate_rk4`` with one
field slot per field strength); this module turns their dipole (or magnetic
moment) trajectories into properties, following Section 2.2 of the paper:

* finite-field stencils (Section 2.2.2): from runs at field amplitudes
  ``A, -A, 2A, -2A`` (and 0) the first- and second-order moments
  ``mu1 = (8[mu(A) - mu(-A)] - [mu(2A) - mu(-2A)]) / (12 A)`` and
  ``mu2 = (16[mu(A) + mu(-A)] - [mu(2A) + mu(-2A)] - 30 mu(0)) / (24 A^2)``;
* cosine fits (Section 2.2.2): ``mu1(t) = alpha cos(wt)`` gives the
  polarisability, ``mu2(t) = 1/4 [beta_SHG cos(2wt) + beta_OR]`` the
  second-harmonic-generation and optical-rectification first
  hyperpolarisabilities, each with its coefficient of determination R^2,
  over the part of the trajectory after the ramp;
* the magnetic analogue (Section 2.2.3): ``m1(t) = G' sin(wt)``;
* a least-squares polynomial in the static field strength over a set of
  static-field runs (``mu(F) = c0 + c1 F + c2 F^2 + ...``: alpha = c1,
  beta = 2 c2);
* the absorption spectrum of a delta-like pulse (Section 2.2.1):
  ``alpha_bb(w) = mu~_b(w) / E~_b(w)``, ``I(w) ~ Im sum_b alpha_bb(w)``.
"""
from __future__ import annotations

import numpy as np


def stencil_first(mu_p1, mu_m1, mu_p2, mu_m2, amplitude):
    """First-order moment from the runs at A, -A, 2A, -2A (five-point stencil)."""
    mu_p1, mu_m1, mu_p2, mu_m2 = (np.asarray(x) for x in (mu_p1, mu_m1, mu_p2, mu_m2))
    return (8.0 * (mu_p1 - mu_m1) - (mu_p2 - mu_m2)) / (12.0 * amplitude)


def stencil_second(mu_0, mu_p1, mu_m1, mu_p2, mu_m2, amplitude):
    """Second-order moment from the runs at 0, A, -A, 2A, -2A."""
    mu_0, mu_p1, mu_m1, mu_p2, mu_m2 = (np.asarray(x) for x in (mu_0, mu_p1, mu_m1, mu_p2, mu_m2))
    return (16.0 * (mu_p1 + mu_m1) - (mu_p2 + mu_m2) - 30.0 * mu_0) / (24.0 * amplitude ** 2)


def _lstsq(basis, y):
    """Least-squares coefficients of y on the columns of `basis`, and R^2."""
    y = np.asarray(y, dtype=np.float64)
    coef, *_ = np.linalg.lstsq(basis, y, rcond=None)
    resid = y - basis @ coef
    ss_tot = float(np.sum((y - y.mean()) ** 2))
    r2 = 1.0 - float(np.sum(resid ** 2)) / ss_tot if ss_tot > 0.0 else 1.0
    return coef, r2


def fit_polarizability(times, mu1, omega, t_start=0.0):
    """alpha(w) from mu1(t) = alpha cos(wt) on t >= t_start; returns (alpha, R^2)."""
    t = np.asarray(times, dtype=np.float64)
    sel = t >= t_start
    coef, r2 = _lstsq(np.cos(omega * t[sel])[:, None], np.asarray(mu1, dtype=np.float64)[sel])
    return float(coef[0]), r2


def fit_hyperpolarizability(times, mu2, omega, t_start=0.0):
    """(beta_SHG, beta_OR) from mu2(t) = 1/4 [beta_SHG cos(2wt) + beta_OR] on
    t >= t_start; returns (beta_SHG, beta_OR, R^2)."""
    t = np.asarray(times, dtype=np.float64)
    sel = t >= t_start
    basis = 0.25 * np.stack([np.cos(2.0 * omega * t[sel]), np.ones(int(sel.sum()))], axis=1)
    coef, r2 = _lstsq(basis, np.asarray(mu2, dtype=np.float64)[sel])
    return float(coef[0]), float(coef[1]), r2


def fit_gprime(times, m1, omega, t_start=0.0):
    """G'(w) from the first-order magnetic moment m1(t) = G' sin(wt); (G', R^2)."""
    t = np.asarray(times, dtype=np.float64)
    sel = t >= t_start
    coef, r2 = _lstsq(np.sin(omega * t[sel])[:, None], np.asarray(m1, dtype=np.float64)[sel])
    return float(coef[0]), r2


def static_polynomial(fields, mu, degree=4):
    """Least-squares polynomial mu(F) = sum_k c_k F^k over static-field runs;
    returns (alpha, beta, coefficients) with alpha = c1 and beta = 2 c2."""
    F = np.asarray(fields, dtype=np.float64)
    basis = np.stack([F ** k for k in range(degree + 1)], axis=1)
    coef, _ = _lstsq(basis, np.asarray(mu, dtype=np.float64))
    return float(coef[1]), 2.0 * float(coef[2]), coef


def absorption_spectrum(times, dipoles, fields, damping=0.0, omega_max=None):
    """Dipole strength function of delta-like pulses along x, y, z.

    times: (N,) equally spaced; dipoles: (3, N) the induced dipole along the
    field direction of each of three runs (field along x, y, z); fields: (3, N)
    the field strengths of those runs.  The Fourier transforms are taken as
    discrete sums (the constant 1/2pi cancels in the ratio), optionally with an
    exponential damping exp(-damping t) of the dipole.  Returns (omega,
    I(omega)) with I = Im sum_b mu~_b / E~_b for omega in (0, omega_max].
    """
    t = np.asarray(times, dtype=np.float64)
    dt = t[1] - t[0]
    n = t.size
    omega = 2.0 * np.pi * np.fft.rfftfreq(n, dt)
    keep = omega > 0.0
    if omega_max is not None:
        keep &= omega <= omega_max
    w = omega[keep]
    phase = np.exp(1j * np.outer(w, t)) * dt
    damp = np.exp(-damping * (t - t[0]))
    total = np.zeros(w.size, dtype=np.complex128)
    for b in range(3):
        mu = np.asarray(dipoles[b], dtype=np.float64)
        mu = (mu - mu[0]) * damp
        e = np.asarray(fields[b], dtype=np.float64)
        total += (phase @ mu) / (phase @ e)
    return w, total.imag
