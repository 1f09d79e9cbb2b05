"""Host post-processing of the property layer (no GPU): finite-field stencils,
cosine fits, the static-field polynomial and the absorption spectrum, each
against inputs whose answer is known in closed form."""
import numpy as np

from paper_2407_18947_gb300 import properties as P


def test_stencils_exact_on_quintic():
    c = np.array([0.3, -1.7, 2.5, 0.9, -4.0, 1.3])
    mu = lambda F: sum(ck * F ** k for k, ck in enumerate(c))  # noqa: E731
    A = 0.01
    m1 = P.stencil_first(mu(A), mu(-A), mu(2 * A), mu(-2 * A), A)
    m2 = P.stencil_second(mu(0.0), mu(A), mu(-A), mu(2 * A), mu(-2 * A), A)
    # the first-order stencil cancels F^2 and F^3 errors (exact to degree 4)
    assert abs(m1 - (c[1] - 4.0 * c[5] * A ** 4)) < 1e-12
    assert abs(m2 - c[2]) < 1e-9


def test_cosine_fits_recover_alpha_and_beta():
    w = 0.0656
    t = np.linspace(0.0, 3 * 2 * np.pi / w, 4001)
    alpha, bshg, bor = 9.87, -21.5, 3.25
    a, r2 = P.fit_polarizability(t, alpha * np.cos(w * t), w, t_start=t[-1] / 3)
    assert abs(a - alpha) < 1e-10 and r2 > 1 - 1e-12
    mu2 = 0.25 * (bshg * np.cos(2 * w * t) + bor)
    b1, b2, r2 = P.fit_hyperpolarizability(t, mu2, w, t_start=t[-1] / 3)
    assert abs(b1 - bshg) < 1e-10 and abs(b2 - bor) < 1e-10 and r2 > 1 - 1e-12
    g, r2 = P.fit_gprime(t, 0.7 * np.sin(w * t), w)
    assert abs(g - 0.7) < 1e-12


def test_fit_r2_flags_a_wrong_frequency():
    w = 0.0656
    t = np.linspace(0.0, 4 * 2 * np.pi / w, 2001)
    _, r2 = P.fit_polarizability(t, np.cos(1.3 * w * t), w)
    assert r2 < 0.5


def test_static_polynomial():
    F = np.array([0.0, 0.001, -0.001, 0.002, -0.002, 0.004, -0.004])
    mu = 0.1 + 5.0 * F + 0.5 * 30.0 * F ** 2 + 7.0 * F ** 3 + 11.0 * F ** 4
    alpha, beta, _ = P.static_polynomial(F, mu)
    assert abs(alpha - 5.0) < 1e-7 and abs(beta - 30.0) < 1e-4


def test_absorption_spectrum_peak_of_a_damped_oscillator():
    # linear response chi(t) = f sin(w0 t) exp(-g t) to a narrow Gaussian pulse
    w0, g, f = 0.8, 0.01, 0.5
    dt = 0.05
    t = np.arange(0.0, 600.0, dt)
    E = 1e-3 * np.exp(-(t - 2.0) ** 2 / (2 * 0.2 ** 2))
    chi = f * np.sin(w0 * t) * np.exp(-g * t)
    mu = np.convolve(E, chi)[: t.size] * dt
    w, I = P.absorption_spectrum(t, [mu, mu, mu], [E, E, E], omega_max=2.0)
    assert abs(w[np.argmax(I)] - w0) < 2 * (w[1] - w[0])
    assert I.max() > 0
