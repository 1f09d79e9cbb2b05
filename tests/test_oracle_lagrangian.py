"""Pin the oracle's lambda side and density.

* Exact dynamics: for two electrons CC3 has no triples and CCSD is exact, so
  the RT-CC dipole (density D = dL/dw contracted with mu, lambda propagated by
  Eq. A13-A14, classical RK4) must follow the exact TDSE dipole to the RK4
  error.  This fixes the Lagrangian normalisation, the Euler-Lagrange
  convention and the field/time handling.
* Finite differences of the *brute-force* Lagrangian (second quantisation,
  Eq. A6 with t3 eliminated) reproduce the oracle's autograd lambda residuals
  and density with triples and a field on.
"""
import numpy as np
import pytest
import torch

from oracle import cc3
from paper_2407_18947_gb300.synth import random_amplitudes, random_probe

from _oracle_helpers import tiny


@pytest.mark.parametrize("field", [
    cc3.FieldSpec(cc3.FIELD_STATIC, 0.05, direction=(0.3, -0.5, 1.0)),
    cc3.FieldSpec(cc3.FIELD_COS, 0.08, omega=0.5, direction=(1.0, 0.2, -0.4)),
    cc3.FieldSpec(cc3.FIELD_GAUSS, 0.1, center=0.2, width=0.1, direction=(0.0, 1.0, 0.0)),
])
def test_rt_dipole_matches_exact_tdse_two_electrons(field):
    s, ham, bf = tiny(1, 4, seed=21)
    y0 = cc3.solve_ground_state(ham)
    h, nsteps = 0.01, 40
    _, dips, ens = cc3.propagate_rk4(ham, field, y0, h, nsteps)
    e0, psi0 = bf.exact_ground_state()
    times = np.arange(nsteps + 1) * h
    wt = lambda t: ham.field_operator(field.vector(t)).numpy()
    hint = 0.01 if field.kind == cc3.FIELD_STATIC else 2e-4
    psis = bf.propagate_exact(psi0, wt, times, h_int=hint)
    ex = np.array([[bf.expectation_one_body(p, s.dipole[x]) for x in range(3)] for p in psis])
    assert np.abs(ex - ex[0]).max() > 1e-4  # the field does something
    assert np.abs(dips - ex).max() < 2e-10
    assert np.abs(dips.imag).max() < 1e-12


def _fd(fun, h):
    """Central difference with one Richardson step."""
    d1 = (fun(h) - fun(-h)) / (2 * h)
    d2 = (fun(h / 2) - fun(-h / 2)) / h
    return (4 * d2 - d1) / 3


@pytest.mark.parametrize("ov,fld", [((2, 2), 0.0), ((2, 2), 0.2), ((3, 2), 0.1)])
def test_lambda_residual_equals_fd_of_bruteforce_lagrangian(ov, fld):
    o, v = ov
    s, ham, bf = tiny(o, v, seed=13)
    t1, t2, l1, l2 = random_amplitudes(o, v, seed=4, t1_scale=0.05, t2_scale=0.05,
                                       l1_scale=0.3, l2_scale=0.3)
    w = ham.field_operator([0.0, 0.5 * fld, fld]).numpy()
    res = cc3.evaluate(ham, t1, t2, l1, l2, w)
    d1 = random_probe(t1.shape, seed=101)
    d2 = random_probe(t2.shape, seed=102)
    d2 = 0.5 * (d2 + d2.transpose(1, 0, 3, 2))
    dw = random_probe(w.shape, seed=103).real
    dw = 0.5 * (dw + dw.T)
    L = lambda h: bf.lagrangian(t1 + h * d1, t2 + h * d2, l1, l2, w)
    fd = _fd(L, 1e-3)
    an = np.sum(res.r_l1.numpy() * d1) + 0.5 * np.sum(res.r_l2.numpy() * d2)
    assert abs(fd - an) < 1e-9 * max(1.0, abs(an))
    Lw = lambda h: bf.lagrangian(t1, t2, l1, l2, w + h * dw)
    fdw = _fd(Lw, 1e-3)
    anw = np.sum(res.density.numpy() * dw)
    assert abs(fdw - anw) < 1e-9 * max(1.0, abs(anw))
    # T residuals are the lambda-derivative of the same Lagrangian
    Ll = lambda h: bf.lagrangian(t1, t2, l1 + h * d1, l2 + h * d2, w)
    fdl = _fd(Ll, 1e-2)
    anl = np.sum(res.r_t1.numpy() * d1) + 0.5 * np.sum(res.r_t2.numpy() * d2)
    assert abs(fdl - anl) < 1e-10 * max(1.0, abs(anl))


def test_lambda_residual_pair_symmetric():
    s, ham, bf = tiny(3, 4, seed=5)
    t1, t2, l1, l2 = random_amplitudes(3, 4, seed=8)
    w = ham.field_operator([0.0, 0.0, 0.05]).numpy()
    res = cc3.evaluate(ham, t1, t2, l1, l2, w)
    for x in (res.r_t2, res.r_l2):
        x = x.numpy()
        assert np.abs(x - x.transpose(1, 0, 3, 2)).max() < 1e-15
