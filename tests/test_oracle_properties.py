"""Structural properties of the oracle that the paper fixes.

* ``W_ijk^abc = W_jik^bac`` and the other simultaneous pair permutations
  (Eq. A30 makes W invariant under them).
* dressed integrals keep only ``<pq|rs>~ = <qp|sr>~`` (Section 4.1).
* a converged zero-field CC3 ground state is stationary: zero residuals and a
  constant dipole / energy under RK4 (the right-hand sides of Eqs. 2-3 are
  the ground-state residuals).
* classical RK4 is fourth order: halving h cuts the error ~16x.
* the finite-field stencils of Eqs. 19-20 are exact for quartic mu(A).
* the weak static-field limit: mu(F) from the density equals -dE/dF of the
  converged field-dependent ground state (Hellmann-Feynman for the CC3
  Lagrangian).
"""
import numpy as np
import pytest
import torch

from oracle import cc3, finite_field
from paper_2407_18947_gb300.synth import make_system, random_amplitudes

from _oracle_helpers import tiny


def test_W_permutational_symmetry():
    s = make_system(3, 4, seed=2)
    ham = cc3.Hamiltonian.from_system(s)
    t1, t2, _, _ = random_amplitudes(3, 4, seed=1)
    gt, ft, wt, ht = cc3.dress(ham, cc3._ct(t1), torch.zeros(ham.n, ham.n, dtype=cc3.CD))
    W = cc3.triples_W(ham, gt, cc3._ct(t2))
    scale = float(W.abs().max())
    for perm in ['jikbac', 'ikjacb', 'kjicba', 'kijcab', 'jkibca']:
        Wp = torch.einsum(perm + '->ijkabc', W)
        assert float((Wp - W).abs().max()) < 1e-14 * scale


def test_dressed_integral_symmetry():
    s = make_system(3, 4, seed=2)
    ham = cc3.Hamiltonian.from_system(s)
    t1, _, _, _ = random_amplitudes(3, 4, seed=1, t1_scale=0.1)
    gt, _, _, _ = cc3.dress(ham, cc3._ct(t1), torch.zeros(ham.n, ham.n, dtype=cc3.CD))
    phys = torch.einsum('prqs->pqrs', gt)  # <pq|rs>~ = (pr|qs)~
    assert float((phys - torch.einsum('qpsr->pqrs', phys)).abs().max()) < 1e-15
    # the untransformed eightfold symmetry is broken, e.g. <pq|rs> != <rq|ps>
    assert float((phys - torch.einsum('rqps->pqrs', phys)).abs().max()) > 1e-4


@pytest.fixture(scope="module")
def ground():
    s = make_system(2, 5, seed=17)
    ham = cc3.Hamiltonian.from_system(s)
    return ham, cc3.solve_ground_state(ham)


def test_ground_state_is_stationary(ground):
    ham, y0 = ground
    w = torch.zeros(ham.n, ham.n, dtype=cc3.CD)
    res = cc3.evaluate(ham, *y0, w)
    for r in (res.r_t1, res.r_t2, res.r_l1, res.r_l2):
        assert float(r.abs().max()) < 1e-11
    none = cc3.FieldSpec(cc3.FIELD_NONE)
    _, dips, ens = cc3.propagate_rk4(ham, none, y0, 0.01, 10)
    assert np.abs(dips - dips[0]).max() < 1e-12
    assert np.abs(ens - ens[0]).max() < 1e-12


def test_rk4_fourth_order(ground):
    ham, y0 = ground
    field = cc3.FieldSpec(cc3.FIELD_COS, 0.05, omega=0.3, direction=(0.0, 0.0, 1.0))
    T = 0.4
    ref = cc3.propagate_rk4(ham, field, y0, T / 32, 32)[1][-1]
    errs = []
    for nst in (4, 8):
        d = cc3.propagate_rk4(ham, field, y0, T / nst, nst)[1][-1]
        errs.append(np.abs(d - ref).max())
    ratio = errs[0] / errs[1]
    assert 12.0 < ratio < 20.0, ratio


def test_stencils_exact_on_quartic():
    A = 0.002
    c = np.array([0.3, -1.7, 4.2, 11.0, -250.0])
    mu = lambda F: sum(ck * F ** k for k, ck in enumerate(c))
    m1 = finite_field.first_order(mu(A), mu(-A), mu(2 * A), mu(-2 * A), A)
    m2 = finite_field.second_order(mu(0), mu(A), mu(-A), mu(2 * A), mu(-2 * A), A)
    # both stencils are exact for polynomials through F^4
    assert abs(m1 - c[1]) < 1e-10
    assert abs(m2 - c[2]) < 1e-7


def test_static_limit_hellmann_feynman():
    """mu_z from the CC3 density equals -dE/dF of the field-dependent ground
    state (triples with the field solved by iteration)."""
    s = make_system(2, 4, seed=19)
    ham = cc3.Hamiltonian.from_system(s)
    F = 0.01

    def energy_and_dipole(f):
        w = ham.field_operator([0.0, 0.0, f])
        t1, t2, l1, l2 = _ground_state_with_field(ham, w)
        res = cc3.evaluate(ham, t1, t2, l1, l2, w)
        return res.energy, res.dipole[2]
    e_p, _ = energy_and_dipole(F)
    e_m, _ = energy_and_dipole(-F)
    e_p2, _ = energy_and_dipole(F / 2)
    e_m2, _ = energy_and_dipole(-F / 2)
    _, mu0 = energy_and_dipole(0.0)
    d1 = (e_p - e_m) / (2 * F)
    d2 = (e_p2 - e_m2) / F
    dEdF = (4 * d2 - d1) / 3
    assert abs(mu0 - (-dEdF)) < 1e-8


def _ground_state_with_field(ham, w, tol=1e-12):
    d1, d2 = ham.denominators()
    d1, d2 = d1.to(cc3.CD), d2.to(cc3.CD)
    o, v = ham.o, ham.v
    t1 = torch.zeros(o, v, dtype=cc3.CD)
    t2 = torch.zeros(o, o, v, v, dtype=cc3.CD)
    for _ in range(300):
        r1, r2, _, _ = cc3.forward(ham, t1, t2, w, True, field_on=True)
        if max(float(r1.abs().max()), float(r2.abs().max())) < tol:
            break
        t1, t2 = t1 - r1 / d1, t2 - r2 / d2
    else:
        raise RuntimeError("T amplitudes with the static field did not converge")
    l1 = torch.zeros(o, v, dtype=cc3.CD)
    l2 = torch.zeros(o, o, v, v, dtype=cc3.CD)
    for _ in range(300):
        res = cc3.evaluate(ham, t1, t2, l1, l2, w)
        if max(float(res.r_l1.abs().max()), float(res.r_l2.abs().max())) < tol:
            break
        l1, l2 = l1 - res.r_l1 / d1, l2 - res.r_l2 / d2
    else:
        raise RuntimeError("lambda amplitudes with the static field did not converge")
    return t1, t2, l1, l2
