"""Pin the oracle's T side to brute-force second quantisation.

The brute-force engine (oracle/bruteforce.py) evaluates Eqs. A10-A12 in the
full N-electron determinant space with the spin-adapted amplitudes of
Eqs. A17-A19 mapped through the generators E_pq, and solves the triples
equation (Eq. 4) over every spin-orbital triple excitation.  The oracle's
spin-adapted closed-shell expressions must agree to round-off: this fixes the
CCSD residual (not printed in the paper), the T1 dressing, X1 (Eq. A21), X2
(Eq. A22), the triples with a field (Eq. A25 read per the commutator) and the
energy (Eq. A8).
"""
import numpy as np
import pytest
import torch

from oracle import cc3
from paper_2407_18947_gb300.synth import random_amplitudes

from _oracle_helpers import tiny

CASES = [((2, 2), 0.0), ((2, 3), 0.05), ((3, 2), 0.04), ((2, 2), 0.08)]


@pytest.mark.parametrize("ov,fld", CASES)
@pytest.mark.parametrize("triples", [False, True])
def test_residuals_match_bruteforce(ov, fld, triples):
    o, v = ov
    s, ham, bf = tiny(o, v, seed=7 + o + v)
    t1, t2, _, _ = random_amplitudes(o, v, seed=3, t1_scale=0.05, t2_scale=0.05)
    w = ham.field_operator([0.3 * fld, -0.2 * fld, fld]).numpy()
    R1, R2, E, _ = bf.residuals(t1, t2, w, triples=triples)
    r1, r2, e, _ = cc3.forward(ham, cc3._ct(t1), cc3._ct(t2), cc3._ct(w), triples=triples)
    assert np.abs(R1 - r1.numpy()).max() < 1e-13
    assert np.abs(R2 - r2.numpy()).max() < 1e-13
    assert abs(E - complex(e)) < 1e-13


def test_triples_state_matches_bruteforce_o3():
    """Distinct i<j<k: the oracle's t3 (mapped with Eq. A19) reproduces the
    brute-force spin-orbital T3|0> including the field coupling."""
    o, v = 3, 3
    s, ham, bf = tiny(o, v, seed=11)
    t1, t2, _, _ = random_amplitudes(o, v, seed=5, t1_scale=0.05, t2_scale=0.05)
    w = ham.field_operator([0.02, -0.03, 0.05]).numpy()
    R1, R2, E, T3 = bf.residuals(t1, t2, w, triples=True)
    r1, r2, e, t3 = cc3.forward(ham, cc3._ct(t1), cc3._ct(t2), cc3._ct(w), triples=True)
    ref = T3 @ bf.fs.phi0
    got = bf.fs.T3_on_ref(t3.numpy())
    assert np.abs(ref).max() > 1e-4
    assert np.abs(got - ref).max() < 1e-14
    assert np.abs(R1 - r1.numpy()).max() < 1e-13
    assert np.abs(R2 - r2.numpy()).max() < 1e-13
    assert abs(E - complex(e)) < 1e-13


def test_planted_sign_error_is_caught():
    """A flipped sign in the occupied field slot (the reading of Eq. A25 the
    paper prints) must fail against brute force: the pin is sensitive."""
    o, v = 2, 3
    s, ham, bf = tiny(o, v, seed=9)
    t1, t2, _, _ = random_amplitudes(o, v, seed=3, t1_scale=0.05, t2_scale=0.05)
    w = ham.field_operator([0.0, 0.0, 0.3]).numpy()
    R1, R2, _, _ = bf.residuals(t1, t2, w, triples=True)
    orig = cc3.triples_slot_op

    def wrong(woo, wvv, t3):
        return orig(-woo, wvv, t3)  # paper's printed '+ v_il' reading
    cc3.triples_slot_op = wrong
    try:
        r1, r2, _, _ = cc3.forward(ham, cc3._ct(t1), cc3._ct(t2), cc3._ct(w), triples=True)
    finally:
        cc3.triples_slot_op = orig
    assert np.abs(R2 - r2.numpy()).max() > 1e-9


def test_ccsd_equals_fci_for_two_electrons():
    """For two electrons CCSD (= CC3, no triples exist) is exact: the converged
    ground-state energy is the lowest FCI eigenvalue."""
    s, ham, bf = tiny(1, 4, seed=21)
    t1, t2, l1, l2 = cc3.solve_ground_state(ham)
    r1, r2, e, _ = cc3.forward(ham, t1, t2, torch.zeros(ham.n, ham.n, dtype=cc3.CD))
    efci, _ = bf.exact_ground_state()
    assert abs(e.real - (efci - bf.e_ref)) < 1e-12
    assert abs(e.imag) < 1e-14
