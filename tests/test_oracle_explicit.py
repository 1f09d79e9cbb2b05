"""The paper's printed lambda-side formulas against the Lagrangian derivatives.

``oracle.cc3`` obtains the lambda residuals and the density as holomorphic
derivatives of the reduced CC3 Lagrangian (Eq. A6); ``oracle.explicit``
evaluates the closed forms of the appendix (lambda3 Eq. A26, Y1 Eq. A23,
Y2 Eq. A24, the triples density Eqs. A31-A33).  The two routes share only
the dressing and the t3 solve, so agreement to 1e-12 pins both the printed
formulas (with the readings listed in ``oracle/explicit.py``) and the
derivative route of the oracle.
"""
import pytest
import torch

from oracle import cc3, explicit
from paper_2407_18947_gb300.synth import make_system, random_amplitudes

CD = cc3.CD


def _setup(o, v, seed, scale=1e-2):
    s = make_system(o, v, seed=seed)
    ham = cc3.Hamiltonian.from_system(s)
    t1, t2, l1, l2 = [cc3._ct(x) for x in random_amplitudes(o, v, seed=seed + 3,
                                                          t1_scale=scale, t2_scale=scale)]
    # t_ij^ab = t_ji^ba and lambda_ab^ij = lambda_ba^ji, as the amplitudes are
    t2 = 0.5 * (t2 + t2.permute(1, 0, 3, 2))
    l2 = 0.5 * (l2 + l2.permute(1, 0, 3, 2))
    return ham, t1, t2, l1, l2


def _lagrangian_grads(ham, t1, t2, l1, l2, w, triples):
    t1_ = t1.clone().requires_grad_(True)
    t2_ = t2.clone().requires_grad_(True)
    w_ = w.clone().requires_grad_(True)
    r1, r2, e, _ = cc3.forward(ham, t1_, t2_, w_, triples, field_on=True)
    lag = e + (l1 * r1).sum() + 0.5 * (l2 * r2).sum()
    g1, g2, gw = cc3._holo_grad(lag, [t1_, t2_, w_])
    return g1, g2 + g2.permute(1, 0, 3, 2), gw


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("o,v,seed", [(2, 3, 11), (3, 4, 12), (3, 5, 13)])
def test_printed_lambda3_is_the_multiplier_of_the_triples_equation(o, v, seed):
    """Eq. A26 at zero field equals -P_ijk^abc(dL/dt3)/eps, the multiplier of the
    triples equation, with dL/dt3 the cotangent of lambda1.X1 + 1/2 lambda2.X2."""
    ham, t1, t2, l1, l2 = _setup(o, v, seed)
    w = torch.zeros(ham.n, ham.n, dtype=CD)
    gt, ft, wt, _ = cc3.dress(ham, t1, w)
    t3 = cc3.solve_t3(ham, cc3.triples_W(ham, gt, t2), None, wt, False)
    t3l = t3.clone().requires_grad_(True)
    X1, X2 = cc3.triples_X(ham, gt, ft, t3l)
    ybar = cc3._holo_grad((l1 * X1).sum() + 0.5 * (l2 * X2).sum(), [t3l])[0]
    want = -cc3.P6(ybar) / ham.triples_denominator()
    got = explicit.lambda3(ham, gt, ft, wt, l1, l2, field_on=False)
    assert _rel(got, want) < 1e-12
    # invariant under the simultaneous permutations, as Eq. A30 requires
    assert _rel(torch.einsum('jikbac->ijkabc', got), got) < 1e-14


@pytest.mark.parametrize("o,v,seed", [(2, 3, 21), (3, 4, 22), (3, 5, 23)])
def test_printed_y1_y2_are_the_triples_part_of_the_lambda_residuals(o, v, seed):
    """R_lambda(CC3) - R_lambda(CCSD) at the same amplitudes, zero field, equals
    Y1 (Eq. A23) and Y2 (Eq. A24) with the printed lambda3."""
    ham, t1, t2, l1, l2 = _setup(o, v, seed)
    w = torch.zeros(ham.n, ham.n, dtype=CD)
    a1, a2, _ = _lagrangian_grads(ham, t1, t2, l1, l2, w, True)
    b1, b2, _ = _lagrangian_grads(ham, t1, t2, l1, l2, w, False)
    gt, ft, wt, _ = cc3.dress(ham, t1, w)
    t3 = cc3.solve_t3(ham, cc3.triples_W(ham, gt, t2), None, wt, False)
    l3 = explicit.lambda3(ham, gt, ft, wt, l1, l2, field_on=False)
    # the differences are small against the residuals they come from: the
    # tolerance is relative to the full CC3 residual
    y1 = explicit.y1(ham, gt, t2, t3, l2, l3)
    y2 = explicit.y2(ham, gt, l3)
    assert float((y1 - (a1 - b1)).abs().max()) < 1e-12 * float(a1.abs().max())
    assert float((y2 - (a2 - b2)).abs().max()) < 1e-12 * float(a2.abs().max())
    # and the triples terms are not negligible at this size
    assert float((a1 - b1).abs().max()) > 1e-4 * float(a1.abs().max())


def test_dropping_a_printed_y1_term_is_caught():
    """A plausible transcription mistake (the sixth term of Eq. A23 read as
    printed, with its duplicated i replaced by k) leaves a visible error."""
    o, v = 3, 4
    ham, t1, t2, l1, l2 = _setup(o, v, 22)
    w = torch.zeros(ham.n, ham.n, dtype=CD)
    a1, _, _ = _lagrangian_grads(ham, t1, t2, l1, l2, w, True)
    b1, _, _ = _lagrangian_grads(ham, t1, t2, l1, l2, w, False)
    gt, ft, wt, _ = cc3.dress(ham, t1, w)
    t3 = cc3.solve_t3(ham, cc3.triples_W(ham, gt, t2), None, wt, False)
    l3 = explicit.lambda3(ham, gt, ft, wt, l1, l2, field_on=False)
    O, V = slice(0, o), slice(o, ham.n)
    L = explicit._L(explicit._phys(gt))[O, O, V, V]
    good = torch.einsum('jklbcd,ljab,kicd->ia', t3, L, l2)
    bad = torch.einsum('jklbcd,ijab,klcd->ia', t3, L, l2)
    y = explicit.y1(ham, gt, t2, t3, l2, l3) + good - bad
    assert _rel(y, a1 - b1) > 1e-3


@pytest.mark.parametrize("o,v,seed,field", [(2, 3, 31, 0.0), (3, 4, 32, 0.0),
                                            (2, 3, 33, 0.02), (3, 4, 34, 0.01)])
def test_printed_triples_density_is_the_triples_part_of_dL_dv(o, v, seed, field):
    """D_ij, D_ab, D_ia (Eqs. A31-A33) with the printed lambda3 (fixed point of
    Eq. A26 when the field is on) equal the triples part of dL/dv~, the
    derivative with respect to the dressed perturbation, with and without a
    static field and with t1 != 0."""
    ham, t1, t2, l1, l2 = _setup(o, v, seed)
    w = ham.field_operator([0.3 * field, -0.2 * field, field])
    _, _, gw3 = _lagrangian_grads(ham, t1, t2, l1, l2, w, True)
    _, _, gw2 = _lagrangian_grads(ham, t1, t2, l1, l2, w, False)
    # dL/dv~ = Y^T (dL/dw) X^T for v~ = X w Y with X = 1 - tau, Y = 1 + tau
    n, o_ = ham.n, ham.o
    tau = torch.zeros(n, n, dtype=CD)
    tau[o_:, :o_] = t1.T
    X = torch.eye(n, dtype=CD) - tau
    Y = torch.eye(n, dtype=CD) + tau
    want = Y.T @ (gw3 - gw2) @ X.T
    gt, ft, wt, _ = cc3.dress(ham, t1, w)
    on = field != 0.0
    src = cc3.triples_field_source(ham, wt, t2) if on else None
    t3 = cc3.solve_t3(ham, cc3.triples_W(ham, gt, t2), src, wt, on)
    l3 = explicit.lambda3(ham, gt, ft, wt, l1, l2, field_on=on)
    got = explicit.triples_density(ham, t2, t3, l2, l3)
    assert _rel(got, want) < 1e-11
    # the virtual-occupied block gets no triples term
    assert float(want[o_:, :o_].abs().max()) < 1e-14 * float(want.abs().max())
