"""The paper's printed lambda-side triples formulas, term by term.  TEST INFRASTRUCTURE ONLY.

The oracle's main route (``oracle.cc3``) obtains the lambda residuals and the
one-electron density as holomorphic derivatives of the reduced CC3 Lagrangian
(Eq. A6).  This module evaluates instead the closed forms printed in the
paper's appendix, so that the two routes can be compared element by element:

* ``lambda3``  -- the triples multipliers, Eq. A26 (solved by fixed point when
  the field is on, as the triples amplitudes are);
* ``y1``, ``y2`` -- the triples terms of the Lambda1 and Lambda2 equations,
  Eqs. A23 and A24 (printed for zero field only);
* ``triples_density`` -- the triples terms of the one-electron density,
  Eqs. A31-A33.

Conventions are those of ``oracle.cc3``: chemists' dressed integrals
``g[p,q,r,s] = (pq|rs)~`` so that the paper's ``<pq|rs>~`` is ``(pr|qs)~``;
``t2[i,j,a,b] = t_ij^ab``, ``t3[i,j,k,a,b,c] = t_ijk^abc``,
``l1[i,a] = lambda_a^i``, ``l2[i,j,a,b] = lambda_ab^ij``,
``l3[i,j,k,a,b,c] = lambda_abc^ijk``; lambda1 and lambda2 are normalised as in
``L = E + sum l1 R1 + 1/2 sum l2 R2``.

Readings (each confirmed by the tests in ``tests/test_oracle_explicit.py``,
which compare against the Lagrangian derivatives to 1e-12):

* Eq. A26 prints the right-hand side of the lambda3 equation; as for t3
  (Eq. 6) the multipliers are ``-eps^-1`` times it.  With this, lambda3 is the
  Lagrange multiplier of the triples equation in the normalisation
  ``L += 1/6 sum lambda3 * Omega3``.  Inside ``P_ijk^abc`` the ``1/2 P_ij^ab``
  is the identity.  With a field the two ``beta/2`` terms contain lambda3
  itself (the transpose of the field coupling of the t3 equation), so the
  equation is solved by the same fixed point as t3.
* Eq. A23: the first six integrals are printed without a tilde; they are
  ov-ov blocks, which the T1 transformation leaves unchanged.  The sixth term,
  printed ``t_jkl^bcd L_ijab lambda_cd^il`` (i twice, k absent), is read as
  ``t_jkl^bcd L_ljab lambda_cd^ki``; the tenth, printed
  ``t_jk^bc <di|la>~ lambda_acd^jkl`` (a twice, b absent), is read as
  ``t_jk^bc <di|lb>~ lambda_acd^jkl``.  All printed signs are kept.
* Eqs. A31-A33 are the triples parts of ``D_pq = dL/dv~_pq`` (the dressed
  perturbation): ``D_ij`` fills the occupied-occupied block, ``D_ab`` the
  virtual-virtual block and ``D_ia`` the occupied-virtual block.
"""
from __future__ import annotations

import torch

from . import cc3

E = torch.einsum


def _phys(gt):
    """``<pq|rs>~`` as a tensor ``P[p,q,r,s] = g[p,r,q,s]`` (Eq. A27)."""
    return gt.permute(0, 2, 1, 3)


def _L(P):
    """``L_pqrs = 2<pq|rs> - <pq|sr>`` (Eq. A28)."""
    return 2.0 * P - P.permute(0, 1, 3, 2)


def lambda3_rhs(ham, gt, ft, l1, l2):
    """The bracket of Eq. A26 without its field terms, summed by ``P_ijk^abc``:
    ``P{(L_ijab l_c^k - L_ijac l_b^k) + (f~_ia l_bc^jk + sum_l <kj|al>~ l_bc^li
    - sum_d <kd|ab>~ l_cd^ij) - f~_ja l_bc^ik - sum_l L~_ijal l_bc^lk
    + sum_d L~_djab l_cd^ki}``."""
    o, n = ham.o, ham.n
    O, V = slice(0, o), slice(o, n)
    P = _phys(gt)
    L = _L(P)
    f = ft[O, V]
    Z = (E('ijab,kc->ijkabc', L[O, O, V, V], l1) - E('ijac,kb->ijkabc', L[O, O, V, V], l1)
         + E('ia,jkbc->ijkabc', f, l2)
         + E('kjal,libc->ijkabc', P[O, O, V, O], l2)
         - E('kdab,ijcd->ijkabc', P[O, V, V, V], l2)
         - E('ja,ikbc->ijkabc', f, l2)
         - E('ijal,lkbc->ijkabc', L[O, O, V, O], l2)
         + E('djab,kicd->ijkabc', L[V, O, V, V], l2))
    return cc3.P6(Z)


def lambda3(ham, gt, ft, wt, l1, l2, field_on: bool, tol: float = 1e-15, maxiter: int = 200):
    """lambda_abc^ijk of Eq. A26: ``eps lambda3 = -(rhs + field terms)`` where the
    field terms are ``1/2 P_ijk^abc (sum_d v~_da lambda_dbc^ijk - sum_l v~_il
    lambda_abc^ljk)``, i.e. the transpose of the field coupling of the t3
    equation on every slot; fixed-point iteration when the field is on."""
    o, n = ham.o, ham.n
    O, V = slice(0, o), slice(o, n)
    D3 = ham.triples_denominator()
    rhs = -lambda3_rhs(ham, gt, ft, l1, l2)
    lam = rhs / D3
    if not field_on:
        return lam
    woo, wvv = wt[O, O], wt[V, V]
    for _ in range(maxiter):
        half = (E('da,ijkdbc->ijkabc', wvv, lam) - E('il,ljkabc->ijkabc', woo, lam))
        new = (rhs - 0.5 * cc3.P6(half)) / D3
        delta = float((new - lam).abs().max())
        scale = float(new.abs().max())
        lam = new
        if delta <= tol * max(scale, 1e-300):
            break
    return lam


def y1(ham, gt, t2, t3, l2, l3):
    """Y_a^i of Eq. A23 (triples terms of the Lambda1 equation, zero field)."""
    o, n = ham.o, ham.n
    O, V = slice(0, o), slice(o, n)
    P = _phys(gt)
    L = _L(P)
    oovv, Loovv = P[O, O, V, V], L[O, O, V, V]
    y = (E('jklbcd,ijcd,klab->ia', t3, oovv, l2)
         + E('jklbcd,klab,ijcd->ia', t3, oovv, l2)
         + E('jklbcd,ijab,klcd->ia', t3, Loovv, l2)
         - E('jklbcd,ijac,klbd->ia', t3, Loovv, l2)
         - E('jklbcd,jibc,klad->ia', t3, Loovv, l2)
         - E('jklbcd,ljab,kicd->ia', t3, Loovv, l2)
         - E('jkbc,jdla,lkibcd->ia', t2, P[O, V, O, V], l3)
         - E('jkbc,djla,iklbcd->ia', t2, P[V, O, O, V], l3)
         - E('jkbc,idlb,lkjacd->ia', t2, P[O, V, O, V], l3)
         - E('jkbc,dilb,jklacd->ia', t2, P[V, O, O, V], l3)
         + E('jkbc,deab,kijcde->ia', t2, P[V, V, V, V], l3)
         + E('jkbc,ijlm,lmkabc->ia', t2, P[O, O, O, O], l3))
    return y


def y2(ham, gt, l3):
    """Y_ab^ij of Eq. A24: ``P_ij^ab{sum_lde <de|al>~ l_dbe^ijl - sum_lmd <id|ml>~ l_abd^mjl}``."""
    o, n = ham.o, ham.n
    O, V = slice(0, o), slice(o, n)
    P = _phys(gt)
    S = E('deal,ijldbe->ijab', P[V, V, V, O], l3) - E('idml,mjlabd->ijab', P[O, V, O, O], l3)
    return S + S.permute(1, 0, 3, 2)


def triples_density(ham, t2, t3, l2, l3):
    """Triples terms of the one-electron density (Eqs. A31-A33), as an
    ``n x n`` matrix in the T1-transformed basis:
    ``D_ij = -1/2 sum t_ilk^abc l_abc^jlk``, ``D_ab = 1/2 sum t_ijk^bdc l_adc^ijk``,
    ``D_ia = sum (t_ijk^abc - t_ijk^bac) l_bc^jk - sum l_bcd^jkl t_il^cd t_kj^ab``."""
    o, n = ham.o, ham.n
    O, V = slice(0, o), slice(o, n)
    D = torch.zeros(n, n, dtype=cc3.CD)
    D[O, O] = -0.5 * E('ilkabc,jlkabc->ij', t3, l3)
    D[V, V] = 0.5 * E('ijkbdc,ijkadc->ab', t3, l3)
    D[O, V] = (E('ijkabc,jkbc->ia', t3 - t3.permute(0, 1, 2, 4, 3, 5), l2)
               - E('jklbcd,ilcd,kjab->ia', l3, t2, t2))
    return D
