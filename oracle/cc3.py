"""Plain FP64 complex oracle of real-time CC3 (RT-CC3).  TEST INFRASTRUCTURE ONLY.

Everything is written as full tensors with ``torch.einsum`` on the CPU in
complex128; no blocking, fusion or reordering beyond the equations.  Index
conventions (closed shell, spatial orbitals, occupied first):

* chemists' integrals ``g[p,q,r,s] = (pq|rs)``; the paper's ``<pq|rs>``
  (Eq. A27/A28, physicists' order) is ``(pr|qs)``, and
  ``L_pqrs = 2<pq|rs> - <pq|sr>`` (Eq. A28).
* amplitudes ``t1[i,a] = t_i^a``, ``t2[i,j,a,b] = t_ij^ab = t_ji^ba``,
  ``t3[i,j,k,a,b,c] = t_ijk^abc`` (Eqs. A17-A19),
  ``l1[i,a] = lambda_a^i``, ``l2[i,j,a,b] = lambda_ab^ij``.
* the perturbation is a one-electron operator ``w = beta V`` (Eq. 1, Eq. 10:
  ``V = -mu . E(t)``), held as an ``nmo x nmo`` matrix.

Readings of the paper taken here (each pinned by a brute-force test):

* T1 dressing (Eq. 8, Eq. A4): ``o -> (1 - tau) o (1 + tau)``, ``tau[a,i] = t_i^a``
  (``tau^2 = 0``), applied to the one-electron part *including* the field and
  to the DF factors.
* The dressed Fock matrix in X2 and lambda_3 is the full one-electron part of
  the dressed Hamiltonian (core + field + dressed mean field).
* Triples are not propagated: t3 is the instantaneous solution of the T3
  stationarity condition Eq. 4 / Eq. A12 with ``dt3/dt := 0``; with a field
  the equation is solved by fixed-point iteration on the full stored tensor
  (the paper's own scheme, Section 2.1).  The field couples through the
  commutator ``[V~, T3]``: ``+V~_vv`` on each virtual slot and ``-V~_oo`` on
  each occupied slot.
* Residuals are the biorthogonal projections (equal to the alpha / alpha-beta
  spin-orbital components); the Lagrangian is
  ``L = E + sum l1*R1 + 1/2 sum l2*R2`` (Eq. A6 with lambda_0 = 1), so the
  Euler-Lagrange equations (Eqs. A13-A14) give ``R_l1 = dL/dt1`` and
  ``R_l2 = dL/dt2 + (dL/dt2)^T`` (pair transpose), and the one-electron
  density is ``D = dL/dw``.  Derivatives are holomorphic (plain transpose).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

CD = torch.complex128
RD = torch.float64

FIELD_NONE, FIELD_STATIC, FIELD_COS, FIELD_GAUSS, FIELD_LRCW, FIELD_QRCW = 0, 1, 2, 3, 4, 5


def _ct(x):
    if torch.is_tensor(x):
        return x.to(CD)
    return torch.as_tensor(np.asarray(x), dtype=CD)


class Hamiltonian:
    """Closed-shell Hamiltonian of Eqs. A1-A3 from orbital energies and DF factors.

    ``(pq|rs) = sum_P L[P,p,q] L[P,r,s]``, or the dense chemists' integrals
    themselves (``eri``, then ``Lfac`` is None and the T1 transformation
    acts on the four-index tensor directly).  The core operator is
    ``h = f - G[D_ref]`` with ``G_pq = sum_k 2(pq|kk) - (pk|kq)`` so that the
    reference Fock operator is exactly ``F = sum_p eps_p E_pp`` (Eq. A2).
    """

    def __init__(self, eps, Lfac, dipole, nocc: int, eri=None):
        self.o = int(nocc)
        self.eps = torch.as_tensor(np.asarray(eps), dtype=RD)
        self.n = self.eps.numel()
        self.v = self.n - self.o
        self.mu = torch.as_tensor(np.asarray(dipole), dtype=RD)
        o = self.o
        if eri is not None:
            self.L = None
            g = torch.as_tensor(np.asarray(eri), dtype=RD).reshape(self.n, self.n, self.n, self.n)
            self.g = g
        else:
            self.L = torch.as_tensor(np.asarray(Lfac), dtype=RD)
            g = torch.einsum('Ppq,Prs->pqrs', self.L, self.L)
        J = torch.einsum('pqkk->pq', g[:, :, :o, :o])
        K = torch.einsum('pkkq->pq', g[:, :o, :o, :])
        self.h = torch.diag(self.eps) - (2.0 * J - K)
        # reference energy without nuclear repulsion: sum_i (h_ii + eps_i)
        self.e_ref = float((torch.diagonal(self.h)[:o] + self.eps[:o]).sum())

    @classmethod
    def from_system(cls, sysm):
        return cls(sysm.eps, sysm.Lfac, sysm.dipole, sysm.nocc)

    def field_operator(self, efield) -> torch.Tensor:
        """``w = -E . mu`` (Eq. 10) for a Cartesian field vector ``efield``."""
        e = torch.as_tensor(np.asarray(efield, dtype=np.float64))
        return (-torch.einsum('x,xpq->pq', e, self.mu)).to(CD)

    def denominators(self):
        o = self.o
        eo, ev = self.eps[:o], self.eps[o:]
        d1 = ev[None, :] - eo[:, None]
        d2 = (ev[None, None, :, None] + ev[None, None, None, :]
              - eo[:, None, None, None] - eo[None, :, None, None])
        return d1, d2

    def triples_denominator(self):
        """``eps_ijk^abc = e_a + e_b + e_c - e_i - e_j - e_k`` (Eq. 6, Eq. A16)."""
        o = self.o
        eo, ev = self.eps[:o], self.eps[o:]
        occ = eo[:, None, None] + eo[None, :, None] + eo[None, None, :]
        vir = ev[:, None, None] + ev[None, :, None] + ev[None, None, :]
        return (vir[None, None, None] - occ[:, :, :, None, None, None]).to(CD)


@dataclass
class FieldSpec:
    """Time profile of the field (Eq. 14 cosine, Eq. 32 Gaussian, static, or the
    linear / quadratic ramped continuous waves of Section 2.2.4)."""

    kind: int = FIELD_NONE
    amplitude: float = 0.0
    omega: float = 0.0
    center: float = 0.0
    width: float = 1.0
    direction: tuple = (0.0, 0.0, 1.0)

    def strength(self, t: float) -> float:
        if self.kind == FIELD_NONE:
            return 0.0
        if self.kind == FIELD_STATIC:
            return self.amplitude
        if self.kind == FIELD_COS:
            return self.amplitude * math.cos(self.omega * t)
        if self.kind == FIELD_GAUSS:
            return self.amplitude * math.exp(-(t - self.center) ** 2 / (2.0 * self.width ** 2))
        if self.kind in (FIELD_LRCW, FIELD_QRCW):
            # ramped continuous waves of Section 2.2.4, ramp duration t_r = width
            if t < 0.0:
                return 0.0
            tr = self.width
            c = math.cos(self.omega * t)
            if t >= tr:
                return self.amplitude * c
            if self.kind == FIELD_LRCW:
                return self.amplitude * (t / tr) * c
            if t < 0.5 * tr:
                return self.amplitude * (2.0 * t * t / (tr * tr)) * c
            return self.amplitude * (1.0 - 2.0 * (t - tr) ** 2 / (tr * tr)) * c
        raise ValueError(f"unknown field kind {self.kind}")

    def vector(self, t: float) -> np.ndarray:
        return self.strength(t) * np.asarray(self.direction, dtype=np.float64)


# --------------------------------------------------------------------------
# T1 dressing (Eq. 8, Eq. A4)
# --------------------------------------------------------------------------
def dress(ham: Hamiltonian, t1: torch.Tensor, w: torch.Tensor):
    """T1-transformed integrals.

    Returns ``(g~, f~, w~, h~)``: dressed chemists' two-electron integrals
    ``(n,n,n,n)``, dressed Fock matrix ``f~_pq = h~_pq + sum_k 2 g~_pqkk - g~_pkkq``
    (``h~`` includes the field), the dressed perturbation ``w~`` and ``h~``.
    """
    o, v, n = ham.o, ham.v, ham.n
    zero_top = torch.zeros(o, n, dtype=CD)
    bottom = torch.cat([t1.transpose(0, 1), torch.zeros(v, v, dtype=CD)], dim=1)
    tau = torch.cat([zero_top, bottom], dim=0)  # tau[a,i] = t_i^a
    eye = torch.eye(n, dtype=CD)
    X = eye - tau
    Y = eye + tau
    ht = X @ (ham.h.to(CD) + w) @ Y
    wt = X @ w @ Y
    if ham.L is not None:
        Lt = torch.einsum('pr,Prs,sq->Ppq', X, ham.L.to(CD), Y)
        gt = torch.einsum('Ppq,Prs->pqrs', Lt, Lt)
    else:
        # (pq|rs)~ = sum X_pt Y_uq X_rv Y_ws (tu|vw), one index at a time
        g = ham.g.to(CD)
        g = torch.einsum('pt,tuvw->puvw', X, g)
        g = torch.einsum('puvw,uq->pqvw', g, Y)
        g = torch.einsum('rv,pqvw->pqrw', X, g)
        gt = torch.einsum('pqrw,ws->pqrs', g, Y)
    J = torch.einsum('pqkk->pq', gt[:, :, :o, :o])
    K = torch.einsum('pkkq->pq', gt[:, :o, :o, :])
    ft = ht + 2.0 * J - K
    return gt, ft, wt, ht


def _blocks(ham):
    o, n = ham.o, ham.n
    return slice(0, o), slice(o, n)


# --------------------------------------------------------------------------
# CCSD part of the residuals (Eqs. A10-A11 without the T3 terms)
# --------------------------------------------------------------------------
def ccsd_residual(ham, gt, ft, t2):
    """Spin-adapted closed-shell CCSD residual in the T1-transformed Hamiltonian.

    ``R1 = <mu1|H + [H,T2]|0>`` and ``R2 = <mu2|H + [H,T2] + 1/2[[H,T2],T2]|0>``,
    the CCSD components of Eqs. A10-A11 (the paper adds the triples to
    "the existing CCSD equations", Section 2.1, without printing them).
    """
    O, V = _blocks(ham)
    T = t2
    u = 2.0 * T - T.transpose(2, 3)  # u_ij^ab = 2 t_ij^ab - t_ij^ba
    g_ovov = gt[O, V, O, V]
    # singles
    r1 = torch.einsum('kicd,adkc->ia', u, gt[V, V, O, V])  # u_ki^cd (ad|kc)~
    r1 = r1 - torch.einsum('klac,kilc->ia', u, gt[O, O, O, V])
    r1 = r1 + torch.einsum('ikac,kc->ia', u, ft[O, V])
    r1 = r1 + ft[V, O].transpose(0, 1)
    # doubles: A (source + particle ladder), B (hole ladder)
    A2 = torch.einsum('aibj->ijab', gt[V, O, V, O]) + torch.einsum('ijcd,acbd->ijab', T, gt[V, V, V, V])
    Wkilj = gt[O, O, O, O] + torch.einsum('ijcd,kcld->kilj', T, g_ovov)
    B2 = torch.einsum('klab,kilj->ijab', T, Wkilj)
    # C, D, E terms, symmetrised with P_ij^ab
    Xc = gt[O, O, V, V] - 0.5 * torch.einsum('liad,kdlc->kiac', T, g_ovov)
    C2 = -0.5 * torch.einsum('kjbc,kiac->ijab', T, Xc) - torch.einsum('kibc,kjac->ijab', T, Xc)
    Lt_voov = 2.0 * gt[V, O, O, V] - torch.einsum('acki->aikc', gt[V, V, O, O])
    L_ovov = 2.0 * g_ovov - torch.einsum('lckd->ldkc', g_ovov)
    Xd = torch.einsum('aikc->iakc', Lt_voov) + 0.5 * torch.einsum('ilad,ldkc->iakc', u, L_ovov)
    D2 = 0.5 * torch.einsum('jkbc,iakc->ijab', u, Xd)
    Fvv = ft[V, V] - torch.einsum('klbd,ldkc->bc', u, g_ovov)
    Foo = ft[O, O] + torch.einsum('ljcd,kdlc->kj', u, g_ovov)
    E2 = torch.einsum('ijac,bc->ijab', T, Fvv) - torch.einsum('ikab,kj->ijab', T, Foo)
    S = C2 + D2 + E2
    r2 = A2 + B2 + S + S.permute(1, 0, 3, 2)
    return r1, r2


def ccsd_energy(ham, gt, ht, t2):
    """``<0|H + [H,T2]|0> - E_ref`` with the dressed H (Eq. A8; phase equation)."""
    O, V = _blocks(ham)
    goooo = gt[O, O, O, O]
    e = 2.0 * torch.einsum('ii->', ht[O, O])
    e = e + 2.0 * torch.einsum('iijj->', goooo) - torch.einsum('ijji->', goooo)
    g_ovov = gt[O, V, O, V]
    L = 2.0 * g_ovov - torch.einsum('ibja->iajb', g_ovov)
    e = e + torch.einsum('ijab,iajb->', t2, L)
    return e - ham.e_ref


# --------------------------------------------------------------------------
# Triples (Eqs. 4, 6, A12, A25, A30)
# --------------------------------------------------------------------------
def P6(Z):
    """``P_ijk^abc`` of Eq. A30: plain sum of the six simultaneous permutations."""
    return (Z + torch.einsum('jikbac->ijkabc', Z) + torch.einsum('ikjacb->ijkabc', Z)
            + torch.einsum('kjicba->ijkabc', Z) + torch.einsum('kijcab->ijkabc', Z)
            + torch.einsum('jkibca->ijkabc', Z))


def triples_W(ham, gt, t2):
    """Connected triples ``W = <mu3|[U,T2]|0>`` (Eq. 6 numerator, Eq. A25):
    ``P_ijk^abc { sum_e t_ij^ae <cb|ke>~ - sum_m t_im^ab <mc|jk>~ }``."""
    O, V = _blocks(ham)
    Z = torch.einsum('ijae,ckbe->ijkabc', t2, gt[V, O, V, V])   # <cb|ke>~ = (ck|be)~
    Z = Z - torch.einsum('imab,mjck->ijkabc', t2, gt[O, O, V, O])  # <mc|jk>~ = (mj|ck)~
    return P6(Z)


def triples_field_source(ham, wt, t2):
    """``<mu3| 1/2 [[V~,T2],T2] |0>``: ``-P_ijk^abc sum_ld v~_ld t_ij^ad t_kl^cb``
    (the beta-term of Eq. A25 written as part of the source, sign per the
    commutator)."""
    O, V = _blocks(ham)
    Z = torch.einsum('ld,ijad,klcb->ijkabc', wt[O, V], t2, t2)
    return -P6(Z)


def triples_slot_op(wt_oo, wt_vv, t3):
    """``<mu3|[V~, T3]|0>``: ``+v~_ad`` on every virtual slot, ``-v~_li`` on every
    occupied slot (field coupling of Eq. 4 / Eq. A12)."""
    r = (torch.einsum('ad,ijkdbc->ijkabc', wt_vv, t3)
         + torch.einsum('bd,ijkadc->ijkabc', wt_vv, t3)
         + torch.einsum('cd,ijkabd->ijkabc', wt_vv, t3))
    r = r - (torch.einsum('li,ljkabc->ijkabc', wt_oo, t3)
             + torch.einsum('lj,ilkabc->ijkabc', wt_oo, t3)
             + torch.einsum('lk,ijlabc->ijkabc', wt_oo, t3))
    return r


def solve_t3(ham, W, src, wt, field_on: bool, tol: float = 1e-15, maxiter: int = 200):
    """Solve ``eps3 t3 + [V~,T3] = -(W + src)`` (Eq. 4 with dt3/dt = 0).

    Field-free: the closed form of Eq. 6.  With a field: fixed-point
    iteration on the full stored tensor until ``max|dt3| <= tol max|t3|``
    (Section 2.1 keeps the full triples and iterates).
    """
    D3 = ham.triples_denominator()
    rhs = -(W + src) if src is not None else -W
    t3 = rhs / D3
    if not field_on:
        return t3
    O, V = _blocks(ham)
    woo, wvv = wt[O, O], wt[V, V]
    for _ in range(maxiter):
        new = (rhs - triples_slot_op(woo, wvv, t3)) / D3
        delta = float((new - t3).detach().abs().max())
        scale = float(new.detach().abs().max())
        t3 = new
        if delta <= tol * max(scale, 1e-300):
            break
    return t3


def triples_X(ham, gt, ft, t3):
    """Triples contributions to the T1 and T2 residuals: X1 (Eq. A21), X2 (Eq. A22)."""
    O, V = _blocks(ham)
    g_ovov = gt[O, V, O, V]
    Ljkbc = 2.0 * torch.einsum('jbkc->jkbc', g_ovov) - torch.einsum('jckb->jkbc', g_ovov)
    d = t3 - torch.einsum('ijkcba->ijkabc', t3)  # t_ijk^abc - t_ijk^cba
    X1 = torch.einsum('ijkabc,jkbc->ia', d, Ljkbc)
    Xa = torch.einsum('ijkabc,kc->ijab', d, ft[O, V])
    # (2 t^cbe - t^ceb - t^ebc) indexed [i,j,k,c,b,e]
    Ub = 2.0 * t3 - torch.einsum('ijkxzy->ijkxyz', t3) - torch.einsum('ijkzyx->ijkxyz', t3)
    Xb = torch.einsum('ijkcbe,acke->ijab', Ub, gt[V, V, O, V])  # <ak|ce>~ = (ac|ke)~
    # (2 t_mjk^cba - t_mjk^bca - t_mjk^abc) indexed [m,j,k,c,b,a]
    Uc = 2.0 * t3 - torch.einsum('mjkyxz->mjkxyz', t3) - torch.einsum('mjkzyx->mjkxyz', t3)
    Xc = -torch.einsum('mjkcba,kimc->ijab', Uc, gt[O, O, O, V])  # <km|ic>~ = (ki|mc)~
    S = Xa + Xb + Xc
    X2 = S + S.permute(1, 0, 3, 2)
    return X1, X2


# --------------------------------------------------------------------------
# One residual evaluation (one RK4 stage) and its Lagrangian derivatives
# --------------------------------------------------------------------------
@dataclass
class StageResult:
    r_t1: torch.Tensor
    r_t2: torch.Tensor
    r_l1: torch.Tensor | None
    r_l2: torch.Tensor | None
    energy: complex
    density: torch.Tensor | None
    dipole: np.ndarray | None
    t3: torch.Tensor | None = None


def forward(ham, t1, t2, w, triples: bool = True, field_on: bool | None = None, keep_t3=False):
    """The T side: (R1, R2, E[, t3]) as differentiable functions of (t1, t2, w)."""
    gt, ft, wt, ht = dress(ham, t1, w)
    r1, r2 = ccsd_residual(ham, gt, ft, t2)
    t3 = None
    if triples:
        if field_on is None:
            field_on = bool(w.detach().abs().max() > 0)
        W = triples_W(ham, gt, t2)
        src = triples_field_source(ham, wt, t2) if field_on else None
        t3 = solve_t3(ham, W, src, wt, field_on)
        X1, X2 = triples_X(ham, gt, ft, t3)
        r1 = r1 + X1
        r2 = r2 + X2
    e = ccsd_energy(ham, gt, ht, t2)
    return r1, r2, e, t3


def lagrangian(ham, t1, t2, l1, l2, w, triples=True):
    """Reduced CC3 Lagrangian ``E + sum l1 R1 + 1/2 sum l2 R2`` (Eq. A6 with t3
    eliminated through its stationarity condition and lambda_0 = 1)."""
    r1, r2, e, _ = forward(ham, t1, t2, w, triples)
    return e + (l1 * r1).sum() + 0.5 * (l2 * r2).sum()


def _holo_grad(out, inputs):
    """Holomorphic derivative d out / d z for complex leaves (plain transpose)."""
    gs = torch.autograd.grad(out.real, inputs, allow_unused=True)
    return [None if g is None else g.conj().resolve_conj() for g in gs]


def evaluate(ham, t1, t2, l1, l2, w, triples: bool = True, need_lambda: bool = True,
             keep_t3: bool = False) -> StageResult:
    """One RK4-stage evaluation: T residuals (Eqs. A10-A11), lambda residuals
    (Eqs. A13-A14 via the Euler-Lagrange derivative of the Lagrangian), the
    energy (Eq. A8) and the one-electron density ``D = dL/dw``."""
    t1 = _ct(t1).detach().clone().requires_grad_(need_lambda)
    t2 = _ct(t2).detach().clone().requires_grad_(need_lambda)
    w = _ct(w).detach().clone().requires_grad_(need_lambda)
    l1 = _ct(l1).detach()
    l2 = _ct(l2).detach()
    with torch.set_grad_enabled(need_lambda):
        # the field-coupling terms of the triples equation always enter the
        # graph when derivatives are taken: at w = 0 they vanish in value but
        # not in dL/dw (the D_ij, D_ab, D_ia triples density terms)
        r1, r2, e, t3 = forward(ham, t1, t2, w, triples, field_on=True if need_lambda else None)
        if not need_lambda:
            return StageResult(r1.detach(), r2.detach(), None, None, complex(e.detach()), None, None,
                               t3.detach() if (keep_t3 and t3 is not None) else None)
        lag = e + (l1 * r1).sum() + 0.5 * (l2 * r2).sum()
        g1, g2, gw = _holo_grad(lag, [t1, t2, w])
    rl1 = g1
    rl2 = g2 + g2.permute(1, 0, 3, 2)
    D = gw
    dip = torch.einsum('pq,xpq->x', D, ham.mu.to(CD)).numpy()
    return StageResult(r1.detach(), r2.detach(), rl1.detach(), rl2.detach(), complex(e.detach()),
                       D.detach(), dip, t3.detach() if (keep_t3 and t3 is not None) else None)


# --------------------------------------------------------------------------
# Ground state (zero field) and RK4 propagation
# --------------------------------------------------------------------------
class DIIS:
    """Pulay extrapolation over the last ``size`` Jacobi iterates."""

    def __init__(self, size=8):
        self.size, self.vecs, self.errs = size, [], []

    def __call__(self, x, e):
        self.vecs.append(x)
        self.errs.append(e)
        if len(self.vecs) > self.size:
            self.vecs.pop(0)
            self.errs.pop(0)
        m = len(self.vecs)
        if m < 2:
            return x
        E = torch.stack(self.errs)
        B = torch.zeros(m + 1, m + 1, dtype=CD)
        B[:m, :m] = E.conj() @ E.T
        B[m, :m] = -1.0
        B[:m, m] = -1.0
        rhs = torch.zeros(m + 1, dtype=CD)
        rhs[m] = -1.0
        c = torch.linalg.solve(B, rhs)[:m]
        return sum(ci * vi for ci, vi in zip(c, self.vecs))


def _jacobi_diis(step_fn, x1, x2, d1, d2, tol, maxiter, label, verbose):
    """Iterate ``x <- x - R(x)/D`` with DIIS until ``max|R| < tol``."""
    diis = DIIS()
    o_v = x1.numel()
    for it in range(maxiter):
        r1, r2 = step_fn(x1, x2)
        err = max(float(r1.abs().max()), float(r2.abs().max()))
        if verbose:
            print(label, it, err)
        if err < tol:
            return x1, x2
        e = torch.cat([(-r1 / d1).flatten(), (-r2 / d2).flatten()])
        x = torch.cat([x1.flatten(), x2.flatten()]) + e
        x = diis(x, e)
        x1, x2 = x[:o_v].reshape(x1.shape), x[o_v:].reshape(x2.shape)
    raise RuntimeError(f'{label} amplitudes did not converge')


def solve_ground_state(ham, triples=True, tol=1e-12, maxiter=400, verbose=False):
    """Zero-field ground state: Jacobi steps ``t <- t - R/D`` (orbital-energy
    denominators) accelerated by DIIS, first for T then for lambda."""
    o, v, n = ham.o, ham.v, ham.n
    d1, d2 = ham.denominators()
    d1, d2 = d1.to(CD), d2.to(CD)
    w = torch.zeros(n, n, dtype=CD)

    def tstep(x1, x2):
        r1, r2, _, _ = forward(ham, x1, x2, w, triples, field_on=False)
        return r1, r2
    t1, t2 = _jacobi_diis(tstep, torch.zeros(o, v, dtype=CD), torch.zeros(o, o, v, v, dtype=CD),
                          d1, d2, tol, maxiter, 'T', verbose)

    def lstep(x1, x2):
        res = evaluate(ham, t1, t2, x1, x2, w, triples)
        return res.r_l1, res.r_l2
    l1, l2 = _jacobi_diis(lstep, torch.zeros(o, v, dtype=CD), torch.zeros(o, o, v, v, dtype=CD),
                          d1, d2, tol, maxiter, 'L', verbose)
    return t1, t2, l1, l2


def time_derivative(ham, field: FieldSpec, t, y, triples=True):
    """``dt/dt = -i R_T`` (Eq. 2 / A10-A11), ``dl/dt = +i R_l`` (Eq. 3 / A13-A14)."""
    t1, t2, l1, l2 = y
    w = ham.field_operator(field.vector(t))
    res = evaluate(ham, t1, t2, l1, l2, w, triples)
    dy = (-1j * res.r_t1, -1j * res.r_t2, 1j * res.r_l1, 1j * res.r_l2)
    return dy, res


def propagate_rk4(ham, field: FieldSpec, y0, h: float, nsteps: int, triples=True, t0: float = 0.0):
    """Classical RK4 with stage times t, t+h/2, t+h/2, t+h.

    Returns the final state and the dipole (nsteps+1, 3) and energy (nsteps+1,)
    trajectories; entry n is evaluated from the state at t0 + n h.
    """
    y = tuple(_ct(x) for x in y0)
    dips, ens = [], []
    t = t0
    for step in range(nsteps):
        k1, res = time_derivative(ham, field, t, y, triples)
        dips.append(res.dipole)
        ens.append(res.energy)
        y2 = tuple(a + 0.5 * h * b for a, b in zip(y, k1))
        k2, _ = time_derivative(ham, field, t + 0.5 * h, y2, triples)
        y3 = tuple(a + 0.5 * h * b for a, b in zip(y, k2))
        k3, _ = time_derivative(ham, field, t + 0.5 * h, y3, triples)
        y4 = tuple(a + h * b for a, b in zip(y, k3))
        k4, _ = time_derivative(ham, field, t + h, y4, triples)
        y = tuple(a + (h / 6.0) * (b1 + 2.0 * b2 + 2.0 * b3 + b4)
                  for a, b1, b2, b3, b4 in zip(y, k1, k2, k3, k4))
        t = t0 + (step + 1) * h
    w = ham.field_operator(field.vector(t))
    res = evaluate(ham, *y, w, triples)
    dips.append(res.dipole)
    ens.append(res.energy)
    return y, np.array(dips), np.array(ens)
