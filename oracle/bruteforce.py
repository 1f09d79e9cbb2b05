"""Brute-force second quantisation in the N-electron determinant space.

TEST INFRASTRUCTURE ONLY.  For tiny systems (a few spatial orbitals) this
module builds fermionic operators as explicit matrices and evaluates the
CC3 equations exactly as the paper states them in operator form, with no
spin adaptation and no algebraic simplification:

* ``H = sum h_pq E_pq + 1/2 sum (pq|rs) (E_pq E_rs - delta_qr E_ps)``,
  ``E_pq`` the singlet generators of Eq. A20;
* ``T1``, ``T2``, spin-adapted ``T3`` built from generators as in Eqs. A17-A19;
* the T1 transformation ``e^{-T1} O e^{T1}`` (Eq. 8, Eq. A4) by exact
  (nilpotent) matrix exponentials;
* the triples from the stationarity condition Eq. 4 / Eq. A12 (with
  ``dt3/dt := 0``), solved as a dense linear system over every triply
  excited determinant (spin-orbital triples, no spin adaptation);
* residuals as the alpha (singles) and alpha-beta (doubles) components of
  ``H~ + [H~,T2] + [H~,T3] (+ 1/2 [[H~,T2],T2])`` acting on the reference
  (Eqs. A10-A11), and the energy of Eq. A8.

Spin orbital ``2p`` is p-alpha, ``2p+1`` is p-beta; determinants are bit
masks; the reference occupies the lowest ``2 nocc`` spin orbitals.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def _popcount(x: int) -> int:
    return bin(x).count("1")


class FockSpace:
    def __init__(self, nmo: int, nocc: int):
        self.n = nmo
        self.o = nocc
        self.v = nmo - nocc
        self.nso = 2 * nmo
        self.N = 2 * nocc
        dets = []
        for occ in itertools.combinations(range(self.nso), self.N):
            m = 0
            for s in occ:
                m |= 1 << s
            dets.append(m)
        self.dets = dets
        self.index = {d: k for k, d in enumerate(dets)}
        self.dim = len(dets)
        self.ref = (1 << self.N) - 1
        self.phi0 = np.zeros(self.dim, dtype=complex)
        self.phi0[self.index[self.ref]] = 1.0
        self._ca = {}
        self._E = {}

    # a^+_P a_Q on spin orbitals
    def ca(self, P: int, Q: int) -> sp.csr_matrix:
        key = (P, Q)
        if key in self._ca:
            return self._ca[key]
        rows, cols, vals = [], [], []
        for k, d in enumerate(self.dets):
            if not (d >> Q) & 1:
                continue
            s = _popcount(d & ((1 << Q) - 1))
            d1 = d & ~(1 << Q)
            if (d1 >> P) & 1:
                continue
            s += _popcount(d1 & ((1 << P) - 1))
            d2 = d1 | (1 << P)
            rows.append(self.index[d2])
            cols.append(k)
            vals.append(-1.0 if s & 1 else 1.0)
        m = sp.csr_matrix((vals, (rows, cols)), shape=(self.dim, self.dim))
        self._ca[key] = m
        return m

    def E(self, p: int, q: int) -> sp.csr_matrix:
        """Singlet excitation generator ``E_pq`` (Eq. A20)."""
        key = (p, q)
        if key not in self._E:
            self._E[key] = self.ca(2 * p, 2 * q) + self.ca(2 * p + 1, 2 * q + 1)
        return self._E[key]

    def one_body(self, h: np.ndarray) -> np.ndarray:
        n = self.n
        H = sp.csr_matrix((self.dim, self.dim), dtype=complex)
        for p in range(n):
            for q in range(n):
                if h[p, q] != 0:
                    H = H + h[p, q] * self.E(p, q)
        return H.toarray()

    def hamiltonian(self, h: np.ndarray, g: np.ndarray) -> np.ndarray:
        """``sum h_pq E_pq + 1/2 sum g_pqrs (E_pq E_rs - delta_qr E_ps)``, g chemists'."""
        n = self.n
        H = sp.csr_matrix(self.one_body(h))
        hk = -0.5 * np.einsum('pqqs->ps', g)
        H = H + sp.csr_matrix(self.one_body(hk))
        for r in range(n):
            for s in range(n):
                Ors = sp.csr_matrix((self.dim, self.dim), dtype=complex)
                for p in range(n):
                    for q in range(n):
                        if g[p, q, r, s] != 0:
                            Ors = Ors + g[p, q, r, s] * self.E(p, q)
                H = H + 0.5 * (Ors @ self.E(r, s))
        return H.toarray()

    # excitation operators in the spin-adapted parametrisation (Eqs. A17-A19)
    def T1(self, t1):
        o = self.o
        T = sp.csr_matrix((self.dim, self.dim), dtype=complex)
        for i in range(o):
            for a in range(self.v):
                T = T + t1[i, a] * self.E(o + a, i)
        return T.toarray()

    def T2(self, t2):
        o, v = self.o, self.v
        T = sp.csr_matrix((self.dim, self.dim), dtype=complex)
        for i, j, a, b in itertools.product(range(o), range(o), range(v), range(v)):
            if t2[i, j, a, b] != 0:
                T = T + 0.5 * t2[i, j, a, b] * (self.E(o + a, i) @ self.E(o + b, j))
        return T.toarray()

    def T3_on_ref(self, t3):
        """``T3 |0>`` for spin-adapted ``t3[i,j,k,a,b,c]`` (Eq. A19)."""
        o, v = self.o, self.v
        out = np.zeros(self.dim, dtype=complex)
        for i, j, k in itertools.product(range(o), repeat=3):
            for a, b, c in itertools.product(range(v), repeat=3):
                x = t3[i, j, k, a, b, c]
                if x == 0:
                    continue
                vec = self.E(o + c, k) @ self.phi0
                vec = self.E(o + b, j) @ vec
                vec = self.E(o + a, i) @ vec
                out += (x / 6.0) * vec
        return out

    # projections
    def single_bra(self, i, a):
        """``a^+_{a alpha} a_{i alpha} |0>`` (the alpha single)."""
        return self.ca(2 * (self.o + a), 2 * i) @ self.phi0

    def double_bra(self, i, j, a, b):
        """``a^+_{a alpha} a_{i alpha} a^+_{b beta} a_{j beta} |0>``."""
        o = self.o
        vec = self.ca(2 * (o + b) + 1, 2 * j + 1) @ self.phi0
        return self.ca(2 * (o + a), 2 * i) @ vec

    def triples_basis(self):
        """Spin-orbital triple excitation operators ``a+_A a_I a+_B a_J a+_C a_K``."""
        occ = list(range(self.N))
        vir = list(range(self.N, self.nso))
        ops = []
        for I, J, K in itertools.combinations(occ, 3):
            for A, B, C in itertools.combinations(vir, 3):
                ops.append((self.ca(A, I) @ self.ca(B, J) @ self.ca(C, K)).toarray())
        return ops


def expm_nilpotent(T: np.ndarray) -> np.ndarray:
    """``exp(T)`` for a nilpotent matrix by its terminating series."""
    out = np.eye(T.shape[0], dtype=complex)
    term = np.eye(T.shape[0], dtype=complex)
    for k in range(1, T.shape[0] + 1):
        term = term @ T / k
        if not np.any(term):
            break
        out = out + term
    return out


class BruteCC3:
    """CC3 residuals by brute force for a tiny ``(h, g, eps)`` system."""

    def __init__(self, eps, h, g, nocc):
        self.eps = np.asarray(eps, dtype=float)
        self.h = np.asarray(h, dtype=complex)
        self.g = np.asarray(g, dtype=complex)
        self.n = len(eps)
        self.o = nocc
        self.v = self.n - nocc
        self.fs = FockSpace(self.n, nocc)
        fs = self.fs
        self.H0 = fs.hamiltonian(self.h, self.g)
        self.Fhat = fs.one_body(np.diag(self.eps).astype(complex))
        self.e_ref = float(np.real(fs.phi0 @ self.H0 @ fs.phi0))
        self._tau3 = None
        self._Eop = {}

    def op(self, w):
        return self.fs.one_body(np.asarray(w, dtype=complex))

    def tau3(self):
        if self._tau3 is None:
            self._tau3 = self.fs.triples_basis()
        return self._tau3

    def solve_triples(self, Ht, Ft, Vt, T2, field=True):
        """Spin-orbital T3 from ``<mu3|[H~,T2] + [F~+V~,T3] + 1/2[[V~,T2],T2]|0> = 0``."""
        fs = self.fs
        phi = fs.phi0
        taus = self.tau3()
        kets = np.array([t @ phi for t in taus])  # rows: tau_mu |0>
        proj = kets.conj()
        src = Ht @ (T2 @ phi) - T2 @ (Ht @ phi)
        if field:
            C = Vt @ T2 - T2 @ Vt
            src = src + 0.5 * (C @ (T2 @ phi) - T2 @ (C @ phi))
        rhs = proj @ src
        A = Ft + Vt if field else Ft
        M = np.empty((len(taus), len(taus)), dtype=complex)
        Aphi = A @ phi
        for nu, t in enumerate(taus):
            M[:, nu] = proj @ (A @ (t @ phi) - t @ Aphi)
        x = np.linalg.solve(M, -rhs)
        T3 = sum(xv * t for xv, t in zip(x, taus))
        return T3

    def residuals(self, t1, t2, w, triples=True):
        """Return (R1, R2, E, T3 operator) for amplitudes (t1, t2) and field w."""
        fs = self.fs
        o, v = self.o, self.v
        phi = fs.phi0
        T1 = fs.T1(t1)
        eT = expm_nilpotent(T1)
        emT = expm_nilpotent(-T1)
        W = self.op(w)
        Ht = emT @ (self.H0 + W) @ eT
        Ft = emT @ self.Fhat @ eT
        Vt = emT @ W @ eT
        T2 = fs.T2(t2)
        field = bool(np.any(np.asarray(w) != 0))
        psi1 = Ht @ phi + Ht @ (T2 @ phi) - T2 @ (Ht @ phi)
        T3 = None
        if triples:
            T3 = self.solve_triples(Ht, Ft, Vt, T2, field)
            psi1 = psi1 + Ht @ (T3 @ phi) - T3 @ (Ht @ phi)
        C = Ht @ T2 - T2 @ Ht
        psi2 = psi1 + 0.5 * (C @ (T2 @ phi) - T2 @ (C @ phi))
        R1 = np.zeros((o, v), dtype=complex)
        R2 = np.zeros((o, o, v, v), dtype=complex)
        for i in range(o):
            for a in range(v):
                R1[i, a] = fs.single_bra(i, a).conj() @ psi1
        for i, j, a, b in itertools.product(range(o), range(o), range(v), range(v)):
            R2[i, j, a, b] = fs.double_bra(i, j, a, b).conj() @ psi2
        E = phi @ (Ht @ phi + Ht @ (T2 @ phi) - T2 @ (Ht @ phi)) - self.e_ref
        return R1, R2, complex(E), T3

    def lagrangian(self, t1, t2, l1, l2, w, triples=True):
        R1, R2, E, _ = self.residuals(t1, t2, w, triples)
        return E + np.sum(l1 * R1) + 0.5 * np.sum(l2 * R2)

    def exact_ground_state(self):
        """Lowest eigenpair of H0 in the N-electron space (exact for any N)."""
        vals, vecs = np.linalg.eigh(self.H0)
        return vals[0], vecs[:, 0]

    def expectation_one_body(self, psi, m):
        M = self.op(m)
        return complex(np.vdot(psi, M @ psi) / np.vdot(psi, psi))

    def propagate_exact(self, psi0, w_of_t, times, h_int=1e-3):
        """Exact TDSE ``i dpsi/dt = (H0 + W(t)) psi`` by many small exponential
        midpoint steps (second order in ``h_int``; used with ``h_int`` tiny)."""
        out = [psi0.copy()]
        psi = psi0.copy()
        t = times[0]
        for t_next in times[1:]:
            nsub = max(1, int(round((t_next - t) / h_int)))
            dt = (t_next - t) / nsub
            for s in range(nsub):
                tm = t + (s + 0.5) * dt
                Hm = self.H0 + self.op(w_of_t(tm))
                psi = sla.expm(-1j * dt * Hm) @ psi
            t = t_next
            out.append(psi.copy())
        return out
