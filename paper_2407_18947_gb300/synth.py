"""Seeded synthetic inputs for the RT-CC3 triples hot path.

This module holds random-number generation only: none of the method's
arithmetic lives here, so both the CPU oracle and the CUDA path may draw
their inputs from it.

Workload recipe (a stand-in for the paper's water-cluster cc-pVDZ runs,
Section 3 and Table 1, whose integrals and geometries are not available):

* ``nocc = 5 n`` and ``nvir = 19 n`` for the (H2O)_n-sized cases.
* Orbital energies: occupied ``U[-1.5, -0.3]`` Ha, virtual ``U[0.2, 3.0]`` Ha,
  each sorted ascending.
* Density-fitted electron-repulsion factors ``L[P, p, q]`` drawn
  ``N(0, sigma^2)`` for ``p <= q`` and mirrored, ``naux = 3 nmo`` by default,
  so that ``(pq|rs) = sum_P L[P,p,q] L[P,r,s]``.  ``sigma = 0.05 sqrt(72 /
  naux)``: 0.05 at the (H2O)1 size (naux = 72) and scaled so that the
  diagonal and exchange-type integrals ``(pq|pq) ~ naux sigma^2 ~ 0.18`` Ha
  keep that magnitude at every size (with a fixed sigma they would grow with
  naux and the coupled-cluster iterations stop converging beyond (H2O)1).
* Dipole matrices ``mu[x|y|z, p, q]``: real symmetric ``N(0, 0.1^2)``.
* numpy ``PCG64`` with draw order eps_occ, eps_vir, L, mu_x, mu_y, mu_z.

Amplitude generators (for parity tests) draw complex amplitudes with the
closed-shell pair symmetry ``t_ij^ab = t_ji^ba`` imposed by averaging.
"""
from __future__ import annotations

import dataclasses

import numpy as np

BASE_SEED = 240718947

#: (nocc, nvir) of the (H2O)_n-sized workloads, n = 1..5.
WATER_SIZES = {1: (5, 19), 2: (10, 38), 3: (15, 57), 4: (20, 76), 5: (25, 95)}


@dataclasses.dataclass
class System:
    """Molecular-like input: canonical orbital energies, DF factors, dipoles."""

    nocc: int
    nvir: int
    eps: np.ndarray  # (nmo,) float64, occupied first
    Lfac: np.ndarray  # (naux, nmo, nmo) float64, symmetric in the last two
    dipole: np.ndarray  # (3, nmo, nmo) float64, symmetric
    seed: int

    @property
    def nmo(self) -> int:
        return self.nocc + self.nvir

    @property
    def naux(self) -> int:
        return self.Lfac.shape[0]


def make_system(nocc: int, nvir: int, naux: int | None = None, seed: int = BASE_SEED,
                eps_occ_range=(-1.5, -0.3), eps_vir_range=(0.2, 3.0),
                l_sigma: float | None = None, mu_sigma: float = 0.1) -> System:
    """Draw one synthetic closed-shell system (recipe in the module docstring)."""
    if nocc < 1 or nvir < 1:
        raise ValueError("nocc and nvir must be positive")
    nmo = nocc + nvir
    if naux is None:
        naux = 3 * nmo
    if l_sigma is None:
        l_sigma = 0.05 * np.sqrt(72.0 / naux)
    rng = np.random.Generator(np.random.PCG64(seed))
    eps_o = np.sort(rng.uniform(eps_occ_range[0], eps_occ_range[1], nocc))
    eps_v = np.sort(rng.uniform(eps_vir_range[0], eps_vir_range[1], nvir))
    iu = np.triu_indices(nmo)
    L = np.zeros((naux, nmo, nmo))
    draws = rng.normal(0.0, l_sigma, size=(naux, iu[0].size))
    L[:, iu[0], iu[1]] = draws
    L[:, iu[1], iu[0]] = draws
    mu = np.zeros((3, nmo, nmo))
    for x in range(3):
        d = rng.normal(0.0, mu_sigma, size=iu[0].size)
        mu[x, iu[0], iu[1]] = d
        mu[x, iu[1], iu[0]] = d
    return System(nocc, nvir, np.concatenate([eps_o, eps_v]), L, mu, seed)


def water_system(n: int) -> System:
    """The (H2O)_n-sized system: nocc=5n, nvir=19n, naux=3 nmo, seed BASE_SEED+n."""
    o, v = WATER_SIZES[n]
    return make_system(o, v, seed=BASE_SEED + n)


def _crandn(rng, shape, scale):
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


def random_amplitudes(nocc: int, nvir: int, seed: int, t1_scale=1e-2, t2_scale=1e-2,
                      l1_scale=2e-2, l2_scale=2e-2):
    """Complex (t1, t2, l1, l2) with t2/l2 pair symmetry ``x[i,j,a,b] = x[j,i,b,a]``.

    Layout: t1[i,a], t2[i,j,a,b], l1[i,a] (lambda_a^i), l2[i,j,a,b] (lambda_ab^ij).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    t1 = _crandn(rng, (nocc, nvir), t1_scale)
    t2 = _crandn(rng, (nocc, nocc, nvir, nvir), t2_scale)
    t2 = 0.5 * (t2 + t2.transpose(1, 0, 3, 2))
    l1 = _crandn(rng, (nocc, nvir), l1_scale)
    l2 = _crandn(rng, (nocc, nocc, nvir, nvir), l2_scale)
    l2 = 0.5 * (l2 + l2.transpose(1, 0, 3, 2))
    return t1, t2, l1, l2


def random_probe(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """A seeded complex probe vector (for finite-difference checks)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return _crandn(rng, shape, scale)


def magnetic_dipole(nmo: int, seed: int, scale: float = 0.1) -> np.ndarray:
    """Synthetic magnetic-dipole matrices m^{x,y,z} (3, nmo, nmo), complex:
    i times a real antisymmetric N(0, scale^2) matrix (the form of the
    magnetic dipole operator's matrix elements in a real orbital basis),
    from its own seeded stream (the system's draws are not affected)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.normal(0.0, scale, size=(3, nmo, nmo))
    a = a - a.transpose(0, 2, 1)
    return 1j * a
