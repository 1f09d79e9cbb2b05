"""Field profiles and the CCSD-only mode against the oracle (FP64, 1e-10).

Gaussian pulse (Eq. 32) and the linear / quadratic ramped continuous waves
(Section 2.2.4) over steps that cross every piece of their definitions, and
RT-CCSD (triples off, the comparison mode of the paper's tables).
"""
import numpy as np
import pytest

from oracle import cc3
from paper_2407_18947_gb300.synth import make_system, random_amplitudes

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("kind,omega,center,width", [
    (cc3.FIELD_GAUSS, 0.0, 0.05, 0.03),
    (cc3.FIELD_LRCW, 0.9, 0.0, 0.1),
    (cc3.FIELD_QRCW, 0.9, 0.0, 0.1),
])
def test_field_profiles_propagate_like_the_oracle(kind, omega, center, width):
    from paper_2407_18947_gb300.api import RTCC3
    o, v = 4, 11
    s = make_system(o, v, seed=91)
    amps = random_amplitudes(o, v, seed=92)
    direction = (0.3, -0.2, 1.0)
    eng = RTCC3(o, v, precision=0)
    eng.set_hamiltonian(s.eps, s.Lfac, s.dipole)
    eng.set_field(0, kind, 0.05, omega=omega, center=center, width=width, direction=direction)
    eng.set_amplitudes(0, *amps)
    dip, en = eng.propagate_rk4(0.04, 4)
    y = eng.get_amplitudes(0)
    eng.close()
    ham = cc3.Hamiltonian.from_system(s)
    field = cc3.FieldSpec(kind=kind, amplitude=0.05, omega=omega, center=center, width=width,
                          direction=direction)
    yr, dr, er = cc3.propagate_rk4(ham, field, amps, 0.04, 4)
    assert _rel(np.asarray(dip)[0], dr) < 1e-10
    assert _rel(np.asarray(en)[0], er) < 1e-10
    for a, b in zip(y, yr):
        assert _rel(a, b.numpy()) < 1e-10


def test_rt_ccsd_mode_matches_oracle():
    from paper_2407_18947_gb300.api import RTCC3
    o, v = 4, 11
    s = make_system(o, v, seed=93)
    amps = random_amplitudes(o, v, seed=94)
    ham = cc3.Hamiltonian.from_system(s)
    eng = RTCC3(o, v, precision=0, triples=False)
    eng.set_hamiltonian(s.eps, s.Lfac, s.dipole)
    eng.set_field(0, 2, 0.02, omega=0.3, direction=(0.0, 0.0, 1.0))
    eng.set_amplitudes(0, *amps)
    got = eng.compute_residuals(0, 0.2)
    ref = cc3.evaluate(ham, *amps, ham.field_operator([0.0, 0.0, 0.02 * np.cos(0.3 * 0.2)]),
                       triples=False)
    for k in ("r_t1", "r_t2", "r_l1", "r_l2"):
        assert _rel(got[k], getattr(ref, k).numpy()) < 1e-10, k
    assert _rel(got["dipole"], ref.dipole) < 1e-10
    eng.set_time(0.0)
    dip, _ = eng.propagate_rk4(0.05, 2)
    eng.close()
    field = cc3.FieldSpec(kind=cc3.FIELD_COS, amplitude=0.02, omega=0.3, direction=(0.0, 0.0, 1.0))
    _, dr, _ = cc3.propagate_rk4(ham, field, amps, 0.05, 2, triples=False)
    assert _rel(np.asarray(dip)[0], dr) < 1e-10


def test_complex64_storage_rounds_the_state_every_step():
    """Complex64 storage (the batched finite-field workload's amplitudes):
    after each RK4 step the state is exactly representable in complex64, and
    the trajectory stays within complex64 rounding of the complex128-state
    run of the same (FP32) graph."""
    from paper_2407_18947_gb300.api import RTCC3
    o, v = 4, 11
    s = make_system(o, v, seed=95)
    amps = random_amplitudes(o, v, seed=96)
    out = {}
    for c64 in (False, True):
        eng = RTCC3(o, v, precision=1, storage_c64=c64)
        eng.set_hamiltonian(s.eps, s.Lfac, s.dipole)
        eng.set_field(0, 1, 0.002, direction=(0.0, 0.0, 1.0))
        eng.set_amplitudes(0, *amps)
        dip, _ = eng.propagate_rk4(0.01, 5)
        out[c64] = (np.asarray(dip)[0], eng.get_amplitudes(0))
        eng.close()
    for x in out[True][1]:
        assert np.array_equal(x, x.astype(np.complex64).astype(np.complex128))
    assert not all(np.array_equal(x, x.astype(np.complex64).astype(np.complex128))
                   for x in out[False][1])
    assert np.abs(out[True][0] - out[False][0]).max() < 1e-6


def test_magnetic_moment_observable_matches_oracle_density():
    """Additional observables (the magnetic dipole of Section 2.2.3): the
    density the GPU records them with is the oracle's dL/dw, so
    sum_pq D_pq m_pq matches; and an observable equal to mu_z reproduces the
    z dipole along a propagation."""
    from paper_2407_18947_gb300.api import RTCC3
    from paper_2407_18947_gb300.synth import magnetic_dipole
    o, v = 4, 11
    s = make_system(o, v, seed=97)
    amps = random_amplitudes(o, v, seed=98)
    m = magnetic_dipole(o + v, seed=99)
    ham = cc3.Hamiltonian.from_system(s)
    eng = RTCC3(o, v, precision=0, nbatch=2)
    eng.set_hamiltonian(s.eps, s.Lfac, s.dipole)
    eng.set_observables(np.concatenate([m, s.dipole[2:3].astype(np.complex128)]))
    for b in range(2):
        eng.set_field(0 if b == 0 else 1, 2, 0.02 * (b + 1), omega=0.4, direction=(0.1, 0.0, 1.0))
        eng.set_amplitudes(b, *amps)
    eng.compute_residuals(0, 0.3)
    got = eng.get_observables(1)[0]
    w = ham.field_operator(np.asarray([0.1, 0.0, 1.0]) * 0.02 * np.cos(0.4 * 0.3))
    ref = cc3.evaluate(ham, *amps, w)
    want = np.einsum('pq,xpq->x', ref.density.numpy(), m)
    assert _rel(got[:3], want) < 1e-10
    dip, _ = eng.propagate_rk4(0.02, 3)
    obs = eng.get_observables(2 * 4).reshape(2, 4, 4)
    eng.close()
    assert _rel(obs[:, :, 3], np.asarray(dip)[:, :, 2]) < 1e-12
