"""Blocked triples (W and t3 recomputed per slab of occupied indices) on the GPU.

The blocked form never stores an o^3 v^3 tensor: the (i,j,k) blocks are
processed in slabs of ``triples_chunk`` first occupied indices, W is rebuilt
from six permuted products per slab in the forward pass and again in the
reverse pass.  It must give the oracle's residuals, lambda residuals, energy
and dipole (FP64: 1e-10 relative; split TF32: 1e-6 max-abs), whatever the
slab size, including ragged last slabs, with and without a field, in the
ground-state solve and in captured RK4 propagation.
"""
import numpy as np
import pytest

from oracle import cc3
from paper_2407_18947_gb300.synth import make_system, random_amplitudes, water_system

pytestmark = pytest.mark.gpu


def _engine(sysm, precision=0, chunk=0, nbatch=1, use_graphs=True):
    from paper_2407_18947_gb300.api import RTCC3
    eng = RTCC3(sysm.nocc, sysm.nvir, nbatch=nbatch, precision=precision,
                triples_chunk=chunk, use_graphs=use_graphs)
    eng.set_hamiltonian(sysm.eps, sysm.Lfac, sysm.dipole)
    return eng


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("ov,chunk,direction,amp", [
    ((3, 7), 1, None, 0.0),
    ((3, 7), 2, (0.0, 0.0, 1.0), 0.02),
    ((4, 11), 3, (0.3, -0.4, 1.0), 0.01),
    ((5, 19), 2, (0.0, 0.0, 1.0), 0.002),
])
def test_blocked_fp64_matches_oracle(ov, chunk, direction, amp):
    o, v = ov
    s = make_system(o, v, seed=61 + o)
    ham = cc3.Hamiltonian.from_system(s)
    t1, t2, l1, l2 = random_amplitudes(o, v, seed=8)
    eng = _engine(s, chunk=chunk)
    kind = 1 if direction else 0
    eng.set_field(0, kind, amp, direction=direction or (0, 0, 1))
    eng.set_amplitudes(0, t1, t2, l1, l2)
    got = eng.compute_residuals(0, time=0.2)
    eng.close()
    w = ham.field_operator(np.asarray(direction or (0, 0, 1)) * (amp if kind else 0.0))
    ref = cc3.evaluate(ham, t1, t2, l1, l2, w)
    for k, r in (("r_t1", ref.r_t1), ("r_t2", ref.r_t2), ("r_l1", ref.r_l1), ("r_l2", ref.r_l2)):
        assert _rel(got[k], r.numpy()) < 1e-10, k
    assert abs(got["energy"] - ref.energy) < 1e-10 * max(1.0, abs(ref.energy))
    assert _rel(got["dipole"], ref.dipole) < 1e-10


@pytest.mark.parametrize("precision,chunk,tol", [(0, 3, 1e-11), (2, 4, 1e-6), (2, 10, 1e-6)])
def test_blocked_matches_stored_at_h2o2_size(precision, chunk, tol):
    """(H2O)2 size (nocc 10, nvir 38), cos field: blocked (ragged slabs of 3
    and 4, and one slab of 10) against the stored form; FP64 relative, split
    TF32 max-abs as for the oracle comparison."""
    s = water_system(2)
    amps = random_amplitudes(s.nocc, s.nvir, seed=12)
    out = {}
    for c in (-1, chunk):
        eng = _engine(s, precision=precision, chunk=c)
        eng.set_field(0, 2, 0.001, omega=0.0656, direction=(0.0, 0.0, 1.0))
        eng.set_amplitudes(0, *amps)
        out[c] = eng.compute_residuals(0, time=0.7)
        eng.close()
    ref, got = out[-1], out[chunk]
    for k in ("r_t1", "r_t2", "r_l1", "r_l2"):
        if precision == 0:
            assert _rel(got[k], ref[k]) < tol, k
        else:
            assert np.abs(got[k] - ref[k]).max() < tol, k
    assert np.abs(np.asarray(got["dipole"]) - np.asarray(ref["dipole"])).max() < \
        (1e-12 if precision == 0 else 1e-7)


def test_blocked_tf32_matches_oracle_monomer():
    s = water_system(1)
    ham = cc3.Hamiltonian.from_system(s)
    amps = random_amplitudes(s.nocc, s.nvir, seed=13)
    eng = _engine(s, precision=2, chunk=2)
    eng.set_field(0, 1, 0.002, direction=(0.0, 0.0, 1.0))
    eng.set_amplitudes(0, *amps)
    got = eng.compute_residuals(0, 0.0)
    eng.close()
    ref = cc3.evaluate(ham, *amps, ham.field_operator([0.0, 0.0, 0.002]))
    for k, r in (("r_t1", ref.r_t1), ("r_t2", ref.r_t2), ("r_l1", ref.r_l1), ("r_l2", ref.r_l2)):
        assert np.abs(got[k] - r.numpy()).max() < 1e-6, k


def test_blocked_ground_state_and_propagation_match_stored():
    """Field-free ground state (the unrotated blocked path) and four captured
    RK4 steps under a cos field, blocked against stored, FP64."""
    s = make_system(4, 13, seed=71)
    res = {}
    for c in (-1, 3):
        eng = _engine(s, chunk=c)
        eng.solve_ground_state(tol=1e-10)
        amps = eng.get_amplitudes(0)
        eng.set_field(0, 2, 0.01, omega=0.1, direction=(0.2, 0.1, 1.0))
        dip, en = eng.propagate_rk4(0.05, 4)
        res[c] = (amps, dip, en, eng.get_amplitudes(0))
        eng.close()
    for a, b in zip(res[3][0], res[-1][0]):
        assert _rel(a, b) < 1e-9
    assert _rel(res[3][1], res[-1][1]) < 1e-10
    assert _rel(res[3][2], res[-1][2]) < 1e-10
    for a, b in zip(res[3][3], res[-1][3]):
        assert _rel(a, b) < 1e-10


def test_autotuner_times_every_form_and_keeps_a_correct_one():
    """The slab-size autotuner times the stored form and slabs of 5, 3, 2, 1
    occupied indices on a water monomer (TF32), keeps the fastest, and the
    residuals with its choice equal those of the stored form."""
    s = water_system(1)
    amps = random_amplitudes(s.nocc, s.nvir, seed=14)
    eng = _engine(s, precision=2)
    eng.set_field(0, 1, 0.002, direction=(0.0, 0.0, 1.0))
    eng.set_amplitudes(0, *amps)
    ref = eng.compute_residuals(0, 0.0)
    choice, ms, table = eng.autotune_triples(0)
    assert set(table) == {-1, 5, 3, 2, 1}
    assert choice in table and ms == min(table.values()) and ms > 0
    got = eng.compute_residuals(0, 0.0)
    eng.close()
    for k in ("r_t1", "r_t2", "r_l1", "r_l2"):
        assert np.abs(got[k] - ref[k]).max() < 1e-6, k
