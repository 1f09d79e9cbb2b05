"""Tensor-core (tcgen05) precision modes against the FP64 oracle.

The triples contractions run on tcgen05 with TF32 or BF16 operands and FP32
accumulation; the CCSD part stays in FP32 on CUDA cores; RK4, denominators
and reductions stay in FP64.  TF32 must keep the residuals within 1e-6
max-abs of the oracle; BF16's error is measured and bounded loosely.
"""
import numpy as np
import pytest

from oracle import cc3
from paper_2407_18947_gb300.synth import random_amplitudes, water_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def w1():
    s = water_system(1)
    ham = cc3.Hamiltonian.from_system(s)
    t1, t2, l1, l2 = random_amplitudes(s.nocc, s.nvir, seed=7)
    w = ham.field_operator([0.0, 0.0, 0.002])
    ref = cc3.evaluate(ham, t1, t2, l1, l2, w)
    ref0 = cc3.evaluate(ham, t1, t2, l1, l2, w, triples=False)
    return s, (t1, t2, l1, l2), ref, ref0


def _run(s, amps, precision):
    from paper_2407_18947_gb300.api import RTCC3
    eng = RTCC3(s.nocc, s.nvir, precision=precision)
    eng.set_hamiltonian(s.eps, s.Lfac, s.dipole)
    eng.set_field(0, 1, 0.002, direction=(0, 0, 1))
    eng.set_amplitudes(0, *amps)
    got = eng.compute_residuals(0, 0.0)
    eng.close()
    return got


KEYS = ("r_t1", "r_t2", "r_l1", "r_l2")


def _errs(got, ref):
    return {k: float(np.abs(got[k] - getattr(ref, k).numpy()).max()) for k in KEYS}


def test_tf32_residuals_within_1e6(w1):
    s, amps, ref, ref0 = w1
    got = _run(s, amps, precision=2)
    errs = _errs(got, ref)
    trip = {k: float(np.abs((getattr(ref, k) - getattr(ref0, k)).numpy()).max()) for k in KEYS}
    assert all(e < 1e-6 for e in errs.values()), (errs, "triples magnitude", trip)
    assert abs(got["energy"] - ref.energy) < 1e-6
    assert np.abs(got["dipole"] - ref.dipole).max() < 1e-6


def test_bf16_residuals_bounded(w1):
    s, amps, ref, ref0 = w1
    got = _run(s, amps, precision=3)
    errs = _errs(got, ref)
    trip = {k: float(np.abs((getattr(ref, k) - getattr(ref0, k)).numpy()).max()) for k in KEYS}
    # BF16 operands (8-bit mantissa): error relative to the triples part itself
    for k in KEYS:
        assert errs[k] < 2e-2 * trip[k] + 1e-6, (k, errs, trip)


def test_tf32_matches_fp32_cuda_cores(w1):
    """The tensor-core route and the CUDA-core route agree to TF32 accuracy."""
    s, amps, ref, ref0 = w1
    a = _run(s, amps, precision=1)
    b = _run(s, amps, precision=2)
    for k in KEYS:
        assert np.abs(a[k] - b[k]).max() < 1e-6, k


def test_tf32_and_fp32_within_1e6_at_h2o2_size():
    """(H2O)2-sized system (nocc 10, nvir 38): the reduced-precision graphs
    against the complex128 graph (itself equal to the oracle to 1e-10 on the
    smaller systems), with a cos field at a nonzero time.  Long sums on the
    tensor cores accumulate in chains of bounded length, which keeps split
    TF32 at FP32 accuracy here."""
    s = water_system(2)
    amps = random_amplitudes(s.nocc, s.nvir, seed=5)
    from paper_2407_18947_gb300.api import RTCC3
    out = {}
    for prec in (0, 1, 2):
        eng = RTCC3(s.nocc, s.nvir, precision=prec)
        eng.set_hamiltonian(s.eps, s.Lfac, s.dipole)
        eng.set_field(0, 2, 0.001, omega=0.0656, direction=(0, 0, 1))
        eng.set_amplitudes(0, *amps)
        out[prec] = eng.compute_residuals(0, 3.0)
        eng.close()
    for prec in (1, 2):
        errs = {k: float(np.abs(out[prec][k] - out[0][k]).max()) for k in KEYS}
        assert all(e < 1e-6 for e in errs.values()), (prec, errs)
        assert np.abs(out[prec]["dipole"] - out[0]["dipole"]).max() < 1e-6
