"""Failure detection on the GPU without a fault.

Every bounded device wait (the tensor-core kernels' pipeline barriers, the
field eigensolver's QR sweeps) gives up after a budget, drains the kernel's
own asynchronous work and returns; the call then reports RTCC3_ERR_TIMEOUT
and the context stays usable.  Here the budgets are made to run out on
purpose (a 1-cycle spin budget, a 1-sweep cap), and a later call with the
default budgets must reproduce the result of an undisturbed context.
"""
import numpy as np
import pytest

from paper_2407_18947_gb300.synth import make_system, random_amplitudes, water_system

pytestmark = pytest.mark.gpu


def _run(eng):
    got = eng.compute_residuals(0, 0.1)
    return np.concatenate([got[k].ravel() for k in ("r_t1", "r_t2", "r_l1", "r_l2")])


def _engine(s, precision):
    from paper_2407_18947_gb300.api import RTCC3
    eng = RTCC3(s.nocc, s.nvir, precision=precision, use_graphs=False)
    eng.set_hamiltonian(s.eps, s.Lfac, s.dipole)
    eng.set_field(0, 1, 0.02, direction=(0.2, 0.1, 1.0))
    eng.set_amplitudes(0, *random_amplitudes(s.nocc, s.nvir, seed=21))
    return eng


def test_eigensolver_sweep_cap_reports_timeout_and_context_recovers():
    from paper_2407_18947_gb300._lib import ERR_TIMEOUT, RTCC3Error
    s = make_system(4, 11, seed=81)
    ref_eng = _engine(s, 0)
    ref = _run(ref_eng)
    ref_eng.close()
    eng = _engine(s, 0)
    eng.set_wait_budgets(0, 1)
    with pytest.raises(RTCC3Error) as ei:
        _run(eng)
    assert ei.value.code == ERR_TIMEOUT and "QR sweeps" in str(ei.value)
    eng.set_wait_budgets(0, 0)
    got = _run(eng)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    eng.close()


def test_tensor_core_wait_budget_reports_timeout_and_context_recovers():
    from paper_2407_18947_gb300._lib import ERR_TIMEOUT, RTCC3Error
    s = water_system(1)
    ref_eng = _engine(s, 2)
    ref = _run(ref_eng)
    ref_eng.close()
    eng = _engine(s, 2)
    eng.set_wait_budgets(1, 0)
    with pytest.raises(RTCC3Error) as ei:
        _run(eng)
    assert ei.value.code == ERR_TIMEOUT and "tensor-core" in str(ei.value)
    eng.set_wait_budgets(0, 0)
    for _ in range(2):
        got = _run(eng)
        assert np.abs(got - ref).max() <= 1e-6
    eng.close()


def test_checked_mode_finds_no_overrun_and_gives_the_same_result():
    """Checked mode (a canary after every device tensor of a stage, verified
    after the stage; no CUDA graphs) on a propagation through the blocked
    triples with split TF32: no overrun is reported and the trajectory
    equals the unchecked one."""
    from paper_2407_18947_gb300.api import RTCC3
    s = water_system(1)
    amps = random_amplitudes(s.nocc, s.nvir, seed=22)
    out = []
    for checked in (False, True):
        eng = RTCC3(s.nocc, s.nvir, precision=2, triples_chunk=2, checked=checked)
        eng.set_hamiltonian(s.eps, s.Lfac, s.dipole)
        eng.set_field(0, 2, 0.002, omega=0.1, direction=(0.0, 0.0, 1.0))
        eng.set_amplitudes(0, *amps)
        out.append(np.asarray(eng.propagate_rk4(0.01, 2)[0]))
        eng.close()
    assert np.abs(out[0] - out[1]).max() < 1e-9
