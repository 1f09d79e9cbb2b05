"""Field-coupled triples: field-dressed eigenbasis against the fixed point.

The default solver rotates the triples equation into the eigenbases of the
dressed O and V matrices (exact, no iteration); the alternative is the
paper's fixed-point iteration on the stored triples.  Both must reproduce
the FP64 oracle (which iterates on the full tensor) with fields strong enough
to matter, including non-Hermitian dressed couplings (t1 != 0) and several
field directions.
"""
import numpy as np
import pytest

from oracle import cc3
from paper_2407_18947_gb300.synth import make_system, random_amplitudes

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("ov,amp,direction", [((3, 7), 0.05, (0.3, -0.2, 1.0)),
                                              ((4, 11), 0.02, (1.0, 0.5, 0.0))])
def test_field_solvers_match_oracle(solver, ov, amp, direction):
    from paper_2407_18947_gb300.api import RTCC3
    o, v = ov
    s = make_system(o, v, seed=50 + o)
    ham = cc3.Hamiltonian.from_system(s)
    t1, t2, l1, l2 = random_amplitudes(o, v, seed=9, t1_scale=0.05)
    eng = RTCC3(o, v, precision=0, field_solver=solver)
    eng.set_hamiltonian(s.eps, s.Lfac, s.dipole)
    eng.set_field(0, 1, amp, direction=direction)
    eng.set_amplitudes(0, t1, t2, l1, l2)
    got = eng.compute_residuals(0, 0.0)
    w = ham.field_operator(np.asarray(direction) * amp)
    ref = cc3.evaluate(ham, t1, t2, l1, l2, w)
    for k in ("r_t1", "r_t2", "r_l1", "r_l2"):
        assert _rel(got[k], getattr(ref, k).numpy()) < 1e-10, k
    assert abs(got["energy"] - ref.energy) < 1e-10
    assert _rel(got["dipole"], ref.dipole) < 1e-10
    eng.close()


def test_rotated_solver_propagation_fp32_matches_fixed_point():
    """Complex64 graph: both solvers give the same trajectory to FP32 accuracy."""
    from paper_2407_18947_gb300.api import RTCC3
    s = make_system(4, 12, seed=3)
    t1, t2, l1, l2 = random_amplitudes(4, 12, seed=4)
    out = []
    for solver in (0, 1):
        eng = RTCC3(4, 12, precision=1, field_solver=solver)
        eng.set_hamiltonian(s.eps, s.Lfac, s.dipole)
        eng.set_field(0, 2, 0.01, omega=0.1, direction=(0, 0, 1))
        eng.set_amplitudes(0, t1, t2, l1, l2)
        out.append(eng.propagate_rk4(0.01, 3)[0])
        eng.close()
    assert _rel(out[0], out[1]) < 1e-5
