"""GPU parity: librtcc3 (through the C ABI) against the FP64 CPU oracle.

FP64 mode must agree to 1e-10 relative (residuals, lambda residuals, energy,
dipole, propagated amplitudes); the FP32 residual graph to 1e-6 max-abs on
the residuals.  Sizes span several 64x64 contraction tiles and ragged tails.
"""
import numpy as np
import pytest
import torch

from oracle import cc3
from paper_2407_18947_gb300.synth import make_system, random_amplitudes, water_system

pytestmark = pytest.mark.gpu


def _engine(sysm, precision=0, nbatch=1, triples=True, use_graphs=True):
    from paper_2407_18947_gb300.api import RTCC3
    eng = RTCC3(sysm.nocc, sysm.nvir, nbatch=nbatch, precision=precision, triples=triples,
                use_graphs=use_graphs)
    eng.set_hamiltonian(sysm.eps, sysm.Lfac, sysm.dipole)
    return eng


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


CASES = [
    ((3, 7), None, 0.0),
    ((4, 11), (0.0, 0.0, 1.0), 0.02),
    ((5, 19), (0.3, -0.4, 1.0), 0.002),
]


@pytest.mark.parametrize("ov,direction,amp", CASES)
def test_residuals_fp64_match_oracle(ov, direction, amp):
    o, v = ov
    s = make_system(o, v, seed=31 + o)
    ham = cc3.Hamiltonian.from_system(s)
    t1, t2, l1, l2 = random_amplitudes(o, v, seed=5)
    eng = _engine(s)
    kind = 1 if direction else 0
    eng.set_field(0, kind, amp, direction=direction or (0, 0, 1))
    eng.set_amplitudes(0, t1, t2, l1, l2)
    got = eng.compute_residuals(0, time=0.3)
    w = ham.field_operator(np.asarray(direction or (0, 0, 1)) * (amp if kind else 0.0))
    ref = cc3.evaluate(ham, t1, t2, l1, l2, w)
    assert _rel(got["r_t1"], ref.r_t1.numpy()) < 1e-10
    assert _rel(got["r_t2"], ref.r_t2.numpy()) < 1e-10
    assert _rel(got["r_l1"], ref.r_l1.numpy()) < 1e-10
    assert _rel(got["r_l2"], ref.r_l2.numpy()) < 1e-10
    assert abs(got["energy"] - ref.energy) < 1e-10 * max(1.0, abs(ref.energy))
    assert _rel(got["dipole"], ref.dipole) < 1e-10
    eng.close()


def test_dense_integrals_match_oracle():
    """rtcc3_set_hamiltonian_eri (dense (pq|rs), factored by the library)
    against the oracle's four-index dressing of the same integrals, and
    against the DF-factor entry point of the same system, FP64, with a field."""
    o, v = 4, 11
    s = make_system(o, v, seed=77)
    eri = np.einsum('Ppq,Prs->pqrs', s.Lfac, s.Lfac)
    ham = cc3.Hamiltonian(s.eps, None, s.dipole, s.nocc, eri=eri)
    t1, t2, l1, l2 = random_amplitudes(o, v, seed=6, t1_scale=0.05)
    from paper_2407_18947_gb300.api import RTCC3
    got = {}
    for form in ("eri", "df"):
        eng = RTCC3(o, v, precision=0)
        if form == "eri":
            eng.set_hamiltonian_eri(s.eps, eri, s.dipole)
        else:
            eng.set_hamiltonian(s.eps, s.Lfac, s.dipole)
        eng.set_field(0, 1, 0.01, direction=(0.3, 0.2, 1.0))
        eng.set_amplitudes(0, t1, t2, l1, l2)
        got[form] = eng.compute_residuals(0, 0.0)
        eng.close()
    ref = cc3.evaluate(ham, t1, t2, l1, l2, ham.field_operator(np.array([0.3, 0.2, 1.0]) * 0.01))
    for k in ("r_t1", "r_t2", "r_l1", "r_l2"):
        assert _rel(got["eri"][k], getattr(ref, k).numpy()) < 1e-10, k
        assert _rel(got["eri"][k], got["df"][k]) < 1e-10, k
    assert abs(got["eri"]["energy"] - ref.energy) < 1e-10 * max(1.0, abs(ref.energy))
    assert _rel(got["eri"]["dipole"], ref.dipole) < 1e-10


def test_residuals_fp32_within_tolerance():
    o, v = 5, 19
    s = make_system(o, v, seed=40)
    ham = cc3.Hamiltonian.from_system(s)
    t1, t2, l1, l2 = random_amplitudes(o, v, seed=6)
    eng = _engine(s, precision=1)
    eng.set_field(0, 1, 0.002, direction=(0, 0, 1))
    eng.set_amplitudes(0, t1, t2, l1, l2)
    got = eng.compute_residuals(0, time=0.0)
    ref = cc3.evaluate(ham, t1, t2, l1, l2, ham.field_operator([0, 0, 0.002]))
    for k, r in (("r_t1", ref.r_t1), ("r_t2", ref.r_t2), ("r_l1", ref.r_l1), ("r_l2", ref.r_l2)):
        assert np.abs(got[k] - r.numpy()).max() < 1e-6, k
    assert abs(got["energy"] - ref.energy) < 1e-6
    eng.close()


@pytest.fixture(scope="module")
def water1():
    s = water_system(1)
    ham = cc3.Hamiltonian.from_system(s)
    y0 = cc3.solve_ground_state(ham)
    return s, ham, y0


def test_rk4_config1_fp64_matches_oracle(water1):
    """nocc=5, nvir=19, static z field 0.002 au, h = 0.01 au, from the oracle's
    converged CC3 ground state (10 steps)."""
    s, ham, y0 = water1
    field = cc3.FieldSpec(cc3.FIELD_STATIC, 0.002, direction=(0.0, 0.0, 1.0))
    nsteps = 10
    yref, dref, eref = cc3.propagate_rk4(ham, field, y0, 0.01, nsteps)
    eng = _engine(s)
    eng.set_field(0, 1, 0.002, direction=(0, 0, 1))
    eng.set_amplitudes(0, *[x.numpy() for x in y0])
    dip, en = eng.propagate_rk4(0.01, nsteps)
    assert _rel(dip[0], dref) < 1e-10
    assert np.abs(en[0] - eref).max() < 1e-10 * max(1.0, np.abs(eref).max())
    got = eng.get_amplitudes(0)
    for g, r in zip(got, yref):
        assert _rel(g, r.numpy()) < 1e-10
    eng.close()


def test_ground_state_fp64_matches_oracle(water1):
    s, ham, y0 = water1
    eng = _engine(s)
    eng.solve_ground_state(tol=1e-11, maxiter=400)
    got = eng.get_amplitudes(0)
    for g, r in zip(got, y0):
        assert np.abs(g - r.numpy()).max() < 1e-9
    eng.close()


def test_graph_replay_equals_eager(water1):
    s, ham, y0 = water1
    outs = []
    for graphs in (True, False):
        eng = _engine(s, use_graphs=graphs)
        eng.set_field(0, 2, 0.001, omega=0.0656, direction=(0, 0, 1))
        eng.set_amplitudes(0, *[x.numpy() for x in y0])
        outs.append(eng.propagate_rk4(0.01, 4))
        eng.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])


def test_checkpoint_resume_bit_identical(water1):
    s, ham, y0 = water1
    eng = _engine(s)
    eng.set_field(0, 2, 0.001, omega=0.0656, direction=(0, 0, 1))
    eng.set_amplitudes(0, *[x.numpy() for x in y0])
    eng.propagate_rk4(0.01, 2)
    snap = eng.get_state()
    d1, e1 = eng.propagate_rk4(0.01, 3)
    eng.set_state(snap)
    d2, e2 = eng.propagate_rk4(0.01, 3)
    assert np.array_equal(d1, d2) and np.array_equal(e1, e2)
    bad = bytearray(snap)
    bad[100] ^= 0xFF
    from paper_2407_18947_gb300._lib import RTCC3Error
    with pytest.raises(RTCC3Error):
        eng.set_state(bytes(bad))
    eng.close()


def test_batched_slots_match_single(water1):
    s, ham, y0 = water1
    fields = [(1, 0.002, (0, 0, 1)), (1, -0.002, (0, 0, 1)), (1, 0.002, (1, 0, 0))]
    eng = _engine(s, nbatch=3)
    for b, (k, a, d) in enumerate(fields):
        eng.set_field(b, k, a, direction=d)
        eng.set_amplitudes(b, *[x.numpy() for x in y0])
    dip, en = eng.propagate_rk4(0.01, 3)
    eng.close()
    for b, (k, a, d) in enumerate(fields):
        e1 = _engine(s)
        e1.set_field(0, k, a, direction=d)
        e1.set_amplitudes(0, *[x.numpy() for x in y0])
        d1, n1 = e1.propagate_rk4(0.01, 3)
        e1.close()
        assert np.array_equal(dip[b], d1[0]) and np.array_equal(en[b], n1[0])


@pytest.mark.parametrize("graphs", [True, False])
def test_chunked_trajectory_equals_one_call(water1, graphs):
    """Chunks of 2 + 3 + 1 steps give the 6-step trajectory of one call
    (entries 0..5) and end in the same state, to rounding: a chunk starts by
    decomposing its first stage's field eigenbasis from the state, where one
    call reuses the basis its previous step looked ahead to (the same matrix
    up to rounding)."""
    s, ham, y0 = water1
    amps = [x.numpy() for x in y0]
    eng = _engine(s, use_graphs=graphs)
    eng.set_field(0, 2, 0.002, omega=0.0656, direction=(0, 0, 1))
    eng.set_amplitudes(0, *amps)
    dip, en = eng.propagate_rk4(0.01, 6)
    end = eng.get_amplitudes(0)
    eng.set_amplitudes(0, *amps)
    eng.set_time(0.0)
    parts = [eng.propagate_rk4_chunk(0.01, n) for n in (2, 3, 1)]
    end_c = eng.get_amplitudes(0)
    eng.close()
    dc = np.concatenate([p[0] for p in parts], axis=1)
    ec = np.concatenate([p[1] for p in parts], axis=1)
    assert dc.shape == (1, 6, 3) and ec.shape == (1, 6)
    assert _rel(dc, dip[:, :6]) < 1e-12 and _rel(ec, en[:, :6]) < 1e-12
    for a, b in zip(end_c, end):
        assert _rel(a, b) < 1e-12


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (2, 1e-6)])
def test_concurrent_streams_equal_serial(water1, precision, tol):
    """The concurrent branches (the two adjoints of each CUDA-core product,
    the CCSD part beside the triples, the field-density pair) give the serial
    results: residuals of one stage and a three-step captured propagation
    (FP64 to rounding, TF32 within its stage tolerance)."""
    s, ham, y0 = water1
    amps = [x.numpy() for x in y0]
    out = {}
    for serial in (False, True):
        from paper_2407_18947_gb300.api import RTCC3
        eng = RTCC3(s.nocc, s.nvir, precision=precision, serial=serial)
        eng.set_hamiltonian(s.eps, s.Lfac, s.dipole)
        eng.set_field(0, 2, 0.002, omega=0.0656, direction=(0.2, 0.0, 1.0))
        eng.set_amplitudes(0, *amps)
        res = eng.compute_residuals(0, 0.1)
        dip, en = eng.propagate_rk4(0.01, 3)
        out[serial] = (res, dip, en)
        eng.close()
    (r0, d0, e0), (r1, d1, e1) = out[False], out[True]
    for k in ("r_t1", "r_t2", "r_l1", "r_l2"):
        if precision == 0:
            assert _rel(r0[k], r1[k]) < tol, k
        else:
            assert np.abs(r0[k] - r1[k]).max() < tol, k
    assert np.abs(d0 - d1).max() < (1e-12 if precision == 0 else 1e-7)
    assert np.abs(e0 - e1).max() < (1e-11 if precision == 0 else 1e-6)


def test_nonfinite_state_is_reported(water1):
    s, ham, y0 = water1
    eng = _engine(s)
    eng.set_amplitudes(0, *[x.numpy() * 1e3 for x in y0])
    from paper_2407_18947_gb300._lib import ERR_NONFINITE, RTCC3Error
    with pytest.raises(RTCC3Error) as ei:
        eng.propagate_rk4(50.0, 40)
    assert ei.value.code == ERR_NONFINITE
    eng.close()


def test_triples_autograd_function_matches_oracle():
    from paper_2407_18947_gb300.autograd import TriplesResidual
    o, v = 4, 9
    s = make_system(o, v, seed=12)
    ham = cc3.Hamiltonian.from_system(s)
    t1, t2, l1, l2 = random_amplitudes(o, v, seed=2)
    eng = _engine(s)
    eng.set_field(0, 1, 0.01, direction=(0, 1, 0))
    dev = torch.device("cuda")
    T1 = torch.tensor(t1, device=dev, requires_grad=True)
    T2 = torch.tensor(t2, device=dev, requires_grad=True)
    X1, X2 = TriplesResidual.apply(T1, T2, eng, 0, 0.0)
    w = ham.field_operator([0.0, 0.01, 0.0])
    r_on = cc3.forward(ham, cc3._ct(t1), cc3._ct(t2), w, True, field_on=True)
    r_off = cc3.forward(ham, cc3._ct(t1), cc3._ct(t2), w, False)
    assert _rel(X1.detach().cpu().numpy(), (r_on[0] - r_off[0]).numpy()) < 1e-10
    assert _rel(X2.detach().cpu().numpy(), (r_on[1] - r_off[1]).numpy()) < 1e-10
    # holomorphic VJP: grad of Re(sum(c1 X1) + sum(c2 X2)) = conj(c^T J)
    c1 = torch.tensor(l1, device=dev)
    c2 = torch.tensor(l2, device=dev)
    L = ((c1 * X1).sum() + (c2 * X2).sum()).real
    g1, g2 = torch.autograd.grad(L, [T1, T2])
    ref = cc3.evaluate(ham, t1, t2, l1, 2 * l2, w, triples=True)
    ref0 = cc3.evaluate(ham, t1, t2, l1, 2 * l2, w, triples=False)
    # evaluate's r_l2 = dL/dt2 + transpose with L containing 1/2 l2 . R2
    exp1 = (ref.r_l1 - ref0.r_l1).numpy()
    got1 = g1.conj().cpu().numpy()
    assert _rel(got1, exp1) < 1e-9
    got2 = g2.conj().cpu().numpy()
    got2 = got2 + got2.transpose(1, 0, 3, 2)
    exp2 = (ref.r_l2 - ref0.r_l2).numpy()
    assert _rel(got2, exp2) < 1e-9
    eng.close()


def test_residuals_fp64_match_oracle_at_h2o2_size():
    """The benchmark's system size (nocc 10, nvir 38, naux 144) with a cos
    field at a nonzero time: the complex128 path against the oracle (one
    residual evaluation with the lambda residuals and the density).  This is
    the size at which the large-gradient, small-output and field-eigenbasis
    code paths all engage."""
    s = water_system(2)
    ham = cc3.Hamiltonian.from_system(s)
    t1, t2, l1, l2 = random_amplitudes(s.nocc, s.nvir, seed=5)
    eng = _engine(s)
    eng.set_field(0, 2, 0.001, omega=0.0656, direction=(0, 0, 1))
    eng.set_amplitudes(0, t1, t2, l1, l2)
    time = 3.0
    got = eng.compute_residuals(0, time)
    field = cc3.FieldSpec(cc3.FIELD_COS, 0.001, omega=0.0656, direction=(0.0, 0.0, 1.0))
    w = ham.field_operator(field.vector(time))
    ref = cc3.evaluate(ham, t1, t2, l1, l2, w)
    for k in ("r_t1", "r_t2", "r_l1", "r_l2"):
        assert _rel(got[k], getattr(ref, k).numpy()) < 1e-10, k
    assert abs(got["energy"] - ref.energy) < 1e-10 * max(1.0, abs(ref.energy))
    assert _rel(got["dipole"], ref.dipole) < 1e-10
    eng.close()
