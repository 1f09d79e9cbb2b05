"""The allocation-free triples map against the allocating one.

Callers that cannot allocate device memory at call time use
rtcc3_triples_forward_noalloc_dev, which takes all of its workspace from the
library's static device region.  It must give the same X1, X2 as
rtcc3_triples_forward_dev, on two calls in a row (the region keeps the
previous call's contents, which must not leak into the next result).  This
file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest
import torch

from paper_2407_18947_gb300.synth import make_system, random_amplitudes

pytestmark = pytest.mark.gpu


def _case(precision, o, v, seed):
    from paper_2407_18947_gb300.api import RTCC3
    s = make_system(o, v, seed=seed)
    eng = RTCC3(o, v, precision=precision)
    eng.set_hamiltonian(s.eps, s.Lfac, s.dipole)
    eng.set_field(0, 1, 0.01, direction=(0.2, 0.0, 1.0))
    t1, t2, _, _ = random_amplitudes(o, v, seed=seed + 1)
    dev = torch.device("cuda")
    T1 = torch.tensor(t1, device=dev)
    T2 = torch.tensor(t2, device=dev)
    return eng, T1, T2


def _forward(eng, T1, T2, noalloc):
    x1 = torch.empty_like(T1)
    x2 = torch.empty_like(T2)
    fn = eng.triples_forward_noalloc_dev if noalloc else eng.triples_forward_dev
    fn(0, 0.1, T1.data_ptr(), T2.data_ptr(), x1.data_ptr(), x2.data_ptr(),
       torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return x1.cpu().numpy(), x2.cpu().numpy()


# FP64 and FP32 on CUDA cores; split TF32 and BF16, at a size whose long
# triples sums (M = o*o*v = 256 rows) take the tcgen05 route, so that the
# tensor-core kernels' tensor maps, packed operands, split-K partials and
# error flag are all served from the static region
@pytest.mark.parametrize("precision,o,v,tol", [(0, 3, 7, 1e-10), (1, 4, 9, 1e-5),
                                               (2, 4, 16, 1e-5), (3, 4, 16, 1e-4)])
def test_noalloc_matches_allocating_entry_point_twice(precision, o, v, tol):
    eng, T1, T2 = _case(precision, o, v, seed=77 + o)
    r1, r2 = _forward(eng, T1, T2, noalloc=False)
    assert np.abs(r2).max() > 0
    for _ in range(2):
        if precision >= 2:
            eng.set_profiling(True)
        a1, a2 = _forward(eng, T1, T2, noalloc=True)
        if precision >= 2:
            tc = sum(st["launches"] for name, st in eng.kernel_stats().items()
                     if name.startswith("contract_tc"))
            eng.set_profiling(False)
            assert tc > 0, "no tensor-core launch in the allocation-free evaluation"
        assert np.abs(a1 - r1).max() <= tol * np.abs(r1).max()
        assert np.abs(a2 - r2).max() <= tol * np.abs(r2).max()
    eng.close()


def test_noalloc_rejects_oversized_system():
    from paper_2407_18947_gb300._lib import ERR_ARG, RTCC3Error
    eng, T1, T2 = _case(0, 9, 30, seed=5)
    with pytest.raises(RTCC3Error) as ei:
        _forward(eng, T1, T2, noalloc=True)
    assert ei.value.code == ERR_ARG and "MiB" in str(ei.value)
    eng.close()
