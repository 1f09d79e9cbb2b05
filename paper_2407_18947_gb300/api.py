"""Thin Python binding over the C ABI of librtcc3 (numpy in, numpy out).

Names follow ``include/rtcc3.h``; complex arrays are numpy complex128 in the
row-major layouts documented there (t1[i,a], t2[i,j,a,b], l1[i,a], l2[i,j,a,b]).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (FIELD_COS, FIELD_GAUSS, FIELD_LRCW, FIELD_NONE, FIELD_QRCW,  # noqa: F401
                   FIELD_STATIC, PREC_BF16, PREC_FP32, PREC_FP64, PREC_TF32, RTCC3Error)


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _c128(a, shape):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    if a.shape != tuple(shape):
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


class RTCC3:
    """One librtcc3 context: ``nbatch`` field slots sharing a Hamiltonian."""

    def __init__(self, nocc: int, nvir: int, nbatch: int = 1, precision: int = PREC_FP64,
                 triples: bool = True, device: int = 0, use_graphs: bool = True,
                 field_tol: float = 0.0, field_solver: int = 0, triples_chunk: int = 0,
                 spin_budget: int = 0, eig_sweep_cap: int = 0, storage_c64: bool = False,
                 tc_scope: int = 0, checked: bool = False, serial: bool = False):
        self.lib = _lib.load()
        self.nocc, self.nvir, self.nbatch = nocc, nvir, nbatch
        opt = _lib.Options()
        self.lib.rtcc3_default_options(ctypes.byref(opt))
        opt.precision = precision
        opt.triples = 1 if triples else 0
        opt.device = device
        opt.use_graphs = 1 if use_graphs else 0
        opt.field_tol = field_tol
        opt.field_solver = field_solver
        opt.triples_chunk = triples_chunk
        opt.spin_budget = spin_budget
        opt.eig_sweep_cap = eig_sweep_cap
        opt.storage = 1 if storage_c64 else 0
        opt.tc_scope = int(tc_scope)
        opt.checked = 1 if checked else 0
        opt.serial = 1 if serial else 0
        h = ctypes.c_void_p()
        rc = self.lib.rtcc3_create(nocc, nvir, nbatch, ctypes.byref(opt), ctypes.byref(h))
        if rc != 0:
            raise RTCC3Error(rc, "rtcc3_create failed")
        self.h = h
        self._nobs = 0

    # -- plumbing ---------------------------------------------------------
    def _check(self, rc):
        if rc != 0:
            msg = self.lib.rtcc3_last_error(self.h)
            raise RTCC3Error(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "h", None):
            self.lib.rtcc3_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def shapes(self):
        o, v = self.nocc, self.nvir
        return (o, v), (o, o, v, v)

    # -- API ----------------------------------------------------------------
    def set_hamiltonian(self, eps, Lfac, dipole):
        n = self.nocc + self.nvir
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        Lfac = np.ascontiguousarray(Lfac, dtype=np.float64)
        dipole = np.ascontiguousarray(dipole, dtype=np.float64)
        if eps.shape != (n,) or Lfac.shape[1:] != (n, n) or dipole.shape != (3, n, n):
            raise ValueError("Hamiltonian arrays have the wrong shape")
        self._check(self.lib.rtcc3_set_hamiltonian(self.h, _dp(eps), Lfac.shape[0], _dp(Lfac),
                                                   _dp(dipole)))

    def set_hamiltonian_eri(self, eps, eri, dipole):
        """Hamiltonian from dense chemists' integrals (pq|rs), factored by the
        library (pivoted Cholesky, ``rtcc3_set_hamiltonian_eri``)."""
        n = self.nocc + self.nvir
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        eri = np.ascontiguousarray(eri, dtype=np.float64)
        dipole = np.ascontiguousarray(dipole, dtype=np.float64)
        if eps.shape != (n,) or eri.shape != (n, n, n, n) or dipole.shape != (3, n, n):
            raise ValueError("Hamiltonian arrays have the wrong shape")
        self._check(self.lib.rtcc3_set_hamiltonian_eri(self.h, _dp(eps), _dp(eri), _dp(dipole)))

    def set_field(self, b, kind, amplitude=0.0, omega=0.0, center=0.0, width=1.0,
                  direction=(0.0, 0.0, 1.0)):
        d = np.ascontiguousarray(direction, dtype=np.float64)
        self._check(self.lib.rtcc3_set_field(self.h, b, kind, amplitude, omega, center, width, _dp(d)))

    def set_amplitudes(self, b, t1=None, t2=None, l1=None, l2=None):
        s1, s2 = self.shapes
        arrs = [None if x is None else _c128(x, s) for x, s in ((t1, s1), (t2, s2), (l1, s1), (l2, s2))]
        self._check(self.lib.rtcc3_set_amplitudes(self.h, b, *[_dp(a) for a in arrs]))

    def get_amplitudes(self, b):
        s1, s2 = self.shapes
        out = [np.zeros(s1, np.complex128), np.zeros(s2, np.complex128),
               np.zeros(s1, np.complex128), np.zeros(s2, np.complex128)]
        self._check(self.lib.rtcc3_get_amplitudes(self.h, b, *[_dp(a) for a in out]))
        return tuple(out)

    def set_time(self, t):
        self._check(self.lib.rtcc3_set_time(self.h, t))

    def get_time(self):
        t = ctypes.c_double()
        self._check(self.lib.rtcc3_get_time(self.h, ctypes.byref(t)))
        return t.value

    def compute_residuals(self, b, time=0.0, lam=True):
        s1, s2 = self.shapes
        r = [np.zeros(s1, np.complex128), np.zeros(s2, np.complex128)]
        rl = [np.zeros(s1, np.complex128), np.zeros(s2, np.complex128)] if lam else [None, None]
        e = np.zeros(1, np.complex128)
        dip = np.zeros(3, np.complex128) if lam else None
        self._check(self.lib.rtcc3_compute_residuals(self.h, b, time, _dp(r[0]), _dp(r[1]), _dp(rl[0]),
                                                     _dp(rl[1]), _dp(e), _dp(dip)))
        return {"r_t1": r[0], "r_t2": r[1], "r_l1": rl[0], "r_l2": rl[1], "energy": complex(e[0]),
                "dipole": dip}

    def solve_ground_state(self, tol=1e-10, maxiter=500):
        self._check(self.lib.rtcc3_solve_ground_state(self.h, tol, maxiter))

    def propagate_rk4(self, h, nsteps):
        dip = np.zeros((self.nbatch, nsteps + 1, 3), np.complex128)
        en = np.zeros((self.nbatch, nsteps + 1), np.complex128)
        self._check(self.lib.rtcc3_propagate_rk4(self.h, h, nsteps, _dp(dip), _dp(en)))
        return dip, en

    def propagate_rk4_dev(self, h, nsteps, dip_ptr, en_ptr, stream_ptr=None):
        self._check(self.lib.rtcc3_propagate_rk4_dev(self.h, h, nsteps, ctypes.c_void_p(dip_ptr),
                                                     ctypes.c_void_p(en_ptr),
                                                     ctypes.c_void_p(stream_ptr or 0)))

    def propagate_rk4_chunk(self, h, nsteps):
        """nsteps RK4 steps recording the state at the start of each step only
        (entries 0..nsteps-1); the final state is entry 0 of the next chunk."""
        dip = np.zeros((self.nbatch, nsteps, 3), np.complex128)
        en = np.zeros((self.nbatch, nsteps), np.complex128)
        self._check(self.lib.rtcc3_propagate_rk4_chunk(self.h, h, nsteps, _dp(dip), _dp(en)))
        return dip, en

    def propagate_rk4_chunk_dev(self, h, nsteps, dip_ptr, en_ptr, stream_ptr=None):
        self._check(self.lib.rtcc3_propagate_rk4_chunk_dev(self.h, h, nsteps,
                                                           ctypes.c_void_p(dip_ptr),
                                                           ctypes.c_void_p(en_ptr),
                                                           ctypes.c_void_p(stream_ptr or 0)))

    def triples_forward_dev(self, b, time, t1_ptr, t2_ptr, x1_ptr, x2_ptr, stream_ptr=None):
        P = ctypes.c_void_p
        self._check(self.lib.rtcc3_triples_forward_dev(self.h, b, time, P(t1_ptr), P(t2_ptr), P(x1_ptr),
                                                       P(x2_ptr), P(stream_ptr or 0)))

    def triples_forward_noalloc_dev(self, b, time, t1_ptr, t2_ptr, x1_ptr, x2_ptr, stream_ptr=None):
        """Same as triples_forward_dev with all device workspace taken from the
        library's static 64 MiB region (no device allocation during the call)."""
        P = ctypes.c_void_p
        self._check(self.lib.rtcc3_triples_forward_noalloc_dev(self.h, b, time, P(t1_ptr), P(t2_ptr),
                                                               P(x1_ptr), P(x2_ptr), P(stream_ptr or 0)))

    def triples_vjp_dev(self, b, time, t1_ptr, t2_ptr, u1_ptr, u2_ptr, g1_ptr, g2_ptr, stream_ptr=None):
        P = ctypes.c_void_p
        self._check(self.lib.rtcc3_triples_vjp_dev(self.h, b, time, P(t1_ptr), P(t2_ptr), P(u1_ptr),
                                                   P(u2_ptr), P(g1_ptr), P(g2_ptr), P(stream_ptr or 0)))

    def get_state(self) -> bytes:
        n = ctypes.c_longlong()
        self._check(self.lib.rtcc3_state_size(self.h, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self._check(self.lib.rtcc3_get_state(self.h, buf, n.value))
        return buf.raw

    def set_state(self, data: bytes):
        buf = ctypes.create_string_buffer(data, len(data))
        self._check(self.lib.rtcc3_set_state(self.h, buf, len(data)))

    def stats(self):
        a, b = ctypes.c_longlong(), ctypes.c_longlong()
        self._check(self.lib.rtcc3_stats(self.h, ctypes.byref(a), ctypes.byref(b)))
        return {"launches": a.value, "device_bytes": b.value}

    def ground_state_history(self):
        """(T max|R| per iteration, lambda max|R| per iteration) of the last
        ground-state solve."""
        cnt, nt = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.rtcc3_ground_state_history(self.h, None, 0, ctypes.byref(cnt),
                                                        ctypes.byref(nt)))
        out = np.zeros(max(cnt.value, 1))
        self._check(self.lib.rtcc3_ground_state_history(self.h, _dp(out), cnt.value,
                                                        ctypes.byref(cnt), ctypes.byref(nt)))
        h = out[:cnt.value]
        return h[:nt.value], h[nt.value:]

    def set_observables(self, ops):
        """Additional one-electron operators (complex, (k, nmo, nmo)) whose
        expectation values sum_pq D_pq O_pq are recorded beside the dipole."""
        if ops is None or len(ops) == 0:
            self._check(self.lib.rtcc3_set_observables(self.h, 0, None))
            self._nobs = 0
            return
        a = np.ascontiguousarray(np.asarray(ops, dtype=np.complex128))
        n = self.nocc + self.nvir
        assert a.ndim == 3 and a.shape[1:] == (n, n)
        self._check(self.lib.rtcc3_set_observables(self.h, a.shape[0], _dp(a.view(np.float64))))
        self._nobs = a.shape[0]

    def get_observables(self, entries: int):
        """Values recorded by the last compute (entries = 1) or propagate call
        (entries = nbatch * (nsteps + 1)): complex array (entries, nops)."""
        out = np.zeros((entries, self._nobs), dtype=np.complex128)
        self._check(self.lib.rtcc3_get_observables(self.h, _dp(out.view(np.float64)), entries))
        return out

    def autotune_triples(self, b: int = 0):
        """Time every storage form of the triples for slot b and keep the
        fastest; returns (choice, ms, {form: ms}) with -1 = whole tensors,
        k > 0 = slabs of k occupied indices."""
        n = 32
        ch, ms, cnt = ctypes.c_int(), ctypes.c_float(), ctypes.c_int()
        cands = (ctypes.c_int * n)()
        cms = (ctypes.c_float * n)()
        self._check(self.lib.rtcc3_autotune_triples(self.h, b, ctypes.byref(ch), ctypes.byref(ms), n,
                                                    cands, cms, ctypes.byref(cnt)))
        k = min(cnt.value, n)
        return ch.value, ms.value, {int(cands[i]): float(cms[i]) for i in range(k)}

    def set_wait_budgets(self, spin_budget: int = 0, eig_sweep_cap: int = 0):
        """Wait budgets of the device kernels (0 restores a default)."""
        self._check(self.lib.rtcc3_set_wait_budgets(self.h, int(spin_budget), int(eig_sweep_cap)))

    def set_profiling(self, enable: bool):
        self._check(self.lib.rtcc3_set_profiling(self.h, 1 if enable else 0))

    def kernel_stats(self):
        """Per-kernel {name: dict(launches, ms, flops, bytes)} since profiling was enabled."""
        cnt = ctypes.c_int()
        self._check(self.lib.rtcc3_kernel_stats(self.h, None, 0, ctypes.byref(cnt)))
        arr = (_lib.KernelStat * max(cnt.value, 1))()
        self._check(self.lib.rtcc3_kernel_stats(self.h, arr, cnt.value, ctypes.byref(cnt)))
        return {arr[i].name.decode(): {"launches": arr[i].launches, "ms": arr[i].ms,
                                        "flops": arr[i].flops, "bytes": arr[i].bytes}
                for i in range(cnt.value)}


def eri_cholesky(eri, tol=1e-12, max_rank=None):
    """Pivoted Cholesky factors L[k, p, q] of dense integrals eri[p, q, r, s]
    (``rtcc3_eri_cholesky``, host only): sum_k L[k,p,q] L[k,r,s] reproduces
    every integral to within tol."""
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    n = eri.shape[0]
    if eri.shape != (n, n, n, n):
        raise ValueError("eri must have shape (n, n, n, n)")
    max_rank = n * n if max_rank is None else int(max_rank)
    L = np.zeros((max_rank, n, n), np.float64)
    rank = ctypes.c_int(0)
    lib = _lib.load()
    rc = lib.rtcc3_eri_cholesky(n, _dp(eri), float(tol), max_rank, _dp(L), ctypes.byref(rank))
    if rc != 0:
        raise RTCC3Error(rc, "rtcc3_eri_cholesky failed")
    return L[:rank.value].copy()


def measure_peaks(device: int = 0) -> dict:
    """Measured dense rates (TFLOP/s) of the device's pipes: TF32 and BF16
    tcgen05 MMA, FP32 and FP64 FMA (``rtcc3_measure_peaks``)."""
    lib = _lib.load()
    out = (ctypes.c_double * 4)()
    rc = lib.rtcc3_measure_peaks(device, out)
    if rc != 0:
        raise RTCC3Error(rc, "rtcc3_measure_peaks failed")
    return {"tf32_mma": out[0], "bf16_mma": out[1], "fp32_fma": out[2], "fp64_fma": out[3]}
