#!/usr/bin/env python3
"""RT-CC3 hot-path benchmark: RK4 steps/s on the (H2O)2-sized synthetic workload.

One timed step is one full RK4 step (four residual evaluations, each the
T1 dressing, CCSD residual, connected triples with field coupling, X1/X2,
energy, and the reverse pass giving the lambda residuals and the density)
plus the FP64 RK4 update, for every field slot, through librtcc3's C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp64|tf32|bf16]
                    [--impl gpu|reference] [--workload 1..5]

Under torchrun each rank propagates its own field (weak scaling, no data-path
collective); rank 0 prints one JSON line.  ``--impl reference`` times the CPU
oracle on the same workload instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RT-CC3 RK4 steps/s at (H2O)n-sized o,v; triples TFLOP/s vs GB300 peak"
UNIT = "RK4 steps/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")

# field per workload (amplitude au, omega au, kind); kind 1 static, 2 cos
WORKLOADS = {
    1: dict(n=1, kind=1, amp=0.002, omega=0.0, h=0.01),
    2: dict(n=2, kind=2, amp=0.001, omega=0.0656, h=0.01),
    3: dict(n=3, kind=1, amp=0.002, omega=0.0, h=0.01),
    4: dict(n=4, kind=1, amp=0.002, omega=0.0, h=0.01),
    5: dict(n=5, kind=1, amp=0.002, omega=0.0, h=0.01),
}
PRECISIONS = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3}
DTYPES = {"fp64": "c128 (f64)", "fp32": "c64 (f32)", "tf32": "c64 (tf32 triples, f32 acc)",
          "bf16": "c64 (bf16 triples, f32 acc)"}


def nominal_flops(o, v):
    """8 (93 o^3 v^4 + 134 o^4 v^3) real flops per RK4 step per field: the
    paper's factorised triples work (t3 and lambda3 once per stage, density
    once per step), counted at 8 flops per complex multiply-add."""
    return 8.0 * (93.0 * o ** 3 * v ** 4 + 134.0 * o ** 4 * v ** 3)


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        finally:
            os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# Profiler names (librtcc3 per-operation timing) grouped by the CUDA kernel
# that runs them, with the roofline that bounds that kernel.
KERNEL_FAMILIES = {
    "k_combine_nd": (("combine", "axpy_gather", "axpy_strided", "copy", "sym6"), "hbm"),
    # the o^3 v^3 permuted sums in the brick thread layouts (k_combine_brick
    # and its several-output form k_combine_brick_multi)
    "k_combine_brick": (("combine_brick",), "hbm"),
    "k_tc_gemm": (("contract_tc_tf32", "contract_tc_bf16"), "tensor"),
    # long sums reading the o^3 v^3 operand from its source (tcgen05, TF32
    # split): N = 10 or 38 complex columns, ~N flop per byte, HBM-bound
    "k_tc_gemm_direct": (("contract_tc_direct_tf32",), "hbm"),
    "k_outer": (("contract_outer_c64", "contract_outer_c128"), "hbm"),
    # the two outer products of the X1 / X2 adjoints in one pass
    "k_outer_pair": (("outer_pair",), "hbm"),
    "k_contract": (("contract_simt_c64", "contract_simt_c128"), "alu"),
    "k_sym6_div": (("sym6_div", "sym3_div"), "hbm"),
    "k_pack": (("tc_pack",), "hbm"),
    "k_reduce_small": (("contract_small_c64", "contract_small_c128"), "hbm"),
    "k_gemv": (("contract_gemv_c64", "contract_gemv_c128"), "hbm"),
    "k_div_eps": (("div_eps",), "hbm"),
    "k_split_reduce": (("split_reduce", "tc_split_finish"), "hbm"),
}

# DRAM bytes (read + write) per launch, averaged over the launches of one RK4
# step, from an ncu capture of this benchmark (dram__bytes_read.sum +
# dram__bytes_write.sum, one pass, full-size workload):
# (kernel, precision, workload) -> bytes.  An entry is removed when its kernel
# changes after the counters were taken.
MEASURED_TRAFFIC = {
    ("k_contract", "tf32", 2): 2.86e6,
    ("k_combine_nd", "tf32", 2): 3.61e6,
    ("k_combine_brick", "tf32", 2): 1755.6e6,
    ("k_sym6_div", "tf32", 2): 1070.54e6,
    ("k_reduce_small", "tf32", 2): 149.09e6,
    ("k_tc_gemm", "tf32", 2): 517.74e6,
    ("k_tc_gemm_direct", "tf32", 2): 485.34e6,
    ("k_outer_pair", "tf32", 2): 377.12e6,
    ("k_gemv", "tf32", 2): 221.78e6,
    ("k_pack", "tf32", 2): 2.01e6,
}


def _family_roofline(fam, st, total_ms, peaks, peak_kind, precision, workload):
    sec = st["ms"] / 1e3
    tflops = st["flops"] / sec / 1e12 if sec > 0 else 0.0
    gbs = st["bytes"] / sec / 1e9 if sec > 0 else 0.0
    bound = KERNEL_FAMILIES[fam][1]
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    if bound == "alu":
        # CUDA-core complex FMA: 152 SMs x 128 FP32 lanes x 2 flop/cycle (FP32),
        # FP64 at the GB300 nominal 1.25 TFLOP/s
        if precision == "fp64":
            peak, note = 1.25, "nominal FP64 (recipe table)"
        else:
            peak, note = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12, "152 SM x 128 FP32 lanes x 2 x max SM clock"
        rl = {"bound": "alu", "achieved": round(tflops, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
              "frac": round(tflops / peak, 4)}
    elif bound == "tensor":
        ratio = 1.1 / 2.25 if precision == "tf32" else 1.0
        peak = peaks["bf16_tflops_sustained"] * ratio
        note = f"{peak_kind} bf16 sustained x nominal dtype ratio ({'tf32' if ratio < 1 else 'bf16'})"
        rl = {"bound": "tensor", "achieved": round(tflops, 2), "peak": round(peak, 1), "unit": "TFLOP/s",
              "frac": round(tflops / peak, 4)}
    else:
        peak = peaks["hbm_gbs"]
        note = f"{peak_kind} hbm_gbs"
        rl = {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
              "frac": round(gbs / peak, 4)}
    rl["traffic"] = MEASURED_TRAFFIC.get((fam, precision, workload))
    rl.update({"kernel": fam, "peak_source": note, "launches": st["launches"],
               "avg_launch_us": round(sec / max(st["launches"], 1) * 1e6, 3),
               "share_of_step": round(st["ms"] / total_ms, 4) if total_ms > 0 else None})
    return rl


def roofline_of(stats, peaks, peak_kind, precision, workload):
    """The dominant kernel (largest summed device time over the profiled
    step) against its own roofline, plus the tensor-core kernel's when it ran."""
    if not stats:
        return None, None
    fams = {}
    for fam, (names, _) in KERNEL_FAMILIES.items():
        acc = {"launches": 0, "ms": 0.0, "flops": 0.0, "bytes": 0.0}
        for nm in names:
            if nm in stats:
                for k in acc:
                    acc[k] += stats[nm][k]
        if acc["launches"]:
            fams[fam] = acc
    total_ms = sum(v["ms"] for v in stats.values())
    dom = max(fams.items(), key=lambda kv: kv[1]["ms"])[0]
    rl = _family_roofline(dom, fams[dom], total_ms, peaks, peak_kind, precision, workload)
    if dom != "k_tc_gemm" and "k_tc_gemm" in fams:
        rl["tensor_kernel"] = _family_roofline("k_tc_gemm", fams["k_tc_gemm"], total_ms, peaks, peak_kind,
                                               precision, workload)
    return rl, dom


def oracle_stage_seconds(wl, threads=None):
    """One oracle residual evaluation (1 of the 4 RK4 stages) on the workload."""
    import torch

    from oracle import cc3
    from paper_2407_18947_gb300.synth import random_amplitudes, water_system
    # the same thread count in both arms: every host core
    torch.set_num_threads(threads or os.cpu_count() or 1)
    s = water_system(wl["n"])
    ham = cc3.Hamiltonian.from_system(s)
    t1, t2, l1, l2 = random_amplitudes(s.nocc, s.nvir, seed=1)
    w = ham.field_operator([0.0, 0.0, wl["amp"]])
    t0 = time.perf_counter()
    cc3.evaluate(ham, t1, t2, l1, l2, w)
    return time.perf_counter() - t0, torch.get_num_threads()


def run_reference(args, wl, rank):
    if rank != 0:
        return
    o, v = 5 * wl["n"], 19 * wl["n"]
    secs, cores = oracle_stage_seconds(wl)
    value = 1.0 / (4.0 * secs)
    sample = (f"one residual evaluation (1 of 4 RK4 stages: forward + Lagrangian derivatives) of the "
              f"nocc={o} nvir={v} workload, extrapolated x4 per RK4 step; the --steps/--warmup loop is "
              f"not repeated because one stage takes ~{secs:.0f} s; torch CPU einsum multi-threaded "
              f"on {cores} threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 4e3 * secs, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128 (f64, CPU)", "data": "synthetic",
            "config": workload_config(wl, "fp64", 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def rank_field_amplitude(amp, rank):
    """Each rank propagates its own field strength: independent problems,
    no data-path collective (weak scaling over field slots)."""
    return amp * (1.0 + 0.25 * rank)


def aggregate_timing(ms_local, steps, world, dist=None, device=None):
    """Max over ranks of the timed region (ms) and the whole-job RK4 steps/s
    (every rank advances its own propagation by `steps`)."""
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * steps / (ms_max / 1e3)


def workload_config(wl, precision, nbatch):
    o, v = wl.get("size", (5 * wl["n"], 19 * wl["n"]))
    field = ("static" if wl["kind"] == 1 else f"cos omega={wl['omega']} au") + f" A={wl['amp']} au along z"
    name = f"(H2O){wl['n']}-sized" if "size" not in wl else "reduced (profiling)"
    return {"workload": f"{name} RT-CC3: nocc={o} nvir={v} naux={3 * (o + v)}, {field}, "
                        f"h={wl['h']} au, T and lambda propagated",
            "nocc": o, "nvir": v, "precision": precision, "fields_per_gpu": nbatch,
            "l2": "working set larger than L2 (o^3 v^3 triples tensors)"}


def first_order_state(s):
    """First-order amplitudes of the synthetic system (an initial state for
    timing where the ground-state iterations do not converge): t2 from the
    orbital-energy denominators, lambda2 = 2 (2 t2 - t2^T) (the first-order
    multipliers in the L = E + l1 R1 + 1/2 l2 R2 normalisation)."""
    o, v = s.nocc, s.nvir
    L = np.asarray(s.Lfac)
    ov = L[:, :o, o:]
    g = np.einsum('Pia,Pjb->ijab', ov, ov, optimize=True)
    eo, ev = np.asarray(s.eps[:o]), np.asarray(s.eps[o:])
    d = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
    t2 = (g / d).astype(np.complex128)
    l2 = 2.0 * (2.0 * t2 - t2.transpose(0, 1, 3, 2))
    z1 = np.zeros((o, v), dtype=np.complex128)
    return z1, t2, z1.copy(), l2


def storage_note(o, v, prec, tune, chunk=0):
    """How the triples were held in this run (the library's automatic rule
    unless the autotuner or --triples-chunk chose)."""
    if tune:
        return dict(tune, rule="autotuned")
    if chunk:
        return {"rule": "given", "choice": "whole o^3 v^3 tensors" if chunk < 0 else
                f"slabs of {chunk} occupied indices"}
    elem = 16 if prec == 0 else 8
    t3 = o ** 3 * v ** 3 * elem
    return {"rule": "automatic", "o3v3_tensor_GB": round(t3 / 1e9, 2)}


def secondary_line(s, wl, precision, dev, stream, steps=3, warmup=1):
    """RK4 steps/s of the same workload in another precision (a short
    device-timed run from that precision's own ground state), for the
    mixed-precision versus FP64 comparison; not the headline."""
    import torch

    from paper_2407_18947_gb300.api import RTCC3
    prec = PRECISIONS[precision]
    eng = RTCC3(s.nocc, s.nvir, precision=prec)
    eng.set_hamiltonian(s.eps, s.Lfac, s.dipole)
    eng.set_field(0, wl["kind"], wl["amp"], omega=wl["omega"], direction=(0.0, 0.0, 1.0))
    t0 = time.perf_counter()
    eng.solve_ground_state(tol=1e-9 if prec == 0 else 1e-5, maxiter=400)
    t_gs = time.perf_counter() - t0
    n = max(steps, warmup) + 1
    dip = torch.zeros((1, n, 3, 2), dtype=torch.float64, device=dev)
    en = torch.zeros((1, n, 2), dtype=torch.float64, device=dev)
    eng.propagate_rk4_dev(wl["h"], warmup, dip.data_ptr(), en.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    eng.propagate_rk4_chunk_dev(wl["h"], steps, dip.data_ptr(), en.data_ptr(), stream.cuda_stream)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1)
    eng.close()
    return {"value": steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
            "warmup": warmup, "dtype": DTYPES[precision], "ground_state_s": round(t_gs, 2)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="tf32", choices=sorted(PRECISIONS))
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", type=int, default=2, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--fields", type=int, default=1,
                    help="field slots propagated together per GPU (batched in one step graph); "
                         "value then counts field-steps/s")
    ap.add_argument("--size", default=None,
                    help="nocc,nvir of a reduced same-recipe system (profiling captures only)")
    ap.add_argument("--init", default=None, choices=["cc3", "ccsd", "mp1"],
                    help="initial state: the CC3 ground state (default up to (H2O)2 size), the "
                         "CCSD ground state (default at (H2O)3 size, where the CC3 iteration costs "
                         "minutes) or first-order amplitudes (default from (H2O)4 size on, where "
                         "the synthetic system's coupled-cluster iterations do not converge)")
    ap.add_argument("--autotune", action="store_true",
                    help="time every triples storage form (whole / slabs of k occupied indices) "
                         "before the warm-up and keep the fastest (stated in config)")
    ap.add_argument("--triples-chunk", type=int, default=0,
                    help="triples storage: 0 automatic, -1 whole o^3 v^3 tensors, k > 0 slabs of k "
                         "occupied indices")
    ap.add_argument("--storage", default="c128", choices=["c128", "c64"],
                    help="propagated state kept in complex128 or rounded to complex64 every step")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64 and BF16 lines of the default workload")
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    if args.size:
        wl["size"] = tuple(int(x) for x in args.size.split(","))
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, wl, rank)
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2407_18947_gb300._lib import ERR_NONFINITE, ERR_NOT_CONVERGED, RTCC3Error
    from paper_2407_18947_gb300.api import RTCC3
    from paper_2407_18947_gb300.synth import BASE_SEED, make_system, water_system

    if "size" in wl:
        s = make_system(*wl["size"], seed=BASE_SEED + wl["n"])
    else:
        s = water_system(wl["n"])
    o, v = s.nocc, s.nvir
    prec = PRECISIONS[args.precision]
    F = max(1, args.fields)
    c64 = args.storage == "c64"
    eng = RTCC3(o, v, nbatch=F, precision=prec, device=local, storage_c64=c64,
                triples_chunk=args.triples_chunk)
    eng.set_hamiltonian(s.eps, s.Lfac, s.dipole)
    # each rank propagates its own field strength (independent problems)
    amp = rank_field_amplitude(wl["amp"], rank)
    # batched slots: the finite-field set 0, +-A, +-2A, +-4A, ... along z
    for b in range(F):
        scale = 0.0 if b == 0 else (1 << ((b - 1) // 2)) * (1.0 if b % 2 else -1.0)
        eng.set_field(b, wl["kind"], amp * (scale if F > 1 else 1.0), omega=wl["omega"],
                      direction=(0.0, 0.0, 1.0))
    def fresh_engine():
        e = RTCC3(o, v, nbatch=F, precision=prec, device=local, storage_c64=c64,
                  triples_chunk=args.triples_chunk)
        e.set_hamiltonian(s.eps, s.Lfac, s.dipole)
        for b in range(F):
            scale = 0.0 if b == 0 else (1 << ((b - 1) // 2)) * (1.0 if b % 2 else -1.0)
            e.set_field(b, wl["kind"], amp * (scale if F > 1 else 1.0), omega=wl["omega"],
                        direction=(0.0, 0.0, 1.0))
        return e

    def ccsd_start(e):
        ccsd = RTCC3(o, v, nbatch=1, precision=prec, triples=False, device=local)
        ccsd.set_hamiltonian(s.eps, s.Lfac, s.dipole)
        ccsd.solve_ground_state(tol=1e-10 if prec == 0 else 1e-5, maxiter=400)
        y = ccsd.get_amplitudes(0)
        ccsd.close()
        for b in range(F):
            e.set_amplitudes(b, *y)

    t0 = time.perf_counter()
    init = args.init or ("cc3" if wl["n"] <= 2 else ("ccsd" if wl["n"] == 3 else "mp1"))
    init_state = "CC3 ground state"
    try:
        if init == "mp1":
            init_state = ("first-order amplitudes t2 = (ia|jb) / (e_i + e_j - e_a - e_b), "
                          "lambda2 = 2 (2 t2 - t2^T), t1 = lambda1 = 0 (chosen: the synthetic "
                          "system's coupled-cluster iterations do not converge at this size)")
            y = first_order_state(s)
            for b in range(F):
                eng.set_amplitudes(b, *y)
        elif init == "ccsd":
            init_state = "CCSD ground state (chosen: the CC3 iteration costs minutes at this size)"
            ccsd_start(eng)
        else:
            eng.solve_ground_state(tol=1e-10 if prec == 0 else 1e-5, maxiter=400)
    except RTCC3Error as err:
        if err.code not in (ERR_NOT_CONVERGED, ERR_NONFINITE):
            raise
        # the CC3 amplitude iteration does not converge for every synthetic
        # system; start from the CCSD ground state then (stated in the line),
        # on a fresh context (nothing of the failed solve is reused)
        eng.close()
        eng = fresh_engine()
        ccsd_start(eng)
        init_state = "CCSD ground state (the CC3 ground-state iteration did not converge)"
    t_gs = time.perf_counter() - t0
    h = wl["h"]
    K, W = args.steps, args.warmup
    dev = torch.device("cuda", local)
    dip = torch.zeros((F, max(K, W) + 1, 3, 2), dtype=torch.float64, device=dev)
    en = torch.zeros((F, max(K, W) + 1, 2), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    y0 = eng.get_amplitudes(0)  # the initial state (re-uploaded by the e2e loop)
    tune = None
    if args.autotune:
        choice, tms, table = eng.autotune_triples(0)
        tune = {"choice": "whole o^3 v^3 tensors" if choice < 0 else f"slabs of {choice} occupied indices",
                "stage_ms": {("whole" if k < 0 else str(k)): round(v_, 2) for k, v_ in table.items()}}
    # warm-up (captures the step graph)
    try:
        eng.propagate_rk4_dev(h, W, dip.data_ptr(), en.data_ptr(), stream.cuda_stream)
    except RTCC3Error as err:
        if err.code != ERR_NONFINITE or not init_state.startswith("CC3"):
            raise
        # a CC3 amplitude solution that the propagation leaves at once (the
        # iteration can settle on a spurious root of the synthetic system):
        # restart from the CCSD ground state on a fresh context
        eng.close()
        eng = fresh_engine()
        ccsd_start(eng)
        init_state = "CCSD ground state (propagation from the CC3 amplitude solution was not finite)"
        y0 = eng.get_amplitudes(0)
        eng.propagate_rk4_dev(h, W, dip.data_ptr(), en.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("rtcc3_timed")
    ev0.record(stream)
    # K RK4 steps, each recording the dipole and energy of the state it
    # starts from (the chunked call: no extra evaluation of the final state)
    eng.propagate_rk4_chunk_dev(h, K, dip.data_ptr(), en.data_ptr(), stream.cuda_stream)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    torch.cuda.nvtx.range_pop()
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    launches = eng.stats()["launches"]
    # every field slot advances K RK4 steps: the whole job counts field-steps
    ms_max, value = aggregate_timing(ms, K * F, world, dist, dev)
    dip_h = dip.cpu().numpy()
    assert np.all(np.isfinite(dip_h[:, :K])), "non-finite dipole trajectory"

    # end to end through the host API: every step uploads the state from
    # pinned host memory, runs one RK4 step and reads back the dipole and
    # energy it records (those of the state the step starts from)
    e2e = None
    if not args.no_e2e:
        ke = max(1, min(K, 5))
        pinned = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory().numpy() for x in y0]
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(ke):
            for b in range(F):
                eng.set_amplitudes(b, *pinned)
            d_h, e_h = eng.propagate_rk4_chunk(h, 1)
        t_e2e = time.perf_counter() - t0
        h2d = F * sum(x.nbytes for x in pinned)
        d2h = d_h.nbytes + e_h.nbytes
        e2e = {"value": world * ke * F / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    # per-kernel device times (CUDA events on the library stream, eager launches)
    for b in range(F):
        eng.set_amplitudes(b, *y0)
    eng.set_profiling(True)
    eng.propagate_rk4_chunk(h, 1)
    kstats = eng.kernel_stats()
    eng.set_profiling(False)
    peaks, peak_kind = load_peaks()
    roofline, dom = roofline_of(kstats, peaks, peak_kind, args.precision,
                                wl.get("size", args.workload))
    # pipe rates of this GPU from the library's probe kernels, beside the
    # GEMM-based peaks the roofline fractions use
    from paper_2407_18947_gb300.api import measure_peaks
    probed = {k: round(v_, 2) for k, v_ in measure_peaks(local).items()}
    for rl in (roofline, (roofline or {}).get("tensor_kernel")):
        if not rl:
            continue
        key = {"alu": "fp64_fma" if args.precision == "fp64" else "fp32_fma",
               "tensor": "bf16_mma" if args.precision == "bf16" else "tf32_mma"}.get(rl["bound"])
        if key:
            rl["frac_of_probed_pipe"] = round(rl["achieved"] / probed[key], 4)
            rl["probed_pipe"] = key
    flops = nominal_flops(o, v)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and o * o * o * v * v * v * 16 > 8e9:
        cpu = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle",
               "sample": f"not run: one o^3 v^3 complex128 tensor of the full-tensor oracle takes "
                         f"{o ** 3 * v ** 3 * 16 / 1e9:.0f} GB of host memory at nocc={o} nvir={v}"}
    elif rank == 0 and world == 1 and not args.no_cpu_baseline:
        secs, cores = oracle_stage_seconds(wl)
        cpu = {"value": 1.0 / (4.0 * secs), "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"one residual evaluation (1 of 4 RK4 stages) of the same workload on the host, "
                         f"{secs:.1f} s, extrapolated x4 per RK4 step; torch CPU einsum multi-threaded "
                         f"on {cores} threads (the same count as the reference arm)"}
    extras = None
    if (rank == 0 and world == 1 and not args.no_extras and args.workload == 2 and "size" not in wl
            and args.precision == "tf32" and F == 1):
        extras = {p_: secondary_line(s, wl, p_, dev, stream) for p_ in ("fp64", "bf16")}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": DTYPES[args.precision], "data": "synthetic",
                "config": dict(workload_config(wl, args.precision, F), initial_state=init_state,
                               triples_storage=storage_note(o, v, prec, tune, args.triples_chunk),
                               state_storage=args.storage),
                "triples_tflops_nominal": round(flops * world * K * F / (ms_max / 1e3) / 1e12, 3),
                "nominal_flops_per_step": flops,
                "roofline": roofline, "peaks_probed_tflops": probed, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches),
                "clocks": clk, "ground_state_s": round(t_gs, 2),
                "kernels": {k: {"launches": v_["launches"], "ms": round(v_["ms"], 4)}
                            for k, v_ in sorted(kstats.items(), key=lambda kv: -kv[1]["ms"])}}
        if extras is not None:
            line["other_precisions"] = extras
        print(json.dumps(line), flush=True)
    eng.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
