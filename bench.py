#!/usr/bin/env python
"""Throughput of the phaseless-AFQMC walker step (propagate + local energy) on B300.

One "step" is one imaginary-time step of every walker (fields, force bias, VHS,
Taylor propagator with the one-body halves, overlap ratio and phaseless weight,
QR every 5th step) followed by the mixed local energy of every walker.  The
metric is walker-steps per second.

The headline workload is the paper's large molecular shape (52 electrons in 290
orbitals, 1500 Cholesky vectors, 640 walkers) stepped in FP64; the same workload in
split precision on the tensor cores, the 100-orbital workload, the batched uneven
systems, the paper's block cadence and the adjoint are reported beside it.

  python bench.py [--gpus N --steps K --warmup W] [--impl afq|reference]

With N > 1 (under torch.distributed.run) every rank runs an independent replica
of the workload with its own seed: the step does not shard, so ranks exchange
nothing on the data path; value = all ranks' walker-steps / max rank time.
"""
from __future__ import annotations

import argparse
import csv
import io
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

METRIC = "walker-steps/s/B300 (propagate+E_loc), FP64 vs mixed, |ΔE| vs FP64 oracle"
UNIT = "walker-steps/s"
WORKLOAD = "c3"
WORKLOAD_TEXT = {
    "c2": ("ph-AFQMC step + E_loc, 100 orbitals, 10a+10b electrons, 400 Cholesky vectors "
           "(geometric norm decay), 128 complex128 walkers, dt 0.005, QR every 5 steps, "
           "Philox fields"),
    "c3": ("ph-AFQMC step + E_loc, 290 orbitals, 26a+26b electrons, 1500 Cholesky vectors "
           "(geometric norm decay), 640 complex128 walkers, dt 0.005, QR every 5 steps, "
           "Philox fields"),
}
# NVIDIA's rated FP64 throughput of B300, and the FP64 ALU peak the FP64 kernels'
# roofline uses: 148 SMs x 4 flops per clock per SM (two FP64 FMA lanes, the count the
# rating implies: 1.25e12 / (148 x 2.032e9) = 4.16) x the 2032 MHz maximum SM clock
FP64_VENDOR_TFLOPS = 1.25
FP64_ALU_TFLOPS = 148 * 4 * 2.032e9 / 1e12
# DRAM bytes (read + write) of the dominant kernel class from one-pass ncu captures of
# these exact workloads: per launch for the FP64 kernels, per step (every launch of
# the class) for the split propagation; absent where no capture of the current
# kernels exists.
TRAFFIC = {("fp64", "c2", "propagate"): 34945792 + 0,
           ("fp64", "c3", "vhs"): 40650807296 + 1304730112,
           ("split_bf16", "c3", "propagate"): 7705380864 + 3032207616}
FP64_KERNELS = {"propagate": "k_propagate_fp64", "exchange": "k_exchange_v / k_exchange_fp64",
                "vhs": "k_vhs_fp64", "force_bias": "k_force_bias_fp64"}
SPLIT_KERNELS = {"propagate": "k_prop_tc (8 GEMM passes) + k_taylor_slice / k_slice_cplx1",
                 "exchange": "k_tc_split<ExVP> + k_exv_dot (stored) / k_exchange_tc (direct)",
                 "vhs": "k_slice_y + k_tc_split<VhsP> + k_slice_cplx1",
                 "force_bias": "k_tc_split<FbP> + reduction"}


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["afq", "reference"], default="afq")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="budget of the oracle CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="headline only: skip the split-precision, c2, batched, block and "
                         "adjoint legs")
    ap.add_argument("--split-steps", type=int, default=50)
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint leg")
    ap.add_argument("--profile-leg", choices=["fp64-c3", "split-c3", "fp64-c2", "split-c2",
                                              "digits7-c3", "digits7-c2",
                                              "mixed-c3", "mixed-c2", "batched",
                                              "batched-fp64", "adjoint", "blocks"],
                    default=None, help="run one leg alone and print its JSON (for ncu); "
                                       "mixed-c3 / mixed-c2 are the split-c3 / split-c2 legs")
    ap.add_argument("--mixed-steps", type=int, default=None,
                    help="timed steps of a mixed-* profile leg (default: --steps)")
    ap.add_argument("--no-mixed", action="store_true", help="the same as --no-extra")
    ap.add_argument("--profile-walkers", type=int, default=0,
                    help="walker count of a --profile-leg step leg (0: the workload's)")
    ap.add_argument("--error-steps", type=int, default=100,
                    help="steps of the split-precision drift check")
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers

def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def job_throughput(total_ms: float, units_per_rank: int, world: int, device="cpu"):
    """Whole-job throughput of independent replicas: every rank processed
    units_per_rank units; the job time is the slowest rank's (MAX over ranks, the only
    collective, outside the data path).  Returns (units per second, max ms)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    return world * units_per_rank / (total_ms / 1e3), total_ms


def host_cores() -> int:
    try:
        from threadpoolctl import threadpool_info
        return max([p.get("num_threads", 1) for p in threadpool_info()] + [1])
    except Exception:
        return os.cpu_count() or 1


def exchange_flops(W, X, M, na, nb, algorithm="direct"):
    """Algorithmic flops of the exchange for W walkers.  direct: T = L~ theta
    (4 n^2 M real flops per g and spin, real x complex) plus sum T_ij T_ji (8 n^2 flops
    per g and spin).  stored: x^T V x over the K (K + 1) / 2 distinct entries of the
    symmetric V (K = n M; real x complex, 4 flops each) plus the dot (8 K)."""
    if algorithm == "stored":
        return W * sum(2 * (n * M) * (n * M + 1) + 8 * n * M for n in (na, nb))
    return W * X * sum(n * n * (4 * M + 8) for n in (na, nb))


def stored_tc_macs(W, M, na, nb):
    """Multiply-adds of the tensor-core stored exchange: per spin the 128-row tiles of
    V' (K = n Mpad) from their diagonal block on, against the 2W theta columns."""
    Mpad = (M + 31) // 32 * 32
    total = 0
    for n in (na, nb):
        Kp = n * Mpad
        for r0 in range(0, Kp, 128):
            total += min(128, Kp - r0) * (Kp - r0) * 2 * W
    return total


def step_flops(W, X, M, na, nb, order=6, exchange="direct"):
    """Algorithmic flops of one FP64 walker step (all walkers), by kernel class."""
    N = na + nb
    Mp = M * (M + 1) // 2
    return {
        "force_bias": W * 4 * X * N * M,
        "vhs": W * 4 * X * Mp,
        # Taylor powers as 3 real products per complex multiply-add (Gauss), the two
        # real P applications as 2
        "propagate": W * (order * 6 + 2 * 4) * M * M * N,
        "overlap_theta": W * sum(4 * M * n * n + 8 * M * n * n for n in (na, nb)),
        "exchange": exchange_flops(W, X, M, na, nb, exchange),
    }


def split_flops(W, X, M, na, nb, algo, S, digits, Sp=4):
    """Digit-product flops of the split-precision tensor-core GEMMs per step, by
    kernel class: each product of an S-digit operand pair with s + t <= S - 1 counts
    the GEMM's algorithmic flops (no padding counted, except the stored exchange's
    128-row tile triangle)."""
    N = na + nb
    Mp = M * (M + 1) // 2
    prods = lambda d: d * (d + 1) // 2  # noqa: E731
    out = {"force_bias": prods(S) * 2 * X * N * M * 2 * W,
           "vhs": prods(Sp) * 2 * Mp * X * 2 * W}
    if digits:
        Sp = max(digits)
        out["vhs"] = prods(Sp) * 2 * Mp * X * 2 * W
        out["propagate"] = W * M * M * N * (4 * (prods(digits[0]) + prods(digits[-1])) +
                                            8 * sum(prods(d) for d in digits[1:-1]))
    if algo == "stored":
        out["exchange"] = prods(S) * 2 * stored_tc_macs(W, M, na, nb)
    else:
        out["exchange"] = prods(S) * exchange_flops(W, X, M, na, nb)
    return out


def algorithmic_bytes(precision, kernel, W, X, M, na, nb, digits=None):
    """Bytes the dominant kernel class must move per launch (FP64) or per step (split
    propagation, every launch of the class) if every operand were read and every
    result written once; None where not modelled.
    FP64 VHS: packed L (X M(M+1)/2 doubles) and y (W X complex) in, A (W M^2 complex)
    and Re A + Im A (W M^2 doubles) out.  FP64 propagation: A, Re A + Im A, P and Phi
    in, Phi out.  Split propagation: per GEMM pass its digit planes (V_z, 2 W M Mpad
    bf16 per digit, or O) and the operand's (2 W N Mpad per digit), the FP64 pass
    output (W N M complex) out; per slicing pass the output in, the FP64 Taylor sum
    read and written, the next digits out; the transposed copy and first slicing of
    Phi; Phi out."""
    N = na + nb
    Mpad = (M + 31) // 32 * 32
    F = W * N * M * 16
    if precision == "fp64":
        if kernel == "vhs":
            return X * (M * (M + 1) // 2) * 8 + W * X * 16 + W * M * M * 24
        if kernel == "propagate":
            return W * M * M * 24 + M * M * 8 + 2 * F
        return None
    if kernel != "propagate" or not digits:
        return None
    V, T, O = 2 * W * M * Mpad * 2, 2 * W * N * Mpad * 2, M * Mpad * 2
    n = len(digits) - 2
    total = 2 * F + F + digits[0] * T                    # transpose, Phi's digits
    total += digits[0] * (O + T) + F                     # first half
    total += 3 * F + digits[1] * T                       # its slicing pass
    for k in range(1, n + 1):
        total += digits[k] * (V + T) + F                 # Taylor pass
        total += 3 * F + digits[k + 1] * T               # slicing pass
    total += digits[-1] * (O + T) + 2 * F                # second half, Phi out
    return total


def fp64_peak() -> dict:
    """FP64 throughput of this GPU: the ALU peak from the unit count and the maximum SM
    clock (the roofline denominator of the FP64 kernels), with two measurements beside
    it: the FMA-loop probe of the library (afq_fp64_fma_rate: independent FMA chains
    filling every SM, CUDA events, best of five) and cuBLAS DGEMM (torch.matmul on
    float64, 4096^3, best of 5, CUDA events)."""
    import torch
    from paper_2209_04015_b300.afqmc import fp64_fma_rate
    fma = fp64_fma_rate(torch.cuda.current_stream().cuda_stream)
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    c = a @ b
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        c = a @ b
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b, c
    torch.cuda.empty_cache()
    return {"tflops": FP64_ALU_TFLOPS,
            "how": "ALU peak: 148 SMs x 4 FP64 flops per clock (2 FMA lanes) x 2032 MHz",
            "fma_probe_tflops": fma,
            "fma_probe_how": "afq_fp64_fma_rate (8 CTAs x 256 threads per SM, 16 independent "
                             "chains per thread), best of 5, CUDA events",
            "dgemm_tflops": 2 * n ** 3 / (best / 1e3) / 1e12,
            "dgemm_how": f"cuBLAS DGEMM {n}^3 (torch.matmul float64), best of 5, CUDA events",
            "vendor_tflops": FP64_VENDOR_TFLOPS}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = gpu_index
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = list(csv.reader(io.StringIO(open(self.path).read())))
        os.unlink(self.path)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(name: str, walkers: int, seconds: float, min_steps: int, max_steps: int,
                  seed_step: int = 0):
    """The FP64 oracle as it stands on a bounded sample of a workload: `walkers` of its
    walkers (started at the trial), steps with Philox fields, the QR cadence and the
    local energy every step, until `seconds` have passed (at least min_steps, at most
    max_steps).  Walkers are independent, so walker-steps/s of the sample carries over
    to the full walker count (the oracle loops over walkers or vectorises them).
    Returns (walker-steps/s, steps, seconds)."""
    from oracle.afqmc import Oracle
    from oracle.philox import gaussian_fields
    from paper_2209_04015_b300.synthetic import make_config, trial_walkers
    s, _ = make_config(name)
    orc = Oracle(s.h1, s.L, s.e0, s.psi_a, s.psi_b, dt=0.005, qr_period=5)
    orc.init_walkers(trial_walkers(s, walkers))
    t0 = time.perf_counter()
    steps = 0
    while True:
        orc.step(gaussian_fields(seed_step + steps, walkers, s.X, 1))
        if orc.nstep % 5 == 0:
            orc.orthogonalise()
        orc.local_energy()
        steps += 1
        el = time.perf_counter() - t0
        if steps >= max_steps or (steps >= min_steps and el > seconds):
            break
    dt = time.perf_counter() - t0
    return walkers * steps / dt, steps, dt


def cpu_baseline(name: str, seconds: float, walkers: int) -> dict:
    from paper_2209_04015_b300.synthetic import CONFIGS
    value, steps, dt = oracle_sample(name, walkers, seconds, 3, 200)
    return {"value": value, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
            "sample": f"{walkers} of the {CONFIGS[name]['W']} walkers of the {name} workload, "
                      f"{steps} steps (step + QR cadence + E_loc every step), {dt:.1f} s of "
                      "host time; walker-steps/s extrapolated to all walkers (walkers are "
                      "independent); set-up excluded"}


# ----------------------------------------------------------------------------- legs

# split precision at FP64 quality: 7 exact digits per operand everywhere (55 bits)
DIGITS7 = dict(split_slices=7, prop_slices=7)


def new_context(s, W, precision, rank, stream, autotune=True, **kw):
    from paper_2209_04015_b300 import AfqContext
    ctx = AfqContext(dt=0.005, qr_period=5, seed=1 + rank, precision=precision,
                     stream=stream.cuda_stream, **kw)
    ctx.init_hamiltonian(s.h1, s.L, s.e0)
    ctx.init_trial(s.psi_a, s.psi_b)
    ctx.init_walkers(W)
    if autotune:
        ctx.autotune()  # launch shapes (set-up, outside the timed region); walkers restored
    return ctx


def step_leg(name: str, precision: str, steps: int, warmup: int, rank: int, world: int,
             local: int, walkers: int = 0, e2e_steps: int = 0, clocks: bool = False,
             **ctx_kw) -> dict:
    """Device-timed steps (propagate + local energy of every walker) of one workload in
    one precision: W untimed warm-up steps, then `steps` steps, each between CUDA events
    on the context's stream with a 256 MB L2 flush before it (outside the events), the
    built-in per-kernel-class event profiler on; the dominant kernel class and its
    roofline; then the same metric end to end through the host-buffer C-ABI calls
    (pinned host fields in, energies out, every step) on a fresh context."""
    import torch
    from paper_2209_04015_b300.synthetic import make_config

    s, c = make_config(name, seed=1 + rank)
    W, X, M, na, nb = walkers or c["W"], s.X, s.M, s.na, s.nb
    stream = torch.cuda.current_stream()
    ctx = new_context(s, W, precision, rank, stream, **ctx_kw)
    e_dev = torch.empty((W, 4, 2), dtype=torch.float64, device="cuda")
    emix_dev = torch.empty(1, dtype=torch.float64, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def step():
        ctx.propagate_dev(None, 1)
        ctx.local_energy_dev(e_dev.data_ptr(), emix_dev.data_ptr())

    for _ in range(max(warmup, 3)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(local) if clocks else None
    if sampler:
        time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    ctx.profile_enable(True)
    n0 = ctx.launch_count()
    torch.cuda.synchronize()
    for k in range(steps):
        flush.zero_()                      # write 256 MB: evicts L2 between timed steps
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    launches = ctx.launch_count() - n0
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    clk = sampler.stop() if sampler else None
    step_ms = [a.elapsed_time(b) for a, b in ev]
    value, total_ms = job_throughput(float(sum(step_ms)), W * steps, world, device="cuda")
    algo = ctx.exchange_algorithm()
    tiles = ctx.get_tiles()
    digits = ctx.prop_digits()[0] if precision != "fp64" else None
    S = ctx.params.split_slices or 4
    Sp = ctx.params.prop_slices or 4
    ctx.close()
    del flush

    # end to end through the public host-buffer API on a fresh context (the synthetic
    # trial lies hundreds of Ha above the projected energy, so with E_shift = E_HF a
    # long-running context's weights eventually overflow -- harmless to the timed
    # kernels, which do not read them, but reported by the checked host-buffer calls)
    e2e = None
    if e2e_steps > 0:
        host_fields = torch.empty((e2e_steps + 1, W, X), dtype=torch.float64).pin_memory()
        host_fields.copy_(torch.from_numpy(
            np.random.default_rng(5 + rank).standard_normal((e2e_steps + 1, W, X))))
        hf = host_fields.numpy()
        ectx = new_context(s, W, precision, rank, stream, **ctx_kw)
        ectx.propagate(hf[0], 1)
        ectx.local_energy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(e2e_steps):
            ectx.propagate(hf[k + 1], 1)
            ectx.local_energy()
        e2e_s = time.perf_counter() - t0
        ectx.close()
        e2e_value, _ = job_throughput(e2e_s * 1e3, W * e2e_steps, world, device="cuda")
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": W * X * 8,
               "d2h_bytes_per_step": W * 4 * 16 + 8, "steps": e2e_steps,
               "api": "afq_propagate (host N(0,1) fields, pinned) + afq_local_energy (host "
                      "energies and weighted estimate) per step; host wall clock"}

    # the dominant kernel class by device time, its algorithmic rate and roofline
    kernels = {k: {"ms_per_step": v[0] / steps, "launches": v[1],
                   "share": v[0] / max(sum(x[0] for x in prof.values()), 1e-30)}
               for k, v in prof.items() if v[1]}
    names = FP64_KERNELS if precision == "fp64" else SPLIT_KERNELS
    dom = max(names, key=lambda k: prof[k][0])
    dom_ms, dom_n = prof[dom]
    out = {"workload": name, "precision": precision, "M": M, "na": na, "nb": nb, "X": X, "W": W,
           "value": value, "unit": UNIT, "ms_per_step": total_ms / steps, "steps": steps,
           "warmup": warmup, "exchange_algorithm": algo, "autotuned_tiles": tiles,
           "kernels": kernels, "gpu_launches": launches, "e2e": e2e, "clocks": clk,
           "l2": "flushed between timed steps (256 MB write, outside the step events)"}
    if precision == "fp64":
        flops = step_flops(W, X, M, na, nb, exchange=algo)
        per_launch = flops[dom] / max(dom_n / steps, 1)
        avg_s = dom_ms / max(dom_n, 1) / 1e3
        out["step_flops"] = sum(flops.values())
        out["step_tflops"] = out["step_flops"] / (out["ms_per_step"] / 1e3) / 1e12
        traffic = TRAFFIC.get(("fp64", name, dom)) if not walkers else None
        algo = algorithmic_bytes("fp64", dom, W, X, M, na, nb)
        out["roofline"] = {"bound": "alu", "kernel": f"{dom} ({FP64_KERNELS[dom]})",
                           "achieved": per_launch / avg_s / 1e12, "unit": "TFLOP/s",
                           "traffic": traffic, "algorithmic_bytes": algo,
                           "traffic_over_algorithmic": (traffic / algo
                                                        if traffic and algo else None),
                           "dram_gbs": traffic / avg_s / 1e9 if traffic else None,
                           "flops_per_launch": per_launch, "avg_launch_ms": avg_s * 1e3,
                           "per": "launch"}
    else:
        flops = split_flops(W, X, M, na, nb, algo, S, digits, Sp)
        per_step = flops[dom]
        dom_s = dom_ms / steps / 1e3
        out["prop_digits"] = digits
        out["split_slices"] = S
        out["tensor_flops_per_step"] = sum(flops.values())
        # the captured split traffic is that of the default digits (4 and 4)
        traffic = (TRAFFIC.get(("split_bf16", name, dom))
                   if not walkers and S == 4 and Sp == 4 else None)
        algo = algorithmic_bytes("split_bf16", dom, W, X, M, na, nb, digits)
        out["roofline"] = {"bound": "tensor", "kernel": f"{dom} ({SPLIT_KERNELS[dom]})",
                           "achieved": per_step / dom_s / 1e12, "unit": "TFLOP/s",
                           "traffic": traffic, "algorithmic_bytes": algo,
                           "traffic_over_algorithmic": (traffic / algo
                                                        if traffic and algo else None),
                           "dram_gbs": traffic / dom_s / 1e9 if traffic else None,
                           "flops_per_step": per_step, "ms_per_step": dom_s * 1e3,
                           "per": "step (every launch of the class, digit slicing included)",
                           "flops_note": "digit products (s + t <= S - 1 of S digits) x the "
                                         "GEMM's algorithmic flops, no padding counted"}
        out["class_rates_tflops"] = {k: flops[k] / (prof[k][0] / steps / 1e3) / 1e12
                                     for k in flops if prof.get(k, (0, 0))[0] > 0}
    return out


def attach_peak(roof: dict, peaks: dict, fp64: dict | None) -> dict:
    """Roofline denominators: measured BF16 (MEASURED_PEAKS.json, burst and sustained)
    for tensor-bound classes, the FP64 ALU peak for FP64 ones; the DRAM rate of the
    captured traffic as a fraction of the measured HBM copy bandwidth beside them."""
    hbm = peaks.get("hbm_gbs", 6400.0)
    if roof.get("dram_gbs"):
        roof["dram_frac_of_hbm"] = roof["dram_gbs"] / hbm
    if roof["bound"] == "tensor":
        burst = peaks.get("bf16_tflops", 1800.0)
        sust = peaks.get("bf16_tflops_sustained", 1400.0)
        roof.update(peak=burst, frac=roof["achieved"] / burst,
                    frac_of_sustained=roof["achieved"] / sust,
                    peak_source="MEASURED_PEAKS.json bf16_tflops (burst, measured; "
                                "bf16_tflops_sustained for frac_of_sustained)"
                    if "bf16_tflops" in peaks else "fallback 1.8 PFLOP/s bf16 burst")
        algo, fl = roof.get("algorithmic_bytes"), roof.get("flops_per_step")
        if algo and fl:
            # the roofline model: below the ridge point the class is bound by HBM, and
            # its roofline is the algorithmic bytes over the measured copy bandwidth
            intensity = fl / algo
            ridge = burst * 1e12 / (hbm * 1e9)
            attainable = min(burst, intensity * hbm * 1e9 / 1e12)
            tensor = {"achieved": roof["achieved"], "unit": "TFLOP/s", "peak": burst,
                      "frac": roof["achieved"] / burst,
                      "frac_of_sustained": roof["achieved"] / sust,
                      "attainable": attainable,
                      "frac_of_attainable": roof["achieved"] / attainable}
            roof.update(intensity_flop_per_byte=intensity, ridge_flop_per_byte=ridge)
            if intensity < ridge:
                sec = roof["ms_per_step"] / 1e3
                gbs = algo / sec / 1e9
                for k in ("frac_of_sustained",):
                    roof.pop(k, None)
                roof.update(bound="hbm", achieved=gbs, unit="GB/s", peak=hbm, frac=gbs / hbm,
                            peak_source="MEASURED_PEAKS.json hbm_gbs (copy bandwidth, "
                                        "measured)" if "hbm_gbs" in peaks
                            else "fallback 6.4 TB/s", tensor=tensor)
            else:
                roof["tensor"] = tensor
    else:
        p = fp64["tflops"]
        roof.update(peak=p, frac=roof["achieved"] / p,
                    frac_of_vendor=roof["achieved"] / FP64_VENDOR_TFLOPS,
                    frac_of_dgemm=roof["achieved"] / fp64["dgemm_tflops"],
                    frac_of_fma_probe=roof["achieved"] / fp64["fma_probe_tflops"],
                    peak_source=f"{fp64['how']} ({p:.3f} TFLOP/s); measured beside it: the "
                                f"FMA-loop probe {fp64['fma_probe_tflops']:.3f} and cuBLAS "
                                f"DGEMM {fp64['dgemm_tflops']:.3f} TFLOP/s; vendor rating "
                                f"{FP64_VENDOR_TFLOPS} TFLOP/s")
    return roof


def mixed_errors(name: str, rank: int, long_steps: int = 100, check_walkers: int = 16) -> dict:
    """Errors of the split-precision path against the FP64 path on the first walkers
    after 1 and after long_steps steps of device Philox fields.  Walkers are
    independent and the Philox counters are keyed by walker index, so an FP64 context
    holding only the first walkers sees exactly the same fields."""
    import torch
    from paper_2209_04015_b300 import AfqContext
    from paper_2209_04015_b300.synthetic import make_config

    s, c = make_config(name, seed=1 + rank)
    W = c["W"]
    stream = torch.cuda.current_stream()

    def context(precision, nw, phi=None):
        ctx = AfqContext(dt=0.005, qr_period=5, seed=1 + rank, precision=precision,
                         stream=stream.cuda_stream)
        ctx.init_hamiltonian(s.h1, s.L, s.e0)
        ctx.init_trial(s.psi_a, s.psi_b)
        ctx.init_walkers(nw, phi)
        return ctx

    def errors(mix, ref, n, gE):
        em, _ = mix.local_energy()
        er, _ = ref.local_energy()
        out = {part: float(np.max(np.abs(em[:n, i] - er[:, i])))
               for i, part in enumerate(("E1", "EJ", "EK", "E_L"))}
        wm, wr = np.abs(mix.get_weights()[:n]), np.abs(ref.get_weights())
        live = wr > 0
        out["w_rel"] = float(np.max(np.abs(wm - wr)[live] / wr[live])) if live.any() else 0.0
        om, orf = mix.get_overlaps()[:n], ref.get_overlaps()
        out["overlap_rel"] = float(np.max(np.abs(om - orf) / np.abs(orf)))
        pm, pr = mix.get_walkers()[:n], ref.get_walkers()
        out["phi_rel"] = float(np.max(np.abs(pm - pr).reshape(n, -1).max(axis=1) /
                                      np.abs(pr).reshape(n, -1).max(axis=1)))
        probe = context("fp64", n, phi=pm)
        gm, gr = probe.local_energy_backward(gE), ref.local_energy_backward(gE)
        probe.close()
        for name_, a, b in zip(("dh1", "dL", "dphi"), gm, gr):
            out[name_ + "_rel"] = float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
        return out

    mix = context("split_bf16", W)
    ref = context("fp64", check_walkers)
    rng = np.random.default_rng(5)
    gE = rng.standard_normal(check_walkers) + 1j * rng.standard_normal(check_walkers)
    errs = {}
    for k in range(1, long_steps + 1):
        mix.propagate(None, 1)
        ref.propagate(None, 1)
        if k in (1, long_steps):
            errs[k] = errors(mix, ref, check_walkers, gE)
    mix.close()
    ref.close()
    return {"after_1_step": errs[1], f"after_{long_steps}_steps": errs[long_steps],
            "dE_L_max_1_step": errs[1]["E_L"],
            f"dE_L_max_{long_steps}_steps": errs[long_steps]["E_L"],
            "reference": f"FP64 path (parity-checked against the FP64 oracle at 1e-10) on the "
                         f"first {check_walkers} of {W} walkers, same Philox fields",
            "units": "E1, EJ, EK, E_L: max |d| in Ha; *_rel: max relative error (weights, "
                     "overlaps per walker; walkers: max element difference over the walker's "
                     "largest element; gradients max |d| / max |ref|, FP64 adjoint at the "
                     "split-propagated walkers, cotangent seeded)"}


def digits7_errors(name: str, rank: int, steps: int = 20, check_walkers: int = 16,
                   digits: int = 7) -> dict:
    """The split path with `digits` exact digits everywhere (7: FP64 quality) against
    the FP64 path on the first walkers after 1 and after `steps` steps of the same
    device Philox fields: max relative error of every energy part, weight, overlap and
    walker element (walker: max element difference over the walker's largest element)."""
    import torch
    from paper_2209_04015_b300 import AfqContext
    from paper_2209_04015_b300.synthetic import make_config

    s, c = make_config(name, seed=1 + rank)
    stream = torch.cuda.current_stream()

    def context(nw, **kw):
        ctx = AfqContext(dt=0.005, qr_period=5, seed=1 + rank, stream=stream.cuda_stream, **kw)
        ctx.init_hamiltonian(s.h1, s.L, s.e0)
        ctx.init_trial(s.psi_a, s.psi_b)
        ctx.init_walkers(nw)
        return ctx

    mix = context(c["W"], precision="split_bf16", split_slices=digits, prop_slices=digits)
    ref = context(check_walkers)
    n, out = check_walkers, {}
    for k in range(1, steps + 1):
        mix.propagate(None, 1)
        ref.propagate(None, 1)
        if k in (1, steps):
            em, _ = mix.local_energy()
            er, _ = ref.local_energy()
            r = {part: float(np.max(np.abs(em[:n, i] - er[:, i]) / np.abs(er[:, i])))
                 for i, part in enumerate(("E1", "EJ", "EK", "E_L"))}
            wm, wr = mix.get_weights()[:n], ref.get_weights()
            r["w"] = float(np.max(np.abs(wm - wr) / np.abs(wr)))
            om, orf = mix.get_overlaps()[:n], ref.get_overlaps()
            r["overlap"] = float(np.max(np.abs(om - orf) / np.abs(orf)))
            pm, pr = mix.get_walkers()[:n], ref.get_walkers()
            r["phi"] = float(np.max(np.abs(pm - pr).reshape(n, -1).max(axis=1) /
                                    np.abs(pr).reshape(n, -1).max(axis=1)))
            out[f"after_{k}_steps"] = r
    mix.close()
    ref.close()
    out["reference"] = (f"FP64 path (parity-checked against the FP64 oracle at 1e-10) on the "
                        f"first {n} of {c['W']} walkers, same Philox fields; all max relative")
    return out


def block_leg(name: str, precision: str, rank: int, blocks: int = 4, block_steps: int = 25) -> dict:
    """The paper's block cadence through the native block driver (afq_run_blocks): 25
    propagation steps, then one local energy, the orthogonalisation (qr_period = 25),
    the energy-shift feedback and population control by the comb, device-event timed
    over `blocks` blocks after one warm-up block.  Context for the per-step metric,
    which evaluates the energy every step and orthogonalises every 5."""
    import torch
    from paper_2209_04015_b300 import AfqContext
    from paper_2209_04015_b300.synthetic import make_config

    s, c = make_config(name, seed=1 + rank)
    W = c["W"]
    stream = torch.cuda.current_stream()
    ctx = AfqContext(dt=0.005, qr_period=block_steps, seed=1 + rank, precision=precision,
                     stream=stream.cuda_stream)
    ctx.init_hamiltonian(s.h1, s.L, s.e0)
    ctx.init_trial(s.psi_a, s.psi_b)
    ctx.init_walkers(W)
    ctx.autotune()
    u = np.random.default_rng(7 + rank).random(blocks + 1)
    # the shift feedback keeps the weights finite: the synthetic trials lie hundreds of
    # Ha above the projected energy, so with E_shift = E_HF they grow ~e^(dt n dE) per
    # block
    ctx.run_blocks(1, block_steps, u=u[:1], shift_feedback=True)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    ctx.run_blocks(blocks, block_steps, u=u[1:], shift_feedback=True)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / blocks
    ctx.close()
    return {"workload": name, "precision": precision, "W": W, "blocks": blocks,
            "ms_per_block": ms, "value": W * block_steps / (ms / 1e3),
            "unit": "walker-steps/s at the block cadence",
            "cadence": f"{block_steps} propagation steps + 1 local energy + QR + shift "
                       "feedback + comb per block (afq_run_blocks)"}


def workflow_leg(name: str, precision: str, rank: int, blocks: int = 160, discard: int = 40,
                 block_steps: int = 25) -> dict:
    """The paper's analysis workflow on one workload: blocks of block_steps steps with
    one energy evaluation, the energy-shift feedback and the comb each, the first
    `discard` blocks dropped for equilibration and the rest reblocked
    (Flyvbjerg-Petersen, optimal level by the Lee-Needs-Drummond criterion) into an
    energy and its error bar."""
    import torch
    from paper_2209_04015_b300 import AfqContext
    from paper_2209_04015_b300.blocking import block_energies, estimate
    from paper_2209_04015_b300.synthetic import make_config

    s, c = make_config(name, seed=1 + rank)
    W = c["W"]
    stream = torch.cuda.current_stream()
    ctx = AfqContext(dt=0.005, qr_period=5, seed=1 + rank, precision=precision,
                     stream=stream.cuda_stream)
    ctx.init_hamiltonian(s.h1, s.L, s.e0)
    ctx.init_trial(s.psi_a, s.psi_b)
    ctx.init_walkers(W)
    e_trial = ctx.trial_energy()
    u = np.random.default_rng(11 + rank).random(blocks)
    t0 = time.perf_counter()
    sums = ctx.run_blocks(blocks, block_steps, u=u, shift_feedback=True)
    seconds = time.perf_counter() - t0
    _, s2_mix = ctx.spin_squared()  # the <S^2> mixed estimator on the final walkers
    t1 = time.perf_counter()
    for _ in range(5):
        ctx.spin_squared()
    s2_ms = (time.perf_counter() - t1) / 5 * 1e3
    ctx.close()
    est = estimate(block_energies(sums), discard=discard)
    return {"workload": name, "precision": precision, "W": W, "blocks": blocks,
            "discarded": discard, "steps_per_block": block_steps, "seconds": seconds,
            "energy": est.mean, "error": est.error, "reblock_level": est.level,
            "trial_energy": e_trial, "s2_mixed_final": s2_mix,
            "s2_call_ms": s2_ms,
            "note": "synthetic Hamiltonian and a random orthonormal (not self-consistent) "
                    "trial, so the projected energy lies far below the trial's: the number "
                    "shows the workflow (blocks, comb, shift feedback, reblocking), not a "
                    "physical energy"}


def batched_leg(rank: int, precision: str, replays: int) -> dict:
    """The eight uneven systems (48..220 orbitals, 0.2 M electrons per spin, X = 5 M,
    512..32 walkers) autotuned and stepped by one CUDA graph (one branch per system,
    5 steps + local energies per replay), against eager stepping of the same contexts."""
    import torch
    from paper_2209_04015_b300 import AfqBatch, AfqContext
    from paper_2209_04015_b300.synthetic import make_c4

    systems = make_c4(seed0=1 + 10 * rank)
    ctxs = []
    for k, (s, W) in enumerate(systems):
        c = AfqContext(dt=0.005, qr_period=5, seed=1 + k, precision=precision)
        c.init_hamiltonian(s.h1, s.L, s.e0)
        c.init_trial(s.psi_a, s.psi_b)
        c.init_walkers(W)
        c.autotune()
        ctxs.append(c)
    walkers = sum(W for _, W in systems)
    # eager: each system in turn, one host call per step and energy (warm up first)
    for c in ctxs:
        c.propagate(None, 5)
        c.local_energy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in ctxs:
        for _ in range(5):
            c.propagate_dev(None, 1)
            c.local_energy_dev(None, None)
    torch.cuda.synchronize()
    eager_s = (time.perf_counter() - t0) / 5
    b = AfqBatch(ctxs)
    b.capture(5)
    b.launch(1)
    b.synchronize()
    t0 = time.perf_counter()
    b.launch(replays)
    b.synchronize()
    graph_s = (time.perf_counter() - t0) / (5 * replays)
    tiles = {f"system{k}": c.get_tiles() for k, c in enumerate(ctxs)}
    b.close()
    grouped = None
    if precision == "fp64":
        # the same contexts with the VHS build and the propagation of all eight systems
        # as one persistent launch each per step (per-system descriptor table)
        bg = AfqBatch(ctxs, grouped=True)
        bg.capture(5)
        bg.launch(1)
        bg.synchronize()
        t0 = time.perf_counter()
        bg.launch(replays)
        bg.synchronize()
        grouped_s = (time.perf_counter() - t0) / (5 * replays)
        bg.close()
        grouped = {"value": walkers / grouped_s, "ms_per_step": grouped_s * 1e3,
                   "vs_per_system_graph": graph_s / grouped_s,
                   "layout": "per step: fields per system (branches), one grouped VHS and "
                             "one grouped propagation launch over all systems' tiles, the "
                             "rest per system (branches)"}
    for c in ctxs:
        c.close()
    out = {"workload": "8 uneven systems: orbitals 48..220, 0.2 M electrons per spin, "
                       f"X = 5 M, walkers 512..32, {precision}",
           "precision": precision, "walkers_total": walkers, "value": walkers / graph_s,
           "unit": UNIT, "ms_per_step": graph_s * 1e3, "eager_value": walkers / eager_s,
           "eager_ms_per_step": eager_s * 1e3, "graph_speedup": eager_s / graph_s,
           "replays": replays, "steps_per_replay": 5,
           "timing": "host wall clock around synchronised replays (graph) or eager steps",
           "autotuned_tiles": tiles}
    if grouped:
        out["grouped"] = grouped
    return out


def adjoint_leg(rank: int, K: int = 20) -> dict:
    """Adjoint on 150 orbitals, 15+15 electrons, 750 Cholesky vectors, 256 walkers:
    the local-energy backward, and a K-step chain (QR every 5 steps, Philox fields)
    forward with its checkpoint tape plus the recomputing backward."""
    import torch
    from paper_2209_04015_b300 import AfqContext
    from paper_2209_04015_b300.synthetic import make_config, perturbed_walkers

    s, c = make_config("c5", seed=1 + rank)
    W = c["W"]
    ctx = AfqContext(dt=0.005, qr_period=5, seed=1 + rank)
    ctx.init_hamiltonian(s.h1, s.L, s.e0)
    ctx.init_trial(s.psi_a, s.psi_b)
    ctx.init_walkers(W, perturbed_walkers(s, W, eps=0.3, seed=9 + rank))
    dev = torch.device("cuda")
    g = torch.ones(W, dtype=torch.complex128, device=dev)
    e = torch.empty((W, 4), dtype=torch.complex128, device=dev)
    dh1 = torch.empty((s.M, s.M), dtype=torch.float64, device=dev)
    dL = torch.empty((s.X, s.M, s.M), dtype=torch.float64, device=dev)
    dphi = torch.empty((W, s.M, s.na + s.nb), dtype=torch.complex128, device=dev)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps

    e_fwd = timed(lambda: ctx.local_energy_dev(e.data_ptr(), None), 5)
    e_bwd = timed(lambda: ctx.local_energy_backward_dev(g.data_ptr(), dh1.data_ptr(),
                                                        dL.data_ptr(), dphi.data_ptr()), 3)
    fwd = timed(lambda: ctx.chain_forward_dev(K, None, e.data_ptr()), 2)
    bwd = timed(lambda: ctx.chain_backward_dev(g.data_ptr(), dh1.data_ptr(), dL.data_ptr(),
                                               dphi.data_ptr()), 2)
    ctx.close()
    return {"workload": f"150 orbitals, 15a+15b electrons, 750 Cholesky vectors, {W} walkers, "
                        f"{K}-step chain, QR every 5 steps, FP64",
            "local_energy_ms": e_fwd * 1e3, "local_energy_backward_ms": e_bwd * 1e3,
            "chain_forward_ms": fwd * 1e3, "chain_backward_ms": bwd * 1e3,
            "backward_over_forward": bwd / fwd,
            "value": W * K / (fwd + bwd), "unit": "walker-steps/s (chain forward + backward)",
            "timing": "host wall clock around synchronised calls (device buffers)"}


# ----------------------------------------------------------------------------- arms

def run_reference(args):
    """The oracle (the reference arm of this build: the paper has no code) on the
    headline workload: each step a bounded sample of 2 of its walkers."""
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    from oracle.afqmc import Oracle
    from oracle.philox import gaussian_fields
    from paper_2209_04015_b300.synthetic import make_config, trial_walkers
    s, c = make_config(WORKLOAD)
    Ws = 2
    orc = Oracle(s.h1, s.L, s.e0, s.psi_a, s.psi_b, dt=0.005, qr_period=5)
    orc.init_walkers(trial_walkers(s, Ws))

    def one(k):
        orc.step(gaussian_fields(k, Ws, s.X, 1))
        if orc.nstep % 5 == 0:
            orc.orthogonalise()
        orc.local_energy()

    for k in range(args.warmup):
        one(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        one(args.warmup + k)
    dt = time.perf_counter() - t0
    value = Ws * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT[WORKLOAD], "name": WORKLOAD,
                       "sample_walkers": Ws},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": host_cores(),
                             "kind": "oracle",
                             "sample": f"{Ws} of {c['W']} walkers per step (walker-steps/s "
                                       "carries over: walkers are independent)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_leg(args) -> int:
    import torch
    torch.cuda.set_device(0)
    leg = args.profile_leg
    if leg.startswith(("fp64", "split", "mixed", "digits7")):
        prec, name = leg.split("-")
        steps = args.mixed_steps if prec == "mixed" and args.mixed_steps else args.steps
        out = step_leg(name, "fp64" if prec == "fp64" else "split_bf16", steps,
                       args.warmup, 0, 1, 0, walkers=args.profile_walkers,
                       **(DIGITS7 if prec == "digits7" else {}))
    elif leg.startswith("batched"):
        out = batched_leg(0, "fp64" if leg.endswith("fp64") else "split_bf16", 2)
    elif leg == "blocks":
        out = {"fp64_c2": block_leg("c2", "fp64", 0),
               "workflow_split_c2": workflow_leg("c2", "split_bf16", 0)}
    else:
        out = adjoint_leg(0)
    print(json.dumps({"leg": leg, **out}), flush=True)
    return 0


def run_afq(args):
    import torch
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    peaks = measured_peaks()
    fp64 = fp64_peak()
    e2e_steps = max(10, min(args.steps, 50))
    head = step_leg(WORKLOAD, "fp64", args.steps, args.warmup, rank, world, local,
                    e2e_steps=e2e_steps, clocks=True)
    attach_peak(head["roofline"], peaks, fp64)
    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return 0

    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Hamiltonian and trial with the paper's 52e/290o shape)",
        "config": {"workload": WORKLOAD_TEXT[WORKLOAD], "name": WORKLOAD, "M": head["M"],
                   "na": head["na"], "nb": head["nb"], "X": head["X"], "W_per_gpu": head["W"],
                   "dt": 0.005, "qr_period": 5, "precision": "fp64",
                   "parallelism": f"replicas x{world}", "l2": head["l2"]},
        "roofline": head["roofline"],
        "e2e": head["e2e"],
        "gpu_launches": head["gpu_launches"],
        "clocks": head["clocks"],
        "fp64_peak": fp64,
        "exchange_algorithm": head["exchange_algorithm"],
        "autotuned_tiles": head["autotuned_tiles"],
        "step_flops": head["step_flops"],
        "step_tflops": head["step_tflops"],
        "kernels": head["kernels"],
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(WORKLOAD, args.cpu_seconds, 2)
    if not (args.no_extra or args.no_mixed):
        split = step_leg(WORKLOAD, "split_bf16", args.split_steps, args.warmup, rank, 1, local,
                         e2e_steps=e2e_steps)
        attach_peak(split["roofline"], peaks, fp64)
        split["speedup_vs_fp64"] = split["value"] / head["value"] * world
        split["errors"] = mixed_errors(WORKLOAD, rank, args.error_steps)
        if "cpu_baseline" in line:
            split["cpu_baseline"] = dict(line["cpu_baseline"],
                                         note="the FP64 oracle (the split path's reference)")
        line["split_bf16"] = split
        d7 = step_leg(WORKLOAD, "split_bf16", args.steps, args.warmup, rank, 1, local,
                      e2e_steps=e2e_steps, **DIGITS7)
        attach_peak(d7["roofline"], peaks, fp64)
        d7["speedup_vs_fp64"] = d7["value"] / head["value"] * world
        d7["precision_note"] = ("split_bf16 with 7 exact 8-bit digits per operand (55 bits) in "
                                "every tensor-core contraction: FP64 quality, held to the FP64 "
                                "path's 1e-10 parity tests against the oracle")
        d7["errors"] = digits7_errors(WORKLOAD, rank)
        line["split_bf16_7digits"] = d7
        d6 = step_leg(WORKLOAD, "split_bf16", args.steps, args.warmup, rank, 1, local,
                      split_slices=6, prop_slices=6)
        attach_peak(d6["roofline"], peaks, fp64)
        d6["speedup_vs_fp64"] = d6["value"] / head["value"] * world
        d6["precision_note"] = ("split_bf16 with 6 exact 8-bit digits per operand (47 bits): "
                                "errors against the FP64 path at its own rounding level, held "
                                "to the FP64 path's 1e-10 parity tests against the oracle")
        d6["errors"] = digits7_errors(WORKLOAD, rank, digits=6)
        line["split_bf16_6digits"] = d6
        c2 = {}
        for prec in ("fp64", "split_bf16"):
            leg = step_leg("c2", prec, 5 * args.steps, args.warmup, rank, 1, local,
                           e2e_steps=e2e_steps)
            attach_peak(leg["roofline"], peaks, fp64)
            c2[prec] = leg
        c2["split_bf16"]["speedup_vs_fp64"] = c2["split_bf16"]["value"] / c2["fp64"]["value"]
        c2["split_bf16"]["errors"] = mixed_errors("c2", rank, args.error_steps)
        if world == 1 and not args.no_cpu_baseline:
            c2["cpu_baseline"] = cpu_baseline("c2", args.cpu_seconds / 2, 8)
        line["c2"] = c2
        line["batched"] = {"fp64": batched_leg(rank, "fp64", 2),
                           "split_bf16": batched_leg(rank, "split_bf16", 8)}
        line["paper_block"] = {"fp64_c2": block_leg("c2", "fp64", rank),
                               "split_c3": block_leg("c3", "split_bf16", rank),
                               "workflow_split_c2": workflow_leg("c2", "split_bf16", rank)}
        if not args.no_adjoint:
            line["adjoint"] = adjoint_leg(rank)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_leg:
        return run_leg(args)
    return run_afq(args)


if __name__ == "__main__":
    sys.exit(main())
