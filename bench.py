#!/usr/bin/env python
"""Throughput of the phaseless-AFQMC walker step (propagate + local energy) on B300.

One "step" is one imaginary-time step of every walker (fields, force bias, VHS,
Taylor propagator with the one-body halves, overlap ratio and phaseless weight,
QR every 5th step) followed by the mixed local energy of every walker.  The
metric is walker-steps per second.

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
WORKLOAD = "c2"
WORKLOAD_TEXT = ("ph-AFQMC step + E_loc, 100 orbitals, 10a+10b electrons, 400 Cholesky "
                 "vectors (geometric norm decay), 128 complex128 walkers, dt 0.005, QR every "
                 "5 steps, Philox fields")
FP64_NOMINAL_TFLOPS = 1.25  # B300 FP64 nominal: 148 SMs x 2032 MHz x ~4.15 flop/clk/SM
# DRAM bytes (read + write) per launch of the dominant kernel, from ncu captures of
# these exact workloads (profiles/propagation_fp64_c2.md, profiles/exchange_tc_c3.md);
# absent where no capture of the current kernel exists.
TRAFFIC = {("split_bf16", "c3", "exchange_direct"): 572279808 + 10032128,
           ("fp64", "c2", "propagate"): 34943232 + 16384}  # captured with 2 columns per CTA
FP64_KERNELS = {"propagate": "k_propagate_fp64", "exchange": "k_exchange_v / k_exchange_fp64",
                "vhs": "k_vhs_fp64", "force_bias": "k_force_bias_fp64"}
SPLIT_PRODUCTS = 6          # bf16 slice products of 3 slices or digits (s + t <= 2)


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["afq", "reference"], default="afq")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="budget of the oracle CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the split-precision legs")
    ap.add_argument("--mixed-steps", type=int, default=20)
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint leg")
    ap.add_argument("--profile-leg", choices=["mixed-c2", "mixed-c3", "batched", "adjoint",
                                              "blocks"],
                    default=None, help="run one secondary leg alone and print its JSON (for ncu)")
    ap.add_argument("--profile-walkers", type=int, default=0,
                    help="walker count of a --profile-leg mixed leg (0: the workload's)")
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
    """Algorithmic flops of one walker step (all walkers), by part."""
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


def cpu_baseline(seconds: float, W_sample: int = 8) -> dict:
    """The FP64 oracle as it stands, on a bounded sample of the same workload."""
    from oracle.afqmc import Oracle
    from oracle.philox import gaussian_fields
    from paper_2209_04015_b300.synthetic import make_config, trial_walkers
    s, c = make_config(WORKLOAD)
    orc = Oracle(s.h1, s.L, s.e0, s.psi_a, s.psi_b, dt=0.005, qr_period=5)
    orc.init_walkers(trial_walkers(s, W_sample))
    t0 = time.perf_counter()
    steps = 0
    while True:
        xi = gaussian_fields(steps, W_sample, s.X, 1)
        orc.step(xi)
        if orc.nstep % 5 == 0:
            orc.orthogonalise()
        orc.local_energy()
        steps += 1
        if time.perf_counter() - t0 > seconds or steps >= 200:
            break
    dt = time.perf_counter() - t0
    try:
        from threadpoolctl import threadpool_info
        cores = max([p.get("num_threads", 1) for p in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count() or 1
    return {"value": W_sample * steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{W_sample} of the {c['W']} walkers of the {WORKLOAD} workload, "
                      f"{steps} steps (step + QR cadence + E_loc), {dt:.1f} s of host time"}


def fp64_step_ms(s, W: int, rank: int, steps: int = 2) -> float:
    """Event-timed FP64 step + local energy on the same system (all walkers)."""
    import torch
    from paper_2209_04015_b300 import AfqContext
    stream = torch.cuda.current_stream()
    ctx = AfqContext(dt=0.005, qr_period=5, seed=1 + rank, stream=stream.cuda_stream)
    ctx.init_hamiltonian(s.h1, s.L, s.e0)
    ctx.init_trial(s.psi_a, s.psi_b)
    ctx.init_walkers(W)
    ctx.propagate_dev(None, 1)
    ctx.local_energy_dev(None, None)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        ctx.propagate_dev(None, 1)
        ctx.local_energy_dev(None, None)
    b.record(stream)
    torch.cuda.synchronize()
    ctx.close()
    return a.elapsed_time(b) / steps


def block_leg(name: str, precision: str, rank: int, blocks: int = 4, block_steps: int = 25) -> dict:
    """The paper's block cadence through the native block driver (afq_run_blocks): 25
    propagation steps, then one local energy, the orthogonalisation (qr_period = 25),
    the energy-shift feedback and population control by the comb, device-event timed
    over `blocks` blocks after one warm-up block.  Context for the per-step metric, which evaluates the energy
    every step and orthogonalises every 5."""
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


def mixed_leg(name: str, steps: int, warmup: int, rank: int, check_walkers: int = 16,
              long_steps: int = 100, walkers: int = 0, fp64_compare: bool = False) -> dict:
    """Split-precision (tcgen05) throughput on one workload, and its errors against
    the FP64 path on the first walkers after 1 and after long_steps steps.  Walkers
    are independent and the Philox counters are keyed by walker index, so an FP64
    context holding only the first walkers sees exactly the same fields."""
    long_steps = max(long_steps, 0)  # 0: no drift check (no FP64 reference context)
    import torch
    from paper_2209_04015_b300 import AfqContext
    from paper_2209_04015_b300.synthetic import make_config

    s, c = make_config(name, seed=1 + rank)
    W, X, M, na, nb = walkers or c["W"], s.X, s.M, s.na, s.nb
    check_walkers = min(check_walkers, W)
    stream = torch.cuda.current_stream()

    def context(precision, nw, phi=None):
        ctx = AfqContext(dt=0.005, qr_period=5, seed=1 + rank, precision=precision,
                         stream=stream.cuda_stream)
        ctx.init_hamiltonian(s.h1, s.L, s.e0)
        ctx.init_trial(s.psi_a, s.psi_b)
        ctx.init_walkers(nw, phi)
        return ctx

    def split_errors(mix, ref, n, gE):
        """Errors of the split-precision walkers against the FP64 path (first n walkers):
        max |dE| per energy part (Ha), max relative error of weights, overlaps and
        walker matrices, and of the local-energy gradients, which the FP64 adjoint
        (the one a split context runs) gives at the split-propagated walkers against
        those at the FP64-propagated ones (max |d| / max |ref| per output)."""
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
        out["phi_rel"] = float(np.max(np.linalg.norm((pm - pr).reshape(n, -1), axis=1) /
                                      np.linalg.norm(pr.reshape(n, -1), axis=1)))
        probe = context("fp64", n, phi=pm)
        gm, gr = probe.local_energy_backward(gE), ref.local_energy_backward(gE)
        probe.close()
        for name_, a, b in zip(("dh1", "dL", "dphi"), gm, gr):
            out[name_ + "_rel"] = float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
        return out

    mix = context("split_bf16", W)
    errs = {1: None, long_steps: None}
    if long_steps > 0:
        ref = context("fp64", check_walkers)
        rng = np.random.default_rng(5)
        gE = rng.standard_normal(check_walkers) + 1j * rng.standard_normal(check_walkers)
        for k in range(1, long_steps + 1):
            mix.propagate(None, 1)
            ref.propagate(None, 1)
            if k in (1, long_steps):
                errs[k] = split_errors(mix, ref, check_walkers, gE)
        ref.close()
    e_dev = torch.empty((W, 4, 2), dtype=torch.float64, device="cuda")
    emix_dev = torch.empty(1, dtype=torch.float64, device="cuda")

    def step():
        mix.propagate_dev(None, 1)
        mix.local_energy_dev(e_dev.data_ptr(), emix_dev.data_ptr())

    for _ in range(max(warmup, 3)):
        step()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    mix.profile_enable(True)
    n0 = mix.launch_count()
    ev0.record(stream)
    for _ in range(steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    prof = mix.profile_read()
    mix.profile_enable(False)
    ms = ev0.elapsed_time(ev1) / steps
    algo = mix.exchange_algorithm()
    digits, xest = mix.prop_digits()
    ex_ms, ex_n = prof["exchange"]
    ex_avg = ex_ms / max(ex_n, 1) / 1e3
    if algo == "stored":
        useful = 2 * stored_tc_macs(W, M, na, nb)
        kname = "exchange (k_tc_split<ExVP>: stored V' x theta, exact digits)"
        note = (f"{SPLIT_PRODUCTS} digit products x 2 x the multiply-adds of the upper block "
                "triangle of V' against theta (padding of M to 32 counted)")
    else:
        useful = exchange_flops(W, X, M, na, nb)
        kname = "exchange (k_exchange_tc, persistent, direct)"
        note = (f"{SPLIT_PRODUCTS} bf16 slice products x the exchange's algorithmic flops "
                "(no padding counted)")
    bf16_flops = SPLIT_PRODUCTS * useful
    peak = measured_peaks().get("bf16_tflops", 1800.0)
    achieved = bf16_flops / ex_avg / 1e12
    out = {"workload": name, "M": M, "na": na, "nb": nb, "X": X, "W": W,
           "value": W / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
           "precision": ("split_bf16: force bias 3 exact 8-bit digits per operand (6 products, "
                         "exact integer sums in TMEM); exchange " +
                         ("stored V' and theta as 3 exact digits (6 products)" if algo == "stored"
                          else "direct, 3 bf16 float slices (6 products, FP32 accumulation)") +
                         "; VHS 4 exact digits; propagator 4 exact digits for the P passes "
                         "and the leading powers, fewer for the small high powers "
                         "(prop_digits); theta double-float; overlaps, inverses, QR and "
                         "weights FP64"),
           "exchange_algorithm": algo,
           "prop_digits": {"per_pass": digits, "sqrt_dt_V2_estimate": xest,
                           "passes": "first P, Taylor powers 1..n, last P"},
           "dE_L_max_1_step": errs[1] and errs[1]["E_L"],
           f"dE_L_max_{long_steps}_steps": errs[long_steps] and errs[long_steps]["E_L"],
           "errors": {"after_1_step": errs[1], f"after_{long_steps}_steps": errs[long_steps],
                      "units": "E1, EJ, EK, E_L: max |d| in Ha; *_rel: max relative error "
                               "(weights, overlaps per walker; walkers Frobenius per walker; "
                               "gradients max |d| / max |ref|, FP64 adjoint at the "
                               "split-propagated walkers, cotangent seeded)"},
           "dE_reference": f"FP64 path (parity-checked against the FP64 oracle at 1e-10) on the "
                           f"first {check_walkers} walkers, same Philox fields",
           "gpu_launches": mix.launch_count() - n0,
           "kernels": {k: {"ms_per_step": v[0] / steps, "launches": v[1]}
                       for k, v in prof.items() if v[1]},
           "roofline": {"bound": "tensor", "kernel": kname,
                        "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": achieved / peak,
                        "traffic": (TRAFFIC.get(("split_bf16", name, "exchange_" + algo))
                                    if W == c["W"] else None),
                        "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst, measured)",
                        "flops_per_launch": bf16_flops, "flops_note": note,
                        "avg_launch_ms": ex_avg * 1e3}}
    # the propagation (the split step's largest part): every digit product of the 8 GEMM
    # passes at its algorithmic flops, over the propagation's event time (which also
    # holds the digit slicing between the passes)
    pr_ms, _ = prof["propagate"]
    pr_s = pr_ms / steps / 1e3
    N = na + nb
    prods = [d * (d + 1) // 2 for d in digits]
    pr_flops = W * M * M * N * (4 * (prods[0] + prods[-1]) + 8 * sum(prods[1:-1]))
    pr_achieved = pr_flops / pr_s / 1e12
    out["propagation_roofline"] = {
        "bound": "tensor", "kernel": "propagation (k_prop_tc, 8 passes per step, with the "
                                     "digit slicing between them)",
        "achieved": pr_achieved, "peak": peak, "unit": "TFLOP/s", "frac": pr_achieved / peak,
        "traffic": None, "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst, measured)",
        "flops_per_step": pr_flops,
        "flops_note": "digit products of each pass (d (d + 1) / 2 for d digits) x 8 M^2 N "
                      "(complex Taylor powers) or 4 M^2 N (real P passes), no padding",
        "ms_per_step": pr_s * 1e3}
    mix.close()
    if fp64_compare:
        f_ms = fp64_step_ms(s, W, rank)
        out["fp64_ms_per_step"] = f_ms
        out["fp64_value"] = W / (f_ms / 1e3)
        out["speedup_vs_fp64"] = f_ms / ms
    return out


def batched_leg(rank: int, replays: int = 8, precision: str = "split_bf16") -> dict:
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
    for c in ctxs:
        c.close()
    return {"workload": "8 uneven systems: orbitals 48..220, 0.2 M electrons per spin, "
                        "X = 5 M, walkers 512..32, split_bf16",
            "walkers_total": walkers, "value": walkers / graph_s, "unit": UNIT,
            "ms_per_step": graph_s * 1e3, "eager_value": walkers / eager_s,
            "eager_ms_per_step": eager_s * 1e3, "graph_speedup": eager_s / graph_s,
            "replays": replays, "steps_per_replay": 5,
            "timing": "host wall clock around synchronised replays (graph) or eager steps",
            "autotuned_tiles": tiles}


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
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    from oracle.afqmc import Oracle
    from oracle.philox import gaussian_fields
    from paper_2209_04015_b300.synthetic import make_config, trial_walkers
    s, c = make_config(WORKLOAD)
    Ws = 4
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
    try:
        from threadpoolctl import threadpool_info
        cores = max([p.get("num_threads", 1) for p in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count() or 1
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT, "name": WORKLOAD, "sample_walkers": Ws},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{Ws} of {c['W']} walkers per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_leg(args) -> int:
    import torch
    torch.cuda.set_device(0)
    leg = args.profile_leg
    if leg.startswith("mixed"):
        out = mixed_leg(leg.split("-")[1], args.mixed_steps, args.warmup, 0,
                        long_steps=args.error_steps, walkers=args.profile_walkers)
    elif leg == "batched":
        out = batched_leg(0)
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
    from paper_2209_04015_b300 import AfqContext
    from paper_2209_04015_b300.synthetic import make_config

    s, c = make_config(WORKLOAD, seed=1 + rank)
    W, X, M, na, nb = c["W"], s.X, s.M, s.na, s.nb
    stream = torch.cuda.current_stream()
    ctx = AfqContext(dt=0.005, qr_period=5, seed=1 + rank, stream=stream.cuda_stream)
    ctx.init_hamiltonian(s.h1, s.L, s.e0)
    ctx.init_trial(s.psi_a, s.psi_b)
    ctx.init_walkers(W)
    ctx.autotune()  # launch shapes (set-up, outside the timed region); walkers restored
    e_dev = torch.empty((W, 4, 2), dtype=torch.float64, device="cuda")
    emix_dev = torch.empty(1, dtype=torch.float64, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def step():
        ctx.propagate_dev(None, 1)
        ctx.local_energy_dev(e_dev.data_ptr(), emix_dev.data_ptr())

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    ctx.profile_enable(True)
    n0 = ctx.launch_count()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()                      # write 256 MB: evicts L2 between timed steps
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    launches = ctx.launch_count() - n0
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    value, total_ms = job_throughput(float(sum(step_ms)), W * args.steps, world, device="cuda")

    # end to end through the public host-buffer API: the step's fields go host -> device
    # from pinned memory, the energies come back to the host, every step
    K2 = max(10, min(args.steps, 50))
    host_fields = torch.empty((K2, W, X), dtype=torch.float64).pin_memory()
    host_fields.copy_(torch.from_numpy(np.random.default_rng(5 + rank).standard_normal((K2, W, X))))
    hf = host_fields.numpy()
    # a fresh context of the same configuration: the synthetic trial lies ~300 Ha above
    # the projected energy, so with E_shift = E_HF the timed context's weights grow
    # ~e^1.6 per step and overflow after ~440 steps (harmless to the timed kernels,
    # which do not read them, but reported by the checked host-buffer calls)
    ectx = AfqContext(dt=0.005, qr_period=5, seed=1 + rank, stream=stream.cuda_stream)
    ectx.init_hamiltonian(s.h1, s.L, s.e0)
    ectx.init_trial(s.psi_a, s.psi_b)
    ectx.init_walkers(W)
    ectx.autotune()
    ectx.propagate(hf[0], 1)
    ectx.local_energy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(K2):
        ectx.propagate(hf[k], 1)
        ectx.local_energy()
    e2e_s = time.perf_counter() - t0
    ectx.close()
    e2e = {"value": W * K2 / e2e_s * world, "unit": UNIT, "h2d_bytes_per_step": W * X * 8,
           "d2h_bytes_per_step": W * 4 * 16 + 8, "steps": K2}

    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return 0

    ex_algo = ctx.exchange_algorithm()
    tiles = ctx.get_tiles()
    flops = step_flops(W, X, M, na, nb, exchange=ex_algo)
    # the dominant FP64 kernel by device time
    dom = max(FP64_KERNELS, key=lambda k: prof[k][0])
    dom_ms, dom_n = prof[dom]
    dom_avg_s = dom_ms / max(dom_n, 1) / 1e3
    dom_achieved = flops[dom] / dom_avg_s / 1e12
    kernels = {k: {"ms_per_step": v[0] / args.steps, "launches": v[1],
                   "share": v[0] / max(sum(x[0] for x in prof.values()), 1e-30)}
               for k, v in prof.items() if v[1]}
    total_flops = sum(flops.values())
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT, "name": WORKLOAD, "M": M, "na": na, "nb": nb,
                   "X": X, "W_per_gpu": W, "dt": 0.005, "qr_period": 5, "precision": "fp64",
                   "parallelism": f"replicas x{world}",
                   "l2": "flushed between timed steps (256 MB write, outside the step events)"},
        "roofline": {"bound": "alu", "kernel": f"{dom} ({FP64_KERNELS[dom]})",
                     "achieved": dom_achieved, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                     "frac": dom_achieved / FP64_NOMINAL_TFLOPS,
                     "traffic": (TRAFFIC.get(("fp64", WORKLOAD, dom))
                                 if W == 128 and (dom != "propagate" or tiles[1] == 2) else None),
                     "peak_source": "FP64 nominal (148 SMs x 2032 MHz x 4.15 flop/clk/SM)",
                     "flops_per_launch": flops[dom], "avg_launch_ms": dom_avg_s * 1e3},
        "exchange_algorithm": ex_algo,
        "autotuned_tiles": tiles,
        "step_flops": total_flops,
        "step_tflops": total_flops / (total_ms / args.steps / 1e3) / 1e12,
        "kernels": kernels,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
    }
    if not args.no_mixed:
        line["mixed"] = {"same_workload": mixed_leg(WORKLOAD, args.mixed_steps * 5, args.warmup,
                                                    rank, long_steps=args.error_steps),
                         "large_shape": mixed_leg("c3", args.mixed_steps, args.warmup, rank,
                                                  long_steps=args.error_steps,
                                                  fp64_compare=True)}
        line["mixed"]["same_workload"]["speedup_vs_fp64"] = (
            line["mixed"]["same_workload"]["value"] / (value / world))
        line["batched"] = batched_leg(rank)
        line["paper_block"] = {"fp64_c2": block_leg("c2", "fp64", rank),
                               "split_c3": block_leg("c3", "split_bf16", rank),
                               "workflow_split_c2": workflow_leg("c2", "split_bf16", rank)}
    if not args.no_adjoint:
        line["adjoint"] = adjoint_leg(rank)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
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
