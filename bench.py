#!/usr/bin/env python
"""Benchmark of the RBE force path on GB300: particle-steps/s of full velocity-Verlet steps.

Workload (one GPU, inputs resident in HBM): 1,048,576 particles at number density
0.1 / A^3 (L = 218.88 A), 10% charged (+/-1 e), single LJ type (eps 0.1 kcal/mol,
sigma 3 A), alpha = 0.09 / A^2 (sqrt(alpha) = 0.3 / A), r_c = 10 A, P = 200 modes,
FP32-compensated form, NVE velocity Verlet, dt = 1 fs. Each step runs every stage of
the path: kick + drift, cell binning and sort, Philox mode sampling, structure factor,
real-space pair forces, k-space gather, kick and energy totals.

Output: one JSON line (rank 0). --impl reference times the FP64 CPU oracle instead.
Under torchrun each rank advances its own replica of the same workload (weak scaling,
no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "RBE force particle-steps/s on 1 GB300, FP32-comp vs FP64 form at stated force error"
UNIT = "particle-steps/s"
FP32_LANES_PER_SM = 128  # FP32 FMA lanes of one Blackwell SM (2 flops each per clock)
PAIR_FLOPS = 20.0  # FP32 flops per unique pair (LJ), the per-unit figure of the roofline
# Algorithmic HBM bytes per particle of the streaming phases (FP32 form): binning = count
# (read s, q; write key, slot: 24 B) + scatter (8 B read, 4 B write) + permute (read slot and
# s, v, id, q, 1/m; write them: 76 B) + charged subset (~2 B at 10%); integration =
# kick-drift (read s, v, F, 1/m; write s, v: 64 B) + kick (read v, F, 1/m; write v: 40 B).
BIN_BYTES = 114.0
INTEGRATE_BYTES = 104.0
# DRAM bytes (read + write) per launch of the dominant kernel on this workload, from one ncu
# capture of the kernel as it stands
TRAFFIC_BYTES = {"cluster": 60.58e6, "cells": 12.94e6, "list_skin_1.0": 2.4174e9}


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of the GB300s (GB/s), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--N", type=int, default=1 << 20)
    ap.add_argument("--P", type=int, default=200)
    ap.add_argument("--precision", default="fp32_comp")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--skin", type=float, default=None,
                    help="Verlet-list skin (A); 0 = cell traversal; default: timed trial of "
                         "0, 0.5, 1.0, 1.5 on the workload itself")
    ap.add_argument("--tuning", default="auto",
                    help="'auto' (rbe_autotune) or fixed values, e.g. pair_test16=1,sf_tile=256 "
                         "(profiling runs: the autotuner's timings are distorted under ncu)")
    ap.add_argument("--ljelec-sizes", default="200000,1400000,7000000,28000000",
                    help="ion counts of --config ljelec")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64 form, e2e, error and CPU legs (profiling runs)")
    ap.add_argument("--no-rbl", action="store_true",
                    help="skip the 2^27-particle random batch list leg")
    ap.add_argument("--config", default="main",
                    choices=["main", "batch96", "sweep16m", "rbl134m", "n3000", "ljelec", "peaks"],
                    help="main: the benchmark line; the others print per-config JSON lines")
    return ap.parse_args()


def workload(args):
    from paper_2609_02694_gb300 import synth
    sy = synth.make_system(args.N, density=0.1, frac_charged=0.1, seed=2)
    desc = (f"N={args.N} charged LJ, 10% +/-1e, density 0.1/A^3, L={sy.box[0]:.3f} A, "
            f"alpha=0.09/A^2, r_c=10 A, P={args.P}, NVE velocity Verlet dt=1 fs")
    return sy, desc


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.lines: list[str] = []
        self.proc = None

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.gpu_id:
            cmd[1:1] = ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, device) -> float:
    """The largest x over all ranks after a barrier (the job's time is its slowest rank's);
    x itself on one rank. `device` is where the process group reduces (cuda for NCCL, cpu
    for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dist.barrier()
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def time_steps(h, stream, flush_buf, K, profile_phase=None):
    """Sum of per-step device times (CUDA events on the library's stream), L2 flushed
    between steps; returns (total_ms, summed phase ms)."""
    import torch
    total = 0.0
    phases = None
    for _ in range(K):
        flush_buf.zero_()  # 256 MiB write evicts the 129 MB L2
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        h.step(1)
        end.record(stream)
        end.synchronize()
        total += start.elapsed_time(end)
        if profile_phase:
            ph, _ = h.profile()
            phases = ph if phases is None else {k: phases[k] + ph[k] for k in ph}
    return total, phases


def sampled_error(orc, sy, F, m, S, n=32, seed=0):
    """Force rel-L2 on n sampled particles against the oracle on the same modes."""
    from paper_2609_02694_gb300 import synth
    rng = np.random.default_rng(seed)
    charged = np.flatnonzero(sy.q != 0)
    idx = np.unique(np.concatenate([rng.choice(sy.n, n, replace=False), charged[: n // 2]]))
    rs = orc.real_space(sy.s, sy.q, sy.types, sy.box, synth.ALPHA, synth.R_CUT,
                        synth.COULOMB_C, sy.eps, sy.sig, i_list=idx)
    rho = orc.rho(sy.s, sy.q, sy.box, m)
    k = 2 * np.pi * m / sy.box
    k2 = (k * k).sum(1)
    th = sy.positions()[idx] @ k.T
    im = rho.imag[None, :] * np.cos(th) - rho.real[None, :] * np.sin(th)
    c = (S / len(m)) * 4 * np.pi * synth.COULOMB_C / (np.prod(sy.box) * k2)
    Fk = -(sy.q[idx][:, None, None] * (c * im)[:, :, None] * k[None, :, :]).sum(1)
    Fo = rs["F"][idx] + Fk
    return float(np.linalg.norm(F[idx] - Fo) / np.linalg.norm(Fo)), len(idx)


def cpu_oracle_step(orc, sy, P, n_sample, seed=0):
    """A bounded sample of one force evaluation of the workload by the oracle as it stands:
    the structure factor and k-space forces of the whole system (Eq. F_long_RBE), and the
    O(N) real-space sums (Eqs. F_i, G_short, LJ) of n_sample random particles, which then
    hold their complete forces. Returns (seconds, particles with complete forces)."""
    from paper_2609_02694_gb300 import synth
    m, S = orc.sample_k(1, 0, 0, sy.box, synth.ALPHA, P)
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(sy.n, n_sample, replace=False))
    t0 = time.perf_counter()
    orc.rbe_kspace(sy.s, sy.q, sy.box, synth.ALPHA, synth.COULOMB_C, m, S)
    orc.real_space(sy.s, sy.q, sy.types, sy.box, synth.ALPHA, synth.R_CUT, synth.COULOMB_C,
                   sy.eps, sy.sig, i_list=idx)
    return time.perf_counter() - t0, n_sample


def cpu_baseline_record(orc, sy, P, n_sample=8192, n_sample_1=512):
    """The oracle as it stands, timed on the host cores with all its OpenMP threads and on
    one thread: one sampled step-0 force evaluation each (cpu_oracle_step); the value is the
    particles given complete forces per second measured, nothing extrapolated. The thread
    count is restored afterwards."""
    cores = orc.num_threads()
    t_all, n_all = cpu_oracle_step(orc, sy, P, n_sample)
    orc.set_num_threads(1)
    try:
        t_one, n_one = cpu_oracle_step(orc, sy, P, n_sample_1, seed=1)
    finally:
        orc.set_num_threads(cores)

    def sample(n, s):
        return ("one step-0 force evaluation of the workload: structure factor and k-space "
                f"forces of all {sy.n} particles and the real-space sums of {n} random "
                f"particles, which then have complete forces ({s:.2f} s measured); value = "
                f"{n} / that time")

    return {"value": n_all / t_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": sample(n_all, t_all),
            "single_thread": {"value": n_one / t_one, "unit": UNIT, "cores": 1,
                              "sample": sample(n_one, t_one)}}


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    import oracle
    sy, desc = workload(args)
    orc = oracle
    orc.lib()
    n_sample = 1024
    for k in range(args.warmup):
        cpu_oracle_step(orc, sy, args.P, 64, seed=1000 + k)
    tot = 0.0
    done = 0
    for k in range(args.steps):
        t, n = cpu_oracle_step(orc, sy, args.P, n_sample, seed=k)
        tot += t
        done += n
    value = done / tot
    sample = (f"per step: structure factor and k-space forces of all {sy.n} particles and the "
              f"real-space sums of {n_sample} random particles, which then have complete "
              f"forces; value = particles with complete forces / measured time")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc + ", FP64 CPU oracle, sampled rows"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": orc.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def subbox_errors(orc, binding, stream, Ps):
    """Errors on the 65,536-particle box of the workload's composition and density, in both
    forms, at P modes: forces against the oracle on the same modes and against the full Ewald
    sum (the RBE sampling error of Eq. F_long_RBE against Eq. F_i; Fourier modes of weight
    >= 1e-6, charged particles only, as neutral ones have no k-space force), and the total
    energy and pressure against the oracle on the same modes and against full Ewald."""
    from paper_2609_02694_gb300 import synth
    sm = synth.sub_box()
    A, RC, C = synth.ALPHA, synth.R_CUT, synth.COULOMB_C
    rs = orc.real_space(sm.s, sm.q, sm.types, sm.box, A, RC, C, sm.eps, sm.sig)
    ch = sm.q != 0
    Fe = np.zeros((sm.n, 3))
    Fe[ch], Ue, We = orc.ewald_kspace_tol(sm.s[ch], sm.q[ch], sm.box, A, C, 1e-6)
    Us = orc.self_energy(sm.q, A, C)
    V = float(np.prod(sm.box))
    K2 = (sm.mass[:, None] * sm.v ** 2).sum() / synth.ACCEL_KAPPA  # 2 K
    U_e = rs["U_real"] + rs["U_lj"] + Ue - Us
    p_e = (K2 + rs["W_real"] + rs["W_lj"] + We) / (3 * V)
    F_e = rs["F"] + Fe
    res = {"N": sm.n, "full_ewald": "Fourier modes of weight >= 1e-6"}
    for P in Ps:
        res[f"P{P}"] = _subbox_forms(orc, binding, stream, sm, P, rs, Us, V, K2, F_e, U_e, p_e)
    return res


def _subbox_forms(orc, binding, stream, sm, P, rs, Us, V, K2, F_e, U_e, p_e):
    from paper_2609_02694_gb300 import synth
    A, RC, C = synth.ALPHA, synth.R_CUT, synth.COULOMB_C
    m, S = orc.sample_k(1, 0, 0, sm.box, A, P)
    Fk, Uk, Wk = orc.rbe_kspace(sm.s, sm.q, sm.box, A, C, m, S)
    U_o = rs["U_real"] + rs["U_lj"] + Uk - Us
    p_o = (K2 + rs["W_real"] + rs["W_lj"] + Wk) / (3 * V)
    F_o = rs["F"] + Fk
    out = {}
    for form in ("fp32_comp", "fp64"):
        with binding.from_system(sm, P=P, alpha=A, r_c=RC, coulomb_C=C, dt=1.0,
                                 kappa=synth.ACCEL_KAPPA, precision=form,
                                 stream=stream.cuda_stream) as h:
            F, E, W = h.forces_f64(0)
            mg, _ = h.sample_k(0)
        p = (K2 + W["total"]) / (3 * V)
        out[form] = {"modes_equal_oracle_draw": bool(np.array_equal(mg, m)),
                     "force_rel_l2_vs_oracle_same_modes": rel(F, F_o),
                     "force_rel_l2_vs_full_ewald": rel(F, F_e),
                     "energy_rel_vs_oracle_same_modes": abs(E["total"] - U_o) / abs(U_o),
                     "pressure_rel_vs_oracle_same_modes": abs(p - p_o) / abs(p_o),
                     "energy_rel_vs_full_ewald": abs(E["total"] - U_e) / abs(U_e),
                     "pressure_rel_vs_full_ewald": abs(p - p_e) / abs(p_e)}
    return out


def p1000_leg(binding, sy, mk, stream, flush, skin):
    """The headline workload at P = 1,000 modes, FP32-compensated and FP64 forms: full
    Verlet steps timed as the headline (L2 flushed between steps), each form autotuned."""
    out = {}
    for form, K in (("fp32_comp", 10), ("fp64", 3)):
        kw = dict(mk)
        kw["P"] = 1000
        h = binding.from_system(sy, precision=form, **kw)
        h.set_neighbor_list(skin)
        tuned = h.autotune(1)
        h.step(2)
        ms, _ = time_steps(h, stream, flush, K)
        out[form] = {"value": sy.n * K / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / K,
                     "steps": K, "autotuned": tuned}
        h.close()
    return out


def rbl_leg(binding, stream, K=2):
    """2^27 particles (5% charged, density 0.1), random batch list r_core = 5 A, r_s = 10 A,
    p = 10, P = 500, FP32-compensated: a few Verlet steps and the device bytes per particle."""
    import torch
    from paper_2609_02694_gb300 import synth
    t0 = time.perf_counter()
    sy = synth.make_system(1 << 27, density=0.1, frac_charged=0.05, seed=5)
    h = binding.from_system(sy, P=500, alpha=synth.ALPHA, r_c=synth.R_CUT,
                            coulomb_C=synth.COULOMB_C, dt=1.0, kappa=synth.ACCEL_KAPPA,
                            r_core=5.0, p_rbl=10, stream=stream.cuda_stream)
    n = sy.n
    del sy
    setup_s = time.perf_counter() - t0
    h.step(1)
    torch.cuda.synchronize()
    ms = _timed(lambda: h.step(1), K, stream)
    out = {"N": n, "value": n * K / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / K,
           "steps": K, "device_bytes_per_particle": h.memory_bytes() / n,
           "setup_s": setup_s,
           "config": "5% +/-1e, density 0.1, RBL r_core 5 A, r_s 10 A, p 10, P 500, FP32-comp"}
    h.close()
    return out


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def pick_traversal(binding, sy, mk, args, stream):
    """Short-range traversal: cells every step (skin 0) or a Verlet list with skin, each
    timed over real Verlet steps (list builds included) from the same initial state."""
    cands = [0.0, 0.5, 1.0, 1.5] if args.skin is None else [args.skin]
    if len(cands) == 1:
        return cands[0], None
    res = {}
    for skin in cands:
        h = binding.from_system(sy, precision=args.precision, **mk)
        h.set_neighbor_list(skin)
        h.step(3)
        res[skin] = _timed(lambda: h.step(1), 10, stream) / 10
        h.close()
    return min(res, key=res.get), {str(k): v for k, v in res.items()}


def run_ours(args):
    import torch
    ws, rank, local = dist_info()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2609_02694_gb300 import binding, build, synth
    build.build()
    binding.lib()
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()
    sy, desc = workload(args)
    mk = dict(P=args.P, alpha=synth.ALPHA, r_c=synth.R_CUT, coulomb_C=synth.COULOMB_C,
              dt=1.0, kappa=synth.ACCEL_KAPPA, replica=rank, stream=stream.cuda_stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    skin, trial = pick_traversal(binding, sy, mk, args, stream)
    h = binding.from_system(sy, precision=args.precision, **mk)
    h.set_neighbor_list(skin)
    if args.tuning == "auto":
        tuned = h.autotune(3)
    else:
        tuned = {}
        for kv in args.tuning.split(","):
            k, v = kv.split("=")
            h.set_tuning(k, int(v))
            tuned[k] = int(v)
    # exact unique-pair count of step 0 (the roofline's units) and the force sample
    F0, E0, _ = h.forces_f64(0)
    nbr, _ = h.neighbor_counts()
    pairs = float(nbr.astype(np.int64).sum()) / 2.0
    m0, S0 = h.sample_k(0)
    for _ in range(args.warmup):
        h.step(1)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:  # noqa: BLE001
        pass
    with ClockSampler(uuid) as clk:
        time.sleep(0.5)  # let the sampler start; warm steps keep the GPU loaded meanwhile
        for _ in range(2):
            h.step(1)
        total_ms, _ = time_steps(h, stream, flush, args.steps)
    torch.cuda.synchronize()
    total_ms = max_over_ranks(total_ms, dev)
    clocks = clk.summary()
    # per-phase device times (and the dominant kernel's launch time) from a second pass of
    # K steps with the library's per-phase events inside the captured graph; the headline
    # above ran without them
    h.set_profiling(True)
    h.step(1)
    prof_ms, phases = time_steps(h, stream, flush, args.steps, profile_phase=True)
    h.set_profiling(False)
    kps = h.kernels_per_step()
    props = torch.cuda.get_device_properties(dev)
    mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
    fp32_peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    peaks = measured_peaks()
    hbm = hbm_peak_gbs()
    nq_pairs = float((sy.q != 0).sum()) * args.P
    E1, _ = h.energies()
    # force evaluation alone (no integration), forces left on the device
    F_dev = torch.empty((sy.n, 3), dtype=torch.float32, device=dev)
    for k in range(2):
        h.forces(1000 + k, out=F_dev, energies=False)
    f_ms = _timed(lambda: h.forces(1002, out=F_dev, energies=False), args.steps, stream) / args.steps
    value = sy.n * args.steps * ws / (total_ms / 1e3)
    pair_ms = phases["pair"] / args.steps
    achieved = pairs * PAIR_FLOPS / (pair_ms / 1e3) / 1e12 if pair_ms > 0 else None
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision != "fp64" else "f64", "data": "synthetic",
            "config": {"workload": desc + f", {args.precision} form",
                       "l2": "flushed between timed steps (256 MiB write); per-step CUDA events",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "autotuned": tuned,
                       "short_range": (f"Verlet list, skin {skin} A" if skin > 0
                                       else "cell traversal every step"),
                       "traversal_trial_ms_per_step": trial},
            "gpu_launches": kps * args.steps,
            "force_only": {"value": sy.n / (f_ms / 1e3), "unit": UNIT, "ms_per_eval": f_ms,
                           "call": "rbe_forces (forces kept on the device, no energies read)"},
            "phases_ms_per_step": {k: v / args.steps for k, v in phases.items()},
            "phases_pass": {"ms_per_step": prof_ms / args.steps,
                            "note": "second pass of the same K steps with per-phase CUDA "
                                    "events in the graph; the headline ran without them"},
            "roofline": {"bound": "alu",
                         "kernel": ("list_pair_kernel (Verlet-list LJ)" if skin > 0
                                    else "cpair_kernel (cluster pairs, LJ)"
                                    if tuned.get("pair_cluster")
                                    else "pair_kernel (cell-list LJ)"),
                         "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp32_peak if achieved else None,
                         "traffic": (TRAFFIC_BYTES["list_skin_1.0"] if skin == 1.0 else None
                                     if skin > 0 else TRAFFIC_BYTES["cluster"]
                                     if tuned.get("pair_cluster") else TRAFFIC_BYTES["cells"]),
                         "traffic_note": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch",
                         "pair_ms_per_launch": pair_ms,
                         "units": f"{pairs:.0f} unique pairs x {PAIR_FLOPS:.0f} flops",
                         "peak_source": (f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} "
                                         f"FP32 lanes x 2 flops x {mhz:.0f} MHz (median SM clock "
                                         "sampled in the timed region; derived)")},
            "rooflines_other": {
                "structure_factor": {"bound": "sfu", "unit": "sincos pairs/s",
                                     "achieved": nq_pairs / (phases["sf"] / args.steps / 1e3),
                                     "peak": peaks["sincos_pairs"],
                                     "frac": nq_pairs / (phases["sf"] / args.steps / 1e3) / peaks["sincos_pairs"]},
                "gather": {"bound": "sfu", "unit": "sincos pairs/s",
                           "achieved": nq_pairs / (phases["gather"] / args.steps / 1e3),
                           "peak": peaks["sincos_pairs"],
                           "frac": nq_pairs / (phases["gather"] / args.steps / 1e3) / peaks["sincos_pairs"]},
                "pair_vs_measured_fp32": achieved * 1e12 / peaks["fp32_flops"] if achieved else None,
                "bin": {"bound": "hbm", "unit": "GB/s", "bytes_per_particle": BIN_BYTES,
                        "achieved": sy.n * BIN_BYTES / (phases["bin"] / args.steps / 1e3) / 1e9,
                        "peak": hbm[0], "peak_source": hbm[1],
                        "frac": sy.n * BIN_BYTES / (phases["bin"] / args.steps / 1e3) / 1e9 / hbm[0]},
                "integrate": {"bound": "hbm", "unit": "GB/s", "bytes_per_particle": INTEGRATE_BYTES,
                              "achieved": sy.n * INTEGRATE_BYTES / ((phases["kick_drift"] + phases["tail"]) / args.steps / 1e3) / 1e9,
                              "peak": hbm[0], "peak_source": hbm[1],
                              "frac": sy.n * INTEGRATE_BYTES / ((phases["kick_drift"] + phases["tail"]) / args.steps / 1e3) / 1e9 / hbm[0],
                              "note": "kick-drift + (kick, kinetic energy and totals)"},
                "peak_source": "own probes (rbe_measure_peak) at the run's clock"},
            "clocks": clocks,
            "neighbor_list": h.neighbor_list_stats() if skin > 0 else None,
            "energy": {"total_step0": E0["total"], "total_after": E1["total"],
                       "kinetic_after": E1["kinetic"]}}
    if rank == 0 and not args.no_extras:
        import oracle
        orc = oracle
        orc.lib()
        err32, ns = sampled_error(orc, sy, F0, m0, S0)
        line["force_error"] = {"rel_l2_vs_oracle_same_modes": err32,
                               "sample": f"{ns} particles (step 0)"}
        # FP64 form on the same workload
        h64 = binding.from_system(sy, precision="fp64", **mk)
        h64.set_neighbor_list(skin)
        line["fp64_form_autotuned"] = h64.autotune(1)
        h64.set_profiling(True)
        F64, _, _ = h64.forces_f64(0)
        for _ in range(2):
            h64.step(1)
        ms64, ph64 = time_steps(h64, stream, flush, args.fp64_steps, profile_phase=True)
        err64, _ = sampled_error(orc, sy, F64, m0, S0)
        line["fp64_form"] = {"value": sy.n * args.fp64_steps / (ms64 / 1e3), "unit": UNIT,
                             "ms_per_step": ms64 / args.fp64_steps,
                             "rel_l2_vs_oracle_same_modes": err64,
                             "phases_ms_per_step": {k: v / args.fp64_steps for k, v in ph64.items()}}
        h64.close()
        # end to end through the C ABI with pinned host buffers
        pos_h = torch.from_numpy(sy.positions()).pin_memory()
        F_h = torch.empty((sy.n, 3), dtype=torch.float32).pin_memory()
        h.set_profiling(False)
        for k in range(2):
            h.set_positions(pos_h)
            h.forces(k, out=F_h)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            h.set_positions(pos_h)
            h.forces(k, out=F_h)
        t1 = time.perf_counter()
        line["e2e"] = {"value": sy.n * args.steps / (t1 - t0), "unit": UNIT,
                       "h2d_bytes_per_step": sy.n * 3 * 8,
                       "d2h_bytes_per_step": sy.n * 3 * 4 + 8 * (6 + 4) + 4,
                       "call": "rbe_set_positions(host f64) + rbe_forces(host f32 F, energies)"}
        # errors on the 65,536-particle box (same modes; full Ewald), headline P and 1,000
        line["errors_65536_box"] = subbox_errors(orc, binding, stream, (args.P, 1000))
        # the workload at P = 1,000 in both forms
        line["p1000"] = p1000_leg(binding, sy, mk, stream, flush, skin)
        # 96 replicas of uneven size, batched
        line["batch96"] = batch96_leg(binding, stream, args.P)
        # the largest single-GPU system: 2^27 particles with the random batch list
        if not args.no_rbl:
            line["rbl_134m"] = rbl_leg(binding, stream)
        # CPU baseline: the oracle on a bounded sample of the same workload
        line["cpu_baseline"] = cpu_baseline_record(orc, sy, args.P)
    h.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _timed(fn, K, stream):
    """Per-call device time (CUDA events on `stream`, synchronised) summed over K calls."""
    import torch
    tot = 0.0
    for _ in range(K):
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        fn()
        e.record(stream)
        e.synchronize()
        tot += s.elapsed_time(e)
    return tot


def batch96_replicas(binding, stream, P):
    """96 replicas of log-uniform size (2,000..250,000), 10% charged, density 0.1, seeds
    1000 + r, replica keys r; the launch shapes of the largest one (rbe_autotune) applied to
    all, so that they share kernels."""
    from paper_2609_02694_gb300 import synth
    sizes = synth.replica_sizes(96)
    hs = []
    for r, n in enumerate(sizes):
        sy = synth.make_system(n, density=0.1, frac_charged=0.1, seed=1000 + r)
        hs.append(binding.from_system(sy, P=P, alpha=synth.ALPHA, r_c=synth.R_CUT,
                                      coulomb_C=synth.COULOMB_C, dt=1.0,
                                      kappa=synth.ACCEL_KAPPA, replica=r,
                                      stream=stream.cuda_stream))
    big = int(np.argmax(sizes))
    tuned = hs[big].autotune(1)
    for h in hs:
        for k, v in tuned.items():
            h.set_tuning(k, v)
    return hs, sizes, tuned


def batch96_leg(binding, stream, P, K=5, W=3):
    """Batched Verlet steps of the 96 replicas: one graph launch per step, each kernel of the
    step once per class of like replicas over all of their blocks."""
    import torch
    hs, sizes, tuned = batch96_replicas(binding, stream, P)
    total_n = sum(sizes)
    with binding.Batch(hs, stream=stream.cuda_stream) as b:
        ncls, nbat, kern = b.info()
        b.step(W)
        torch.cuda.synchronize()
        ms = _timed(lambda: b.step(1), K, stream)
    for h in hs:
        h.close()
    return {"replicas": 96, "particles": total_n, "size_range": [min(sizes), max(sizes)],
            "P": P, "value": total_n * K / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / K,
            "steps": K, "classes": ncls, "replicas_in_classes": nbat,
            "kernel_launches_per_step": kern, "autotuned": tuned,
            "note": "inputs larger than L2 (4.5 M particles)"}


def run_batch96(args):
    """The 96-replica batch against per-box sequential graph launches."""
    import torch
    from paper_2609_02694_gb300 import binding, build
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    rec = batch96_leg(binding, stream, args.P, args.steps, args.warmup)
    hs, sizes, _ = batch96_replicas(binding, stream, args.P)
    total_n = sum(sizes)
    for h in hs:
        h.step(args.warmup)
    torch.cuda.synchronize()

    def seq():
        for h in hs:
            h.step(1)
    ms_s = _timed(seq, args.steps, stream)
    for h in hs:
        h.close()
    rec["sequential_per_box"] = {"value": total_n * args.steps / (ms_s / 1e3), "unit": UNIT,
                                 "ms_per_step": ms_s / args.steps}
    print(json.dumps(dict(config="batch96", **rec)), flush=True)


def run_sweep16m(args):
    """Precision sweep: throughput at 16,777,216 particles for each form and P, and force /
    energy / virial errors on a 65,536-particle box of the same composition against the
    FP64 oracle on the same modes."""
    import torch
    import oracle
    from paper_2609_02694_gb300 import binding, build, synth
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    big = synth.make_system(1 << 24, density=0.1, frac_charged=0.1, seed=3)
    small = synth.sub_box()
    rs = oracle.real_space(small.s, small.q, small.types, small.box, synth.ALPHA, synth.R_CUT,
                           synth.COULOMB_C, small.eps, small.sig)
    ke = 0.5 * (small.mass[:, None] * small.v ** 2).sum() / synth.ACCEL_KAPPA
    V = float(np.prod(small.box))
    peaks = measured_peaks()
    hbm = hbm_peak_gbs()
    nq_big = int((big.q != 0).sum())
    for P in (100, 500, 2000):
        m, S = oracle.sample_k(1, 0, 0, small.box, synth.ALPHA, P)
        Fk, Uk, Wk = oracle.rbe_kspace(small.s, small.q, small.box, synth.ALPHA, synth.COULOMB_C,
                                       m, S)
        Fo = rs["F"] + Fk
        Uo = rs["U_real"] + rs["U_lj"] + Uk - oracle.self_energy(small.q, synth.ALPHA,
                                                                 synth.COULOMB_C)
        Wo = rs["W_real"] + rs["W_lj"] + Wk
        for form in ("fp32_comp", "fp32", "fp64"):
            kw = dict(P=P, alpha=synth.ALPHA, r_c=synth.R_CUT, coulomb_C=synth.COULOMB_C,
                      dt=1.0, kappa=synth.ACCEL_KAPPA, precision=form, stream=stream.cuda_stream)
            with binding.from_system(small, **kw) as h:
                F, E, W = h.forces_f64(0)
            errs = {"force_rel_l2": float(np.linalg.norm(F - Fo) / np.linalg.norm(Fo)),
                    "energy_rel": abs(E["total"] - Uo) / abs(Uo),
                    "pressure_rel": abs((2 * ke + W["total"]) - (2 * ke + Wo)) / abs(2 * ke + Wo)}
            h = binding.from_system(big, **kw)
            h.step(1)
            torch.cuda.synchronize()
            K = 2 if form == "fp64" else 3
            ms = _timed(lambda: h.step(1), K, stream)
            h.set_profiling(True)
            h.step(1)
            ph, _ = h.profile()
            h.close()
            pairs = nq_big * P
            line = {"config": "sweep16m", "form": form, "P": P,
                    "value": big.n * K / (ms / 1e3), "unit": UNIT,
                    "ms_per_step": ms / K, "errors_65536_box": errs,
                    "pressure_A3": (2 * ke + Wo) / (3 * V),
                    "phases_ms_one_step": ph}
            if form != "fp64":
                line["rooflines"] = {
                    "structure_factor": {"bound": "sfu", "unit": "sincos pairs/s",
                                         "achieved": pairs / (ph["sf"] / 1e3),
                                         "frac": pairs / (ph["sf"] / 1e3) / peaks["sincos_pairs"]},
                    "gather": {"bound": "sfu", "unit": "sincos pairs/s",
                               "achieved": pairs / (ph["gather"] / 1e3),
                               "frac": pairs / (ph["gather"] / 1e3) / peaks["sincos_pairs"]},
                    "bin": {"bound": "hbm", "unit": "GB/s",
                            "achieved": big.n * BIN_BYTES / (ph["bin"] / 1e3) / 1e9,
                            "frac": big.n * BIN_BYTES / (ph["bin"] / 1e3) / 1e9 / hbm[0]},
                    "integrate": {"bound": "hbm", "unit": "GB/s",
                                  "achieved": big.n * INTEGRATE_BYTES / ((ph["kick_drift"] + ph["tail"]) / 1e3) / 1e9,
                                  "frac": big.n * INTEGRATE_BYTES / ((ph["kick_drift"] + ph["tail"]) / 1e3) / 1e9 / hbm[0]},
                    "peaks": {"sincos_pairs": peaks["sincos_pairs"], "hbm_gbs": hbm[0]}}
            print(json.dumps(line), flush=True)


def run_rbl134m(args):
    """2^27 particles (5% charged, density 0.1) with the random batch list (r_core = 5 A,
    r_s = 10 A, p = 10), P = 500, FP32-compensated: throughput and device bytes/particle."""
    import torch
    from paper_2609_02694_gb300 import binding, build, synth
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    N = args.N if args.N != (1 << 20) else (1 << 27)
    sy = synth.make_system(N, density=0.1, frac_charged=0.05, seed=5)
    t0 = time.perf_counter()
    h = binding.from_system(sy, P=500, alpha=synth.ALPHA, r_c=synth.R_CUT,
                            coulomb_C=synth.COULOMB_C, dt=1.0, kappa=synth.ACCEL_KAPPA,
                            r_core=5.0, p_rbl=10, stream=stream.cuda_stream)
    init_s = time.perf_counter() - t0
    h.set_profiling(True)
    F, E, W = h.forces_f64(0)  # (records the neighbour counts read below)
    net = np.abs(F.sum(0)).max() / np.abs(F).sum()
    n_core, n_shell = h.neighbor_counts()
    core_mean, shell_mean = float(n_core.mean()), float(n_shell.mean())
    for _ in range(max(1, args.warmup)):
        h.step(1)
    torch.cuda.synchronize()
    K = max(1, min(args.steps, 5))
    ph_tot = None
    tot = 0.0
    for _ in range(K):
        tot += _timed(lambda: h.step(1), 1, stream)
        ph, _ = h.profile()
        ph_tot = ph if ph_tot is None else {k: ph_tot[k] + ph[k] for k in ph}
    print(json.dumps({"config": "rbl134m", "N": N, "value": N * K / (tot / 1e3), "unit": UNIT,
                      "ms_per_step": tot / K, "steps": K,
                      "device_bytes_per_particle": h.memory_bytes() / N,
                      "phases_ms_per_step": {k: v / K for k, v in ph_tot.items()},
                      "net_force_over_sum_abs": float(net), "init_s": init_s,
                      "per_particle": {"core_pairs": core_mean, "shell_members": shell_mean,
                                       "drawn_pairs": 10},
                      "rbl_kernel": {"ms": ph_tot["pair"] / K,
                                     "pair_evaluations_per_s": N * (core_mean + 10) / (ph_tot["pair"] / K / 1e3),
                                     "note": "core pairs + p draws per particle; every stencil "
                                             "candidate is classified once"}}), flush=True)
    h.close()


def run_n3000(args):
    """3,000 point charges (1,500 each sign) in L = 32 A, FP64 form: one force evaluation
    against the oracle on the same modes and against the full Ewald sum (RBE sampling
    error), then 100 graph-replayed Verlet steps (dt = 1 fs) with the energy drift."""
    import torch
    import oracle
    from paper_2609_02694_gb300 import binding, build, synth
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    sy = synth.make_system(3000, L=32.0, all_charged=True, seed=1)
    out = {"config": "n3000"}
    for form in ("fp64", "fp32_comp"):
        with binding.from_system(sy, P=100, alpha=synth.ALPHA, r_c=synth.R_CUT,
                                 coulomb_C=synth.COULOMB_C, dt=1.0, kappa=synth.ACCEL_KAPPA,
                                 precision=form, stream=stream.cuda_stream) as h:
            F, E, W = h.forces_f64(0)
            m, S = h.sample_k(0)
            ref = oracle.total_forces(sy.s, sy.q, sy.types, sy.box, synth.ALPHA, synth.R_CUT,
                                      synth.COULOMB_C, sy.eps, sy.sig, m, S)
            Fe, Ue, We = oracle.ewald_kspace(sy.s, sy.q, sy.box, synth.ALPHA, synth.COULOMB_C)
            rs = oracle.real_space(sy.s, sy.q, sy.types, sy.box, synth.ALPHA, synth.R_CUT,
                                   synth.COULOMB_C, sy.eps, sy.sig)
            Fewald = rs["F"] + Fe
            h.step(1)
            torch.cuda.synchronize()
            E0, _ = h.energies()
            ms = _timed(lambda: h.step(1), 100, stream)
            E1, _ = h.energies()
            out[form] = {"force_rel_l2_vs_oracle_same_modes":
                         float(np.linalg.norm(F - ref["F"]) / np.linalg.norm(ref["F"])),
                         "force_rel_l2_vs_full_ewald":
                         float(np.linalg.norm(F - Fewald) / np.linalg.norm(Fewald)),
                         "energy_rel_vs_oracle": abs(E["total"] - ref["U_total"]) / abs(ref["U_total"]),
                         "value": 3000 * 100 / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / 100,
                         "E_total_step1": E0["total"] + E0["kinetic"],
                         "E_total_step101": E1["total"] + E1["kinetic"]}
    print(json.dumps(out), flush=True)


def measured_peaks():
    """Measured FP32 flop/s, sincos pairs/s and FP64 flop/s of this GPU (own probes)."""
    from paper_2609_02694_gb300 import binding
    return {"fp32_flops": binding.measure_peak("fp32"),
            "sincos_pairs": binding.measure_peak("sincos"),
            "fp64_flops": binding.measure_peak("fp64")}


def run_peaks(args):
    import torch
    from paper_2609_02694_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    print(json.dumps({"config": "peaks", **measured_peaks()}), flush=True)


def run_ljelec(args):
    """LJ electrolyte in reduced units (all ions charged, density 200,000 / 271^3), random
    batch list (r_s = 8, r_c = 4, p = 30), P = 200, Nose-Hoover T = 1: the O(N) sweep of the
    full step, with the k-space kernels against the measured sincos throughput."""
    import torch
    from paper_2609_02694_gb300 import binding, build, synth
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    peaks = measured_peaks()
    prm = synth.LJ_ELECTROLYTE
    for N in [int(x) for x in args.ljelec_sizes.split(",")]:
        sy = synth.lj_electrolyte(N)
        h = binding.from_system(sy, P=prm["P"], alpha=prm["alpha"], r_c=prm["r_c"],
                                r_core=prm["r_core"], p_rbl=prm["p_rbl"],
                                coulomb_C=prm["coulomb_C"], dt=prm["dt"], kappa=prm["kappa"],
                                stream=stream.cuda_stream)
        h.set_thermostat(prm["T"], prm["tau"], prm["kB"])
        h.set_profiling(True)
        h.step(max(2, args.warmup))
        torch.cuda.synchronize()
        K = 5
        tot, ph_tot = 0.0, None
        for _ in range(K):
            tot += _timed(lambda: h.step(1), 1, stream)
            ph, _ = h.profile()
            ph_tot = ph if ph_tot is None else {k: ph_tot[k] + ph[k] for k in ph}
        E, _ = h.energies()
        T_inst = 2 * E["kinetic"] / ((3 * N - 3) * prm["kB"])
        sf = ph_tot["sf"] / K
        ga = ph_tot["gather"] / K
        pairs = N * prm["P"]
        print(json.dumps({"config": "ljelec", "N": N, "L": float(sy.box[0]),
                          "value": N * K / (tot / 1e3), "unit": UNIT, "ms_per_step": tot / K,
                          "phases_ms_per_step": {k: v / K for k, v in ph_tot.items()},
                          "kspace_rooflines": {
                              "structure_factor": {"bound": "sfu", "achieved": pairs / (sf / 1e3),
                                                   "peak": peaks["sincos_pairs"],
                                                   "unit": "sincos pairs/s",
                                                   "frac": pairs / (sf / 1e3) / peaks["sincos_pairs"]},
                              "gather": {"bound": "sfu", "achieved": pairs / (ga / 1e3),
                                         "peak": peaks["sincos_pairs"], "unit": "sincos pairs/s",
                                         "frac": pairs / (ga / 1e3) / peaks["sincos_pairs"]}},
                          "temperature": T_inst,
                          "rbl_eager": h.get_tuning("rbl_eager")}), flush=True)
        h.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "batch96":
        run_batch96(args)
    elif args.config == "sweep16m":
        run_sweep16m(args)
    elif args.config == "rbl134m":
        run_rbl134m(args)
    elif args.config == "n3000":
        run_n3000(args)
    elif args.config == "ljelec":
        run_ljelec(args)
    elif args.config == "peaks":
        run_peaks(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
