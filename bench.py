#!/usr/bin/env python3
"""Throughput of the phase-space lattice step on GB300, in phase-space cell updates per second.

Default workload: the 1D ensemble -- 4096 independent seeded flow realisations with N_x drawn
uniformly from {1024, 2048, 4096, 8192}, N_v = 65, St cycling {0.1, 1, 10}, FP32 storage,
advanced by one persistent launch per step captured in one CUDA graph.  A "step" advances every
instance by one lattice time step (stream, drag, diffusion).  The inputs (two 4.1 GB ping-pong
buffers) are larger than L2, so no flush is needed between steps.

--impl reference times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "phase-space cell updates/s (GCUPS) and % HBM roofline, plain vs FP16/learned"
UNIT = "GCUPS"
NV = 65
N_INST = 4096
SEED = 1234
WORKLOAD = ("1D ensemble FP32: 4096 seeded OU flow realisations, N_x uniform over "
            "{1024,2048,4096,8192}, N_v=65, St in {0.1,1,10}, kappa=1e-3")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--no-cpu-pool", action="store_true",
                   help="skip the all-cores oracle timing of the cpu_baseline leg")
    p.add_argument("--instances", type=int, default=N_INST,
                   help="ensemble size (smaller cases are for profiling only)")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--no-per-instance", action="store_true")
    p.add_argument("--no-forms", action="store_true")
    p.add_argument("--workload", default="ensemble",
                   choices=["ensemble", "2d", "2d_f16", "2d_bf16", "2d_learned"])
    p.add_argument("--scheme", default="upwind", choices=["upwind", "koren"],
                   help="drag scheme of the 1D ensemble workload (koren: flux-limited, "
                        "mu = 2/3, Heun's method)")
    p.add_argument("--size", type=int, default=0,
                   help="grid size N (N x N) of a 2D workload instead of its default "
                        "(profiling a smaller case)")
    p.add_argument("--launch", default=None,
                   help="kernel,block,blocks_per_sm instead of autotuning (profiling runs)")
    return p.parse_args()


def measured_peaks(key: str = "hbm_gbs"):
    """A measured peak of the GB300s (HBM copy GB/s, or dense BF16 TFLOP/s as a burst),
    else the fallback figures of the profiling recipe."""
    fallback = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk[key]), "measured"
    except Exception:
        return fallback[key], "fallback"


def rank_seeds(rank: int):
    """Seeds of one rank's ensemble and flow: every rank advances its own independent set of
    realisations (weak scaling, no data-path collective)."""
    return SEED + rank, SEED + 7 + rank


def max_over_ranks(ms: float, world: int, dist, torch, dev) -> float:
    """The job's time is the slowest rank's time."""
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(cells_per_rank: int, steps: int, world: int, ms_max: float) -> float:
    """Whole-job phase-space cell updates per second, in units of 1e9."""
    return world * cells_per_rank * steps / (ms_max / 1e3) / 1e9


def parse_profile(txt: str) -> dict:
    """The roofline inputs of an ncu summary: its `- key: value` lines."""
    vals = {}
    for line in txt.splitlines():
        line = line.strip().lstrip("- ")
        if ":" in line and line.startswith(("traffic_bytes_per_launch", "source_sha256",
                                            "units_per_launch")):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    return vals


# The ncu summary each timed workload takes its DRAM traffic from, and the source files its
# dominant kernel is compiled from (the summary's hash covers them, in this order).
_CSRC = "paper_1508_02899_gb300/csrc/"
# the learned closure's trained parameters (python -m paper_1508_02899_gb300.train, recipe inside)
CLOSURE_PARAMS = os.path.join(ROOT, "paper_1508_02899_gb300", "closure_params.npz")
EVAL_FINE_STEPS = (100, 400)

KERNEL_PROFILES = {
    "ensemble": ("step1d_ensemble_fp32_nv65.md", (_CSRC + "step1d.cu", _CSRC + "f32x2.h")),
    "ensemble_koren": ("step1d_ensemble_koren_fp32_nv65.md",
                       (_CSRC + "step1d.cu", _CSRC + "f32x2.h")),
    "2d": ("step2d_512_fp32_nv33.md", (_CSRC + "step2d.cu", _CSRC + "step2d_dev.h",
                                       _CSRC + "step2d_x2.h", _CSRC + "f32x2.h")),
    "2d_f16": ("step2d_1024_f16_nv33.md", (_CSRC + "step2d_h.cu", _CSRC + "step2d_dev.h")),
    "2d_bf16": ("step2d_1024_bf16_nv33.md", (_CSRC + "step2d_h.cu", _CSRC + "step2d_dev.h")),
    "2d_learned": ("learn_tc_2048_nv9.md", (_CSRC + "learn_tc.cu",)),
}


def source_hash(src) -> str:
    """First 16 hex digits of the SHA-256 of the kernel's source files, concatenated in order."""
    import hashlib
    srcs = (src,) if isinstance(src, str) else tuple(src)
    m = hashlib.sha256()
    for f in srcs:
        m.update(open(os.path.join(ROOT, f), "rb").read())
    return m.hexdigest()[:16]


def profile_traffic(kernel_file: str, src):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on this source
    (src: one file or the files the kernel is compiled from)."""
    path = os.path.join(ROOT, "profiles", kernel_file)
    try:
        txt = open(path).read()
    except OSError:
        return None
    h = source_hash(src)
    vals = parse_profile(txt)
    if vals.get("source_sha256") != h or "traffic_bytes_per_launch" not in vals:
        return None
    return float(vals["traffic_bytes_per_launch"]), float(vals.get("units_per_launch", "nan"))


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
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
            os.unlink(self.path)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline leg)
# ---------------------------------------------------------------------------------------------
class OracleSample:
    """The FP64 oracle, as it stands, on the first instances of the benchmark ensemble
    (about `sample_cells` phase-space cells per step)."""

    def __init__(self, sample_cells: int = 2_000_000, scheme: str = "upwind", start: int = 0):
        from oracle import lattice as O
        from oracle import limiter as K
        from paper_1508_02899_gb300 import inputs as I
        self.O = O
        self.koren = scheme == "koren"
        self.step_1d = ((lambda *a: K.step_1d(*a, mu=KOREN_MU)) if self.koren else O.step_1d)
        self.tab = I.ensemble_table(N_INST, SEED, nv=NV,
                                    cfl_factor=1 + KOREN_MU if self.koren else 1.0)
        self.idx, self.cells = [], 0
        while self.cells < sample_cells:
            self.idx.append(start + len(self.idx))
            self.cells += int(self.tab.nx[self.idx[-1]]) * NV
        f0 = I.ensemble_initial(self.tab, NV, None, None, instances=self.idx)
        self.fl = I.flow1d_inputs(SEED, 1, n_inst=len(self.idx))
        self.state = {i: (f0[i], self.fl.amp0[j].copy()) for j, i in enumerate(self.idx)}

    def step(self):
        O, tab, fl = self.O, self.tab, self.fl
        for j, i in enumerate(self.idx):
            f, amp = self.state[i]
            nx = int(tab.nx[i])
            dv = (tab.L[i] / nx) / tab.dt[i]
            u = O.flow1d_u(amp, fl.k, nx)
            f = self.step_1d(f, u, tab.tau_p[i], tab.kappa[i], tab.dt[i], dv)
            amp = O.ou_advance(amp, fl.noise[0, j], tab.dt[i], fl.tau_f, fl.sigma)
            self.state[i] = (f, amp)

    def describe(self, steps):
        return (f"instances {self.idx[0]}..{self.idx[-1]} of 4096 ({self.cells} cells per step), "
                f"{steps} steps" + (", flux-limited drag" if self.koren else ""))

    def time_for(self, budget_s: float):
        steps, t0 = 0, time.perf_counter()
        while True:
            self.step()
            steps += 1
            el = time.perf_counter() - t0
            if el >= budget_s:
                return steps, el


def _oracle_worker(job):
    """One process of the all-cores oracle timing: its own disjoint instances, timed for a budget
    (a top-level function, so that a spawned process can import it)."""
    start, budget, scheme = job
    smp = OracleSample(scheme=scheme, start=start)
    steps, el = smp.time_for(budget)
    return smp.cells * steps / el / 1e9


def oracle_all_cores(budget: float, scheme: str):
    """The oracle, as it stands, in one process per host core on disjoint instances (spawned: no
    process is forked from one that has touched the GPU).  Aggregate GCUPS and the core count."""
    import multiprocessing as mp
    n = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(n) as pool:
        rates = pool.map(_oracle_worker, [(16 * w, budget, scheme) for w in range(n)])
    return float(sum(rates)), n


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    smp = OracleSample(scheme=args.scheme)
    for _ in range(args.warmup):
        smp.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        smp.step()
    el = time.perf_counter() - t0
    value = smp.cells * args.steps / el / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "reference": "FP64 CPU oracle (numpy, one core)",
                   "sample": smp.describe(args.steps)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": smp.describe(args.steps)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------------
WORKLOAD_2D = ("2D FP32: periodic 512x512 grid, 33x33 velocity lattice (2.85e8 cells), St=1, "
               "kappa=1e-3, incompressible random-phase flow |k|<=8, k^-3 spectrum, OU phases")
WORKLOAD_LEARNED = ("2D learned coarse lattice: periodic {n}x{n} grid, 9x9 velocities (the 33x33 "
                    "lattice restricted: dv x4, dt / 4), St=1, kappa=1e-3, random-phase flow; "
                    "16-64-64-2 network in BF16 on tcgen05 tensor cores, random-init weights")
LEARN_FLOP_PER_CELL = 2 * (16 * 64 + 64 * 64 + 64 * 2)  # useful multiply-adds x 2
WORKLOAD_2D_16 = ("2D {fmt} storage (per x-line power-of-two scales, FP32 arithmetic): periodic "
                  "{n}x{n} grid, {nv}x{nv} velocity lattice, St=1, kappa=1e-3, incompressible "
                  "random-phase flow |k|<=8, k^-3 spectrum, OU phases")


KOREN_MU = 2.0 / 3.0


def build_ensemble(args, I, lat, torch, dev, rank, nsteps, scheme="upwind"):
    """The 1D ensemble; with scheme "koren" the flux-limited drag (mu = 2/3) and the time steps
    its Courant bound asks for (choose_dt with factor 1 + mu)."""
    n_inst = args.instances
    seed_tab, seed_flow = rank_seeds(rank)
    koren = scheme == "koren"
    tab = I.ensemble_table(n_inst, seed_tab, nv=NV, cfl_factor=1 + KOREN_MU if koren else 1.0)
    fl = I.flow1d_inputs(seed_flow, nsteps, n_inst=n_inst)
    f0 = I.ensemble_initial(tab, NV, torch.float32, dev)
    ens = lat.Ensemble(f0, nv=NV, nx=tab.nx, L=tab.L, tau_p=tab.tau_p, kappa=tab.kappa,
                       dt=tab.dt)
    if koren:
        ens.set_scheme(lat.SCHEME_KOREN, KOREN_MU)
    ens.set_flow_modes(fl.k, fl.amp0, fl.tau_f, fl.sigma)
    ens.set_noise(fl.noise)
    cells = int(tab.nx.sum()) * NV
    desc = WORKLOAD if n_inst == N_INST else f"{WORKLOAD} (profiling case: {n_inst} instances)"
    if koren:
        desc += "; flux-limited drag (Koren limiter, mu = 2/3, Heun's method)"
    return ens, cells, fl.noise, np.zeros((n_inst, 3)), desc


def build_2d(args, I, lat, torch, dev, rank, nsteps, n=512, nv=33, store="f32"):
    """2D lattice, St = 1, kappa = 1e-3, Gaussian velocity start (sigma = 0.2 V_max), uniform in
    space, random-phase flow; store = f32, or f16 / bf16 (encoded from the FP32 start)."""
    L = 2 * math.pi
    tau_p, kappa = L, 1e-3
    dt = I.choose_dt(2, n, L, nv, tau_p, kappa)
    dx = L / n
    dv = dx / dt
    col = I.gaussian_column(1, nv, dx, dv, 0.2 * ((nv - 1) // 2) * dv)
    col2 = torch.tensor(np.outer(col, col) / (n * n), dtype=torch.float32, device=dev)
    f0 = col2[:, :, None, None].expand(nv, nv, n, n).contiguous()
    fl = I.flow2d_inputs(SEED + 11 + rank, nsteps, n, n, dx)
    if store == "f32":
        lt = lat.Lattice(f0, d=2, nx=n, ny=n, nv=nv, L=L, tau_p=tau_p, kappa=kappa, dt=dt)
        desc = WORKLOAD_2D
    else:
        tdt = torch.float16 if store == "f16" else torch.bfloat16
        buf = torch.zeros(f0.shape, dtype=tdt, device=dev)
        lt = lat.Lattice(buf, d=2, nx=n, ny=n, nv=nv, L=L, tau_p=tau_p, kappa=kappa, dt=dt)
        lt.encode(f0)
        desc = WORKLOAD_2D_16.format(fmt=store.upper(), n=n, nv=nv)
    del f0
    lt.set_flow_modes_2d(fl.kvec, fl.a, fl.phi0, fl.tau_f)
    lt.set_noise(fl.noise)
    return lt, n * n * nv * nv, fl.noise, np.zeros(4), desc


def build_cellular(args, I, lat, torch, dev, rank, n=1024, nv=19, koren=False):
    """The tilted cellular flow of Sec. 4.1 (U = 1, L = 2 pi) frozen on an n^2 x 19^2 FP32
    lattice, St = 1/(2 pi), kappa = 8 pi 1e-3, Gaussian velocity start; with `koren` the
    flux-limited drag of the paper's 2D runs (mu = 2/3)."""
    L = 2 * math.pi
    tau_p, kappa = L / (2 * math.pi), 8 * math.pi * 1e-3
    dt = I.choose_dt(2, n, L, nv, tau_p, kappa, u_rms=0.1,  # max |u| = 0.5 = 5 u_rms
                     cfl_factor=1 + KOREN_MU if koren else 1.0)
    dx = L / n
    dv = dx / dt
    col = I.gaussian_column(1, nv, dx, dv, 0.3 * ((nv - 1) // 2) * dv)
    col2 = torch.tensor(np.outer(col, col) / (n * n), dtype=torch.float32, device=dev)
    f0 = col2[:, :, None, None].expand(nv, nv, n, n).contiguous()
    lt = lat.Lattice(f0, d=2, nx=n, ny=n, nv=nv, L=L, tau_p=tau_p, kappa=kappa, dt=dt)
    del f0
    ux, uy = I.cellular_flow(n, n, L, 1.0)
    u = torch.tensor(np.stack([ux, uy]), dtype=torch.float32, device=dev)
    lt.set_flow_field(u)
    lt._keep_field = u
    if koren:
        lt.set_scheme(lat.SCHEME_KOREN, KOREN_MU)
    return lt, n * n * nv * nv


def build_learned(args, I, lat, torch, dev, rank, nsteps, n=2048):
    """Coarse 9x9 lattice of the n^2 x 33^2 FP32 problem with the learned closure (mode 2)."""
    from paper_1508_02899_gb300 import train as T
    L = 2 * math.pi
    tau_p, kappa = L, 1e-3
    dt = I.choose_dt(2, n, L, 33, tau_p, kappa) / T.COARSE_PER_FINE
    dx = L / n
    dv = dx / dt
    nv = 9
    col = I.gaussian_column(1, nv, dx, dv, 0.2 * ((nv - 1) // 2) * dv)
    col2 = torch.tensor(np.outer(col, col) / (n * n), dtype=torch.float32, device=dev)
    f0 = col2[:, :, None, None].expand(nv, nv, n, n).contiguous()
    fl = I.flow2d_inputs(SEED + 13 + rank, nsteps, n, n, dx)
    lt = lat.Lattice(f0, d=2, nx=n, ny=n, nv=nv, L=L, tau_p=tau_p, kappa=kappa, dt=dt)
    lt.set_flow_modes_2d(fl.kvec, fl.a, fl.phi0, fl.tau_f)
    lt.set_noise(fl.noise)
    lt.learn(T.load_params(CLOSURE_PARAMS), 2)  # trained by train.py (recipe in the file)
    return lt, n * n * nv * nv, fl.noise, np.zeros(4), WORKLOAD_LEARNED.format(n=n)


def time_network(lt, reps, torch):
    """CUDA-event time of the tensor-core network alone (lat_learn_corrections reusing the flow
    and the streamed density of a first call), on the current stream."""
    lt.learn_corrections()
    for _ in range(2):
        lt.learn_corrections(reuse_inputs=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        lt.learn_corrections(reuse_inputs=True)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def timed(ctx, K, W, torch, dist, world, local, dev):
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.prepare(W)
    ctx.prepare(K)
    ctx.step(W)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev0.record()
    ctx.step(K)
    ev1.record()
    torch.cuda.synchronize()
    ck = clocks.stop()
    if world > 1:
        dist.barrier()
    return max_over_ranks(ev0.elapsed_time(ev1), world, dist, torch, dev), ck


def end_to_end(ctx, noise, first, glob, steps, torch, pipelined=True):
    """Per step, through the C ABI with host buffers: the step's noise row (rows first, first + 1,
    ... of the flow's noise table) from pinned host memory, one step, and the moments (globals)
    back to host memory, where the host reads them (the total mass).  Pipelined: lat_step_moments_async puts each step's globals in one of two
    pinned buffers, and the host reads step k - 1's once step k is enqueued (its event passed);
    otherwise lat_step_moments, which synchronises every step.  Returns the time, the bytes
    copied per step each way and the masses read."""
    rows = torch.from_numpy(np.ascontiguousarray(noise[first:first + steps])).pin_memory()
    assert rows.shape[0] == steps, "noise table too short"
    outs = [torch.zeros(glob.shape, dtype=torch.float64).pin_memory() for _ in range(2)]
    masses = []
    ctx.prepare(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if pipelined:
        evs = []
        for k in range(steps):
            ctx.set_noise_pinned(rows[k:k + 1])
            # the moments fused into the step where the launch allows it, else a second pass
            ctx.step_moments_async(1, outs[k % 2])
            evs.append(torch.cuda.Event())
            evs[-1].record()
            if k >= 1:
                evs[k - 1].synchronize()
                masses.append(float(outs[(k - 1) % 2].numpy()[..., 0].sum()))
        evs[-1].synchronize()
        masses.append(float(outs[(steps - 1) % 2].numpy()[..., 0].sum()))
        glob[...] = outs[(steps - 1) % 2].numpy()
    else:
        for k in range(steps):
            ctx.set_noise_pinned(rows[k:k + 1])
            ctx.step_moments(1, per_cell=False, globals_out=glob)
            masses.append(float(glob[..., 0].sum()))
    torch.cuda.synchronize()
    return time.perf_counter() - t0, int(rows[0].numel() * 8), int(glob.size * 8), masses


def kernel_label(workload, best, nv):
    k = best["kernel"] if best else 0
    if workload in ("2d_f16", "2d_bf16"):
        t = "__half" if workload == "2d_f16" else "__nv_bfloat16"
        if k >= 4:
            return {4: f"k_step2d_pch<{t},{nv},4,false>", 5: f"k_step2d_pch<{t},{nv},3,false>",
                    6: f"k_step2d_pch<{t},{nv},3,true>", 7: f"k_step2d_pch<{t},{nv},2,true>"}[k]
        return f"k_step2d_plain_h<{t},{nv}>"
    if workload == "2d":
        if k >= 3:
            return {3: f"k_step2d_pc<{nv},4,false,false>", 4: f"k_step2d_pc<{nv},4,true,false>",
                    5: f"k_step2d_pc<{nv},3,true,false>", 6: f"k_step2d_pc<{nv},3,true,true>",
                    7: f"k_step2d_pc<{nv},2,true,true>", 8: f"k_step2d_pc2<{nv},3,false>",
                    9: f"k_step2d_pc2<{nv},3,true>", 10: f"k_step2d_pc2<{nv},2,true>"}[k]
        return f"k_step2d_{'ring' if k == 2 else 'plain'}<{nv}>"
    if k >= 5:
        return f"k_step1d_pc<{nv},{k - 3}>"
    if k >= 2:
        return f"k_step1d_ring<{nv},{k}>"
    return f"k_step1d_reg<float,{nv}>"


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    from paper_1508_02899_gb300 import inputs as I
    from paper_1508_02899_gb300 import lat

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    K, W = args.steps, args.warmup
    K_e2e = max(3, min(K, 50))
    nsteps = W + K + 2 * K_e2e + 2  # warm-up, timed, pipelined and synchronous end to end
    bytes_per_cell, lines = 8, 0
    if args.workload == "2d_learned":
        ctx, cells, noise, glob, desc = build_learned(args, I, lat, torch, dev, rank, nsteps,
                                                          n=args.size or 2048)
        nv = 9
        prof, src = KERNEL_PROFILES["2d_learned"]
        launches_per_step = 4  # flow, streamed density, network, corrected step
    elif args.workload == "2d":
        ctx, cells, noise, glob, desc = build_2d(args, I, lat, torch, dev, rank, nsteps,
                                                     n=args.size or 512)
        nv = 33
        prof, src = KERNEL_PROFILES["2d"]
        launches_per_step = 2  # flow evaluation + fused step
    elif args.workload in ("2d_f16", "2d_bf16"):
        store = args.workload[3:]
        ctx, cells, noise, glob, desc = build_2d(args, I, lat, torch, dev, rank, nsteps,
                                                     n=args.size or 1024, store=store)
        nv = 33
        prof, src = KERNEL_PROFILES[args.workload]
        launches_per_step = 3  # flow evaluation + output scales + fused step
        bytes_per_cell, lines = 4, nv * nv * (args.size or 1024)
    else:
        ctx, cells, noise, glob, desc = build_ensemble(args, I, lat, torch, dev, rank, nsteps,
                                                           scheme=args.scheme)
        nv = NV
        prof, src = KERNEL_PROFILES["ensemble" if args.scheme == "upwind" else "ensemble_koren"]
        launches_per_step = 1
    best = None
    if args.launch:
        kern, blk, bps = (int(v) for v in args.launch.split(","))
        ctx.set_launch(kernel=kern, block=blk, blocks_per_sm=bps)
        best = {"kernel": kern, "block": blk, "blocks_per_sm": bps, "us_per_step": None}
    elif not args.no_autotune:
        best = ctx.autotune(reps=3)

    per_inst_ms = None
    if args.workload == "ensemble" and not args.no_per_instance:
        # unbatched baseline: one launch per instance per step (context, not the headline)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ctx.set_launch(mode=1)
        torch.cuda.synchronize()
        ev0.record()
        ctx.step(1)
        ev1.record()
        torch.cuda.synchronize()
        per_inst_ms = ev0.elapsed_time(ev1)
        ctx.set_launch(mode=0)

    ms_max, ck = timed(ctx, K, W, torch, dist, world, local, dev)
    status = ctx.status()
    value = job_throughput(cells, K, world, ms_max)
    first = ctx.steps_done  # the noise rows after those of the steps taken so far
    e2e_s, h2d, d2h, masses = end_to_end(ctx, noise, first, glob, K_e2e, torch)
    e2e_value = world * cells * K_e2e / e2e_s / 1e9
    e2e_status = ctx.status()
    sync_s, _, _, _ = end_to_end(ctx, noise, first + K_e2e, glob, K_e2e, torch,
                                 pipelined=False)
    e2e_sync = world * cells * K_e2e / sync_s / 1e9
    mass_drift = (max(masses) - min(masses)) / abs(masses[0]) if masses and masses[0] else None

    peak, peak_src = measured_peaks()
    # one read and one write of every cell; 16-bit storage adds per line its input scale, its
    # output scale and its recorded maximum (4 bytes each)
    bytes_per_launch = cells * bytes_per_cell + lines * 12
    achieved = bytes_per_launch / (ms_max / K / 1e3) / 1e9
    roof = None
    if args.workload == "2d_learned":
        # dominant kernel: the tensor-core network, timed alone with CUDA events
        net_ms = time_network(ctx, max(5, min(K, 50)), torch)
        flops = cells * LEARN_FLOP_PER_CELL
        tpeak, tsrc = measured_peaks(key="bf16_tflops")
        tf = flops / (net_ms / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": tf, "peak": tpeak, "unit": "TFLOP/s",
                "frac": tf / tpeak, "traffic": None, "peak_source": tsrc,
                "kernel": "k_mlp_tc_units<9>", "flop_per_launch": flops, "ms_per_launch": net_ms}
    tr = profile_traffic(prof, src)
    traffic = None
    if tr is not None:
        tb, units = tr
        traffic = tb * (cells / units) if units == units and units > 0 else tb
    if roof is not None:
        roof["traffic"] = traffic
    ctx.close()
    del ctx
    torch.cuda.empty_cache()

    forms = None
    if args.workload == "ensemble" and not args.no_forms and args.instances == N_INST:
        lt, c2, *_ = build_2d(args, I, lat, torch, dev, rank, 2 * 40 + 4)
        b2 = lt.autotune(reps=3)
        ms2, _ = timed(lt, 40, 3, torch, dist, world, local, dev)
        g2 = c2 * 40 / (ms2 / 1e3) / 1e9
        forms = {"2d_fp32_512x512_33x33": {
            "gcups": g2, "ms_per_step": ms2 / 40, "hbm_frac": g2 * 8 / peak,
            "kernel": kernel_label("2d", b2, 33), "steps": 40}}
        lt.close()
        del lt
        torch.cuda.empty_cache()
        # FP32 storage at the 16-bit forms' size: their speedup is taken against this
        lt, c2, *_ = build_2d(args, I, lat, torch, dev, rank, 2 * 40 + 4, n=1024)
        b2 = lt.autotune(reps=3)
        ms32, _ = timed(lt, 40, 3, torch, dist, world, local, dev)
        g2 = c2 * 40 / (ms32 / 1e3) / 1e9
        forms["2d_fp32_1024x1024_33x33"] = {
            "gcups": g2, "ms_per_step": ms32 / 40, "hbm_frac": g2 * 8 / peak,
            "kernel": kernel_label("2d", b2, 33), "steps": 40, "status": lt.status()}
        lt.close()
        del lt
        torch.cuda.empty_cache()
        for store in ("f16", "bf16"):
            lt, c2, *_ = build_2d(args, I, lat, torch, dev, rank, 2 * 40 + 4, n=1024,
                                  store=store)
            b2 = lt.autotune(reps=3)
            ms2, _ = timed(lt, 40, 3, torch, dist, world, local, dev)
            st2 = lt.status()
            g2 = c2 * 40 / (ms2 / 1e3) / 1e9
            forms[f"2d_{store}_1024x1024_33x33"] = {
                "gcups": g2, "ms_per_step": ms2 / 40,
                "hbm_frac": (g2 * 4 + g2 / 1024 * 12) / peak,
                "speedup_vs_fp32_storage": ms32 / ms2,
                "kernel": kernel_label(f"2d_{store}", b2, 33), "steps": 40, "status": st2}
            lt.close()
            del lt
            torch.cuda.empty_cache()
        if args.scheme == "upwind":
            lt, c2, *_ = build_ensemble(args, I, lat, torch, dev, rank, 2 * 40 + 4,
                                        scheme="koren")
            b2 = lt.autotune(reps=3)
            ms2, _ = timed(lt, 40, 3, torch, dist, world, local, dev)
            st2 = lt.status()
            g2 = c2 * 40 / (ms2 / 1e3) / 1e9
            forms["ensemble_koren_fp32_nv65"] = {
                "gcups": g2, "ms_per_step": ms2 / 40, "hbm_frac": g2 * 8 / peak,
                "kernel": kernel_label("ensemble", b2, NV), "steps": 40, "status": st2}
            lt.close()
            del lt
            torch.cuda.empty_cache()
        lt, c2 = build_cellular(args, I, lat, torch, dev, rank)
        b2 = lt.autotune(reps=3)
        ms2, _ = timed(lt, 40, 3, torch, dist, world, local, dev)
        st2 = lt.status()
        g2 = c2 * 40 / (ms2 / 1e3) / 1e9
        forms["2d_cellular_fp32_1024x1024_19x19"] = {
            "gcups": g2, "ms_per_step": ms2 / 40, "hbm_frac": g2 * 8 / peak,
            "kernel": kernel_label("2d", b2, 19), "steps": 40, "status": st2,
            "flow": "tilted cellular flow (Sec. 4.1), frozen field, St = 1/(2 pi), "
                    "kappa = 8 pi 1e-3"}
        lt.close()
        del lt
        torch.cuda.empty_cache()
        lt, c2 = build_cellular(args, I, lat, torch, dev, rank, koren=True)
        ms2, _ = timed(lt, 20, 3, torch, dist, world, local, dev)  # the fused FP32-pair kernel
        st2 = lt.status()
        lt.set_launch(kernel=1)  # the three passes, for comparison
        ms3, _ = timed(lt, 20, 3, torch, dist, world, local, dev)
        st2 = st2 or lt.status()
        g2 = c2 * 20 / (ms2 / 1e3) / 1e9
        forms["2d_cellular_koren_fp32_1024x1024_19x19"] = {
            "gcups": g2, "ms_per_step": ms2 / 20, "hbm_frac_of_8B": g2 * 8 / peak,
            "kernel": "k_lim2d_packed<19,32,2,4>", "bound": "alu (instruction issue)",
            "three_pass_ms_per_step": ms3 / 20, "speedup_vs_three_pass": ms3 / ms2,
            "steps": 20, "status": st2,
            "flow": "tilted cellular flow, flux-limited drag (Koren, mu = 2/3), Heun's method"}
        lt.close()
        del lt
        torch.cuda.empty_cache()
        # observables of the ensemble state (Eqs. def_coarse, def_eulS1): one call each
        lt, c2, *_ = build_ensemble(args, I, lat, torch, dev, rank, 8)
        lt.step(4)
        widths = [1, 2, 4, 8, 16, 32, 64, 128, 256, 512]
        seps = [0, 1, 2, 4, 8, 16, 32, 64]
        lt.coarse_moment(widths)
        lt.s1(seps)
        t0 = time.perf_counter()
        lt.coarse_moment(widths)
        t1 = time.perf_counter()
        lt.s1(seps)
        t2 = time.perf_counter()
        forms["observables_ensemble_fp32_nv65"] = {
            "coarse_moment_ms": 1e3 * (t1 - t0), "widths": len(widths),
            "s1_ms": 1e3 * (t2 - t1), "separations": len(seps),
            "s1_pair_gcups": c2 * len(seps) / (t2 - t1) / 1e9,
            "note": "host-timed calls (each synchronises), per-cell moments included",
            "status": lt.status()}
        lt.close()
        del lt
        torch.cuda.empty_cache()
        lt, c2, *_ = build_learned(args, I, lat, torch, dev, rank, 2 * 20 + 4)
        ms2, _ = timed(lt, 20, 3, torch, dist, world, local, dev)
        st2 = lt.status()
        net_ms = time_network(lt, 10, torch)
        tpeak, _ = measured_peaks(key="bf16_tflops")
        tf = c2 * LEARN_FLOP_PER_CELL / (net_ms / 1e3) / 1e12
        forms["2d_learned_2048x2048_9x9"] = {
            "gcups": c2 * 20 / (ms2 / 1e3) / 1e9, "ms_per_step": ms2 / 20,
            "network_ms": net_ms, "network_tflops": tf, "network_frac_bf16": tf / tpeak,
            "kernel": "k_mlp_tc_units<9> + k_step2d_pc<9,4,0,0,0,1>", "steps": 20, "status": st2}
        lt.close()
        del lt
        torch.cuda.empty_cache()
        # the fine lattice the closure stands in for: plain FP32 33^2 at 2048^2 (2 x 18 GB);
        # one fine step spans COARSE_PER_FINE coarse steps
        from paper_1508_02899_gb300 import train as T
        lt, c2, *_ = build_2d(args, I, lat, torch, dev, rank, 2 * 20 + 4, n=2048)
        b2 = lt.autotune(reps=2)
        msf, _ = timed(lt, 20, 3, torch, dist, world, local, dev)
        forms["2d_fp32_2048x2048_33x33"] = {
            "gcups": c2 * 20 / (msf / 1e3) / 1e9, "ms_per_step": msf / 20,
            "kernel": kernel_label("2d", b2, 33), "steps": 20, "status": lt.status()}
        forms["2d_learned_2048x2048_9x9"]["speedup_vs_fine_fp32"] = (
            msf / (T.COARSE_PER_FINE * ms2))
        forms["2d_learned_2048x2048_9x9"]["coarse_steps_per_fine_step"] = T.COARSE_PER_FINE
        lt.close()
        del lt
        torch.cuda.empty_cache()
        # the stated error: <|v|^2> and <rho_r^2> (r = 16 cells) of the plain 9^2 lattice and of
        # the closure against the plain 33^2 lattice, frozen random-phase flow, same start
        ev = T.evaluate(T.load_params(CLOSURE_PARAMS), 2048, 33, 1.0, 1e-3, flow_seed=505,
                        init_seed=506, times=EVAL_FINE_STEPS, r=16, kmax=8, mode=2)
        forms["2d_learned_2048x2048_9x9"]["error_vs_fine_33x33"] = {
            "fine_steps": list(EVAL_FINE_STEPS), "r_cells": 16,
            "flow": "frozen random-phase flow |k| <= 8 (seed 505), St = 1, kappa = 1e-3",
            "plain_9x9": {"v2_rel": [e[0] for e in ev["plain"]],
                          "rho_r2_rel": [e[1] for e in ev["plain"]]},
            "learned_9x9": {"v2_rel": [e[0] for e in ev["learned"]],
                            "rho_r2_rel": [e[1] for e in ev["learned"]]}}
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        scheme = args.scheme if args.workload == "ensemble" else "upwind"
        smp = OracleSample(scheme=scheme)
        c_steps, c_el = smp.time_for(args.cpu_seconds)
        cpu = {"value": smp.cells * c_steps / c_el / 1e9, "unit": UNIT, "cores": 1,
               "kind": "oracle", "sample": smp.describe(c_steps)}
        if not args.no_cpu_pool:
            v_all, n_all = oracle_all_cores(args.cpu_seconds, scheme)
            cpu["all_cores"] = {"value": v_all, "unit": UNIT, "cores": n_all,
                                "sample": f"{n_all} spawned processes, each on its own 2.3e6-cell "
                                          f"sample of the ensemble for {args.cpu_seconds:g} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": ms_max / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"2d_f16": "f16 storage, f32 math", "2d_bf16": "bf16 storage, f32 math",
                      "2d_learned": "f32 state, bf16 network (f32 accumulation)"}.get(
                args.workload, "f32"),
            "data": "synthetic",
            "config": {"workload": desc, "nv": nv, "cells_per_step_per_gpu": cells,
                       "l2": "inputs larger than L2 (FP32 ping-pong buffers of GBs); no flush",
                       "launch": best, "status": status},
            "roofline": roof or {"bound": "hbm", "achieved": achieved, "peak": peak,
                                 "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                                 "peak_source": peak_src,
                                 "kernel": kernel_label(args.workload, best, nv),
                                 "bytes_per_launch": bytes_per_launch},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "steps": K_e2e,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "api": "lat_step_moments_async, globals read one step behind",
                    "sync_value": e2e_sync, "sync_api": "lat_step_moments (synchronises)",
                    "status": e2e_status, "mass_rel_spread": mass_drift},
            "gpu_launches": launches_per_step * K + 1,
            "clocks": ck,
        }
        if per_inst_ms is not None:
            line["batching"] = {"persistent_graph_gcups": value / world,
                                "per_instance_launch_gcups": cells / (per_inst_ms / 1e3) / 1e9}
        if forms:
            line["forms"] = forms
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
