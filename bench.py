#!/usr/bin/env python3
"""Benchmark: PIC particle-steps/s of the GB300 PIC/MCC step (deposit + solve +
push + MCC + injection + sort + ionization + compaction) on the 128x128x256-cell,
~1e7-macroparticle workload (h = 2.5 nm, emitter radius 40 nm, 60/30/10 % e/Cu/Cu+),
mixed precision (FP32 particles/deposit/gather/smoothing, FP64 CG residual and
refinement) as `value`, the FP64 plain path measured beside it.

One JSON line on rank 0. Under torchrun every rank runs an independent replica
(its own seed, no collective in the data path): value = all ranks' particle
pushes / max-over-ranks time ("scaling": "weak").

--impl reference times the FP64 CPU oracle on the host cores instead (a bounded
sample of the same workload per step: the 64x64x128-cell sub-box of the same
cell size and particle density).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "PIC particle-steps/s (deposit+solve+push+MCC), 1 GB300, vs FP64 plain; HBM %"
UNIT = "particle-steps/s"
WORKLOADS = {
    "c1": ("32x32x64 cells h=5nm, 1e4 macroparticles at weight 100 (60% e, 30% Cu, 10% Cu+), J=1e12 A/m2 "
           "from a 10 nm disk, Cu flux 1e27, 3 kV, sort every 20", 10_000),
    "c2": ("128x128x256 cells h=2.5nm, 1e7 macroparticles (60% e, 30% Cu, 10% Cu+), J~U[5e11,5e12] A/m2, "
           "Cu flux 1e28, sort every 20", 10_000_000),
    "c3": ("256x256x512 cells h=1.25nm (same box), 5e7 macroparticles (60% e, 30% Cu, 10% Cu+), "
           "J~U[5e11,5e12] A/m2, Cu flux 1e28, sort every 20", 50_000_000),
    "c4": ("ensemble of 48 independent instances in one handle: grids (n,n,2n), n in {32,64,96,128}, h=2.5nm, "
           "field U[5,15] GV/m, emitter radius U[5,40] nm, 1e4-2e6 macroparticles each (log-uniform), "
           "sort interval per instance from the autotuner", None),
}
WORKLOAD = WORKLOADS["c2"][0]
FALLBACK_HBM_GBS = 6800.0

# Algorithmic bytes per particle of the fused gather/push/collide/compact kernel:
# read the particle record and write it once (the node field is gathered from L2).
BYTES_PER_PARTICLE = {"mixed": 32 + 32, "fp64": 52 + 52}
# DRAM bytes (read + write) per launch of the forward convolutions captured with ncu
# (profiles/unet_conv_d0a_forward_128x128x256.md); layers without a capture are absent
UNET_NCU_TRAFFIC = {"d0a": 536.2e6}
# DRAM bytes (read + write) per pushed electron of the same kernel from one ncu capture of the
# current kernel (profiles/k_push_mixed_electrons_128x128x256.md: 145.12 MB for 2 593 379
# electrons; profiles/k_push_fp64_electrons_128x128x256.md: 266.88 MB); None where no
# capture of the current kernel exists
NCU_TRAFFIC_PER_PARTICLE = {"mixed": 55.96, "fp64": 102.91}
# The FP64 electron push is bound by GB300's FP64 pipe (2 FP64 operations per cycle
# and SM), not by HBM: FP64 warp instructions x 32 per pushed electron from one ncu
# capture of the current kernel (profiles/k_push_fp64_electrons_128x128x256.md:
# 9 274 288 instructions for 2 593 379 electrons, the pipe active 84 % of cycles)
FP64_PIPE_SLOTS_PER_ELECTRON = 114.44
FP64_OPS_PER_SM_CYCLE = 2


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peak_tflops():
    """Sustained BF16 tensor throughput (the network runs inside a long step)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["bf16_tflops_sustained"]), "measured, sustained"
    except Exception:
        return 1700.0, "fallback, sustained"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.tmp.read().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.tmp.name)
        if sm:
            out["sm_mhz"] = statistics.median(sm)
            out["sm_max_mhz"] = max(smax)
            out["samples"] = len(sm)
        out["reasons"] = sorted(reasons)
        return out


class NvmlClockSampler:
    """SM clock and clock-event reasons read through NVML (the NVIDIA driver's management library,
    read-only queries) every millisecond from a thread during the timed region;
    the device is found by its UUID, so it is the one being timed."""

    # clock-event reason bits of the public NVML API
    REASONS = {0x8: "hw_slowdown", 0x40: "hw_thermal_slowdown", 0x20: "sw_thermal_slowdown", 0x4: "sw_power_cap"}

    def __init__(self, local):
        import ctypes
        import threading
        self.ct, self.threading = ctypes, threading
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.dev = ctypes.c_void_p()
        import torch
        uuid = getattr(torch.cuda.get_device_properties(local), "uuid", None)
        ok = False
        if uuid is not None:
            ok = self.lib.nvmlDeviceGetHandleByUUID(f"GPU-{uuid}".encode(), ctypes.byref(self.dev)) == 0
        if not ok and self.lib.nvmlDeviceGetHandleByIndex_v2(local, ctypes.byref(self.dev)) != 0:
            raise RuntimeError("no NVML device")
        self.samples, self.stop_flag, self.thread = [], False, None

    def _read(self):
        ct = self.ct
        sm, smax, r = ct.c_uint(), ct.c_uint(), ct.c_ulonglong()
        try:
            if self.lib.nvmlDeviceGetClockInfo(self.dev, 1, ct.byref(sm)) != 0:  # NVML_CLOCK_SM
                return None
            self.lib.nvmlDeviceGetMaxClockInfo(self.dev, 1, ct.byref(smax))
            self.lib.nvmlDeviceGetCurrentClocksEventReasons(self.dev, ct.byref(r))
        except Exception:
            return None
        return sm.value, smax.value, r.value

    def _loop(self):
        while not self.stop_flag:
            v = self._read()
            if v is not None:
                self.samples.append(v)
            time.sleep(0.001)

    def start(self):
        self.samples, self.stop_flag = [], False
        v = self._read()  # one sample before the region starts
        if v is not None:
            self.samples.append(v)
        self.thread = self.threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    def stop(self):
        self.stop_flag = True
        self.thread.join(timeout=5)
        v = self._read()
        if v is not None:
            self.samples.append(v)
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "source": "nvml, 1 ms"}
        if self.samples:
            out["sm_mhz"] = statistics.median(x[0] for x in self.samples)
            out["sm_max_mhz"] = max(x[1] for x in self.samples)
            out["samples"] = len(self.samples)
            out["reasons"] = sorted({n for x in self.samples for b, n in self.REASONS.items() if x[2] & b})
        return out


def clock_sampler(local):
    """NVML sampling where NVIDIA's management library loads, else nvidia-smi."""
    try:
        return NvmlClockSampler(local)
    except Exception:
        return ClockSampler(local)


def with_cx(wl, cx_sigma):
    """The workload with resonant charge exchange Cu+ + Cu added at a constant
    cross-section (m^2); unchanged for cx_sigma = 0."""
    if not cx_sigma:
        return wl
    import numpy as np
    from paper_2606_05893_gb300 import workloads as W
    wl.xsec = list(wl.xsec) + [W.XSec(W.XS_CHARGE_EXCHANGE, 2, 1, 1, 0.0, np.array([1.0]), np.array([cx_sigma]))]
    return wl


def cx_label(cx_sigma):
    return f" + charge exchange Cu+ + Cu at a constant {cx_sigma:g} m2" if cx_sigma else ""


def make_workload(name, seed, n_preload, cx_sigma=0.0):
    from paper_2606_05893_gb300 import workloads as W
    if name == "c1":
        return with_cx(W.config_small(seed=42 + seed, n_preload=n_preload), cx_sigma)
    if name == "c3":
        return with_cx(W.config_mixed_large(seed=seed, n_preload=n_preload), cx_sigma)
    return with_cx(W.config_scale(seed=seed, n_preload=n_preload), cx_sigma)


def run_gpu(args, rank, ws, local):
    import torch
    import paper_2606_05893_gb300 as pkg

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    wl = make_workload(args.workload, args.seed + rank, args.n_preload, args.cx_sigma)
    results = {}
    precisions = ["mixed", "fp64"] if args.precision == "both" else [args.precision]
    stream = torch.cuda.current_stream()
    for prec in precisions:
        p = pkg.PIC_MIXED if prec == "mixed" else pkg.PIC_FP64
        sim = pkg.Simulation(wl, precision=p)
        for _ in range(args.warmup):
            sim.step(1)
        # the timed window must hold its share of cell sorts, ceil(K / interval):
        # if the next K steps hold fewer, untimed steps move it to a sort step
        if wl.sort_interval > 0:
            iv, s0 = wl.sort_interval, sim.moments()["step"]
            if sum(1 for t in range(s0, s0 + args.steps) if t % iv == 0) < -(-args.steps // iv):
                while sim.moments()["step"] % iv != 0:
                    sim.step(1)
        m0 = sim.moments()
        l0, k0 = pkg.pic_launch_count(), pkg.pic_kernel_count()
        clocks = clock_sampler(local)
        barrier()
        clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sim.step(1)
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        clk = clocks.stop()
        ms = e0.elapsed_time(e1)
        launch_ops = pkg.pic_launch_count() - l0
        launches = pkg.pic_kernel_count() - k0
        m1 = sim.moments()
        pushes = sum(m1["pushed"]) - sum(m0["pushed"])
        push_e = m1["pushed"][0] - m0["pushed"][0]
        # profiled pass: per-phase CUDA-event times on the library's stream
        pkg.pic_set_profiling(sim.h, True)
        mp0 = sim.moments()
        for _ in range(args.profile_steps):
            sim.step(1)
        torch.cuda.synchronize()
        phases = pkg.pic_get_phase_times(sim.h, 0)
        mp1 = sim.moments()
        pkg.pic_set_profiling(sim.h, False)
        prof_push_e = mp1["pushed"][0] - mp0["pushed"][0]
        # end to end through the public API with host buffers: every step uploads a
        # batch of particles handed over by the surface model (pinned host arrays),
        # steps, and reads the moments back.
        batch = args.e2e_batch
        rng = np.random.default_rng(1234 + rank)
        Lx, Ly, Lz = wl.L
        hx = torch.empty((batch, 3), dtype=torch.float64, pin_memory=True)
        hv = torch.empty((batch, 3), dtype=torch.float64, pin_memory=True)
        xb = np.stack([Lx / 2 + (rng.random(batch) - 0.5) * 40e-9, Ly / 2 + (rng.random(batch) - 0.5) * 40e-9,
                       rng.random(batch) * 5e-9], 1)
        hx.numpy()[:] = xb
        hv.numpy()[:] = rng.standard_normal((batch, 3)) * 800.0

        def e2e_step():
            pkg.pic_inject_particles(sim.h, 0, 1, hx.numpy(), hv.numpy())
            sim.step(1)
            _ = pkg.pic_moments(sim.h, 0)

        # untimed warm-up of the same loop, as for the device-timed steps: the
        # first upload allocates the pinned staging and the first steps after
        # it record their step graphs
        for _ in range(args.warmup):
            e2e_step()
        me0 = sim.moments()
        barrier()
        e2 = torch.cuda.Event(enable_timing=True)
        e3 = torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        t2 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        e3.record(stream)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        me1 = sim.moments()
        e2e_pushes = sum(me1["pushed"]) - sum(me0["pushed"])
        # a longer window of the same instance further into the run (the population
        # drains through the anode, so the first window is a transient)
        steady = None
        if prec == precisions[0] and args.steady_steps > 0:
            sim.step(1)
            ms0 = sim.moments()
            sim.step(1)
            ms1 = sim.moments()
            torch.cuda.synchronize()
            e4 = torch.cuda.Event(enable_timing=True)
            e5 = torch.cuda.Event(enable_timing=True)
            e4.record(stream)
            sim.step(args.steady_steps)
            e5.record(stream)
            torch.cuda.synchronize()
            ms2 = sim.moments()
            sim.step(1)
            ms3 = sim.moments()
            st_ms = e4.elapsed_time(e5)
            st_push = sum(ms2["pushed"]) - sum(ms1["pushed"])
            steady = {"first_step": ms1["step"], "steps": args.steady_steps, "value": st_push / (st_ms * 1e-3),
                      "ms_per_step": st_ms / args.steady_steps,
                      "pushes_per_step_at_start": sum(ms1["pushed"]) - sum(ms0["pushed"]),
                      "pushes_per_step_at_end": sum(ms3["pushed"]) - sum(ms2["pushed"]),
                      "particles_at_end": sum(ms3["count"])}
        results[prec] = dict(ms=ms, wall=wall, pushes=pushes, push_e=push_e, launches=launches, launch_ops=launch_ops, clocks=clk,
                             phases=phases, prof_push_e=prof_push_e, prof_steps=args.profile_steps,
                             e2e_s=(t3 - t2), e2e_pushes=e2e_pushes, cg_iters=m1["cg_iters"],
                             counts=m1["count"], moments=m1, steady=steady)
        sim.close()
        torch.cuda.synchronize()

    agg = {prec: reduce_over_ranks(r, dist, "cuda") for prec, r in results.items()}
    if dist is not None:
        dist.barrier()
    return results, agg, wl


def run_gpu_ensemble(args, rank, ws, local):
    """Batched ensemble: every instance steps on its own stream inside one
    pic_step call; the autotuner picks each instance's sort interval first."""
    import torch
    import paper_2606_05893_gb300 as pkg
    from paper_2606_05893_gb300 import workloads as W
    from paper_2606_05893_gb300.autotune import tune

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    wls = W.config_ensemble(seed=args.seed + rank)
    n_inst = len(wls)
    sim = pkg.Simulation(wls, precision=pkg.PIC_MIXED)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        sim.step(1)
    t_tune = time.perf_counter()
    chosen, measured = tune(sim, window=args.tune_window)
    tune_s = time.perf_counter() - t_tune

    def pushed_all():
        return [sum(sim.moments(i)["pushed"]) for i in range(n_inst)]

    p0 = pushed_all()
    l0, k0 = pkg.pic_launch_count(), pkg.pic_kernel_count()
    clocks = clock_sampler(local)
    barrier()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        sim.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    launch_ops = pkg.pic_launch_count() - l0
    launches = pkg.pic_kernel_count() - k0
    p1 = pushed_all()
    pushes = sum(p1) - sum(p0)
    # per-instance device time (phase events; instances then run one after another)
    pkg.pic_set_profiling(sim.h, True)
    q0 = [sim.moments(i) for i in range(n_inst)]
    sim.step(args.profile_steps)
    per_inst, push_e_ms, push_e_n = [], 0.0, 0
    for i in range(n_inst):
        ph = pkg.pic_get_phase_times(sim.h, i)
        q1 = sim.moments(i)
        t = sum(v[0] for v in ph.values())
        per_inst.append((sum(q1["pushed"]) - sum(q0[i]["pushed"])) / (t * 1e-3))
        push_e_ms += ph["push_electron"][0]
        push_e_n += q1["pushed"][0] - q0[i]["pushed"][0]
    pkg.pic_set_profiling(sim.h, False)
    # end to end: a host batch of neutrals into the instance with the most room
    # left for them, one ensemble step, that instance's moments
    tgt = max(range(n_inst), key=lambda i: wls[i].species[1].capacity - sim.count(1, i))
    batch = args.e2e_batch
    rng = np.random.default_rng(1234 + rank)
    Lx, Ly, Lz = wls[tgt].L
    hx = torch.empty((batch, 3), dtype=torch.float64, pin_memory=True)
    hv = torch.empty((batch, 3), dtype=torch.float64, pin_memory=True)
    hx.numpy()[:] = np.stack([Lx / 2 + (rng.random(batch) - 0.5) * 0.2 * Lx,
                              Ly / 2 + (rng.random(batch) - 0.5) * 0.2 * Ly, rng.random(batch) * 0.01 * Lz], 1)
    hv.numpy()[:] = rng.standard_normal((batch, 3)) * 800.0

    def e2e_step():
        pkg.pic_inject_particles(sim.h, tgt, 1, hx.numpy(), hv.numpy())
        sim.step(1)
        _ = pkg.pic_moments(sim.h, tgt)

    for _ in range(args.warmup):  # untimed, as in the single-instance leg
        e2e_step()
    pe0 = pushed_all()
    barrier()
    t2 = time.perf_counter()
    for _ in range(args.e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    e2e_pushes = sum(pushed_all()) - sum(pe0)
    sim.close()
    r = dict(ms=ms, pushes=pushes, e2e_s=t3 - t2, e2e_pushes=e2e_pushes)
    agg = reduce_over_ranks(r, dist, "cuda")
    if dist is not None:
        dist.barrier()
    info = dict(launches=launches, launch_ops=launch_ops, clocks=clk, per_inst=per_inst, chosen=chosen,
                tune_ms={f"interval {k[0]}, {k[1]} blocks/SM": float(np.sum([x for x in v if x is not None]))
                         for k, v in measured.items()}, tune_s=tune_s,
                push_e_ms=push_e_ms, push_e_n=push_e_n, prof_push_launches=n_inst * args.profile_steps,
                sizes=[w.nx for w in wls], n_total=sum(w.n_particles() for w in wls))
    return info, agg


def run_c4_leg(args, local, peak, peak_kind):
    """The batched ensemble (48 instances of uneven grids and populations in one
    handle, autotuned, each ensemble step one recorded graph launch) as an extra
    leg of the default run: a shorter tuning window and timed window than
    `--workload c4` (one replica, this rank's GPU)."""
    import copy
    a2 = copy.copy(args)
    a2.steps, a2.warmup, a2.profile_steps, a2.e2e_steps = args.c4_steps, 3, 2, 2
    a2.tune_window = 20
    t0 = time.perf_counter()
    info, a = run_gpu_ensemble(a2, 0, 1, local)
    pi = sorted(info["per_inst"])
    achieved = BYTES_PER_PARTICLE["mixed"] * info["push_e_n"] / (info["push_e_ms"] * 1e-3) / 1e9
    return {"workload": WORKLOADS["c4"][0], "instances": len(info["sizes"]), "macroparticles": info["n_total"],
            "steps": a2.steps, "warmup": a2.warmup, "value": a["pushes"] / (a["ms"] * 1e-3), "unit": UNIT,
            "ms_per_step": a["ms"] / a2.steps,
            "e2e": {"value": a["e2e_pushes"] / a["e2e_s"], "unit": UNIT},
            "per_instance_particle_steps_s": {"min": pi[0], "median": pi[len(pi) // 2], "max": pi[-1]},
            "launch_ops_per_step": info["launch_ops"] / a2.steps, "kernels_per_step": info["launches"] / a2.steps,
            "roofline": {"bound": "hbm", "kernel": "k_push (electrons, all instances, isolated launches)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "bytes_per_particle": BYTES_PER_PARTICLE["mixed"], "traffic": None},
            "autotune": {"chosen_interval_blocks_per_sm": info["chosen"], "window": a2.tune_window,
                         "seconds": round(info["tune_s"], 1)},
            "leg_s": round(time.perf_counter() - t0, 1)}


def run_c3_leg(args, peak, peak_kind):
    """The largest single-GPU workload: 256x256x512 cells of 1.25 nm (the same box),
    5e7 macroparticles, mixed precision; device-timed steps and the electron push's
    roofline, as for the headline."""
    import torch
    import paper_2606_05893_gb300 as pkg
    from paper_2606_05893_gb300 import workloads as W
    t0 = time.perf_counter()
    wl = W.config_mixed_large(seed=0, n_preload=args.c3_n_preload)
    sim = pkg.Simulation(wl, precision=pkg.PIC_MIXED)
    setup_s = time.perf_counter() - t0
    sim.step(3)
    stream = torch.cuda.current_stream()
    m0 = sim.moments()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.c3_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    m1 = sim.moments()
    pushes = sum(m1["pushed"]) - sum(m0["pushed"])
    pkg.pic_set_profiling(sim.h, True)
    mp0 = sim.moments()
    sim.step(3)
    ph = pkg.pic_get_phase_times(sim.h, 0)
    mp1 = sim.moments()
    pkg.pic_set_profiling(sim.h, False)
    sim.close()
    push_ms, push_n = ph["push_electron"]
    e_per = (mp1["pushed"][0] - mp0["pushed"][0]) / max(push_n, 1)
    per_ms = push_ms / max(push_n, 1)
    achieved = BYTES_PER_PARTICLE["mixed"] * e_per / (per_ms * 1e-3) / 1e9
    return {"workload": WORKLOADS["c3"][0], "n_preload": args.c3_n_preload, "steps": args.c3_steps, "warmup": 3,
            "value": pushes / (ms * 1e-3), "ms_per_step": ms / args.c3_steps, "setup_s": round(setup_s, 1),
            "cg_iters_last_step": m1["cg_iters"],
            "phase_ms_per_step": {k: round(v[0] / 3, 4) for k, v in ph.items()},
            "roofline": {"bound": "hbm", "kernel": "k_push (electrons)", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                         "bytes_per_particle": BYTES_PER_PARTICLE["mixed"], "particles_per_launch": e_per,
                         "launch_ms": per_ms, "traffic": None}}


def run_warm_start_leg(args, peak_tflops, peak_kind):
    """Learned warm start on the 128x128x256 grid: samples from runs at random field,
    J and Cu flux, training on the GPU with the library's kernels (residual
    objective), then on a held-out run the solve's iterations, the network's
    inference time and the step throughput with and without it, both solved to the
    workload's 1e-8 relative residual."""
    import torch
    import paper_2606_05893_gb300 as pkg
    from paper_2606_05893_gb300 import unet_inputs
    from paper_2606_05893_gb300 import warmstart as WS
    from paper_2606_05893_gb300 import workloads as W
    t_all = time.perf_counter()
    n_pre = args.c5_n_preload
    runs = [W.config_warm_start(seed=100 + k, n_preload=n_pre) for k in range(args.c5_runs)]
    held = W.config_warm_start(seed=1000, n_preload=n_pre)
    D, H, Wd = held.nz, held.ny, held.nx
    net = pkg.UNet(D, H, Wd)
    w0 = np.concatenate([w.reshape(-1) for w in unet_inputs.init_weights(pkg.UNET_WEIGHT_SHAPES, seed=0)])
    net.set_weights(w0.astype(np.float32))
    t0 = time.perf_counter()
    samples = WS.collect(runs, args.c5_samples, 5, net, precision=pkg.PIC_MIXED)
    collect_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    losses = WS.train(net, samples, args.c5_iters, lr=args.c5_lr, seed=0)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    ratio = WS.residual_ratio(net, samples, range(0, samples.n, max(1, samples.n // 6)))
    # inference: CUDA events around whole forward passes and around each convolution
    x = samples.X[0]
    for _ in range(3):
        net.forward(x)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.c5_infer):
        net.forward(x)
    e1.record(stream)
    torch.cuda.synchronize()
    infer_ms = e0.elapsed_time(e1) / args.c5_infer
    pkg.unet_set_profiling(net.net, True)
    for _ in range(args.c5_infer):
        net.forward(x)
    lt = pkg.unet_get_layer_times(net.net)
    pkg.unet_set_profiling(net.net, False)
    flops = {}
    for name, ci, co in pkg.UNET_LAYERS:
        lev = int(name[1])
        flops[name] = 2.0 * (D >> lev) * (H >> lev) * (Wd >> lev) * 27 * ci * co
    top = max(lt, key=lambda k: lt[k][0])
    top_ms = lt[top][0] / max(lt[top][1], 1)
    achieved = flops[top] / (top_ms * 1e-3) / 1e12
    net_flops = sum(flops.values())
    out = {"workload": "128x128x256 cells h=2.5nm, 1e7 macroparticles per run, field U[5,15] GV/m, J U[5e11,5e12], "
                       "Cu flux logU[1e26,1e28]; network 4 levels 16/32/64/128 channels, 3x3x3, BF16/FP32",
           "samples": samples.n, "runs": len(runs), "collect_s": round(collect_s, 1),
           "train_iters": len(losses), "train_s": round(train_s, 1),
           "train_ms_per_iter": round(1e3 * train_s / max(len(losses), 1), 2),
           "loss_first_last": [float(np.mean(losses[:50])), float(np.mean(losses[-50:]))],
           "train_residual_ratio": float(np.mean(ratio)),
           "inference_ms": infer_ms, "network_gflop": net_flops / 1e9,
           "network_tflops": net_flops / (infer_ms * 1e-3) / 1e12,
           "roofline": {"bound": "tensor",
                        "kernel": f"{'k_conv3z' if dict((n, co) for n, _, co in pkg.UNET_LAYERS)[top] <= 16 else 'k_conv3'}"
                                  f" forward, layer {top}", "achieved": achieved,
                        "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                        "peak_kind": peak_kind, "flop_per_launch": flops[top], "launch_ms": top_ms,
                        "traffic": UNET_NCU_TRAFFIC.get(top)},
           "layer_ms": {k: round(v[0] / max(v[1], 1), 4) for k, v in lt.items()}}
    for prec_name, prec in (("mixed", pkg.PIC_MIXED), ("fp64", pkg.PIC_FP64)):
        ev = WS.evaluate(held, net, args.c5_eval_steps, warmup=5, precision=prec)
        res = {}
        for mode in ("plain", "unet"):
            sim = pkg.Simulation(held, precision=prec)
            if mode == "unet":
                pkg.pic_set_warm_unet(sim.h, 0, net.net)
            sim.step(5)
            m0 = sim.moments()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sim.step(args.c5_eval_steps)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            m1 = sim.moments()
            pushes = sum(m1["pushed"]) - sum(m0["pushed"])
            res[mode] = {"ms_per_step": ms / args.c5_eval_steps, "particle_steps_s": pushes / (ms * 1e-3),
                         "cg_iters_mean": float(np.mean(ev[mode]["iters"])),
                         "solve_ms": ev[mode]["solve_ms"], "max_resid": float(np.max(ev[mode]["resid"]))}
            sim.close()
        res["iterations_saved_per_step"] = res["plain"]["cg_iters_mean"] - res["unet"]["cg_iters_mean"]
        res["speedup_unet_over_plain"] = res["unet"]["particle_steps_s"] / res["plain"]["particle_steps_s"]
        out[prec_name] = res
    net.close()
    out["leg_s"] = round(time.perf_counter() - t_all, 1)
    return out


def reduce_over_ranks(r, dist, device):
    """Whole-job numbers of independent replicas: the slowest rank's time and the
    sum of every rank's particle pushes (no collective touches the data path)."""
    if dist is None:
        return dict(ms=r["ms"], pushes=float(r["pushes"]), e2e_s=r["e2e_s"], e2e_pushes=float(r["e2e_pushes"]))
    import torch

    def red(v, op):
        t = torch.tensor([float(v)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=op)
        return float(t.item())
    return dict(ms=red(r["ms"], dist.ReduceOp.MAX), pushes=red(r["pushes"], dist.ReduceOp.SUM),
                e2e_s=red(r["e2e_s"], dist.ReduceOp.MAX), e2e_pushes=red(r["e2e_pushes"], dist.ReduceOp.SUM))


def _oracle_sample(workload, cx_sigma, seed=0):
    """The bounded CPU sample of a workload: the 64x64x128-cell sub-box (1/8 of the
    volume, same h and particle density), or for the small 32x32x64 workload the
    workload itself."""
    from paper_2606_05893_gb300 import workloads as W
    if workload == "c1":
        return (make_workload("c1", seed, WORKLOADS["c1"][1], cx_sigma),
                "the 32x32x64 workload itself (1e4 macroparticles)")
    return (with_cx(W.config_scale(seed=seed, n_preload=1_250_000, nx=64, ny=64, nz=128, h=2.5e-9), cx_sigma),
            "the 64x64x128-cell sub-box (same h = 2.5 nm and particle density, 1.25e6 macroparticles)")


def _time_oracle(wl, omp, seconds_target, steps_max):
    """Steps of the oracle until steps_max or seconds_target; (pushes/s, steps, s)."""
    import oracle
    o = oracle.Oracle(wl, omp=omp)
    t0 = time.perf_counter()
    pushes = 0
    steps = 0
    while steps < steps_max:
        n = sum(o.count(s) for s in range(3))
        o.step()
        pushes += n  # particles present at the start of the step (injected ones added below)
        steps += 1
        if time.perf_counter() - t0 > seconds_target:
            break
    dt = time.perf_counter() - t0
    pushes += sum(o.moments()["injected"])
    o.close()
    return pushes / dt, steps, dt


def cpu_baseline(seconds_target=10.0, steps_max=10, workload="c2", cx_sigma=0.0):
    """The FP64 oracle as it stands on a bounded sample of the workload, timed twice:
    its OpenMP build on every core this process may use (the line's value), and
    the single-threaded build beside it over the same steps. The two builds give
    bit-identical results (every sum keeps one fixed order)."""
    import oracle
    wl, what = _oracle_sample(workload, cx_sigma)
    if workload == "c1":
        steps_max = 1000
    v1, steps, dt1 = _time_oracle(wl, False, seconds_target, steps_max)
    avail = len(os.sched_getaffinity(0))
    threads = oracle.set_threads(avail)
    wl, _ = _oracle_sample(workload, cx_sigma)
    vp, steps_p, dtp = _time_oracle(wl, True, 1e30, steps)
    return {"value": vp, "unit": UNIT, "cores": threads, "cores_available": avail, "kind": "oracle",
            "build": "OpenMP build of the oracle source (bit-identical to the serial build)",
            "sample": f"{steps_p} oracle steps of {what}, FP64, {threads} threads, {dtp:.1f} s",
            "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                              "sample": f"{steps} oracle steps of the same sample, serial build, {dt1:.1f} s"}}


def run_reference(args, rank, ws):
    """The oracle as the reference arm: its OpenMP build on every core this process
    may use, on the bounded sample of the workload (rank 0 only)."""
    if rank != 0:
        return 0
    import oracle
    wl, sample = _oracle_sample(args.workload, args.cx_sigma, args.seed)
    threads = oracle.set_threads(len(os.sched_getaffinity(0)))
    o = oracle.Oracle(wl, omp=True)
    for _ in range(args.warmup):
        o.step()
    m0 = o.moments()
    n_start = sum(m0["count"])
    t0 = time.perf_counter()
    pushes = 0
    for _ in range(args.steps):
        n = sum(o.count(s) for s in range(3))
        inj0 = sum(o.moments()["injected"])
        o.step()
        pushes += n + (sum(o.moments()["injected"]) - inj0)
    dt = time.perf_counter() - t0
    o.close()
    value = pushes / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOADS[args.workload][0] + cx_label(args.cx_sigma),
                                            "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads,
                             "cores_available": len(os.sched_getaffinity(0)), "kind": "oracle",
                             "build": "OpenMP build of the oracle source (bit-identical to the serial build)",
                             "sample": f"{args.steps} timed oracle steps of {sample}, started with "
                                       f"{n_start} particles, {threads} threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="both", choices=["both", "mixed", "fp64"])
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS),
                    help="c1: 32x32x64, 1e4 particles; c2: 128x128x256, 1e7 particles (the headline); "
                         "c3: 256x256x512, 5e7 particles; c4: 48-instance ensemble")
    ap.add_argument("--n-preload", type=int, default=None, help="macroparticles preloaded (default per workload)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--profile-steps", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--e2e-batch", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tune-window", type=int, default=None,
                    help="steps per autotuner candidate (c4; default: one common period of the candidate intervals)")
    ap.add_argument("--steady-steps", type=int, default=100,
                    help="a second, longer timed window of the headline instance (0: off)")
    ap.add_argument("--no-c3", dest="c3", action="store_false",
                    help="skip the 256x256x512 / 5e7 leg (on by default with the c2 workload)")
    ap.add_argument("--c3-steps", type=int, default=10)
    ap.add_argument("--no-c4", dest="c4", action="store_false",
                    help="skip the batched-ensemble leg of the default run")
    ap.add_argument("--c4-steps", type=int, default=10)
    ap.add_argument("--c3-n-preload", type=int, default=50_000_000)
    ap.add_argument("--no-c5", dest="c5", action="store_false",
                    help="skip the learned warm start leg (on by default with the c2 workload)")
    ap.add_argument("--c5-runs", type=int, default=4, help="warm start: sample runs")
    ap.add_argument("--c5-samples", type=int, default=40, help="warm start: samples per run")
    ap.add_argument("--c5-iters", type=int, default=800, help="warm start: training iterations")
    ap.add_argument("--c5-lr", type=float, default=5e-4)
    ap.add_argument("--c5-infer", type=int, default=20, help="warm start: timed forward passes")
    ap.add_argument("--c5-eval-steps", type=int, default=20)
    ap.add_argument("--c5-n-preload", type=int, default=10_000_000)
    ap.add_argument("--cx-sigma", type=float, default=0.0,
                    help="add resonant charge exchange Cu+ + Cu at this constant cross-section (m^2) "
                         "to c1-c3; 0 (default): off, the headline workload")
    args = ap.parse_args()
    if args.n_preload is None:
        args.n_preload = WORKLOADS[args.workload][1]
    if args.workload == "c4":
        args.precision = "mixed"
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if args.cx_sigma and args.workload == "c4":
        ap.error("--cx-sigma applies to c1-c3")
    if args.cx_sigma < 0:
        ap.error("--cx-sigma must be >= 0")
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, ws)

    if args.workload == "c4":
        return report_ensemble(args, rank, ws, local)
    results, agg, wl = run_gpu(args, rank, ws, local)
    if rank != 0:
        return 0
    peak, peak_kind = peaks()
    head = "mixed" if "mixed" in results else "fp64"
    r, a = results[head], agg[head]
    value = a["pushes"] / (a["ms"] * 1e-3)
    ph = r["phases"]
    push_ms, push_n = ph["push_electron"]
    per_launch_ms = push_ms / max(push_n, 1)
    e_per_launch = r["prof_push_e"] / max(push_n, 1)
    bpp = BYTES_PER_PARTICLE[head]
    achieved = bpp * e_per_launch / (per_launch_ms * 1e-3) / 1e9
    traffic_pp = NCU_TRAFFIC_PER_PARTICLE[head]
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": (traffic_pp * e_per_launch if traffic_pp else None),
                "kernel": "k_push (electrons: gather+push+absorb+MCC+compact)",
                "peak_kind": peak_kind, "bytes_per_particle": bpp, "particles_per_launch": e_per_launch,
                "launch_ms": per_launch_ms}
    steps_total = r["prof_steps"]
    phase_ms = {k: round(v[0] / max(steps_total, 1), 4) for k, v in ph.items()}
    h2d = args.e2e_batch * 48
    import ctypes
    import paper_2606_05893_gb300 as pkg
    d2h = ctypes.sizeof(pkg.pic_moments_t) + 600 + 512
    e2e = {"value": a["e2e_pushes"] / a["e2e_s"], "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "steps": args.e2e_steps, "warmup": args.warmup,
           "api": "pic_inject_particles(host batch) + pic_step(1) + pic_moments per step"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": a["ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if head == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload][0] + cx_label(args.cx_sigma), "precision": head,
                       "n_preload": args.n_preload,
                       "grid": [wl.nx, wl.ny, wl.nz], "h": wl.h, "dt": wl.dt,
                       "parallelism": f"replicas x{ws}",
                       "l2": "inputs larger than L2 (particle stores of 0.3 GB and more per buffer)",
                       "sort": f"every {wl.sort_interval} steps; the timed window holds ceil(steps / {wl.sort_interval}) sorts"},
            "e2e": e2e, "gpu_launches": r["launches"], "launch_ops": r["launch_ops"], "clocks": r["clocks"], "roofline": roofline,
            "phase_ms_per_step": phase_ms, "cg_iters_last_step": r["cg_iters"]}
    # the whole step against HBM by the scope's byte model: particles (64 B each in the
    # mixed store, 104 B in FP64) + per unknown node 12 B (charge, counts, potential)
    # + 128 B per PCG iteration (mixed; 180 B in FP64)
    nu = wl.nx * wl.ny * (wl.nz - 1)
    pushes_step = a["pushes"] / args.steps
    per_it = 128 if head == "mixed" else 180
    step_bytes = pushes_step * BYTES_PER_PARTICLE[head] + nu * (12 + r["cg_iters"] * per_it)
    step_gbs = step_bytes / (a["ms"] / args.steps * 1e-3) / 1e9
    line["step_roofline"] = {"bound": "hbm", "achieved": step_gbs, "peak": peak, "unit": "GB/s",
                             "frac": step_gbs / peak, "bytes_per_step": step_bytes,
                             "model": f"{BYTES_PER_PARTICLE[head]} B per push + (12 + {per_it} x CG iterations) B per unknown node"}
    if "fp64" in results and head != "fp64":
        f, fa = results["fp64"], agg["fp64"]
        fph = f["phases"]
        fpush_ms, fpush_n = fph["push_electron"]
        line["fp64_plain"] = {"value": fa["pushes"] / (fa["ms"] * 1e-3), "ms_per_step": fa["ms"] / args.steps,
                              "speedup_mixed_over_fp64": value / (fa["pushes"] / (fa["ms"] * 1e-3)),
                              "phase_ms_per_step": {k: round(v[0] / max(f["prof_steps"], 1), 4) for k, v in fph.items()},
                              "push_kernel_ms": fpush_ms / max(fpush_n, 1), "clocks": f["clocks"]}
        # its push against the FP64 pipe (the bound) and against HBM
        import torch
        f_e = f["prof_push_e"] / max(fpush_n, 1)
        f_s = fpush_ms / max(fpush_n, 1) * 1e-3
        sm_mhz = (f["clocks"] or {}).get("sm_mhz") or 2070.0
        nsm = torch.cuda.get_device_properties(0).multi_processor_count
        f_peak = nsm * FP64_OPS_PER_SM_CYCLE * sm_mhz * 1e6 / 1e12
        f_ach = FP64_PIPE_SLOTS_PER_ELECTRON * f_e / f_s / 1e12
        f_hbm = BYTES_PER_PARTICLE["fp64"] * f_e / f_s / 1e9
        line["fp64_plain"]["push_roofline"] = {
            "bound": "fp64", "achieved": f_ach, "peak": f_peak, "unit": "T FP64 ops/s", "frac": f_ach / f_peak,
            "peak_kind": f"{nsm} SMs x {FP64_OPS_PER_SM_CYCLE} FP64 ops per cycle at the sampled {sm_mhz:.0f} MHz",
            "ops_per_particle": FP64_PIPE_SLOTS_PER_ELECTRON, "particles_per_launch": f_e,
            "hbm": {"achieved": f_hbm, "peak": peak, "unit": "GB/s", "frac": f_hbm / peak,
                    "bytes_per_particle": BYTES_PER_PARTICLE["fp64"],
                    "traffic": NCU_TRAFFIC_PER_PARTICLE["fp64"] * f_e}}
    if r.get("steady"):
        line["steady_state"] = r["steady"]
    if args.c3 and args.workload == "c2":
        line["c3_mixed"] = run_c3_leg(args, peak, peak_kind)
    if args.c4 and args.workload == "c2":
        line["c4_ensemble"] = run_c4_leg(args, dist_env()[2], peak, peak_kind)
    if args.c5 and args.workload == "c2":
        ptf, pkind = peak_tflops()
        line["learned_warm_start"] = run_warm_start_leg(args, ptf, pkind)
    if not args.no_cpu_baseline and ws >= 1:
        line["cpu_baseline"] = cpu_baseline(workload=args.workload, cx_sigma=args.cx_sigma)
    print(json.dumps(line), flush=True)
    return 0


def report_ensemble(args, rank, ws, local):
    info, a = run_gpu_ensemble(args, rank, ws, local)
    if rank != 0:
        return 0
    peak, peak_kind = peaks()
    value = a["pushes"] / (a["ms"] * 1e-3)
    bpp = BYTES_PER_PARTICLE["mixed"]
    achieved = bpp * info["push_e_n"] / (info["push_e_ms"] * 1e-3) / 1e9
    pi = sorted(info["per_inst"])
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": a["ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOADS["c4"][0], "precision": "mixed", "instances": len(info["sizes"]),
                       "macroparticles": info["n_total"], "parallelism": f"replicas x{ws}",
                       "l2": "inputs larger than L2 (about 2.3e7 particles in the handle)"},
            "e2e": {"value": a["e2e_pushes"] / a["e2e_s"], "unit": UNIT, "h2d_bytes_per_step": args.e2e_batch * 48,
                    "d2h_bytes_per_step": 1712,
                    "api": "pic_inject_particles(host batch into the instance with the most room) + pic_step(1) of the ensemble + pic_moments"},
            "gpu_launches": info["launches"], "launch_ops": info["launch_ops"], "clocks": info["clocks"],
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "kernel": "k_push (electrons, all instances, isolated launches)",
                         "peak_kind": peak_kind, "bytes_per_particle": bpp},
            "per_instance_particle_steps_s": {"min": pi[0], "median": pi[len(pi) // 2], "max": pi[-1]},
            "autotune": {"chosen_interval_blocks_per_sm": info["chosen"], "ms_per_step_summed": info["tune_ms"],
                         "seconds": round(info["tune_s"], 1),
                         "method": "every candidate timed from the same checkpointed state of every instance"}}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
