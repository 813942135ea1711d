"""Benchmark of the hydro RK2 step: cell-updates/s on one GB300.

Workload (the metric's configuration): 3D adiabatic Euler, gamma = 5/3, periodic 256^3
in 64 MeshBlocks of 64^3, PLM + HLLC + RK2, CFL 0.3, rho = 1, p = 1, seeded
random-phase Gaussian velocity field with shell spectrum E(k) ~ k^-2 on 2 <= |k| <= 8,
rms Mach 0.5.  A step is one full RK2 step: ghost fill, stage 1, ghost fill, stage 2
with the CFL reduction, dt finalisation -- all in libak's CUDA kernels, dt device
resident (no host round trip inside the timed region).  `value` is the FP64 form; the
`mixed` object is the same workload in the mixed FP32/FP64 form.  The line also carries
the other configurations, each with its own roofline: `smr` (the static-refinement batch,
1016 leaves), and `large` -- 512^3 in 128^3 blocks with PPM4 + RK3 (FP64 and mixed) and
768^3 in 96^3 blocks at Mach 2 (mixed, 50 steps).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
N > 1 (under torchrun) runs independent replicas, one per GPU (weak scaling, no data
exchange: the build targets one GPU per box).
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/sec per full RK2 step on 1 GB300 (FP64 vs mixed FP32) at stated L1 error"
UNIT = "cell-updates/s"
ROOT_NX = (256, 256, 256)
BLOCK_NX = (64, 64, 64)
WORKLOAD = "256^3 periodic, 64 MeshBlocks of 64^3, PLM+HLLC+RK2, k^-2 turbulence Mach 0.5"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")

# Algorithmic work per cell and stage:
#  FP64 flops of the scheme (each +,-,*,/,sqrt counted once): cons->prim 11, PLM
#  (slope once per cell, 2 face states) 150, HLLC 3 faces x 99, divergence 45, RK
#  update 17.5 (mean of the two stages), CFL 21 on the last stage (10.5 mean)
FLOP_PER_CELL_STAGE = 531.0
#  bytes: stage 1 reads U_in and writes U_out (2 x 40 B); stage 2 also reads U0
BYTES_STAGE = {1: 80.0, 2: 120.0}
# FP64 peak from unit counts and clock: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP64 pipe busy fraction of the FP64 stage kernel in the ncu capture of these sources
# (sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active, mean of the two stages):
# the unit the form is bound by
FP64_PIPE_BUSY_NCU = 0.792
# FP64 instructions (DADD + DMUL + DFMA, thread level) per cell of the FP64 stage kernel
# in the same capture (smsp__sass_thread_inst_executed_op_{dadd,dmul,dfma}_pred_on),
# stages 1 and 2: set against the measured FP64 instruction rate (ak_probe_fp64_rate)
FP64_INST_PER_CELL_NCU = (283.6, 313.0)
# DRAM bytes per cell of the stage kernels (dram__bytes_read.sum + dram__bytes_write.sum
# of one ncu capture per launch: PLM + RK2 on 192^3 in 64^3 blocks, PPM4 + RK3 on 256^3 in
# 128^3 blocks; the per-cell figures carry over to grids of the same block size), valid
# for the kernel sources with this hash (else traffic = null)
TRAFFIC_SRC_HASH = "2556c102381adc8594a48b1df549027742c73cbe"
TRAFFIC_B_PER_CELL = {"fp64": (85.61, 128.22), "mixed": (83.91, 126.89),
                      "ppm4_mixed": (92.80, 138.51, 135.43)}


def kernel_source_hash():
    """sha1 over the sha1sum lines of the stage kernel's sources (as sha1sum prints them)."""
    import hashlib
    d = os.path.join(ROOT, "paper_2409_16053_gb300", "csrc")
    lines = ""
    for f in ("stage_kernel.cuh", "ak_stage_plm.cu", "ak_stage_mx.cu", "stage_mx.cuh",
              "stage_common.cuh", "hydro_ops.cuh", "lanes.cuh", "fastmath.cuh", "exchange.cuh"):
        h = hashlib.sha1(open(os.path.join(d, f), "rb").read()).hexdigest()
        lines += f"{h}  ../paper_2409_16053_gb300/csrc/{f}\n"
    return hashlib.sha1(lines.encode()).hexdigest()


def traffic_per_launch(form, cells):
    """Measured DRAM bytes per stage launch (mean over the step's stages), or None if the
    kernel changed since the counters were taken."""
    if kernel_source_hash() != TRAFFIC_SRC_HASH:
        return None
    b = TRAFFIC_B_PER_CELL[form]
    return sum(b) / len(b) * cells


def linear_wave_l1(ak, precision, n=32):
    """L1 error of the 3D sound-wave test (n^3, one block, PLM+HLLC+RK2, CFL 0.3, one
    period), run on the GPU outside the timed region."""
    import numpy as np
    import pgen
    U0, T = pgen.linear_wave((n, n, n))
    m = ak.Mesh((n, n, n), (n, n, n), precision=precision, ref_rho=1.0, ref_p=0.6)
    m.upload(U0)
    t, dt = 0.0, m.new_dt()
    while t < T:
        dt = min(dt, T - t)
        dn = m.step(dt)
        t += dt
        dt = dn
    U = m.download()
    m.close()
    return float(np.sqrt(sum(np.mean(np.abs(U[k] - U0[k])) ** 2 for k in range(5))))


def max_over_ranks(dist, v, device="cuda"):
    """The slowest rank's time: the job's time (v itself without a process group)."""
    if not dist:
        return v
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(ws, cells_per_rank, steps, t_ms):
    """Whole-job cell-updates/s: every rank advances its own replica (weak scaling)."""
    return ws * cells_per_rank * steps / (t_ms * 1e-3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(prefix="ak_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smmax, reasons = [], [], set()
        lines = open(self.path).read().splitlines()
        os.unlink(self.path)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smmax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smmax) if smmax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def time_form(ak, torch, precision, U0, steps, warmup):
    """Times `steps` RK2 steps of one form.  Returns a dict of measurements."""
    mesh = ak.Mesh(ROOT_NX, BLOCK_NX, precision=precision, ref_rho=1.0, ref_p=1.0)
    mesh.upload(U0)
    schedule = mesh.autotune()  # library autotuner, outside the timed region
    mesh.upload(U0)
    mesh.new_dt()
    h = mesh.handle
    stream = mesh.stream

    def one_step(evs=None):
        # the same launches as ak_step: a ghost fill before each stage unless the stage
        # kernels read halos from the neighbour blocks directly
        if not mesh.direct:
            ak.ak_fill_ghosts(h, 0)
        if evs:
            evs[0].record(stream)
        ak.ak_stage(h, 1, 0.0)
        if evs:
            evs[1].record(stream)
        if not mesh.direct:
            ak.ak_fill_ghosts(h, 1)
        if evs:
            evs[2].record(stream)
        ak.ak_stage(h, 2, 0.0)
        if evs:
            evs[3].record(stream)

    for _ in range(warmup):
        one_step()
    stream.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    for s in range(steps):
        one_step(evs[s])
    end.record(stream)
    end.synchronize()
    total_ms = start.elapsed_time(end)
    st1 = [e[0].elapsed_time(e[1]) for e in evs]
    st2 = [e[2].elapsed_time(e[3]) for e in evs]
    per_step = [e[0].elapsed_time(e[3]) for e in evs]  # stage 1 start to stage 2 end
    dt_next, status = ak.ak_new_dt(h, 0)
    counters = mesh.counters()
    direct = mesh.direct
    mesh.close()
    del mesh
    torch.cuda.empty_cache()
    return {"total_ms": total_ms, "stage1_ms": statistics.mean(st1),
            "stage2_ms": statistics.mean(st2),
            "step_ms": {"best": min(per_step), "median": statistics.median(per_step)},
            "dt_after": dt_next, "counters": counters,
            "direct": direct,
            "schedule": {"tile": schedule[0], "x3_segments": schedule[1],
                         "order": schedule[2]}}


def e2e_form(ak, torch, precision, U0, steps):
    """Whole job through the public API with host buffers: upload the initial state from
    pinned host memory, `steps` x ak_step with the dt round trip to the host every step,
    download the final state to pinned host memory."""
    import numpy as np
    mesh = ak.Mesh(ROOT_NX, BLOCK_NX, precision=precision, ref_rho=1.0, ref_p=1.0)
    packed = torch.from_numpy(mesh.pack(U0)).pin_memory()
    out = torch.empty_like(packed).pin_memory()
    ak.ak_upload(mesh.handle, 0, packed.data_ptr())      # warm-up: schedule, graph capture
    ak.ak_mesh_autotune(mesh.handle)
    ak.ak_upload(mesh.handle, 0, packed.data_ptr())
    dt, _ = ak.ak_new_dt(mesh.handle, 0)
    ak.ak_step(mesh.handle, dt, True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ak.ak_upload(mesh.handle, 0, packed.data_ptr())
    dt, _ = ak.ak_new_dt(mesh.handle, 0)
    for _ in range(steps):
        dt, _ = ak.ak_step(mesh.handle, dt, True)
    ak.ak_download(mesh.handle, 0, out.data_ptr())
    t1 = time.perf_counter()
    ok = bool(np.isfinite(out.numpy()).all())
    nbytes = packed.numel() * 8
    mesh.close()
    torch.cuda.empty_cache()
    cells = ROOT_NX[0] * ROOT_NX[1] * ROOT_NX[2]
    return {"value": cells * steps / (t1 - t0), "unit": UNIT,
            "h2d_bytes_per_step": (nbytes + 8 * (steps + 1)) / steps,
            "d2h_bytes_per_step": (nbytes + 8 * (steps + 1)) / steps,
            "finite": ok}


def time_smr(ak, torch, precision, steps, warmup):
    """The static-refinement workload: root 128^3 in 32^3 blocks and two nested levels of
    16^3 blocks over the central 1/2 and 1/4 cubes (1016 leaves, 5,767,168 cells) on
    [-1/2, 1/2]^3, Sedov deposit (energy 1 in r < 0.02, rho = 1, p = 1e-5), PLM + HLLC +
    RK2, one dt for all levels.  A step is one graph-replayed ak_step (the ghost fill at
    level boundaries -- restrictions, prolongations; same-level halos are read by the
    stage kernels directly --, flux correction, stage, twice, and the dt reduction)."""
    import pgen
    t = pgen.nested_refinement_blocks()
    P = pgen.sedov_blocks(t, 128)
    m = ak.Mesh((128, 128, 128), table=t, precision=precision, xmin=(-0.5,) * 3,
                xmax=(0.5,) * 3, ref_rho=1.0, ref_p=1e-5)
    m.upload_packed(P)
    schedule = m.autotune()
    m.upload_packed(P)
    m.new_dt()
    for _ in range(warmup):
        m.step(0.0, want_dt_next=False)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(m.stream)
    for _ in range(steps):
        m.step(0.0, want_dt_next=False)
    b.record(m.stream)
    b.synchronize()
    ms = a.elapsed_time(b)
    cells = int(np.prod(t[:, 4:7].astype(np.int64), axis=1).sum())
    c = m.counters()
    m.close()
    torch.cuda.empty_cache()
    value = cells * steps / (ms * 1e-3)
    peaks, peak_kind = load_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    gbs = value * 200.0 / 1e9
    return {"value": value, "unit": UNIT, "ms_per_step": ms / steps,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                         "frac": gbs / hbm, "bytes_per_cell_update": 200.0,
                         "cells": "leaf cells", "traffic": None,
                         "peak_source": f"{peak_kind} hbm_gbs"},
            "counters": c, "schedule": {"tile": schedule[0], "x3_segments": schedule[1],
                                        "order": schedule[2], "fused": schedule[4]}}


def cpu_baseline(sample_n=96, budget_s=12.0, steps_max=None):
    """The oracle (as it stands) on this host's cores: RK2 steps of a periodic sample_n^3
    box with the benchmark's turbulence recipe until budget_s of CPU work."""
    import oracle
    import pgen
    oracle.build()
    n = (sample_n,) * 3
    U = pgen.turbulence(n, seed=1, kmin=2, kmax=8, mach=0.5)
    g = oracle.Grid(n)
    steps, t0 = 0, time.perf_counter()
    while True:
        dt = oracle.new_dt(U, g, 0.3)
        U, _ = oracle.rk_step(U, g, dt, 2)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (steps_max is not None and steps >= steps_max):
            break
    return {"value": sample_n ** 3 * steps / el, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{steps} RK2 steps of a periodic {sample_n}^3 box (same turbulence "
                      f"recipe, FP64 oracle, OpenMP), {el:.1f} s"}


def cpu_baseline_one_core(sample_n=48, budget_s=5.0):
    """The same oracle sample on one host core (a child process with OMP_NUM_THREADS=1,
    since the thread count is fixed when the oracle library loads)."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.cpu_baseline(sample_n=%d, budget_s=%r)))"
            % (ROOT, sample_n, budget_s))
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                           env=env, timeout=120)
        return json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as e:  # reported, not fatal: the headline numbers do not depend on it
        return {"unavailable": str(e)[:200]}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    import pgen
    oracle.build()
    n = (64, 64, 64)
    U = pgen.turbulence(n, seed=1, kmin=2, kmax=8, mach=0.5)
    g = oracle.Grid(n)
    for _ in range(args.warmup):
        U, _ = oracle.rk_step(U, g, oracle.new_dt(U, g, 0.3), 2)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U, _ = oracle.rk_step(U, g, oracle.new_dt(U, g, 0.3), 2)
    el = time.perf_counter() - t0
    value = 64 ** 3 * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "64^3 periodic box per step (bounded)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": f"{args.steps} RK2 steps of a periodic 64^3 box"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_profile_case(args):
    """Small cases for ncu captures, one form, `steps` graph-replayed steps: 192^3 in 27
    MeshBlocks of 64^3 with PLM + RK2 (two registers of ~0.34 GB, larger than L2);
    profile-ppm: 256^3 in 8 MeshBlocks of 128^3 with PPM4 + RK3; profile-smr: the
    static-refinement mesh."""
    import torch
    import pgen
    from paper_2409_16053_gb300 import ak
    prec = ak.AK_MIXED if args.form == "mixed" else ak.AK_FP64
    if args.case == "profile-smr":
        t = pgen.nested_refinement_blocks()
        m = ak.Mesh((128, 128, 128), table=t, precision=prec, xmin=(-0.5,) * 3,
                    xmax=(0.5,) * 3, ref_rho=1.0, ref_p=1e-5)
        m.upload_packed(pgen.sedov_blocks(t, 128))
        m.new_dt()
        for _ in range(args.steps):
            m.step(0.0)
        c = m.counters()
        m.close()
        print(json.dumps({"case": "profile-smr", "form": args.form, "steps": args.steps,
                          "counters": c}), flush=True)
        return 0 if c[:2] == [0, 0] else 1
    if args.case == "profile-ppm":
        # the 512^3 PPM4 + RK3 configuration's kernels on 256^3 in 128^3 blocks
        root = (256, 256, 256)
        U0 = pgen.turbulence(root, seed=3, kmin=2, kmax=8, mach=0.5)
        m = ak.Mesh(root, (128, 128, 128), recon=ak.AK_PPM4, rk=3, precision=prec,
                    ref_rho=1.0, ref_p=1.0)
        m.upload(U0)
        m.new_dt()
        for _ in range(args.steps):
            m.step(0.0)
        c = m.counters()
        m.close()
        print(json.dumps({"case": "profile-ppm", "form": args.form, "cells": 256 ** 3,
                          "steps": args.steps, "counters": c}), flush=True)
        return 0 if c[:2] == [0, 0] else 1
    root = (192, 192, 192)
    U0 = pgen.turbulence(root, seed=1, kmin=2, kmax=8, mach=0.5)
    m = ak.Mesh(root, (64, 64, 64), precision=prec, ref_rho=1.0, ref_p=1.0)
    m.upload(U0)
    dt = m.new_dt()
    for _ in range(args.steps):
        dt = m.step(0.0)
    c = m.counters()
    m.close()
    print(json.dumps({"case": "profile", "form": args.form, "cells": 192 ** 3,
                      "steps": args.steps, "dt": dt, "counters": c}), flush=True)
    return 0 if c[:2] == [0, 0] else 1


def time_large(ak, torch, case, steps, warmup):
    """The large configurations, timed like the main line (graph-replayed ak_step with the
    device-resident dt, CUDA events on the mesh's stream, clocks sampled meanwhile):
      c3: 512^3 in 64 MeshBlocks of 128^3, PPM4 + HLLC + RK3, k^-2 turbulence Mach 0.5,
          FP64 and mixed;
      c5: 768^3 in 512 MeshBlocks of 96^3, PLM + HLLC + RK2, mixed, solenoidal k^-2
          (2 <= |k| <= 16) turbulence, rms Mach 2, at least 50 steps.
    Inputs come from the torch form of the turbulence recipe, generated on the GPU.  For
    c3 the first step of both forms starts from the same state, and the line reports the
    L1 difference of the mixed state from the FP64 one after it, sqrt(sum_k L1_k^2) with
    L1_k the mean |U_k(mixed) - U_k(FP64)| over all cells (the FP64 GPU path itself
    matches the FP64 oracle to 1e-12 on sub-box replays, tests/test_gpu_large.py)."""
    import pgen
    c3 = case == "c3"
    root = 512 if c3 else 768
    nblk = 128 if c3 else 96
    rk = 3 if c3 else 2
    recon = ak.AK_PPM4 if c3 else ak.AK_PLM
    steps = steps if c3 else max(steps, 50)
    forms = [("fp64", ak.AK_FP64), ("mixed", ak.AK_MIXED)] if c3 else [("mixed", ak.AK_MIXED)]
    gen = dict(seed=3, kmin=2, kmax=8, mach=0.5) if c3 else \
        dict(seed=5, kmin=2, kmax=16, mach=2.0, solenoidal=True)
    cells = root ** 3
    peaks, peak_kind = load_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    bytes_cu = 320.0 if rk == 3 else 200.0
    out = {"workload": (
        f"{root}^3 periodic in {(root // nblk) ** 3} MeshBlocks of {nblk}^3, "
        + ("PPM4+HLLC+RK3, k^-2 turbulence Mach 0.5" if c3 else
           "PLM+HLLC+RK2, solenoidal k^-2 turbulence (2<=|k|<=16) Mach 2")),
        "cells": cells, "steps": steps, "warmup": warmup,
        "l2": "inputs larger than L2"}
    ref = None
    for name, prec in forms:
        U0 = pgen.turbulence_device((root,) * 3, **gen)
        m = ak.Mesh((root,) * 3, (nblk,) * 3, recon=recon, rk=rk, precision=prec,
                    ref_rho=1.0, ref_p=1.0)
        m.upload_device(U0)
        del U0
        torch.cuda.empty_cache()
        dt0 = m.new_dt()
        m.step(dt0, want_dt_next=False)
        m.stream.synchronize()  # the state is read on another stream below
        g = m.ng
        inner = m.register_view(0)[:, :, g:-g, g:-g, g:-g]
        l1 = None
        if c3 and name == "fp64":
            ref = inner.clone()
        elif c3 and ref is not None:
            l1 = float(torch.sqrt(sum(((inner[:, v] - ref[:, v]).abs().mean()) ** 2
                                      for v in range(5))))
            ref = None
            torch.cuda.empty_cache()
        del inner
        for _ in range(warmup):
            m.step(0.0, want_dt_next=False)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        a.record(m.stream)
        for _ in range(steps):
            m.step(0.0, want_dt_next=False)
        b.record(m.stream)
        b.synchronize()
        clk = clocks.stop()
        ms = a.elapsed_time(b)
        value = cells * steps / (ms * 1e-3)
        gbs = value * bytes_cu / 1e9
        f = {"value": value, "unit": UNIT, "ms_per_step": ms / steps,
             "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                          "frac": gbs / hbm, "bytes_per_cell_update": bytes_cu,
                          "traffic": None, "peak_source": f"{peak_kind} hbm_gbs"},
             "dt0": dt0, "counters": m.counters(), "clocks": clk}
        if name == "fp64":
            f["roofline"]["note"] = "FP64 form: bound by the FP64 unit, not by HBM"
        elif c3:
            # mean DRAM bytes of the step's three stage launches
            f["roofline"]["traffic"] = traffic_per_launch("ppm4_mixed", cells)
            f["roofline"]["algorithmic_bytes_per_launch"] = bytes_cu / 3 * cells
        if l1 is not None:
            f["l1_vs_fp64_after_one_step"] = l1
        out[name] = f
        m.close()
        del m
        torch.cuda.empty_cache()
    return out


def run_large_case(args):
    """--case c3 / c5: one large configuration on its own, printed as one JSON line."""
    import torch
    from paper_2409_16053_gb300 import ak
    out = time_large(ak, torch, args.case, args.steps, args.warmup)
    out["case"] = args.case
    print(json.dumps(out), flush=True)
    forms = [v for k, v in out.items() if k in ("fp64", "mixed")]
    return 0 if all(f["counters"][:2] == [0, 0] for f in forms) else 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 512^3 PPM4+RK3 and 768^3 Mach-2 legs")
    ap.add_argument("--case", default="bench",
                    choices=["bench", "profile", "profile-smr", "profile-ppm", "c3", "c5"])
    ap.add_argument("--form", default="fp64", choices=["fp64", "mixed"])
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.case in ("profile", "profile-smr", "profile-ppm"):
        return run_profile_case(args)
    if args.case in ("c3", "c5"):
        return run_large_case(args)

    ws, rank, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import pgen
    from paper_2409_16053_gb300 import ak
    U0 = pgen.turbulence(ROOT_NX, seed=1 + rank, kmin=2, kmax=8, mach=0.5)

    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    r64 = time_form(ak, torch, ak.AK_FP64, U0, args.steps, args.warmup)
    rmx = time_form(ak, torch, ak.AK_MIXED, U0, args.steps, args.warmup)
    clk = clocks.stop()
    if dist:
        dist.barrier()

    def tmax(v):
        return max_over_ranks(dist, v)

    smr = None
    if rank == 0:
        smr = {"workload": "static refinement: 128^3 root in 32^3 blocks + 2 nested levels "
                           "of 16^3 blocks, 1016 leaves, 5,767,168 cells, Sedov, PLM+HLLC+RK2",
               "fp64": time_smr(ak, torch, ak.AK_FP64, args.steps, args.warmup),
               "mixed": time_smr(ak, torch, ak.AK_MIXED, args.steps, args.warmup)}
    t64 = tmax(r64["total_ms"])
    tmx = tmax(rmx["total_ms"])
    cells = ROOT_NX[0] * ROOT_NX[1] * ROOT_NX[2]
    value64 = job_rate(ws, cells, args.steps, t64)
    valuemx = job_rate(ws, cells, args.steps, tmx)

    large = None
    if rank == 0 and not args.no_large:
        large = {"c3": time_large(ak, torch, "c3", min(args.steps, 3), max(args.warmup, 3)),
                 "c5": time_large(ak, torch, "c5", 50, max(args.warmup, 3))}
    e2e = e2e_form(ak, torch, ak.AK_FP64, U0, max(2, args.steps // 2)) if rank == 0 else None
    e2e_mx = e2e_form(ak, torch, ak.AK_MIXED, U0, max(2, args.steps // 2)) if rank == 0 else None

    peaks, peak_kind = load_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    # FP64 stage kernel: ALU bound (FP64 pipe); per launch = mean of the two stages
    st64 = 0.5 * (r64["stage1_ms"] + r64["stage2_ms"])
    ach64 = FLOP_PER_CELL_STAGE * cells / (st64 * 1e-3) / 1e12
    # the FP64 instructions the kernel issues against the rate this GPU sustains
    fp64_rate = None
    if rank == 0:
        dfma_s = ak.ak_probe_fp64_rate(torch.cuda.current_stream().cuda_stream)
        inst_s = sum(FP64_INST_PER_CELL_NCU) / 2 * cells / (st64 * 1e-3)
        fp64_rate = {"inst_per_cell_stage_ncu": list(FP64_INST_PER_CELL_NCU),
                     "achieved_inst_per_s": inst_s, "measured_dfma_per_s": dfma_s,
                     "measured_per_clock_per_sm": dfma_s / (152 * clk["sm_mhz"] * 1e6)
                     if clk.get("sm_mhz") else None,
                     "frac_of_measured": inst_s / dfma_s,
                     "source": "ak_probe_fp64_rate: 8 independent DFMA chains per thread, "
                               "8 CTAs of 256 threads per SM"}
    # mixed stage kernel: HBM roofline on the algorithmic bytes per launch
    stmx = 0.5 * (rmx["stage1_ms"] + rmx["stage2_ms"])
    bytes_mx = 0.5 * (BYTES_STAGE[1] + BYTES_STAGE[2]) * cells
    ach_mx = bytes_mx / (stmx * 1e-3) / 1e9
    l1 = None
    if rank == 0:
        e64 = linear_wave_l1(ak, ak.AK_FP64)
        emx = linear_wave_l1(ak, ak.AK_MIXED)
        l1 = {"test": "3D sound wave, 32^3, amplitude 1e-6, one period, PLM+HLLC+RK2",
              "fp64": e64, "mixed": emx, "mixed_over_fp64": emx / e64}
    line = {
        "metric": METRIC, "value": value64, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t64 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "form": "FP64", "cells": cells,
                   "schedule": r64["schedule"], "schedule_mixed": rmx["schedule"],
                   "l2": "inputs larger than L2: 2 registers x 805 MB",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "roofline": {"bound": "alu", "achieved": ach64, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": ach64 / FP64_PEAK_TFLOPS,
                     "traffic": traffic_per_launch("fp64", cells),
                     "kernel": "stage_kernel<PLM, FP64> (mean of stage 1 and 2 launches)",
                     "peak_source": "derived: 152 SM x 2 DFMA/clk x 2 flop x 2.07 GHz "
                                    "(ncu's peak_sustained for DFMA: 304 per clock on "
                                    "152 SMs)",
                     "fp64_pipe_busy_ncu": FP64_PIPE_BUSY_NCU,
                     "measured_fp64_rate": fp64_rate},
        "mixed": {
            "value": valuemx, "unit": UNIT, "ms_per_step": tmx / args.steps, "dtype": "f32+f64",
            "roofline": {"bound": "hbm", "achieved": ach_mx, "peak": hbm, "unit": "GB/s",
                         "frac": ach_mx / hbm, "traffic": traffic_per_launch("mixed", cells),
                         "kernel": "stage_mx_kernel<PLM> (paired; mean of stage 1 and 2 "
                                   "launches)",
                         "peak_source": f"{peak_kind} hbm_gbs"},
            "e2e": e2e_mx,
        },
        "stage_ms": {"fp64": [r64["stage1_ms"], r64["stage2_ms"]],
                     "mixed": [rmx["stage1_ms"], rmx["stage2_ms"]]},
        "step_ms_best_median": {"fp64": r64["step_ms"], "mixed": rmx["step_ms"]},
        "counters": {"fp64": r64["counters"], "mixed": rmx["counters"]},
        "l1_error": l1,
        "smr": smr,
        "large": large,
        "e2e": e2e,
        # per form and step: 2 stage launches, the dt finalisation, and a ghost fill
        # before each stage unless the stage kernels read halos directly
        "gpu_launches": args.steps * 2 * (3 + 2 * (not r64["direct"])),
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
        line["cpu_baseline"]["one_core"] = cpu_baseline_one_core()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
