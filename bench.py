#!/usr/bin/env python
"""Throughput of the D3Q19 stream + collide step on GB300, in MLUPS and as a
fraction of the measured HBM roofline.

Default workload: periodic 256^3 lattice, FP32 storage, SRT, D3Q19-I
(improved) equilibrium, tau = 0.8, transverse shear wave u_y = 0.01 sin(2 pi
x / 256) on a background flow U_x = 0.1.  A bench "step" is one lattice time
step over all 256^3 cells (one launch of the fused stream + collide kernel).
The 2 x 1.27 GB of population grids are ~20x the 129 MB L2, so every step
streams from HBM (no L2 flush needed).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Prints one JSON line (rank 0).  With --gpus N > 1 (torchrun, one process per
GPU) each rank runs an independent replica of the workload ("replicas only":
the method's single-GPU path has no exchange step); value = total lattice
updates of all ranks / max-over-ranks time.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "D3Q19 MLUPS & % HBM roofline (FP32 vs 16-bit storage); adjoint/forward cost"
BYTES_PER_LUP = {"f64": 304, "f32": 152, "f16s": 76, "bf16s": 76}
# GB300 HBM3e nominal bandwidth (vendor figure); the measured copy bandwidth of
# MEASURED_PEAKS.json is the primary denominator, and a kernel that streams as
# well as that copy reads slightly above 1.0 against it.
NOMINAL_HBM_GBS = 7900.0
# Velocity-profile error of the walled channel after its 5000 steps against the
# FP64 oracle, per storage precision (tests/test_gpu_workloads.py): 16-bit
# storage cannot carry the per-step body-force increment of the shifted
# populations, so those rates buy no usable channel result.
CHANNEL_PROFILE_ERR = {"f32": "< 1e-5", "f16s": "1.0 (flow never starts)", "bf16s": "about 0.82 (stagnates)"}
DTYPE_NAME = {"f64": "f64", "f32": "f32", "f16s": "f16", "bf16s": "bf16"}


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["native", "reference"], default="native")
    p.add_argument("--n", type=int, default=256, help="lattice edge (workload is n^3)")
    p.add_argument("--precision", choices=["f64", "f32", "f16s", "bf16s"], default="f32")
    p.add_argument("--pattern", choices=["ab", "aa"], default="ab")
    p.add_argument("--collision", choices=["srt", "trt", "mrt"], default="srt")
    p.add_argument("--equilibrium", choices=["standard", "improved"], default="improved")
    p.add_argument("--tau", type=float, default=0.8)
    p.add_argument("--block", type=str, default=None, help="step kernel block 'bx,by'")
    p.add_argument("--cells-x", type=int, choices=[1, 2, 4], default=None,
                   help="step kernel cells per thread along x (default: library's choice)")
    p.add_argument("--graphs", type=int, choices=[0, 1], default=None,
                   help="1: lbm_step replays 16-step CUDA graphs (library default); 0: one launch per step")
    p.add_argument("--only-adjoint", action="store_true",
                   help="time only the adjoint workload (128^3) and print its figures")
    p.add_argument("--no-extras", action="store_true", help="main line only (profiling runs)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    return p.parse_args(argv)


# ------------------------------------------------------------------ helpers

def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("nccl")
        return dist, int(os.environ["RANK"]), ws, int(os.environ.get("LOCAL_RANK", "0"))
    return None, 0, 1, 0


def max_over_ranks(value, dist, device):
    """Max of a float over all ranks (identity without a process group)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while a region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.6)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = []
        smax = None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        load = [s for s in sm if smax and s > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def read_traffic(kernel_key):
    """DRAM bytes per launch of `kernel_key` from the committed ncu summary, or
    None when the summary is absent or was taken on a different kernel source."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.txt")
    if not os.path.exists(path):
        return None, None
    entries = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        if "kernel" in parts:
            entries[parts["kernel"]] = parts
    e = entries.get(kernel_key)
    if not e:
        return None, None
    src = b""
    for f in ("lbm_device.cuh", "lbm_step.cuh"):
        src += open(os.path.join(ROOT, "paper_1803_04937_gb300", "csrc", f), "rb").read()
    sha = hashlib.sha256(src).hexdigest()[:16]
    if e.get("source_sha") != sha:
        return None, sha
    return float(e["dram_bytes_per_lup"]), sha


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def shear_workload(nx, ny, nz, device):
    from paper_1803_04937_gb300 import inputs
    return inputs.shear_wave(nx, ny, nz, U=(0.1, 0.0, 0.0), amplitude=0.01, device=device)


# ------------------------------------------------------------------ GPU timing

GRAPH_STEPS = 16  # lbm_step replays CUDA graphs of this many steps


def warm(sim, warmup):
    """`warmup` untimed steps, then GRAPH_STEPS more so that the CUDA graph for
    the grid (A/B) or parity (AA) the timed steps start from is captured
    before the timed region (an even count returns to the same grid)."""
    sim.step(warmup)
    sim.step(GRAPH_STEPS)
    return warmup + GRAPH_STEPS


def time_steps(sim, steps, warmup):
    """Average device time (s) per lattice step over `steps` launches, after
    `warmup` launches; CUDA events on the simulation's stream."""
    import torch
    s = sim.stream
    warm(sim, warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    sim.step(steps)
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1e-3 / steps


def make_sim(args, n, precision=None, pattern=None, collision=None, equilibrium=None, device="cuda", stencil=19):
    from paper_1803_04937_gb300.lbm import Simulation
    block = tuple(int(x) for x in args.block.split(",")) if args.block else None
    sim = Simulation(n, n, n, equilibrium=equilibrium or args.equilibrium, collision=collision or args.collision,
                     tau=args.tau, precision=precision or args.precision, pattern=pattern or args.pattern,
                     device=device, block=block, cells_x=args.cells_x, stencil=stencil,
                     graphs=None if args.graphs is None else bool(args.graphs))
    rho, u = shear_workload(n, n, n, device)
    sim.init(rho, u.float() if (precision or args.precision) != "f64" else u)
    del rho, u
    return sim


def variant_mlups(args, n, **kw):
    import torch
    sim = make_sim(args, n, **kw)
    t = time_steps(sim, 400, 10)
    prec = kw.get("precision") or args.precision
    bpl = BYTES_PER_LUP[prec] * kw.get("stencil", 19) // 19
    out = {"mlups": n ** 3 / t / 1e6, "gbs": bpl * n ** 3 / t / 1e9}
    sim.close()
    del sim
    torch.cuda.empty_cache()
    return out


def config_variants(peak):
    """Throughput on the other workload configurations, each on its own lattice:
    the walled channel 512x256x256 (TRT 3/16, tau 0.6, body force; FP32 / FP16S /
    BF16S with A/B, and FP32 with the in-place AA pattern) and decaying
    turbulence at 768^3 (SRT, tau 0.51, FP32 / FP16S with the memory-lean
    in-place AA pattern, and FP16S with A/B, which fits as well)."""
    import torch

    from paper_1803_04937_gb300 import inputs
    from paper_1803_04937_gb300.lbm import Simulation
    out = {}
    nu = (0.6 - 0.5) / 3
    a = 8 * nu * 0.05 / 256 ** 2
    for prec, pattern in (("f32", "ab"), ("f16s", "ab"), ("bf16s", "ab"), ("f32", "aa")):
        sim = Simulation(512, 256, 256, equilibrium="improved", collision="trt", tau=0.6, precision=prec,
                         force=(a, 0.0, 0.0), walls=(False, True, False), pattern=pattern)
        rho, u = inputs.rest(512, 256, 256, device="cuda")
        sim.init(rho, u.float() if prec != "f64" else u)
        del rho, u
        t = time_steps(sim, 200, 10)
        cells = 512 * 256 * 256
        key = "channel_512x256x256_" + prec + ("" if pattern == "ab" else "_aa")
        out[key] = {"mlups": cells / t / 1e6, "gbs": BYTES_PER_LUP[prec] * cells / t / 1e9,
                    "profile_err_after_5000_steps": CHANNEL_PROFILE_ERR[prec]}
        sim.close()
        del sim
        torch.cuda.empty_cache()
    n = 768
    _, u = inputs.hit_spectrum(n, n, n, u_rms=0.04, seed=4, device="cuda")
    u = u.float()
    for prec, pattern in (("f32", "aa"), ("f16s", "aa"), ("f16s", "ab")):
        sim = Simulation(n, n, n, equilibrium="improved", collision="srt", tau=0.51, precision=prec, pattern=pattern)
        sim.init(None, u)
        t = time_steps(sim, 64, 4)
        out["hit_768_%s_%s" % (pattern, prec)] = {"mlups": n ** 3 / t / 1e6,
                                                  "gbs": BYTES_PER_LUP[prec] * n ** 3 / t / 1e9}
        sim.close()
        del sim
        torch.cuda.empty_cache()
    del u
    torch.cuda.empty_cache()
    for v in out.values():
        v["frac"] = v["gbs"] / peak
    return out


def adjoint_ratio(args, n=128, horizon=400):
    """Adjoint cost on the adjoint workload's lattice (periodic n^3, FP32, SRT,
    D3Q19-I, tau = 0.7): per-step kernel times, and the whole differentiable
    run (forward with sqrt(T) checkpoints, then backward = recompute + adjoint)
    through the autograd.Function."""
    import ctypes

    import torch

    from paper_1803_04937_gb300 import _lib, adjoint, inputs
    from paper_1803_04937_gb300.lbm import Simulation
    sim = Simulation(n, n, n, equilibrium="improved", collision="srt", tau=0.7, precision="f32")
    rho, u = inputs.random_solenoidal(n, n, n, kmax=8, u_rms=0.02, seed=1, device="cuda")
    _, tgt = inputs.random_solenoidal(n, n, n, kmax=8, u_rms=0.02, seed=2, device="cuda")
    sim.init(None, u.float())
    t_fwd = time_steps(sim, 200, 10)
    lib = _lib.load()
    lam = [torch.zeros((19, n, n, n), dtype=torch.float32, device="cuda") for _ in range(2)]
    gw = torch.zeros(2, dtype=torch.float64, device="cuda")
    gwp = ctypes.cast(ctypes.c_void_p(gw.data_ptr()), ctypes.POINTER(ctypes.c_double))
    state = ctypes.c_void_p(sim.grids[0].data_ptr())  # any A/B grid is a valid state for timing
    lp = [ctypes.c_void_p(t.data_ptr()) for t in lam]
    s = sim.stream
    # deferred dL/domega sums, as the autograd backward runs them (flushed inside the timed region)
    _lib.check(lib.lbm_set_option(sim.handle, _lib.OPT_ADJ_DEFER_SUM, 1.0), sim.handle)
    for i in range(10):
        _lib.check(lib.lbm_adjoint_step(sim.handle, state, lp[i % 2], lp[1 - i % 2], gwp), sim.handle)
    _lib.check(lib.lbm_adjoint_flush(sim.handle), sim.handle)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = 200
    e0.record(s)
    for i in range(reps):
        lib.lbm_adjoint_step(sim.handle, state, lp[i % 2], lp[1 - i % 2], gwp)
    lib.lbm_adjoint_flush(sim.handle)
    e1.record(s)
    torch.cuda.synchronize()
    t_adj = e0.elapsed_time(e1) * 1e-3 / reps
    sim.close()
    del lam, sim
    # whole differentiable run (second of two, so the caching allocator holds
    # the checkpoint and recompute buffers)
    for _ in range(2):
        u0 = u.float().clone().requires_grad_(True)
        tau = torch.tensor(0.7, dtype=torch.float64, requires_grad=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, uT = adjoint.simulate(u0, tau, horizon, n, n, n, precision="f32")
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        L = 0.5 * ((uT.double() - tgt) ** 2).sum()
        L.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
    return {"grid": "%d^3" % n, "horizon": horizon, "forward_step_ms": t_fwd * 1e3, "adjoint_step_ms": t_adj * 1e3,
            "adjoint_kernel_gbs": 228 * n ** 3 / t_adj / 1e9,
            "ratio_recompute_plus_adjoint_over_forward": (t_fwd + t_adj) / t_fwd,
            "forward_pass_s": t1 - t0, "backward_pass_s": t2 - t1,
            "ratio_backward_over_forward_pass": (t2 - t1) / (t1 - t0)}


def e2e(args, n, dist=None, device=None, calls=3, steps_per_call=(100, 2000)):
    """Same metric through the C ABI from pinned host buffers: each call is
    lbm_init reading rho, u from host memory, steps_per_call steps, and
    lbm_moments writing rho, u to host memory, then a stream synchronise (the
    host-device transfers are inside the timed region: the init and moments
    kernels read and write the pinned host buffers directly).  Reported for
    100 steps per call (the headline figure) and for the shear-wave
    configuration's 2000 steps per call.  Under torchrun every rank runs its
    replica; barrier before, max-over-ranks time, all ranks' updates counted
    (bytes per step are per rank)."""
    import torch
    from paper_1803_04937_gb300.lbm import Simulation
    ws = dist.get_world_size() if dist else 1
    sim = Simulation(n, n, n, equilibrium=args.equilibrium, collision=args.collision, tau=args.tau,
                     precision=args.precision, pattern=args.pattern, device=device or "cuda")
    dt = torch.float64 if args.precision == "f64" else torch.float32
    rho, u = shear_workload(n, n, n, "cpu")
    rho_h = rho.to(dt).pin_memory()
    u_h = u.to(dt).pin_memory()
    out = (torch.empty(rho_h.shape, dtype=dt, pin_memory=True), torch.empty(u_h.shape, dtype=dt, pin_memory=True))
    bi = rho_h.numel() * rho_h.element_size() + u_h.numel() * u_h.element_size()
    bo = out[0].numel() * out[0].element_size() + out[1].numel() * out[1].element_size()
    res = {}
    for spc in steps_per_call:
        sim.run_host(rho_h, u_h, spc, out)  # warm-up (also captures the step graph)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(calls):
            sim.run_host(rho_h, u_h, spc, out)
        t = max_over_ranks(time.perf_counter() - t0, dist, device)
        res[spc] = {"value": ws * n ** 3 * spc * calls / t / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": bi / spc,
                    "d2h_bytes_per_step": bo / spc, "lbm_steps_per_call": spc, "h2d_bytes_per_call": bi,
                    "d2h_bytes_per_call": bo, "calls": calls}
    sim.close()
    head = dict(res[steps_per_call[0]])
    head["api"] = "C ABI lbm_init / lbm_step / lbm_moments on pinned host buffers (zero-copy reads and writes)"
    for spc in steps_per_call[1:]:
        head["at_%d_steps_per_call" % spc] = {"value": res[spc]["value"], "h2d_bytes_per_step": res[spc][
            "h2d_bytes_per_step"], "d2h_bytes_per_step": res[spc]["d2h_bytes_per_step"]}
    return head


# ------------------------------------------------------------------ CPU oracle

def oracle_sample(target_seconds, cross=32, single_thread_seconds=0.0):
    """Times the FP64 CPU oracle on a 256 x c x c periodic slab of the shear-wave
    workload (the flow is invariant in y and z, so every slab is an exact
    sample of the 256^3 lattice), sized to about `target_seconds`."""
    import numpy as np

    import oracle
    nx = 256
    cfg1 = oracle.Config(nx, 8, 8, equilibrium=oracle.IMPROVED, collision=oracle.SRT, tau=0.8)
    rho, u = shear_workload(nx, 8, 8, "cpu")
    f = oracle.init(cfg1, rho.numpy(), u.numpy())
    t0 = time.perf_counter()
    oracle.step(cfg1, f, 2)
    rate = 2 * cfg1.ncell / max(time.perf_counter() - t0, 1e-6)  # LUP/s
    c = int(max(4, min(cross, math.sqrt(max(rate * target_seconds / nx, 16)))))
    cfg = oracle.Config(nx, c, c, equilibrium=oracle.IMPROVED, collision=oracle.SRT, tau=0.8)
    rho, u = shear_workload(nx, c, c, "cpu")
    f = oracle.init(cfg, rho.numpy(), u.numpy())
    steps = max(1, int(round(rate * target_seconds / cfg.ncell)))
    t0 = time.perf_counter()
    f = oracle.step(cfg, f, steps)
    t = time.perf_counter() - t0
    assert np.isfinite(f).all()
    out = {"value": cfg.ncell * steps / t / 1e6, "unit": "MLUPS", "cores": oracle.max_threads(), "kind": "oracle",
           "sample": "FP64 C oracle, %d steps of a periodic 256x%dx%d slab of the shear-wave workload "
                     "(y,z-invariant, so an exact sample of 256^3), %.1f s" % (steps, c, c, t)}
    if single_thread_seconds > 0:
        # the same oracle on one thread, on a slab sized to about single_thread_seconds
        cfg.nthreads = 1
        f = oracle.init(cfg, rho.numpy(), u.numpy())
        t0 = time.perf_counter()
        oracle.step(cfg, f, 1)
        t1 = time.perf_counter() - t0
        steps1 = max(1, int(single_thread_seconds / max(t1, 1e-6)))
        t0 = time.perf_counter()
        oracle.step(cfg, f, steps1)
        t1 = time.perf_counter() - t0
        out["value_1_thread"] = cfg.ncell * steps1 / t1 / 1e6
        out["sample_1_thread"] = "%d steps of the same slab on 1 thread, %.1f s" % (steps1, t1)
        # the thread count is process-wide in OpenMP: restore it
        tiny = oracle.Config(1, 1, 1, nthreads=out["cores"])
        oracle.step(tiny, oracle.init(tiny, np.ones((1, 1, 1)), np.zeros((3, 1, 1, 1))), 1)
    return out


def run_reference(args):
    dist, rank, ws, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    nx = 256
    probe = oracle_sample(1.0, cross=8)
    rate = probe["value"] * 1e6
    budget = 90.0  # seconds for warmup + steps
    c = int(max(2, min(32, math.sqrt(rate * budget / (nx * max(1, args.steps + args.warmup))))))
    cfg = oracle.Config(nx, c, c, equilibrium=oracle.IMPROVED if args.equilibrium == "improved" else oracle.STANDARD,
                        collision={"srt": oracle.SRT, "trt": oracle.TRT, "mrt": oracle.MRT}[args.collision],
                        tau=args.tau)
    rho, u = shear_workload(nx, c, c, "cpu")
    f = oracle.init(cfg, rho.numpy(), u.numpy())
    f = oracle.step(cfg, f, args.warmup)
    t0 = time.perf_counter()
    f = oracle.step(cfg, f, args.steps)
    t = time.perf_counter() - t0
    value = cfg.ncell * args.steps / t / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "D3Q19 shear wave, periodic 256^3 (timed on a 256x%dx%d slab sample), %s, %s, "
                               "tau=%g" % (c, c, args.equilibrium, args.collision, args.tau),
                   "precision": "f64 (CPU oracle)"},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": oracle.max_threads(), "kind": "oracle",
                         "sample": "each step: one oracle time step of a periodic 256x%dx%d slab (exact y,z sample "
                                   "of the 256^3 shear wave)" % (c, c)},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ main

def run_native(args):
    import torch
    dist, rank, ws, local = _dist()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    n = args.n
    sim = make_sim(args, n, device=device)
    warmup_run = warm(sim, args.warmup)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    with sampler:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(sim.stream)
        sim.step(args.steps)
        e1.record(sim.stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_local = e0.elapsed_time(e1) * 1e-3
    t = max_over_ranks(t_local, dist, device)
    red = sim.reduce()
    ok = red["nonfinite"] == 0
    sim.close()
    del sim
    torch.cuda.empty_cache()

    cells = n ** 3
    value = ws * cells * args.steps / t / 1e6
    per_launch = t_local / args.steps
    peak, peak_kind = measured_peaks()
    achieved = BYTES_PER_LUP[args.precision] * cells / per_launch / 1e9
    cx = args.cells_x or (4 if args.precision in ("f16s", "bf16s") else 1)
    if args.pattern == "ab":
        kname = "k_ab%d<%s>" % (cx, args.precision) + ("[mrt]" if args.collision == "mrt" else "")
    else:
        kname = "k_aa_even%d+k_aa_odd%d<%s>" % (cx, cx, args.precision) + ("[mrt]" if args.collision == "mrt" else "")
    traffic_per_lup, _ = read_traffic(kname)
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE_NAME[args.precision], "data": "synthetic",
        "config": {"workload": "D3Q19 shear wave u_y=0.01 sin(2 pi x/%d) on U_x=0.1, periodic %d^3" % (n, n),
                   "equilibrium": args.equilibrium, "collision": args.collision, "tau": args.tau,
                   "warmup_steps_run": warmup_run,
                   "precision": args.precision, "pattern": args.pattern,
                   "l2": "inputs larger than L2 (%.2f GB per grid vs 129 MB L2)" % (
                       BYTES_PER_LUP[args.precision] / 2 * cells / 1e9),
                   "parallelism": "replicas x%d" % ws, "finite": ok},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "peak_nominal": NOMINAL_HBM_GBS, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                     "algorithmic_bytes_per_lup": BYTES_PER_LUP[args.precision],
                     "traffic": traffic_per_lup * cells if traffic_per_lup else None,
                     "kernel": kname},
        "gpu_launches": args.steps,
        "clocks": sampler.summary(),
    }
    if not args.no_extras and ws > 1:
        line["e2e"] = e2e(args, n, dist, device)  # every rank takes part
    if rank == 0 and not args.no_extras and ws == 1:
        line["e2e"] = e2e(args, n)
        variants = {}
        for prec in ("f16s", "bf16s"):
            variants[prec] = variant_mlups(args, n, precision=prec)
        variants["aa_" + args.precision] = variant_mlups(args, n, pattern="aa")
        variants["aa_f16s"] = variant_mlups(args, n, pattern="aa", precision="f16s")
        variants["trt_" + args.precision] = variant_mlups(args, n, collision="trt")
        variants["mrt_" + args.precision] = variant_mlups(args, n, collision="mrt")
        variants["mrt_f16s"] = variant_mlups(args, n, collision="mrt", precision="f16s")
        variants["standard_" + args.precision] = variant_mlups(args, n, equilibrium="standard")
        variants["d3q27_" + args.precision] = variant_mlups(args, n, equilibrium="standard", stencil=27)
        variants["d3q27_f16s"] = variant_mlups(args, n, equilibrium="standard", stencil=27, precision="f16s")
        for k, v in variants.items():
            v["frac"] = v["gbs"] / peak
        variants["f16s"]["speedup_vs_main"] = variants["f16s"]["mlups"] / value
        variants["bf16s"]["speedup_vs_main"] = variants["bf16s"]["mlups"] / value
        variants["d3q27_" + args.precision]["d3q19_speedup_over_d3q27"] = value / variants["d3q27_" + args.precision][
            "mlups"]
        line["variants"] = variants
        line["configs"] = config_variants(peak)
        line["adjoint"] = adjoint_ratio(args)
    elif rank == 0 and args.no_extras:
        line["e2e"] = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample(12.0, single_thread_seconds=4.0)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.only_adjoint:
        print(json.dumps({"adjoint": adjoint_ratio(args)}), flush=True)
        return 0
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
