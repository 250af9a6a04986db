#!/usr/bin/env python3
"""Benchmark: D3Q19 N+1-phase lattice Boltzmann step of the Diffuse Solid Method.

Workload: the plain FP32 D3Q19 pillar-slab lattice, 256x256x192 = 12,582,912
nodes (square pillars 10 wide, 30 high, pitch 32 on an 8-node base, liquid slab
z in [38, 98), contact angle drawn in [90, 150] degrees from seed 0), synthetic.
One "step" = one full lattice Boltzmann time step through libdsm: the moments
pass plus the fused pass over every node.  Inputs (3.9 GB of populations) are
far larger than the 129 MB L2, so no flush is needed between steps.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the host cores on a bounded slice of the same workload instead.

Multi-GPU (torchrun, N ranks): every rank runs its own independent lattice
(replicas; the method has no exchange between independent problems); value =
all ranks' node updates / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "D3Q19 N+1-phase LBM MLUPS & HBM-roofline %; sweep solves/s with p50/p99 latency"


def lu_bytes(lattice: str, prec: str, g_eq: bool):
    """Algorithmic bytes per lattice update of the fused pass and of the moments
    pass.  Population form: read and write f and g once, read C1 (FP32 D3Q19:
    308 B; 16-bit storage with FP32 g_0: 160 B).  g held as g_eq (tau_g = 1):
    read and write f, read C1, write A and u in the fused pass; read A, u and the
    previous C and write C in the moments pass.  The fused pass's read of C, just
    written by the moments pass, is not counted (an L2-resident field)."""
    q, d = (19, 3) if lattice == "D3Q19" else (9, 2)
    real = 8 if prec == "f64" else 4
    st = {"f64": 8, "f32": 4, "bf16": 2, "f16": 2}[prec]
    g_read = (q - 1) * st + 4 if st == 2 else q * st
    if g_eq:
        return 2 * q * st + real + (1 + d) * real, (1 + d) * real + 2 * real
    return 2 * q * st + 2 * g_read + real, g_read + real


def lu_bytes_single(prec: str):
    """Algorithmic bytes per lattice update of the one-pass step (D3Q19, g held
    as g_eq): read and write f, read and write (A, u) and C, read C1.  FP32:
    152 + 40 + 4 = 196 B; 16-bit storage of f: 76 + 40 + 4 = 120 B."""
    real = 8 if prec == "f64" else 4
    st = {"f64": 8, "f32": 4, "bf16": 2, "f16": 2}[prec]
    return 2 * 19 * st + 2 * 5 * real + real
SHAPE = (256, 256, 192)
WORKLOAD = "D3Q19 FP32 pillar-slab 256x256x192 (12.58M nodes), plain method, stage-2 LB step"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        with open(self.path) as f:
            lines = f.readlines()
        os.unlink(self.path)
        return parse_clocks(lines)


def parse_clocks(lines):
    """Median SM clock, maximum SM clock and the throttle reasons seen in the
    CSV lines of the ClockSampler query (header and malformed lines skipped)."""
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [s.strip() for s in line.split(",")]
        if len(parts) < 9 or not parts[1].split() or not parts[1].split()[0].isdigit():
            continue
        sm.append(float(parts[1].split()[0]))
        mx = float(parts[2].split()[0])
        for nm, v in zip(names, parts[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
    sm.sort()
    return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(sm)}


def aggregate(t_local: float, units_local: float, dist=None):
    """Replica timing over ranks: the job time is the slowest rank's, the
    throughput all ranks' units over that time.  Returns (t_max, units/t_max)."""
    t_max, units = t_local, units_local
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        import torch
        dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" \
            else torch.device("cpu")
        tt = torch.tensor([t_local, units_local], dtype=torch.float64, device=dev)
        t = tt[:1].clone()
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        u = tt[1:].clone()
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        t_max, units = float(t.item()), float(u.item())
    return t_max, units / t_max


def shard(items, rank: int, world: int):
    """Independent problems are split across replicas by index."""
    return [it for i, it in enumerate(items) if i % world == rank]


def measured_traffic(name="zstep_kernel_d3q19_f32"):
    """DRAM bytes per launch of the fused kernel from the committed ncu summary,
    or None when the kernel source has changed since the counters were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", name + "_traffic.txt")
    if not os.path.exists(path):
        return None
    rec = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            rec[k.strip()] = v.strip()
    h = hashlib.sha256()
    for f in ("dsm_lb_impl.cuh", "dsm_common.cuh", "dsm_zstep.cuh"):
        with open(os.path.join(ROOT, "paper_2504_19941_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != rec.get("kernel_source_sha256_16"):
        return None
    return float(rec["bytes_per_launch"])


def make_case(shape, lattice="D3Q19"):
    import synthetic as S
    if lattice == "D2Q9":
        return S.pillar_row_2d(*shape, liquid=(38, min(98, shape[1] - 4)))
    if tuple(shape) == SHAPE:
        return S.pillar_slab_3d(*SHAPE)
    nz = shape[2]
    return S.pillar_slab_3d(*shape, liquid=(38, min(98, nz - 4)))


class OracleSlice:
    """The FP64 oracle, as it stands, on a 64x64x48 slice of the workload: the
    bounded sample both the CPU baseline and the reference arm time."""
    SHAPE = (64, 64, 48)

    def __init__(self):
        import numpy as np
        import oracle as O
        import synthetic as S
        self.O = O
        case = S.pillar_slab_3d(*self.SHAPE, pitch=32, width=10, height=12, base=4, liquid=(16, 32))
        k, _ = O.kappa_from_angle(case.theta_deg, case.g23, case.g12)
        self.p = O.make_params(O.D3Q19, self.SHAPE, k, alpha_s=case.alpha_s)
        self.c1 = O.solid_profile(case.solid_sd, case.alpha_s)
        self.f, self.g = O.lb_init(self.p, 2, self.c1, case.c2)
        self.n = int(np.prod(self.SHAPE))

    def run(self, max_seconds):
        """Oracle steps, two at a time, until max_seconds have passed: (steps, seconds)."""
        steps, t0 = 0, time.perf_counter()
        while True:
            self.f, self.g = self.O.lb_run(self.p, 2, self.c1, self.f, self.g, 2)
            steps += 2
            if time.perf_counter() - t0 > max_seconds:
                break
        return steps, time.perf_counter() - t0

    @staticmethod
    def cores():
        return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def cpu_baseline(max_seconds=15.0):
    """The FP64 oracle, as it stands, on a 64x64x48 slice of the workload."""
    sl = OracleSlice()
    sl.run(0.0)  # warm
    steps, dt = sl.run(max_seconds)
    return {"value": sl.n * steps / dt / 1e6, "unit": "MLUPS", "cores": sl.cores(), "kind": "oracle",
            "sample": f"D3Q19 FP64 oracle, 64x64x48 pillar-slab slice, {steps} steps, {dt:.1f} s"}


def oracle_single_core(max_seconds=5.0):
    """The same oracle slice on one host core (a child process with one OpenMP
    thread): the single-core figure next to the all-cores one."""
    import subprocess
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-one-core",
                        str(max_seconds)], env=env, capture_output=True, text=True, timeout=300)
    try:
        return json.loads(r.stdout.strip().splitlines()[-1])
    except (ValueError, IndexError):
        return {"error": (r.stderr or r.stdout)[-200:]}


def run_reference(args, rank, world):
    """The reference arm: the oracle timed on the host cores.  Each of the K
    timed steps (after W untimed ones) is a bounded sample of the workload --
    oracle steps on the 64x64x48 slice for about 100 s / (K + W), at least 0.2 s
    -- so that the whole run takes about two minutes."""
    if rank != 0:
        return 0
    per_step = min(20.0, max(0.2, 100.0 / max(args.steps + args.warmup, 1)))
    sl = OracleSlice()
    lu, secs, steps_done = 0, 0.0, 0
    for i in range(args.warmup + args.steps):
        steps, dt = sl.run(per_step)
        if i >= args.warmup:
            lu += sl.n * steps
            secs += dt
            steps_done += steps
    value = lu / secs / 1e6
    out = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup,
           # one step of the full workload at the sampled rate
           "ms_per_step": SHAPE[0] * SHAPE[1] * SHAPE[2] / (value * 1e6) * 1e3,
           "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference", "config": gpu_config(SHAPE, world, "populations"),
           "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": sl.cores(), "kind": "oracle",
                            "sample": f"each step: D3Q19 FP64 oracle LB steps on a 64x64x48 "
                                      f"pillar-slab slice for {per_step:.2f} s ({steps_done} oracle "
                                      f"steps in {secs:.1f} s timed)"},
           "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0},
           "cpu_single_core": oracle_single_core()}
    print(json.dumps(out), flush=True)
    return 0


def gpu_config(shape, world, g_storage, lattice="D3Q19", rho3=1.0, tau3=1.0, faces=None):
    nodes = 1
    for v in shape:
        nodes *= int(v)
    if lattice == "D2Q9":
        name = f"D2Q9 FP32 pillar-row {shape[0]}x{shape[1]}"
    elif tuple(shape) == SHAPE:
        name = WORKLOAD
    else:
        name = f"D3Q19 FP32 pillar-slab {shape[0]}x{shape[1]}x{shape[2]} (profiling size)"
    if rho3 != 1.0 or tau3 != 1.0:
        name += f", gas density {rho3}, gas tau {tau3} (liquid 1, 1)"
    if faces:
        name += ", faces " + "/".join(faces)
    return {"workload": name, "lattice": lattice, "nodes": nodes,
            "global_batch": world, "parallelism": f"replicas x{world}",
            "g_storage": g_storage,
            "l2": f"f populations alone {nodes * (9 if lattice == 'D2Q9' else 19) * 4 / 1e9:.1f} GB "
                  "per buffer, larger than L2; no flush"}


def run_gpu(args, rank, world):
    import torch
    import paper_2504_19941_gb300 as P
    from paper_2504_19941_gb300 import _lib

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    shape = tuple(int(v) for v in args.shape.split(","))
    lattice = args.lattice
    if lattice == "D2Q9" and len(shape) != 2:
        shape = (4096, 4096)
    case = make_case(shape, lattice)
    faces = tuple(args.faces.split(",")) if args.faces else None
    store = args.storage
    params = P.make_params(lattice, shape, store, theta_deg=case.theta_deg, g12=case.g12,
                           g23=case.g23, alpha_s=case.alpha_s, rho3=args.rho3, tau3=args.tau3,
                           faces=faces)
    lat = P.Lattice(params, device=dev)
    lat.set_g_storage(args.g_storage)
    lat.set_step_form(args.step_form, args.zrun)
    sd_h = torch.as_tensor(case.solid_sd, dtype=torch.float32).pin_memory()
    c2_h = torch.as_tensor(case.c2, dtype=torch.float32).pin_memory()
    sd_d = sd_h.to(dev, non_blocking=True)
    c2_d = c2_h.to(dev, non_blocking=True)
    lat.set_solid_distance(sd_d)
    lat.set_fluid(c2_d)
    n = lat.n
    h = lat.h
    # the one-pass step where the lattice allows it (one launch per step),
    # else the moments pass and the fused pass (two launches)
    single = lat.single_pass

    def one_step():
        if single:
            _lib.dsm_step(h, 1)
        else:
            _lib.dsm_step_moments(h)
            _lib.dsm_step_collide(h)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    g_eq = lat.g_implicit
    if single:
        k2_b, k1_b = lu_bytes_single(store), 0
    else:
        k2_b, k1_b = lu_bytes(lattice, store, g_eq)
    stream = torch.cuda.current_stream(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        e0.record(stream)
        for k in range(args.steps):
            if single:
                ev[k][0].record(stream)
                _lib.dsm_step(h, 1)
            else:
                _lib.dsm_step_moments(h)
                ev[k][0].record(stream)
                _lib.dsm_step_collide(h)
            ev[k][1].record(stream)
        e1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_total = e0.elapsed_time(e1) / 1e3
    t_k2 = sum(a.elapsed_time(b) for a, b in ev) / len(ev) / 1e3
    obs = lat.observables()
    assert obs["nonfinite"] == 0, "non-finite state after the timed steps"
    t_max, lups = aggregate(t_total, float(n * args.steps), dist)
    value = lups / 1e6

    # end to end through the public API with host buffers: H2D of the geometry
    # and the liquid field, set_solid, set_fluid, K steps, D2H of the liquid field
    out_h = torch.empty(n, dtype=torch.float32).pin_memory()
    lat2 = lat
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    sd_d.copy_(sd_h, non_blocking=True)
    c2_d.copy_(c2_h, non_blocking=True)
    lat2.set_solid_distance(sd_d)
    lat2.set_fluid(c2_d)
    lat2.step(args.steps)
    f_out = lat2.field("C2")
    out_h.copy_(f_out, non_blocking=True)
    s1.record(stream)
    torch.cuda.synchronize()
    t_e2e, lups_e2e = aggregate(s0.elapsed_time(s1) / 1e3, float(n * args.steps), dist)
    e2e = {"value": lups_e2e / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": 2 * 4 * n / args.steps, "d2h_bytes_per_step": 4 * n / args.steps}

    peak, peak_kind = _peaks()
    achieved = k2_b * n / t_k2 / 1e9
    default = (shape == SHAPE and lattice == "D3Q19" and args.rho3 == 1.0 and args.tau3 == 1.0
               and not faces and store == "f32")
    if single:
        traffic = measured_traffic("zstep_kernel_d3q19_f32") if default else None
    else:
        traffic = (measured_traffic("node_kernel_d3q19_f32_geq" if g_eq else "node_kernel_d3q19_f32")
                   if default else None)
    step_achieved = (k2_b + k1_b) * n / (t_max / args.steps) / 1e9
    # the two secondary fractions of the measurement definitions: DRAM bytes
    # that ncu measured per lattice update, and B_min, one read and one write
    # of f and g per node plus a read of C1 (a form that moves less, as the
    # g_eq form does, is credited for the bytes it avoids)
    b_min = lu_bytes(lattice, store, False)[0]  # the population form's fused-pass bytes
    lups_gpu = n * args.steps / t_max  # one GPU's lattice updates per second

    if rank == 0:
        cb = cpu_baseline() if world == 1 and not args.no_cpu_baseline else None
        out = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f32" if store == "f32" else store + "-storage/f32",
               "data": "synthetic",
               "config": gpu_config(shape, world,
                                    "g_eq (tau_g = 1): A, u per node" if g_eq else "populations",
                                    lattice, args.rho3, args.tau3, faces),
               "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                            "frac": achieved / peak, "traffic": traffic,
                            "kernel": ("zstep_kernel<f32,f32%s> (one pass per step, %d z planes "
                                       "per block)" % (",density contrast" if args.rho3 != 1.0 else "",
                                                       _lib.dsm_step_info(h)[1]))
                                      if single else
                                      "node_kernel<%s,f32,stage2,step,%s%s>" %
                                      (lattice, "g_eq" if g_eq else "populations",
                                       ",density contrast" if args.rho3 != 1.0 else ""),
                            "bytes_per_lu": k2_b, "peak_source": peak_kind,
                            "k2_ms": t_k2 * 1e3, "step_bytes_per_lu": k1_b + k2_b,
                            "step_achieved": step_achieved, "step_frac": step_achieved / peak,
                            "measured_bytes_per_lu": traffic / n if traffic else None,
                            "measured_frac": (traffic / n * lups_gpu / 1e9 / peak) if traffic else None,
                            "b_min_per_lu": b_min, "useful_frac": b_min * lups_gpu / 1e9 / peak},
               "clocks": clk.summary(), "e2e": e2e,
               "gpu_launches": (1 if single else 2) * args.steps,
               "cpu_baseline": cb,
               "observables": {"mass_c2": obs["mass_c2"], "max_u": obs["max_u"]}}
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_serve(args, rank, world):
    """Served form: a Poisson stream of wetting studies through the
    continuous-batching scheduler, against serving the same stream one request
    at a time.  Requests: 50 % D2Q9 (side 64..512), 50 % D3Q19 (side 64..160),
    random pillars / sinusoidal walls / sphere packings, contact angle
    U[30, 150] degrees, step budgets U[2000, 20000] scaled by --serve-scale.
    By default 48 requests arrive at once with full step budgets, which
    saturates the GPU (throughput and the latency of a burst); a rate below
    capacity (e.g. --serve-rate 1.0) measures latency under load.  Policy: at
    most --serve-max-large large lattices active together, taken shortest work
    first (--serve-order sjf)."""
    import torch
    import synthetic as S
    from paper_2504_19941_gb300.serving import GpuExecutor, Scheduler, serial_run, summarize

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    reqs = S.serving_stream(n_req=args.serve_requests, rate=args.serve_rate, seed=0,
                            scale_steps=args.serve_scale)
    mine = shard(reqs, rank, world)   # replicas: requests split across ranks
    # a request arrives with its fields (geometry and liquid), as a client sends
    # them: build them before the clock starts
    for r in mine:
        r.payload = r.case()
    warm = S.serving_stream(n_req=4, rate=1000.0, seed=99, min_side=32, max_side_2d=96, max_side_3d=48,
                            steps=(20, 40))
    policy = dict(max_large=args.serve_max_large if args.serve_max_large > 0 else None,
                  order=args.serve_order)
    Scheduler(GpuExecutor("f32"), 200 << 30, quantum=args.serve_quantum, **policy).run(warm)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        recs = Scheduler(GpuExecutor("f32"), 200 << 30, quantum=args.serve_quantum,
                         **policy).run(mine)
        wall = time.perf_counter() - t0
    s = summarize(recs, wall)
    thetas = [r.result.get("theta_deg") for r in recs if r.status == "done"]
    s["theta_deg_measured"] = sum(1 for t in thetas if t is not None and math.isfinite(t))
    base = None
    if not args.no_serial_baseline:
        t0 = time.perf_counter()
        srecs = serial_run(GpuExecutor("f32"), mine)
        base = summarize(srecs, time.perf_counter() - t0)
    if rank == 0:
        out = {"metric": "served wetting sweeps: solves/s (p50/p99 latency)",
               "value": s["solves_per_s"] * world, "unit": "solves/s", "n_gpus": world,
               "steps": len(mine), "warmup": len(warm), "ms_per_step": None,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic",
               "config": {"workload": f"{args.serve_requests} requests, Poisson {args.serve_rate}/s, "
                                      f"steps x{args.serve_scale}", "quantum": args.serve_quantum,
                          "max_large": policy["max_large"], "order": policy["order"],
                          "executor": "asynchronous: per-lattice CUDA events, large lattices on "
                                      "their own streams, small ones in one batched launch",
                          "result": "observables and the apparent contact angle of the drop",
                          "parallelism": f"replicas x{world}"},
               "serving": s, "one_at_a_time": base, "clocks": clk.summary()}
        print(json.dumps(out), flush=True)
    return 0


def _time_steps(lat, steps, warmup):
    """Per-step and dominant-kernel times (CUDA events) of `steps` steps: the
    one-pass step's launch, or the fused pass of the two-pass step."""
    import torch
    from paper_2504_19941_gb300 import _lib
    for _ in range(warmup):
        lat.step(1)
    torch.cuda.synchronize()
    single = lat.single_pass
    stream = lat.stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(steps):
        if single:
            ev[k][0].record(stream)
            _lib.dsm_step(lat.h, 1)
        else:
            _lib.dsm_step_moments(lat.h)
            ev[k][0].record(stream)
            _lib.dsm_step_collide(lat.h)
        ev[k][1].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / steps, sum(a.elapsed_time(b) for a, b in ev) / steps / 1e3


def run_precision(args, rank, world):
    """Precision forms on the 384x384x256 capillary-rise lattice (D3Q19): FP32
    storage and BF16 / FP16 storage of the populations, FP32 arithmetic."""
    import torch
    import synthetic as S
    import paper_2504_19941_gb300 as P
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    case = S.plates_rise_3d()
    peak, peak_kind = _peaks()
    out = {}
    for prec in ("f32", "bf16", "f16"):
        p = P.make_params("D3Q19", case.shape, prec, theta_deg=case.theta_deg, g12=case.g12,
                          g23=case.g23, alpha_s=case.alpha_s, body=case.body)
        lat = P.Lattice(p, device=dev)
        lat.set_g_storage(args.g_storage)
        lat.set_solid_distance(torch.as_tensor(case.solid_sd, dtype=torch.float32, device=dev))
        lat.set_fluid(torch.as_tensor(case.c2, dtype=torch.float32, device=dev))
        lat.set_step_form(args.step_form, args.zrun)
        t_step, t_k2 = _time_steps(lat, args.steps, args.warmup)
        bmin = (lu_bytes_single(prec) if lat.single_pass
                else lu_bytes("D3Q19", prec, lat.g_implicit)[0])
        ob = lat.observables()
        out[prec] = {"MLUPS": lat.n / t_step / 1e6, "ms_per_step": t_step * 1e3,
                     "single_pass": lat.single_pass,
                     "k2_ms": t_k2 * 1e3, "bytes_per_lu": bmin,
                     "roofline_frac": bmin * lat.n / t_k2 / 1e9 / peak,
                     "nonfinite": ob["nonfinite"]}
        del lat
        torch.cuda.empty_cache()
    if rank == 0:
        print(json.dumps({"metric": "D3Q19 precision forms MLUPS (384x384x256 capillary rise)",
                          "value": out["bf16"]["MLUPS"], "unit": "MLUPS", "n_gpus": 1,
                          "steps": args.steps, "warmup": args.warmup, "dtype": "bf16-storage/f32",
                          "higher_is_better": True, "data": "synthetic", "peak_gbs": peak,
                          "peak_source": peak_kind, "g_storage": args.g_storage,
                          "forms": out}), flush=True)
    return 0


def run_ramp(args, rank, world):
    """The cfg2 physics run: the 256x256x192 pillar slab (gaps vented through
    the base plate) under a body force on the liquid ramped linearly along -z
    from 0 to twice the square-pillar critical-pressure estimate over
    --ramp-steps steps, one run per seed (contact angle drawn in [90, 150]).
    Reports per seed the critical pressure (the ramp's f H when the mean
    C2 = 1/2 height next to the pillars falls 2 nodes below the pillar tops,
    or None when the slab stays pinned through the ramp), the estimate, and
    the MLUPS of the ramp's steps with the one-pass kernel's HBM fraction."""
    import numpy as np
    import torch
    import synthetic as S
    import paper_2504_19941_gb300 as P
    from paper_2504_19941_gb300.ramp import pillar_ring, pressure_ramp
    from paper_2504_19941_gb300 import _lib
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    peak, peak_kind = _peaks()
    seeds = shard(list(range(args.ramp_seeds)), rank, world)
    runs = []
    lu_total, t_total = 0.0, 0.0
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for seed in seeds:
            case = S.pillar_slab_3d(seed=seed, vent=10)
            nx, ny, nz = case.shape
            params = P.make_params("D3Q19", case.shape, "f32", theta_deg=case.theta_deg,
                                   g12=case.g12, g23=case.g23, alpha_s=case.alpha_s)
            lat = P.Lattice(params, device=dev)
            lat.set_solid_distance(torch.as_tensor(case.solid_sd, dtype=torch.float32, device=dev))
            lat.set_fluid(torch.as_tensor(case.c2, dtype=torch.float32, device=dev))
            c1 = lat.field("C1").double().cpu().numpy().reshape(nz, ny, nx)
            ring = pillar_ring(c1[20])
            thick = 98 - 38
            f_max = case.extra["f_max"]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(lat.stream)
            r = pressure_ramp(lat, f_max, args.ramp_steps, c1, ring, 38, thick,
                              check_every=100, stop_at_depinning=False)
            e1.record(lat.stream)
            torch.cuda.synchronize()
            secs = e0.elapsed_time(e1) / 1e3
            est = f_max * thick / 2.0
            runs.append({"seed": seed, "theta_deg": case.theta_deg, "dp_estimate": est,
                         "dp_crit": r["dp_crit"],
                         "dp_crit_over_estimate": None if r["dp_crit"] is None
                         else r["dp_crit"] / est,
                         "dp_max": f_max * thick, "steps": r["steps"],
                         "contact_line_start": r["history"][0][2],
                         "contact_line_end": r["history"][-1][2],
                         "single_pass": lat.single_pass,
                         "seconds": secs, "MLUPS": lat.n * r["steps"] / secs / 1e6})
            lu_total += lat.n * r["steps"]
            t_total += secs
            del lat
            torch.cuda.empty_cache()
    t_max, lups = aggregate(t_total, lu_total, dist)
    value = lups / 1e6
    achieved = lu_bytes_single("f32") * value * 1e6 / 1e9
    if rank == 0:
        print(json.dumps({
            "metric": "cfg2 pressure ramp: critical pressure per contact angle; ramp MLUPS",
            "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.ramp_steps,
            "warmup": 0, "ms_per_step": t_total / max(1, sum(r["steps"] for r in runs)) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "D3Q19 FP32 pillar slab 256x256x192, base plate vented under "
                                   "each gap, body force on the liquid ramped 0 -> 2x the "
                                   "square-pillar estimate along -z",
                       "seeds": seeds, "check_every": 100,
                       "timing": "CUDA events around each ramp: its steps, the force updates "
                                 "and the field reads of the detector"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "zstep_kernel<f32,f32> (one pass per step)",
                         "bytes_per_lu": lu_bytes_single("f32"), "peak_source": peak_kind},
            "clocks": clk.summary(), "runs": runs}), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def meniscus_between_plates(c2_zyx, c1_zyx, yc, half_gap, x_lo, margin=3.0):
    """Meniscus of a capillary rise between plates normal to y (rise along +x):
    returns (height, theta_deg).  The z-averaged liquid field is taken in the
    (x, y) plane; the height is where C2 crosses 1/2 along the gap's centre line
    (first crossing above x_lo, linear interpolation); theta comes from a Kasa
    circle fit of the C2 = 1/2 points in the gap at least `margin` nodes from
    the plates (cos theta = w / R, w the half distance between the plates'
    C1 = 1/2 planes)."""
    import numpy as np
    from paper_2504_19941_gb300.analysis import level_points, sphere_fit
    c2 = c2_zyx.mean(axis=0)                  # (ny, nx)
    col = c2[yc, x_lo:]
    below = np.nonzero(col < 0.5)[0]
    if below.size == 0 or below[0] == 0:
        return math.nan, math.nan
    k = below[0]
    h = x_lo + (k - 1) + (col[k - 1] - 0.5) / (col[k - 1] - col[k])
    # the plates' C1 = 1/2 planes on either side of the centre line
    c1 = c1_zyx.mean(axis=0)[:, int(round(h))]
    lo = yc
    while lo > 0 and c1[lo - 1] < 0.5:
        lo -= 1
    hi = yc
    while hi < c1.size - 1 and c1[hi + 1] < 0.5:
        hi += 1
    w = 0.5 * ((hi + (c1[hi] - 0.5) / (c1[hi] - c1[hi + 1]) if hi + 1 < c1.size else hi)
               - (lo - (c1[lo] - 0.5) / (c1[lo] - c1[lo - 1]) if lo > 0 else lo))
    pts, _ = level_points(c2[max(0, yc - half_gap):yc + half_gap + 1, :], 0.5)
    pts[:, 1] += max(0, yc - half_gap)
    keep = (np.abs(pts[:, 1] - yc) < w - margin) & (np.abs(pts[:, 0] - h) < 2 * half_gap)
    pts = pts[keep]
    if pts.shape[0] < 8:
        return h, math.nan
    _, R = sphere_fit(pts)
    return h, math.degrees(math.acos(max(-1.0, min(1.0, w / R)))) if R > 0 else math.nan


def run_cfg3(args, rank, world):
    """Precision forms on the capillary rise between plates (384x384x256, gap
    40, 45 degrees, gravity for a Jurin rise of 120 nodes): FP64, FP32 and BF16
    / FP16 storage run the same steps (50k, or fewer when FP64's measured speed
    would take longer than --cfg3-budget seconds); every --cfg3-check steps the
    meniscus height and angle of each; at the end the errors of C2, rho, pt and
    u against the FP64 run, and each form's MLUPS.  --cfg3-reference f32
    compares the 16-bit forms with FP32 instead and does not run FP64 (whose
    steps cost 25 times FP32's on this GPU)."""
    import numpy as np
    import torch
    import synthetic as S
    import paper_2504_19941_gb300 as P
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    shape = tuple(int(v) for v in args.cfg3_shape.split(","))
    if shape == (384, 384, 256):
        case = S.plates_rise_3d()
    else:  # proportionally scaled geometry
        sc = shape[0] / 384.0
        case = S.plates_rise_3d(*shape, gap=int(round(40 * sc)), thick=max(3, int(round(8 * sc))),
                                x0=int(round(40 * sc)), x1=int(round(340 * sc)),
                                reservoir=int(round(60 * sc)), lid=max(3, int(round(8 * sc))),
                                target_rise=120.0 * sc)
    nx, ny, nz = case.shape
    yc, half_gap = ny // 2, case.extra["gap"] // 2
    x_lo = int(round(60 * nx / 384.0))

    def make(prec):
        p = P.make_params("D3Q19", case.shape, prec, theta_deg=case.theta_deg, g12=case.g12,
                          g23=case.g23, alpha_s=case.alpha_s, body=case.body)
        lat = P.Lattice(p, device=dev)
        lat.set_solid_distance(torch.as_tensor(case.solid_sd, dtype=lat.real, device=dev))
        lat.set_fluid(torch.as_tensor(case.c2, dtype=lat.real, device=dev))
        return lat

    ref_prec = args.cfg3_reference
    f64_step = None
    steps = args.cfg3_steps
    if ref_prec == "f64":
        # FP64's speed decides how many steps every form runs
        probe = make("f64")
        probe.step(5)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        probe.step(50)
        torch.cuda.synchronize()
        f64_step = (time.perf_counter() - t0) / 50
        del probe
        torch.cuda.empty_cache()
        steps = min(args.cfg3_steps,
                    int(args.cfg3_budget / f64_step) // args.cfg3_check * args.cfg3_check)
        steps = max(steps, args.cfg3_check)
    c1 = None
    results, finals = {}, {}
    forms = ("f64", "f32", "bf16", "f16") if ref_prec == "f64" else ("f32", "bf16", "f16")
    for prec in forms:
        lat = make(prec)
        if c1 is None:
            c1 = lat.field("C1").double().cpu().numpy().reshape(nz, ny, nx)
        m0 = lat.observables()["mass_c2"]
        hist = []
        secs = 0.0
        for done in range(args.cfg3_check, steps + 1, args.cfg3_check):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lat.step(args.cfg3_check)
            torch.cuda.synchronize()
            secs += time.perf_counter() - t0
            c2 = lat.field("C2").double().cpu().numpy().reshape(nz, ny, nx)
            h, th = meniscus_between_plates(c2, c1, yc, half_gap, x_lo)
            hist.append((done, h, th))
        ob = lat.observables(check=False)
        finals[prec] = {k: lat.field(k).double().cpu().numpy()
                        for k in ("C2", "rho", "pt", "ux", "uy", "uz")}
        results[prec] = {"MLUPS": lat.n * steps / secs / 1e6, "single_pass": lat.single_pass,
                         "meniscus": hist, "mass_drift": (ob["mass_c2"] - m0) / m0,
                         "nonfinite": ob["nonfinite"]}
        del lat
        torch.cuda.empty_cache()
    ref = finals[ref_prec]
    umax = max(np.abs(ref[k]).max() for k in ("ux", "uy", "uz"))
    for prec in [f for f in forms if f != ref_prec]:
        got = finals[prec]
        err = {k: float(np.abs(got[k] - ref[k]).max() / np.abs(ref[k]).max())
               for k in ("C2", "rho", "pt")}
        err["u"] = float(max(np.abs(got[k] - ref[k]).max() for k in ("ux", "uy", "uz")) / umax)
        h_ref, th_ref = results[ref_prec]["meniscus"][-1][1:]
        h, th = results[prec]["meniscus"][-1][1:]
        err["meniscus_height"] = h - h_ref
        err["theta_deg"] = th - th_ref
        results[prec]["error_vs_" + ref_prec] = err
    if rank == 0:
        print(json.dumps({
            "metric": "cfg3 precision forms: errors against FP64 and MLUPS (capillary rise between plates)",
            "value": results["bf16"]["MLUPS"], "unit": "MLUPS", "n_gpus": 1, "steps": steps,
            "warmup": 0, "dtype": "bf16-storage/f32", "higher_is_better": True, "data": "synthetic",
            "config": {"workload": f"D3Q19 capillary rise between plates {nx}x{ny}x{nz}, gap "
                                   f"{case.extra['gap']}, 45 deg, gamma 1e-2, Jurin rise 120 "
                                   f"(scaled), {steps} steps (asked {args.cfg3_steps})",
                       "reference": ref_prec,
                       "f64_ms_per_step": None if f64_step is None else f64_step * 1e3,
                       "check_every": args.cfg3_check,
                       "jurin_height": x_lo + 120.0 * nx / 384.0},
            "forms": results}), flush=True)
    return 0


def run_plain_fp64(args, rank, world):
    """The plain FP64 D2Q9 128x64 wall-drop case: per-step launches against one
    persistent batched launch of all its steps, in both storage forms of g."""
    import torch
    import synthetic as S
    import paper_2504_19941_gb300 as P
    from paper_2504_19941_gb300 import _lib
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    case = S.wall_drop_2d()
    res = {}
    for form in ("auto", "populations"):
        for mode in ("per_step_launches", "persistent_launch"):
            p = P.make_params("D2Q9", case.shape, "f64", theta_deg=case.theta_deg, g12=case.g12,
                              g23=case.g23, alpha_s=case.alpha_s)
            lat = P.Lattice(p, device=dev)
            lat.set_g_storage(form)
            lat.set_solid_distance(torch.as_tensor(case.solid_sd, dtype=torch.float64, device=dev))
            lat.set_fluid(torch.as_tensor(case.c2, dtype=torch.float64, device=dev))
            nb = _lib.dsm_batch_scratch_bytes([lat.h])
            scratch = torch.empty(nb, dtype=torch.uint8, device=dev)
            lat.step(10)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if mode == "per_step_launches":
                lat.step(case.steps)
            else:
                _lib.dsm_batch_step([lat.h], [case.steps], scratch, nb)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            key = ("g_eq" if form == "auto" else "populations") + "/" + mode
            res[key] = {"us_per_step": dt / case.steps * 1e6, "MLUPS": lat.n * case.steps / dt / 1e6}
    best = min(res, key=lambda k: res[k]["us_per_step"])
    # the oracle on the same case, on the host cores (200 steps)
    import oracle as O
    k, _ = O.kappa_from_angle(case.theta_deg, case.g23, case.g12)
    po = O.make_params(O.D2Q9, case.shape, k, alpha_s=case.alpha_s)
    c1 = O.solid_profile(case.solid_sd, case.alpha_s)
    f, g = O.lb_init(po, 2, c1, case.c2)
    t0 = time.perf_counter()
    O.lb_run(po, 2, c1, f, g, 200)
    t_or = (time.perf_counter() - t0) / 200
    oracle = {"us_per_step": t_or * 1e6, "MLUPS": case.n / t_or / 1e6,
              "cores": OracleSlice.cores(), "kind": "oracle", "sample": "200 steps of the same case"}
    if rank == 0:
        print(json.dumps({"metric": "D2Q9 FP64 128x64 wall drop, 2000 steps", "unit": "us/step",
                          "value": res[best]["us_per_step"], "best": best,
                          "higher_is_better": False, "n_gpus": 1, "dtype": "f64",
                          "data": "synthetic", "modes": res, "cpu_baseline": oracle}),
              flush=True)
    return 0


def run_capillary(args, rank, world):
    """The capillary-filling lattice (Sec. IV): D2Q9 FP32 1750x450 with mirror
    faces top and bottom, an inclined channel through a solid slab, the solid
    relaxed first (5000 stage-1 steps).  Mirror faces keep g as populations.
    Its state (f and g, 2 x 57 MB) is about L2's size, so L2 is flushed before
    every timed step and only the step's two launches are timed."""
    import torch
    import synthetic as S
    import paper_2504_19941_gb300 as P
    from paper_2504_19941_gb300 import _lib
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    case = S.capillary_channel_2d()
    p = P.make_params("D2Q9", case.shape, "f32", theta_deg=case.theta_deg, g12=case.g12,
                      g23=case.g23, tau2=case.tau2, tau3=case.tau3, tau_g=case.tau_g,
                      faces=case.faces)
    lat = P.Lattice(p, device=dev)
    mask = torch.as_tensor(case.extra["mask"], device=dev)
    lat.set_solid_c1(mask.to(torch.float32))
    lat.relax_solid(mask, case.extra["solid_steps"], case.extra["beta"], case.extra["omega"])
    c1 = lat.field("C1").clamp(0.0, 1.0)
    c2 = torch.as_tensor(case.c2, dtype=torch.float32, device=dev).clamp(0.0, 1.0) * (1.0 - c1)
    lat.set_fluid(c2)
    m0 = lat.observables()["mass_c2"]
    for _ in range(args.warmup):
        lat.step(1)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    torch.cuda.synchronize()
    with ClockSampler(dev.index or 0) as clk:
        time.sleep(0.3)
        for k in range(args.steps):
            flush.fill_(k & 255)
            ev[k][0].record(stream)
            _lib.dsm_step_moments(lat.h)
            ev[k][1].record(stream)
            _lib.dsm_step_collide(lat.h)
            ev[k][2].record(stream)
        torch.cuda.synchronize()
    t_step = sum(a.elapsed_time(c) for a, _, c in ev) / args.steps / 1e3
    t_k2 = sum(b.elapsed_time(c) for _, b, c in ev) / args.steps / 1e3
    ob = lat.observables()
    k2_b, k1_b = lu_bytes("D2Q9", "f32", lat.g_implicit)
    peak, peak_kind = _peaks()
    achieved = k2_b * lat.n / t_k2 / 1e9
    if rank == 0:
        print(json.dumps({
            "metric": "D2Q9 capillary filling 1750x450 (mirror top/bottom) MLUPS", "unit": "MLUPS",
            "value": lat.n / t_step / 1e6, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "D2Q9 FP32 capillary channel 1750x450, 20 deg incline, "
                                   "mirror top/bottom", "nodes": lat.n,
                       "g_storage": "g_eq" if lat.g_implicit else "populations",
                       "l2": "state about L2's size: L2 flushed (256 MB write) before each "
                             "timed step, outside the timed events"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "node_kernel<D2Q9,f32,stage2,step,populations,faces>",
                         "bytes_per_lu": k2_b, "peak_source": peak_kind, "k2_ms": t_k2 * 1e3,
                         "step_bytes_per_lu": k1_b + k2_b},
            "clocks": clk.summary(), "gpu_launches": 2 * args.steps,
            "observables": {"mass_drift": ob["mass_c2"] / m0 - 1.0, "max_u": ob["max_u"],
                            "nonfinite": ob["nonfinite"]}}), flush=True)
    return 0


def run_multi(args, rank, world):
    """N fluid components (dsm_ml_*): three (--nfluid 3) or four fluids on the
    D3Q19 FP32 pillar slab 256x256x192, the liquid split into two fluids (x
    below and above the middle; four fluids: the gas above z = 150 is fluid 4's).
    tau_g = 1 and periodic faces, so g is held as g_eq, and the planes tile into
    32 x 8 blocks, so each step is one pass (--step-form two_pass: the moments
    passes and the fused pass).  Algorithmic bytes per lattice update with NF
    free fluids: read and write f (152), read C1 (4), read and write A_f and C_f
    of every free fluid (16 NF) and u (24): 212 B for three fluids, 228 B for
    four; the two-pass form moves the same bytes (176 + 36 for three fluids).
    Population form: f and every g_f in and out plus C1 in the fused pass, the
    g_f in and C_f out in the moments passes, 2 * 76 (NF + 1) + 4 + 80 NF bytes
    (620 for three fluids)."""
    import torch
    import paper_2504_19941_gb300 as P
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    shape = tuple(int(v) for v in args.shape.split(","))
    case = make_case(shape)
    nx = shape[0]
    c2 = torch.as_tensor(case.c2, dtype=torch.float32, device=dev)
    xs = torch.arange(c2.numel(), device=dev) % nx
    nfl = args.nfluid
    C = [c2 * (xs < nx // 2), c2 * (xs >= nx // 2)]
    if nfl == 4:  # the upper gas becomes fluid 4
        zs = torch.arange(c2.numel(), device=dev) // (shape[0] * shape[1])
        c1 = torch.as_tensor(case.solid_sd, dtype=torch.float32, device=dev)
        free = 1.0 - 0.5 * (1.0 + torch.tanh(c1 / (2.0 * case.alpha_s)))
        C.append(((free - c2) * (zs >= int(0.78 * shape[2]))).clamp(min=0.0))
    C = torch.stack(C).contiguous()
    p = P.make_params("D3Q19", shape, "f32", theta_deg=case.theta_deg, g12=case.g12,
                      g23=case.g23, alpha_s=case.alpha_s)
    k = P._lib.dsm_kappa(p)
    kappa = [k[0]] + [k[1]] * (nfl - 1) + [k[2]]  # the liquids alike, the gases alike
    ml = P.MultiLattice(p, nfl, kappa, (1.0,) * nfl, (1.0,) * nfl, device=dev)
    ml.set_step_form(args.step_form, args.zrun)
    ml.set_solid_distance(torch.as_tensor(case.solid_sd, dtype=torch.float32, device=dev))
    ml.set_fluids(C)
    for _ in range(args.warmup):
        ml.step(1)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with ClockSampler(dev.index or 0) as clk:
        time.sleep(0.3)
        e0.record(stream)
        ml.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / args.steps
    ux = ml.field("ux")
    assert torch.isfinite(ux).all(), "non-finite velocity after the timed steps"
    peak, peak_kind = _peaks()
    nf = nfl - 1
    single = ml.single_pass
    b = 180 + 16 * nf if ml.g_implicit else 2 * 19 * 4 * (nf + 1) + 4 + 80 * nf
    launches = 1 if single else (nf + 1 if ml.g_implicit else 2)
    names = {3: "three", 4: "four"}
    if rank == 0:
        print(json.dumps({
            "metric": "D3Q19 %s-fluid LB MLUPS (%dx%dx%d pillar slab)" % ((names[nfl],) + shape),
            "unit": "MLUPS",
            "value": ml.n / t / 1e6, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "D3Q19 FP32 pillar slab %dx%dx%d, %s fluids" % (shape + (names[nfl],)),
                       "nodes": ml.n,
                       "g_storage": "g_eq (A_f, u per node)" if ml.g_implicit else "populations",
                       "step": "one pass (zrun %d)" % P._lib.dsm_ml_step_info(ml.h)[1]
                       if single else "two passes",
                       "l2": "f alone 1.0 GB per buffer, larger than L2; no flush"},
            "roofline": {"bound": "hbm", "step_bytes_per_lu": b,
                         "achieved": b * ml.n / t / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": b * ml.n / t / 1e9 / peak, "peak_source": peak_kind},
            "clocks": clk.summary(), "gpu_launches": launches * args.steps}), flush=True)
    return 0


def _em_iterations(args, case, p, dev):
    """A fixed number of L-BFGS iterations (tol 0) on the 128^3 sphere case, for
    profiling one iteration: prints the wall time per iteration."""
    import torch
    import paper_2504_19941_gb300 as P
    from paper_2504_19941_gb300.energy import FreeEnergy, lbfgs
    lat = P.Lattice(P.make_params("D3Q19", case.shape, "f32", theta_deg=case.theta_deg,
                                  g23=case.g23, g12=case.g12, alpha_s=1.0), device=dev)
    lat.set_solid_distance(torch.as_tensor(case.solid_sd, dtype=torch.float32, device=dev))
    c1 = lat.field("C1")
    del lat
    c2 = torch.as_tensor(case.c2, dtype=torch.float32, device=dev)
    fe = FreeEnergy(p, device=dev)
    V0 = float(c2.double().sum())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, E, info = lbfgs(fe, c2, c1, active=2, kcs=1e-2, V0=V0, tol=0.0, max_iter=args.lbfgs_iters)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    print(json.dumps({"metric": "L-BFGS wall time per iteration (128^3 sphere at the interface)",
                      "value": wall / max(info["iterations"], 1) * 1e6, "unit": "us",
                      "higher_is_better": False, "iterations": info["iterations"],
                      "evaluations": info["evaluations"]}), flush=True)
    return 0


def run_critical(args, rank, world):
    """Critical pressure of the Cassie-Baxter to Wenzel transition on 2D pillars
    (Sec. III) by bisection over GPU energy minimisations, for a sweep of five
    contact angles on a 160x200 box with gap s = 81, served as concurrent
    searches (one host thread and CUDA stream per angle): the value is sweep
    points per second.  The same sweep one search at a time is timed beside it,
    and the two must give identical results; each point reports dP_c against
    -2 gamma cos(theta) / s."""
    import torch
    import synthetic as S
    from paper_2504_19941_gb300 import critical as C
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    thetas = (60.0, 80.0, 100.0, 112.0, 135.0)
    warm = S.pillar_gap_2d(period=40, height=64, width=16, pillar=24, base=4)
    C.critical_sweep([warm, warm])  # module, context and thread-pool warm-up
    cases = [S.pillar_gap_2d(period=160, height=200, width=79, pillar=100, base=6, theta=t)
             for t in thetas]
    t0 = time.perf_counter()
    one = [C.critical_pressure(c, tol=1e-4) for c in cases]
    wall_one = time.perf_counter() - t0
    res, wall = C.critical_sweep(cases, tol=1e-4)
    same = all(a["dP_c"] == b["dP_c"] and a["iterations"] == b["iterations"]
               for a, b in zip(one, res))
    pts = [{"theta": t, "dP_c": r["dP_c"], "theory": r["theory"], "ratio": r["ratio"],
            "probes": r["probes"], "lbfgs_iterations": r["iterations"],
            "seconds": r["seconds"], "ms_per_lbfgs_iteration": r["seconds"] / max(
                r["iterations"], 1) * 1e3} for t, r in zip(thetas, res)]
    if rank == 0:
        print(json.dumps({"metric": "critical-pressure sweep points/s (2D pillars, bisection to 1e-4)",
                          "value": len(pts) / wall, "unit": "points/s", "n_gpus": 1,
                          "higher_is_better": True, "dtype": "f32 fields / f64 energy",
                          "data": "synthetic",
                          "config": {"workload": "160x200 box, pillar width 79, gap 81, height 100",
                                     "searches": "concurrent, one thread and stream per angle"},
                          "one_at_a_time": {"value": len(pts) / wall_one, "unit": "points/s",
                                            "wall_s": wall_one},
                          "identical_to_one_at_a_time": same, "wall_s": wall,
                          "points": pts}), flush=True)
    return 0 if same else 1


def lbfgs_bytes_per_node(m: int = 10) -> int:
    """Algorithmic bytes per node of one L-BFGS iteration of the native loop
    with m stored pairs and one line-search trial: the trial point, its energy
    and gradient and g.d (12 + 12 + 8); the direction from the history and g
    (2m + 1 vectors read, one written); the new pair (s: 8, y: 12); the dots
    of every stored vector against y and g (2m + 2 vectors read); s.s and g.g
    (4 + 4).  m = 10: 236 B."""
    return 32 + (2 * m + 2) * 4 + 8 + 12 + (2 * m + 2) * 4 + 8


def run_em(args, rank, world):
    """Energy-minimisation twin on a 128^3 grid (sphere of radius 20 at a flat
    liquid/gas interface): energy + gradient evaluations per second, and L-BFGS
    iterations per second with the time to an rms gradient of 1e-6 for both
    128^3 cases (the sphere at the interface and the drop on the sinusoidal
    wall, each volume-constrained)."""
    import torch
    import synthetic as S
    import paper_2504_19941_gb300 as P
    from paper_2504_19941_gb300.energy import FreeEnergy, lbfgs
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    case = S.em_sphere_interface()
    n = case.n
    p = P.make_params("D3Q19", case.shape, "f32", theta_deg=case.theta_deg, g23=case.g23,
                      g12=case.g12)
    if args.lbfgs_iters > 0:
        return _em_iterations(args, case, p, dev)
    # the solid's tanh profile of Sec. II.A, written by the library from the distance
    lat_p = P.make_params("D3Q19", case.shape, "f32", theta_deg=case.theta_deg, g23=case.g23,
                          g12=case.g12, alpha_s=1.0)
    lat = P.Lattice(lat_p, device=dev)
    lat.set_solid_distance(torch.as_tensor(case.solid_sd, dtype=torch.float32, device=dev))
    c1 = lat.field("C1")
    del lat
    c2 = torch.as_tensor(case.c2, dtype=torch.float32, device=dev)
    fe = FreeEnergy(p, device=dev)
    E = torch.empty(1, dtype=torch.float64, device=dev)
    g = torch.empty(n, dtype=torch.float32, device=dev)
    for _ in range(5):
        fe(c1, c2, energy=E, grad=g, kcs=1e-2, V0=float(c2.double().sum()))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 200
    V0 = float(c2.double().sum())
    e0.record()
    for _ in range(reps):
        fe(c1, c2, energy=E, grad=g, kcs=1e-2, V0=V0)
    e1.record()
    torch.cuda.synchronize()
    t_eval = e0.elapsed_time(e1) / 1e3 / reps
    peak, peak_kind = _peaks()
    minimisations = {}
    for name in ("sphere_at_interface", "sinusoid_drop"):
        if name == "sphere_at_interface":
            xc, c1c, pc = c2, c1, p
        else:
            cs = S.em_sinusoid_drop()
            pc = P.make_params("D3Q19", cs.shape, "f32", theta_deg=cs.theta_deg, g23=cs.g23,
                               g12=cs.g12)
            lat_s = P.Lattice(P.make_params("D3Q19", cs.shape, "f32", theta_deg=cs.theta_deg,
                                            g23=cs.g23, g12=cs.g12, alpha_s=cs.alpha_s), device=dev)
            lat_s.set_solid_distance(torch.as_tensor(cs.solid_sd, dtype=torch.float32, device=dev))
            c1c = lat_s.field("C1")
            del lat_s
            xc = torch.as_tensor(cs.c2, dtype=torch.float32, device=dev)
        fec = FreeEnergy(pc, device=dev)
        V0c = float(xc.double().sum())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xm, Em, inf = lbfgs(fec, xc, c1c, active=2, kcs=1e-2, V0=V0c, tol=1e-6,
                            max_iter=args.em_iters)
        torch.cuda.synchronize()
        t_m = time.perf_counter() - t0
        it_s = inf["iterations"] / t_m
        bpi = lbfgs_bytes_per_node() * n
        minimisations[name] = {"iterations": inf["iterations"], "evaluations": inf["evaluations"],
                               "rms_grad": inf["rms_grad"], "converged": bool(inf["converged"]),
                               "energy": Em, "seconds_to_tol": t_m, "iters_per_s": it_s,
                               "bytes_per_iteration": bpi,
                               "achieved_gbs": bpi * it_s / 1e9,
                               "frac": bpi * it_s / 1e9 / peak,
                               "volume_drift": float(xm.double().sum()) / V0c - 1.0}
    info = {k: minimisations["sphere_at_interface"][k] for k in ("iterations", "evaluations",
                                                                  "rms_grad")}
    Emin = minimisations["sphere_at_interface"]["energy"]
    t_lb = minimisations["sphere_at_interface"]["seconds_to_tol"]
    # N fluid components: the same lattice with the liquid split into N - 1
    # free fluids; algorithmic bytes per node 4 (2 (N - 1) + 1): read C1 and the
    # free planes, write their gradients
    from paper_2504_19941_gb300.energy import FreeEnergyMulti
    multi = {}
    for nfluid in (2, 3, 4):
        nf = nfluid - 1
        C = (c2 / nf).repeat(nf, 1).contiguous()
        kap = [0.0] + [float(k) for k in P._lib.dsm_kappa(p)[1:]] + [0.9] * (nfluid - 2)
        kap[0] = float(P._lib.dsm_kappa(p)[0])
        fm = FreeEnergyMulti(p, nfluid, kap, device=dev)
        Em = torch.empty(1, dtype=torch.float64, device=dev)
        gm = torch.empty((nf, n), dtype=torch.float32, device=dev)
        for _ in range(5):
            fm(c1, C, energy=Em, grad=gm)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fm(c1, C, energy=Em, grad=gm)
        e1.record()
        torch.cuda.synchronize()
        t_m = e0.elapsed_time(e1) / 1e3 / reps
        b = 4 * (2 * nf + 1)
        multi[f"N={nfluid}"] = {"eval_ms": t_m * 1e3, "bytes_per_node": b,
                                "achieved_gbs": b * n / t_m / 1e9,
                                "frac": b * n / t_m / 1e9 / peak}
    if rank == 0:
        print(json.dumps({"metric": "EM energy+gradient evaluations/s (128^3, D3Q19 stencil)",
                          "value": 1.0 / t_eval, "unit": "evals/s", "n_gpus": 1,
                          "higher_is_better": True, "dtype": "f32 fields / f64 energy",
                          "data": "synthetic",
                          "roofline": {"bound": "hbm", "bytes_per_node": 12,
                                       "achieved": 12 * n / t_eval / 1e9, "peak": peak,
                                       "unit": "GB/s", "frac": 12 * n / t_eval / 1e9 / peak,
                                       "peak_source": peak_kind},
                          "eval_ms": t_eval * 1e3,
                          "lbfgs": {"iterations": info["iterations"],
                                    "evaluations": info["evaluations"],
                                    "rms_grad": info["rms_grad"], "energy": Emin,
                                    "seconds": t_lb, "iters_per_s": info["iterations"] / t_lb,
                                    "tol": 1e-6, "m": 10,
                                    "bytes_per_node_per_iteration": lbfgs_bytes_per_node(),
                                    "cases": minimisations},
                          "multi_fluid": multi}), flush=True)
    return 0


def main():
    if len(sys.argv) == 3 and sys.argv[1] == "--oracle-one-core":
        sl = OracleSlice()
        sl.run(0.0)
        steps, dt = sl.run(float(sys.argv[2]))
        print(json.dumps({"value": sl.n * steps / dt / 1e6, "unit": "MLUPS", "cores": 1,
                          "kind": "oracle",
                          "sample": f"64x64x48 slice, {steps} steps, {dt:.1f} s, one thread"}))
        return 0
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="dsm", choices=["dsm", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--lattice", default="D3Q19", choices=["D3Q19", "D2Q9"],
                    help="D2Q9: a 2D pillar row (default 4096x4096 unless --shape has two sizes)")
    ap.add_argument("--rho3", type=float, default=1.0, help="gas density (liquid 1)")
    ap.add_argument("--tau3", type=float, default=1.0, help="gas relaxation time (liquid 1)")
    ap.add_argument("--faces", default="",
                    help="six comma-separated faces x-,x+,y-,y+,z-,z+: periodic, mirror or wall")
    ap.add_argument("--step-form", default="auto", choices=["auto", "two_pass"],
                    help="auto: one pass per step where the lattice allows it")
    ap.add_argument("--lbfgs-iters", type=int, default=0,
                    help="--workload em: only this many L-BFGS iterations (tol 0), for profiling")
    ap.add_argument("--nfluid", type=int, default=3, choices=[3, 4],
                    help="fluid components of --workload multi")
    ap.add_argument("--zrun", type=int, default=0,
                    help="z planes per block of the one-pass step (0: automatic)")
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "f16"],
                    help="population storage of the default workload (arithmetic in FP32)")
    ap.add_argument("--g-storage", default="auto", choices=["auto", "populations"],
                    help="g held as g_eq when tau_g = 1 (auto) or as populations")
    ap.add_argument("--shape", default=",".join(map(str, SHAPE)),
                    help="lattice size nx,ny,nz (default: the benchmark workload)")
    ap.add_argument("--workload", default="lb",
                    choices=["lb", "serve", "precision", "fp64", "em", "critical", "capillary",
                             "multi", "ramp", "cfg3"])
    ap.add_argument("--cfg3-steps", type=int, default=50000)
    ap.add_argument("--cfg3-check", type=int, default=5000)
    ap.add_argument("--cfg3-budget", type=float, default=900.0,
                    help="seconds the FP64 run may take; fewer steps if it would take longer")
    ap.add_argument("--cfg3-shape", default="384,384,256")
    ap.add_argument("--cfg3-reference", default="f64", choices=["f64", "f32"],
                    help="the form the others are compared with (f32: FP64 is not run)")
    ap.add_argument("--ramp-seeds", type=int, default=5)
    ap.add_argument("--ramp-steps", type=int, default=10000)
    ap.add_argument("--em-iters", type=int, default=20000)
    # default: a saturating burst (every request at once, full step budgets)
    ap.add_argument("--serve-requests", type=int, default=48)
    ap.add_argument("--serve-rate", type=float, default=1000.0)
    ap.add_argument("--serve-scale", type=float, default=1.0)
    ap.add_argument("--serve-quantum", type=int, default=200)
    ap.add_argument("--serve-max-large", type=int, default=2,
                    help="large lattices active at once (0: no cap)")
    ap.add_argument("--serve-order", default="sjf", choices=["fifo", "sjf"])
    ap.add_argument("--no-serial-baseline", action="store_true")
    args = ap.parse_args()
    assert args.warmup >= 3, "at least 3 warm-up steps"
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "serve":
        return run_serve(args, rank, world)
    if args.workload == "precision":
        return run_precision(args, rank, world)
    if args.workload == "fp64":
        return run_plain_fp64(args, rank, world)
    if args.workload == "em":
        return run_em(args, rank, world)
    if args.workload == "multi":
        return run_multi(args, rank, world)
    if args.workload == "capillary":
        return run_capillary(args, rank, world)
    if args.workload == "critical":
        return run_critical(args, rank, world)
    if args.workload == "ramp":
        return run_ramp(args, rank, world)
    if args.workload == "cfg3":
        return run_cfg3(args, rank, world)
    return run_gpu(args, rank, world)


if __name__ == "__main__":
    sys.exit(main())
