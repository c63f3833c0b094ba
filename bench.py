"""Throughput of the pseudopotential-LBM wetting step on GB300.

Workload: the paper-shaped sweep -- 72 sessile droplets on 400 x 200
lattices (radius 50 on a flat wall; density-based, pseudopotential-based and
modified interactions at 12 G_w values each over the ranges of Sec. III.C;
vapour/liquid viscosity ratios 1 and 10) held as one batched context.  One
bench step = one time step of all 72 lattices (5.76 M nodes).  `value` is the
FP32 shifted-population path (MLUPS, all nodes counted); the FP64 path is
reported under "fp64".  Inputs are larger than L2 (415 MB FP32, 830 MB FP64
of populations), so no L2 flush is needed between steps.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX, NY, R = 400, 200, 50.0
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
BYTES_PER_NODE = {"fp32": 72.0, "fp32_f64": 72.0, "fp64": 144.0}
KERNEL_SRC = os.path.join(ROOT, "paper_1410_2569_gb300", "csrc", "lbm_kernels.cu")
PROFILE = os.path.join(ROOT, "profiles", "step_kernel_sweep.md")


def kernel_sha():
    import hashlib
    with open(KERNEL_SRC, "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()


def profile_figures():
    """Per-launch counters of the step kernels from the committed ncu summary
    (lines `key: value`), or {} when that summary was taken on a different
    kernel source than the one built now."""
    try:
        with open(PROFILE) as fh:
            kv = dict(ln.strip().split(": ", 1) for ln in fh
                      if re.match(r"[a-z0-9_-]+: ", ln))
    except OSError:
        return {}
    if kv.get("kernel-source-sha256", "").strip() != kernel_sha():
        return {}
    out = {}
    for k, v in kv.items():
        try:
            out[k] = float(v.split()[0])
        except (ValueError, IndexError):
            pass
    return out


def sweep_instances(prec, world_size=1, rank=0):
    from paper_1410_2569_gb300 import default_params, inputs
    solid = inputs.flat_walls(NX, NY)
    out = []
    for c in inputs.sweep_cases(world_size, rank):
        p = default_params(prec=prec, tau_nu_L=c["tau_nu_L"], tau_nu_V=c["tau_nu_V"])
        out.append(dict(nx=NX, ny=NY, params=p, solid=solid, fsi=c["fsi"],
                        gw=inputs.wall_gw(solid, c["gw"])))
    return out


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
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
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def fp64_rate():
    """FP64 pipe throughput of this GPU, DFMA instructions per second, from
    the library's probe (lbm_selftest_fp64_rate), measured in this run."""
    import ctypes
    import paper_1410_2569_gb300 as lbm
    v = ctypes.c_double()
    if lbm.load().lbm_selftest_fp64_rate(ctypes.byref(v)) != 0:
        return None
    return v.value


def measured_peaks():
    try:
        with open(PEAKS_FILE) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def droplet_density(nx, ny, x0, y0, R, W, rho_L=500.0, rho_V=1.0):
    """Host input of the end-to-end leg: a sessile-droplet density field with
    a tanh interface of width W (minimum image in x)."""
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    dx = x - x0
    dx -= nx * np.floor(dx / nx + 0.5)
    r = np.sqrt(dx * dx + (y - y0) ** 2)
    return rho_V + 0.5 * (rho_L - rho_V) * (1.0 - np.tanh(2.0 * (r - R) / W))


def max_over_ranks(value, dist=None, device="cpu"):
    """The largest value over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def time_device(lat, stream, steps, warmup):
    import torch
    lat.step(warmup)
    lat.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stream.synchronize()
    e0.record(stream)
    lat.step(steps)
    e1.record(stream)
    e1.synchronize()
    lat.sync()
    return e0.elapsed_time(e1) / 1000.0


def run_ours(args, ws, rank, local):
    import torch
    import paper_1410_2569_gb300 as lbm
    from paper_1410_2569_gb300 import inputs

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.Stream()
    nodes = len(inputs.sweep_cases()) * NX * NY
    results = {}
    y_w = inputs.wall_height("copy")
    precs = ("fp32", "fp32_f64", "fp64") if args.prec == "both" else (args.prec,)
    for prec in precs:
        insts = sweep_instances(prec, ws, rank)
        lat = lbm.Lattice(insts, stream=stream)
        for k in range(len(insts)):
            lat.init_droplet(NX / 2, y_w, R, inputs.SWEEP_WIDTH, inst=k)
        if args.launch:
            v = [int(x) for x in args.launch.split(",")]
            bx, h, pers, graph = v[:4]
            lat.set_launch(bx, h, pers, graph, v[4] if len(v) > 4 else 0)
        # warm-up, then the timed region bracketed by barrier + synchronize
        lat.step(args.warmup)
        lat.sync()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        with Clocks(local) as clk:
            dt = time_device(lat, stream, args.steps, 0)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        dt = max_over_ranks(dt, dist, "cuda")
        mlups = ws * nodes * args.steps / dt / 1e6
        results[prec] = dict(dt=dt, mlups=mlups, clocks=clk.summary(), lat=lat)
        if prec != "fp32":
            lat.close()
            results[prec].pop("lat")
    # the large single lattice (8192 x 4096, striped wall, 2000 droplets):
    # an extra figure beside the sweep, one lattice far larger than L2
    large = None
    if args.large and args.prec == "both":
        large = {}
        lnx, lny = 8192, 4096
        solid_l, gw_l, drops_l = inputs.large_striped(lnx, lny, 2000, seed=0)
        rho_l = inputs.droplet_field(lnx, lny, drops_l, 4.0)
        for prec, nsteps in (("fp32", 50), ("fp64", 10)):
            lat = lbm.Lattice.single(lnx, lny, lbm.default_params(prec=prec), solid_l, "modified",
                                     gw_l, stream=stream)
            lat.set_density(rho_l)
            lat.step(3)
            lat.sync()
            dt_l = max_over_ranks(time_device(lat, stream, nsteps, 0), dist, "cuda")
            ml = ws * lnx * lny * nsteps / dt_l / 1e6
            large[prec] = {"value": round(ml, 1), "unit": "MLUPS", "steps": nsteps,
                           "ms_per_step": round(dt_l / nsteps * 1e3, 4),
                           "algorithmic_GBps": round(ml * 1e6 * BYTES_PER_NODE[prec] / 1e9 / ws, 1)}
            lat.close()
    accuracy = None
    if args.accuracy and args.prec == "both" and rank == 0:
        accuracy = sweep_accuracy()
    extra = None
    if args.extra and args.prec == "both" and rank == 0:
        extra = {"batched_uneven": batched_uneven(stream), "adjoint": adjoint_cost(stream)}
    # end-to-end through the C ABI with host buffers: host density fields in,
    # `chunk` steps, host rho/ux/uy fields out, per e2e iteration
    e2e = None
    if not args.no_e2e and "fp32" in results:
        lat = results["fp32"]["lat"]
        n_inst = len(inputs.sweep_cases())
        total = lat.total_nodes
        chunk, iters = max(1, args.steps // 2), 2
        # pinned host fields of the whole batch, concatenated in instance
        # order: one upload and one read-back per field and iteration; each
        # iteration's fields land in their own host arrays
        host_rho = torch.empty(total, dtype=torch.float64).pin_memory().numpy()
        host_out = [{k: torch.empty(total, dtype=torch.float64).pin_memory().numpy()
                     for k in ("rho", "ux", "uy")} for _ in range(iters)]
        one = droplet_density(NX, NY, NX / 2, y_w, R, inputs.SWEEP_WIDTH)
        for v in lat.split(host_rho):
            v[:] = one
        # one untimed iteration: the library makes its copy streams and the
        # upload staging buffer on first use
        lat.set_density_all(host_rho)
        lat.step(1)
        lat.fields_all(host_out[0])
        lat.sync()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # the library overlaps each upload with the steps queued before it
        # and each read-back with the steps queued after it; one
        # synchronisation at the end, inside the timed region
        for it in range(iters):
            lat.set_density_all(host_rho)
            lat.step(chunk)
            lat.fields_all(host_out[it])
        lat.sync()
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        for o in host_out:  # every iteration's fields arrived
            assert np.isfinite(o["rho"]).all() and o["rho"].max() > 100.0
        e2e = {"value": round(ws * nodes * chunk * iters / te / 1e6, 2), "unit": "MLUPS",
               "h2d_bytes_per_step": n_inst * NX * NY * 8 / chunk,
               "d2h_bytes_per_step": 3 * n_inst * NX * NY * 8 / chunk,
               "steps_per_call": chunk}
    for r in results.values():
        r.pop("lat", None)
    if rank != 0 or args.prec != "both":
        if dist:
            dist.destroy_process_group()
        if rank == 0:
            print(json.dumps({k: {kk: vv for kk, vv in v.items() if kk != "clocks"}
                              for k, v in results.items()}))
        return
    hbm, peak_kind = measured_peaks()
    f32, f64, f3264 = results["fp32"], results["fp64"], results["fp32_f64"]
    prof = profile_figures()

    def roof(prec, dt, steps):
        achieved = nodes * BYTES_PER_NODE[prec] * steps / dt / 1e9  # per GPU
        return achieved
    ach32 = roof("fp32", f32["dt"], args.steps)
    ach64 = roof("fp64", f64["dt"], args.steps)
    # FP64 step: FP64-pipe instructions per node counted by ncu
    # (smsp__inst_executed_pipe_fp64 x 32 / nodes) in the committed profile,
    # else the count from the source arithmetic (density 8, psi ~12,
    # collision ~120)
    fp64_ops_node = prof.get("fp64_pipe_thread_ops_per_node", 140.0)
    fp64_alu = nodes * fp64_ops_node * args.steps / f64["dt"] / 1e9
    fp64_peak = fp64_rate()  # after the timed regions
    cpu = cpu_baseline(args) if not args.no_cpu else None
    line = {
        "metric": "D2Q9 MLUPS & % HBM roofline, FP32 vs FP64 at <=0.5 deg contact-angle error",
        "value": round(f32["mlups"], 2),
        "unit": "MLUPS",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(f32["dt"] / args.steps * 1e3, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "paper-shaped sweep: 72 sessile droplets, 400x200 each, "
                               "3 interactions x 12 G_w x viscosity ratio {1,10}, R=50",
                   "nodes_per_gpu": nodes, "lattice": [NX, NY], "instances": 72,
                   "l2": "inputs larger than L2 (415 MB FP32 populations), no flush",
                   "parallelism": f"independent sweeps per GPU x{ws}",
                   "precision": "FP32 populations stored as f - w rho_ref; density and psi "
                                "from compensated FP32 sums (error-free transformations, "
                                "FP64-grade, no FP64 instruction); FP64 density and psi "
                                "instructions: fp32_f64"},
        "roofline": {"bound": "hbm", "achieved": round(ach32, 1), "peak": hbm,
                     "unit": "GB/s", "frac": round(ach32 / hbm, 4),
                     "traffic": prof.get("fp32_dram_bytes_per_launch"),
                     "peak_kind": peak_kind,
                     "algorithmic_bytes_per_node": BYTES_PER_NODE["fp32"]},
        "fp64": {"value": round(f64["mlups"], 2), "unit": "MLUPS",
                 "ms_per_step": round(f64["dt"] / args.steps * 1e3, 4),
                 "roofline": {"bound": "alu", "achieved": round(fp64_alu, 1),
                              "peak": None if fp64_peak is None else round(fp64_peak / 1e9, 1),
                              "unit": "G FP64 ops/s",
                              "frac": None if fp64_peak is None else
                              round(fp64_alu * 1e9 / fp64_peak, 4),
                              "peak_kind": "measured in this run: DFMA probe "
                                           "(lbm_selftest_fp64_rate)",
                              "fp64_ops_per_node": fp64_ops_node,
                              "fp64_ops_per_node_source": "ncu profile" if
                              "fp64_pipe_thread_ops_per_node" in prof else "source count",
                              "hbm_achieved_gbs": round(ach64, 1),
                              "hbm_frac": round(ach64 / hbm, 4)},
                 "clocks": f64["clocks"]},
        "fp32_f64": {"value": round(f3264["mlups"], 2), "unit": "MLUPS",
                     "ms_per_step": round(f3264["dt"] / args.steps * 1e3, 4),
                     "what": "FP32 populations with density and psi in FP64 instructions",
                     "hbm_frac": round(nodes * BYTES_PER_NODE["fp32_f64"] * args.steps /
                                       f3264["dt"] / 1e9 / hbm, 4)},
        "accuracy": accuracy,
        "e2e": e2e,
        "large_lattice": None if large is None else dict(
            large, workload="8192x4096, bottom wall in 64-node G_w stripes -0.1/0.3, "
                            "2000 droplets R 10-40, modified interaction",
            hbm_frac_fp32=round(large["fp32"]["algorithmic_GBps"] / hbm, 4)),
        "batched_uneven": None if extra is None else extra["batched_uneven"],
        "adjoint": None if extra is None else extra["adjoint"],
        "gpu_launches": args.steps,
        "clocks": f32["clocks"],
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    append_log(args, line)
    if dist:
        dist.destroy_process_group()


def sweep_accuracy(steps=30000):
    """The metric's accuracy condition on sampled sweep lattices: each
    interaction at both ends of its G_w range at viscosity ratios 1 and 10
    (12 lattices), `steps` steps in FP32 (default storage), FP32 with FP64
    density and psi, and FP64; the largest differences from FP64 over the
    sample.  Outside the timed region."""
    import paper_1410_2569_gb300 as lbm
    from paper_1410_2569_gb300 import inputs
    cases = [c for c in inputs.sweep_cases()
             if any(np.isclose(c["gw"], v) for v in inputs.GW_RANGES[c["fsi"]])]
    solid = inputs.flat_walls(NX, NY)
    fluid = solid == 0
    res = {}
    for prec in ("fp64", "fp32", "fp32_f64"):
        specs = [dict(nx=NX, ny=NY, params=lbm.default_params(prec=prec, tau_nu_L=c["tau_nu_L"],
                                                               tau_nu_V=c["tau_nu_V"]),
                      solid=solid, fsi=c["fsi"], gw=inputs.wall_gw(solid, c["gw"]))
                 for c in cases]
        lat = lbm.Lattice(specs)
        for k in range(len(cases)):
            lat.init_droplet(NX / 2, 0.5, R, inputs.SWEEP_WIDTH, inst=k)
        lat.step(steps)
        lat.sync()
        res[prec] = [(lat.fields(k)["rho"], lat.diagnostics(inst=k, y_w=0.5, x_ref=NX / 2))
                     for k in range(len(cases))]
        lat.close()
    out = {"steps": steps, "lattices": len(cases),
           "sample": "each interaction at the lowest and highest G_w of its range, viscosity "
                     "ratios 1 and 10, 400x200, R=50; differences from the FP64 step"}
    for prec in ("fp32", "fp32_f64"):
        th, ext, pt, frac, scale = 0.0, 0.0, 0.0, 0.0, 0.0
        for (r, d), (r64, d64) in zip(res[prec], res["fp64"]):
            th = max(th, abs(d["theta_deg"] - d64["theta_deg"]))
            ext = max(ext, *(abs(d[k] / d64[k] - 1.0) for k in ("rho_max", "rho_min", "mass")))
            diff = np.abs(r - r64)[fluid]
            rel = diff / r64[fluid]
            pt, frac = max(pt, float(rel.max())), max(frac, float(np.mean(rel > 1e-4)))
            scale = max(scale, float(diff.max()) / 499.0)
        out[prec] = {"theta_max_abs_diff_deg": th, "rho_extrema_mass_max_rel": ext,
                     "rho_node_max_rel": pt, "rho_node_frac_above_1e-4": frac,
                     "rho_node_max_abs_over_range": scale}
    return out


def batched_uneven(stream, steps=1000):
    """The batched workload: 64 lattices of seeded log-uniform sizes (128x64
    to 512x256), random interaction and G_w per lattice, droplets of radius
    ny/4, FP32 storage.  MLUPS (all nodes) over `steps` steps for each launch
    mode: warp strips one launch per step (the FP32 column-pair strips:
    every width here is a multiple of 8); the same in a CUDA graph of
    `steps` launches; one persistent cooperative launch per `steps` steps
    captured in a graph, block rows with a grid barrier per step or the
    column-pair strips each waiting on its neighbours; the shape
    lbm_autotune picks."""
    import paper_1410_2569_gb300 as lbm
    from paper_1410_2569_gb300 import inputs
    cases = inputs.batch_instances(64, seed=0)
    specs = []
    for c in cases:
        solid = inputs.flat_walls(c["nx"], c["ny"])
        specs.append(dict(nx=c["nx"], ny=c["ny"], params=lbm.default_params(prec="fp32"),
                          solid=solid, fsi=c["fsi"], gw=inputs.wall_gw(solid, c["gw"])))
    lat = lbm.Lattice(specs, stream=stream)
    y_w = inputs.wall_height("copy")
    for k, c in enumerate(cases):
        lat.init_droplet(c["nx"] / 2, y_w, c["R"], 2.0, inst=k)
    nodes = sum(c["nx"] * c["ny"] for c in cases)
    out = {"instances": len(cases), "nodes": nodes, "steps": steps, "unit": "MLUPS"}
    modes = (("warp_strips", dict(stages=0)), ("warp_strips_graph", dict(stages=0, graph=True)),
             ("persistent_graph", dict(stages=1, persistent=True, graph=True)),
             ("persistent_warp_strips_graph", dict(stages=0, persistent=True, graph=True)))
    for name, kw in modes:
        lat.set_launch(**kw)
        dt = time_device(lat, stream, steps, steps)  # the warm-up captures the graph
        out[name] = round(nodes * steps / dt / 1e6, 1)
    lat.set_launch()
    t = lat.autotune(steps=20)
    dt = time_device(lat, stream, steps, steps)
    out["autotuned"] = round(nodes * steps / dt / 1e6, 1)
    out["autotuned_shape"] = {k: t[k] for k in ("bx", "h", "stages", "persistent")}
    lat.close()
    return out


def adjoint_cost(stream, T=2000):
    """The differentiation workload: 256x128, droplet of radius 32, modified
    interaction, a G_w field of 256 wall-node parameters (0.1), FP64; the
    loss (theta - theta_target)^2 with theta_target 10 deg above the initial
    angle.  Wall time of lbm_adjoint over T steps (forward with checkpoints,
    seed, reverse sweep, gradient) against T forward steps alone."""
    import paper_1410_2569_gb300 as lbm
    from paper_1410_2569_gb300 import inputs
    nx, ny = 256, 128
    solid = inputs.flat_walls(nx, ny)
    gw = inputs.wall_gw(solid, 0.1)

    def fresh():
        lat = lbm.Lattice.single(nx, ny, lbm.default_params(prec="fp64"), solid, "modified", gw,
                                 stream=stream)
        lat.init_droplet(nx / 2, 0.5, 32.0, 2.0)
        return lat
    lat = fresh()
    target = lat.diagnostics(y_w=0.5, x_ref=nx / 2)["theta_deg"] + 10.0
    lat.step(T)  # warm-up: module load, graphs of the step
    lat.sync()
    lat.close()
    lat = fresh()
    dt_fwd = time_device(lat, stream, T, 0)
    lat.close()
    lat = fresh()
    t0 = time.perf_counter()
    loss, theta, grad = lat.adjoint(T, target, 0.5, nx / 2, 3.0)
    dt_adj = time.perf_counter() - t0
    lat.close()
    assert np.isfinite(grad).all() and np.abs(grad[0]).max() > 0.0
    return {"lattice": [nx, ny], "steps": T, "forward_ms": round(dt_fwd * 1e3, 2),
            "adjoint_ms": round(dt_adj * 1e3, 2), "adjoint_over_forward": round(dt_adj / dt_fwd, 2),
            "parameters": int(np.count_nonzero(gw)), "loss": loss, "theta_deg": theta}


def cpu_baseline(args, budget_s=None):
    """The FP64 oracle as it stands on this host's cores: a bounded sample of
    the sweep (the first instances of the batch for a few steps)."""
    import oracle
    from paper_1410_2569_gb300 import inputs
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    budget = budget_s if budget_s is not None else args.cpu_seconds
    solid = inputs.flat_walls(NX, NY)
    cases = inputs.sweep_cases()
    y_w = inputs.wall_height("copy")
    done_nodes, t_used, n_inst, steps_each = 0, 0.0, 0, 0
    t0 = time.perf_counter()
    k = 0
    while time.perf_counter() - t0 < budget and k < len(cases):
        c = cases[k]
        p = oracle.paper_params(tau_nu_L=c["tau_nu_L"], tau_nu_V=c["tau_nu_V"])
        o = oracle.Lattice(NX, NY, p, solid, c["fsi"], inputs.wall_gw(solid, c["gw"]))
        o.init_droplet(NX / 2, y_w, R, inputs.SWEEP_WIDTH)
        ts = time.perf_counter()
        steps = 0
        while time.perf_counter() - t0 < budget and steps < 200:
            o.step(10)
            steps += 10
        t_used += time.perf_counter() - ts
        done_nodes += NX * NY * steps
        n_inst += 1
        steps_each = max(steps_each, steps)
        k += 1
    # the same oracle on one thread: the first sweep lattice for a short slice
    oracle.set_threads(1)
    c = cases[0]
    p = oracle.paper_params(tau_nu_L=c["tau_nu_L"], tau_nu_V=c["tau_nu_V"])
    o = oracle.Lattice(NX, NY, p, solid, c["fsi"], inputs.wall_gw(solid, c["gw"]))
    o.init_droplet(NX / 2, y_w, R, inputs.SWEEP_WIDTH)
    ts, steps1 = time.perf_counter(), 0
    while time.perf_counter() - ts < max(1.0, 0.15 * budget) and steps1 < 200:
        o.step(5)
        steps1 += 5
    one = NX * NY * steps1 / (time.perf_counter() - ts) / 1e6
    oracle.set_threads(cores)
    # the same oracle, all cores and one thread, on the small single lattice
    # (100x60, psi-based G_w = 1.0, R = 20) and on a 1024x512 slice of the
    # large lattice's pattern (G_w stripes, 30 droplets): about a second each
    other = {}
    slice_s = max(0.5, 0.05 * budget)
    s1 = inputs.flat_walls(100, 60)
    s5, g5, d5 = inputs.large_striped(1024, 512, 30, seed=0)
    rho5 = inputs.droplet_field(1024, 512, d5, 4.0)
    for threads, key in ((cores, "cores"), (1, "1thread")):
        oracle.set_threads(threads)
        o = oracle.Lattice(100, 60, oracle.paper_params(), s1, "psi", inputs.wall_gw(s1, 1.0))
        o.init_droplet(50.0, y_w, 20.0, 2.0)
        other.setdefault("100x60", {})[key] = _oracle_rate(o, 100 * 60, slice_s)
        o = oracle.Lattice(1024, 512, oracle.paper_params(), s5, "modified", g5)
        o.set_density(rho5)
        other.setdefault("1024x512 striped slice", {})[key] = _oracle_rate(o, 1024 * 512,
                                                                           slice_s)
    oracle.set_threads(cores)
    return {"value": round(done_nodes / t_used / 1e6, 3), "unit": "MLUPS", "cores": cores,
            "kind": "oracle", "cpu_model": cpu_model(), "value_1thread": round(one, 3),
            "other_lattices_mlups": other,
            "sample": f"{n_inst} of the 72 sweep lattices (400x200), up to {steps_each} steps "
                      f"each, {t_used:.1f} s of CPU time; one thread: the first lattice, "
                      f"{steps1} steps"}


def _oracle_rate(o, nodes, seconds):
    """MLUPS of oracle lattice o stepped for about `seconds`"""
    ts, steps = time.perf_counter(), 0
    while time.perf_counter() - ts < seconds and steps < 2000:
        o.step(2)
        steps += 2
    return round(nodes * steps / (time.perf_counter() - ts) / 1e6, 3)


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def run_reference(args, ws, rank):
    if rank != 0:
        return
    cpu = cpu_baseline(args, budget_s=max(5.0, args.cpu_seconds))
    line = {
        "metric": "D2Q9 MLUPS & % HBM roofline, FP32 vs FP64 at <=0.5 deg contact-angle error",
        "value": cpu["value"], "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(72 * NX * NY / (cpu["value"] * 1e6) * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": "paper-shaped sweep: 72 sessile droplets, 400x200 each, "
                               "3 interactions x 12 G_w x viscosity ratio {1,10}, R=50",
                   "nodes_per_gpu": 72 * NX * NY, "lattice": [NX, NY], "instances": 72},
        "cpu_baseline": cpu,
        "e2e": {"value": cpu["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    append_log(args, line)


def append_log(args, line):
    """--log: append the line with the git commit, the host's core count and
    the GPU's name to a JSONL file (one record per run)."""
    if not args.log:
        return
    rec = dict(line)
    try:
        rec["git_commit"] = subprocess.run(["git", "rev-parse", "HEAD"], cwd=ROOT,
                                           capture_output=True, text=True,
                                           timeout=10).stdout.strip() or None
    except (OSError, subprocess.SubprocessError):
        rec["git_commit"] = None
    rec["host_cores"] = os.cpu_count()
    try:
        import torch
        rec["gpu_name"] = torch.cuda.get_device_name(0) if torch.cuda.is_available() else None
    except Exception:
        rec["gpu_name"] = None
    rec["time_utc"] = time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())
    with open(args.log, "a") as fh:
        fh.write(json.dumps(rec) + "\n")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--launch", default="",
                    help="bx,h,persistent,graph[,stages] as in lbm_set_launch")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", dest="extra", action="store_false",
                    help="skip the batched-uneven and adjoint figures")
    ap.add_argument("--log", default="",
                    help="also append the JSON line, with the git commit, host cores and GPU "
                         "name, to this JSONL file")
    ap.add_argument("--no-accuracy", dest="accuracy", action="store_false",
                    help="skip the 30,000-step FP32-vs-FP64 accuracy sample")
    ap.add_argument("--no-large", dest="large", action="store_false",
                    help="skip the extra 8192x4096 single-lattice figure")
    ap.add_argument("--prec", default="both", choices=["both", "fp32", "fp32_f64", "fp64"],
                    help="a single precision prints only its timings (profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
