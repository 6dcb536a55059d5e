"""Benchmark: lattice updates per second of the coupled LBM-DEM step on GB300.

Workload (synthetic): 256^3 D3Q19 box, periodic in x and y, walls in z with
the top one sliding at 0.05; tau0 = 0.51, Smagorinsky C = 0.17; 2000 spheres
of radius 4 placed by seeded random sequential addition (solid fraction
0.032), velocities uniform in [-0.01, 0.01]^3, density ratio 2.5, k_n = 1e3,
restitution 0.8, 16 DEM sub-steps per lattice step.  One step = geometry,
refill, fused collide-stream, bounce-back + momentum exchange, DEM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|bf16|fp16]
  python bench.py --impl reference ...   # the FP64 CPU oracle, bounded sample

Prints one JSON line (rank 0).  MLUPS counts every node of the box.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & % HBM roofline at 256^3 + 2000 spheres; FP32 vs BF16-storage vs FP64 err"
BOX = (256, 256, 256)
NSPH = 2000
PHYS = dict(tau0=0.51, cs=0.17, g=(0.0, 0.0, 0.0), u_lo=(0.0, 0.0, 0.0), u_hi=(0.05, 0.0, 0.0), rho_s=2.5,
            kn=1e3, restitution=0.8, dem_substeps=16)
BYTES = {"fp32": 4, "bf16": 2, "fp16": 2}


def workload_name(prec, nsph=None, dense=False):
    name = "slurry box %d^3, %d spheres R=4, sliding lid 0.05, tau0=0.51, Cs=0.17, %s storage" % (
        BOX[0], NSPH if nsph is None else nsph, prec)
    if dense:
        name += ", solid fraction 0.13 (phi-matched count), tangential friction"
    return name


def workload_spheres(args):
    """Spheres of the timed workload: the 2000-sphere box, or with
    --workload dense the same box at the solid fraction 0.13 it names."""
    from paper_1703_05158_gb300 import inputs

    if getattr(args, "workload", "slurry") == "dense":
        return inputs.phi_matched_slurry(box=BOX)
    return oracle_sample(BOX, NSPH)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def collide_source_sha():
    """First 16 hex digits of the SHA-256 of the collide kernel's sources."""
    import hashlib

    h = hashlib.sha256()
    for name in ("lbm_collide.cu", "lbm_collide_node.cuh", "lbm_stream.cuh"):
        with open(os.path.join(ROOT, "paper_1703_05158_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(prec):
    """DRAM bytes per collide launch from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "stream_collide_256cubed_%s.md" % prec)
    try:
        text = open(path).read()
        sha = collide_source_sha()
        vals = dict(l.split(":", 1) for l in text.splitlines() if l.startswith(("traffic_bytes_per_launch:",
                                                                                  "collide_source_sha256_16:")))
        if vals.get("collide_source_sha256_16:".rstrip(":"), "").strip() != sha:
            return None
        return float(vals["traffic_bytes_per_launch"])
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                s, m = float(f[1]), float(f[2])
            except ValueError:
                continue
            sm.append(s)
            mx = max(mx, m)
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        load = sorted(sm)[len(sm) // 4:] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(box, nsph, seed_offset=0):
    from paper_1703_05158_gb300 import inputs

    return inputs.slurry_box(box=box, n=nsph, seed=inputs.SEED_BASE + 2 + seed_offset)


def error_vs_fp64(precision, steps=200):
    """Relative L2 velocity error (nodes fluid on both sides) and largest
    relative sphere-force error of the GPU path at this storage precision
    against the FP64 oracle, on a 64^3 sub-box of the production physics at
    the same sphere density (31 spheres of radius 4), after 200 steps."""
    import numpy as np

    import oracle
    from paper_1703_05158_gb300 import inputs, lbm

    box = (64, 64, 64)
    p = inputs.slurry_box(box=box, n=31, radius=4.0, seed=inputs.SEED_BASE + 8)
    lat = lbm.Lattice(*box, precision=precision, max_particles=31, max_radius=4.0, **PHYS)
    orc = oracle.Oracle(*box, **PHYS)
    for o in (lat, orc):
        o.set_particles(p["X"], V=p["V"], Om=p["Om"], R=p["R"])
    lat.step(steps)
    orc.step(steps)
    _, ug = lat.fields()
    _, uo = orc.fields()
    fluid = (orc.owner() < 0) & (lat.owner() < 0)
    a, b = ug[:, fluid].astype(np.float64), uo[:, fluid]
    Fg, _ = lat.forces()
    Fo, _ = orc.forces()
    lat.close()
    return {"relative_l2_velocity": float(np.linalg.norm(a - b) / np.linalg.norm(b)),
            "max_relative_force": float((np.linalg.norm(Fg - Fo, axis=1) / np.linalg.norm(Fo, axis=1)).max()),
            "case": "64^3 sub-box, 31 spheres R=4, %d steps, against the FP64 oracle" % steps}


def precision_form(args, prec, p, stream, dev, fp32_ms):
    """The same workload with populations stored as 16-bit deviations: MLUPS
    over the same number of timed steps (after the same warm-up), the ratio
    to the FP32 line, and the velocity / force error against the FP64 oracle
    on the 64^3 sub-box."""
    import torch

    from paper_1703_05158_gb300 import lbm

    lat = lbm.Lattice(*BOX, precision=prec, max_particles=len(p["R"]), max_radius=4.0, stream=ctypes_stream(stream),
                      device=dev, schedule=args.schedule, **PHYS)
    lat.set_particles(p["X"], V=p["V"], Om=p["Om"], R=p["R"])
    lat.step(args.warmup)
    lat.sync()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    lat.step(args.steps)
    end.record(stream)
    torch.cuda.synchronize()
    lat.sync()
    ms = start.elapsed_time(end) / args.steps
    lat.close()
    out = {"value": BOX[0] * BOX[1] * BOX[2] / (ms * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": ms,
           "ratio_to_fp32": fp32_ms / ms}
    if not args.no_error_check:
        out["error_vs_fp64"] = error_vs_fp64(prec)
    return out


def cpu_baseline(steps=2):
    """The oracle as it stands on the host cores, on the full workload for a
    couple of steps (bounded sample)."""
    import oracle

    p = oracle_sample(BOX, NSPH)
    o = oracle.Oracle(*BOX, **PHYS)
    o.set_particles(p["X"], V=p["V"], Om=p["Om"], R=p["R"])
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    n = BOX[0] * BOX[1] * BOX[2]
    return {"value": n * steps / dt / 1e6, "unit": "MLUPS", "cores": int(os.environ.get("OMP_NUM_THREADS",
                                                                                        os.cpu_count())),
            "kind": "oracle", "sample": "%d steps of the full 256^3 + 2000-sphere workload, FP64, %.1f s" % (steps, dt),
            "single_thread": single_thread_baseline()}


def single_thread_baseline(steps=3):
    """The oracle on one host thread (a child process with OMP_NUM_THREADS=1)
    on a 64^3 box at the workload's sphere density (31 spheres of radius 4)."""
    code = ("import time, bench, oracle\n"
            "from paper_1703_05158_gb300 import inputs\n"
            "p = inputs.slurry_box(box=(64, 64, 64), n=31, radius=4.0, seed=inputs.SEED_BASE + 8)\n"
            "o = oracle.Oracle(64, 64, 64, **bench.PHYS)\n"
            "o.set_particles(p['X'], V=p['V'], Om=p['Om'], R=p['R'])\n"
            "t = time.perf_counter(); o.step(%d); print(time.perf_counter() - t)\n" % steps)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, stdout=subprocess.PIPE,
                       stderr=subprocess.DEVNULL, text=True, timeout=600)
    dt = float(r.stdout.strip().splitlines()[-1])
    return {"value": 64 ** 3 * steps / dt / 1e6, "unit": "MLUPS", "cores": 1,
            "sample": "%d steps of a 64^3 box with 31 spheres R=4 (the workload's density), %.1f s" % (steps, dt)}


def max_over_ranks(x, world):
    """Maximum of a host float over the ranks of the job (every rank calls
    it; NCCL with GPUs, gloo in the CPU tests)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def whole_job_mlups(updates_per_rank, world, seconds):
    """Node updates of all ranks (replicas) over the slowest rank's time."""
    return world * updates_per_rank / seconds / 1e6


def friction_params(args):
    """Tangential contact law of the --friction and --workload dense runs
    (none by default)."""
    if not (getattr(args, "friction", False) or getattr(args, "workload", "slurry") == "dense"):
        return {}
    return dict(kt=0.5 * PHYS["kn"], mu=0.3, restitution_t=0.6)


def zieb_params(args):
    """ZIEB face of the --zieb runs (none by default)."""
    if not getattr(args, "zieb", False):
        return {}
    A = float(BOX[0] * BOX[1])
    return dict(zieb=dict(area=A, volume=40.0 * A, vp=0.005))


def run_reference(args, rank, world):
    """--impl reference: the FP64 oracle on the host, each step a bounded
    sample of the workload (a 48^3 box at the same solid fraction: 13 spheres
    of radius 4)."""
    if rank != 0:
        return
    import oracle

    box, nsph = (48, 48, 48), 13
    p = oracle_sample(box, nsph, seed_offset=100)
    corr = bool(getattr(args, "momentum_correction", False))
    o = oracle.Oracle(*box, momentum_correction=corr, **PHYS, **friction_params(args))
    o.set_particles(p["X"], V=p["V"], Om=p["Om"], R=p["R"])
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    n = box[0] * box[1] * box[2]
    val = n * args.steps / dt / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count()))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.precision), "sample": "48^3 box, 13 spheres R=4 per step",
                       "momentum_correction": corr, "friction": friction_params(args) or None},
            "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": "48^3 box with 13 spheres (solid fraction of the workload), %d steps" %
                                       args.steps},
            "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_1703_05158_gb300 import lbm

    torch.cuda.set_device(local_rank)
    dev = local_rank
    stream = torch.cuda.Stream(device=dev)
    p = workload_spheres(args)
    nsph = len(p["R"])
    dense = args.workload == "dense"
    lat = lbm.Lattice(*BOX, precision=args.precision, max_particles=nsph, max_radius=4.0,
                      stream=ctypes_stream(stream), device=dev, schedule=args.schedule,
                      momentum_correction=args.momentum_correction, mea=args.mea, **PHYS, **friction_params(args),
                      **zieb_params(args))
    lat.set_particles(p["X"], V=p["V"], Om=p["Om"], R=p["R"])
    N = BOX[0] * BOX[1] * BOX[2]

    # warm-up
    lat.step(args.warmup)
    lat.sync()
    info = lat.info()

    # timed region: events on the library's stream (the steps replay the
    # library's step graphs; the phase profiler is off here)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with Clocks(dev) as clk:
        start.record(stream)
        lat.step(args.steps)
        end.record(stream)
        torch.cuda.synchronize()
    lat.sync()
    ms = start.elapsed_time(end)
    # per-phase device times from a separate profiled run (events around each
    # phase on the launching stream; these steps launch kernel by kernel)
    lat.profile(True)
    lat.step(min(args.steps, 400))
    lat.sync()
    phases, psteps = lat.profile_read()
    lat.profile(False)
    ms_max = max_over_ranks(ms, world)
    value = whole_job_mlups(N * args.steps, world, ms_max * 1e-3)

    # end to end through the public API with host buffers: every step uploads
    # the external load (force, torque) from pinned host memory, steps, and
    # reads the hydrodynamic force, torque and the centres back
    n = nsph
    hF = torch.zeros((n, 3), dtype=torch.float64).pin_memory()
    hT = torch.zeros((n, 3), dtype=torch.float64).pin_memory()
    oF = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    oT = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    oX = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    ke = args.e2e_steps
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ke):
        lbm.lbm_set_particle_load(lat.h, hF, hT)
        lbm.lbm_step(lat.h, 1)
        lbm.lbm_particle_state(lat.h, oF, oT, oX)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_val = whole_job_mlups(N * ke, world, max_over_ranks(e2e_s, world))

    if rank != 0:
        return
    s = BYTES[args.precision]
    nf = info["fluid_nodes"]
    walls = 2 * BOX[0] * BOX[1] * 5 * s
    # the collide launch(es) read the flag (and, overlapped, the near tag) and
    # 19 + 19 populations of every fluid node once
    bytes_collide = nf * 2 * 19 * s + (2 if args.schedule == "overlap" else 1) * N + walls
    collide_ms = (phases["collide"] + phases["collide_far"]) / max(psteps, 1)
    step_bytes = bytes_collide + 16 * info["links"]
    achieved = bytes_collide / (collide_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    traffic = profiled_traffic(args.precision)
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(args.precision, nsph, dense), "box": list(BOX), "spheres": nsph,
                   "radius": 4.0, "solid_fraction": round(float(np.sum(4 / 3 * np.pi * p["R"] ** 3)) / N, 4),
                   "storage": args.precision, "schedule": args.schedule, "fluid_nodes": nf, "links": info["links"],
                   "momentum_correction": args.momentum_correction, "friction": friction_params(args) or None,
                   "zieb": zieb_params(args).get("zieb"), "mea": args.mea,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (populations %.2f GB)" % (19 * N * s / 1e9)},
        "roofline": {"bound": "hbm", "kernel": "k_stream_collide" + (" (near + far launches)" if args.schedule == "overlap" else ""),
                     "achieved": achieved,
                     "peak": peak,
                     "peak_kind": "%s hbm_gbs" % peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "algorithmic_bytes_per_launch": bytes_collide,
                     "avg_launch_ms": collide_ms, "frac_of_nominal_7900": achieved / 7900.0,
                     # the whole step: the collide bytes plus 16 B per cut link, over the step time
                     "step_bytes": step_bytes, "step_frac": step_bytes / (ms_max / args.steps * 1e-3) / 1e9 / peak,
                     "path_frac": step_bytes / (ms_max / args.steps * 1e-3) / 1e9 / peak},
        "mflups_fluid": value * nf / N,
        "phases_ms_per_step": {k: v / max(psteps, 1) for k, v in phases.items()},
        "clocks": clk.summary(),
        "e2e": {"value": e2e_val, "unit": "MLUPS", "steps": ke,
                "h2d_bytes_per_step": int(hF.numel() * 8 + hT.numel() * 8),
                "d2h_bytes_per_step": int((oF.numel() + oT.numel() + oX.numel()) * 8)},
        # per step with spheres: overlapped = far collide, near marks, near list, marks, refill,
        # near collide, links, neighbours, DEM; serial = marks, refill, collide, links, neighbours, DEM
        "gpu_launches": args.steps * (((9 if args.schedule == "overlap" else 6) if nsph else 1) + int(args.zieb)),
    }
    if world == 1 and not args.no_cpu_baseline and not dense:
        line["cpu_baseline"] = cpu_baseline()
    if world == 1 and not args.no_error_check and not dense:
        line["error_vs_fp64"] = error_vs_fp64(args.precision)
    lat.close()
    if world == 1 and args.precision == "fp32" and not dense and not args.no_precision_forms:
        line["precision_forms"] = {q: precision_form(args, q, p, stream, dev, ms_max / args.steps)
                                   for q in ("bf16", "fp16")}
    print(json.dumps(line), flush=True)


def run_batched(args, rank, world, local_rank):
    """The batched form: 64 independent instances of a parameter sweep (box
    edges from {48, 64, 96, 128, 160}, radii in [2, 6], solid fraction in
    [0.05, 0.25], Cs in [0.1, 0.2], tau0 in [0.51, 0.8], body force in
    [1e-6, 1e-5]), FP32, stepped together; MLUPS over all nodes of all
    instances."""
    import numpy as np
    import torch

    from paper_1703_05158_gb300 import inputs, lbm

    torch.cuda.set_device(local_rank)
    dev = local_rank
    stream = torch.cuda.Stream(device=dev)
    inst = inputs.batch_instances(count=args.batch)
    cfgs = [dict(nx=i["box"][0], ny=i["box"][1], nz=i["box"][2], precision=args.precision, **i["params"])
            for i in inst]
    batch = lbm.Batch(cfgs, stream=ctypes_stream(stream), device=dev)
    for m, i in zip(batch.members, inst):
        if len(i["parts"]["R"]):
            m.set_particles(i["parts"]["X"], V=i["parts"]["V"], R=i["parts"]["R"])
    tpb, grid, tune_ms = batch.tune()
    batch.step(args.warmup)
    batch.sync()
    infos = [m.info() for m in batch.members]
    N = sum(int(np.prod(i["box"])) for i in inst)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with Clocks(dev) as clk:
        start.record(stream)
        batch.step(args.steps)
        end.record(stream)
        torch.cuda.synchronize()
    batch.sync()
    ms = max_over_ranks(start.elapsed_time(end), world)
    value = whole_job_mlups(N * args.steps, world, ms * 1e-3)
    if rank != 0:
        batch.close()
        return
    s = BYTES[args.precision]
    bytes_collide = sum(inf["fluid_nodes"] * 2 * 19 * s + inf["nodes"] + 2 * i["box"][0] * i["box"][1] * 5 * s
                        for inf, i in zip(infos, inst))
    achieved = bytes_collide / (tune_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    line = {
        "metric": "MLUPS (all nodes of all instances) & % HBM roofline, batched parameter sweep", "value": value,
        "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else args.precision, "data": "synthetic",
        "config": {"workload": "batched sweep: %d instances, edges {48..160}, r in [2,6], phi in [0.05,0.25], "
                               "%s storage" % (len(inst), args.precision),
                   "instances": len(inst), "nodes": N, "spheres": int(sum(len(i["parts"]["R"]) for i in inst)),
                   "mean_phi": round(float(np.mean([i["phi"] for i in inst])), 4),
                   "collide_launch": {"threads": tpb, "blocks": grid},
                   "l2": "inputs larger than L2 (populations %.2f GB)" % (19 * N * s / 1e9)},
        "roofline": {"bound": "hbm", "kernel": "k_collide_batch", "achieved": achieved, "peak": peak,
                     "peak_kind": "%s hbm_gbs" % peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "algorithmic_bytes_per_launch": bytes_collide, "avg_launch_ms": tune_ms},
        "clocks": clk.summary(),
        "e2e": None,
        # per step: one graph of marks, refill, collide, links, neighbours, DEM
        "gpu_launches": args.steps * 6,
    }
    print(json.dumps(line), flush=True)
    batch.close()


def run_adjoint(args, rank, world, local_rank):
    """The differentiation form: a 128 x 64 x 64 channel (inlet peak 0.04,
    pressure outlet, 4 x 40 x 40 plate at x = 80, 200 fixed spheres of radius
    3, Cs = 0.15, tau0 = 0.6, g = 1e-6), 500 steps, checkpoints every 50, J =
    plate drag averaged over steps 301..500; one timed "step" is a full
    gradient evaluation (forward run plus adjoint sweep); MLUPS counts the
    forward lattice updates of it (N x 500 per evaluation)."""
    import numpy as np
    import torch

    from paper_1703_05158_gb300 import inputs, lbm

    torch.cuda.set_device(local_rank)
    stream = torch.cuda.Stream(device=local_rank)
    X, R = inputs.channel_spheres()
    cfg = dict(nx=128, ny=64, nz=64, tau0=0.6, cs=0.15, gx=1e-6, u_peak=0.04, plate_lo=(80, 12, 12),
               plate_hi=(83, 51, 51), steps=500, avg_from=301)
    ch = lbm.Channel(**cfg, checkpoint_every=50, X=X, R=R, device=local_rank, stream=ctypes_stream(stream))
    for _ in range(args.warmup):
        ch.forward()
        ch.backward()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    tf = tb = 0.0
    barrier(world)
    torch.cuda.synchronize()
    with Clocks(local_rank) as clk:
        for _ in range(args.steps):
            ev[0].record(stream)
            J = ch.forward()
            ev[1].record(stream)
            g = ch.backward()
            ev[2].record(stream)
            torch.cuda.synchronize()
            tf += ev[0].elapsed_time(ev[1])
            tb += ev[1].elapsed_time(ev[2])
    tf, tb = max_over_ranks(tf, world), max_over_ranks(tb, world)
    if rank != 0:
        return
    N, S = 128 * 64 * 64, 500
    ms = (tf + tb) / args.steps
    # reverse sweep, per node and step, FP32: recompute (read G^{s-1}, write G^s and f^s) and adjoint
    # step (read lambda^{s+1} and f^s, write lambda^s): 6 x 19 x 4 B; the link fractions are read at
    # cut nodes only and the per-node masks (16 B) are left out
    bytes_bwd = N * S * (6 * 19 * 4)
    achieved = bytes_bwd / (tb / args.steps * 1e-3) / 1e9
    peak, peak_kind = peaks()
    line = {
        "metric": "gradient evaluations of the mean plate drag (forward + adjoint), MLUPS of the forward updates",
        "value": whole_job_mlups(N * S, world, ms * 1e-3), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "differentiation form: 128x64x64 channel, plate 4x40x40 at x=80, 200 fixed spheres "
                               "R=3, Cs=0.15, tau0=0.6, 500 steps, checkpoints every 50",
                   "forward_ms": tf / args.steps, "backward_ms": tb / args.steps, "J": J, "grad": list(g),
                   "l2": "inputs larger than L2 (checkpoint segment states %.2f GB)" % (50 * 19 * N * 4 / 1e9)},
        "roofline": {"bound": "hbm", "kernel": "reverse sweep (k_chan_step recompute + k_chan_adj)",
                     "achieved": achieved, "peak": peak, "peak_kind": "%s hbm_gbs" % peak_kind, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "algorithmic_bytes_per_launch": bytes_bwd // S},
        "clocks": clk.summary(),
        "e2e": None,
        "gpu_launches": args.steps * chan_launches(S, 50),
    }
    print(json.dumps(line), flush=True)
    ch.close()


def chan_launches(S, K):
    """Kernel launches of one gradient evaluation of the differentiation form:
    the forward run (one launch for the initial collision, one per step; the
    boundary planes ride in the same launches), then per checkpoint segment
    the recompute (as the forward) and one adjoint launch per step, and the
    final sum of the gradient parts."""
    n = S + 1
    for seg in range(S // K, -1, -1):
        s0, s1 = seg * K, min(seg * K + K - 1, S)
        n += (s1 - s0 + 1 if s1 > s0 else 0) + (s1 - s0 + 1)
    return n + 1


def ctypes_stream(stream):
    return stream.cuda_stream


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "bf16", "fp16"], default="fp32")
    ap.add_argument("--e2e-steps", type=int, default=300)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-error-check", action="store_true",
                    help="skip the 64^3 velocity / force error against the FP64 oracle")
    ap.add_argument("--no-precision-forms", action="store_true",
                    help="skip the BF16 / FP16 storage lines of the FP32 run")
    ap.add_argument("--schedule", choices=["serial", "overlap"], default="serial",
                    help="order of the kernels inside a step (same results)")
    ap.add_argument("--mea", choices=["paper", "galilean"], default="paper",
                    help="momentum exchange on sphere links (Eqs. 25, 26, or its Galilean-invariant form)")
    ap.add_argument("--zieb", action="store_true",
                    help="ZIEB face on z = 0 onto a piston cylinder (A_p = nx ny, V_0 = 40 A_p, v_p = 0.005)")
    ap.add_argument("--friction", action="store_true",
                    help="tangential contact law (Eqs. 2, 3) with k_t = k_n / 2, mu = 0.3, e_t = 0.6 (slurry workload)")
    ap.add_argument("--momentum-correction", action="store_true",
                    help="covered / uncovered nodes exchange their momentum with the spheres (slurry workload)")
    ap.add_argument("--workload", choices=["slurry", "dense", "batched", "adjoint"], default="slurry",
                    help="slurry: the 256^3 box with 2000 spheres; dense: the same box at solid fraction 0.13 "
                         "(8136 spheres) with tangential friction; batched: the parameter-sweep batch; "
                         "adjoint: gradient evaluations of the differentiation form")
    ap.add_argument("--batch", type=int, default=64, help="instances of the batched workload")
    ap.add_argument("--box", type=int, default=256,
                    help="cubic box edge for profiling runs; sphere count scaled to keep the solid fraction")
    args = ap.parse_args()
    if args.box != 256:
        global BOX, NSPH
        BOX = (args.box,) * 3
        NSPH = int(round(2000 * (args.box / 256.0) ** 3))
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    if args.workload == "batched":
        run_batched(args, rank, world, local_rank)
    elif args.workload == "adjoint":
        run_adjoint(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
