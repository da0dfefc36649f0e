"""Throughput benchmark of the fused collide-stream step.

Workload (one "step" = one time step of the whole path over the lattice):
the 8192 x 8192 periodic square -- NH lambda = 1.5, mu = 0.75, c = 5,
omega = 2, a seeded 16-mode random velocity field (amplitude 0.05, seed 1),
F = I -- with FP32 populations and an FP64 displacement accumulator. Every
step is one launch of the fused kernel (pull streaming, collision, the
displacement quadrature).

Reported (one JSON line on rank 0):
  value     MLUPS with the state resident in HBM, timed with CUDA events on
            the library's stream over exactly --steps steps;
  e2e       MLUPS through the public C ABI with host buffers: the initial
            state copied in from pinned memory and initialized, the steps,
            and the final state and displacement copied out, all inside the
            timed region (with the time of each part; the median of five
            passes when --steps <= 200);
  roofline  the step kernel's algorithmic bytes per launch (224 B per node)
            over its mean launch duration in the timed region (CUDA events
            around the region, which holds only that kernel), against the
            measured HBM copy bandwidth;
  forms     the same step on the 4096 x 2048 clamped specimen (clamped left
            edge, traction-free top and bottom, traction ramp on the right)
            with FP32, FP64, BF16 and FP16 populations, the 8192^2 field with
            BF16 and FP16 populations, 256 specimens of uneven size and
            material in batched launches (FP32), and the adjoint's cost
            relative to the forward on the 1024^2 differentiation workload
            (FP32, 2000 steps);
  cpu_baseline  the FP64 CPU oracle on bounded samples: the headline field
            at 512 x 512 (the value), and the 64^2 shear wave, the 512^2
            field and the specimen scaled to 512 x 256 at one thread and at
            every host core.
--impl reference times the oracle alone as the reference arm.
Multi-GPU (torchrun): every rank runs an independent replica (weak scaling);
the path is not decomposed across GPUs.
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

METRIC = "MLUPS and achieved HBM GB/s vs peak (FP32/BF16 vs FP64), adjoint/forward step cost"
UNIT = "MLUPS"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=4000)
    p.add_argument("--warmup", type=int, default=50)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-forms", action="store_true", help="skip the side measurements (other storages, the clamped specimen, batch, adjoint)")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    p.add_argument("--form", choices=["batch", "adjoint", "bf16"], default=None,
                   help="run only this side measurement and print its JSON (profiling); not a bench line")
    p.add_argument("--form-steps", type=int, default=None, help="steps of the --form run")
    p.add_argument("--batch-members", type=int, default=None,
                   help="--form batch with only the first so many specimens (profiling)")
    p.add_argument("--size", type=int, default=8192,
                   help="side of the periodic square (profiling of smaller cases; the workload is 8192)")
    return p.parse_args()


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, None
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "ours":
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist.init_process_group("gloo")
    return rank, ws, dist


def max_over_ranks(x, dist, device):
    """The largest of every rank's x (x itself without a process group)."""
    if not dist:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.15)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def setup_ctx(lbm, w, storage, U0, u0):
    L = lbm.Lattice(w.nx, w.ny, dx=w.dx, c=w.c, omega=w.omega, storage=storage)
    lbm.lbm_set_material(L.ctx, lbm.LBM_LAW_NH, [w.lam, w.mu])
    lbm.lbm_set_body_force(L.ctx, *w.body_force)
    kinds = {"periodic": lbm.LBM_BC_PERIODIC, "velocity": lbm.LBM_BC_VELOCITY, "traction": lbm.LBM_BC_TRACTION}
    tfs = {"const": 0, "linear_ramp": 1, "sin2_ramp": 2, "sin_pulse": 3, "ricker": 4}
    for e, ed in enumerate(w.edges):
        lbm.lbm_set_boundary(L.ctx, e, kinds[ed.kind], ed.value, tfs[ed.timefn], ed.tparams, ed.profile)
    if U0 is not None:
        lbm.lbm_init(L.ctx, U0, u0, 2)
    return L


def timed_steps(lbm, torch, L, steps, warmup, dist, census_steps=10):
    """Device time (ms) of exactly `steps` steps, CUDA events on the stream
    the kernels run on, with nothing else in the timed region. A short
    untimed run with the library's per-launch events beforehand counts the
    launches per step and splits a step between the bulk and the edge
    kernel; the bulk kernel's average launch duration over the timed region
    is then the region's time per step times its share."""
    st = torch.cuda.current_stream()
    lbm.lbm_step(L.ctx, warmup)
    lbm.lbm_profile(L.ctx, True)
    lbm.lbm_step(L.ctx, census_steps)
    prof = lbm.lbm_profile_read(L.ctx)
    lbm.lbm_profile(L.ctx, False)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    lbm.lbm_step_async(L.ctx, steps)
    e1.record(st)
    e1.synchronize()
    lbm.lbm_sync(L.ctx)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    (ns, ts), (ne, te) = prof["step"], prof["edges"]
    share = ts / (ts + te) if ts + te > 0 else 1.0
    info = {"launches_per_step": (ns + ne) / census_steps, "step_kernel_ms": ms / steps * share,
            "edge_kernel_ms": te / max(ne, 1), "step_variant": lbm.lbm_step_variant(L.ctx)}
    return ms, info


def recorded_fp64_counts():
    """FP64 instructions per node-update of the FP64 step kernel (committed
    ncu record) and the FP64 instruction rate of the GPU derived from its
    nominal FP64 rate, or None when the kernel source changed since."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "fp64_step_kernel_counts.txt")
    try:
        kv = dict(ln.split("=", 1) for ln in open(path).read().split() if "=" in ln)
        h = hashlib.sha256()
        for f in ("lbm_step_kernels.cuh", "lbm_step_core.cuh", "lbm_device.cuh", "lbm_edges.cuh"):
            h.update(open(os.path.join(ROOT, "paper_2605_26677_gb300", "csrc", f), "rb").read())
        if kv.get("source_sha256") != h.hexdigest():
            return None
        return float(kv["fp64_inst_per_node"]), float(kv["fp64_inst_peak_per_s"])
    except Exception:
        return None


def _kernel_sources_sha():
    import hashlib

    h = hashlib.sha256()
    for f in ("lbm_step_kernels.cuh", "lbm_step_core.cuh", "lbm_device.cuh", "lbm_edges.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2605_26677_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def recorded_traffic(workload):
    """DRAM bytes per node of one step-kernel launch on `workload` from the
    committed ncu summary (profiles/step_kernel_traffic.txt, one line per
    workload), or None when there is none or the kernel source changed
    since the capture."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.txt")
    try:
        lines = open(path).read().splitlines()
    except Exception:
        return None
    sha = _kernel_sources_sha()
    for ln in lines:
        kv = dict(t.split("=", 1) for t in ln.split() if "=" in t)
        if kv.get("workload") == workload and kv.get("source_sha256") == sha:
            try:
                return float(kv["bytes_per_node"])
            except (KeyError, ValueError):
                return None
    return None


def e2e_run(lbm, torch, w, U0, steps, warmup):
    """MLUPS through the public C ABI with host buffers: lbm_init from a
    pinned host copy of U0 (zero initial displacement, passed as NULL),
    `steps` steps, then lbm_read_state (U) and lbm_read_displacement into
    pinned host arrays, all inside the timed region; every call returns
    only after its work is done. Short runs (steps <= 200, where the host
    copies weigh and host-side delays of tens of ms hit some passes) take
    the median of five such passes, longer ones one pass. Returns (MLUPS, h2d
    bytes, d2h bytes, the time of each part in ms of the pass taken, the
    total ms of every pass)."""
    U0p = torch.from_numpy(U0).pin_memory().numpy()
    uout = torch.empty((2, w.ny, w.nx), dtype=torch.float64).pin_memory().numpy()
    Uout = torch.empty((6, w.ny, w.nx), dtype=torch.float64).pin_memory().numpy()
    L = setup_ctx(lbm, w, lbm.LBM_STORE_F32, None, None)
    lbm.lbm_init(L.ctx, U0p, None, 2)  # warm-up of every call
    lbm.lbm_step(L.ctx, warmup)
    lbm.lbm_read_state(L.ctx, Uout, None, want_P=False)
    lbm.lbm_read_displacement(L.ctx, uout)
    passes = []
    for _ in range(5 if steps <= 200 else 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lbm.lbm_init(L.ctx, U0p, None, 2)
        t1 = time.perf_counter()
        lbm.lbm_step(L.ctx, steps)
        t2 = time.perf_counter()
        lbm.lbm_read_state(L.ctx, Uout, None, want_P=False)
        lbm.lbm_read_displacement(L.ctx, uout)
        t3 = time.perf_counter()
        passes.append((t3 - t0, {"init_ms": (t1 - t0) * 1e3, "steps_ms": (t2 - t1) * 1e3, "read_ms": (t3 - t2) * 1e3}))
    L.close()
    N = w.nx * w.ny
    total, parts = sorted(passes, key=lambda p: p[0])[len(passes) // 2]
    return (N * steps / total / 1e6, U0p.nbytes, Uout.nbytes + uout.nbytes, parts,
            [round(p[0] * 1e3, 1) for p in passes])


def run_ours(args, rank, ws, dist):
    import torch

    from paper_2605_26677_gb300 import build

    build.build()
    from paper_2605_26677_gb300 import lbm
    from synth import clamped_specimen, fourier_periodic

    dev = torch.cuda.current_device()
    peak, peak_kind = peaks()
    wp = fourier_periodic(n=args.size)
    Up, up = wp.fields()
    N = wp.nx * wp.ny
    L = setup_ctx(lbm, wp, lbm.LBM_STORE_F32, Up, up)
    with ClockSampler(dev) as clk:
        ms, tinfo = timed_steps(lbm, torch, L, args.steps, args.warmup, dist)
    clocks = clk.summary()
    bpn = lbm.lbm_bytes_per_node_update(L.ctx)
    L.close()
    ms_max = max_over_ranks(ms, dist, "cuda")
    value = N * args.steps * ws / (ms_max * 1e-3) / 1e6

    # roofline of the step kernel: its average launch duration over the timed region
    kern_ms = tinfo["step_kernel_ms"]
    achieved = bpn * N / (kern_ms * 1e-3) / 1e9
    traffic_bpn = recorded_traffic("fourier_periodic_%dx%d_f32" % (wp.nx, wp.ny))

    e2e, h2d, d2h, parts, e2e_passes = e2e_run(lbm, torch, wp, Up, args.steps, args.warmup)

    forms = {}
    if not args.no_forms:
        k = max(50, min(args.steps // 10, 400))
        for name, st in (("bf16", lbm.LBM_STORE_BF16), ("f16", lbm.LBM_STORE_F16)):
            L = setup_ctx(lbm, wp, st, Up, up)
            ms8, i8 = timed_steps(lbm, torch, L, k, 5, None)
            b8 = lbm.lbm_bytes_per_node_update(L.ctx)
            L.close()
            gbs = b8 * N / (i8["step_kernel_ms"] * 1e-3) / 1e9
            forms[name + "_periodic_8192x8192"] = {
                "value": N * k / (ms8 * 1e-3) / 1e6, "unit": UNIT, "steps": k, "kernel_GBs": gbs,
                "roofline_frac": gbs / peak, "bytes_per_node": b8, "step_variant": i8["step_variant"],
                "note": "16-mode random velocity field, NH lambda=1.5 mu=0.75, omega=2; populations stored as "
                        "%s offsets from the rest equilibrium, FP32 compute, FP64 u*" % name}
        del Up, up
        w = clamped_specimen()
        U0, u0 = w.fields()
        Nc = w.nx * w.ny
        L = setup_ctx(lbm, w, lbm.LBM_STORE_F32, U0, u0)
        msc, ic = timed_steps(lbm, torch, L, k, 5, None)
        bc = lbm.lbm_bytes_per_node_update(L.ctx)
        L.close()
        gbs = bc * Nc / (ic["step_kernel_ms"] * 1e-3) / 1e9
        tc = recorded_traffic("clamped_specimen_4096x2048_f32")
        forms["fp32_clamped_specimen_4096x2048"] = {
            "value": Nc * k / (msc * 1e-3) / 1e6, "unit": UNIT, "steps": k, "kernel_GBs": gbs,
            "roofline_frac": gbs / peak, "bytes_per_node": bc, "traffic_bytes_per_node": tc,
            "step_variant": ic["step_variant"],
            "note": "clamped left, traction-free top and bottom, traction ramp 0.3 mu on the right, NH lambda=2 "
                    "mu=1, body force 1e-6, c=5, omega=1.95; edge rules fused into the step kernel"}
        L = setup_ctx(lbm, w, lbm.LBM_STORE_F64, U0, u0)
        ms64, i64 = timed_steps(lbm, torch, L, k, 5, None)
        b64 = lbm.lbm_bytes_per_node_update(L.ctx)
        L.close()
        forms["fp64_clamped_specimen_4096x2048"] = {
            "value": Nc * k / (ms64 * 1e-3) / 1e6, "unit": UNIT, "steps": k,
            "kernel_GBs": b64 * Nc / (i64["step_kernel_ms"] * 1e-3) / 1e9, "bytes_per_node": b64,
            "step_variant": i64["step_variant"],
            "note": "FP64 populations (parity mode); FP64 ALU-bound on GB300"}
        fp64 = recorded_fp64_counts()
        if fp64 is not None:
            ach = fp64[0] * Nc / (i64["step_kernel_ms"] * 1e-3)
            forms["fp64_clamped_specimen_4096x2048"]["roofline"] = {
                "bound": "alu", "achieved": ach, "peak": fp64[1], "unit": "FP64 inst/s", "frac": ach / fp64[1],
                "fp64_inst_per_node": fp64[0],
                "peak_source": "derived: nominal 1.25 TFLOP/s FP64 = 2 FMA per SM per clock x 152 SMs x 2070 MHz; "
                               "every FP64 instruction (FMA, add, multiply) occupies the FP64 pipe alike"}
        for name, st in (("bf16", lbm.LBM_STORE_BF16), ("f16", lbm.LBM_STORE_F16)):
            L = setup_ctx(lbm, w, st, U0, u0)
            msh, ih = timed_steps(lbm, torch, L, k, 5, None)
            bh = lbm.lbm_bytes_per_node_update(L.ctx)
            L.close()
            gbs = bh * Nc / (ih["step_kernel_ms"] * 1e-3) / 1e9
            forms[name + "_clamped_specimen_4096x2048"] = {
                "value": Nc * k / (msh * 1e-3) / 1e6, "unit": UNIT, "steps": k, "kernel_GBs": gbs,
                "roofline_frac": gbs / peak, "bytes_per_node": bh, "step_variant": ih["step_variant"],
                "note": "populations stored as %s offsets from the rest equilibrium, FP32 compute, FP64 u*" % name}
        del U0, u0

        forms["batch_256_specimens_fp32"] = batch_form(lbm, torch, peak, k)
        forms["adjoint_1024x1024_fp32"] = adjoint_form(lbm, torch)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline()

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(wp, ws, bpn),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_source": peak_kind,
                     "frac_of_nominal_7900": round(achieved / 7900.0, 4),
                     "traffic": None if traffic_bpn is None else traffic_bpn * N,
                     "kernel": "k_step (fused pull-stream + collide + quadrature)",
                     "bytes_per_node_update": bpn, "launch_ms": kern_ms, "step_variant": tinfo["step_variant"],
                     "edge_kernel_ms": tinfo["edge_kernel_ms"],
                     "launch_ms_source": "CUDA events around the timed region / launches (no per-launch events in it)"},
        "e2e": {"value": round(e2e, 1), "unit": UNIT, "h2d_bytes_per_step": h2d / args.steps,
                "d2h_bytes_per_step": d2h / args.steps, "parts": parts, "passes_ms": e2e_passes,
                "note": "lbm_init from pinned host U0 (u0 = 0 passed as NULL), %d steps, lbm_read_state (U) and "
                        "lbm_read_displacement into pinned host arrays; %s" % (
                            args.steps, "median of %d passes" % len(e2e_passes) if len(e2e_passes) > 1 else "one pass")},
        "gpu_launches": int(round(tinfo["launches_per_step"] * args.steps)),
        "clocks": clocks,
        "forms": forms,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    return line


def workload_config(wp, ws, bpn):
    N = wp.nx * wp.ny
    return {"workload": "periodic square %dx%d, 16-mode random velocity field (amplitude 0.05, seed 1), NH "
                        "lambda=1.5 mu=0.75, c=5, omega=2, FP32 populations + FP64 displacement" % (wp.nx, wp.ny),
            "nx": wp.nx, "ny": wp.ny, "global_batch": N * ws, "parallelism": "replicas" if ws > 1 else "single",
            "l2": "inputs larger than L2 (%.1f GB moved per step)" % (bpn * N / 1e9)}


def batch_form(lbm, torch, peak, steps, graph_steps=20, members=None):
    """256 specimens of uneven size and material (FP32) advanced by the
    batched launches: tuned tiles replayed from a CUDA graph (the value), and
    beside it the same with direct launches and with the default tiles.
    members: only the first so many specimens (profiling of a smaller case)."""
    from synth.generators import specimen_batch

    ws = specimen_batch()
    if members:
        ws = ws[:members]
    kinds = {"velocity": lbm.LBM_BC_VELOCITY, "traction": lbm.LBM_BC_TRACTION}
    Ls = []
    for w in ws:
        L = lbm.Lattice(w.nx, w.ny, dx=w.dx, c=w.c, omega=w.omega, storage=lbm.LBM_STORE_F32)
        lbm.lbm_set_material(L.ctx, lbm.LBM_LAW_NH, [w.lam, w.mu])
        for e, E in enumerate(w.edges):
            lbm.lbm_set_boundary(L.ctx, e, kinds[E.kind], E.value)
        U0, u0 = w.fields()
        lbm.lbm_init(L.ctx, U0, u0, 2)
        Ls.append(L)
    nodes = sum(w.nx * w.ny for w in ws)
    bpn = lbm.lbm_bytes_per_node_update(Ls[0].ctx)
    b = lbm.lbm_batch_create([L.ctx for L in Ls])
    st = torch.cuda.current_stream()

    def run(gs):
        lbm.lbm_batch_step(b, 2 * graph_steps, gs)  # warm-up (and capture)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        lbm.lbm_batch_step(b, steps, gs)
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1)

    default_tiles = lbm.lbm_batch_get_tiles(b)
    ms_default = run(graph_steps)
    tiles, us = lbm.lbm_batch_tune(b, reps=10)
    orders = lbm.lbm_batch_get_task_orders(b)
    ms = run(graph_steps)
    ms_direct = run(0)
    info = lbm.lbm_batch_info(b)
    lbm.lbm_batch_destroy(b)
    for L in Ls:
        L.close()
    gbs = bpn * nodes * steps / (ms * 1e-3) / 1e9
    return {"value": nodes * steps / (ms * 1e-3) / 1e6, "unit": UNIT, "steps": steps, "kernel_GBs": gbs,
            "roofline_frac": gbs / peak, "bytes_per_node": bpn, "nodes": nodes,
            "launches_per_step": info["launches_per_step"], "graph_steps": graph_steps,
            "tiles": tiles, "task_orders_dynamic": orders, "default_tiles": default_tiles,
            "tune_us": [[round(x, 1) for x in row] for row in us.tolist()],
            "value_direct_launches": nodes * steps / (ms_direct * 1e-3) / 1e6,
            "value_default_tiles": nodes * steps / (ms_default * 1e-3) / 1e6,
            "note": "seed-2 specimens, N log-uniform 64^2..1024^2, aspect 1..4, NH mu U(0.2,2), lambda/mu "
                    "U(1,4), clamped left, other edges clamped or traction-free; GB/s over the whole step"}


def adjoint_form(lbm, torch, steps=2000, all_states=True):
    """Gradient of the right-edge sensor misfit with respect to mu(X) and v0
    on the 1024^2 differentiation workload (FP32, 2000 steps, sqrt(N)
    checkpoints): device time of the forward (with checkpoints and sensor
    reads) and of the backward (segment recomputation included), per step,
    and their ratio; also the ratio with every state kept (no recomputation)."""
    from synth.generators import adjoint_specimen

    w = adjoint_specimen(steps=steps)
    p = w.params
    U0, _ = w.fields()
    U0d = torch.from_numpy(U0).cuda()
    out = {}
    for name, K in (("sqrtN", 0), ("all_states", 1))[: 2 if all_states else 1]:
        L = lbm.Lattice(w.nx, w.ny, dx=w.dx, c=w.c, omega=w.omega, storage=lbm.LBM_STORE_F32)
        lbm.lbm_set_material_field(L.ctx, lbm.LBM_LAW_NH, p["mu"], p["lam_ratio"])
        kinds = {"velocity": lbm.LBM_BC_VELOCITY, "traction": lbm.LBM_BC_TRACTION}
        for e, E in enumerate(w.edges):
            lbm.lbm_set_boundary(L.ctx, e, kinds[E.kind], E.value)
        A = lbm.lbm_adjoint_create(L.ctx, steps, K)
        lbm.lbm_adjoint_set_loss(A, p["sensors"], p["records"], p["target"])
        gmu = torch.zeros((w.ny, w.nx), dtype=torch.float64, device="cuda")
        gv0 = torch.zeros((2, w.ny, w.nx), dtype=torch.float64, device="cuda")
        for _ in range(2):  # the first pass warms up
            loss = lbm.lbm_adjoint_forward(A, U0d)
            lbm.lbm_adjoint_backward(A, gmu, gv0)
        info = lbm.lbm_adjoint_info(A)
        lbm.lbm_adjoint_destroy(A)
        L.close()
        out[name] = {"checkpoint_every": info["checkpoint_every"], "stored_states": info["stored_states"],
                     "forward_ms_per_step": info["forward_ms"] / steps,
                     "backward_ms_per_step": info["backward_ms"] / steps,
                     "adjoint_over_forward": info["backward_ms"] / info["forward_ms"], "loss": loss}
    N = w.nx * w.ny
    r = out["sqrtN"]
    return {"value": r["adjoint_over_forward"], "unit": "backward time / forward time", "steps": steps,
            "forward_MLUPS": N / (r["forward_ms_per_step"] * 1e-3) / 1e6,
            "backward_MLUPS": N / (r["backward_ms_per_step"] * 1e-3) / 1e6, "checkpointing": out,
            "note": "1024^2 clamped-left specimen, mu = exp(0.3 GRF, corr 64), lambda = 2 mu, velocity pulse, "
                    "64 right-edge sensors recorded every 20 steps; backward includes segment recomputation"}


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_lattice(name):
    """An oracle lattice with the initial state of a bounded sample:
    'fourier512' the headline field (same 16 waves in normalised
    coordinates) on 512 x 512, 'shear64' the 64^2 shear wave, 'specimen'
    the clamped specimen scaled to 512 x 256."""
    from oracle import oracle as orc
    from synth import clamped_specimen, fourier_periodic, shear_wave_64

    w = {"fourier512": lambda: fourier_periodic(n=512), "shear64": shear_wave_64,
         "specimen": lambda: clamped_specimen(nx=512, ny=256)}[name]()
    U0, u0 = w.fields()
    O = orc.Lattice(w.nx, w.ny, w.dx, w.c, w.omega)
    O.set_law(orc.NH, [w.lam, w.mu])
    O.set_body_force(*w.body_force)
    kinds = {"periodic": orc.PERIODIC, "velocity": orc.VELOCITY, "traction": orc.TRACTION}
    tfs = {"const": 0, "linear_ramp": 1, "sin2_ramp": 2, "sin_pulse": 3, "ricker": 4}
    for e, ed in enumerate(w.edges):
        O.set_edge(e, kinds[ed.kind], ed.value, tfs[ed.timefn], ed.tparams, ed.profile)
    O.init(U0, u0, 2)
    return O, w.nx * w.ny, "%s %dx%d" % (w.name, w.nx, w.ny)


def _time_oracle(O, n, seconds, chunk):
    O.step(1)
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        O.step(chunk)
        steps += chunk
    dt = time.perf_counter() - t0
    return n * steps / dt / 1e6, steps, dt


def cpu_baseline(seconds=2.5):
    """The FP64 oracle (as it stands) on bounded samples at one thread and at
    every host core; the value is the headline field's 512^2 sample at every
    core. About 6 x `seconds` of CPU time."""
    from oracle import oracle as orc

    cores = _host_cores()
    runs = []
    value = None
    for name, chunk in (("fourier512", 1), ("shear64", 20), ("specimen", 2)):
        O, n, label = oracle_lattice(name)
        for threads in (1, cores):
            orc.set_threads(threads)
            v, steps, dt = _time_oracle(O, n, seconds, chunk)
            runs.append({"sample": label, "threads": threads, "MLUPS": round(v, 3), "steps": steps,
                         "seconds": round(dt, 2)})
            if name == "fourier512" and threads == cores:
                value = (v, steps, dt)
    orc.set_threads(cores)
    return {"value": round(value[0], 3), "unit": UNIT, "cores": cores, "nproc": os.cpu_count(), "kind": "oracle",
            "sample": "the headline field's 16 waves on a 512x512 periodic square, %d steps (%.1f s) on %d threads"
                      % (value[1], value[2], cores), "runs": runs}


def run_reference(args, rank, ws):
    """Reference arm: the FP64 CPU oracle, every step one step of the
    headline workload's 512 x 512 sample, on every host core."""
    if rank != 0:
        return None
    from oracle import oracle as orc
    from synth import fourier_periodic

    cores = _host_cores()
    orc.set_threads(cores)
    O, n, label = oracle_lattice("fourier512")
    O.step(max(args.warmup, 0))
    t0 = time.perf_counter()
    O.step(args.steps)
    dt = time.perf_counter() - t0
    v = n * args.steps / dt / 1e6
    wp = fourier_periodic()
    return {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(wp, ws, 224.0),
            "cpu_baseline": {"value": round(v, 3), "unit": UNIT, "cores": cores, "nproc": os.cpu_count(),
                             "kind": "oracle",
                             "sample": "each step one FP64 oracle step of the same 16-wave field on a 512x512 "
                                       "periodic square (%s), %d steps on %d threads" % (label, args.steps, cores)},
            "e2e": {"value": round(v, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, ws, dist = dist_setup(args)
    if args.form is not None:
        import torch

        from paper_2605_26677_gb300 import build

        build.build()
        from paper_2605_26677_gb300 import lbm

        if args.form == "batch":
            line = {"form": "batch", **batch_form(lbm, torch, peaks()[0], args.form_steps or 200,
                                                  members=args.batch_members)}
        elif args.form == "bf16":
            from synth import clamped_specimen

            w = clamped_specimen()
            U0, u0 = w.fields()
            L = setup_ctx(lbm, w, lbm.LBM_STORE_BF16, U0, u0)
            k = args.form_steps or 200
            ms, ti = timed_steps(lbm, torch, L, k, 5, None)
            L.close()
            line = {"form": "bf16", "value": w.nx * w.ny * k / (ms * 1e-3) / 1e6, "unit": UNIT, "steps": k,
                    "kernel_us": ti["step_kernel_ms"] * 1e3, "step_variant": ti["step_variant"]}
        else:
            line = {"form": "adjoint", **adjoint_form(lbm, torch, args.form_steps or 2000, all_states=False)}
    elif args.impl == "reference":
        line = run_reference(args, rank, ws)
    else:
        line = run_ours(args, rank, ws, dist)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
