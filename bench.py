"""Benchmark of the coalesced-ghost translation step (one JSON line on rank 0).

A step is one full translation step of the whole workload through the library: 27-cell
block union and slot indexing, work list, the sweep kernel(s) (fused Ghost Translation
tile kernel by default, or the 3-pass classical form), and the sparsity rule with FP64
mass accounting.  Default workload: the uniform-mesh configuration, 64^3 periodic
cells x 32^3 velocity cells (512 blocks of 4^3 per cell, 8.6e9 phase-space cells,
34 GB of float32 f per copy), dt = 0.05 with dx = 1.

Metric: phase-space cell updates per second (one update = one velocity cell of one
spatial cell advanced through the full x->y->z step), whole job.  The state (34 GB)
is far larger than L2 (129 MB), so no L2 flush is needed between steps.

--impl reference times the FP64 CPU oracle on the machine's host cores instead, on a
bounded window of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2504_21450_gb300 import inputs  # noqa: E402

METRIC = "phase-space cell updates/s (xyz)"
UNIT = "updates/s"
BYTES_PER_UPDATE = {"fused": 8.0, "3pass": 8.0}  # per launch, FP32 storage: read f once, write once
# bytes per stored value: 16-bit codes plus their chunk's FP32 scale (4 B per 16 values)
STORAGE_BYTES = {"f32": 4, "bf16": 2.25, "f16": 2.25}
KERNEL = {"fused": "k_gt3", "fused-rows": "k_fused", "3pass": "k_pass"}
KERNEL_OPT = {"default": 0, "batched": 1, "rows": 2}
LAUNCHES_PER_STEP = {"fused": 1, "3pass": 3}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def traffic_for(kernel: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the kernel
    source as it is now (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(f"{kernel}:{workload}")
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    src = os.path.join(ROOT, "paper_2504_21450_gb300", "csrc", rec["source"])
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    return rec["bytes_per_launch"] if h == rec.get("sha256_16") else None


def cpu_baseline(cfg, budget_s=20.0):
    """The FP64 oracle as it stands, on all host cores, on a 16^3 window of the workload
    (the full velocity mesh), repeated until about budget_s of CPU work."""
    import oracle
    size = (16, 16, 16)
    thr = inputs.threshold(cfg)
    init = inputs.generate(cfg, size=size, thr=thr)
    mesh = oracle.Mesh(n=size, nv=cfg.nv, vmin=cfg.vmin, dv=cfg.dv, dx=cfg.dx)
    blk = oracle.as_blocks(init.off, init.ids, init.vals.astype(np.float64))
    cores = oracle.max_threads()
    updates, t0, reps = 0, time.perf_counter(), 0
    while True:
        oracle.step(mesh, blk, cfg.dt, thr, "xyz", nthreads=cores)
        updates += blk.nblocks * 64
        reps += 1
        if time.perf_counter() - t0 >= budget_s * 0.5 or reps >= 20:
            break
    el = time.perf_counter() - t0
    # the same oracle on one core, on an 8^3-cell window (one step)
    small = (8, 8, 8)
    init1 = inputs.generate(cfg, size=small, thr=thr)
    mesh1 = oracle.Mesh(n=small, nv=cfg.nv, vmin=cfg.vmin, dv=cfg.dv, dx=cfg.dx)
    blk1 = oracle.as_blocks(init1.off, init1.ids, init1.vals.astype(np.float64))
    t1 = time.perf_counter()
    oracle.step(mesh1, blk1, cfg.dt, thr, "xyz", nthreads=1)
    single = blk1.nblocks * 64 / (time.perf_counter() - t1)
    return {"value": updates / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{reps} step(s) of a periodic 16^3-cell window x {cfg.nv[0]}^3 velocity "
                      f"cells ({blk.nblocks * 64:.3g} updates/step), FP64, OpenMP over block ids",
            "single_core": {"value": single, "unit": UNIT,
                            "sample": f"1 step of a periodic 8^3-cell window "
                                      f"({blk1.nblocks * 64:.3g} updates), FP64, one thread"}}


def aggregate(el_ms: float, updates: float, dist=None, device="cuda"):
    """Whole-job figures of the ranks: the slowest rank's time and the sum of the updates
    (each rank advances its own replica of the workload)."""
    import torch
    t = torch.tensor([el_ms, float(updates)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t[0:1], op=dist.ReduceOp.MAX)
        dist.all_reduce(t[1:2], op=dist.ReduceOp.SUM)
    return float(t[0]), float(t[1])


def workload_name(cfg) -> str:
    """The workload both arms report in config.workload."""
    return (f"{cfg.name}: {cfg.n[0]}x{cfg.n[1]}x{cfg.n[2]} periodic cells x "
            f"{cfg.nv[0]}x{cfg.nv[1]}x{cfg.nv[2]} velocity cells (4^3 blocks), "
            f"dt={cfg.dt}, rel. threshold {cfg.rel_threshold:g}")


def run_reference(args, cfg):
    """Reference arm: the FP64 oracle timed on the host cores, bounded window per step."""
    import oracle
    rank, world, _ = dist_env()
    if rank != 0:
        return
    thr = inputs.threshold(cfg)
    # size the window so that the whole run stays within a few minutes
    budget = 150.0 / max(1, args.steps + args.warmup)
    edge = 16 if budget >= 3.0 else (12 if budget >= 1.2 else 8)
    size = (edge, edge, edge)
    init = inputs.generate(cfg, size=size, thr=thr)
    mesh = oracle.Mesh(n=size, nv=cfg.nv, vmin=cfg.vmin, dv=cfg.dv, dx=cfg.dx)
    blk = oracle.as_blocks(init.off, init.ids, init.vals.astype(np.float64))
    cores = oracle.max_threads()
    for _ in range(args.warmup):
        blk = oracle.step(mesh, blk, cfg.dt, thr, "xyz", nthreads=cores)[0]
    updates = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        updates += blk.nblocks * 64
        blk = oracle.step(mesh, blk, cfg.dt, thr, "xyz", nthreads=cores)[0]
    el = time.perf_counter() - t0
    value = updates / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(cfg), "order": "xyz",
                   "sample": f"each step: a periodic {edge}^3-cell window of the workload "
                             f"({edge ** 3} cells, the full velocity mesh)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"periodic {edge}^3-cell window of the workload per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def state_bytes(cfg) -> float:
    """Rough float32 bytes of one copy of the initial state (for choosing where to stage)."""
    if cfg.rel_threshold <= 1e-12 or len(cfg.pops) == 1:
        return cfg.ncells * cfg.nb * 256.0
    return cfg.ncells * 900 * 256.0


def generate_host(cfg, device, slab=2):
    """Initial state staged in host memory: generated on the GPU slab by slab (two
    passes: counts, then values), so that the device never holds it besides the
    library's own copy."""
    import torch
    thr = inputs.threshold(cfg)
    nx, ny, nz = cfg.n
    plane = nx * ny
    counts = np.zeros(cfg.ncells, np.int64)
    for z0 in range(0, nz, slab):
        dz = min(slab, nz - z0)
        off, _, _, _ = inputs.generate_torch(cfg, device, origin=(0, 0, z0), size=(nx, ny, dz), thr=thr)
        counts[z0 * plane:(z0 + dz) * plane] = torch.diff(off).cpu().numpy()
        del off
        torch.cuda.empty_cache()
    off = np.zeros(cfg.ncells + 1, np.int64)
    np.cumsum(counts, out=off[1:])
    ids_h = np.empty(int(off[-1]), np.uint16)
    vals_h = np.empty((int(off[-1]), 64), np.float32)
    for z0 in range(0, nz, slab):
        dz = min(slab, nz - z0)
        _, ids, vals, _ = inputs.generate_torch(cfg, device, origin=(0, 0, z0), size=(nx, ny, dz), thr=thr)
        a, b = off[z0 * plane], off[(z0 + dz) * plane]
        ids_h[a:b] = ids.cpu().numpy().astype(np.uint16)
        vals_h[a:b] = vals.cpu().numpy()
        del ids, vals
        torch.cuda.empty_cache()
    return off, ids_h, vals_h, thr


PRESIZE_EDGE = 8       # cost-model tiles: 8^3 cells
PRESIZE_MARGIN = 0.05  # capacity = (1 + margin) x the summed tile predictions


def train_cost_model(horizon, local):
    """The pre-sizing model, trained with seed 0 on solver traces of the uniform and
    shock workloads (windows: their full sizes do not fit beside the timed state)."""
    import torch
    from paper_2504_21450_gb300 import costmodel, vlasov
    X_l, T_l, info = [], [], []
    for name, size, nsteps in (("uniform", (32, 32, 16), horizon + 8), ("shock", (128, 32, 16), horizon + 40)):
        cfg = inputs.CONFIGS[name]
        off, ids, vals, thr = inputs.generate_torch(cfg, f"cuda:{local}", size=size)
        g = vlasov.Grid(size, cfg.nv, cfg.vmin, cfg.dv, cfg.dx, threshold=thr, device=local)
        g.set_blocks(off, ids, vals)
        del off, ids, vals
        tr = costmodel.record_run(g, cfg.dt, nsteps, edge=PRESIZE_EDGE)
        X, T = tr.dataset(horizon)
        g.close()
        del tr
        X_l.append(X)
        T_l.append(T)
        info.append(f"{name} {size[0]}x{size[1]}x{size[2]} cells, {nsteps} steps")
        torch.cuda.empty_cache()
    X, T = torch.cat(X_l), torch.cat(T_l)
    model = costmodel.CostModel(seed=0)
    epochs = 3000
    t0 = time.perf_counter()
    losses = model.train(X, T, epochs, lr=3e-3)
    return model, {"traces": "; ".join(info), "samples": int(X.shape[0]), "epochs": epochs,
                   "loss_first": losses[0], "loss_last": losses[-1],
                   "train_s": round(time.perf_counter() - t0, 3)}


def run_ours(args, cfg):
    import torch
    from paper_2504_21450_gb300 import vlasov

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        quiet_nccl()
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    form = {"fused": vlasov.VL_FORM_FUSED, "3pass": vlasov.VL_FORM_3PASS,
            "auto": vlasov.VL_FORM_AUTO}[args.form]
    storage = {"f32": vlasov.VL_STORE_F32, "bf16": vlasov.VL_STORE_BF16_SCALED,
               "f16": vlasov.VL_STORE_F16_SCALED}[args.storage]
    kern = KERNEL_OPT[args.kernel]

    model, train_info = None, None
    if args.presize == "mlp":
        model, train_info = train_cost_model(args.chunk or args.steps, local)
    host = None
    e2e_note = None
    big = state_bytes(cfg) > 40e9
    if big:
        off, ids, vals, thr = generate_host(cfg, f"cuda:{local}")
        g = vlasov.Grid(cfg.n, cfg.nv, cfg.vmin, cfg.dv, cfg.dx, threshold=thr, storage=storage,
                        device=local)
        g.set_blocks(off, ids, vals)
        del off, ids, vals
        e2e_note = "not measured: the state is staged in pageable host memory for this workload"
    else:
        off, ids, vals, thr = inputs.generate_torch(cfg, f"cuda:{local}")
        g = vlasov.Grid(cfg.n, cfg.nv, cfg.vmin, cfg.dv, cfg.dx, threshold=thr, storage=storage,
                        device=local)
        g.set_blocks(off, ids, vals)
        if args.e2e:
            host = (off.cpu().pin_memory(), ids.to(torch.int16).cpu().pin_memory(), vals.cpu().pin_memory())
        del off, ids, vals
    torch.cuda.empty_cache()

    chunk = args.chunk or args.steps
    cap = int(g.block_count() * 1.08) if (args.graph and args.presize == "fixed") else 0
    step_calls = [chunk] * (args.steps // chunk) + ([args.steps % chunk] if args.steps % chunk else []) \
        if args.graph else [1] * args.steps
    caps = []   # capacity asked for per captured call
    held = []   # blocks the pools held after it
    unions = []  # union blocks of its last step
    cap_ms = []  # host time of the capacity decision (features + model) per call

    def capacity_for_call():
        """Pool capacity of the next captured call: fixed (1.08 x the blocks present),
        exact (0: the library's default, the last union's exact count + 25%), or the
        learned model's prediction for the next `chunk` steps."""
        t0 = time.perf_counter()
        if args.presize == "mlp":
            c = model.capacity(g.tile_features(PRESIZE_EDGE)[0], PRESIZE_MARGIN)
        else:
            c = cap
        cap_ms.append(round((time.perf_counter() - t0) * 1e3, 3))
        caps.append(c)
        return c

    tune = None
    if form == vlasov.VL_FORM_AUTO:
        # the autotuner's probe steps (one warm-up and one timed step per candidate),
        # before and apart from the warm-up below
        g.translate(cfg.dt, args.order, 8, form, ghost=args.ghost, kernel=kern)
        st = g.stats()
        # per candidate: the sweep kernels' ms in its timed probe step (the library compares
        # them per updated cell), 0 = not applicable, -1 = ruled out by the prior
        tune = {"probe_sweep_ms": dict(zip(["fused_batched", "fused_rows16", "fused_rows8", "3pass"],
                                        [round(x, 3) for x in st.tune_ms])),
                "chosen": {vlasov.VL_FORM_FUSED: "fused", vlasov.VL_FORM_3PASS: "3pass"}.get(st.form_used),
                "kernel": {1: "batched", 2: "rows"}.get(int(st.kernel_used)),
                "tile_rows": int(st.tile_rows_used)}
    if args.graph:
        # warm-up with the same step count, so that the timed call replays a cached graph
        g.translate(cfg.dt, args.order, chunk, form, graph=True, capacity=capacity_for_call(),
                    ghost=args.ghost, kernel=kern)
        if args.presize == "fixed":
            cap = max(cap, g.stats().capacity)
        for _ in range(max(0, args.warmup - 1)):
            g.translate(cfg.dt, args.order, 1, form, ghost=args.ghost, kernel=kern)
        caps.clear()
        cap_ms.clear()
    else:
        for _ in range(args.warmup):
            g.translate(cfg.dt, args.order, 1, form, ghost=args.ghost, kernel=kern)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    updates = 0
    sweep_ms = 0.0
    launches = 0
    regrows = 0
    replays = 0
    phases = {"index_ms": 0.0, "sweep_ms": 0.0, "prune_ms": 0.0, "tail_ms": 0.0}
    stats = None
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for n in step_calls:
            g.translate(cfg.dt, args.order, n, form, graph=args.graph,
                        capacity=capacity_for_call() if args.graph else 0, ghost=args.ghost, kernel=kern)
            s = g.stats()
            updates += s.updates
            sweep_ms += s.sweep_ms
            launches += s.launches
            regrows += s.capacity_regrows
            replays += s.graph_replays
            held.append(int(s.capacity))
            unions.append(int(s.union_blocks))
            stats = s
            for k in phases:
                phases[k] += getattr(s, k)
        ev1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    el_ms, total_updates = aggregate(ev0.elapsed_time(ev1), updates, dist, "cuda")
    value = total_updates / (el_ms / 1e3)

    # end to end through the public API with host buffers: each step uploads the state
    # from page-locked host memory (vl_set_blocks), advances it (vl_translate) and reads
    # the advanced state back into the same host buffers (vl_get_blocks), so successive
    # steps form a host-driven time loop
    e2e = None
    if args.e2e and host is not None:
        h_off, h_ids, h_vals = host
        cap = int(h_vals.shape[0])
        nb = cap
        e_steps = max(1, min(args.steps, 3))
        e_updates = 0
        h2d = d2h = 0
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e_steps):
            vlasov.vl_set_blocks(g.handle, nb, h_off.data_ptr(), h_ids.data_ptr(), h_vals.data_ptr(), 0)
            h2d += h_off.numel() * 8 + nb * 2 + nb * 256
            e_updates += nb * 64
            g.translate(cfg.dt, args.order, 1, form, ghost=args.ghost, kernel=kern)
            vlasov.vl_get_blocks(g.handle, cap, h_off.data_ptr(), h_ids.data_ptr(), h_vals.data_ptr(), 0)
            nb = int(h_off[-1])
            d2h += h_off.numel() * 8 + nb * 2 + nb * 256
        torch.cuda.synchronize()
        e_el = time.perf_counter() - t0
        if dist:
            te = torch.tensor([e_el], dtype=torch.float64, device="cuda")
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
            e_el = float(te[0])
        e2e = {"value": e_updates * world / e_el, "unit": UNIT, "h2d_bytes_per_step": int(h2d // e_steps),
               "d2h_bytes_per_step": int(d2h // e_steps), "steps": e_steps,
               "transfer": "page-locked host buffers read and written in place by the scatter/gather kernels"}
    elif e2e_note:
        e2e = {"value": None, "unit": UNIT, "note": e2e_note}

    peak, peak_kind = measured_peak_hbm()
    form_used = {vlasov.VL_FORM_FUSED: "fused", vlasov.VL_FORM_3PASS: "3pass"}.get(stats.form_used, "fused")
    kernel_key = "fused-rows" if (form_used == "fused" and int(stats.kernel_used) == 2) else form_used
    launches_sweep = LAUNCHES_PER_STEP[form_used] * args.steps
    per_launch_updates = updates / args.steps  # every sweep launch touches every update once
    avg_launch_s = (sweep_ms / launches_sweep) / 1e3 if sweep_ms > 0 else float("nan")
    bytes_per_update = BYTES_PER_UPDATE[form_used] * STORAGE_BYTES[args.storage] / 4
    achieved = bytes_per_update * per_launch_updates / avg_launch_s / 1e9
    workload = cfg.name if args.storage == "f32" else f"{cfg.name}-{args.storage}"
    if args.ghost != 3:
        workload += f"-gt{args.ghost}"
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": peak_kind,
                "kernel": KERNEL[kernel_key],
                "traffic": traffic_for(KERNEL[kernel_key], workload),
                "algorithmic_bytes_per_launch": bytes_per_update * per_launch_updates,
                "avg_launch_ms": avg_launch_s * 1e3}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(cfg),
                   "form": form_used, "storage": args.storage, "order": args.order, "parallelism": f"replicas{world}",
                   "ghost": args.ghost,
                   "kernel": KERNEL[kernel_key],
                   "graph": bool(args.graph), "capacity_regrows": regrows,
                   "l2": f"state ({updates / args.steps * STORAGE_BYTES[args.storage] / 1e9:.1f} GB per copy) larger than L2; no flush",
                   "blocks_per_step": updates / args.steps / 64},
        "roofline": roofline,
        **({"autotune": tune} if tune else {}),
        **({"presize": {"mode": args.presize, "chunk": chunk, "capacity_blocks": caps,
                        "held_blocks": held, "union_blocks_at_end": unions, "decision_ms": cap_ms,
                        "blocks_present_last": int(stats.blocks), "union_blocks_last": int(stats.union_blocks),
                        "capacity_regrows": regrows, "graph_replays": replays, "train": train_info}}
           if args.graph else {}),
        "phases_ms_per_step": {k: v / args.steps for k, v in phases.items()},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "e2e": e2e,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg)
    g.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def quiet_nccl():
    """Rank 0 prints one JSON line on stdout: keep NCCL's version banner off it unless the
    user asked for NCCL's own logging."""
    if os.environ.get("NCCL_DEBUG", "VERSION").upper() == "VERSION":
        os.environ["NCCL_DEBUG"] = "WARN"


def run_slab(args, cfg):
    """N > 1 GPUs: the spatial domain split into z-slabs over the ranks (weak scaling: each
    rank owns the per-GPU workload's nz planes of a global grid of nz * N planes).  A timed
    step is one coalesced ghost update (3 planes from each neighbour over NCCL, Section 3)
    followed by one translation step of each rank's local grid (its planes plus 3 ghost
    planes on either side)."""
    import dataclasses

    import torch
    import torch.distributed as dist
    from paper_2504_21450_gb300 import slab, vlasov

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if "MASTER_ADDR" not in os.environ:  # one rank started without a launcher
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=os.environ.get("MASTER_PORT", "29517"),
                          RANK="0", WORLD_SIZE="1")
    quiet_nccl()
    dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    form = {"fused": vlasov.VL_FORM_FUSED, "3pass": vlasov.VL_FORM_3PASS,
            "auto": vlasov.VL_FORM_AUTO}[args.form]
    storage = {"f32": vlasov.VL_STORE_F32, "bf16": vlasov.VL_STORE_BF16_SCALED,
               "f16": vlasov.VL_STORE_F16_SCALED}[args.storage]
    kern = KERNEL_OPT[args.kernel]
    gcfg = dataclasses.replace(cfg, n=(cfg.n[0], cfg.n[1], cfg.n[2] * world), name=f"{cfg.name}-slabs{world}")
    sl = slab.slabs(gcfg.n[2], world)[rank]
    ln = (cfg.n[0], cfg.n[1], sl.local_nz)
    off, ids, vals, thr = inputs.generate_torch(gcfg, f"cuda:{local}", origin=(0, 0, sl.origin_z), size=ln)
    g = vlasov.Grid(ln, cfg.nv, cfg.vmin, cfg.dv, cfg.dx, threshold=thr, storage=storage, device=local)
    g.set_blocks(off, ids, vals)
    del off, ids, vals
    torch.cuda.empty_cache()
    planes = slab.GridPlanes(g)
    ex = slab.TorchExchange(sl, dist, f"cuda:{local}")
    owned_window = ((0, 0, slab.GHOST), (ln[0], ln[1], sl.owned))

    def step():
        slab.ghost_update(sl, planes.get, planes.set, ex)
        g.translate(cfg.dt, args.order, 1, form, ghost=args.ghost, kernel=kern)

    for _ in range(max(args.warmup, 8 if form == vlasov.VL_FORM_AUTO else 0)):
        step()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dist.barrier()
    torch.cuda.synchronize()
    updates = 0
    sweep_ms = 0.0
    launches = 0
    local_updates = 0
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            updates += vlasov.vl_get_block_count_window(g.handle, *owned_window) * 64
            step()
            s = g.stats()
            sweep_ms += s.sweep_ms
            launches += s.launches
            local_updates += s.updates
        ev1.record(stream)
        torch.cuda.synchronize()
    dist.barrier()
    el_ms, total_updates = aggregate(ev0.elapsed_time(ev1), updates, dist, "cuda")
    peak, peak_kind = measured_peak_hbm()
    form_used = {vlasov.VL_FORM_FUSED: "fused", vlasov.VL_FORM_3PASS: "3pass"}.get(s.form_used, "fused")
    kernel_key = "fused-rows" if (form_used == "fused" and int(s.kernel_used) == 2) else form_used
    launches_sweep = LAUNCHES_PER_STEP[form_used] * args.steps
    avg_launch_s = (sweep_ms / launches_sweep) / 1e3 if sweep_ms > 0 else float("nan")
    bytes_per_update = BYTES_PER_UPDATE[form_used] * STORAGE_BYTES[args.storage] / 4
    achieved = bytes_per_update * (local_updates / args.steps) / avg_launch_s / 1e9
    line = {
        "metric": METRIC, "value": total_updates / (el_ms / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": workload_name(gcfg), "form": form_used, "kernel": KERNEL[kernel_key],
                   "storage": args.storage, "order": args.order, "parallelism": f"slabs{world}",
                   "decomposition": {"axis": "z", "owned_planes_rank0": sl.owned,
                                     "ghost_planes": 2 * slab.GHOST, "exchange": "NCCL send/recv, once per step"},
                   "l2": "state larger than L2; no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind, "kernel": KERNEL[kernel_key],
                     "traffic": None, "avg_launch_ms": avg_launch_s * 1e3,
                     "note": "local grid (owned and ghost planes) per launch"},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "e2e": {"value": None, "unit": UNIT, "note": "not measured in the slab decomposition"},
    }
    g.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="auto", choices=["fused", "3pass", "auto"],
                    help="auto: the library's autotuner times the fused form (16- and 8-row "
                         "tiles) and the 3-pass form on this workload and keeps the fastest")
    ap.add_argument("--kernel", default="default", choices=sorted(KERNEL_OPT),
                    help="fused form: plane-batched kernel, row-segment kernel, or the default choice")
    ap.add_argument("--ghost", type=int, default=3, choices=[1, 2, 3],
                    help="GT-k ghost depth of the fused form: 3 is exact, 1 and 2 are the reduced "
                         "(approximate) GT1 and GT2 of Section 3.2")
    ap.add_argument("--graph", action="store_true",
                    help="run the timed steps as one captured CUDA graph (no host sync per step)")
    ap.add_argument("--config", default="uniform", choices=sorted(inputs.CONFIGS))
    ap.add_argument("--order", default="xyz")
    ap.add_argument("--storage", default="f32", choices=sorted(STORAGE_BYTES),
                    help="storage of f (arithmetic is FP32 in every case)")
    ap.add_argument("--grid", type=int, nargs=3, default=None,
                    help="override the spatial extent (smaller cases for profiling)")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--presize", default="fixed", choices=["fixed", "exact", "mlp"],
                    help="pool capacity of captured calls: 1.08 x blocks present, the last exact "
                         "union count + 25%%, or the learned cost model")
    ap.add_argument("--chunk", type=int, default=0, help="steps per captured call (default: all)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--decomp", default="auto", choices=["auto", "slabs", "replicas"],
                    help="auto: z-slabs with one ghost update per step when N > 1, else one "
                         "domain; slabs: the slab path also for one rank (its own planes are its "
                         "ghosts); replicas: N independent copies of the workload")
    args = ap.parse_args()
    if args.ghost != 3 and args.form != "fused":
        ap.error("--ghost 1 or 2 needs --form fused (GT1/GT2 exist in the fused form only)")
    cfg = inputs.CONFIGS[args.config]
    if args.grid:
        import dataclasses
        cfg = dataclasses.replace(cfg, n=tuple(args.grid), name=f"{cfg.name}-{'x'.join(map(str, args.grid))}")
    if args.impl == "reference":
        run_reference(args, cfg)
    elif args.decomp == "slabs" or (args.decomp == "auto" and dist_env()[1] > 1):
        run_slab(args, cfg)
    else:
        run_ours(args, cfg)


if __name__ == "__main__":
    main()
