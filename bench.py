"""Throughput of the fused two-component Shan-Chen step on GB300.

Workload: D3Q19, 128^3 periodic, symmetric interactions (G_AA = G_BB = 0),
spherical A-rich droplet of radius 24 (tanh profile, +/-1e-3 seeded noise),
FP32 deviation storage.  One benchmark step = 2048 fused time steps (the
convergence-check interval delta t = 2^11 of the paper's section 4) followed by
the radial pressure-tensor profile (0.5 lattice-unit bins), the bulk pressure
at the centre node and at the far corner, and the sigma[R] minimum -- every
stage of the hot path, all in this library's kernels.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on the same workload (a bounded sample per step) on the host cores.
"""
from __future__ import annotations

import argparse
import math
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % of HBM roofline (D3Q19 2-comp); FP32 vs FP16-storage at stated σ error"
SHAPE = (128, 128, 128)
RADIUS = 24.0
G_CROSS = 3.6  # G c_s^2 = 1.2: the largest tested coupling that is stable in three dimensions at tau = 1
INNER = 2048  # time steps per benchmark step (section 4: delta t = 2^11); --inner overrides for profiling
# algorithmic bytes per site update: 2 comps x 19 pops x (read + write) x storage bytes
BYTES_PER_SITE = {"f32": 304, "f16": 152, "bf16": 152, "f64": 608}
# bytes the 16-bit forms move in addition: the FP32 reference-density pair of each site (read + write)
LOCAL_REF_BYTES = {"f16": 16, "bf16": 16}
# DRAM bytes (read + write) of one step launch on this workload, from an ncu capture of the
# launch; reported only while the kernel sources still hash to the captured version.
KERNEL_SOURCES = ["paper_2112_02574_gb300/csrc/sc_common.cuh", "paper_2112_02574_gb300/csrc/sc_step_kernel.cuh",
                  "paper_2112_02574_gb300/csrc/sc_step_staged.cuh"]
# DRAM bytes per step launch (dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture), keyed by the
# kernel sources' hash, the storage and the launch (tile_y, stages, blocks_per_sm, blocks); a change to any of
# them drops the figure (reported as null) until it is measured again
MEASURED_TRAFFIC = {
    ("386a06ff5cd3c81c", "f32", "v2 ty8 ns1 mb3 g456"): 605.263104e6,
    ("386a06ff5cd3c81c", "f16", "v2 ty8 ns1 mb3 g456"): 312.314880e6,
}


def workload_config(storage: str):
    return {
        "workload": f"D3Q19 two-component Shan-Chen, 128^3 periodic droplet R=24, symmetric G (G c_s^2 = 1.2), "
                    f"tau = 1, {storage.upper()} deviation storage; {INNER} fused steps + radial P-tensor "
                    f"profile + sigma[R] minimum per step",
        "lattice": "D3Q19",
        "sites": SHAPE[0] * SHAPE[1] * SHAPE[2],
        "time_steps_per_step": INNER,
        "storage": storage,
        "l2": "inputs larger than L2 (two population buffers of 2*19*128^3*4 B = 319 MB each)",
    }


def fields():
    import sc_synth

    return sc_synth.droplet(SHAPE[::-1], (64, 64, 64), RADIUS, n_in=0.95, n_out=0.05, amplitude=1e-3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
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
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_key(cfg) -> str:
    return "v{variant} ty{tile_y} ns{stages} mb{blocks_per_sm} g{blocks}".format(**cfg)


def kernel_hash() -> str:
    import hashlib

    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_baseline(budget_s: float = 12.0, shape=(64, 64, 64)):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample:
    the same droplet workload scaled to 64^3 (R = 12), steps until the budget."""
    import oracle
    import sc_synth

    op = oracle.Params(shape=shape, lattice=oracle.D3Q19, psi_self=oracle.PSI_EXP, G=G_CROSS)
    nA, nB = sc_synth.droplet(shape[::-1], tuple(s // 2 for s in shape), RADIUS * shape[0] / SHAPE[0])
    f = oracle.init(op, nA, nB)
    oracle.step(op, f, 1)  # warm
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        f = oracle.step(op, f, 2)
        n += 2
    dt = time.perf_counter() - t0
    sites = shape[0] * shape[1] * shape[2]
    return {"value": sites * n / dt / 1e6, "unit": "MLUPS", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{n} FP64 oracle time steps of the same droplet workload at {shape[0]}^3 (R = "
                      f"{RADIUS * shape[0] / SHAPE[0]:g}), {dt:.1f} s"}


PRECISION_STEPS = 4096  # two convergence-check intervals of the bench workload


def surface_of_tension_after(B, storage_code, steps, dev, stream):
    """(dP, R_s, sigma_s) of the bench droplet after `steps` fused steps in one storage mode."""
    params = B.make_params(SHAPE, lattice=B.SC_D3Q19, stencil=B.SC_FORCE_E4, psi_self=B.SC_PSI_EXP,
                           storage=storage_code, tau=(1.0, 1.0), G=G_CROSS, G_self=(0.0, 0.0))
    nA0, nB0 = fields()
    import torch

    with torch.cuda.stream(stream):
        sim = B.Simulation(params, nA0, nB0, device=dev, stream=stream)
        sim.step(steps)
        _, out = B.surface_of_tension(sim, (64.0, 64.0, 64.0), 0.5, nbins=128)
        B.sc_sync(sim.ctx)
        o = out.cpu().numpy()
    return {"dP": float(o[0]), "Rs": float(o[2]), "sigma_s": float(o[3])}


def precision_block(B, storages, dev, stream):
    """Errors of dP, R_s and sigma_s against the FP64-storage path (itself within 1e-13 per step of the
    FP64 CPU oracle) after PRECISION_STEPS steps of the bench workload."""
    ref = surface_of_tension_after(B, B.SC_STORE_F64, PRECISION_STEPS, dev, stream)
    out = {"steps": PRECISION_STEPS, "reference": "FP64-storage GPU path", "reference_values": ref}
    codes = {"f32": B.SC_STORE_F32, "f16": B.SC_STORE_F16, "bf16": B.SC_STORE_BF16}
    for st in storages:
        got = surface_of_tension_after(B, codes[st], PRECISION_STEPS, dev, stream)
        out[st] = {k + "_rel_err": abs(got[k] - ref[k]) / abs(ref[k]) for k in ("dP", "Rs", "sigma_s")}
    return out


def run_reference(args, rank, world):
    """The oracle arm: rank 0 only, FP64 on the host cores, same metric and unit."""
    if rank != 0:
        return
    import oracle
    import oracle.sigma as SG
    import sc_synth

    shape = SHAPE
    op = oracle.Params(shape=shape, lattice=oracle.D3Q19, psi_self=oracle.PSI_EXP, G=G_CROSS)
    nA, nB = fields()
    f = oracle.init(op, nA, nB)
    sample = 2  # oracle time steps per benchmark step (bounded sample of the 2048)
    sites = shape[0] * shape[1] * shape[2]

    def one():
        nonlocal f
        f = oracle.step(op, f, sample)
        a, b, _ = oracle.moments(op, f, with_u=False)
        rows = oracle.profile(op, a, b, oracle.RADIAL, (64, 64, 64), 0.5, 128)
        r, _, pt, _, _ = SG.clean_profile(rows)
        c = 64 + 128 * (64 + 128 * 64)
        SG.surface_of_tension(r, pt, oracle.bulk_pressure(op, a[c], b[c]), oracle.bulk_pressure(op, a[-1], b[-1]))

    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    dt = time.perf_counter() - t0
    value = sites * sample * args.steps / dt / 1e6
    line = {"metric": METRIC, "value": value, "unit": "MLUPS", "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args.storage),
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": oracle.threads(), "kind": "oracle",
                             "sample": f"each benchmark step a bounded sample of the workload: {sample} of its "
                                       f"{INNER} time steps at 128^3 (FP64 oracle), then the radial profile "
                                       f"and the sigma[R] minimum"},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(ms: float, device) -> float:
    """The slowest rank's time (ms): the whole job's time of a replica run."""
    import torch
    import torch.distributed as tdist

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(sites: int, steps_per_rank: int, world: int, ms: float) -> float:
    """Site updates of all ranks (each rank a full replica) / the job's time."""
    return sites * steps_per_rank * world / (ms * 1e-3) / 1e6


def run_gpu(args, rank, world, local_rank):
    import torch

    from paper_2112_02574_gb300 import binding as B

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    storage = args.storage
    st = {"f32": B.SC_STORE_F32, "f16": B.SC_STORE_F16, "bf16": B.SC_STORE_BF16, "f64": B.SC_STORE_F64}[storage]
    params = B.make_params(SHAPE, lattice=B.SC_D3Q19, stencil=B.SC_FORCE_E4, psi_self=B.SC_PSI_EXP, storage=st,
                           tau=(1.0, 1.0), G=G_CROSS, G_self=(0.0, 0.0), tile_y=args.tile_y, tile_z=args.tile_z,
                           variant=args.variant, stages=args.stages, blocks_per_sm=args.blocks_per_sm)
    nA0, nB0 = fields()
    stream = torch.cuda.Stream(dev)
    sites = SHAPE[0] * SHAPE[1] * SHAPE[2]
    with torch.cuda.stream(stream):
        sim = B.Simulation(params, nA0, nB0, device=dev, stream=stream)
        step_cfg = sim.step_config
        rows = torch.empty(128 * 6, dtype=torch.float64, device=dev)
        pio = torch.empty(2, dtype=torch.float64, device=dev)
        sig = torch.empty(8, dtype=torch.float64, device=dev)
    centre = (64.0, 64.0, 64.0)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    step_ms = []

    def one(record=False):
        if record:
            ev[0].record(stream)
        B.sc_step(sim.ctx, INNER)
        if record:
            ev[1].record(stream)
        B.sc_pressure_profile(sim.ctx, B.SC_PROFILE_RADIAL, centre, 0.5, 128, rows)
        B.sc_bulk_pressure_at(sim.ctx, (64, 64, 64), pio[0:1])
        B.sc_bulk_pressure_at(sim.ctx, (127, 127, 127), pio[1:2])
        B.sc_sigma_minimum(rows.view(128, 6), pio, 3, 0.01, 64.0, 0.01, sig, stream)
        if record:
            ev[1].synchronize()
            step_ms.append(ev[0].elapsed_time(ev[1]))

    for _ in range(args.warmup):
        one()
    B.sc_sync(sim.ctx)
    launches0 = sim.launches
    dist = world > 1
    if dist:
        import torch.distributed as tdist
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        if dist:
            tdist.barrier()
        torch.cuda.synchronize(dev)
        start.record(stream)
        for _ in range(args.steps):
            one(record=args.kernel_events)
        stop.record(stream)
        torch.cuda.synchronize(dev)
        if dist:
            tdist.barrier()
    B.sc_sync(sim.ctx)
    ms = start.elapsed_time(stop)
    if dist:
        ms = max_over_ranks(ms, dev)
    step_launches = sim.launches - launches0
    # per bench step: INNER fused steps + fields + profile partials + profile finalise + 2 bulk + sigma
    launches = step_launches + args.steps * 6

    # kernel-only timing of the fused step (events around the INNER launches, separate pass)
    if not step_ms:
        for _ in range(3):
            one(record=True)
    kern_ms = statistics.median(step_ms) / INNER
    alg_bytes = BYTES_PER_SITE[storage] * sites
    peak, peak_kind = measured_peak()
    achieved = alg_bytes / (kern_ms * 1e-3) / 1e9

    value = whole_job_mlups(sites, INNER * args.steps, world, ms)

    # end to end through the host-buffer entry point, the same work as one benchmark step plus the copies:
    # H2D of the initial fields, create, INNER steps, the radial profile, P_in / P_out and the sigma[R]
    # minimum, D2H of the densities and the 8 results
    e2e = None
    if not args.no_e2e:
        ws = sim.workspace  # reuse the device workspace (the simulation above is finished)
        hA = torch.from_numpy(nA0.reshape(-1)).pin_memory()
        hB = torch.from_numpy(nB0.reshape(-1)).pin_memory()
        oA, oB = torch.empty_like(hA).pin_memory(), torch.empty_like(hB).pin_memory()
        res = torch.empty(8, dtype=torch.float64).pin_memory()
        run = lambda: B.sc_run_host_sigma(params, hA, hB, INNER, centre, 0.5, 128, oA, oB, res, ws, stream)
        with torch.cuda.stream(stream):
            run()  # warm
            t0 = time.perf_counter()
            reps = max(1, args.steps // 2)
            for _ in range(reps):
                run()
            e2e_s = (time.perf_counter() - t0) / reps
        if world > 1:
            e2e_s = max_over_ranks(e2e_s * 1e3, dev) * 1e-3
        e2e = {"value": whole_job_mlups(sites, INNER, world, e2e_s * 1e3), "unit": "MLUPS",
               "h2d_bytes_per_step": 2 * sites * 8, "d2h_bytes_per_step": 2 * sites * 8 + 8 * 8,
               "result": {"dP": float(res[0]), "R_s": float(res[2]), "sigma_s": float(res[3])},
               "note": f"sc_run_host_sigma per step: H2D of n_A0, n_B0 (FP64), create, {INNER} steps, radial "
                       f"profile + P_in, P_out + sigma[R] minimum, D2H of n_A, n_B and the 8 results"}

    precision = None
    if not args.no_precision and rank == 0:
        others = [st for st in ("f32", "f16") if st != storage]
        precision = precision_block(B, [storage] + others, dev, stream)
        # the other storage mode's throughput, measured like `value` (same steps, same workload)
        if "f16" in others or "f32" in others:
            alt = others[0]
            precision["throughput"] = {alt: alt_throughput(B, alt, args, dev, stream)}

    batch = None
    if not args.no_batch and rank == 0:
        batch = batch_block(B, dev, stream, value / world if storage == "f32" else None)

    e6 = None
    if not args.no_batch and rank == 0:
        e6 = e6_slab_block(B, dev, stream)

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": storage, "data": "synthetic", "config": workload_config(storage),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": MEASURED_TRAFFIC.get((kernel_hash(), storage, traffic_key(step_cfg))),
                     "kernel": "sc_step_staged" if step_cfg["variant"] == 2 else "sc_step_kernel",
                     "launch": step_cfg,
                     "bytes_per_site": BYTES_PER_SITE[storage], "algorithmic_bytes_per_launch": alg_bytes,
                     "kernel_ms": kern_ms, "peak_source": peak_kind,
                     **({"frac_with_local_reference": (alg_bytes + LOCAL_REF_BYTES[storage] * sites)
                         / (kern_ms * 1e-3) / 1e9 / peak} if storage in LOCAL_REF_BYTES else {})},
        "hbm_roofline_mlups_frac": value / world * 1e6 * BYTES_PER_SITE[storage] / (peak * 1e9),
        "gpu_launches": launches, "clocks": clk.summary(), "e2e": e2e, "precision": precision,
        "batch_sweep": batch, "e6_slab": e6,
        "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    print(json.dumps(line), flush=True)


def sweep_droplets():
    """The batched radius sweep: 16 droplets, R_k = 8 + 32 k / 15, cubes of side 4 ceil(R_k) (about 4R,
    a multiple of 4 so that every member takes the staged kernel; centre on a node), even k symmetric,
    odd k asymmetric (G_AA c_s^2 = -0.2)."""
    import math

    import sc_synth

    out = []
    for k in range(16):
        R = 8.0 + 32.0 * k / 15.0
        L = 4 * math.ceil(R)
        G_self = (0.0, 0.0) if k % 2 == 0 else (-0.6, 0.0)
        f = sc_synth.droplet((L, L, L), (L // 2,) * 3, R, n_in=0.95, n_out=0.05, amplitude=1e-3,
                             seed=20211206 + 3 + k)
        out.append((L, R, G_self, f))
    return out


BATCH_CANDIDATES = [(8, 64, 1, 3), (8, 32, 1, 3), (8, 64, 1, 2), (4, 32, 1, 3), (4, 64, 1, 3), (4, 128, 1, 3),
                    (4, 64, 2, 2)]


def batch_block(B, dev, stream, plain_mlups, steps=128):
    """Throughput of the batched radius sweep in FP32, FP16 and BF16 storage; (tile_y, tile_z, stages,
    blocks_per_sm) and the launch form of whole 32-step runs (one persistent launch, or one launch per
    step from a CUDA graph) chosen by the autotuner on the whole batch; both forms of the chosen block
    shape are reported."""
    import torch

    from paper_2112_02574_gb300 import tune

    drops = sweep_droplets()
    sites = sum(L ** 3 for L, _, _, _ in drops)
    res = {"lattices": len(drops), "sites": sites, "sides": [L for L, _, _, _ in drops]}
    fields_ = [f for _, _, _, f in drops]
    for name, code in (("f32", B.SC_STORE_F32), ("f16", B.SC_STORE_F16), ("bf16", B.SC_STORE_BF16)):
        plist = [B.make_params((L, L, L), lattice=B.SC_D3Q19, psi_self=B.SC_PSI_EXP, storage=code, G=G_CROSS,
                               G_self=gs) for L, _, gs, _ in drops]
        cfg, _, table = tune.tune_batch(plist, fields_, BATCH_CANDIDATES, steps=32, device=dev)
        plist = [tune.with_config(p, cfg) for p in plist]

        def timed(batch):
            batch.step(64)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            batch.step(steps)
            b.record(stream)
            b.synchronize()
            for m in batch.members:
                m.sync()
            return a.elapsed_time(b)

        with torch.cuda.stream(stream):
            batch = B.Batch(plist, fields_, device=dev, stream=stream)
            forms = {}
            if batch.persistent:  # both launch forms of the tuned block shape
                for persistent in (True, False):
                    batch.persistent = persistent
                    forms["persistent" if persistent else "per_step"] = timed(batch) / steps
            batch.persistent = cfg[4]
            ms = timed(batch)
        mlups = sites * steps / (ms * 1e-3) / 1e6
        res[name] = {"MLUPS": mlups, "ms_per_step": ms / steps, "staged": batch.staged, "persistent": cfg[4],
                     "ms_per_step_by_launch_form": forms,
                     "config": dict(zip(("tile_y", "tile_z", "stages", "blocks_per_sm", "persistent"), cfg)),
                     "vs_plain_f32": mlups / plain_mlups if plain_mlups else None,
                     "tuning": [[list(c), round(m, 4)] for c, m in table]}
        del batch
    return res


def e6_slab_block(B, dev, stream, steps=1024):
    """The flat-interface slab workload: D3Q19 64 x 64 x 256, an A-rich band of width 128 along z, the
    extended (E6) forcing stencil, asymmetric couplings (G_AA c_s^2 = -0.2) with psi = exp(-1/n), FP32
    storage.  Fused steps timed with CUDA events on the launching stream; roofline on the 304-B
    algorithmic bytes per site update of the step kernel (the generic kernel: E6 reaches two sites)."""
    import torch

    import sc_synth

    shape = (64, 64, 256)
    nA0, nB0 = sc_synth.slab(shape[::-1], 128.0, amplitude=1e-3)
    params = B.make_params(shape, lattice=B.SC_D3Q19, stencil=B.SC_FORCE_E6, psi_self=B.SC_PSI_EXP,
                           storage=B.SC_STORE_F32, G=G_CROSS, G_self=(-0.6, 0.0))
    with torch.cuda.stream(stream):
        sim = B.Simulation(params, nA0, nB0, device=dev, stream=stream)
        B.sc_step(sim.ctx, 128)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        B.sc_step(sim.ctx, steps)
        b.record(stream)
        b.synchronize()
        B.sc_sync(sim.ctx)
    ms = a.elapsed_time(b) / steps
    sites = shape[0] * shape[1] * shape[2]
    peak, peak_kind = measured_peak()
    achieved = BYTES_PER_SITE["f32"] * sites / (ms * 1e-3) / 1e9
    return {"workload": "D3Q19 64x64x256 slab, A-rich band of width 128, E6 stencil, G_AA c_s^2 = -0.2, FP32",
            "MLUPS": sites / (ms * 1e-3) / 1e6, "kernel_ms": ms, "launch": sim.step_config,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "bytes_per_site": BYTES_PER_SITE["f32"], "peak_source": peak_kind}}


def alt_throughput(B, storage, args, dev, stream):
    """MLUPS of the fused step alone in another storage mode (same workload, same timing rules)."""
    import torch

    code = {"f32": B.SC_STORE_F32, "f16": B.SC_STORE_F16, "bf16": B.SC_STORE_BF16}[storage]
    params = B.make_params(SHAPE, lattice=B.SC_D3Q19, stencil=B.SC_FORCE_E4, psi_self=B.SC_PSI_EXP, storage=code,
                           tau=(1.0, 1.0), G=G_CROSS, G_self=(0.0, 0.0))
    nA0, nB0 = fields()
    with torch.cuda.stream(stream):
        sim = B.Simulation(params, nA0, nB0, device=dev, stream=stream)
        B.sc_step(sim.ctx, 3 * INNER // 4)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        B.sc_step(sim.ctx, INNER)
        b.record(stream)
        b.synchronize()
        B.sc_sync(sim.ctx)
    ms = a.elapsed_time(b)
    sites = SHAPE[0] * SHAPE[1] * SHAPE[2]
    return {"MLUPS": sites * INNER / (ms * 1e-3) / 1e6, "kernel_ms": ms / INNER,
            "hbm_frac": sites * BYTES_PER_SITE[storage] / (ms / INNER * 1e-3) / 1e9 / measured_peak()[0]}


STUDY_RADII = (8, 10, 12, 16, 20, 24, 32, 40)


def precision_study(args, dev):
    """Errors of every result against the FP64-storage GPU path (itself within 1e-13 per step of the FP64
    oracle): (1) the Tolman sweep -- 8 radii x (A-rich, B-rich) droplets in cubes of side 4 ceil(R) as one
    batch, a 64x64x256 slab for sigma_0, Eq. sigma_c fitted on the device -- for the asymmetric (G_AA c_s^2 =
    -0.2) and the symmetric coupling set; (2) the large droplet (side --study-size, R = side * 3/16,
    asymmetric): dP, R_s, sigma_s, densities and velocity."""
    import torch

    import sc_synth
    from paper_2112_02574_gb300 import binding as B
    from paper_2112_02574_gb300 import tolman

    codes = {"f64": B.SC_STORE_F64, "f32": B.SC_STORE_F32, "f16": B.SC_STORE_F16, "bf16": B.SC_STORE_BF16}
    T = args.study_steps
    mk = lambda shape, centre, R, a_rich: sc_synth.droplet(shape, centre, R, n_in=0.95, n_out=0.05, amplitude=1e-3,
                                                           a_rich=a_rich)
    slab = lambda shape: sc_synth.slab(shape, shape[0] / 2, amplitude=1e-3)
    out = {"study": "precision of every result vs the FP64-storage path; Tolman length from Eq. sigma_c",
           "tolman_steps": T, "radii": list(STUDY_RADII), "sides": [tolman.droplet_side(R) for R in STUDY_RADII]}
    for name, gs in (("asymmetric", (-0.6, 0.0)), ("symmetric", (0.0, 0.0))):
        per = {}
        for st in ("f64", "f32", "f16", "bf16"):
            t0 = time.perf_counter()
            kw = dict(lattice=B.SC_D3Q19, psi_self=B.SC_PSI_EXP, storage=codes[st], G=G_CROSS, G_self=gs)
            drops = tolman.droplet_sweep(STUDY_RADII, (1, -1), mk, kw, T, device=dev)
            s0 = tolman.flat_sigma0((64, 64, 256), slab, kw, T, device=dev)
            per[st] = {"droplets": drops, "sigma0_flat": float(s0.item()), "fit_fixed_sigma0": tolman.fit(drops, s0),
                       "fit_free_sigma0": tolman.fit(drops, None), "seconds": time.perf_counter() - t0}
            torch.cuda.empty_cache()
        ref = per["f64"]
        for st in ("f32", "f16", "bf16"):
            got = per[st]
            rel = lambda k: max(abs(a[k] - b[k]) / abs(b[k]) for a, b in zip(got["droplets"], ref["droplets"]))
            got["errors_vs_f64"] = {
                "dP_max_rel": rel("dP"), "R_s_max_rel": rel("R_s"), "sigma_s_max_rel": rel("sigma_s"),
                "sigma0_rel": abs(got["sigma0_flat"] - ref["sigma0_flat"]) / abs(ref["sigma0_flat"]),
                "delta_abs": abs(got["fit_fixed_sigma0"]["delta"] - ref["fit_fixed_sigma0"]["delta"]),
                "rigidity_abs": abs(got["fit_fixed_sigma0"]["rigidity"] - ref["fit_fixed_sigma0"]["rigidity"])}
        out[name] = per
    # the large droplet
    n = args.study_size
    shape = (n, n, n)
    R = n * 3.0 / 16.0
    nA0, nB0 = sc_synth.droplet(shape, (n // 2,) * 3, R, n_in=0.95, n_out=0.05, amplitude=1e-3)
    big = {"shape": list(shape), "R": R, "steps": args.study_size_steps}
    refm = None
    for st in ("f64", "f32", "f16", "bf16"):
        t0 = time.perf_counter()
        p = B.make_params(shape, lattice=B.SC_D3Q19, psi_self=B.SC_PSI_EXP, storage=codes[st], G=G_CROSS,
                          G_self=(-0.6, 0.0))
        sim = B.Simulation(p, nA0, nB0, device=dev)
        sim.step(args.study_size_steps)
        _, o = B.surface_of_tension(sim, (n // 2,) * 3, 0.5)
        nA, nB, u = sim.moments()
        sim.sync()
        o = o.cpu().numpy()
        res = {"dP": float(o[0]), "R_s": float(o[2]), "sigma_s": float(o[3]), "seconds": time.perf_counter() - t0}
        if refm is None:
            refm = (nA, nB, u, res)
        else:
            rA, rB, ru, rres = refm
            res["errors_vs_f64"] = {
                **{k + "_rel": abs(res[k] - rres[k]) / abs(rres[k]) for k in ("dP", "R_s", "sigma_s")},
                "n_max_rel": max(float((nA - rA).abs().max() / rA.abs().max()),
                                 float((nB - rB).abs().max() / rB.abs().max())),
                "u_max_abs": float((u - ru).abs().max()), "u_max": float(ru.abs().max())}
            del nA, nB, u
        big[st] = res
        del sim
        torch.cuda.empty_cache()
    out["large_droplet"] = big
    print(json.dumps(out), flush=True)


def large_droplet_study(args, dev):
    """The large droplet of the workload configurations at a formed droplet: side --study-size (default 256,
    the half-size fallback of 512^3), R = 3 side / 16, asymmetric couplings (G_AA c_s^2 = -0.2), psi =
    exp(-1/n), --study-large-steps time steps in every storage.  The pressure jump of Eq. bulkp is
    recorded every 2^11 steps (section 4's check interval) with its relative change; dP, R_s, sigma_s,
    densities and velocity of FP32, FP16 and BF16 storage are compared with the FP64-storage run."""
    import torch

    import sc_synth
    from paper_2112_02574_gb300 import binding as B

    n = args.study_size
    shape = (n, n, n)
    R = n * 3.0 / 16.0
    T = args.study_large_steps
    nA0, nB0 = sc_synth.droplet(shape, (n // 2,) * 3, R, n_in=0.95, n_out=0.05, amplitude=1e-3)
    kw = dict(lattice=B.SC_D3Q19, psi_self=B.SC_PSI_EXP, G=G_CROSS, G_self=(-0.6, 0.0))
    out = {"study": "large droplet at a formed droplet", "shape": list(shape), "R": R, "steps": T,
           "couplings": {"G": G_CROSS, "G_self": [-0.6, 0.0]}}

    def run(storage):
        t0 = time.perf_counter()
        sim = B.Simulation(B.make_params(shape, storage=storage, **kw), nA0, nB0, device=dev)
        jump = lambda: float((sim.bulk_pressure((n // 2,) * 3) - sim.bulk_pressure((n - 1,) * 3)).item())
        hist, t, prev = [], 0, None
        while t < T:
            w = min(2048, T - t)
            sim.step(w)
            t += w
            dp = jump()
            hist.append([t, dp, abs(dp - prev) / abs(prev) if prev else None])
            prev = dp
        _, o = B.surface_of_tension(sim, (n // 2,) * 3, 0.5)
        nA, nB, u = sim.moments()
        sim.sync()
        o = o.cpu().numpy()
        res = {"dP": float(o[0]), "R_s": float(o[2]), "sigma_s": float(o[3]), "dP_history": hist,
               "seconds": time.perf_counter() - t0}
        return res, (nA, nB, u), sim

    ref, (rA, rB, ru), sim = run(B.SC_STORE_F64)
    del sim
    torch.cuda.empty_cache()
    out["f64"] = ref
    for name, code in (("f32", B.SC_STORE_F32), ("f16", B.SC_STORE_F16), ("bf16", B.SC_STORE_BF16)):
        res, (nA, nB, u), sim = run(code)
        res["errors_vs_f64"] = {
            **{k + "_rel": abs(res[k] - ref[k]) / abs(ref[k]) for k in ("dP", "R_s", "sigma_s")},
            "n_max_rel": max(float((nA - rA).abs().max() / rA.abs().max()), float((nB - rB).abs().max() / rB.abs().max())),
            "u_max_abs": float((u - ru).abs().max()), "u_max": float(ru.abs().max())}
        out[name] = res
        del sim, nA, nB, u
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)


# The workloads (synthetic stand-ins with section 4's shapes): name -> setup
STUDY_CONFIGS = {
    "D2Q9 64^2 droplet": dict(shape=(64, 64, 1), lattice="d2q9", stencil="e4", psi="n", G=4.2, G_self=(0.0, 0.0),
                        init=("droplet", 12.0), gpu_steps=2000, storages=("f32",), orc=(400, 100)),
    "D3Q19 128^3 droplet": dict(shape=(128, 128, 128), lattice="d3q19", stencil="e4", psi="exp", G=3.6,
                          G_self=(0.0, 0.0), init=("droplet", 24.0), gpu_steps=2048,
                          storages=("f32", "f16", "bf16"), orc=(6, 2)),
    "D3Q19 64x64x256 slab, E6": dict(shape=(64, 64, 256), lattice="d3q19", stencil="e6", psi="exp", G=3.6,
                                G_self=(-0.6, 0.0), init=("slab", 128.0), gpu_steps=1024, storages=("f32",),
                                orc=(4, 1)),
    "D3Q19 512^3 droplet": dict(shape=(512, 512, 512), lattice="d3q19", stencil="e4", psi="exp", G=3.6,
                          G_self=(-0.6, 0.0), init=("droplet", 96.0), gpu_steps=64,
                          storages=("f32", "f16", "bf16"), orc=(1, 1), orc_shape=(256, 256, 256)),
}


def _config_fields(cfg, shape):
    import sc_synth

    kind, size = cfg["init"]
    if kind == "slab":
        return sc_synth.slab(shape[::-1], size, amplitude=1e-3)
    R = size * shape[0] / cfg["shape"][0]
    return sc_synth.droplet(shape[::-1], tuple(n // 2 for n in shape), R, n_in=0.95, n_out=0.05, amplitude=1e-3)


def _oracle_rate(name, steps, q=None):
    """MLUPS of the FP64 oracle on configuration `name` (at its oracle shape) over `steps` steps."""
    import oracle

    cfg = STUDY_CONFIGS[name]
    shape = cfg.get("orc_shape", cfg["shape"])
    op = oracle.Params(shape=shape, lattice=oracle.D3Q19 if cfg["lattice"] == "d3q19" else oracle.D2Q9,
                       stencil=1 if cfg["stencil"] == "e6" else 0,
                       psi_self=oracle.PSI_EXP if cfg["psi"] == "exp" else oracle.PSI_N, G=cfg["G"],
                       G_self=cfg["G_self"])
    f = oracle.init(op, *_config_fields(cfg, shape))
    t0 = time.perf_counter()
    f = oracle.step(op, f, steps)
    dt = time.perf_counter() - t0
    res = {"MLUPS": shape[0] * shape[1] * shape[2] * steps / dt / 1e6, "threads": oracle.threads(),
           "shape": list(shape), "steps": steps, "seconds": dt}
    if q is not None:
        q.put(res)
    return res


def _oracle_one_thread(name, steps, q):
    os.environ["OMP_NUM_THREADS"] = "1"
    _oracle_rate(name, steps, q)


def configs_study(args, dev):
    """Each workload configuration: the GPU step rate (CUDA events, fused steps only) in its storage modes,
    and the FP64 oracle's rate on the host cores (all threads, and one thread in a spawned process)."""
    import multiprocessing as mp

    import torch

    from paper_2112_02574_gb300 import binding as B

    codes = {"f32": B.SC_STORE_F32, "f16": B.SC_STORE_F16, "bf16": B.SC_STORE_BF16}
    out = {"study": "workload configurations: GPU step rate and FP64 oracle rate", "configs": {}}
    ctx = mp.get_context("spawn")
    for name, cfg in STUDY_CONFIGS.items():
        if args.study_config and args.study_config not in name:
            continue
        res = {"shape": list(cfg["shape"]), "gpu": {}}
        if not args.no_cpu_baseline:
            # the oracle first: one thread in a spawned child, then all threads here
            q = ctx.Queue()
            pr = ctx.Process(target=_oracle_one_thread, args=(name, cfg["orc"][1], q))
            pr.start()
            res["oracle_1_thread"] = q.get()
            pr.join()
            res["oracle_all_threads"] = _oracle_rate(name, cfg["orc"][0])
        shape = cfg["shape"]
        nA, nB = _config_fields(cfg, shape)
        for st in cfg["storages"]:
            p = B.make_params(shape, lattice=B.SC_D3Q19 if cfg["lattice"] == "d3q19" else B.SC_D2Q9,
                              stencil=B.SC_FORCE_E6 if cfg["stencil"] == "e6" else B.SC_FORCE_E4,
                              psi_self=B.SC_PSI_EXP if cfg["psi"] == "exp" else B.SC_PSI_N, storage=codes[st],
                              G=cfg["G"], G_self=cfg["G_self"])
            sim = B.Simulation(p, nA, nB, device=dev)
            sim.step(max(8, cfg["gpu_steps"] // 8))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(sim.stream)
            sim.step(cfg["gpu_steps"])
            b.record(sim.stream)
            b.synchronize()
            sim.sync()
            ms = a.elapsed_time(b) / cfg["gpu_steps"]
            sites = shape[0] * shape[1] * shape[2]
            res["gpu"][st] = {"MLUPS": sites / (ms * 1e-3) / 1e6, "us_per_step": ms * 1e3,
                              "hbm_frac": sites * BYTES_PER_SITE[st] / (ms * 1e-3) / 1e9 / measured_peak()[0],
                              "launch": sim.step_config}
            del sim
            torch.cuda.empty_cache()
        out["configs"][name] = res
        print(json.dumps({name: res}), flush=True)
    print(json.dumps(out), flush=True)


PAPER_SIDES = (25, 31, 37, 41, 51, 57, 65)  # section 4's system sizes up to 65; R = L / 4
PAPER_DGAB = (0.0, 0.48, -0.48, 0.88, -0.88)


def paper_couplings(dGAB: float, dGc: float = 0.4):
    """Eq. self_p: G_AA = G_c [1 - dG_c (1 + dG_AB)], G_BB = G_c (1 - dG_c), with G_c c_s^2 = -e^2 / 3
    (the critical self coupling of psi = exp(-1/n), printed as -2.463) and G c_s^2 = 0.5 (section 4)."""
    Gc = -math.e ** 2
    return dict(G=1.5, G_self=(Gc * (1.0 - dGc * (1.0 + dGAB)), Gc * (1.0 - dGc)))


def paper_tolman_study(args, dev):
    """The Tolman sweep on the paper's couplings (section 4): per dG_AB a flat-interface pre-run (slab
    16 x 16 x 128) gives the bulk densities and sigma_0; A-rich and B-rich droplets of side L (odd, the
    paper's sizes) and R = L / 4 start from those densities; all droplets of all dG_AB run as one batch
    until each has converged by section 4's criteria (then it retires from the batch); Eq. sigma_c is
    fitted on the device with sigma_0 held at the slab value."""
    import sc_synth
    from paper_2112_02574_gb300 import binding as B
    from paper_2112_02574_gb300 import tolman

    code = {"f64": B.SC_STORE_F64, "f32": B.SC_STORE_F32, "f16": B.SC_STORE_F16, "bf16": B.SC_STORE_BF16}[
        args.study_storage]
    T = args.study_steps
    ntot = args.study_density
    sides = tuple(int(v) for v in args.study_sides.split(",")) if args.study_sides else PAPER_SIDES
    dgabs = tuple(float(v) for v in args.study_dgab.split(",")) if args.study_dgab else PAPER_DGAB
    out = {"study": "Tolman length on the couplings of Eq. self_p (dG_c = 0.4, G c_s^2 = 0.5, psi = exp(-1/n))",
           "steps": T, "storage": args.study_storage, "total_density": ntot, "sides": list(sides), "sets": {}}
    members, flats = [], {}
    for d in dgabs:
        kw = dict(lattice=B.SC_D3Q19, psi_self=B.SC_PSI_EXP, storage=code, **paper_couplings(d))
        slab = lambda shape: sc_synth.slab(shape, shape[0] / 2, n_rich=0.95 * ntot, n_poor=0.05 * ntot,
                                           amplitude=1e-3)
        fl = tolman.flat_densities((16, 16, 128), slab, kw, T, device=dev)
        flats[d] = fl
        for L in sides:
            for sign in (1, -1):
                inside = (fl["A_in"], fl["B_in"]) if sign > 0 else (fl["A_out"], fl["B_out"])
                outside = (fl["A_out"], fl["B_out"]) if sign > 0 else (fl["A_in"], fl["B_in"])
                # section 4's initial profile as printed: no noise (the slab pre-run keeps its +-1e-3)
                f = sc_synth.droplet_ab((L, L, L), (L // 2,) * 3, L / 4.0, inside[0], outside[0], inside[1],
                                        outside[1], amplitude=0.0)
                members.append({"L": L, "R": L / 4.0, "sign": sign, "params": kw, "fields": f, "tag": d})
    t0 = time.perf_counter()
    drops = tolman.sweep(members, T, device=dev, converge=True)
    out["sweep_seconds"] = time.perf_counter() - t0
    out["convergence"] = "section 4: every 2048 steps, |dP change| / dP < 1e-5 or dU < 1e-12; converged " \
                         "droplets retire from the batch; at most --study-steps steps"
    import torch

    for d in dgabs:
        ds = [x for x in drops if x["tag"] == d]
        s0 = torch.tensor([flats[d]["sigma0"]], dtype=torch.float64, device=dev)
        free = tolman.fit(ds, None, device=dev)
        # section 4, Fig. 3a: the droplets' R_s -> infinity limit (Eq. sigma_c with sigma_0 free) against the
        # slab, over all sizes and over the larger sizes only (the expansion in 1/R_s holds better there)
        limits = {}
        for lmin in sorted({min(sides), 51, 97}):
            sub = [x for x in ds if x["L"] >= lmin]
            f = tolman.fit(sub, None, device=dev)
            limits[f"L>={lmin}"] = {"sigma0": f["sigma0"], "delta": f["delta"], "used": f["used"],
                                    "rel_to_slab": (f["sigma0"] - flats[d]["sigma0"]) / flats[d]["sigma0"]}
        out["sets"][f"{d:+.2f}"] = {"flat": flats[d], "fit_fixed_sigma0": tolman.fit(ds, s0, device=dev),
                                    "fit_free_sigma0": free,
                                    "sigma0_limit_vs_slab": (free["sigma0"] - flats[d]["sigma0"]) / flats[d]["sigma0"],
                                    "droplet_limit_by_size": limits,
                                    "converged": sum(1 for x in ds if x["converged"]),
                                    "steps_range": [min(x["steps"] for x in ds), max(x["steps"] for x in ds)],
                                    "max_com_offset": max(x["com_offset"] for x in ds),
                                    "com_accepted": sum(1 for x in ds if x["com_offset"] < 1e-3),
                                    "max_dP_change": max(x["dP_change"] for x in ds), "droplets": ds}
    print(json.dumps(out), flush=True)


def main():
    global INNER
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16", "f64"])
    ap.add_argument("--tile-y", type=int, default=0)
    ap.add_argument("--tile-z", type=int, default=0)
    ap.add_argument("--variant", type=int, default=0, help="step kernel: 0 auto, 1 generic, 2 cp.async-staged")
    ap.add_argument("--stages", type=int, default=0, help="staged kernel pipeline stages (0 default, 1, 2)")
    ap.add_argument("--blocks-per-sm", type=int, default=0, help="staged kernel register budget (0 default)")
    ap.add_argument("--kernel-events", action="store_true", help="record per-step kernel events in the timed loop")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-precision", action="store_true", help="skip the sigma / R_s / dP error block")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched radius sweep block")
    ap.add_argument("--inner", type=int, default=INNER, help="time steps per benchmark step (profiling runs)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--study", choices=["precision", "paper", "configs", "large"],
                    help="run only a study (minutes) and print its JSON line: precision = every result in each "
                         "storage against the FP64 path; paper = Tolman length on the couplings of Eq. self_p; "
                         "configs = GPU and oracle rates of every workload configuration")
    ap.add_argument("--study-config", default="",
                    help="configs study: only the configurations whose name contains this text")
    ap.add_argument("--study-storage", default="f32", choices=["f64", "f32", "f16", "bf16"])
    ap.add_argument("--study-density", type=float, default=2.0, help="total density of the paper study")
    ap.add_argument("--study-steps", type=int, default=16384, help="time steps of the Tolman sweep and slab")
    ap.add_argument("--study-size", type=int, default=512, help="side of the large droplet of the study")
    ap.add_argument("--study-size-steps", type=int, default=4096, help="time steps of the large droplet")
    ap.add_argument("--study-sides", default="", help="paper study: comma-separated cube sides (default: 25..65)")
    ap.add_argument("--study-dgab", default="", help="paper study: comma-separated dG_AB values")
    ap.add_argument("--study-large-steps", type=int, default=16384, help="large study: time steps per storage")
    args = ap.parse_args()
    INNER = args.inner
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # no launcher: start one rank per GPU on this node and pass the arguments through
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
               "--master-addr", "127.0.0.1", "--master-port", os.environ.get("MASTER_PORT", "29511"),
               os.path.abspath(__file__), *sys.argv[1:]]
        sys.exit(subprocess.call(cmd))
    if args.gpus != world:
        sys.exit(f"bench.py: --gpus {args.gpus} but the launcher started {world} rank(s)")
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.study:
        if rank == 0:
            {"precision": precision_study, "paper": paper_tolman_study, "configs": configs_study,
             "large": large_droplet_study}[args.study](args, "cuda")
        return
    if world > 1:
        import torch
        import torch.distributed as tdist

        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
    try:
        run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as tdist

            tdist.destroy_process_group()


if __name__ == "__main__":
    main()
