#!/usr/bin/env python
"""Benchmark: cells/s assembled + solved by the ROM-accelerated BDDC path.

Workload: 132 x 132 = 17,424 cells, p = 6, quartic maps from a smooth random
field, circle-hole and cross families mixed 50/50, one reduced model of rank 60
per family (trained by the library's GPU trainer before timing), rho = 5e-4,
left edge clamped, unit downward traction on the right edge, PCG rtol 1e-8.

One step = romb_assemble (theta + contraction) -> romb_factor (local BDDC
set-up + coarse Cholesky) -> romb_bddc_solve (PCG + interior recovery).
`value` times steps whose inputs are already resident in HBM (device pointers);
`e2e` times the same calls with pinned host inputs and a host read of the
displacement inside the timed region.  L2 is flushed (a 512 MB write) between
timed steps, outside the timed events.

--impl reference times the CPU oracle on bounded samples of the same workload
(independent tiles, one per host core), with models trained by the oracle.
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
sys.path.insert(0, ROOT)

METRIC = "cells/s assembled+solved at 17,424 cells p=6; FP32 vs FP64 form at ≤1e-6 error"
CONFIG = 3
SAMPLE_NX = SAMPLE_NY = 12      # tile of the reference arm (one per host core per step)
BASE_NX = BASE_NY = 24          # bounded CPU sample of the cpu_baseline leg (~15 s)
FP64_PEAK_GFLOPS = 1250.0       # nominal dense FP64 rate of GB300 (profiling recipe)
# DRAM bytes (read + write) per cell of the local factor kernel, from an ncu
# capture of one launch on the first 66 x 66 cells of the 132 x 132 p = 6
# workload (4,356 cells; per-cell traffic, scaled to the launch by the cell
# count; profiles/factor_kernel_132x132_p6.md)
FACTOR_TRAFFIC_PER_CELL = (172553984 + 312830976) / 4356


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "fp64", "fp32split", "bf16split"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-fp64-form", action="store_true")
    ap.add_argument("--workload", type=int, default=3, choices=[3, 4, 5, 6, 7],
                    help="3: the headline (132 x 132, p = 6); 4: the compliance gradient on 64 x 64 cells; "
                         "5: 256 x 256 cells, p = 8, 16 load sets sharing one factorisation; "
                         "6: the quarter-annulus Schwarz Diamond benchmark, p = 8, 16 clusters; "
                         "7: the wrench-like layout of Schoen IWP cells, 90 and 7,290 cells, p = 8")
    ap.add_argument("--sub", type=int, default=0,
                    help="profiling only: run the first N x N cells of the workload")
    ap.add_argument("--cpu-sample-json", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--rom-dir", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--small-models", action="store_true", help=argparse.SUPPRESS)
    return ap.parse_args()


# ---------------------------------------------------------------------------
# shared set-up
# ---------------------------------------------------------------------------
def train_models(rom_dir: str, compare_host: bool = True):
    """Offline phase (Sec. 4.2): the library's GPU trainer on the LHS samples
    from the seeded inputs; the host trainer on the same samples is timed
    beside it (its files are not used)."""
    import lattice_inputs as LI
    import paper_2604_09113_gb300 as romb
    paths = []
    gpu_s = host_s = 0.0
    for spec in LI.rom_specs(CONFIG):
        path = os.path.join(rom_dir, f"family{spec.family}.rom")
        S = LI.lhs(spec.n_s, spec.lo, spec.hi, seed=spec.seed)
        if not os.path.exists(path):
            t0 = time.perf_counter()
            romb.romb_train_gpu(spec.family, 0, spec.p, spec.r, spec.n_r, spec.lo, spec.hi, S, path)
            gpu_s += time.perf_counter() - t0
            if compare_host:
                t0 = time.perf_counter()
                romb.romb_train(spec.family, 0, spec.p, spec.r, spec.n_r, spec.lo, spec.hi, S, path + ".host")
                host_s += time.perf_counter() - t0
                os.unlink(path + ".host")
        paths.append(path)
    info = {"gpu_s": gpu_s, "models": "rank 60, 400 samples, 2,401 grid nodes, two families"}
    if compare_host:
        info["host_s"] = host_s
        info["host_threads"] = os.cpu_count()
    return paths, info


def sub_lattice(lat, sx: int, sy: int):
    import lattice_inputs as LI
    return LI.sub_lattice(lat, sx, sy)


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


_TILE_ROMS = {}


def _oracle_tile_job(args):
    """One independent tile of the workload through the oracle's online phase
    (MDEIM assembly, BDDC set-up, PCG rtol 1e-8, recovery); runs in a pool
    worker.  Returns (seconds, cells)."""
    rom_paths, x0, y0, sx, sy = args
    import lattice_inputs as LI
    from oracle import bddc as obddc, pipeline, rom as orom
    key = tuple(rom_paths)
    if key not in _TILE_ROMS:
        _TILE_ROMS[key] = {R.family: R for R in (orom.read(p) for p in rom_paths)}
    lat = LI.tile_lattice(LI.config(CONFIG), x0, y0, sx, sy)
    t0 = time.perf_counter()
    K = pipeline.matrices_rom(lat, _TILE_ROMS[key])
    pipeline.solve(lat, K, obddc.lattice_loads(lat), rtol=1e-8)
    return time.perf_counter() - t0, lat.ncells


def tiles(count: int, size: int):
    """`count` tiles of size x size cells of the 132 x 132 workload, row by row
    (repeated when the workload has fewer)."""
    per = 132 // size
    return [((k % (per * per)) % per * size, (k % (per * per)) // per * size) for k in range(count)]


def spawn_pool(n: int):
    """Process pool started with spawn (safe after CUDA initialisation), one
    single-threaded worker per core."""
    import multiprocessing as mp
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        return mp.get_context("spawn").Pool(n)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def oracle_tiles_seconds(pool, rom_paths, count: int, size: int):
    """Wall time of `count` independent tiles run concurrently by the pool."""
    jobs = [(list(rom_paths), x0, y0, size, size) for x0, y0 in tiles(count, size)]
    t0 = time.perf_counter()
    res = pool.map(_oracle_tile_job, jobs, chunksize=1)
    return time.perf_counter() - t0, sum(c for _, c in res)


def oracle_models(train: bool, small: bool = False):
    """Oracle-trained models of the workload (cached per machine); None when
    train is False and they are not cached.  small: the rank-60 models on 80
    samples with r = 2 (for a quick check of the line's format only; weaker
    models leave some cells of this lattice indefinite)."""
    import dataclasses
    import lattice_inputs as LI
    from oracle import offline
    specs = LI.rom_specs(CONFIG)
    if small:
        specs = [dataclasses.replace(s, n_s=80, r=2) for s in specs]
    return offline.workload_models(specs, lambda n, lo, hi, seed: LI.lhs(n, lo, hi, seed=seed), train=train)


def cpu_baseline(rom_paths):
    """The oracle on the host cores, in a child process (threads fixed before
    numpy loads): one 24 x 24 tile single-threaded, then one tile per core
    run concurrently.  Uses the oracle-trained models when a reference-arm
    run on this machine has cached them, else the benchmark's model files
    (the timing does not depend on the model's values)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    with tempfile.NamedTemporaryFile(suffix=".json", delete=False) as f:
        out = f.name
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-sample-json", out, "--rom-dir",
           os.path.dirname(rom_paths[0])]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=900)
    if r.returncode != 0:
        return {"value": None, "unit": "cells/s", "cores": 1, "kind": "oracle", "error": r.stderr[-400:]}
    d = json.load(open(out))
    os.unlink(out)
    return d


def cpu_sample(rom_dir: str, out: str):
    """Body of the cpu_baseline child process."""
    models = oracle_models(train=False)
    src = "oracle-trained models"
    if models is None:
        models = sorted(os.path.join(rom_dir, f) for f in os.listdir(rom_dir) if f.endswith(".rom"))
        src = "the benchmark's model files"
    nproc = os.cpu_count() or 1
    single, cells1 = _oracle_tile_job((models, 0, 0, BASE_NX, BASE_NY))
    with spawn_pool(nproc) as pool:
        oracle_tiles_seconds(pool, models, nproc, 8)          # workers import numpy / scipy
        wall, cells_all = oracle_tiles_seconds(pool, models, nproc, BASE_NX)
    json.dump({"value": cells1 / single, "unit": "cells/s", "cores": 1, "kind": "oracle",
               "sample": f"{cells1} cells: first {BASE_NX}x{BASE_NY} cells of the workload, MDEIM assembly + "
                         f"BDDC set-up + PCG + recovery, single thread ({src})",
               "seconds": single, "cpu_model": cpu_model(), "nproc": nproc,
               "all_cores": {"value": cells_all / wall, "unit": "cells/s", "cores": nproc, "seconds": wall,
                             "sample": f"{nproc} independent {BASE_NX}x{BASE_NY} tiles of the workload, one "
                                       f"single-threaded process per core, run concurrently"}},
              open(out, "w"))


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.file = tempfile.NamedTemporaryFile(suffix=".csv", delete=False)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.file.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    pass
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, v in enumerate(fl) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def aggregate(total_ms: float, cells_per_rank: int, world: int, device=None):
    """Whole-job throughput of independent replicas: every rank processes its own
    copy of the workload; the job time is the slowest rank's (all_reduce MAX)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, world * cells_per_rank / (total_ms / 1e3)


# ---------------------------------------------------------------------------
# flop models (algorithmic counts per cell)
# ---------------------------------------------------------------------------
def factor_flops(p: int) -> float:
    NI, NU = 2 * (p - 1) ** 2, 8 * p
    NK = NU - 8
    f = NI ** 3 / 3 + NI ** 2 * NU + NU * (NU + 1) * NI          # chol K_II, W, S
    f += NK ** 3 / 3 + NK ** 2 * 12 + 12 * 13 * NK               # chol Shat, Y, That
    f += 2 * NK ** 2 * 20 + 2 * 12 * NK * 20 + 2 * 144 * 20      # Z, R, Lambda
    f += 2 * NK * 12 * 20 + NK ** 2 * 20                         # Y Lambda, Lhat^-T
    f += 2 * NU * NU * 20 + 2 * 400 * NU                         # S Psi, Psi^T S Psi
    f += NK ** 3 / 3 + 144 * NK + 12 * NK ** 2 + NK * NK * (NK / 3 + 12)   # M, V, N, F
    return f


def nd_fronts(nx: int, ny: int, dmask: int) -> list:
    """(ns, nb) of every front of the library's geometric nested dissection
    of the coarse problem: coarse DoFs on vertices (2) and edges (3),
    rectangles bisected across the longer side down to 2 x 2 cells; separator
    DoFs of a rectangle are eliminated there (ns), DoFs on its internal sides
    are its update rows (nb); clamped DoFs are absent."""
    def vdir(vx, vy):
        return ((dmask & 1) and vx == 0) or ((dmask & 2) and vx == nx) or ((dmask & 4) and vy == 0) or \
            ((dmask & 8) and vy == ny)

    def groups(x0, x1, y0, y1):
        out = []
        for py in range(2 * y0, 2 * y1 + 1):
            for px in range(2 * x0, 2 * x1 + 1):
                ex, ey = px % 2 == 0, py % 2 == 0
                if not ex and not ey:
                    continue
                if ex and ey:
                    if not vdir(px // 2, py // 2):
                        out.append((px, py, 2))
                elif ey:
                    vy = py // 2
                    if not ((vy == 0 and dmask & 4) or (vy == ny and dmask & 8)):
                        out.append((px, py, 3))
                else:
                    vx = px // 2
                    if not ((vx == 0 and dmask & 1) or (vx == nx and dmask & 2)):
                        out.append((px, py, 3))
        return out

    fronts = []
    stack = [(0, nx, 0, ny)]
    while stack:
        x0, x1, y0, y1 = stack.pop()
        w, h = x1 - x0, y1 - y0
        leaf = w <= 2 and h <= 2
        xm = x0 + w // 2 if (not leaf and w >= h) else -1
        ym = y0 + h // 2 if (not leaf and w < h) else -1
        ns = nb = 0
        for px, py, nd in groups(x0, x1, y0, y1):
            if (px == 2 * x0 and x0 > 0) or (px == 2 * x1 and x1 < nx) or (py == 2 * y0 and y0 > 0) or \
                    (py == 2 * y1 and y1 < ny):
                nb += nd
            elif leaf or (xm >= 0 and px == 2 * xm) or (ym >= 0 and py == 2 * ym):
                ns += nd
        fronts.append((ns, nb))
        if not leaf:
            if xm >= 0:
                stack += [(x0, xm, y0, y1), (xm, x1, y0, y1)]
            else:
                stack += [(x0, x1, y0, ym), (x0, x1, ym, y1)]
    return fronts


def coarse_solve_fma(nx: int, ny: int, dmask: int) -> float:
    """FMAs of one coarse solve (FP32 in the split forms): both sweeps apply every front's
    B = [L11^-T | -(L21 L11^-1)^T] once (ns(ns+1)/2 + ns nb entries)."""
    return sum(2.0 * (ns * (ns + 1) / 2 + ns * nb) for ns, nb in nd_fronts(nx, ny, dmask))


def pcg_cell_fma(p: int) -> float:
    """FMAs per cell and PCG iteration: S p (nU^2), D F D r on its non-zero
    (nU-8)^2 block, Phi^T r and Phi g (2 nU 20); all FP64 in the FP64 form,
    all but S p FP32 in the split forms (the preconditioner)."""
    NU = 8 * p
    return NU * NU + (NU - 8) ** 2 + 2 * NU * 20


def assembly_flops(p: int, n_r: int) -> float:
    nB = (p + 1) ** 2
    pairs = nB * (nB + 1) // 2
    return 2.0 * (n_r + 1) * 36 * pairs + 2.0 * 4 * 36 * pairs


def tensor_peak_tflops(form: str):
    """Dense tensor-core peak for the split form's operand type: the measured
    bf16 burst rate of this machine (MEASURED_PEAKS.json), times the nominal
    TF32 / BF16 ratio (1.1 / 2.25 PFLOP/s) for the TF32 form."""
    src = "measured bf16 burst (MEASURED_PEAKS.json)"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            bf16 = float(json.load(fh)["bf16_tflops"])
    except (OSError, ValueError, KeyError):
        bf16, src = 1900.0, "fallback bf16 burst 1.9 PFLOP/s"
    if form == "fp32split":
        return bf16 * 1.1 / 2.25, src + " x 1.1/2.25 (nominal TF32/BF16)"
    return bf16, src


def fma_rates(romb, torch, stream, sms: int) -> dict:
    """FP64 and FP32 FMA issue rates of this GPU, measured by the library's
    probe kernel (8 independent FMA chains per thread, 8 warps per block,
    8 blocks per SM) on the benchmark's stream with CUDA events, best of 5
    launches of ~20 ms after a warm-up launch."""
    out = {}
    blocks, threads = 8 * sms, 256
    for name, prec, dt in (("fp64_gflops", 0, torch.float64), ("fp32_gflops", 1, torch.float32)):
        buf = torch.empty(blocks * threads, dtype=dt, device=torch.device("cuda", torch.cuda.current_device()))
        iters = 64
        best = 0.0
        for rep in range(7):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fl = romb.romb_fma_probe(prec, blocks, threads, iters, stream.cuda_stream, buf)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            if rep == 0:           # size the launches for ~20 ms
                iters = max(16, int(iters * 20.0 / max(ms, 1e-3)))
                continue
            if rep >= 2:
                best = max(best, fl / (ms / 1e3) / 1e9)
        out[name] = best
    out["how"] = (f"romb_fma_probe: {blocks} blocks x {threads} threads x 8 independent FMA chains, "
                  "best of 5 launches of ~20 ms, CUDA events on the benchmark stream")
    return out


def assembly_report(phase_ms, ncells: int, p: int, n_r: int, form: str, world: int = 1,
                    fp64_gflops: float = FP64_PEAK_GFLOPS) -> dict:
    """Assembly alone (theta + contraction phases): cells/s, and the
    contraction's algorithmic rate (assembly_flops per cell, K symmetry used)
    against the tensor-core peak of its operand type, or against the FP64 rate
    for the FP64 form."""
    asm_ms = float(phase_ms[0] + phase_ms[1])
    fl = assembly_flops(p, n_r) * ncells
    out = {"cells_per_s": world * ncells / (asm_ms / 1e3), "ms": asm_ms,
           "contraction_ms": float(phase_ms[1]),
           "contraction_tflops": fl / (float(phase_ms[1]) / 1e3) / 1e12,
           "units": f"{ncells} cells x {assembly_flops(p, n_r):.0f} flop"}
    if form == "fp64":
        out["peak_tflops"], out["peak_source"] = fp64_gflops / 1e3, "measured FP64 FMA rate (fma_rates)"
    else:
        out["peak_tflops"], out["peak_source"] = tensor_peak_tflops(form)
    out["frac"] = out["contraction_tflops"] / out["peak_tflops"]
    return out


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(a):
    import numpy as np
    import torch
    import lattice_inputs as LI
    import paper_2604_09113_gb300 as romb

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    rom_dir = a.rom_dir or tempfile.mkdtemp(prefix="romb_models_")
    paths, train_info = train_models(rom_dir)
    lat = LI.config(CONFIG)
    if a.sub:
        lat = sub_lattice(lat, a.sub, a.sub)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = romb.Context(local, 0, stream.cuda_stream)
    for p_ in paths:
        romb.romb_train_load(ctx.h, p_)
    nodes = (lat.p * lat.nx + 1) * (lat.p * lat.ny + 1)
    darr = {"ctrl": torch.from_numpy(lat.ctrl).to(dev), "mu": torch.from_numpy(lat.mu).to(dev),
            "family": torch.from_numpy(lat.family).to(dev),
            "traction": torch.from_numpy(lat.traction.reshape(8).copy()).to(dev)}
    u_dev = torch.zeros((1, nodes, 2), dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device=dev)   # 512 MB > L2

    have_tc = a.precision != "fp64"
    precisions = {"fp64": romb.ROMB_FP64, "fp32split": romb.ROMB_FP32_SPLIT,
                  "bf16split": romb.ROMB_BF16_SPLIT}
    if a.precision == "auto":
        try:
            romb.romb_assemble(ctx.h, lat, romb.ROMB_FP32_SPLIT, device_arrays=darr)
        except romb.RombError:
            have_tc = False
    if a.precision == "auto":
        form = "fp32split" if have_tc else "fp64"
    else:
        form = a.precision
    prec = precisions[form]

    def step(pr, host=None):
        if host is None:
            romb.romb_assemble(ctx.h, lat, pr, device_arrays=darr)
        else:
            romb.romb_assemble(ctx.h, host["lat"], pr)
        romb.romb_factor(ctx.h)
        out = u_dev if host is None else host["u"]
        _, its, rel = romb.romb_bddc_solve(ctx.h, nodes, rtol=1e-8, maxit=500, out=out)
        return int(its[0]), float(rel[0])

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(a.warmup):
        step(prec)
    barrier()
    rates = fma_rates(romb, torch, stream, torch.cuda.get_device_properties(dev).multi_processor_count)
    peak64 = rates["fp64_gflops"] or FP64_PEAK_GFLOPS
    barrier()
    clocks = Clocks(local)
    clocks.start()
    l0 = romb.romb_launch_count(ctx.h)
    times, phases, iters = [], [], []
    for _ in range(a.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        it, rel = step(prec)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        phases.append(romb.romb_stats(ctx.h)[0].copy())
        iters.append(it)
    launches = (romb.romb_launch_count(ctx.h) - l0) // max(1, a.steps)
    barrier()
    clk = clocks.stop()
    total_ms, _ = aggregate(sum(times), lat.ncells, world, dev)
    ms = total_ms / a.steps
    value = world * lat.ncells / (ms / 1e3)
    ph = np.mean(np.array(phases), axis=0)

    # accuracy of the split form against the FP64 form (same device, same inputs)
    u_form = u_dev.clone()
    acc = {}
    fp64_form = None
    names = ["theta", "contraction", "local_factor", "coarse_factor", "pcg", "recovery"]
    if form != "fp64" and not a.no_fp64_form:
        # the all-FP64 GPU form on the same lattice, timed like the chosen form
        # (L2 flushed between steps; fewer steps: it is ~2.5x slower)
        step(romb.ROMB_FP64)
        k64 = max(1, min(a.steps, 5))
        t64, ph64, it64 = [], [], []
        for _ in range(k64):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            it, _ = step(romb.ROMB_FP64)
            e1.record(stream)
            e1.synchronize()
            t64.append(e0.elapsed_time(e1))
            ph64.append(romb.romb_stats(ctx.h)[0].copy())
            it64.append(it)
        ms64, _ = aggregate(sum(t64), lat.ncells, world, dev)
        ms64 /= k64
        p64 = np.mean(np.array(ph64), axis=0)
        fp64_form = {"value": world * lat.ncells / (ms64 / 1e3), "unit": "cells/s", "ms_per_step": ms64,
                     "steps": k64, "pcg_iters": it64[-1],
                     "phase_ms": {n: float(v) for n, v in zip(names + ["copies", "total"], p64)},
                     "speedup_of_chosen_form": ms64 / ms}
    if have_tc and not a.no_accuracy:
        # every split form against the FP64 form, untimed, on the same lattice
        if form == "fp64":
            u_ref = u_form
        else:
            step(romb.ROMB_FP64)
            u_ref = u_dev.clone()
        den = torch.linalg.vector_norm(u_ref).item()
        for name in ("fp32split", "bf16split"):
            if name == form:
                u_s = u_form
            else:
                step(precisions[name])
                u_s = u_dev.clone()
            acc["disp_rel_l2_%s_vs_fp64" % name] = torch.linalg.vector_norm(u_s - u_ref).item() / den
        step(prec)

    # end to end: pinned host inputs, host output, through the public API
    e2e = None
    if not a.no_e2e:
        pin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory()
               for k, v in {"ctrl": lat.ctrl, "mu": lat.mu, "family": lat.family,
                            "traction": lat.traction}.items()}
        hl = LI.Lattice(**{**lat.__dict__, "ctrl": pin["ctrl"].numpy(), "mu": pin["mu"].numpy(),
                           "family": pin["family"].numpy(), "traction": pin["traction"].numpy()})
        u_host = torch.zeros((1, nodes, 2), dtype=torch.float64).pin_memory().numpy()
        host = {"lat": hl, "u": u_host}
        step(prec, host)
        et = []
        for _ in range(a.steps):
            flush.zero_()
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(prec, host)
            e1.record(stream)
            e1.synchronize()
            et.append(e0.elapsed_time(e1))
        ems = sum(et) / len(et)
        if world > 1:
            t = torch.tensor([ems], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            ems = float(t.item())
        h2d = lat.ctrl.nbytes + lat.mu.nbytes + lat.family.nbytes + lat.traction.nbytes
        e2e = {"value": world * lat.ncells / (ems / 1e3), "unit": "cells/s", "ms_per_step": ems,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(u_host.nbytes)}

    # roofline of the dominant single kernel (the local factor kernel; the PCG
    # phase is ~40 small kernels per iteration), from its CUDA-event time on the
    # context stream, plus the PCG phase as a whole against the same FP64 peak
    n_r = max(s.n_r for s in LI.rom_specs(CONFIG))
    fl = factor_flops(lat.p) * lat.ncells
    roof = {"kernel": f"factor_kernel<{lat.p}>", "bound": "alu", "achieved": fl / (ph[2] / 1e3) / 1e9,
            "peak": peak64, "unit": "GFLOP/s (FP64)", "traffic": (FACTOR_TRAFFIC_PER_CELL * lat.ncells
                                                                         if FACTOR_TRAFFIC_PER_CELL else None),
            "units": f"{lat.ncells} cells x {factor_flops(lat.p):.0f} flop",
            "peak_source": "measured FP64 FMA rate of this GPU (fma_rates: romb_fma_probe)"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    # the split forms apply the preconditioner in FP32 (D F D, Phi, the coarse
    # substitutions); S p stays FP64
    NU = 8 * lat.p
    pre_fma = (pcg_cell_fma(lat.p) - NU * NU) * lat.ncells + coarse_solve_fma(lat.nx, lat.ny,
                                                                             int(lat.dirichlet_mask))
    sp_fma = NU * NU * lat.ncells
    pcg_s = ph[4] / 1e3
    if form == "fp64":
        roof_pcg = {"phase": "pcg", "bound": "alu", "achieved": iters[-1] * 2.0 * (sp_fma + pre_fma) / pcg_s / 1e9,
                    "peak": peak64, "unit": "GFLOP/s (FP64)", "iterations": iters[-1]}
    else:
        peak32 = rates.get("fp32_gflops") or None
        roof_pcg = {"phase": "pcg", "bound": "alu", "achieved": iters[-1] * 2.0 * sp_fma / pcg_s / 1e9,
                    "peak": peak64, "unit": "GFLOP/s (FP64: S p)", "iterations": iters[-1],
                    "fp32_preconditioner": {"achieved": iters[-1] * 2.0 * pre_fma / pcg_s / 1e9, "peak": peak32,
                                            "unit": "GFLOP/s (FP32: D F D, Phi, coarse substitutions)"}}
        if peak32:
            roof_pcg["fp32_preconditioner"]["frac"] = roof_pcg["fp32_preconditioner"]["achieved"] / peak32
    roof_pcg["frac"] = roof_pcg["achieved"] / roof_pcg["peak"]
    asm = assembly_report(ph, lat.ncells, lat.p, n_r, form, world, peak64)

    cpu = None
    if rank == 0 and not a.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(paths)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp64": "f64", "fp32split": "tf32x3+f64", "bf16split": "bf16x10+f64"}[form], "data": "synthetic",
            "config": {"workload": "132x132 lattice, p=6, quartic maps, circle/cross 50/50, n_r=60 per family",
                       "cells": lat.ncells, "p": lat.p, "assembly_form": form,
                       "l2": "flushed (512 MB write) between timed steps", "pcg_rtol": 1e-8},
            "clocks": clk, "e2e": e2e, "gpu_launches": int(launches), "roofline": roof, "roofline_pcg": roof_pcg,
            "assembly": asm,
            "cpu_baseline": cpu, "pcg_iters": iters[-1],
            "phase_ms": {n: float(v) for n, v in zip(names + ["copies", "total"], ph)},
            "offline_train": train_info, "accuracy": acc or None, "fp64_form": fp64_form,
            "fma_rates": rates,
        }
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------------------
# the other two workloads (opt-in lines; the headline is workload 3)
# ---------------------------------------------------------------------------
def _setup(a, k: int):
    import torch
    import lattice_inputs as LI
    import paper_2604_09113_gb300 as romb
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    rom_dir = a.rom_dir or tempfile.mkdtemp(prefix="romb_models_")
    t0 = time.time()
    paths = []
    for spec in LI.rom_specs(k):
        path = os.path.join(rom_dir, f"w{k}_family{spec.family}.rom")
        if not os.path.exists(path):
            romb.romb_train_gpu(spec.family, 0, spec.p, spec.r, spec.n_r, spec.lo, spec.hi,
                                LI.lhs(spec.n_s, spec.lo, spec.hi, seed=spec.seed), path)
        paths.append(path)
    train_s = time.time() - t0
    lat = LI.config(k)
    if a.sub:
        lat = LI.sub_lattice(lat, a.sub, a.sub)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    free0 = torch.cuda.mem_get_info(dev)[0]
    ctx = romb.Context(0, 0, stream.cuda_stream)
    for p_ in paths:
        romb.romb_train_load(ctx.h, p_)
    darr = {"ctrl": torch.from_numpy(lat.ctrl).to(dev), "mu": torch.from_numpy(lat.mu).to(dev),
            "family": torch.from_numpy(lat.family).to(dev),
            "traction": torch.from_numpy(lat.traction.reshape(8).copy()).to(dev)}
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device=dev)   # 512 MB > L2
    return dev, stream, ctx, lat, darr, flush, train_s, free0


def _timed(torch, stream, flush, steps: int, fn):
    times, out = [], []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        out.append(r)
    return times, out


def run_workload5(a):
    """256 x 256 cells, p = 8, quartic maps, graded circle holes, rank-80 model,
    split-precision assembly (BF16 form unless --precision says otherwise),
    16 seeded load sets sharing one factorisation; one step = assembly,
    factor, and the 16 solves."""
    import numpy as np
    import torch
    import lattice_inputs as LI
    import paper_2604_09113_gb300 as romb
    dev, stream, ctx, lat, darr, flush, train_s, free0 = _setup(a, 5)
    nrhs = 16
    tr = torch.from_numpy(LI.traction_sets(nrhs, seed=1005).reshape(nrhs, 8)).to(dev)
    nodes = (lat.p * lat.nx + 1) * (lat.p * lat.ny + 1)
    u = torch.zeros((nrhs, nodes, 2), dtype=torch.float64, device=dev)
    forms = {"fp64": romb.ROMB_FP64, "fp32split": romb.ROMB_FP32_SPLIT, "bf16split": romb.ROMB_BF16_SPLIT}
    form = "bf16split" if a.precision == "auto" else a.precision

    def step(pr, k=nrhs):
        romb.romb_assemble(ctx.h, lat, pr, device_arrays=darr)
        romb.romb_factor(ctx.h)
        _, its, rel = romb.romb_bddc_solve(ctx.h, nodes, nrhs=k, traction_sets=tr[:k], rtol=1e-8, maxit=800,
                                          out=u[:k])
        return its.tolist()

    for _ in range(a.warmup):
        step(forms[form])
    torch.cuda.synchronize(dev)
    held = free0 - torch.cuda.mem_get_info(dev)[0]
    clocks = Clocks(0)
    clocks.start()
    times, its = _timed(torch, stream, flush, a.steps, lambda: (step(forms[form]), romb.romb_stats(ctx.h)[0].copy()))
    clk = clocks.stop()
    ms = sum(times) / len(times)
    ph = np.mean(np.array([p for _, p in its]), axis=0)
    names = ["theta", "contraction", "local_factor", "coarse_factor", "pcg", "recovery", "copies", "total"]
    acc = {}
    if not a.no_accuracy:
        ref = None
        for name in ("fp64", "fp32split", "bf16split"):
            step(forms[name], 2)
            v = u[:2].clone()
            if ref is None:
                ref = v
                continue
            acc[f"disp_rel_l2_{name}_vs_fp64"] = [
                (torch.linalg.vector_norm(v[k] - ref[k]) / torch.linalg.vector_norm(ref[k])).item() for k in range(2)]
    line = {"metric": "cells/s assembled+solved at 65,536 cells p=8, 16 load sets sharing one factorisation",
            "value": lat.ncells / (ms / 1e3), "unit": "cells/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32split": "tf32x3+f64", "bf16split": "bf16x10+f64"}[form],
            "data": "synthetic",
            "config": {"workload": "256x256 lattice, p=8, quartic maps, graded circle holes 0.2-0.42, n_r=80",
                       "cells": lat.ncells, "p": lat.p, "assembly_form": form, "load_sets": nrhs,
                       "l2": "flushed (512 MB write) between timed steps", "pcg_rtol": 1e-8},
            "clocks": clk, "pcg_iters": its[-1][0], "phase_ms": {n: float(v) for n, v in zip(names, ph)},
            "device_bytes_held": int(held), "offline_train_s": train_s, "accuracy": acc or None}
    print(json.dumps(line))
    ctx.close()


def run_workload6(a):
    """The paper's benchmark lattice (Sec. 5.1.2, Eq. RES multi map): quarter
    annulus, Schwarz Diamond cells with thresholds 0.9 - 0.8 s, p = 8,
    rho = 5e-4, E = 5, nu = 0.25, clamped at s = 0, traction 0.1 downward at
    s = 1; reduced models with n_k = 2 (16 clusters), n_r = 40, r = 6 and 100
    samples per cluster (Sec. 4.3), trained on the GPU.  One step = assembly,
    factor and solve to 1e-8 (split assembly form unless --precision says
    otherwise), at 2,048 cells (64 x 32) and 16,200 cells (180 x 90), the first
    and fourth rows of Table RES weak (15 and 17 iterations there)."""
    import numpy as np
    import torch
    import lattice_inputs as LI
    import paper_2604_09113_gb300 as romb
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    rom_dir = a.rom_dir or tempfile.mkdtemp(prefix="romb_models_")
    path = os.path.join(rom_dir, "w6_schwarz_d_nk2.rom")
    t0 = time.time()
    if not os.path.exists(path):
        romb.romb_train_gpu_clustered(LI.FAMILY_SCHWARZ_D, 0, 8, 6, 40, 0.1, 0.9, 2,
                                      LI.cluster_samples(100, 0.1, 0.9, 2, seed=2006), path)
    train_s = time.time() - t0
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device=dev)   # 512 MB > L2
    forms = {"fp64": romb.ROMB_FP64, "fp32split": romb.ROMB_FP32_SPLIT, "bf16split": romb.ROMB_BF16_SPLIT}
    form = "fp32split" if a.precision == "auto" else a.precision
    names = ["theta", "contraction", "local_factor", "coarse_factor", "pcg", "recovery", "copies", "total"]
    sizes = {}
    clocks = Clocks(0)
    clocks.start()
    for (nx, ny, paper_its) in ((64, 32, 15), (180, 90, 17)):
        lat = LI.quarter_annulus(nx, ny, p=8)
        nodes = (lat.p * nx + 1) * (lat.p * ny + 1)
        ctx = romb.Context(0, 0, stream.cuda_stream)
        romb.romb_train_load(ctx.h, path)
        darr = {"ctrl": torch.from_numpy(lat.ctrl).to(dev), "mu": torch.from_numpy(lat.mu).to(dev),
                "family": torch.from_numpy(lat.family).to(dev),
                "traction": torch.from_numpy(lat.traction.reshape(8).copy()).to(dev)}
        u = torch.zeros((1, nodes, 2), dtype=torch.float64, device=dev)

        def step(pr):
            romb.romb_assemble(ctx.h, lat, pr, device_arrays=darr)
            romb.romb_factor(ctx.h)
            _, its, rel = romb.romb_bddc_solve(ctx.h, nodes, rtol=1e-8, maxit=500, out=u)
            return int(its[0])

        for _ in range(a.warmup):
            step(forms[form])
        torch.cuda.synchronize(dev)
        times, its = _timed(torch, stream, flush, a.steps, lambda: (step(forms[form]), romb.romb_stats(ctx.h)[0].copy()))
        ms = sum(times) / len(times)
        ph = np.mean(np.array([p_ for _, p_ in its]), axis=0)
        entry = {"cells": lat.ncells, "ms_per_step": ms, "cells_per_s": lat.ncells / (ms / 1e3),
                 "pcg_iters": its[-1][0], "paper_iters": paper_its,
                 "phase_ms": {n: float(v) for n, v in zip(names, ph)}}
        if not a.no_accuracy:
            v = u.clone()
            step(romb.ROMB_FP64)
            entry["disp_rel_l2_vs_fp64"] = (torch.linalg.vector_norm(v - u) / torch.linalg.vector_norm(u)).item()
        sizes[f"{nx}x{ny}"] = entry
        ctx.close()
    clk = clocks.stop()
    big = sizes["180x90"]
    line = {"metric": "cells/s assembled+solved, quarter annulus Schwarz Diamond p=8, 16 clusters",
            "value": big["cells_per_s"], "unit": "cells/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": big["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32split": "tf32x3+f64", "bf16split": "bf16x10+f64"}[form],
            "data": "synthetic",
            "config": {"workload": "quarter annulus (Eq. RES multi map), Schwarz Diamond, thresholds 0.9-0.8s, p=8, "
                                   "n_k=2, n_r=40, r=6", "assembly_form": form,
                       "l2": "flushed (512 MB write) between timed steps", "pcg_rtol": 1e-8},
            "clocks": clk, "sizes": sizes, "offline_train_s": train_s}
    print(json.dumps(line))


def run_workload7(a):
    """The lattice-wrench application (Sec. 5.2.2) on a wrench-like layout:
    a round head with a clamped hole and a handle loaded at its end, cells of
    an 18 x 8 (x scale) grid of which the others are absent, Schoen IWP cells
    with thresholds drawn per cell from [-2.5, 2.5]^4, p = 8, E = 5,
    nu = 0.25, rho = 5e-4; a reduced model with n_k = 2 (16 clusters),
    n_r = 40, r = 6 and 100 samples per cluster, trained on the GPU.  One
    step = assembly, factor and solve to 1e-8, at 90 cells (scale 1) and
    7,290 cells (scale 9), the paper's two wrench lattices (15 and 18
    iterations there, on its own geometry)."""
    import numpy as np
    import torch
    import lattice_inputs as LI
    import paper_2604_09113_gb300 as romb
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    rom_dir = a.rom_dir or tempfile.mkdtemp(prefix="romb_models_")
    path = os.path.join(rom_dir, "w7_schoen_iwp_nk2.rom")
    t0 = time.time()
    if not os.path.exists(path):
        romb.romb_train_gpu_clustered(LI.FAMILY_SCHOEN_IWP, 0, 8, 6, 40, -2.5, 2.5, 2,
                                      LI.cluster_samples(100, -2.5, 2.5, 2, seed=2007), path)
    train_s = time.time() - t0
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device=dev)   # 512 MB > L2
    forms = {"fp64": romb.ROMB_FP64, "fp32split": romb.ROMB_FP32_SPLIT, "bf16split": romb.ROMB_BF16_SPLIT}
    form = "fp32split" if a.precision == "auto" else a.precision
    names = ["theta", "contraction", "local_factor", "coarse_factor", "pcg", "recovery", "copies", "total"]
    sizes = {}
    clocks = Clocks(0)
    clocks.start()
    for scale, paper_its in ((1, 15), (9, 18)):
        lat = LI.wrench(scale, p=8)
        cells = int(lat.present.sum())
        nodes = (lat.p * lat.nx + 1) * (lat.p * lat.ny + 1)
        ctx = romb.Context(0, 0, stream.cuda_stream)
        romb.romb_train_load(ctx.h, path)
        darr = {"ctrl": torch.from_numpy(lat.ctrl).to(dev), "mu": torch.from_numpy(lat.mu).to(dev),
                "family": torch.from_numpy(lat.family).to(dev),
                "traction": torch.from_numpy(lat.traction.reshape(8).copy()).to(dev),
                "present": torch.from_numpy(lat.present.astype(np.uint8)).to(dev),
                "edge_clamped": torch.from_numpy(lat.edge_clamped.astype(np.uint8).reshape(-1)).to(dev)}
        u = torch.zeros((1, nodes, 2), dtype=torch.float64, device=dev)

        def step(pr):
            romb.romb_assemble(ctx.h, lat, pr, device_arrays=darr)
            romb.romb_factor(ctx.h)
            _, its, rel = romb.romb_bddc_solve(ctx.h, nodes, rtol=1e-8, maxit=500, out=u)
            return int(its[0])

        for _ in range(a.warmup):
            step(forms[form])
        torch.cuda.synchronize(dev)
        times, its = _timed(torch, stream, flush, a.steps, lambda: (step(forms[form]), romb.romb_stats(ctx.h)[0].copy()))
        ms = sum(times) / len(times)
        ph = np.mean(np.array([p_ for _, p_ in its]), axis=0)
        _, flags = romb.romb_stats(ctx.h, cells)
        entry = {"cells": cells, "grid": f"{lat.nx}x{lat.ny}", "ms_per_step": ms, "cells_per_s": cells / (ms / 1e3),
                 "pcg_iters": its[-1][0], "paper_iters": paper_its,
                 "exact_fallback_cells": int(np.count_nonzero(flags & 16)),
                 "phase_ms": {n: float(v) for n, v in zip(names, ph)}}
        if not a.no_accuracy:
            v = u.clone()
            step(romb.ROMB_FP64)
            entry["disp_rel_l2_vs_fp64"] = (torch.linalg.vector_norm(v - u) / torch.linalg.vector_norm(u)).item()
        sizes[str(cells)] = entry
        ctx.close()
    clk = clocks.stop()
    big = sizes["7290"]
    line = {"metric": "cells/s assembled+solved, wrench-like layout of Schoen IWP cells, p=8, 16 clusters",
            "value": big["cells_per_s"], "unit": "cells/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": big["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32split": "tf32x3+f64", "bf16split": "bf16x10+f64"}[form],
            "data": "synthetic",
            "config": {"workload": "wrench-like layout (round head with a clamped hole, loaded handle), Schoen IWP, "
                                   "thresholds U[-2.5,2.5]^4 per cell, p=8, n_k=2, n_r=40, r=6",
                       "assembly_form": form, "l2": "flushed (512 MB write) between timed steps", "pcg_rtol": 1e-8},
            "clocks": clk, "sizes": sizes, "offline_train_s": train_s}
    print(json.dumps(line))


def run_workload4(a):
    """The compliance gradient workload: 64 x 64 cells, cubic maps, one hole
    radius per cell, p = 6, rank-40 model; one step = FP64-form assembly,
    factor, solve and the adjoint gradient with respect to every control
    point and radius (device outputs).  Untimed: central differences of the
    compliance along seeded directions against the adjoint gradient."""
    import numpy as np
    import torch
    import lattice_inputs as LI
    import paper_2604_09113_gb300 as romb
    import ctypes
    dev, stream, ctx, lat, darr, flush, train_s, free0 = _setup(a, 4)
    nodes = (lat.p * lat.nx + 1) * (lat.p * lat.ny + 1)
    u = torch.zeros((1, nodes, 2), dtype=torch.float64, device=dev)
    gx = torch.zeros(lat.ctrl.shape, dtype=torch.float64, device=dev)
    gR = torch.zeros(lat.ncells, dtype=torch.float64, device=dev)
    cval = ctypes.c_double()
    ev = {}

    def step(lt=None, darr_=None):
        romb.romb_assemble(ctx.h, lt or lat, romb.ROMB_FP64, device_arrays=darr_ or darr)
        romb.romb_factor(ctx.h)
        romb.romb_bddc_solve(ctx.h, nodes, rtol=1e-12, maxit=1000, out=u)
        ev["g0"] = torch.cuda.Event(enable_timing=True)
        ev["g1"] = torch.cuda.Event(enable_timing=True)
        ev["g0"].record(stream)
        st = romb._lib.romb_compliance_grad(ctx.h, ctypes.byref(cval), ctypes.c_void_p(gx.data_ptr()),
                                            ctypes.c_void_p(gR.data_ptr()), None)
        ev["g1"].record(stream)
        if st != 0:
            raise romb.RombError(st, "romb_compliance_grad")
        return cval.value

    for _ in range(a.warmup):
        step()
    times, gms = [], []
    for _ in range(a.steps):
        t, _ = _timed(torch, stream, flush, 1, step)
        times += t
        gms.append(ev["g0"].elapsed_time(ev["g1"]))
    ms = sum(times) / len(times)
    c0 = step()
    g_ctrl, g_R = gx.cpu().numpy().copy(), gR.cpu().numpy().copy()
    nfd = 20
    V = LI.directions(nfd, lat.ctrl.size + lat.ncells, seed=1000 + 4)
    gnorm = float(np.sqrt((g_ctrl ** 2).sum() + (g_R ** 2).sum()))
    worst, h = 0.0, 2e-5
    for v in V:
        vx, vr = v[:lat.ctrl.size].reshape(lat.ctrl.shape), v[lat.ctrl.size:]
        cs = []
        for sgn in (1, -1):
            lp = LI.Lattice(**{**lat.__dict__, "ctrl": lat.ctrl + sgn * h * vx, "mu": lat.mu + sgn * h * vr[:, None]})
            dp = {"ctrl": torch.from_numpy(lp.ctrl).to(dev), "mu": torch.from_numpy(lp.mu).to(dev),
                  "family": darr["family"], "traction": darr["traction"]}
            cs.append(step(lp, dp))
        fd = (cs[0] - cs[1]) / (2 * h)
        worst = max(worst, abs(fd - ((g_ctrl * vx).sum() + (g_R * vr).sum())) / gnorm)
    line = {"metric": "compliance gradients/s at 4,096 cells p=6 (adjoint, all control points and radii)",
            "value": 1e3 / ms, "unit": "gradients/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "64x64 lattice, p=6, cubic maps, circle hole radius per cell, n_r=40",
                       "cells": lat.ncells, "control_points": len(lat.ctrl), "pcg_rtol": 1e-12,
                       "l2": "flushed (512 MB write) between timed steps",
                       "step": "FP64 assembly + factor + solve + adjoint gradient"},
            "grad_ms": float(np.mean(gms)), "compliance": c0,
            "fd_check": {"directions": nfd, "h": h, "worst_abs_err_over_grad_norm": worst},
            "offline_train_s": train_s}
    print(json.dumps(line))
    ctx.close()


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle on a bounded sample
# ---------------------------------------------------------------------------
def run_reference(a):
    """The oracle on the host cores: every step runs one 16 x 16 tile of the
    workload per core, concurrently (independent sub-problems, oracle-trained
    models; training is not timed)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    paths = oracle_models(train=True, small=a.small_models)
    nproc = os.cpu_count() or 1
    with spawn_pool(nproc) as pool:
        for _ in range(max(1, min(a.warmup, 1))):
            oracle_tiles_seconds(pool, paths, nproc, SAMPLE_NX)
        times = []
        for _ in range(a.steps):
            t, cells = oracle_tiles_seconds(pool, paths, nproc, SAMPLE_NX)
            times.append(t)
    s = sum(times) / len(times)
    v = cells / s
    sample = (f"{nproc} independent {SAMPLE_NX}x{SAMPLE_NY} tiles of the workload per step ({cells} cells), one "
              f"single-threaded oracle process per core; oracle-trained models"
              + (" (reduced: 80 samples, r = 2, format check only)" if a.small_models else ""))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "cells/s", "n_gpus": 1, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "132x132 lattice, p=6, quartic maps, circle/cross 50/50, n_r=60 per family",
                       "sample": sample},
            "cpu_baseline": {"value": v, "unit": "cells/s", "cores": nproc, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
            "e2e": {"value": v, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    a = args_parse()
    if a.cpu_sample_json:
        cpu_sample(a.rom_dir, a.cpu_sample_json)
        return
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == 5:
        run_workload5(a)
    elif a.workload == 4:
        run_workload4(a)
    elif a.workload == 6:
        run_workload6(a)
    elif a.workload == 7:
        run_workload7(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
