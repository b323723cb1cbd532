#!/usr/bin/env python
"""Benchmark of the docking hot path on GB300.

One step = one complete docking of the paper-scale workload through adg_dock:
64^3 FP32 maps (9) of a 3,000-atom pseudo-receptor, one ligand of 40 heavy
atoms + 4 polar H with 8 torsions, 100 LGA runs x population 150 x 2.5M
evaluations per run, ADADELTA local search (300 iterations) on analytic
gradients.  Metric: energy(+gradient) evaluations per second (and docked
ligands per second) on 1 GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank docks its own
ligand (replicas; no data-path collective), value = all ranks' evaluations /
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import functools
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "energy+gradient evals/s and docked ligands/s on 1 GB300 vs plain form, at tol"
UNIT = "evals/s"
SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ_FALLBACK = 2070.0


# ---------------------------------------------------------------- algorithmic work per evaluation
def flops_per_eval(natoms: int, npairs: int, sum_moving: int, grad: bool) -> float:
    """Per-unit algorithmic FP32 work of one evaluation (FMA = 2 flops; MUFU
    ops not counted): pose 18 (N + sum|S_k|), intermolecular 130 N,
    intramolecular 55 P, gradient reductions 9 (N + sum|S_k|) (energy+gradient only)."""
    f = 18.0 * (natoms + sum_moving) + 130.0 * natoms + 55.0 * npairs
    if grad:
        f += 9.0 * (natoms + sum_moving)
    return f


def fp32_peak_tflops() -> tuple[float, str]:
    mhz = SM_MAX_MHZ_FALLBACK
    src = "recipe max SM clock"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
            src = "MEASURED_PEAKS.json sm_max_mhz"
    except Exception:
        pass
    return SM_COUNT * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12, src


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self) -> dict:
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [l.split(",") for l in open(self.path) if l.strip()]
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if sm:
            sm.sort()
            out.update(sm_mhz=sm[len(sm) // 2], sm_max_mhz=max(mx), reasons=sorted(reasons), samples=len(sm))
        return out


# ---------------------------------------------------------------- CPU oracle (baseline / reference arm)
def _oracle_worker(args):
    maps_path, nev, run = args
    import numpy as np
    import oracle as O
    from paper_2007_03678_gb300 import synth as S
    grid, rec, lig = S.workload_inputs(S.PAPER)
    maps = np.load(maps_path)
    p = O.SearchParams(nrun=1, pop_size=S.PAPER["pop"], nev=nev, ls_method=2)
    t0 = time.perf_counter()
    best, _, evals, gens, _ = O.lga_run(S.forcefield(), grid, maps, O.Ligand(lig), p, run=run)
    return evals, time.perf_counter() - t0


def oracle_sample(nev: int, cores: int, maps_path: str, run0: int = 0) -> dict:
    """Run `cores` single-threaded oracle LGA runs of the paper-scale ligand in
    parallel (spawned processes), each until `nev` evaluations; return the
    aggregate evaluation rate."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(cores) as pool:
        t0 = time.perf_counter()
        out = pool.map(_oracle_worker, [(maps_path, nev, run0 + i) for i in range(cores)])
        wall = time.perf_counter() - t0
    evals = sum(e for e, _ in out)
    return dict(evals=evals, wall=wall, rate=evals / wall)


def _oracle_plain_worker(args):
    maps_path, run = args
    import numpy as np
    import oracle as O
    from paper_2007_03678_gb300 import synth as S
    grid, rec, lig = S.workload_inputs(S.PLAIN)
    maps = np.load(maps_path)
    p = O.SearchParams(nrun=1, pop_size=S.PLAIN["pop"], nev=S.PLAIN["nev"], ls_method=1)
    best, _, evals, gens, _ = O.lga_run(S.forcefield(), grid, maps, O.Ligand(lig), p, run=run)
    return evals


def _oracle_diff_worker(args):
    maps_path, specs = args
    import numpy as np
    import oracle as O
    from paper_2007_03678_gb300 import synth as S
    grid = S.make_grid(S.PAPER["grid_n"])
    maps = np.load(maps_path)
    ff = S.forcefield()
    n = 0
    for n_heavy, n_tors, seed, i in specs:
        lig = S.make_ligand(n_heavy, n_tors, seed)
        genes = S.random_genes(lig, 256, grid, 40000 + i, spread=0.3).astype(np.float32).astype(np.float64)
        O.score(ff, grid, maps, O.Ligand(lig), genes)
        n += len(genes)
    return n


def oracle_other_configs(cores: int, paper_maps_path: str, diff_specs) -> dict:
    """The FP64 oracle on the plain config (its 10 runs as 10 parallel
    single-thread processes) and on the differentiation workload (energy +
    gradient of its 65,536 poses, ligands spread over `cores` processes;
    ligand set-up included in the time)."""
    import multiprocessing as mp
    import numpy as np
    import oracle as O
    from paper_2007_03678_gb300 import synth as S
    grid, rec, lig = S.workload_inputs(S.PLAIN)
    fd, plain_path = tempfile.mkstemp(suffix=".npy")
    os.close(fd)
    np.save(plain_path, O.maps_build(S.forcefield(), grid, rec).astype(np.float32).astype(np.float64))
    try:
        nrun = S.PLAIN["nrun"]
        with mp.get_context("spawn").Pool(min(cores, nrun)) as pool:
            pool.map(_oracle_plain_worker, [(plain_path, 0)])  # warm the workers' imports
            t0 = time.perf_counter()
            evals = sum(pool.map(_oracle_plain_worker, [(plain_path, r) for r in range(nrun)]))
            t_plain = time.perf_counter() - t0
        chunks = [diff_specs[i::cores] for i in range(cores)]
        with mp.get_context("spawn").Pool(cores) as pool:
            pool.map(_oracle_diff_worker, [(paper_maps_path, [])] * cores)
            t0 = time.perf_counter()
            poses = sum(pool.map(_oracle_diff_worker, [(paper_maps_path, c) for c in chunks]))
            t_diff = time.perf_counter() - t0
    finally:
        os.unlink(plain_path)
    return {"plain_config": {"ligands_per_s": 1.0 / t_plain, "evals_per_s": evals / t_plain, "seconds": t_plain,
                             "cores": min(cores, nrun),
                             "sample": f"the whole plain config: {nrun} single-thread oracle LGA runs in parallel"},
            "differentiation": {"poses_per_s": poses / t_diff, "seconds": t_diff, "cores": cores,
                                "sample": f"all {poses} poses of the differentiation workload, energy + gradient"}}


def oracle_maps_file() -> str:
    import numpy as np
    import oracle as O
    from paper_2007_03678_gb300 import synth as S
    grid, rec, lig = S.workload_inputs(S.PAPER)
    maps = O.maps_build(S.forcefield(), grid, rec).astype(np.float32).astype(np.float64)
    fd, path = tempfile.mkstemp(suffix=".npy")
    os.close(fd)
    np.save(path, maps)
    return path


ORACLE_SAMPLE_NEV = 150 + 45150  # initial population + one ADADELTA generation
BATCH_LIGANDS, BATCH_NRUN, BATCH_NEV = 256, 20, 100_000


def cpu_cores() -> int:
    return max(1, min(os.cpu_count() or 1, 16))


def run_reference(args, rank: int) -> None:
    if rank != 0:
        return
    cores = cpu_cores()
    maps_path = oracle_maps_file()
    try:
        for w in range(args.warmup):
            oracle_sample(150 + 1500, cores, maps_path)
        rates, walls, evals = [], [], 0
        for s in range(args.steps):
            r = oracle_sample(ORACLE_SAMPLE_NEV, cores, maps_path, run0=s * cores)
            walls.append(r["wall"])
            evals += r["evals"]
        value = evals / sum(walls)
    finally:
        os.unlink(maps_path)
    sample = (f"{cores} parallel single-thread oracle LGA runs of the paper-scale ligand per step, "
              f"each stopped after {ORACLE_SAMPLE_NEV} evaluations (initial population + 1 ADADELTA generation)")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(walls) / len(walls), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def workload_config(nrun=None, nev=None) -> dict:
    from paper_2007_03678_gb300 import synth as S
    w = dict(S.PAPER)
    w["nrun"] = nrun or w["nrun"]
    w["nev"] = nev or w["nev"]
    return {"workload": "paper-scale docking: 64^3 x 9 FP32 maps (0.375 A) of a 3000-atom pseudo-receptor, "
                        "one ligand of 40 heavy atoms + 4 polar H with 8 torsions, "
                        f"{w['nrun']} LGA runs x pop 150 x {w['nev']:,} evals, ADADELTA local search",
            "grid": w["grid_n"], "receptor_atoms": w["rec_atoms"], "ligand_atoms": w["n_heavy"] + w["n_hd"],
            "torsions": w["n_tors"], "nrun": w["nrun"], "pop": w["pop"], "nev": w["nev"], "local_search": "adadelta",
            "l2": "flushed between steps (256 MB write); maps (58.7 MB packed) are meant to stay L2-resident within a step",
            "parallelism": "replicas"}


TRIAGE_TRAIN, TRIAGE_STREAM = 4000, 20000
# Figures of the generation kernel taken from ncu captures, valid only for
# the kernel source they were taken on: the bench reports them only while
# the SHA-256 (first 16 hex digits) of adg_kernels.cu + adg_internal.h
# equals `source_sha16`, and null otherwise.  The same hash heads the capture
# summaries under profiles/.
#   traffic_bytes: DRAM bytes (read + write) per generation of all 100 runs
#     (both launches), from
#     ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum --clock-control none
#         -k regex:k_dock_generation -s 60 -c 2 python bench.py --steps 1 --warmup 3 --no-cpu-baseline
#         --no-e2e --no-batching --no-triage --no-graphs
#   l1_pipe_frac: the L1 / shared-memory data pipe's share of its peak
#     (l1tex__data_pipe_lsu_wavefronts.avg.pct_of_peak_sustained_elapsed) in
#     the full-section capture of one launch.
GEN_CAPTURE = {"source_sha16": "7f8f4d03637f8cfc", "traffic_bytes": 36.42e6, "l1_pipe_frac": 0.676}


def kernel_source_sha16() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("adg_kernels.cu", "adg_internal.h"):
        with open(os.path.join(ROOT, "paper_2007_03678_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def gen_capture_figures() -> tuple:
    """(traffic bytes, L1-pipe fraction) of the generation kernel if the
    captures were taken on the current kernel source, else (None, None)."""
    if GEN_CAPTURE["source_sha16"] != kernel_source_sha16():
        return None, None
    return GEN_CAPTURE["traffic_bytes"], GEN_CAPTURE["l1_pipe_frac"]


def run_mlp_inference(ctx, rows=1_000_000, reps=10):
    """Triage-network inference throughput on `rows` random feature rows, for
    both engines (tcgen05 with tensor-memory accumulators, and warp-level
    MMAs); device-timed, mean of `reps` launches."""
    import json as _json
    import numpy as np
    import torch
    from paper_2007_03678_gb300 import adg
    nin = 26
    net = adg.MLP(ctx, nin, seed=1)
    net.set_norm(np.zeros(nin), np.ones(nin), 0.0, 1.0)
    x = torch.randn(rows, nin, device=f"cuda:{ctx.device}")
    flops = 2.0 * rows * (32 * 256 + 256 * 256 + 256)  # input width padded to 32 on the tensor cores
    out = {"rows": rows, "network": f"{nin}-256-256-1, BF16 weights / FP32 accumulate", "flops_per_call": flops}
    peak = None
    try:
        peak = float(_json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                  "MEASURED_PEAKS.json")))["bf16_tflops"])
    except Exception:
        pass
    for eng, name in ((adg.MLP_TCGEN05, "tcgen05"), (adg.MLP_MMA_SYNC, "mma_sync")):
        net.set_engine(eng)
        for _ in range(3):
            net.forward(x)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            net.forward(x)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms": ms, "tflops": flops / ms / 1e9,
                     "frac_of_bf16_peak": (flops / ms / 1e9 / peak) if peak else None}
    net.check()
    net.close()
    return out


def run_mlp_training(ctx, rows=65536, reps=10):
    """Triage-network gradient (forward, backward, weight gradients) on `rows`
    random rows for both engines; device-timed, mean of `reps` calls."""
    import numpy as np
    import torch
    from paper_2007_03678_gb300 import adg
    nin = 26
    net = adg.MLP(ctx, nin, seed=2)
    net.set_norm(np.zeros(nin), np.ones(nin), 0.0, 1.0)
    x = torch.randn(rows, nin, device=f"cuda:{ctx.device}")
    t = torch.randn(rows, device=f"cuda:{ctx.device}")
    # forward (two layers, K padded to 32), dh1 = dh2 W2, dW2 and dW1
    flops = 2.0 * rows * (32 * 256 + 256 * 256) + 2.0 * rows * 256 * 256 + 2.0 * rows * (256 * 256 + 256 * 32)
    out = {"rows": rows, "flops_per_call": flops}
    for eng, name in ((adg.MLP_TCGEN05, "tcgen05"), (adg.MLP_MMA_SYNC, "mma_sync")):
        net.set_engine(eng)
        for _ in range(3):
            net.grad(x, t)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            net.grad(x, t)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms": ms, "tflops": flops / ms / 1e9}
    net.check()
    net.close()
    return out


def run_plain_config(ctx, ff, reps=5):
    """The plain configuration: 40^3 maps of a 600-atom pseudo-receptor, one
    16+2-atom ligand with 3 torsions, 10 runs x pop 150 x 50,000 evals,
    Solis-Wets.  Device-timed per docking call (best of `reps`)."""
    import numpy as np
    import torch
    from paper_2007_03678_gb300 import adg, synth as S
    grid, rec, lig = S.workload_inputs(S.PLAIN)
    maps = adg.maps_build(ctx, ff, grid, rec)
    R = adg.Receptor(ctx, grid, maps)
    L = adg.Ligand(ctx, ff, lig)
    p = adg.search_params(nrun=S.PLAIN["nrun"], pop_size=S.PLAIN["pop"], nev=S.PLAIN["nev"],
                          ls_method=adg.LS_SOLIS_WETS, seed=S.SEARCH_SEED)
    adg.dock(ctx, R, L, p)
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        r = adg.dock(ctx, R, L, p)[0]
        e1.record(ctx.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    ev = int(r["evals"].sum())
    return {"workload": "plain: 40^3 maps, 600-atom pseudo-receptor, 16+2 atoms, 3 torsions, 10 runs x 150 x "
                        "50,000 evals, Solis-Wets", "evals_per_s": ev / (best / 1e3), "ligands_per_s": 1e3 / best,
            "ms_per_ligand": best, "best_energy_median": float(np.median(r["best_energy"]))}


@functools.lru_cache(maxsize=1)
def differentiation_ligands():
    """The differentiation workload's 256 seeded ligands (20-50 atoms, 2-12
    torsions) and the (heavy atoms, torsions, seed, index) that make each."""
    import numpy as np
    from paper_2007_03678_gb300 import synth as S
    rng = np.random.default_rng(2024)
    specs, ligs, seed = [], [], 30000
    while len(ligs) < 256:
        seed += 1
        n_heavy, n_tors = int(rng.integers(18, 46)), int(rng.integers(2, 13))
        try:
            lig = S.make_ligand(n_heavy, n_tors, seed)
        except RuntimeError:
            continue
        if 20 <= lig.natoms <= 50:
            specs.append((n_heavy, n_tors, seed, len(ligs)))
            ligs.append(lig)
    return specs, ligs


def run_differentiation(ctx, R, ff, reps=5):
    """65,536 random poses across 256 ligands (20-50 atoms, 2-12 torsions):
    energy + gene gradient through torch.autograd, forward and backward,
    device-timed (best of `reps`): all ligands in one batched call
    (adg_score_multi, one launch per atoms-per-lane width), and, for
    comparison, one call per ligand."""
    import numpy as np
    import torch
    from paper_2007_03678_gb300 import adg, synth as S
    from paper_2007_03678_gb300.autograd import score, score_batch, score_rows
    specs, ligs = differentiation_ligands()
    grid = S.make_grid(S.PAPER["grid_n"])
    L = [adg.Ligand(ctx, ff, l) for l in ligs]
    X = [torch.from_numpy(S.random_genes(l, 256, grid, 40000 + i, spread=0.3).astype(np.float32)).cuda()
         for i, l in enumerate(ligs)]

    def timed(step):
        best = None
        for _ in range(reps + 1):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            step()
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        return best

    npose = [x.shape[0] for x in X]
    rows = torch.cat([torch.nn.functional.pad(x, (0, adg.MAX_GENES - x.shape[1])) for x in X], 0)

    def packed():
        rows.requires_grad_(True)
        score_rows(rows, ctx, R, L, npose).sum().backward()
        rows.grad = None

    def batched():
        xs = [x.requires_grad_(True) for x in X]
        torch.stack([e.sum() for e in score_batch(xs, ctx, R, L)]).sum().backward()
        for x in xs:
            x.grad = None

    def per_ligand():
        for Lg, x in zip(L, X):
            x.requires_grad_(True)
            score(x, ctx, R, Lg).sum().backward()
            x.grad = None

    ms_rows = timed(packed)
    ms_batch = timed(batched)
    ms_each = timed(per_ligand)
    for Lg in L:
        Lg.close()
    return {"workload": "65,536 poses over 256 ligands (20-50 atoms, 2-12 torsions), energy + gene gradient, "
                        "forward + backward through torch.autograd", "poses_per_s": 65536 / (ms_rows / 1e3),
            "ms": ms_rows, "calls": "packed rows [65536, 23], one autograd call (adg_score_multi)",
            "list_of_tensors": {"poses_per_s": 65536 / (ms_batch / 1e3), "ms": ms_batch,
                                "calls": "256 per-ligand tensors padded and concatenated inside autograd"},
            "per_ligand_calls": {"poses_per_s": 65536 / (ms_each / 1e3), "ms": ms_each}}


def run_batching_full(ctx, R, ff, nlig=4096, nrun=20, nev=1_000_000):
    """The full batching configuration in one adg_dock call (the ligand
    groups' graphs on concurrent streams), after one short call that tunes
    every shape bucket.  Host-timed around the one call."""
    import torch
    from paper_2007_03678_gb300 import adg, synth as S
    t0 = time.perf_counter()
    bl = S.make_batch(nlig, seed=7, workers=0)
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    L = [adg.Ligand(ctx, ff, l) for l in bl]
    t_setup = time.perf_counter() - t0
    p = adg.search_params(nrun=nrun, pop_size=150, nev=nev, ls_method=adg.LS_ADADELTA, seed=S.SEARCH_SEED)
    wp = adg.search_params(nrun=1, pop_size=150, nev=600, ls_method=adg.LS_ADADELTA, seed=S.SEARCH_SEED)
    adg.dock(ctx, R, L, wp)
    ctx.stats(reset=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = adg.dock(ctx, R, L, p)
    dt = time.perf_counter() - t0
    ev = int(sum(r["evals"].sum() for r in res))
    out = {"workload": f"batching: {nlig} seeded ligands, {nrun} runs x 150 x {nev:,} evals, ADADELTA, "
                       "one adg_dock call", "seconds": dt, "ligands_per_s": nlig / dt,
           "evals_per_s": ev / dt, "evals": ev, "groups": ctx.stats()["dock_groups"],
           "ligand_setup_s": t_setup, "ligand_generation_s": t_gen,
           "atoms": [min(l.natoms for l in bl), max(l.natoms for l in bl)],
           "torsions": [min(len(l.tors) for l in bl), max(len(l.tors) for l in bl)]}
    for lg in L:
        lg.close()
    return out


def run_triage(ctx, R, ff):
    """Learned triage against the plain path on a seeded stream: the network
    is trained on full dockings of a training set, then the stream is docked
    both ways (plain: full search of every ligand; triaged: early search of
    every ligand, full search of the survivors).  Host-timed end to end.
    Recall of the plain path's top 1 % is reported with its 95 % Wilson
    interval, beside the same survival fraction chosen by the early energy
    alone (no network) and at other survival fractions."""
    import numpy as np
    from paper_2007_03678_gb300 import adg, synth as S, triage as T
    cfg = T.TriageConfig()
    t0 = time.perf_counter()
    lt, ls = S.make_batch(TRIAGE_TRAIN, seed=101, workers=0), S.make_batch(TRIAGE_STREAM, seed=202, workers=0)
    t_gen = time.perf_counter() - t0
    LT = [adg.Ligand(ctx, ff, l) for l in lt]
    LS = [adg.Ligand(ctx, ff, l) for l in ls]
    T.assign_stream_ids(LT, 1_000_000)
    T.assign_stream_ids(LS, 2_000_000)
    y_tr, x_tr, ev_tr, t_tr = T.dock_full(ctx, R, LT, cfg)
    tri = T.Triage(ctx, cfg, seed=3)
    t0 = time.perf_counter()
    tri.fit(x_tr, y_tr)
    t_fit = time.perf_counter() - t0
    T.dock_early(ctx, R, LS[:8], cfg)  # warm-up of the early geometry
    y_st, x_st, ev_plain, t_plain = T.dock_full(ctx, R, LS, cfg)
    out = T.screen(ctx, R, LS, tri)
    keep = out["keep"]
    hits, ntop = T.recall_counts(y_st, keep, cfg.top_frac)
    keep_early = T.early_rule_survivors(x_st, cfg)
    hits_e, _ = T.recall_counts(y_st, keep_early, cfg.top_frac)
    pred = tri.predict(x_st)
    curve = {}
    for frac in (0.05, 0.10, 0.20):
        kn, ke = T.keep_best(pred, frac), T.keep_best(x_st[:, adg.NDESC + cfg.early_gen - 1], frac)
        curve[str(frac)] = {"network": T.recall(y_st, kn, cfg.top_frac), "early_energy": T.recall(y_st, ke, cfg.top_frac)}
    for l in LT + LS:
        l.close()
    return {"train_ligands": TRIAGE_TRAIN, "stream_ligands": TRIAGE_STREAM,
            "search": {"nrun": cfg.nrun, "pop": cfg.pop, "generations": cfg.max_gen, "early_generations": cfg.early_gen,
                       "local_search": "adadelta", "ls_max_iters": cfg.ls_max_iters},
            "network": f"{cfg.nin}-256-256-1 ReLU, BF16 weights / FP32 accumulate, ensemble of {tri.folds}",
            "ligands_per_s_plain": TRIAGE_STREAM / t_plain, "ligands_per_s_triaged": TRIAGE_STREAM / out["seconds"],
            "speedup": t_plain / out["seconds"], "recall_top1pct": hits / ntop, "top1pct_ligands": ntop,
            "recall_top1pct_ci95_wilson": list(T.wilson_interval(hits, ntop)),
            "recall_top1pct_early_energy_rule": hits_e / ntop,
            "recall_top1pct_early_energy_rule_ci95_wilson": list(T.wilson_interval(hits_e, ntop)),
            "network_vs_early_rule_mcnemar": T.mcnemar_exact(y_st, keep, keep_early, cfg.top_frac),
            "recall_by_survivor_fraction": curve,
            "survivors": float(keep.mean()), "evals_ratio": out["evals"] / ev_plain,
            "survivors_match_plain": bool(np.array_equal(out["energy"][keep], y_st[keep])),
            "seconds": {"ligand_generation": t_gen, "train_docking": t_tr, "fit": t_fit, "plain": t_plain,
                        "triaged": out["seconds"], "early": out["seconds_early"], "full_survivors": out["seconds_full"]},
            "sample": f"seeded stand-in for the 10^6-ligand stream: {TRIAGE_TRAIN:,} training and {TRIAGE_STREAM:,} "
                      f"stream ligands (heavy atoms 10-60, torsions 0-15); search {cfg.nrun} runs x {cfg.pop} x "
                      f"{cfg.max_gen} generations of ADADELTA ({cfg.ls_max_iters} iterations), early search "
                      f"= the first {cfg.early_gen} generations"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end pass (profiling runs)")
    ap.add_argument("--no-batching", action="store_true", help="skip the batching comparison (profiling runs)")
    ap.add_argument("--no-triage", action="store_true", help="skip the learned-triage screen")
    ap.add_argument("--no-graphs", action="store_true",
                    help="host-driven generation loop (kernel profilers cannot see kernels in conditional graphs)")
    ap.add_argument("--nrun", type=int, default=None, help="override the run count (small profiling cases)")
    ap.add_argument("--nev", type=int, default=None, help="override the evaluation budget (small profiling cases)")
    ap.add_argument("--mlp-only", action="store_true",
                    help="instead of the bench line: the triage network's inference and training throughput only "
                         "(profiling runs)")
    ap.add_argument("--no-batching-full", action="store_true",
                    help="skip the full batching configuration (4,096 seeded ligands of 10-60 heavy atoms and 0-15 "
                         "torsions, 20 runs x 150 x 1,000,000 evals, ADADELTA, one adg_dock call; ~5 min)")
    args = ap.parse_args()
    if args.mlp_only:
        from paper_2007_03678_gb300 import adg, build
        build.build()
        ctx = adg.Context(0)
        print(json.dumps({"mlp_inference": run_mlp_inference(ctx), "mlp_training": run_mlp_training(ctx)}), flush=True)
        ctx.close()
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import numpy as np
    import torch
    from paper_2007_03678_gb300 import adg, build, synth as S
    from paper_2007_03678_gb300.replicas import reduce_run

    build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        # the other workloads (batching, triage, the triage network, the plain
        # configuration, differentiation) are single-GPU measurements reported
        # from the one-GPU run; replicas time the paper-scale docking only
        args.no_batching = args.no_triage = args.no_batching_full = True
    ff = S.forcefield()
    w = S.PAPER
    grid, rec, lig_desc = S.workload_inputs(w, lig_index=rank)
    stream = torch.cuda.Stream()
    ctx = adg.Context(local, stream=stream)
    if args.no_graphs:
        ctx.set_graphs(False)
    maps = adg.maps_build(ctx, ff, grid, rec)
    R = adg.Receptor(ctx, grid, maps)
    ctx.sync()
    del maps
    L = adg.Ligand(ctx, ff, lig_desc)
    nrun = args.nrun or w["nrun"]
    nev = args.nev or w["nev"]
    p = adg.search_params(nrun=nrun, pop_size=w["pop"], nev=nev, ls_method=adg.LS_ADADELTA,
                          seed=S.SEARCH_SEED, lig_id=rank)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")

    for _ in range(args.warmup):
        adg.dock(ctx, R, L, p)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    ctx.stats(reset=True)
    ctx.set_timing(True)
    step_ms, evals, results = [], 0, None
    barrier()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            results = adg.dock(ctx, R, L, p)[0]
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            evals += int(results["evals"].sum())
    barrier()
    ctx.set_timing(False)
    st = ctx.stats(reset=True)
    total_ms, evals = reduce_run(sum(step_ms), evals, dist, device=f"cuda:{local}")
    value = evals / (total_ms / 1e3)
    ligands_per_s = world * args.steps / (total_ms / 1e3)

    # roofline of the dominant kernel (the GA-generation kernel: selection + ADADELTA).  One
    # generation of the 100 runs is two concurrent launches of 50 runs each (the library docks
    # one ligand's runs as concurrent halves); the figures are per generation of all runs.
    gens = int(results["generations"][0])
    iters = p.ls_max_iters
    f_eg = flops_per_eval(L.natoms, L.npairs, L.sum_moving, True)
    f_e = flops_per_eval(L.natoms, L.npairs, L.sum_moving, False)
    gen_flops_per_step = p.nrun * gens * ((p.pop_size - 1) * f_e + p.pop_size * iters * f_eg)
    gen_ms = st["gen_kernel_ms"] / max(1, st["gen_timed"])
    flops_per_gen = gen_flops_per_step / gens
    achieved = flops_per_gen / (gen_ms / 1e3) / 1e12
    peak, peak_src = fp32_peak_tflops()
    traffic, l1_frac = gen_capture_figures()
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_unit": "bytes per generation of all runs (dram read + write)",
                "l1_shared_pipe_frac_ncu": l1_frac, "kernel_source_sha16": kernel_source_sha16(),
                "kernel": "k_dock_generation<2,ADADELTA>",
                "generation_ms": gen_ms, "flops_per_generation": flops_per_gen,
                "gen_share_of_step": st["gen_kernel_ms"] / total_ms if world == 1 else None,
                "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {peak_src}"}

    # the same kernel against its three unit limits as measured on this GPU
    # (FP32 flops, special-function results, L2 random gathers), after the
    # timed region; the binding one is the evaluation's roofline
    if rank == 0:
        pk = adg.probe_peaks(ctx)
        evals_per_gen = p.nrun * ((p.pop_size - 1) + p.pop_size * iters)
        # per pair two exponentials (ex2) and one rsqrt and one reciprocal (rsqrt rate)
        per_eval = {"flops": flops_per_gen / evals_per_gen, "mufu": 4.0 * L.npairs,
                    "l2_bytes": 96.0 * L.natoms}
        t_unit = {"fp32": per_eval["flops"] / (pk["fp32_tflops"] * 1e12),
                  "mufu": 2.0 * L.npairs / (pk["mufu_gops"] * 1e9) + 2.0 * L.npairs / (pk["mufu_rsqrt_gops"] * 1e9),
                  "l2_gather": per_eval["l2_bytes"] / (pk["l2_gather_gbs"] * 1e9)}
        binding = max(t_unit, key=t_unit.get)
        limit = 1.0 / t_unit[binding]
        got = evals_per_gen / (gen_ms / 1e3)
        roofline["measured_units"] = {
            "fp32_tflops": pk["fp32_tflops"], "fp32_scalar_tflops": pk["fp32_scalar_tflops"],
            "fp32x2_tflops": pk["fp32x2_tflops"], "mufu_ex2_gops": pk["mufu_gops"],
            "mufu_rsqrt_gops": pk["mufu_rsqrt_gops"],
            "l2_gather_gbs": pk["l2_gather_gbs"], "gather_buffer_bytes": pk["gather_bytes"],
            "frac_of_measured_fp32": achieved / pk["fp32_tflops"],
            "per_eval": per_eval, "binding_unit": binding, "evals_per_s_limit": limit,
            "evals_per_s_kernel": got, "frac_of_limit": got / limit}

    # end to end through the public API with host buffers: ligand upload + dock + results read back
    ctx.stats(reset=True)
    e2e_t, e2e_evals = 1e-30, 0
    for _ in range(0 if args.no_e2e else args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Lh = adg.Ligand(ctx, ff, lig_desc)
        r = adg.dock(ctx, R, Lh, p)[0]
        Lh.close()
        e2e_t += time.perf_counter() - t0
        e2e_evals += int(r["evals"].sum())
    st2 = ctx.stats(reset=True)
    e2e = None if args.no_e2e else {
        "value": e2e_evals / e2e_t * (world if dist is not None else 1), "unit": UNIT,
        "h2d_bytes_per_step": st2["h2d_bytes"] // args.steps, "d2h_bytes_per_step": st2["d2h_bytes"] // args.steps,
        "ligands_per_s": args.steps / e2e_t * world}

    # batching (shape classes on concurrent streams, one graph each) against one call per ligand
    batching = None
    if not args.no_batching:
        bl = S.make_batch(BATCH_LIGANDS, seed=7, workers=0)
        BL = [adg.Ligand(ctx, ff, l) for l in bl]
        bp = adg.search_params(nrun=BATCH_NRUN, pop_size=150, nev=BATCH_NEV, ls_method=adg.LS_ADADELTA,
                               seed=S.SEARCH_SEED)
        # warm-up of every path; tunes the launch geometry of every shape bucket once
        wp = adg.search_params(nrun=1, pop_size=150, nev=600, ls_method=adg.LS_ADADELTA, seed=S.SEARCH_SEED)
        ctx.stats(reset=True)
        t0 = time.perf_counter()
        adg.dock(ctx, R, BL, wp)
        t_tune = time.perf_counter() - t0
        tune_launches = ctx.stats()["tune_launches"]
        torch.cuda.synchronize()
        ctx.stats(reset=True)
        t0 = time.perf_counter()
        rb = adg.dock(ctx, R, BL, bp)
        t_batch = time.perf_counter() - t0
        groups = ctx.stats()["dock_groups"]
        ctx.set_geometry(adg.GEO_HEURISTIC)  # the same batch under the fixed launch rule
        adg.dock(ctx, R, BL, wp)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        adg.dock(ctx, R, BL, bp)
        t_fixed = time.perf_counter() - t0
        ctx.set_geometry(adg.GEO_TUNED)
        t0 = time.perf_counter()
        for i, lg in enumerate(BL):
            bp.lig_id = i
            adg.dock(ctx, R, lg, bp)
        t_one = time.perf_counter() - t0
        ev = int(sum(r["evals"].sum() for r in rb))
        batching = {"ligands": BATCH_LIGANDS, "atoms": [min(l.natoms for l in bl), max(l.natoms for l in bl)],
                    "nrun": BATCH_NRUN, "pop": 150, "nev": BATCH_NEV, "local_search": "adadelta",
                    "ligands_per_s_batched": BATCH_LIGANDS / t_batch,
                    "ligands_per_s_one_by_one": BATCH_LIGANDS / t_one, "speedup": t_one / t_batch,
                    "ligands_per_s_batched_fixed_rule": BATCH_LIGANDS / t_fixed,
                    "evals_per_s_batched": ev / t_batch, "groups": groups,
                    "tuning": {"buckets": len(ctx.tuned()), "launches": tune_launches,
                               "first_call_s": round(t_tune, 3)}}

    triage = mlp = None
    if not args.no_triage:
        triage = run_triage(ctx, R, ff)
        mlp = run_mlp_inference(ctx)
        mlp["training"] = run_mlp_training(ctx)
    plain = differentiation = batching_full = None
    if not args.no_batching:
        plain = run_plain_config(ctx, ff)
        differentiation = run_differentiation(ctx, R, ff)
    if not args.no_batching_full:
        batching_full = run_batching_full(ctx, R, ff)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = cpu_cores()
        path = oracle_maps_file()
        try:
            r = oracle_sample(ORACLE_SAMPLE_NEV, cores, path)
            others = oracle_other_configs(cores, path, differentiation_ligands()[0])
        finally:
            os.unlink(path)
        cpu = {"value": r["rate"], "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{cores} parallel single-thread oracle LGA runs of the paper-scale ligand, each stopped "
                         f"after {ORACLE_SAMPLE_NEV} evaluations ({r['evals']} evals in {r['wall']:.1f} s)",
               "other_configs": others}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(args.nrun, args.nev), "ligands_per_s": ligands_per_s,
                "best_energy_median": float(np.median(results["best_energy"])),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(), "batching": batching,
                "batching_full": batching_full,
                "triage": triage, "mlp_inference": mlp, "plain": plain, "differentiation": differentiation,
                "gpu_launches": st["kernel_launches"]}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
