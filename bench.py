#!/usr/bin/env python
"""Benchmark of the exchange build: K-build time per SCF iteration.

One step = one rix_build_K + rix_energy on the resident inputs of the
workload (default: the largest single-GPU workload, the ice-like supercell of
3,072 atoms, nbasis 24,576, 8 A images), launched eagerly (--graph 1: one
step captured into a CUDA graph and replayed).  Prints one JSON line; the
per-stage times and the per-launch times of the tensor-core GEMM come from
CUDA events recorded inside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config 4] [--precision both|fp64|mixed]

By default both paths run; the headline value is the mixed path (the
contraction stages on the BF16 tensor cores by error-free slicing), with the
FP64 path's time and the mixed-vs-FP64 errors in the same line.
  python bench.py --impl reference ...   (the FP64 CPU oracle on a bounded row sample)

Inputs are synthetic (seeded), larger than L2 (C alone is 24.6 GB for the
default workload), so no L2 flush is needed between steps.  With N > 1 (one
process per GPU under torchrun) every rank runs an independent replica of the
whole build (the build is not sharded across GPUs).
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "K-build ms per SCF iteration (rix_build_K + rix_energy)"
WORKLOAD_NAMES = {
    0: "(H2O)8 cluster, 24 atoms, nbasis 192, no cutoff",
    1: "(H2O)64 cluster, 192 atoms, nbasis 1536, 8 A cutoff, tau 1e-10",
    2: "ice-like periodic, 768 atoms (256 H2O), nbasis 6144, 8 A images",
    3: "perovskite-like periodic, 1536 atoms, nbasis 24911, 8 A images",
    4: "ice-like periodic, 3072 atoms (1024 H2O), nbasis 24576, 8 A images",
}
STAGE_KERNEL = {"flags": "k_flags", "T": "k_T", "U2": "k_U2", "X12": "k_X12",
                "TC12": "k_gemm_sliced (terms 1 and 2)", "Z": "k_Z", "X34": "k_X34", "sym": "k_sym"}
# in mixed precision the TC12 and X34 stages are packing kernels + k_gemm_sliced (TC12 is empty in FP64),
# and the Z stage is k_Z for some middle atoms plus k_gemm_sliced for the others
TENSOR_STAGE = {"X34": (0,), "TC12": (1, 2), "Z": (3,), "T": (4,)}


def screened(stats, cnt):
    """The setup-time statistics with the FLOP counts replaced by those of this D after block screening."""
    out = dict(stats)
    out["flops_fp64_unscreened"] = stats["flops_fp64"]
    out["flops_stage"] = [cnt[k] for k in ("T", "U2", "X12", "Z", "X34", "sym")]
    out["flops_fp64"] = sum(out["flops_stage"])
    out["flops_term2"] = cnt["term2"]
    out["flops_term1_tc"] = cnt["term1_tc"]
    out["flops_z_tc"] = cnt["z_tc"]
    out["flops_t_tc"] = cnt["t_tc"]
    return out


def stage_flops(stats, st, precision):
    """Algorithmic FP64-equivalent FLOPs of one stage as the path runs it.

    In mixed precision the TC12 stage holds term 2 on the tensor cores and, with a
    single row block, term 1 on the tensor cores; with several row blocks term 1 runs
    per block while T is resident, inside the X12 stage.
    """
    fs = stats["flops_stage"]
    mixed = precision == "mixed"
    t1_in_x12 = mixed and stats.get("n_row_blocks", 1) > 1
    tc12 = stats["flops_term2"] + (0.0 if t1_in_x12 else stats["flops_term1_tc"])
    return {"T": fs[0], "U2": fs[1], "X12": fs[2] - tc12 if mixed else fs[2], "TC12": tc12 if mixed else 0.0,
            "Z": fs[3], "X34": fs[4]}.get(st, 0.0)


def stage_fp64_share(stats, st, precision):
    """Fraction of a stage's algorithmic FLOPs left on the FP64 pipe."""
    if precision != "mixed":
        return 1.0
    if st in ("X34", "TC12"):
        return 0.0
    if st == "Z":
        fz = stats["flops_stage"][3]
        return (fz - stats["flops_z_tc"]) / fz if fz > 0 else 0.0
    if st == "T":
        ft = stats["flops_stage"][0]
        return (ft - stats["flops_t_tc"]) / ft if ft > 0 else 0.0
    return 1.0
# FP64 peak of GB300 (recipe table: FP64 1.25 TFLOP/s), used when no measured FP64 peak exists.
FP64_PEAK_TFLOPS_NOMINAL = 1.25


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.dir = tempfile.mkdtemp(prefix="rix_clocks")
        self.path = os.path.join(self.dir, "clocks.csv")
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            try:
                os.rmdir(self.dir)
            except OSError:
                pass
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax = float(f[2])
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
            os.unlink(self.path)
        except OSError:
            pass
        try:
            os.rmdir(self.dir)
        except OSError:
            pass
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


class OracleSampler:
    """The FP64 oracle on a bounded row sample of a workload, scaled to a full build.

    The full build's FLOP count comes from the oracle's own dry run (counted
    once); each timed sample builds the K rows of the sample atoms and is
    scaled by the exact FLOP ratio.
    """

    def __init__(self, system, pk):
        from oracle.oracle import Oracle
        self.Oracle = Oracle
        self.o = Oracle(system)
        self.o.set_data(pk.C, pk.V, pk.D)
        self.o.kpattern()
        self.o.build_K(dry=True)
        self.full = self.o.flops()

    def run(self, rows, threads=0):
        if threads:
            self.Oracle.set_threads(threads)
        try:
            self.o.kpattern(rows)
            t0 = time.perf_counter()
            self.o.build_K()
            dt = time.perf_counter() - t0
            used = self.Oracle.threads()
        finally:
            if threads:
                self.Oracle.set_threads(0)
        return dt, self.o.flops(), used

    def ms_full(self, rows, threads=0):
        dt, sf, used = self.run(rows, threads)
        return dt * self.full / sf * 1e3, dt, sf, used

    def ms_full_blocks(self, keys, threads=0):
        """The same scaling for a sample of K blocks (the oracle builds exactly those)."""
        if threads:
            self.Oracle.set_threads(threads)
        try:
            self.o.kpattern_blocks(keys)
            t0 = time.perf_counter()
            self.o.build_K()
            dt = time.perf_counter() - t0
        finally:
            if threads:
                self.Oracle.set_threads(0)
        sf = self.o.flops()
        return dt * self.full / sf * 1e3, dt, sf


def sample_rows(system, n_mol=1):
    """A whole molecule (or the first atoms) near the middle of the atom list."""
    mid = (system.n_atoms // 2) // 3 * 3
    return list(range(mid, min(system.n_atoms, mid + 3 * n_mol)))


def light_row(system):
    """One atom of the lightest species near the middle (a bounded single-thread sample)."""
    sp = int(np.argmin(system.nbas * system.naux))
    atoms = np.nonzero(system.species == sp)[0]
    return [int(atoms[len(atoms) // 2])]


def cpu_baseline(system, pk, sampler=None):
    """The oracle on the host cores: all cores on a molecule's rows, one core on one light row."""
    smp = sampler or OracleSampler(system, pk)
    rows = sample_rows(system)
    ms, dt, sf, used = smp.ms_full(rows)
    # one core: the diagonal K block and a few neighbours of one light atom (a bounded sample)
    one = light_row(system)[0]
    kk = smp.o.kpattern([one])
    want = kk[:4]
    ms1, dt1, sf1 = smp.ms_full_blocks(want, threads=1)
    return {"value": ms, "unit": "ms", "cores": used, "kind": "oracle",
            "sample": f"rows {rows} of {system.n_atoms} atoms ({sf:.3g} of {smp.full:.3g} FLOP, {dt:.1f} s on "
                      f"{used} threads), scaled to a full build by the oracle's own FLOP count",
            "single_thread": {"value": ms1, "unit": "ms", "cores": 1,
                              "sample": f"{len(want)} K blocks of row {one} ({sf1:.3g} FLOP, {dt1:.1f} s on 1 "
                                        f"thread), scaled likewise"}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import rix_inputs as ri
    s = ri.config(args.config)
    pk = ri.generate(s)
    smp = OracleSampler(s, pk)
    rows = light_row(s) if s.n_atoms > 1000 else sample_rows(s)
    for _ in range(args.warmup):
        smp.run(rows)
    times, sf, used = [], 0.0, 1
    for _ in range(args.steps):
        ms, dt, sf, used = smp.ms_full(rows)
        times.append(ms)
    ms = float(np.mean(times))
    line = {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAMES[args.config], "precision": "fp64", "l2": "inputs larger than L2"},
        "cpu_baseline": {"value": ms, "unit": "ms", "cores": used, "kind": "oracle",
                         "sample": f"each step: rows {rows} of {s.n_atoms} ({sf:.3g} of {smp.full:.3g} FLOP), "
                                   f"time scaled by the oracle's own FLOP ratio"},
        "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def max_over_ranks(x, world, dev):
    """The largest value over the ranks: the job's step time is its slowest rank's."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


# DRAM bytes (read + write) per MMA of k_gemm_sliced (one 128 x 80 x 16 product of one slice
# pair): ncu dram__bytes_read.sum + dram__bytes_write.sum over the 13 GEMM launches of a
# (H2O)64 cluster build (192 atoms; 1.59e11 bytes for 4.65e8 MMAs, three builds 337-343),
# scaled to a launch of the bench workload by its MMA count (None: not measured for the
# kernel as it stands)
GEMM_DRAM_BYTES_PER_STAGE_PAIR = 340.0
GEMM_STAGE_PAIR_FLOPS = 2.0 * 128 * 80 * 16


def measure(args, s, pk, precision, dev, world, steps, warmup, graph, e2e_steps):
    """Warm up, time `steps` builds (+ energy) and the end-to-end variant; returns a dict."""
    import torch
    import torch.distributed as dist
    from paper_2403_10343_gb300.rix import Exchange

    # leave room for the caller's D and K (and the end-to-end copies) beside the library's workspace
    cap = 0
    if s.n_atoms > 1000:
        cap = int(torch.cuda.mem_get_info(dev)[0] - (24 << 30))
    kw = {"n_slices": args.slices, "n_slices_regrouped": args.slices_regrouped} if precision == "mixed" else {}
    prof = 2 if (precision == "mixed" and not graph) else 1
    ex = Exchange.from_system(s, precision=precision, profile=prof, max_workspace_bytes=cap, verbose=args.verbose,
                              **kw)
    assert np.array_equal(ex.pair_keys(), pk.keys)
    ex.set_CV(pk.C, pk.V)          # straight from host memory (copied into library storage)
    D = torch.from_numpy(pk.D).to(dev)
    K = torch.empty(ex.k_elems, dtype=torch.float64, device=dev)
    Ex = torch.empty(1, dtype=torch.float64, device=dev)
    tiles = None
    if args.autotune and precision == "fp64":
        # tile budgets of the FP64 contraction kernels, timed on this system (not in the timed region)
        tiles = ex.autotune(D, os.path.join(tempfile.gettempdir(), "rix_tiles.txt"))

    def step(Dd):
        ex.build_K(Dd, K)
        ex.energy(Dd, K, Ex)

    for _ in range(warmup):
        step(D)
    torch.cuda.synchronize()
    stage_ms, nb = ex.stage_times()
    if prof == 2:
        ex.gemm_profile()
    if graph:
        # one step captured into a CUDA graph; the timed steps are replays
        g = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream(device=dev)
        cs.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(cs):
            step(D)
        torch.cuda.current_stream().wait_stream(cs)
        torch.cuda.synchronize()
        with torch.cuda.graph(g):
            step(D)
        torch.cuda.synchronize()
        run = g.replay
        ex.stage_times()
    else:
        def run():
            step(D)
    st = torch.cuda.current_stream()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        run()
    e1.record(st)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1) / steps
    if not graph:
        # per-stage and per-GEMM-launch events recorded inside the timed region
        sm, nb = ex.stage_times()
        stage_ms = sm
    stage_ms = {k: v / max(1, nb) for k, v in stage_ms.items()}
    gemm = None
    if prof == 2:
        gms, glaunch, gpairs = ex.gemm_profile()
        gemm = {"ms_per_build": gms / steps, "launches_per_build": glaunch / steps,
                "stage_pairs_per_build": gpairs / steps}
    ms = max_over_ranks(ms, world, dev)
    # end to end through the same API with host buffers: D in, K and E_x out, every step
    Dh = torch.from_numpy(pk.D).pin_memory()
    Kh = torch.empty(ex.k_elems, dtype=torch.float64).pin_memory()
    Exh = torch.empty(1, dtype=torch.float64).pin_memory()
    Dd = torch.empty_like(D)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(e2e_steps):
        Dd.copy_(Dh, non_blocking=True)
        if graph:
            D.copy_(Dd)        # the graph reads D
            run()
        else:
            step(Dd)
        Kh.copy_(K, non_blocking=True)
        Exh.copy_(Ex, non_blocking=True)
    e1.record(st)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    ex.stage_times()
    if prof == 2:
        ex.gemm_profile()
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    stats = screened(ex.stats(), ex.count_flops(D))
    launches = stats["launches_build"] + 3  # build + energy kernels
    out = {"ms": ms, "e2e_ms": e2e_ms, "stage_ms": stage_ms, "stats": stats, "clocks": clocks, "graph": graph,
           "tiles": tiles, "gemm": gemm, "E_x": Exh.item(), "E_x_dev": Ex.item(), "K": K, "launches": launches,
           "h2d": int(D.numel() * 8), "d2h": int(K.numel() * 8 + 8), "steps": steps, "warmup": warmup,
           "e2e_steps": e2e_steps}
    ex.close()
    return out


def tensor_alg_flops(stats):
    """Algorithmic FP64-equivalent FLOPs (screened, unpadded, 2 per multiply-add) done by k_gemm_sliced."""
    return (stats["flops_t_tc"] + stats["flops_term1_tc"] + stats["flops_term2"] + stats["flops_z_tc"] +
            stats["flops_stage"][4])


def roofline(precision, r):
    """The dominant kernel's roofline.

    Mixed: k_gemm_sliced, achieved = the algorithmic FP64-equivalent FLOPs of
    the work it does per build / its summed launch time per build (CUDA events
    around every launch in the timed region), against the measured sustained
    BF16 peak; the BF16 FLOPs it issued (every slice pair, padded tiles) are
    reported beside it.  FP64: the longest FP64 stage on the FP64 pipe.
    """
    stats, stage_ms = r["stats"], r["stage_ms"]
    pk_peaks, src = peaks()
    if precision == "mixed" and r.get("gemm"):
        gm = r["gemm"]
        alg = tensor_alg_flops(stats)
        t = gm["ms_per_build"] * 1e-3
        peak = pk_peaks["bf16_tflops_sustained"]
        issued = gm["stage_pairs_per_build"] * GEMM_STAGE_PAIR_FLOPS
        per_launch = gm["stage_pairs_per_build"] / max(1.0, gm["launches_per_build"])
        traffic = None if GEMM_DRAM_BYTES_PER_STAGE_PAIR is None else GEMM_DRAM_BYTES_PER_STAGE_PAIR * per_launch
        return {"bound": "tensor", "kernel": "k_gemm_sliced", "achieved": alg / t / 1e12, "peak": peak,
                "unit": "TFLOP/s", "frac": alg / t / 1e12 / peak, "traffic": traffic,
                "traffic_unit": "bytes per launch",
                "traffic_source": "ncu DRAM bytes per 128x80x16 MMA over the GEMM launches of the 192-atom cluster "
                                  "build, times the MMAs of an average launch here",
                "peak_source": f"bf16 sustained (a kernel timed inside a long step), {src}",
                "alg_flops_per_build": alg, "kernel_ms_per_build": gm["ms_per_build"],
                "launches_per_build": gm["launches_per_build"],
                "issued_bf16_flops_per_build": issued, "issued_tflops": issued / t / 1e12,
                "issued_frac": issued / t / 1e12 / peak,
                "alg_definition": "FP64-equivalent, screened, unpadded: T, terms 1-4 and Z products moved to the "
                                  "tensor cores (2 FLOP per multiply-add)"}
    fp64_stages = [k for k in ("T", "U2", "X12", "Z", "X34") if stage_fp64_share(stats, k, precision) >= 0.5]
    dom = max(fp64_stages, key=lambda k: stage_ms.get(k, 0.0))
    flops = stage_flops(stats, dom, precision) * stage_fp64_share(stats, dom, precision)
    achieved = flops / (stage_ms[dom] * 1e-3) / 1e12
    peak = pk_peaks.get("fp64_tflops", FP64_PEAK_TFLOPS_NOMINAL)
    return {"bound": "alu", "kernel": STAGE_KERNEL[dom], "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None,
            "peak_source": "FP64 pipe, nominal 1.25 TFLOP/s (recipe table); measured DFMA 1.01, DMMA 1.06"}


def stage_rates(precision, r):
    """Every stage: its event time and its algorithmic FP64-equivalent FLOP rate."""
    stats, stage_ms = r["stats"], r["stage_ms"]
    out = {}
    for st in ("T", "U2", "X12", "TC12", "Z", "X34"):
        ms = stage_ms.get(st, 0.0)
        fl = stage_flops(stats, st, precision)
        if ms > 0 and fl > 0:
            out[st] = {"ms": round(ms, 4), "alg_tflops": round(fl / (ms * 1e-3) / 1e12, 4)}
    return out


def run_rix(args):
    import torch
    import torch.distributed as dist
    import rix_inputs as ri

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    s = ri.config(args.config)
    pk = ri.generate(s)
    big = s.n_atoms > 1000
    # eager launches by default, so that the per-launch GEMM events fall inside the timed region
    graph = bool(args.graph)
    precs = ["mixed", "fp64"] if args.precision == "both" else [args.precision]
    res = {}
    for p in precs:
        if p == "fp64" and "mixed" in precs and big:
            # the FP64 path of the large workloads takes minutes per build: a shorter run, labelled
            res[p] = measure(args, s, pk, p, dev, world, 1, 0, False, 1)
        else:
            res[p] = measure(args, s, pk, p, dev, world, args.steps, args.warmup, graph,
                             min(args.steps, 3) if big else args.steps)
    head = "mixed" if "mixed" in res else "fp64"
    r = res[head]
    roof = roofline(head, r)
    extra = {}
    if len(res) == 2:
        K64, Km = res["fp64"]["K"], res["mixed"]["K"]
        r64 = res["fp64"]
        extra["fp64"] = {"ms": r64["ms"], "steps": r64["steps"], "warmup": r64["warmup"],
                         "e2e_ms": r64["e2e_ms"], "E_x": r64["E_x"],
                         "stage_ms": {k: round(v, 4) for k, v in r64["stage_ms"].items()},
                         "roofline": roofline("fp64", r64), "stage_rates": stage_rates("fp64", r64),
                         "note": "timed over fewer steps than the mixed path" if r64["steps"] < args.steps else ""}
        extra["mixed_vs_fp64"] = {"dE_x_Ha": res["mixed"]["E_x"] - r64["E_x"],
                                  "K_rel_fro": float(torch.linalg.norm(Km - K64) / torch.linalg.norm(K64)),
                                  "speedup": r64["ms"] / res["mixed"]["ms"]}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(s, pk)
    if rank == 0:
        stats = r["stats"]
        line = {
            "metric": METRIC, "value": r["ms"], "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if head == "fp64" else "bf16-slices+f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_NAMES[args.config], "precision": head,
                       "n_slices": args.slices if head == "mixed" else None,
                       "n_slices_regrouped": (args.slices_regrouped or args.slices + 1) if head == "mixed" else None,
                       "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas{world}",
                       "timing": "CUDA graph replay" if r["graph"] else "eager launches",
                       "autotuned_tiles_x12_z_x34": r["tiles"]},
            "e2e": {"value": r["e2e_ms"], "unit": "ms", "h2d_bytes_per_step": r["h2d"],
                    "d2h_bytes_per_step": r["d2h"], "steps": r["e2e_steps"]},
            "gpu_launches": r["launches"] * args.steps,
            "clocks": r["clocks"],
            "roofline": roof,
            "cpu_baseline": cpu,
            "stage_ms": {k: round(v, 4) for k, v in r["stage_ms"].items()},
            "stage_rates": stage_rates(head, r),
            "alg_flops": stats["flops_fp64"],
            "alg_flops_unscreened": stats["flops_fp64_unscreened"],
            "alg_tflops": stats["flops_fp64"] / (r["ms"] * 1e-3) / 1e12,
            "E_x": r["E_x"],
        }
        line.update(extra)
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", type=int, default=4,
                    help="workload 0-4 (default 4: the largest single-GPU one, the 3,072-atom ice supercell)")
    ap.add_argument("--precision", default="both", choices=["fp64", "mixed", "both"])
    ap.add_argument("--impl", default="rix", choices=["rix", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--graph", type=int, default=0,
                    help="1: time CUDA graph replays of one step; 0 (default): eager launches, with CUDA events "
                         "around every tensor-core GEMM launch for the kernel roofline")
    ap.add_argument("--autotune", type=int, default=1, help="1: rix_autotune of the FP64 path (default)")
    ap.add_argument("--slices", type=int, default=5,
                    help="mixed path: BF16 slices per operand (the regrouped plans take one more); 3 = the "
                         "three-term split")
    ap.add_argument("--slices-regrouped", type=int, default=0,
                    help="mixed path: slices of the regrouped plans (term 1, Z, T); 0 = --slices + 1")
    ap.add_argument("--verbose", type=int, default=0, help="1: the library prints its plan to stderr")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        from paper_2403_10343_gb300 import build
        build.build()
        run_rix(args)


if __name__ == "__main__":
    main()
