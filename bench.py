#!/usr/bin/env python
"""Benchmark of the exchange build: K-build time per SCF iteration.

One step = one rix_build_K + rix_energy on the resident inputs of the
workload (default: the (H2O)64 cluster, 192 atoms, nbasis 1536, 8 A cutoff),
captured once into a CUDA graph and replayed (--graph 0: eager launches).
Prints one JSON line; per-stage times come from CUDA events of the eager
warm-up steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config 1] [--precision both|fp64|mixed]

By default both paths run; the headline value is the mixed path (terms 3+4 on
the BF16 tensor cores by error-free slicing), with the FP64 path's time and the
mixed-vs-FP64 errors in the same line.
  python bench.py --impl reference ...   (the FP64 CPU oracle on a bounded row sample)

Inputs are synthetic (seeded), larger than L2 (C alone is 0.87 GB for the
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
    """Algorithmic FP64-equivalent FLOPs of one stage as the path runs it."""
    fs = stats["flops_stage"]
    tc12 = stats["flops_term2"] + stats["flops_term1_tc"]
    mixed = precision == "mixed"
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


def oracle_sample(system, pk, rows):
    """Time the FP64 oracle on a row sample; return (seconds, sample FLOPs, full FLOPs, threads)."""
    from oracle.oracle import Oracle
    o = Oracle(system)
    o.set_data(pk.C, pk.V, pk.D)
    o.kpattern()
    o.build_K(dry=True)
    full = o.flops()
    o.kpattern(rows)
    t0 = time.perf_counter()
    o.build_K()
    dt = time.perf_counter() - t0
    return dt, o.flops(), full, Oracle.threads()


def sample_rows(system, n_mol=1):
    """A whole molecule (or the first atoms) near the middle of the atom list."""
    mid = (system.n_atoms // 2) // 3 * 3
    return list(range(mid, min(system.n_atoms, mid + 3 * n_mol)))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import rix_inputs as ri
    s = ri.config(args.config)
    pk = ri.generate(s)
    rows = sample_rows(s)
    for _ in range(args.warmup):
        oracle_sample(s, pk, rows[:1])
    times, sf, ff, thr = [], 0, 0, 1
    for _ in range(args.steps):
        dt, sf, ff, thr = oracle_sample(s, pk, rows)
        times.append(dt * ff / sf * 1e3)
    ms = float(np.mean(times))
    line = {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAMES[args.config], "precision": "fp64", "l2": "inputs larger than L2"},
        "cpu_baseline": {"value": ms, "unit": "ms", "cores": thr, "kind": "oracle",
                         "sample": f"rows {rows} of {s.n_atoms} ({sf:.3g} of {ff:.3g} FLOP), "
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


def measure(args, s, pk, precision, dev, world, rank, local):
    """Warm up, time args.steps builds (+ energy) and the end-to-end variant; returns a dict."""
    import torch
    import torch.distributed as dist
    from paper_2403_10343_gb300.rix import Exchange

    # leave room for the caller's D and K (and the end-to-end copies) beside the library's workspace
    cap = 0
    if s.n_atoms > 1000:
        cap = int(torch.cuda.mem_get_info(dev)[0] - (24 << 30))
    kw = {"n_slices": args.slices} if precision == "mixed" else {}
    ex = Exchange.from_system(s, precision=precision, profile=1, max_workspace_bytes=cap, verbose=args.verbose,
                              **kw)
    assert np.array_equal(ex.pair_keys(), pk.keys)
    ex.set_CV(pk.C, pk.V)          # straight from host memory (copied into library storage)
    D = torch.from_numpy(pk.D).to(dev)
    K = torch.empty(ex.k_elems, dtype=torch.float64, device=dev)
    Ex = torch.empty(1, dtype=torch.float64, device=dev)
    tiles = None
    if args.autotune:
        # tile budgets of the FP64 contraction kernels, timed on this system (not in the timed region)
        tiles = ex.autotune(D, os.path.join(tempfile.gettempdir(), "rix_tiles.txt"))

    def step(Dd):
        ex.build_K(Dd, K)
        ex.energy(Dd, K, Ex)

    # warm-up steps run eagerly and carry the per-stage CUDA events
    for _ in range(args.warmup):
        step(D)
    torch.cuda.synchronize()
    stage_ms, nb = ex.stage_times()
    stage_ms = {k: v / max(1, nb) for k, v in stage_ms.items()}
    eager_ms = None
    if args.graph:
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
    clk = Clocks(local)
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        run()
    e1.record(st)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ex.stage_times()
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
    for _ in range(args.steps):
        Dd.copy_(Dh, non_blocking=True)
        if args.graph:
            D.copy_(Dd)        # the graph reads D
            run()
        else:
            step(Dd)
        Kh.copy_(K, non_blocking=True)
        Exh.copy_(Ex, non_blocking=True)
    e1.record(st)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    ex.stage_times()
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    stats = screened(ex.stats(), ex.count_flops(D))
    launches = stats["launches_build"] + 3  # build + energy kernels
    out = {"ms": ms, "e2e_ms": e2e_ms, "stage_ms": stage_ms, "stats": stats, "clocks": clocks, "graph": args.graph,
           "tiles": tiles,
           "E_x": Ex.item(), "K": K, "launches": launches, "h2d": int(D.numel() * 8), "d2h": int(K.numel() * 8 + 8)}
    ex.close()
    return out


def roofline(args, precision, r):
    stats, stage_ms = r["stats"], r["stage_ms"]
    pk_peaks, src = peaks()
    fp64_stages = [k for k in ("T", "U2", "X12", "Z", "X34") if stage_fp64_share(stats, k, precision) >= 0.5]
    dom = max(fp64_stages, key=lambda k: stage_ms.get(k, 0.0))
    flops = stage_flops(stats, dom, precision) * stage_fp64_share(stats, dom, precision)
    achieved = flops / (stage_ms[dom] * 1e-3) / 1e12
    roof_tc = None
    if precision == "mixed":
        # terms 1-4 and Z on the tensor cores: issued BF16 FLOPs (all slice pairs, padded tiles)
        ms = sum(stage_ms.get(k, 0.0) for k in TENSOR_STAGE if stage_fp64_share(stats, k, precision) < 0.5)
        if ms > 0:
            tc = stats["tensor_flops"] / (ms * 1e-3) / 1e12
            peak_tc = pk_peaks["bf16_tflops_sustained"]
            roof_tc = {"bound": "tensor", "kernel": "k_gemm_sliced (+ packing): terms 1-4 and Z",
                       "achieved": tc, "peak": peak_tc, "unit": "TFLOP/s", "frac": tc / peak_tc, "traffic": None,
                       "peak_source": f"bf16 sustained, {src}",
                       "fp64_equivalent_tflops": (stage_flops(stats, "X34", precision) +
                                                  stage_flops(stats, "TC12", precision) +
                                                  stats["flops_z_tc"] + stats["flops_t_tc"]) / (ms * 1e-3) / 1e12}
            # the headline bound is the stage that takes longest: FP64 kernel or tensor-core stages
            if ms > stage_ms.get(dom, 0.0):
                return roof_tc, roof_tc
    peak = pk_peaks.get("fp64_tflops", FP64_PEAK_TFLOPS_NOMINAL)
    roof = {"bound": "alu", "kernel": STAGE_KERNEL[dom], "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None,
            "peak_source": "FP64 pipe, nominal 1.25 TFLOP/s (recipe table); measured DFMA 1.01, DMMA 1.06"}
    return roof, roof_tc


def stage_roofline(precision, r):
    """Every stage: algorithmic FP64-equivalent FLOPs over its event time, against the pipe it runs on."""
    stats, stage_ms = r["stats"], r["stage_ms"]
    pk_peaks, src = peaks()
    out = {}
    for st in ("T", "U2", "X12", "TC12", "Z", "X34"):
        ms = stage_ms.get(st, 0.0)
        fl = stage_flops(stats, st, precision)
        if ms <= 0 or fl <= 0:
            continue
        ach = fl / (ms * 1e-3) / 1e12
        if precision == "mixed" and st in TENSOR_STAGE and stage_fp64_share(stats, st, precision) < 0.5:
            tc = sum(stats["tensor_flops_stage"][i] for i in TENSOR_STAGE[st]) / (ms * 1e-3) / 1e12
            peak = pk_peaks["bf16_tflops_sustained"]
            out[st] = {"ms": round(ms, 4), "pipe": "tensor (bf16 slices)", "issued_tflops": round(tc, 2),
                       "peak": peak, "frac": round(tc / peak, 4), "fp64_equivalent_tflops": round(ach, 3)}
        else:
            peak = pk_peaks.get("fp64_tflops", FP64_PEAK_TFLOPS_NOMINAL)
            out[st] = {"ms": round(ms, 4), "pipe": "fp64", "achieved_tflops": round(ach, 4), "peak": peak,
                       "frac": round(ach / peak, 4)}
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
    precs = ["fp64", "mixed"] if args.precision == "both" else [args.precision]
    res = {p: measure(args, s, pk, p, dev, world, rank, local) for p in precs}
    head = "mixed" if "mixed" in res else "fp64"
    r = res[head]
    roof, roof_tc = roofline(args, head, r)
    extra = {}
    if len(res) == 2:
        K64, Km = res["fp64"]["K"], res["mixed"]["K"]
        extra["fp64"] = {"ms": res["fp64"]["ms"], "e2e_ms": res["fp64"]["e2e_ms"], "E_x": res["fp64"]["E_x"],
                         "stage_ms": {k: round(v, 4) for k, v in res["fp64"]["stage_ms"].items()},
                         "roofline": roofline(args, "fp64", res["fp64"])[0],
                         "stage_roofline": stage_roofline("fp64", res["fp64"])}
        extra["mixed_vs_fp64"] = {"dE_x_Ha": res["mixed"]["E_x"] - res["fp64"]["E_x"],
                                  "K_rel_fro": float(torch.linalg.norm(Km - K64) / torch.linalg.norm(K64)),
                                  "speedup": res["fp64"]["ms"] / res["mixed"]["ms"]}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rows = sample_rows(s)
        dt, sf, ff, thr = oracle_sample(s, pk, rows)
        cpu = {"value": dt * ff / sf * 1e3, "unit": "ms", "cores": thr, "kind": "oracle",
               "sample": f"rows {rows} of {s.n_atoms} ({sf:.3g} of {ff:.3g} FLOP, {dt:.1f} s), "
                         f"scaled to a full build by the oracle's own FLOP ratio"}
    if rank == 0:
        stats = r["stats"]
        line = {
            "metric": METRIC, "value": r["ms"], "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if head == "fp64" else "bf16-slices+f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_NAMES[args.config], "precision": head,
                       "n_slices": args.slices if head == "mixed" else None,
                       "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas{world}",
                       "timing": "CUDA graph replay" if args.graph else "eager launches",
                       "autotuned_tiles_x12_z_x34": r["tiles"]},
            "e2e": {"value": r["e2e_ms"], "unit": "ms", "h2d_bytes_per_step": r["h2d"],
                    "d2h_bytes_per_step": r["d2h"]},
            "gpu_launches": r["launches"] * args.steps,
            "clocks": r["clocks"],
            "roofline": roof,
            "roofline_tensor_stage": roof_tc,
            "cpu_baseline": cpu,
            "stage_ms": {k: round(v, 4) for k, v in r["stage_ms"].items()},
            "stage_roofline": stage_roofline(head, r),
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
    ap.add_argument("--config", type=int, default=1)
    ap.add_argument("--precision", default="both", choices=["fp64", "mixed", "both"])
    ap.add_argument("--impl", default="rix", choices=["rix", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--graph", type=int, default=1, help="1: time CUDA graph replays of one step (default)")
    ap.add_argument("--autotune", type=int, default=1, help="1: rix_autotune before the warm-up (default)")
    ap.add_argument("--slices", type=int, default=5,
                    help="mixed path: BF16 slices per operand (the regrouped plans take one more); 3 = the "
                         "three-term split")
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
