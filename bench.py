"""Benchmark: FP64 tiled Cholesky as a device-scheduled STF task graph on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl spx|reference]
                    [--n 16384] [--tile 512]

One step = the whole hot path on one synthetic SPD matrix resident in HBM:
insert the task graph (default: spx_cholesky_insert_ozaki, FP64 results with
the SYRK/GEMM and inverse-panel products split on the tensor cores;
--arith f64: spx_cholesky_insert, everything on the FP64 pipe), derive the
DAG on the device, run it in the persistent kernel, wait.  The matrix is
restored from a pristine copy before each step (outside the timed events).
Inputs (2.1 GB) are larger than L2, so no flush is needed.

Printed: one JSON line (rank 0) with GFLOP/s (n^3/3 per step), tasks/s,
p50/p99 step latency, the one-launch-per-task and four-stream baselines on
the same GPU, the small-matrix latency case (n=512, tile 64), the roofline
of the persistent kernel (the BF16 tensor rate on the split path, the FP64
SIMT peak on the FP64 pipe) with its DRAM traffic from the committed ncu
summary, the end-to-end number through pinned host buffers, the CPU oracle
on a bounded sample, and the SM clocks seen.

--impl reference times the CPU oracle (plain single-threaded FP64 loops,
insertion order) on a bounded sample of the same workload.

Under torchrun (N > 1) every rank factors its own matrix (replicas: the
workload has no exchange step); value = all ranks' flops / max rank time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import threading
import time

import numpy as np

METRIC = "Cholesky GFLOP/s & tasks/s (device DAG vs per-task launch); p50/p99 latency"
PEAKS_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
ROOT = os.path.dirname(os.path.abspath(__file__))
DRAM_PROFILE = os.path.join(ROOT, "profiles", "persistent_kernel_dram_cholesky_n16384_t512.md")
GEMM_DRAM_PROFILE = os.path.join(ROOT, "profiles", "split_gemm_dag_n8192_t512.md")


def kernel_source_hash() -> str:
    """SHA-256 (first 16 hex digits) of the device sources the kernels are
    built from: the .cu files and the headers they include (host-only graph
    builders and bindings do not change a kernel)."""
    import glob
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2308_15964_b300", "csrc")
    files = sorted(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh")) +
                   glob.glob(os.path.join(csrc, "*.h")))
    for f in files:
        if os.path.isfile(f):
            h.update(os.path.basename(f).encode())
            h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(path: str = DRAM_PROFILE):
    """DRAM bytes (read + write) of one launch from a committed ncu summary,
    or None when the kernel sources changed since that capture."""
    if not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        if ":" in line and line.split(":", 1)[0].strip() in ("source-hash", "traffic-bytes-per-launch"):
            k, v = line.split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    if fields.get("source-hash") != kernel_source_hash() or "traffic-bytes-per-launch" not in fields:
        return None
    return int(fields["traffic-bytes-per-launch"])
# FP64 SIMT peak: 2 DFMA per clock per SM (measured by spx_probe: 1.127 TFLOP/s
# at 1942 MHz on 148 SMs) x 2 flop x 148 SMs x 2032 MHz maximum SM clock.
FP64_DFMA_PER_CLK_SM = 2
ORACLE_SAMPLE_N = 4096      # CPU baseline sample (about 10 s on one core)
COMPARATOR_STEPS = 5        # timed steps of each comparison executor
REFERENCE_STEP_N = 2048     # --impl reference: one step of the oracle


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="spx", choices=["spx", "reference"])
    p.add_argument("--n", type=int, default=16384)
    p.add_argument("--tile", type=int, default=512)
    p.add_argument("--sigma", type=float, default=0.1)
    p.add_argument("--arith", default="ozaki", choices=["ozaki", "f64"],
                   help="cholesky: FP64 trailing updates emulated on the tensor cores by "
                        "splitting (ozaki) or on the FP64 SIMT pipe (f64)")
    p.add_argument("--no-extras", action="store_true", help="skip baseline / e2e / cpu legs")
    p.add_argument("--workload", default="cholesky", choices=["cholesky", "gemm", "batch", "mixed", "serve", "tc",
                                                      "overhead", "axpy", "nbody", "splitgemm", "stream"],
                   help="batch: 4096 uneven solves (n in 32..1024, 1..16 RHS) in one launch")
    p.add_argument("--gemm-rows", default="all", choices=["all", "split", "f64"],
                   help="gemm: which DAG forms to time (split products, FP64 pipe, or both)")
    p.add_argument("--count", type=int, default=4096)
    p.add_argument("--rate", type=float, default=200.0, help="serve: offered requests per second")
    p.add_argument("--duration", type=float, default=60.0, help="serve: seconds of arrivals")
    return p.parse_args()


class Clocks:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            self.p.wait()

    def summary(self):
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit()),
                "samples": len(rows), "reasons": reasons}


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_oracle_gflops(n: int, b: int, sigma: float, seed: int):
    from oracle import oracle as O
    from paper_2308_15964_b300 import inputs
    A = inputs.spd_matrix(n, sigma, seed).numpy()
    dt, info = O.timed_tiled_cholesky(A, b)
    assert info == 0
    return n ** 3 / 3.0 / dt / 1e9, dt


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n, b = REFERENCE_STEP_N, args.tile
    times = []
    for i in range(args.warmup + args.steps):
        gf, dt = cpu_oracle_gflops(n, b, args.sigma, seed=2)
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = args.steps * (n ** 3 / 3.0) / total / 1e9
    sample = (f"tiled Cholesky oracle (single-threaded FP64 loops, insertion order) on n={n}, "
              f"tile {b}, sigma {args.sigma}: one factorization per step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"tiled Cholesky FP64, sample n={n} tile={b} of the n={args.n} workload",
                   "n": n, "tile": b},
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def ozaki_work(n, b):
    """(BF16 tensor flops, FP64 SIMT flops) of the split-path Cholesky with
    inverse panels, tiles b (the last one may be ragged: counted as full)."""
    T = -(-n // b)
    nbr, nbc = -(-b // 128), -(-b // 64)
    full = nbr * nbc
    syrk_blocks = sum(min(2 * (i + 1), nbc) for i in range(nbr))
    gemm_tiles = sum((T - k - 1) * (T - k - 2) // 2 for k in range(T))
    syrk_tiles = T * (T - 1) // 2
    inv_tiles = sum(max(0, T - k - 2) for k in range(T))
    block_flops = 36 * 2 * 128 * 64 * b
    tensor_flops = ((gemm_tiles + inv_tiles) * full + syrk_tiles * syrk_blocks) * block_flops
    fp64_flops = T * b ** 3 / 3 + (T - 1) * b ** 3 + T * b ** 3 / 3
    return tensor_flops, fp64_flops


def ozaki_roofline(n, b, kernel_ms, fp64_peak, traffic):
    """Roofline of the persistent kernel on the split path (inverse panels).
    Tensor work: every 128 x 64 output block with K digits issues MMAs over
    N = 64 (8 - p) columns for the eight planes p of A, i.e. 36 digit-pair
    products of 2 * 128 * 64 * K flops; summed over the GEMM tasks' tiles, the
    SYRK tasks' lower blocks and the TRSM_INV products (tiles i >= k + 2).
    FP64 SIMT work: POTRF (b^3 / 3), the critical panel tile's substitution
    (b^3) and TRTRI (b^3 / 3) per k.  The bound is the tensor-core rate; the
    FP64 share is given beside."""
    tensor_flops, fp64_flops = ozaki_work(n, b)
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    bf16 = peaks.get("bf16_tflops", 1800.0)
    ach = tensor_flops / (kernel_ms * 1e-3) / 1e12
    return {"bound": "tensor", "achieved": ach, "peak": bf16, "unit": "TFLOP/s", "frac": ach / bf16,
            "traffic": traffic,
            "kernel": "persistent_kernel<split products> (one CTA per SM)",
            "kernel_ms": kernel_ms,
            "peak_note": "measured cuBLAS bf16 burst rate (MEASURED_PEAKS.json)"
                         if "bf16_tflops" in peaks else "fallback bf16 peak",
            "tensor_tflop_per_launch": tensor_flops / 1e12,
            "fp64_simt": {"flops_per_launch": fp64_flops,
                          "achieved_tflops": fp64_flops / (kernel_ms * 1e-3) / 1e12,
                          "peak_tflops": fp64_peak,
                          "frac": fp64_flops / (kernel_ms * 1e-3) / 1e12 / fp64_peak},
            "note": "FP64-equivalent rate n^3/3 over the kernel time: "
                    f"{n ** 3 / 3 / (kernel_ms * 1e-3) / 1e12:.2f} TFLOP/s"}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    world, rank, local = dist_setup()
    import torch
    torch.cuda.set_device(local)
    from paper_2308_15964_b300 import cholesky, inputs, spx
    if args.workload == "batch":
        run_batch(args, world, rank, local)
        return
    if args.workload == "mixed":
        run_mixed(args, world, rank, local)
        return
    if args.workload == "serve":
        run_serve(args, world, rank, local)
        return
    if args.workload == "tc":
        run_tc(args, world, rank, local)
        return
    if args.workload == "stream":
        run_stream(args, world, rank, local)
        return
    if args.workload == "splitgemm":
        run_splitgemm(args, world, rank, local)
        return
    if args.workload == "overhead":
        run_overhead(args, world, rank, local)
        return
    if args.workload == "gemm":
        run_gemm(args, world, rank, local)
        return
    if args.workload == "axpy":
        run_axpy(args, world, rank, local)
        return
    if args.workload == "nbody":
        run_nbody(args, world, rank, local)
        return

    n, b = args.n, args.tile
    flops = cholesky.cholesky_flops(n)
    A0 = inputs.spd_matrix(n, args.sigma, seed=2, device="cuda")
    A = torch.empty_like(A0)
    stream = torch.cuda.current_stream()
    g = spx.Graph()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    oz = args.arith == "ozaki"
    # split path: inverse panel solves (TRTRI + split products), the diagonal
    # inverses in V
    store = cholesky.ozaki_store(n, b, inverse_panels=True) if oz else None
    V = torch.zeros((n, b), dtype=torch.float64, device="cuda") if oz else None

    def build_graph(graph, ozaki=oz, inverse=True):
        if ozaki:
            cholesky.cholesky_ozaki_graph(graph, A, b, S=store, V=V if inverse else None)
        else:
            cholesky.cholesky_graph(graph, A, b)

    def step(graph, record=None, ozaki=oz, inverse=True):
        A.copy_(A0)
        ev[0].record()
        graph.clear()
        build_graph(graph, ozaki, inverse)
        graph.execute(stream)
        rc, info = graph.wait()
        ev[1].record()
        ev[1].synchronize()
        assert rc == spx.OK, (rc, info)
        if record is not None:
            record.append((ev[0].elapsed_time(ev[1]), graph.timing()[1]))

    for _ in range(args.warmup):
        step(g)
    ntasks, nedges, _, _ = g.sizes()
    recs = []
    torch.cuda.synchronize()
    barrier(world)
    with Clocks(local) as clk:
        t0 = time.perf_counter()
        torch.cuda.nvtx.range_push("spx_timed")
        for _ in range(args.steps):
            step(g, recs)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        barrier(world)
        wall = time.perf_counter() - t0
    clocks = clk.summary()
    step_ms = [r[0] for r in recs]
    run_ms = [r[1] for r in recs]
    total_ms = max_over_ranks(sum(step_ms), world)
    value = world * args.steps * flops / (total_ms * 1e-3) / 1e9
    stats = g.stats()

    out = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": ("f64 (SYRK/GEMM products emulated by Ozaki splitting: bf16 digit planes on tcgen05, "
                  "exact fp32 digit sums, one fp64 rounding; POTRF/TRSM fp64)") if oz else "f64",
        "data": "synthetic",
        "config": {"workload": f"tiled Cholesky FP64 n={n} tile={b} ({ntasks} tasks, {nedges} edges); "
                               "step = insert + device DAG derivation + persistent execution; "
                               + ("trailing updates and panel solves (TRTRI + inverse products) "
                                  "by splitting on the tensor cores, POTRF and the critical panel "
                                  "tile on the FP64 pipe" if oz
                                  else "all tile ops on the FP64 SIMT pipe"),
                   "arith": args.arith,
                   "n": n, "tile": b, "tasks": ntasks, "edges": nedges, "sigma": args.sigma,
                   "l2": "inputs larger than L2 (matrix 8n^2 bytes)",
                   "parallelism": f"replicas x{world}"},
        "tasks_per_s": ntasks / (statistics.mean(step_ms) * 1e-3),
        "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
        "wall_s": wall,
        "gpu_launches": 2 * args.steps,
        "clocks": clocks,
        "sched": {"parts": stats["parts"], "ctas": stats["ctas"],
                  "busy_frac": stats["busy_cycles"] / max(1, stats["total_cycles"]),
                  "queue_hiwater": stats["queue_hiwater"]},
    }

    # Roofline of the dominant kernel (the persistent executor): algorithmic
    # flops n^3/3 per launch / its CUDA-event duration, against the FP64 SIMT
    # peak derived from the measured DFMA rate per SM and the max SM clock.
    sms = spx.lib.spx_device_sm_count()
    max_mhz = clocks.get("sm_max_mhz") or 2032.0
    peak = FP64_DFMA_PER_CLK_SM * 2 * sms * max_mhz * 1e6 / 1e12
    run_mean = statistics.mean(run_ms)
    probe_rate, _ = spx.probe(0, 4000)
    # the committed capture is of the split path's launch (the default arithmetic)
    traffic = measured_traffic() if (n, b) == (16384, 512) and oz else None
    traffic_note = ("dram__bytes_read.sum + dram__bytes_write.sum of one launch, from the committed "
                    "ncu summary of this workload; null when the kernel sources differ from the "
                    "captured ones, and for the FP64 path (not captured)")
    if oz:
        out["roofline"] = ozaki_roofline(n, b, run_mean, peak, traffic)
        out["roofline"]["traffic_note"] = traffic_note
    else:
        achieved = flops / (run_mean * 1e-3) / 1e12
        out["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                           "frac": achieved / peak, "traffic": traffic, "traffic_note": traffic_note,
                           "kernel": "persistent_kernel (FP64 DFMA tile ops)",
                           "kernel_ms": run_mean,
                           "peak_note": "2 DFMA/clk/SM x 148 SMs x max SM clock (derived); "
                                        f"live DFMA probe {probe_rate / 1e12:.3f} TFLOP/s"}
    out["sched"]["op_share"] = {k: round(v / max(1, stats["busy_cycles"]), 3)
                                for k, v in stats["op_cycles"].items()}

    if oz and rank == 0 and not args.no_extras:
        # the same factorization with every tile op on the FP64 SIMT pipe, and
        # the two factors compared (the splitting's accuracy at this size)
        L_oz = torch.tril(A)
        # the split path with every panel tile by FP64 substitution
        gsub = spx.Graph()
        step(gsub, inverse=False)
        srec_ = []
        for _ in range(3):
            step(gsub, srec_, inverse=False)
        gsub.close()
        subms = [r[0] for r in srec_]
        out["ozaki_substitution_panels"] = {
            "value": flops / (statistics.mean(subms) * 1e-3) / 1e9, "unit": "GFLOP/s",
            "ms_per_step": statistics.mean(subms), "p99_ms": float(np.percentile(subms, 99)),
            "steps": len(subms)}
        gf = spx.Graph()
        step(gf, ozaki=False)
        frec = []
        for _ in range(3):
            step(gf, frec, ozaki=False)
        gf.close()
        L_f = torch.tril(A)
        fms = [r[0] for r in frec]
        frun = statistics.mean(r[1] for r in frec)
        gen = torch.Generator(device="cuda").manual_seed(7)
        v = torch.rand(n, 4, dtype=torch.float64, device="cuda", generator=gen) * 2 - 1
        fr = lambda L: float(((A0 @ v - L @ (L.T @ v)).norm() / (A0.norm() * v.norm())).item())
        out["f64_dfma"] = {"value": flops / (statistics.mean(fms) * 1e-3) / 1e9, "unit": "GFLOP/s",
                           "ms_per_step": statistics.mean(fms),
                           "p50_ms": float(np.percentile(fms, 50)),
                           "p99_ms": float(np.percentile(fms, 99)), "steps": len(fms),
                           "roofline": {"bound": "alu", "achieved": flops / (frun * 1e-3) / 1e12,
                                        "peak": peak, "unit": "TFLOP/s",
                                        "frac": flops / (frun * 1e-3) / 1e12 / peak,
                                        "kernel": "persistent_kernel (FP64 DFMA tile ops)"}}
        out["accuracy"] = {"max_rel_entry_diff_vs_dfma": float(((L_oz - L_f).abs().max()
                                                               / L_f.abs().max()).item()),
                           "freivalds_ozaki": fr(L_oz), "freivalds_dfma": fr(L_f),
                           "note": "||A v - L L^T v|| / (||A||_F ||v||) with 4 random v; the "
                                   "factors of the two arithmetics compared entry by entry"}
        del L_oz, L_f

    if rank == 0 and not args.no_extras:
        # one-launch-per-task baseline, same tile code, same stream
        gb = spx.Graph(executor=spx.EXEC_PER_TASK)
        step(gb)
        brec = []
        for _ in range(COMPARATOR_STEPS):
            step(gb, brec)
        bms = [r[0] for r in brec]
        out["baseline_per_task"] = {"value": flops / (statistics.mean(bms) * 1e-3) / 1e9,
                                    "unit": "GFLOP/s", "ms_per_step": statistics.mean(bms),
                                    "tasks_per_s": ntasks / (statistics.mean(bms) * 1e-3),
                                    "p99_ms": float(np.percentile(bms, 99)), "steps": len(bms)}
        gb.close()
        # the paper's GPU set-up: per-task launches over four streams, an event
        # wait per cross-stream predecessor
        gs = spx.Graph(executor=spx.EXEC_STREAMS)
        step(gs)
        srec = []
        for _ in range(COMPARATOR_STEPS):
            step(gs, srec)
        sms_ = [r[0] for r in srec]
        out["baseline_streams"] = {"value": flops / (statistics.mean(sms_) * 1e-3) / 1e9,
                                   "unit": "GFLOP/s", "ms_per_step": statistics.mean(sms_),
                                   "tasks_per_s": ntasks / (statistics.mean(sms_) * 1e-3),
                                   "p99_ms": float(np.percentile(sms_, 99)), "steps": len(sms_)}
        gs.close()
        # one launch per task, the launch sequence replayed through a CUDA graph
        # (inserted once; re-runs reset and replay)
        gg = spx.Graph(executor=spx.EXEC_PER_TASK, cuda_graph=True)
        A.copy_(A0)
        build_graph(gg)
        assert gg.run()[0] == spx.OK
        grec = []
        for i in range(COMPARATOR_STEPS + 1):
            A.copy_(A0)
            gg.reset()
            ev[0].record()
            rc_, _ = gg.run()
            ev[1].record()
            ev[1].synchronize()
            assert rc_ == spx.OK
            if i > 0:                     # the first reset run captures the graph
                grec.append(ev[0].elapsed_time(ev[1]))
        out["baseline_per_task_cudagraph"] = {"value": flops / (statistics.mean(grec) * 1e-3) / 1e9,
                                              "unit": "GFLOP/s", "ms_per_step": statistics.mean(grec),
                                              "note": "execution only (the graph is inserted once)"}
        gg.close()
        # the same workload with priorities from the critical path
        gp = spx.Graph(priorities=1)
        step(gp)
        prec_ = []
        for _ in range(COMPARATOR_STEPS):
            step(gp, prec_)
        pms = [r[0] for r in prec_]
        out["bottom_level_priorities"] = {"value": flops / (statistics.mean(pms) * 1e-3) / 1e9,
                                          "unit": "GFLOP/s", "ms_per_step": statistics.mean(pms),
                                          "p99_ms": float(np.percentile(pms, 99)),
                                          "steps": len(pms)}
        gp.close()
        out["latency_small"] = small_latency(spx, cholesky, inputs, torch)
        out["gemm_dag"] = gemm_dag(spx, cholesky, inputs, torch, 8192, b, args.warmup, args.steps,
                                   max_mhz, comparators=True)

        # end to end through host buffers: H2D of A, the step, D2H of L
        Ah = A0.cpu().pin_memory()
        Lh = torch.empty_like(Ah).pin_memory()
        e2e = []
        for i in range(3):
            ev[0].record()
            A.copy_(Ah, non_blocking=True)
            g.clear()
            build_graph(g)
            g.execute(stream)
            rc, _ = g.wait()
            assert rc == spx.OK
            Lh.copy_(A, non_blocking=True)
            ev[1].record()
            ev[1].synchronize()
            if i > 0:
                e2e.append(ev[0].elapsed_time(ev[1]))
        whole = {"value": flops / (statistics.mean(e2e) * 1e-3) / 1e9, "unit": "GFLOP/s",
                 "h2d_bytes_per_step": 8 * n * n, "d2h_bytes_per_step": 8 * n * n,
                 "ms_per_step": statistics.mean(e2e),
                 "how": "whole matrix copied in, graph run, whole matrix copied out"}
        if oz and V is not None:
            # the library's host-buffer entry: the lower triangle's column
            # blocks uploaded while the kernel runs, the factor's copied back
            lower = sum((n - j * b) * min(b, n - j * b) * 8 for j in range(-(-n // b)))
            Lh.zero_()
            e2e = []
            gh = spx.Graph()  # cleared and reused: its device buffers stay allocated
            for i in range(4):
                gh.clear()
                ev[0].record()
                rc, info = cholesky.cholesky_host_ozaki(gh, Ah, Lh, b, dev_A=A, S=store, V=V)
                ev[1].record()
                ev[1].synchronize()
                assert rc == spx.OK and info == 0
                if i > 0:
                    e2e.append(ev[0].elapsed_time(ev[1]))
            gh.close()
            assert torch.equal(torch.tril(Lh), torch.tril(A.cpu()))
            out["e2e"] = {"value": flops / (statistics.mean(e2e) * 1e-3) / 1e9, "unit": "GFLOP/s",
                          "h2d_bytes_per_step": lower, "d2h_bytes_per_step": lower,
                          "ms_per_step": statistics.mean(e2e),
                          "how": "spx_cholesky_host_ozaki: pinned host matrix in, factor out; "
                                 "the lower triangle's column blocks uploaded while the kernel "
                                 "runs, the factor's downloaded as each one's last writers "
                                 "finish", "whole_matrix_copies": whole}
        else:
            out["e2e"] = whole
        del Ah, Lh
        sizes = {}
        for ns in (1024, 2048):
            if ns < ORACLE_SAMPLE_N:
                sizes[ns] = cpu_oracle_gflops(ns, b, args.sigma, seed=2)[1]
        gf, dt = cpu_oracle_gflops(ORACLE_SAMPLE_N, b, args.sigma, seed=2)
        sizes[ORACLE_SAMPLE_N] = dt
        out["cpu_baseline"] = {"value": gf, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                               "sample": f"tiled Cholesky oracle, n={ORACLE_SAMPLE_N} tile {b} "
                                         f"(same tile and recipe, {dt:.1f} s on one host core; "
                                         f"host has {os.cpu_count()} cores)",
                               "seconds_by_n": {str(k): v for k, v in sizes.items()},
                               "extrapolated_s_at_n": {
                                   "n": n, "seconds": dt * (n / ORACLE_SAMPLE_N) ** 3,
                                   "note": "n^3 extrapolation of the n=%d time, not measured"
                                           % ORACLE_SAMPLE_N}}
    g.close()
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def gemm_dag(spx, cholesky, inputs, torch, n, b, warmup, steps, max_mhz, comparators=False,
             rows="all"):
    """The paper's tiled GEMM whose tasks depend on the blocks of C (section
    "Numerical applications"): C += A B, one GEMM_NN_ADD task per (i, j, k),
    each with a WRITE on C_ij (the 16 tasks of a block form a chain) or a
    COMMUTATIVE_WRITE (any order, one at a time).  Entries uniform[-1, 1)
    (seeds 3, 4, 5).  Step = insert + derive + execute + wait; value = 2 n^3
    over the step's device time.  Inputs 3 x 8 n^2 bytes, larger than L2."""
    A = inputs.uniform((n, n), 3, device="cuda")
    B = inputs.uniform((n, n), 4, device="cuda")
    C0 = inputs.uniform((n, n), 5, device="cuda")
    C = torch.empty_like(C0)
    flops = cholesky.gemm_flops(n)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    stream = torch.cuda.current_stream()
    sms = spx.lib.spx_device_sm_count()
    peak = FP64_DFMA_PER_CLK_SM * 2 * sms * max_mhz * 1e6 / 1e12
    res = {"workload": f"tiled GEMM C += A B as a task graph, FP64, n={n} tile={b}, "
                       "one task per (i, j, k) on C_ij (WRITE chain or COMMUTATIVE_WRITE run)",
           "n": n, "tile": b, "flops_per_step": flops}

    T = -(-n // b)
    S = torch.empty(2 * T * T * spx.lib.spx_ozaki_slot_bytes(b), dtype=torch.uint8, device="cuda")

    def timed(g, commutative, nsteps, nwarm, split=False):
        rec = []
        for i in range(nwarm + nsteps):
            C.copy_(C0)
            ev[0].record()
            g.clear()
            if split:
                cholesky.gemm_ozaki_graph(g, A, B, C, b, commutative=commutative, S=S)
            else:
                cholesky.gemm_graph(g, A, B, C, b, commutative=commutative)
            g.execute(stream)
            rc, _ = g.wait()
            ev[1].record()
            ev[1].synchronize()
            assert rc == spx.OK, rc
            if i >= nwarm:
                rec.append((ev[0].elapsed_time(ev[1]), g.timing()[1]))
        return rec

    for mode, comm in (("write", False), ("commutative", True)) if rows != "split" else ():
        g = spx.Graph()
        rec = timed(g, comm, steps, warmup)
        ntasks, nedges, _, _ = g.sizes()
        g.close()
        ms = [r[0] for r in rec]
        kern = statistics.mean(r[1] for r in rec)
        row = {"value": flops / (statistics.mean(ms) * 1e-3) / 1e9, "unit": "GFLOP/s",
               "ms_per_step": statistics.mean(ms), "steps": len(ms), "tasks": ntasks,
               "edges": nedges, "tasks_per_s": ntasks / (statistics.mean(ms) * 1e-3),
               "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
               "roofline": {"bound": "alu", "achieved": flops / (kern * 1e-3) / 1e12, "peak": peak,
                            "unit": "TFLOP/s", "frac": flops / (kern * 1e-3) / 1e12 / peak,
                            "kernel": "persistent_kernel (FP64 DFMA tile ops)", "kernel_ms": kern}}
        # comparators on the WRITE DAG only: a commutative task runs as one
        # part (one CTA), so one launch per task would serialise 4096
        # single-CTA GEMMs (minutes per step) and measure nothing new
        if comparators and not comm:
            for name, ex in (("baseline_per_task", spx.EXEC_PER_TASK),
                             ("baseline_streams", spx.EXEC_STREAMS)):
                gb = spx.Graph(executor=ex)
                brec = timed(gb, comm, COMPARATOR_STEPS, 1)
                gb.close()
                bms = [r[0] for r in brec]
                row[name] = {"value": flops / (statistics.mean(bms) * 1e-3) / 1e9,
                             "unit": "GFLOP/s", "ms_per_step": statistics.mean(bms),
                             "tasks_per_s": ntasks / (statistics.mean(bms) * 1e-3),
                             "p99_ms": float(np.percentile(bms, 99)), "steps": len(bms)}
        res[mode] = row
    # the same DAG with each task's product split on the tensor cores (SPLIT
    # tasks for the tiles of A, SPLIT_T for B, then the GEMM_NN_ADD tasks)
    block_flops = 36 * 2 * 128 * 64 * b
    tensor_flops = T ** 3 * (-(-b // 128)) * (-(-b // 64)) * block_flops
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    bf16 = peaks.get("bf16_tflops", 1800.0)
    for mode, comm in (("split_write", False), ("split_commutative", True)) if rows != "f64" else ():
        g = spx.Graph()
        rec = timed(g, comm, steps, warmup, split=True)
        ntasks, nedges, _, _ = g.sizes()
        g.close()
        ms = [r[0] for r in rec]
        kern = statistics.mean(r[1] for r in rec)
        ach = tensor_flops / (kern * 1e-3) / 1e12
        res[mode] = {"value": flops / (statistics.mean(ms) * 1e-3) / 1e9, "unit": "GFLOP/s",
                     "ms_per_step": statistics.mean(ms), "steps": len(ms), "tasks": ntasks,
                     "edges": nedges, "tasks_per_s": ntasks / (statistics.mean(ms) * 1e-3),
                     "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
                     "arith": "FP64 by split products (Ozaki) on the BF16 tensor cores",
                     "roofline": {"bound": "tensor", "achieved": ach, "peak": bf16,
                                  "unit": "TFLOP/s", "frac": ach / bf16,
                                  "traffic": measured_traffic(GEMM_DRAM_PROFILE)
                                  if (n, b) == (8192, 512) else None,
                                  "kernel": "persistent_kernel<split products> (one CTA per SM)",
                                  "kernel_ms": kern,
                                  "tensor_tflop_per_launch": tensor_flops / 1e12}}
    del A, B, C, C0, S
    torch.cuda.empty_cache()
    # CPU oracle (one host core, insertion order): bounded samples (about 4 s
    # in all; n = 2048 takes 40 s), n^3 extrapolation to the workload size
    from oracle import oracle as O
    secs = {}
    for ns in (512, 1024):
        Ah = inputs.uniform((ns, ns), 3).numpy()
        Bh = inputs.uniform((ns, ns), 4).numpy()
        Ch = inputs.uniform((ns, ns), 5).numpy()
        t0 = time.perf_counter()
        assert O.tiled_gemm(Ah, Bh, Ch, b) == 0
        secs[ns] = time.perf_counter() - t0
    top = max(secs)
    res["cpu_baseline"] = {"value": cholesky.gemm_flops(top) / secs[top] / 1e9, "unit": "GFLOP/s",
                           "cores": 1, "kind": "oracle",
                           "sample": f"tiled GEMM oracle (WRITE order), n in {sorted(secs)}, tile {b}",
                           "seconds_by_n": {str(k): v for k, v in secs.items()},
                           "extrapolated_s_at_n": {"n": n, "seconds": secs[top] * (n / top) ** 3,
                                                   "note": f"n^3 extrapolation of the n={top} time, "
                                                           "not measured"}}
    return res


def run_gemm(args, world, rank, local):
    """--workload gemm: the tiled GEMM DAG alone (n = 8192, tile 512)."""
    import torch
    from paper_2308_15964_b300 import cholesky, inputs, spx
    n = args.n if args.n != 16384 else 8192
    with Clocks(local) as clk:
        rows = args.gemm_rows
        if rows == "all" and args.no_extras:  # the line's own form only
            rows = "split" if args.arith == "ozaki" else "f64"
        res = gemm_dag(spx, cholesky, inputs, torch, n, args.tile, args.warmup, args.steps, 2032.0,
                       comparators=not args.no_extras, rows=rows)
    clocks = clk.summary()
    # the line's value: the split-product DAG (--arith ozaki, default) or
    # the FP64 SIMT DAG (--arith f64), WRITE form; every row in gemm_dag
    oz = args.arith == "ozaki"
    w = res["split_write" if oz else "write"]
    out = {"metric": METRIC, "value": w["value"], "unit": "GFLOP/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": w["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": ("f64 (products emulated by Ozaki splitting: bf16 digit planes on tcgen05, "
                     "exact fp32 digit sums, one fp64 rounding per task)") if oz else "f64",
           "data": "synthetic",
           "config": {"workload": res["workload"] + (", products split on the tensor cores "
                                                     "(SPLIT / SPLIT_T tasks first)" if oz else ""),
                      "arith": args.arith, "n": n, "tile": args.tile,
                      "l2": "inputs larger than L2 (3 x 8 n^2 bytes)"},
           "roofline": w["roofline"], "cpu_baseline": res["cpu_baseline"], "gemm_dag": res,
           "clocks": clocks, "gpu_launches": 2 * args.steps}
    if rank == 0:
        print(json.dumps(out))


def timed_graph_runs(spx, torch, build, restore, nsteps, nwarm, executor=0):
    """Run `build(g)` (insert) + execute + wait nwarm + nsteps times on a
    fresh graph each step (the full hot path); returns [(step_ms, kernel_ms)]."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    g = spx.Graph(executor=executor)
    rec = []
    for i in range(nwarm + nsteps):
        restore()
        ev[0].record()
        g.clear()
        build(g)
        g.execute()
        rc, _ = g.wait()
        ev[1].record()
        ev[1].synchronize()
        assert rc == spx.OK, rc
        if i >= nwarm:
            rec.append((ev[0].elapsed_time(ev[1]), g.timing()[1]))
    ntasks = g.sizes()[0]
    g.close()
    return rec, ntasks


def run_axpy(args, world, rank, local):
    """The paper's AXPY test case (FP32, a vector split into independent
    pieces): n = 2^28 values (x, y 1 GiB each), pieces of 2^14 .. 2^22 values;
    step = insert + derive + execute + wait.  HBM-bound: 12 bytes per value
    (read x, read and write y)."""
    import ctypes
    import torch
    from paper_2308_15964_b300 import inputs, spx
    n = args.n if args.n != 16384 else 1 << 28
    x = inputs.uniform((n,), 21, device="cuda").to(torch.float32)
    y0 = inputs.uniform((n,), 22, device="cuda").to(torch.float32)
    y = y0.clone()
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    hbm = peaks.get("hbm_gbs", 6400.0)
    nbytes = 12.0 * n
    alpha = 1.5

    def build_for(piece):
        def build(g):
            spx._check(spx.lib.spx_axpy_insert(g._h, ctypes.c_void_p(x.data_ptr()),
                                               ctypes.c_void_p(y.data_ptr()), n, piece, alpha,
                                               None), "spx_axpy_insert")
        return build

    rows = []
    with Clocks(local) as clk:
        for lg in (14, 16, 18, 20, 22):
            piece = 1 << lg
            row = {"piece": piece, "tasks": -(-n // piece)}
            for name, ex in (("persistent", spx.EXEC_PERSISTENT), ("per_task", spx.EXEC_PER_TASK),
                             ("streams", spx.EXEC_STREAMS)):
                steps = args.steps if name == "persistent" else COMPARATOR_STEPS
                rec, nt = timed_graph_runs(spx, torch, build_for(piece), lambda: None, steps,
                                           args.warmup if name == "persistent" else 1, ex)
                ms = statistics.mean(r[0] for r in rec)
                kern = statistics.mean(r[1] for r in rec)
                row[name] = {"ms_per_step": ms, "GBps": nbytes / (ms * 1e-3) / 1e9,
                             "tasks_per_s": nt / (ms * 1e-3), "kernel_ms": kern,
                             "kernel_GBps": nbytes / (kern * 1e-3) / 1e9,
                             "p99_ms": float(np.percentile([r[0] for r in rec], 99))}
            rows.append(row)
    clocks = clk.summary()
    head = [r for r in rows if r["piece"] == 1 << 20][0]
    # CPU oracle: the same loop on one host core over a bounded sample
    from oracle import oracle as O
    m = 1 << 24
    xs, ys = x[:m].cpu().numpy(), y0[:m].cpu().numpy().copy()
    t0 = time.perf_counter()
    O.axpy_f32(xs, ys, alpha)
    dt = time.perf_counter() - t0
    out = {"metric": METRIC, "value": head["persistent"]["GBps"], "unit": "GB/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": head["persistent"]["ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"AXPY FP32 y += {alpha} x, n = {n}, pieces of 2^20 "
                                  "(other piece sizes in rows); step = insert + derive + "
                                  "execute + wait", "n": n,
                      "l2": "inputs larger than L2 (8 n bytes)"},
           "tasks_per_s": head["persistent"]["tasks_per_s"], "rows": rows,
           "roofline": {"bound": "hbm", "achieved": head["persistent"]["kernel_GBps"],
                        "peak": hbm, "unit": "GB/s",
                        "frac": head["persistent"]["kernel_GBps"] / hbm, "traffic": None,
                        "kernel": "persistent_kernel (AXPY tile op)",
                        "note": "12 bytes per value: x read, y read and written; peak = the "
                                "measured copy bandwidth"},
           "cpu_baseline": {"value": 12.0 * m / dt / 1e9, "unit": "GB/s", "cores": 1,
                            "kind": "oracle", "sample": f"the oracle's FP32 loop on {m} values"},
           "clocks": clocks, "gpu_launches": 2 * args.steps}
    if rank == 0:
        print(json.dumps(out))


NBODY_FLOPS = 20   # per interaction: 3 sub, r^2 (5), sqrt, division, 3 mul, add, 3 FMA (6)


def run_nbody(args, world, rank, local):
    """The paper's particle test case (FP64 direct Coulomb sum, dependencies on
    whole groups): G = 64 groups of 128 .. 2048 particles (seeded), positions
    and charges uniform in [-1, 1]; tasks SELF(i) and PAIR(i, j) with WRITE on
    the groups (and a COMMUTATIVE_WRITE row).  Interactions = N (N - 1) per
    step; ALU-bound, against the measured rate of the same arithmetic."""
    import ctypes
    import torch
    from paper_2308_15964_b300 import inputs, spx
    G = 64
    u = inputs.uniform((G,), 61).numpy()
    sizes = (128 + np.floor((u + 1) / 2 * (2048 - 128 + 1))).astype(np.int64)
    sizes = np.minimum(sizes, 2048)
    N = int(sizes.sum())
    P0 = torch.zeros((N, 8), dtype=torch.float64, device="cuda")
    P0[:, 0:3] = inputs.uniform((N, 3), 62, device="cuda")
    P0[:, 3] = inputs.uniform((N,), 63, device="cuda")
    P = P0.clone()
    offs = np.concatenate([[0], np.cumsum(sizes)])
    ptrs = (ctypes.c_void_p * G)(*[P.data_ptr() + 64 * int(o) for o in offs[:-1]])
    sz = (ctypes.c_int * G)(*[int(v) for v in sizes])
    inter = float(N) * (N - 1)

    def build_for(comm):
        def build(g):
            spx._check(spx.lib.spx_nbody_insert(g._h, G, ptrs, sz, comm, None), "spx_nbody_insert")
        return build

    def restore():
        P.copy_(P0)

    probe_rate, _ = spx.probe(14, 2000)
    res = {}
    with Clocks(local) as clk:
        for name, ex, comm in (("write", spx.EXEC_PERSISTENT, 0),
                               ("commutative", spx.EXEC_PERSISTENT, 1),
                               ("per_task", spx.EXEC_PER_TASK, 0),
                               ("streams", spx.EXEC_STREAMS, 0)):
            steps = args.steps if name == "write" else COMPARATOR_STEPS
            rec, nt = timed_graph_runs(spx, torch, build_for(comm), restore, steps,
                                       args.warmup if name == "write" else 1, ex)
            ms = statistics.mean(r[0] for r in rec)
            kern = statistics.mean(r[1] for r in rec)
            res[name] = {"ms_per_step": ms, "interactions_per_s": inter / (ms * 1e-3),
                         "gflops": NBODY_FLOPS * inter / (ms * 1e-3) / 1e9, "tasks": nt,
                         "tasks_per_s": nt / (ms * 1e-3), "kernel_ms": kern,
                         "p99_ms": float(np.percentile([r[0] for r in rec], 99))}
    clocks = clk.summary()
    w = res["write"]
    # CPU oracle on a bounded sample: the first 4 groups
    from oracle import oracle as O
    k = 4
    Ph = P0[:int(offs[k])].cpu().numpy().copy()
    t0 = time.perf_counter()
    assert O.nbody(Ph, [int(v) for v in sizes[:k]]) == 0
    dt = time.perf_counter() - t0
    ns = int(offs[k])
    out = {"metric": METRIC, "value": w["gflops"], "unit": "GFLOP/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": w["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": f"particle interactions FP64: {G} groups, N = {N} particles "
                                  f"(sizes 128..2048), {len(sizes) * (len(sizes) + 1) // 2} tasks, "
                                  f"{NBODY_FLOPS} flops per interaction; step = insert + derive "
                                  "+ execute + wait", "groups": G, "N": N},
           "interactions_per_s": w["interactions_per_s"], "tasks_per_s": w["tasks_per_s"],
           "p50_ms": w["ms_per_step"], "p99_ms": w["p99_ms"], "executors": res,
           "roofline": {"bound": "alu", "achieved": inter / (w["kernel_ms"] * 1e-3),
                        "peak": probe_rate, "unit": "interactions/s",
                        "frac": inter / (w["kernel_ms"] * 1e-3) / probe_rate, "traffic": None,
                        "kernel": "persistent_kernel (NBODY tile ops)",
                        "note": "peak = spx_probe(SPX_PROBE_NBODY): the same FP64 interaction "
                                "arithmetic on register data over all SMs"},
           "cpu_baseline": {"value": NBODY_FLOPS * ns * (ns - 1) / dt / 1e9, "unit": "GFLOP/s",
                            "cores": 1, "kind": "oracle",
                            "sample": f"the oracle's task list on the first {k} groups "
                                      f"({ns} particles)"},
           "clocks": clocks, "gpu_launches": 2 * args.steps}
    if rank == 0:
        print(json.dumps(out))


def run_overhead(args, world, rank, local):
    """The paper's engine-overhead pattern on the device scheduler: T chains
    (T = the persistent CTAs) of N tasks that only busy-wait D; every task of a
    chain accesses the same d data objects with WRITE or COMMUTATIVE_WRITE.
    Execution ~ N (D + O): O = run time / N - D is the per-task overhead of
    the executor; I = host insertion time / (T N).  Also the global atomic
    rates behind the queue (probe)."""
    import ctypes
    from paper_2308_15964_b300 import spx
    T = 2 * spx.lib.spx_device_sm_count()  # the FP64 persistent kernel runs 2 CTAs per SM
    rows = []
    for comm in (0, 1):
        for d in (1, 5, 10, 16):
            for D_ns in (0, 10_000, 100_000):
                N = 20 if D_ns >= 100_000 else 40
                g = spx.Graph()
                nt = ctypes.c_longlong()
                t0 = time.perf_counter()
                spx._check(spx.lib.spx_overhead_insert(g._h, T, N, d, comm, D_ns, ctypes.byref(nt)),
                           "spx_overhead_insert")
                ins_ms = (time.perf_counter() - t0) * 1e3
                rc, _ = g.run()
                assert rc == spx.OK, rc
                prep_ms = g.timing()[0]
                runs = []
                for _ in range(3):
                    g.reset()
                    rc, _ = g.run()
                    assert rc == spx.OK, rc
                    runs.append(g.timing()[1])
                run_ms = min(runs)
                g.close()
                rows.append({"mode": "commutative" if comm else "write", "deps": d, "D_us": D_ns / 1e3,
                             "chains": T, "tasks_per_chain": N,
                             "overhead_us": run_ms * 1e3 / N - D_ns / 1e3,
                             "insert_us_per_task": ins_ms * 1e3 / (T * N),
                             "derive_ms": prep_ms, "run_ms": run_ms,
                             "tasks_per_s": T * N / (run_ms * 1e-3)})
    same, _ = spx.probe(3, 2000)
    distinct, _ = spx.probe(4, 2000)
    nop = [r for r in rows if r["mode"] == "write" and r["deps"] == 1 and r["D_us"] == 0][0]
    out = {"metric": METRIC, "value": nop["tasks_per_s"], "unit": "tasks/s", "n_gpus": world,
           "steps": 3, "warmup": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "data": "synthetic",
           "config": {"workload": "engine overhead: T chains x N busy-wait tasks, d data objects per "
                                  "task (write or commutative write), D in {0, 10, 100} us"},
           "atomics_per_s": {"same_address": same, "distinct_addresses": distinct},
           "rows": rows}
    if rank == 0:
        print(json.dumps(out))


def run_stream(args, world, rank, local):
    """Streaming insertion (spx_stream_begin / flush / end) on the split-path
    Cholesky with substitution panels: the host inserts panel k's tasks one
    call at a time (Python, spx_task_insert) and flushes them while the
    kernel runs the earlier panels.  Time to solution by the host clock, from
    the first insertion to the return of the wait, against inserting every
    task first (the same Python calls) and then executing, and against the
    C insertion of the whole graph (spx_cholesky_insert_ozaki) + execution."""
    import torch
    from paper_2308_15964_b300 import cholesky, inputs, spx
    n, b = args.n, args.tile
    T = -(-n // b)
    A0 = inputs.spd_matrix(n, args.sigma, seed=2, device="cuda")
    A = torch.empty_like(A0)
    store = cholesky.ozaki_store(n, b)
    slot = spx.lib.spx_ozaki_slot_bytes(b)
    OZ, R, W = spx.F64_OZAKI, spx.READ, spx.WRITE

    def tiles(g):
        g.register_ozaki(store.data_ptr(), max(1, T * (T - 1) // 2), b)
        h = [[None] * T for _ in range(T)]
        for i in range(T):
            for j in range(i + 1):
                lo = store.data_ptr() + (i * (i - 1) // 2 + j) * slot if i > j else 0
                h[i][j] = g.register(A[i * b:, j * b:].data_ptr(), min(b, n - i * b),
                                     min(b, n - j * b), n, spx.DT_F64, lo, b if lo else 0)
        return h

    def panel(g, h, k):
        t = g.insert(spx.OP_POTRF, [h[k][k]], [W], 2)
        g.set_arg(t, k * b)
        for i in range(k + 1, T):
            g.insert(spx.OP_TRSM, [h[k][k], h[i][k]], [R, W], 2 if i == k + 1 else 1, OZ)
        for i in range(k + 1, T):
            g.insert(spx.OP_SYRK, [h[i][k], h[i][i]], [R, W], 2 if i == k + 1 else 1, OZ)
        for j in range(k + 1, T):
            for i in range(j + 1, T):
                g.insert(spx.OP_GEMM_NT_SUB, [h[i][k], h[j][k], h[i][j]], [R, R, W],
                         (2 if i == k + 2 else 1) if j == k + 1 else 0, OZ)

    ntasks = T + T * (T - 1) + T * (T - 1) * (T - 2) // 6
    rows = {"streamed": [], "insert_then_execute": [], "c_insert_then_execute": []}
    L = {}
    for it in range(args.warmup + args.steps):
        for mode in rows:
            A.copy_(A0)
            torch.cuda.synchronize()
            g = spx.Graph()
            h = tiles(g) if mode != "c_insert_then_execute" else None
            t0 = time.perf_counter()
            if mode == "streamed":
                panel(g, h, 0)  # fixes the kernel family (split tasks)
                g.stream_begin(max_tasks=2 * ntasks + 4 * T, max_tiles=T * T, max_records=4 * ntasks,
                               max_preds=16 * ntasks)
                for k in range(1, T):
                    panel(g, h, k)
                    g.stream_flush()
                g.stream_end()
                rc, _ = g.wait()
            elif mode == "insert_then_execute":
                for k in range(T):
                    panel(g, h, k)
                rc, _ = g.run()
            else:
                cholesky.cholesky_ozaki_graph(g, A, b, S=store)
                rc, _ = g.run()
            dt = time.perf_counter() - t0
            assert rc == spx.OK, (mode, rc)
            g.close()
            if it >= args.warmup:
                rows[mode].append(dt)
            if it == args.warmup + args.steps - 1:
                L[mode] = torch.tril(A).clone()
    flops = n ** 3 / 3.0
    same = all(torch.equal(L["streamed"], L[m]) for m in L)
    out = {"metric": "Cholesky GFLOP/s, time to solution with streamed insertion (host clock)",
           "value": flops / statistics.mean(rows["streamed"]) / 1e9, "unit": "GFLOP/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * statistics.mean(rows["streamed"]), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64 (split products)",
           "data": "synthetic",
           "config": {"workload": f"split-path Cholesky n={n} tile={b} ({ntasks} tasks), tasks "
                                  "inserted from Python one call each, flushed per panel",
                      "n": n, "tile": b, "tasks": ntasks},
           "rows_ms": {m: {"mean": 1e3 * statistics.mean(v), "p99": 1e3 * float(np.percentile(v, 99))}
                       for m, v in rows.items()},
           "factors_bit_identical": bool(same),
           "gpu_launches": 1}
    if rank == 0:
        print(json.dumps(out))


def run_splitgemm(args, world, rank, local):
    """Stand-alone rate of the split-FP64 product: the T (T - 1) GEMM_NT_SUB
    tasks C_ij -= A_i A_j^T (i != j) of T = n / b tiles in one graph, after
    each A_i was split by a TRSM with an identity diagonal tile (which solves
    nothing: only its split phase matters).  The product time is the run
    with the products minus the run with the splits alone."""
    import torch
    from paper_2308_15964_b300 import spx
    b = args.tile
    T = max(2, args.n // b)
    slot = spx.lib.spx_ozaki_slot_bytes(b)
    store = torch.zeros(T * slot, dtype=torch.uint8, device="cuda")
    gen = torch.Generator(device="cuda").manual_seed(11)
    A = [torch.rand(b, b, dtype=torch.float64, device="cuda", generator=gen) * 2 - 1 for _ in range(T)]
    C = torch.zeros(T * b, T * b, dtype=torch.float64, device="cuda")
    eye = torch.eye(b, dtype=torch.float64, device="cuda")

    def graph(products):
        g = spx.Graph()
        g.register_ozaki(store.data_ptr(), T, b)
        hI = g.register_tensor(eye)
        hA = [g.register(A[i].data_ptr(), b, b, b, spx.DT_F64, store.data_ptr() + i * slot, b)
              for i in range(T)]
        for i in range(T):
            g.insert(spx.OP_TRSM, [hI, hA[i]], [spx.READ, spx.WRITE], prec=spx.F64_OZAKI)
        for i in range(T if products else 0):
            for j in range(T):
                if i != j:
                    hc = g.register(C[i * b:(i + 1) * b, j * b:(j + 1) * b].data_ptr(), b, b,
                                    T * b, spx.DT_F64)
                    g.insert(spx.OP_GEMM_NT_SUB, [hA[i], hA[j], hc], [spx.READ, spx.READ, spx.WRITE],
                             prec=spx.F64_OZAKI)
        return g

    def timed(products):
        g = graph(products)
        ms = []
        for i in range(args.warmup + args.steps):
            if i:
                g.reset()
            rc, _ = g.run()
            assert rc == spx.OK
            if i >= args.warmup:
                ms.append(g.timing()[1])
        st = g.stats()
        g.close()
        return ms, st

    with Clocks(local) as clk:
        split_ms, _ = timed(False)
        full_ms, st = timed(True)
    prod_ms = statistics.mean(full_ms) - statistics.mean(split_ms)
    tasks = T * (T - 1)
    fp64_flops = tasks * 2.0 * b ** 3
    tensor_flops = 36.0 * fp64_flops
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    bf16 = peaks.get("bf16_tflops", 1800.0)
    ach = tensor_flops / (prod_ms * 1e-3) / 1e12
    out = {"metric": "split-FP64 GEMM TFLOP/s (FP64-equivalent)", "value": fp64_flops / (prod_ms * 1e-3) / 1e12,
           "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": prod_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64 (Ozaki split, bf16 digit planes)", "data": "synthetic uniform[-1,1)",
           "config": {"workload": f"{tasks} GEMM_NT_SUB tasks on {T} split {b} x {b} tiles, one launch",
                      "tile": b, "tiles": T, "tasks": tasks},
           "kernel_ms": {"splits_only": statistics.mean(split_ms), "splits_and_products": statistics.mean(full_ms)},
           "gpu_launches": 2 * args.steps,
           "roofline": {"bound": "tensor", "achieved": ach, "peak": bf16, "unit": "TFLOP/s",
                        "frac": ach / bf16, "traffic": None,
                        "kernel": "persistent_kernel<split products> (one CTA per SM)",
                        "note": "36 digit-pair products of 2 b^3 flops per task over the product time"},
           "sched": {"busy_frac": st["busy_cycles"] / max(1, st["total_cycles"])},
           "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(out))


def run_tc(args, world, rank, local):
    """Stand-alone tensor-core tile update C (FP64, m x m) -= A B^T with BF16 and
    TF32 operands (m x K): the trailing-update kernel of the mixed path."""
    import ctypes
    import torch
    from paper_2308_15964_b300 import spx
    m, K = args.n if args.n != 16384 else 8192, args.tile if args.tile != 512 else 1024
    C = torch.zeros((m, m), dtype=torch.float64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = {"metric": METRIC, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "data": "synthetic", "config": {"workload": f"tensor-core tile update C(fp64 {m}x{m}) -= "
                                                       f"A({m}x{K}) B({m}x{K})^T", "m": m, "K": K}}
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    P = ctypes.c_void_p
    st = torch.cuda.current_stream()
    for name, prec, dt in (("bf16", spx.BF16, torch.bfloat16), ("tf32", spx.TF32, torch.float32)):
        A = (torch.rand((m, K), device="cuda") * 2 - 1).to(dt)
        B = (torch.rand((m, K), device="cuda") * 2 - 1).to(dt)
        call = lambda: spx.lib.spx_tc_gemm_nt(P(C.data_ptr()), m, m, m, P(A.data_ptr()), K,
                                              P(B.data_ptr()), K, K, prec, P(err.data_ptr()),
                                              P(st.cuda_stream))
        for _ in range(args.warmup):
            call()
        ev[0].record()
        for _ in range(args.steps):
            call()
        ev[1].record()
        ev[1].synchronize()
        ms = ev[0].elapsed_time(ev[1]) / args.steps
        flops = 2.0 * m * m * K
        bytes_ = 16.0 * m * m + 2 * m * K * A.element_size()
        out[name] = {"ms": ms, "tflops": flops / ms / 1e9, "gbs": bytes_ / ms / 1e6,
                     "frac_hbm": bytes_ / ms / 1e6 / peaks.get("hbm_gbs", 6451.5),
                     "frac_bf16_peak": flops / ms / 1e9 / peaks.get("bf16_tflops", 1736.0)}
    assert int(err.item()) == 0
    out["value"] = out["bf16"]["tflops"]
    out["ms_per_step"] = out["bf16"]["ms"]
    out["roofline"] = {"bound": "hbm", "achieved": out["bf16"]["gbs"], "peak": peaks.get("hbm_gbs", 6451.5),
                       "unit": "GB/s", "frac": out["bf16"]["frac_hbm"], "traffic": None,
                       "kernel": "tc_gemm_kernel<bf16>",
                       "note": "algorithmic bytes: FP64 C read+write 16 m^2 + operands"}
    if rank == 0:
        print(json.dumps(out))


def run_serve(args, world, rank, local):
    """Serving: Poisson stream (seeded) of Cholesky-solve requests, n log-uniform
    in [64, 16384], 1..64 RHS, FP64 or TF32 + 4 FP64 refinement sweeps,
    admitted under a 120 GB HBM budget into one resident server kernel."""
    from paper_2308_15964_b300 import serve
    with Clocks(local) as clk:
        out = serve.serve(rate=args.rate, duration=args.duration, budget=120e9, seed=6 + rank,
                          drain=False, max_wall=args.duration + 120,
                          split_fp64=args.arith == "ozaki")
    res = {"metric": METRIC, "value": out["gflops"], "unit": "GFLOP/s", "n_gpus": world,
           "steps": 1, "warmup": 0, "ms_per_step": out["wall_s"] * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": ("f64 (orders >= %d by split products on the tensor cores) / tf32+f64 refinement"
                     % serve.SPLIT_MIN_N) if args.arith == "ozaki" else "f64 / tf32+f64 refinement",
           "data": "synthetic",
           "config": {"workload": f"serving: Poisson {args.rate}/s for {args.duration} s, n log-uniform "
                                  "64..16384, 1..64 RHS, 50% TF32+refinement, 120 GB budget",
                      "rate": args.rate, "duration_s": args.duration, "arith": args.arith},
           "p50_ms": out["p50_ms"], "p99_ms": out["p99_ms"], "serve": out, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(res))


def run_mixed(args, world, rank, local):
    """Mixed precision: TF32 and BF16 tensor-core trailing updates, FP64 POTRF,
    FP64 refinement of 8 right-hand sides to eta <= 1e-14 (n = 32768, tile 512,
    sigma = 1e-3 unless given)."""
    import torch
    from paper_2308_15964_b300 import cholesky, inputs, mixed, spx
    n = args.n if args.n != 16384 else 32768
    b, nrhs = args.tile, 8
    sigma = args.sigma if args.sigma != 0.1 else 1e-3
    A0 = inputs.spd_matrix(n, sigma, seed=4 + rank, device="cuda")
    B = inputs.rhs(n, nrhs, seed=4 + rank, device="cuda")
    out = {"metric": METRIC, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "tf32/bf16 updates, f64 potrf+refinement", "data": "synthetic",
           "config": {"workload": f"mixed-precision Cholesky n={n} tile={b}, {nrhs} RHS, "
                                  f"A = B B^T/n + {sigma} I, FP64 refinement to eta <= 1e-14",
                      "n": n, "tile": b, "nrhs": nrhs, "sigma": sigma}}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    last = {}
    with Clocks(local) as clk:
        for name, prec in (("tf32", spx.TF32), ("bf16", spx.BF16)):
            runs = []
            for i in range(args.warmup + args.steps):
                last.pop(name, None)
                ev[0].record()
                X, L, info = mixed.mixed_solve(A0, B, b=b, prec=prec)
                ev[1].record()
                ev[1].synchronize()
                if i >= args.warmup:
                    runs.append((ev[0].elapsed_time(ev[1]), info))
                last[name] = (X, L)
                del X, L
            ms = statistics.mean(r[0] for r in runs)
            inf = runs[-1][1]
            fac = statistics.mean(r[1]["factor_ms"] for r in runs)
            flops = cholesky.cholesky_flops(n, nrhs)
            out[name] = {"ms_per_solve": ms, "factor_ms": fac,
                         "refine_ms": statistics.mean(r[1]["refine_ms"] for r in runs),
                         "ms_per_solve_runs": [round(r[0], 2) for r in runs],
                         "gflops_total": flops / (ms * 1e-3) / 1e9,
                         "factor_gflops": n ** 3 / 3 / (fac * 1e-3) / 1e9,
                         "converged": inf["converged"], "iterations": inf["iterations"],
                         "eta_device": inf["eta_final"],
                         "eta_history": inf["eta"],
                         "eta_history_compensated": inf["eta_compensated"],
                         "correction_solve": inf.get("correction"),
                         "factor_cta_time_share": {k: round(v, 4) for k, v in
                                                   inf.get("factor_op_share", {}).items()}}
    # GMRES-based refinement from the same kind of factor (Carson-Higham):
    # each step solves the correction equation by FP64 GMRES preconditioned
    # with the factor
    for name, prec in (("tf32", spx.TF32), ("bf16", spx.BF16)):
        gr = []
        for i in range(1 + args.steps):
            ev[0].record()
            X, L, info = mixed.gmres_ir_solve(A0, B, b=b, prec=prec)
            ev[1].record()
            ev[1].synchronize()
            if i >= 1:
                gr.append((ev[0].elapsed_time(ev[1]), info))
            last[name + "_gmres"] = (X, L)
            del X, L
        gi = gr[-1][1]
        out[name]["gmres_ir"] = {"ms_per_solve": statistics.mean(r[0] for r in gr),
                                 "factor_ms": statistics.mean(r[1]["factor_ms"] for r in gr),
                                 "refine_ms": statistics.mean(r[1]["refine_ms"] for r in gr),
                                 "converged": gi["converged"], "outer": gi["outer"],
                                 "inner": gi["inner"], "eta_device": gi["eta_final"]}
    if rank == 0:
        # The oracle's checks of the last run of each precision (host, one
        # core): normwise backward error of X with compensated residuals, and
        # a Freivalds probe ||A v - L (L^T v)|| / (||A||_F ||v||) of the
        # low-precision factor (its backward error, of order the precision).
        from oracle import oracle as O
        A0h, Bh = A0.cpu().numpy(), B.cpu().numpy()
        v = inputs.gaussian(n, 9)
        for name in ("tf32", "bf16"):
            X, L = last[name]
            Xh = X.cpu().numpy()
            del X
            t0 = time.perf_counter()
            eta = O.solve_backward_error(A0h, Xh, Bh)
            t1 = time.perf_counter()
            Lh = L.cpu().numpy()
            del L
            fr = O.freivalds(A0h, Lh, v)
            t2 = time.perf_counter()
            del Lh
            out[name]["eta_oracle"] = float(eta.max())
            out[name]["eta_oracle_per_rhs"] = [float(x) for x in eta]
            out[name]["factor_freivalds_oracle"] = fr
            out[name]["oracle_check_s"] = {"eta": t1 - t0, "freivalds": t2 - t1}
            Xg, _ = last[name + "_gmres"]
            out[name]["gmres_ir"]["eta_oracle"] = float(
                O.solve_backward_error(A0h, Xg.cpu().numpy(), Bh).max())
        del A0h
    last.clear()
    out["value"] = out["tf32"]["gflops_total"]
    out["ms_per_step"] = out["tf32"]["ms_per_solve"]
    out["clocks"] = clk.summary()
    # Roofline of the factorization (the trailing updates dominate its bytes
    # and flops): with the factor tiles' low-precision copies as operands and
    # the trailing matrix in FP64 (read and written, 16 bytes per element per
    # update), the algorithmic traffic is sum_k 16 (n - k b)^2 / 2 ~ 16 n^3 /
    # (6 b) bytes; the n^3 / 3 flops on the tensor cores take less time at
    # the measured BF16 rate (TF32: half of it), so HBM bounds it.
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    hbm = peaks.get("hbm_gbs", 6400.0)
    tbytes = 16.0 * n ** 3 / (6.0 * b)
    fac_ms = out["tf32"]["factor_ms"]
    out["roofline"] = {"bound": "hbm", "achieved": tbytes / (fac_ms * 1e-3) / 1e9, "peak": hbm,
                       "unit": "GB/s", "frac": tbytes / (fac_ms * 1e-3) / 1e9 / hbm,
                       "traffic": None,
                       "kernel": "persistent_kernel<tensor cores> (TF32 factorization)",
                       "note": f"algorithmic trailing-update bytes 16 n^3 / (6 b) = "
                               f"{tbytes / 1e9:.0f} GB over the TF32 factor time "
                               f"({fac_ms:.0f} ms, insertion and derivation included); the "
                               "factor is bound by its chain of FP64 diagonal POTRF steps "
                               "(64 x about 1.3 ms), not by HBM"}
    if rank == 0:
        print(json.dumps(out))


def run_batch(args, world, rank, local):
    """Batched uneven solves: one graph, one persistent launch per batch; the
    autotuner picks each order's tile; re-runs replay a CUDA graph."""
    import torch
    from paper_2308_15964_b300 import batch as Bt
    from paper_2308_15964_b300 import spx
    n, r = Bt.problem_sizes(args.count, seed=5 + rank)
    split = args.arith == "ozaki"
    t0 = time.perf_counter()
    best, table = Bt.autotune(n, split=split)
    tune_s = time.perf_counter() - t0
    tiles = [best[int(k)] for k in n]
    bt = Bt.Batch(n, r, seed=5 + rank)
    flops = bt.flops()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    g = spx.Graph(cuda_graph=True)
    # full hot path once per warm-up step: insert + derive + execute
    full = []
    for _ in range(max(1, args.warmup)):
        bt.restore()
        ev[0].record()
        g.clear()
        ntasks = Bt.insert(g, bt, tiles, split=split)
        rc, _ = g.run()
        ev[1].record()
        ev[1].synchronize()
        assert rc == spx.OK, rc
        full.append(ev[0].elapsed_time(ev[1]))
    g.reset()
    bt.restore()
    assert g.run()[0] == spx.OK          # captures the replay graph
    recs = []
    torch.cuda.synchronize()
    barrier(world)
    with Clocks(local) as clk:
        for _ in range(args.steps):
            g.reset()
            bt.restore()
            ev[0].record()
            rc, _ = g.run()
            ev[1].record()
            ev[1].synchronize()
            assert rc == spx.OK
            recs.append((ev[0].elapsed_time(ev[1]), g.timing()[1]))
        barrier(world)
    step_ms = [x[0] for x in recs]
    total_ms = max_over_ranks(sum(step_ms), world)
    value = world * args.steps * flops / (total_ms * 1e-3) / 1e9
    sms = spx.lib.spx_device_sm_count()
    clocks = clk.summary()
    peak = FP64_DFMA_PER_CLK_SM * 2 * sms * (clocks.get("sm_max_mhz") or 2032.0) * 1e6 / 1e12
    kern = statistics.mean(x[1] for x in recs)
    out = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f64 (trailing updates and panel products split on the tensor cores)" if split
           else "f64", "data": "synthetic",
           "config": {"workload": f"batched uneven Cholesky solves: {args.count} problems, n in "
                                  "32..1024 (multiples of 32), 1..16 RHS, autotuned tiles, "
                                  "one persistent launch, CUDA-graph replay",
                      "count": args.count, "tasks": ntasks, "parallelism": f"replicas x{world}",
                      "arith": args.arith},
           "tasks_per_s": ntasks / (statistics.mean(step_ms) * 1e-3),
           "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
           "full_step_ms": statistics.mean(full),
           "autotune": {"seconds": tune_s, "tile_of_n": {str(k): v for k, v in best.items()}},
           "gpu_launches": 2 * args.steps, "clocks": clocks,
           "roofline": {"bound": "alu", "achieved": flops / (kern * 1e-3) / 1e12, "peak": peak,
                        "unit": "TFLOP/s", "frac": flops / (kern * 1e-3) / 1e12 / peak,
                        "traffic": None, "kernel": "persistent_kernel", "kernel_ms": kern}}
    if split:  # the tensor-core bound over the digit-pair flops, the FP64 share beside it
        tf, ff = (sum(x) for x in zip(*(ozaki_work(int(k), int(b)) for k, b in zip(n, tiles))))
        bf16 = (json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}).get(
            "bf16_tflops", 1800.0)
        ach = tf / (kern * 1e-3) / 1e12
        out["roofline"] = {"bound": "tensor", "achieved": ach, "peak": bf16, "unit": "TFLOP/s",
                           "frac": ach / bf16, "traffic": None,
                           "kernel": "persistent_kernel<split products> (one CTA per SM)",
                           "kernel_ms": kern, "tensor_tflop_per_launch": tf / 1e12,
                           "fp64_simt": {"flops_per_launch": ff,
                                         "frac": ff / (kern * 1e-3) / 1e12 / peak}}
    if rank == 0:
        gb = spx.Graph(executor=spx.EXEC_PER_TASK, cuda_graph=True)
        Bt.insert(gb, bt, tiles, split=split)
        bms = []
        for i in range(3):
            bt.restore()
            ev[0].record()
            rc, _ = gb.run()
            ev[1].record()
            ev[1].synchronize()
            assert rc == spx.OK
            gb.reset()
            if i > 0:
                bms.append(ev[0].elapsed_time(ev[1]))
        out["baseline_per_task_cudagraph"] = {"value": flops / (statistics.mean(bms) * 1e-3) / 1e9,
                                              "unit": "GFLOP/s", "ms_per_step": statistics.mean(bms)}
        gb.close()
        print(json.dumps(out))
    g.close()


def small_latency(spx, cholesky, inputs, torch, reps=200):
    """Latency of the small case: n=512, tile 64, A = B B^T/n + I (seed 1),
    one right-hand side: the factorization (120 tasks) and the block solve
    (72 tasks) in one graph of 192 tasks.  Host wall time of execute -> wait
    on a reset graph, persistent vs the per-task executors (one stream; the
    same through a CUDA graph; four streams with event waits); the
    factorization alone beside it.  Then the critical path of one traced
    persistent run, split into the time tasks run and the time between a
    predecessor's end and the task's start (release + pop)."""
    n, b = 512, 64
    A0 = inputs.spd_matrix(n, 1.0, seed=1, device="cuda")
    X0 = inputs.rhs(n, 1, seed=1, device="cuda")
    A, X = torch.empty_like(A0), torch.empty_like(X0)
    flops_fs = cholesky.cholesky_flops(n, 1)
    res = {}
    for name, ex, rederive, cg, solve, la in (
            ("persistent", spx.EXEC_PERSISTENT, False, False, True, 1),
            ("persistent_all_critical", spx.EXEC_PERSISTENT, False, False, True, 2),
            ("persistent_bottom_level", -1, False, False, True, 1),
            ("persistent_factor_only", spx.EXEC_PERSISTENT, False, False, False, 1),
            ("persistent_insert_derive", spx.EXEC_PERSISTENT, True, False, True, 1),
            ("per_task", spx.EXEC_PER_TASK, False, False, True, 1),
            ("per_task_cudagraph", spx.EXEC_PER_TASK, False, True, True, 1),
            ("streams", spx.EXEC_STREAMS, False, False, True, 1)):
        g = (spx.Graph(priorities=1) if ex < 0 else spx.Graph(executor=ex, cuda_graph=cg))
        Xs = X if solve else None
        ntasks = cholesky.cholesky_graph(g, A, b, Xs, lookahead=la)
        lat = []
        for i in range(reps + 5):
            A.copy_(A0)
            X.copy_(X0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if rederive and i > 0:
                g.clear()
                cholesky.cholesky_graph(g, A, b, Xs, lookahead=la)
            g.execute()
            rc, _ = g.wait()
            t1 = time.perf_counter()
            assert rc == spx.OK
            if not rederive:
                g.reset()
            if i >= 5:
                lat.append((t1 - t0) * 1e3)
        fl = flops_fs if solve else cholesky.cholesky_flops(n)
        res[name] = {"tasks": ntasks, "p50_ms": float(np.percentile(lat, 50)),
                     "p99_ms": float(np.percentile(lat, 99)),
                     "gflops": fl / (np.median(lat) * 1e-3) / 1e9}
        g.close()
    res["workload"] = ("n=512 tile=64, 1 RHS: factorization + block solve, 192 tasks (the "
                       "_factor_only row: the 120 factorization tasks); host wall time of "
                       "execute->wait over %d runs; the graph is reset and re-run, except "
                       "persistent_insert_derive, which inserts and derives every time; "
                       "_bottom_level: priorities from the critical path (cfg.priorities = 1) "
                       "instead of the look-ahead marks; _all_critical: every task on the "
                       "critical-path queue with the finer parts (lookahead = 2)" % reps)
    res["critical_path"] = critical_path_trace(spx, cholesky, torch, A, A0, X, X0, b)
    res["critical_path_bottom_level"] = critical_path_trace(spx, cholesky, torch, A, A0, X, X0, b,
                                                            priorities=1)
    return res


def critical_path_trace(spx, cholesky, torch, A, A0, X, X0, b, priorities=0):
    """Critical path of one traced persistent run of the small case: walk back
    from the last task to finish, each time to the predecessor that finished
    last; per task on that path, the time it ran (first part start to last
    part end, %globaltimer) and the gap since that predecessor's end (the
    release of its successors, the pop, and the wait for a free CTA)."""
    g = spx.Graph(trace=True, priorities=priorities)
    cholesky.cholesky_graph(g, A, b, X)
    runs = []
    for _ in range(6):
        A.copy_(A0)
        X.copy_(X0)
        torch.cuda.synchronize()
        g.execute()
        assert g.wait()[0] == spx.OK
        runs.append(g.trace().astype(np.int64))
        g.reset()
    rp, col, _ = g.edges()
    ops, prio = g.task_ops()
    g.close()
    N = len(ops)
    preds = [[] for _ in range(N)]
    for u in range(N):
        for v in col[rp[u]:rp[u + 1]]:
            preds[int(v)].append(u)
    out = []
    for tr in runs[1:]:
        start, end = tr[:, 0], tr[:, 1]
        u = int(np.argmax(end))
        chain = [u]
        while preds[u]:
            u = max(preds[u], key=lambda p: end[p])
            chain.append(u)
        chain.reverse()
        rows = []
        for i, t in enumerate(chain):
            gap = 0 if i == 0 else int(start[t] - end[chain[i - 1]])
            rows.append((spx.OP_NAMES[ops[t]], int(end[t] - start[t]), gap, int(tr[t, 3])))
        out.append({"span_us": (end.max() - start.min()) / 1e3, "rows": rows})
    best = min(out, key=lambda r: r["span_us"])
    by_op = {}
    for name, run_ns, gap_ns, parts in best["rows"]:
        d = by_op.setdefault(name, {"tasks": 0, "run_us": 0.0, "gap_us": 0.0, "parts": 0})
        d["tasks"] += 1
        d["run_us"] += run_ns / 1e3
        d["gap_us"] += gap_ns / 1e3
        d["parts"] += parts
    run_us = sum(r[1] for r in best["rows"]) / 1e3
    gap_us = sum(r[2] for r in best["rows"]) / 1e3
    return {"tasks_on_path": len(best["rows"]), "span_us": best["span_us"],
            "run_us": run_us, "gap_us": gap_us,
            "per_task_us": best["span_us"] / len(best["rows"]),
            "spans_us_of_5_runs": [round(r["span_us"], 1) for r in out],
            "by_op": {k: {kk: round(vv, 2) if isinstance(vv, float) else vv
                          for kk, vv in v.items()} for k, v in by_op.items()},
            "path": [{"op": r[0], "run_us": round(r[1] / 1e3, 2), "gap_us": round(r[2] / 1e3, 2),
                      "parts": r[3]} for r in best["rows"]],
            "note": "device %globaltimer; the fastest of 5 traced runs; gap = start of the task "
                    "minus end of its latest-finishing predecessor"}


if __name__ == "__main__":
    main()
