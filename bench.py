"""Benchmark: PCG solves/s at a true relative residual of 1e-6, mixed
precision against plain float64, on the precision-form instance (n = 65536
uniform locations in a 1 km square, d = 64, lambda = 1e-4, 8 transmitters,
N_r = 2048 random directions, 512 x 512 query grid).

One step = the whole hot path on one instance: kernel construction, CCCP
preconditioner fit, mixed-precision PCG (split-bf16 tensor-core operator,
float64 scalars, float64-accurate residual every 20 products) to the true
tolerance, radio-map evaluation.  Inputs are resident in HBM when the timed
region starts (`value`); `e2e` repeats the step through the same public API
with pinned host buffers copied in and the results copied out inside the timed
region.  The plain float64 path (the paper's method run in float64
throughout) is timed on the same instance in the same run, and the line
reports the mixed alpha's error against it and the dB RMSE of the two maps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload n65536_d64|n16384_d32|n1024_fp64|batched|learned|
                              sweep|variants|combined|streaming]

Multi-GPU: the instance does not shard; N ranks run N independent replicas
(different seeds), `value` = instances solved by all ranks / max rank time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2604_25138_gb300 import synth  # noqa: E402

METRIC = "PCG solves/s at rel-res 1e-6 (mixed, vs plain FP64)"
UNIT = "solves/s"
# single-instance workloads: the precision form (headline) and the larger
# plain-method instance
SINGLE = {
    "n65536_d64": dict(name="precision form: single instance, n=65536 uniform, d=64, lambda=1e-4, 8 Tx, 512x512 grid",
               n=65536, d=64, lam=1e-4, n_tx=8, layout="uniform", grid=512, tol=1e-6, refine_every=20, seed=3000),
    "n16384_d32": dict(name="single instance, n=16384 (70% uniform, 30% in 5 blobs), d=32, lambda=1e-4, 8 Tx, 512x512 grid",
               n=16384, d=32, lam=1e-4, n_tx=8, layout="clustered", grid=512, tol=1e-6, refine_every=20, seed=2000),
    "n1024_fp64": dict(name="plain method in float64: single instance, n=1024 uniform, d=16, lambda=1e-3, 3 Tx, 64x64 grid",
               n=1024, d=16, lam=1e-3, n_tx=3, layout="uniform", grid=64, tol=1e-8, refine_every=0, seed=1000,
               precision="FP64"),
}
# the bounded oracle sample timed on the host cores: the same generator as the
# workload at n = 2048 (the dense oracle's CCCP costs O(n^3) per iteration:
# ~12 s at n = 2048, ~50 s at n = 4096 and ~5 min at n = 8192 on 8 cores)
CPU_SAMPLE_N = 2048
CPU_SAMPLE_GRID = 64
# DRAM bytes (read + write) of one k_mf_bf16x3<64> launch at n = 65536, d = 64
# from a one-pass ncu capture of the current kernel (17.09 MB read: the split
# operands once; 13.70 MB written: partials); profiles/k_mf_bf16x3_n16384_d64.md
# gives the command.  None for any other workload.
MF_TRAFFIC_BYTES_C3 = 30.79e6
SFU_EX2_PER_CLK_PER_SM = 32   # ex2.approx results per clock per SM (micro-benchmarked on GB300)
FP64_NOMINAL_TFLOPS = 1.25    # dense float64 rate of GB300 (nominal)


def workload(cfg: dict, seed: int, n: int | None = None, grid: int | None = None):
    n = cfg["n"] if n is None else n
    inst = synth.make_instance(n, cfg["d"], cfg["lam"], n_tx=cfg["n_tx"], seed=seed, layout=cfg["layout"],
                               grid=cfg["grid"] if grid is None else grid)
    n_r = synth.default_num_directions(n)
    Z = synth.directions(n, n_r, seed)
    return inst, Z, n_r


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p["hbm_gbs"], "measured"
    except Exception:
        return 6800.0, "fallback"


def peaks_bf16():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p["bf16_tflops"], "measured"
    except Exception:
        return 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, device: int):
        self.proc = None
        self.device = device
        where = os.environ.get("LAKER_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(where, f"laker_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()
        return False

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# Our CUDA path
# ---------------------------------------------------------------------------

def rank_env():
    """(world size, rank, local rank) of a torchrun launch; (1, 0, 0) without one."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def job_ms(ms: float, world: int, device) -> float:
    """The job's time for `world` replicas: the slowest rank's, by a MAX
    all-reduce over the process group (every rank gets it)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, ms: float) -> float:
    """Whole-job throughput: the units all ranks processed over the job's time."""
    return world * units_per_rank / (ms / 1e3)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2604_25138_gb300 import build
    from paper_2604_25138_gb300 import laker as L

    cfg = SINGLE[args.workload]
    world, rank, local = rank_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    build.build()
    dev_t = torch.device("cuda", local)
    inst, Zh, n_r = workload(cfg, cfg["seed"] + rank)
    n = inst.n

    def to_dev(x):
        return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device=dev_t)

    Q, y, Z, Qg = to_dev(inst.Q), to_dev(inst.y), to_dev(Zh), to_dev(inst.Qg)
    ctx = L.Context(local)

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(ctx.stream)
        return e

    def step(Q, y, Z, Qg, precision, refine, tol, keep=False, phases=None):
        e0 = ev()
        op = L.laker_build_kernel(ctx, Q, inst.scale, inst.lam, precision)
        e1 = ev()
        P = L.laker_fit_preconditioner(ctx, op, Z)
        e2 = ev()
        alpha, info = L.laker_pcg_solve(ctx, op, P, y, tol, max_iter=40000, refine_every=refine)
        e3 = ev()
        fmap = L.laker_eval_map(ctx, op, Qg, alpha)
        e4 = ev()
        if phases is not None:
            e4.synchronize()
            phases.append({"build": e0.elapsed_time(e1), "fit": e1.elapsed_time(e2), "solve": e2.elapsed_time(e3),
                           "map": e3.elapsed_time(e4)})
        P.close()
        if not keep:
            op.close()
            op = None
        return alpha, fmap, info, P.info, op

    prec_name = cfg.get("precision", "BF16X3")
    fp64_only = prec_name == "FP64"
    mixed = dict(precision=getattr(L, prec_name), refine=cfg["refine_every"], tol=cfg["tol"])
    for _ in range(args.warmup):
        step(Q, y, Z, Qg, **mixed)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches0 = ctx.launches()
    phases = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0 = ev()
        t0 = time.perf_counter()
        infos = []
        for _ in range(args.steps):
            alpha, fmap, info, finfo, _ = step(Q, y, Z, Qg, phases=phases, **mixed)
            infos.append((info, finfo))
        ev1 = ev()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    launches = ctx.launches() - launches0
    dev_ms = ev0.elapsed_time(ev1)
    ms = job_ms(max(dev_ms, wall * 1e3), world, dev_t)
    ms_per_step = ms / args.steps
    value = job_throughput(args.steps, world, ms)
    info, finfo = infos[-1]
    alpha_m, fmap_m = alpha.clone(), fmap.clone()

    # end to end through the public API with pinned host buffers
    hosts = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (inst.Q, inst.y, Zh, inst.Qg)]
    h2d = sum(h.numel() * 8 for h in hosts)
    out_a = torch.empty(n, dtype=torch.float64).pin_memory()
    out_m = torch.empty(inst.Qg.shape[0], dtype=torch.float64).pin_memory()
    d2h = (out_a.numel() + out_m.numel()) * 8
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 2))
    for _ in range(e2e_steps):
        dQ, dy, dZ, dQg = (h.to(dev_t, non_blocking=True) for h in hosts)
        a, fm, _, _, _ = step(dQ, dy, dZ, dQg, **mixed)
        out_a.copy_(a, non_blocking=True)
        out_m.copy_(fm, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = job_ms((time.perf_counter() - t0) / e2e_steps * 1e3, world, dev_t) / 1e3

    # roofline of the dominant kernel: the matrix-free product.  The method's
    # own work per unique pair (n(n+1)/2 pairs; the operator is symmetric) is
    # the three split-bf16 products hi.hi + hi.lo + lo.hi of 2 d flops each on
    # the tensor pipe and one ex2 on the MUFU pipe; the roof is the larger of
    # the two times.  The kernel's fourth product (lo.lo) and the padding of
    # the tiles are implementation work and are not counted.  The time is that
    # of the whole product as PCG issues it (preparation, tensor-core kernel,
    # finish).
    x = to_dev(synth.random_vector(n, 1))
    ldk = (n + 3) // 4 * 4
    hbm, hbm_kind = peaks()
    if fp64_only:
        # the plain method: the float64 G (8 MiB at n = 1024, L2-resident) is
        # streamed by the float64 product, bound by the float64 FMA rate
        op = L.laker_build_kernel(ctx, Q, inst.scale, inst.lam, L.FP64)
        prod_ms = L.laker_op_time_product(ctx, op, x, reps=50)
        op.close()
        flops = 2.0 * n * n
        achieved = flops / (prod_ms * 1e-3) / 1e12
        roofline = {"kernel": "k_matvec_mat<double> (float64 G, L2-resident)", "bound": "alu",
                    "achieved": achieved, "peak": FP64_NOMINAL_TFLOPS,
                    "peak_kind": "nominal dense float64 rate of GB300 (not in MEASURED_PEAKS.json)",
                    "unit": "TFLOP/s", "frac": achieved / FP64_NOMINAL_TFLOPS, "traffic": None,
                    "flops_per_product": flops, "ms_per_product": prod_ms,
                    "note": "G fits in L2; the product is latency- and float64-bound, not an HBM stream"}
        variant_cmp = None
    else:
        op = L.laker_build_kernel(ctx, Q, inst.scale, inst.lam, L.BF16X3)
        prod_ms = L.laker_op_time_product(ctx, op, x, reps=20)
        main_ms = L.laker_op_time_operator(ctx, op, x, reps=20)
        op.close()
        pairs = n * (n + 1) / 2.0
        flops = pairs * 3 * 2 * inst.d
        bf16_peak, peak_kind = peaks_bf16()
        sfu_peak = SFU_EX2_PER_CLK_PER_SM * 152 * 2.07e9
        t_tensor = flops / (bf16_peak * 1e12)
        t_sfu = pairs / sfu_peak
        achieved = flops / (prod_ms * 1e-3) / 1e12
        roofline = {"kernel": "matrix-free product: k_mf_prep + k_mf_bf16x3 (tcgen05 split-bf16 logits, ex2, row and "
                              "column sums) + k_mf_finish",
                    "bound": "tensor" if t_tensor >= t_sfu else "sfu", "achieved": achieved, "peak": bf16_peak,
                    "peak_kind": peak_kind + " bf16 burst (kernel timed alone)", "unit": "TFLOP/s",
                    "frac": achieved / bf16_peak,
                    "traffic": MF_TRAFFIC_BYTES_C3 if (n == 65536 and inst.d == 64) else None,
                    "method_flops_per_product": flops, "unique_pairs": pairs,
                    "ms_per_product": prod_ms, "ms_main_kernel": main_ms,
                    "tensor_roof_ms": t_tensor * 1e3, "sfu_roof_ms": t_sfu * 1e3,
                    "sfu_peak_ex2_per_s": sfu_peak,
                    "frac_of_binding_roof": max(t_tensor, t_sfu) * 1e3 / prod_ms}
        # the streamed float32 materialised product, for the variant choice per n
        opm = L.laker_build_kernel(ctx, Q, inst.scale, inst.lam, L.FP32, L.MATERIALISED)
        mat_ms = L.laker_op_time_product(ctx, opm, x, reps=10)
        opm.close()
        mat_gbs = (n * ldk * 4 + 3 * n * 8) / (mat_ms * 1e-3) / 1e9
        variant_cmp = {"ms_per_product": mat_ms, "achieved_gbs": mat_gbs, "peak_gbs": hbm, "peak_kind": hbm_kind,
                       "frac": mat_gbs / hbm, "vs_matrix_free": mat_ms / prod_ms}

    # plain float64 path on the same instance (the paper's method in float64)
    plain = None
    accuracy = None
    if args.plain_steps > 0 and not fp64_only:
        torch.cuda.synchronize()
        p0 = time.perf_counter()
        for k in range(args.plain_steps):
            a64, f64, pinfo, pfinfo, op64 = step(Q, y, Z, Qg, precision=L.FP64, refine=0, tol=cfg["tol"],
                                                  keep=(k == args.plain_steps - 1))
        torch.cuda.synchronize()
        pm = (time.perf_counter() - p0) * 1e3 / args.plain_steps
        plain = {"solves_per_s": 1e3 / pm, "ms_per_step": pm, "iterations": pinfo["iterations"],
                 "cccp_iterations": pfinfo["iterations"], "rel_res_true": pinfo["rel_res_true"]}
        # accuracy of the mixed run against the float64 run: alpha, the map in
        # dB over the whole grid, and the mixed alpha's true residual by the
        # float64 operator
        w = L.laker_op_matvec(ctx, op64, alpha_m)
        res_m = float(torch.linalg.norm(y - w) / torch.linalg.norm(y))
        op64.close()
        accuracy = {"alpha_rel_err": float(torch.linalg.norm(alpha_m - a64) / torch.linalg.norm(a64)),
                    "map_db_rmse": float(inst.y_sigma * torch.sqrt(torch.mean((fmap_m - f64) ** 2))),
                    "map_db_max": float(inst.y_sigma * torch.max(torch.abs(fmap_m - f64))),
                    "rel_res_true_fp64_operator": res_m,
                    "reference": "float64 GPU run of the same instance (float64 operator, fit, PCG and map)"}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = oracle_baseline(cfg, ctx, L, to_dev)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if fp64_only else "bf16 split (hi/lo) logits, f32 exp and sums, f64 scalars and residual",
        "data": "synthetic",
        "config": {"workload": cfg["name"] + ", N_r=%d, tol %g true residual" % (n_r, cfg["tol"]),
                   "n": n, "d": inst.d, "lambda": inst.lam, "n_r": n_r, "grid": cfg["grid"] ** 2,
                   "operator": ("materialised float64 G" if fp64_only else
                                "matrix-free tcgen05 split-bf16 logits + ex2, float64-accurate residual every "
                                "%d products from the packed upper-triangular float32 pair" % cfg["refine_every"]),
                   "l2": ("working set fits in L2 (G: %.1f MB float64)" % (n * ldk * 8 / 1e6) if fp64_only else
                          "working set larger than L2 (129 MB): directions %.2f GB, packed float32 pair %.1f GB"
                          % (n * n_r * 8 / 1e9, n * (n + 1) / 2 * 8 / 1e9)),
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "phases_ms_last_step": phases[-1] if phases else None,
        "solve": {"iterations": info["iterations"], "true_residuals": info["true_residuals"],
                  "rel_res_true": info["rel_res_true"], "cccp_iterations": finfo["iterations"],
                  "eig_sweeps": finfo["eig_sweeps"]},
        "plain_fp64": plain,
        "speedup_vs_plain_fp64": (value / plain["solves_per_s"]) if plain else None,
        "accuracy_vs_fp64": accuracy,
        "e2e": {"value": world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": roofline,
        "materialised_fp32_matvec": variant_cmp,
        "ms_per_pcg_product": (phases[-1]["solve"] / max(1, info["iterations"])) if phases else None,
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def run_batched(args):
    """Batching workload: 256 independent instances (n log-uniform in
    [512, 8192], d in {16, 32}, lambda log-uniform in [1e-5, 1e-2], 1-8
    transmitters), float32 operators with float64-accurate residual
    replacement, CCCP preconditioners.  A step is one laker_pcg_solve_batched
    call over all instances to a true relative residual of 1e-6 (operators and
    preconditioners are built and fitted before the timed region; their times
    are reported separately)."""
    import torch

    from paper_2604_25138_gb300 import build
    from paper_2604_25138_gb300 import laker as L

    torch.cuda.set_device(0)
    build.build()
    dev_t = torch.device("cuda", 0)
    specs = synth.batch_specs(synth.CONFIGS["batch256"]["count"], 4000)
    tol = synth.CONFIGS["batch256"]["tol"]
    ctx = L.Context(0)

    def to_dev(x):
        return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device=dev_t)

    insts, ops, precs, ys = [], [], [], []
    torch.cuda.synchronize()
    tb = time.perf_counter()
    build_s = fit_s = 0.0
    for sp in specs:
        inst = synth.make_instance(sp["n"], sp["d"], sp["lam"], n_tx=sp["n_tx"], seed=sp["seed"],
                                   layout=sp["layout"], freq_hz=sp["freq_hz"], grid=2)
        insts.append(inst)
        Q, Z = to_dev(inst.Q), to_dev(synth.directions(inst.n, synth.default_num_directions(inst.n), sp["seed"]))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        op = L.laker_build_kernel(ctx, Q, inst.scale, inst.lam, L.FP32)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        P = L.laker_fit_preconditioner(ctx, op, Z)
        torch.cuda.synchronize()
        build_s += t1 - t0
        fit_s += time.perf_counter() - t1
        ops.append(op)
        precs.append(P)
        ys.append(to_dev(inst.y))
    setup_s = time.perf_counter() - tb
    items = [(op, P, y, None) for op, P, y in zip(ops, precs, ys)]
    for _ in range(args.warmup):
        L.laker_pcg_solve_batched(ctx, items, tol, max_iter=20000, refine_every=20)
    torch.cuda.synchronize()
    launches0 = ctx.launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        ev0.record(ctx.stream)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            alphas, infos, done = L.laker_pcg_solve_batched(ctx, items, tol, max_iter=20000, refine_every=20)
        ev1.record(ctx.stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    launches = ctx.launches() - launches0
    ms = max(ev0.elapsed_time(ev1), wall * 1e3)
    count = len(items)
    value = count * args.steps / (ms / 1e3)
    # end to end: y from pinned host memory, alpha back, inside the timed region
    hy = [torch.from_numpy(np.ascontiguousarray(i.y)).pin_memory() for i in insts]
    ha = [torch.empty(i.n, dtype=torch.float64).pin_memory() for i in insts]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dys = [h.to(dev_t, non_blocking=True) for h in hy]
    a2, _, _ = L.laker_pcg_solve_batched(ctx, [(op, P, y, None) for op, P, y in zip(ops, precs, dys)], tol,
                                         max_iter=20000, refine_every=20)
    for h, a in zip(ha, a2):
        h.copy_(a, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    # the same solves as concurrent single-instance solves on 16 streams
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, cinfos, _ = L.laker_pcg_solve_concurrent(ctx, items, tol, max_iter=20000, refine_every=20, streams=16,
                                                allow_maxiter=True)
    torch.cuda.synchronize()
    conc_s = time.perf_counter() - t0
    # algorithmic HBM bytes of the solve: each product streams the float32 G
    # (n x ldk x 4 bytes); each float64-accurate residual streams the pair
    gbytes = 0.0
    for inst, info in zip(insts, infos):
        ldk = (inst.n + 3) // 4 * 4
        gbytes += inst.n * ldk * 4.0 * info["iterations"] + inst.n * ldk * 8.0 * (info["true_residuals"] + 1)
    step_ms = ms / args.steps
    achieved = gbytes / (step_ms * 1e-3) / 1e9
    hbm, hbm_kind = peaks()
    it = np.array([f["iterations"] for f in infos])
    worst = max(f["rel_res_true"] for f in infos)
    dn = np.array(done)
    line = {
        "metric": "batched PCG solves/s at rel-res 1e-6 (mixed)", "value": value, "unit": "solves/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "batching: 256 instances, n log-uniform in [512, 8192], d in {16, 32}, "
                               "lambda log-uniform in [1e-5, 1e-2], 1-8 Tx, CCCP (N_r default schedule), "
                               "tol 1e-6 true residual, one persistent launch per step",
                   "sum_n": int(sum(i.n for i in insts)), "sum_n2": float(sum(float(i.n) ** 2 for i in insts)),
                   "l2": "working set larger than L2 (float32 pairs, %.1f GB)" %
                         (sum(i.n * ((i.n + 3) // 4 * 4) * 8.0 for i in insts) / 1e9),
                   "setup_s": setup_s, "build_s": build_s, "fit_s": fit_s,
                   "fit_note": "fits are outside the timed step; solves/s including them would be "
                               "%.2f" % (count / (fit_s + build_s + step_ms / 1e3))},
        "per_instance_ms": {"p50": float(np.percentile(dn, 50)), "p99": float(np.percentile(dn, 99)),
                            "max": float(dn.max())},
        "iterations": {"p50": float(np.median(it)), "max": int(it.max()), "sum": int(it.sum())},
        "worst_rel_res_true": worst,
        "concurrent_16_streams": {"solves_per_s": count / conc_s,
                                  "converged": sum(int(f["converged"] == 1) for f in cinfos),
                                  "worst_rel_res_true": max(f["rel_res_true"] for f in cinfos),
                                  "note": "laker_pcg_solve_concurrent on the same instances, one call"},
        "e2e": {"value": count / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": int(sum(i.n for i in insts) * 8),
                "d2h_bytes_per_step": int(sum(i.n for i in insts) * 8)},
        "gpu_launches": launches,
        "roofline": {"kernel": "k_batch_pcg (one persistent launch)", "bound": "hbm", "achieved": achieved,
                     "peak": hbm, "peak_kind": hbm_kind, "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                     "bytes_per_step": gbytes},
        "clocks": clk.summary(),
        "cpu_baseline": None,
    }
    print(json.dumps(line))


def run_learned(args):
    """Learned-preconditioner workload (scaled down for the time budget): the
    set network is trained on the method's own CCCP fits of seeded training
    instances (n uniform in [1024, 4096], d = 32, lambda log-uniform in
    [1e-5, 1e-2], 1-8 Tx), then held-out instances of the same distribution and
    a few at n = 16384 are solved with: the cold CCCP fit, the warm-started fit,
    the prediction used as Sigma_* (with CCCP as the fallback when it needs more
    than 1.2x CCCP's PCG iterations), Jacobi and no preconditioner."""
    import torch

    from paper_2604_25138_gb300 import build
    from paper_2604_25138_gb300 import laker as L
    from paper_2604_25138_gb300 import learned

    torch.cuda.set_device(0)
    build.build()
    ctx = L.Context(0)
    rng = np.random.default_rng(5005)

    def draw(k0, count, n_fixed=None):
        out = []
        for k in range(count):
            n = n_fixed or int(rng.integers(1024, 4097))
            lam = float(10 ** rng.uniform(-5, -2))
            out.append(synth.make_instance(n, 32, lam, n_tx=int(rng.integers(1, 9)), seed=k0 + k, grid=2))
        return out

    n_train, n_test, n_big = args.learned_train, args.learned_test, args.learned_big
    t0 = time.perf_counter()
    train_set = [learned.fit_example(ctx, inst, seed=inst.seed) for inst in draw(50000, n_train)]
    gen_s = time.perf_counter() - t0
    net = L.SetNet(ctx, 32 + 3, 256, 64, seed=5)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = learned.train(ctx, net, train_set, steps=args.learned_steps, batch=16, lr=1e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    rows = []
    for inst in draw(70000, n_test) + draw(80000, n_big, n_fixed=16384):
        r = learned.compare(ctx, net, inst, seed=inst.seed)
        r["n"] = inst.n
        rows.append(r)

    def summary(sel):
        out = {}
        for k in ("cccp", "warm", "learned", "jacobi", "none"):
            it = [r[k]["iterations"] for r in sel]
            fit = [r[k]["fit_s"] for r in sel]
            sol = [r[k]["solve_s"] for r in sel]
            conv = sum(int(r[k]["converged"] == 1) for r in sel)
            out[k] = {"pcg_iterations_mean": float(np.mean(it)), "fit_ms_mean": 1e3 * float(np.mean(fit)),
                      "solve_ms_mean": 1e3 * float(np.mean(sol)), "converged": conv,
                      "solves_per_s": len(sel) / float(np.sum(fit) + np.sum(sol)),
                      "kappa_PA_median": float(np.median([r[k]["kappa_PA"] for r in sel]))}
            if k in ("cccp", "warm"):
                out[k]["cccp_iterations_mean"] = float(np.mean([r[k]["cccp_iterations"] for r in sel]))
        # learned with the fallback: CCCP's time and iterations are charged when it falls back
        fb = [r["fallback"] for r in sel]
        t = [(r["learned"]["fit_s"] + r["learned"]["solve_s"]) + ((r["cccp"]["fit_s"] + r["cccp"]["solve_s"])
                                                                 if r["fallback"] else 0.0) for r in sel]
        out["learned_with_fallback"] = {"fallback_rate": float(np.mean(fb)), "solves_per_s": len(sel) / float(np.sum(t))}
        return out

    small = [r for r in rows if r["n"] < 16384]
    big = [r for r in rows if r["n"] == 16384]
    line = {
        "metric": "end-to-end solves/s with the learned preconditioner (fit or prediction + mixed PCG to 1e-6)",
        "value": summary(small)["learned_with_fallback"]["solves_per_s"], "unit": "solves/s", "n_gpus": 1,
        "steps": len(small), "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 net, f32 operator, f64 scalars", "data": "synthetic",
        "config": {"workload": "learned preconditioner: train on %d CCCP fits (n in [1024, 4096], d = 32, lambda "
                               "log-uniform in [1e-5, 1e-2], 1-8 Tx), test on %d held-out + %d at n = 16384"
                               % (n_train, n_test, n_big),
                   "train_examples_s": gen_s, "train_s": train_s, "train_steps": args.learned_steps,
                   "loss_first": float(np.mean(losses[:20])), "loss_last": float(np.mean(losses[-20:]))},
        "held_out": summary(small),
        "n16384": summary(big) if big else None,
    }
    print(json.dumps(line))


def run_sweep(args):
    """The problem-size sweep of Sec. V-B (Table II, Fig. 2) on the GPU:
    lambda = 1e-2, 10-dimensional embedding, the unscaled kernel exp(<e_i,e_j>),
    n uniform points in a 100 m square, gamma = 0.1, N_r from the default
    schedule, float64 throughout.  Per n: kappa(lambda I + G) and kappa(P A)
    from the Lanczos tridiagonals of the solves' own coefficients, iterations
    to the objective gap TAR.TOL = 1e-3 (Eq. iterations) for CCCP, Jacobi, no
    preconditioner and gradient descent, the final residual at PCG.TOL =
    1e-10, the objective gap and prediction discrepancy against a reference
    solve (CCCP-PCG to 1e-13, standing in for the paper's convex solver), and
    the time of the fit + solve.  The paper's Table II values are quoted for
    context (its hardware and embedding are not stated)."""
    import torch

    from paper_2604_25138_gb300 import build
    from paper_2604_25138_gb300 import laker as L

    torch.cuda.set_device(0)
    build.build()
    ctx = L.Context(0)
    dev_t = torch.device("cuda", 0)

    def to_dev(x):
        return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device=dev_t)

    paper = {50: dict(kappa_A=5.05e3, kappa_PA=1.33e2, its_laker=16, its_jacobi=21, time_s=0.009),
             200: dict(kappa_A=2.02e4, kappa_PA=1.95e2, its_laker=21, its_jacobi=32, time_s=0.043),
             500: dict(kappa_A=5.04e4, kappa_PA=2.07e2, its_laker=25, its_jacobi=42, time_s=0.162),
             1000: dict(kappa_A=1.01e5, kappa_PA=1.79e2, its_laker=28, its_jacobi=47, time_s=0.411),
             2000: dict(kappa_A=2.02e5, kappa_PA=2.09e2, its_laker=30, its_jacobi=59, time_s=1.699)}
    rows = []
    launches0 = ctx.launches()
    t_all = time.perf_counter()
    for n in args.sweep_sizes:
        inst = synth.make_instance(n, 10, 1e-2, n_tx=3, seed=5000 + n, side=100.0, grid=45, scale=1.0)
        y = to_dev(inst.y)
        n_r = synth.default_num_directions(n)
        op = L.laker_build_kernel(ctx, to_dev(inst.Q), inst.scale, inst.lam, L.FP64)
        Pc = L.laker_fit_preconditioner_seeded(ctx, op, 5000 + n, n_r)
        a_ref, _ = L.laker_pcg_solve(ctx, op, Pc, y, 1e-13, max_iter=20000, allow_maxiter=True)
        # R(alpha_ref) by the float64 operator: |G a - y|^2 + lambda a^T G a with G a = A a - lambda a
        w = L.laker_op_matvec(ctx, op, a_ref)
        Ga = w - inst.lam * a_ref
        R_ref = float(torch.sum((Ga - y) ** 2) + inst.lam * torch.dot(a_ref, Ga))
        row = {"n": n, "n_r": n_r}
        for name, P in (("cccp", Pc), ("jacobi", L.laker_precond_jacobi(ctx, op)), ("none", None)):
            alpha, info, trace = L.laker_pcg_solve_trace(ctx, op, P, y, 1e-10, max_iter=20000)
            lo, hi = L.laker_lanczos_extremes(trace)
            row[name] = {"kappa_est": hi / lo, "gap_iterations": L.laker_trace_gap_iterations(trace, R_ref, 1e-3),
                         "iterations_to_1e-10": info["iterations"], "rel_res_true": info["rel_res_true"],
                         "prediction_discrepancy": L.laker_prediction_discrepancy(ctx, op, alpha, a_ref)}
        # time of the whole method (seeded fit + PCG to 1e-10), median of 3
        ts = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            P = L.laker_fit_preconditioner_seeded(ctx, op, 5000 + n, n_r)
            L.laker_pcg_solve(ctx, op, P, y, 1e-10, max_iter=20000)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
            P.close()
        row["cccp"]["time_s"] = statistics.median(ts)
        # gradient descent with the step picked by a small grid search over
        # multiples of 1/L, within an iteration budget
        best = None
        for c in (0.5, 1.0, 1.9):
            mu = L.laker_op_lambda_max(ctx, op, 50)
            eta = c / (2 * mu * (mu + inst.lam))
            a_gd, ginfo, _, gtr = L.laker_gd_solve(ctx, op, y, eta=eta, tol=0.0, max_iter=args.gd_steps,
                                                  trace_cap=args.gd_steps)
            gap = abs(gtr[-1, 1] - R_ref) / abs(R_ref)
            if best is None or gap < best["objective_gap"]:
                hit = np.nonzero(np.abs(gtr[:, 1] - R_ref) <= 1e-3 * abs(R_ref))[0]
                best = {"eta_over_1_by_L": c, "steps": ginfo["iterations"], "objective_gap": gap,
                        "rel_res_true": ginfo["rel_res_true"],
                        "gap_iterations": int(hit[0]) + 1 if hit.size else None,
                        "prediction_discrepancy": L.laker_prediction_discrepancy(ctx, op, a_gd, a_ref)}
        row["gd"] = best
        row["paper_table_ii"] = paper.get(n)
        rows.append(row)
        Pc.close()
        op.close()
    wall = time.perf_counter() - t_all
    line = {"metric": "Table II sweep: kappa, iterations to objective gap 1e-3 and solve time vs n",
            "value": float(np.mean([r["cccp"]["gap_iterations"] for r in rows])), "unit": "iterations (mean, CCCP)",
            "n_gpus": 1, "steps": len(rows), "warmup": 0, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "Sec. V-B sweep: n in %s, lambda=1e-2, d=10, exp(<e_i,e_j>) (scale 1), 100 m "
                                   "square, 3 Tx, gamma=0.1, N_r default schedule, PCG.TOL 1e-10, TAR.TOL 1e-3, "
                                   "GD %d steps" % (list(args.sweep_sizes), args.gd_steps)},
            "rows": rows, "gpu_launches": ctx.launches() - launches0, "wall_s": wall}
    print(json.dumps(line))


def run_variants(args):
    """The per-n choice of the float32-class operator: for n from 512 to
    32768 (d = 32, the field and layout of the n = 16384 instance), an FP32 operator built with
    LAKER_AUTO times one product of the materialised variant (stream of the
    float32 G) and of the matrix-free one (split-bf16 tcgen05 kernel) and keeps
    the faster; the line reports both times, the choice, and the algorithmic
    HBM rate of the materialised product."""
    import torch

    from paper_2604_25138_gb300 import build
    from paper_2604_25138_gb300 import laker as L

    torch.cuda.set_device(0)
    build.build()
    ctx = L.Context(0)
    dev_t = torch.device("cuda", 0)
    rows = []
    for n in args.variant_sizes:
        inst = synth.make_instance(n, 32, 1e-4, n_tx=8, seed=2000 + n, layout="clustered", grid=2)
        Q = torch.as_tensor(np.ascontiguousarray(inst.Q), dtype=torch.float64, device=dev_t)
        op = L.laker_build_kernel(ctx, Q, inst.scale, inst.lam, L.FP32, L.AUTO)
        dsc = L.laker_op_describe(op)
        x = torch.ones(n, dtype=torch.float64, device=dev_t)
        t_kept = L.laker_op_time_product(ctx, op, x, reps=20)
        ldk = (n + 3) // 4 * 4
        rows.append({"n": n, "t_materialised_ms": dsc["t_materialised_ms"], "t_matrix_free_ms": dsc["t_matrix_free_ms"],
                     "chosen": "matrix-free" if dsc["variant"] == L.MATRIX_FREE else "materialised",
                     "t_chosen_ms_20reps": t_kept,
                     "materialised_gbs": (n * ldk * 4 + 3 * n * 8) / (dsc["t_materialised_ms"] * 1e-3) / 1e9})
        op.close()
    print(json.dumps({"metric": "float32-class operator: variant chosen per n (AUTO)", "rows": rows,
                      "peak_hbm_gbs": peaks()[0]}))


def run_combined(args):
    """The target comparison: the mixed, batched, learned-preconditioner form
    against plain float64 PCG on the same GB300, in solves/s at a true
    relative residual of 1e-6.

    A set network is trained once, outside the timed region, on the method's
    own CCCP fits of training instances (n uniform in [1024, 4096], d = 32,
    lambda log-uniform in [1e-5, 1e-2], 1-8 Tx).  A timed step takes
    `--combined-count` held-out instances of the same distribution through:
    * combined: float32 operators, the network's prediction used as Sigma_*
      (no CCCP iteration), the solves of all instances together: concurrent
      single-instance solves on 16 streams (`--combined-solver concurrent`,
      the default, measured faster) or one persistent batched launch
      (`batched`; the line reports the other solver's time too); an instance
      that has not converged after `--combined-cap` products falls back to a
      CCCP fit and a single solve (charged to the step);
    * mixed batched CCCP: the same, with CCCP fits;
    * plain float64: float64 operator, CCCP fit and PCG per instance, one at
      a time (the paper's method as printed)."""
    import torch

    from paper_2604_25138_gb300 import build
    from paper_2604_25138_gb300 import laker as L
    from paper_2604_25138_gb300 import learned

    torch.cuda.set_device(0)
    build.build()
    ctx = L.Context(0)
    rng = np.random.default_rng(6006)

    def draw(k0, count):
        out = []
        for k in range(count):
            n = int(rng.integers(1024, 4097))
            lam = float(10 ** rng.uniform(-5, -2))
            out.append(synth.make_instance(n, 32, lam, n_tx=int(rng.integers(1, 9)), seed=k0 + k, grid=2))
        return out

    t0 = time.perf_counter()
    train_set = [learned.fit_example(ctx, inst, seed=inst.seed) for inst in draw(90000, args.learned_train)]
    net = L.SetNet(ctx, 32 + 3, 256, 64, seed=6)
    losses = learned.train(ctx, net, train_set, steps=args.learned_steps, batch=16, lr=1e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    insts = draw(95000, args.combined_count)
    tol = 1e-6

    def dev(x):
        return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")

    ins = [(dev(i.Q), dev(i.y), dev(synth.directions(i.n, synth.default_num_directions(i.n), i.seed)),
            learned.instance_inputs(ctx, i)) for i in insts]

    phase_ms = {}

    def mark(name, t0):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        phase_ms[name] = 1e3 * (t1 - t0)
        return t1

    def solve_all(items, solver):
        if solver == "concurrent":
            return L.laker_pcg_solve_concurrent(ctx, items, tol, max_iter=args.combined_cap, refine_every=20,
                                                streams=16, allow_maxiter=True)
        return L.laker_pcg_solve_batched(ctx, items, tol, max_iter=args.combined_cap, refine_every=20,
                                         allow_maxiter=True)

    def combined_step(mode, solver=args.combined_solver):
        phase_ms.clear()
        ops, precs = [], []
        t = time.perf_counter()
        for inst, (Q, y, Z, X) in zip(insts, ins):
            ops.append(L.laker_build_kernel(ctx, Q, inst.scale, inst.lam, L.FP32, L.MATERIALISED))
        t = mark("build", t)
        for op, (Q, y, Z, X) in zip(ops, ins):
            if mode == "learned":
                precs.append(L.laker_fit_preconditioner_learned(ctx, op, Z, net, X, mode=1))
            else:
                precs.append(L.laker_fit_preconditioner(ctx, op, Z))
        t = mark("precondition", t)
        items = [(op, P, y, None) for op, P, (_, y, _, _) in zip(ops, precs, ins)]
        alphas, infos, _ = solve_all(items, solver)
        t = mark("solve_" + solver, t)
        fallback = 0
        if mode == "learned":
            for k, f in enumerate(infos):
                if f["converged"] != 1:
                    fallback += 1
                    P = L.laker_fit_preconditioner(ctx, ops[k], ins[k][2])
                    _, f2 = L.laker_pcg_solve(ctx, ops[k], P, ins[k][1], tol, max_iter=40000, refine_every=20)
                    infos[k] = f2
                    P.close()
        worst = max(f["rel_res_true"] for f in infos)
        for P in precs:
            P.close()
        for op in ops:
            op.close()
        mark("fallback_and_release", t)
        return infos, fallback, worst, dict(phase_ms)

    def plain_step():
        worst, its = 0.0, []
        for inst, (Q, y, Z, _) in zip(insts, ins):
            op = L.laker_build_kernel(ctx, Q, inst.scale, inst.lam, L.FP64)
            P = L.laker_fit_preconditioner(ctx, op, Z)
            _, f = L.laker_pcg_solve(ctx, op, P, y, tol, max_iter=40000)
            worst = max(worst, f["rel_res_true"])
            its.append(f["iterations"])
            P.close()
            op.close()
        return its, worst

    def timed(fn, steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            out = fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / steps, out

    for _ in range(max(1, args.warmup)):
        combined_step("learned")
        combined_step("cccp")
    count = len(insts)
    launches0 = ctx.launches()
    with ClockSampler(0) as clk:
        s_l, (inf_l, fb, worst_l, ph_l) = timed(lambda: combined_step("learned"), args.steps)
    launches = ctx.launches() - launches0
    s_c, (inf_c, _, worst_c, ph_c) = timed(lambda: combined_step("cccp"), 1)
    other = "batched" if args.combined_solver == "concurrent" else "concurrent"
    s_o, (_, _, worst_o, ph_o) = timed(lambda: combined_step("learned", other), 1)
    s_p, (its_p, worst_p) = timed(plain_step, 1)
    line = {
        "metric": "solves/s at true rel-res 1e-6: mixed + batched + learned preconditioner vs plain FP64 PCG",
        "value": count / s_l, "unit": "solves/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": s_l * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 operator + f64 scalars/residual, bf16 set network", "data": "synthetic",
        "config": {"workload": "combined form: %d held-out instances, n uniform in [1024, 4096], d = 32, lambda "
                               "log-uniform in [1e-5, 1e-2], 1-8 Tx; network trained on %d CCCP fits (%d Adam steps, "
                               "%.1f s, outside the timed step)" % (count, args.learned_train, args.learned_steps,
                                                                     train_s),
                   "loss_first": float(np.mean(losses[:20])), "loss_last": float(np.mean(losses[-20:]))},
        "combined": {"solves_per_s": count / s_l, "fallbacks": fb, "worst_rel_res_true": worst_l,
                     "pcg_products_mean": float(np.mean([f["iterations"] for f in inf_l])),
                     "phases_ms_last_step": ph_l},
        "mixed_batched_cccp": {"solves_per_s": count / s_c, "worst_rel_res_true": worst_c,
                               "pcg_products_mean": float(np.mean([f["iterations"] for f in inf_c])),
                               "phases_ms": ph_c},
        "plain_fp64": {"solves_per_s": count / s_p, "worst_rel_res_true": worst_p,
                       "pcg_products_mean": float(np.mean(its_p))},
        "speedup_vs_plain_fp64": s_p / s_l,
        "solver": args.combined_solver,
        "other_solver": {"solver": other, "solves_per_s": count / s_o, "worst_rel_res_true": worst_o,
                         "phases_ms": ph_o},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    print(json.dumps(line))


def run_streaming(args):
    """Streaming update (the paper's future work: measurements that arrive
    sequentially).  The 16384-point clustered instance (d = 32, lambda = 1e-4,
    8 Tx) is solved once; then `--stream-steps` batches of `--stream-m` new
    points of the same field arrive.  A timed update is: laker_op_append
    (reusing the stored entries), the CCCP fit warm-started from the previous
    (c, D), and PCG warm-started from the previous alpha (zeros for the new
    points), mixed split-bf16, to a true relative residual of 1e-6.  The
    baseline redoes each update cold: build, fit from Sigma_0 = I, PCG from
    0.  N_r stays at the first instance's value so that the warm fit keeps its
    directions (Z grows by rows)."""
    import torch

    from paper_2604_25138_gb300 import build
    from paper_2604_25138_gb300 import laker as L

    torch.cuda.set_device(0)
    build.build()
    ctx = L.Context(0)
    n0, m, steps = 16384, args.stream_m, args.stream_steps
    n = n0 + m * steps
    inst = synth.make_instance(n, 32, 1e-4, n_tx=8, seed=2000, layout="clustered", grid=2)
    n_r = synth.default_num_directions(n0)
    tol = 1e-6

    def dev(x):
        return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")

    Q, y, Z = dev(inst.Q), dev(inst.y), dev(synth.directions(n, n_r, 2000))

    def first():
        op = L.laker_build_kernel(ctx, Q[:n0].contiguous(), inst.scale, inst.lam, L.BF16X3)
        P = L.laker_fit_preconditioner(ctx, op, Z[:n0].contiguous())
        a, f = L.laker_pcg_solve(ctx, op, P, y[:n0].contiguous(), tol, max_iter=40000, refine_every=20)
        return op, P, a

    def warm_run():
        op, P, a = first()
        rows = []
        for s_ in range(steps):
            k = n0 + (s_ + 1) * m
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            op1 = L.laker_op_append(ctx, op, Q[k - m:k].contiguous())
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            P1 = L.laker_fit_preconditioner_warm(ctx, op1, Z[:k].contiguous(), P)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            a0 = torch.cat([a, torch.zeros(m, dtype=torch.float64, device="cuda")])
            a, f = L.laker_pcg_solve_warm(ctx, op1, P1, y[:k].contiguous(), a0, tol, max_iter=40000,
                                          refine_every=20)
            torch.cuda.synchronize()
            t3 = time.perf_counter()
            rows.append(dict(n=k, append_ms=1e3 * (t1 - t0), fit_ms=1e3 * (t2 - t1), solve_ms=1e3 * (t3 - t2),
                             products=f["iterations"], cccp_iterations=P1.info["iterations"],
                             rel_res_true=f["rel_res_true"], restarts=f["restarts"]))
            P.close()
            op.close()
            op, P = op1, P1
        P.close()
        op.close()
        return rows

    def cold_run():
        rows = []
        for s_ in range(steps):
            k = n0 + (s_ + 1) * m
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            op = L.laker_build_kernel(ctx, Q[:k].contiguous(), inst.scale, inst.lam, L.BF16X3)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            P = L.laker_fit_preconditioner(ctx, op, Z[:k].contiguous())
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            a, f = L.laker_pcg_solve(ctx, op, P, y[:k].contiguous(), tol, max_iter=40000, refine_every=20)
            torch.cuda.synchronize()
            t3 = time.perf_counter()
            rows.append(dict(n=k, build_ms=1e3 * (t1 - t0), fit_ms=1e3 * (t2 - t1), solve_ms=1e3 * (t3 - t2),
                             products=f["iterations"], cccp_iterations=P.info["iterations"],
                             rel_res_true=f["rel_res_true"]))
            P.close()
            op.close()
        return rows

    warm_run()   # warm-up (also compiles nothing: the library is built)
    launches0 = ctx.launches()
    with ClockSampler(0) as clk:
        warm = warm_run()
    launches = ctx.launches() - launches0
    cold = cold_run()

    def tot(rows, keys):
        return sum(sum(r[k] for k in keys) for r in rows)

    warm_ms = tot(warm, ("append_ms", "fit_ms", "solve_ms"))
    cold_ms = tot(cold, ("build_ms", "fit_ms", "solve_ms"))
    line = {
        "metric": "streaming updates/s at true rel-res 1e-6 (append + warm CCCP + warm PCG, mixed)",
        "value": steps / (warm_ms / 1e3), "unit": "updates/s", "n_gpus": 1, "steps": steps, "warmup": 1,
        "ms_per_step": warm_ms / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x3 operator, f64 residual and scalars", "data": "synthetic",
        "config": {"workload": "streaming: n0 = 16384 clustered (d = 32, lambda = 1e-4, 8 Tx), %d batches of %d "
                               "new points, N_r = %d" % (steps, m, n_r)},
        "cold_updates_per_s": steps / (cold_ms / 1e3),
        "speedup_vs_cold": cold_ms / warm_ms,
        "warm": warm, "cold": cold,
        "worst_rel_res_true": max(r["rel_res_true"] for r in warm),
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# The FP64 oracle on the host cores (bounded sample of the same workload)
# ---------------------------------------------------------------------------

def oracle_solve(inst, Z, n_r, tol):
    """One whole solve by the float64 oracle as it stands: kernel matrix,
    random directions, dense shrinkage CCCP, Sigma_*^-1/2 by a dense
    eigendecomposition, PCG to the tolerance and the map on the sample grid.
    Returns the wall-clock seconds and the PCG / CCCP iteration counts."""
    from oracle import laker_oracle as O
    t0 = time.perf_counter()
    r = O.laker(inst.Q, inst.y, inst.lam, inst.scale, Z, tol=tol, Eg=inst.Qg)
    dt = time.perf_counter() - t0
    return dt, r.pcg.iterations, r.cccp.iterations


def oracle_baseline(cfg, ctx=None, L=None, to_dev=None):
    """The oracle timed on the host cores on a bounded sample of the workload:
    one whole solve of an n = CPU_SAMPLE_N instance from the same generator
    (same d, lambda, field and layout, N_r from the default schedule, map on a
    CPU_SAMPLE_GRID^2 grid).  When the GPU library is at hand, the mixed GPU
    path is timed on the same sample instance beside it."""
    inst, Z, n_r = workload(cfg, cfg["seed"] + 77, n=CPU_SAMPLE_N, grid=CPU_SAMPLE_GRID)
    dt, its, cits = oracle_solve(inst, Z, n_r, cfg["tol"])
    out = {"value": 1.0 / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
           "sample": "numpy float64 oracle, one whole solve (kernel, directions, dense CCCP, dense "
                     "Sigma^-1/2, PCG to %g, map on a %dx%d grid) of an n=%d instance of the same generator "
                     "(d=%d, N_r=%d): %.2f s, %d PCG products, %d CCCP iterations; BLAS threads = all cores"
                     % (cfg["tol"], CPU_SAMPLE_GRID, CPU_SAMPLE_GRID, CPU_SAMPLE_N, cfg["d"], n_r, dt, its, cits)}
    if L is not None:
        import torch
        Qd, yd, Zd, Qgd = to_dev(inst.Q), to_dev(inst.y), to_dev(Z), to_dev(inst.Qg)
        times = []
        for k in range(4):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            op = L.laker_build_kernel(ctx, Qd, inst.scale, inst.lam, L.BF16X3)
            P = L.laker_fit_preconditioner(ctx, op, Zd)
            a, _ = L.laker_pcg_solve(ctx, op, P, yd, cfg["tol"], max_iter=40000, refine_every=cfg["refine_every"])
            L.laker_eval_map(ctx, op, Qgd, a)
            torch.cuda.synchronize()
            if k > 0:
                times.append(time.perf_counter() - t0)
            P.close()
            op.close()
        out["gpu_same_sample"] = {"value": 1.0 / statistics.median(times), "unit": UNIT,
                                  "note": "mixed GPU path on the same n=%d sample instance, median of 3" % CPU_SAMPLE_N}
    return out


def run_reference(args):
    """The reference arm: the float64 oracle as it stands, on the host cores;
    each step is one whole oracle solve of the bounded sample instance of the
    workload (see oracle_baseline)."""
    world, rank, _ = rank_env()
    if rank != 0:
        return
    cfg = SINGLE[args.workload if args.workload in SINGLE else "n65536_d64"]
    inst, Z, n_r = workload(cfg, cfg["seed"] + 77, n=CPU_SAMPLE_N, grid=CPU_SAMPLE_GRID)
    for _ in range(args.warmup):
        oracle_solve(inst, Z, n_r, cfg["tol"])
    t0 = time.perf_counter()
    its = []
    for _ in range(args.steps):
        _, it, cit = oracle_solve(inst, Z, n_r, cfg["tol"])
        its.append((it, cit))
    wall = time.perf_counter() - t0
    v = args.steps / wall
    sample = ("numpy float64 oracle, one whole solve per step (kernel, directions, dense CCCP, dense Sigma^-1/2, "
              "PCG to %g, map on a %dx%d grid) of an n=%d instance of the workload's generator (d=%d, N_r=%d); "
              "%d PCG products, %d CCCP iterations; %.1f s for %d steps"
              % (cfg["tol"], CPU_SAMPLE_GRID, CPU_SAMPLE_GRID, CPU_SAMPLE_N, cfg["d"], n_r, its[-1][0], its[-1][1],
                 wall, args.steps))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg["name"] + " (bounded sample: n=%d of the same generator)" % CPU_SAMPLE_N},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--plain-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep-sizes", type=int, nargs="+", default=[50, 200, 500, 1000, 2000, 4000, 8000])
    ap.add_argument("--gd-steps", type=int, default=2000)
    ap.add_argument("--variant-sizes", type=int, nargs="+", default=[512, 1024, 2048, 4096, 8192, 16384, 32768])
    ap.add_argument("--workload", default="n65536_d64", choices=["n65536_d64", "n16384_d32", "n1024_fp64", "batched", "learned", "sweep", "variants", "combined", "streaming"],
                    help="n65536_d64: the precision-form instance (the headline line); n16384_d32: the clustered "
                         "n=16384 instance; n1024_fp64: the small float64 instance; batched: 256 instances; learned: the set-network preconditioner")
    ap.add_argument("--learned-train", type=int, default=256)
    ap.add_argument("--learned-test", type=int, default=32)
    ap.add_argument("--learned-big", type=int, default=4)
    ap.add_argument("--learned-steps", type=int, default=2000)
    ap.add_argument("--combined-count", type=int, default=96)
    ap.add_argument("--combined-cap", type=int, default=4000)
    ap.add_argument("--combined-solver", default="concurrent", choices=["concurrent", "batched"])
    ap.add_argument("--stream-m", type=int, default=512)
    ap.add_argument("--stream-steps", type=int, default=8)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "sweep":
        run_sweep(args)
    elif args.workload == "variants":
        run_variants(args)
    elif args.workload == "combined":
        run_combined(args)
    elif args.workload == "streaming":
        run_streaming(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
