"""Benchmark: retarded-V pair integrals per second on the level-3 icosphere,
T = 4, 32 jittered slabs (122,880 space-time panels).

A step is one pass of the assembly hot path of the energetic single-layer
Galerkin matrix: outer quadrature points, the bit-exact sparsity pattern, the
light-cone-clipped quadrature of every admissible panel pair and the
block-banded assembly (mixed precision: FP64 cone geometry, FP32 arcs).
`value` = admissible pairs (pattern entries) / device time per step, summed
over ranks (weak scaling: rank r assembles its own jittered mesh, seed 1+r).
`e2e` times the public C ABI from host arrays: mesh upload, assembly,
right-hand side, GMRES solve (FP32 inner solves, FP64 refinement, tol 1e-8)
and the density read back to the host.

`--impl reference` times the FP64 CPU oracle (test infrastructure) on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "retarded-V pair integrals/s"
WORKLOADS = {
    "c2": "icosphere L3 (1280 triangles), T=4, 32 slabs, +-20% time jitter: 122,880 panels; m_Q=3",
    "l3x16": "icosphere L3 (1280 triangles), T=4, 16 slabs, +-20% time jitter: 61,440 panels; m_Q=3",
    "l3x8": "icosphere L3 (1280 triangles), T=4, 8 slabs, +-20% time jitter: 30,720 panels; m_Q=3",
    "l2x8": "icosphere L2 (320 triangles), T=2, 8 slabs, +-20% time jitter: 7,680 panels; m_Q=3",
}
WORKLOAD = WORKLOADS["c2"]
L2_BYTES = 129e6


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(mesh_np, seconds=12.0, seed=11):
    """Oracle pair integrals/s on the host cores on a sample of the workload:
    random test panels, their exact pattern rows, random admissible pairs."""
    import oracle
    om = oracle.Mesh.from_spacetime(mesh_np)
    rng = np.random.default_rng(seed)
    rows = rng.choice(mesh_np.n_tet, 24, replace=False).astype(np.int32)
    t0 = time.time()
    cols = om.pattern_rows(rows)
    t_pat = time.time() - t0
    pairs = np.array([(r, c) for r, cs in zip(rows, cols) for c in cs], dtype=np.int32)
    rng.shuffle(pairs)
    nthreads = os.cpu_count() or 1
    # calibrate, then fill the time budget
    n0 = min(len(pairs), 64 * nthreads)
    t0 = time.time()
    om.entries(pairs[:n0], nthreads=nthreads, use_pattern=False)
    dt0 = time.time() - t0
    n1 = int(min(len(pairs), max(n0, n0 * seconds / max(dt0, 1e-3))))
    t0 = time.time()
    om.entries(pairs[:n1], nthreads=nthreads, use_pattern=False)
    dt = time.time() - t0
    return {"value": n1 / dt, "unit": "pairs/s", "cores": nthreads, "kind": "oracle",
            "sample": f"{n1} admissible pairs from the exact pattern rows of 24 random test panels of the "
                      f"same mesh ({dt:.1f} s of quadrature; pattern rows {t_pat:.1f} s not counted)"}


def run_reference(args):
    rank = _env_int("RANK", 0)
    if rank != 0:
        return
    from paper_2103_16841_gb300 import inputs
    m = inputs.workload_c2(seed=1)
    vals = []
    cb = None
    for k in range(max(1, args.steps)):
        cb = cpu_baseline(m, seconds=max(5.0, 60.0 / max(1, args.steps)), seed=11 + k)
        vals.append(cb["value"])
    v = float(np.mean(vals))
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "pairs/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "sample": "bounded sample per step, see cpu_baseline"},
           "cpu_baseline": {"value": v, "unit": "pairs/s", "cores": cb["cores"], "kind": "oracle",
                            "sample": cb["sample"]},
           "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def aggregate(ms, pairs, device):
    """Whole-job numbers of a weak-scaling step: the slowest rank's time and
    the pairs of all ranks (each rank assembles its own mesh; no collective
    touches the data path)."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(ms), float(pairs)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    n = torch.tensor([float(pairs)], dtype=torch.float64, device=device)
    tdist.all_reduce(n)
    return float(t.item()), float(n.item())


def product_only(args):
    """Profiling aid: the tensor-core product of 64 right-hand sides on the
    workload's mixed operator, timed with CUDA events after the shape tuning;
    one more product runs between cudaProfilerStart/Stop (for ncu
    --profile-from-start off). Prints one JSON line."""
    import torch
    import paper_2103_16841_gb300 as stb
    from paper_2103_16841_gb300 import inputs
    m = {"c2": inputs.workload_c2, "l3x16": lambda: inputs.sphere_mesh(3, 16, 4.0, 0.2, seed=1),
         "l3x8": lambda: inputs.sphere_mesh(3, 8, 4.0, 0.2, seed=1),
         "l2x8": lambda: inputs.sphere_mesh(2, 8, 2.0, 0.2, seed=3)}[args.workload]()
    ctx = stb.Context(0)
    op = stb.Operator(ctx, stb.Mesh.from_spacetime(ctx, m), "mixed")
    g = torch.Generator(device="cuda").manual_seed(3)
    x = 0.5 + 0.5 * torch.rand((64, m.n_tet), dtype=torch.float64, device="cuda", generator=g)
    y = torch.empty_like(x)
    dt = args.product_only
    op.matvec(x, y=y, dtype=dt)   # tunes the launch shape
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        op.matvec(x, y=y, dtype=dt)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 5
    torch.cuda.profiler.start()
    op.matvec(x, y=y, dtype=dt)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    st = op.stats()
    print(json.dumps({"workload": WORKLOADS[args.workload], "dtype": dt, "nrhs": 64, "ms_per_product": ms,
                      "stored_values": st["stored"],
                      "note": "bem_matvec_dtype from device arrays in caller order (permutations and packing "
                              "included)"}), flush=True)


def run_ours(args):
    import torch
    import paper_2103_16841_gb300 as stb
    from paper_2103_16841_gb300 import inputs

    rank, world = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)

    def barrier():
        if dist:
            import torch.distributed as tdist
            tdist.barrier()
        torch.cuda.synchronize()

    prec = args.precision
    ctx0 = stb.Context(local if dist else 0)
    alu = ctx0.alu_peaks()      # FP32 / FP64 FMA rates of this GPU, before the timed region
    ctx0.close()
    if args.workload == "c2":
        m = inputs.workload_c2(seed=1 + rank)
    elif args.workload == "l3x16":
        m = inputs.sphere_mesh(3, 16, 4.0, 0.2, seed=1 + rank)
    elif args.workload == "l3x8":
        m = inputs.sphere_mesh(3, 8, 4.0, 0.2, seed=1 + rank)
    else:
        m = inputs.sphere_mesh(2, 8, 2.0, 0.2, seed=3)
    ctx = stb.Context(local if dist else 0)
    ctx.set_tuning(1)           # the quadrature's CTAs per SM timed on the first assembly (not timed below)
    mesh = stb.Mesh.from_spacetime(ctx, m)
    op = stb.Operator(ctx, mesh, prec, store_fp32=True)
    st = op.stats()
    nnz = st["nnz"]
    n_inner = op.inner_integrals()
    stream = torch.cuda.Stream()
    for _ in range(args.warmup):
        op.reassemble(stream)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local if dist else 0) as clk:
        barrier()
        ev0.record(stream)
        phases = []
        for _ in range(args.steps):
            op.reassemble(stream)
            phases.append(op.timings())
        ev1.record(stream)
        ev1.synchronize()
        barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    ms, total_pairs = aggregate(ms, nnz, "cuda")
    value = total_pairs / (ms / 1e3)
    quad_ms = float(np.mean([p["quadrature_ms"] for p in phases]))

    # end to end through the C ABI with host buffers
    b_host = None
    prm = inputs.pulse_params(1, seed=2, fixed_c=1.5)
    e2e_times, solve_info = [], None
    h2d = m.svert.nbytes + m.stv_sv.nbytes + m.stv_t.nbytes + m.tets.nbytes + prm.nbytes
    for k in range(args.e2e_steps):
        barrier()
        t0 = time.perf_counter()
        mesh2 = stb.Mesh.from_spacetime(ctx, m)
        op2 = stb.Operator(ctx, mesh2, prec, store_fp32=True)
        b_host = op2.rhs(stb.DATA_PULSE, prm)[:, 0]
        w, info = op2.solve(b_host, tol=1e-8, restart=50, maxit=400, inner="fp32", max_refine=8,
                            allow_unconverged=True)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
        solve_info = info[0]
        op2.close()
        mesh2.close()
    t_e2e = max(e2e_times) if e2e_times else float("nan")
    t_e2e, _ = aggregate(t_e2e, 0, "cuda")
    d2h = m.n_tet * 8 + m.n_tet * 8  # rhs vector and density back to the host

    acc = accuracy_leg(ctx, mesh, op, m, args) if (args.accuracy and rank == 0) else None
    multi = (multi_rhs_leg(op, m, args, ref=acc.pop("_W64") if acc else None)
             if (args.multi_rhs > 0 and rank == 0) else None)
    serving = serving_leg(ctx, args) if (args.serve_requests > 0 and rank == 0) else None
    batched = batch_leg(ctx, args) if (args.batch > 0 and rank == 0) else None

    if rank != 0:
        if dist:
            import torch.distributed as tdist
            tdist.destroy_process_group()
        return

    pk = peaks()
    prof = load_profile_summary()
    roof = None
    inner_per_s = n_inner / (quad_ms / 1e3)
    if prof and "fp32_flops_per_inner" in prof:
        # executed flops per inner integral of the quadrature kernel, from an ncu
        # capture of the same kernel on a mesh whose values exceed L2 (level-3
        # sphere, 8 slabs), times this run's inner integrals, over the kernel's
        # CUDA-event time; peaks measured on this GPU in this run
        f32 = prof["fp32_flops_per_inner"] * n_inner / (quad_ms / 1e3) / 1e12
        f64 = prof["fp64_flops_per_inner"] * n_inner / (quad_ms / 1e3) / 1e12
        traffic = prof["dram_bytes_per_inner"] * n_inner if prof.get("dram_bytes_per_inner") else None
        roof = {"bound": "alu", "achieved": round(f32, 3), "peak": round(alu["fp32_tflops"], 2), "unit": "TFLOP/s",
                "frac": round(f32 / alu["fp32_tflops"], 4), "traffic": traffic,
                "kernel": "k_quad_blocks<mixed>",
                "fp64": {"achieved": round(f64, 4), "peak": round(alu["fp64_tflops"], 3), "unit": "TFLOP/s",
                         "frac": round(f64 / alu["fp64_tflops"], 4)},
                "inner_integrals_per_launch": n_inner,
                "note": "achieved = executed FP32 (FP64) flops per inner integral from ncu (SASS op counters, "
                        "FFMA counted 2) on the level-3 sphere with 8 slabs x inner integrals of this launch / "
                        "its CUDA-event time; peak = FMA rate measured on this GPU in this run (bem_alu_peaks; "
                        "152 SMs x 128 lanes x 2 x 2.07 GHz = 80.5 TFLOP/s nominal)"}
    cb = cpu_baseline(m, seconds=args.cpu_seconds) if args.cpu_seconds > 0 else None
    vbytes = st["stored"] * (4 if prec == "mixed" else 12)  # FP32 values; FP64 operators also keep FP64
    out = {
        "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if prec == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "precision": prec, "pairs_per_rank": nnz,
                   "inner_integrals_per_rank": n_inner,
                   "stored_values": st["stored"], "parallelism": f"independent meshes per rank (x{world})",
                   "quadrature_launch": op.tuning(),
                   "l2": f"each step writes the {vbytes / 1e9:.2f} GB value array: "
                         + ("larger than L2" if vbytes > L2_BYTES else "smaller than L2 (profiling case)")},
        "phases_ms": {k: round(float(np.mean([p[k] for p in phases])), 2) for k in phases[0]},
        "e2e": None if not e2e_times else {"value": total_pairs / t_e2e, "unit": "pairs/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "seconds_per_step": t_e2e,
                "includes": "mesh upload, assembly, RHS, GMRES(FP32 inner + FP64 refinement, tol 1e-8), "
                            "density to host",
                "solve": solve_info},
        "gpu_launches": 3 * args.steps,
        "clocks": clk.summary(),
        "roofline": roof,
        "cpu_baseline": cb,
        "accuracy": acc,
        "multi_rhs": multi,
        "serving": serving,
        "batch": batched,
        "inner_integrals_per_s": inner_per_s,
        "peaks": {"hbm_gbs": pk.get("hbm_gbs"), "bf16_tflops": pk.get("bf16_tflops"),
                  "fp32_tflops_measured": alu["fp32_tflops"], "fp64_tflops_measured": alu["fp64_tflops"]},
    }
    print(json.dumps(out), flush=True)
    if dist:
        import torch.distributed as tdist
        tdist.destroy_process_group()


def accuracy_leg(ctx, mesh, op, m, args):
    """The reduced-precision form against the FP64 operator on the same mesh
    (the GPU FP64 path, itself checked against the oracle to 1e-11 in the
    tests): the FP64 operator is assembled, the single-RHS solution of the
    benchmark's data is compared with its FP64 GMRES solution, and the 64-RHS
    reference (pulses with centres in [1, 2]) is the refinement whose
    residual uses the FP64 operator (bem_solve_refined), which converges to
    the FP64 operator's solution."""
    import torch
    import paper_2103_16841_gb300 as stb
    from paper_2103_16841_gb300 import inputs
    t0 = time.perf_counter()
    op64 = stb.Operator(ctx, mesh, "fp64", store_fp32=False)
    torch.cuda.synchronize()
    out = {"fp64_operator_s": round(time.perf_counter() - t0, 2),
           "fp64_quadrature_ms": round(op64.timings()["quadrature_ms"], 1)}
    b = op.rhs(stb.DATA_PULSE, inputs.pulse_params(1, seed=2, fixed_c=1.5))[:, 0]
    w64, i64 = op64.solve(b, tol=1e-12, restart=100, maxit=4000, inner="fp64", allow_unconverged=True)
    wm, im = op.solve(b, tol=1e-8, restart=50, maxit=400, inner="fp32", max_refine=8, allow_unconverged=True)
    t1 = time.perf_counter()
    wr, ir = op.solve_refined(op64, b, tol=1e-10, restart=50, maxit=600, inner="fp32", max_refine=20,
                              allow_unconverged=True)
    t_ref = time.perf_counter() - t1
    rel = lambda w: float(np.linalg.norm(w - w64) / np.linalg.norm(w64))
    out["single_rhs"] = {"fp64_gmres_iterations": i64[0]["iterations"],
                         "mixed_fp32_inner_tol_1e-8": {"rel_error_vs_fp64_operator": rel(wm),
                                                       "rel_residual": im[0]["rel_residual"]},
                         "mixed_with_fp64_residual_tol_1e-10": {"rel_error_vs_fp64_operator": rel(wr),
                                                                "seconds": round(t_ref, 2),
                                                                "refinements": ir[0]["refinements"]}}
    W64 = None
    if args.multi_rhs > 0:
        prm = inputs.pulse_params(args.multi_rhs, seed=2)
        B = op.rhs(stb.DATA_PULSE, prm)
        t1 = time.perf_counter()
        W64, info = op.solve_refined(op64, B, tol=1e-11, restart=50, maxit=800, inner="tf32", max_refine=30,
                                     allow_unconverged=True)
        out["multi_rhs_reference"] = {"how": "TF32 inner solves on the mixed operator, FP64 residual of the FP64 "
                                             "operator, tol 1e-11", "seconds": round(time.perf_counter() - t1, 2),
                                      "converged": int(sum(i["converged"] for i in info)),
                                      "rel_residual_max": float(max(i["rel_residual"] for i in info))}
    op64.close()
    out["_W64"] = W64
    return out


def multi_rhs_leg(op, m, args, ref=None):
    """Many right-hand sides on the assembled operator: the block matvec in
    FP32 (CUDA cores), TF32 and BF16 (tensor cores) with the values read once
    per product, and GMRES with TF32 / BF16 inner solves plus FP64
    refinement to 1e-8; errors per RHS against the FP64 operator's solution
    (from the accuracy leg) when given, else against the TF32-inner solution
    of the same operator refined to 1e-12."""
    import torch
    import paper_2103_16841_gb300 as stb
    from paper_2103_16841_gb300 import inputs
    nrhs = args.multi_rhs
    st = op.stats()
    n = m.n_tet
    prm = inputs.pulse_params(nrhs, seed=2)
    b = op.rhs(stb.DATA_PULSE, prm)
    x = torch.tensor(np.ascontiguousarray(b.T), device="cuda")
    out = {"nrhs": nrhs, "pulses": "exp(-((t - x.d - c)/0.25)^2), d seeded unit vectors, c ~ U[1, 2]",
           "products": {}, "solves": {}}
    stream = torch.cuda.Stream()
    hbm = peaks().get("hbm_gbs")
    # one vector, FP32 values (the inner-solve product): HBM-bound
    x1 = x[:1].contiguous()
    y1 = op.matvec(x1, dtype="fp32", stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(10):
        e0.record(stream)
        op.matvec(x1, y1, dtype="fp32", stream=stream)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms1 = float(np.median(ts))
    gbs1 = st["stored"] * 4 / (ms1 / 1e3) / 1e9
    out["products"]["fp32_x1"] = {"ms": round(ms1, 3), "value_GBps": round(gbs1, 1),
                                  "frac_of_measured_hbm": round(gbs1 / hbm, 3) if hbm else None,
                                  "note": "4 B per stored value over the call (conversions and permutations "
                                          "included), against the measured HBM copy bandwidth"}
    for dt in ["fp32", "tf32", "bf16"]:
        y = op.matvec(x, dtype=dt, stream=stream)          # first call: workspace, autotune
        reps = 5
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ts = []
        for _ in range(reps):
            e0.record(stream)
            op.matvec(x, y, dtype=dt, stream=stream)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = float(np.median(ts))
        vbytes = st["stored"] * (2 if dt == "bf16" else 4)
        out["products"][dt] = {"ms": round(ms, 3), "value_bytes": vbytes,
                               "value_GBps": round(vbytes / (ms / 1e3) / 1e9, 1),
                               "frac_of_measured_hbm": round(vbytes / (ms / 1e3) / 1e9 / hbm, 3) if hbm else None,
                               "passes_over_values": math.ceil(nrhs / 4) if dt == "fp32" else math.ceil(nrhs / 64),
                               "note": "includes the FP64 <-> packed-operand conversions and the caller-order "
                                       "permutations of bem_matvec_dtype"}
    runs = [("tf32", "tf32", 1e-8), ("bf16", "bf16", 1e-8)]
    key_err = "rel_error_vs_fp64_operator_per_rhs"
    if ref is None:
        runs = [("reference_tf32_1e-12", "tf32", 1e-12)] + runs
        key_err = "rel_error_vs_same_operator_refined_per_rhs"
    for key, inner, tol in runs:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        w, info = op.solve(b, tol=tol, restart=50, maxit=600, inner=inner, max_refine=30, allow_unconverged=True)
        dt_s = time.perf_counter() - t0
        rec = {"seconds": round(dt_s, 3), "tol": tol, "converged": int(sum(i["converged"] for i in info)),
               "iterations_max": int(max(i["iterations"] for i in info)),
               "refinements": int(info[0]["refinements"]),
               "rel_residual_max": float(max(i["rel_residual"] for i in info))}
        if ref is None:
            ref = w
        else:
            err = np.linalg.norm(w - ref, axis=0) / np.linalg.norm(ref, axis=0)
            rec[key_err] = [float("%.3e" % e) for e in err]
            rec["rel_error_max"] = float(err.max())
        out["solves"][key] = rec
    return out


def batch_leg(ctx, args):
    """Batched small scatterers: seeded ellipsoids (icosphere level 1 or 2
    scaled by semi-axes in [0.5, 1.5], 8-16 slabs, T = 4, +-20% jitter, 1-4
    pulse RHS each) assembled by one persistent launch per pass over all
    operators and solved as one block-diagonal GMRES (CUDA graphs; FP32 inner
    solves, FP64 refinement, tol 1e-8)."""
    import torch
    import paper_2103_16841_gb300 as stb
    from paper_2103_16841_gb300 import inputs
    probs = inputs.scatterer_meshes(args.batch, seed=3)
    meshes = [stb.Mesh.from_spacetime(ctx, m) for m, _ in probs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch = stb.Batch(ctx, meshes, precision="mixed")
    t1 = time.perf_counter()
    ws, infos = batch.solve([p for _, p in probs], tol=1e-8, restart=50, maxit=2000, inner="fp32", max_refine=10,
                            allow_unconverged=True)
    t2 = time.perf_counter()
    st = batch.stats()
    batch.close()
    flat = [i for inf in infos for i in inf]
    return {"scatterers": len(probs), "panels": st["n_tet"], "pairs": st["nnz"],
            "rhs": len(flat), "assemble_ms": round(st["assemble_ms"], 1),
            "pairs_per_s": st["nnz"] / (st["assemble_ms"] / 1e3),
            "create_s": round(t1 - t0, 3), "solve_s": round(t2 - t1, 3),
            "converged": int(sum(i["converged"] for i in flat)),
            "iterations_max": int(max(i["iterations"] for i in flat)),
            "rel_residual_max": float(max(i["rel_residual"] for i in flat)),
            "scatterers_per_s": len(probs) / (t2 - t0)}


def serving_leg(ctx, args):
    """Poisson stream of Dirichlet solves through the continuous-batching
    server: the mixed-precision form (FP32 quadrature, FP32 inner GMRES, FP64
    refinement) against the plain FP64 path (FP64 quadrature and GMRES), on
    the same trace and server settings, both keeping assembled operators
    resident (a later request on the same mesh skips the assembly). Requests
    are drawn uniformly from icosphere levels x slab counts x right-hand-side
    counts (T = 4, +-20% jitter, one seeded mesh per (level, slabs) shape,
    pulse data with per-request seeds); latency = submission to completion.
    Each request's mixed-precision density is compared with its FP64 one:
    the mixed path solves to 1e-8 (FP32 inner GMRES, FP64 refinement), the
    FP64 path to 1e-10, so that its densities are a reference for the mixed
    path's error (the FP64 path's time is almost all assembly, so the tighter
    tolerance costs it little). Requests on a mesh that another request is
    assembling or using wait for that operator (the server's coalescing)."""
    import paper_2103_16841_gb300 as stb
    from paper_2103_16841_gb300 import inputs
    rng = np.random.default_rng(4)
    levels = [1, 2, 3] if args.serve_full else [1, 2]
    slabs = [8, 16, 32] if args.serve_full else [8, 16]
    nrhs_set = [1, 4, 16]
    n = args.serve_requests
    arrivals = np.cumsum(rng.exponential(1.0 / args.serve_rate, n))
    shapes = {}
    reqs = []
    for k in range(n):
        lv, sl, nr = int(rng.choice(levels)), int(rng.choice(slabs)), int(rng.choice(nrhs_set))
        if (lv, sl) not in shapes:
            shapes[(lv, sl)] = inputs.sphere_mesh(lv, sl, 4.0, 0.2, seed=1000 + 10 * lv + sl)
        reqs.append((shapes[(lv, sl)], inputs.pulse_params(nr, seed=2000 + k), f"{k}:L{lv}x{sl}x{nr}"))
    out = {"requests": n, "poisson_rate_per_s": args.serve_rate, "slots": args.serve_slots,
           "mix": {"levels": levels, "slabs": slabs, "nrhs": nrhs_set}, "mesh_shapes_in_trace": len(shapes),
           "resident_operators": True, "paths": {}}
    dens = {}
    for name, prec, inner, tol in [("mixed", "mixed", "fp32", 1e-8), ("fp64", "fp64", "fp64", 1e-10)]:
        srv = stb.Server(ctx, max_slots=args.serve_slots, precision=prec, inner=inner, tol=tol, restart=50,
                         maxit=5000, max_refine=12, cache_operators=True)
        t0 = time.perf_counter()
        tickets = []
        for (m, prm, _), ta in zip(reqs, arrivals):
            dt = t0 + ta - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets.append(srv.submit(m, params=prm))
        res = srv.wait(tickets, timeout_s=3600)
        t_end = time.perf_counter()
        st = srv.stats()
        srv.close()
        lat = np.array([res[t]["latency_ms"] for t in tickets])
        ok = sum(res[t]["status"] == 0 for t in tickets)
        dens[name] = [res[t]["w"] for t in tickets]
        out["paths"][name] = {
            "precision": prec, "inner": inner, "tol": tol, "completed": int(ok),
            "solves_per_s": round(float(st["solves_per_s"]), 3),
            "p50_ms": round(float(np.percentile(lat, 50)), 1), "p99_ms": round(float(np.percentile(lat, 99)), 1),
            "mean_ms": round(float(lat.mean()), 1), "wall_s": round(t_end - t0, 2),
            "peak_running": int(st["peak_running"]), "cache_hits": int(st["cache_hits"]),
            "rel_residual_max": float(max(res[t]["rel_residual"] for t in tickets))}
    errs = []
    for wm, w64 in zip(dens["mixed"], dens["fp64"]):
        if wm is not None and w64 is not None:
            errs.append(float((np.linalg.norm(wm - w64, axis=1) / np.linalg.norm(w64, axis=1)).max()))
    out["mixed_vs_fp64_rel_error_per_request"] = {lab: float("%.3e" % e) for (_, _, lab), e in zip(reqs, errs)}
    out["mixed_vs_fp64_rel_error_per_request_max"] = max(errs) if errs else None
    out["mixed_vs_fp64_rel_error_per_request_median"] = float(np.median(errs)) if errs else None
    mx, fp = out["paths"]["mixed"], out["paths"]["fp64"]
    out["speedup_solves_per_s"] = round(mx["solves_per_s"] / max(fp["solves_per_s"], 1e-12), 2)
    return out


def load_profile_summary():
    """Per-pair FP32 work and DRAM traffic of the quadrature kernel from the
    committed ncu summary (profiles/quad_kernel_mixed.json)."""
    p = os.path.join(ROOT, "profiles", "quad_kernel_mixed.json")
    try:
        return json.load(open(p))
    except Exception:
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--e2e-steps", dest="e2e_steps", type=int, default=1)
    ap.add_argument("--cpu-seconds", dest="cpu_seconds", type=float, default=12.0)
    ap.add_argument("--accuracy", type=int, default=1,
                    help="1: assemble the FP64 operator of the same mesh and report the mixed form's errors "
                         "against its solutions (0: skip)")
    ap.add_argument("--multi-rhs", dest="multi_rhs", type=int, default=64,
                    help="right-hand sides of the multi-RHS leg (0: skip)")
    ap.add_argument("--batch", type=int, default=512,
                    help="small scatterers of the batch leg (0: skip; 512, the default, is the full batch)")
    ap.add_argument("--serve-requests", dest="serve_requests", type=int, default=12,
                    help="requests of the serving leg (0: skip)")
    ap.add_argument("--serve-rate", dest="serve_rate", type=float, default=200.0,
                    help="Poisson arrivals per second (200: the offered load exceeds capacity, so solves/s is the "
                         "server's capacity)")
    ap.add_argument("--serve-slots", dest="serve_slots", type=int, default=4)
    ap.add_argument("--serve-small", dest="serve_full", action="store_false",
                    help="draw from levels 1-2 and 8/16 slabs only (default: the full mix, levels 1-3 x 8/16/32 "
                         "slabs x 1/4/16 RHS)")
    ap.add_argument("--product-only", dest="product_only", default=None, choices=["tf32", "bf16", "fp32"],
                    help="profiling aid: time the 64-RHS product of the workload's operator in this arithmetic "
                         "and run one more under cudaProfilerStart/Stop, then exit")
    ap.add_argument("--workload", default="c2", choices=["c2", "l3x16", "l3x8", "l2x8"],
                    help="l3x16 / l3x8 / l2x8: the level-3 sphere with 16 or 8 slabs (T = 4) / the level-2 sphere "
                         "with 8 slabs (T = 2), jittered, for profiler captures only")
    args = ap.parse_args()
    if args.product_only:
        product_only(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
