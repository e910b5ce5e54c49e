"""Probe solves/s of the eddy-current FE solver on the 4M-DOF tube + support-plate workload.

Workload (config 2 of the benchmark table): 53 x 53 x 356-node jittered Kuhn
tetrahedral mesh (1,000,004 nodes, 4,000,016 complex unknowns, 5,759,520 tets)
of a 30 x 30 x 200 mm box around a tube (sigma 1e6) through a quatrefoil
support plate (sigma 1.4e6, the defect configuration) at 100 kHz; the probe's
coil pair sits at the plate edge.  One probe position = 4 solves (2 coils x
{vacuum, defect}) + Delta Z.  Inputs are synthetic and seeded (ect_inputs).

A step is one batch of probe positions through the whole hot path: coil
sources, batched solves of both systems, Delta Z.  Assembly and the
preconditioner set-up are done once before timing (the matrix does not
depend on the probe position) and reported separately.

  value       solves/s with the sources already in HBM (ect_solve on device
              buffers + the Delta Z reduction), mixed FP32/FP64 + batched
  e2e         the same metric through ect_impedance with host buffers (host
              positions in, host Delta Z out, copies inside the timed region)
  fp64_plain  solves/s of the plain FP64 flexible GMRES, one position
  roofline    the dominant kernel (FP32 SpMM inside the mixed solve), timed
              with CUDA events on the library stream

--impl reference times the CPU oracle (the reference for this workload) on a
bounded sample of the same workload on the host cores.
Multi-GPU: positions are sharded across ranks (no collective on the data
path); value = all ranks' solves / max-over-ranks time.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return PEAKS_FALLBACK, "fallback"


def profiled_traffic(kernel, nnzb):
    """DRAM bytes per launch of `kernel` from profiles/traffic.json, scaled to nnzb blocks.

    The record holds dram__bytes_read.sum + dram__bytes_write.sum of one captured launch on a
    mid-size case and that case's nnzb; traffic grows with the matrix (blocks and the vectors of
    the same rows), so it is scaled by the ratio of block counts.  None when the kernel has no
    capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    return rec["bytes"] * nnzb / rec["nnzb"]


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # raw samples beside the process (summarised into the JSON line); ECT_CLOCKS_DIR overrides
        self.path = os.path.join(os.environ.get("ECT_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"ect_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x, device):
    """Max of a host scalar over all ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput: the units all ranks processed over the max-over-ranks time."""
    return units_per_rank * world / seconds


def probe_positions(n, rank=0, world=1):
    """Positions around the plate edge (z = 10 mm), 0.5 mm apart, sharded by rank."""
    z = 10.0e-3 + 0.5e-3 * (np.arange(n * world) - (n * world) // 2)
    return z[rank * n:(rank + 1) * n]


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------

def run_gpu(args):
    import torch
    import torch.distributed as dist

    import ect_inputs as E
    from paper_1602_03207_gb300 import build as B
    from paper_1602_03207_gb300 import ect

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    B.build()
    ect.load_library()

    t0 = time.time()
    p = E.make_config(args.config)
    m = p.mesh
    gen_s = time.time() - t0
    ctx = ect.Context()
    ctx.load_problem(p)
    n = 4 * m.n_nodes
    mask = ect.ECT_F64 | ect.ECT_F32
    st = torch.cuda.current_stream()

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    if args.block_split:
        ctx.set_block_split(args.block_split)
    asm_ms = [timed(lambda w=w: ctx.assemble(w, mask)) for w in (0, 1)]
    pc_ms = [timed(lambda w=w: ctx.precond_setup(w, mask)) for w in (0, 1)]
    _, nnzb = ctx.matrix_info()

    P = args.positions
    zs = probe_positions(P, rank, world)
    cur = [c.current for c in p.coils]
    base = ect.default_options(tol=args.tol, mode=ect.ECT_MODE_MIXED, restart=args.outer_restart,
                               inner_iters=args.inner_iters, max_iters=args.max_outer, use_graph=1,
                               reorth=args.reorth, spmm_rows=args.spmm_rows)
    plain = ect.default_options(tol=args.tol, mode=ect.ECT_MODE_F64, restart=args.restart, use_graph=1,
                                max_iters=args.max_iters)
    # device-resident sources: [P][2][n] (position-major, coil minor)
    Bsrc = torch.empty(P, 2, n, dtype=torch.complex128, device="cuda")
    for c in range(2):
        tmp = torch.empty(P, n, dtype=torch.complex128, device="cuda")
        ctx.coil_rhs(p.coils[c], zs, tmp)
        Bsrc[:, c] = tmp
    del tmp
    U0 = torch.empty_like(Bsrc)
    Ud = torch.empty_like(Bsrc)
    k = 2 * P
    tune = None
    mixed = base
    if not args.no_autotune:
        # tune on each of the step's two systems, then keep the winner whose vacuum + defect
        # solves take least time (one option set serves both, as in ect_impedance)
        t_at = time.time()
        cands = [ctx.autotune(w, Bsrc, U0, k, base)[0] for w in (0, 1)]
        best_ms = None
        for o in cands:
            ms_pair = ctx.solve(0, Bsrc, U0, k, o)["ms"] + ctx.solve(1, Bsrc, Ud, k, o)["ms"]
            if best_ms is None or ms_pair < best_ms:
                mixed, best_ms = o, ms_pair
        tune = {"rhs_tile": mixed.rhs_tile, "spmm_rows": mixed.spmm_rows, "block_split": ctx.block_split(),
                "restart": mixed.restart,
                "inner_iters": mixed.inner_iters,
                "reorth": mixed.reorth, "seconds": time.time() - t_at, "pair_ms": best_ms,
                "tuned_on": "vacuum and defect systems; the faster option set on both"}

    stats = {}

    def step_device(opts, tag):
        s0 = ctx.solve(0, Bsrc, U0, k, opts)
        s1 = ctx.solve(1, Bsrc, Ud, k, opts)
        for q in range(P):
            ctx.delta_z(U0[q], Ud[q], None, cur)
        stats[tag] = (s0, s1)
        return s0["launches"] + s1["launches"] + P

    for _ in range(args.warmup):
        step_device(mixed, "mixed")
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    e0.record(st)
    for _ in range(args.steps):
        launches += step_device(mixed, "mixed")
    e1.record(st)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(ms, "cuda")
    value = job_rate(4 * P * args.steps, world, ms / 1000.0)

    # e2e: the public host-buffer call (host positions in, host Delta Z out)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    dz_e2e = None
    for _ in range(args.steps):
        dz_e2e, _ = ctx.impedance(p.coils, zs, mixed)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t1, "cuda")
    e2e = job_rate(4 * P * args.steps, world, e2e_s)

    # plain FP64 flexible GMRES, one position (4 solves), the same preconditioner in FP64
    plain_ms = None
    dz_plain = None
    if not args.skip_plain:
        z1 = zs[:1]
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        dz_plain, sp = ctx.impedance(p.coils, z1, plain)
        torch.cuda.synchronize()
        plain_ms = (time.perf_counter() - t2) * 1000.0
        stats["plain"] = sp
    dz_err = None
    if dz_plain is not None and dz_e2e is not None:
        dz_err = float(np.abs(dz_e2e[0] - dz_plain[0]).max() / np.abs(dz_plain[0]).max())

    # kernels, timed with CUDA events on the library's stream
    ctx_stream = torch.cuda.ExternalStream(ctx.stream.cuda_stream)

    def ktime(fn, reps=20):
        fn()
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(ctx_stream)
        for _ in range(reps):
            fn()
        a1.record(ctx_stream)
        torch.cuda.synchronize()
        return a0.elapsed_time(a1) / reps

    kk = min(k, 8)
    ctx.set_spmm_rows(mixed.spmm_rows)
    staged = mixed.spmm_rows != -1
    xs = torch.randn(kk, n, dtype=torch.complex64, device="cuda")
    ys = torch.empty_like(xs)
    spmv_ms = ktime(lambda: ctx.spmv(0, xs, ys, kk, precision=ect.ECT_F32))
    mg_ms = ktime(lambda: ctx.precond_apply(0, xs, ys, kk, precision=ect.ECT_F32), reps=5)
    Vb = torch.randn(10, n, dtype=torch.complex64, device="cuda")
    wv = torch.randn(n, dtype=torch.complex64, device="cuda")
    cgs_ms = ktime(lambda: ctx.cgs2(Vb, wv, precision=ect.ECT_F32), reps=5)
    del xs, ys, Vb, wv
    nrows = m.n_nodes
    # matrix values and one column index per block (16-bit local index when staged, 32-bit
    # otherwise), row pointers, x and y once per right-hand side (the staged kernel's tile lists,
    # ~1 % of these bytes, are not counted)
    spmv_bytes = nnzb * (16 * 8 + (2 if staged else 4)) + 4 * (nrows + 1) + 2 * kk * n * 8
    kname = "k_spmm_pipe" if staged else "k_spmv_f32<8>"
    achieved = spmv_bytes / (spmv_ms / 1000.0) / 1e9
    peaks, src = load_peaks()
    hbm = float(peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))
    s_mixed = stats["mixed"]

    rec = {
        "metric": "probe solves/s at 4M complex DOF, FP64 plain vs mixed+batched, dZ err<=1e-6",
        "value": value,
        "unit": "solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "c64/c128 (mixed FP32 inner, FP64 outer)",
        "data": "synthetic (seeded jittered Kuhn mesh, ect_inputs)",
        "config": {"workload": f"{args.config}: {m.n_nodes} nodes / {n} complex dof / {m.n_tets} tets, "
                               f"{P} probe positions per rank per step (= {4 * P} solves), tol {args.tol}",
                   "positions_per_step": P * world, "rhs_per_solve_call": k, "nnzb": nnzb,
                   "inner_iters": mixed.inner_iters, "outer_restart": mixed.restart,
                   "reorth": mixed.reorth, "rhs_tile": mixed.rhs_tile, "spmm_rows": mixed.spmm_rows,
                   "block_split": ctx.block_split(),
                   "l2": "inputs larger than L2 (matrices 3.8 GB FP64 / 1.9 GB FP32 each)",
                   "parallelism": f"positions sharded over {world} GPU(s)"},
        "clocks": clocks,
        "e2e": {"value": e2e, "unit": "solves/s", "h2d_bytes_per_step": 8 * P + 2 * 40,
                "d2h_bytes_per_step": 64 * P},
        "autotune": tune,
        "fp64_plain": {"value": (4.0 / (plain_ms / 1000.0)) if plain_ms else None, "unit": "solves/s",
                       "ms_per_position": plain_ms,
                       "stats": stats.get("plain")},
        "dz_rel_err_mixed_vs_fp64": dz_err,
        "solver_stats": {"mixed_vacuum": s_mixed[0], "mixed_defect": s_mixed[1],
                         "preconditioner": "aggregation multigrid on the subdomain blocks (W-cycle)"},
        "kernels_ms": {"spmv_f32_k%d" % kk: spmv_ms, "multigrid_cycle_f32_k%d" % kk: mg_ms,
                       "cgs2_f32_j10_k1": cgs_ms},
        "setup_ms": {"mesh_gen_s": gen_s * 1000, "assemble": asm_ms, "precond": pc_ms},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": profiled_traffic(kname, nnzb) if kk == 8 else None,
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch on a "
                                       "mid-size case, scaled by nnzb (profiles/traffic.json)",
                     "kernel": f"{kname} (SpMM, {kk} rhs, spmm_rows {mixed.spmm_rows})", "ms_per_launch": spmv_ms,
                     "algorithmic_bytes": spmv_bytes, "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)"},
        "gpu_launches": int(launches),
    }
    if rank == 0 and not args.no_cpu_baseline:
        rec["cpu_baseline"] = cpu_baseline(args, stats)
    if rank == 0:
        print(json.dumps(rec))
    if world > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ----------------------------------------------------------------------------

def oracle_setup(args):
    """The oracle's FP64 system of a slab of the workload and its multigrid hierarchy.

    The slab keeps the full 53 x 53 cross-section and 40 node layers of the
    z-range around the plate edge (same h, materials, jitter recipe)."""
    import ect_inputs as E
    from oracle import fem, rhs, solve

    shape, lengths, jitter = E.CONFIGS[args.config]
    nz = 40
    Lz = lengths[2] * (nz - 1) / (shape[2] - 1)
    p = E.tsp_problem((shape[0], shape[1], nz), (lengths[0], lengths[1], Lz), jitter=jitter, z_pos=(0.0,))
    t0 = time.time()
    M = fem.system_matrix(p, "defect")
    asm_s = time.time() - t0
    t = fem.scaling(M)
    S = fem.scaled(M, t)
    s1, _ = fem.effective_coefficients(p.sigma, p.nu, p.sigma_d, p.nu_d, "defect")
    cond = fem.conducting_nodes(p.mesh.n_nodes, p.mesh.tets, s1)
    d, v = fem.fixed_dofs(p.mesh.bc_mask, cond)
    levels = solve.amg_setup(S, solve.near_null_weights(t, np.concatenate([d, v])), p.mesh.block_of_node,
                             solve.node_graph_from_tets(p.mesh.n_nodes, p.mesh.tets))
    setup_s = time.time() - t0
    b = fem.constrain_rhs(rhs.coil_rhs(p.mesh.xyz, p.mesh.tets, p.coils[0].as_tuple(), 0.0), p, "defect")
    return {"S": S, "levels": levels, "rhs": t * b, "n_small": 4 * p.mesh.n_nodes,
            "n_full": 4 * shape[0] * shape[1] * shape[2], "shape": (shape[0], shape[1], nz),
            "assembly_s": asm_s, "setup_s": setup_s}


def oracle_iterate(o, budget_s):
    """FGMRES(30) iterations of the oracle for about budget_s seconds; (iterations, seconds)."""
    from oracle import solve
    it = 0
    x = None
    t1 = time.time()
    while time.time() - t1 < budget_s:
        x, info = solve.fgmres(o["S"], o["rhs"], lambda r: solve.amg_apply(o["levels"], r), tol=1e-30,
                               restart=30, maxiter=10, x0=x)
        it += info["iters"]
    return it, time.time() - t1


def oracle_rate(o, it, el, ips):
    """Full-size solves/s extrapolated from a sample: seconds per iteration per unknown, scaled
    to the workload's unknowns and to ips iterations per solve."""
    return 1.0 / (el / it / o["n_small"] * o["n_full"] * ips)


def _superlu_child(shape, lengths, q):
    import ect_inputs as E
    from oracle import fem, rhs, solve
    p = E.tsp_problem(shape, lengths, z_pos=(0.0,))
    t0 = time.time()
    M = fem.system_matrix(p, "defect")
    t1 = time.time()
    b = fem.constrain_rhs(rhs.coil_rhs(p.mesh.xyz, p.mesh.tets, p.coils[0].as_tuple(), 0.0), p, "defect")
    _, lu = solve.superlu_solve(M, b)
    t2 = time.time()
    for _ in range(4):
        lu.solve(b)
    t3 = time.time()
    q.put({"unknowns": 4 * p.mesh.n_nodes, "assembly_s": t1 - t0, "factor_s": t2 - t1, "solve_s": (t3 - t2) / 4})


def superlu_leg(limit_s):
    """SciPy SuperLU (the paper's solver family) on the oracle's matrix: a config-1-size mesh
    measured, and the next size up attempted within limit_s seconds (child process, started
    with spawn)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = []
    for shape, lengths, lim in (((16, 16, 32), (30e-3, 30e-3, 60e-3), 10 * limit_s),
                                ((20, 20, 40), (30e-3, 30e-3, 60e-3), limit_s)):
        q = ctx.Queue()
        pr = ctx.Process(target=_superlu_child, args=(shape, lengths, q))
        t0 = time.time()
        pr.start()
        pr.join(lim)
        if pr.is_alive():
            pr.terminate()
            pr.join()
            out.append({"mesh": "x".join(map(str, shape)), "unknowns": 4 * shape[0] * shape[1] * shape[2],
                        "completed": False, "note": f"did not complete in {lim:.0f} s"})
        else:
            r = q.get() if not q.empty() else {}
            out.append(dict(r, mesh="x".join(map(str, shape)), completed=bool(r),
                            wall_s=time.time() - t0,
                            solves_per_s=(1.0 / r["solve_s"]) if r.get("solve_s") else None))
    return out


def cpu_baseline(args, stats):
    ips = None
    if stats.get("plain"):
        ips = stats["plain"].get("iters") or None
    ips = ips or args.ref_iters
    o = oracle_setup(args)
    it, el = oracle_iterate(o, args.cpu_budget)
    rec = {"value": oracle_rate(o, it, el, ips), "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": (f"oracle FP64 FGMRES(30) with its aggregation-multigrid W-cycle on a "
                      f"{'x'.join(map(str, o['shape']))}-node slab of the workload ({o['n_small']} unknowns): "
                      f"{it} iterations in {el:.1f} s, scaled to {o['n_full']} unknowns and {ips} iterations per "
                      f"solve ({'the GPU FP64 run' if stats.get('plain') else 'the FP64 count at this size'}); "
                      f"slab assembly {o['assembly_s']:.1f} s, assembly + hierarchy {o['setup_s']:.1f} s"),
           "oracle_assembly": {"unknowns": o["n_small"], "seconds": o["assembly_s"]}}
    if args.superlu_limit > 0:
        rec["superlu"] = superlu_leg(args.superlu_limit)
    return rec


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, on the host cores.  Each step is one
    timed sample of FGMRES iterations on the slab (ms_per_step is that measured time); the
    value is the full-size rate extrapolated from the samples."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    t0 = time.time()
    o = oracle_setup(args)
    samples = []
    for _ in range(args.warmup + args.steps):
        samples.append(oracle_iterate(o, args.ref_budget))
    v = samples[-args.steps:]
    rates = [oracle_rate(o, it, el, args.ref_iters) for it, el in v]
    value = statistics.median(rates)
    ms = 1000.0 * sum(el for _, el in v) / len(v)
    sample = (f"per step: {statistics.median([it for it, _ in v])} oracle FGMRES(30) iterations (multigrid W-cycle) "
              f"on a {'x'.join(map(str, o['shape']))}-node slab of the workload ({o['n_small']} unknowns), "
              f"{ms / 1000:.1f} s; value extrapolated to {o['n_full']} unknowns and {args.ref_iters} iterations "
              f"per solve (the FP64 count at this size on a GB300, bench line fp64_plain); setup {o['setup_s']:.1f} s")
    rec = {"impl": "reference", "metric": "probe solves/s at 4M complex DOF, FP64 plain vs mixed+batched, "
           "dZ err<=1e-6", "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "ms_per_step_basis": "measured wall time of one oracle sample",
           "value_basis": "extrapolated from the timed samples",
           "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "c128", "data": "synthetic (seeded, ect_inputs)",
           "config": {"workload": f"{args.config} (oracle sample)"},
           "cpu_baseline": {"value": value, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "wall_s": time.time() - t0}
    print(json.dumps(rec))


def kernel_probe(args):
    """A few launches of the hot kernels on a mid-size case, for profiler captures.

    53 x 53 x 120-node TSP mesh (1,348,320 complex dof): FP32 SpMM and the
    preconditioner (block-Jacobi, or the multigrid cycle with --probe-mg) on 8
    right-hand sides, 3 times each, then CGS2 against 10 vectors twice."""
    import torch

    import ect_inputs as E
    from paper_1602_03207_gb300 import build as B
    from paper_1602_03207_gb300 import ect

    B.build()
    p = E.tsp_problem((53, 53, 120), (30e-3, 30e-3, 67.4e-3), (2, 2, 4), 0.15, 0, z_pos=(10e-3,))
    ctx = ect.Context()
    ctx.load_problem(p)
    ctx.assemble(0, ect.ECT_F64 | ect.ECT_F32)
    ctx.precond_setup(0, ect.ECT_F64 | ect.ECT_F32, -1 if args.probe_mg else 0)
    ctx.set_spmm_rows(args.spmm_rows)
    n = 4 * p.mesh.n_nodes
    k = 8
    x = torch.randn(k, n, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    for _ in range(3):
        ctx.spmv(0, x, y, k, precision=ect.ECT_F32)
        ctx.precond_apply(0, y, x, k, precision=ect.ECT_F32)
    V = torch.randn(10, n, dtype=torch.complex64, device="cuda")
    w = torch.randn(n, dtype=torch.complex64, device="cuda")
    for _ in range(2):
        ctx.cgs2(V, w, precision=ect.ECT_F32)
    torch.cuda.synchronize()
    print(json.dumps({"kernel_probe": "ok", "dof": n, "nnzb": int(ctx.matrix_info()[1]),
                      "preconditioner": "multigrid" if args.probe_mg else "block-Jacobi"}))


def dz_record(args):
    """Delta Z of the mixed solve (to args.tol) against the plain FP64 solve (to 1e-10) at one
    probe position of args.config, both through ect_impedance: the error record config 4 asks
    for (mixed precision to 1e-8 at 16M unknowns)."""
    import torch

    import ect_inputs as E
    from paper_1602_03207_gb300 import build as B
    from paper_1602_03207_gb300 import ect

    B.build()
    p = E.make_config(args.config)
    ctx = ect.Context()
    ctx.load_problem(p)
    for w in (0, 1):
        ctx.assemble(w, ect.ECT_F64 | ect.ECT_F32)
        ctx.precond_setup(w, ect.ECT_F64 | ect.ECT_F32, -1)
    mixed = ect.default_options(tol=args.tol, mode=ect.ECT_MODE_MIXED, restart=args.outer_restart,
                                inner_iters=args.inner_iters, max_iters=args.max_outer, reorth=args.reorth,
                                spmm_rows=args.spmm_rows)
    plain = ect.default_options(tol=1e-10, mode=ect.ECT_MODE_F64, restart=args.restart, max_iters=args.max_iters)
    t0 = time.time()
    dz_m, st_m = ctx.impedance(p.coils, p.z_pos, mixed)
    t1 = time.time()
    dz_p, st_p = ctx.impedance(p.coils, p.z_pos, plain)
    t2 = time.time()
    torch.cuda.synchronize()
    err = float(np.abs(dz_m - dz_p).max() / np.abs(dz_p).max())
    print(json.dumps({"dz_record": args.config, "n_nodes": p.mesh.n_nodes, "unknowns": 4 * p.mesh.n_nodes,
                      "mixed_tol": args.tol, "fp64_tol": 1e-10, "dz_rel_err_mixed_vs_fp64": err,
                      "dz_fp64": [[[float(z.real), float(z.imag)] for z in row] for row in dz_p[0]],
                      "mixed": {"s": t1 - t0, "iters": st_m["iters"], "relres": st_m["relres_max"]},
                      "fp64": {"s": t2 - t1, "iters": st_p["iters"], "relres": st_p["relres_max"]}}))


def mlp_probe(args):
    """Surrogate MLP on the tensor cores: forward and one Adam step at batch 65536 (the largest the
    library takes), timed with CUDA events; FLOPs count the real layer sizes (6->256, 4x 256->256)."""
    import torch

    from paper_1602_03207_gb300 import build as B
    from paper_1602_03207_gb300 import ect

    B.build()
    bt = 65536
    net = ect.Surrogate(batch=bt)
    rng = np.random.default_rng(0)
    sizes = ect.MLP_SIZES
    layers = [(rng.normal(scale=1.0 / np.sqrt(fi), size=(fo, fi)), np.zeros(fo)) for fi, fo in zip(sizes[:-1], sizes[1:])]
    net.set_params(ect.mlp_flatten(layers))
    x = torch.randn(bt, sizes[0], device="cuda")
    y = torch.empty(bt, sizes[-1], device="cuda")
    t = torch.randn(bt, sizes[-1], device="cuda") * 0.1
    fwd_flop = 2.0 * bt * sum(fi * fo for fi, fo in zip(sizes[:-1], sizes[1:]))

    def timed(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    f_ms = timed(lambda: net.forward(x, y), 20)
    s_ms = timed(lambda: net.train_step(x, t, 1e-4), 10)
    peaks, src = load_peaks()
    pk = float(peaks.get("bf16_tflops", PEAKS_FALLBACK["bf16_tflops"]))
    hbm = float(peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))
    # algorithmic bytes of the inference forward: per layer the bf16 input once (the first layer's
    # padded to 16 columns), the bf16 activations written once (the output layer: fp32), the bf16
    # weights once; x read and y copied out at the ends
    fwd_bytes = bt * sizes[0] * 4 + 2 * bt * sizes[-1] * 4
    for l, (fi, fo) in enumerate(zip(sizes[:-1], sizes[1:])):
        fwd_bytes += bt * (16 if l == 0 else fi) * 2 + bt * fo * (4 if l == len(sizes) - 2 else 2) + fo * fi * 2
    rec = {"mlp_probe": "ok", "batch": bt, "forward_ms": f_ms, "forward_tflops": fwd_flop / f_ms / 1e9,
           "forward_bytes": fwd_bytes, "forward_gbs": fwd_bytes / f_ms / 1e6,
           "forward_hbm_frac": fwd_bytes / f_ms / 1e6 / hbm,
           "train_step_ms": s_ms, "train_step_tflops": 3 * fwd_flop / s_ms / 1e9,
           "bf16_peak_tflops": pk, "peak_source": src,
           "forward_frac": fwd_flop / f_ms / 1e9 / pk, "train_step_frac": 3 * fwd_flop / s_ms / 1e9 / pk}
    print(json.dumps(rec))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="c2")
    ap.add_argument("--positions", type=int, default=4)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--max-iters", type=int, default=6000)
    ap.add_argument("--outer-restart", type=int, default=10)
    ap.add_argument("--max-outer", type=int, default=400)
    ap.add_argument("--inner-iters", type=int, default=20)
    ap.add_argument("--reorth", type=int, default=1, help="Gram-Schmidt variant when not autotuned (0-3)")
    ap.add_argument("--block-split", type=int, default=0,
                    help="smoothing blocks per subdomain when not autotuned (0: the library's default, 1)")
    ap.add_argument("--spmm-rows", type=int, default=0,
                    help="FP32 SpMM row tiling when not autotuned (0 auto, -1 unstaged)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--kernel-probe", action="store_true", help="only launch the hot kernels on a mid-size case")
    ap.add_argument("--dz-record", action="store_true",
                    help="only compare Delta Z of the mixed solve (--tol) with the FP64 solve on --config")
    ap.add_argument("--probe-mg", action="store_true")
    ap.add_argument("--mlp-probe", action="store_true", help="only time the surrogate MLP on the tensor cores")
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--superlu-limit", type=float, default=60.0,
                    help="seconds allowed for the SuperLU attempt at 64,000 unknowns (0: skip the SuperLU leg)")
    ap.add_argument("--ref-budget", type=float, default=10.0)
    ap.add_argument("--ref-iters", type=int, default=504,
                    help="FP64 FGMRES(30) iterations per solve at this size (the GPU's FP64 leg with the "
                         "autotuned preconditioner), used to extrapolate the reference arm's samples")
    args = ap.parse_args()
    if args.kernel_probe:
        kernel_probe(args)
        return
    if args.dz_record:
        dz_record(args)
        return
    if args.mlp_probe:
        mlp_probe(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
