"""Benchmark: solved DoF/s of one multigrid-preconditioned CG solve on GB300.

Workload (one "step" = one nnmg_pcg_solve of all right-hand sides to a 1e-8
relative residual): 3D Poisson on the unit cube, Q2, four independently
jittered non-nested hex levels (6^3, 13^3, 27^3, 55^3 cells, +-0.15h, seeds
1-4), f = 1 plus seven N(0,1) right-hand sides (seeds 1001-1007), Chebyshev
degree 3 around Jacobi, FP64 direct coarse solve, V-cycle in FP32 inside FP64
CG.  Inputs (mesh hierarchy and right-hand sides) are resident in HBM when the
timed region starts; the working set (~1 GB of vectors and metric terms) is
far larger than the 129 MB L2, so no flush is needed between steps.

Also reported: the same solve with the V-cycle in FP64 (plain FP64 GPU
multigrid), V-cycle and operator GDoF/s, p50/p99 solve latency, the roofline
of the dominant kernel, the end-to-end number through the host-buffer C call,
and the FP64 CPU oracle timed on a bounded sample of the same workload.

Multi-GPU: replicas only (one independent solve per rank, weak scaling).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solved DoF/s at 1e-8 rel. residual, FP32-MG vs FP64-MG; V-cycle GDoF/s; p50/p99"
UNIT = "DoF/s"
CONFIG = "c2_3d_q2"
WORKLOAD = ("3D Poisson unit cube, Q2, 4 non-nested jittered hex levels 6^3/13^3/27^3/55^3 "
            "(+-0.15h, seeds 1-4), f=1 + 7 N(0,1) RHS, Chebyshev(3)-Jacobi, FP64 direct coarse, "
            "FP32 V-cycle in FP64 PCG, rtol 1e-8")
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 CUDA-core peak of GB300: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz;
# the FP64 pipe takes one FMA, MUL or ADD per slot: 152 x 2 x 2.07e9 op/s.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP64_PIPE_TOPS = 152 * 2 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# DRAM bytes per (cell, right-hand side) of the FP64 fine-level operator, from
# ncu's dram__bytes_read.sum + dram__bytes_write.sum of one launch on config 2
# (412.5 + 66.8 MB over 166,375 cells x 8 RHS, padded metric rows), keyed by
# the kernel choice the counters were taken on (-1: op_reg_kernel<3,2,double>).
# The launch's traffic is this times its cells x RHS; another choice reports
# null.
OP64_TRAFFIC_PER_UNIT = {-1: (412489472 + 66762496) / (166375 * 8)}


def op64_traffic(choice, n_cells, nrhs):
    per = OP64_TRAFFIC_PER_UNIT.get(choice)
    return None if per is None else per * n_cells * nrhs


def poisson3d_work(n):
    """(flops, FP64 pipe ops) per cell and right-hand side of the 3D Poisson
    operator with n = k + 1 points per direction, as the sweeps run them:
    12 line sweeps (3 interpolations, 3 derivatives, their transposes; two of
    the transposed derivatives accumulate) and 9 multiply-adds of the metric
    per quadrature point.  For odd n the sweeps skip S's unit middle row and
    Dg's zero middle diagonal entry (exact for symmetric point sets)."""
    odd = n % 2
    rows = n - odd                                   # S rows that are not the unit row
    s_flops, s_ops = rows * (2 * n - 1), rows * n    # S and S^T lines (same count)
    d_flops = n * (2 * n - 1) - 2 * odd               # Dg or Dg^T line
    d_ops = n * n - odd
    da_flops, da_ops = 2 * n * n - 2 * odd, n * n - odd   # Dg^T accumulating into a line
    lines = n * n
    flops = lines * (6 * s_flops + 4 * d_flops + 2 * da_flops) + 15 * n ** 3
    ops = lines * (6 * s_ops + 4 * d_ops + 2 * da_ops) + 9 * n ** 3
    return flops, ops


def fine_level_kernel_bytes(dim, k, kc, ncomp, nrhs, s, cheb, fine, coarse):
    """Algorithmic DRAM bytes of the fine level's V-cycle kernels, per launch
    (operator, restriction, prolongation) or per V-cycle (vector kernels).

    fine / coarse: (n_nodes, n_free, n_cells) of the two levels; k, kc their
    degrees; s the value size.  Vectors are [rows][ncomp * nrhs].
    operator: read x and write y at free rows, plus per cell the metric terms
      (6 (3D) / 3 (2D) Poisson, 9 elasticity, s bytes each) and the node
      indices (4 B) of its (k+1)^d quadrature points / nodes.
    vector kernels of one V-cycle: Chebyshev start (read f, write d, x) and
      2m-1 Chebyshev steps (read f, t, d, x; write d, x, t), plus the Jacobi
      diagonal per row in each of the 2m (the residual is formed inside the
      restriction).
    restriction: at the located points read f and t = A x with their node
      index (4 B) and reference point (d s B) and reset t to zero (the fused
      residual r = f - t), write the coarse vector, and the cell-local buffer
      of the deterministic two-phase gather (written, read back) with its
      gather list (4 B per cell-local entry).
    prolongation: read the coarse vector once and the coarse cells' node
      indices, read and write the fine vector at the located points with
      their node index and reference point."""
    nn_f, nf_f, nc_f = fine
    nn_c, nf_c, nc_c = coarse
    ch = ncomp * nrhs
    nloc, nloc_c = (k + 1) ** dim, (kc + 1) ** dim
    nmetric = 9 if ncomp == 3 else (6 if dim == 3 else 3)
    rows_f = nn_f * ncomp
    op = 2 * nf_f * ch * s + nc_f * nloc * (nmetric * s + 4)
    vec = rows_f * nrhs * s * (3 + (2 * cheb - 1) * 7) + 2 * cheb * rows_f * s
    n_pts = nf_f
    pts = n_pts * (4 + dim * s)
    buf = nc_c * nloc_c * ch * s
    restrict = 3 * n_pts * ch * s + pts + nn_c * ch * s + 2 * buf + nc_c * nloc_c * 4
    prolong = nn_c * ch * s + nc_c * nloc_c * 4 + 2 * n_pts * ch * s + pts
    return {"operator": op, "vector": vec, "restrictor": restrict, "prolongator": prolong}


def vcycle_kernel_table(H, degrees, ncomp, nrhs, cheb, hbm_gbs, reps=5):
    """Per-level V-cycle breakdown (paper Sec. 5 components) in FP32 and the
    achieved HBM bandwidth of the fine level's kernels, from the library's
    event-timed profile run (nnmg_vcycle_profile)."""
    import numpy as np
    import torch
    from paper_2412_10910_gb300 import _abi
    top = H.n_levels - 1
    r = torch.randn(H.rows(top), nrhs, dtype=torch.float32, device="cuda")
    r[torch.tensor(np.repeat(H.constrained(top), ncomp), device="cuda")] = 0
    z = torch.empty_like(r)
    H.vcycle_profile(r, z)                        # warm-up
    acc, cnt = None, None
    for _ in range(reps):
        ms, cnt = H.vcycle_profile(r, z)
        acc = ms if acc is None else acc + ms
    ms = acc / reps
    cols = _abi.PROF_COLUMNS
    breakdown = {f"level{lv}": {c: round(float(ms[lv, i]), 4) for i, c in enumerate(cols[:6])
                                if cnt[lv, i] > 0}
                 for lv in range(H.n_levels)}
    dim = H.dim
    fine, coarse = H.info(top), H.info(top - 1)
    by = fine_level_kernel_bytes(dim, degrees[top], degrees[top - 1], ncomp, nrhs, 4, cheb,
                                 fine, coarse)
    col = {c: i for i, c in enumerate(cols)}
    kern = {}
    for name, per_launch in (("operator", True), ("vector", False), ("restrictor", True),
                             ("prolongator", True)):
        n = int(cnt[top, col[name]]) if per_launch else 1
        t_ms = float(ms[top, col[name]]) / max(n, 1)
        gbs = by[name] / (t_ms / 1e3) / 1e9
        kern[name] = {"ms_per_launch" if per_launch else "ms_per_vcycle": round(t_ms, 5),
                      "algorithmic_bytes": int(by[name]), "achieved_gbs": round(gbs, 1),
                      "frac_of_measured_hbm": round(gbs / hbm_gbs, 3)}
    return breakdown, kern


def operator_kernel_name(choice, k, dtype):
    if choice == -1:
        return f"op_reg_kernel<3,{k},{dtype}> (register-resident)"
    if choice == -2:
        return f"op_reg2_kernel<3,{k}> (paired FP32 register-resident)"
    if choice > 0:
        return f"op3d_kernel<{k},{dtype},1> ({choice} units per block)"
    if choice <= -100:
        return f"op3d_kernel<{k},f2,1> (paired FP32, {-100 - choice} (cell, pair) units per block)"
    return f"default rule for <3,{k},{dtype}>"


def _peaks():
    try:
        with open(PEAKS) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def _rhs(n_rows, free_mask_rows, H, top, nrhs):
    import numpy as np
    import torch
    from synthetic import normal_rhs
    b = torch.zeros(n_rows, nrhs, dtype=torch.float64, device="cuda")
    H.load_vector(top, np.ones(1), b, col=0)              # f = 1
    if nrhs > 1:
        r = normal_rhs(n_rows, [1000 + j for j in range(1, nrhs)])
        r[~free_mask_rows] = 0.0
        b[:, 1:] = torch.tensor(r, device="cuda")
    return b


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self):
        self.p = None
        self.path = None

    def start(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        dev = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={dev}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.p is None:
            return out
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [t.strip() for t in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                   "reasons": sorted(reasons), "samples": len(sm)}
        return out


def replica_aggregate(local_ms, local_units, world, reduce_max, reduce_sum):
    """Whole-job numbers of `world` independent replicas: the slowest rank's
    time and the units all ranks processed (weak scaling, no data exchange).
    reduce_max / reduce_sum combine one float across ranks."""
    ms = reduce_max(local_ms) if world > 1 else local_ms
    units = reduce_sum(local_units) if world > 1 else local_units
    return ms, units, units / (ms / 1e3)


def kernels_per_solve(n_levels, cheb, iters):
    """Kernel launches of one PCG solve run as the device-side graph loop:
    init 2 and the loop's arming kernel, per iteration the V-cycle (per level
    above the coarsest: 1 + 2(m-1) pre, 1 residual operator pass, 2 restriction
    (the first forms the residual), 1 prolongation, 2m post; the coarse solve
    and its fixed-order segment sum),
    8 CG kernels (two dots, beta, p, operator, alpha, update with the FP32 copy
    of r, check) and the loop's re-arming kernel."""
    per_level = 1 + 2 * (cheb - 1) + 1 + 2 + 1 + 2 * cheb
    return 3 + iters * ((n_levels - 1) * per_level + 2 + 8 + 1)


def cpu_baseline_sample(nrhs_sample=8, steps=1, warmup=0):
    """Time the FP64 oracle (as it stands) on a bounded sample of the workload in
    a subprocess: the three coarsest levels of the same family (finest 27^3 Q2
    cells), f = 1 in every column, FP32 V-cycle inside FP64 CG.  The oracle
    hierarchy is built once (untimed); the right-hand sides are solved in
    parallel, one column per worker process (forked after the build, each
    single-threaded), on min(nrhs, host cores) cores; each step is one solve of
    all columns.  The full four-level hierarchy is not sampled: the oracle's
    brute-force point location of its 1.3M fine points over 19,683 coarse cells
    alone takes about 15 minutes."""
    code = r"""
import json, os, sys, time, numpy as np, multiprocessing as mp
sys.path.insert(0, %r)
from synthetic import config_levels
from oracle.hierarchy import OracleHierarchy
lv = config_levels("c2_3d_q2", n_levels=3)
H = OracleHierarchy(lv, 2, cheb_degree=3)
top = len(H.levels) - 1
b = H.load_vector(top, lambda x: np.ones((len(x), 1)))
nrhs = %d

def solve(j):
    x, its, rel, tr = H.pcg(b[:, None], "fp32", rtol=1e-8)
    return int(its[0])

if __name__ == "__main__":
    cores = max(1, min(nrhs, os.cpu_count() or 1))
    with mp.get_context("fork").Pool(cores) as pool:
        pool.map(solve, range(cores))               # workers up and warm
        for _ in range(%d):
            pool.map(solve, range(nrhs))
        ts, its = [], []
        for _ in range(%d):
            t = time.perf_counter()
            its = pool.map(solve, range(nrhs))
            ts.append(time.perf_counter() - t)
    print(json.dumps({"seconds": ts, "free": int(H.levels[top].free_dofs.size), "nrhs": nrhs,
                      "cores": cores, "iters": its}))
""" % (ROOT, nrhs_sample, warmup, steps)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("oracle baseline failed: " + r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    sec = statistics.mean(d["seconds"])
    v = d["free"] * d["nrhs"] / sec
    return {"value": v, "unit": UNIT, "cores": d["cores"], "kind": "oracle",
            "seconds_per_step": sec,
            "sample": (f"FP64 numpy/scipy oracle, same family with the 3 coarsest levels (finest "
                       f"27^3 Q2 cells, {d['free']} free DoFs; the full 4-level hierarchy is not "
                       f"sampled because the oracle's brute-force point location of its 1.3M fine "
                       f"points takes ~15 min), {d['nrhs']} RHS f=1 solved one column per "
                       f"single-threaded worker on {d['cores']} host cores, FP32 V-cycle in FP64 "
                       f"PCG to 1e-8, {d['iters'][0]} iterations, {sec:.2f} s per solve")}


def run_reference(args, rank, world):
    """Reference arm: the oracle timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    cb = cpu_baseline_sample(8, steps=args.steps, warmup=args.warmup)
    v = cb["value"]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * cb["seconds_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD + " (oracle: bounded sample)"},
            "cpu_baseline": {"kind": "oracle", "cores": cb["cores"], "sample": cb["sample"],
                             "value": v, "unit": UNIT},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_configs(args, rank):
    """Every configuration: setup time, then p50/p99 of timed solves (after
    warm-up) in the three modes, the per-level V-cycle breakdown and the fine
    level's kernels against HBM, one JSON line per configuration."""
    import numpy as np
    import torch
    from paper_2412_10910_gb300 import _abi, nnmg
    from synthetic import config_levels, normal_rhs
    from synthetic.meshes import CONFIGS

    cases = [("c1_2d_q1", None, None), ("c2_3d_q2", None, None),
             ("c3_3d_q4_deformed", None, None),
             ("c3_3d_q4_deformed", "pmg", None),        # polynomial-multigrid coarse solver
             ("c4_3d_q2_elasticity", None, None),
             ("c4_3d_q2_elasticity", None, [(8, 2, 2), (19, 5, 5), (41, 11, 11), (85, 23, 23)])]
    for name, variant, cells in cases:
        cfg = CONFIGS[name]
        levels = config_levels(name, cells=cells)
        degs = None
        if variant == "pmg":
            k = cfg["degree"]
            levels = [levels[0]] * (k - 1) + levels
            degs = list(range(1, k)) + [k] * (len(levels) - k + 1)
        torch.cuda.synchronize()
        t = time.perf_counter()
        H = nnmg.Hierarchy(levels, cfg["degree"], cfg["ncomp"], cfg.get("lame", (1.0, 1.0)),
                           cfg["cheb"], max_nrhs=16, level_degrees=degs)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t
        top = H.n_levels - 1
        rows = H.rows(top)
        nn, nfree, nc = H.info(top)
        nrhs = cfg["nrhs"]
        b = H.vector(top, nrhs)
        if name.startswith("c1"):
            xq = H.quadrature_points(top)
            fq = 2 * np.pi ** 2 * np.sin(np.pi * xq[..., 0]) * np.sin(np.pi * xq[..., 1])
            H.load_vector(top, fq.reshape(-1), b, col=0, per_qp=True)
        elif name.startswith("c4"):
            H.load_vector(top, np.array([0.0, 0.0, -1.0]), b, col=0)
        else:
            H.load_vector(top, np.ones(1), b, col=0)
        if nrhs > 1:
            r = normal_rhs(rows, [1000 + j for j in range(1, nrhs)])
            b[:, 1:] = torch.tensor(r, device="cuda")
        out = {"config": name + ("_" + variant if variant else ""),
               "levels": [list(lv.n) for lv in levels], "level_degrees": degs, "fine_free_dofs":
               int(nfree) * cfg["ncomp"], "nrhs": nrhs, "setup_s": setup_s,
               "setup_dofs_per_s": int(nn) * cfg["ncomp"] / setup_s,
               "setup_phases_s": H.setup_seconds(),
               "hierarchy_bytes": H.hierarchy_bytes()}
        for mode, tag in [(_abi.FP32_MG_FP64_CG, "fp32_mg_fp64_cg"), (_abi.FP64_MG, "fp64_mg"),
                          (_abi.FP32_MG_DW_CG, "fp32_mg_dw_cg")]:
            x = torch.zeros_like(b)
            steps = args.steps if nfree * nrhs < 5e6 else max(5, args.steps // 10)
            for _ in range(max(3, args.warmup)):
                st, its, rel = H.pcg(b, x, mode=mode)
            ts = []
            for _ in range(steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                st, its, rel = H.pcg(b, x, mode=mode)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            ts.sort()
            med = ts[len(ts) // 2]
            out[tag] = {"p50_ms": med, "p99_ms": ts[min(len(ts) - 1, int(0.99 * len(ts)))],
                        "solves": steps, "iterations": [int(i) for i in its],
                        "max_relres": float(max(rel)),
                        "solved_dofs_per_s": nfree * cfg["ncomp"] * nrhs / (med / 1e3)}
        # FP32 V-cycle per level and component, and the fine level's kernels
        # against the measured HBM bandwidth
        peaks, _ = _peaks()
        out["vcycle_breakdown_ms"], out["fine_level_kernels_hbm"] = vcycle_kernel_table(
            H, degs or [cfg["degree"]] * H.n_levels, cfg["ncomp"], nrhs, cfg["cheb"],
            peaks["hbm_gbs"])
        if rank == 0:
            print(json.dumps(out), flush=True)
        H.close()
    run_nested_cube(args, rank)


def run_nested_cube(args, rank):
    """The paper's nested cube (Sec. 5 comparison of global coarsening and the
    non-nested transfer): [-1,1]^3, Q4, levels 2^3 .. 32^3 cells by global
    refinement, f = 1.  Same hierarchy solved with the non-nested point
    evaluation and with the nested sum-factorized transfer."""
    import numpy as np
    import torch
    from paper_2412_10910_gb300 import _abi, nnmg
    from synthetic.meshes import Level, boundary_vertex_mask, refine_nested, structured_grid

    v, c = structured_grid((2, 2, 2), (2.0, 2.0, 2.0))
    lv = [Level(3, v - 1.0, c, boundary_vertex_mask(v, (2.0, 2.0, 2.0)).astype(np.uint8), (2, 2, 2))]
    par = [None]
    for _ in range(4):
        f, p_, c_ = refine_nested(lv[-1])
        lv.append(f)
        par.append((p_, c_))
    H = nnmg.Hierarchy(lv, 4, cheb_degree=3, max_nrhs=16)
    top = len(lv) - 1
    nn_, nfree, _ = H.info(top)
    b = H.vector(top, 1)
    H.load_vector(top, np.ones(1), b, col=0)
    x = torch.zeros_like(b)
    out = {"config": "nested_cube_q4 (paper Sec. 5 cube, levels 2^3..32^3)", "fine_free_dofs": nfree}
    for tag in ("non_nested", "nested_gc"):
        for l in range(1, len(lv)):
            H.set_nested(l, *(par[l] if tag == "nested_gc" else (None, None)))
        for _ in range(3):
            st, its, rel = H.pcg(b, x)
        ts = []
        for _ in range(max(5, args.steps // 2)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st, its, rel = H.pcg(b, x)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ts.sort()
        xc = torch.randn(H.rows(top - 1), 1, dtype=torch.float32, device="cuda")
        xf = H.vector(top, 1, torch.float32)
        rc = H.vector(top - 1, 1, torch.float32)
        tr = []
        for i in range(13):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            H.prolongate(top, xc, xf)
            e1.record()
            H.restrict(top, xf, rc)
            e2.record()
            torch.cuda.synchronize()
            if i >= 3:
                tr.append((e0.elapsed_time(e1), e1.elapsed_time(e2)))
        out[tag] = {"solve_p50_ms": ts[len(ts) // 2], "iterations": [int(i) for i in its],
                    "max_relres": float(max(rel)),
                    "finest_prolongation_ms": statistics.median(t[0] for t in tr),
                    "finest_restriction_ms": statistics.median(t[1] for t in tr)}
    if rank == 0:
        print(json.dumps(out), flush=True)
    H.close()


def run_serving(args, rank):
    """Serving mix: 12 cached mesh families, Poisson arrivals, continuous batching."""
    line = serving_mix(args.requests, args.rate)
    if rank == 0:
        print(json.dumps(line), flush=True)


def serving_mix(n_requests, fixed_rate=0.0):
    """The serving mix's line: calibration burst, then n_requests Poisson
    arrivals at fixed_rate (0: 0.8 x the calibrated service rate)."""
    import numpy as np
    import torch
    from paper_2412_10910_gb300.serving import FamilySpec, Request, Server, latency_stats
    from synthetic.serving import request_rhs, serving_families, serving_requests

    fams = serving_families()
    specs = {f["name"]: FamilySpec(f["levels"], f["degree"]) for f in fams}
    budget = int(0.5 * torch.cuda.get_device_properties(0).total_memory)
    server = Server(specs, budget_bytes=budget)
    t = time.perf_counter()
    server.prepare([f["name"] for f in fams])
    setup_s = time.perf_counter() - t

    def make(reqs):
        out = []
        for rid, (fi, m, arr) in enumerate(reqs):
            f = fams[fi]
            out.append(Request(rid, f["name"], request_rhs(f["n_nodes"], m, rid), arrival=arr))
        return out

    # calibration: a closed burst (all requests at t = 0) gives the service rate
    ncal = max(60, n_requests // 20)
    cal = make(serving_requests(fams, ncal, seed=7, rate=1e9))
    t = time.perf_counter()
    server.run(cal)
    cal_rate = ncal / (time.perf_counter() - t)
    rate = fixed_rate if fixed_rate else 0.8 * cal_rate
    for e in server.engines.values():          # occupancy of the timed run only
        e.iterations = e.column_iterations = e.width_iterations = 0
        e.host_copy_s = 0.0
    reqs = make(serving_requests(fams, n_requests, seed=6, rate=rate))
    t = time.perf_counter()
    done = server.run(reqs)
    span = time.perf_counter() - t
    dofs = sum(next(f for f in fams if f["name"] == r.family)["n_free"] * r.nrhs for r in done)
    ok = all(all(s == 0 for s in r.status) and max(r.relres) <= 1e-8 for r in done)
    per_family = {}
    for f in fams:
        mine = [r for r in done if r.family == f["name"]]
        eng = server.engines.get(f["name"])
        if not mine:
            continue
        lat = np.array([r.t_done - r.arrival for r in mine])
        per_family[f["name"]] = {
            "requests": len(mine), "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)),
            # occupied slots per iteration / 16, and per column the batch computed
            "slot_occupancy": (eng.column_iterations / max(1, eng.iterations * eng.nslots)
                               if eng is not None else None),
            "occupied_per_computed_column": (eng.column_iterations / max(1, eng.width_iterations)
                                             if eng is not None else None),
            "host_copy_s": eng.host_copy_s if eng is not None else None}
    line = {"metric": "serving: solved DoF/s and p50/p99 request latency", "value": dofs / span,
            "unit": UNIT, "requests": len(done), "arrival_rate_per_s": rate,
            "calibration_rate_per_s": cal_rate, "makespan_s": span,
            "latency": latency_stats(done), "all_converged": ok, "setup_s_12_families": setup_s,
            "evictions": server.evictions, "budget_bytes": budget, "per_family": per_family,
            "families": [f["name"] for f in fams], "data": "synthetic",
            "config": {"workload": "serving mix: 12 jittered non-nested families (seed 5), "
                                   "Poisson arrivals (seed 6), 1-16 N(0,1) RHS, FP32 V-cycle / "
                                   "FP64 CG to 1e-8, continuous batching over 16 slots per family"}}
    server.close()
    return line


# requests of the serving mix appended to the full line
SERVING_REQUESTS = 600

# FMA-chain iterations per probe launch (about 50 ms each on GB300)
PROBE_ITERS = {0: 4000, 1: 200000, 2: 100000}


def pipe_rates(reps=3):
    """Best of `reps` FMA-chain probe launches per pipe (nnmg_pipe_rate), in
    multiply-adds per second: FP64 (DFMA), FP32 (FFMA), packed FP32 (FFMA2)."""
    from paper_2412_10910_gb300 import nnmg
    return {name: max(nnmg.nnmg_pipe_rate(kind, PROBE_ITERS[kind]) for _ in range(reps))
            for kind, name in ((0, "fp64"), (1, "fp32"), (2, "fp32_packed"))}


def run_peaks(args, rank):
    """The arithmetic pipe rates of this GPU (the ALU rooflines' denominators),
    with the SM clock sampled while the probes run: rate / (SMs x median clock)
    gives the multiply-adds per clock and SM the pipe sustains."""
    import torch
    clocks = Clocks()
    clocks.start()
    rates = pipe_rates(reps=max(3, args.steps))
    torch.cuda.synchronize()
    clk = clocks.stop()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = clk.get("sm_mhz") or 2070.0
    per_clk = {k: v / (sms * mhz * 1e6) for k, v in rates.items()}
    if rank == 0:
        print(json.dumps({"only": "peaks", "fma_per_s": rates, "sms": sms,
                          "fma_per_clock_per_sm": per_clk, "clocks": clk,
                          "fp64_tflops": 2 * rates["fp64"] / 1e12,
                          "fp32_tflops": 2 * max(rates["fp32"], rates["fp32_packed"]) / 1e12}),
              flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true",
                    help="leave the shortened serving mix out of the full line")
    ap.add_argument("--only", choices=["solve", "solve64", "solvedw", "vcycle", "op64", "op32",
                                       "opdw", "prolong", "restrict", "serving", "configs", "peaks"],
                    default=None, help="run only one timed section (for profiler launch lists), "
                    "or the serving mix")
    ap.add_argument("--requests", type=int, default=2000, help="serving mix: number of requests")
    ap.add_argument("--rate", type=float, default=0.0,
                    help="serving mix: arrivals per second (default 0.8 x the calibrated rate)")
    ap.add_argument("--config", default=CONFIG, choices=["c1_2d_q1", "c2_3d_q2", "c3_3d_q4_deformed"],
                    help="Poisson configuration of the --only sections (the full line always "
                         "measures config 2)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2412_10910_gb300 import _abi, nnmg
    from synthetic import config_levels
    from synthetic.meshes import CONFIGS

    torch.cuda.set_device(local)
    if args.only == "peaks":
        return run_peaks(args, rank)
    if args.only == "serving":
        return run_serving(args, rank)
    if args.only == "configs":
        return run_configs(args, rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def _reduce(v, op):
        t = torch.tensor([v], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=op)
        return float(t.item())

    def max_over_ranks(v):
        return v if world == 1 else _reduce(v, dist.ReduceOp.MAX)

    def sum_over_ranks(v):
        return v if world == 1 else _reduce(v, dist.ReduceOp.SUM)

    name = args.config if args.only else CONFIG
    cfg = CONFIGS[name]
    levels = config_levels(name)
    nrhs = cfg["nrhs"]
    H = nnmg.Hierarchy(levels, cfg["degree"], 1, cheb_degree=cfg["cheb"], max_nrhs=16)
    top = H.n_levels - 1
    n_nodes, n_free, n_cells = H.info(top)
    rows = H.rows(top)
    free_rows = ~H.constrained(top)
    b = _rhs(rows, free_rows, H, top, nrhs)
    x = torch.zeros_like(b)
    stream = torch.cuda.current_stream()

    def solve(mode):
        return H.pcg(b, x, mode=mode, rtol=1e-8, maxit=100)

    if args.only:
        fns = {"solve": lambda: solve(_abi.FP32_MG_FP64_CG), "solve64": lambda: solve(_abi.FP64_MG),
               "solvedw": lambda: solve(_abi.FP32_MG_DW_CG)}
        if args.only in ("vcycle",):
            r32 = torch.randn(rows, nrhs, dtype=torch.float32, device="cuda")
            z32 = torch.empty_like(r32)
            fns["vcycle"] = lambda: H.vcycle(r32, z32)
        if args.only in ("prolong", "restrict"):
            # the finest pair's FP32 transfers (nnmg_prolongate zeroes the fine
            # vector first; nnmg_restrict runs both phases)
            xc = torch.randn(H.rows(top - 1), nrhs, device="cuda")
            xf = torch.randn(rows, nrhs, device="cuda")
            fns["prolong"] = lambda: H.prolongate(top, xc, xf)
            fns["restrict"] = lambda: H.restrict(top, xf, xc)
        if args.only in ("op64", "op32", "opdw"):
            dt = torch.float32 if args.only == "op32" else torch.float64
            xo = torch.randn(rows, nrhs, dtype=dt, device="cuda")
            yo = torch.empty_like(xo)
            fns[args.only] = lambda: H.apply(top, xo, yo, double_word=(args.only == "opdw"))
        fn = fns[args.only]
        for _ in range(args.warmup):
            fn()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed")      # profilers select this range
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        barrier()
        if rank == 0:
            choice = {p: H.operator_choice(top, p, nrhs) for p in (_abi.F32, _abi.F64, _abi.F64_DW)}
            print(json.dumps({"only": args.only, "config": name,
                              "ms_per_step": e0.elapsed_time(e1) / args.steps,
                              "operator_choice_top": {"f32": choice[_abi.F32], "f64": choice[_abi.F64],
                                                      "f64_dw": choice[_abi.F64_DW]}}))
        H.close()
        return

    def timed(fn, k, w):
        for _ in range(w):
            fn()
        barrier()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(k)]
        out = None
        for e0, e1 in evs:
            e0.record(stream)
            out = fn()
            e1.record(stream)
        barrier()
        ts = [e0.elapsed_time(e1) for e0, e1 in evs]
        return ts, out

    # ---- headline: FP32 V-cycle inside FP64 CG
    clocks = Clocks()
    for _ in range(args.warmup):
        solve(_abi.FP32_MG_FP64_CG)
    barrier()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    per_step = []
    iters = None
    ev0.record(stream)
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, its, rel = solve(_abi.FP32_MG_FP64_CG)
        e1.record(stream)
        per_step.append((e0, e1))
        iters = its
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    lat = sorted(e0.elapsed_time(e1) for e0, e1 in per_step)
    dofs = n_free * nrhs
    total_ms, total_units, _ = replica_aggregate(ev0.elapsed_time(ev1), dofs * args.steps, world,
                                                 max_over_ranks, sum_over_ranks)
    ms = total_ms / args.steps
    value = total_units / (total_ms / 1e3)
    relres = [float(r) for r in rel]

    # ---- comparator: plain FP64 multigrid
    ts64, (st64, its64, rel64) = timed(lambda: solve(_abi.FP64_MG), max(2, args.steps // 3), 1)
    ms64 = max_over_ranks(statistics.mean(ts64))
    # ---- variant: the CG's operator in double-word arithmetic on the FP32 pipes
    tsdw, (stdw, itsdw, reldw) = timed(lambda: solve(_abi.FP32_MG_DW_CG), max(3, args.steps // 2), 2)
    msdw = max_over_ranks(statistics.mean(tsdw))

    # ---- V-cycle and operator throughput (fine level, all RHS)
    r32 = torch.randn(rows, nrhs, dtype=torch.float32, device="cuda")
    z32 = torch.empty_like(r32)
    tv, _ = timed(lambda: H.vcycle(r32, z32), 10, 3)
    x64 = torch.randn(rows, nrhs, dtype=torch.float64, device="cuda")
    y64 = torch.empty_like(x64)
    top64, _ = timed(lambda: H.apply(top, x64, y64), 10, 3)
    x32 = x64.float()
    y32 = torch.empty_like(x32)
    top32, _ = timed(lambda: H.apply(top, x32, y32), 10, 3)
    topdw, _ = timed(lambda: H.apply(top, x64, y64, double_word=True), 10, 3)

    # ---- per-level V-cycle breakdown and HBM fraction of the fine level's kernels
    peaks, peak_kind = _peaks()
    breakdown, kern_hbm = vcycle_kernel_table(H, [cfg["degree"]] * H.n_levels, 1, nrhs, cfg["cheb"],
                                              peaks["hbm_gbs"])

    # ---- end to end through the host-buffer C call
    bh = torch.empty(rows * nrhs, dtype=torch.float64, pin_memory=True)
    bh.copy_(b.reshape(-1).cpu())
    xh = torch.empty_like(bh)
    for _ in range(2):
        H.pcg_host(bh, xh, nrhs)
    barrier()
    t0 = time.perf_counter()
    ke = max(2, args.steps // 2)
    for _ in range(ke):
        H.pcg_host(bh, xh, nrhs)
    barrier()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / ke)

    # ---- roofline of the dominant kernel: the FP64 fine-level operator (ALU bound),
    # against the FP64 pipe rate measured now by the FMA-chain probe
    rates = pipe_rates(reps=3)
    fp64_peak = rates["fp64"] / 1e12
    flops_cell, ops_cell = poisson3d_work(cfg["degree"] + 1)
    flops = float(flops_cell) * n_cells * nrhs
    op64_ms = statistics.mean(top64)
    achieved = flops / (op64_ms / 1e3) / 1e12
    pipe = ops_cell * n_cells * nrhs / (op64_ms / 1e3) / 1e12
    from paper_2412_10910_gb300 import _abi
    choice64 = H.operator_choice(top, _abi.F64, nrhs)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "fine_free_dofs": n_free, "nrhs": nrhs,
                   "levels": [list(lv.n) for lv in levels], "parallelism": f"replicas{world}",
                   "l2": "working set > L2 (no flush)"},
        "iterations": [int(i) for i in iters], "relres": relres,
        "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
        "fp64_mg": {"value": dofs * world / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64,
                    "iterations": [int(i) for i in its64]},
        "fp32_mg_dw_cg": {"value": dofs * world / (msdw / 1e3), "unit": UNIT, "ms_per_step": msdw,
                          "iterations": [int(i) for i in itsdw],
                          "max_relres": float(max(reldw)),
                          "note": "CG operator in double-word (2 x FP32, ~48-bit) arithmetic; "
                                  "vectors, dots and updates FP64"},
        "vcycle_gdofs": dofs / (statistics.mean(tv) / 1e3) / 1e9,
        "operator_gdofs": {"f32": n_nodes * nrhs / (statistics.mean(top32) / 1e3) / 1e9,
                           "f64": n_nodes * nrhs / (op64_ms / 1e3) / 1e9,
                           "f64_double_word": n_nodes * nrhs / (statistics.mean(topdw) / 1e3) / 1e9},
        # The FP64 pipe takes one FMA, MUL or ADD per slot, 2 per clock per SM:
        # the roofline counts the kernel's FP64 operations against those slots
        # (flops beside it: an ADD is one flop in a full slot).
        "roofline": {"kernel": operator_kernel_name(choice64, cfg["degree"], "double")
                     + ", FP64 fine-level operator, 8 RHS",
                     "bound": "alu", "achieved": pipe, "peak": fp64_peak,
                     "unit": "T FP64-pipe op/s (FMA, MUL or ADD)", "frac": pipe / fp64_peak,
                     "ops_per_cell_rhs": ops_cell, "flops_per_cell_rhs": flops_cell,
                     "achieved_tflops": achieved, "peak_tflops": 2 * fp64_peak,
                     "nominal_peak": FP64_PIPE_TOPS, "frac_of_nominal": pipe / FP64_PIPE_TOPS,
                     # DRAM bytes read + written per launch: ncu's bytes per (cell, RHS)
                     # for this kernel on this workload, times the launch's cells x RHS
                     "traffic": op64_traffic(choice64, n_cells, nrhs),
                     "peak_source": "measured in this run: FMA-chain probe (nnmg_pipe_rate, "
                                    "best of 3, DFMA chains on every SM); nominal "
                                    "152 SM x 2 FP64 op/clk x 2.07 GHz beside it"},
        "pipe_rates_fma_per_s": rates,
        # FP32 V-cycle per level and component (ms, event-timed eager run) and the
        # fine level's kernels against the measured HBM copy bandwidth
        "vcycle_breakdown_ms": breakdown,
        "fine_level_kernels_hbm": kern_hbm,
        "e2e": {"value": dofs * world / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": rows * nrhs * 8, "d2h_bytes_per_step": rows * nrhs * 8},
        "gpu_launches": kernels_per_solve(H.n_levels, cfg["cheb"], int(max(iters))) * args.steps,
        "clocks": clk,
        "hbm_peak_gbs": peaks.get("hbm_gbs"), "peak_kind": peak_kind,
    }
    # the records after the timed solves: a failure there is reported in the
    # line, which is printed in any case
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline_sample(8)
        except Exception as exc:                       # noqa: BLE001
            line["cpu_baseline"] = {"kind": "oracle", "error": str(exc)[-500:]}
    H.close()
    if rank == 0 and world == 1 and not args.no_serving:
        # the serving mix, shortened (`--only serving` runs the 2000-request mix)
        try:
            sv = serving_mix(SERVING_REQUESTS)
            line["serving"] = {k: sv[k] for k in ("metric", "value", "unit", "requests",
                                                 "arrival_rate_per_s", "calibration_rate_per_s",
                                                 "makespan_s", "latency", "all_converged",
                                                 "setup_s_12_families")}
            line["serving"]["workload"] = sv["config"]["workload"]
        except Exception as exc:                       # noqa: BLE001
            line["serving"] = {"error": str(exc)[-500:]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
