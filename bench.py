#!/usr/bin/env python
"""Benchmark of the scaled-stencil vector operator apply (physical stencil scaling, Sec. 2 of
arXiv 1908.08666) on one GB300, through the libhhgs C ABI.

Workload: 3D linear elasticity (nu = 0.3) on the unit cube split into 6 Kuhn macro
tetrahedra, refined to level 7 (129^3 = 2,146,689 nodes, 6.44 MDoF); Young's modulus a
lognormal field (exp of a Gaussian random field smoothed with correlation length 0.1,
sigma = 1, seed 2); input vector i.i.d. uniform[-1, 1] (seed 3).  One step = one full FP32
operator application y = A x: the macro-interior scaled-stencil kernels plus the macro
skeleton (interface) kernel.  The L2 cache is flushed (256 MB write, outside the timed
events) before every timed step.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle instead (the
reference arm of this build: the paper has no code; its FP64 definition-level oracle is
the baseline).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

LEVEL = 7
NU = 0.3
# algorithmic cost of one macro-interior node of the FP32 apply
BYTES_PER_NODE_F32 = 28  # read x (12 B) and k (4 B), write y (12 B)
STORED_BYTES_PER_NODE_F32 = 135 * 4 + 24  # the 15 stored 3x3 blocks, x and y
FLOPS_PER_NODE = 723     # FMA = 2 flops, as the kernel evaluates the scaled stencil
METRIC = "scaled-stencil vector matvec GDoF/s & % of HBM peak; time to 1e-8 residual"
WORKLOAD = "elasticity, 6-macro Kuhn unit cube, level 7 (129^3 nodes), lognormal E, FP32 physical-scaling apply"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--level", type=int, default=LEVEL)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-stokes", action="store_true")
    ap.add_argument("--no-plume", action="store_true")
    ap.add_argument("--no-elastostatics", action="store_true")
    ap.add_argument("--no-foam", action="store_true")
    ap.add_argument("--no-twod", action="store_true")
    ap.add_argument("--foam-level", type=int, default=7)
    ap.add_argument("--elastostatics-level", type=int, default=6)
    ap.add_argument("--plume-level", type=int, default=5)
    ap.add_argument("--no-kernel-table", action="store_true")
    ap.add_argument("--no-carreau", action="store_true")
    ap.add_argument("--carreau-level", type=int, default=8)
    ap.add_argument("--no-learn", action="store_true")
    ap.add_argument("--learn-train-level", type=int, default=6)
    ap.add_argument("--learn-level", type=int, default=8)
    ap.add_argument("--learn-seeds", type=int, default=24)
    ap.add_argument("--learn-steps", type=int, default=4000)
    ap.add_argument("--learn-coarsen", type=int, default=1)
    ap.add_argument("--learn-coarse-train-level", type=int, default=6)
    ap.add_argument("--learn-coarse-seeds", type=int, default=12)
    ap.add_argument("--no-learn-stokes", action="store_true")
    ap.add_argument("--learn-stokes-fields", type=int, default=8)
    ap.add_argument("--learn-stokes-steps", type=int, default=2000)
    ap.add_argument("--learn-stokes-level", type=int, default=8)
    return ap.parse_args()


def max_over_ranks(v, world, device="cuda"):
    """The largest v over all ranks (the job takes as long as its slowest rank)."""
    if world <= 1:
        return float(v)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(dofs_per_rank, ms_per_step, world):
    """Whole-job throughput in GDoF/s: every rank applies its own replica (weak scaling)."""
    return world * dofs_per_rank / (ms_per_step * 1e-3) / 1e9


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------- clocks


class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def fp32_peak(B, torch, h, stream, reps=5):
    """FP32 FMA issue rate measured by the library's probe kernel (hhg_fp32_fma_probe: 8
    independent FMA chains per thread on SMs x 8 blocks of 256 threads), timed with CUDA events on
    the context's stream: the best of `reps` launches of the plain (fma.rn.f32) and the packed
    two-lane (fma.rn.f32x2) form.  Returns the higher rate, both rates and the SM count."""
    out = torch.zeros(1, device="cuda")
    res = {}
    sms = None
    for packed in (0, 1):
        iters = 100000
        B.hhg_fp32_fma_probe(h, packed, iters, out)
        torch.cuda.synchronize()
        best = None
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fl, sms = B.hhg_fp32_fma_probe(h, packed, iters, out)
            b.record(stream)
            torch.cuda.synchronize()
            r = fl / (a.elapsed_time(b) * 1e-3) / 1e12
            best = r if best is None else max(best, r)
        res["fma_f32x2" if packed else "fma_f32"] = round(best, 2)
    return max(res.values()), res, sms


# ---------------------------------------------------------------------------- workload


def workload_fields(coords, level):
    import hhg_inputs as hi

    N = 1 << level
    kgrid = hi.lognormal_grid(N, seed=2)
    xgrid = hi.uniform_grid(N, seed=3)
    return hi.sample_grid(kgrid[..., None], coords)[:, 0], hi.sample_grid(xgrid, coords)


def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("hhg_sweep.cu", "hhg_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_1908_08666_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per interior-kernel launch from the committed ncu summary, if it was taken
    on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "interior_apply_f32_cube6_l7.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("kernel_source_sha") != kernel_source_sha():
        return None
    return d.get("dram_bytes_per_launch")


_GRIDS = {}


def _grids(level):
    import hhg_inputs as hi

    if level not in _GRIDS:
        N = 1 << level
        _GRIDS[level] = (hi.lognormal_grid(N, seed=2), hi.uniform_grid(N, seed=3))
    return _GRIDS[level]


_BW = {}

# The CPU baseline applies the oracle's assembled operator on a level the oracle can assemble
# in seconds (its element-record assembly needs about 2 GB at level 5 and grows 8x per level)
BASELINE_LEVEL = 5


def _baseline_operator(level, workload_level):
    """The oracle's FP64 physical-scaling operator (scipy CSR, Dirichlet identity rows) of the
    benchmark workload on the 6-macro cube at `level`: lognormal E of the workload's grid
    (seed 2, correlation length 0.1), nu = 0.3; x from the workload's uniform field (seed 3)."""
    import hhg_inputs as hi
    from oracle import fem, mesh, operators as op

    xyz, tets = hi.kuhn_cube(1)
    lv = mesh.build_level(mesh.MacroMesh.build(xyz, tets), level)
    kgrid, xgrid = _grids(workload_level)
    k = hi.sample_grid(kgrid[..., None], lv.coords)[:, 0]
    x = hi.sample_grid(xgrid, lv.coords)
    ce, cd = fem.elasticity_coefficients(NU)
    K = fem.element_stiffness(lv.coords[lv.elems], ce, cd)
    A = op.with_dirichlet_rows(op.scaled_operator(lv, K, k), lv.dirichlet)
    return A.tocsr(), np.ascontiguousarray(x.reshape(-1)), lv


def _baseline_worker_init(path):
    d = np.load(path, allow_pickle=True)
    _BW.update(blocks=list(d["blocks"]), x=d["x"])


def _baseline_apply(job):
    """reps applications of row block q of the oracle's operator (y_q = A_q x)."""
    q, reps = job
    A, x = _BW["blocks"][q], _BW["x"]
    y = None
    for _ in range(reps):
        y = A @ x
    return float(y[0]) if y is not None and len(y) else 0.0


class CpuBaseline:
    """The oracle's FP64 operator apply (its assembled scipy CSR matrix, y = A x) on every host
    core: the rows are split into one block per core, each block applied by its own spawned
    process (spawn, not fork: the parent holds a CUDA context); throughput = 3 x nodes x reps /
    the wall-clock time of the whole pool round (after an untimed warm-up round)."""

    def __init__(self, level=BASELINE_LEVEL, workload_level=7, cores=None):
        import multiprocessing as mp
        import tempfile

        self.level = level
        self.cores = cores or len(os.sched_getaffinity(0))
        t0 = time.perf_counter()
        A, x, lv = _baseline_operator(level, workload_level)
        self.setup_s = time.perf_counter() - t0
        self.nodes = lv.num_nodes
        self.nfree = int((~lv.dirichlet).sum())
        rows = A.shape[0]
        cuts = np.linspace(0, rows // 3, self.cores + 1).astype(np.int64) * 3
        blocks = np.empty(self.cores, dtype=object)
        for q in range(self.cores):
            blocks[q] = A[cuts[q]:cuts[q + 1]]
        self.tmp = tempfile.NamedTemporaryFile(suffix=".npz", delete=False)
        self.tmp.close()
        np.savez(self.tmp.name, blocks=blocks, x=x)
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_baseline_worker_init,
                                                 initargs=(self.tmp.name,))
        t0 = time.perf_counter()
        self.pool.map(_baseline_apply, [(q, 1) for q in range(self.cores)])  # every worker initialised
        self.round_s = max(1e-4, time.perf_counter() - t0)

    def _round(self, reps):
        t0 = time.perf_counter()
        self.pool.map(_baseline_apply, [(q, reps) for q in range(self.cores)])
        return time.perf_counter() - t0

    def measure(self, budget_s):
        reps = 1
        while True:  # calibrate: a round long enough that the pool's dispatch cost is negligible
            dt = self._round(reps)
            if dt > 0.2 * budget_s or reps > 1 << 20:
                break
            reps *= 4
        reps = max(1, int(reps * budget_s / dt))
        dt = self._round(reps)
        return {"value": 3.0 * self.nodes * reps / dt / 1e9, "unit": "GDoF/s", "cores": self.cores, "kind": "oracle",
                "free_dof_value": 3.0 * self.nfree * reps / dt / 1e9,
                "sample": "y = A x by the oracle's assembled FP64 physical-scaling operator (scipy CSR, built "
                          "once in %.1f s outside the timing) of the same workload on the 6-macro cube at level "
                          "%d (%d nodes; the level-%d lognormal E and x sampled at its nodes), rows split over "
                          "%d spawned processes, %d applications each, %.2f s wall clock for the whole pool"
                          % (self.setup_s, self.level, self.nodes, 7, self.cores, reps, dt)}

    def close(self):
        self.pool.close()
        self.pool.join()
        os.unlink(self.tmp.name)


def c1_pcg_baseline():
    """The oracle's Jacobi-preconditioned CG (textbook, Saad Alg. 9.1) on the single unit macro
    tetrahedron at level 5 (6545 nodes), E = 1 + 0.5 sin sin sin, nu = 0.3, f ~ U[-1, 1] (seed 1),
    to a relative residual of 1e-10; one host core."""
    import hhg_inputs as hi
    from oracle import fem, mesh, operators as op, solvers as S

    xyz, tets = hi.unit_tet()
    lv = mesh.build_level(mesh.MacroMesh.build(xyz, tets), 5)
    ce, cd = fem.elasticity_coefficients(NU)
    K = fem.element_stiffness(lv.coords[lv.elems], ce, cd)
    A = op.with_dirichlet_rows(op.scaled_operator(lv, K, hi.young_sine(lv.coords)), lv.dirichlet)
    f = hi.node_noise(lv.coords, seed=1)
    f[lv.dirichlet] = 0.0
    D = S.point_diagonal(A, lv.dirichlet)
    t0 = time.perf_counter()
    x, it = S.pcg(A, lv.dirichlet, f, np.zeros_like(f), lambda r: r / D, 1e-10, 5000)
    dt = time.perf_counter() - t0
    r = S.residual(A, lv.dirichlet, f, x)
    return {"seconds": round(dt, 4), "iterations": int(it), "nodes": lv.num_nodes, "cores": 1,
            "rel_residual": float(np.sqrt((r**2).sum() / (f[~lv.dirichlet]**2).sum()))}


def cpu_baseline(budget_s=12.0):
    """The oracle timed on this host's cores: the all-core operator apply, plus the C1 solve."""
    b = CpuBaseline()
    try:
        out = b.measure(budget_s)
    finally:
        b.close()
    out["c1_jacobi_pcg"] = c1_pcg_baseline()
    return out


def solve_times(B, torch, h, level, coords_u):
    """Time to an FP64 relative residual of 1e-8 on the same workload (f ~ U[-1, 1], seed 3,
    x0 = 0): FP64 iterative refinement around FP32 MG-CG, and plain FP64 MG-CG (V(2,2)
    Chebyshev, exact coarse solve on level 2)."""
    import hhg_inputs as hi

    N = 1 << level
    E, U, _ = B.hhg_num_nodes(h, level)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B.hhg_mg_setup(h)
    setup_s = time.perf_counter() - t0
    fu = hi.sample_grid(hi.uniform_grid(N, seed=3), coords_u)
    src = torch.as_tensor(np.ascontiguousarray(fu.T).reshape(-1), dtype=torch.float64, device="cuda")
    f = torch.empty(3 * E, dtype=torch.float64, device="cuda")
    B.hhg_scatter_unique(h, level, B.F64, 3, src, f)
    out = {"rtol": 1e-8, "setup_s": round(setup_s, 4)}
    for name, method, kw in (("ir_fp64_over_fp32_mgcg", B.SOLVE_IR_MG_CG, dict(inner_rtol=1e-3, inner_max_iter=50)),
                             ("fp64_mgcg", B.SOLVE_MG_CG, {})):
        best = None
        for _ in range(2):
            x = torch.zeros_like(f)
            torch.cuda.synchronize()
            rep = B.hhg_solve(h, f, x, method=method, level=level, dt=B.F64, rtol=1e-8, max_iter=100, **kw)
            if best is None or rep["seconds"] < best["seconds"]:
                best = rep
        r = torch.empty_like(f)
        r2 = B.hhg_residual(h, level, B.F64, f, x, r, want_norm=True)
        out[name] = {"seconds": round(best["seconds"], 5), "iterations": best["iterations"],
                     "inner_iterations": best["inner_iterations"], "rel_residual_fp64": float(np.sqrt(r2)) /
                     best["residual0"], "converged": bool(best["converged"])}
    out["speedup_ir_vs_fp64"] = round(out["fp64_mgcg"]["seconds"] / out["ir_fp64_over_fp32_mgcg"]["seconds"], 3)
    # the paper's solver (Sec. 5.1.2): stationary V(3,3) cycles with the hybrid Gauss-Seidel smoother
    B.hhg_set_mg_params(h, smoother=B.SMOOTH_HYBRID_GS, pre=3, post=3)
    B.hhg_mg_setup(h)
    x = torch.zeros_like(f)
    torch.cuda.synchronize()
    rep = B.hhg_solve(h, f, x, method=B.SOLVE_MG, level=level, dt=B.F64, rtol=1e-8, max_iter=200,
                      allow_not_converged=True)
    r = torch.empty_like(f)
    r2 = B.hhg_residual(h, level, B.F64, f, x, r, want_norm=True)
    out["fp64_mg_v33_hybrid_gs"] = {"seconds": round(rep["seconds"], 5), "iterations": rep["iterations"],
                                    "rel_residual_fp64": float(np.sqrt(r2)) / rep["residual0"],
                                    "converged": bool(rep["converged"]),
                                    "note": "stationary V(3,3) cycles, hybrid Gauss-Seidel smoother (omega 2/3 on the "
                                            "skeleton), exact coarse solve at level 2"}
    B.hhg_set_mg_params(h)
    B.hhg_mg_setup(h)
    return out


# algorithmic bytes per node of each sweep (every array touched once): x (3 comps), k, y;
# + f for the residual and a Jacobi step; x, f, k, d read and x, d written for a Chebyshev step
SWEEP_BYTES = {("apply", 8): 56, ("residual", 8): 80, ("jacobi", 8): 80, ("chebyshev", 8): 128,
               ("apply", 4): 28, ("residual", 4): 40, ("jacobi", 4): 40, ("chebyshev", 4): 64,
               ("apply_bf16_k", 4): 26}
for _name in ("apply_tile_kernel", "apply_per_macro_launches", "apply_one_launch"):
    SWEEP_BYTES[(_name, 8)], SWEEP_BYTES[(_name, 4)] = 56, 28


def kernel_table(B, torch, dev, stream, levels=(7, 8), reps=10):
    """Every sweep of the hot path on the C2 workload (lognormal E seed 2, x and f U[-1, 1]
    seed 3) at each level: apply, residual, one Jacobi and one Chebyshev step in FP64 and FP32,
    and the FP32 apply with the BF16 coefficient.  Device time of the whole sweep per call
    (CUDA events; the L2 is flushed before each call), GDoF/s = 3 x unique nodes / t, the
    algorithmic bytes per node and their rate against the measured copy bandwidth."""
    import hhg_inputs as hi

    hbm_peak, peak_kind = measured_peaks()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    out = {"workload": "C2: 6-macro cube, lognormal E (seed 2), x and f ~ U[-1,1] (seed 3)",
           "hbm_peak_gbs": hbm_peak, "hbm_peak_source": peak_kind, "reps": reps, "rows": []}
    xyz, tets = hi.kuhn_cube(1)
    for level in levels:
        h = B.hhg_create(dev, stream.cuda_stream)
        try:
            B.hhg_set_macro_mesh(h, xyz, tets)
            B.hhg_refine(h, level)
            B.hhg_set_problem(h, nu=NU)
            E, U, _ = B.hhg_num_nodes(h, level)
            ce = B.hhg_entry_coords(h, level)
            e2u, udir = B.hhg_entry_to_unique(h, level)
            first = np.full(U, -1, dtype=np.int64)
            first[e2u[::-1]] = np.arange(E)[::-1]
            k_u, x_u = workload_fields(ce[first], level)
            x_u[udir] = 0.0
            kl = torch.empty(E, dtype=torch.float64, device="cuda")
            B.hhg_scatter_unique(h, level, B.F64, 1, torch.as_tensor(k_u, dtype=torch.float64, device="cuda"), kl)
            B.hhg_set_coefficient(h, kl, B.F64)
            B.hhg_mg_setup(h)
            xs = torch.as_tensor(np.ascontiguousarray(x_u.T).reshape(-1), dtype=torch.float64, device="cuda")
            x64 = torch.empty(3 * E, dtype=torch.float64, device="cuda")
            B.hhg_scatter_unique(h, level, B.F64, 3, xs, x64)
            f64 = 0.5 * x64
            bufs = {B.F64: (x64, f64, torch.empty_like(x64)), B.F32: (x64.float(), f64.float(), None)}
            bufs[B.F32] = bufs[B.F32][:2] + (torch.empty_like(bufs[B.F32][0]),)

            def timed(call):
                for _ in range(2):
                    call()
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(reps)]
                for q, (a, b) in enumerate(ev):
                    flush.fill_(float(q))
                    a.record(stream)
                    call()
                    b.record(stream)
                torch.cuda.synchronize()
                return statistics.median(a.elapsed_time(b) for a, b in ev)

            def row(kind, dt, ms):
                w = 8 if dt == B.F64 else 4
                byts = SWEEP_BYTES[(kind, w)]
                gbs = byts * U / (ms * 1e-3) / 1e9
                out["rows"].append({"level": level, "kernel": kind, "dtype": "f64" if w == 8 else "f32",
                                    "ms": round(ms, 5), "gdofs": round(3 * U / (ms * 1e-3) / 1e9, 3),
                                    "bytes_per_node": byts, "gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm_peak, 4)})

            for dt in (B.F64, B.F32):
                x, f, y = bufs[dt]
                row("apply", dt, timed(lambda: B.hhg_apply(h, level, dt, x, y)))
                row("residual", dt, timed(lambda: B.hhg_residual(h, level, dt, f, x, y)))
                for kind, sm in (("jacobi", B.SMOOTH_JACOBI), ("chebyshev", B.SMOOTH_CHEBYSHEV)):
                    B.hhg_set_mg_params(h, smoother=sm)
                    y.copy_(x)
                    row(kind, dt, timed(lambda: B.hhg_smooth(h, level, dt, 1, f, y)))
                B.hhg_set_mg_params(h)
            # the other macro-interior kernels on the same sweeps: the shared-memory tile kernel
            # (1), the point kernels with one launch per macro (2) and with one launch for all (3)
            for kern, name in ((1, "apply_tile_kernel"), (2, "apply_per_macro_launches"), (3, "apply_one_launch")):
                B.hhg_set_interior_kernel(h, kern)
                for dt in (B.F64, B.F32):
                    x, f, y = bufs[dt]
                    row(name, dt, timed(lambda: B.hhg_apply(h, level, dt, x, y)))
            B.hhg_set_interior_kernel(h, 0)
            x, f, y = bufs[B.F32]
            B.hhg_set_coefficient(h, kl.to(torch.bfloat16).view(torch.int16), B.BF16)
            row("apply_bf16_k", B.F32, timed(lambda: B.hhg_apply(h, level, B.F32, x, y)))
        finally:
            B.hhg_destroy(h)
    return out


def stokes_bench(B, torch, level, dev, stream, steps=20):
    """Stokes with variable viscosity (Sec. 5.2) on the same cube and level: mu = 1 inside a
    sphere of radius 0.25 around the centre and 1e3 outside (tanh blend of width 0.02), body
    force i.i.d. uniform[-1, 1] (seed 4).  FP32 saddle-operator apply throughput (4 DoFs per
    node, L2 flushed before each apply) and the time to an FP64 relative residual of 1e-8
    with FP64 iterative refinement around FP32 block-preconditioned MINRES."""
    import hhg_inputs as hi

    xyz, tets = hi.kuhn_cube(1)
    h = B.hhg_create(dev, stream.cuda_stream)
    try:
        B.hhg_set_macro_mesh(h, xyz, tets)
        B.hhg_refine(h, level)
        B.hhg_set_problem(h, kind=B.STOKES)
        E, U, _ = B.hhg_num_nodes(h, level)
        ce = B.hhg_entry_coords(h, level)
        e2u, udir = B.hhg_entry_to_unique(h, level)
        first = np.full(U, -1, dtype=np.int64)
        first[e2u[::-1]] = np.arange(E)[::-1]
        cu = ce[first]
        mu = hi.viscosity_sphere(cu)
        mul = torch.empty(E, dtype=torch.float64, device="cuda")
        B.hhg_scatter_unique(h, level, B.F64, 1, torch.as_tensor(mu, device="cuda"), mul)
        B.hhg_set_coefficient(h, mul, B.F64)
        fu = hi.sample_grid(hi.uniform_grid(1 << level, seed=4), cu)
        fu[udir] = 0.0
        src = np.zeros((4, U))
        src[:3] = fu.T
        f = torch.empty(4 * E, dtype=torch.float64, device="cuda")
        B.hhg_scatter_unique(h, level, B.F64, 4, torch.as_tensor(src.reshape(-1), device="cuda"), f)
        x32 = f.float()
        y32 = torch.empty_like(x32)
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        for _ in range(3):
            B.hhg_stokes_apply(h, level, B.F32, x32, y32)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            flush.fill_(1.0)
            a.record(stream)
            B.hhg_stokes_apply(h, level, B.F32, x32, y32)
            b.record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        B.hhg_mg_setup(h)
        out = {"workload": "Stokes, 6-macro cube, level %d, viscosity sphere 1 / 1e3, f ~ U[-1,1] (seed 4)" % level,
               "apply_ms": round(ms, 5), "apply_gdofs": round(4 * U / (ms * 1e-3) / 1e9, 3)}
        for name, method, inner in (("ir_minres", B.SOLVE_STOKES_IR_MINRES, 400),
                                    ("ir_uzawa_mg", B.SOLVE_STOKES_IR_UZAWA, 40),
                                    ("ir_fgcr_uzawa_mg", B.SOLVE_STOKES_IR_FGCR, 60)):
            x = torch.zeros_like(f)
            rep = B.hhg_solve(h, f, x, method=method, level=level, dt=B.F64, rtol=1e-8, max_iter=30,
                              inner_rtol=1e-3, inner_max_iter=inner, allow_not_converged=True)
            out[name] = {k: (float("%.4g" % v) if isinstance(v, float) else v) for k, v in rep.items()}
        # the paper's solver settings (Sec. 5.2.1): hybrid Gauss-Seidel velocity smoothing, one
        # step per Uzawa step, pressure relaxation 0.3, variable V(3,3) cycles with two more steps
        # per coarser level
        B.hhg_set_mg_params(h, smoother=B.SMOOTH_HYBRID_GS, uzawa_pre=3, uzawa_post=3, uzawa_extra=2,
                            uzawa_vsteps=1, uzawa_omega=0.3)
        for name, method, inner in (("ir_uzawa_mg_hybrid_gs", B.SOLVE_STOKES_IR_UZAWA, 40),
                                    ("ir_fgcr_uzawa_mg_hybrid_gs", B.SOLVE_STOKES_IR_FGCR, 60)):
            x = torch.zeros_like(f)
            rep = B.hhg_solve(h, f, x, method=method, level=level, dt=B.F64, rtol=1e-8, max_iter=30,
                              inner_rtol=1e-3, inner_max_iter=inner, allow_not_converged=True)
            out[name] = {k: (float("%.4g" % v) if isinstance(v, float) else v) for k, v in rep.items()}
        B.hhg_set_mg_params(h)
        return out
    finally:
        B.hhg_destroy(h)


def elastostatics_bench(B, torch, level, m, dev, stream):
    """The linear elastostatics benchmark setup of Sec. 5.1.2: the unit cube as 384 macro
    tetrahedra (4 x 4 x 4 cubes of 6 Kuhn tetrahedra), E = cos(m pi x y z) + 2, nu = 0.34,
    Dirichlet data u* on the whole boundary, solved from the boundary values (interior 0) to a
    relative residual of 1e-8 by stationary V(3,3) cycles with the hybrid Gauss-Seidel smoother
    and an exact solve on the coarsest level 0 (the macro mesh), in FP64 as in the paper.  The
    right-hand side is A I_h u* on the free rows (the discrete solution is then I_h u*; the
    paper uses the consistent load of -div sigma(u*), which the library does not assemble),
    so the error column reports how closely the solve reaches I_h u*."""
    import hhg_inputs as hi

    xyz, tets = hi.kuhn_cube(4)
    h = B.hhg_create(dev, stream.cuda_stream)
    try:
        B.hhg_set_macro_mesh(h, xyz, tets)
        B.hhg_set_coarsest_level(h, 0)
        B.hhg_refine(h, level)
        B.hhg_set_problem(h, nu=0.34)
        E, U, _ = B.hhg_num_nodes(h, level)
        ce = B.hhg_entry_coords(h, level)
        e2u, udir = B.hhg_entry_to_unique(h, level)
        first = np.full(U, -1, dtype=np.int64)
        first[e2u[::-1]] = np.arange(E)[::-1]
        cu = ce[first]
        kl = torch.empty(E, dtype=torch.float64, device="cuda")
        B.hhg_scatter_unique(h, level, B.F64, 1, torch.as_tensor(hi.young_cos(cu, m), device="cuda"), kl)
        B.hhg_set_coefficient(h, kl, B.F64)
        us = hi.u_star(cu)
        u = torch.empty(3 * E, dtype=torch.float64, device="cuda")
        B.hhg_scatter_unique(h, level, B.F64, 3, torch.as_tensor(np.ascontiguousarray(us.T).reshape(-1),
                                                                  device="cuda"), u)
        f = torch.empty_like(u)
        B.hhg_apply(h, level, B.F64, u, f)  # free rows: A I_h u*; Dirichlet rows: u*
        x0s = us * udir[:, None]
        x0 = torch.empty_like(u)
        B.hhg_scatter_unique(h, level, B.F64, 3, torch.as_tensor(np.ascontiguousarray(x0s.T).reshape(-1),
                                                                  device="cuda"), x0)
        out = {"workload": "elastostatics benchmark setup (Sec. 5.1.2), 384-macro cube, level %d (%d free DoFs), "
                           "m = %d, nu = 0.34, coarsest level 0" % (level, 3 * int((~udir).sum()), m),
               "paper": "32 V(3,3) cycles at this level and m = 1 (1 core of SuperMUC-NG: 1125 s at level 6, "
                        "143 s at level 5)"}
        B.hhg_set_mg_params(h, smoother=B.SMOOTH_HYBRID_GS, pre=3, post=3)
        B.hhg_mg_setup(h)
        h3 = (1.0 / (4 << level)) ** 3
        for name, method, kw in (("fp64_mg_v33_hybrid_gs", B.SOLVE_MG, {}),
                                 ("ir_fp64_over_fp32_mgcg_v33_hybrid_gs", B.SOLVE_IR_MG_CG,
                                  dict(inner_rtol=1e-3, inner_max_iter=50))):
            x = x0.clone()
            torch.cuda.synchronize()
            rep = B.hhg_solve(h, f, x, method=method, level=level, dt=B.F64, rtol=1e-8, max_iter=200,
                              allow_not_converged=True, **kw)
            xu = torch.empty(3 * U, dtype=torch.float64, device="cuda")
            B.hhg_gather_unique(h, level, B.F64, 3, x, xu)
            err = xu.cpu().numpy().reshape(3, U).T - us
            out[name] = {"seconds": round(rep["seconds"], 4), "iterations": rep["iterations"],
                         "inner_iterations": rep["inner_iterations"], "rel_residual": float("%.4g" % rep["rel_residual"]),
                         "converged": bool(rep["converged"]),
                         "l2_error_vs_interpolant": float("%.4g" % np.sqrt(h3 * (err**2).sum()))}
        return out
    finally:
        B.hhg_destroy(h)


def foam_bench(B, torch, level, dev, stream):
    """The boundary conditions of the foam block of Sec. 5.1.3: the box (0,4) x (0,2) x (0,1) as
    48 macro tetrahedra, clamped at z = 0, traction (0, 0, -1) on the top plane z = 1
    (`hhg_traction_load`), the other faces traction-free, nu = 0.3; the CT-derived modulus is
    replaced by a Schwarz-P open-cell field (E = 1 in the struts, 1e-2 in the pores).  At level 7
    the free DoFs (5.06e7) match the paper's 5.05e7.  FP64 V(3,3) hybrid Gauss-Seidel cycles
    (the paper: 19 V-cycles) and FP64 refinement around FP32 MG-CG with the same cycle."""
    import hhg_inputs as hi

    xyz, tets = hi.kuhn_box(4, 2, 1)
    dflags = np.zeros((len(tets), 4), dtype=np.int32)
    tflags = np.zeros_like(dflags)
    for m, t in enumerate(tets):
        for f in range(4):
            z = xyz[[int(t[q]) for q in range(4) if q != f], 2]
            dflags[m, f] = np.all(z == 0.0)
            tflags[m, f] = np.all(z == 1.0)
    h = B.hhg_create(dev, stream.cuda_stream)
    try:
        B.hhg_set_macro_mesh(h, xyz, tets, dflags)
        B.hhg_refine(h, level)
        B.hhg_set_problem(h, nu=0.3)
        E, U, _ = B.hhg_num_nodes(h, level)
        ce = B.hhg_entry_coords(h, level)
        e2u, udir = B.hhg_entry_to_unique(h, level)
        first = np.full(U, -1, dtype=np.int64)
        first[e2u[::-1]] = np.arange(E)[::-1]
        cu = ce[first]
        kl = torch.empty(E, dtype=torch.float64, device="cuda")
        B.hhg_scatter_unique(h, level, B.F64, 1, torch.as_tensor(hi.foam_modulus(cu), device="cuda"), kl)
        B.hhg_set_coefficient(h, kl, B.F64)
        tr = np.zeros((3, U))
        tr[2] = -1.0
        t = torch.empty(3 * E, dtype=torch.float64, device="cuda")
        B.hhg_scatter_unique(h, level, B.F64, 3, torch.as_tensor(tr.reshape(-1), device="cuda"), t)
        f = torch.zeros_like(t)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.hhg_traction_load(h, level, B.F64, tflags, t, f)
        load_s = time.perf_counter() - t0
        out = {"workload": "foam block boundary conditions (Sec. 5.1.3), 48 macros, level %d (%d free DoFs), "
                           "Schwarz-P modulus stand-in" % (level, 3 * int((~udir).sum())),
               "traction_load_s": round(load_s, 4),
               "paper": "19 V-cycles (48 cores of SuperMUC-NG: 19.2 s physical scaling)"}
        B.hhg_set_mg_params(h, smoother=B.SMOOTH_HYBRID_GS, pre=3, post=3)
        B.hhg_mg_setup(h)
        for name, method, kw in (("fp64_mg_v33_hybrid_gs", B.SOLVE_MG, {}),
                                 ("ir_fp64_over_fp32_mgcg_v33_hybrid_gs", B.SOLVE_IR_MG_CG,
                                  dict(inner_rtol=1e-3, inner_max_iter=50))):
            x = torch.zeros_like(f)
            torch.cuda.synchronize()
            # the stationary cycles diverge on this field (capped at 20); MG-CG converges
            rep = B.hhg_solve(h, f, x, method=method, level=level, dt=B.F64, rtol=1e-8,
                              max_iter=20 if method == B.SOLVE_MG else 60, allow_not_converged=True, **kw)
            out[name] = {k: (float("%.4g" % v) if isinstance(v, float) else v) for k, v in rep.items()}
        xu = torch.empty(3 * U, dtype=torch.float64, device="cuda")
        B.hhg_gather_unique(h, level, B.F64, 3, x, xu)
        out["max_downward_displacement"] = float("%.4g" % -xu[2 * U:].min().item())
        return out
    finally:
        B.hhg_destroy(h)


def twod_bench(B, torch, level, dev, stream, steps=20):
    """The 2D variant (Sec. 2.3) on one skewed macro triangle at 2^level intervals per edge:
    FP32 and FP64 physical-scaling and FP32 nodal-integration apply throughput (2 DoFs per point, L2 flushed before each
    call, median of the calls) and the algorithmic bytes per point (x 2, k 1 read; y 2 write)."""
    tri = np.array([[0.2, 0.1], [1.3, 0.4], [0.5, 1.7]])
    n = 1 << level
    N = (n + 1) * (n + 2) // 2
    h = B.hhg_create(dev, stream.cuda_stream)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    out = {"workload": "2D physical scaling, one macro triangle, %d intervals per edge (%d points)" % (n, N)}
    try:
        g = torch.Generator(device="cuda").manual_seed(5)
        for name, dt, tdt, size, var in (("f32", B.F32, torch.float32, 4, B.PHYSICAL),
                                         ("f64", B.F64, torch.float64, 8, B.PHYSICAL),
                                         ("f32_nodal", B.F32, torch.float32, 4, B.NODAL)):
            k = 1.0 + 0.5 * torch.rand(N, dtype=tdt, device="cuda", generator=g)
            x = torch.rand(2 * N, dtype=tdt, device="cuda", generator=g)
            y = torch.empty_like(x)
            for _ in range(3):
                B.hhg_apply_2d(h, tri, level, 0.3, var, dt, k, x, y)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for a, b in ev:
                flush.fill_(1.0)
                a.record(stream)
                B.hhg_apply_2d(h, tri, level, 0.3, var, dt, k, x, y)
                b.record(stream)
            torch.cuda.synchronize()
            ms = statistics.median(a.elapsed_time(b) for a, b in ev)
            bytes_pt = 5 * size
            out[name] = {"ms": round(ms, 5), "gdofs": round(2 * N / (ms * 1e-3) / 1e9, 3),
                         "bytes_per_point": bytes_pt, "gbs": round(bytes_pt * N / (ms * 1e-3) / 1e9, 1)}
        out["rel_time_physical_over_nodal_f32"] = round(out["f32"]["ms"] / out["f32_nodal"]["ms"], 4)
        return out
    finally:
        B.hhg_destroy(h)


def plume_bench(B, torch, level, dev, stream):
    """The stationary plume workload (Sec. 5.2.1) on the 384-macro cube (4 x 4 x 4 cubes of 6
    Kuhn tetrahedra each; macro faces on z = 3/4 carry the viscosity jump): mu = exp(-theta),
    times 1e-2 above z = 3/4, body force theta (0, 0, 10), no-slip walls.  Multigrid from the
    coarsest level 1 (the level-2 direct solve would be too large), the paper's smoother
    settings (hybrid Gauss-Seidel, pressure relaxation 0.3, variable V(3,3) + 2 per coarser
    level) inside flexible GCR (FP32) and FP64 refinement to an FP64 relative residual of 1e-8.
    With the 1e-2 jump the cycles diverge (the injected coarse viscosity at the plane z = 3/4
    over-corrects the pressure; the oracle's cycle does the same at small levels), so the line
    also reports the field without the jump."""
    import hhg_inputs as hi

    xyz, tets = hi.kuhn_cube(4)
    h = B.hhg_create(dev, stream.cuda_stream)
    try:
        B.hhg_set_macro_mesh(h, xyz, tets)
        B.hhg_set_coarsest_level(h, 1)
        B.hhg_refine(h, level)
        B.hhg_set_problem(h, kind=B.STOKES)
        E, U, _ = B.hhg_num_nodes(h, level)
        ce = B.hhg_entry_coords(h, level)
        e2u, udir = B.hhg_entry_to_unique(h, level)
        first = np.full(U, -1, dtype=np.int64)
        first[e2u[::-1]] = np.arange(E)[::-1]
        cu = ce[first]
        mul = torch.empty(E, dtype=torch.float64, device="cuda")
        src = np.zeros((4, U))
        fu = hi.plume_force(cu)
        fu[udir] = 0.0
        src[:3] = fu.T
        f = torch.empty(4 * E, dtype=torch.float64, device="cuda")
        B.hhg_scatter_unique(h, level, B.F64, 4, torch.as_tensor(src.reshape(-1), device="cuda"), f)
        B.hhg_set_mg_params(h, smoother=B.SMOOTH_HYBRID_GS, uzawa_pre=3, uzawa_post=3, uzawa_extra=2,
                            uzawa_vsteps=1, uzawa_omega=0.3)
        out = {"workload": "Stokes plume (Sec. 5.2.1), 384-macro cube, level %d (%d nodes, %d DoFs), coarsest "
                           "level 1" % (level, U, 4 * U), "macros": len(tets)}
        # the paper's viscosity, and the same without the factor 1e-2 above z = 3/4
        for field, mu in (("with_jump", hi.plume_viscosity(cu)), ("without_jump", np.exp(-hi.plume_temperature(cu)))):
            B.hhg_scatter_unique(h, level, B.F64, 1, torch.as_tensor(mu, device="cuda"), mul)
            B.hhg_set_coefficient(h, mul, B.F64)
            B.hhg_mg_setup(h)
            x = torch.zeros_like(f)
            try:
                # with the jump the cycles do not converge: two refinement steps (120 cycles) show it
                rep = B.hhg_solve(h, f, x, method=B.SOLVE_STOKES_IR_FGCR, level=level, dt=B.F64, rtol=1e-8,
                                  max_iter=2 if field == "with_jump" else 30, inner_rtol=1e-3, inner_max_iter=60,
                                  allow_not_converged=True)
                out["ir_fgcr_uzawa_mg_hybrid_gs_" + field] = {
                    k: (float("%.4g" % v) if isinstance(v, float) else v) for k, v in rep.items()}
            except B.HhgError as e:
                out["ir_fgcr_uzawa_mg_hybrid_gs_" + field] = {"error": str(e)}
        return out
    finally:
        B.hhg_destroy(h)


def carreau_bench(B, torch, level, dev, stream):
    """Generalised Newtonian Stokes (Sec. 5.2.2): Carreau law with n = 0.5, eta0 = 1,
    eta_inf = 1e-3, lambda = 1 (kappa = lambda^2, r = (n-1)/2), lid-driven cavity on the
    6-macro cube; Picard iterations (Alg. 1) with the FP64 viscosity update."""
    import hhg_inputs as hi

    xyz, tets = hi.kuhn_cube(1)
    h = B.hhg_create(dev, stream.cuda_stream)
    try:
        B.hhg_set_macro_mesh(h, xyz, tets)
        B.hhg_refine(h, level)
        B.hhg_set_problem(h, kind=B.STOKES)
        E, U, _ = B.hhg_num_nodes(h, level)
        ce = B.hhg_entry_coords(h, level)
        e2u, _ = B.hhg_entry_to_unique(h, level)
        first = np.full(U, -1, dtype=np.int64)
        first[e2u[::-1]] = np.arange(E)[::-1]
        cu = ce[first]
        one = torch.ones(E, dtype=torch.float64, device="cuda")
        B.hhg_set_coefficient(h, one, B.F64)
        x0 = np.zeros((4, U))
        x0[:3] = hi.lid_velocity(cu).T
        x = torch.empty(4 * E, dtype=torch.float64, device="cuda")
        B.hhg_scatter_unique(h, level, B.F64, 4, torch.as_tensor(x0.reshape(-1), device="cuda"), x)
        f = torch.zeros_like(x)
        torch.cuda.synchronize()
        rep = B.hhg_picard(h, f, x, level, eta0=1.0, eta_inf=1e-3, kappa=1.0, r=-0.25, picard_tol=1e-3,
                           max_picard=40, step_rtol=1e-2, step_max_iter=100, final_rtol=1e-3,
                           allow_not_converged=True)
        return {"workload": "Carreau Stokes (n=0.5, eta0=1, eta_inf=1e-3, lambda=1), lid-driven 6-macro cube, "
                            "level %d (%d nodes)" % (level, U),
                "picard": {k: (float("%.4g" % v) if isinstance(v, float) else v) for k, v in rep.items()}}
    finally:
        B.hhg_destroy(h)


# ---------------------------------------------------------------------------- our arm


def learned_bench(B, torch, dev, stream, train_level, eval_level, nseed, nrhs, iters, steps, coarsen=0,
                  coarse_train_level=7, coarse_seeds=12):
    """Learned preconditioner: training pairs from the errors of MG-preconditioned CG
    solves at train_level (lognormal E with seeds 100.., f ~ U[-1, 1]), GPU training of the
    conv net (Adam, batches of 8 random 32^3 crops), then the time to an FP64 relative
    residual of 1e-8 at eval_level on the bench field (seed 2, f seed 3): FP64 refinement
    around FP32 flexible CG with the V-cycle plus the learned correction, against the same
    solver with the V-cycle alone and plain FP64 MG-CG.  Also the conv-net forward
    throughput on the eval grid (tensor-core roofline of the dominant learned kernel).
    With coarsen = q > 0 also the coarse-grid mode: the network trained on pairs from
    coarse_train_level stored q levels lower, and applied q levels below eval_level."""
    import hhg_inputs as hi

    xyz, tets = hi.kuhn_cube(1)

    def make(level):
        h = B.hhg_create(dev, stream.cuda_stream)
        B.hhg_set_macro_mesh(h, xyz, tets)
        B.hhg_refine(h, level)
        B.hhg_set_problem(h, nu=NU)
        E, U, _ = B.hhg_num_nodes(h, level)
        ce = B.hhg_entry_coords(h, level)
        e2u, udir = B.hhg_entry_to_unique(h, level)
        first = np.full(U, -1, dtype=np.int64)
        first[e2u[::-1]] = np.arange(E)[::-1]
        return h, E, U, ce[first], udir

    def scatter(h, level, u, comps, dt):
        tdt = torch.float64 if dt == B.F64 else torch.float32
        src = torch.as_tensor(np.ascontiguousarray(np.asarray(u).reshape(-1, comps).T).reshape(-1), dtype=tdt,
                              device="cuda")
        E = B.hhg_num_nodes(h, level)[0]
        dst = torch.empty(comps * E, dtype=tdt, device="cuda")
        B.hhg_scatter_unique(h, level, dt, comps, src, dst)
        return dst

    def train(level, seeds, q, crop):
        """Pairs from MG-CG errors on `seeds` lognormal fields at `level` (stored q levels
        lower), GPU training; returns (parameters, report, pair-generation seconds)."""
        h, E, U, cu, udir = make(level)
        Nt = 1 << level
        B.hhg_learn_set_coarsening(h, q)
        B.hhg_learn_reserve_pairs(h, level, seeds * nrhs * iters)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in range(seeds):
            B.hhg_set_coefficient(h, scatter(h, level, hi.sample_grid(hi.lognormal_grid(Nt, 100 + s), cu), 1, B.F64),
                                  B.F64)
            B.hhg_mg_setup(h)
            for q2 in range(nrhs):
                f = np.random.default_rng(1000 * s + q2).uniform(-1, 1, size=(U, 3))
                f[udir] = 0.0
                B.hhg_learn_collect_cg(h, level, scatter(h, level, f, 3, B.F32), iters)
        torch.cuda.synchronize()
        gen_s = time.perf_counter() - t0
        B.hhg_learn_init(h, 1)
        tr = B.hhg_learn_train(h, steps=steps, batch=8, crop=crop, lr=2e-3, seed=2)
        params = B.hhg_learn_get_params(h)
        B.hhg_destroy(h)
        return params, tr, gen_s

    # training pairs and training
    params, tr, gen_s = train(train_level, nseed, 0, 32)

    # evaluation
    h, E, U, cu, udir = make(eval_level)
    N = 1 << eval_level
    B.hhg_set_coefficient(h, scatter(h, eval_level, hi.sample_grid(hi.lognormal_grid(N, 2), cu), 1, B.F64), B.F64)
    B.hhg_mg_setup(h)
    B.hhg_learn_set_params(h, params)
    f = scatter(h, eval_level, hi.sample_grid(hi.uniform_grid(N, seed=3), cu), 3, B.F64)
    out = {"train": {"level": train_level, "coefficient_seeds": "%d..%d" % (100, 100 + nseed - 1),
                     "pairs": int(tr["pairs"]), "pair_source": "errors of %d MG-CG iterations x %d RHS per field"
                     % (iters, nrhs), "pair_generation_s": round(gen_s, 3), "steps": steps, "batch": "8 x 32^3",
                     "loss_first": tr["loss_first"], "loss_last": tr["loss_last"],
                     "train_s": round(tr["seconds"], 3)},
           "eval_level": eval_level, "rtol": 1e-8}
    for name, method, kw in (("ir_fcg_learned", B.SOLVE_IR_FCG_LEARNED, dict(inner_rtol=1e-3, inner_max_iter=100)),
                             ("ir_fcg_vcycle", B.SOLVE_IR_FCG, dict(inner_rtol=1e-3, inner_max_iter=100)),
                             ("fp64_mgcg", B.SOLVE_MG_CG, {})):
        best = None
        for _ in range(2):
            x = torch.zeros_like(f)
            B.hhg_learn_stats(h, reset=True)
            torch.cuda.synchronize()
            rep = B.hhg_solve(h, f, x, method=method, level=eval_level, dt=B.F64, rtol=1e-8, max_iter=100, **kw)
            st = B.hhg_learn_stats(h)
            if best is None or rep["seconds"] < best[0]["seconds"]:
                best = (rep, st)
        rep, st = best
        r = torch.empty_like(f)
        r2 = B.hhg_residual(h, eval_level, B.F64, f, x, r, want_norm=True)
        out[name] = {"seconds": round(rep["seconds"], 5), "iterations": rep["iterations"],
                     "inner_iterations": rep["inner_iterations"],
                     "rel_residual_fp64": float(np.sqrt(r2)) / rep["residual0"], "converged": bool(rep["converged"])}
        if method == B.SOLVE_IR_FCG_LEARNED:
            out[name].update({"net_applications": st["applications"], "fallbacks": st["fallbacks"],
                              "mean_weight_b_over_a": round(st["alpha_mean"], 4),
                              "mean_extra_energy_reduction": round(st["gain_mean"], 5)})
    out["iterations_saved_vs_vcycle"] = out["ir_fcg_vcycle"]["inner_iterations"] - out["ir_fcg_learned"]["inner_iterations"]
    out["speedup_learned_vs_fp64_mgcg"] = round(out["fp64_mgcg"]["seconds"] / out["ir_fcg_learned"]["seconds"], 3)
    if coarsen > 0:
        # coarse-grid mode: the network on the node grid `coarsen` levels below the solve's
        cp, ctr, cgen = train(coarse_train_level, coarse_seeds, coarsen, 32)
        B.hhg_learn_set_params(h, cp)
        B.hhg_learn_set_coarsening(h, coarsen)
        best = None
        for _ in range(2):
            x = torch.zeros_like(f)
            B.hhg_learn_stats(h, reset=True)
            torch.cuda.synchronize()
            rep = B.hhg_solve(h, f, x, method=B.SOLVE_IR_FCG_LEARNED, level=eval_level, dt=B.F64, rtol=1e-8,
                              max_iter=100, inner_rtol=1e-3, inner_max_iter=100)
            st = B.hhg_learn_stats(h)
            if best is None or rep["seconds"] < best[0]["seconds"]:
                best = (rep, st)
        rep, st = best
        B.hhg_learn_set_coarsening(h, 0)
        B.hhg_learn_set_params(h, params)
        out["ir_fcg_learned_coarse"] = {
            "coarsen": coarsen, "network_level": eval_level - coarsen,
            "train": {"level": coarse_train_level, "pair_grid_level": coarse_train_level - coarsen,
                      "pairs": int(ctr["pairs"]), "pair_generation_s": round(cgen, 3),
                      "loss_first": ctr["loss_first"], "loss_last": ctr["loss_last"]},
            "seconds": round(rep["seconds"], 5), "iterations": rep["iterations"],
            "inner_iterations": rep["inner_iterations"], "converged": bool(rep["converged"]),
            "net_applications": st["applications"], "fallbacks": st["fallbacks"],
            "mean_extra_energy_reduction": round(st["gain_mean"], 5),
            "iterations_saved_vs_vcycle": out["ir_fcg_vcycle"]["inner_iterations"] - rep["inner_iterations"]}
    # conv-net forward throughput on the eval grid (4 layers, 27 taps, 16 x 16 channels)
    (D, H, W), _ = B.hhg_learn_grid(h, eval_level)
    V = D * H * W
    xin = torch.randn(V * 7, device="cuda")
    yo = torch.empty(V * 3, device="cuda")
    for _ in range(3):
        B.hhg_learn_forward(h, xin, 7, 1, D, H, W, yo)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    reps = 10
    for _ in range(reps):
        B.hhg_learn_forward(h, xin, 7, 1, D, H, W, yo)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    # the same forward pass on the tcgen05 kernel
    B.hhg_learn_set_conv_kernel(h, 1)
    for _ in range(3):
        B.hhg_learn_forward(h, xin, 7, 1, D, H, W, yo)
    a.record(stream)
    for _ in range(reps):
        B.hhg_learn_forward(h, xin, 7, 1, D, H, W, yo)
    b.record(stream)
    torch.cuda.synchronize()
    ms_u = a.elapsed_time(b) / reps
    B.hhg_learn_set_conv_kernel(h, 2)
    for _ in range(3):
        B.hhg_learn_forward(h, xin, 7, 1, D, H, W, yo)
    a.record(stream)
    for _ in range(reps):
        B.hhg_learn_forward(h, xin, 7, 1, D, H, W, yo)
    b.record(stream)
    torch.cuda.synchronize()
    ms_p = a.elapsed_time(b) / reps
    B.hhg_learn_set_conv_kernel(h, 0)
    flops = V * 4 * 27 * 16 * 16 * 2
    peak = None
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        peak = float(json.load(open(pp))["bf16_tflops"])
        src = "measured (cuBLAS bf16 burst)"
    else:
        peak, src = 1900.0, "fallback"
    tf = flops / (ms * 1e-3) / 1e12
    out["conv_forward"] = {"grid": [D, H, W], "ms": round(ms, 4), "tflops": round(tf, 2), "peak_tflops": peak,
                           "frac": round(tf / peak, 4), "peak_source": src,
                           "kernel": "k_conv (mma.sync m16n8k16 BF16, FP32 accumulate), 4 launches",
                           "tcgen05": {"ms": round(ms_u, 4), "tflops": round(flops / (ms_u * 1e-3) / 1e12, 2),
                                       "frac": round(flops / (ms_u * 1e-3) / 1e12 / peak, 4),
                                       "kernel": "k_conv_umma (tcgen05.mma kind::f16, TMEM accumulators)"},
                           "tma_tcgen05": {"ms": round(ms_p, 4), "tflops": round(flops / (ms_p * 1e-3) / 1e12, 2),
                                           "frac": round(flops / (ms_p * 1e-3) / 1e12 / peak, 4),
                                           "kernel": "k_conv_tma (TMA loads, tcgen05.mma, TMEM double buffer)"}}
    B.hhg_destroy(h)
    return out


def learned_stokes_bench(B, torch, dev, stream, train_level, eval_level, nfield, nrhs, iters, steps):
    """Learned preconditioner for Stokes: training pairs from the errors of flexible GCR
    with the inexact Uzawa V-cycle at train_level (viscosity 1 inside / 1e3 outside a sphere
    of seeded centre in [0.35, 0.65]^3 and radius in [0.15, 0.3], tanh width 0.02; body
    force U[-1, 1] per seed), GPU training (4 output channels: velocity and pressure),
    then the time to an FP64 relative residual of 1e-8 at eval_level on the Stokes bench
    workload (sphere at the centre, radius 0.25; f seed 4): FP64 refinement around FP32
    flexible GCR with the Uzawa V-cycle plus the learned correction, against the same
    solver with the V-cycle alone."""
    import hhg_inputs as hi

    xyz, tets = hi.kuhn_cube(1)

    def make(level):
        h = B.hhg_create(dev, stream.cuda_stream)
        B.hhg_set_macro_mesh(h, xyz, tets)
        B.hhg_refine(h, level)
        B.hhg_set_problem(h, kind=B.STOKES)
        E, U, _ = B.hhg_num_nodes(h, level)
        ce = B.hhg_entry_coords(h, level)
        e2u, udir = B.hhg_entry_to_unique(h, level)
        first = np.full(U, -1, dtype=np.int64)
        first[e2u[::-1]] = np.arange(E)[::-1]
        return h, E, U, ce[first], udir

    def scatter(h, level, u, comps, dt):
        tdt = torch.float64 if dt == B.F64 else torch.float32
        src = torch.as_tensor(np.ascontiguousarray(np.asarray(u).reshape(-1, comps).T).reshape(-1), dtype=tdt,
                              device="cuda")
        E = B.hhg_num_nodes(h, level)[0]
        dst = torch.empty(comps * E, dtype=tdt, device="cuda")
        B.hhg_scatter_unique(h, level, dt, comps, src, dst)
        return dst

    h, E, U, cu, udir = make(train_level)
    B.hhg_learn_reserve_pairs(h, train_level, nfield * nrhs * iters)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(nfield):
        rng = np.random.default_rng(500 + s)
        ctr = rng.uniform(0.35, 0.65, size=3)
        rad = rng.uniform(0.15, 0.3)
        mu = hi.viscosity_sphere(cu - (ctr - 0.5), radius=rad)
        B.hhg_set_coefficient(h, scatter(h, train_level, mu, 1, B.F64), B.F64)
        B.hhg_mg_setup(h)
        for q in range(nrhs):
            f = np.zeros((U, 4))
            f[:, :3] = rng.uniform(-1, 1, size=(U, 3))
            f[udir, :3] = 0.0
            B.hhg_learn_collect_cg(h, train_level, scatter(h, train_level, f, 4, B.F32), iters)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    # per-channel RMS of the inputs and targets over the stored pairs (every 6th pair)
    dims, _ = B.hhg_learn_grid(h, train_level)
    xs, ts = [], []
    for j in range(0, nfield * nrhs * iters, 6):
        xp, tp = B.hhg_learn_get_pair(h, j, dims, nc=4)
        xs.append(np.sqrt((xp.reshape(-1, 9).astype(np.float64) ** 2).mean(axis=0)))
        ts.append(np.sqrt((tp.reshape(-1, 4).astype(np.float64) ** 2).mean(axis=0)))
    B.hhg_learn_init(h, 1)
    tr = B.hhg_learn_train(h, steps=steps, batch=8, crop=32, lr=2e-3, seed=2)
    params = B.hhg_learn_get_params(h)
    B.hhg_destroy(h)

    h, E, U, cu, udir = make(eval_level)
    try:
        B.hhg_set_coefficient(h, scatter(h, eval_level, hi.viscosity_sphere(cu), 1, B.F64), B.F64)
        B.hhg_mg_setup(h)
        B.hhg_learn_set_params(h, params)
        fu = hi.sample_grid(hi.uniform_grid(1 << eval_level, seed=4), cu)
        fu[udir] = 0.0
        f4 = np.zeros((U, 4))
        f4[:, :3] = fu
        f = scatter(h, eval_level, f4, 4, B.F64)
        out = {"train": {"level": train_level, "fields": nfield, "pairs": int(tr["pairs"]),
                         "pair_source": "errors of %d FGCR iterations x %d RHS per field" % (iters, nrhs),
                         "pair_generation_s": round(gen_s, 3), "steps": steps, "batch": "8 x 32^3",
                         "loss_first": tr["loss_first"], "loss_last": tr["loss_last"],
                         "train_s": round(tr["seconds"], 3),
                         "input_rms_per_channel": [round(float(v), 4) for v in np.mean(xs, axis=0)],
                         "target_rms_per_channel": [round(float(v), 4) for v in np.mean(ts, axis=0)]},
               "eval_level": eval_level, "rtol": 1e-8,
               "workload": "Stokes, 6-macro cube, level %d, viscosity sphere 1 / 1e3, f ~ U[-1,1] (seed 4)"
                           % eval_level}
        for name, method in (("ir_fgcr_learned", B.SOLVE_STOKES_IR_FGCR_LEARNED),
                             ("ir_fgcr_uzawa", B.SOLVE_STOKES_IR_FGCR)):
            x = torch.zeros_like(f)
            B.hhg_learn_stats(h, reset=True)
            torch.cuda.synchronize()
            rep = B.hhg_solve(h, f, x, method=method, level=eval_level, dt=B.F64, rtol=1e-8, max_iter=30,
                              inner_rtol=1e-3, inner_max_iter=60, allow_not_converged=True)
            st = B.hhg_learn_stats(h)
            out[name] = {"seconds": round(rep["seconds"], 5), "iterations": rep["iterations"],
                         "inner_iterations": rep["inner_iterations"],
                         "rel_residual": float("%.4g" % rep["rel_residual"]), "converged": bool(rep["converged"])}
            if method == B.SOLVE_STOKES_IR_FGCR_LEARNED:
                out[name].update({"net_applications": st["applications"], "fallbacks": st["fallbacks"],
                                  "mean_weight_b_over_a": round(st["alpha_mean"], 4),
                                  "mean_extra_residual_reduction": round(st["gain_mean"], 5)})
        out["iterations_saved_vs_vcycle"] = (out["ir_fgcr_uzawa"]["inner_iterations"] -
                                             out["ir_fgcr_learned"]["inner_iterations"])
        return out
    finally:
        B.hhg_destroy(h)


def run_ours(args):
    import torch

    from paper_1908_08666_gb300 import binding as B
    import hhg_inputs as hi

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()
    level = args.level
    xyz, tets = hi.kuhn_cube(1)
    h = B.hhg_create(dev, stream.cuda_stream)
    B.hhg_set_macro_mesh(h, xyz, tets)
    B.hhg_refine(h, level)
    B.hhg_set_problem(h, nu=NU)
    E, U, F = B.hhg_num_nodes(h, level)
    coords_e = B.hhg_entry_coords(h, level)
    e2u, _ = B.hhg_entry_to_unique(h, level)
    first = np.full(U, -1, dtype=np.int64)
    first[e2u[::-1]] = np.arange(E)[::-1]
    k_u, x_u = workload_fields(coords_e[first], level)
    ku = torch.as_tensor(k_u, dtype=torch.float64, device="cuda")
    kl = torch.empty(E, dtype=torch.float64, device="cuda")
    B.hhg_scatter_unique(h, level, B.F64, 1, ku, kl)
    B.hhg_set_coefficient(h, kl, B.F64)
    xu = torch.as_tensor(np.ascontiguousarray(x_u.T).reshape(-1), dtype=torch.float32, device="cuda")
    x = torch.empty(3 * E, dtype=torch.float32, device="cuda")
    B.hhg_scatter_unique(h, level, B.F32, 3, xu, x)
    y = torch.empty_like(x)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > 2x L2
    n = 1 << level
    nmacro = tets.shape[0]
    interior_per_macro = (n - 1) * (n - 2) * (n - 3) // 6
    dofs = 3 * U

    for _ in range(max(3, args.warmup)):
        B.hhg_apply(h, level, B.F32, x, y)
    torch.cuda.synchronize()
    alu_peak, alu_probe, sm_count = fp32_peak(B, torch, h, stream)

    clocks = Clocks(dev)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    B.hhg_profile(h, 1)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for s in range(args.steps):
        flush.fill_(float(s))
        starts[s].record(stream)
        B.hhg_apply(h, level, B.F32, x, y)
        ends[s].record(stream)
    torch.cuda.synchronize()
    prof_ms, prof_launches = B.hhg_profile(h, 0, read=True)
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    total_ms = max_over_ranks(float(sum(step_ms)), world)
    median_ms = statistics.median(step_ms)
    # end-to-end: host buffers through the C ABI (H2D copy, apply, D2H copy, wait)
    xh = torch.empty(3 * E, dtype=torch.float32, pin_memory=True)
    xh.copy_(x.cpu())
    yh = torch.empty_like(xh, pin_memory=True)
    for _ in range(2):
        B.hhg_apply_host(h, level, B.F32, xh, yh)
    e2e_steps = max(3, min(args.steps, 20))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        B.hhg_apply_host(h, level, B.F32, xh, yh)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    time.sleep(0.2)
    clk = clocks.stop()
    assert torch.isfinite(y).all()
    # BF16 coefficient option: the same apply with k rounded to BF16 (the macro-interior
    # kernels read it as 2 bytes per node); error against the FP32-coefficient apply above
    kb = kl.to(torch.bfloat16)
    B.hhg_set_coefficient(h, kb.view(torch.int16), B.BF16)
    yb = torch.empty_like(y)
    for _ in range(3):
        B.hhg_apply(h, level, B.F32, x, yb)
    torch.cuda.synchronize()
    B.hhg_profile(h, 1)
    evb = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for s, (a0, a1) in enumerate(evb):
        flush.fill_(float(s))
        a0.record(stream)
        B.hhg_apply(h, level, B.F32, x, yb)
        a1.record(stream)
    torch.cuda.synchronize()
    pb_ms, pb_l = B.hhg_profile(h, 0, read=True)
    bms = sum(a0.elapsed_time(a1) for a0, a1 in evb) / args.steps
    bf16 = {"ms_per_step": round(bms, 5), "value": round(dofs / (bms * 1e-3) / 1e9, 3), "unit": "GDoF/s",
            "interior_launch_ms": round(pb_ms[0] / max(1, pb_l[0]), 5),
            "bytes_per_interior_node": BYTES_PER_NODE_F32 - 2,
            "rel_error_vs_fp32_coefficient": float((yb.double() - y.double()).norm() / y.double().norm()),
            "max_abs_error_over_max_abs": float((yb - y).abs().max() / y.abs().max())}
    B.hhg_set_coefficient(h, kl, B.F64)
    # the paper's arithmetic: the same apply in FP64 (x widened from the FP32 input)
    x64 = x.double()
    y64 = torch.empty_like(x64)
    for _ in range(3):
        B.hhg_apply(h, level, B.F64, x64, y64)
    torch.cuda.synchronize()
    ev64 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(20)]
    for s_, (a0, a1) in enumerate(ev64):
        flush.fill_(float(s_))
        a0.record(stream)
        B.hhg_apply(h, level, B.F64, x64, y64)
        a1.record(stream)
    torch.cuda.synchronize()
    ms64 = statistics.median(a0.elapsed_time(a1) for a0, a1 in ev64)
    fp64 = {"ms_per_step": round(ms64, 5), "value": round(dofs / (ms64 * 1e-3) / 1e9, 3), "unit": "GDoF/s",
            "free_dof_value": round(3 * F / (ms64 * 1e-3) / 1e9, 3), "steps": 20, "statistic": "median",
            "rel_difference_fp32_vs_fp64": float((y.double() - y64).norm() / y64.norm())}
    del x64, y64
    # the paper's comparison method: nodal integration a_h on the fly (same coefficient, same x)
    B.hhg_set_problem(h, nu=NU, variant=B.NODAL)
    yn = torch.empty_like(y)
    for _ in range(3):
        B.hhg_apply(h, level, B.F32, x, yn)
    evn = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for s, (a0, a1) in enumerate(evn):
        flush.fill_(float(s))
        a0.record(stream)
        B.hhg_apply(h, level, B.F32, x, yn)
        a1.record(stream)
    torch.cuda.synchronize()
    nms = sum(a0.elapsed_time(a1) for a0, a1 in evn) / args.steps
    nodal = {"ms_per_step": round(nms, 5), "value": round(dofs / (nms * 1e-3) / 1e9, 3), "unit": "GDoF/s",
             "rel_time_physical_over_nodal": round(total_ms / args.steps / nms, 4),
             "rel_difference_vs_physical": float((yn.double() - y.double()).norm() / y.double().norm())}
    # the paper's third method: stored stencils (135 values per macro-interior node, streamed)
    B.hhg_set_problem(h, nu=NU, variant=B.STORED)
    ys = torch.empty_like(y)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B.hhg_apply(h, level, B.F32, x, ys)  # computes the stored blocks, then applies
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    for _ in range(3):
        B.hhg_apply(h, level, B.F32, x, ys)
    torch.cuda.synchronize()
    B.hhg_profile(h, 1)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for s_, (a0, a1) in enumerate(evs):
        flush.fill_(float(s_))
        a0.record(stream)
        B.hhg_apply(h, level, B.F32, x, ys)
        a1.record(stream)
    torch.cuda.synchronize()
    ps_ms, ps_l = B.hhg_profile(h, 0, read=True)
    sms = sum(a0.elapsed_time(a1) for a0, a1 in evs) / args.steps
    s_launch = ps_ms[0] / max(1, ps_l[0])
    s_bytes = STORED_BYTES_PER_NODE_F32 * interior_per_macro
    hbm_peak0, peak_kind0 = measured_peaks()
    stored = {"ms_per_step": round(sms, 5), "value": round(dofs / (sms * 1e-3) / 1e9, 3), "unit": "GDoF/s",
              "build_s": round(build_s, 4), "interior_launch_ms": round(s_launch, 5),
              "bytes_per_interior_node": STORED_BYTES_PER_NODE_F32,
              "interior_hbm_gbs": round(s_bytes / (s_launch * 1e-3) / 1e9, 1),
              "interior_hbm_frac": round(s_bytes / (s_launch * 1e-3) / 1e9 / hbm_peak0, 4), "peak_source": peak_kind0,
              "stored_bytes": int(135 * 4 * E),
              "rel_difference_vs_physical": float((ys.double() - y.double()).norm() / y.double().norm()),
              "rel_time_physical_over_stored": round(total_ms / args.steps / sms, 4)}
    B.hhg_set_problem(h, nu=NU)
    solve = None if args.no_solve else solve_times(B, torch, h, level, coords_e[first])
    B.hhg_destroy(h)
    stokes = None if args.no_stokes else stokes_bench(B, torch, level, dev, stream)
    if stokes is not None and not args.no_plume:
        stokes["plume"] = plume_bench(B, torch, args.plume_level, dev, stream)
    ktable = None if args.no_kernel_table else kernel_table(B, torch, dev, stream, (level, level + 1))
    elasto = None if args.no_elastostatics else elastostatics_bench(B, torch, args.elastostatics_level, 1, dev,
                                                                      stream)
    twod = None if args.no_twod else twod_bench(B, torch, 12, dev, stream)
    if elasto is not None and not args.no_foam:
        elasto["foam"] = foam_bench(B, torch, args.foam_level, dev, stream)
    carreau = None if args.no_carreau else carreau_bench(B, torch, args.carreau_level, dev, stream)
    learned = None if args.no_learn else learned_bench(B, torch, dev, stream, args.learn_train_level,
                                                       args.learn_level, args.learn_seeds, 2, 6, args.learn_steps,
                                                       args.learn_coarsen, args.learn_coarse_train_level,
                                                       args.learn_coarse_seeds)
    learned_stokes = None if args.no_learn_stokes else learned_stokes_bench(
        B, torch, dev, stream, args.learn_train_level, args.learn_stokes_level, args.learn_stokes_fields, 2, 6,
        args.learn_stokes_steps)

    ms_per_step = total_ms / args.steps
    value = job_value(dofs, ms_per_step, world)
    hbm_peak, peak_kind = measured_peaks()
    launch_ms = prof_ms[0] / max(1, prof_launches[0])
    bytes_per_launch = interior_per_macro * BYTES_PER_NODE_F32
    flops_per_launch = interior_per_macro * FLOPS_PER_NODE
    hbm_achieved = bytes_per_launch / (launch_ms * 1e-3) / 1e9
    alu_achieved = flops_per_launch / (launch_ms * 1e-3) / 1e12
    traffic = profiled_traffic()
    hbm_frac = hbm_achieved / hbm_peak
    alu_frac = alu_achieved / alu_peak
    if alu_frac >= hbm_frac:
        roof = {"bound": "alu", "achieved": round(alu_achieved, 3), "peak": round(alu_peak, 2), "unit": "TFLOP/s",
                "frac": round(alu_frac, 4),
                "peak_source": "measured in this run: FP32 FMA probe kernel (hhg_fp32_fma_probe) on %d SMs, "
                               "best of fma.rn.f32 %.1f / fma.rn.f32x2 %.1f TFLOP/s" %
                               (sm_count, alu_probe["fma_f32"], alu_probe["fma_f32x2"])}
    else:
        roof = {"bound": "hbm", "achieved": round(hbm_achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(hbm_frac, 4), "peak_source": peak_kind}
    roof.update({"kernel": "k_interior_pair<APPLY> (FP32, pairs of neighbouring points; one launch per macro)",
                 "traffic": traffic,
                 "algorithmic_bytes_per_launch": bytes_per_launch,
                 "algorithmic_flops_per_launch": flops_per_launch,
                 "launch_ms": round(launch_ms, 5),
                 "hbm": {"achieved_gbs": round(hbm_achieved, 1), "peak_gbs": hbm_peak, "frac": round(hbm_frac, 4),
                         "peak_source": peak_kind},
                 "sm_count": sm_count,
                 "alu": {"achieved_tflops": round(alu_achieved, 3), "peak_tflops": round(alu_peak, 2),
                         "probe_tflops": alu_probe,
                         "frac": round(alu_frac, 4)},
                 "skeleton_ms_per_step": round(prof_ms[1] / args.steps, 5),
                 # the paper's unit (Sec. 4.2 benchmark: 222 ns per node update and CPU rank)
                 "ns_per_interior_node_update": round(launch_ms * 1e6 / interior_per_macro, 5)})
    out = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "GDoF/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_per_step, 5),
        "ms_per_step_median": round(median_ms, 5),
        "free_dof_value": round(job_value(3 * F, ms_per_step, world), 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "level": level, "macros": int(nmacro), "nodes": int(U),
                   "dofs": int(dofs), "free_dofs": int(3 * F), "entries": int(E),
                   "l2": "flushed before every step (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roof,
        "e2e": {"value": round(world * dofs / e2e_s / 1e9, 3), "unit": "GDoF/s",
                "h2d_bytes_per_step": int(xh.numel() * 4), "d2h_bytes_per_step": int(yh.numel() * 4)},
        "gpu_launches": int(prof_launches[0] + prof_launches[1]),
        "solve": solve,
        "kernels": ktable,
        "stokes": stokes,
        "elastostatics": elasto,
        "twod": twod,
        "carreau": carreau,
        "bf16_coefficient": bf16,
        "fp64_apply": fp64,
        "nodal_integration": nodal,
        "stored_stencils": stored,
        "learned": learned,
        "learned_stokes": learned_stokes,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline()
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------- reference arm


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    base = CpuBaseline()
    try:
        for _ in range(max(0, args.warmup)):
            base.measure(0.2)
        per_step = max(0.5, min(6.0, 100.0 / max(1, args.steps)))
        meas = [base.measure(per_step) for _ in range(args.steps)]
    finally:
        base.close()
    value = statistics.mean(m["value"] for m in meas)
    out = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "GDoF/s",
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": None,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD.replace("FP32", "FP64 oracle"), "level": args.level,
                   "sample_level": base.level},
        "cpu_baseline": {"value": value, "unit": "GDoF/s", "cores": base.cores, "kind": "oracle",
                         "sample": "each step: " + meas[-1]["sample"]},
        "e2e": {"value": value, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
