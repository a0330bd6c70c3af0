#!/usr/bin/env python3
"""Benchmark of the direct-sum boundary-integral PB hot path on GB300.

One step = one pass of the whole hot path on one charge configuration that
is already resident on the device: source term, mixed-precision GMRES(10)
solve to a true relative residual of 1e-8 (FP32 mat-vecs inside GMRES, the
refinement residual b - A x in double-float arithmetic -- two FP32 words,
~48 bits, verified against FP64 to 2e-12 -- FP64 Krylov recurrences and
sums), solvation energy (read back to the host).  The same solve with a
native-FP64 refinement residual and the plain FP64 GMRES solve are timed
beside it (solve_ms_mixed_fp64_residual, solve_ms_fp64), and so are the
mixed and FP64 solves with the element self-block preconditioner of Sec.
2.2.4 (solve_ms_mixed_precond_self, solve_ms_fp64_precond_self), which the
paper's GPU pipeline leaves out and the step therefore leaves out too.

Default workload: the Kirkwood sphere (icosphere level 5, N = 20480
triangles, 2N = 40960 unknowns, radius 20 A, 50 charges, eps 1/80,
kappa 0.1257 1/A).  ``--workload protein_like`` selects the displaced
level-6 sphere (N = 81920, 2000 charges).

value = pair interactions evaluated per second over the step (every mat-vec
pair N(N-1), plus the N*Nc source and energy pairs), in Gpairs/s.  The JSON
line also carries the FP64 GMRES solve time of the same system, single
mat-vec throughputs, the roofline of the dominant kernel, the CPU oracle
baseline, the end-to-end number through the host API and the SM clocks.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BIE matvec Gpairs/s; GMRES solve time at 1e-8 rel. residual, mixed vs FP64"
TOL = 1e-8
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2

# Algorithmic work per ordered pair of the mat-vec (the unit of the roofline):
# the pair of Eqs. 5-6 written out term by term (d, r^2, r, s^2 and s^3, the
# exponent argument, c_i, c_j, c_ij, t and w, K1..K4, four accumulations) is
# about 43 FP32-pipe instructions, about 20 of them FMAs, i.e. 63 flops,
# plus 2 MUFU operations.  The kernels execute fewer (the symmetric kernel
# about 23 FP32-pipe instructions per ordered pair, since it evaluates each
# unordered pair once for both rows), so achieved / peak can exceed the pipe's
# busy fraction; the ncu FMA-pipe fraction is reported beside it.
PAIR_FLOPS = 63
PAIR_PIPE_INSTR = 43
# Measured FP32 FFMA throughput (bench.py --mode peaks, the microbenchmark
# microbench/alu_peaks.cu): 3.65e13 lane-ops/s on 152 SMs at a median SM clock
# of 1987 MHz, i.e. 120.9 FMA lanes per SM per clock of the nominal 128.  The
# roofline's peak is this per-clock rate at the SM clock sampled in the timed
# region (2 flop per FMA).
FFMA_LANES_PER_SM_MEASURED = 3.65e13 / (152 * 1987e6)
# ncu FMA-pipe busy fraction of the FP32 mat-vec pair kernel (symmetric variant
# 9) on the Kirkwood workload, from profiles/k_sym_fp32_kirkwood.md
NCU_FMA_PIPE_FRAC_FP32_KIRKWOOD = {9: 0.691}
# DRAM bytes (read + write) per launch of the FP32 mat-vec kernel on the Kirkwood
# workload, by variant, from one ncu capture of that variant's kernel (the
# records and partial sums stay in L2); variants without a capture report null
DRAM_BYTES_FP32_KIRKWOOD = {5: 1.369088e6, 9: 0.702976e6}
FP32_LANES_PER_SM = 128  # FP32 FMA lanes per SM per clock
FP64_LANES_PER_SM = 2    # FP64 FMA lanes per SM per clock (1.25 TFLOP/s nominal at 2.07 GHz, 152 SMs)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="kirkwood", choices=["kirkwood", "protein_like", "adjoint"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison solve")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-API measurement")
    ap.add_argument("--no-extra", action="store_true", help="skip the single mat-vec timings")
    ap.add_argument("--no-config3", action="store_true", help="skip the protein-like (N = 81920) solves")
    ap.add_argument("--cuda-core-residual", action="store_true",
                    help="--mode matvecdfm: df64 multiply-adds on the CUDA cores instead of exact tensor-core digits")
    ap.add_argument("--no-config4a", action="store_true",
                    help="skip the batched 64-charge-set solves on the tensor cores")
    ap.add_argument("--inner", default="direct", choices=["direct", "tree"],
                    help="Krylov mat-vec of the step's mixed solve: the direct FP32 sum (the paper's pipeline) or "
                         "the far-field treecode of Sec. 2.2.3 (MIXED_TREE; the residual stays direct)")
    ap.add_argument("--precond", default="none", choices=["none", "self"],
                    help="preconditioner of the step's solve (none: the paper's GPU pipeline; self: element "
                         "self blocks of Sec. 2.2.4)")
    ap.add_argument("--clocks-csv", default="", help="also keep the raw nvidia-smi clock samples in this file")
    ap.add_argument("--variant", type=int, default=-1,
                    help="FP32 mat-vec variant (default: autotuned; --mode matvec32: the handle's default)")
    ap.add_argument("--ordered-pairs", action="store_true",
                    help="FP64 / double-float mat-vecs visit every ordered pair (default: unordered pairs once)")
    ap.add_argument("--configs", default="3,4a,4b,4bs,5",
                    help="--mode configs: which larger configurations (5fd: the full-size central-difference check)")
    ap.add_argument("--mode", default="solve",
                    choices=["solve", "matvec32", "matvec64", "matvecdf", "matvecdfm", "matvectc", "matvectree",
                             "configs", "peaks"],
                    help="matvec32/matvec64: only W+K single mat-vecs of the workload (for profilers)")
    return ap.parse_args()


def workload(name):
    import synth

    p = synth.problem_by_name(name)
    desc = {
        "kirkwood": "Kirkwood sphere: icosphere level 5 (N=20480 triangles, 40960 unknowns), R=20 A, 50 charges "
                    "in r<16 A, eps 1/80, kappa 0.1257/A; source + mixed-precision GMRES(10) to 1e-8 + energy",
        "protein_like": "protein-like surface: displaced icosphere level 6 (N=81920), R=25 A, 2000 charges, "
                        "eps 1/80, kappa 0.1257/A; source + mixed-precision GMRES(10) to 1e-8 + energy",
        "adjoint": "displaced icosphere level 7 (N=327680), R=45 A, 10000 charges, eps 1/80, kappa 0.1257/A; "
                   "source + mixed-precision GMRES(10) to 1e-8 + energy",
    }[name]
    return p, desc


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, path=None):
        self.index = index
        self.proc = None
        self.keep = bool(path)  # keep the raw samples only where asked
        self.path = path or os.path.join(tempfile.gettempdir(), f"bipb_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            if os.path.dirname(self.path):
                os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception as e:  # nvidia-smi missing: report no clocks
            log("clock sampling unavailable:", e)
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            lines = f.readlines()
        if not self.keep:
            os.remove(self.path)
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def _load_for(step, seconds):
    """Untimed steps for about `seconds` (keeps the GPU under load around the timed region)."""
    import torch

    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        step()
        torch.cuda.synchronize()


# ------------------------------------------------------------------ CPU oracle
def cpu_oracle_rate(prob, budget_s=10.0):
    """Oracle FP64 mat-vec pair rate on this host: full mat-vecs until the budget is used."""
    import oracle

    oracle.build()
    eps = prob.eps_out / prob.eps_in
    u = np.random.default_rng(0).standard_normal(2 * prob.n)
    n = prob.n
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle.matvec(prob.centroids, prob.normals, prob.areas, eps, prob.kappa, u)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or el / reps * (reps + 1) > 2.5 * budget_s:
            break
    pairs = reps * n * (n - 1)
    return {"value": pairs / el / 1e9, "unit": "Gpairs/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{reps} full FP64 oracle mat-vec(s) of the workload ({n}x{n - 1} pairs each), {el:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    prob, desc = workload(args.workload)
    import oracle

    oracle.build()
    eps = prob.eps_out / prob.eps_in
    n = prob.n
    rows = max(64, int(2e9 / 2.0 / n) // 16 * 16)  # ~1e9 pairs per step
    rows = min(rows, 2 * n)
    rng = np.random.default_rng(1)
    u = rng.standard_normal(2 * n)
    sel = np.sort(rng.choice(2 * n, rows, replace=False))
    for _ in range(args.warmup):
        oracle.matvec_rows(prob.centroids, prob.normals, prob.areas, eps, prob.kappa, u, sel[:64])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.matvec_rows(prob.centroids, prob.normals, prob.areas, eps, prob.kappa, u, sel)
    el = time.perf_counter() - t0
    value = args.steps * rows * (n - 1) / el / 1e9
    sample = f"{rows} sampled rows of the FP64 mat-vec per step ({rows * (n - 1):.3g} pairs)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gpairs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": desc, "n": n, "nc": prob.nc},
            "cpu_baseline": {"value": value, "unit": "Gpairs/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "Gpairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_configs(args):
    """The CPU oracle on every configuration, on this host: one FP64 mat-vec
    on all cores and on one core (rows sampled where a full one would take
    long, scaled to N(N-1) pairs), and the oracle's GMRES(10) solve to 1e-8
    for the Born and Kirkwood systems; the larger solves are extrapolated
    from the mat-vec time (stated in each line)."""
    import platform

    import oracle
    import synth

    oracle.build()
    cores = oracle.num_threads()
    host = {"machine": platform.machine(), "cpus": os.cpu_count(), "oracle_threads": cores}
    rng = np.random.default_rng(7)

    def matvec_s(prob, threads, max_pairs):
        """Seconds per full mat-vec, from the rows that make up about max_pairs pairs."""
        n = prob.n
        eps = prob.eps_out / prob.eps_in
        u = rng.standard_normal(2 * n)
        rows = int(min(2 * n, max(threads * 8, max_pairs // (n - 1))))
        sel = np.sort(rng.choice(2 * n, rows, replace=False))
        oracle.set_threads(threads)
        try:
            t0 = time.perf_counter()
            oracle.matvec_rows(prob.centroids, prob.normals, prob.areas, eps, prob.kappa, u, sel)
            el = time.perf_counter() - t0
        finally:
            oracle.set_threads(cores)
        return el * (n * (n - 1)) / (rows * (n - 1)), rows

    cfgs = (("1: Born ion, level 3", synth.born_problem(level=3), True),
            ("2: Kirkwood sphere, level 5", synth.kirkwood_problem(level=5), True),
            ("3: protein-like, level 6", synth.protein_like_problem(), False),
            ("5: displaced sphere, level 7", synth.adjoint_problem(), False))
    per_solve_mv = None
    for name, prob, full in cfgs:
        n = prob.n
        t_all, r_all = matvec_s(prob, cores, 2.0e9 * cores / 16)
        t_one, r_one = matvec_s(prob, 1, 1.2e8)
        line = {"impl": "reference", "mode": "configs", "config": name, "n": n, "host": host,
                "matvec_s_all_cores": t_all, "matvec_s_one_core": t_one,
                "matvec_sample_rows": {"all_cores": r_all, "one_core": r_one, "of": 2 * n},
                "gpairs_all_cores": n * (n - 1) / t_all / 1e9,
                "pairs_per_s_per_core": n * (n - 1) / t_one}
        if full:
            t0 = time.perf_counter()
            sol = oracle.solve(prob, method="gmres", tol=1e-8, restart=10)
            line["solve_s"] = time.perf_counter() - t0
            line["solve"] = f"measured: oracle GMRES(10) to 1e-8, {sol.info.get('iters')} iterations"
            per_solve_mv = sol.info.get("iters", 0) + 1
        else:
            mv = per_solve_mv or 29
            line["solve_s"] = mv * t_all
            line["solve"] = f"extrapolated: {mv} mat-vecs (the Kirkwood solve's count) x the all-core mat-vec"
            if name.startswith("3"):
                line["solve_s_64_rhs"] = 64 * mv * t_all
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def run_matvec_only(args):
    """W + K single mat-vecs of one precision on the workload (a small, fixed launch sequence)."""
    import torch

    from paper_2312_10044_gb300.build import build

    build()
    import paper_2312_10044_gb300 as bipb

    prob, desc = workload(args.workload)
    prec = {"matvec32": bipb.FP32, "matvec64": bipb.FP64, "matvecdf": bipb.DF64, "matvecdfm": bipb.DF64,
            "matvectc": bipb.TENSOR, "matvectree": bipb.TREE32}[args.mode]
    n_vec = 64 if args.mode in ("matvectc", "matvecdfm") else 1
    med = bipb.medium(prob.eps_in, prob.eps_out, prob.kappa)
    with bipb.Surface(prob.centroids, prob.normals, prob.areas) as s:
        if args.variant >= 0:
            s.set_variant(args.variant)
        if args.ordered_pairs:
            s.symmetric_pairs(False)
        if args.cuda_core_residual:
            s.exact_tensor_residual(False)
        u = torch.randn(n_vec, 2 * prob.n, dtype=torch.float64, device="cuda")
        y = torch.empty_like(u)
        for _ in range(args.warmup):
            s.matvec(u, y, precision=prec, med=med)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for _ in range(args.steps):
            s.matvec(u, y, precision=prec, med=med)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / args.steps
    print(json.dumps({"mode": args.mode, "workload": desc, "n_vec": n_vec, "ms_per_matvec": ms,
                      "gpairs": prob.n * (prob.n - 1) / ms / 1e6,
                      "g_pair_rhs": n_vec * prob.n * (prob.n - 1) / ms / 1e6}), flush=True)


def _timed(fn, torch):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    out = fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b), out


def run_configs(args):
    """One timed run of each larger configuration (after one untimed warm-up
    of the same call): protein-like single solve, 64-RHS batched solve on the
    tensor-core path vs CUDA cores, uneven batch of 8 surfaces, and the
    level-7 adjoint (forward + adjoint solve + gradient).  Prints one JSON
    line per configuration."""
    import torch

    import synth
    from paper_2312_10044_gb300.build import build

    build()
    import paper_2312_10044_gb300 as bipb

    which = args.configs.split(",")
    out = []

    def emit(d):
        print(json.dumps(d), flush=True)
        out.append(d)

    if "3" in which:
        p = synth.protein_like_problem()
        med = bipb.medium(p.eps_in, p.eps_out, p.kappa)
        with bipb.Surface(p.centroids, p.normals, p.areas) as s:
            s.set_charges(p.charge_pos, p.q)
            v, mv = s.autotune(med, reps=2)
            res = {"config": "protein-like N=81920, 2000 charges", "matvec32_variant": v, "matvec32_ms": mv}
            for name, prec, pc in (("mixed_df64", bipb.MIXED_DF64, bipb.PRECOND_NONE),
                                   ("mixed_fp64_residual", bipb.MIXED, bipb.PRECOND_NONE),
                                   ("mixed_df64_precond_self", bipb.MIXED_DF64, bipb.PRECOND_SELF)):
                prm = bipb.solve_params(p.eps_in, p.eps_out, p.kappa, tol=TOL, precision=prec, precond=pc)
                s.solve(prm)
                ms, info = _timed(lambda: s.solve(prm), torch)
                res[f"solve_ms_{name}"] = ms
                res[f"{name}_info"] = info[0]
            res["energy_kcal"] = float(s.energy()[0])
            # potential maps (10^4 points in the molecule, 10^4 in the solvent) and the free energy
            rng = np.random.default_rng(11)
            dirs = rng.standard_normal((20000, 3))
            dirs /= np.linalg.norm(dirs, axis=1)[:, None]
            radii = np.concatenate([rng.uniform(0.0, 20.0, 10000), rng.uniform(31.0, 80.0, 10000)])
            pts = dirs * radii[:, None]
            s.potential_at(pts[:10000], inside=True)
            ms_in, _ = _timed(lambda: s.potential_at(pts[:10000], inside=True), torch)
            ms_out, _ = _timed(lambda: s.potential_at(pts[10000:], inside=False), torch)
            ms_free, (ef, ec) = _timed(lambda: s.energy_free(), torch)
            res["potential_ms_10k_inside"] = ms_in
            res["potential_ms_10k_outside"] = ms_out
            res["energy_free_ms"] = ms_free
            res["energy_free_kcal"] = float(ef[0])
            res["energy_coulomb_kcal"] = float(ec[0])
            res.update(far_field_timings(bipb, torch, s, p))
            # plain FP64 GMRES: one run (26+ FP64 mat-vecs of ~0.7 s)
            if not args.no_fp64:
                prm = bipb.solve_params(p.eps_in, p.eps_out, p.kappa, tol=TOL, precision=bipb.FP64)
                ms, info = _timed(lambda: s.solve(prm), torch)
                res["solve_ms_fp64"] = ms
                res["fp64_info"] = info[0]
            emit(res)
    if "4a" in which:
        base = synth.protein_like_problem()
        p = synth.batched_charges(base, n_rhs=64, n_charges=2000)
        med = bipb.medium(p.eps_in, p.eps_out, p.kappa)
        with bipb.Surface(p.centroids, p.normals, p.areas) as s:
            s.set_charges(p.charge_pos, p.q)
            n = p.n
            U = torch.randn(64, 2 * n, dtype=torch.float64, device="cuda")
            Y = torch.empty_like(U)
            res = {"config": "batched: protein-like N=81920, 64 charge sets x 2000"}
            for name, prec in (("tensor", bipb.TENSOR), ("fp32_cuda_cores", bipb.FP32)):
                s.matvec(U, Y, precision=prec, med=med)
                ms, _ = _timed(lambda: s.matvec(U, Y, precision=prec, med=med), torch)
                res[f"matvec64rhs_ms_{name}"] = ms
                res[f"pair_rhs_per_s_{name}"] = 64 * n * (n - 1) / (ms / 1e3)
            prm = bipb.solve_params(p.eps_in, p.eps_out, p.kappa, tol=TOL, precision=bipb.MIXED_TENSOR)
            s.solve(prm)  # untimed: the once-per-surface row scales of the tensor-core residual
            bipb.timer_enable(s, True)
            ms, info = _timed(lambda: s.solve(prm), torch)
            t = bipb.timer_read(s)
            bipb.timer_enable(s, False)
            res["solve_ms_mixed_tensor_64rhs"] = ms
            res["kernel_ms"] = {k: v[1] for k, v in t.items() if v[0]}
            res["iters_max"] = max(i["iters"] for i in info)
            res["refine_steps_max"] = max(i["refine_steps"] for i in info)
            res["refine_steps_hist"] = {str(k): sum(1 for i in info if i["refine_steps"] == k)
                                        for k in sorted({i["refine_steps"] for i in info})}
            res["rel_residual_max"] = max(i["rel_residual"] for i in info)
            # the same with the element self-block preconditioner (Sec. 2.2.4)
            prm.precond = bipb.PRECOND_SELF
            bipb.timer_enable(s, True)
            ms, info = _timed(lambda: s.solve(prm), torch)
            t = bipb.timer_read(s)
            bipb.timer_enable(s, False)
            res["solve_ms_mixed_tensor_64rhs_precond_self"] = ms
            res["kernel_ms_precond_self"] = {k: v[1] for k, v in t.items() if v[0]}
            res["kernel_launches_precond_self"] = {k: v[0] for k, v in t.items() if v[0]}
            res["iters_max_precond_self"] = max(i["iters"] for i in info)
            res["rel_residual_max_precond_self"] = max(i["rel_residual"] for i in info)
            emit(res)
    if "4b" in which:
        probs = synth.uneven_batch_problems()
        with bipb.BatchSurface([(q.centroids, q.normals, q.areas) for q in probs]) as s:
            s.set_charges([(q.charge_pos, q.q[0]) for q in probs])
            prm = bipb.solve_params(probs[0].eps_in, probs[0].eps_out, probs[0].kappa, tol=TOL,
                                    precision=bipb.MIXED_DF64)
            s.solve(prm)
            ms, info = _timed(lambda: s.solve(prm), torch)
            res = {"config": "uneven batch: 8 displaced spheres, levels 4,4,4,5,5,5,6,6",
                   "sizes": [q.n for q in probs], "sum_n2": sum(q.n * q.n for q in probs),
                   "solve_ms_mixed_df64": ms, "iters": [i["iters"] for i in info],
                   "rel_residual_max": max(i["rel_residual"] for i in info)}
            # the same surfaces one at a time
            tot = 0.0
            for q in probs:
                with bipb.Surface(q.centroids, q.normals, q.areas) as s1:
                    s1.set_charges(q.charge_pos, q.q)
                    s1.solve(prm)
                    m1, _ = _timed(lambda: s1.solve(prm), torch)
                    tot += m1
            res["solve_ms_one_at_a_time"] = tot
            emit(res)
    if "4bs" in which:
        # many small uneven surfaces, where one launch per pass over all of them
        # (instead of one solve per surface) pays
        probs = synth.uneven_batch_problems(levels=(2, 3, 3, 4) * 8, seed0=4200)
        with bipb.BatchSurface([(q.centroids, q.normals, q.areas) for q in probs]) as s:
            s.set_charges([(q.charge_pos, q.q[0]) for q in probs])
            prm = bipb.solve_params(probs[0].eps_in, probs[0].eps_out, probs[0].kappa, tol=TOL,
                                    precision=bipb.MIXED_DF64)
            s.solve(prm)
            ms, info = _timed(lambda: s.solve(prm), torch)
            res = {"config": "uneven batch of small surfaces: 32 displaced spheres, levels 2,3,3,4 x 8",
                   "sizes": [q.n for q in probs], "sum_n2": sum(q.n * q.n for q in probs),
                   "solve_ms_mixed_df64": ms, "iters_max": max(i["iters"] for i in info),
                   "rel_residual_max": max(i["rel_residual"] for i in info)}
            tot = 0.0
            for q in probs:
                with bipb.Surface(q.centroids, q.normals, q.areas) as s1:
                    s1.set_charges(q.charge_pos, q.q)
                    s1.solve(prm)
                    m1, _ = _timed(lambda: s1.solve(prm), torch)
                    tot += m1
            res["solve_ms_one_at_a_time"] = tot
            emit(res)
    if "5" in which:
        p = synth.adjoint_problem()
        with bipb.Surface(p.centroids, p.normals, p.areas) as s:
            s.set_charges(p.charge_pos, p.q)
            prm = bipb.solve_params(p.eps_in, p.eps_out, p.kappa, tol=TOL, precision=bipb.MIXED_DF64)
            s.solve(prm)  # untimed warm-up of both calls
            s.energy_grad(prm)
            ms_f, info = _timed(lambda: s.solve(prm), torch)
            ms_g, (dq, dy) = _timed(lambda: s.energy_grad(prm), torch)
            res = {"config": "adjoint: displaced icosphere level 7 (N=327680), R=45, 10000 charges",
                   "solve_ms_mixed_df64": ms_f, "energy_grad_ms": ms_g, "info": info[0],
                   "energy_kcal": float(s.energy()[0]), "max_abs_force": float(np.abs(dy).max())}
            # the same with the element self-block preconditioner (Sec. 2.2.4)
            prm.precond = bipb.PRECOND_SELF
            ms_fp, info_p = _timed(lambda: s.solve(prm), torch)
            ms_gp, (dqp, dyp) = _timed(lambda: s.energy_grad(prm), torch)
            res.update({"solve_ms_mixed_df64_precond_self": ms_fp, "energy_grad_ms_precond_self": ms_gp,
                        "info_precond_self": info_p[0],
                        "max_rel_force_difference_precond": float(np.abs(dyp - dy).max() / np.abs(dy).max())})
            res.update(far_field_timings(bipb, torch, s, p))
            emit(res)
    if "5fd" in which:
        emit(config5_central_differences(bipb, torch))
    return out


def far_field_timings(bipb, torch, s, p):
    """The far-field (treecode) FP32 mat-vec of Sec. 2.2.3 with its default
    parameters (and its transpose) against the direct FP32 mat-vec, and the
    mixed solve with it (MIXED_TREE, plain and with the self-block
    preconditioner) against the direct mixed solve, plus the energy gradient
    whose adjoint solve takes the far-field transpose; s is a handle of
    problem p with its charges set."""
    n = p.n
    med = bipb.medium(p.eps_in, p.eps_out, p.kappa)
    u = torch.randn(2 * n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(u)
    out = {}
    pairs, far, leaves = s.treecode_stats()
    out["tree_pairs_per_matvec"] = pairs
    out["tree_pairs_frac_of_direct"] = pairs / (n * (n - 1))
    out["tree_far_clusters"], out["tree_leaves"] = far, leaves
    for name, prec, reps, tr in (("tree32", bipb.TREE32, 10, False), ("fp32_direct", bipb.FP32, 5, False),
                                 ("tree32_transpose", bipb.TREE32, 10, True),
                                 ("fp32_direct_transpose", bipb.FP32, 5, True)):
        s.matvec(u, y, precision=prec, transpose=tr, med=med)
        ms, _ = _timed(lambda: [s.matvec(u, y, precision=prec, transpose=tr, med=med) for _ in range(reps)], torch)
        out[f"matvec_ms_{name}"] = ms / reps
    bipb.timer_enable(s, True)
    s.matvec(u, y, precision=bipb.TREE32, med=med)
    t = bipb.timer_read(s)
    bipb.timer_enable(s, False)
    out["tree_kernel_ms"] = t["matvec_tree"][1]
    out["tree_kernel_gpairs"] = pairs / (t["matvec_tree"][1] / 1e3) / 1e9 if t["matvec_tree"][1] > 0 else None
    for name, prec, pc in (("mixed_tree", bipb.MIXED_TREE, bipb.PRECOND_NONE),
                           ("mixed_tree_precond_self", bipb.MIXED_TREE, bipb.PRECOND_SELF)):
        prm = bipb.solve_params(p.eps_in, p.eps_out, p.kappa, tol=TOL, precision=prec, precond=pc)
        s.solve(prm)
        ms, info = _timed(lambda: s.solve(prm), torch)
        out[f"solve_ms_{name}"] = ms
        out[f"{name}_info"] = dict(info[0], energy_kcal=float(s.energy()[0]))
        gms, _ = _timed(lambda: s.energy_grad(prm), torch)
        out[f"energy_grad_ms_{name}"] = gms
    return out


def config5_central_differences(bipb, torch):
    """Full-size check of the adjoint gradient on 32 seeded atoms (level 7).

    Moving charge k by +-h e_d changes only its own term of the source b and
    of the energy row c, so E(y +- h e_d) - E(y) = 1/2 [dc.u + c.du + dc.du]
    with A du = db, where db and dc are the source and energy row of the
    charge pair {(y_k +- h e_d, q_k), (y_k, -q_k)}.  The 192 pair systems are
    solved together (tensor-core Krylov + double-float residual, tol 1e-9), and each
    term is a reaction-energy pass: no difference of two large energies is
    taken.  dE/dq_k (E is quadratic in q, so central differences are exact)
    = 1/2 (c_k.u + c.u_k) with u_k the solution for a unit charge at y_k.
    """
    import synth

    p = synth.adjoint_problem()
    n, y, q = p.n, p.charge_pos, p.q[0]
    med = bipb.medium(p.eps_in, p.eps_out, p.kappa)
    atoms = np.sort(np.random.default_rng(7).choice(p.nc, 32, replace=False))
    h = 1e-4
    res = {"config": "adjoint gradient vs central differences: level 7 (N=327680), 10000 charges, 32 seeded "
                      "atoms, h=1e-4 A (solution differences)"}
    t0 = time.perf_counter()
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        s.set_charges(y, q)
        base = bipb.solve_params(p.eps_in, p.eps_out, p.kappa, tol=1e-10, precision=bipb.MIXED_DF64)
        s.solve(base)
        phi, dphi = s.surface_potential()
        u0 = np.concatenate([phi[0], dphi[0]]) / bipb.KCAL
        dq, dy = s.energy_grad(base)
        pos_sets, q_sets = [], []
        for k in atoms:
            for d in range(3):
                for sg in (1.0, -1.0):
                    yp = y[k].copy()
                    yp[d] += sg * h
                    pos_sets.append([yp, y[k]])
                    q_sets.append([q[k], -q[k]])
        for k in atoms:  # unit charge at y_k (the second charge is empty)
            pos_sets.append([y[k], y[k]])
            q_sets.append([1.0, 0.0])
        B = len(q_sets)
        s.set_charges(np.array(pos_sets), np.array(q_sets))
        prm = bipb.solve_params(p.eps_in, p.eps_out, p.kappa, tol=1e-9, precision=bipb.MIXED_TENSOR)
        ms, info = _timed(lambda: s.solve(prm), torch)
        res["pair_solves"] = {"systems": B, "ms": ms, "converged": int(sum(i["converged"] for i in info)),
                              "rel_residual_max": max(i["rel_residual"] for i in info)}
        phi, dphi = s.surface_potential()
        du = torch.tensor(np.concatenate([phi, dphi], axis=1) / bipb.KCAL, dtype=torch.float64, device="cuda")
        del phi, dphi
        e_b = torch.empty(B, dtype=torch.float64, device="cuda")
        s.reaction(du, None, e_b, med)  # 1/2 dc.du
        e_a = torch.empty_like(e_b)
        s.reaction(torch.tensor(u0, device="cuda").repeat(B, 1), None, e_a, med)  # 1/2 dc.u
        s.set_charges(y[None], np.repeat(q[None], B, axis=0))
        e_c = torch.empty_like(e_b)
        s.reaction(du, None, e_c, med)  # 1/2 c.du
    D = (e_a + e_b + e_c).cpu().numpy()
    g_fd = ((D[0:192:2] - D[1:192:2]) / (2 * h)).reshape(32, 3)
    g_adj = dy[0][atoms]
    dq_fd = (e_a + e_c).cpu().numpy()[192:]
    dq_adj = dq[0][atoms]
    res["dE_dy_max_rel_err"] = float(np.abs(g_fd - g_adj).max() / np.abs(g_adj).max())
    res["dE_dy_per_atom_rel_err_max"] = float(
        (np.linalg.norm(g_fd - g_adj, axis=1) / np.linalg.norm(g_adj, axis=1)).max())
    res["dE_dq_max_rel_err"] = float(np.abs(dq_fd - dq_adj).max() / np.abs(dq_adj).max())
    res["max_abs_force"] = float(np.abs(g_adj).max())
    res["seconds_total"] = time.perf_counter() - t0
    return res


def config3_solves(bipb, torch):
    """The largest single-RHS configuration beside the headline: the
    protein-like surface (displaced icosphere level 6, N = 81920, 2000
    charges), source + solve to 1e-8 + energy, each solve timed once after an
    untimed run of the same call: mixed (FP32 Krylov, double-float residual),
    mixed with an FP64 residual, plain FP64 GMRES, and the mixed solve with
    the element self-block preconditioner; then the far-field mat-vec and the
    mixed solves on it (far_field_timings)."""
    import synth

    p = synth.protein_like_problem()
    out = {"config3_workload": "protein-like surface: displaced icosphere level 6 (N=81920), R=25 A, 2000 charges, "
                               "eps 1/80, kappa 0.1257/A, tol 1e-8"}
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        s.set_charges(p.charge_pos, p.q)
        for key, prec, pre in (("mixed", bipb.MIXED_DF64, bipb.PRECOND_NONE),
                               ("mixed_fp64_residual", bipb.MIXED, bipb.PRECOND_NONE),
                               ("fp64", bipb.FP64, bipb.PRECOND_NONE),
                               ("mixed_precond_self", bipb.MIXED_DF64, bipb.PRECOND_SELF)):
            prm = bipb.solve_params(p.eps_in, p.eps_out, p.kappa, tol=TOL, restart=10, precision=prec,
                                    precond=pre)
            if key != "fp64":  # the FP64 solve takes seconds: one run, no warm-up
                s.solve(prm)
            ms, info = _timed(lambda: (s.solve(prm)[0], s.energy()[0]), torch)
            out[f"config3_solve_ms_{key}"] = ms
            out[f"config3_{key}_info"] = dict(info[0], energy_kcal=info[1])
        out.update({f"config3_{k}": v for k, v in far_field_timings(bipb, torch, s, p).items()})
    return out


def config4a_solves(bipb, torch):
    """The batched configuration: 64 charge sets of 2000 charges (each with its
    own positions) on the protein-like surface, solved together with the
    tensor-core Krylov mat-vec and the exact tensor-core double-float
    residual (BIPB_MIXED_TENSOR) to 1e-8, plain and with the element
    self-block preconditioner, each timed once after an untimed run of the
    same call, and the 64 energy gradients (forward and adjoint solves); the
    64-RHS mat-vec, its transpose and the residual timed alone."""
    import synth

    base = synth.protein_like_problem()
    p = synth.batched_charges(base, n_rhs=64, n_charges=2000)
    med = bipb.medium(p.eps_in, p.eps_out, p.kappa)
    out = {"config4a_workload": "protein-like surface (N=81920), 64 charge sets x 2000 charges, eps 1/80, "
                                "kappa 0.1257/A, tol 1e-8"}
    with bipb.Surface(p.centroids, p.normals, p.areas) as s:
        s.set_charges(p.charge_pos, p.q)
        U = torch.randn(64, 2 * p.n, dtype=torch.float64, device="cuda")
        Y = torch.empty_like(U)
        for key, prec, tr in (("tensor", bipb.TENSOR, False), ("tensor_transpose", bipb.TENSOR, True),
                              ("df64_tensor", bipb.DF64, False)):
            s.matvec(U, Y, precision=prec, transpose=tr, med=med)
            ms, _ = _timed(lambda: s.matvec(U, Y, precision=prec, transpose=tr, med=med), torch)
            out[f"config4a_matvec64rhs_ms_{key}"] = ms
        for key, pre in (("mixed_tensor", bipb.PRECOND_NONE), ("mixed_tensor_precond_self", bipb.PRECOND_SELF)):
            prm = bipb.solve_params(p.eps_in, p.eps_out, p.kappa, tol=TOL, restart=10,
                                    precision=bipb.MIXED_TENSOR, precond=pre)
            s.solve(prm)
            ms, info = _timed(lambda: s.solve(prm), torch)
            out[f"config4a_solve_ms_{key}"] = ms
            out[f"config4a_{key}_iters_max"] = max(i["iters"] for i in info)
            out[f"config4a_{key}_refine_steps_max"] = max(i["refine_steps"] for i in info)
            out[f"config4a_{key}_rel_residual_max"] = max(i["rel_residual"] for i in info)
            if pre == bipb.PRECOND_NONE:  # the 64 energy gradients: forward and adjoint solves on the tensor cores
                s.energy_grad(prm)
                gms, _ = _timed(lambda: s.energy_grad(prm), torch)
                out["config4a_energy_grad_ms_mixed_tensor"] = gms
    return out


def run_peaks(args):
    """Measured throughput of the FP32 FFMA, FP64 DFMA and MUFU pipes (the
    microbenchmark microbench/alu_peaks.cu, built here with nvcc), against the
    nominal unit counts at the SM clock sampled meanwhile."""
    here = os.path.dirname(os.path.abspath(__file__))
    src = os.path.join(here, "paper_2312_10044_gb300", "microbench", "alu_peaks.cu")
    exe = os.path.join(here, "_build", "alu_peaks")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe, src])
    clocks = ClockSampler(0, args.clocks_csv or None)
    clocks.start()
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    clk = clocks.stop()
    vals = dict(line.split(None, 1) for line in out.splitlines() if line.strip())
    if vals.get("status", "").strip() != "ok":
        raise RuntimeError(out)
    sms = int(vals["sms"])
    f = (clk["sm_mhz"] if clk else 2070.0) * 1e6
    res = {"mode": "peaks", "sms": sms, "clocks": clk}
    for name, lanes in (("ffma", FP32_LANES_PER_SM), ("dfma", FP64_LANES_PER_SM), ("mufu", 16)):
        v = float(vals[f"{name}_per_s"])
        nominal = sms * lanes * f
        res[f"{name}_per_s"] = v
        res[f"{name}_nominal_per_s"] = nominal
        res[f"{name}_frac_of_nominal"] = v / nominal
    print(json.dumps(res), flush=True)
    return res


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference_configs(args) if args.mode == "configs" else run_reference(args)
    if args.mode == "configs":
        return run_configs(args)
    if args.mode == "peaks":
        return run_peaks(args)
    if args.mode != "solve":
        return run_matvec_only(args)
    import torch

    from paper_2312_10044_gb300 import replicas
    from paper_2312_10044_gb300.build import build

    world, rank, local = replicas.init("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    if rank == 0:
        build()
    replicas.barrier(world)
    import paper_2312_10044_gb300 as bipb

    prob, desc = workload(args.workload)
    n, nc = prob.n, prob.nc
    params = bipb.solve_params(prob.eps_in, prob.eps_out, prob.kappa, tol=TOL, restart=10,
                               precision=bipb.MIXED_TREE if args.inner == "tree" else bipb.MIXED_DF64,
                               precond=bipb.PRECOND_SELF if args.precond == "self" else bipb.PRECOND_NONE)
    s = bipb.Surface(prob.centroids, prob.normals, prob.areas)
    s.set_charges(prob.charge_pos, prob.q)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        info = s.solve(params)
        e = s.energy()
        return info[0], e[0]

    if args.variant >= 0:  # fixed variant (profiling runs: the autotuner's timings under a profiler differ)
        s.set_variant(args.variant)
        variant = args.variant
        log(f"FP32 mat-vec variant {variant} (fixed)")
    else:
        variant, mv_ms = s.autotune(bipb.medium(prob.eps_in, prob.eps_out, prob.kappa), reps=3)
        log(f"autotune: FP32 mat-vec variant {variant}, {mv_ms:.4f} ms")
    for _ in range(args.warmup):
        info, e = step()
    log(f"warm-up: {info} E={e:.6f} kcal/mol")

    # ---- timed region: K steps, events per step, L2 flushed between steps.
    # The clock sampler starts during untimed steps before the region and
    # stops after untimed steps behind it, so that its samples (one per 100
    # ms) cover the whole region with the GPU under load.
    cs = ClockSampler(local, args.clocks_csv)
    cs.start()
    _load_for(step, 0.6)
    bipb.timer_enable(s, True)
    launches0 = bipb.launch_count(s)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    replicas.barrier(world)
    torch.cuda.synchronize()
    infos = []
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record()
        infos.append(step())
        evs[k][1].record()
    torch.cuda.synchronize()
    launches = bipb.launch_count(s) - launches0
    timers = bipb.timer_read(s)
    bipb.timer_enable(s, False)
    _load_for(step, 0.3)
    clocks = cs.stop()
    replicas.barrier(world)
    ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = replicas.max_over_ranks(float(sum(ms)), world, dev)
    info0 = infos[-1][0]
    mv = info0["matvecs32"] + info0["matvecs64"]
    pairs_step = mv * n * (n - 1) + 2 * n * nc
    tree_pairs = None
    if args.inner == "tree":  # the Krylov mat-vecs evaluate the far-field operator's pairs only
        tree_pairs = s.treecode_stats()[0]
        pairs_step = info0["matvecs32"] * tree_pairs + info0["matvecs64"] * n * (n - 1) + 2 * n * nc
    value = replicas.whole_job_rate(args.steps * pairs_step, world, total_ms / 1e3) / 1e9

    # ---- dominant kernel and its roofline (from the events around each launch)
    # the dominant kernel; with the far-field Krylov mat-vec, the roofline is that kernel's
    dom = "matvec_tree" if args.inner == "tree" else max(timers, key=lambda k: timers[k][1])
    cnt, tms = timers[dom]
    # launches that found their system converged return at once; average over the effective ones
    eff = {"matvec32": info0["matvecs32"] * args.steps, "matvec_tree": info0["matvecs32"] * args.steps}.get(dom, cnt)
    avg_ms = tms / max(min(cnt, eff), 1)
    f_mhz = clocks["sm_mhz"] if clocks else 2070.0
    lanes = FP64_LANES_PER_SM if dom.startswith("matvec64") else FP32_LANES_PER_SM
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    pairs_launch = tree_pairs if dom == "matvec_tree" else n * (n - 1)
    fp32 = lanes == FP32_LANES_PER_SM
    lanes_meas = FFMA_LANES_PER_SM_MEASURED if fp32 else lanes
    achieved = pairs_launch * PAIR_FLOPS / (avg_ms / 1e3) / 1e12
    peak = nsm * lanes_meas * 2 * f_mhz * 1e6 / 1e12
    peak_nominal = nsm * lanes * 2 * f_mhz * 1e6 / 1e12
    instr_frac = pairs_launch * PAIR_PIPE_INSTR / (avg_ms / 1e3) / (nsm * lanes_meas * f_mhz * 1e6)
    traffic = None
    if dom == "matvec32" and args.workload == "kirkwood":
        traffic = DRAM_BYTES_FP32_KIRKWOOD.get(variant)
    ncu_pipe = NCU_FMA_PIPE_FRAC_FP32_KIRKWOOD.get(variant) if dom == "matvec32" and args.workload == "kirkwood" \
        else None
    roofline = {"bound": "alu", "kernel": f"{dom} pair kernel", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                "pipe": "fp32" if fp32 else "fp64",
                "definition": f"achieved = {PAIR_FLOPS} flops x {pairs_launch} ordered (target, source) pairs per "
                              "launch / mean launch time; "
                              f"peak = {nsm} SMs x {lanes_meas:.1f} measured {'FFMA' if fp32 else 'DFMA'} lanes per "
                              f"SM per clock x 2 flop x {f_mhz:.0f} MHz (median SM clock sampled in the timed "
                              "region); the symmetric kernel evaluates each unordered pair once for both rows, so "
                              "it executes fewer instructions than the algorithmic count and frac can exceed 1",
                "peak_nominal": peak_nominal, "frac_of_nominal": achieved / peak_nominal,
                "instr_frac": instr_frac,
                "instr_note": f"{PAIR_PIPE_INSTR} FP32-pipe instructions per ordered pair over the measured issue "
                              "peak (can exceed 1 for the same reason)",
                "ncu_fma_pipe_frac": ncu_pipe,
                "ncu_note": "FMA-pipe busy fraction of this kernel from one ncu capture "
                            "(profiles/k_sym_fp32_kirkwood.md): how busy the pipe actually is",
                "pairs_per_launch": pairs_launch, "sms": nsm, "sm_mhz": f_mhz,
                "avg_launch_ms": avg_ms, "launches": cnt, "effective_launches": min(cnt, eff),
                "kernel_ms": {k: v[1] for k, v in timers.items() if v[0]},
                "kernel_launches": {k: v[0] for k, v in timers.items() if v[0]}}

    extra = {}
    # ---- single mat-vec throughputs (device-resident, events around 10 launches each)
    u = torch.randn(2 * n, dtype=torch.float64, device=dev)
    y = torch.empty_like(u)
    med = bipb.medium(prob.eps_in, prob.eps_out, prob.kappa)
    for prec, name, reps in (() if args.no_extra else ((bipb.FP32, "fp32", 20), (bipb.FP64, "fp64", 3),
                                                          (bipb.DF64, "df64", 5))):
        s.matvec(u, y, precision=prec, med=med)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            s.matvec(u, y, precision=prec, med=med)
        b.record()
        torch.cuda.synchronize()
        extra[f"matvec_{name}_gpairs"] = reps * n * (n - 1) / (a.elapsed_time(b) / 1e3) / 1e9
    # ---- FP64 GMRES solve of the same system
    if not args.no_fp64:
        p64 = bipb.solve_params(prob.eps_in, prob.eps_out, prob.kappa, tol=TOL, restart=10, precision=bipb.FP64)
        s.solve(p64)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        i64 = s.solve(p64)[0]
        b.record()
        torch.cuda.synchronize()
        extra["solve_ms_fp64"] = a.elapsed_time(b)
        extra["fp64_info"] = i64
        # the same mixed solve with a native FP64 refinement residual
        pm = bipb.solve_params(prob.eps_in, prob.eps_out, prob.kappa, tol=TOL, restart=10, precision=bipb.MIXED)
        s.solve(pm)
        a.record()
        im = s.solve(pm)[0]
        b.record()
        torch.cuda.synchronize()
        extra["solve_ms_mixed_fp64_residual"] = a.elapsed_time(b)
        extra["mixed_fp64_residual_info"] = im
        # plain FP64 GMRES with the element self-block preconditioner (Sec. 2.2.4)
        p64.precond = bipb.PRECOND_SELF
        s.solve(p64)
        a.record()
        ip = s.solve(p64)[0]
        b.record()
        torch.cuda.synchronize()
        extra["solve_ms_fp64_precond_self"] = a.elapsed_time(b)
        extra["fp64_precond_self_info"] = ip
    # the step's mixed solve with the element self-block preconditioner (Sec.
    # 2.2.4, applied on the right): same true-residual target, fewer FP32 mat-vecs
    pp = bipb.solve_params(prob.eps_in, prob.eps_out, prob.kappa, tol=TOL, restart=10,
                           precision=bipb.MIXED_DF64, precond=bipb.PRECOND_SELF)
    s.solve(pp)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(5):
        ipp = s.solve(pp)[0]
    b.record()
    torch.cuda.synchronize()
    extra["solve_ms_mixed_precond_self"] = a.elapsed_time(b) / 5
    extra["mixed_precond_self_info"] = ipp
    extra["solve_ms_mixed"] = total_ms / args.steps
    extra["mixed_info"] = info0
    extra["energy_kcal"] = infos[-1][1]
    if args.workload == "kirkwood" and not args.no_config3:
        extra.update(config3_solves(bipb, torch))
    if args.workload == "kirkwood" and not args.no_config4a:
        extra.update(config4a_solves(bipb, torch))

    # ---- end to end through the host API: geometry + charges from pinned host
    # memory, create, solve, energy back to the host, destroy
    cen = torch.from_numpy(prob.centroids).pin_memory()
    nrm = torch.from_numpy(prob.normals).pin_memory()
    area = torch.from_numpy(prob.areas).pin_memory()
    pos = torch.from_numpy(np.ascontiguousarray(prob.charge_pos)).pin_memory()
    qq = torch.from_numpy(np.ascontiguousarray(prob.q)).pin_memory()
    e2e_steps = 0 if args.no_e2e else max(2, min(args.steps, 5))
    torch.cuda.synchronize()
    replicas.barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        with bipb.Surface(cen.numpy(), nrm.numpy(), area.numpy()) as s2:
            s2.set_charges(pos.numpy(), qq.numpy())
            s2.solve(params)
            s2.energy()
    torch.cuda.synchronize()
    e2e_s = replicas.max_over_ranks((time.perf_counter() - t0) / max(e2e_steps, 1), world, dev)
    h2d = cen.numel() * 8 + nrm.numel() * 8 + area.numel() * 8 + pos.numel() * 8 + qq.numel() * 8
    e2e = None if not e2e_steps else {
        "value": replicas.whole_job_rate(pairs_step, world, e2e_s) / 1e9, "unit": "Gpairs/s",
        "h2d_bytes_per_step": int(h2d),
        "d2h_bytes_per_step": 8, "ms_per_step": e2e_s * 1e3,
        "api": "bipb_surface_create + bipb_charges_set + bipb_solve + bipb_energy + bipb_surface_destroy"}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_oracle_rate(prob)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "Gpairs/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32 (Krylov mat-vecs) + df64 (residual) + f64",
                "data": "synthetic",
                "config": {"workload": desc, "n": n, "nc": nc, "tol": TOL, "restart": 10, "l2": "flushed",
                           "parallelism": f"replicas{world}", "matvec32_variant": variant,
                           "precond": args.precond, "inner": args.inner},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clocks}
        line.update(extra)
        print(json.dumps(line), flush=True)
    s.close()
    replicas.finish(world)


if __name__ == "__main__":
    main()
