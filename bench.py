#!/usr/bin/env python3
"""Time to rtol 1e-8 of Chebyshev-basis s-step PCG with FGS Gram solves, against classical PCG
from the same CUDA library, on the 3D 7-point Poisson problem (256^3 interior unknowns,
stencil form, Jacobi), one GB300 per rank.  Prints one JSON line (rank 0).

A step is one whole solve: r0 = b - A x0, the outer iterations of PCG-S to ||r|| <= 1e-8 ||b||
(MPK, Gram reduction + reduced solves, fused block update, stop test) and the true residual.
Inputs (b, x0) are resident in device memory when the timed region starts; every vector is
134 MB, larger than L2, and the working set is several GB.

--impl reference times the FP64 CPU oracle on the host cores on bounded samples of the same
workload, extrapolated to a whole solve with the oracle's own iteration count.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1e-8 rel. residual, s-step vs classical PCG, 256^3 Poisson; HBM GB/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
COUNTS_FILE = os.path.join(ROOT, "tests", "golden", "oracle_counts_256.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
# FP64 pipe of GB300: 2 FMA per clock per SM x 152 SMs x 2.07 GHz x 2 flops = 1.259 TFLOP/s
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=256, help="grid edge (n^3 unknowns)")
    p.add_argument("--s", type=int, default=4)
    p.add_argument("--sweeps", type=int, default=3)
    p.add_argument("--algo", choices=["literal", "onesync"], default="literal")
    p.add_argument("--form", choices=["stencil", "csr"], default="stencil")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--extra", default="4:30,4:3:fp32_rr,4:30:fp32_rr",
                   help="extra s-step configs 's:nu[:precision]' to time once each, e.g. "
                        "'4:30,4:3:fp32_rr' (precision fp64 or fp32_rr)")
    p.add_argument("--batch", default="64:16",
                   help="batched workload 'nsys:nrhs' (7-point systems, edges uniform in 32..96); "
                        "empty to skip")
    p.add_argument("--adjoint", type=int, default=128,
                   help="edge of the differentiated Q1 workload (theta ~ N(0, 0.5^2) per cell, unit "
                        "right-hand side); 0 skips")
    p.add_argument("--batch-shape", default="0:0",
                   help="'cluster:threads' of the batched launches (0: autotuned)")
    p.add_argument("--hpcg", type=int, default=200,
                   help="edge of the 27-point Poisson benchmark with unit right-hand side "
                        "(s in 4..10, eta diagnostics); 0 skips")
    p.add_argument("--q1", type=int, default=192,
                   help="edge of the Q1 log-normal diffusion workload (FP32 basis, s = 8); 0 skips")
    p.add_argument("--grid", default="2,4,8:2,3",
                   help="s values:nu values of the FP64 configuration grid timed once each at the "
                        "headline size, stencil and CSR forms; empty skips")
    p.add_argument("--oracle-full", default="",
                   help="run the FP64 oracle to completion on the n^3 7-point workload for one "
                        "configuration ('pcg' or '<literal|onesync>_s<S>nu<NU>') on one host "
                        "thread, print its time as one JSON line and exit (no GPU work)")
    p.add_argument("--small", type=int, default=64,
                   help="edge of the 2D 5-point CSR workload (s = 4, nu = 2; GPU and oracle times); "
                        "0 skips")
    return p.parse_args()


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_median": float(np.median(power)) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- algorithmic work per kernel

def kernel_work(s, n, points=7, sym_blocks=False):
    """Algorithmic bytes and FP64 flops of each kernel launch (FP64 values, 8 bytes).

    A multiply-add counts 2 flops.  Literal form (default): b2 = -Q^T AZ (s^2 products),
    Q/AQ update fused with W = Q^T AQ (symmetric: its upper triangle, s (s + 1) / 2 products),
    b1 = Q^T r and the previous step's deferred x += Q alpha (2 s^2 + s (s + 1) / 2 + 2 s
    multiply-adds), r update (s + 1).  One-reduction form: one Gram pass (4 s^2 + 2 s products,
    or 2 s^2 + 3 s with the symmetric shortcut) and one update pass (2 s^2 + 2 s + 1)."""
    V = 8.0 * n
    sp_flops = {5: 5, 7: 7, 27: 27}[points]  # Poisson: (points-1) adds + 1 multiply per row
    rec = 4  # z_{q+1} = c1 d (Az) - c2 z_q - z_{q-1}: 2 multiplies + 2 adds
    ne = (2 * s * s + 3 * s) if sym_blocks else (4 * s * s + 2 * s)
    mpk_bytes = (4 * (s - 1) + 2) * V if s > 1 else 3 * V
    return {
        "mpk_step": {"bytes": mpk_bytes / s, "flops": (sp_flops + rec) * n},
        "gram_b2": {"bytes": 2 * s * V, "flops": 2.0 * s * s * n},
        # the update also adds the previous step's x += Q alpha (read and write x, s FMAs); the
        # r update reads AQ and r and writes r
        "update_w": {"bytes": (6 * s + 3) * V,
                     "flops": 2.0 * (2 * s * s + s * (s + 1) // 2 + s + s) * n},
        "update_xr": {"bytes": (s + 2) * V, "flops": (2.0 * (s + 1) + 2) * n},
        "gram": {"bytes": (4 * s + 1) * V, "flops": 2.0 * ne * n},
        "update": {"bytes": (6 * s + 4) * V, "flops": 2.0 * (2 * s * s + 2 * s + 1) * n},
        "pcg_spmv_dot": {"bytes": 2 * V, "flops": (sp_flops + 2) * n},
        "pcg_update": {"bytes": 6 * V, "flops": 10.0 * n},
        "pcg_pdir": {"bytes": 3 * V, "flops": 3.0 * n},
    }


def source_hash(*files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def load_traffic(kernel, workload, src_hash):
    try:
        data = json.load(open(TRAFFIC_FILE))
        rec = data.get(kernel + "@" + workload)
        if rec and rec.get("source_hash") == src_hash:
            return rec["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


def hbm_peak():
    try:
        return float(json.load(open(PEAKS_FILE))["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- oracle (CPU) timing

def oracle_sample(n_edge, s, nu, gpu_lambda=None, outer_sample=2, algo="literal"):
    """Time the oracle on bounded samples of the workload and extrapolate to a whole solve.

    Returns (seconds_per_solve, description, details).  The extrapolation multiplies the
    per-outer-iteration time by the oracle's own iteration count for this workload when it is
    recorded (tests/golden/oracle_counts_256.json), else by the count given by the caller.
    """
    import oracle as O
    from paper_2603_09790_gb300 import inputs as I

    dims = (n_edge,) * 3
    A = O.CSR(*I.poisson_csr(dims, 7))
    xt, b = I.poisson_problem(dims, 7)
    v0 = I.power_start(A.n)
    t = time.perf_counter()
    lam2, _ = O.power(A, "jacobi", v0, 2, 0.0)
    t_power = (time.perf_counter() - t) / 2 * 20  # 20 power iterations
    lam = gpu_lambda if gpu_lambda else lam2
    t = time.perf_counter()
    O.pcgs(A, b, s=s, nu=nu, rtol=0.0, max_outer=outer_sample, algo=algo, lambda_max=lam)
    t_outer_s = (time.perf_counter() - t) / outer_sample
    t = time.perf_counter()
    O.pcg(A, b, rtol=0.0, max_iters=4 * outer_sample)
    t_pcg_it = (time.perf_counter() - t) / (4 * outer_sample)
    return t_power, t_outer_s, t_pcg_it


def oracle_counts():
    try:
        return json.load(open(COUNTS_FILE))
    except Exception:
        return {}


# ---------------------------------------------------------------- ranks

def reduce_over_ranks(value, world, device):
    """Max over ranks of a per-rank time (replicas: every rank solves its own copy of the
    problem; the job's time per step is that of the slowest rank)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- reference arm

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    counts = oracle_counts()
    key = f"{args.algo}_s{args.s}nu{args.sweeps}"
    if args.n != 256 or key not in counts:
        print(json.dumps({"impl": "reference", "unavailable":
                          f"no recorded oracle iteration count for n={args.n}, {key}"}))
        return 0
    N_outer = counts[key]["iters"]
    times = []
    for k in range(args.warmup + args.steps):
        t_power, t_outer, _ = oracle_sample(args.n, args.s, args.sweeps, outer_sample=1,
                                            algo=args.algo)
        if k >= args.warmup:
            times.append(t_power + t_outer * N_outer)
    v = float(np.mean(times))
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"poisson7_{args.n}^3_{args.form}_jacobi_s{args.s}_nu{args.sweeps}",
                   "algo": f"PCG-S {args.algo} form, FP64 oracle (plain C, sequential)"},
        "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle",
                         "sample": f"per step: 1 outer iteration + 2 power iterations of the oracle "
                                   f"at {args.n}^3, extrapolated to 20 power iterations and the oracle's "
                                   f"recorded {N_outer} outer iterations"},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- our arm

def run_grid(spec, N, dev, sstep, I, torch, b, v0d):
    """The FP64 configuration grid at N^3: stencil and CSR forms x s x nu (literal form), plus
    classical PCG per form.  One solve per configuration (its graph capture included, about a
    millisecond); set-up (operator copy, Jacobi, Gershgorin bound, 20 power iterations) timed
    separately and added into the total."""
    s_list, nu_list = ([int(v) for v in part.split(",")] for part in spec.split(":"))
    dims = (N, N, N)
    rp, ci, vv = I.poisson_csr(dims, 7)
    ops = {"stencil": lambda: sstep.Stencil(N, N, N, 7),
           "csr": lambda: sstep.CSR(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev),
                                    torch.from_numpy(vv).to(dev))}
    bd = torch.from_numpy(b).to(dev)
    common = dict(rtol=1e-8, power_iters=20, power_tol=0.0, power_v0=v0d, lambda_min=-1.0)
    out = {"workload": f"poisson7_{N}^3_jacobi_literal", "rtol": 1e-8,
           "timing": "setup_s: host wall time of sstep_setup (power method included); solve_s: "
                     "sstep_info.ms_solve of one solve (device buffers; first solve of the handle, "
                     "graph capture included); total_s = setup_s + solve_s"}
    for form, mk in ops.items():
        A = mk()
        cases = [(f"s{s_}_nu{nu_}", dict(s=s_, sweeps=nu_)) for s_ in s_list for nu_ in nu_list]
        cases.append(("pcg", dict(algo="pcg")))
        for label, kw in cases:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            S = sstep.Solver(A, **common, **kw)
            t_setup = time.perf_counter() - t0
            x = torch.zeros_like(bd)
            info = S.solve(bd, x)
            S.free()
            out[f"{form}_{label}"] = {
                "setup_s": t_setup, "solve_s": info.ms_solve / 1e3,
                "total_s": t_setup + info.ms_solve / 1e3, "outer_iters": info.outer_iters,
                "inner_equiv": info.inner_equiv, "status": info.status,
                "relres_true": info.relres_true}
        del A
        torch.cuda.empty_cache()
    for form in ops:
        pcg = out[f"{form}_pcg"]["solve_s"]
        for k in list(out):
            if k.startswith(form + "_s") and isinstance(out[k], dict):
                out[k]["solve_over_pcg"] = out[k]["solve_s"] / pcg
    return out


def run_small(N, dev, sstep, I, torch, with_oracle):
    """2D 5-point Poisson on an N x N grid, FP64 CSR, Jacobi, s = 4, nu = 2, Chebyshev interval
    from 20 power iterations and the Gershgorin lower bound, rtol 1e-8; against classical PCG
    of the library; the FP64 oracle run to completion on the same input (one host thread)."""
    dims = (N, N)
    rp, ci, vv = I.poisson_csr(dims, 5)
    xt, b = I.poisson_problem(dims, 5)
    v0 = I.power_start(N * N)
    A = sstep.CSR(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev), torch.from_numpy(vv).to(dev))
    bd = torch.from_numpy(b).to(dev)
    common = dict(rtol=1e-8, power_iters=20, power_tol=0.0, power_v0=torch.from_numpy(v0).to(dev),
                  lambda_min=-1.0)
    out = {"workload": f"poisson5_{N}x{N}_csr_jacobi_literal_s4_nu2", "n": N * N, "nnz": int(rp[-1]),
           "timing": "median of 5 solves (sstep_info.ms_solve, device buffers) after a warm-up; "
                     "setup_s: host wall time of sstep_setup"}
    lam = None
    for label, kw in (("sstep", dict(s=4, sweeps=2)), ("pcg", dict(algo="pcg"))):
        t0 = time.perf_counter()
        S = sstep.Solver(A, **common, **kw)
        t_setup = time.perf_counter() - t0
        x = torch.zeros_like(bd)
        S.solve(bd, x)
        ts, info = [], None
        for _ in range(5):
            x.zero_()
            info = S.solve(bd, x)
            ts.append(info.ms_solve / 1e3)
        if label == "sstep":
            lam = S.get_basis_info()["lambda_max"]
        S.free()
        out[label] = {"setup_s": t_setup, "solve_s": float(np.median(ts)),
                      "outer_iters": info.outer_iters, "relres_true": info.relres_true,
                      "x_rel_error_vs_true": float(np.linalg.norm(x.cpu().numpy() - xt) / np.linalg.norm(xt))}
    out["sstep_over_pcg"] = out["sstep"]["solve_s"] / out["pcg"]["solve_s"]
    if with_oracle:
        import oracle as O
        Ac = O.CSR(rp, ci, vv)
        t0 = time.perf_counter()
        lam_o, _ = O.power(Ac, "jacobi", v0, 20, 0.0)
        ref = O.pcgs(Ac, b, s=4, nu=2, rtol=1e-8, algo="literal",
                     lambda_min=O.gershgorin_lower(Ac, "jacobi"), lambda_max=lam_o)
        t_or = time.perf_counter() - t0
        t0 = time.perf_counter()
        refp = O.pcg(Ac, b, rtol=1e-8)
        t_orp = time.perf_counter() - t0
        out["oracle"] = {"sstep_s": t_or, "sstep_outer_iters": ref.iters, "pcg_s": t_orp,
                         "pcg_iters": refp.iters, "cores": 1,
                         "what": "the FP64 C oracle (plain sequential loops) run to completion, "
                                 "power method included, one host thread"}
        out["lambda_max_gpu_vs_oracle"] = [lam, lam_o]
    return out


def run_batch(spec, dev, sstep, I, torch, shape="0:0"):
    """Batched workload: nsys 7-point Poisson systems with edges drawn uniformly in 32..96
    (seed 0), nrhs right-hand sides each (U[-1,1), seed 1 + system), Jacobi, nu = 3, rtol 1e-8,
    solved by one persistent launch per call; against the plain FP64 form (one single-system
    handle per system, right-hand sides one after another)."""
    nsys, nrhs = (int(v) for v in spec.split(":"))
    grids = I.batch_grids(nsys, 32, 96, seed=0)
    n = [int(np.prod(g)) for g in grids]
    A = [sstep.Stencil(*g, points=7) for g in grids]
    bd, xd = [], []
    for i in range(nsys):
        rhs = torch.from_numpy(I.batch_rhs(i, n[i], nrhs)).to(dev)
        for j in range(nrhs):
            bd.append(rhs[j].contiguous())
            xd.append(torch.zeros(n[i], dtype=torch.float64, device=dev))
    out = {"workload": f"batch_{nsys}x{nrhs}_poisson7_edges32-96_jacobi_nu30",
           "unknowns_per_rhs": int(sum(n)), "problems": nsys * nrhs,
           "sweeps": "30 (the paper's own FGS sweep count; the batched configuration names none)"}
    cl, nt = (int(v) for v in shape.split(":"))
    common = dict(sweeps=30, rtol=1e-8, power_iters=20, power_tol=0.0, cluster=cl, block_threads=nt)

    def zero():
        for x in xd:
            x.zero_()
        torch.cuda.synchronize()

    for label, kw in (("fp64_s4", dict(s=4)), ("fp64_autotuned", dict(s=0)),
                      ("fp32_rr_s4", dict(s=4, precision="fp32_rr")),
                      ("fp32_rr_autotuned", dict(s=0, precision="fp32_rr")),
                      ("fp64_autotuned_nu3", dict(s=0, sweeps=3))):
        kw = dict(common, **kw)
        t0 = time.perf_counter()
        S = sstep.Solver(A, **kw)
        t_setup = time.perf_counter() - t0
        zero()
        S.solve_batched(bd, xd)  # warm-up (graph instantiation)
        zero()
        t0 = time.perf_counter()
        infos = S.solve_batched(bd, xd)
        t = time.perf_counter() - t0
        cfg = S.get_batch_config()
        S.free()
        its = [i.outer_iters for i in infos]
        out[label] = {"s": t, "setup_s": t_setup, "config": cfg,
                      "outer_iters_mean": float(np.mean(its)), "outer_iters_max": int(max(its)),
                      "all_converged": all(i.status == sstep.OK for i in infos),
                      "max_relres_true": float(max(i.relres_true for i in infos)),
                      "launches_per_solve": int(infos[0].launches)}
    # the plain FP64 form on a sample of the right-hand sides, scaled to all of them
    sample = min(2, nrhs)
    t_plain = 0.0
    for i in range(nsys):
        S = sstep.Solver(A[i], s=4, **{k: v for k, v in common.items() if k not in ("cluster", "block_threads")})
        xs = [torch.zeros(n[i], dtype=torch.float64, device=dev) for _ in range(sample)]
        S.solve(bd[i * nrhs], xs[0])  # graph instantiation
        for x in xs:
            x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.solve_batched(bd[i * nrhs:i * nrhs + sample], xs)
        t_plain += time.perf_counter() - t0
        S.free()
    out["plain_fp64_s4_sequential_s"] = t_plain * nrhs / sample
    out["plain_sample"] = f"{sample} of {nrhs} right-hand sides of every system, time scaled by {nrhs / sample:g}"
    out["fp64_s4_speedup_vs_plain"] = out["plain_fp64_s4_sequential_s"] / out["fp64_s4"]["s"]
    out["timing"] = "host wall time of one synchronous sstep_solve_batched call, after a warm-up call"
    return out


def run_q1(N, dev, sstep, I, torch):
    """Q1 trilinear diffusion with log-normal conductivity (sigma 1, correlation 8 cells) on an
    N^3 grid of interior vertices, Jacobi, s = 8, rtol 1e-8: the FP32-basis form against the
    FP64 form and classical PCG of the same library (FP64, and in the FP32-basis recipe with
    the CSR matrix), with the assembled CSR matrix and with the matrix-free operator (keys
    mf_*) on the same conductivities."""
    dims = (N, N, N)
    t0 = time.perf_counter()
    (rp, ci, v), kappa, xt, b = I.q1_lognormal_problem(dims)
    t_gen = time.perf_counter() - t0
    n = N ** 3
    ops = {"": sstep.CSR(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev),
                         torch.from_numpy(v).to(dev)),
           "mf_": sstep.Q1(N, N, N, torch.from_numpy(np.ascontiguousarray(kappa)).to(dev))}
    bd = torch.from_numpy(b).to(dev)
    xtd = torch.from_numpy(xt).to(dev)
    out = {"workload": f"q1_lognormal_{N}^3_jacobi_literal_s8", "n": n, "nnz": int(rp[-1]),
           "operators": {"(no prefix)": "CSR assembled by the input generator",
                         "mf_": "matrix-free Q1 from the cell conductivities"},
           "generation_s": t_gen}
    sol = {}
    for pre, A in ops.items():
        for label, kw in (("fp64_s8_nu30", dict(s=8, sweeps=30)),
                          ("fp32_rr_s8_nu30", dict(s=8, sweeps=30, precision="fp32_rr", rr_period=8)),
                          ("fp32_rr_s8_nu3", dict(s=8, sweeps=3, precision="fp32_rr", rr_period=8)),
                          ("fp32_rr_s4_nu30", dict(s=4, sweeps=30, precision="fp32_rr", rr_period=4)),
                          ("fp64_pcg", dict(algo="pcg")),
                          ("fp32_rr_pcg", dict(algo="pcg", precision="fp32_rr"))):
            S = sstep.Solver(A, rtol=1e-8, power_iters=20, power_tol=0.0, lambda_min=-1.0, **kw)
            x = torch.zeros_like(bd)
            S.solve(bd, x)  # warm-up (graph instantiation)
            x.zero_()
            torch.cuda.synchronize()
            info = S.solve(bd, x)
            ph = S.profile(bd, iters=3) if "pcg" not in label else None
            S.free()
            key = pre + label
            sol[key] = x
            out[key] = {"s": info.ms_solve / 1e3, "status": info.status,
                        "outer_iters": info.outer_iters, "relres_true": info.relres_true,
                        "rel_error_vs_x_true": float(torch.linalg.norm(x - xtd) / torch.linalg.norm(xtd))}
            if ph is not None:
                out[key]["phase_ms_per_outer"] = {"mpk": ph[0], "gram_b2": ph[1], "update_w": ph[2],
                                                  "update_xr": ph[3]}
    ref = sol["fp64_s8_nu30"]
    for key in sol:
        if key == "fp64_s8_nu30":
            continue
        out[key]["rel_diff_vs_fp64_s8"] = float(torch.linalg.norm(sol[key] - ref) / torch.linalg.norm(ref))
        out[key]["time_over_fp64_s8"] = out[key]["s"] / out["fp64_s8_nu30"]["s"]
    out["timing"] = "host wall time of one sstep_solve (device buffers) after a warm-up solve"
    return out


def run_hpcg27(N, dev, sstep, torch):
    """The paper's own benchmark problem on one GPU: 27-point Poisson on N^3 interior points
    (N = 200 is one GPU's share of its 64-GPU run), unit right-hand side, Jacobi, rtol 1e-8,
    s in {4, 6, 8, 10} at nu = 30, FP64; outer counts, times, the reduced-solve residuals
    eta_alpha / eta_beta of every outer iteration, and the diagonally normalised Gram pattern
    for s = 10 at outer iterations 5..8 (mean |W_ij| / sqrt(W_ii W_jj) by distance |i - j|)."""
    A = sstep.Stencil(N, N, N, 27)
    b = torch.ones(N ** 3, dtype=torch.float64, device=dev)
    out = {"workload": f"poisson27_{N}^3_stencil_jacobi_unit_rhs_literal_nu30", "n": N ** 3}
    # the paper's power-method rule (relative change 1e-3, at most 50 iterations)
    common = dict(rtol=1e-8, power_iters=50, power_tol=1e-3, lambda_min=-1.0)
    for s_ in (4, 6, 8, 10):
        S = sstep.Solver(A, s=s_, sweeps=30, **common)
        x = torch.zeros_like(b)
        S.solve(b, x)  # warm-up (graph instantiation)
        x.zero_()
        info = S.solve(b, x)
        d = S.get_diagnostics()
        S.free()
        ea, eb = d["eta_a"], d["eta_b"]
        e = {"s": info.ms_solve / 1e3, "outer_iters": info.outer_iters,
             "inner_equiv": info.inner_equiv, "relres_true": info.relres_true,
             "eta_alpha_max": float(ea.max()) if ea.size else None,
             "eta_alpha_median": float(np.median(ea)) if ea.size else None,
             "eta_beta_max": float(eb.max()) if eb.size else None,
             "eta_beta_median": float(np.median(eb)) if eb.size else None}
        if s_ == 10 and d["W"].shape[0] >= 9:
            pat = []
            for k in range(5, 9):
                W = d["W"][k]
                dg = np.sqrt(np.diag(W))
                Wn = np.abs(W) / np.outer(dg, dg)
                pat.append([float(np.mean(np.diag(Wn, off))) for off in range(s_)])
            e["gram_pattern_k5_8_by_offset"] = pat
        out[f"s{s_}_nu30"] = e
    # exact reduced solves at s = 10: how much of the outer convergence FGS costs
    S = sstep.Solver(A, s=10, gram="cholesky", algo="onesync", **common)
    x = torch.zeros_like(b)
    S.solve(b, x)
    x.zero_()
    info = S.solve(b, x)
    S.free()
    out["s10_cholesky"] = {"s": info.ms_solve / 1e3, "outer_iters": info.outer_iters,
                           "inner_equiv": info.inner_equiv, "relres_true": info.relres_true}
    P = sstep.Solver(A, algo="pcg", **common)
    x = torch.zeros_like(b)
    P.solve(b, x)
    x.zero_()
    info = P.solve(b, x)
    P.free()
    out["pcg"] = {"s": info.ms_solve / 1e3, "iters": info.outer_iters, "relres_true": info.relres_true}
    out["timing"] = "sstep_info.ms_solve (host wall time of one solve, device buffers) after a warm-up"
    return out


def run_adjoint(N, dev, sstep, I, torch):
    """Differentiated solve: Q1 diffusion on N^3 interior vertices with kappa = exp(theta),
    theta ~ N(0, 0.5^2) iid per cell (seed 0), b = 1, loss = ||x - x_target||^2 with x_target
    the solution for theta = 0.  Forward + backward through autograd.q1_solve (kappa = exp(theta),
    device assembly of the CSR values for the AMG preconditioner, x recomputed in backward,
    adjoint s-step solve, per-cell gradient kernel) against one plain FP64 set-up + solve of the
    same system; the gradient is checked by central differences on 32 random cells (seed 2,
    h = 1e-3, solves at rtol 1e-12 with the matrix-free operator and Jacobi)."""
    from paper_2603_09790_gb300 import autograd as AG
    dims = (N, N, N)
    t0 = time.perf_counter()
    patt = AG.Q1Pattern(dims, dev)
    t_pat = time.perf_counter() - t0
    ncell = (N + 1) ** 3
    theta0 = torch.from_numpy(0.5 * I.normal_pm(0, ncell)).to(dev)
    b = torch.ones(N ** 3, dtype=torch.float64, device=dev)
    opts = dict(s=4, sweeps=30, rtol=1e-8, power_iters=20, power_tol=0.0, precond="amg",
                amg_coarse_max=512)
    with torch.no_grad():
        x_target = AG.q1_solve(torch.zeros_like(theta0), b, patt, **dict(opts, precond="jacobi"))

    def loss_of(th, o):
        x = AG.q1_solve(th, b, patt, **o)
        return torch.sum((x - x_target) ** 2)

    th = theta0.clone().requires_grad_(True)
    loss_of(th, opts).backward()  # warm-up
    th = theta0.clone().requires_grad_(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = loss_of(th, opts)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    loss.backward()
    torch.cuda.synchronize()
    t_all = time.perf_counter() - t0
    g = th.grad
    # plain FP64 set-up + solve of the same system, AMG and Jacobi, set-up and solve apart
    kappa = torch.empty_like(theta0)
    sstep.q1_exp(theta0, kappa)
    vals = patt.values(kappa)
    A = sstep.CSR(patt.pattern.rowptr, patt.pattern.colind, vals)
    plain = {}
    for label, op, kw in (("amg_csr", A, opts), ("jacobi_csr", A, dict(opts, precond="jacobi")),
                          ("jacobi_matrix_free", sstep.Q1(N, N, N, kappa), dict(opts, precond="jacobi"))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S = sstep.Solver(op, **kw)
        t_setup = time.perf_counter() - t0
        x = torch.zeros_like(b)
        S.solve(b, x)  # graph capture
        x.zero_()
        info = S.solve(b, x)
        S.free()
        plain[label] = {"setup_s": t_setup, "solve_s": info.ms_solve / 1e3,
                        "outer_iters": info.outer_iters, "relres_true": info.relres_true}
    # central differences on 32 random cells, solves at rtol 1e-12 (matrix-free, Jacobi)
    o12 = dict(opts, rtol=1e-12, precond="jacobi")
    rng = np.random.default_rng(2)
    cells = rng.choice(ncell, 32, replace=False)
    h = 1e-3
    fd_err = []
    t0 = time.perf_counter()
    gmax = max(abs(g).max().item(), 1e-300)
    with torch.no_grad():
        for c in cells:
            tp, tm = theta0.clone(), theta0.clone()
            tp[c] += h
            tm[c] -= h
            fd = (loss_of(tp, o12).item() - loss_of(tm, o12).item()) / (2 * h)
            fd_err.append(abs(fd - g[c].item()) / gmax)
    t_fd = time.perf_counter() - t0
    return {"workload": f"q1_theta_{N}^3_amg_literal_s4_nu30_adjoint", "n": N ** 3,
            "amg": "double pairwise aggregation, l1-Jacobi V-cycle, dense coarse solve at <= 512; "
                   "hierarchy set up on the host, V-cycle on the device",
            "cells": ncell, "pattern_s": t_pat, "loss": float(loss.item()),
            "forward_s": t_fwd, "forward_backward_s": t_all,
            "plain_fp64": plain,
            "forward_backward_over_plain_amg": t_all / (plain["amg_csr"]["setup_s"] + plain["amg_csr"]["solve_s"]),
            "fd_cells": [int(c) for c in cells], "fd_step": h,
            "fd_max_err_rel_to_max_grad": float(max(fd_err)), "fd_s": t_fd,
            "timing": "host wall time (synchronised); forward/backward include every handle set-up "
                      "(AMG hierarchy included); plain_fp64 splits set-up and solve"}


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        info = dict(l.split(":", 1) for l in out.splitlines() if ":" in l)
        return {k: info.get(k, "").strip() for k in ("Architecture", "Model name", "CPU(s)", "Vendor ID")}
    except Exception:
        return {}


def run_oracle_full(args):
    """The FP64 oracle run to completion (rtol 1e-8) on the n^3 7-point workload, one host
    thread: power method (20 iterations, start vector seed 1) + PCG-S or PCG."""
    import oracle as O
    from paper_2603_09790_gb300 import inputs as I
    dims = (args.n,) * 3
    A = O.CSR(*I.poisson_csr(dims, 7))
    xt, b = I.poisson_problem(dims, 7)
    cfg = args.oracle_full
    t0 = time.perf_counter()
    lam, _ = O.power(A, "jacobi", I.power_start(A.n), 20, 0.0)
    t_power = time.perf_counter() - t0
    t0 = time.perf_counter()
    if cfg == "pcg":
        r = O.pcg(A, b, rtol=1e-8)
    else:
        algo, rest = cfg.split("_")
        s_, nu_ = rest[1:].split("nu")
        r = O.pcgs(A, b, s=int(s_), nu=int(nu_), rtol=1e-8, algo=algo,
                   lambda_min=O.gershgorin_lower(A, "jacobi"), lambda_max=lam)
    t_solve = time.perf_counter() - t0
    print(json.dumps({"oracle_full": cfg, "n": A.n, "power_s": t_power, "solve_s": t_solve,
                      "total_s": t_power + t_solve, "iters": r.iters, "status": r.status,
                      "relres_true": r.relres_true, "cores": 1, "cpu": cpu_model()}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.oracle_full:
        return run_oracle_full(args)

    import torch
    import torch.distributed as dist

    from paper_2603_09790_gb300 import inputs as I
    from paper_2603_09790_gb300 import sstep

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    if world > 1:
        # replicas: every rank times the headline solve; the side workloads are reported by the
        # single-GPU run and would only hold the other GPUs here
        args.extra, args.batch, args.q1, args.adjoint, args.hpcg = "", "", 0, 0, 0

    def barrier():
        if world > 1:
            dist.barrier()

    N = args.n
    dims = (N, N, N)
    n = N ** 3
    xt, b = I.poisson_problem(dims, 7)
    v0 = I.power_start(n)
    bd = torch.from_numpy(b).to(dev)
    v0d = torch.from_numpy(v0).to(dev)
    stream = torch.cuda.Stream(device=dev)
    if args.form == "stencil":
        A = sstep.Stencil(N, N, N, 7)
    else:
        rp, ci, vv = I.poisson_csr(dims, 7)
        A = sstep.CSR(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev),
                      torch.from_numpy(vv).to(dev))
    common = dict(rtol=1e-8, power_iters=20, power_tol=0.0, power_v0=v0d, lambda_min=-1.0,
                  stream=stream)

    def timed_solves(S, xd, K, W):
        for _ in range(W):
            xd.zero_()
            S.solve(bd, xd)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        evs = []
        infos = []
        for _ in range(K):
            with torch.cuda.stream(stream):
                xd.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            infos.append(S.solve(bd, xd))
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        barrier()
        ms = [a.elapsed_time(b_) for a, b_ in evs]
        return ms, infos

    # ---- s-step (headline)
    S = sstep.Solver(A, s=args.s, sweeps=args.sweeps, algo=args.algo, **common)
    xd = torch.zeros(n, dtype=torch.float64, device=dev)
    gpu_id = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    sampler = ClockSampler(("GPU-" + str(gpu_id)) if gpu_id else local)
    for _ in range(args.warmup):
        xd.zero_()
        S.solve(bd, xd)
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    ms, infos = timed_solves(S, xd, args.steps, 0)
    clocks = sampler.stop()
    ms_step = float(np.mean(ms))
    ms_max = reduce_over_ranks(ms_step, world, dev)
    info = infos[-1]
    basis = S.get_basis_info()

    # ---- end to end through the public API with host (pinned) buffers
    bh = torch.from_numpy(b).pin_memory()
    xh = torch.zeros(n, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for k in range(max(1, args.steps)):
        xh.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.solve(bh, xh)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    x_host = xh.numpy()
    err_true = float(np.linalg.norm(x_host - xt) / np.linalg.norm(xt))

    # ---- per-phase device times (CUDA events between the phases of eager outer iterations)
    S.profile(bd, iters=2)
    ph = S.profile(bd, iters=5)
    S.free()

    # ---- classical PCG from the same library
    P = sstep.Solver(A, algo="pcg", **common)
    xp = torch.zeros(n, dtype=torch.float64, device=dev)
    pms, pinfos = timed_solves(P, xp, args.steps, args.warmup)
    P.profile(bd, iters=2)
    pph = P.profile(bd, iters=5)
    P.free()

    # ---- classical PCG in the FP32-basis precision recipe (FP32 p, A p; double-float x, r;
    # FP64 residual replacement every 16 iterations), the comparator of the FP32 s-step forms
    PF = sstep.Solver(A, algo="pcg", precision="fp32_rr", **common)
    xpf = torch.zeros(n, dtype=torch.float64, device=dev)
    pfms, pfinfos = timed_solves(PF, xpf, args.steps, args.warmup)
    PF.profile(bd, iters=2)
    pfph = PF.profile(bd, iters=5)
    PF.free()

    # ---- optional extra s-step configurations
    extra = {}
    x_fp64 = torch.from_numpy(x_host).to(dev)  # the headline FP64 solution
    xe = torch.zeros_like(xd)
    for item in filter(None, args.extra.split(",")):
        parts = item.split(":")
        s_, nu_ = int(parts[0]), int(parts[1])
        prec = parts[2] if len(parts) > 2 else "fp64"
        E = sstep.Solver(A, s=s_, sweeps=nu_, algo="literal" if prec != "fp64" else args.algo,
                         precision=prec, **common)
        ems, einfos = timed_solves(E, xe, 1, 1)
        err = float(torch.linalg.norm(xe - x_fp64) / torch.linalg.norm(x_fp64))
        key = f"s{s_}_nu{nu_}" + ("" if prec == "fp64" else "_" + prec)
        extra[key] = {
            "s": ems[0] / 1e3, "outer_iters": einfos[0].outer_iters,
            "relres_true": einfos[0].relres_true, "rel_diff_vs_fp64_solution": err,
            "time_over_fp64_pcg": ems[0] / float(np.mean(pms))}
        if prec == "fp32_rr":
            extra[key]["time_over_fp32_pcg"] = ems[0] / float(np.mean(pfms))
        if prec == "fp32_rr":  # the FP32 kernels are HBM-bound: GB/s per launch
            E.profile(bd, iters=2)
            fph = E.profile(bd, iters=5)
            F = 4.0 * n
            fb = {"mpk_step": (4 * (s_ - 1) + 2) * F / s_, "gram_b2": 2 * s_ * F,
                  "update_w": (6 * s_ + 6) * F, "update_xr": (s_ + 4) * F}
            fms = {"mpk_step": fph[0] / s_, "gram_b2": fph[1], "update_w": fph[2], "update_xr": fph[3]}
            hbm_, _ = hbm_peak()
            extra[key]["per_kernel"] = {
                k: {"ms_per_launch": fms[k], "GB_s": fb[k] / (fms[k] * 1e-3) / 1e9,
                    "hbm_frac": fb[k] / (fms[k] * 1e-3) / 1e9 / hbm_} for k in fb}
            extra[key]["ms_per_outer"] = float(sum(fph[:4]))
            extra[key]["hbm_frac_whole_outer"] = sum(fb[k] * (s_ if k == "mpk_step" else 1)
                                                     for k in fb) / (sum(fph[:4]) * 1e-3) / 1e9 / hbm_
        E.free()

    grid = run_grid(args.grid, N, dev, sstep, I, torch, b, v0d) if args.grid else None
    small = run_small(args.small, dev, sstep, I, torch,
                      rank == 0 and not args.no_cpu_baseline) if args.small > 0 else None
    batch = run_batch(args.batch, dev, sstep, I, torch, args.batch_shape) if args.batch else None
    q1 = run_q1(args.q1, dev, sstep, I, torch) if args.q1 > 0 else None
    adjoint = run_adjoint(args.adjoint, dev, sstep, I, torch) if args.adjoint > 0 else None
    hpcg = run_hpcg27(args.hpcg, dev, sstep, torch) if args.hpcg > 0 else None

    # ---- roofline of each kernel from the phase times
    work = kernel_work(args.s, n)
    hbm, hbm_src = hbm_peak()
    if args.algo == "literal":
        phases = {"mpk": ph[0], "gram_b2": ph[1], "update_w": ph[2], "update_xr": ph[3]}
        kernels = (("mpk_step", ph[0] / args.s), ("gram_b2", ph[1]), ("update_w", ph[2]),
                   ("update_xr", ph[3]))
        phase_kernel = {"mpk": "mpk_step", "gram_b2": "gram_b2", "update_w": "update_w",
                        "update_xr": "update_xr"}
    else:
        phases = {"mpk": ph[0], "gram": ph[1], "update": ph[2]}
        kernels = (("mpk_step", ph[0] / args.s), ("gram", ph[1]), ("update", ph[2]))
        phase_kernel = {"mpk": "mpk_step", "gram": "gram", "update": "update"}
    per = {}
    for name, t_ms in kernels + (("pcg_spmv_dot", pph[0]), ("pcg_update", pph[1]),
                                 ("pcg_pdir", pph[2])):
        w = work[name]
        per[name] = {"ms_per_launch": t_ms, "GB_s": w["bytes"] / (t_ms * 1e-3) / 1e9,
                     "TFLOP_s": w["flops"] / (t_ms * 1e-3) / 1e12,
                     "hbm_frac": w["bytes"] / (t_ms * 1e-3) / 1e9 / hbm,
                     "fp64_frac": w["flops"] / (t_ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS}
    # the dominant kernel: the largest share of a step's time.  The MPK phase is s launches of
    # two or three kernels (first step, middle steps, last step); its heaviest kernel is the
    # middle-step one, (s - 1) / s of the phase at most.
    share = dict(phases)
    share["mpk"] = phases["mpk"] * max(1, args.s - 1) / args.s
    dom = max(share, key=share.get)
    dom_kernel = phase_kernel[dom]
    d = per[dom_kernel]
    workload = f"poisson7_{N}^3_{args.form}_jacobi_{args.algo}_s{args.s}_nu{args.sweeps}"
    # the counters stay valid only while the kernel's source is the one they were taken on
    kfile = "k_operator.cu" if dom_kernel == "mpk_step" else "k_blas.cu"
    src = source_hash("paper_2603_09790_gb300/csrc/" + kfile, "paper_2603_09790_gb300/csrc/common.cuh")
    traffic = load_traffic(dom_kernel, workload, src)
    roofline = {"bound": "alu", "kernel": dom_kernel, "achieved": d["TFLOP_s"],
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": d["TFLOP_s"] / FP64_PEAK_TFLOPS,
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz",
                "traffic": traffic, "algorithmic_bytes": work[dom_kernel]["bytes"],
                "algorithmic_flops": work[dom_kernel]["flops"],
                "hbm_GB_s": d["GB_s"], "hbm_peak_GB_s": hbm, "hbm_peak_source": hbm_src,
                "hbm_frac": d["hbm_frac"],
                "timing": "CUDA events on the solver's stream between the phases of 5 outer "
                          "iterations launched right after the timed solves"}

    line = {
        "metric": METRIC, "value": ms_max / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload, "n": n, "grid": list(dims), "stencil": 7, "form": args.form,
                   "precond": "jacobi", "algo": args.algo, "s": args.s, "sweeps": args.sweeps,
                   "rtol": 1e-8,
                   "power_iters": 20, "lambda_min": basis["lambda_min"],
                   "lambda_max": basis["lambda_max"], "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2 (each vector 134 MB; working set > 4 GB)"},
        "outer_iters": info.outer_iters, "inner_equiv": info.inner_equiv,
        "relres": info.relres, "relres_true": info.relres_true, "x_rel_error_vs_true": err_true,
        "pcg": {"s": float(np.mean(pms)) / 1e3, "iters": pinfos[-1].outer_iters,
                "relres_true": pinfos[-1].relres_true},
        "sstep_over_pcg_time": ms_step / float(np.mean(pms)),
        "pcg_fp32_rr": {"s": float(np.mean(pfms)) / 1e3, "iters": pfinfos[-1].outer_iters,
                        "relres_true": pfinfos[-1].relres_true, "rr_period": 16,
                        "phase_ms": {"spmv_pap": pfph[0], "update": pfph[1], "pdir": pfph[2]}},
        "setup_s": {"headline_sstep": info.ms_setup / 1e3},
        "configs_fp64_256": grid,
        "poisson5_64x64_csr": small,
        "extra_configs": extra,
        "batched": batch,
        "q1_diffusion": q1,
        "differentiated": adjoint,
        "poisson27_unit_rhs": hpcg,
        "e2e": {"value": float(np.mean(e2e_ms)) / 1e3, "unit": "s", "h2d_bytes_per_step": 16 * n,
                "d2h_bytes_per_step": 8 * n},
        "gpu_launches": int(info.launches),
        "phase_ms_per_outer": phases,
        "per_kernel": per, "roofline": roofline, "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_power, t_outer, t_pcg = oracle_sample(N, args.s, args.sweeps, basis["lambda_max"],
                                                algo=args.algo)
        counts = oracle_counts().get(f"{args.algo}_s{args.s}nu{args.sweeps}")
        n_outer = counts["iters"] if counts and N == 256 else info.outer_iters
        v = t_power + t_outer * n_outer
        line["cpu_baseline"] = {
            "value": v, "unit": "s", "cores": 1, "kind": "oracle",
            "sample": f"2 power + 2 outer iterations + 8 PCG iterations of the FP64 C oracle at {N}^3 "
                      f"(single thread), extrapolated to 20 power and {n_outer} outer iterations",
            "pcg_value": t_pcg * (oracle_counts().get("pcg", {}).get("iters") or pinfos[-1].outer_iters),
            "cpu": cpu_model()}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
