#!/usr/bin/env python
"""Benchmark: time per right-hand side of the deflated mixed-precision HISQ
propagator solve on one GB300, next to plain mixed-precision CG on the same GPU.

Workload (synthetic stand-in for the paper's MILC ensembles, Section 2 Table 1),
by default the largest single-GPU one, in the light-mass regime: 64^3 x 96
lattice, thin links exp(i 0.25 A) (seed 4), fat = 9/8 U, long = -1/24 UUU (two
rows stored, the third rebuilt), antiperiodic time, m = 0.0008, 200 eigenpairs
of the squared massless even-site operator (block thick-restart Lanczos) stored
in FP16, 12 right-hand sides per step (4 Gaussian sources x 3 colours) solved
together.  One step = one batch through the whole hot path: source preparation,
deflated initial guesses (Eq. 4, tensor-core GEMMs), sloppy CG with FP64
reliable updates and re-deflation (Section 3), odd reconstruction and the FP64
full residual, to |eta - M psi| / |eta| <= 1e-10.  Link upload and the
eigensolve are setup (excluded from the solve time, as in the paper) and
reported separately.  Plain mixed-precision CG on the same GPU is timed the
same way (warm-up steps, CUDA events on the solve stream, the same step count).
--config c2 / c3 select the 32^3 x 64 single-RHS and 24-RHS workloads.

usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs independent replicas (different sources); the
time is the max over ranks and value = time / (right-hand sides of all ranks).
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time/RHS to 1e-10 residual, deflated vs plain CG on 1 GB300; Dslash HBM GB/s"
SOURCE_SEED = 11
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", default="c5")
    ap.add_argument("--sloppy", type=int, default=16, help="sloppy colour-vector storage: 32 or 16")
    ap.add_argument("--recon", type=int, default=12, help="long links: 18 reals, 12 (two rows + SU(3) row) or 8 (a2, a3, b1 and two phases)")
    ap.add_argument("--links", type=int, default=32, help="sloppy link storage: 32 or 16")
    ap.add_argument("--reliable", type=int, choices=[64, 48], default=64,
                    help="reliable-update residual arithmetic of the headline: 64 (FP64, the paper's) or 48 "
                         "(double-float on the FP32 units, certified in FP64); the other one is timed beside it "
                         "where its links fit (not at c5)")
    ap.add_argument("--n-ev", type=int, default=None)
    ap.add_argument("--n-kr", type=int, default=None)
    ap.add_argument("--cheby", type=int, default=60)
    ap.add_argument("--amin", type=float, default=-2.0,
                    help="Chebyshev window edge: > 0 given, -f: where about f n_ev eigenvalues lie below it")
    ap.add_argument("--eig-tol", type=float, default=1e-6)
    ap.add_argument("--eig-cache", default=None, metavar="PATH",
                    help="save the eigenpairs to PATH after the eigensolve, or reload them from it if it exists")
    ap.add_argument("--eig-block", type=int, default=64,
                    help="eigensolver block size (1: thick-restart Lanczos; b: block thick-restart Lanczos)")
    ap.add_argument("--eig-prec", type=int, default=None,
                    help="eigenvector storage: 32 (FP32), 16 (FP16 + per-site scale), 15 (BF16), 14 (FP16 x 2^e); "
                         "default FP16 x 2^e for c5, BF16 for c3, FP32 otherwise")
    ap.add_argument("--plain-steps", type=int, default=None,
                    help="timed steps of the plain-CG comparison (default: --steps)")
    ap.add_argument("--plain-warmup", type=int, default=None,
                    help="warm-up steps of the plain-CG comparison (default: --warmup)")
    ap.add_argument("--e2e-steps", type=int, default=3, help="steps of the end-to-end host-API measurement")
    ap.add_argument("--persistent", type=int, choices=[0, 1], default=0,
                    help="batched solves: 1 = one cooperative launch per stretch of sloppy iterations, "
                         "0 = three launches per iteration replayed as CUDA graphs")
    ap.add_argument("--source-pool-gb", type=float, default=30.0,
                    help="device memory for distinct source batches (cycled over the steps)")
    ap.add_argument("--cpu-iters", type=int, default=2, help="oracle CG iterations per CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--learned", action="store_true", help="learned initial guess workload (24^3x48)")
    ap.add_argument("--learned-pairs", type=int, default=512)
    ap.add_argument("--learned-epochs", type=int, default=30)
    ap.add_argument("--learned-lr", type=float, default=2e-3)
    ap.add_argument("--sweep", choices=["delta_tr", "mass", "cheby"], default=None,
                    help="precision/re-deflation sweep (Fig. 2 analogue) or iterations vs mass (Fig. 1 analogue) "
                         "on the 32^3x64 lattice; prints one JSON line per table")
    ap.add_argument("--capture", action="store_true",
                    help="profiler-capture run: --iters CG iterations (no timing, no JSON line)")
    ap.add_argument("--iters", type=int, default=4, help="--capture: CG iterations")
    ap.add_argument("--mrhs", type=int, default=0, help="--capture: solve this many Gaussian RHS together")
    ap.add_argument("--tc", type=int, default=0, help="--capture: also run the tensor-core batched deflation "
                                                      "with this many random eigenvectors (24 RHS)")
    ap.add_argument("--tc-prec", type=int, default=32, help="--capture: eigenvector storage for --tc (32, 15, 14)")
    ap.add_argument("--mrhs-shape", default=None, metavar="KIND,R,BUDGET",
                    help="--capture: fixed launch shape of the batched operator (hisq_set_batched_kernel)")
    ap.add_argument("--traffic-from", default=None, metavar="REPORT",
                    help="--capture: write profiles/dslash_traffic.json from an ncu report of a capture run")
    ap.add_argument("--traffic-key", default="s16_r12", help="--capture: key suffix (sloppy bits, recon)")
    ap.add_argument("--traffic-command", default="", help="--capture: the ncu command that made the report")
    ap.add_argument("--rhs-per-step", type=int, default=None,
                    help="right-hand sides solved together per step (batched); default 1, 24 for c3, 12 for c5")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def replica_time(elapsed_ms: float, steps: int, device="cpu"):
    """Replicas only: every rank solves its own right-hand sides; the job time is
    the slowest rank's and value = time / (right-hand sides of all ranks).
    Returns (max elapsed ms, ms per RHS of the whole job)."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    if world > 1:
        t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    return elapsed_ms, elapsed_ms / (steps * world)


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "of measured"
    except Exception:
        return FALLBACK_HBM_GBS, "of fallback"


def kernel_source_hash():
    from paper_2502_00152_gb300.build import dslash_source_hash

    return dslash_source_hash()


def ncu_traffic(kernel_key: str, sites: int):
    """dram bytes per launch of the Dslash from the committed ncu summary, if it
    was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "dslash_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("kernel_source_hash") != kernel_source_hash():
            return None
        per_site = d["dram_bytes_per_output_site"].get(kernel_key)
        return None if per_site is None else per_site * sites
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for r in csv.reader(io.StringIO(f.read())):
                if len(r) >= 9:
                    rows.append([x.strip() for x in r])
        os.unlink(self.path)
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        smax = max((float(r[2]) for r in rows if r[2].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows)}


def link_bytes_per_site(recon: int, link_prec: int = 32) -> int:
    # 8 fat + 8 long hop matrices of 18 reals (12 or 8 for the long ones with recon 12 or 8)
    rb = link_prec // 8
    return 8 * 18 * rb + 8 * recon * rb


def spinor_bytes_per_site(prec: int) -> int:
    return {64: 48, 32: 24, 16: 16}[prec]


# ------------------------------------------------------------------ our arm
def run_ours(a):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_2502_00152_gb300 import build as B

    if rank == 0:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2502_00152_gb300 import hisq as H
    from paper_2502_00152_gb300 import inputs as I

    cfg = I.lattice_config(a.config)
    dims, m, tol = cfg["dims"], cfg["mass"], cfg["tol"]
    V = I.volume(dims)
    Vh = V // 2
    n_ev = a.n_ev if a.n_ev is not None else cfg.get("n_ev", 0)
    if a.eig_prec is None:
        a.eig_prec = {"c5": H.HISQ_PREC_HALF_EV, "c3": H.HISQ_PREC_BF16}.get(a.config, 32)
    eig_name = {32: "FP32", 16: "FP16 + per-site scale", 15: "BF16", 14: "FP16"}.get(a.eig_prec, str(a.eig_prec))
    n_kr = a.n_kr if a.n_kr is not None else max(int(1.5 * n_ev), n_ev + 32)

    t0 = time.time()
    fat, lng = I.hisq_links(dims, cfg["seed"], cfg["eps"])
    t_links = time.time() - t0
    # the library works on a stream of its own (not the legacy default stream),
    # so that its CG iterations are captured and replayed as CUDA graphs
    stream = torch.cuda.Stream(device=local)
    torch.cuda.set_stream(stream)
    ctx = H.hisq_create(dims, t_antiperiodic=True, device=local, cuda_stream=stream.cuda_stream)
    H.hisq_load_links(ctx, fat, lng, long_recon=a.recon, long_scale=I.C3_NAIK if a.recon != 18 else 1.0)
    H.hisq_set_mass(ctx, m)

    # setup: eigensolve (excluded from the solve time, reported), or the pairs
    # of an earlier run reloaded from --eig-cache (eigenvalues recomputed as FP64
    # Rayleigh quotients on load, as the paper recomputes them from stored vectors)
    eig = {}
    cache_info = (a.eig_cache + ".json") if a.eig_cache else None
    if n_ev > 0 and a.eig_cache and os.path.exists(a.eig_cache) and os.path.exists(cache_info):
        torch.cuda.synchronize()
        t0 = time.time()
        H.hisq_load_eigvecs(ctx, a.eig_cache)
        torch.cuda.synchronize()
        with open(cache_info) as f:
            eig = json.load(f)
        eig["loaded_from_cache_seconds"] = round(time.time() - t0, 2)
    elif n_ev > 0:
        ep = H.hisq_default_eig_params(n_ev=n_ev, n_kr=n_kr, tol=a.eig_tol, max_restarts=100, cheby_degree=a.cheby,
                                       a_min=a.amin, a_max=0.0, storage_precision=a.eig_prec, seed=1000 + rank,
                                       block_size=a.eig_block)
        torch.cuda.synchronize()
        t0 = time.time()
        eps, nconv = H.hisq_eigensolve(ctx, ep)
        torch.cuda.synchronize()
        eig = dict(seconds=round(time.time() - t0, 2), n_ev=n_ev, n_kr=n_kr, block_size=a.eig_block,
                   converged=nconv, cheby_degree=a.cheby, eps_min=float(eps[0]), eps_max=float(eps[-1]),
                   storage=eig_name)
        if a.eig_cache:
            H.hisq_save_eigvecs(ctx, a.eig_cache)
            with open(cache_info, "w") as f:
                json.dump(eig, f)

    # sources: resident in HBM before the timed region (FP64 full-lattice fields)
    keep_links = (fat, lng) if (rank == 0 and world == 1 and not a.no_cpu_baseline) else (None, None)
    kps = a.rhs_per_step if a.rhs_per_step is not None else {"c3": 24, "c5": 12}.get(a.config, 1)
    plain_steps = a.steps if a.plain_steps is None else a.plain_steps
    plain_warmup = a.warmup if a.plain_warmup is None else a.plain_warmup
    # a pool of distinct source batches, resident in HBM, cycled over the steps
    # (a 12-RHS batch of the largest lattice is 14.5 GB of FP64 fields)
    batch_bytes = V * 48 * kps
    nsrc = max(1, min(a.warmup + a.steps, int(a.source_pool_gb * 1e9 // batch_bytes)))
    if kps == 1:
        srcs = [I.gaussian_source(dims, SOURCE_SEED, rank * 1000 + k) for k in range(nsrc)]
    elif a.config == "c5":
        # Gaussian sources x 3 colours (colour-diluted)
        srcs = [np.stack([I.gaussian_colour_source(dims, SOURCE_SEED, (rank * 1000 + k) * 64 + q // 3, q % 3)
                          for q in range(kps)]) for k in range(nsrc)]
    else:
        # Z2 wall sources: 8 timeslices x 3 colours per 24 right-hand sides
        srcs = [np.stack([I.z2_wall_source(dims, SOURCE_SEED + 97 * (rank * 1000 + k) + q // 24, (q % 24) // 3, q % 3)
                          for q in range(kps)]) for k in range(nsrc)]
    eta_dev = [torch.from_numpy(s).to(f"cuda:{local}") for s in srcs]
    if keep_links[0] is None:
        del fat, lng
    psi_dev = torch.zeros_like(eta_dev[0])
    rel_prec = a.reliable
    def params(deflate, rel):
        return H.hisq_default_solve_params(tol=tol, precision_sloppy=a.sloppy, link_precision_sloppy=a.links,
                                           deflate=deflate, compute_full_residual=1, precision_reliable=rel,
                                           persistent=a.persistent)
    prm_defl = params(1 if n_ev > 0 else 0, rel_prec)
    prm_plain = params(0, rel_prec)

    def solve(k, prm):
        st, status = H.hisq_solve_device(ctx, eta_dev[k], psi_dev, kps, prm)
        if status != H.HISQ_OK:
            raise RuntimeError(f"solve did not converge: {st}")
        if kps == 1:
            return st[0]
        agg = dict(st[0])
        for key in ("iterations", "reliable_updates", "redeflations", "profiled_iterations"):
            agg[key] = max(s[key] for s in st)
        agg["profiled_rhs_launches"] = sum(s["profiled_iterations"] for s in st)
        for key in ("seconds_dslash_oe", "seconds_dslash_eo"):
            agg[key] = sum(s[key] for s in st)
        agg["full_residual"] = max(s["full_residual"] for s in st)
        return agg

    def timed(prm, warmup, steps, profile=False, sample_clocks=False):
        """warm-up steps, then `steps` steps between CUDA events on the solve
        stream (a barrier and a synchronize on both sides); ms per step"""
        for k in range(warmup):
            solve(k % nsrc, prm)
        H.hisq_set_profiling(ctx, profile)
        clocks = Clocks(local) if sample_clocks else None
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        l0 = H.hisq_kernel_launches(ctx)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed")
        ev0.record(stream)
        st = [solve((warmup + k) % nsrc, prm) for k in range(steps)]
        ev1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        launches = H.hisq_kernel_launches(ctx) - l0
        clk = clocks.stop() if clocks else None
        H.hisq_set_profiling(ctx, False)
        elapsed_ms, per_rhs = replica_time(ev0.elapsed_time(ev1), max(steps, 1) * kps, f"cuda:{local}")
        return st, elapsed_ms, per_rhs, launches, clk

    # headline: the deflated solve
    stats, elapsed_ms, value, launches, clk = timed(prm_defl, a.warmup, a.steps, profile=True, sample_clocks=True)
    fp64_s, fp64_n = H.hisq_profiled_fp64(ctx)  # the FP64 Dslash launches of the timed steps
    if world > 1:
        torch.distributed.barrier()
    ms_per_step = elapsed_ms / a.steps  # one step = kps right-hand sides
    # plain mixed-precision CG on the same GPU, timed the same way
    plain, _, plain_ms, _, _ = timed(prm_plain, plain_warmup, plain_steps) if plain_steps > 0 else ([], 0, None, 0, None)

    # end to end through the host API: pinned host source -> psi on the host
    pin_eta = torch.from_numpy(np.ascontiguousarray(srcs[a.warmup % nsrc])).pin_memory()
    pin_psi = torch.empty_like(pin_eta).pin_memory()  # the result lands in pinned host memory
    e2e_ms = []
    for k in range(max(1, a.e2e_steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, st_h, status = H.hisq_solve(ctx, pin_eta.numpy(), prm_defl, out=pin_psi.numpy())
        e2e_ms.append((time.perf_counter() - t0) * 1e3 / kps)
        if status != H.HISQ_OK:
            raise RuntimeError("host-API solve did not converge")

    # the same solves with the other reliable-update arithmetic (comparison);
    # the double-float links need as much memory as the FP64 copy (2304 B per
    # site), which the largest workload does not have left
    other = 64 if rel_prec != 64 else H.HISQ_PREC_DF64
    mem = {"library_bytes_before_comparison": H.hisq_device_bytes(ctx),
           "device_free_bytes_before_comparison": torch.cuda.mem_get_info(local)[0]}
    try:
        s2, e2, v2, _, _ = timed(params(1 if n_ev > 0 else 0, other), 1, max(1, min(2, a.steps)))
        other_rel = {"ms_per_rhs": round(v2, 3), "iterations": [x["iterations"] for x in s2],
                     "reliable_updates": [x["reliable_updates"] for x in s2],
                     "true_residual_max": max(x["full_residual"] for x in s2)}
    except Exception as e:  # e.g. no room for the double-float links
        other_rel = {"unavailable": str(e)[:200]}
    mem["library_bytes_after_comparison"] = H.hisq_device_bytes(ctx)

    # Dslash roofline from the event-timed kernels of the timed solves
    it = sum(s["profiled_iterations"] for s in stats)
    t_oe = sum(s["seconds_dslash_oe"] for s in stats) / max(it, 1)
    t_eo = sum(s["seconds_dslash_eo"] for s in stats) / max(it, 1)
    sp = spinor_bytes_per_site(a.sloppy)
    lb = link_bytes_per_site(a.recon, a.links)
    bytes_oe = Vh * (lb + 2 * sp)
    xb = 24  # FP32 x in the fused update
    bytes_eo = Vh * (lb + sp + sp + 2 * sp + 2 * xb)
    peak, peak_src = measured_peak_hbm()
    ach = bytes_oe / t_oe / 1e9 if t_oe > 0 else None
    key = f"oe_s{a.sloppy}_r{a.recon}" + ("" if a.links == 32 else f"_l{a.links}")
    traffic = ncu_traffic(key, Vh)
    flops_site = 1146
    res_max = max(s["full_residual"] for s in stats)
    if kps == 1:
        roof = {
            "bound": "hbm", "achieved": None if ach is None else round(ach, 1), "peak": peak, "unit": "GB/s",
            "frac": None if ach is None else round(ach / peak, 4), "traffic": traffic,
            "peak_source": peak_src, "kernel": "k_dslash D_oe (tmp = D_oe p, |tmp|^2)",
            "algorithmic_bytes_per_launch": bytes_oe, "launch_us": round(t_oe * 1e6, 2),
            "fused_eo_kernel": {"algorithmic_bytes_per_launch": bytes_eo, "launch_us": round(t_eo * 1e6, 2),
                                "achieved_gbs": round(bytes_eo / t_eo / 1e9, 1) if t_eo > 0 else None},
            "dslash_gflops": round(flops_site * Vh / t_oe / 1e9, 1) if t_oe > 0 else None,
        }
    else:
        # batched D_oe kernel: one launch serves every active right-hand side;
        # at 12-24 RHS its intensity (8-14 flop/B) is at or past the FP32 ridge,
        # so the bound is the FP32 FMA rate: 152 SMs x 128 lanes x 2 flop x 2.07 GHz
        n_launch = sum(s["profiled_iterations"] for s in stats)
        rhs_launch = sum(s["profiled_rhs_launches"] for s in stats)
        t_all = sum(s["seconds_dslash_oe"] for s in stats)
        t_all_eo = sum(s["seconds_dslash_eo"] for s in stats)
        peak32 = 152 * 128 * 2 * 2.07e9 / 1e12
        tf = flops_site * Vh * rhs_launch / t_all / 1e12 if t_all > 0 else None
        roof = {
            "bound": "alu", "achieved": None if tf is None else round(tf, 2), "peak": round(peak32, 1),
            "unit": "TFLOP/s", "frac": None if tf is None else round(tf / peak32, 4),
            "traffic": ncu_traffic(f"mrhs{kps}_oe_s{a.sloppy}_r{a.recon}", Vh),
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (nominal clock)",
            "kernel": f"k_dslash_mrhs D_oe ({kps} RHS per launch)",
            "flops_per_rhs_site": flops_site,
            "launch_us": round(t_all / max(n_launch, 1) * 1e6, 2),
            "mean_rhs_per_launch": round(rhs_launch / max(n_launch, 1), 2),
            "hbm_view": {"algorithmic_bytes_per_launch": Vh * (lb + 2 * sp * kps),
                         "achieved_gbs": round(Vh * (lb * n_launch + 2 * sp * rhs_launch) / t_all / 1e9, 1)
                         if t_all > 0 else None, "peak": peak},
            "fused_eo_kernel": {"launch_us": round(t_all_eo / max(n_launch, 1) * 1e6, 2),
                                "achieved_tflops": round(flops_site * Vh * rhs_launch / t_all_eo / 1e12, 2)
                                if t_all_eo > 0 else None},
        }

    # the FP64 Dslash (reliable-update residuals, source preparation, odd
    # reconstruction, residual checks) is FP64-ALU bound: 1146 flop per output
    # site against GB300's nominal 1.25 TFLOP/s FP64 rate
    if fp64_n > 0 and fp64_s > 0:
        tf64 = flops_site * Vh * fp64_n / fp64_s / 1e12
        roof["fp64_dslash_kernel"] = {
            "kernel": "k_dslash FP64 (reliable updates, source preparation, reconstruction, residual checks)",
            "launches": fp64_n, "launch_us": round(fp64_s / fp64_n * 1e6, 2), "achieved_tflops": round(tf64, 3),
            "peak": 1.25, "peak_source": "nominal GB300 dense FP64 rate", "frac": round(tf64 / 1.25, 4),
            "share_of_timed": round(fp64_s * 1e3 / elapsed_ms, 4)}
    rel_name = "FP64 reliable updates" if rel_prec == 64 else "double-float reliable updates, final residual in FP64"
    out = {
        "metric": METRIC,
        "value": round(value, 4),
        "unit": "ms/RHS",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if a.sloppy != 64 else "f64",
        "data": "synthetic",
        "config": {
            "workload": f"HISQ {dims[0]}^3x{dims[3]}, m={m}, {n_ev} eigenpairs ({eig_name}), deflated "
                        f"mixed-precision CG (FP{a.sloppy} vectors, FP{a.links} links recon {a.recon}, {rel_name}), "
                        + ("1 Gaussian RHS per step" if kps == 1 else
                           (f"{kps} RHS per step ({kps // 3} Gaussian sources x 3 colours), batched"
                            if a.config == "c5" else f"{kps} Z2 wall RHS per step, batched"))
                        + f", tol {tol}",
            "rhs_per_step": kps,
            "lattice": list(dims), "mass": m, "n_ev": n_ev, "eigenvectors": eig_name,
            "sloppy_vectors": f"fp{a.sloppy}", "links": f"fp{a.links} recon {a.recon}",
            "l2": "inputs larger than L2 (links and eigenvectors are GBs)",
            "parallelism": f"replicas{world}",
            "graphs": ("off (persistent launch)" if a.persistent and kps > 1 else
                       "on (CG iterations replayed as CUDA graphs on the library's stream)"),
            "persistent": "on (one cooperative launch per stretch of sloppy iterations)" if a.persistent and kps > 1
                          else "off",
            "sources": f"{nsrc} distinct batches resident in HBM, cycled over the steps",
        },
        "roofline": roof,
        "e2e": {"value": round(sorted(e2e_ms)[len(e2e_ms) // 2], 4), "unit": "ms/RHS",
                "h2d_bytes_per_step": V * 48 * kps, "d2h_bytes_per_step": V * 48 * kps,
                "steps": len(e2e_ms)},
        "gpu_launches": int(launches),
        "clocks": clk,
        "plain_cg": {"ms_per_rhs": None if plain_ms is None else round(plain_ms, 3),
                     "iterations": [s["iterations"] for s in plain], "steps": plain_steps, "warmup": plain_warmup,
                     "timing": "CUDA events on the solve stream after warm-up, as the headline"},
        "speedup_vs_plain_cg": round(plain_ms / value, 3) if plain_ms and value > 0 else None,
        "reliable_updates_arithmetic": "fp64" if rel_prec == 64 else "double-float (FP32 hi+lo), FP64-confirmed",
        ("double_float_reliable_updates" if other == H.HISQ_PREC_DF64 else "fp64_reliable_updates"): other_rel,
        "iterations_deflated": [s["iterations"] for s in stats],
        "reliable_updates": [s["reliable_updates"] for s in stats],
        "redeflations": [s["redeflations"] for s in stats],
        "true_residual_max": res_max,
        "eigensolve": eig,
        "eigensolve_break_even_rhs": (round(eig["seconds"] * 1e3 / (plain_ms - value), 1)
                                      if eig and plain_ms and plain_ms > value else None),
        "link_generation_s": round(t_links, 2),
        "device_memory": mem,
    }
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(a, dims, cfg, 1, *keep_links)
    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------ oracle timing
def oracle_iterations(name: str):
    path = os.path.join(ROOT, "tests", "golden", f"oracle_plain_cg_{name}.json")
    try:
        with open(path) as f:
            return int(json.load(f)["iterations"]), "oracle plain CG iteration count from tests/golden"
    except Exception:
        return None, "no stored oracle iteration count"


_ORACLE_CACHE = {}


def cpu_baseline(a, dims, cfg, samples: int = 1, fat=None, lng=None):
    """The FP64 oracle as it stands, on the host cores: time per CG iteration on
    the benchmark workload (a bounded sample of a.cpu_iters iterations), scaled
    to one right-hand side by the oracle's iteration count."""
    from oracle.oracle import Oracle, num_threads
    from paper_2502_00152_gb300 import inputs as I

    key = (tuple(dims), cfg["seed"], cfg["eps"], cfg["mass"])
    if key not in _ORACLE_CACHE:
        if fat is None:
            fat, lng = I.hisq_links(dims, cfg["seed"], cfg["eps"])
        o = Oracle(dims, fat, lng, t_antiperiodic=True)
        eta = I.gaussian_source(dims, SOURCE_SEED, 0)
        _ORACLE_CACHE.clear()
        _ORACLE_CACHE[key] = (o, o.prepare_source(cfg["mass"], eta))
    o, b = _ORACLE_CACHE[key]
    per_it = []
    for _ in range(samples):
        t0 = time.perf_counter()
        o.cg(cfg["mass"], b, None, 1e-300, maxiter=a.cpu_iters)
        per_it.append((time.perf_counter() - t0) / (a.cpu_iters + 2))  # + initial and final residual applies
    n_it, src = oracle_iterations(a.config)
    t_it = min(per_it)
    return {"value": round(t_it * n_it * 1e3, 1) if n_it else None, "unit": "ms/RHS", "cores": num_threads(),
            "threads": num_threads(), "nproc": os.cpu_count(), "kind": "oracle",
            "sample": f"{a.cpu_iters} FP64 oracle CG iterations on the full {dims[0]}^3x{dims[3]} lattice "
                      f"({t_it * 1e3:.1f} ms per iteration incl. residual applies), x {n_it} iterations "
                      f"({src}); extrapolated, plain CG without deflation"}


def run_reference(a):
    rank, world, local = dist_env()
    if rank != 0:
        return
    from oracle import build as OB
    from paper_2502_00152_gb300 import inputs as I

    OB.build()
    cfg = I.lattice_config(a.config)
    dims = cfg["dims"]
    fat, lng = I.hisq_links(dims, cfg["seed"], cfg["eps"])
    for _ in range(a.warmup):
        cpu_baseline(a, dims, cfg, 1, fat, lng)
    vals = []
    t0 = time.time()
    for _ in range(a.steps):
        vals.append(cpu_baseline(a, dims, cfg, 1, fat, lng))
    wall = time.time() - t0
    v = sorted(x["value"] for x in vals if x["value"] is not None)
    value = v[len(v) // 2] if v else None
    cb = dict(vals[-1])
    cb["value"] = value
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ms/RHS", "n_gpus": world,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(wall * 1e3 / a.steps, 1),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"HISQ {dims[0]}^3x{dims[3]}, m={cfg['mass']}, plain FP64 CG (oracle), "
                                  f"1 Gaussian RHS per step, tol {cfg['tol']}", "lattice": list(dims)},
           "cpu_baseline": cb,
           "e2e": {"value": value, "unit": "ms/RHS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------ profiler captures
def run_capture(a):
    """A few CG iterations on a benchmark lattice, in the launch configuration of
    the solve, for a profiler to capture the kernels (ncu -k ... -c ...): source
    preparation and initial residual (three FP64 Dslash launches), then per CG
    iteration the D_oe kernel, the fused D_eo + update kernel and the direction
    update; --mrhs K solves K Gaussian right-hand sides together (batched
    operator); --tc N also runs the tensor-core batched deflation twice with N
    random orthonormalised eigenvectors and 24 right-hand sides.
    --traffic-from REPORT instead writes profiles/dslash_traffic.json from an ncu
    report of such a run."""
    from paper_2502_00152_gb300 import build as B
    from paper_2502_00152_gb300 import hisq as H
    from paper_2502_00152_gb300 import inputs as I

    if a.traffic_from:
        out = os.path.join(ROOT, "profiles", "dslash_traffic.json")
        write_traffic(a.traffic_from, a.config, a.traffic_key, out, a.traffic_command, a.mrhs)
        return
    B.build()
    c = I.lattice_config(a.config)
    dims = c["dims"]
    fat, lng = I.hisq_links(dims, c["seed"], c["eps"])
    ctx = H.hisq_create(dims, t_antiperiodic=True, device=0)
    H.hisq_load_links(ctx, fat, lng, long_recon=a.recon, long_scale=I.C3_NAIK if a.recon != 18 else 1.0)
    H.hisq_set_mass(ctx, c["mass"])
    if a.mrhs_shape:
        H.hisq_set_batched_kernel(ctx, *[int(x) for x in a.mrhs_shape.split(",")])
    if a.mrhs > 1:
        import numpy as np

        eta = np.stack([I.gaussian_source(dims, 11, j) for j in range(a.mrhs)])
    else:
        eta = I.gaussian_source(dims, 11, 0)
    prm = H.hisq_default_solve_params(tol=1e-14, max_iter=a.iters, precision_sloppy=a.sloppy,
                                      compute_full_residual=0, batch=1 if a.mrhs > 1 else 0,
                                      precision_reliable=a.reliable)
    _, st, status = H.hisq_solve(ctx, eta, prm)
    print(f"{a.config} {dims}: {st[0]['iterations']} iterations, status {status}")
    if a.tc > 0:
        import numpy as np

        from paper_2502_00152_gb300.inputs import random_normal

        V = I.volume(dims)
        par = (np.indices(dims[::-1]).sum(axis=0) & 1).reshape(-1)
        vecs = random_normal(5, 77, 0, 6 * V * a.tc).reshape(a.tc, V, 3, 2)
        vecs = vecs[..., 0] + 1j * vecs[..., 1]
        vecs[:, par == 1] = 0
        vecs /= np.linalg.norm(vecs.reshape(a.tc, -1), axis=1)[:, None, None]
        H.hisq_set_eigvecs(ctx, vecs, np.linspace(0.01, 0.1, a.tc), a.tc_prec)
        bs = np.stack([I.gaussian_field(dims, 40 + j) for j in range(24)])
        for _ in range(2):
            H.hisq_deflate_batch(ctx, bs)
        print(f"tensor-core deflation: {a.tc} vectors x 24 right-hand sides done")
    ctx.close()


def write_traffic(report: str, config: str, key: str, out: str, command: str, mrhs: int = 0) -> None:
    """Per-output-site DRAM bytes of the sloppy Dslash launches in an ncu report
    of this driver: the single-RHS D_oe (EpiXpay) and fused D_eo + update (EpiCG)
    kernels, or with mrhs = K the batched ones (BEpiStore, BEpiCG) for K
    right-hand sides, keyed "mrhsK_...".  Entries are merged into `out` when it
    was written on the same kernel sources (the hash of the Dslash sources is
    stored with them; the benchmark uses them only while it matches)."""
    import csv
    import io
    import json
    import subprocess

    from paper_2502_00152_gb300 import inputs as I
    from paper_2502_00152_gb300.build import dslash_source_hash

    txt = subprocess.run(["ncu", "-i", report, "--page", "raw", "--csv"], check=True, capture_output=True,
                         text=True).stdout
    rows = list(csv.reader(io.StringIO(txt)))
    hdr, data = rows[0], rows[2:]
    col = {n: hdr.index(n) for n in ("Kernel Name", "dram__bytes_read.sum", "dram__bytes_write.sum")}
    units = rows[1]
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    dims = I.lattice_config(config)["dims"]
    dims_s = f"{dims[0]}^3x{dims[3]}"
    vh = I.volume(dims) // 2
    per_site = {}
    for r in data:
        name = r[col["Kernel Name"]]
        if "k_dslash_mrhs" in name:
            kind = "oe" if "BEpiStore" in name else ("eo" if "BEpiCG" in name else None)
            prefix = f"mrhs{mrhs}_"
        else:
            kind = "oe" if "EpiXpay" in name else ("eo" if "EpiCG" in name else None)
            prefix = ""
        if kind is None or (prefix != "") != (mrhs > 1):
            continue
        b = sum(float(r[col[m]].replace(",", "")) * scale[units[col[m]]]
                for m in ("dram__bytes_read.sum", "dram__bytes_write.sum"))
        per_site.setdefault(f"{prefix}{kind}_{key}", []).append(b / vh)
    h = dslash_source_hash()
    doc = {"what": "DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per output site of the sloppy Dslash "
                   "kernels (keys mrhsK_...: the batched kernel for K right-hand sides), from ncu captures on the "
                   f"{dims_s} lattice (Vh = {vh}); traffic scales with the number of output sites, so the benchmark "
                   "multiplies by its own Vh",
           "commands": [], "kernel_source_hash": h, "dram_bytes_per_output_site": {}}
    try:
        with open(out) as f:
            old = json.load(f)
        if old.get("kernel_source_hash") == h:
            doc["commands"] = list(old.get("commands", []))
            doc["dram_bytes_per_output_site"].update(old.get("dram_bytes_per_output_site", {}))
    except (OSError, ValueError):
        pass
    if command and command not in doc["commands"]:
        doc["commands"].append(command)
    doc["dram_bytes_per_output_site"].update({k: round(sum(v) / len(v), 1) for k, v in per_site.items()})
    with open(out, "w") as f:
        json.dump(doc, f, indent=1)
    print(json.dumps(doc["dram_bytes_per_output_site"]))



# ------------------------------------------------------------ learned guess
def run_learned(a):
    """24^3 x 48, m = 0.003, 128 eigenpairs; the parallel-transport network is
    trained on (eta, psi) pairs from the deflated solver (Gaussian sources, seed
    3) and a held-out set of right-hand sides is solved from a zero guess, from
    the deflated guess, and from deflation plus the network's guess, all to the
    same 1e-10 FP64 true residual."""
    import numpy as np
    import torch

    from paper_2502_00152_gb300 import build as B
    from paper_2502_00152_gb300 import hisq as H
    from paper_2502_00152_gb300 import inputs as I
    from paper_2502_00152_gb300.learned import GuessNet

    B.build()
    cfg = I.lattice_config("c4")
    dims, m = cfg["dims"], cfg["mass"]
    V = I.volume(dims)
    fat, lng = I.hisq_links(dims, cfg["seed"], cfg["eps"])
    ctx = H.hisq_create(dims, True, 0, torch.cuda.current_stream().cuda_stream)
    H.hisq_load_links(ctx, fat, lng, long_recon=a.recon, long_scale=I.C3_NAIK if a.recon != 18 else 1.0)
    H.hisq_set_mass(ctx, m)
    del fat, lng
    t0 = time.time()
    H.hisq_eigensolve(ctx, H.hisq_default_eig_params(n_ev=cfg["n_ev"], n_kr=int(1.5 * cfg["n_ev"]), tol=1e-6,
                                                     max_restarts=100, cheby_degree=a.cheby, a_min=a.amin))
    t_eig = time.time() - t0
    prm = H.hisq_default_solve_params(deflate=1, batch=1, precision_sloppy=a.sloppy)
    par = torch.from_numpy((np.indices(dims[::-1]).sum(axis=0) & 1).reshape(-1)).cuda()
    even = (par == 0).to(torch.complex64)[None, :, None]
    par_np = par.cpu().numpy()
    n_pairs = a.learned_pairs
    # training pairs (seed 3): psi from the batched deflated solver, deflated guess from the library
    t0 = time.time()
    X, T = [], []
    for k0 in range(0, n_pairs, 24):
        kb = min(24, n_pairs - k0)
        etas = np.stack([I.gaussian_source(dims, 3, k0 + q) for q in range(kb)])
        psi, st, s = H.hisq_solve(ctx, etas, prm)
        for q in range(kb):
            # target: the part of psi_e the deflated guess does not give
            xd = H.hisq_deflate(ctx, _even_rhs(H, ctx, etas[q], m, par_np))
            tgt = psi[q] * (par_np == 0)[:, None] - xd
            X.append(etas[q].astype(np.complex64))
            T.append(tgt.astype(np.complex64))
    t_pairs = time.time() - t0
    samples = [(torch.from_numpy(np.stack(X[i:i + 3])).cuda(), torch.from_numpy(np.stack(T[i:i + 3])).cuda())
               for i in range(0, len(X) - 2, 3)]
    net = GuessNet(ctx, seed=1, bf16=True)
    t0 = time.time()
    losses = []
    for ep in range(a.learned_epochs):
        el = [net.train_step(x, t, even, lr=a.learned_lr) for x, t in samples]
        losses.append(float(np.mean(el)))
    torch.cuda.synchronize()
    t_train = time.time() - t0
    # held-out right-hand sides
    etas = np.stack([I.gaussian_source(dims, 3, 100000 + q) for q in range(24)])
    eta_dev = torch.from_numpy(etas).cuda()
    psi_dev = torch.zeros_like(eta_dev)
    res = {}
    for name, p, use_net in (("zero", H.hisq_default_solve_params(deflate=0, batch=1, precision_sloppy=a.sloppy), False),
                             ("deflated", prm, False),
                             ("deflated+learned", H.hisq_default_solve_params(deflate=1, batch=1, guess=1,
                                                                              precision_sloppy=a.sloppy), True)):
        psi_dev.zero_()
        H.hisq_solve_device(ctx, eta_dev[:3].contiguous(), psi_dev[:3].contiguous(), 3, p)  # warm-up
        torch.cuda.synchronize()
        t0 = time.time()
        psi_dev.zero_()
        if use_net:  # the guess is produced on the device and read there by the solve
            with torch.no_grad():
                xin = eta_dev.to(torch.complex64)
                for i in range(0, 24, 3):
                    psi_dev[i:i + 3] = net(xin[i:i + 3]).to(torch.complex128)
        st, s = H.hisq_solve_device(ctx, eta_dev, psi_dev, 24, p)
        torch.cuda.synchronize()
        dt = (time.time() - t0) * 1e3 / 24
        res[name] = dict(ms_per_rhs=round(dt, 3), iterations=float(np.mean([x["iterations"] for x in st])),
                         true_residual_max=max(x["full_residual"] for x in st), status=int(s))
    out = {"metric": METRIC, "value": res["deflated+learned"]["ms_per_rhs"], "unit": "ms/RHS",
           "higher_is_better": False, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"HISQ {dims[0]}^3x{dims[3]}, m={m}, {cfg['n_ev']} eigenpairs, learned initial "
                                  f"guess (3-16-16-16-3 parallel-transport network, BF16 weights) trained on "
                                  f"{n_pairs} deflated-solver pairs, 24 held-out Gaussian RHS, tol 1e-10",
                      "lattice": list(dims)},
           "learned": {"solves": res, "train_loss_first_last": [losses[0], losses[-1]], "epochs": a.learned_epochs,
                       "pairs_seconds": round(t_pairs, 1), "train_seconds": round(t_train, 1),
                       "eigensolve_seconds": round(t_eig, 1)}}
    print(json.dumps(out), flush=True)
    ctx.close()


def _even_rhs(H, ctx, eta, m, par_np):
    """y_e = (M^dag eta)_e = 2m eta_e - D_eo eta_o with the library's FP64 Dslash."""
    d = H.hisq_apply_dslash(ctx, 0, 64, eta)
    y = 2.0 * m * eta - d
    y[par_np == 1] = 0
    return y


# ------------------------------------------------------------ sweeps
def run_sweep(a):
    """32^3x64, m = 0.002 (seed 2, eps 0.3), Gaussian sources, single-RHS solves
    to the 1e-10 FP64 true residual.
    delta_tr: re-deflation threshold x eigenvector storage (FP32, BF16) with
    256 eigenpairs; delta_tr = 0 switches re-deflation off (Fig. 2 analogue).
    mass: plain and deflated CG iterations and time per RHS against the quark
    mass, with one set of massless eigenpairs (lambda_i = eps_i + 4 m^2; Fig. 1
    analogue).
    cheby: eigensolve time against the Chebyshev filter degree."""
    import numpy as np
    import torch

    from paper_2502_00152_gb300 import build as B
    from paper_2502_00152_gb300 import hisq as H
    from paper_2502_00152_gb300 import inputs as I

    B.build()
    cfg = I.lattice_config("c2")
    dims, m0 = cfg["dims"], cfg["mass"]
    fat, lng = I.hisq_links(dims, cfg["seed"], cfg["eps"])
    stream = torch.cuda.current_stream()
    ctx = H.hisq_create(dims, t_antiperiodic=True, device=0, cuda_stream=stream.cuda_stream)
    H.hisq_load_links(ctx, fat, lng, long_recon=a.recon, long_scale=I.C3_NAIK if a.recon != 18 else 1.0)
    del fat, lng
    H.hisq_set_mass(ctx, m0)
    n_ev = a.n_ev if a.n_ev is not None else 256
    srcs = [torch.from_numpy(I.gaussian_source(dims, SOURCE_SEED, 500 + k)).cuda() for k in range(2)]
    psi = torch.zeros_like(srcs[0])

    def eigensolve(prec):
        ep = H.hisq_default_eig_params(n_ev=n_ev, n_kr=max(int(1.5 * n_ev), n_ev + 32), tol=a.eig_tol,
                                       max_restarts=100, cheby_degree=a.cheby, a_min=a.amin, storage_precision=prec)
        t0 = time.time()
        H.hisq_eigensolve(ctx, ep)
        torch.cuda.synchronize()
        return time.time() - t0

    def solve(prm):
        out = []
        for e in srcs:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, status = H.hisq_solve_device(ctx, e, psi, 1, prm)
            torch.cuda.synchronize()
            out.append(dict(ms=(time.perf_counter() - t0) * 1e3, iterations=st[0]["iterations"],
                            redeflations=st[0]["redeflations"], reliable_updates=st[0]["reliable_updates"],
                            full_residual=st[0]["full_residual"], status=int(status)))
        return dict(ms_per_rhs=round(float(np.mean([o["ms"] for o in out])), 2),
                    iterations=[o["iterations"] for o in out], redeflations=[o["redeflations"] for o in out],
                    reliable_updates=[o["reliable_updates"] for o in out],
                    true_residual_max=max(o["full_residual"] for o in out), status=[o["status"] for o in out])

    base = dict(tol=1e-10, precision_sloppy=a.sloppy, link_precision_sloppy=a.links, compute_full_residual=1)
    if a.sweep == "delta_tr":
        rows = []
        for prec, name in ((32, "FP32"), (15, "BF16")):
            t_eig = eigensolve(prec)
            solve(H.hisq_default_solve_params(deflate=1, **base))  # warm-up
            for dtr in (0.0, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6):
                r = solve(H.hisq_default_solve_params(deflate=1, delta_tr=dtr, max_iter=20000, **base))
                rows.append(dict(eigvecs=name, delta_tr=dtr, **r))
            rows.append(dict(eigvecs=name, eigensolve_seconds=round(t_eig, 1)))
        plain = solve(H.hisq_default_solve_params(deflate=0, **base))
        print(json.dumps({"sweep": "delta_tr", "lattice": list(dims), "mass": m0, "n_ev": n_ev,
                          "plain_cg": plain, "rows": rows}), flush=True)
    elif a.sweep == "cheby":
        # eigensolve time against the Chebyshev filter degree (0 = no filter),
        # and the deflated solve that the pairs give
        rows = []
        for deg in (0, 20, 40, 60, 100, 150):
            ep = H.hisq_default_eig_params(n_ev=n_ev, n_kr=max(int(1.5 * n_ev), n_ev + 32), tol=a.eig_tol,
                                           max_restarts=200 if deg == 0 else 100, cheby_degree=deg, a_min=a.amin)
            torch.cuda.synchronize()
            t0 = time.time()
            try:
                eps, nconv = H.hisq_eigensolve(ctx, ep)
            except H.HisqError as e:
                rows.append(dict(cheby_degree=deg, error=str(e)))
                continue
            torch.cuda.synchronize()
            t_eig = time.time() - t0
            r = solve(H.hisq_default_solve_params(deflate=1, **base))
            rows.append(dict(cheby_degree=deg, eigensolve_seconds=round(t_eig, 2), converged=int(nconv),
                             eps_min=float(eps[0]), eps_max=float(eps[-1]), deflated=r))
        print(json.dumps({"sweep": "cheby", "lattice": list(dims), "mass": m0, "n_ev": n_ev, "rows": rows}),
              flush=True)
    else:
        eigensolve(32)
        rows = []
        for m in (0.05, 0.02, 0.01, 0.005, 0.002, 0.001, 0.0005):
            H.hisq_set_mass(ctx, m)
            p = solve(H.hisq_default_solve_params(deflate=0, max_iter=20000, **base))
            d = solve(H.hisq_default_solve_params(deflate=1, max_iter=20000, **base))
            rows.append(dict(mass=m, plain=p, deflated=d))
        print(json.dumps({"sweep": "mass", "lattice": list(dims), "n_ev": n_ev, "rows": rows}), flush=True)
    ctx.close()


if __name__ == "__main__":
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.capture:
        run_capture(args)
    elif args.sweep:
        run_sweep(args)
    elif args.learned:
        run_learned(args)
    else:
        run_ours(args)
