"""Benchmark: Gauss-IRK steps/s on 2D viscous Burgers 512^2 (one GB300).

A bench "step" is one IRK step at Newton relative residual 1e-10: the whole
hot path (stage states, residual, Algorithm-1 block solves with FGMRES and
V-cycles, updates) over the 512^2 (u, v) field, FP64 throughout (the plain
FP64 GPU method).  Workload: nu = 5e-3, dt = 2e-3, seeded random-Fourier
initial field (16 modes, |k| <= 8), Gauss s = 2 (headline) and s = 3.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line on rank 0.  Timing: CUDA events on the solver's stream around
each step, L2 flushed (a 512 MiB write) between steps outside the events;
max over ranks; each rank runs an independent replica (weak scaling, no
collective on the data path).  `e2e` times the same steps through the C ABI
with host buffers, as a caller streaming one trajectory: the state in from
pinned host memory (set_state_keep_stages), the step, get_state back to host.  `--impl reference` times the FP64 CPU oracle on the same
workload (a bounded number of steps on the host cores).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# The reference arm times the oracle on one host thread (reported as cores =
# 1): the BLAS thread pools read these when numpy is first imported, so they
# are set here, before any import that loads numpy.
def _impl_arg(argv):
    for i, a in enumerate(argv):
        if a == "--impl" and i + 1 < len(argv):
            return argv[i + 1]
        if a.startswith("--impl="):
            return a.split("=", 1)[1]
    return "ours"


if _impl_arg(sys.argv) == "reference":
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[_v] = "1"

N = 512
NU = 5e-3
DT = 2e-3
SEED = 1
OP = "burgers2d"
LENGTH = 1.0
# the other full-size workload that fits the timed path: the vorticity-
# streamfunction DAE, double shear layer 1024^2, Re = 1000, Gauss s=5, dt = 5e-3
VSF_1024 = dict(N=1024, NU=1e-3, DT=5e-3, SEED=2, OP="vsf", LENGTH=2 * 3.141592653589793)
METRIC = "IRK steps/s at 1e-10 Newton resid"
UNIT = "steps/s"
FP64_PEAK_TFLOPS_DERIVED = 152 * 2.070e9 * 4 / 1e12  # 2 DFMA/clk/SM at 2070 MHz
FP32_PEAK_TFLOPS_DERIVED = 152 * 2.070e9 * 256 / 1e12  # 128 FFMA/clk/SM at 2070 MHz


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--stages", type=int, default=None, help="default 2 (burgers2d_512), 5 (vsf_1024)")
    ap.add_argument("--workload", default="burgers2d_512", choices=["burgers2d_512", "vsf_1024"],
                    help="timed workload; the extras and the reference arm run on burgers2d_512 only")
    ap.add_argument("--mg-precision", type=int, default=0)
    ap.add_argument("--no-extras", action="store_true", help="skip the s=3 / FP32 / e2e / CPU legs")
    ap.add_argument("--serving-requests", type=int, default=512,
                    help="requests of the 512-request serving mix to run (0 = skip)")
    ap.add_argument("--serving-rates", default="50,100,400",
                    help="Poisson arrival rates to sweep, req/s (comma-separated)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo", init_method="env://")
    return rank, world


def job_throughput(local_ms: float, steps_per_rank: int, world: int):
    """Whole-job steps/s: the steps of all ranks over the slowest rank's time
    (max over ranks, then a barrier).  Returns (steps/s, max time in ms)."""
    t = float(local_ms)
    if world > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([t], dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt[0])
        dist.barrier()
    return steps_per_rank * world / (t / 1e3), t


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline_leg(stages: int, save_path: str = "") -> dict:
    """The oracle, as it stands, on one IRK step of the same workload, run in
    a fresh interpreter limited to one BLAS/OpenMP thread.  The oracle's
    u_{n+1} is saved to save_path (if given) for the precision report."""
    code = (
        "import time, json, sys; sys.path.insert(0, %r)\n"
        "import numpy as np\n"
        "import workloads\n"
        "from oracle import irk\n"
        "from oracle.operators import Problem\n"
        "p = Problem('burgers2d', %d, %r)\n"
        "u0 = workloads.random_fourier_2d(%d, seed=%d)\n"
        "t = time.perf_counter(); u1, K, info = irk.step(p, %d, u0, 0.0, %r, linear='gmres')\n"
        "sec = time.perf_counter() - t\n"
        "if %r: np.save(%r, u1)\n"
        "print(json.dumps({'sec': sec}))\n"
    ) % (ROOT, N, NU, N, SEED, stages, DT, bool(save_path), save_path)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=600)
    sec = json.loads(r.stdout.strip().splitlines()[-1])["sec"]
    return {"value": 1.0 / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"1 IRK step (Gauss s={stages}) of the 512^2 workload from u0: exact Newton, "
                      "SciPy GMRES rtol 1e-13 on the assembled Jacobian, 1 thread"}


def workload_config(args, world: int) -> dict:
    """The `config` of the JSON line, the same for both arms: the workload,
    its sizes and the accuracy every step reaches."""
    return {"workload": f"{OP}_{N}_gauss{args.stages}", "n": N, "nu": NU, "dt": DT,
            "stages": args.stages, "mg_precision": ["fp64", "fp32", "bf16"][args.mg_precision],
            "newton_rtol": 1e-10,
            "l2": "GPU arm: flushed between steps (512 MiB write)",
            "parallelism": f"replicas x{world}"}


# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import numpy as np
    import workloads
    from oracle import irk
    from oracle.operators import Problem
    p = Problem("burgers2d", N, NU)
    u = workloads.random_fourier_2d(N, seed=SEED)
    # the requested warm-up steps run in full; the timed steps stop once
    # `budget` seconds of oracle work have been timed (each is a full step)
    budget = 150.0
    warm = args.warmup
    t = 0.0
    for _ in range(warm):
        u, _, _ = irk.step(p, args.stages, u, t, DT, linear="gmres")
        t += DT
    times = []
    t_start = time.perf_counter()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        u, _, _ = irk.step(p, args.stages, u, t, DT, linear="gmres")
        times.append(time.perf_counter() - t0)
        t += DT
        if time.perf_counter() - t_start > budget:
            break
    sec = sum(times) / len(times)
    val = 1.0 / sec
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": len(times), "warmup": warm, "ms_per_step": 1e3 * sec, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, 1),
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1,
                         "kind": "oracle",
                         "sample": f"{len(times)} timed IRK steps (of {args.steps} requested, "
                                   f"{budget:.0f} s budget) after {warm} warm-up, FP64 exact Newton "
                                   "with SciPy GMRES on the host cores"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
def run_ours(args, rank, world):
    global np
    import numpy as np
    import torch
    import workloads
    from paper_2101_01776_gb300 import build as pbuild
    if not os.path.exists(pbuild.LIB):
        pbuild.build()
    from paper_2101_01776_gb300 import binding as B

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # a dedicated stream: the solver's kernels and the timing events share it
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    if OP == "vsf":
        u0 = np.zeros((2, N, N))
        u0[0] = workloads.double_shear_layer_vorticity(N, seed=SEED + rank)
    else:
        u0 = workloads.random_fourier_2d(N, seed=SEED + rank)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def make(stages, prec, profile, variant=None, **kw):
        # variant None: the library's default nonlinear iteration
        if variant is not None:
            kw["nonlinear_variant"] = variant
        cfg = B.irk_config_default(op=OP, n=N, nu=NU, stages=stages, length=LENGTH,
                                   mg_precision=prec, profile=profile, **kw)
        h = B.irk_create(cfg, torch.from_numpy(u0).to(dev), stream)
        return h

    def timed_steps(h, nsteps, warm, t0=0.0):
        t = t0
        for _ in range(warm):
            B.irk_step(h, t, DT, 1)
            t += DT
        torch.cuda.synchronize(dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(nsteps)]
        tot = {"newton_its": 0, "krylov_its": 0, "vcycles": 0, "prec_apps": 0, "launches": 0,
               "outer_its": 0}
        for k in range(nsteps):
            flush.zero_()
            ev[k][0].record(stream)
            st = B.irk_step(h, t, DT, 1)
            ev[k][1].record(stream)
            t += DT
            tot["newton_its"] += st.newton_its
            tot["krylov_its"] += st.krylov_its
            tot["vcycles"] += st.vcycles
            tot["prec_apps"] += st.prec_apps
            tot["launches"] += st.kernel_launches
            tot["outer_its"] += st.outer_its
        torch.cuda.synchronize(dev)
        ms = [a.elapsed_time(b) for a, b in ev]
        return ms, tot, t

    # ---- ALU ceilings of this GPU, measured (FMA chains on every SM) -------
    alu_peaks = {"fp64": B.irk_measure_alu_peak(0, stream), "fp32": B.irk_measure_alu_peak(1, stream)}
    # ---- headline: plain FP64 GPU method -----------------------------------
    h = make(args.stages, args.mg_precision, 0)
    hbm_peak, peak_src = peaks()
    clocks = ClockSampler(local)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize(dev)
    t = 0.0
    for _ in range(args.warmup):
        B.irk_step(h, t, DT, 1)
        t += DT
    torch.cuda.synchronize(dev)
    clocks.start()
    ms, tot, t = timed_steps(h, args.steps, 0, t)
    clk = clocks.stop()
    B.irk_destroy(h)
    # ---- per-kernel CUDA-event timing: an instrumented repeat of the timed
    # steps (events around every launch slow the host's launch rate, so the
    # headline above runs without them; kernel durations are unaffected)
    h = make(args.stages, args.mg_precision, 1)
    for _ in range(args.warmup):
        B.irk_step(h, 0.0, DT, 1)
    torch.cuda.synchronize(dev)
    B.irk_reset_kernel_stats(h)
    _ms_prof, _tot_prof, _ = timed_steps(h, args.steps, 0, args.warmup * DT)
    kstats = B.irk_kernel_stats(h)
    B.irk_destroy(h)
    step_ms = sum(ms) / len(ms)
    value, local_time = job_throughput(sum(ms), args.steps, world)

    # ---- roofline of the dominant kernel class (CUDA-event time inside the timed region)

    def roofline_of(k):
        # V-cycle classes compute in FP32 when their storage is FP32 or BF16
        # (the velocity and conversion classes read FP64 fields)
        fp32 = (args.mg_precision > 0 and k["name"].startswith("mg_")
                and k["name"] not in ("mg_setup", "mg_convert"))
        alu_peak = alu_peaks["fp32" if fp32 else "fp64"]
        intensity = k["flops"] / max(k["bytes"], 1.0)
        if intensity > alu_peak * 1e12 / (hbm_peak * 1e9):
            achieved = k["flops"] / (k["ms"] / 1e3) / 1e12
            r = {"bound": "alu", "achieved": achieved, "peak": alu_peak,
                 "unit": "TFLOP/s", "frac": achieved / alu_peak,
                 "peak_source": ("measured on this GPU by irk_measure_alu_peak (%s FMA chains, "
                                 "8 x 256 threads per SM, best of 5); derived %.3f"
                                 % ("FP32" if fp32 else "FP64",
                                    FP32_PEAK_TFLOPS_DERIVED if fp32 else FP64_PEAK_TFLOPS_DERIVED))}
        else:
            achieved = k["bytes"] / (k["ms"] / 1e3) / 1e9
            r = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                 "frac": achieved / hbm_peak, "peak_source": f"{peak_src} hbm_gbs"}
        r.update({"traffic": read_traffic(k["name"], f"{OP}_{N}_gauss{args.stages}"), "kernel": k["name"],
                  "launches": k["launches"],
                  "avg_launch_us": 1e3 * k["ms"] / max(k["launches"], 1),
                  "algorithmic_bytes_per_launch": k["bytes"] / max(k["launches"], 1),
                  "algorithmic_flops_per_launch": k["flops"] / max(k["launches"], 1)})
        return r

    ranked = sorted(kstats, key=lambda k: -k["ms"])
    dom = ranked[0]
    roof = roofline_of(dom)
    roof["timing"] = ("CUDA events around each launch on the solver stream, "
                      "instrumented repeat of the timed steps")
    # the next classes by time, for context (same definitions)
    roof_next = [roofline_of(k) for k in ranked[1:4] if k["ms"] > 0]
    kernel_table = sorted(
        ({"name": k["name"], "launches": k["launches"], "ms": round(k["ms"], 3),
          "share": round(k["ms"] / sum(x["ms"] for x in kstats), 4),
          "GBps": round(k["bytes"] / max(k["ms"], 1e-9) / 1e6, 1),
          "TFLOPs": round(k["flops"] / max(k["ms"], 1e-9) / 1e9, 4)} for k in kstats),
        key=lambda r: -r["ms"])
    step_bytes = sum(k["bytes"] for k in kstats) / args.steps

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, world),
        "roofline": roof,
        "roofline_next": roof_next,
        "gpu_launches": tot["launches"],
        "clocks": clk,
        "alu_peaks_measured_tflops": alu_peaks,
        "solver": {"newton_its_per_step": tot["newton_its"] / args.steps,
                   "krylov_its_per_step": tot["krylov_its"] / args.steps,
                   "prec_apps_per_step": tot["prec_apps"] / args.steps,
                   "vcycles_per_step": tot["vcycles"] / args.steps,
                   "vcycles_per_s": tot["vcycles"] / (sum(ms) / 1e3),
                   "algorithmic_GB_per_step": step_bytes / 1e9,
                   "step_hbm_frac": step_bytes / (step_ms / 1e3) / (hbm_peak * 1e9)},
        "kernels": kernel_table,
    }

    if not args.no_extras and rank == 0:
        # ---- e2e through the C ABI with host buffers -------------------------
        h = make(args.stages, args.mg_precision, 0)
        host_in = torch.from_numpy(u0.copy()).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        # a caller streaming one trajectory through pinned host memory: per
        # step the state goes in (keeping the last step's stages as the Newton
        # guess), one IRK step runs, and the new state comes back
        tt = 0.0
        for _ in range(2):
            B.irk_set_state_keep_stages(h, host_in)
            B.irk_step(h, tt, DT, 1)
            B.irk_get_state(h, host_out)
            host_in.copy_(host_out)
            tt += DT
        e2e_n = max(3, min(args.steps, 5))
        t_e = 0.0
        for _ in range(e2e_n):
            flush.zero_()
            torch.cuda.synchronize(dev)
            a = time.perf_counter()
            B.irk_set_state_keep_stages(h, host_in)
            B.irk_step(h, tt, DT, 1)
            B.irk_get_state(h, host_out)
            t_e += time.perf_counter() - a
            host_in.copy_(host_out)
            tt += DT
        B.irk_destroy(h)
        nbytes = u0.size * 8
        line["e2e"] = {"value": e2e_n / t_e, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                       "d2h_bytes_per_step": nbytes}
        # ---- what one copy launch of a given size reaches (the HBM floor) ----
        line["copy_floor"] = copy_floor_leg(torch, dev, stream, flush, hbm_peak)
        # ---- the other stage count and the FP32 V-cycle, same workload ------
        extra = {}
        # (the *_transfer runs: the residual-restriction fusion against the
        # automatic choice, fused with FP32 storage, two kernels with FP64)
        for label, stages, prec, var, kw in (
                ("gauss3_fp64", 3, 0, None, {}), ("gauss2_mg_fp32", 2, 1, None, {}),
                ("gauss3_mg_fp32", 3, 1, None, {}), ("gauss3_fp64_variant3", 3, 0, 3, {}),
                ("gauss2_fp64_fused_transfer", 2, 0, None, dict(mg_fuse_transfer=1)),
                ("gauss2_mg_fp32_separate_transfer", 2, 1, None, dict(mg_fuse_transfer=2))):
            h = make(stages, prec, 0, var, **kw)
            ms2, tot2, _ = timed_steps(h, 3, 2)
            B.irk_destroy(h)
            extra[label] = {"steps_per_s": 1e3 / (sum(ms2) / len(ms2)),
                            "krylov_its_per_step": tot2["krylov_its"] / 3,
                            "newton_its_per_step": tot2["newton_its"] / 3}
        extra["vsf1024_gauss5"] = vsf_leg(B, torch, dev, stream, flush, timed_steps)
        line["variants"] = extra
        # ---- the nonlinear iterations of Sec. 3.2 side by side (same workload,
        # Gauss s=3, FP64): simplified Newton (0), Newton-like (1)-(3), exact
        # Newton (4); gamma = eta against gamma*; the eigenvector basis; and
        # the Radau IIA / Lobatto IIIC rows of Table 1 at s=3
        cmp_ = {}
        for label, kw in (("variant0", dict(nonlinear_variant=0)),
                          ("variant1", dict(nonlinear_variant=1)),
                          ("variant2", dict(nonlinear_variant=2)),
                          ("variant3", dict(nonlinear_variant=3)),
                          ("variant4_exact_newton", dict(nonlinear_variant=4)),
                          ("variant3_gamma_eta", dict(nonlinear_variant=3, gamma_mode=1)),
                          ("variant3_eigen_basis", dict(nonlinear_variant=3, basis=1)),
                          ("radau_iia3", dict(nonlinear_variant=3, family=1)),
                          ("lobatto_iiic3", dict(nonlinear_variant=3, family=2))):
            kw = dict(kw)
            var = kw.pop("nonlinear_variant")
            h = make(3, 0, 0, var, **kw)
            ms2, tot2, _ = timed_steps(h, 3, 2)
            B.irk_destroy(h)
            cmp_[label] = {"steps_per_s": 1e3 / (sum(ms2) / len(ms2)),
                           "newton_its_per_step": tot2["newton_its"] / 3,
                           "krylov_its_per_step": tot2["krylov_its"] / 3,
                           "outer_its_per_step": tot2["outer_its"] / 3,
                           "vcycles_per_step": tot2["vcycles"] / 3}
        line["solver_comparison"] = {"workload": "burgers2d 512^2, s=3, dt=2e-3, FP64 V-cycles",
                                     "runs": cmp_}
        # ---- fully implicit against SDIRK of equal order (the comparison of
        # Sec. 7: preconditioner applications per step), same workload and dt;
        # SDIRK solves its stages one after another
        dirk = {}
        for label, fam, ns in (("gauss1_order2", 0, 1), ("sdirk2_order2", 3, 2),
                               ("radau_iia2_order3", 1, 2), ("sdirk3_order3", 3, 3),
                               ("gauss2_order4", 0, 2), ("sdirk5_order4", 3, 5),
                               ("gauss3_order6", 0, 3)):
            h = make(ns, 0, 0, family=fam)
            ms2, tot2, _ = timed_steps(h, 3, 2)
            B.irk_destroy(h)
            dirk[label] = {"steps_per_s": 1e3 / (sum(ms2) / len(ms2)),
                           "newton_its_per_step": tot2["newton_its"] / 3,
                           "krylov_its_per_step": tot2["krylov_its"] / 3,
                           "prec_apps_per_step": tot2["prec_apps"] / 3,
                           "vcycles_per_step": tot2["vcycles"] / 3}
        line["gauss_vs_sdirk"] = {"workload": "burgers2d 512^2, dt=2e-3, FP64 V-cycles, "
                                              "3 steps after 2", "runs": dirk}
        line["vsf_dae_solvers"] = vsf_dae_leg(B, torch, dev, stream, flush)
        # ---- the empirical autotuner on the headline workload (2 timed steps
        # per candidate), then the same timed steps as the headline
        h = make(args.stages, args.mg_precision, 0)
        for _ in range(2):
            B.irk_step(h, 0.0, DT, 1)
        t_tune = time.perf_counter()
        chosen = B.irk_autotune(h, 2 * DT, DT, 2)
        t_tune = time.perf_counter() - t_tune
        ms3, tot3, _ = timed_steps(h, args.steps, args.warmup, 2 * DT)
        B.irk_destroy(h)
        line["autotuned"] = {
            "steps_per_s": 1e3 / (sum(ms3) / len(ms3)), "tuning_s": t_tune,
            "krylov_its_per_step": tot3["krylov_its"] / args.steps,
            "chosen": {"mg_shifted_sweeps": chosen.mg_shifted_sweeps,
                       "mg_coarse_smoother": chosen.mg_coarse_smoother,
                       "mg_coarse_reduction": chosen.mg_coarse_reduction,
                       "mg_tile_rows": chosen.mg_tile_rows, "mg_levels": chosen.mg_levels,
                       "mg_fuse_transfer": chosen.mg_fuse_transfer}}
        if args.serving_requests > 0:
            # the mix at several Poisson arrival rates, from below the
            # service rate to saturation; 8 slots (the lowest step latency at
            # the mix's throughput; 16 measured the same steps/s at 4x the p50
            # step latency); 32 slots at the highest rate trade tail latency
            # for throughput (host threads then outnumber the host cores)
            rates = [float(r) for r in args.serving_rates.split(",") if r]
            line["serving"] = {
                "requests": args.serving_requests, "of_mix": 512, "slots": 8,
                "per_rate": [serving_leg(B, args.serving_requests, r, slots=8) for r in rates]}
            line["serving_32_slots"] = serving_leg(B, args.serving_requests, rates[-1],
                                                   slots=32, budget_gib=48)
            # the batched form: every resident request in one graph launch
            # per step (include/irk_batch.h), same mix and rates
            # (n >= 512 on 8 stream workers beside the batch: those grids fill
            # the GPU alone and would hold the batch to their step time)
            line["batched_serving"] = {
                "requests": args.serving_requests, "of_mix": 512, "capacity": 32,
                "stream_slots_for_512": 8,
                "per_rate": [serving_leg(B, args.serving_requests, r, slots=32, budget_gib=48,
                                         batched=True, streams_for_large=8) for r in rates]}
            # the 64^2/128^2 part of the mix at the highest rate, both forms
            small = [r for r in workloads.serving_requests(512, seed=4)[:args.serving_requests]
                     if r["n"] <= 128]
            line["serving_small_grids"] = {
                "requests": len(small), "grids": [64, 128], "arrival_rate_per_s": rates[-1],
                "streams_8_slots": serving_leg(B, 0, rates[-1], slots=8, reqs=small),
                "streams_32_slots": serving_leg(B, 0, rates[-1], slots=32, budget_gib=48, reqs=small),
                "batched_32": serving_leg(B, 0, rates[-1], slots=32, budget_gib=48, batched=True,
                                          reqs=small)}
        # ---- precision report: one step from u0 per V-cycle storage precision
        prec_u = {}
        for prec, name in ((0, "fp64"), (1, "fp32"), (2, "bf16")):
            h = make(args.stages, prec, 0)
            st = B.irk_step(h, 0.0, DT, 1)
            out = torch.empty(u0.shape, dtype=torch.float64, device=dev)
            B.irk_get_state(h, out)
            B.irk_destroy(h)
            prec_u[name] = (out.cpu().numpy(), st)
        if world == 1:
            import tempfile
            tmp = os.path.join(tempfile.mkdtemp(), "oracle_u1.npy")
            try:
                line["cpu_baseline"] = cpu_baseline_leg(args.stages, tmp)
                ref = np.load(tmp)
            except Exception as e:  # report, never hide
                line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                        "sample": f"failed: {e!r}"[:200]}
                ref = None
            rep = {}
            for name, (u1, st) in prec_u.items():
                rep[name] = {"krylov_its": st.krylov_its, "newton_its": st.newton_its,
                             "vcycles": st.vcycles, "final_rel_res": st.final_rel_res,
                             "rel_l2_err_vs_oracle": (float(np.linalg.norm(u1 - ref) / np.linalg.norm(ref))
                                                      if ref is not None else None)}
            line["precision"] = {"burgers2d_512": {"workload": "one IRK step from u0 (512^2, Gauss s=%d)"
                                                               % args.stages, "per_precision": rep},
                                 "vsf_1024": vsf_precision_leg(B, torch, dev, stream)}
    elif "e2e" not in line:
        line["e2e"] = None
    if rank == 0:
        # the side results go last, the most read last of all, rounded to
        # four significant digits (the tail of the line is what logs keep)
        for k in ("copy_floor", "kernels", "roofline_next", "variants", "solver_comparison", "gauss_vs_sdirk",
                  "vsf_dae_solvers", "autotuned", "serving_32_slots", "serving",
                  "serving_small_grids", "batched_serving", "precision"):
            if k in line:
                line[k] = _round(line.pop(k))
        print(json.dumps(line), flush=True)
    return 0


def copy_floor_leg(torch, dev, stream, flush, hbm_peak):
    """Device-to-device copies of 1 to 512 MB, one launch each after an L2
    flush (CUDA events on the stream): the bandwidth a single launch of that
    many bytes reaches, against which the 1-40 MB kernels of the V-cycle and
    the Krylov loop are read."""
    out = []
    for mb in (1, 4, 16, 64, 512):
        n = mb * 1024 * 1024 // 8
        src = torch.ones(n, dtype=torch.float64, device=dev)
        dst = torch.empty_like(src)
        for _ in range(3):
            dst.copy_(src)
        reps, tot = 10, 0.0
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            dst.copy_(src)
            b.record(stream)
            b.synchronize()
            tot += a.elapsed_time(b)
        us = 1e3 * tot / reps
        gbs = 2.0 * n * 8 / (us * 1e-6) / 1e9  # bytes read + written
        out.append({"MB": mb, "us": us, "GBps": gbs, "frac_of_peak": gbs / hbm_peak})
        del src, dst
    return {"what": "one copy launch (read + write) after an L2 flush, mean of 10", "sizes": out}


def _round(x):
    if isinstance(x, float):
        return float(f"{x:.4g}")
    if isinstance(x, dict):
        return {k: _round(v) for k, v in x.items()}
    if isinstance(x, list):
        return [_round(v) for v in x]
    return x


def vsf_dae_leg(B, torch, dev, stream, flush):
    """The two DAE solvers of Sec. 7.2 on the double shear layer, 256^2,
    Re=1000, dt=5e-3, FP64, 2 steps after 1: Eq. vsf-system-1 (dae_solver 0:
    FGMRES on each (omega, psi) block, one omega and one psi V-cycle per
    preconditioner application) and the block forward solve of Eq.
    vsf-system-2 (dae_solver 1); Gauss s=1..5 and SDIRK of orders 1-4.
    Reports omega and psi V-cycles per step (the paper's AIR and AMG
    iteration counts of Table dsl-iters)."""
    import math
    import workloads
    n, nu, dt = 256, 1e-3, 5e-3
    u0 = np.zeros((2, n, n))
    u0[0] = workloads.double_shear_layer_vorticity(n, seed=2)
    runs = {}
    for fam, name, stages in ((0, "gauss", (1, 2, 3, 4, 5)), (3, "sdirk", (1, 2, 3, 5))):
        for ns in stages:
            for ds in (0, 1):
                cfg = B.irk_config_default(op="vsf", n=n, nu=nu, stages=ns, family=fam,
                                           length=2 * math.pi, dae_solver=ds)
                h = B.irk_create(cfg, torch.from_numpy(u0).to(dev), stream)
                t = 0.0
                B.irk_step(h, t, dt, 1)
                t += dt
                ms, agg = [], {"newton_its": 0, "prec_apps": 0, "vcycles": 0, "poisson_vcycles": 0}
                for _ in range(2):
                    flush.zero_()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    st = B.irk_step(h, t, dt, 1)
                    e1.record(stream)
                    torch.cuda.synchronize(dev)
                    ms.append(e0.elapsed_time(e1))
                    for k in agg:
                        agg[k] += getattr(st, k)
                    t += dt
                B.irk_destroy(h)
                runs[f"{name}{ns}_system{ds + 1}"] = {
                    "steps_per_s": 1e3 / (sum(ms) / len(ms)),
                    "newton_its_per_step": agg["newton_its"] / 2,
                    "prec_apps_per_step": agg["prec_apps"] / 2,
                    "omega_vcycles_per_step": (agg["vcycles"] - agg["poisson_vcycles"]) / 2,
                    "psi_vcycles_per_step": agg["poisson_vcycles"] / 2}
    return {"workload": "vsf 256^2 double shear layer, Re=1000, dt=5e-3, FP64", "runs": runs}


def vsf_leg(B, torch, dev, stream, flush, timed_steps):
    """Vorticity-streamfunction DAE, double shear layer 1024^2, Re=1000, Gauss
    s=5, dt=5e-3, FP64 (and FP32 V-cycle): steps/s over 2 steps after 1."""
    import math
    import workloads
    n, nu, dt = 1024, 1e-3, 5e-3
    w0 = workloads.double_shear_layer_vorticity(n, seed=2)
    u0 = np.zeros((2, n, n))
    u0[0] = w0
    out = {}
    # the default block-diagonal variant 2 (FP64 / FP32 V-cycle) and the block
    # upper triangular variant 3 (Sec. 3.2), which keeps the small d_kl
    # off-diagonal terms of the transformed Jacobian (same fixed point)
    for label, prec, var in (("fp64", 0, 2), ("mg_fp32", 1, 2), ("mg_bf16", 2, 2),
                             ("fp64_variant3", 0, 3), ("mg_fp32_variant3", 1, 3)):
        cfg = B.irk_config_default(op="vsf", n=n, nu=nu, stages=5, length=2 * math.pi,
                                   mg_precision=prec, nonlinear_variant=var)
        h = B.irk_create(cfg, torch.from_numpy(u0).to(dev), stream)
        t, ms = 0.0, []
        st = B.irk_step(h, t, dt, 1)
        t += dt
        kry = newt = 0
        for _ in range(2):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = B.irk_step(h, t, dt, 1)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(e0.elapsed_time(e1))
            kry += st.krylov_its
            newt += st.newton_its
            t += dt
        B.irk_destroy(h)
        out[label] = {
            "steps_per_s": 1e3 / (sum(ms) / len(ms)), "krylov_its_per_step": kry / 2,
            "newton_its_per_step": newt / 2}
    return out


def vsf_precision_leg(B, torch, dev, stream):
    """Config [3] on the DAE: one IRK step from the double shear layer 1024^2
    (Re=1000, Gauss s=5, dt=5e-3) per V-cycle precision (FP64; FP32; BF16
    storage with FP32 arithmetic), FP64 everywhere else.  Error of omega
    against the oracle's first step, read from the stored trajectory that
    tests/golden/make_trajectories.py writes with the oracle."""
    import math
    import workloads
    path = os.path.join(ROOT, "tests", "golden", "traj_vsf_1024_gauss5.npz")
    ref = np.load(path)["u_step1"] if os.path.exists(path) else None
    n, nu, dt = 1024, 1e-3, 5e-3
    u0 = np.zeros((2, n, n))
    u0[0] = workloads.double_shear_layer_vorticity(n, seed=2)
    rep = {}
    for prec, name in ((0, "fp64"), (1, "fp32"), (2, "bf16")):
        cfg = B.irk_config_default(op="vsf", n=n, nu=nu, stages=5, length=2 * math.pi,
                                   mg_precision=prec)
        h = B.irk_create(cfg, torch.from_numpy(u0).to(dev), stream)
        st = B.irk_step(h, 0.0, dt, 1)
        out = torch.empty((2, n, n), dtype=torch.float64, device=dev)
        B.irk_get_state(h, out)
        B.irk_destroy(h)
        w1 = out[0].cpu().numpy()
        rep[name] = {"krylov_its": st.krylov_its, "newton_its": st.newton_its,
                     "vcycles": st.vcycles, "final_rel_res": st.final_rel_res,
                     "rel_l2_err_omega_vs_oracle": (float(np.linalg.norm(w1 - ref) / np.linalg.norm(ref))
                                                    if ref is not None else None)}
    return {"workload": "one IRK step from the double shear layer (1024^2, Gauss s=5, dt=5e-3)",
            "per_precision": rep}


def serving_leg(B, count, rate, slots=8, budget_gib=24, batched=False, reqs=None,
                streams_for_large=0):
    """Config [4]: the first `count` requests of the seeded 512-request mix
    (2D Burgers, grid from {64,128,256,512}^2, nu log-uniform in [1e-3,1e-1],
    Gauss s in {2,3,4}, random-Fourier initial field seeded by request id,
    20 steps at dt=1e-3), or the given `reqs`, Poisson arrivals at `rate`
    req/s, served by the continuous-batching runtime with `slots` slots (one
    stream and host thread each) or, batched, by the batched server with
    `slots` resident requests stepped together (and, with streams_for_large,
    the 512^2 requests on that many stream workers beside the batch), within
    an HBM budget."""
    import threading
    import workloads
    if reqs is None:
        reqs = workloads.serving_requests(512, seed=4)[:count]
    count = len(reqs)
    u0s = {}
    for r in reqs:
        u0s[r["id"]] = workloads.random_fourier_2d(r["n"], seed=r["seed"])
    srv = (B.irk_server_create_batched(slots, budget_gib << 30, stream_slots=streams_for_large,
                                       stream_min_n=512 if streams_for_large else 0) if batched
           else B.irk_server_create(slots, budget_gib << 30))
    ids = [None] * len(reqs)
    rng = np.random.default_rng(5)
    gaps = rng.exponential(1.0 / rate, size=len(reqs))

    def producer():
        for k, r in enumerate(reqs):
            cfg = B.irk_config_default(op="burgers2d", n=r["n"], stages=r["s"], nu=r["nu"])
            ids[k] = B.irk_server_submit(srv, cfg, u0s[r["id"]], 0.0, 1e-3, 20)
            time.sleep(float(gaps[k]))
    th = threading.Thread(target=producer)
    th.start()
    th.join()
    failed = 0
    for k, r in enumerate(reqs):
        try:
            B.irk_server_wait(srv, ids[k], u0s[r["id"]].shape, 20)
        except B.IrkError:
            failed += 1
    st = B.irk_server_stats_get(srv)
    B.irk_server_destroy(srv)
    return {"requests": count, "of_mix": 512, "arrival_rate_per_s": rate, "slots": slots,
            "form": ("batched + %d streams for 512^2" % streams_for_large if streams_for_large
                     else "batched") if batched else "streams",
            "budget_GiB": budget_gib, "failed": failed, "steps": st["steps"],
            "steps_per_s": st["steps_per_s"], "wall_s": st["wall_s"],
            "p50_step_ms": st["p50_step_ms"], "p99_step_ms": st["p99_step_ms"],
            "p50_request_ms": st["p50_request_ms"], "p99_request_ms": st["p99_request_ms"],
            "p50_queue_ms": st["p50_queue_ms"], "p99_queue_ms": st["p99_queue_ms"],
            "peak_active": st["peak_active"], "peak_GiB": st["peak_bytes"] / 2 ** 30}


def read_traffic(kernel_class: str, workload: str = "burgers2d_512_gauss2"):
    """DRAM bytes per launch of the kernel class on this workload from the
    committed ncu summary, or None when absent or taken on a different kernel
    source."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    import hashlib
    for line in open(path):
        if line.startswith("#") or "=" not in line:
            continue
        kv = dict(x.split("=", 1) for x in line.split())
        if kv.get("class") != kernel_class or kv.get("workload") != workload:
            continue
        # the kernel's source and the solver that sets its launch mix
        srcs = [os.path.join(ROOT, "paper_2101_01776_gb300", "csrc", f)
                for f in kv.get("source", "").split(",")]
        if not srcs or not all(os.path.exists(f) for f in srcs):
            return None
        hsh = hashlib.sha256()
        for f in srcs:
            hsh.update(open(f, "rb").read())
        sha = hsh.hexdigest()[:16]
        if sha != kv.get("sha"):
            return None
        return float(kv["dram_bytes_per_launch"])
    return None


def main():
    args = parse()
    if args.workload == "vsf_1024":
        globals().update(VSF_1024)
        args.no_extras = True
    if args.stages is None:
        args.stages = 5 if OP == "vsf" else 2
    rank, world = dist_setup(args)
    if args.impl == "reference" and OP != "burgers2d":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the oracle on "
                              "the burgers2d_512 workload only"}), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world)


if __name__ == "__main__":
    sys.exit(main())
