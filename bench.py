"""Benchmark of the dynamic-tomography hot path on GB300.

Workload (default): 16 slices of 256^2 voxels, 256 detector bins, K = 1800
projections over 10 continuous half-turns, m = 8 real Fourier coefficient
volumes, nt = 10 frames, moving-ellipsoid phantom with Poisson noise (1e4
photons), FP32 -- reconstructed with ADMM-CG (4 CG steps per u-step).

One step = one ADMM-CG iteration: 5 dynamic forward projections, 5 dynamic
back-projections (1 residual + 4 CG), the 4D TV stencils, the prox and the
FP64 inner products, replayed as a CUDA graph by admm_solve.  The metric is
voxel-projection updates per second: each projector application counts K * V
voxel-projection pairs, 10 applications per iteration.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs one independent replica per GPU (the path has no exchange step
at this size: weak scaling, no collective on the data path).  The reference
arm times the FP64 CPU oracle on the host cores on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP32 FMA pipe: 152 SMs x 128 lanes x 2 flop x 2.07 GHz (maximum SM clock).
SMS, FP32_LANES, SM_MAX_GHZ = 152, 128, 2.07


def smem_peak_tbs():
    """Shared-memory bandwidth: 128 bytes per clock per SM (one wavefront)."""
    return SMS * 128 * SM_MAX_GHZ * 1e9 / 1e12


def hbm_peak_gbs():
    """Measured copy bandwidth of this GPU model (generated file), else
    the fallback figure of an earlier GB300 measurement."""
    try:
        with open(PEAKS_PATH) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json copy bandwidth)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback (6.8 TB/s, earlier GB300 copy measurement)"


def fp32_peak_tflops(sm_mhz=None):
    ghz = (sm_mhz / 1000.0) if sm_mhz else SM_MAX_GHZ
    return SMS * FP32_LANES * 2 * ghz * 1e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ellipsoids256")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-jobs", type=int, default=24)
    ap.add_argument("--no-slabs", action="store_true", help="skip the slab-streaming measurement")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the BF16-operator, FBP and slab-streaming measurements")
    ap.add_argument("--fold-strip", type=int, default=0,
                    help="with --variant: fix the folded forward's strip height (lines) instead of the default")
    ap.add_argument("--variant", default=None,
                    help="force projector variants 'fwd,adj' (0 direct, 1 fold, 2 fold in two kernels: forward "
                         "only); default: autotuned")
    ap.add_argument("--fold2-config", default=None,
                    help="with --variant 2,x or --profile-small: fix the two-kernel folded forward's "
                         "'group,threads,lines[,split[,async[,rays_per_thread]]]' instead of the default")
    ap.add_argument("--fold-adj-angles", type=int, default=0,
                    help="with --variant x,1 or --profile-small: fix the folded adjoint's distinct angles per "
                         "pipeline stage instead of the default")
    ap.add_argument("--profile-small", action="store_true",
                    help="run only one launch of each projector kernel on the workload (for ncu captures)")
    return ap.parse_args()


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running: one
    nvidia-smi child in its loop mode (every 100 ms), stopped on exit."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._proc = None
        self._th = None

    def _read(self):
        for line in self._proc.stdout:
            line = line.strip()
            if line:
                self.samples.append([x.strip() for x in line.split(",")])

    def __enter__(self):
        try:
            self._proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                           "--format=csv,noheader,nounits", "-lms", "100"],
                                          stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._th = threading.Thread(target=self._read, daemon=True)
            self._th.start()
            time.sleep(0.15)  # first sample before the timed region starts
        except Exception:
            self._proc = None
        return self

    def __exit__(self, *a):
        if self._proc is not None:
            time.sleep(0.15)
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()
        if self._th:
            self._th.join(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if len(s) > 4 + i and
                          s[4 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def dist_init(n):
    """One process per GPU under torchrun (NCCL); gloo when no GPU is present.
    Replicas only exchange the timing maximum, never data."""
    if n <= 1 and "RANK" not in os.environ:
        return 0, 1, None
    import torch
    import torch.distributed as tdist
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if not tdist.is_initialized():
        tdist.init_process_group(backend=backend)
    return tdist.get_rank(), tdist.get_world_size(), tdist


def barrier_max(tdist, value: float, device):
    """Maximum of a per-rank value over all ranks (the job's wall time)."""
    if tdist is None:
        return value
    import torch
    dev = device if tdist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def replica_units(units_per_rank: float, world: int) -> float:
    """Whole-job work of N independent replicas (weak scaling)."""
    return units_per_rank * world


def set_fold2_config(plan, text):
    """Apply 'group,threads,lines[,split[,async[,rays_per_thread]]]' to the two-kernel folded forward."""
    v = [int(x) for x in text.split(",")]
    plan.set_fold_groups(v[0], v[2], v[1], v[5] if len(v) > 5 else 0)
    plan.set_fold_march(v[3] if len(v) > 3 else 1, v[4] if len(v) > 4 else 0)


def joseph_samples(theta, nx, ny, ns, distinct=True):
    """Number of Joseph interpolation samples of one static transform per
    slice: for every angle (distinct angles mod pi when `distinct`), bin and
    step line, the samples whose interpolation pair touches the grid (the
    sample at xi contributes when -1 <= xi < n along the interpolated axis)."""
    th = np.mod(np.asarray(theta, dtype=np.float64), np.pi) if distinct else np.asarray(theta, dtype=np.float64)
    if distinct:
        th = np.unique(np.round(th, 11))
    sb = np.arange(ns) - 0.5 * (ns - 1)
    total = 0
    for a in th:
        c, s = np.cos(a), np.sin(a)
        if abs(c) >= abs(s):  # step over rows, interpolate in x
            y = np.arange(ny) - 0.5 * (ny - 1)
            xi = (sb[None, :] - y[:, None] * s) / c + 0.5 * (nx - 1)
            n = nx
        else:  # step over columns, interpolate in y
            x = np.arange(nx) - 0.5 * (nx - 1)
            xi = (sb[None, :] - x[:, None] * c) / s + 0.5 * (ny - 1)
            n = ny
        total += int(np.count_nonzero((xi >= -1.0) & (xi < n)))
    return total


def algorithmic_smem_bytes(w, theta, variant, U):
    """Shared-memory bytes one projector application needs to read: every
    Joseph sample of the folded forward reads two neighbouring pixel vectors
    of m FP32 coefficients from the staged strip; the folded adjoint reads,
    per voxel and distinct angle, two bins of the m folded sinograms from its
    staged window.  (The direct variants stage data per projection.)  The
    two-kernel folded forward (variant 2) reads the same samples in its
    static-transform kernel."""
    if variant in (1, 2):
        return 2 * w.m * 4 * joseph_samples(theta, w.N, w.N, w.ns) * w.nz
    return 2 * w.m * 4 * w.K * w.voxels()


def algorithmic_flops(w, variant, U):
    """FP32 flops of one projector application (FMA = 2 flops).

    direct (every projection at its own angle): per voxel-projection pair m
    FMAs of the basis combine + 2 of the interpolation / footprint:
        2 (m + 2) K V.
    half-turn fold (Sec. 4): per voxel and distinct angle mod pi, 2 FMAs of
    the interpolation for each of the m coefficients, plus m FMAs per
    detector sample to distribute (fold) over the K projections:
        2 (2 m U V + m K ns nz).
    The two-kernel folded forward does the same arithmetic in two launches."""
    if variant in (1, 2):
        return 2.0 * (2 * w.m * U * w.voxels() + w.m * w.K * w.ns * w.nz)
    return 2.0 * (w.m + 2) * w.K * w.voxels()


def run_ours(a):
    import torch

    from paper_1809_09725_gb300 import dynrecon as dr
    from paper_1809_09725_gb300 import synth

    rank, world, tdist = dist_init(a.gpus)
    local = int(os.environ.get("LOCAL_RANK", rank))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = synth.WORKLOADS[a.workload]
    theta, t, g_np = synth.make_data(w)
    plan = dr.Plan(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt, dr.F32)
    g = torch.from_numpy(g_np.astype(np.float32)).to(dev)
    u = torch.zeros(plan.u_shape(), dtype=torch.float32, device=dev)
    units_per_iter = 2 * (w.n_cg + 1) * w.K * w.voxels()  # projector applications x K V
    if a.variant:
        fv, av = (int(x) for x in a.variant.split(","))
        plan.set_variant(fv, av)
        if a.fold_strip > 0:
            plan.set_fold_strip(a.fold_strip, False)
        if fv == dr.FOLD2 and a.fold2_config:
            set_fold2_config(plan, a.fold2_config)
        if av == dr.FOLD and a.fold_adj_angles > 0:
            plan.set_fold_adj_stage(a.fold_adj_angles)

    if a.profile_small:
        # one forward and one adjoint of each variant (direct, half-turn fold)
        # on the benchmark workload, for profiler captures
        uin = torch.randn(plan.u_shape(), dtype=torch.float32, device=dev)
        gout = torch.empty_like(g)
        for var in (dr.DIRECT, dr.FOLD):
            plan.set_variant(var, var)
            if var == dr.FOLD and a.fold_strip > 0:
                plan.set_fold_strip(a.fold_strip, False)
            if var == dr.FOLD and a.fold_adj_angles > 0:
                plan.set_fold_adj_stage(a.fold_adj_angles)
            dr.dyn_radon_fwd(plan, uin, gout)
            dr.dyn_radon_adj(plan, g, u)
        # the two-kernel folded forward (static transforms + distribution)
        plan.set_variant(dr.FOLD2, dr.FOLD)
        if a.fold2_config:
            set_fold2_config(plan, a.fold2_config)
        dr.dyn_radon_fwd(plan, uin, gout)
        # the folded forward on BF16 storage (bf16 strip)
        pb = dr.Plan(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt, dr.BF16)
        pb.set_variant(dr.FOLD, dr.FOLD)
        pb.set_fold_strip(6, False)
        gb = torch.empty(pb.g_shape(), dtype=torch.bfloat16, device=dev)
        dr.dyn_radon_fwd(pb, uin.to(torch.bfloat16), gb)
        torch.cuda.synchronize()
        print(json.dumps({"profile_small": True}))
        return

    prm = dr.solve_params(dr.ADMM_CG, iters=a.warmup, n_cg=w.n_cg, lambda1=w.lambda1, lambda2=w.lambda2,
                          rho=w.rho)
    dr.admm_solve(plan, g, u, prm, want_objective=False)  # warm-up iterations (untimed)
    u.zero_()
    torch.cuda.synchronize()
    prm = dr.solve_params(dr.ADMM_CG, iters=a.steps, n_cg=w.n_cg, lambda1=w.lambda1, lambda2=w.lambda2,
                          rho=w.rho)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        if tdist is not None:
            tdist.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        res = dr.admm_solve(plan, g, u, prm, want_objective=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if tdist is not None:
            tdist.barrier()
    ms = e0.elapsed_time(e1)
    ms = barrier_max(tdist, ms, dev)
    total_units = replica_units(units_per_iter * a.steps, world)
    value = total_units / (ms * 1e-3)
    obj = res["objective"]

    # dominant kernels: time the projector pair alone on the same stream, in
    # the variant the solver selected (autotuned inside admm_solve)
    info = plan.info()
    tune = plan.autotune() if not a.variant else None
    p_in = torch.randn(plan.u_shape(), dtype=torch.float32, device=dev)
    gbuf = torch.empty(plan.g_shape(), dtype=torch.float32, device=dev)
    ubuf = torch.empty(plan.u_shape(), dtype=torch.float32, device=dev)
    for _ in range(3):
        dr.dyn_radon_fwd(plan, p_in, gbuf)
        dr.dyn_radon_adj(plan, gbuf, ubuf)
    reps = 10
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(reps):
        dr.dyn_radon_fwd(plan, p_in, gbuf)
    ev[1].record(stream)
    for _ in range(reps):
        dr.dyn_radon_adj(plan, gbuf, ubuf)
    ev[2].record(stream)
    torch.cuda.synchronize()
    fwd_ms = ev[0].elapsed_time(ev[1]) / reps
    adj_ms = ev[1].elapsed_time(ev[2]) / reps
    U = info["unique_angles"]
    if fwd_ms >= adj_ms:
        variant = info["fwd_variant"]
        kname = {1: "fold_fwd_kernel", 2: "fold_fwd_kernel(static)+fold_dist_kernel"}.get(variant, "fwd_kernel")
        launch_ms = fwd_ms
    else:
        variant = info["adj_variant"]
        kname = "fold_adj_kernel+fold_data_kernel" if variant == 1 else "adj_kernel"
        launch_ms = adj_ms
    flops = algorithmic_flops(w, variant, U)
    achieved = flops / (launch_ms * 1e-3) / 1e12
    clocks = clk.summary()
    peak = fp32_peak_tflops()
    traffic = load_traffic(kname)
    if fwd_ms >= adj_ms:
        smem_bytes = algorithmic_smem_bytes(w, theta, variant, U)
    else:
        smem_bytes = 2 * w.m * 4 * (U if variant == 1 else w.K) * w.voxels()
    smem_achieved = smem_bytes / (launch_ms * 1e-3) / 1e12
    smem_peak = smem_peak_tbs()

    # the projector pair on BF16 storage (FP32 accumulation) next to FP32
    bf16_ops = None
    if rank == 0 and not a.no_extras:
        pb = dr.Plan(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt, dr.BF16)
        pb.autotune()
        ub = p_in.to(torch.bfloat16)
        gb = torch.empty(pb.g_shape(), dtype=torch.bfloat16, device=dev)
        uab = torch.empty_like(ub)
        for _ in range(3):
            dr.dyn_radon_fwd(pb, ub, gb)
            dr.dyn_radon_adj(pb, gb, uab)
        bev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize()
        bev[0].record(stream)
        for _ in range(reps):
            dr.dyn_radon_fwd(pb, ub, gb)
        bev[1].record(stream)
        for _ in range(reps):
            dr.dyn_radon_adj(pb, gb, uab)
        bev[2].record(stream)
        torch.cuda.synchronize()
        bf16_ops = {"fwd_ms": bev[0].elapsed_time(bev[1]) / reps, "adj_ms": bev[1].elapsed_time(bev[2]) / reps,
                    "fp32_fwd_ms": fwd_ms, "fp32_adj_ms": adj_ms,
                    "note": "dyn_radon_fwd / dyn_radon_adj on bf16 u and g (FP32 accumulation), same workload"}
        del pb, ub, gb, uab

    # FBP initial guess (Sec. 5), one window per half-turn: filter + one back-projection
    fbp = None
    tv_kernels = None
    if not a.no_extras:
        fbp = run_fbp(plan, g, w, dev, stream)
        tv_kernels = run_tv_kernels(plan, w, dev, stream)

    # end to end through the public call with host buffers (one full job per call)
    e2e = None
    if not a.no_e2e:
        gh = torch.from_numpy(g_np.astype(np.float32)).pin_memory()
        uh = torch.zeros(plan.u_shape(), dtype=torch.float32).pin_memory()
        ghn, uhn = gh.numpy(), uh.numpy()
        jobs = 2
        prm_e = dr.solve_params(dr.ADMM_CG, iters=w.iters, n_cg=w.n_cg, lambda1=w.lambda1, lambda2=w.lambda2,
                                rho=w.rho)
        dr.admm_solve(plan, ghn, uhn, dr.solve_params(dr.ADMM_CG, iters=2, n_cg=w.n_cg, lambda1=w.lambda1,
                                                      lambda2=w.lambda2, rho=w.rho), want_objective=False)
        torch.cuda.synchronize()
        if tdist is not None:
            tdist.barrier()
        t0 = time.perf_counter()
        for _ in range(jobs):
            uhn[...] = 0.0
            dr.admm_solve(plan, ghn, uhn, prm_e, want_objective=False)
        torch.cuda.synchronize()
        el = barrier_max(tdist, time.perf_counter() - t0, dev)
        e2e = {"value": units_per_iter * w.iters * jobs * world / el, "unit": "voxel*projection/s",
               "h2d_bytes_per_step": int(g_np.size * 4 + uhn.nbytes), "d2h_bytes_per_step": int(uhn.nbytes),
               "step": "one %d-iteration reconstruction job via admm_solve on pinned host buffers" % w.iters,
               "jobs": jobs, "s_per_job": el / jobs}

    serving = None
    if not a.no_serving:
        serving = {name: run_serving(a, local, prec) for name, prec in (("fp32", dr.F32), ("bf16", dr.BF16))}
        if rank == 0 and not a.no_extras:
            serving["load_sweep_fp32"] = run_serving_sweep(a, local)

    batched = None
    if rank == 0 and not a.no_extras:
        batched = run_batched(dev)

    slabs = None
    if rank == 0 and not (a.no_slabs or a.no_extras):
        slabs = run_slabs(w, theta, t, g_np, dev)

    cpu = None
    accuracy = None
    if rank == 0 and not a.no_cpu_baseline:
        cpu = cpu_baseline(w, theta, t, g_np)
        cpu["one_thread"] = cpu_baseline_1thread(w)
        accuracy = accuracy_vs_oracle(w, theta, t, g_np, dev)

    if rank == 0:
        # per ADMM-CG iteration: n_cg + 1 forwards and adjoints (the folded
        # adjoint is two launches: data fold + back-projection), n_cg + 1 D^T D
        # (right-hand side + CG steps), prox, D^T w, n_cg updates, n_cg - 1
        # direction updates, the fidelity dot, the iteration counter
        # (the two-kernel folded forward is two launches too: static transforms +
        # distribution).  With both folded, the CG steps' R*R p is the folded
        # normal operator: static transforms, Gram mix, back-projection.
        adj_launches = 2 if info["adj_variant"] == 1 else 1
        fwd_launches = 2 if info["fwd_variant"] == 2 else 1
        normal_launches = 3 if (info["fwd_variant"], info["adj_variant"]) == (2, 1) else fwd_launches + adj_launches
        launches_per_iter = ((1 + fwd_launches + adj_launches) + w.n_cg * (1 + normal_launches) + 2 * w.n_cg + 3)
        line = {
            "metric": "voxel*projection updates/s (dynamic projector + back-projector applications "
                      "inside ADMM-CG iterations)",
            "value": value, "unit": "voxel*projection/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded moving ellipsoids, Poisson 1e4)",
            "config": bench_config(world),
            "admm_iters_per_s": a.steps * world / (ms * 1e-3),
            "objective_first_last": [float(obj[0]), float(obj[-1])],
            "clocks": clocks,
            "e2e": e2e,
            "gpu_launches": launches_per_iter * a.steps + fwd_launches + 1,  # + the final fidelity (forward + dot)
            "roofline": {"bound": "smem", "kernel": kname, "achieved": smem_achieved, "peak": smem_peak,
                         "unit": "TB/s", "frac": smem_achieved / smem_peak, "traffic": traffic,
                         "algorithmic_smem_bytes_per_launch": smem_bytes,
                         "peak_source": "derived: 152 SMs x 128 B/clk shared-memory bandwidth x 2.07 GHz max SM clock",
                         "alu": {"achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                                 "algorithmic_flops_per_launch": flops,
                                 "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"},
                         "launch_ms": launch_ms, "fwd_ms": fwd_ms, "adj_ms": adj_ms,
                         "variants": {"unique_angles": U, "fwd": info["fwd_variant"], "adj": info["adj_variant"],
                                      "fold_lines": info["fold_lines"], "fold_async": info["fold_async"],
                                      "fold_adj_angles_per_stage": info["fold_adj_angles"],
                                      "fold2_group_threads_lines_split_async_rpt": [
                                          info["fold2_group"], info["fold2_threads"], info["fold2_lines"],
                                          info["fold2_split"], info["fold2_async"], info["fold2_rays_per_thread"]],
                                      "autotune_ms_fwd_direct_fold_adj_direct_fold_fwd_fold2": tune}},
            "cpu_baseline": cpu,
            "serving": serving,
            "accuracy_vs_fp64_oracle": accuracy,
            "batched_jobs": batched,
            "fbp_init": fbp,
            "tv_kernels": tv_kernels,
            "bf16_operators": bf16_ops,
            "slab_streaming": slabs,
        }
        print(json.dumps(line))


def serving_jobs(n, seed=180905):
    """A stream of uneven reconstruction requests: Poisson arrivals at 4 jobs/s;
    grid 128 or 256, 4-16 slices, 4-20 continuous half-turns at 90 or 180
    projections per half-turn, m in {4, 8, 16}, Fourier or Legendre, 30
    ADMM-CG iterations; data are exact line integrals of 5 moving disks."""
    from paper_1809_09725_gb300 import synth
    rng = synth.rng_for(seed)
    t_arr = np.cumsum(rng.exponential(1.0 / 4.0, size=n))
    jobs = []
    for i in range(n):
        N = int(rng.choice([128, 256]))
        nz = int(rng.integers(4, 17))
        ht = int(rng.integers(4, 21))
        per = int(rng.choice([90, 180]))
        K = ht * per
        m = int(rng.choice([4, 8, 16]))
        basis = int(rng.integers(0, 2))
        theta, t = synth.scan(K, ht)
        blobs = synth.disks(rng, N, 5)
        g = np.repeat(synth.sinogram(blobs, theta, t, N, 1), nz, axis=0)
        jobs.append(dict(arrival=float(t_arr[i]), N=N, nz=nz, K=K, m=m, basis=basis, nt=ht, theta=theta, t=t,
                         g=g))
    return jobs


def run_serving(a, device, prec):
    """Submit the request stream to the serving loop in real time; report
    latency percentiles and aggregate projector throughput."""
    from paper_1809_09725_gb300 import dynrecon as dr
    jobs = serving_jobs(a.serving_jobs)
    descs = []
    for j in jobs:
        if prec == dr.BF16:
            import torch
            gh = torch.from_numpy(j["g"]).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
            uh = np.zeros((j["nz"], j["N"], j["N"], j["m"]), dtype=np.uint16)
        else:
            gh = j["g"].astype(np.float32)
            uh = np.zeros((j["nz"], j["N"], j["N"], j["m"]), dtype=np.float32)
        prm = dr.solve_params(dr.ADMM_CG, iters=30, n_cg=4, lambda1=1e-3, lambda2=1.0, rho=1e-2)
        descs.append(dr.job_desc(j["N"], j["N"], j["nz"], j["N"], j["theta"], j["t"], j["basis"], j["m"], j["nt"],
                                 prec, prm, gh, uh))
    srv = dr.Server(device=device, budget_bytes=150 * 10 ** 9, slots=8)
    t0 = time.perf_counter()
    ids = []
    for j, d in zip(jobs, descs):
        dt = j["arrival"] - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        ids.append(srv.submit(d))
    res = [srv.wait(i, timeout_s=600.0) for i in ids]
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    units = sum(2 * 5 * 30 * j["K"] * j["N"] * j["N"] * j["nz"] for j in jobs)
    return {"jobs": len(jobs), "completed": st["completed"], "failed": st["failed"],
            "p50_latency_s": st["p50_latency_s"], "p99_latency_s": st["p99_latency_s"],
            "voxel_projection_per_s": units / wall, "wall_s": wall,
            "peak_device_gb": st["peak_device_bytes"] / 1e9, "budget_gb": 150,
            "stream": "Poisson 4 jobs/s, first %d arrivals; N in {128,256}, nz 4-16, K 360-3600 over 4-20 "
                      "half-turns, m in {4,8,16}, 30 ADMM-CG iterations" % len(jobs),
            "max_queue_s": max(r["queue_s"] for r in res),
            "errors": [{"job": i, "rc": r["rc"], "error": r["error"]} for i, r in enumerate(res) if r["rc"] != 0]}


def run_tv_kernels(plan, w, dev, stream, reps=10):
    """The HBM-bound TV stencils through the C ABI on the workload's volume:
    tv4d_prox (shrink + dual update: reads u and mu, writes mu and w),
    tv4d_grad_adj (D^T p: reads p, writes u) and tv4d_grad (D u: reads u,
    writes p), each timed alone with CUDA events; achieved = algorithmic
    bytes / time against the measured HBM copy bandwidth."""
    import torch

    from paper_1809_09725_gb300 import dynrecon as dr

    V = w.voxels()
    ub = w.m * V * 4  # u, float
    fb = 4 * w.nt * V * 4  # one dual field, float
    u = torch.randn(plan.u_shape(), dtype=torch.float32, device=dev)
    mu = torch.randn(plan.field_shape(), dtype=torch.float32, device=dev) * 1e-3
    wf = torch.empty_like(mu)
    ua = torch.empty_like(u)
    peak, src = hbm_peak_gbs()
    calls = {
        "prox": (lambda: dr.tv4d_prox(plan, u, mu, wf, w.rho, w.lambda1, w.lambda2), ub + 3 * fb),
        "grad_adj": (lambda: dr.tv4d_grad_adj(plan, wf, ua, w.lambda2), fb + ub),
        "grad": (lambda: dr.tv4d_grad(plan, u, wf, w.lambda2), ub + fb),
        "normal": (lambda: dr.tv4d_normal(plan, u, ua, w.lambda2, 1.0), 3 * ub),
    }
    out = {"hbm_peak_gbs": peak, "peak_source": src,
           "note": "one call each through the C ABI, inputs %.0f MB > L2; algorithmic bytes: prox u + 3 fields, "
                   "grad_adj and grad one field + u, normal (out += D^T D x, as in a CG step) 3 x u; u alone "
                   "(%.0f MB) fits in L2" % ((ub + fb) / 1e6, ub / 1e6)}
    for name, (fn, nbytes) in calls.items():
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        gbs = nbytes / (ms * 1e-3) / 1e9
        out[name] = {"ms": ms, "bytes": nbytes, "achieved_gbs": gbs, "frac": gbs / peak}
    return out


def run_fbp(plan, g, w, dev, stream):
    """FBP initial guess with one window per half-turn, timed on the device."""
    import torch

    from paper_1809_09725_gb300 import dynrecon as dr

    ufbp = torch.empty(plan.u_shape(), dtype=torch.float32, device=dev)
    n_win = int(round(w.n_halfturns))
    for _ in range(3):
        dr.fbp_init(plan, g, ufbp, n_win)
    torch.cuda.synchronize()
    fe0, fe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fe0.record(stream)
    for _ in range(5):
        dr.fbp_init(plan, g, ufbp, n_win)
    fe1.record(stream)
    torch.cuda.synchronize()
    fbp = {"ms": fe0.elapsed_time(fe1) / 5, "windows": n_win,
           "note": "Shepp-Logan filter of nz*K rows + one folded back-projection; includes the "
                   "blocking table upload of each call"}
    return fbp


def run_slabs(w, theta, t, g_np, dev, slab=4, iters=10):
    """Chambolle-Pock with the volume in pinned host memory, streamed in slabs
    (cp_solve_slabs), against the same iterations with the volume resident on
    the device; the same operator norm for both."""
    import torch

    from paper_1809_09725_gb300 import dynrecon as dr

    plan = dr.Plan(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt, dr.F32)
    g = torch.from_numpy(g_np.astype(np.float32)).to(dev)
    u = torch.zeros(plan.u_shape(), dtype=torch.float32, device=dev)
    prm = dr.solve_params(dr.CHAMBOLLE_POCK, iters=1, lambda1=w.lambda1, lambda2=w.lambda2)
    L = dr.admm_solve(plan, g, u, prm, want_objective=False)["op_norm"]
    prm = dr.solve_params(dr.CHAMBOLLE_POCK, iters=iters, lambda1=w.lambda1, lambda2=w.lambda2, op_norm=L)
    u.zero_()
    dr.admm_solve(plan, g, u, prm, want_objective=False)
    u.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dr.admm_solve(plan, g, u, prm, want_objective=False)
    torch.cuda.synchronize()
    t_in = time.perf_counter() - t0
    gh = torch.from_numpy(g_np.astype(np.float32)).pin_memory().numpy()
    uh = np.zeros(plan.u_shape(), dtype=np.float32)
    dr.cp_solve_slabs(plan, gh, uh, dr.solve_params(dr.CHAMBOLLE_POCK, iters=1, lambda1=w.lambda1,
                                                    lambda2=w.lambda2, op_norm=L), slab, want_objective=False)
    # per-iteration cost = difference of two runs (removes the per-call set-up:
    # pinned host state, device buffers, first-touch of the host arrays)
    times = []
    for n_it in (iters, 3 * iters):
        uh[...] = 0.0
        prm_n = dr.solve_params(dr.CHAMBOLLE_POCK, iters=n_it, lambda1=w.lambda1, lambda2=w.lambda2, op_norm=L)
        t0 = time.perf_counter()
        dr.cp_solve_slabs(plan, gh, uh, prm_n, slab, want_objective=False)
        times.append(time.perf_counter() - t0)
    t_sl = (times[1] - times[0]) / 2.0
    setup_s = times[0] - t_sl
    V = w.voxels()
    per_slice = (w.N * w.N * w.m * 4, w.K * w.ns * 4, w.N * w.N * w.nt * 16)  # u, data, dual field
    nslab = (w.nz + slab - 1) // slab
    h2d = w.nz * (2 * per_slice[0] + 2 * per_slice[1] + per_slice[2]) + (nslab - 1) * per_slice[0]
    d2h = w.nz * (2 * per_slice[0] + per_slice[1] + per_slice[2])
    return {"slab_nz": slab, "iters": iters, "ms_per_iter_streamed": 1e3 * t_sl / iters,
            "ms_per_iter_in_core": 1e3 * t_in / iters,
            "streamed_voxel_projection_per_s": 2.0 * w.K * V * iters / t_sl,
            "h2d_bytes_per_iter": int(h2d), "d2h_bytes_per_iter": int(d2h),
            "copy_gbs": (h2d + d2h) * iters / t_sl / 1e9, "setup_s_per_call": setup_s,
            "note": "Chambolle-Pock, same operator norm; streamed = volume in pinned host memory, per-iteration "
                    "time from the difference of a %d- and a %d-iteration call" % (iters, 3 * iters)}


def load_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    (profiles/traffic.txt), or None if that kernel was not captured."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        for line in open(path):
            parts = line.split()
            if len(parts) == 2 and not line.startswith("#") and parts[0] == kernel:
                return int(parts[1])
    except OSError:
        pass
    return None


def cpu_baseline(w, theta, t, g_np, sample_slices=None):
    """The FP64 oracle as it stands, on the host cores: one forward and one
    back-projection of the same workload (bounded sample)."""
    import oracle
    nz = w.nz if sample_slices is None else sample_slices
    P = oracle.Problem(w.N, w.N, nz, w.ns, theta, t, w.basis, w.m, w.nt)
    rng = np.random.default_rng(1)
    u = rng.standard_normal((nz, w.N, w.N, w.m))
    t0 = time.perf_counter()
    P.fwd(u)
    P.adj(g_np[:nz])
    el = time.perf_counter() - t0
    units = 2 * w.K * w.N * w.N * nz
    return {"value": units / el, "unit": "voxel*projection/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "one forward + one back-projection, FP64 oracle, %d slices of the workload (%.1f s)"
                      % (nz, el)}


def cpu_baseline_1thread(w):
    """The oracle on one host thread (OMP_NUM_THREADS=1, a separate process):
    one forward and one back-projection of one slice of the workload."""
    code = (
        "import sys, time, numpy as np; sys.path.insert(0, %r); import oracle\n"
        "from paper_1809_09725_gb300 import synth\n"
        "w = synth.WORKLOADS[%r]; theta, t = synth.scan(w.K, w.n_halfturns, w.mod_pi)\n"
        "P = oracle.Problem(w.N, w.N, 1, w.ns, theta, t, w.basis, w.m, w.nt)\n"
        "rng = np.random.default_rng(1); u = rng.standard_normal((1, w.N, w.N, w.m))\n"
        "g = rng.standard_normal((1, w.K, w.ns))\n"
        "t0 = time.perf_counter(); P.fwd(u); P.adj(g); print(time.perf_counter() - t0)\n"
    ) % (os.path.dirname(os.path.abspath(__file__)), w.name)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        el = float(out.stdout.strip().splitlines()[-1])
    except Exception as exc:  # noqa: BLE001 -- reported in the JSON line
        return {"error": repr(exc)[:200]}
    units = 2 * w.K * w.N * w.N
    return {"value": units / el, "unit": "voxel*projection/s", "cores": 1, "kind": "oracle",
            "sample": "one forward + one back-projection, FP64 oracle, 1 slice, one thread (%.1f s)" % el}


def accuracy_vs_oracle(w, theta, t, g_np, dev, iters=3):
    """Relative L2 error of the GPU solve against the FP64 oracle running the
    same ADMM-CG iterations on a 1-slice cut of the workload."""
    import torch

    import oracle
    from paper_1809_09725_gb300 import dynrecon as dr

    g1 = g_np[:1]
    P = oracle.Problem(w.N, w.N, 1, w.ns, theta, t, w.basis, w.m, w.nt)
    t0 = time.perf_counter()
    uo, oo, _ = P.admm_cg(g1, np.zeros((1, w.N, w.N, w.m)), iters, w.n_cg, w.lambda1, w.lambda2, w.rho)
    t_or = time.perf_counter() - t0
    out = {"cut": "slice 0 of the workload, %d ADMM-CG iterations from zero" % iters, "oracle_s": t_or}
    for name, prec in (("fp32", dr.F32), ("bf16", dr.BF16)):
        plan = dr.Plan(w.N, w.N, 1, w.ns, theta, t, w.basis, w.m, w.nt, prec)
        dt = getattr(torch, plan.storage_dtype)
        u = torch.zeros(plan.u_shape(), dtype=dt, device=dev)
        prm = dr.solve_params(dr.ADMM_CG, iters=iters, n_cg=w.n_cg, lambda1=w.lambda1, lambda2=w.lambda2, rho=w.rho)
        res = dr.admm_solve(plan, torch.from_numpy(g1).to(dt).to(dev), u, prm)
        uu = u.to(torch.float64).cpu().numpy()
        out[name] = {"rel_l2_u": float(np.linalg.norm(uu - uo) / np.linalg.norm(uo)),
                     "rel_objective": float(abs(res["objective"][-1] - oo[-1]) / abs(oo[-1]))}
    return out


def run_serving_sweep(a, device, utilisations=(0.5, 0.8, 0.95)):
    """The reduced request stream at arrival rates giving the stated
    utilisations: rho = lambda E[S], E[S] the mean time of a job solved alone."""
    from paper_1809_09725_gb300 import dynrecon as dr
    jobs = serving_jobs(a.serving_jobs)
    prm = lambda: dr.solve_params(dr.ADMM_CG, iters=30, n_cg=4, lambda1=1e-3, lambda2=1.0, rho=1e-2)
    service = []
    for j in jobs:  # each job alone, through the same public call as a worker
        plan = dr.Plan(j["N"], j["N"], j["nz"], j["N"], j["theta"], j["t"], j["basis"], j["m"], j["nt"], dr.F32)
        uh = np.zeros((j["nz"], j["N"], j["N"], j["m"]), dtype=np.float32)
        gh = j["g"].astype(np.float32)
        t0 = time.perf_counter()
        dr.admm_solve(plan, gh, uh, prm(), want_objective=False)
        service.append(time.perf_counter() - t0)
        plan.close()
    es = float(np.mean(service))
    out = {"mean_service_s": es, "points": []}
    for rho in utilisations:
        rng = np.random.default_rng(int(rho * 1000))
        arrivals = np.cumsum(rng.exponential(es / rho, size=len(jobs)))
        descs, keep = [], []
        for j in jobs:
            gh = j["g"].astype(np.float32)
            uh = np.zeros((j["nz"], j["N"], j["N"], j["m"]), dtype=np.float32)
            keep.append((gh, uh))
            descs.append(dr.job_desc(j["N"], j["N"], j["nz"], j["N"], j["theta"], j["t"], j["basis"], j["m"],
                                     j["nt"], dr.F32, prm(), gh, uh))
        srv = dr.Server(device=device, budget_bytes=150 * 10 ** 9, slots=8)
        t0 = time.perf_counter()
        ids = []
        for arr, d in zip(arrivals, descs):
            wait = arr - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            ids.append(srv.submit(d))
        res = [srv.wait(i, timeout_s=600.0) for i in ids]
        st = srv.stats()
        srv.close()
        out["points"].append({"utilisation": rho, "arrival_rate_per_s": rho / es,
                              "p50_latency_s": st["p50_latency_s"], "p99_latency_s": st["p99_latency_s"],
                              "completed": st["completed"], "failed": st["failed"],
                              "max_queue_s": max(r["queue_s"] for r in res)})
    return out


def run_batched(dev, n_jobs=16, iters=10, seed=180903):
    """Uneven jobs of the batched configuration (N in {128,256,512}, nz in
    [1,32], K in {720,1800,3600} over 4-20 half-turns, m in {4,8,16}, Fourier or
    Legendre; first n_jobs of the seeded list, seeded random data) solved
    together by admm_solve_batch (one CUDA graph per iteration)."""
    import torch

    from paper_1809_09725_gb300 import dynrecon as dr
    from paper_1809_09725_gb300 import synth
    rng = np.random.default_rng(seed)
    plans, gs, us, prms, units = [], [], [], [], 0
    for i in range(n_jobs):
        N = int(rng.choice([128, 256, 512]))
        nz = int(rng.integers(1, 33))
        K = int(rng.choice([720, 1800, 3600]))
        ht = int(rng.integers(4, 21))
        m = int(rng.choice([4, 8, 16]))
        basis = int(rng.integers(0, 2))
        theta, t = synth.scan(K, ht)
        p = dr.Plan(N, N, nz, N, theta, t, basis, m, ht, dr.F32)
        plans.append(p)
        gen = torch.Generator(device=dev).manual_seed(seed * 1000 + i)
        gs.append(torch.randn(p.g_shape(), generator=gen, device=dev))
        us.append(torch.zeros(p.u_shape(), device=dev))
        prms.append(dr.solve_params(dr.ADMM_CG, iters=iters, n_cg=4, lambda1=1e-3, lambda2=1.0, rho=1e-2))
        units += 2 * 5 * iters * K * N * N * nz
    t_setup = time.perf_counter()
    for p in plans:
        p.autotune()
    t_setup = time.perf_counter() - t_setup
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dr.admm_solve_batch(plans, gs, us, prms)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    # the same jobs one after another (same plans, same variants)
    for u in us:
        u.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for p, g, u, prm in zip(plans, gs, us, prms):
        dr.admm_solve(p, g, u, prm, want_objective=False)
    torch.cuda.synchronize()
    el_seq = time.perf_counter() - t0
    folded = sum(1 for p in plans if p.info()["fwd_variant"] in (1, 2))
    return {"jobs": n_jobs, "iters": iters, "seconds": el, "voxel_projection_per_s": units / el,
            "sequential_seconds": el_seq, "sequential_voxel_projection_per_s": units / el_seq,
            "jobs_on_folded_projectors": folded, "autotune_s": t_setup,
            "note": "seeded random data of each job's shape (throughput does not depend on the values); "
                    "autotuning timed separately; jobs whose angles do not repeat mod pi use the direct pair"}


def bench_config(world: int) -> dict:
    """The workload both arms are quoted on."""
    return {"workload": "ellipsoids256: nz=16 x 256^2 voxels, 256 bins, K=1800 over 10 half-turns, "
                        "m=8 Fourier, nt=10, ADMM-CG n_cg=4, FP32",
            "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": "per-iteration working set 0.54 GB > 129 MB L2 (duals stream through every iteration)"}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1809_09725_gb300 import synth
    w = synth.WORKLOADS[a.workload]
    theta, t, g_np = synth.make_data(w)
    # slices per step: 4 (about half a second on 16 host cores), fewer for
    # long runs, so that the whole reference run stays within minutes
    nz = 4 if a.steps <= 100 else (2 if a.steps <= 200 else 1)
    for _ in range(a.warmup):
        cpu_baseline(w, theta, t, g_np, sample_slices=1)
    t0 = time.perf_counter()
    vals = []
    for _ in range(a.steps):
        vals.append(cpu_baseline(w, theta, t, g_np, sample_slices=nz))
    el = time.perf_counter() - t0
    units = 2 * w.K * w.N * w.N * nz * a.steps
    value = units / el
    line = {"impl": "reference", "metric": "voxel*projection updates/s (dynamic projector + back-projector "
                                           "applications inside ADMM-CG iterations)",
            "value": value, "unit": "voxel*projection/s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": el * 1e3 / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded moving ellipsoids, Poisson 1e4)",
            "config": bench_config(1),
            "cpu_baseline": {"value": value, "unit": "voxel*projection/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": "per step: one forward + one back-projection on %d of "
                                                         "the %d slices of the workload, FP64 oracle on the host "
                                                         "cores (no GPU used)" % (nz, w.nz)},
            "e2e": {"value": value, "unit": "voxel*projection/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
