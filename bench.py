"""Benchmark of the dynamic-tomography hot path on GB300.

Workload (default, the large mixed-precision volume): 64 slices of
1024^2 voxels, 1024 detector bins, K = 6000 projections over 20 continuous
half-turns, m = 16 shifted-Legendre coefficient volumes, nt = 20 frames,
sharp-edged moving ellipsoids with Poisson noise (1e4 photons), FP32,
reconstructed with ADMM-CG (4 CG steps per u-step).

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
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ellipsoids1024")
    ap.add_argument("--op-reps", type=int, default=5, help="timed launches of each projector for the roofline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-iters", type=int, default=5, help="ADMM-CG iterations of each end-to-end job")
    ap.add_argument("--e2e-jobs", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-jobs", type=int, default=24, help="jobs of the reduced serving stream")
    ap.add_argument("--serving-window", type=float, default=30.0,
                    help="seconds the full-size serving stream runs before the backlog is canceled")
    ap.add_argument("--batch-jobs", type=int, default=64)
    ap.add_argument("--extra-workloads", default="ellipsoids256",
                    help="comma-separated workloads also timed (FP32 ADMM-CG) as extra keys")
    ap.add_argument("--no-slabs", action="store_true", help="skip the slab-streaming measurement")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the BF16, TV-kernel, FBP, extra-workload, batched, slab and serving measurements")
    ap.add_argument("--variant", default=None,
                    help="force projector variants 'fwd,adj' (0 direct, 1 fold, 2 fold in two kernels: forward "
                         "only); default: autotuned")
    ap.add_argument("--fold2-config", default=None,
                    help="with --variant 2,x: fix the two-kernel folded forward's "
                         "'group,threads,lines[,split[,async[,rays_per_thread]]]' instead of the default")
    ap.add_argument("--fold-adj-angles", type=int, default=0,
                    help="with --variant x,1: fix the folded adjoint's distinct angles per pipeline stage")
    ap.add_argument("--slices", type=int, default=0,
                    help="with --profile-small: the workload's geometry on this many slices (a small case for ncu)")
    ap.add_argument("--profile-small", action="store_true",
                    help="run only one launch of each projector call and of each TV stencil on the workload "
                         "(for ncu captures)")
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


def time_projectors(plan, dev, stream, reps=5, dtype=None):
    """Mean device time (CUDA events on the launching stream) of one forward
    and one back-projection through the C ABI, in the variants the plan
    selected, on random inputs of the plan's shapes."""
    import torch

    from paper_1809_09725_gb300 import dynrecon as dr
    dt = dtype or getattr(torch, plan.storage_dtype)
    p_in = torch.randn(plan.u_shape(), dtype=torch.float32, device=dev).to(dt)
    gbuf = torch.empty(plan.g_shape(), dtype=dt, device=dev)
    ubuf = torch.empty(plan.u_shape(), dtype=dt, device=dev)
    for _ in range(2):
        dr.dyn_radon_fwd(plan, p_in, gbuf)
        dr.dyn_radon_adj(plan, gbuf, ubuf)
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
    out = ev[0].elapsed_time(ev[1]) / reps, ev[1].elapsed_time(ev[2]) / reps
    del p_in, gbuf, ubuf
    return out


def roofline_of(w, theta, info, fwd_ms, adj_ms, tune=None):
    """Roofline of the dominant projector call (the slower of the pair):
    FP32 ALU flops of the half-turn fold (or of the direct form) against
    the derived FP32 pipe peak; algorithmic HBM bytes against the measured
    copy bandwidth; algorithmic shared-memory bytes against the derived
    shared-memory bandwidth (side key)."""
    U = info["unique_angles"]
    if fwd_ms >= adj_ms:
        variant = info["fwd_variant"]
        kname = {1: "fold_fwd_kernel", 2: "fold_fwd_kernel(static)+fold_dist_kernel"}.get(variant, "fwd_kernel")
        launch_ms = fwd_ms
        smem_bytes = algorithmic_smem_bytes(w, theta, variant, U)
    else:
        variant = info["adj_variant"]
        kname = "fold_adj_kernel+fold_data_kernel" if variant == 1 else "adj_kernel"
        launch_ms = adj_ms
        smem_bytes = 2 * w.m * 4 * (U if variant == 1 else w.K) * w.voxels()
    flops = algorithmic_flops(w, variant, U)
    achieved = flops / (launch_ms * 1e-3) / 1e12
    peak = fp32_peak_tflops()
    hbm_bytes = 4 * (w.m * w.voxels() + w.K * w.ns * w.nz)  # read u + write g (or the reverse), FP32
    hbm_peak, hbm_src = hbm_peak_gbs()
    hbm_gbs = hbm_bytes / (launch_ms * 1e-3) / 1e9
    smem_achieved = smem_bytes / (launch_ms * 1e-3) / 1e12
    samples = joseph_samples(theta, w.N, w.N, w.ns) * w.nz if variant in (1, 2) else None
    traffic = load_traffic(kname, w.name)
    return {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic,
            "algorithmic_flops_per_launch": flops,
            "flops_formula": ("2 (2 m U V + m K ns nz), U distinct angles mod pi" if variant in (1, 2)
                              else "2 (m + 2) K V"),
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (max SM clock)",
            "joseph_samples_per_launch": samples,
            "hbm": {"achieved_gbs": hbm_gbs, "peak_gbs": hbm_peak, "frac": hbm_gbs / hbm_peak,
                    "algorithmic_bytes": hbm_bytes, "traffic": traffic, "peak_source": hbm_src},
            "smem": {"achieved_tbs": smem_achieved, "peak_tbs": smem_peak_tbs(),
                     "frac": smem_achieved / smem_peak_tbs(), "algorithmic_bytes": smem_bytes,
                     "peak_source": "derived: 152 SMs x 128 B/clk x 2.07 GHz"},
            "launch_ms": launch_ms, "fwd_ms": fwd_ms, "adj_ms": adj_ms,
            "variants": {"unique_angles": U, "fwd": info["fwd_variant"], "adj": info["adj_variant"],
                         "fold2_group_threads_lines_split_async_rpt": [
                             info["fold2_group"], info["fold2_threads"], info["fold2_lines"],
                             info["fold2_split"], info["fold2_async"], info["fold2_rays_per_thread"]],
                         "fold_adj_angles_per_stage": info["fold_adj_angles"],
                         "autotune_ms_fwd_direct_fold_adj_direct_fold_fwd_fold2": tune}}


def launches_per_iteration(info, n_cg):
    """Kernels one ADMM-CG iteration launches: n_cg + 1 forwards and adjoints
    (the folded adjoint is two launches: data fold + back-projection; the
    two-kernel folded forward too: static transforms + distribution; with
    both folded, a CG step's R*R p is the folded normal operator: static
    transforms, Gram mix, back-projection), n_cg + 1 D^T D (right-hand side +
    CG steps), prox, D^T w, n_cg updates, n_cg - 1 direction updates, the
    fidelity dot and the iteration counter."""
    adj_launches = 2 if info["adj_variant"] == 1 else 1
    fwd_launches = 2 if info["fwd_variant"] == 2 else 1
    normal_launches = 3 if (info["fwd_variant"], info["adj_variant"]) == (2, 1) else fwd_launches + adj_launches
    per_iter = (1 + fwd_launches + adj_launches) + n_cg * (1 + normal_launches) + 2 * n_cg + 3
    return per_iter, fwd_launches


def solve_timed(plan, g, u, w, steps, warmup, tdist, dev, local, want_obj=True):
    """W untimed ADMM-CG iterations (autotuning on the first call), then
    exactly `steps` iterations in one admm_solve call bracketed by a barrier
    and a device synchronisation, timed with CUDA events on the plan's
    stream, clocks sampled meanwhile."""
    import torch

    from paper_1809_09725_gb300 import dynrecon as dr
    prm = dr.solve_params(dr.ADMM_CG, iters=warmup, n_cg=w.n_cg, lambda1=w.lambda1, lambda2=w.lambda2,
                          rho=w.rho)
    dr.admm_solve(plan, g, u, prm, want_objective=False)
    u.zero_()
    torch.cuda.synchronize()
    prm = dr.solve_params(dr.ADMM_CG, iters=steps, n_cg=w.n_cg, lambda1=w.lambda1, lambda2=w.lambda2,
                          rho=w.rho)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        if tdist is not None:
            tdist.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        res = dr.admm_solve(plan, g, u, prm, want_objective=want_obj)
        e1.record(stream)
        torch.cuda.synchronize()
        if tdist is not None:
            tdist.barrier()
    ms = barrier_max(tdist, e0.elapsed_time(e1), dev)
    return ms, res, clk.summary()


def run_ours(a):
    import torch

    from paper_1809_09725_gb300 import dynrecon as dr
    from paper_1809_09725_gb300 import synth

    rank, world, tdist = dist_init(a.gpus)
    local = int(os.environ.get("LOCAL_RANK", rank))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    w = synth.WORKLOADS[a.workload]
    if a.profile_small and a.slices > 0:
        import dataclasses
        w = dataclasses.replace(w, nz=a.slices)
    t_data = time.perf_counter()
    theta, t, g_np = synth.make_data(w)
    g32 = g_np.astype(np.float32)
    del g_np
    t_data = time.perf_counter() - t_data
    plan = dr.Plan(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt, dr.F32)
    g = torch.from_numpy(g32).to(dev)
    u = torch.zeros(plan.u_shape(), dtype=torch.float32, device=dev)
    units_per_iter = 2 * (w.n_cg + 1) * w.K * w.voxels()  # projector applications x K V
    if a.variant:
        fv, av = (int(x) for x in a.variant.split(","))
        plan.set_variant(fv, av)
        if fv == dr.FOLD2 and a.fold2_config:
            set_fold2_config(plan, a.fold2_config)
        if av == dr.FOLD and a.fold_adj_angles > 0:
            plan.set_fold_adj_stage(a.fold_adj_angles)

    if a.profile_small:
        # one launch of the selected projector pair on the workload, for profiler captures
        if not a.variant:
            plan.autotune()
        uin = torch.randn(plan.u_shape(), dtype=torch.float32, device=dev)
        gout = torch.empty_like(g)
        dr.dyn_radon_fwd(plan, uin, gout)
        dr.dyn_radon_adj(plan, g, u)
        # and one launch of each TV stencil (D^T D, D^T, prox, D) on the same volume
        mu = torch.randn(plan.field_shape(), dtype=torch.float32, device=dev) * 1e-3
        wf = torch.empty_like(mu)
        dr.tv4d_normal(plan, uin, u, w.lambda2, 1.0)
        dr.tv4d_grad_adj(plan, mu, u, w.lambda2)
        dr.tv4d_prox(plan, uin, mu, wf, w.rho, w.lambda1, w.lambda2)
        dr.tv4d_grad(plan, uin, wf, w.lambda2)
        torch.cuda.synchronize()
        print(json.dumps({"profile_small": True, "info": plan.info()}))
        return

    t_tune = time.perf_counter()
    tune = plan.autotune() if not a.variant else None
    t_tune = time.perf_counter() - t_tune
    ms, res, clocks = solve_timed(plan, g, u, w, a.steps, a.warmup, tdist, dev, local)
    value = replica_units(units_per_iter * a.steps, world) / (ms * 1e-3)
    obj = res["objective"]
    info = plan.info()

    # the dominant kernels alone, on the same stream, in the variants the solver used
    fwd_ms, adj_ms = time_projectors(plan, dev, stream, reps=a.op_reps)
    roof = roofline_of(w, theta, info, fwd_ms, adj_ms, tune)
    per_iter, fwd_launches = launches_per_iteration(info, w.n_cg)

    # end to end through the public call with host buffers: each step is one
    # reconstruction job of e2e_iters iterations from pinned host memory
    e2e = None
    if not a.no_e2e:
        e2e = run_e2e(plan, g32, w, a.e2e_iters, a.e2e_jobs, tdist, dev, units_per_iter, world)

    extras = {}
    cpu = None
    if rank == 0 and not a.no_cpu_baseline:
        cpu, acc_ops = cpu_baseline_and_accuracy(plan, w, theta, t, g32, dev)
        cpu["one_thread"] = cpu_baseline_1thread(w)
        extras["operator_accuracy_vs_fp64_oracle"] = acc_ops
    del g, u
    torch.cuda.empty_cache()

    u_ref = None
    if rank == 0 and not a.no_extras:
        extras["tv_kernels"] = guarded(run_tv_kernels, plan, w, dev, stream)
        extras["fbp_init"] = guarded(run_fbp, plan, torch.from_numpy(g32).to(dev), w, dev, stream)
        torch.cuda.empty_cache()
        # the FP32 plan's iterate after a few iterations, for the reduced-precision variants
        u_ref = torch.zeros(plan.u_shape(), dtype=torch.float32, device=dev)
        dr.admm_solve(plan, torch.from_numpy(g32).to(dev), u_ref,
                      dr.solve_params(dr.ADMM_CG, iters=3, n_cg=w.n_cg, lambda1=w.lambda1, lambda2=w.lambda2,
                                      rho=w.rho), want_objective=False)
        fp32_solver_gb = plan.device_bytes() / 1e9
    plan.close()
    torch.cuda.empty_cache()
    if rank == 0 and not a.no_extras:
        extras["reduced_precision"] = guarded(run_precision_variants, w, theta, t, g32, u_ref, 3, dev, stream, a)
        if isinstance(extras["reduced_precision"], dict) and "error" not in extras["reduced_precision"]:
            extras["reduced_precision"]["fp32_solver_device_gb"] = fp32_solver_gb
        del u_ref
        torch.cuda.empty_cache()
    del g32
    if rank == 0 and not a.no_extras:
        for name in a.extra_workloads.split(",") if a.extra_workloads else []:
            extras[name] = guarded(run_workload_line, name, dev, stream, local, a)
            torch.cuda.empty_cache()
        extras["disks64_fp64_whole_solve"] = guarded(run_disks_fp64, dev)
        extras["batched_jobs"] = guarded(run_batched, dev, a.batch_jobs)
        if not a.no_slabs:
            extras["slab_streaming"] = guarded(run_slabs_workload, "ellipsoids256", dev)
    if not a.no_serving and rank == 0 and not a.no_extras:
        extras["serving"] = {name: guarded(run_serving_c5, local, prec, a.serving_window) for name, prec in
                             (("c5_fp32", dr.F32), ("c5_fp32_bf16fields", dr.F32 | dr.FIELDS_BF16))}
        outs = {}
        for name, prec in (("reduced_fp32", dr.F32), ("reduced_fp32_bf16fields", dr.F32 | dr.FIELDS_BF16),
                           ("reduced_bf16", dr.BF16)):
            outs[name] = []
            extras["serving"][name] = guarded(run_serving, a, local, prec, outs[name])
        extras["serving"]["reduced_rel_l2_vs_fp32"] = guarded(serving_differences, outs)
        extras["serving"]["load_sweep_reduced_fp32"] = guarded(run_serving_sweep, a, local)

    if rank == 0:
        line = {
            "metric": "voxel*projection updates/s (dynamic projector + back-projector applications "
                      "inside ADMM-CG iterations)",
            "value": value, "unit": "voxel*projection/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded %s, exact line integrals + Poisson noise at 1e4 photons)" % (
                "sharp-edged moving ellipsoids" if w.name == "ellipsoids1024" else "moving ellipsoids"),
            "config": bench_config(w, world),
            "admm_iters_per_s": a.steps * world / (ms * 1e-3),
            "objective_first_last": [float(obj[0]), float(obj[-1])],
            "clocks": clocks,
            "e2e": e2e,
            "gpu_launches": per_iter * a.steps + fwd_launches + 1,  # + the final fidelity (forward + dot)
            "roofline": roof,
            "cpu_baseline": cpu,
            "setup_s": {"data": t_data, "autotune": t_tune},
        }
        line.update(extras)
        print(json.dumps(line))


def guarded(fn, *args, **kw):
    """Run one optional measurement; its failure is reported in its key
    instead of ending the benchmark."""
    try:
        return fn(*args, **kw)
    except Exception as exc:  # noqa: BLE001 -- reported in the JSON line
        import traceback
        return {"error": repr(exc)[:300], "where": traceback.format_exc().splitlines()[-3:]}


def run_e2e(plan, g32, w, iters, jobs, tdist, dev, units_per_iter, world):
    """The same metric through admm_solve on pinned host buffers: every job
    copies its data and initial guess in and its result out inside the
    timed region (host wall clock, device synchronised on both sides)."""
    import torch

    from paper_1809_09725_gb300 import dynrecon as dr
    gh = torch.from_numpy(g32).pin_memory()
    uh = torch.zeros(plan.u_shape(), dtype=torch.float32).pin_memory()
    ghn, uhn = gh.numpy(), uh.numpy()
    prm = lambda n: dr.solve_params(dr.ADMM_CG, iters=n, n_cg=w.n_cg, lambda1=w.lambda1, lambda2=w.lambda2,
                                    rho=w.rho)
    dr.admm_solve(plan, ghn, uhn, prm(1), want_objective=False)  # staging buffers allocated once
    torch.cuda.synchronize()
    if tdist is not None:
        tdist.barrier()
    t0 = time.perf_counter()
    for _ in range(jobs):
        uhn[...] = 0.0
        dr.admm_solve(plan, ghn, uhn, prm(iters), want_objective=False)
    torch.cuda.synchronize()
    el = barrier_max(tdist, time.perf_counter() - t0, dev)
    out = {"value": units_per_iter * iters * jobs * world / el, "unit": "voxel*projection/s",
           "h2d_bytes_per_step": int(g32.nbytes + uhn.nbytes), "d2h_bytes_per_step": int(uhn.nbytes),
           "step": "one %d-iteration reconstruction job via admm_solve on pinned host buffers "
                   "(data and initial guess in, result out)" % iters,
           "jobs": jobs, "s_per_job": el / jobs}
    del gh, uh
    return out


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


def run_serving(a, device, prec, results=None):
    """Submit the request stream to the serving loop in real time; report
    latency percentiles and aggregate projector throughput.  results: a list
    that receives each job's reconstruction (host arrays)."""
    from paper_1809_09725_gb300 import dynrecon as dr
    jobs = serving_jobs(a.serving_jobs)
    descs, outs = [], []
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
        outs.append(uh)
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
    if results is not None:
        results.extend(outs)
    units = sum(2 * 5 * 30 * j["K"] * j["N"] * j["N"] * j["nz"] for j in jobs)
    return {"jobs": len(jobs), "completed": st["completed"], "failed": st["failed"],
            "p50_latency_s": st["p50_latency_s"], "p99_latency_s": st["p99_latency_s"],
            "voxel_projection_per_s": units / wall, "wall_s": wall,
            "peak_device_gb": st["peak_device_bytes"] / 1e9, "budget_gb": 150,
            "stream": "Poisson 4 jobs/s, first %d arrivals; N in {128,256}, nz 4-16, K 360-3600 over 4-20 "
                      "half-turns, m in {4,8,16}, 30 ADMM-CG iterations" % len(jobs),
            "max_queue_s": max(r["queue_s"] for r in res),
            "errors": [{"job": i, "rc": r["rc"], "error": r["error"]} for i, r in enumerate(res) if r["rc"] != 0]}


def serving_stream_c5(n=64, seed=180905):
    """The serving stream of 4D reconstruction requests: Poisson arrivals at
    4 jobs/s; grid N uniform in {256, 512, 1024, 2048}, nz in 8..128, K in
    900..7200 projections over 4..20 continuous half-turns, m in 4..32,
    Fourier or Legendre, 30 ADMM-CG iterations.  Sizes only: a job's data
    are made when it is submitted."""
    from paper_1809_09725_gb300 import synth
    rng = synth.rng_for(seed)
    t_arr = np.cumsum(rng.exponential(1.0 / 4.0, size=n))
    jobs = []
    for i in range(n):
        N = int(rng.choice([256, 512, 1024, 2048]))
        nz = int(rng.integers(8, 129))
        K = int(rng.integers(900, 7201))
        m = int(rng.integers(4, 33))
        ht = int(rng.integers(4, 21))
        basis = int(rng.integers(0, 2))
        jobs.append(dict(arrival=float(t_arr[i]), N=N, nz=nz, K=K, m=m, ht=ht, basis=basis, seed=seed * 100 + i))
    return jobs


def run_serving_c5(device, prec, window_s=60.0, n=64, budget=150 * 10 ** 9, slots=8):
    """The serving stream in real time against the 150 GB budget: jobs whose
    state cannot fit the budget are refused at submission (DR_ENOMEM); the
    rest queue and are admitted as memory and slots free up.  At window_s
    after the first arrival every job not finished is canceled (running ones
    stop between iterations).  Latency is counted from each job's scheduled
    arrival (the submission can lag it while a large job's data are made)."""
    import torch

    from paper_1809_09725_gb300 import dynrecon as dr
    from paper_1809_09725_gb300 import synth
    jobs = serving_stream_c5(n)
    prm = lambda: dr.solve_params(dr.ADMM_CG, iters=30, n_cg=4, lambda1=1e-3, lambda2=1.0, rho=1e-2)
    srv = dr.Server(device=device, budget_bytes=budget, slots=slots)
    refused, live, keep = [], {}, {}
    t0 = time.perf_counter()
    for i, j in enumerate(jobs):
        dt = j["arrival"] - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        if time.perf_counter() - t0 > window_s:
            break
        theta, t = synth.scan(j["K"], j["ht"])
        size_only = dr.job_desc(j["N"], j["N"], j["nz"], j["N"], theta, t, j["basis"], j["m"], j["ht"], prec, prm(),
                                None, None)
        need = dr.job_device_bytes(size_only)
        if need > budget:
            refused.append({"job": i, "N": j["N"], "nz": j["nz"], "K": j["K"], "m": j["m"], "gb": need / 1e9})
            continue
        # data: exact line integrals of 5 moving disks, the same on every slice
        blobs = synth.disks(synth.rng_for(j["seed"]), j["N"], 5)
        g1 = synth.sinogram(blobs, theta, t, j["N"], 1)[0].astype(np.float32)
        if prec & ~dr.FIELDS_BF16 == dr.BF16:
            g1 = torch.from_numpy(g1).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
        g = np.empty((j["nz"], j["K"], j["N"]), dtype=g1.dtype)
        g[...] = g1[None]
        u = np.zeros((j["nz"], j["N"], j["N"], j["m"]), dtype=g1.dtype)
        d = dr.job_desc(j["N"], j["N"], j["nz"], j["N"], theta, t, j["basis"], j["m"], j["ht"], prec, prm(), g, u)
        jid = srv.submit(d)
        live[jid] = (i, time.perf_counter() - t0 - j["arrival"])
        keep[jid] = (d, g, u)
    left = window_s - (time.perf_counter() - t0)
    deadline = time.perf_counter() + max(0.0, left)
    done = {}
    for jid in list(live):
        r = srv.wait(jid, timeout_s=max(0.0, deadline - time.perf_counter()))
        if r["rc"] != dr.DR_ETIMEOUT:
            done[jid] = r
    for jid in live:
        if jid not in done:
            try:
                srv.cancel(jid)
            except Exception:  # noqa: BLE001 -- finished between the wait and the cancel
                pass
    for jid in live:
        if jid not in done:
            done[jid] = srv.wait(jid, timeout_s=600.0)
    st = srv.stats()
    srv.close()
    lat = sorted(done[jid]["latency_s"] + live[jid][1] for jid in live if done[jid]["state"] == dr.JOB_DONE)
    units = 0.0
    for jid in live:
        if done[jid]["state"] == dr.JOB_DONE:
            j = jobs[live[jid][0]]
            units += 2 * 5 * 30 * j["K"] * j["N"] * j["N"] * j["nz"]
    pct = lambda q: float(np.percentile(lat, q)) if lat else None
    return {"stream": "first %d Poisson arrivals at 4 jobs/s; N in {256,512,1024,2048}, nz 8-128, K 900-7200 "
                      "over 4-20 half-turns, m 4-32, 30 ADMM-CG iterations, %s" % (n, "BF16" if prec == dr.BF16 else
                                                                                   "FP32"),
            "window_s": window_s, "budget_gb": budget / 1e9, "slots": slots,
            "submitted": len(live), "refused_enomem": len(refused), "not_arrived_in_window": n - len(live) - len(refused),
            "completed": st["completed"], "canceled_at_window_end": st["canceled"], "failed": st["failed"],
            "p50_latency_s": pct(50), "p99_latency_s": pct(99),
            "voxel_projection_per_s": units / window_s, "peak_device_gb": st["peak_device_bytes"] / 1e9,
            "max_submit_lag_s": max([v[1] for v in live.values()] + [0.0]),
            "refused": refused[:16],
            "note": "the stream's admitted work is ~1e15 voxel*projection updates (tens of minutes of this GPU): "
                    "the window shows the latency of the jobs it completes and the backlog it leaves"}


def run_tv_kernels(plan, w, dev, stream, reps=5):
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
    out = {"hbm_peak_gbs": peak, "peak_source": src, "workload": w.name,
           "note": "one call each through the C ABI, inputs %.0f MB > L2; algorithmic bytes: prox u + 3 fields, "
                   "grad_adj and grad one field + u, normal (out += D^T D x, as in a CG step) 3 x u (u: %.0f MB)"
                   % ((ub + fb) / 1e6, ub / 1e6)}
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


def serving_differences(outs):
    """Largest relative L2 difference of the served reconstructions from the
    FP32 ones, per variant (the same jobs and parameters)."""
    import torch
    ref = outs["reduced_fp32"]
    res = {}
    for name, arrs in outs.items():
        if name == "reduced_fp32" or len(arrs) != len(ref):
            continue
        worst = 0.0
        for a_, b_ in zip(arrs, ref):
            av = (torch.from_numpy(a_.view(np.int16)).view(torch.bfloat16).double().numpy() if a_.dtype == np.uint16
                  else a_.astype(np.float64))
            bv = b_.astype(np.float64)
            nb = np.linalg.norm(bv)
            if nb > 0:
                worst = max(worst, float(np.linalg.norm(av - bv) / nb))
        res[name] = worst
    return res


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


def run_batched(dev, n_jobs=64, iters=10, seed=180903):
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
    batch_u = [u.clone() for u in us]
    # the same jobs one after another (same plans, same variants)
    for u in us:
        u.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for p, g, u, prm in zip(plans, gs, us, prms):
        dr.admm_solve(p, g, u, prm, want_objective=False)
    torch.cuda.synchronize()
    el_seq = time.perf_counter() - t0
    identical = sum(1 for a, b in zip(batch_u, us) if torch.equal(a, b))
    folded = sum(1 for p in plans if p.info()["fwd_variant"] in (1, 2))
    dev_gb = sum(p.device_bytes() for p in plans) / 1e9
    for p in plans:
        p.close()
    return {"jobs": n_jobs, "iters": iters, "seconds": el, "voxel_projection_per_s": units / el,
            "sequential_seconds": el_seq, "sequential_voxel_projection_per_s": units / el_seq,
            "jobs_bit_identical_to_alone": identical, "device_gb": dev_gb,
            "jobs_on_folded_projectors": folded, "autotune_s": t_setup,
            "note": "seeded random data of each job's shape (throughput does not depend on the values); "
                    "autotuning timed separately; jobs whose angles do not repeat mod pi use the direct pair"}


def load_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summary (profiles/traffic.txt: kernel, workload, bytes), or None if that
    kernel was not captured since it last changed."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        for line in open(path):
            parts = line.split()
            if len(parts) == 3 and not line.startswith("#") and parts[0] == kernel and parts[1] == workload:
                return int(parts[2])
    except OSError:
        pass
    return None


def cpu_baseline_and_accuracy(plan, w, theta, t, g32, dev):
    """The FP64 oracle as it stands, on the host cores: one forward and one
    back-projection of one slice of the workload with all K projections
    (bounded sample).  The same inputs go through the GPU plan (slice 0 of
    an otherwise zero volume / data set) and the outputs are compared."""
    import torch

    import oracle
    from paper_1809_09725_gb300 import dynrecon as dr
    P = oracle.Problem(w.N, w.N, 1, w.ns, theta, t, w.basis, w.m, w.nt)
    rng = np.random.default_rng(1)
    u0 = rng.standard_normal((1, w.N, w.N, w.m)).astype(np.float32).astype(np.float64)
    g0 = g32[:1].astype(np.float64)
    t0 = time.perf_counter()
    ref_g = P.fwd(u0)
    ref_u = P.adj(g0)
    el = time.perf_counter() - t0
    units = 2 * w.K * w.N * w.N
    cpu = {"value": units / el, "unit": "voxel*projection/s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": "one forward + one back-projection of 1 of the %d slices with all %d projections, FP64 "
                     "oracle (%.1f s)" % (w.nz, w.K, el)}
    uin = torch.zeros(plan.u_shape(), dtype=torch.float32, device=dev)
    uin[0] = torch.from_numpy(u0[0].astype(np.float32)).to(dev)
    gout = torch.empty(plan.g_shape(), dtype=torch.float32, device=dev)
    dr.dyn_radon_fwd(plan, uin, gout)
    gin = torch.zeros(plan.g_shape(), dtype=torch.float32, device=dev)
    gin[0] = torch.from_numpy(g32[0]).to(dev)
    dr.dyn_radon_adj(plan, gin, uin)
    torch.cuda.synchronize()
    got_g = gout[0].double().cpu().numpy()
    got_u = uin[0].double().cpu().numpy()

    def errs(a, b):
        return {"rel_l2": float(np.linalg.norm(a - b) / np.linalg.norm(b)),
                "max_abs_over_max_ref": float(np.max(np.abs(a - b)) / np.max(np.abs(b)))}

    acc = {"forward": errs(got_g, ref_g[0]), "adjoint": errs(got_u, ref_u[0]),
           "sample": "slice 0: random N(0,1) coefficients (forward), the workload's data (adjoint); the plan's "
                     "autotuned variants", "info": plan.info()}
    del uin, gout, gin
    return cpu, acc


def cpu_baseline_1thread(w, kproj=100):
    """The oracle on one host thread (OMP_NUM_THREADS=1, a separate process):
    one forward and one back-projection of one slice with the first `kproj`
    projections of the workload."""
    code = (
        "import sys, time, numpy as np; sys.path.insert(0, %r); import oracle\n"
        "from paper_1809_09725_gb300 import synth\n"
        "w = synth.WORKLOADS[%r]; theta, t = w.geometry(); kp = %d\n"
        "P = oracle.Problem(w.N, w.N, 1, w.ns, theta[:kp], t[:kp], w.basis, w.m, w.nt)\n"
        "rng = np.random.default_rng(1); u = rng.standard_normal((1, w.N, w.N, w.m))\n"
        "g = rng.standard_normal((1, kp, w.ns))\n"
        "t0 = time.perf_counter(); P.fwd(u); P.adj(g); print(time.perf_counter() - t0)\n"
    ) % (os.path.dirname(os.path.abspath(__file__)), w.name, kproj)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        el = float(out.stdout.strip().splitlines()[-1])
    except Exception as exc:  # noqa: BLE001 -- reported in the JSON line
        return {"error": repr(exc)[:200]}
    units = 2 * kproj * w.N * w.N
    return {"value": units / el, "unit": "voxel*projection/s", "cores": 1, "kind": "oracle",
            "sample": "one forward + one back-projection, FP64 oracle, 1 slice, first %d projections, one "
                      "thread (%.1f s)" % (kproj, el)}


def run_precision_variants(w, theta, t, g32, u_ref, iters, dev, stream, a):
    """The workload on reduced-precision storage (FP32 arithmetic and
    accumulation throughout): FP32 data and coefficients with the solver's
    dual fields in bf16 (DR_FIELDS_BF16), and BF16 data and coefficients with
    bf16 fields.  Per variant: the projector pair on its storage type, the
    ADMM-CG iteration time, the solver's device bytes, and u after `iters`
    iterations from zero against the FP32 plan's (u_ref)."""
    import torch

    from paper_1809_09725_gb300 import dynrecon as dr
    out = {}
    for label, prec in (("fp32_bf16fields", dr.F32 | dr.FIELDS_BF16), ("bf16_bf16fields", dr.BF16 | dr.FIELDS_BF16)):
        pb = dr.Plan(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt, prec)
        t0 = time.perf_counter()
        pb.autotune()
        t_tune = time.perf_counter() - t0
        sd = getattr(torch, pb.storage_dtype)
        fwd_ms, adj_ms = time_projectors(pb, dev, stream, reps=a.op_reps)
        gb = torch.from_numpy(g32).to(dev).to(sd)
        ub = torch.zeros(pb.u_shape(), dtype=sd, device=dev)
        prm = dr.solve_params(dr.ADMM_CG, iters=iters, n_cg=w.n_cg, lambda1=w.lambda1, lambda2=w.lambda2, rho=w.rho)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        dr.admm_solve(pb, gb, ub, prm, want_objective=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / iters  # the first iteration runs eagerly, the rest from a graph
        diff = float(torch.linalg.vector_norm(ub.float() - u_ref) / torch.linalg.vector_norm(u_ref))
        out[label] = {"fwd_ms": fwd_ms, "adj_ms": adj_ms, "admm_ms_per_iter": ms, "autotune_s": t_tune,
                      "voxel_projection_per_s": 2 * (w.n_cg + 1) * w.K * w.voxels() / (ms * 1e-3),
                      "solver_device_gb": (pb.device_bytes()) / 1e9,
                      "rel_l2_u_vs_fp32_after_%d_iters" % iters: diff, "info": pb.info()}
        del gb, ub
        pb.close()
        torch.cuda.empty_cache()
    out["note"] = ("dual fields in bf16: one rounding per store, FP32 arithmetic; BF16 storage also rounds g and u; "
                   "u compared with the FP32 plan's after the same iterations from zero")
    return out


def run_workload_line(name, dev, stream, local, a, steps=20, warmup=3):
    """Another workload's headline numbers (FP32, autotuned, ADMM-CG)."""
    import torch

    from paper_1809_09725_gb300 import dynrecon as dr
    from paper_1809_09725_gb300 import synth
    w = synth.WORKLOADS[name]
    theta, t, g_np = synth.make_data(w)
    plan = dr.Plan(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt, dr.F32)
    g = torch.from_numpy(g_np.astype(np.float32)).to(dev)
    u = torch.zeros(plan.u_shape(), dtype=torch.float32, device=dev)
    tune = plan.autotune()
    ms, res, clocks = solve_timed(plan, g, u, w, steps, warmup, None, dev, local, want_obj=False)
    fwd_ms, adj_ms = time_projectors(plan, dev, stream, reps=10)
    roof = roofline_of(w, theta, plan.info(), fwd_ms, adj_ms, tune)
    units = 2 * (w.n_cg + 1) * w.K * w.voxels() * steps
    out = {"workload": bench_config(w, 1)["workload"], "value": units / (ms * 1e-3), "unit": "voxel*projection/s",
           "steps": steps, "ms_per_step": ms / steps, "clocks": clocks,
           "roofline_alu_frac": roof["frac"], "roofline": roof}
    del g, u
    plan.close()
    return out


def run_disks_fp64(dev):
    """The plain method in FP64 on the single-slice disks problem, timed
    whole (20 ADMM-CG iterations x 4 CG steps): the GPU FP64 plan against the
    FP64 oracle on the host cores, with the relative difference of u."""
    import torch

    import oracle
    from paper_1809_09725_gb300 import dynrecon as dr
    from paper_1809_09725_gb300 import synth
    w = synth.WORKLOADS["disks64"]
    theta, t, g_np = synth.make_data(w)
    plan = dr.Plan(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt, dr.F64)
    g = torch.from_numpy(g_np).to(dev)
    u = torch.zeros(plan.u_shape(), dtype=torch.float64, device=dev)
    prm = lambda: dr.solve_params(dr.ADMM_CG, iters=w.iters, n_cg=w.n_cg, lambda1=w.lambda1, lambda2=w.lambda2,
                                  rho=w.rho)
    dr.admm_solve(plan, g, u, prm(), want_objective=False)
    u.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dr.admm_solve(plan, g, u, prm(), want_objective=False)
    torch.cuda.synchronize()
    t_gpu = time.perf_counter() - t0
    P = oracle.Problem(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt)
    t0 = time.perf_counter()
    uo, _, _ = P.admm_cg(g_np, np.zeros(plan.u_shape()), w.iters, w.n_cg, w.lambda1, w.lambda2, w.rho)
    t_or = time.perf_counter() - t0
    uu = u.cpu().numpy()
    units = 2 * (w.n_cg + 1) * w.K * w.voxels() * w.iters
    plan.close()
    return {"workload": "disks64: 64^2, 1 slice, 64 bins, K=256 over 4 half-turns (mod pi), m=4 Fourier, "
                        "20 ADMM x 4 CG, FP64",
            "gpu_s": t_gpu, "oracle_s": t_or, "oracle_cores": os.cpu_count(),
            "gpu_voxel_projection_per_s": units / t_gpu, "oracle_voxel_projection_per_s": units / t_or,
            "rel_l2_u_gpu_vs_oracle": float(np.linalg.norm(uu - uo) / np.linalg.norm(uo))}


def run_slabs_workload(name, dev):
    from paper_1809_09725_gb300 import synth
    w = synth.WORKLOADS[name]
    theta, t, g_np = synth.make_data(w)
    out = run_slabs(w, theta, t, g_np, dev)
    out["workload"] = name
    return out


def bench_config(w, world: int) -> dict:
    """The workload both arms are quoted on."""
    basis = {0: "Fourier", 1: "Legendre"}[w.basis]
    ws = {"ellipsoids1024": "per-iteration working set ~65 GB > 129 MB L2",
          "ellipsoids256": "per-iteration working set 0.54 GB > 129 MB L2 (duals stream through every iteration)"}
    return {"workload": "%s: nz=%d x %d^2 voxels, %d bins, K=%d over %g half-turns, m=%d %s, nt=%d, "
                        "ADMM-CG n_cg=%d, FP32" % (w.name, w.nz, w.N, w.ns, w.K, w.n_halfturns, w.m, basis, w.nt,
                                                   w.n_cg),
            "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": ws.get(w.name, "inputs larger than L2")}


def reference_sample(w, steps, warmup):
    """Projections per reference step: one slice with the first kp
    projections, so that warm-up + timed steps stay within a few minutes."""
    n = steps + warmup
    kp = 600 if n <= 40 else (300 if n <= 100 else 150)
    return min(kp, w.K)


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_1809_09725_gb300 import synth
    w = synth.WORKLOADS[a.workload]
    theta, t = w.geometry()
    kp = reference_sample(w, a.steps, a.warmup)
    P = oracle.Problem(w.N, w.N, 1, w.ns, theta[:kp], t[:kp], w.basis, w.m, w.nt)
    rng = np.random.default_rng(1)
    u = rng.standard_normal((1, w.N, w.N, w.m))
    g = rng.standard_normal((1, kp, w.ns))
    for _ in range(a.warmup):
        P.fwd(u)
        P.adj(g)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        P.fwd(u)
        P.adj(g)
    el = time.perf_counter() - t0
    units = 2 * kp * w.N * w.N * a.steps
    value = units / el
    sample = ("per step: one forward + one back-projection of 1 of the %d slices with the first %d of the %d "
              "projections, FP64 oracle on the host cores (no GPU used)" % (w.nz, kp, w.K))
    line = {"impl": "reference", "metric": "voxel*projection updates/s (dynamic projector + back-projector "
                                           "applications inside ADMM-CG iterations)",
            "value": value, "unit": "voxel*projection/s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": el * 1e3 / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded random coefficients and data of the "
                                                         "workload's shape)",
            "config": bench_config(w, 1),
            "cpu_baseline": {"value": value, "unit": "voxel*projection/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
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
