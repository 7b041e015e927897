"""GPU parity of the dynamic projector pair against the FP64 oracle.

Forward g = R u (Eq. radapr) and adjoint u = R* g (Eq. radadjapr) through
the C ABI, element by element against the oracle on the same seeded inputs:
FP64 plans to 1e-12, FP32 plans to 1e-5 relative L2, BF16 storage against the
oracle fed the same bf16-rounded inputs.  Sizes span several tiles with
ragged tails, odd detector widths (plain-load staging instead of TMA), wide
and narrow detectors, every template size of m, both bases, and the full
16-slice 256^2 x 1800-projection workload the benchmark times.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1809_09725_gb300 import dynrecon as dr
from paper_1809_09725_gb300 import synth

from _common import assert_close, dev_tensor, host_values, rel, to_bf16_f64

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# name: nx, ny, nz, ns, K, half-turns, mod_pi, basis, m, nt
CASES = {
    "disks64": (64, 64, 1, 64, 256, 4, True, dr.FOURIER, 4, 4),
    "ragged": (37, 29, 3, 45, 100, 3.3, False, dr.LEGENDRE, 5, 3),
    "wide_det": (40, 40, 2, 70, 33, 2.0, False, dr.FOURIER, 3, 2),
    "narrow_det": (48, 52, 2, 24, 65, 5.0, False, dr.FOURIER, 8, 5),
    "single_proj": (20, 20, 1, 20, 1, 1.0, False, dr.FOURIER, 2, 1),
    "m1_static": (33, 33, 2, 33, 47, 2.0, False, dr.FOURIER, 1, 2),
    "m12": (24, 24, 2, 28, 40, 3.0, False, dr.LEGENDRE, 12, 4),
    "m16": (24, 32, 1, 32, 70, 4.0, False, dr.FOURIER, 16, 8),
    "m24": (20, 20, 2, 24, 36, 3.0, False, dr.FOURIER, 24, 6),
    "m32": (16, 24, 1, 20, 50, 6.0, False, dr.LEGENDRE, 32, 6),
    "haar": (30, 28, 2, 33, 120, 4.0, False, dr.HAAR, 6, 4),
    "heaviside": (26, 26, 2, 29, 90, 3.0, False, dr.HEAVISIDE, 5, 5),
    "orthonormal": (32, 32, 1, 32, 128, 4.0, True, dr.FOURIER | dr.ORTHONORMAL, 4, 4),
    "complex_m8": (36, 30, 2, 40, 160, 8.0, False, dr.COMPLEX_FOURIER, 16, 8),
    "complex_m4": (28, 28, 1, 28, 96, 4.0, True, dr.COMPLEX_FOURIER, 8, 4),
    "thin": (3, 41, 2, 23, 40, 2.0, False, dr.FOURIER, 3, 2),
    "flat": (57, 5, 1, 31, 44, 3.0, False, dr.LEGENDRE, 4, 3),
    "tiny_det": (9, 8, 1, 3, 30, 2.0, False, dr.FOURIER, 2, 2),
    # lines wider than one 256-pixel TMA box, with a partial last box
    "wide300": (300, 270, 2, 310, 90, 3.0, False, dr.FOURIER, 4, 3),
}


def _setup(case, seed=0):
    nx, ny, nz, ns, K, ht, mp, basis, m, nt = CASES[case]
    theta, t = synth.scan(K, ht, mp)
    rng = synth.rng_for(1000 + seed + sum(map(ord, case)))
    u = rng.standard_normal((nz, ny, nx, m))
    g = rng.standard_normal((nz, K, ns))
    P = oracle.Problem(nx, ny, nz, ns, theta, t, basis, m, nt)
    return (nx, ny, nz, ns, theta, t, basis, m, nt), u, g, P


def _plan(args, prec):
    nx, ny, nz, ns, theta, t, basis, m, nt = args
    return dr.Plan(nx, ny, nz, ns, theta, t, basis, m, nt, prec)


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec,tol", [(dr.F64, 1e-12), (dr.F32, 1e-5)])
def test_forward_matches_oracle(case, prec, tol):
    args, u, _, P = _setup(case)
    if prec == dr.F32:
        u = u.astype(np.float32).astype(np.float64)
    plan = _plan(args, prec)
    plan.set_variant(dr.DIRECT, dr.DIRECT)
    g = torch.zeros(plan.g_shape(), dtype=getattr(torch, plan.storage_dtype), device="cuda")
    dr.dyn_radon_fwd(plan, dev_tensor(u, prec), g)
    plan.sync()
    assert_close(host_values(g), P.fwd(u), tol)


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec,tol", [(dr.F64, 1e-12), (dr.F32, 1e-5)])
def test_adjoint_matches_oracle(case, prec, tol):
    args, _, g, P = _setup(case)
    if prec == dr.F32:
        g = g.astype(np.float32).astype(np.float64)
    plan = _plan(args, prec)
    plan.set_variant(dr.DIRECT, dr.DIRECT)
    u = torch.zeros(plan.u_shape(), dtype=getattr(torch, plan.storage_dtype), device="cuda")
    dr.dyn_radon_adj(plan, dev_tensor(g, prec), u)
    plan.sync()
    assert_close(host_values(u), P.adj(g), tol)


@pytest.mark.parametrize("case", ["disks64", "ragged", "m16"])
def test_adjoint_beta_accumulates(case):
    args, u0, g, P = _setup(case, seed=3)
    plan = _plan(args, dr.F64)
    u = dev_tensor(u0, dr.F64)
    dr.dyn_radon_adj(plan, dev_tensor(g, dr.F64), u, beta=-0.75)
    plan.sync()
    assert_close(host_values(u), -0.75 * u0 + P.adj(g), 1e-12)


@pytest.mark.parametrize("case", ["disks64", "ragged", "m32"])
def test_gpu_pair_is_adjoint(case):
    """<R u, g> = <u, R* g> for the GPU pair itself (FP64 plan)."""
    args, u, g, _ = _setup(case, seed=5)
    plan = _plan(args, dr.F64)
    gu = torch.zeros(plan.g_shape(), dtype=torch.float64, device="cuda")
    ua = torch.zeros(plan.u_shape(), dtype=torch.float64, device="cuda")
    dr.dyn_radon_fwd(plan, dev_tensor(u, dr.F64), gu)
    dr.dyn_radon_adj(plan, dev_tensor(g, dr.F64), ua)
    plan.sync()
    lhs = float(np.vdot(host_values(gu), g))
    rhs = float(np.vdot(u, host_values(ua)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("case", ["disks64", "ragged", "narrow_det", "m16"])
def test_bf16_storage(case):
    """BF16 storage, FP32 accumulation: against the oracle fed the same
    bf16-rounded inputs and rounded to bf16 the same way (1e-3), and the
    end-to-end error including the output rounding (bounded by 2^-8)."""
    args, u, g, P = _setup(case, seed=7)
    ub, gb = to_bf16_f64(u), to_bf16_f64(g)
    plan = _plan(args, dr.BF16)
    plan.set_variant(dr.DIRECT, dr.DIRECT)
    go = torch.zeros(plan.g_shape(), dtype=torch.bfloat16, device="cuda")
    uo = torch.zeros(plan.u_shape(), dtype=torch.bfloat16, device="cuda")
    dr.dyn_radon_fwd(plan, dev_tensor(ub, dr.BF16), go)
    dr.dyn_radon_adj(plan, dev_tensor(gb, dr.BF16), uo)
    plan.sync()
    ref_g, ref_u = P.fwd(ub), P.adj(gb)
    assert_close(host_values(go), to_bf16_f64(ref_g), 1e-3)
    assert_close(host_values(uo), to_bf16_f64(ref_u), 1e-3)
    assert_close(host_values(go), ref_g, 2.0 ** -8)
    assert_close(host_values(uo), ref_u, 2.0 ** -8)


def test_half_turn_symmetry_on_gpu():
    """Sec. 4: R f(theta + pi, s) = R f(theta, -s) for a static object."""
    N, K = 48, 24
    th0 = np.linspace(0.05, math.pi - 0.05, K // 2)
    theta = np.concatenate([th0, th0 + math.pi])
    t = np.zeros(K)
    plan = dr.Plan(N, N, 1, N, theta, t, dr.FOURIER, 1, 1, dr.F64)
    u = synth.rng_for(9).standard_normal((1, N, N, 1))
    g = torch.zeros(plan.g_shape(), dtype=torch.float64, device="cuda")
    dr.dyn_radon_fwd(plan, dev_tensor(u, dr.F64), g)
    plan.sync()
    gh = host_values(g)[0]
    np.testing.assert_allclose(gh[K // 2:], gh[:K // 2, ::-1], atol=1e-11)


def test_full_workload_256x16x1800_fp32():
    """The benchmarked workload (16 slices of 256^2, 1800 projections over 10
    half-turns, m = 8 Fourier) at full size, in the launch configuration the
    benchmark uses, against the oracle on every output element."""
    w = synth.WORKLOADS["ellipsoids256"]
    theta, t = w.geometry()
    rng = synth.rng_for(4242)
    u = rng.standard_normal((w.nz, w.N, w.N, w.m)).astype(np.float32).astype(np.float64)
    g = rng.standard_normal((w.nz, w.K, w.ns)).astype(np.float32).astype(np.float64)
    plan = dr.Plan(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt, dr.F32)
    plan.set_variant(dr.DIRECT, dr.DIRECT)
    P = oracle.Problem(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt)
    go = torch.zeros(plan.g_shape(), dtype=torch.float32, device="cuda")
    uo = torch.zeros(plan.u_shape(), dtype=torch.float32, device="cuda")
    dr.dyn_radon_fwd(plan, dev_tensor(u, dr.F32), go)
    dr.dyn_radon_adj(plan, dev_tensor(g, dr.F32), uo)
    plan.sync()
    assert_close(host_values(go), P.fwd(u), 1e-5)
    assert_close(host_values(uo), P.adj(g), 1e-5)


def test_invalid_arguments_raise():
    theta, t = synth.scan(8, 1.0)
    with pytest.raises(dr.DynreconError):
        dr.Plan(0, 8, 1, 8, theta, t, dr.FOURIER, 2, 2, dr.F32)
    with pytest.raises(dr.DynreconError):
        dr.Plan(8, 8, 1, 8, theta, t, dr.FOURIER, 33, 2, dr.F32)
    with pytest.raises(dr.DynreconError):
        dr.Plan(8, 8, 1, 4096, theta, t, dr.FOURIER, 2, 2, dr.F32)
    bad = theta.copy()
    bad[3] = np.nan
    with pytest.raises(dr.DynreconError):
        dr.Plan(8, 8, 1, 8, bad, t, dr.FOURIER, 2, 2, dr.F32)
    plan = dr.Plan(8, 8, 1, 8, theta, t, dr.FOURIER, 2, 2, dr.F32)
    with pytest.raises(TypeError):
        dr.dyn_radon_fwd(plan, torch.zeros(plan.u_shape(), dtype=torch.float64, device="cuda"),
                         torch.zeros(plan.g_shape(), dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        dr.dyn_radon_fwd(plan, torch.zeros((1, 8, 8, 3), dtype=torch.float32, device="cuda"),
                         torch.zeros(plan.g_shape(), dtype=torch.float32, device="cuda"))


# --------------------------------------------------------------------------- #
# Half-turn fold (Sec. 4): same operator as the direct form, up to rounding
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("case", sorted(CASES))
def test_fold_variant_matches_oracle(case):
    args, u, g, P = _setup(case, seed=11)
    u = u.astype(np.float32).astype(np.float64)
    g = g.astype(np.float32).astype(np.float64)
    plan = _plan(args, dr.F32)
    plan.set_variant(dr.FOLD, dr.FOLD)
    go = torch.zeros(plan.g_shape(), dtype=torch.float32, device="cuda")
    uo = torch.zeros(plan.u_shape(), dtype=torch.float32, device="cuda")
    dr.dyn_radon_fwd(plan, dev_tensor(u, dr.F32), go)
    dr.dyn_radon_adj(plan, dev_tensor(g, dr.F32), uo)
    plan.sync()
    assert_close(host_values(go), P.fwd(u), 1e-5)
    assert_close(host_values(uo), P.adj(g), 1e-5)


# the bf16 strip layouts: M = 4 (8-byte vectors), M = 8 with m = 8 (16-byte
# copies) and m = 5 (element copies), M = 1, 12, 16, 24, 32 (odd slot counts)
@pytest.mark.parametrize("case", ["disks64", "narrow_det", "ragged", "m1_static", "m12", "m16", "m24", "m32",
                                  "thin", "tiny_det"])
def test_fold_variant_bf16(case):
    args, u, g, P = _setup(case, seed=13)
    ub, gb = to_bf16_f64(u), to_bf16_f64(g)
    plan = _plan(args, dr.BF16)
    plan.set_variant(dr.FOLD, dr.FOLD)
    go = torch.zeros(plan.g_shape(), dtype=torch.bfloat16, device="cuda")
    uo = torch.zeros(plan.u_shape(), dtype=torch.bfloat16, device="cuda")
    dr.dyn_radon_fwd(plan, dev_tensor(ub, dr.BF16), go)
    dr.dyn_radon_adj(plan, dev_tensor(gb, dr.BF16), uo, beta=0.0)
    plan.sync()
    assert_close(host_values(go), to_bf16_f64(P.fwd(ub)), 1e-3)
    assert_close(host_values(uo), to_bf16_f64(P.adj(gb)), 1e-3)


def test_fold_groups_angles_across_pi():
    """Angles a hair below pi fold onto 0 with reversed bins; repeated
    half-turns fold onto their base angle."""
    base = np.array([0.0, 0.3, 1.2, 2.5])
    theta = np.concatenate([base, base + np.pi, base + 2 * np.pi, [np.pi - 1e-13, 3 * np.pi - 2e-13]])
    K = theta.size
    t = np.linspace(0.0, 0.99, K)
    args = (30, 26, 2, 33, theta, t, dr.FOURIER, 3, 3)
    plan = _plan(args, dr.F32)
    info = plan.info()
    assert info["unique_angles"] == 4 and info["max_group"] == 5
    rng = synth.rng_for(21)
    u = rng.standard_normal((2, 26, 30, 3)).astype(np.float32).astype(np.float64)
    g = rng.standard_normal((2, K, 33)).astype(np.float32).astype(np.float64)
    P = oracle.Problem(30, 26, 2, 33, theta, t, dr.FOURIER, 3, 3)
    plan.set_variant(dr.FOLD, dr.FOLD)
    go = torch.zeros(plan.g_shape(), dtype=torch.float32, device="cuda")
    uo = torch.zeros(plan.u_shape(), dtype=torch.float32, device="cuda")
    dr.dyn_radon_fwd(plan, dev_tensor(u, dr.F32), go)
    dr.dyn_radon_adj(plan, dev_tensor(g, dr.F32), uo)
    plan.sync()
    assert_close(host_values(go), P.fwd(u), 1e-5)
    assert_close(host_values(uo), P.adj(g), 1e-5)


def test_fold_full_workload_and_autotune():
    w = synth.WORKLOADS["ellipsoids256"]
    theta, t = w.geometry()
    plan = dr.Plan(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt, dr.F32)
    info = plan.info()
    assert info["unique_angles"] == 180 and info["max_group"] == 10
    times = plan.autotune()
    info = plan.info()
    assert info["tuned"] == 1 and all(x > 0 for x in times)
    # the benchmark's path: the variants and launch configurations the
    # autotuner chose (kept, not forced), folded on this geometry
    assert info["fwd_variant"] in (dr.FOLD, dr.FOLD2) and info["adj_variant"] == dr.FOLD
    rng = synth.rng_for(4243)
    u = rng.standard_normal((w.nz, w.N, w.N, w.m)).astype(np.float32).astype(np.float64)
    g = rng.standard_normal((w.nz, w.K, w.ns)).astype(np.float32).astype(np.float64)
    P = oracle.Problem(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt)
    go = torch.zeros(plan.g_shape(), dtype=torch.float32, device="cuda")
    uo = torch.zeros(plan.u_shape(), dtype=torch.float32, device="cuda")
    dr.dyn_radon_fwd(plan, dev_tensor(u, dr.F32), go)
    dr.dyn_radon_adj(plan, dev_tensor(g, dr.F32), uo)
    plan.sync()
    assert_close(host_values(go), P.fwd(u), 1e-5)
    assert_close(host_values(uo), P.adj(g), 1e-5)


def test_fold_is_unavailable_for_f64_plans():
    args, _, _, _ = _setup("disks64")
    plan = _plan(args, dr.F64)
    assert plan.info()["unique_angles"] == 0
    with pytest.raises(dr.DynreconError):
        plan.set_variant(dr.FOLD, dr.FOLD)


def test_dependent_basis_is_rejected():
    """Orthonormalising Heaviside steps sampled only on [0, 1/2): the steps at
    t >= 1/2 vanish on every acquisition, so the basis is dependent there."""
    theta, t = synth.scan(40, 2.0)
    t = t * 0.5
    with pytest.raises(dr.DynreconError):
        dr.Plan(16, 16, 1, 16, theta, t, dr.HEAVISIDE | dr.ORTHONORMAL, 8, 4, dr.F32)


def test_complex_basis_rejects_odd_m_and_orthonormalisation():
    theta, t = synth.scan(40, 2.0)
    with pytest.raises(dr.DynreconError):
        dr.Plan(16, 16, 1, 16, theta, t, dr.COMPLEX_FOURIER, 5, 2, dr.F32)
    with pytest.raises(dr.DynreconError):
        dr.Plan(16, 16, 1, 16, theta, t, dr.COMPLEX_FOURIER | dr.ORTHONORMAL, 8, 2, dr.F32)


@pytest.mark.parametrize("prec", [dr.F32, dr.BF16])
def test_fold_strip_choices_are_bitwise_identical(prec):
    """Every strip height and staging mode of the folded forward marches each
    ray over the same lines in the same order: identical results."""
    N, K = 48, 180
    theta, t = synth.scan(K, 6.0)
    rng = synth.rng_for(91)
    u = rng.standard_normal((2, N, N, 8))
    plan = dr.Plan(N, N, 2, N, theta, t, dr.FOURIER, 8, 6, prec)
    plan.set_variant(dr.FOLD, dr.FOLD)
    ud = dev_tensor(u, prec)
    outs = []
    for lines, asy in ((1, False), (2, False), (5, False), (1, True), (3, True)):
        plan.set_fold_strip(lines, asy)
        g = torch.zeros(plan.g_shape(), dtype=getattr(torch, plan.storage_dtype), device="cuda")
        dr.dyn_radon_fwd(plan, ud, g)
        plan.sync()
        outs.append(host_values(g))
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])
    with pytest.raises(dr.DynreconError):
        plan.set_fold_strip(0, False)


@pytest.mark.parametrize("prec,tol", [(dr.F64, 1e-13), (dr.F32, 1e-6)])
def test_hand_worked_2x2_example_on_gpu(prec, tol):
    """The Joseph sums of the 2 x 2 image worked by hand (tests/golden), computed
    by the GPU forward with a static basis (m = 1)."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "joseph_2x2.json")))
    theta = np.array([math.atan2(gold["sin"], gold["cos"])])
    plan = dr.Plan(2, 2, 1, gold["ns"], theta, np.array([0.0]), dr.FOURIER, 1, 1, prec)
    img = np.array(gold["image_rows_y_then_x"], dtype=np.float64)[None, :, :, None]
    g = torch.zeros(plan.g_shape(), dtype=getattr(torch, plan.storage_dtype), device="cuda")
    dr.dyn_radon_fwd(plan, dev_tensor(img, prec), g)
    plan.sync()
    np.testing.assert_allclose(host_values(g)[0, 0], gold["expected"], rtol=0, atol=tol * 10)


@pytest.mark.parametrize("case", sorted(c for c in CASES if CASES[c][8] >= 4))
def test_fold2_variant_matches_oracle(case):
    """The fold in two kernels (static transforms of coefficient groups, then
    distribution) is the same operator as the direct form."""
    args, u, _, P = _setup(case, seed=17)
    u = u.astype(np.float32).astype(np.float64)
    plan = _plan(args, dr.F32)
    plan.set_variant(dr.FOLD2, dr.FOLD)
    go = torch.zeros(plan.g_shape(), dtype=torch.float32, device="cuda")
    dr.dyn_radon_fwd(plan, dev_tensor(u, dr.F32), go)
    plan.sync()
    assert_close(host_values(go), P.fwd(u), 1e-5)


@pytest.mark.parametrize("case", ["narrow_det", "m12", "m16", "m32", "ragged"])
def test_fold2_variant_bf16(case):
    args, u, _, P = _setup(case, seed=19)
    ub = to_bf16_f64(u)
    plan = _plan(args, dr.BF16)
    plan.set_variant(dr.FOLD2, dr.FOLD)
    go = torch.zeros(plan.g_shape(), dtype=torch.bfloat16, device="cuda")
    dr.dyn_radon_fwd(plan, dev_tensor(ub, dr.BF16), go)
    plan.sync()
    assert_close(host_values(go), to_bf16_f64(P.fwd(ub)), 1e-3)


def test_fold2_modes_match_fold():
    """The residual (R u - g) and Chambolle-Pock dual epilogues of the
    distribution kernel, through a short solve of each algorithm: the two
    fold forms agree to FP32 rounding."""
    args, _, g, P = _setup("narrow_det", seed=23)
    g = g.astype(np.float32)
    out = {}
    for v in (dr.FOLD, dr.FOLD2):
        for algo in (dr.ADMM_CG, dr.CHAMBOLLE_POCK):
            plan = _plan(args, dr.F32)
            plan.set_variant(v, dr.FOLD)
            u = torch.zeros(plan.u_shape(), dtype=torch.float32, device="cuda")
            prm = dr.solve_params(algo, iters=3, n_cg=3, lambda1=0.05, lambda2=1.0, rho=0.5, op_norm=40.0)
            dr.admm_solve(plan, torch.from_numpy(g).cuda(), u, prm)
            out[(v, algo)] = host_values(u)
    for algo in (dr.ADMM_CG, dr.CHAMBOLLE_POCK):
        assert_close(out[(dr.FOLD2, algo)], out[(dr.FOLD, algo)], 1e-4)


@pytest.mark.parametrize("prec", [dr.F32, dr.BF16])
def test_fold2_group_sizes_agree(prec):
    """Every coefficient group size of the two-kernel forward computes the same
    static transforms (each coefficient's ray sums run the same march): the
    projections agree bit for bit."""
    N, K = 40, 120
    theta, t = synth.scan(K, 4.0)
    rng = synth.rng_for(97)
    u = rng.standard_normal((2, N, N, 8))
    plan = dr.Plan(N, N, 2, N, theta, t, dr.LEGENDRE, 8, 4, prec)
    plan.set_variant(dr.FOLD2, dr.FOLD)
    ud = dev_tensor(u, prec)
    outs = []
    for group, threads, rpt in ((4, 256, 0), (8, 256, 0), (4, 512, 0), (8, 512, 0), (4, 1024, 0), (8, 1024, 0),
                                (4, 512, 4), (8, 512, 2)):
        plan.set_fold_groups(group, 2, threads, rpt)
        assert plan.info()["fold2_rays_per_thread"] == (rpt or (32 if threads < 1024 else 16) // group)
        g = torch.zeros(plan.g_shape(), dtype=getattr(torch, plan.storage_dtype), device="cuda")
        dr.dyn_radon_fwd(plan, ud, g)
        plan.sync()
        outs.append(host_values(g))
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])


@pytest.mark.parametrize("case,nsplit", [("narrow_det", 2), ("m16", 3), ("ragged", 4), ("flat", 8),
                                         ("complex_m8", 3)])
def test_fold2_line_split_matches_oracle(case, nsplit):
    """Splitting the two-kernel forward's march into chunks of image lines
    (some chunks empty when the image is thinner than nsplit lines, as in
    'flat') computes the same operator: the distribution adds the chunks'
    partial sums before the basis weights."""
    args, u, _, P = _setup(case, seed=29)
    u = u.astype(np.float32).astype(np.float64)
    plan = _plan(args, dr.F32)
    plan.set_variant(dr.FOLD2, dr.FOLD)
    plan.set_fold_march(nsplit)
    go = torch.zeros(plan.g_shape(), dtype=torch.float32, device="cuda")
    dr.dyn_radon_fwd(plan, dev_tensor(u, dr.F32), go)
    plan.sync()
    assert plan.info()["fold2_split"] == nsplit
    assert_close(host_values(go), P.fwd(u), 1e-5)


def test_fold2_line_split_bf16():
    args, u, _, P = _setup("m16", seed=37)
    ub = to_bf16_f64(u)
    plan = _plan(args, dr.BF16)
    plan.set_variant(dr.FOLD2, dr.FOLD)
    plan.set_fold_march(3)
    go = torch.zeros(plan.g_shape(), dtype=torch.bfloat16, device="cuda")
    dr.dyn_radon_fwd(plan, dev_tensor(ub, dr.BF16), go)
    plan.sync()
    assert_close(host_values(go), to_bf16_f64(P.fwd(ub)), 1e-3)


def test_fold2_line_split_inside_solvers():
    """A split march inside both solvers' captured iterations (residual and
    dual epilogues): repeatable bit for bit, and equal to the unsplit march
    to FP32 rounding."""
    args, _, g, P = _setup("narrow_det", seed=31)
    gd = torch.from_numpy(g.astype(np.float32)).cuda()
    for algo in (dr.ADMM_CG, dr.CHAMBOLLE_POCK):
        outs = []
        for nsplit in (1, 3, 3):
            plan = _plan(args, dr.F32)
            plan.set_variant(dr.FOLD2, dr.FOLD)
            plan.set_fold_march(nsplit)
            u = torch.zeros(plan.u_shape(), dtype=torch.float32, device="cuda")
            prm = dr.solve_params(algo, iters=3, n_cg=3, lambda1=0.05, lambda2=1.0, rho=0.5, op_norm=40.0)
            dr.admm_solve(plan, gd, u, prm)
            outs.append(host_values(u))
        np.testing.assert_array_equal(outs[1], outs[2])
        assert_close(outs[1], outs[0], 1e-4)


@pytest.mark.parametrize("prec", [dr.F32, dr.BF16])
@pytest.mark.parametrize("case", ["m16", "ragged", "narrow_det"])
def test_fold2_async_strips_bitwise(case, prec):
    """Double- and triple-buffered cp.async strips stage the same lines for
    the same march (whole 16-byte groups by cp.async, the rest through
    registers): projections identical bit for bit, with and without line
    chunks, at several strip heights (strips of one line to more lines than
    the image has)."""
    args, u, _, _ = _setup(case, seed=41)
    plan = _plan(args, prec)
    plan.set_variant(dr.FOLD2, dr.FOLD)
    ud = dev_tensor(u, prec)
    for lines in (1, 3, 16):
        for nsplit in (1, 3):
            outs = []
            for async_stage in (0, 1, 2, 3):
                try:
                    plan.set_fold_groups(4, lines, 256, 0)
                except dr.DynreconError:
                    pytest.skip("strip of %d lines exceeds the budget" % lines)
                plan.set_fold_march(nsplit, async_stage)
                g = torch.zeros(plan.g_shape(), dtype=getattr(torch, plan.storage_dtype), device="cuda")
                dr.dyn_radon_fwd(plan, ud, g)
                plan.sync()
                outs.append(host_values(g))
            for o in outs[1:]:
                np.testing.assert_array_equal(o, outs[0])


@pytest.mark.parametrize("case", ["m16", "narrow_det", "m12", "complex_m8", "wide300", "flat", "ragged"])
def test_fold2_tma_strips_match_oracle(case):
    """Static transforms with TMA-staged strips (staging mode 3: even and odd
    pixels of each line copied by tensor maps with element stride 2, two
    buffers on mbarriers; 4- and 8-coefficient groups): the oracle's projections, and the same
    bits as synchronous staging, at strip heights of one line, a few lines
    and the most that fit, with and without line chunks; a plan whose m is
    not a multiple of 4 ('ragged', m = 5) falls back to cp.async buffers."""
    args, u, _, P = _setup(case, seed=53)
    u = u.astype(np.float32).astype(np.float64)
    plan = _plan(args, dr.F32)
    plan.set_variant(dr.FOLD2, dr.FOLD)
    ud = dev_tensor(u, dr.F32)
    ref = P.fwd(u)
    groups = (4, 8) if args[7] > 4 else (4,)  # 8-coefficient groups: two 16-byte planes per pixel
    checked = 0
    for group in groups:
        for lines in (1, 4, 16):
            try:
                plan.set_fold_groups(group, lines, 256, 0)
            except dr.DynreconError:
                continue  # strip taller than the budget allows
            for nsplit in (1, 2):
                outs = []
                for async_stage in (0, 3):
                    plan.set_fold_march(nsplit, async_stage)
                    g = torch.zeros(plan.g_shape(), dtype=torch.float32, device="cuda")
                    dr.dyn_radon_fwd(plan, ud, g)
                    plan.sync()
                    outs.append(host_values(g))
                np.testing.assert_array_equal(outs[1], outs[0])
                assert_close(outs[1], ref, 1e-5)
                checked += 1
    assert checked >= 4


def test_fold2_tma_strips_inside_solver():
    """TMA-staged static transforms inside the captured ADMM-CG iterations
    (the folded normal operator of the CG steps): repeatable bit for bit and
    the same as synchronous staging."""
    args, _, g, P = _setup("narrow_det", seed=59)
    gd = torch.from_numpy(g.astype(np.float32)).cuda()
    outs = []
    for async_stage in (0, 3, 3):
        plan = _plan(args, dr.F32)
        plan.set_variant(dr.FOLD2, dr.FOLD)
        plan.set_fold_march(1, async_stage)
        u = torch.zeros(plan.u_shape(), dtype=torch.float32, device="cuda")
        prm = dr.solve_params(dr.ADMM_CG, iters=4, n_cg=3, lambda1=0.05, lambda2=1.0, rho=0.5)
        dr.admm_solve(plan, gd, u, prm)
        outs.append(host_values(u))
    np.testing.assert_array_equal(outs[1], outs[0])
    np.testing.assert_array_equal(outs[2], outs[0])


@pytest.mark.parametrize("case", ["narrow_det", "m16", "ragged"])
def test_fold_adjoint_stage_sizes_bitwise(case):
    """The folded adjoint sums the distinct angles in the same order whatever
    the angles per pipeline stage (a ragged last stage included): the
    back-projections agree bit for bit, and match the oracle."""
    args, _, g, P = _setup(case, seed=43)
    g = g.astype(np.float32).astype(np.float64)
    plan = _plan(args, dr.F32)
    plan.set_variant(dr.FOLD, dr.FOLD)
    gd = dev_tensor(g, dr.F32)
    outs = []
    for angles in (8, 7, 6, 5, 1, 32):
        plan.set_fold_adj_stage(angles)
        u = torch.zeros(plan.u_shape(), dtype=torch.float32, device="cuda")
        dr.dyn_radon_adj(plan, gd, u)
        plan.sync()
        assert plan.info()["fold_adj_angles"] == angles
        outs.append(host_values(u))
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])
    assert_close(outs[0], P.adj(g), 1e-5)


@pytest.mark.parametrize("case", ["narrow_det", "m16", "ragged", "complex_m8"])
def test_fold2_angle_blocks_bitwise(case):
    """Spreading the distinct angles over more, smaller CTA blocks changes
    which CTA marches a ray, not the march: projections identical bit for
    bit, and equal to the oracle."""
    args, u, _, P = _setup(case, seed=47)
    u = u.astype(np.float32).astype(np.float64)
    plan = _plan(args, dr.F32)
    plan.set_variant(dr.FOLD2, dr.FOLD)
    ud = dev_tensor(u, dr.F32)
    outs, sizes = [], []
    for extra in range(4):
        try:
            plan.set_fold_blocks(extra)
        except dr.DynreconError:
            break  # this plan has no smaller blocks
        g = torch.zeros(plan.g_shape(), dtype=torch.float32, device="cuda")
        dr.dyn_radon_fwd(plan, ud, g)
        plan.sync()
        outs.append(host_values(g))
        sizes.append(plan.info()["fold2_angles"])
    assert sizes == sorted(sizes, reverse=True) and len(set(sizes)) == len(sizes)
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])
    assert_close(outs[0], P.fwd(u), 1e-5)


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """Failure detection without a fault: a kernel waits, with the bounded
    mbarrier wait the TMA pipelines use, on a barrier nothing arrives at.
    The wait gives up after its limit, the status word reports it
    (DR_ETIMEOUT, cleared on read), and the same plan then computes a
    correct forward projection."""
    args, u, _, P = _setup("ragged", seed=77)
    plan = _plan(args, dr.F32)
    assert plan.wait_selftest(0.05) == dr.DR_ETIMEOUT
    plan.sync()  # status word cleared: no error now
    g = torch.zeros(plan.g_shape(), dtype=torch.float32, device="cuda")
    dr.dyn_radon_fwd(plan, dev_tensor(u, dr.F32), g)
    plan.sync()
    assert_close(host_values(g), P.fwd(u.astype(np.float32).astype(np.float64)), 1e-5)
    assert plan.wait_selftest(3.0) == dr.DR_EINVAL
