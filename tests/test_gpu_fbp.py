"""GPU parity of the FBP initial guess (Sec. 5: Shepp-Logan FBP as the
starting point of the iterations) against the oracle.

dr_fbp_init filters every projection row with the discrete Shepp-Logan
kernel and back-projects once with the windowed least-squares table in place
of the basis table; the oracle filters, back-projects window by window and
fits the coefficients by a dense minimum-norm least-squares solve.  Cases:
several bases and window counts (one of them redundant), ragged sizes, both
projector variants, FP64 / FP32 / BF16 plans, a two-slice cut of the 256^2 x
1800 workload, and bad arguments.
"""
import numpy as np
import pytest

import oracle
from paper_1809_09725_gb300 import dynrecon as dr
from paper_1809_09725_gb300 import synth

from _common import assert_close, dev_tensor, host_values, rel, to_bf16_f64

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# nx, ny, nz, ns, K, half-turns, basis, m, nt, windows
CASES = {
    "disks64_static": (64, 64, 1, 64, 256, 4.0, dr.FOURIER, 4, 4, 1),
    "disks64_halfturns": (64, 64, 1, 64, 256, 4.0, dr.FOURIER, 4, 4, 4),
    "ragged": (37, 29, 3, 45, 150, 3.0, dr.LEGENDRE, 5, 3, 3),
    "heaviside": (40, 40, 2, 40, 160, 4.0, dr.HEAVISIDE, 4, 4, 4),
    "m16_orthonormal": (24, 26, 2, 31, 200, 5.0, dr.LEGENDRE | dr.ORTHONORMAL, 16, 5, 5),
    "wide_det": (20, 20, 1, 300, 64, 2.0, dr.FOURIER, 3, 2, 2),
    "complex_redundant": (30, 30, 2, 32, 128, 4.0, dr.COMPLEX_FOURIER, 8, 4, 4),
}


def _setup(case, seed=0):
    nx, ny, nz, ns, K, ht, basis, m, nt, nw = CASES[case]
    theta, t = synth.scan(K, ht)
    rng = synth.rng_for(700 + seed + sum(map(ord, case)))
    g = rng.standard_normal((nz, K, ns)) * 4.0
    P = oracle.Problem(nx, ny, nz, ns, theta, t, basis, m, nt)
    return (nx, ny, nz, ns, theta, t, basis, m, nt), g, P, nw


def _run(args, g, prec, nw, variant=None):
    plan = dr.Plan(*args, prec=prec)
    if variant is not None:
        plan.set_variant(dr.DIRECT, variant)
    u = torch.full(plan.u_shape(), 7.0, dtype=getattr(torch, plan.storage_dtype), device="cuda")
    dr.fbp_init(plan, dev_tensor(g, prec), u, nw)
    plan.sync()
    return host_values(u)


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec,tol", [(dr.F64, 1e-11), (dr.F32, 1e-5)])
def test_fbp_init_matches_oracle(case, prec, tol):
    args, g, P, nw = _setup(case)
    if prec == dr.F32:
        g = g.astype(np.float32).astype(np.float64)
    u = _run(args, g, prec, nw)
    assert_close(u, P.fbp_init(g, nw), tol)


@pytest.mark.parametrize("case", ["disks64_halfturns", "ragged", "heaviside"])
def test_fbp_init_both_variants(case):
    args, g, P, nw = _setup(case, seed=1)
    g = g.astype(np.float32).astype(np.float64)
    ref = P.fbp_init(g, nw)
    for v in (dr.DIRECT, dr.FOLD):
        assert_close(_run(args, g, dr.F32, nw, variant=v), ref, 1e-5)


@pytest.mark.parametrize("case", ["disks64_static", "ragged"])
def test_fbp_init_bf16(case):
    """BF16 data and coefficients, FP32 arithmetic: against the oracle fed the
    same bf16 data and rounded the same way, and end to end (2^-8)."""
    args, g, P, nw = _setup(case, seed=2)
    gb = to_bf16_f64(g)
    u = _run(args, gb, dr.BF16, nw)
    ref = P.fbp_init(gb, nw)
    assert_close(u, to_bf16_f64(ref), 1e-3)
    assert_close(u, ref, 2.0 ** -8)


def test_fbp_init_reconstructs_disks():
    """Exact line integrals of static disks: the constant coefficient of the
    one-window FBP is the disk image (density 1 inside)."""
    N, K = 96, 384
    theta, t = synth.scan(K, 3.0)
    blobs = [synth.Blob(-12.0, 6.0, 0, 0, 0, 0, 15.0, 15.0, 1e9, 0, 1.0, 0, 0),
             synth.Blob(20.0, -14.0, 0, 0, 0, 0, 9.0, 9.0, 1e9, 0, 1.0, 0, 0)]
    g = synth.sinogram(blobs, theta, np.zeros(K), N, 1)
    plan = dr.Plan(N, N, 1, N, theta, t, dr.FOURIER, 5, 3, dr.F32)
    u = torch.zeros(plan.u_shape(), dtype=torch.float32, device="cuda")
    dr.fbp_init(plan, dev_tensor(g, dr.F32), u, 1)
    u = host_values(u)
    c = np.arange(N) - 0.5 * (N - 1)
    X, Y = np.meshgrid(c, c)
    for bl in blobs:
        inside = np.hypot(X - bl.x0, Y - bl.y0) < 0.7 * bl.A
        assert abs(u[0, :, :, 0][inside].mean() - 1.0) < 0.01
    assert np.max(np.abs(u[..., 1:])) < 1e-4


def test_fbp_init_ellipsoids256_cut():
    """Two slices of the 256^2, K = 1800 (10 half-turns), m = 8 workload, one
    window per half-turn, at the launch configuration the solver uses."""
    w = synth.WORKLOADS["ellipsoids256"]
    theta, t, g = synth.make_data(w)
    g = g[:2].astype(np.float32).astype(np.float64)
    P = oracle.Problem(w.N, w.N, 2, w.ns, theta, t, w.basis, w.m, w.nt)
    ref = P.fbp_init(g, 10)
    plan = dr.Plan(w.N, w.N, 2, w.ns, theta, t, w.basis, w.m, w.nt, dr.F32)
    u = torch.zeros(plan.u_shape(), dtype=torch.float32, device="cuda")
    dr.fbp_init(plan, dev_tensor(g, dr.F32), u, 10)
    assert_close(host_values(u), ref, 1e-5)


def test_fbp_init_then_solve_lowers_objective():
    """The FBP start is closer to the data than zero, and ADMM-CG from it
    keeps a lower objective after the same iterations."""
    w = synth.WORKLOADS["disks64"]
    theta, t, g = synth.make_data(w)
    plan = dr.Plan(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt, dr.F32)
    gd = dev_tensor(g, dr.F32)
    u_fbp = torch.zeros(plan.u_shape(), dtype=torch.float32, device="cuda")
    dr.fbp_init(plan, gd, u_fbp, 1)
    P = oracle.Problem(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt)
    zero = np.zeros(plan.u_shape())
    assert P.objective(g, host_values(u_fbp), w.lambda1, w.lambda2) < 0.2 * P.objective(g, zero, w.lambda1, w.lambda2)
    prm = dr.solve_params(dr.ADMM_CG, iters=3, n_cg=w.n_cg, lambda1=w.lambda1, lambda2=w.lambda2, rho=w.rho)
    u0 = torch.zeros_like(u_fbp)
    r0 = dr.admm_solve(plan, gd, u0, prm)
    r1 = dr.admm_solve(plan, gd, u_fbp, prm)
    assert r1["objective"][-1] < r0["objective"][-1]


def test_fbp_init_rejects_bad_arguments():
    args, g, P, nw = _setup("ragged")
    plan = dr.Plan(*args, prec=dr.F32)
    gd = dev_tensor(g, dr.F32)
    u = torch.zeros(plan.u_shape(), dtype=torch.float32, device="cuda")
    for bad in (0, -1, plan.K + 1):
        with pytest.raises(dr.DynreconError) as err:
            dr.fbp_init(plan, gd, u, bad)
        assert err.value.status == dr.DR_EINVAL


def test_fbp_init_dependent_basis_takes_minimum_norm_fit():
    """m = 4 Legendre functions sampled at only 3 distinct times are dependent:
    the fit is the minimum-norm least-squares one, as in the oracle."""
    theta = np.linspace(0.0, np.pi, 12, endpoint=False)
    t = np.repeat([0.1, 0.5, 0.9], 4)
    rng = synth.rng_for(777)
    g = rng.standard_normal((1, 12, 16))
    P = oracle.Problem(16, 16, 1, 16, theta, t, oracle.LEGENDRE, 4, 2)
    u = _run((16, 16, 1, 16, theta, t, dr.LEGENDRE, 4, 2), g, dr.F64, 3)
    assert_close(u, P.fbp_init(g, 3), 1e-9)
