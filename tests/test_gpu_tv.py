"""GPU parity of the 4D TV stencils and the ADMM prox against the oracle.

D = nabla_{lambda2} o PhiF (Eq. TV1 on the synthesised frames), its adjoint
(Sec. 3, K_2^* = -div), and the shrink/dual step of the ADMM split, through
the C ABI on seeded inputs with ragged sizes, every TV template size of m,
and nz = 1 (no z neighbours).
"""
import numpy as np
import pytest

import oracle
from paper_1809_09725_gb300 import dynrecon as dr
from paper_1809_09725_gb300 import synth

from _common import assert_close, dev_tensor, host_values, rel, to_bf16_f64

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# nx, ny, nz, basis, m, nt
CASES = {
    "c1like": (64, 64, 1, dr.FOURIER, 4, 4),
    "ragged": (37, 29, 5, dr.LEGENDRE, 5, 3),
    "m8": (33, 40, 4, dr.FOURIER, 8, 10),
    "m1": (20, 17, 3, dr.FOURIER, 1, 2),
    "m13": (16, 18, 3, dr.LEGENDRE, 13, 7),
    "m32": (12, 10, 3, dr.FOURIER, 32, 5),
    "nt1": (21, 22, 2, dr.FOURIER, 3, 1),
    "haar": (20, 18, 3, dr.HAAR, 4, 8),
    "orthonormal": (18, 20, 2, dr.LEGENDRE | dr.ORTHONORMAL, 5, 6),
    "complex": (19, 17, 3, dr.COMPLEX_FOURIER, 8, 6),
    # a row of u plus the dual fields takes so many bytes that the stencils
    # walk the volume in bands of rows (21 rows in FP32 with a partial last
    # band / 10 in FP64 here, 27 / 13 in banded_m8, both with a partial band)
    "banded": (512, 100, 3, dr.LEGENDRE, 16, 20),
    "banded_m8": (300, 60, 4, dr.FOURIER, 8, 30),
}


def _to_field(a):
    """Oracle layout [nz][ny][nx][nt][4] -> the library's [nz][nt][ny][nx][4]."""
    return np.ascontiguousarray(np.asarray(a).transpose(0, 3, 1, 2, 4))


def _from_field(a):
    """The library's [nz][nt][ny][nx][4] -> oracle layout [nz][ny][nx][nt][4]."""
    return np.asarray(a).transpose(0, 2, 3, 1, 4)


def _setup(case, seed=0):
    nx, ny, nz, basis, m, nt = CASES[case]
    K = 8
    theta, t = synth.scan(K, 2.0)
    plan_args = (nx, ny, nz, 9, theta, t, basis, m, nt)
    P = oracle.Problem(nx, ny, nz, 9, theta, t, basis, m, nt)
    rng = synth.rng_for(500 + seed + sum(map(ord, case)))
    u = rng.standard_normal((nz, ny, nx, m))
    p = rng.standard_normal((nz, ny, nx, nt, 4))
    mu = rng.standard_normal((nz, ny, nx, nt, 4))
    return plan_args, P, u, p, mu


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec,tol", [(dr.F64, 1e-12), (dr.F32, 1e-5)])
def test_grad_and_adjoint(case, prec, tol):
    args, P, u, p, _ = _setup(case)
    lam2 = 1.7
    if prec == dr.F32:
        u = u.astype(np.float32).astype(np.float64)
        p = p.astype(np.float32).astype(np.float64)
    plan = dr.Plan(*args, prec=prec)
    fdt = getattr(torch, plan.field_dtype)
    pg = torch.zeros(plan.field_shape(), dtype=fdt, device="cuda")
    dr.tv4d_grad(plan, dev_tensor(u, prec), pg, lam2)
    ua = torch.zeros(plan.u_shape(), dtype=getattr(torch, plan.storage_dtype), device="cuda")
    dr.tv4d_grad_adj(plan, dev_tensor(_to_field(p), prec), ua, lam2)
    plan.sync()
    assert_close(_from_field(host_values(pg)), P.D(u, lam2), tol)
    assert_close(host_values(ua), P.DT(p, lam2), tol)


@pytest.mark.parametrize("case", ["ragged", "m8", "banded", "banded_m8"])
@pytest.mark.parametrize("prec,tol", [(dr.F64, 1e-12), (dr.F32, 1e-5)])
def test_grad_adj_beta(case, prec, tol):
    """u = beta u + D^T p (in FP32 with nt m <= 448 the frame tables come from
    the constant bank; the banded cases walk in several bands)."""
    args, P, u, p, _ = _setup(case, seed=1)
    if prec == dr.F32:
        u = u.astype(np.float32).astype(np.float64)
        p = p.astype(np.float32).astype(np.float64)
    plan = dr.Plan(*args, prec=prec)
    ut = dev_tensor(u, prec)
    dr.tv4d_grad_adj(plan, dev_tensor(_to_field(p), prec), ut, 0.6, beta=2.5)
    plan.sync()
    assert_close(host_values(ut), 2.5 * u + P.DT(p, 0.6), tol)


@pytest.mark.parametrize("case", ["m8", "banded_m8"])
def test_grad_adj_bf16_storage(case):
    """D^T p into bf16 coefficients (BF16 plan: float fields, FP32 sums, one
    rounding to bf16 per stored coefficient)."""
    args, P, _, p, _ = _setup(case, seed=5)
    p = p.astype(np.float32).astype(np.float64)
    plan = dr.Plan(*args, prec=dr.BF16)
    ua = torch.zeros(plan.u_shape(), dtype=torch.bfloat16, device="cuda")
    dr.tv4d_grad_adj(plan, dev_tensor(_to_field(p), dr.F32), ua, 0.6)
    plan.sync()
    ref = P.DT(p, 0.6)
    # bf16 keeps 8 significant bits: each stored value within 2^-8 of itself
    got = host_values(ua)
    assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-6 * np.max(np.abs(ref)))


# Tall volumes: many slices per row of the walk, ragged nx and ny, and m
# below the template size.
TALL = {"tall_m8": (40, 20, 400, dr.FOURIER, 8, 3), "tall_m5": (33, 9, 700, dr.LEGENDRE, 5, 4),
        "tall_m16": (70, 17, 150, dr.FOURIER, 16, 2)}


@pytest.mark.parametrize("case", sorted(CASES) + sorted(TALL))
@pytest.mark.parametrize("prec,tol", [(dr.F64, 1e-12), (dr.F32, 1e-5)])
def test_normal_matches_oracle(case, prec, tol):
    """out = beta out + D^T D x against the oracle's D^T (D x)."""
    if case in TALL:
        nx, ny, nz, basis, m, nt = TALL[case]
        theta, t = synth.scan(8, 2.0)
        args = (nx, ny, nz, 9, theta, t, basis, m, nt)
        P = oracle.Problem(*args)
        rng = synth.rng_for(900 + sum(map(ord, case)))
        x = rng.standard_normal((nz, ny, nx, m))
    else:
        args, P, x, _, _ = _setup(case, seed=3)
    o0 = synth.rng_for(17).standard_normal(x.shape)
    lam2, beta = 1.9, -0.75
    if prec == dr.F32:
        x = x.astype(np.float32).astype(np.float64)
        o0 = o0.astype(np.float32).astype(np.float64)
    plan = dr.Plan(*args, prec=prec)
    cdt = np.float64 if prec == dr.F64 else np.float32
    xd = torch.from_numpy(x.astype(cdt)).cuda()
    od = torch.from_numpy(o0.astype(cdt)).cuda()
    dr.tv4d_normal(plan, xd, od, lam2, beta)
    plan.sync()
    ref = beta * o0 + P.DT(P.D(x, lam2), lam2)
    assert_close(host_values(od), ref, tol)


def test_normal_rejects_aliasing():
    args, _, x, _, _ = _setup("m1")
    plan = dr.Plan(*args, prec=dr.F32)
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    with pytest.raises(dr.DynreconError):
        dr.tv4d_normal(plan, xd, xd, 1.0)


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec,tol", [(dr.F64, 1e-12), (dr.F32, 1e-5)])
def test_prox_matches_oracle(case, prec, tol):
    args, P, u, _, mu0 = _setup(case, seed=2)
    rho, lam1, lam2 = 0.7, 0.4, 1.3
    if prec == dr.F32:
        u = u.astype(np.float32).astype(np.float64)
        mu0 = mu0.astype(np.float32).astype(np.float64)
    plan = dr.Plan(*args, prec=prec)
    mu = dev_tensor(_to_field(mu0), prec if prec != dr.BF16 else dr.F32)
    w = torch.zeros_like(mu)
    res = dr.tv4d_prox(plan, dev_tensor(u, prec), mu, w, rho, lam1, lam2, want_residual=True)
    mu_o, w_o = mu0.copy(), np.zeros_like(mu0)
    tv_o, pr_o = oracle.tv4d_prox(u, mu_o, w_o, P.PhiF, rho, lam1, lam2)
    assert_close(_from_field(host_values(mu)), mu_o, tol)
    assert_close(_from_field(host_values(w)), w_o, tol)
    assert abs(res - np.sqrt(pr_o)) <= 10 * tol * np.sqrt(pr_o)


def test_prox_bf16_coefficients():
    args, P, u, _, mu0 = _setup("m8", seed=4)
    ub = to_bf16_f64(u)
    mu0 = mu0.astype(np.float32).astype(np.float64)
    plan = dr.Plan(*args, prec=dr.BF16)
    mu = dev_tensor(_to_field(mu0), dr.F32)
    w = torch.zeros_like(mu)
    dr.tv4d_prox(plan, dev_tensor(ub, dr.BF16), mu, w, 0.7, 0.4, 1.3)
    plan.sync()
    mu_o, w_o = mu0.copy(), np.zeros_like(mu0)
    oracle.tv4d_prox(ub, mu_o, w_o, P.PhiF, 0.7, 0.4, 1.3)
    assert_close(_from_field(host_values(mu)), mu_o, 1e-5)
    assert_close(_from_field(host_values(w)), w_o, 1e-5)


def test_prox_rejects_bad_parameters():
    args, _, u, _, mu0 = _setup("m1")
    plan = dr.Plan(*args, prec=dr.F32)
    mu = dev_tensor(_to_field(mu0), dr.F32)
    w = torch.zeros_like(mu)
    with pytest.raises(dr.DynreconError):
        dr.tv4d_prox(plan, dev_tensor(u, dr.F32), mu, w, 0.0, 0.4, 1.3)
    with pytest.raises(dr.DynreconError):
        dr.tv4d_prox(plan, dev_tensor(u, dr.F32), mu, w, 1.0, -0.4, 1.3)
