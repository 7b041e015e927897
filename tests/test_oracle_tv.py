"""Pins of the oracle's 4D gradient/divergence and proximal maps.

Checks against: the adjoint relation div = -nabla^T (Sec. 3, K_2^*), exact
derivatives of constants and ramps along each axis (which also fixes the
component order and where lambda2 enters, Eq. TV1), closed-form and
brute-force minimisers of the proximal problems (Eq. prox), and the Moreau
identity linking the shrink and the projection.
"""
import math

import numpy as np
import pytest
from scipy import optimize

import oracle
from paper_1809_09725_gb300 import synth


def test_div_is_minus_grad_transpose():
    rng = synth.rng_for(10)
    F = rng.standard_normal((3, 5, 6, 4))
    p = rng.standard_normal((3, 5, 6, 4, 4))
    lam2 = 1.7
    lhs = np.vdot(oracle.grad4(F, lam2), p)
    rhs = -np.vdot(F, oracle.div4(p, lam2))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_grad_of_constant_is_zero():
    F = np.full((2, 3, 4, 5), 2.5)
    assert np.all(oracle.grad4(F, 3.0) == 0.0)


def test_grad_of_ramps_fixes_component_order():
    nz, ny, nx, nt = 3, 4, 5, 6
    z, y, x, l = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), np.arange(nt),
                             indexing="ij")
    lam2 = 2.5
    for axis, ramp, n in ((0, x, nx), (1, y, ny), (2, z, nz), (3, l, nt)):
        p = oracle.grad4(ramp.astype(float), lam2)
        scale = lam2 if axis == 3 else 1.0
        idx = [z, y, x, l][[2, 1, 0, 3][axis]]
        expect = np.where(idx < n - 1, scale, 0.0)
        np.testing.assert_array_equal(p[..., axis], expect)
        for other in range(4):
            if other != axis:
                assert np.all(p[..., other] == 0.0)


def test_D_and_DT_are_adjoint_and_synthesise_frames():
    rng = synth.rng_for(11)
    nz, ny, nx, m, nt = 2, 4, 5, 3, 6
    PhiF = oracle.frame_table(oracle.FOURIER, m, nt)
    u = rng.standard_normal((nz, ny, nx, m))
    p = rng.standard_normal((nz, ny, nx, nt, 4))
    lhs = np.vdot(oracle.D(u, PhiF, 0.8), p)
    rhs = np.vdot(u, oracle.DT(p, PhiF, 0.8))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # u_1 = 1 (the cos 2 pi t coefficient): frames are cos(2 pi l / nt) everywhere
    u1 = np.zeros((1, 2, 2, m))
    u1[..., 1] = 1.0
    F = oracle.frames(u1, PhiF)
    np.testing.assert_allclose(F[0, 0, 0], np.cos(2 * np.pi * np.arange(nt) / nt), atol=1e-15)
    p1 = oracle.D(u1, PhiF, 0.8)
    dt = 0.8 * np.diff(np.cos(2 * np.pi * np.arange(nt) / nt))
    np.testing.assert_allclose(p1[0, 1, 1, :-1, 3], dt, atol=1e-15)
    assert p1[0, 1, 1, -1, 3] == 0.0
    assert np.all(p1[..., :3] == 0.0)


@pytest.mark.parametrize("kappa", [0.0, 0.3, 2.0, 10.0])
def test_shrink_minimises_its_objective(kappa):
    rng = synth.rng_for(12)
    for _ in range(5):
        v = rng.standard_normal(4)
        out = oracle.shrink4(v, kappa)
        obj = lambda q: kappa * np.linalg.norm(q) + 0.5 * np.sum((v - q) ** 2)
        best = optimize.minimize(obj, v * 0.5, method="Nelder-Mead",
                                 options={"xatol": 1e-10, "fatol": 1e-14, "maxiter": 20000})
        assert obj(out) <= best.fun + 1e-9
        n = np.linalg.norm(v)
        expect = v * max(0.0, 1.0 - kappa / n)
        np.testing.assert_allclose(out, expect, atol=1e-15)


def test_shrink_zero_vector():
    assert np.all(oracle.shrink4(np.zeros(4), 1.0) == 0.0)


def test_moreau_identity():
    rng = synth.rng_for(13)
    for kappa in (0.1, 1.0, 3.0):
        v = rng.standard_normal(4) * 2
        lhs = oracle.shrink4(v, kappa) + kappa * oracle.project4(v / kappa, 1.0)
        np.testing.assert_allclose(lhs, v, atol=1e-14)


def test_projection_is_nearest_point_of_ball():
    rng = synth.rng_for(14)
    lam = 0.7
    for _ in range(6):
        h = rng.standard_normal(4)
        out = oracle.project4(h, lam)
        assert np.linalg.norm(out) <= lam + 1e-15
        cons = {"type": "ineq", "fun": lambda q: lam ** 2 - np.sum(q ** 2)}
        best = optimize.minimize(lambda q: np.sum((q - h) ** 2), np.zeros(4), constraints=[cons],
                                 method="SLSQP", options={"ftol": 1e-14, "maxiter": 500})
        np.testing.assert_allclose(out, best.x, atol=1e-6)


def test_cp_h1_prox_closed_form():
    """Sec. 3: prox of sigma F_1^* is (h - sigma g)/(1 + sigma); brute force on a scalar."""
    for h, g, sigma in ((0.3, -1.2, 0.5), (2.0, 0.7, 3.0)):
        f = lambda q: q * g + 0.5 * q * q + (h - q) ** 2 / (2 * sigma)
        best = optimize.minimize_scalar(f, bracket=(-10, 10), tol=1e-14)
        assert abs(best.x - (h - sigma * g) / (1 + sigma)) < 1e-7


def _prox_case():
    rng = synth.rng_for(15)
    nz, ny, nx, m, nt = 2, 4, 5, 3, 4
    PhiF = oracle.frame_table(oracle.FOURIER, m, nt)
    u = rng.standard_normal((nz, ny, nx, m))
    mu = rng.standard_normal((nz, ny, nx, nt, 4))
    return u, mu, PhiF


def test_tv4d_prox_limits():
    u, mu0, PhiF = _prox_case()
    lam2, rho = 1.3, 2.0
    Du = oracle.D(u, PhiF, lam2)
    # lambda1 = 0: psi = D u + mu/rho, mu -> 0, w = psi
    mu, w = mu0.copy(), np.zeros_like(mu0)
    tv, pr = oracle.tv4d_prox(u, mu, w, PhiF, rho, 0.0, lam2)
    np.testing.assert_allclose(mu, 0.0, atol=1e-14)
    np.testing.assert_allclose(w, Du + mu0 / rho, atol=1e-14)
    assert abs(tv - np.sum(np.linalg.norm(Du, axis=-1))) < 1e-12 * tv
    assert abs(pr - np.sum((mu0 / rho) ** 2)) < 1e-12 * pr
    # lambda1 huge: psi = 0, mu -> mu + rho D u, w = -mu/rho
    mu, w = mu0.copy(), np.zeros_like(mu0)
    oracle.tv4d_prox(u, mu, w, PhiF, rho, 1e12, lam2)
    np.testing.assert_allclose(mu, mu0 + rho * Du, atol=1e-12)
    np.testing.assert_allclose(w, -(mu0 + rho * Du) / rho, atol=1e-12)


def test_tv4d_prox_matches_pointwise_shrink():
    u, mu0, PhiF = _prox_case()
    lam1, lam2, rho = 0.9, 1.3, 2.0
    Du = oracle.D(u, PhiF, lam2)
    mu, w = mu0.copy(), np.zeros_like(mu0)
    oracle.tv4d_prox(u, mu, w, PhiF, rho, lam1, lam2)
    v = (Du + mu0 / rho).reshape(-1, 4)
    psi = np.stack([oracle.shrink4(q, lam1 / rho) for q in v]).reshape(Du.shape)
    np.testing.assert_allclose(mu, mu0 + rho * (Du - psi), atol=1e-13)
    np.testing.assert_allclose(w, psi - mu / rho, atol=1e-13)
    # psi is the minimiser of lam1 |psi| + rho/2 |v - psi|^2: check one point by brute force
    q = v[7]
    obj = lambda s: lam1 * np.linalg.norm(s) + 0.5 * rho * np.sum((q - s) ** 2)
    best = optimize.minimize(obj, q, method="Nelder-Mead",
                             options={"xatol": 1e-11, "fatol": 1e-15, "maxiter": 40000})
    assert obj(psi.reshape(-1, 4)[7]) <= best.fun + 1e-9
