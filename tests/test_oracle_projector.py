"""Pins of the oracle's projector pair and bases against facts fixed outside it.

Each test checks the FP64 oracle against mathematics the paper fixes: the
adjoint identity of Eq. (radadjapr), the half-turn symmetry of Sec. 4, exact
line sums at special angles, a hand-worked 2x2 example, brute-force matrix
transposes, closed-form line integrals of disks and ellipses, and textbook
basis values.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1809_09725_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _dense_fwd(nx, ny, ns, theta):
    """Matrix of the oracle's single-angle Joseph projector, column by column."""
    A = np.zeros((ns, ny * nx))
    for q in range(ny * nx):
        e = np.zeros(ny * nx)
        e[q] = 1.0
        A[:, q] = oracle.joseph_fwd_slice(e.reshape(ny, nx), theta, ns)
    return A


def _dense_adj(nx, ny, ns, theta):
    B = np.zeros((ny * nx, ns))
    for b in range(ns):
        e = np.zeros(ns)
        e[b] = 1.0
        B[:, b] = oracle.joseph_adj_slice(e, theta, nx, ny).ravel()
    return B


ANGLES = [0.0, math.pi / 2, math.pi / 4, 3 * math.pi / 4, 0.3, 1.1, 2.0, 2.9, 3.5, 5.0, -0.7,
          math.atan2(0.6, 0.8)]


@pytest.mark.parametrize("nx,ny,ns", [(8, 8, 8), (8, 6, 11), (5, 7, 6)])
@pytest.mark.parametrize("theta", ANGLES)
def test_gather_adjoint_is_exact_transpose(nx, ny, ns, theta):
    A = _dense_fwd(nx, ny, ns, theta)
    B = _dense_adj(nx, ny, ns, theta)
    assert np.max(np.abs(A.T - B)) <= 1e-14 * max(1.0, np.max(np.abs(A)))


def test_hand_worked_2x2_example():
    gold = json.load(open(os.path.join(GOLD, "joseph_2x2.json")))
    img = np.array(gold["image_rows_y_then_x"])
    theta = math.atan2(gold["sin"], gold["cos"])
    out = oracle.joseph_fwd_slice(img, theta, gold["ns"])
    np.testing.assert_allclose(out, gold["expected"], rtol=0, atol=1e-13)


def test_special_angles_are_exact_line_sums():
    rng = synth.rng_for(1)
    N = 9
    F = rng.standard_normal((N, N))
    # theta = 0: line x = s -> column sums; theta = pi/2: line y = s -> row sums
    np.testing.assert_allclose(oracle.joseph_fwd_slice(F, 0.0, N), F.sum(axis=0), atol=1e-12)
    np.testing.assert_allclose(oracle.joseph_fwd_slice(F, math.pi / 2, N), F.sum(axis=1), atol=1e-12)
    # theta = pi: x = -s -> reversed column sums
    np.testing.assert_allclose(oracle.joseph_fwd_slice(F, math.pi, N), F.sum(axis=0)[::-1],
                               atol=1e-12)
    # theta = pi/4, centre bin: samples on the anti-diagonal, weight sqrt(2)
    g = oracle.joseph_fwd_slice(F, math.pi / 4, N)
    anti = sum(F[j, N - 1 - j] for j in range(N))
    assert abs(g[N // 2] - math.sqrt(2.0) * anti) < 1e-12
    # theta = 3pi/4 (cos < 0), centre bin: main diagonal
    g = oracle.joseph_fwd_slice(F, 3 * math.pi / 4, N)
    assert abs(g[N // 2] - math.sqrt(2.0) * np.trace(F)) < 1e-12


@pytest.mark.parametrize("theta", [0.2, 0.9, 1.7, 2.6, math.pi / 4])
def test_half_turn_symmetry(theta):
    """Sec. 4: R f(theta + pi, s) = R f(theta, -s), exact on the symmetric bin grid."""
    rng = synth.rng_for(2)
    F = rng.standard_normal((10, 12))
    a = oracle.joseph_fwd_slice(F, theta, 15)
    b = oracle.joseph_fwd_slice(F, theta + math.pi, 15)
    np.testing.assert_allclose(b, a[::-1], atol=1e-12)


@pytest.mark.parametrize("basis", [oracle.FOURIER, oracle.LEGENDRE])
def test_dynamic_adjoint_dot_product(basis):
    """<R u, g> = <u, R* g> (Sec. 4, the adjoint equality behind Eq. radadjapr)."""
    rng = synth.rng_for(3)
    nz, ny, nx, m, K, ns = 2, 12, 10, 5, 37, 15
    theta, t = synth.scan(K, 3.3)
    Phi = oracle.basis_table(basis, m, t)
    u = rng.standard_normal((nz, ny, nx, m))
    g = rng.standard_normal((nz, K, ns))
    lhs = np.vdot(oracle.dyn_fwd(u, theta, Phi, ns), g)
    rhs = np.vdot(u, oracle.dyn_adj(g, theta, Phi, nx, ny))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_static_reduction_m1():
    """m = 1 with phi_0 = 1: the dynamic operator is the static Radon transform."""
    rng = synth.rng_for(4)
    nz, ny, nx, K, ns = 2, 9, 9, 11, 9
    theta, t = synth.scan(K, 2.0)
    Phi = oracle.basis_table(oracle.FOURIER, 1, t)
    assert np.all(Phi == 1.0)
    u = rng.standard_normal((nz, ny, nx, 1))
    g = oracle.dyn_fwd(u, theta, Phi, ns)
    for z in range(nz):
        for k in range(K):
            np.testing.assert_allclose(g[z, k], oracle.joseph_fwd_slice(u[z, :, :, 0], theta[k], ns),
                                       atol=1e-12)


def test_time_dependence_special_times():
    """f(t) = U + cos(2 pi t) V: at t = 0, 1/2, 1/4 the projection is of U+V, U-V, U."""
    rng = synth.rng_for(5)
    n, ns = 8, 8
    U, V = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    u = np.stack([U, V], axis=-1)[None]
    t = np.array([0.0, 0.5, 0.25])
    theta = np.array([0.4, 1.3, 2.2])
    Phi = oracle.basis_table(oracle.FOURIER, 2, t)
    g = oracle.dyn_fwd(u, theta, Phi, ns)[0]
    np.testing.assert_allclose(g[0], oracle.joseph_fwd_slice(U + V, theta[0], ns), atol=1e-12)
    np.testing.assert_allclose(g[1], oracle.joseph_fwd_slice(U - V, theta[1], ns), atol=1e-12)
    np.testing.assert_allclose(g[2], oracle.joseph_fwd_slice(U, theta[2], ns), atol=1e-12)


def test_fourier_basis_values_and_orthogonality():
    P = oracle.basis_table(oracle.FOURIER, 5, [0.25, 0.125])
    # phi = {1, cos 2pi t, sin 2pi t, cos 4pi t, sin 4pi t}
    np.testing.assert_allclose(P[0], [1, 0, 1, -1, 0], atol=1e-15)
    np.testing.assert_allclose(P[1], [1, math.sqrt(0.5), math.sqrt(0.5), 0, 1], atol=1e-15)
    K = 64
    Pk = oracle.basis_table(oracle.FOURIER, 7, np.arange(K) / K)
    G = Pk.T @ Pk
    np.testing.assert_allclose(G, np.diag([K] + [K / 2] * 6), atol=1e-11)


def test_legendre_textbook_values():
    # shifted Legendre phi_j(t) = P_j(2t - 1)
    P = oracle.basis_table(oracle.LEGENDRE, 5, [1.0, 0.0, 0.5, 0.75])
    np.testing.assert_allclose(P[0], [1, 1, 1, 1, 1], atol=1e-15)
    np.testing.assert_allclose(P[1], [1, -1, 1, -1, 1], atol=1e-15)
    np.testing.assert_allclose(P[2], [1, 0, -0.5, 0, 0.375], atol=1e-15)
    np.testing.assert_allclose(P[3][:4], [1, 0.5, -0.125, -0.4375], atol=1e-15)
    # orthogonality on [0,1]: int phi_i phi_j dt = delta_ij / (2j+1), Gauss-Legendre quadrature
    x, wq = np.polynomial.legendre.leggauss(20)
    Pq = oracle.basis_table(oracle.LEGENDRE, 6, (x + 1) / 2)
    G = (Pq * (wq / 2)[:, None]).T @ Pq
    np.testing.assert_allclose(G, np.diag(1.0 / (2 * np.arange(6) + 1)), atol=1e-13)


def test_disk_line_integrals_converge():
    """Joseph sums of an area-sampled disk approach the closed-form line integral
    2 sqrt(r^2 - s^2) as the grid is refined (error falls roughly like 1/N)."""
    errs = []
    for N in (32, 64, 128):
        h = 2.0 / N  # field of view [-1, 1]
        blob = synth.Blob(0.21 / h, -0.13 / h, 0, 0, 0, 0, 0.37 / h, 0.37 / h, 1e9, 0, 1.0, 0, 0)
        img = synth.rasterize([blob], N, 1, 0.0, supersample=8)[0]
        thetas = np.array([0.1, 0.7, 1.3, 2.2])
        exact = synth.sinogram([blob], thetas, np.zeros(4), N, 1)[0]
        approx = np.stack([oracle.joseph_fwd_slice(img, th, N) for th in thetas])
        errs.append(np.linalg.norm(approx - exact) / np.linalg.norm(exact))
    assert errs[0] < 0.05
    assert errs[1] < 0.75 * errs[0]
    assert errs[2] < 0.75 * errs[1]


def _ellipse_chord(A, B, psi, cx, cy, theta, s):
    """Length of the chord that the line x cos(theta) + y sin(theta) = s cuts
    from the ellipse with semi-axes A (along angle psi) and B centred at
    (cx, cy): the line p(tau) = s n + tau n_perp put into the ellipse's frame,
    the two roots of the quadratic (u + tau v)^T diag(1/A^2, 1/B^2) (u + tau v) = 1."""
    n = np.array([math.cos(theta), math.sin(theta)])
    d = np.array([-math.sin(theta), math.cos(theta)])
    rot = np.array([[math.cos(psi), math.sin(psi)], [-math.sin(psi), math.cos(psi)]])
    out = np.zeros(len(s))
    for i, si in enumerate(s):
        u = rot @ (si * n - np.array([cx, cy]))
        v = rot @ d
        qa = v[0] ** 2 / A ** 2 + v[1] ** 2 / B ** 2
        qb = 2.0 * (u[0] * v[0] / A ** 2 + u[1] * v[1] / B ** 2)
        qc = u[0] ** 2 / A ** 2 + u[1] ** 2 / B ** 2 - 1.0
        disc = qb * qb - 4.0 * qa * qc
        out[i] = math.sqrt(disc) / qa if disc > 0.0 else 0.0
    return out


def test_ellipse_line_integrals_converge():
    """Closed-form line integrals of an ellipse (chord lengths from the roots of
    a quadratic) equal the phantom generator's exact sinogram, and Joseph sums
    of the area-sampled rotated ellipse approach them as the grid is refined
    (error falls roughly like 1/N)."""
    errs = []
    thetas = np.array([0.1, 0.7, 1.3, 2.2, 2.9])
    for N in (32, 64, 128):
        h = 2.0 / N  # field of view [-1, 1]
        A, B, psi, cx, cy = 0.55 / h, 0.23 / h, 0.6, 0.12 / h, -0.2 / h
        blob = synth.Blob(cx, cy, 0, 0, 0, 0, A, B, 1e9, psi, 1.0, 0, 0)
        sb = np.arange(N) - 0.5 * (N - 1)
        exact = np.stack([_ellipse_chord(A, B, psi, cx, cy, th, sb) for th in thetas])
        gen = synth.sinogram([blob], thetas, np.zeros(len(thetas)), N, 1)[0]
        np.testing.assert_allclose(gen, exact, rtol=1e-9, atol=1e-9 * exact.max())
        img = synth.rasterize([blob], N, 1, 0.0, supersample=8)[0]
        approx = np.stack([oracle.joseph_fwd_slice(img, th, N) for th in thetas])
        errs.append(np.linalg.norm(approx - exact) / np.linalg.norm(exact))
    assert errs[0] < 0.08  # the minor axis is under 4 pixels at N = 32
    assert errs[1] < 0.75 * errs[0]
    assert errs[2] < 0.75 * errs[1]


def test_haar_values_and_orthogonality():
    # phi_0 = 1; phi_1 = psi(t); phi_2 = psi(2t); phi_3 = psi(2t - 1); psi = +1 on [0,1/2), -1 on [1/2,1)
    P = oracle.basis_table(oracle.HAAR, 4, [0.1, 0.3, 0.6, 0.9])
    np.testing.assert_array_equal(P, [[1, 1, 1, 0], [1, 1, -1, 0], [1, -1, 0, 1], [1, -1, 0, -1]])
    K = 64
    Pk = oracle.basis_table(oracle.HAAR, 8, (np.arange(K) + 0.5) / K)
    G = Pk.T @ Pk
    # levels 0 (j=1), 1 (j=2,3), 2 (j=4..7): supports of length 1, 1/2, 1/4
    np.testing.assert_allclose(G, np.diag([64, 64, 32, 32, 16, 16, 16, 16]), atol=0)


def test_heaviside_values():
    P = oracle.basis_table(oracle.HEAVISIDE, 4, [0.0, 0.249, 0.25, 0.6, 0.99])
    np.testing.assert_array_equal(P, [[1, 0, 0, 0], [1, 0, 0, 0], [1, 1, 0, 0], [1, 1, 1, 0], [1, 1, 1, 1]])


@pytest.mark.parametrize("kind", [oracle.FOURIER, oracle.LEGENDRE, oracle.HEAVISIDE])
def test_orthonormalised_basis(kind):
    """Gram-Schmidt over the acquisition times: Phi^T Phi = I, and the new
    functions span the same space (same frames up to the triangular change)."""
    theta, t = synth.scan(40, 3.0)
    P = oracle.Problem(6, 6, 1, 7, theta, t, kind | oracle.ORTHONORMAL, 4, 5)
    np.testing.assert_allclose(P.Phi.T @ P.Phi, np.eye(4), atol=1e-13)
    raw = oracle.basis_table(kind, 4, t)
    # raw = Phi Rm with Rm upper triangular: Phi^T raw = Rm
    M = P.Phi.T @ raw
    assert np.max(np.abs(np.tril(M, -1))) < 1e-12
    # the frame table transforms with the same matrix
    rawF = oracle.frame_table(kind, 4, 5)
    Rm = np.linalg.lstsq(P.Phi, raw, rcond=None)[0]
    np.testing.assert_allclose(P.PhiF @ Rm, rawF, atol=1e-11)


def _complex_coeffs(u_real):
    """u[..., 2j] + i u[..., 2j+1]: the complex coefficients of the channels."""
    return u_real[..., 0::2] + 1j * u_real[..., 1::2]


def test_complex_fourier_channels_against_complex_arithmetic():
    """Sec. 5 basis phi_j(t) = exp(2 pi i t (j - M/2)): the real channel table
    reproduces Re sum_j u_j phi_j(t) computed with complex numbers, and its
    transpose is the paper's adjoint weight conj(phi_j) (Eq. radadjapr)."""
    M = 6
    rng = synth.rng_for(40)
    t = rng.uniform(0.0, 1.0, 50)
    Phi = oracle.basis_table(oracle.COMPLEX_FOURIER, 2 * M, t)
    a = rng.standard_normal(2 * M)
    uc = _complex_coeffs(a)
    freqs = np.arange(M) - M // 2
    E = np.exp(2j * np.pi * np.outer(t, freqs))  # [K][M]
    np.testing.assert_allclose(Phi @ a, (E @ uc).real, atol=1e-13)
    x = rng.standard_normal(t.size)
    adj = E.conj().T @ x  # sum_k conj(phi_j(t_k)) x_k
    back = Phi.T @ x
    np.testing.assert_allclose(back[0::2], adj.real, atol=1e-12)
    np.testing.assert_allclose(back[1::2], adj.imag, atol=1e-12)
    with pytest.raises(ValueError):
        oracle.basis_table(oracle.COMPLEX_FOURIER, 5, t)


def test_complex_fourier_dynamic_projection():
    """R applied to the complex-basis object equals Re of the complex sum of
    the Radon transforms of the coefficient images (linearity, Eq. radapr)."""
    M, n, ns = 4, 9, 11
    rng = synth.rng_for(41)
    theta, t = synth.scan(12, 2.0)
    u = rng.standard_normal((1, n, n, 2 * M))
    Phi = oracle.basis_table(oracle.COMPLEX_FOURIER, 2 * M, t)
    g = oracle.dyn_fwd(u, theta, Phi, ns)[0]
    uc = _complex_coeffs(u[0])
    freqs = np.arange(M) - M // 2
    for k in range(theta.size):
        Rre = np.stack([oracle.joseph_fwd_slice(uc[..., j].real, theta[k], ns) for j in range(M)], axis=-1)
        Rim = np.stack([oracle.joseph_fwd_slice(uc[..., j].imag, theta[k], ns) for j in range(M)], axis=-1)
        ph = np.exp(2j * np.pi * t[k] * freqs)
        np.testing.assert_allclose(g[k], ((Rre + 1j * Rim) @ ph).real, atol=1e-12)
