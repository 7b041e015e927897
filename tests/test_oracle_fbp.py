"""Pins of the oracle's FBP initial guess (Sec. 5: the iterations start from
the filtered back-projection with the Shepp-Logan filter) against facts fixed
outside it: closed-form partial sums and the frequency response of the
discrete Shepp-Logan kernel, the reconstruction of disks from their exact
line integrals, and least-squares fits that the basis reproduces exactly.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1809_09725_gb300 import synth


def test_tap_values():
    # h(n) = -2 / (pi^2 (4 n^2 - 1)): h(0) = 2/pi^2, h(+-1) = -2/(3 pi^2)
    assert oracle.shepp_logan_tap(0) == pytest.approx(2.0 / math.pi ** 2, abs=1e-16)
    assert oracle.shepp_logan_tap(1) == pytest.approx(-2.0 / (3 * math.pi ** 2), abs=1e-16)
    assert oracle.shepp_logan_tap(-1) == oracle.shepp_logan_tap(1)
    assert oracle.shepp_logan_tap(5) == pytest.approx(-2.0 / (99 * math.pi ** 2), abs=1e-16)


@pytest.mark.parametrize("L", [3, 10, 41])
def test_constant_row_closed_forms(L):
    """sum_{n=1}^{N} 1/(4n^2-1) = N/(2N+1) (telescoping), so on a constant row
    of length 2L+1 the centre output is 2/(pi^2 (2L+1)) and the end output is
    (2/pi^2) (2L+1)/(4L+1)."""
    ns = 2 * L + 1
    q = oracle.shepp_logan_filter(np.ones((1, ns)))[0]
    assert q[L] == pytest.approx(2.0 / (math.pi ** 2 * ns), rel=1e-12)
    N = ns - 1
    end = 2.0 / math.pi ** 2 * (N + 1) / (2 * N + 1)
    assert q[0] == pytest.approx(end, rel=1e-12)
    assert q[-1] == pytest.approx(end, rel=1e-12)


def test_impulse_response_and_frequency_response():
    """The filtered unit impulse is the kernel itself, centred on the impulse;
    its DTFT is |sin(w/2)|/pi (Fourier series of |sin x|) up to the tail
    sum_{|n|>L} |h(n)| = 2/(pi^2 (2L+1))."""
    L = 400
    ns = 2 * L + 1
    d = np.zeros((1, ns))
    d[0, L] = 1.0
    q = oracle.shepp_logan_filter(d)[0]
    n = np.arange(ns) - L
    np.testing.assert_allclose(q, -2.0 / (math.pi ** 2 * (4.0 * n * n - 1.0)), rtol=0, atol=1e-15)
    # an off-centre impulse shifts the response (no index offset)
    d2 = np.zeros((1, 9))
    d2[0, 2] = 1.0
    q2 = oracle.shepp_logan_filter(d2)[0]
    np.testing.assert_allclose(q2, [oracle.shepp_logan_tap(b - 2) for b in range(9)], atol=1e-16)
    tail = 2.0 / (math.pi ** 2 * (2 * L + 1))
    for w in (0.0, 0.1, 0.7, 1.5, 2.5, math.pi):
        H = float(np.sum(q * np.cos(n * w)))
        assert abs(H - abs(math.sin(w / 2)) / math.pi) <= tail + 1e-14


def _disk_sino(blobs, N, K, n_halfturns=1.0):
    theta, t = synth.scan(K, n_halfturns)
    return theta, t, synth.sinogram(blobs, theta, np.zeros(K), N, 1)


def _region_means(img, x0, y0, r, N):
    c = np.arange(N) - 0.5 * (N - 1)
    X, Y = np.meshgrid(c, c)
    R = np.hypot(X - x0, Y - y0)
    inner = img[R < 0.7 * r]
    ring = img[(R > r + 4) & (np.hypot(X, Y) < 0.45 * N)]
    return inner.mean(), np.abs(inner - 1.0).max(), ring.mean(), np.abs(ring).max()


def test_fbp_reconstructs_a_disk():
    """Exact line integrals of a unit disk: the FBP image is 1 inside and 0
    outside, up to discretisation (a dropped pi/K, a sign or a wrong filter
    scale fails by far)."""
    N, K = 128, 256
    x0, y0, r = 9.0, -14.0, 23.0
    blob = synth.Blob(x0, y0, 0, 0, 0, 0, r, r, 1e9, 0, 1.0, 0, 0)
    theta, t, g = _disk_sino([blob], N, K)
    f = oracle.fbp_windows(g, theta, t, N, N, 1)[0, 0]
    mean_in, max_in, mean_out, max_out = _region_means(f, x0, y0, r, N)
    assert abs(mean_in - 1.0) < 0.01
    assert max_in < 0.05
    assert abs(mean_out) < 0.005
    assert max_out < 0.1


def test_fbp_over_several_half_turns_equals_one_half_turn():
    """Sec. 4 half-turn symmetry: a static object scanned over 3 half-turns
    (K = 3 x 128) gives the same FBP image as one half-turn of 128 views."""
    N = 64
    blob = synth.Blob(5.0, 3.0, 0, 0, 0, 0, 14.0, 9.0, 1e9, 0.4, 1.0, 0, 0)
    th1, t1, g1 = _disk_sino([blob], N, 128, 1.0)
    th3, t3, g3 = _disk_sino([blob], N, 384, 3.0)
    f1 = oracle.fbp_windows(g1, th1, t1, N, N, 1)
    f3 = oracle.fbp_windows(g3, th3, t3, N, N, 1)
    np.testing.assert_allclose(f3, f1, atol=1e-12)


def test_fbp_windows_separate_half_turns():
    """Two half-turns of two different static disks: window w reconstructs the
    disk seen during half-turn w."""
    N, Kh = 96, 192
    a = synth.Blob(-15.0, 4.0, 0, 0, 0, 0, 16.0, 16.0, 1e9, 0, 1.0, 0, 0)
    b = synth.Blob(18.0, -10.0, 0, 0, 0, 0, 12.0, 12.0, 1e9, 0, 1.0, 0, 0)
    theta, t = synth.scan(2 * Kh, 2.0)
    g = np.concatenate([synth.sinogram([a], theta[:Kh], np.zeros(Kh), N, 1),
                        synth.sinogram([b], theta[Kh:], np.zeros(Kh), N, 1)], axis=1)
    f = oracle.fbp_windows(g, theta, t, N, N, 2)[0]
    for img, bl in ((f[0], a), (f[1], b)):
        mean_in, max_in, mean_out, _ = _region_means(img, bl.x0, bl.y0, bl.A, N)
        assert abs(mean_in - 1.0) < 0.015 and max_in < 0.06
        assert abs(mean_out) < 0.005


def test_fbp_init_static_fourier_is_constant_in_time():
    """One window: the target is the same image at every time; the constant
    function is in the Fourier span, so the fitted curve equals it at every
    acquisition time and every frame time."""
    N, K = 40, 120
    rng = synth.rng_for(31)
    theta, t = synth.scan(K, 2.0)
    g = rng.standard_normal((2, K, N))
    f = oracle.fbp_windows(g, theta, t, N, N, 1)
    P = oracle.Problem(N, N, 2, N, theta, t, oracle.FOURIER, 5, 4)
    u = P.fbp_init(g, 1)
    at_t = np.einsum("kj,zyxj->zkyx", P.Phi, u)
    np.testing.assert_allclose(at_t, np.broadcast_to(f[:, :1], at_t.shape), atol=1e-10)
    np.testing.assert_allclose(u[..., 0], f[:, 0], atol=1e-10)
    assert np.max(np.abs(u[..., 1:])) < 1e-10


def test_fbp_init_heaviside_reproduces_every_window():
    """m = nw Heaviside steps at j/m span exactly the functions constant on the
    windows [w/nw, (w+1)/nw): the fit reproduces f_{w(k)} at every t_k."""
    N, K, nw = 32, 160, 4
    rng = synth.rng_for(32)
    theta, t = synth.scan(K, 4.0)
    g = rng.standard_normal((1, K, N))
    f = oracle.fbp_windows(g, theta, t, N, N, nw)
    P = oracle.Problem(N, N, 1, N, theta, t, oracle.HEAVISIDE, nw, nw)
    u = P.fbp_init(g, nw)
    w = np.floor(t * nw).astype(int)
    at_t = np.einsum("kj,zyxj->zkyx", P.Phi, u)
    np.testing.assert_allclose(at_t, f[:, w], atol=1e-10)


def test_fbp_init_least_squares_normal_equations():
    """The fit residual over the acquisition times is orthogonal to every basis
    function (normal equations), for a basis that cannot fit the windows exactly."""
    N, K, nw = 24, 90, 3
    rng = synth.rng_for(33)
    theta, t = synth.scan(K, 3.0)
    g = rng.standard_normal((1, K, N))
    f = oracle.fbp_windows(g, theta, t, N, N, nw)
    P = oracle.Problem(N, N, 1, N, theta, t, oracle.LEGENDRE, 2, 3)
    u = P.fbp_init(g, nw)
    w = np.floor(t * nw).astype(int)
    resid = np.einsum("kj,zyxj->zkyx", P.Phi, u) - f[:, w]
    proj = np.einsum("kj,zkyx->zyxj", P.Phi, resid)
    assert np.max(np.abs(proj)) < 1e-9 * max(1.0, np.max(np.abs(f)))
    assert np.max(np.abs(resid)) > 1e-3  # the fit is not exact


def test_fbp_init_minimum_norm_for_a_redundant_basis():
    """The complex Fourier basis of Sec. 5 is redundant as a real basis
    (cos(-w t) = cos(w t), and the zero-frequency sine vanishes): the fit is
    the minimum-norm least-squares solution, so for one window the constant
    channel holds the image and every other channel is zero."""
    N, K, M = 24, 96, 4
    rng = synth.rng_for(34)
    theta, t = synth.scan(K, 2.0)
    g = rng.standard_normal((1, K, N))
    f = oracle.fbp_windows(g, theta, t, N, N, 1)
    P = oracle.Problem(N, N, 1, N, theta, t, oracle.COMPLEX_FOURIER, 2 * M, 2)
    u = P.fbp_init(g, 1)
    const = 2 * (M // 2)  # channel of cos(0 t) = 1
    np.testing.assert_allclose(u[..., const], f[:, 0], atol=1e-10)
    others = np.delete(u, const, axis=-1)
    assert np.max(np.abs(others)) < 1e-10
