"""Seeded synthetic inputs shaped like the paper's continuous-rotation workloads.

This module holds none of the reconstruction method's arithmetic: it makes
acquisition geometries, moving phantoms (disks and z-rotated ellipsoids with
closed-form line integrals), measurement noise and random test vectors.  Both
the CUDA path's tests/benchmark and the CPU oracle's tests take their inputs
from here, so neither side ever produces the other's inputs.

Coordinates are in pixel units about the grid centre (pixel i sits at
``i - (n-1)/2``), the same convention as the projectors.  Continuous
rotation (Sec. 2): projection k is taken at angle ``theta_k`` and time
``t_k = k/K`` in [0, 1).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

FOURIER = 0
LEGENDRE = 1


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


# --------------------------------------------------------------------------- #
# Acquisition
# --------------------------------------------------------------------------- #
def scan(K: int, n_halfturns: float, mod_pi: bool = False):
    """Continuous rotation over ``n_halfturns`` half-turns: theta_k = pi*n*k/K."""
    k = np.arange(K, dtype=np.float64)
    theta = math.pi * n_halfturns * k / K
    if mod_pi:
        theta = np.mod(theta, math.pi)
    t = k / K
    return theta, t


# --------------------------------------------------------------------------- #
# Phantoms with closed-form line integrals
# --------------------------------------------------------------------------- #
@dataclasses.dataclass
class Blob:
    """Ellipsoid (or disk when A == B and nz == 1) moving linearly in t.

    Semi-axes A, B in the xy-plane (A along angle ``psi``), C along z.
    Intensity a + b*sin(2*pi*t + c).
    """
    x0: float
    y0: float
    z0: float
    vx: float
    vy: float
    vz: float
    A: float
    B: float
    C: float
    psi: float
    a: float
    b: float
    c: float

    def intensity(self, t):
        return self.a + self.b * np.sin(2.0 * math.pi * t + self.c)


def disks(rng: np.random.Generator, N: int, count: int = 5, rmin=3.0, rmax=12.0):
    """Static-position disks (radius rmin..rmax px) inside the inscribed circle,
    intensity a + b sin(2 pi t + c) with a in [0.2,1], b in [0,0.3], c in [0,2pi)."""
    out = []
    for _ in range(count):
        r = rng.uniform(rmin, rmax)
        rad = N / 2.0 - r
        # uniform position in the disk of radius N/2 - r
        rr = rad * math.sqrt(rng.uniform(0.0, 1.0))
        ph = rng.uniform(0.0, 2.0 * math.pi)
        out.append(Blob(rr * math.cos(ph), rr * math.sin(ph), 0.0, 0.0, 0.0, 0.0, r, r, 1e9, 0.0,
                        rng.uniform(0.2, 1.0), rng.uniform(0.0, 0.3), rng.uniform(0.0, 2 * math.pi)))
    return out


def ellipsoids(rng: np.random.Generator, N: int, nz: int, count: int, amin=4.0, amax=40.0,
               vmax=20.0, sharp: bool = False):
    """Moving ellipsoids rotated about z; centres move linearly at up to ``vmax``
    voxels per unit time and stay inside the field of view."""
    out = []
    amax = min(amax, N / 4.0)
    for _ in range(count):
        A, B = rng.uniform(amin, amax), rng.uniform(amin, amax)
        C = rng.uniform(amin, max(amin, min(amax, nz)))
        lim = N / 2.0 - max(A, B) - vmax
        lim = max(lim, 1.0)
        rr = lim * math.sqrt(rng.uniform(0.0, 1.0))
        ph = rng.uniform(0.0, 2.0 * math.pi)
        sp = rng.uniform(0.0, vmax)
        dirn = rng.uniform(0.0, 2.0 * math.pi)
        z0 = rng.uniform(-nz / 2.0, nz / 2.0)
        a = rng.uniform(0.2, 1.0) * (1.0 if rng.uniform() < 0.7 else -0.5)
        b = 0.0 if sharp else rng.uniform(0.0, 0.3)
        out.append(Blob(rr * math.cos(ph), rr * math.sin(ph), z0, sp * math.cos(dirn),
                        sp * math.sin(dirn), 0.0, A, B, C, rng.uniform(0.0, math.pi), a, b,
                        rng.uniform(0.0, 2 * math.pi)))
    return out


def sinogram(blobs, theta, t, ns: int, nz: int = 1, slices=None) -> np.ndarray:
    """Exact line integrals of the moving phantom: g[z, k, b] for the detector
    bin centres s_b = b - (ns-1)/2 and slice centres z - (nz-1)/2.

    For an ellipse with semi-axes A, B (A at angle psi) centred at c, the line
    x cos(theta) + y sin(theta) = s carries 2 I A B sqrt(a2 - s'^2) / a2 with
    a2 = A^2 cos^2(theta-psi) + B^2 sin^2(theta-psi), s' = s - c.n.

    Each blob is evaluated only on the bins its shadow can reach (|s'| is at
    most the larger semi-axis), slices vectorised; the bins outside add
    exact zeros, so the values equal an evaluation over the whole detector.
    ``slices``: the slice indices to return (default all nz), the phantom
    still being placed in an nz-slice volume."""
    theta = np.asarray(theta, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    K = theta.size
    zsel = np.arange(nz) if slices is None else np.asarray(slices, dtype=np.int64)
    nzo = zsel.size
    cth, sth = np.cos(theta), np.sin(theta)
    half = 0.5 * (ns - 1)
    rmax = max([max(bl.A, bl.B) for bl in blobs] + [1.0])
    pad = int(math.ceil(min(rmax, 4.0 * ns))) + 4
    g = np.zeros((nzo, K, ns + 2 * pad), dtype=np.float64)
    zc = zsel.astype(np.float64) - 0.5 * (nz - 1) if nz > 1 else np.zeros(nzo)
    kk = np.arange(K)
    for bl in blobs:
        if nz > 1:
            zz = zc[:, None] - (bl.z0 + bl.vz * t)[None, :]
        else:
            zz = np.zeros((nzo, K))
        frac = 1.0 - (zz / bl.C) ** 2
        live = frac > 0.0
        zl = np.nonzero(np.any(live, axis=1))[0]
        if zl.size == 0:
            continue
        live = live[zl]
        sc = np.sqrt(np.where(live, frac[zl], 0.0))
        A = bl.A * sc
        B = bl.B * sc
        x0 = bl.x0 + bl.vx * t
        y0 = bl.y0 + bl.vy * t
        cen = x0 * cth + y0 * sth
        a2 = (A * np.cos(theta - bl.psi)) ** 2 + (B * np.sin(theta - bl.psi)) ** 2
        a2 = np.where(live, a2, 1.0)
        R = min(max(bl.A, bl.B), 4.0 * ns)
        wd = int(2 * math.ceil(R)) + 4
        b0 = np.floor(cen + half - R).astype(np.int64) - 1
        b0 = np.clip(b0, -pad, ns + pad - wd)
        bidx = b0[:, None] + np.arange(wd)[None, :]
        sb = bidx.astype(np.float64) - half
        sp = sb - cen[:, None]
        inside = a2[:, :, None] - (sp ** 2)[None, :, :]
        val = 2.0 * (A * B)[:, :, None] * np.sqrt(np.clip(inside, 0.0, None)) / a2[:, :, None]
        val *= (bl.intensity(t)[None, :] * live)[:, :, None]
        g[zl[:, None, None], kk[None, :, None], (bidx + pad)[None, :, :]] += val
    return np.ascontiguousarray(g[:, :, pad:pad + ns])


def rasterize(blobs, N: int, nz: int, t: float, supersample: int = 4) -> np.ndarray:
    """Area-averaged image of the phantom at time t, shape [nz][N][N]."""
    ss = supersample
    off = (np.arange(ss) + 0.5) / ss - 0.5
    c = np.arange(N, dtype=np.float64) - 0.5 * (N - 1)
    X = (c[None, :, None, None] + off[None, None, None, :])
    Y = (c[:, None, None, None] + off[None, None, :, None])
    img = np.zeros((nz, N, N), dtype=np.float64)
    for z in range(nz):
        zc = z - 0.5 * (nz - 1) if nz > 1 else 0.0
        acc = np.zeros((N, N, ss, ss))
        for bl in blobs:
            zz = zc - (bl.z0 + bl.vz * t) if nz > 1 else 0.0
            frac = 1.0 - (zz / bl.C) ** 2
            if frac <= 0.0:
                continue
            A = bl.A * math.sqrt(frac)
            B = bl.B * math.sqrt(frac)
            dx = X - (bl.x0 + bl.vx * t)
            dy = Y - (bl.y0 + bl.vy * t)
            cp, sp = math.cos(bl.psi), math.sin(bl.psi)
            xr = dx * cp + dy * sp
            yr = -dx * sp + dy * cp
            acc += bl.intensity(t) * ((xr / A) ** 2 + (yr / B) ** 2 <= 1.0)
        img[z] = acc.mean(axis=(2, 3))
    return img


# --------------------------------------------------------------------------- #
# Noise
# --------------------------------------------------------------------------- #
def gaussian_noise(rng: np.random.Generator, g: np.ndarray, frac: float) -> np.ndarray:
    """Additive Gaussian noise with sigma = frac * max|g|."""
    return g + rng.standard_normal(g.shape) * (frac * float(np.max(np.abs(g))))


def poisson_noise(rng: np.random.Generator, g: np.ndarray, photons: float) -> np.ndarray:
    """Photon-counting noise: g is scaled so its maximum is 1, counts are drawn
    from Poisson(photons * exp(-g)) and the log is taken back (clamped at one
    count), then scaled back to the original units."""
    gmax = float(np.max(np.abs(g)))
    if gmax == 0.0:
        return g.copy()
    out = np.empty_like(g)
    flat, res = g.reshape(-1), out.reshape(-1)
    step = 1 << 22  # drawn in order in chunks: the same counts as one draw over the array
    for i in range(0, flat.size, step):
        gs = flat[i:i + step] / gmax
        counts = rng.poisson(photons * np.exp(-gs))
        res[i:i + step] = -np.log(np.maximum(counts, 1) / photons) * gmax
    return out


# --------------------------------------------------------------------------- #
# Random test vectors
# --------------------------------------------------------------------------- #
def random_u(rng, nz, ny, nx, m, dtype=np.float64):
    return rng.standard_normal((nz, ny, nx, m)).astype(dtype)


def random_g(rng, nz, K, ns, dtype=np.float64):
    return rng.standard_normal((nz, K, ns)).astype(dtype)


def random_field(rng, nz, ny, nx, nt, dtype=np.float64):
    return rng.standard_normal((nz, ny, nx, nt, 4)).astype(dtype)


# --------------------------------------------------------------------------- #
# Named workloads
# --------------------------------------------------------------------------- #
@dataclasses.dataclass
class Workload:
    name: str
    N: int
    nz: int
    ns: int
    K: int
    n_halfturns: float
    mod_pi: bool
    basis: int
    m: int
    nt: int
    iters: int
    n_cg: int
    lambda1: float
    lambda2: float
    seed: int

    @property
    def rho(self) -> float:
        return 10.0 * self.lambda1

    def geometry(self):
        return scan(self.K, self.n_halfturns, self.mod_pi)

    def voxels(self) -> int:
        return self.N * self.N * self.nz


# lambda_space = lambda1; lambda_time = lambda1 * lambda2 (Eq. TV1 weights
# the time derivative by lambda2 inside the norm scaled by lambda1).
WORKLOADS = {
    # single slice, 4 half-turns, angles taken mod pi, 5 disks, Gaussian 1 %
    "disks64": Workload("disks64", 64, 1, 64, 256, 4, True, FOURIER, 4, 4, 20, 4, 1e-3, 1.0, 180901),
    # 16 slices of 256^2, 10 half-turns, m = 8 Fourier, Poisson 1e4 photons
    "ellipsoids256": Workload("ellipsoids256", 256, 16, 256, 1800, 10, False, FOURIER, 8, 10, 50,
                              4, 1e-3, 1.0, 180902),
    # large volume, 20 half-turns, m = 16 Legendre
    "ellipsoids1024": Workload("ellipsoids1024", 1024, 64, 1024, 6000, 20, False, LEGENDRE, 16, 20,
                               30, 4, 1e-3, 1.0, 180904),
}


def make_data(w: Workload, nz: int | None = None):
    """Phantom data for a named workload: returns (theta, t, g[nz][K][ns])."""
    rng = rng_for(w.seed)
    theta, t = w.geometry()
    nz = w.nz if nz is None else nz
    if w.name == "disks64":
        blobs = disks(rng, w.N, 5)
        g = sinogram(blobs, theta, t, w.ns, 1)
        g = gaussian_noise(rng, g, 0.01)
    else:
        count = int(rng.integers(20, 41))
        blobs = ellipsoids(rng, w.N, w.nz, count, sharp=(w.name == "ellipsoids1024"))
        g = sinogram(blobs, theta, t, w.ns, w.nz, slices=np.arange(nz))
        g = poisson_noise(rng, g, 1e4)
    return theta, t, g
