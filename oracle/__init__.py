"""Plain FP64 CPU oracle for the dynamic-tomography hot path (arXiv 1809.09725).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library: the arithmetic lives in ``dynrecon_oracle.c`` (plain C,
double precision, compiled with ``-ffp-contract=off``); this module only builds
it with gcc and marshals numpy arrays through ctypes.

Every function follows a passage of the paper:
  * ``basis_table``            Sec. 4, Eq. (repr): real Fourier, shifted Legendre,
                               Haar, Heaviside; Sec. 5 complex Fourier (real channels)
  * ``ORTHONORMAL`` flag        Gram-Schmidt over the acquisition times (Sec. 4)
  * ``joseph_fwd_slice``       static Radon transform R of Eq. (radapr), Joseph rule
  * ``joseph_adj_slice``       its exact transpose (pixel-driven gather)
  * ``dyn_fwd`` / ``dyn_adj``  Eqs. (Rfwd)/(radapr) and (radadjapr)
  * ``grad4`` / ``div4``       nabla_{lambda2} of Eq. (TV1), div = -nabla^T (Sec. 3)
  * ``D`` / ``DT``             nabla_{lambda2} composed with the frame synthesis
  * ``shrink4`` / ``project4`` pointwise proximal maps (Sec. 3, prox of sigma F_2^*)
  * ``tv4d_prox``              ADMM shrink and dual update on psi = D u
  * ``admm_cg``                ADMM with a CG u-step for Eq. (lr12)
  * ``chambolle_pock``         Sec. 3, Fig. 2
  * ``power_norm``             operator norm for tau, sigma (Fig. 2 footnote)
  * ``objective``              Eq. (lr12)
  * ``shepp_logan_filter``     the Shepp-Logan filter of the FBP start (Sec. 5)
  * ``fbp_windows`` / ``fbp_init``  windowed FBP images and their least-squares
                               fit to the basis (the initial guess of Sec. 5)

Parity unpinned: none of the functions above; each has a pin in
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dynrecon_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

FOURIER = 0
LEGENDRE = 1
HAAR = 2
HEAVISIDE = 3
COMPLEX_FOURIER = 4  # exp(2 pi i t (j - M/2)) as 2M real channels (Re, Im of each u_j)
ORTHONORMAL = 0x100  # flag: Gram-Schmidt orthonormalise over the acquisition times

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i = ctypes.c_int
_i64 = ctypes.c_int64
_d = ctypes.c_double
_pd = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile ``dynrecon_oracle.c`` into ``liboracle.so`` next to it (gcc, OpenMP)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fPIC", "-shared",
            _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        sig = {
            "or_basis_table": (_i, [_i, _i, _dp, _i64, _dp]),
            "or_orthonormalise": (_i, [_dp, _i64, _i, _dp, _i64]),
            "or_joseph_fwd_slice": (None, [_dp, _i, _i, _d, _i, _dp]),
            "or_joseph_adj_slice": (None, [_dp, _i, _d, _i, _i, _dp]),
            "or_dyn_fwd": (None, [_dp, _i, _i, _i, _i, _i, _dp, _dp, _i, _dp]),
            "or_dyn_adj": (None, [_dp, _i, _i, _i, _i, _i, _dp, _dp, _i, _dp]),
            "or_frames": (None, [_dp, _i64, _i, _dp, _i, _dp]),
            "or_frames_T": (None, [_dp, _i64, _i, _dp, _i, _dp]),
            "or_grad4": (None, [_dp, _i, _i, _i, _i, _d, _dp]),
            "or_div4": (None, [_dp, _i, _i, _i, _i, _d, _dp]),
            "or_D": (None, [_dp, _i, _i, _i, _i, _dp, _i, _d, _dp]),
            "or_DT": (None, [_dp, _i, _i, _i, _i, _dp, _i, _d, _dp]),
            "or_shrink4": (None, [_dp, _d, _dp]),
            "or_project4": (None, [_dp, _d, _dp]),
            "or_tv4d_prox": (None, [_dp, _dp, _dp, _i, _i, _i, _i, _dp, _i, _d, _d, _d, _pd, _pd]),
            "or_admm_cg_flat": (_i, [_i, _i, _i, _i, _i, _i, _i, _dp, _dp, _dp, _dp, _dp, _i, _i,
                                     _d, _d, _d, _pd, _pd]),
            "or_chambolle_pock_flat": (_i, [_i, _i, _i, _i, _i, _i, _i, _dp, _dp, _dp, _dp, _dp, _i,
                                            _d, _d, _d, _d, _pd]),
            "or_power_norm_flat": (_d, [_i, _i, _i, _i, _i, _i, _i, _dp, _dp, _dp, _d, _i]),
            "or_splitmix_uniform": (_d, [ctypes.c_uint64, ctypes.c_uint64]),
            "or_objective_flat": (_d, [_i, _i, _i, _i, _i, _i, _i, _dp, _dp, _dp, _dp, _dp, _d, _d]),
            "or_shepp_logan_tap": (_d, [_i64]),
            "or_shepp_logan_filter": (None, [_dp, _i64, _i, _dp]),
            "or_fbp_windows": (_i, [_dp, _i, _i, _i, _i, _dp, _dp, _i, _i, _dp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _optbuf(n: int, want: bool):
    if not want:
        return None, None
    arr = np.zeros(n, dtype=np.float64)
    return arr, arr.ctypes.data_as(_pd)


# --------------------------------------------------------------------------- #
# Bases and single-slice Joseph pair
# --------------------------------------------------------------------------- #
def basis_table(kind: int, m: int, t) -> np.ndarray:
    """``out[i, j] = phi_j(t[i])``; kind FOURIER (real), LEGENDRE (shifted), HAAR,
    HEAVISIDE or COMPLEX_FOURIER (m = 2M real channels)."""
    t = _c(np.atleast_1d(t))
    out = np.zeros((t.size, m), dtype=np.float64)
    if _load().or_basis_table(int(kind), int(m), t, t.size, out) != 0:
        raise ValueError("bad basis kind or m")
    return out


def frame_table(kind: int, m: int, nt: int) -> np.ndarray:
    """Basis on the frame grid t_l = l / nt (Sec. 4, Eq. discrt)."""
    return basis_table(kind, m, np.arange(nt, dtype=np.float64) / nt)


def joseph_fwd_slice(F, theta: float, ns: int) -> np.ndarray:
    F = _c(F)
    ny, nx = F.shape
    out = np.zeros(ns, dtype=np.float64)
    _load().or_joseph_fwd_slice(F, nx, ny, float(theta), ns, out)
    return out


def joseph_adj_slice(g, theta: float, nx: int, ny: int) -> np.ndarray:
    g = _c(g)
    out = np.zeros((ny, nx), dtype=np.float64)
    _load().or_joseph_adj_slice(g, g.size, float(theta), nx, ny, out)
    return out


# --------------------------------------------------------------------------- #
# Dynamic operators: u [nz][ny][nx][m] <-> g [nz][K][ns]
# --------------------------------------------------------------------------- #
def dyn_fwd(u, theta, Phi, ns: int) -> np.ndarray:
    u = _c(u)
    theta = _c(theta)
    Phi = _c(Phi)
    nz, ny, nx, m = u.shape
    K = theta.size
    assert Phi.shape == (K, m)
    g = np.zeros((nz, K, ns), dtype=np.float64)
    _load().or_dyn_fwd(u, nx, ny, nz, m, K, theta, Phi, ns, g)
    return g


def dyn_adj(g, theta, Phi, nx: int, ny: int) -> np.ndarray:
    g = _c(g)
    theta = _c(theta)
    Phi = _c(Phi)
    nz, K, ns = g.shape
    m = Phi.shape[1]
    u = np.zeros((nz, ny, nx, m), dtype=np.float64)
    _load().or_dyn_adj(g, nx, ny, nz, m, K, theta, Phi, ns, u)
    return u


# --------------------------------------------------------------------------- #
# 4D gradient / divergence and the composed D, D^T
# --------------------------------------------------------------------------- #
def grad4(F, lambda2: float) -> np.ndarray:
    F = _c(F)
    nz, ny, nx, nt = F.shape
    p = np.zeros((nz, ny, nx, nt, 4), dtype=np.float64)
    _load().or_grad4(F, nx, ny, nz, nt, float(lambda2), p)
    return p


def div4(p, lambda2: float) -> np.ndarray:
    p = _c(p)
    nz, ny, nx, nt, _ = p.shape
    F = np.zeros((nz, ny, nx, nt), dtype=np.float64)
    _load().or_div4(p, nx, ny, nz, nt, float(lambda2), F)
    return F


def frames(u, PhiF) -> np.ndarray:
    u = _c(u)
    PhiF = _c(PhiF)
    nz, ny, nx, m = u.shape
    nt = PhiF.shape[0]
    F = np.zeros((nz, ny, nx, nt), dtype=np.float64)
    _load().or_frames(u, nz * ny * nx, m, PhiF, nt, F)
    return F


def D(u, PhiF, lambda2: float) -> np.ndarray:
    u = _c(u)
    PhiF = _c(PhiF)
    nz, ny, nx, m = u.shape
    nt = PhiF.shape[0]
    p = np.zeros((nz, ny, nx, nt, 4), dtype=np.float64)
    _load().or_D(u, nx, ny, nz, m, PhiF, nt, float(lambda2), p)
    return p


def DT(p, PhiF, lambda2: float) -> np.ndarray:
    p = _c(p)
    PhiF = _c(PhiF)
    nz, ny, nx, nt, _ = p.shape
    m = PhiF.shape[1]
    u = np.zeros((nz, ny, nx, m), dtype=np.float64)
    _load().or_DT(p, nx, ny, nz, m, PhiF, nt, float(lambda2), u)
    return u


def splitmix_uniform(seed: int, i: int) -> float:
    """i-th output of the counter-based SplitMix64 stream, as a double in [0, 1)."""
    return _load().or_splitmix_uniform(int(seed), int(i))


def shrink4(v, kappa: float) -> np.ndarray:
    out = np.zeros(4, dtype=np.float64)
    _load().or_shrink4(_c(v), float(kappa), out)
    return out


def project4(h, lam: float) -> np.ndarray:
    out = np.zeros(4, dtype=np.float64)
    _load().or_project4(_c(h), float(lam), out)
    return out


def tv4d_prox(u, mu, w, PhiF, rho: float, lambda1: float, lambda2: float):
    """In place on ``mu`` and ``w`` (float64, C-contiguous); returns (sum |Du|, ||Du - psi||^2)."""
    u = _c(u)
    PhiF = _c(PhiF)
    assert mu.dtype == np.float64 and mu.flags.c_contiguous
    assert w.dtype == np.float64 and w.flags.c_contiguous
    nz, ny, nx, m = u.shape
    nt = PhiF.shape[0]
    tv = ctypes.c_double()
    pr = ctypes.c_double()
    _load().or_tv4d_prox(u, mu, w, nx, ny, nz, m, PhiF, nt, float(rho), float(lambda1),
                         float(lambda2), ctypes.byref(tv), ctypes.byref(pr))
    return tv.value, pr.value


# --------------------------------------------------------------------------- #
# FBP initial guess (Sec. 5)
# --------------------------------------------------------------------------- #
def shepp_logan_tap(n: int) -> float:
    """Discrete Shepp-Logan kernel h(n) = -2 / (pi^2 (4 n^2 - 1)), unit spacing."""
    return _load().or_shepp_logan_tap(int(n))


def shepp_logan_filter(g) -> np.ndarray:
    """Linear convolution of every row of g[..., ns] with h along the last axis."""
    g = _c(g)
    ns = g.shape[-1]
    q = np.zeros_like(g)
    _load().or_shepp_logan_filter(g, g.size // ns, ns, q)
    return q


def fbp_windows(g, theta, t, nx: int, ny: int, n_windows: int) -> np.ndarray:
    """FBP image of every time window: f[nz][nw][ny][nx] (see or_fbp_windows)."""
    g = _c(g)
    nz, K, ns = g.shape
    f = np.zeros((nz, n_windows, ny, nx))
    rc = _load().or_fbp_windows(g, nx, ny, nz, K, _c(theta), _c(t), ns, int(n_windows), f)
    if rc != 0:
        raise MemoryError("oracle fbp_windows failed (%d)" % rc)
    return f


def fbp_init(g, theta, t, Phi, nx: int, ny: int, n_windows: int) -> np.ndarray:
    """Initial coefficients from windowed FBP images (Sec. 5 starts the
    iterations from an FBP reconstruction).  The target at acquisition time
    t_k is the FBP image of the window k falls in; the coefficients are the
    least-squares fit over the acquisition times,
        u = argmin sum_k || sum_j phi_j(t_k) u_j - f_{w(k)} ||^2,
    i.e. u_j = sum_w A[j, w] f_w with A = Phi^+ S (the minimum-norm
    least-squares solution; (Phi^T Phi)^{-1} Phi^T S when the functions are
    independent over the acquisition times) and S[k, w] = 1 if projection k
    is in window w.  Returns u[nz][ny][nx][m]."""
    Phi = _c(Phi)
    K, m = Phi.shape
    f = fbp_windows(g, theta, t, nx, ny, n_windows)
    w = np.clip(np.floor(_c(t) * n_windows), 0, n_windows - 1).astype(int)
    S = np.zeros((K, n_windows))
    S[np.arange(K), w] = 1.0
    A = np.linalg.lstsq(Phi, S, rcond=1e-6)[0]
    return np.einsum("jw,zwyx->zyxj", A, f)


# --------------------------------------------------------------------------- #
# Problem + solvers
# --------------------------------------------------------------------------- #
class Problem:
    """Geometry, acquisition and basis of one reconstruction (all FP64)."""

    def __init__(self, nx, ny, nz, ns, theta, t, basis: int, m: int, nt: int):
        self.nx, self.ny, self.nz, self.ns = int(nx), int(ny), int(nz), int(ns)
        self.theta = _c(theta)
        self.t = _c(t)
        self.K = self.theta.size
        self.basis, self.m, self.nt = int(basis), int(m), int(nt)
        kind = int(basis) & 0xff
        self.Phi = basis_table(kind, m, self.t)
        self.PhiF = frame_table(kind, m, nt)
        if int(basis) & ORTHONORMAL:
            if _load().or_orthonormalise(self.Phi, self.K, self.m, self.PhiF, self.nt) != 0:
                raise ValueError("basis columns are linearly dependent over the acquisition times")

    def _head(self):
        return (self.nx, self.ny, self.nz, self.ns, self.K, self.m, self.nt, self.theta, self.Phi,
                self.PhiF)

    def fwd(self, u):
        return dyn_fwd(u, self.theta, self.Phi, self.ns)

    def adj(self, g):
        return dyn_adj(g, self.theta, self.Phi, self.nx, self.ny)

    def D(self, u, lambda2):
        return D(u, self.PhiF, lambda2)

    def DT(self, p, lambda2):
        return DT(p, self.PhiF, lambda2)

    def objective(self, g, u, lambda1, lambda2) -> float:
        return _load().or_objective_flat(*self._head(), _c(g), _c(u), float(lambda1), float(lambda2))

    def fbp_init(self, g, n_windows: int = 1):
        return fbp_init(g, self.theta, self.t, self.Phi, self.nx, self.ny, n_windows)

    def power_norm(self, lambda2, iters: int = 100) -> float:
        return _load().or_power_norm_flat(*self._head(), float(lambda2), int(iters))

    def admm_cg(self, g, u0, iters, n_cg, lambda1, lambda2, rho, want_objective=True,
                want_primal=False):
        u = _c(u0).copy()
        obj, pobj = _optbuf(iters, want_objective)
        pres, ppres = _optbuf(iters, want_primal)
        rc = _load().or_admm_cg_flat(*self._head(), _c(g), u, int(iters), int(n_cg),
                                     float(lambda1), float(lambda2), float(rho), pobj, ppres)
        if rc != 0:
            raise MemoryError("oracle admm_cg failed (%d)" % rc)
        return u, obj, pres

    def chambolle_pock(self, g, u0, iters, lambda1, lambda2, theta_cp=1.0, L=None,
                       want_objective=True):
        if L is None:
            L = self.power_norm(lambda2)
        u = _c(u0).copy()
        obj, pobj = _optbuf(iters, want_objective)
        rc = _load().or_chambolle_pock_flat(*self._head(), _c(g), u, int(iters), float(lambda1),
                                            float(lambda2), float(theta_cp), float(L), pobj)
        if rc != 0:
            raise MemoryError("oracle chambolle_pock failed (%d)" % rc)
        return u, obj
