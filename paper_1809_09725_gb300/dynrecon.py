"""Thin Python binding of the dynrecon C ABI (``include/dynrecon.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library ``libdynrecon.so``.  PyTorch supplies device memory and the stream;
tensors are passed by pointer.  If the library is missing the import of the
entry points fails loudly -- there is no CPU fallback.

The entry points keep the C names: ``dyn_radon_fwd``, ``dyn_radon_adj``,
``tv4d_grad``, ``tv4d_grad_adj``, ``tv4d_prox``, ``admm_solve``.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdynrecon.so")

DR_OK, DR_EINVAL, DR_ENOMEM, DR_ECUDA, DR_ETIMEOUT, DR_ENOTCONV, DR_ECANCELED = 0, -1, -2, -3, -4, -5, -6
FOURIER, LEGENDRE, HAAR, HEAVISIDE, COMPLEX_FOURIER = 0, 1, 2, 3, 4
ORTHONORMAL = 0x100  # flag OR-ed into the basis kind
F32, BF16, F64 = 0, 1, 2
FIELDS_BF16 = 0x10  # flag OR-ed into F32 / BF16: the solvers keep their dual fields in bf16
ADMM_CG, CHAMBOLLE_POCK = 0, 1

_STATUS = {DR_EINVAL: "EINVAL", DR_ENOMEM: "ENOMEM", DR_ECUDA: "ECUDA", DR_ETIMEOUT: "ETIMEOUT",
           DR_ENOTCONV: "ENOTCONV", DR_ECANCELED: "ECANCELED"}

# Every symbol include/dynrecon.h declares.
EXPORTS = ("dr_plan_create", "dr_plan_destroy", "dr_plan_set_stream", "dr_plan_device_bytes",
           "dr_plan_workspace_bytes", "dr_plan_state_bytes", "dr_plan_sync", "dr_plan_wait_selftest", "dr_plan_set_variant", "dr_plan_autotune",
           "dr_plan_set_fold_strip", "dr_plan_set_fold_groups", "dr_plan_set_fold_march", "dr_plan_set_fold_adj_stage", "dr_plan_set_fold_blocks", "dr_plan_info",
           "dyn_radon_fwd", "dyn_radon_adj", "dyn_radon_adj_noalloc", "dr_fbp_init", "tv4d_grad", "tv4d_grad_adj", "tv4d_normal",
           "tv4d_prox", "dr_solve_params_default", "admm_solve", "admm_solve_batch", "cp_solve_slabs",
           "cp_solve_slabs_device_bytes", "dr_job_device_bytes", "dr_job_slab_device_bytes", "dr_server_create",
           "dr_server_submit", "dr_server_cancel", "dr_server_wait", "dr_server_stats", "dr_server_destroy",
           "dr_last_error", "dr_version")

JOB_QUEUED, JOB_RUNNING, JOB_DONE, JOB_FAILED, JOB_CANCELED = 0, 1, 2, 3, 4

DIRECT, FOLD, FOLD2, AUTO = 0, 1, 2, -1  # FOLD2: forward only, the fold in two kernels


class DynreconError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s (%d): %s" % (_STATUS.get(status, "?"), status, msg))
        self.status = status


class PlanInfo(ctypes.Structure):
    _fields_ = [("unique_angles", ctypes.c_int), ("max_group", ctypes.c_int), ("fwd_variant", ctypes.c_int),
                ("adj_variant", ctypes.c_int), ("tuned", ctypes.c_int), ("device_bytes", ctypes.c_size_t),
                ("fold_lines", ctypes.c_int), ("fold_async", ctypes.c_int), ("fold2_group", ctypes.c_int),
                ("fold2_threads", ctypes.c_int),
                ("fold2_rays_per_thread", ctypes.c_int), ("fold2_lines", ctypes.c_int),
                ("fold2_split", ctypes.c_int),
                ("fold2_async", ctypes.c_int), ("fold_adj_angles", ctypes.c_int),
                ("fold2_angles", ctypes.c_int),
                ("fwd_variant_storage", ctypes.c_int)]


class SolveParams(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int), ("iters", ctypes.c_int), ("n_cg", ctypes.c_int),
                ("lambda1", ctypes.c_double), ("lambda2", ctypes.c_double), ("rho", ctypes.c_double),
                ("cp_theta", ctypes.c_double), ("power_iters", ctypes.c_int),
                ("objective_out", ctypes.POINTER(ctypes.c_double)),
                ("primal_res_out", ctypes.POINTER(ctypes.c_double)),
                ("op_norm_out", ctypes.POINTER(ctypes.c_double)), ("op_norm", ctypes.c_double),
                ("state", ctypes.c_void_p), ("resume", ctypes.c_int)]


class JobDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("ns", ctypes.c_int),
                ("K", ctypes.c_int), ("theta", ctypes.POINTER(ctypes.c_double)),
                ("t", ctypes.POINTER(ctypes.c_double)), ("basis", ctypes.c_int), ("m", ctypes.c_int),
                ("nt", ctypes.c_int), ("prec", ctypes.c_int), ("params", SolveParams), ("g", ctypes.c_void_p),
                ("u", ctypes.c_void_p)]


class JobResult(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("status", ctypes.c_int), ("latency_s", ctypes.c_double),
                ("queue_s", ctypes.c_double), ("device_bytes", ctypes.c_size_t), ("slab_nz", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("failed", ctypes.c_int64), ("canceled", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("active", ctypes.c_int), ("p50_latency_s", ctypes.c_double),
                ("p99_latency_s", ctypes.c_double), ("peak_device_bytes", ctypes.c_size_t),
                ("budget_bytes", ctypes.c_size_t), ("voxel_projection_per_s", ctypes.c_double)]


_lib = None


def load(path: str = LIB_PATH):
    """Load ``libdynrecon.so`` and declare the ABI (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libdynrecon.so not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    pd = ctypes.POINTER(ctypes.c_double)
    decl = {
        "dr_plan_create": (i, [ctypes.POINTER(vp), i, i, i, i, i, pd, pd, i, i, i, i, vp]),
        "dr_plan_destroy": (i, [vp]),
        "dr_plan_set_stream": (i, [vp, vp]),
        "dr_plan_device_bytes": (sz, [vp]),
        "dr_plan_workspace_bytes": (sz, [vp, i]),
        "dr_plan_state_bytes": (sz, [vp, i]),
        "dr_plan_sync": (i, [vp]),
        "dr_plan_wait_selftest": (i, [vp, d]),
        "dr_plan_set_variant": (i, [vp, i, i]),
        "dr_plan_autotune": (i, [vp, pd]),
        "dr_plan_set_fold_strip": (i, [vp, i, i]),
        "dr_plan_set_fold_groups": (i, [vp, i, i, i, i]),
        "dr_plan_set_fold_march": (i, [vp, i, i]),
        "dr_plan_set_fold_adj_stage": (i, [vp, i]),
        "dr_plan_set_fold_blocks": (i, [vp, i]),
        "dr_plan_info": (i, [vp, ctypes.POINTER(PlanInfo)]),
        "dyn_radon_fwd": (i, [vp, vp, vp]),
        "dyn_radon_adj": (i, [vp, vp, vp, d]),
        "dyn_radon_adj_noalloc": (i, [vp, vp, vp, d]),
        "dr_fbp_init": (i, [vp, vp, vp, i]),
        "tv4d_grad": (i, [vp, vp, vp, d]),
        "tv4d_grad_adj": (i, [vp, vp, vp, d, d]),
        "tv4d_normal": (i, [vp, vp, vp, d, d]),
        "tv4d_prox": (i, [vp, vp, vp, vp, d, d, d, pd]),
        "dr_solve_params_default": (None, [ctypes.POINTER(SolveParams)]),
        "admm_solve": (i, [vp, vp, vp, ctypes.POINTER(SolveParams)]),
        "admm_solve_batch": (i, [i, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                 ctypes.POINTER(SolveParams)]),
        "cp_solve_slabs": (i, [vp, vp, vp, ctypes.POINTER(SolveParams), i]),
        "cp_solve_slabs_device_bytes": (sz, [vp, i, ctypes.POINTER(SolveParams)]),
        "dr_job_device_bytes": (sz, [ctypes.POINTER(JobDesc)]),
        "dr_job_slab_device_bytes": (sz, [ctypes.POINTER(JobDesc), i]),
        "dr_server_create": (i, [ctypes.POINTER(vp), i, sz, i]),
        "dr_server_submit": (i, [vp, ctypes.POINTER(JobDesc), ctypes.POINTER(ctypes.c_int64)]),
        "dr_server_cancel": (i, [vp, ctypes.c_int64]),
        "dr_server_wait": (i, [vp, ctypes.c_int64, d, ctypes.POINTER(JobResult)]),
        "dr_server_stats": (i, [vp, ctypes.POINTER(ServerStats)]),
        "dr_server_destroy": (i, [vp]),
        "dr_last_error": (ctypes.c_char_p, []),
        "dr_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in decl.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(st: int):
    if st != DR_OK:
        raise DynreconError(st, load().dr_last_error().decode())


def _torch():
    import torch
    return torch


_DTYPES = {F32: "float32", BF16: "bfloat16", F64: "float64"}
_CALC = {F32: "float32", BF16: "float32", F64: "float64"}


def _ptr(x, want_dtype: str, shape, what: str):
    """Device or host pointer of a torch tensor / numpy array after checks."""
    if isinstance(x, np.ndarray):
        if str(x.dtype) != want_dtype and not (want_dtype == "bfloat16" and x.dtype == np.uint16):
            raise TypeError("%s: dtype %s, expected %s" % (what, x.dtype, want_dtype))
        if not x.flags.c_contiguous:
            raise ValueError("%s must be C-contiguous" % what)
        if tuple(x.shape) != tuple(shape):
            raise ValueError("%s: shape %s, expected %s" % (what, tuple(x.shape), tuple(shape)))
        return ctypes.c_void_p(x.ctypes.data)
    torch = _torch()
    if x.dtype != getattr(torch, want_dtype):
        raise TypeError("%s: dtype %s, expected %s" % (what, x.dtype, want_dtype))
    if not x.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    if tuple(x.shape) != tuple(shape):
        raise ValueError("%s: shape %s, expected %s" % (what, tuple(x.shape), tuple(shape)))
    return ctypes.c_void_p(x.data_ptr())


class Plan:
    """A reconstruction geometry: grid (nz, ny, nx), detector bins ns, the
    acquisition (theta_k, t_k), the temporal basis (kind, m) and the frame
    count nt used by the time derivative.  Owns the device tables."""

    def __init__(self, nx: int, ny: int, nz: int, ns: int, theta, t, basis: int = FOURIER, m: int = 4,
                 nt: int = 4, prec: int = F32, stream=None):
        lib = load()
        self.nx, self.ny, self.nz, self.ns = int(nx), int(ny), int(nz), int(ns)
        th = np.ascontiguousarray(theta, dtype=np.float64)
        tt = np.ascontiguousarray(t, dtype=np.float64)
        if th.shape != tt.shape or th.ndim != 1:
            raise ValueError("theta and t must be 1-D of equal length")
        self.K = th.size
        self.basis, self.m, self.nt = int(basis), int(m), int(nt)
        self.prec = int(prec) & ~FIELDS_BF16
        self.fields_bf16 = bool(int(prec) & FIELDS_BF16)
        self._h = ctypes.c_void_p()
        pd = ctypes.POINTER(ctypes.c_double)
        _check(lib.dr_plan_create(ctypes.byref(self._h), self.nx, self.ny, self.nz, self.ns, self.K,
                                  th.ctypes.data_as(pd), tt.ctypes.data_as(pd), self.basis, self.m,
                                  self.nt, int(prec), ctypes.c_void_p(self._stream_handle(stream))))

    @staticmethod
    def _stream_handle(stream) -> int:
        if stream is not None:
            return int(getattr(stream, "cuda_stream", stream))
        try:
            torch = _torch()
            if torch.cuda.is_available():
                return int(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return 0

    def use_current_stream(self):
        _check(load().dr_plan_set_stream(self._h, ctypes.c_void_p(self._stream_handle(None))))

    @property
    def handle(self):
        return self._h

    def u_shape(self):
        return (self.nz, self.ny, self.nx, self.m)

    def g_shape(self):
        return (self.nz, self.K, self.ns)

    def field_shape(self):
        """4-vector fields on frames (D u, the ADMM duals): frame-major within
        each slice, [nz][nt][ny][nx][4]."""
        return (self.nz, self.nt, self.ny, self.nx, 4)

    @property
    def storage_dtype(self) -> str:
        return _DTYPES[self.prec]

    @property
    def field_dtype(self) -> str:
        return _CALC[self.prec]

    def device_bytes(self) -> int:
        return load().dr_plan_device_bytes(self._h)

    def workspace_bytes(self, algo: int = ADMM_CG) -> int:
        return load().dr_plan_workspace_bytes(self._h, int(algo))

    def wait_selftest(self, limit_s: float = 0.05) -> int:
        """Run the bounded-wait failure check; returns the status code
        (DR_ETIMEOUT expected) without raising."""
        return int(load().dr_plan_wait_selftest(self._h, float(limit_s)))

    def state_bytes(self, algo: int = ADMM_CG) -> int:
        """Bytes of the solver state besides u (checkpoint / resume buffer)."""
        return load().dr_plan_state_bytes(self._h, int(algo))

    def sync(self):
        _check(load().dr_plan_sync(self._h))

    def set_variant(self, fwd: int = AUTO, adj: int = AUTO):
        """0 direct, 1 half-turn fold (Sec. 4), 2 (forward) fold in two kernels, -1 automatic."""
        _check(load().dr_plan_set_variant(self._h, int(fwd), int(adj)))

    def autotune(self):
        """Time the projector variants; returns [fwd direct, fwd fold, adj direct, adj fold,
        fwd fold in two kernels] ms."""
        self.use_current_stream()
        t = (ctypes.c_double * 5)()
        _check(load().dr_plan_autotune(self._h, t))
        return list(t)

    def set_fold_strip(self, lines: int, async_copy: bool = False):
        """Fix the folded forward's strip height and staging (results do not change)."""
        _check(load().dr_plan_set_fold_strip(self._h, int(lines), int(bool(async_copy))))

    def set_fold_groups(self, group: int, lines: int, threads: int = 256, rays_per_thread: int = 0):
        """Fix the two-kernel folded forward's coefficient group (4, 8), CTA size,
        rays per thread (0: the most for the group and CTA size) and strip height."""
        _check(load().dr_plan_set_fold_groups(self._h, int(group), int(threads), int(rays_per_thread), int(lines)))

    def set_fold_march(self, nsplit: int = 1, async_stage: int = 0):
        """Two-kernel folded forward: line chunks of each ray's march, and
        strip staging (0 synchronous, 1 double-, 2 triple-buffered cp.async)."""
        _check(load().dr_plan_set_fold_march(self._h, int(nsplit), int(async_stage)))

    def set_fold_adj_stage(self, angles: int):
        """Folded adjoint: distinct angles per pipeline stage."""
        _check(load().dr_plan_set_fold_adj_stage(self._h, int(angles)))

    def set_fold_blocks(self, extra: int):
        """Two-kernel folded forward: extra angle blocks per stepping axis (0..3)."""
        _check(load().dr_plan_set_fold_blocks(self._h, int(extra)))

    def info(self) -> dict:
        inf = PlanInfo()
        _check(load().dr_plan_info(self._h, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in PlanInfo._fields_}

    def close(self):
        if self._h:
            load().dr_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dyn_radon_fwd(plan: Plan, u, g):
    """g = R u (Eq. radapr).  u [nz][ny][nx][m], g [nz][K][ns], device tensors."""
    plan.use_current_stream()
    _check(load().dyn_radon_fwd(plan.handle, _ptr(u, plan.storage_dtype, plan.u_shape(), "u"),
                                _ptr(g, plan.storage_dtype, plan.g_shape(), "g")))
    return g


def dyn_radon_adj(plan: Plan, g, u, beta: float = 0.0):
    """u = beta u + R* g (Eq. radadjapr)."""
    plan.use_current_stream()
    _check(load().dyn_radon_adj(plan.handle, _ptr(g, plan.storage_dtype, plan.g_shape(), "g"),
                                _ptr(u, plan.storage_dtype, plan.u_shape(), "u"), float(beta)))
    return u


def dyn_radon_adj_noalloc(plan: Plan, g, u, beta: float = 0.0):
    """u = beta u + R* g by the half-turn fold, with the folded data in the
    library's fixed 8 MiB device array: allocates no device memory (for
    callers inside a stream capture or under a no-allocation policy)."""
    plan.use_current_stream()
    _check(load().dyn_radon_adj_noalloc(plan.handle, _ptr(g, plan.storage_dtype, plan.g_shape(), "g"),
                                        _ptr(u, plan.storage_dtype, plan.u_shape(), "u"), float(beta)))
    return u


def fbp_init(plan: Plan, g, u, n_windows: int = 1):
    """u = least-squares fit over the acquisition times of the Shepp-Logan FBP
    images of ``n_windows`` time windows (the initial guess of Sec. 5)."""
    plan.use_current_stream()
    _check(load().dr_fbp_init(plan.handle, _ptr(g, plan.storage_dtype, plan.g_shape(), "g"),
                              _ptr(u, plan.storage_dtype, plan.u_shape(), "u"), int(n_windows)))
    return u


def tv4d_grad(plan: Plan, u, p, lambda2: float):
    """p = D u = nabla_{lambda2} of the synthesised frames (Eq. TV1)."""
    plan.use_current_stream()
    _check(load().tv4d_grad(plan.handle, _ptr(u, plan.storage_dtype, plan.u_shape(), "u"),
                            _ptr(p, plan.field_dtype, plan.field_shape(), "p"), float(lambda2)))
    return p


def tv4d_grad_adj(plan: Plan, p, u, lambda2: float, beta: float = 0.0):
    """u = beta u + D^T p."""
    plan.use_current_stream()
    _check(load().tv4d_grad_adj(plan.handle, _ptr(p, plan.field_dtype, plan.field_shape(), "p"),
                                _ptr(u, plan.storage_dtype, plan.u_shape(), "u"), float(lambda2),
                                float(beta)))
    return u


def tv4d_normal(plan: Plan, x, out, lambda2: float, beta: float = 0.0):
    """out = beta out + D^T D x on compute-typed coefficient arrays (the
    plan's field dtype: float for F32/BF16 plans, double for F64)."""
    plan.use_current_stream()
    _check(load().tv4d_normal(plan.handle, _ptr(x, plan.field_dtype, plan.u_shape(), "x"),
                              _ptr(out, plan.field_dtype, plan.u_shape(), "out"), float(lambda2), float(beta)))
    return out


def tv4d_prox(plan: Plan, u, mu, w, rho: float, lambda1: float, lambda2: float,
              want_residual: bool = False) -> Optional[float]:
    """ADMM shrink + dual update on psi = D u (in place on mu, w)."""
    plan.use_current_stream()
    res = ctypes.c_double(0.0)
    _check(load().tv4d_prox(plan.handle, _ptr(u, plan.storage_dtype, plan.u_shape(), "u"),
                            _ptr(mu, plan.field_dtype, plan.field_shape(), "mu"),
                            _ptr(w, plan.field_dtype, plan.field_shape(), "w"), float(rho),
                            float(lambda1), float(lambda2),
                            ctypes.byref(res) if want_residual else None))
    return res.value if want_residual else None


def solve_params(algo: int = ADMM_CG, iters: int = 20, n_cg: int = 4, lambda1: float = 1e-3,
                 lambda2: float = 1.0, rho: float = 0.0, cp_theta: float = 1.0,
                 power_iters: int = 100, op_norm: float = 0.0, state=None, resume: bool = False) -> SolveParams:
    """state: a device tensor of Plan.state_bytes(algo) bytes (kept alive by
    the caller) that receives the solver state at the end of the call;
    resume: start from it instead of zero duals."""
    p = SolveParams()
    load().dr_solve_params_default(ctypes.byref(p))
    p.algo, p.iters, p.n_cg = int(algo), int(iters), int(n_cg)
    p.lambda1, p.lambda2, p.rho, p.cp_theta = float(lambda1), float(lambda2), float(rho), float(cp_theta)
    p.power_iters = int(power_iters)
    p.op_norm = float(op_norm)
    if state is not None:
        if not getattr(state, "is_cuda", False):
            raise ValueError("state must be a device tensor")
        p.state = ctypes.c_void_p(state.data_ptr())
    p.resume = 1 if resume else 0
    return p


def admm_solve(plan: Plan, g, u, params: SolveParams, want_objective: bool = True,
               want_primal: bool = False):
    """Solve Eq. (lr12) in place on u; g and u may live on the host or the
    device.  Returns dict(objective=..., primal_res=..., op_norm=...)."""
    plan.use_current_stream()
    n = max(int(params.iters), 1)
    obj = np.zeros(n, dtype=np.float64)
    pres = np.zeros(n, dtype=np.float64)
    opn = ctypes.c_double(0.0)
    pd = ctypes.POINTER(ctypes.c_double)
    params.objective_out = obj.ctypes.data_as(pd) if want_objective else None
    params.primal_res_out = pres.ctypes.data_as(pd) if want_primal else None
    params.op_norm_out = ctypes.pointer(opn)
    _check(load().admm_solve(plan.handle, _ptr(g, plan.storage_dtype, plan.g_shape(), "g"),
                             _ptr(u, plan.storage_dtype, plan.u_shape(), "u"), ctypes.byref(params)))
    it = int(params.iters)
    return {"objective": obj[:it] if want_objective else None,
            "primal_res": pres[:it] if want_primal else None,
            "op_norm": opn.value}


def cp_solve_slabs(plan: Plan, g: np.ndarray, u: np.ndarray, params: SolveParams, slab_nz: int,
                   want_objective: bool = True):
    """Chambolle-Pock on host-resident g and u, streamed through the GPU in
    slabs of ``slab_nz`` slices (in place on u).  Returns dict(objective, op_norm)."""
    plan.use_current_stream()
    n = max(int(params.iters), 1)
    obj = np.zeros(n, dtype=np.float64)
    opn = ctypes.c_double(0.0)
    pd = ctypes.POINTER(ctypes.c_double)
    params.objective_out = obj.ctypes.data_as(pd) if want_objective else None
    params.primal_res_out = None
    params.op_norm_out = ctypes.pointer(opn)
    _check(load().cp_solve_slabs(plan.handle, _ptr(g, plan.storage_dtype, plan.g_shape(), "g"),
                                 _ptr(u, plan.storage_dtype, plan.u_shape(), "u"), ctypes.byref(params),
                                 int(slab_nz)))
    it = int(params.iters)
    return {"objective": obj[:it] if want_objective else None, "op_norm": opn.value}


def cp_solve_slabs_device_bytes(plan: Plan, slab_nz: int, params: SolveParams) -> int:
    return int(load().cp_solve_slabs_device_bytes(plan.handle, int(slab_nz), ctypes.byref(params)))


def version() -> str:
    return load().dr_version().decode()


def admm_solve_batch(plans, gs, us, params_list):
    """Solve several independent jobs together: one CUDA graph per iteration
    with one branch per job (results equal separate admm_solve calls)."""
    n = len(plans)
    for p in plans:
        p.use_current_stream()
    hp = (ctypes.c_void_p * n)(*[p.handle.value for p in plans])
    hg = (ctypes.c_void_p * n)(*[_ptr(g, p.storage_dtype, p.g_shape(), "g").value for p, g in zip(plans, gs)])
    hu = (ctypes.c_void_p * n)(*[_ptr(u, p.storage_dtype, p.u_shape(), "u").value for p, u in zip(plans, us)])
    prm = (SolveParams * n)(*params_list)
    _check(load().admm_solve_batch(n, hp, hg, hu, prm))


def job_desc(nx, ny, nz, ns, theta, t, basis, m, nt, prec, params: SolveParams, g, u) -> JobDesc:
    """Describe a reconstruction request (g, u: host numpy arrays or device tensors,
    kept alive by the caller until the job finishes).  g = u = None describes
    the job's sizes only (for job_device_bytes; the server refuses it)."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    tt = np.ascontiguousarray(t, dtype=np.float64)
    pd = ctypes.POINTER(ctypes.c_double)
    d = JobDesc()
    d.nx, d.ny, d.nz, d.ns, d.K = int(nx), int(ny), int(nz), int(ns), th.size
    d.theta, d.t = th.ctypes.data_as(pd), tt.ctypes.data_as(pd)
    d.basis, d.m, d.nt, d.prec = int(basis), int(m), int(nt), int(prec)
    d.params = params
    dt = _DTYPES[int(prec) & ~FIELDS_BF16]
    d.g = None if g is None else _ptr(g, dt, (nz, th.size, ns), "g").value
    d.u = None if u is None else _ptr(u, dt, (nz, ny, nx, m), "u").value
    d._keep = (th, tt, g, u)
    return d


def job_device_bytes(desc: JobDesc) -> int:
    return load().dr_job_device_bytes(ctypes.byref(desc))


def job_slab_device_bytes(desc: JobDesc, slab_nz: int) -> int:
    return load().dr_job_slab_device_bytes(ctypes.byref(desc), int(slab_nz))


class Server:
    """Request loop: jobs are admitted under a device-memory budget and run
    concurrently (one worker thread, plan and stream per running job)."""

    def __init__(self, device: int = 0, budget_bytes: int = 1 << 30, slots: int = 4):
        self._h = ctypes.c_void_p()
        _check(load().dr_server_create(ctypes.byref(self._h), int(device), int(budget_bytes), int(slots)))
        self._descs = {}

    def submit(self, desc: JobDesc) -> int:
        jid = ctypes.c_int64(0)
        _check(load().dr_server_submit(self._h, ctypes.byref(desc), ctypes.byref(jid)))
        self._descs[jid.value] = desc
        return jid.value

    def cancel(self, job_id: int):
        _check(load().dr_server_cancel(self._h, ctypes.c_int64(job_id)))

    def wait(self, job_id: int, timeout_s: float = -1.0) -> dict:
        r = JobResult()
        st = load().dr_server_wait(self._h, ctypes.c_int64(job_id), float(timeout_s), ctypes.byref(r))
        out = {f: getattr(r, f) for f, _ in JobResult._fields_}
        out["error"] = load().dr_last_error().decode() if st != DR_OK else ""
        out["rc"] = st
        return out

    def stats(self) -> dict:
        s = ServerStats()
        _check(load().dr_server_stats(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in ServerStats._fields_}

    def close(self):
        if self._h:
            load().dr_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
