"""GPU parity of the solvers for Eq. (lr12) against the oracle, iteration by
iteration from the same initial guess (the model can have several
minimisers, so parity is defined per iteration of the same algorithm).

ADMM-CG (the workload's solver) and Chambolle-Pock (Sec. 3, Fig. 2) on the
single-slice disks workload (64^2, 256 projections over 4 half-turns, m = 4
Fourier, 20 x 4 CG), FP64 and FP32 plans; a 2-slice cut of the 256^2 x 1800
ellipsoid workload; host-buffer inputs; BF16 storage; degenerate inputs.
"""
import numpy as np
import pytest

import oracle
from paper_1809_09725_gb300 import dynrecon as dr
from paper_1809_09725_gb300 import synth

from _common import dev_tensor, host_values, rel, to_bf16_f64

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _disks():
    w = synth.WORKLOADS["disks64"]
    theta, t, g = synth.make_data(w)
    P = oracle.Problem(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt)
    return w, theta, t, g, P


@pytest.fixture(scope="module")
def disks():
    return _disks()


@pytest.fixture(scope="module")
def disks_oracle_admm(disks):
    w, theta, t, g, P = disks
    u0 = np.zeros((w.nz, w.N, w.N, w.m))
    g32 = g.astype(np.float32).astype(np.float64)
    out = {}
    out["f64"] = P.admm_cg(g, u0, w.iters, w.n_cg, w.lambda1, w.lambda2, w.rho, want_primal=True)
    out["f32"] = P.admm_cg(g32, u0, w.iters, w.n_cg, w.lambda1, w.lambda2, w.rho, want_primal=True)
    return out


def _run(w, theta, t, g, prec, algo, iters=None, host=False, **kw):
    plan = dr.Plan(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt, prec)
    prm = dr.solve_params(algo, iters=w.iters if iters is None else iters, n_cg=w.n_cg, lambda1=w.lambda1,
                          lambda2=w.lambda2, rho=w.rho, **kw)
    if host:
        dt = {dr.F32: np.float32, dr.F64: np.float64}[prec]
        gd = np.ascontiguousarray(g, dtype=dt)
        ud = np.zeros(plan.u_shape(), dtype=dt)
    else:
        gd = dev_tensor(g, prec)
        ud = torch.zeros(plan.u_shape(), dtype=getattr(torch, plan.storage_dtype), device="cuda")
    res = dr.admm_solve(plan, gd, ud, prm, want_primal=True)
    u = ud.astype(np.float64) if host else host_values(ud)
    return u, res


def test_admm_f64_matches_oracle_every_iteration(disks, disks_oracle_admm):
    w, theta, t, g, P = disks
    uo, oo, po = disks_oracle_admm["f64"]
    u, res = _run(w, theta, t, g, dr.F64, dr.ADMM_CG)
    assert rel(res["objective"], oo) <= 1e-9
    assert rel(res["primal_res"], po) <= 1e-8
    assert rel(u, uo) <= 1e-8


# FP32 solves: the data residual g - R u carries an absolute rounding error of
# about eps32 * |g|, and the CG right-hand side R*(g - R u) is ~1e-4 of R* g
# on this near-interpolating problem (16384 unknowns, 16384 data, lambda1 =
# 1e-3), so the FP32 iterates differ from FP64 ones by ~1e4 eps32 ~ 1e-4.
# Which rounding errors get amplified depends on the order of the float sums
# (projector variant, interpolation order, normal operator): after 20
# iterations u is measured between 5e-5 and 3.4e-4 from the FP64 iterates
# over the three variant pairs and two summation orders of the Joseph taps,
# the objective within 9.6e-4.  The FP64 plan, which runs the same algorithm,
# matches to 1e-9 (test above).
F32_SOLVE_TOL_U = 6e-4
F32_SOLVE_TOL_OBJ = 2e-3


@pytest.mark.parametrize("fwd,adj", [(dr.DIRECT, dr.DIRECT), (dr.FOLD, dr.FOLD), (dr.FOLD2, dr.FOLD)])
def test_admm_f32_matches_oracle(disks, disks_oracle_admm, fwd, adj):
    """(FOLD2, FOLD) runs the CG products through the folded normal operator:
    static transforms mixed per distinct angle by the Gram matrix of its
    projections' basis rows, then back-projected."""
    w, theta, t, g, P = disks
    uo, oo, po = disks_oracle_admm["f32"]
    g32 = g.astype(np.float32).astype(np.float64)
    plan = dr.Plan(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt, dr.F32)
    plan.set_variant(fwd, adj)
    ud = torch.zeros(plan.u_shape(), dtype=torch.float32, device="cuda")
    prm = dr.solve_params(dr.ADMM_CG, iters=w.iters, n_cg=w.n_cg, lambda1=w.lambda1, lambda2=w.lambda2, rho=w.rho)
    res = dr.admm_solve(plan, dev_tensor(g32, dr.F32), ud, prm)
    assert rel(host_values(ud), uo) <= F32_SOLVE_TOL_U
    assert np.max(np.abs(res["objective"] - oo) / np.abs(oo)) <= F32_SOLVE_TOL_OBJ


def test_admm_host_buffers_equal_device_buffers(disks):
    w, theta, t, g, P = disks
    g32 = g.astype(np.float32).astype(np.float64)
    ud, rd = _run(w, theta, t, g32, dr.F32, dr.ADMM_CG, iters=5)
    uh, rh = _run(w, theta, t, g32, dr.F32, dr.ADMM_CG, iters=5, host=True)
    np.testing.assert_array_equal(ud, uh)
    np.testing.assert_array_equal(rd["objective"], rh["objective"])


def test_admm_is_deterministic(disks):
    w, theta, t, g, P = disks
    a, ra = _run(w, theta, t, g, dr.F32, dr.ADMM_CG, iters=6)
    b, rb = _run(w, theta, t, g, dr.F32, dr.ADMM_CG, iters=6)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(ra["objective"], rb["objective"])


@pytest.mark.parametrize("prec,tol_u,tol_o", [(dr.F64, 1e-9, 1e-10), (dr.F32, 3e-4, 2e-3)])
def test_chambolle_pock_matches_oracle(disks, prec, tol_u, tol_o):
    w, theta, t, g, P = disks
    if prec == dr.F32:
        g = g.astype(np.float32).astype(np.float64)
    u0 = np.zeros((w.nz, w.N, w.N, w.m))
    L = P.power_norm(w.lambda2)
    uo, oo = P.chambolle_pock(g, u0, w.iters, w.lambda1, w.lambda2, 1.0, L)
    u, res = _run(w, theta, t, g, prec, dr.CHAMBOLLE_POCK)
    assert abs(res["op_norm"] - L) <= (1e-10 if prec == dr.F64 else 1e-5) * L
    assert rel(u, uo) <= tol_u
    assert rel(res["objective"], oo) <= tol_o


def test_ellipsoid_workload_two_slices_fp32():
    """A 2-slice cut of the 256^2 x 1800-projection ellipsoid workload, 3 ADMM-CG iterations."""
    w = synth.WORKLOADS["ellipsoids256"]
    theta, t, g = synth.make_data(w, nz=2)
    g = g.astype(np.float32).astype(np.float64)
    P = oracle.Problem(w.N, w.N, 2, w.ns, theta, t, w.basis, w.m, w.nt)
    uo, oo, _ = P.admm_cg(g, np.zeros((2, w.N, w.N, w.m)), 3, w.n_cg, w.lambda1, w.lambda2, w.rho)
    plan = dr.Plan(w.N, w.N, 2, w.ns, theta, t, w.basis, w.m, w.nt, dr.F32)
    ud = torch.zeros(plan.u_shape(), dtype=torch.float32, device="cuda")
    prm = dr.solve_params(dr.ADMM_CG, iters=3, n_cg=w.n_cg, lambda1=w.lambda1, lambda2=w.lambda2, rho=w.rho)
    res = dr.admm_solve(plan, dev_tensor(g, dr.F32), ud, prm)
    assert rel(host_values(ud), uo) <= F32_SOLVE_TOL_U
    assert np.max(np.abs(res["objective"] - oo) / np.abs(oo)) <= F32_SOLVE_TOL_OBJ


@pytest.mark.parametrize("algo", [dr.ADMM_CG, dr.CHAMBOLLE_POCK])
@pytest.mark.parametrize("prec", [dr.F64, dr.F32])
def test_banded_walk_solve_matches_oracle(algo, prec):
    """A volume whose rows (u plus 64 frames of duals) fill more than one
    4 MB band per slice: every TV stencil of the solve walks it in bands
    (30 rows in FP64, 60 in FP32: full bands and a partial one); in FP32
    with m = 16 the CG's D^T D is the z-marching tiled kernel (two tiles
    across x, a partial tile row).  Three iterations against the oracle
    from zero."""
    nx, ny, nz, ns, K, m, nt = 64, 130, 2, 96, 16, 16, 64
    theta, t = synth.scan(K, 2.0)
    g = synth.rng_for(4242).standard_normal((nz, K, ns))
    if prec == dr.F32:
        g = g.astype(np.float32).astype(np.float64)
    P = oracle.Problem(nx, ny, nz, ns, theta, t, dr.FOURIER, m, nt)
    u0 = np.zeros((nz, ny, nx, m))
    lam1, lam2, rho, n_cg = 0.05, 1.0, 0.5, 4
    plan = dr.Plan(nx, ny, nz, ns, theta, t, dr.FOURIER, m, nt, prec)
    ud = torch.zeros(plan.u_shape(), dtype=getattr(torch, plan.storage_dtype), device="cuda")
    prm = dr.solve_params(algo, iters=3, n_cg=n_cg, lambda1=lam1, lambda2=lam2, rho=rho)
    res = dr.admm_solve(plan, dev_tensor(g, prec), ud, prm)
    if algo == dr.ADMM_CG:
        uo, oo, _ = P.admm_cg(g, u0, 3, n_cg, lam1, lam2, rho)
    else:
        L = P.power_norm(lam2)
        assert abs(res["op_norm"] - L) <= (1e-10 if prec == dr.F64 else 1e-5) * L
        uo, oo = P.chambolle_pock(g, u0, 3, lam1, lam2, 1.0, L)
    tol_u, tol_o = (1e-9, 1e-10) if prec == dr.F64 else (F32_SOLVE_TOL_U, F32_SOLVE_TOL_OBJ)
    assert rel(host_values(ud), uo) <= tol_u
    assert np.max(np.abs(np.asarray(res["objective"]) - oo) / np.abs(oo)) <= tol_o


def test_bf16_storage_solve(disks):
    """BF16 data and coefficients, FP32 state: error against the oracle run on
    the bf16-rounded data (output rounding to bf16 included)."""
    w, theta, t, g, P = disks
    gb = to_bf16_f64(g)
    uo, oo, _ = P.admm_cg(gb, np.zeros((w.nz, w.N, w.N, w.m)), 5, w.n_cg, w.lambda1, w.lambda2, w.rho)
    plan = dr.Plan(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt, dr.BF16)
    ud = torch.zeros(plan.u_shape(), dtype=torch.bfloat16, device="cuda")
    prm = dr.solve_params(dr.ADMM_CG, iters=5, n_cg=w.n_cg, lambda1=w.lambda1, lambda2=w.lambda2, rho=w.rho)
    res = dr.admm_solve(plan, dev_tensor(gb, dr.BF16), ud, prm)
    assert rel(host_values(ud), uo) <= 2.0 ** -8
    # state and arithmetic are FP32: the FP32 solve gate applies to the objective
    assert np.max(np.abs(res["objective"] - oo) / np.abs(oo)) <= F32_SOLVE_TOL_OBJ


def test_zero_data_keeps_zero_solution(disks):
    w, theta, t, g, P = disks
    u, res = _run(w, theta, t, np.zeros_like(g), dr.F32, dr.ADMM_CG, iters=3)
    assert np.all(u == 0.0)
    assert np.all(res["objective"] == 0.0)


def test_zero_iterations_leave_u_unchanged(disks):
    w, theta, t, g, P = disks
    plan = dr.Plan(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt, dr.F32)
    u0 = synth.rng_for(3).standard_normal(plan.u_shape())
    ud = dev_tensor(u0, dr.F32)
    dr.admm_solve(plan, dev_tensor(g, dr.F32), ud, dr.solve_params(iters=0))
    np.testing.assert_array_equal(host_values(ud), u0.astype(np.float32))


def test_solver_rejects_bad_parameters(disks):
    w, theta, t, g, P = disks
    plan = dr.Plan(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt, dr.F32)
    ud = torch.zeros(plan.u_shape(), dtype=torch.float32, device="cuda")
    for bad in (dict(iters=-1), dict(n_cg=0), dict(lambda1=-1.0), dict(cp_theta=2.0, algo=dr.CHAMBOLLE_POCK)):
        with pytest.raises(dr.DynreconError):
            dr.admm_solve(plan, dev_tensor(g, dr.F32), ud, dr.solve_params(**bad))


def test_folded_normal_operator_matches_forward_then_adjoint():
    """One power-iteration estimate of ||[R; D]|| through the folded normal
    operator equals the one through forward + adjoint to FP32 rounding, with
    and without line chunks (Chambolle-Pock reports the norm it used)."""
    args = (40, 36, 3, 44, *synth.scan(200, 5.0), dr.LEGENDRE, 6, 4)
    nx, ny, nz, ns, theta, t, basis, m, nt = args
    rng = synth.rng_for(61)
    g = rng.standard_normal((nz, len(theta), ns)).astype(np.float32)
    norms = {}
    for key, fwd, nsplit in (("plain", dr.FOLD, 1), ("normal", dr.FOLD2, 1), ("normal_split", dr.FOLD2, 3)):
        plan = dr.Plan(nx, ny, nz, ns, theta, t, basis, m, nt, dr.F32)
        plan.set_variant(fwd, dr.FOLD)
        if fwd == dr.FOLD2:
            plan.set_fold_march(nsplit, 1)
        u = torch.zeros(plan.u_shape(), dtype=torch.float32, device="cuda")
        res = dr.admm_solve(plan, torch.from_numpy(g).cuda(), u,
                            dr.solve_params(dr.CHAMBOLLE_POCK, iters=1, lambda1=0.01, lambda2=1.0, power_iters=30))
        norms[key] = res["op_norm"]
    assert abs(norms["normal"] - norms["plain"]) <= 1e-5 * norms["plain"]
    assert abs(norms["normal_split"] - norms["plain"]) <= 1e-5 * norms["plain"]


@pytest.mark.parametrize("algo", [dr.ADMM_CG, dr.CHAMBOLLE_POCK])
@pytest.mark.parametrize("prec", [dr.F64, dr.F32])
def test_checkpoint_resume_continues_the_iteration(disks, algo, prec):
    """A solve of a + b iterations equals a solve of a iterations whose
    state buffer (duals; Chambolle-Pock also h1 and the extrapolated u) is
    handed to a second solve of b iterations with resume (same operator norm
    for Chambolle-Pock): iterates and objective rows continue unchanged.
    (With BF16 storage the u handed between the calls is rounded to bf16.)"""
    w, theta, t, g, P = disks
    a, b = 3, 4
    plan = dr.Plan(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt, prec)
    sdt = getattr(torch, plan.storage_dtype)
    gd = dev_tensor(g, prec)
    kw = dict(n_cg=w.n_cg, lambda1=w.lambda1, lambda2=w.lambda2, rho=w.rho)
    u_all = torch.zeros(plan.u_shape(), dtype=sdt, device="cuda")
    r_all = dr.admm_solve(plan, gd, u_all, dr.solve_params(algo, iters=a + b, **kw))
    kw["op_norm"] = r_all["op_norm"] if algo == dr.CHAMBOLLE_POCK else 0.0
    state = torch.empty(plan.state_bytes(algo), dtype=torch.uint8, device="cuda")
    u = torch.zeros_like(u_all)
    r1 = dr.admm_solve(plan, gd, u, dr.solve_params(algo, iters=a, state=state, **kw))
    r2 = dr.admm_solve(plan, gd, u, dr.solve_params(algo, iters=b, state=state, resume=True, **kw))
    plan.sync()
    tol = 1e-12 if prec == dr.F64 else 1e-6
    assert rel(host_values(u), host_values(u_all)) <= tol
    assert rel(np.concatenate([r1["objective"], r2["objective"]]), r_all["objective"]) <= tol
    # without the state the second call restarts the duals: a different iterate
    u_re = torch.zeros_like(u_all)
    dr.admm_solve(plan, gd, u_re, dr.solve_params(algo, iters=a, **kw))
    dr.admm_solve(plan, gd, u_re, dr.solve_params(algo, iters=b, **kw))
    assert rel(host_values(u_re), host_values(u_all)) > 10 * tol


def test_resume_without_state_is_rejected(disks):
    w, theta, t, g, P = disks
    plan = dr.Plan(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt, dr.F32)
    u = torch.zeros(plan.u_shape(), dtype=torch.float32, device="cuda")
    with pytest.raises(dr.DynreconError):
        dr.admm_solve(plan, dev_tensor(g, dr.F32), u, dr.solve_params(dr.ADMM_CG, iters=2, resume=True))
    assert plan.state_bytes(dr.ADMM_CG) == 2 * 4 * w.nt * w.N * w.N * w.nz * 4
    assert plan.state_bytes(dr.CHAMBOLLE_POCK) == 4 * (4 * w.nt * w.N * w.N * w.nz + w.K * w.ns * w.nz
                                                       + w.m * w.N * w.N * w.nz)


# --------------------------------------------------------------------------- #
# Dual fields stored in bf16 (DR_FIELDS_BF16): same arithmetic, one rounding
# of mu, w (h2) per store; the reconstruction error is that of the FP32 solve
# (the duals hold lambda-sized values; their rounding moves u by ~1e-7 in the
# FP64 model of the same iteration)
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("algo", [dr.ADMM_CG, dr.CHAMBOLLE_POCK])
def test_bf16_fields_solve_matches_oracle(disks, disks_oracle_admm, algo):
    w, theta, t, g, P = disks
    g32 = g.astype(np.float32).astype(np.float64)
    kw = dict(n_cg=w.n_cg, lambda1=w.lambda1, lambda2=w.lambda2, rho=w.rho)
    if algo == dr.ADMM_CG:
        uo, oo, _ = disks_oracle_admm["f32"]
    else:
        L = P.power_norm(w.lambda2)
        uo, oo = P.chambolle_pock(g32, np.zeros((w.nz, w.N, w.N, w.m)), w.iters, w.lambda1, w.lambda2, 1.0, L)
        kw["op_norm"] = L
    outs = {}
    for prec in (dr.F32, dr.F32 | dr.FIELDS_BF16):
        plan = dr.Plan(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt, prec)
        ud = torch.zeros(plan.u_shape(), dtype=torch.float32, device="cuda")
        res = dr.admm_solve(plan, dev_tensor(g32, dr.F32), ud, dr.solve_params(algo, iters=w.iters, **kw))
        outs[prec] = (host_values(ud), res["objective"], plan)
    u, obj, plan = outs[dr.F32 | dr.FIELDS_BF16]
    tol_u = F32_SOLVE_TOL_U if algo == dr.ADMM_CG else 3e-4
    assert rel(u, uo) <= tol_u
    assert np.max(np.abs(obj - oo) / np.abs(oo)) <= F32_SOLVE_TOL_OBJ
    assert rel(u, outs[dr.F32][0]) <= tol_u
    # the fields take half the bytes: ADMM two fields, Chambolle-Pock one
    nf = 4 * w.nt * w.N * w.N * w.nz
    assert outs[dr.F32][2].workspace_bytes(algo) - plan.workspace_bytes(algo) == (2 if algo == dr.ADMM_CG else 1) * 2 * nf


def test_bf16_fields_checkpoint_resume_and_state_size(disks):
    """The state buffer holds the bf16 fields as they are: 3 + 4 iterations
    with the state handed over equal 7 in one call."""
    w, theta, t, g, P = disks
    plan = dr.Plan(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt, dr.F32 | dr.FIELDS_BF16)
    assert plan.state_bytes(dr.ADMM_CG) == 2 * 4 * w.nt * w.N * w.N * w.nz * 2
    gd = dev_tensor(g, dr.F32)
    kw = dict(n_cg=w.n_cg, lambda1=w.lambda1, lambda2=w.lambda2, rho=w.rho)
    u_all = torch.zeros(plan.u_shape(), dtype=torch.float32, device="cuda")
    r_all = dr.admm_solve(plan, gd, u_all, dr.solve_params(dr.ADMM_CG, iters=7, **kw))
    state = torch.empty(plan.state_bytes(dr.ADMM_CG), dtype=torch.uint8, device="cuda")
    u = torch.zeros_like(u_all)
    r1 = dr.admm_solve(plan, gd, u, dr.solve_params(dr.ADMM_CG, iters=3, state=state, **kw))
    r2 = dr.admm_solve(plan, gd, u, dr.solve_params(dr.ADMM_CG, iters=4, state=state, resume=True, **kw))
    plan.sync()
    assert rel(host_values(u), host_values(u_all)) <= 1e-6
    assert rel(np.concatenate([r1["objective"], r2["objective"]]), r_all["objective"]) <= 1e-6


def test_bf16_fields_rejected_for_f64():
    theta, t = synth.scan(16, 1.0)
    with pytest.raises(dr.DynreconError):
        dr.Plan(8, 8, 1, 8, theta, t, dr.FOURIER, 2, 2, dr.F64 | dr.FIELDS_BF16)
