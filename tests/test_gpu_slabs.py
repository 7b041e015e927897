"""Slab-streamed Chambolle-Pock (Sec. 6: slabs of slices with the neighbouring
slices for the z derivatives, copies overlapped with the computation) against
the whole-volume solver and the oracle.

* With the same operator norm and projector variants, every slab thickness
  gives the in-core Chambolle-Pock result bit for bit (FP32, FP64, BF16).
* With the streamed power iteration, the FP64 result matches the oracle's
  Chambolle-Pock (and its operator norm).
* Bad arguments, memory estimate, non-finite data.
"""
import numpy as np
import pytest

import oracle
from paper_1809_09725_gb300 import dynrecon as dr
from paper_1809_09725_gb300 import synth

from _common import dev_tensor, host_values, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N, NZ, K, HT, M, NT = 40, 7, 120, 3.0, 4, 3
LAM1, LAM2 = 0.05, 1.0


def _problem(seed=0, nz=NZ):
    theta, t = synth.scan(K, HT)
    rng = synth.rng_for(4200 + seed)
    g = rng.standard_normal((nz, K, N)) * 3.0
    return theta, t, g


def _host(x, prec):
    if prec == dr.BF16:
        return torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16).copy()
    return np.ascontiguousarray(x, dtype=np.float64 if prec == dr.F64 else np.float32)


def _to_f64(a, prec):
    if prec == dr.BF16:
        return torch.from_numpy(a.view(np.int16)).view(torch.bfloat16).to(torch.float64).numpy()
    return a.astype(np.float64)


def _incore(theta, t, g, prec, iters, variant, nz=NZ, op_norm=0.0):
    plan = dr.Plan(N, N, nz, N, theta, t, dr.FOURIER, M, NT, prec)
    plan.set_variant(variant, variant)
    u = torch.zeros(plan.u_shape(), dtype=getattr(torch, plan.storage_dtype), device="cuda")
    prm = dr.solve_params(dr.CHAMBOLLE_POCK, iters=iters, lambda1=LAM1, lambda2=LAM2, op_norm=op_norm)
    res = dr.admm_solve(plan, dev_tensor(g, prec), u, prm)
    return host_values(u), res


def _slabs(theta, t, g, prec, iters, variant, slab, nz=NZ, op_norm=0.0, power_iters=100):
    plan = dr.Plan(N, N, nz, N, theta, t, dr.FOURIER, M, NT, prec)
    if variant is not None:
        plan.set_variant(variant, variant)
    u = _host(np.zeros(plan.u_shape()), prec)
    prm = dr.solve_params(dr.CHAMBOLLE_POCK, iters=iters, lambda1=LAM1, lambda2=LAM2, op_norm=op_norm,
                          power_iters=power_iters)
    res = dr.cp_solve_slabs(plan, _host(g, prec), u, prm, slab)
    return _to_f64(u, prec), res


@pytest.mark.parametrize("prec", [dr.F32, dr.F64, dr.BF16])
@pytest.mark.parametrize("slab", [1, 2, 3, 7, 10])
def test_slabs_equal_incore_bitwise(prec, slab):
    theta, t, g = _problem()
    if prec == dr.BF16:
        g = torch.from_numpy(g).to(torch.bfloat16).to(torch.float64).numpy()
    variants = [dr.DIRECT] if prec == dr.F64 else [dr.DIRECT, dr.FOLD]
    for v in variants:
        u_in, r_in = _incore(theta, t, g, prec, 6, v)
        u_sl, r_sl = _slabs(theta, t, g, prec, 6, v, slab, op_norm=r_in["op_norm"])
        np.testing.assert_array_equal(u_sl, u_in)
        assert rel(r_sl["objective"], r_in["objective"]) <= 1e-12
        assert r_sl["op_norm"] == r_in["op_norm"]


def test_slabs_f64_match_oracle_with_streamed_power_iteration():
    theta, t, g = _problem(seed=1, nz=5)
    P = oracle.Problem(N, N, 5, N, theta, t, oracle.FOURIER, M, NT)
    L = P.power_norm(LAM2)
    uo, oo = P.chambolle_pock(g, np.zeros((5, N, N, M)), 8, LAM1, LAM2, L=L)
    u, res = _slabs(theta, t, g, dr.F64, 8, None, 2, nz=5)
    assert abs(res["op_norm"] - L) <= 1e-10 * L
    assert rel(u, uo) <= 1e-9
    assert rel(res["objective"], oo) <= 1e-10


@pytest.mark.parametrize("slab", [1, 3])
def test_slabs_power_norm_equals_incore(slab):
    theta, t, g = _problem(seed=2)
    _, r_in = _incore(theta, t, g, dr.F32, 1, dr.FOLD)
    _, r_sl = _slabs(theta, t, g, dr.F32, 1, dr.FOLD, slab)
    assert abs(r_sl["op_norm"] - r_in["op_norm"]) <= 1e-5 * r_in["op_norm"]


def test_slabs_device_bytes_grow_with_slab():
    theta, t, _ = _problem()
    plan = dr.Plan(N, N, NZ, N, theta, t, dr.FOURIER, M, NT, dr.F32)
    prm = dr.solve_params(dr.CHAMBOLLE_POCK, iters=4, lambda1=LAM1, lambda2=LAM2)
    b1 = dr.cp_solve_slabs_device_bytes(plan, 1, prm)
    b3 = dr.cp_solve_slabs_device_bytes(plan, 3, prm)
    assert 0 < b1 < b3


def test_slabs_reject_bad_arguments():
    theta, t, g = _problem()
    plan = dr.Plan(N, N, NZ, N, theta, t, dr.FOURIER, M, NT, dr.F32)
    u = np.zeros(plan.u_shape(), dtype=np.float32)
    gh = g.astype(np.float32)
    with pytest.raises(dr.DynreconError) as err:
        dr.cp_solve_slabs(plan, gh, u, dr.solve_params(dr.ADMM_CG, iters=2), 2)
    assert err.value.status == dr.DR_EINVAL
    with pytest.raises(dr.DynreconError):
        dr.cp_solve_slabs(plan, gh, u, dr.solve_params(dr.CHAMBOLLE_POCK, iters=2), 0)
    gd = torch.from_numpy(gh).cuda()
    with pytest.raises(dr.DynreconError):
        dr.cp_solve_slabs(plan, gd, u, dr.solve_params(dr.CHAMBOLLE_POCK, iters=2), 2)


def test_slabs_nonfinite_data():
    theta, t, g = _problem()
    g = g.astype(np.float32)
    g[3, 10, 5] = np.inf
    plan = dr.Plan(N, N, NZ, N, theta, t, dr.FOURIER, M, NT, dr.F32)
    u = np.zeros(plan.u_shape(), dtype=np.float32)
    with pytest.raises(dr.DynreconError) as err:
        dr.cp_solve_slabs(plan, g, u, dr.solve_params(dr.CHAMBOLLE_POCK, iters=3, op_norm=50.0), 2)
    assert err.value.status == dr.DR_ENOTCONV


def test_server_streams_cp_job_over_budget():
    """A Chambolle-Pock job whose whole-volume state exceeds the budget is
    admitted in slabs (the thickest that fit) and gives the result of
    cp_solve_slabs with that slab thickness; an ADMM job of the same size is
    refused."""
    theta, t, g = _problem(seed=3)
    g32 = g.astype(np.float32)
    prm = dr.solve_params(dr.CHAMBOLLE_POCK, iters=4, lambda1=LAM1, lambda2=LAM2, op_norm=60.0)
    u = np.zeros((NZ, N, N, M), dtype=np.float32)
    desc = dr.job_desc(N, N, NZ, N, theta, t, dr.FOURIER, M, NT, dr.F32, prm, g32, u)
    full = dr.job_device_bytes(desc)
    slab = max(s for s in range(1, NZ) if dr.job_slab_device_bytes(desc, s) < full)
    budget = dr.job_slab_device_bytes(desc, slab) + 1
    assert dr.job_slab_device_bytes(desc, slab + 1) > budget
    srv = dr.Server(device=0, budget_bytes=budget, slots=2)
    jid = srv.submit(desc)
    r = srv.wait(jid, timeout_s=300.0)
    with pytest.raises(dr.DynreconError) as err:
        srv.submit(dr.job_desc(N, N, NZ, N, theta, t, dr.FOURIER, M, NT, dr.F32,
                               dr.solve_params(dr.ADMM_CG, iters=2), g32, np.zeros_like(u)))
    assert err.value.status == dr.DR_ENOMEM
    srv.close()
    assert r["rc"] == dr.DR_OK and r["state"] == dr.JOB_DONE, r
    assert r["slab_nz"] == slab and r["device_bytes"] <= budget
    u_ref, _ = _slabs(theta, t, g32.astype(np.float64), dr.F32, 4, None, slab, op_norm=60.0)
    np.testing.assert_array_equal(u.astype(np.float64), u_ref)
