"""Batched uneven jobs and the serving loop.

* admm_solve_batch: jobs of different grids, slices, projection counts,
  bases, m, precision and iteration counts in one CUDA graph per iteration;
  each result must be bit-for-bit the result of solving the job alone.
* Server: jobs admitted under a device-memory budget, running concurrently;
  each result equals the job alone; a job larger than the budget is refused;
  queued jobs can be cancelled; non-finite data make the job fail cleanly.
"""
import numpy as np
import pytest

from paper_1809_09725_gb300 import dynrecon as dr
from paper_1809_09725_gb300 import synth

from _common import dev_tensor, host_values

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# N, nz, K, half-turns, basis, m, nt, prec, iters
JOBS = [
    (48, 2, 120, 4.0, dr.FOURIER, 4, 4, dr.F32, 4),
    (64, 1, 200, 5.0, dr.LEGENDRE, 8, 5, dr.F32, 6),
    (32, 3, 90, 3.0, dr.FOURIER, 3, 3, dr.BF16, 3),
    (40, 2, 160, 8.0, dr.FOURIER, 16, 8, dr.F32, 5),
]


def _job_inputs(i, spec):
    N, nz, K, ht, basis, m, nt, prec, iters = spec
    theta, t = synth.scan(K, ht)
    rng = synth.rng_for(9000 + i)
    g = rng.standard_normal((nz, K, N)) * 3.0
    return theta, t, g


def _params(spec, algo=dr.ADMM_CG):
    return dr.solve_params(algo, iters=spec[8], n_cg=3, lambda1=0.05, lambda2=1.0, rho=0.5)


def _alone(i, spec, algo=dr.ADMM_CG):
    N, nz, K, ht, basis, m, nt, prec, iters = spec
    theta, t, g = _job_inputs(i, spec)
    plan = dr.Plan(N, N, nz, N, theta, t, basis, m, nt, prec)
    u = torch.zeros(plan.u_shape(), dtype=getattr(torch, plan.storage_dtype), device="cuda")
    dr.admm_solve(plan, dev_tensor(g, prec), u, _params(spec, algo))
    return host_values(u)


@pytest.mark.parametrize("algo", [dr.ADMM_CG, dr.CHAMBOLLE_POCK])
def test_batch_equals_each_job_alone(algo):
    alone = [_alone(i, s, algo) for i, s in enumerate(JOBS)]
    plans, gs, us, prms = [], [], [], []
    for i, spec in enumerate(JOBS):
        N, nz, K, ht, basis, m, nt, prec, iters = spec
        theta, t, g = _job_inputs(i, spec)
        p = dr.Plan(N, N, nz, N, theta, t, basis, m, nt, prec)
        plans.append(p)
        gs.append(dev_tensor(g, prec))
        us.append(torch.zeros(p.u_shape(), dtype=getattr(torch, p.storage_dtype), device="cuda"))
        prms.append(_params(spec, algo))
    dr.admm_solve_batch(plans, gs, us, prms)
    for i in range(len(JOBS)):
        np.testing.assert_array_equal(host_values(us[i]), alone[i])


def test_batch_rejects_duplicate_plans():
    spec = JOBS[0]
    theta, t, g = _job_inputs(0, spec)
    p = dr.Plan(spec[0], spec[0], spec[1], spec[0], theta, t, spec[4], spec[5], spec[6], spec[7])
    g1 = dev_tensor(g, spec[7])
    u1 = torch.zeros(p.u_shape(), dtype=torch.float32, device="cuda")
    with pytest.raises(dr.DynreconError):
        dr.admm_solve_batch([p, p], [g1, g1], [u1, u1], [_params(spec), _params(spec)])


def _descs():
    descs, outs = [], []
    for i, spec in enumerate(JOBS):
        N, nz, K, ht, basis, m, nt, prec, iters = spec
        theta, t, g = _job_inputs(i, spec)
        if prec == dr.BF16:
            gh = torch.from_numpy(g).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
            uh = np.zeros((nz, N, N, m), dtype=np.uint16)
        else:
            gh = g.astype(np.float32)
            uh = np.zeros((nz, N, N, m), dtype=np.float32)
        descs.append(dr.job_desc(N, N, nz, N, theta, t, basis, m, nt, prec, _params(spec), gh, uh))
        outs.append(uh)
    return descs, outs


def _host_to_f64(arr, prec):
    if prec == dr.BF16:
        return torch.from_numpy(arr.view(np.int16)).view(torch.bfloat16).to(torch.float64).numpy()
    return arr.astype(np.float64)


def test_server_runs_jobs_concurrently_with_alone_results():
    alone = [_alone(i, s) for i, s in enumerate(JOBS)]
    descs, outs = _descs()
    budget = sum(dr.job_device_bytes(d) for d in descs[:2]) + 1
    srv = dr.Server(device=0, budget_bytes=budget, slots=3)
    ids = [srv.submit(d) for d in descs]
    res = [srv.wait(j, timeout_s=300.0) for j in ids]
    st = srv.stats()
    srv.close()
    for i, r in enumerate(res):
        assert r["rc"] == dr.DR_OK and r["state"] == dr.JOB_DONE, r
        np.testing.assert_array_equal(_host_to_f64(outs[i], JOBS[i][7]), alone[i])
    assert st["completed"] == len(JOBS) and st["failed"] == 0
    assert st["peak_device_bytes"] <= budget
    assert st["p99_latency_s"] >= st["p50_latency_s"] > 0.0


def test_server_refuses_job_larger_than_budget():
    descs, _ = _descs()
    srv = dr.Server(device=0, budget_bytes=dr.job_device_bytes(descs[0]) - 1, slots=1)
    with pytest.raises(dr.DynreconError) as err:
        srv.submit(descs[0])
    assert err.value.status == dr.DR_ENOMEM
    srv.close()


def test_server_cancel_and_nonfinite_data():
    descs, outs = _descs()
    srv = dr.Server(device=0, budget_bytes=1 << 34, slots=1)
    first = srv.submit(descs[1])
    second = srv.submit(descs[3])
    srv.cancel(second)
    r2 = srv.wait(second, timeout_s=300.0)
    assert r2["state"] == dr.JOB_CANCELED and r2["rc"] == dr.DR_ECANCELED
    assert srv.wait(first, timeout_s=300.0)["state"] == dr.JOB_DONE
    # NaN in the data: the solve reports non-finite values instead of a result
    N, nz, K, ht, basis, m, nt, prec, iters = JOBS[0]
    theta, t, g = _job_inputs(0, JOBS[0])
    g = g.astype(np.float32)
    g[0, 3, 5] = np.nan
    u = np.zeros((nz, N, N, m), dtype=np.float32)
    bad = srv.submit(dr.job_desc(N, N, nz, N, theta, t, basis, m, nt, prec, _params(JOBS[0]), g, u))
    r = srv.wait(bad, timeout_s=300.0)
    assert r["state"] == dr.JOB_FAILED and r["rc"] == dr.DR_ENOTCONV
    srv.close()


def test_server_cancels_a_running_job_between_iterations():
    """A running job stops within a few iterations of dr_server_cancel and is
    recorded as canceled; the server then runs the next job to its normal
    result (the same as alone)."""
    import time

    N, nz, K, ht, basis, m, nt, prec, iters = JOBS[1]
    theta, t, g = _job_inputs(1, JOBS[1])
    long_prm = dr.solve_params(dr.ADMM_CG, iters=100000, n_cg=4, lambda1=1e-3, lambda2=1.0, rho=1e-2)
    u_long = np.zeros((nz, N, N, m), dtype=np.float32)
    d_long = dr.job_desc(N, N, nz, N, theta, t, basis, m, nt, dr.F32, long_prm, g.astype(np.float32), u_long)
    srv = dr.Server(device=0, budget_bytes=1 << 34, slots=1)
    jid = srv.submit(d_long)
    descs, outs = _descs()
    nxt = srv.submit(descs[0])
    t0 = time.perf_counter()
    while srv.wait(jid, timeout_s=0.05)["rc"] == dr.DR_ETIMEOUT and time.perf_counter() - t0 < 1.0:
        pass
    assert srv.wait(jid, timeout_s=0.0)["rc"] == dr.DR_ETIMEOUT  # still running after 1 s
    t_cancel = time.perf_counter()
    srv.cancel(jid)
    r = srv.wait(jid, timeout_s=120.0)
    t_stop = time.perf_counter() - t_cancel
    assert r["state"] == dr.JOB_CANCELED and r["rc"] == dr.DR_ECANCELED, r
    assert t_stop < 10.0
    r2 = srv.wait(nxt, timeout_s=300.0)
    st = srv.stats()
    srv.close()
    assert r2["rc"] == dr.DR_OK and r2["state"] == dr.JOB_DONE
    np.testing.assert_array_equal(_host_to_f64(outs[0], JOBS[0][7]), _alone(0, JOBS[0]))
    assert st["canceled"] == 1 and st["completed"] == 1 and st["failed"] == 0
    srv2 = dr.Server(device=0, budget_bytes=1 << 30, slots=1)
    with pytest.raises(dr.DynreconError):
        srv2.cancel(12345)  # unknown job
    srv2.close()


def test_concurrent_plans_with_different_shared_memory_sizes():
    """Plans on several threads launch the same kernels with different dynamic
    shared-memory sizes at once (strip heights, grid sizes); every launch must
    succeed and give the single-threaded result."""
    import threading

    cases = [(48, 2), (160, 5), (96, 1), (224, 3)]
    ref = {}
    for N, lines in cases:
        theta, t = synth.scan(90, 3.0)
        plan = dr.Plan(N, N, 2, N, theta, t, dr.FOURIER, 8, 3, dr.F32)
        plan.set_variant(dr.FOLD, dr.FOLD)
        u = torch.from_numpy(synth.rng_for(N).standard_normal((2, N, N, 8))).float().cuda()
        g = torch.zeros(plan.g_shape(), dtype=torch.float32, device="cuda")
        dr.dyn_radon_fwd(plan, u, g)
        plan.sync()
        ref[N] = (plan, u, host_values(g), lines)
    errors = []

    def worker(N):
        try:
            plan, u, g_ref, lines = ref[N]
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                for rep in range(12):
                    plan.set_fold_strip(1 + (rep + lines) % 3, False)
                    g = torch.zeros(plan.g_shape(), dtype=torch.float32, device="cuda")
                    dr.dyn_radon_fwd(plan, u, g)
                    plan.sync()
                    if not np.array_equal(host_values(g), g_ref):
                        errors.append((N, rep, "mismatch"))
        except Exception as exc:  # noqa: BLE001 -- collected and asserted below
            errors.append((N, repr(exc)))

    threads = [threading.Thread(target=worker, args=(N,)) for N, _ in cases]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors


def test_server_job_with_bf16_fields_equals_its_solve_alone():
    """A served job with DR_FIELDS_BF16 is budgeted with half-size dual fields
    and returns the same result as admm_solve alone on a plan with the flag."""
    spec = JOBS[1]
    N, nz, K, ht, basis, m, nt, prec, iters = spec
    theta, t, g = _job_inputs(1, spec)
    flag = dr.F32 | dr.FIELDS_BF16
    plan = dr.Plan(N, N, nz, N, theta, t, basis, m, nt, flag)
    u_alone = torch.zeros(plan.u_shape(), dtype=torch.float32, device="cuda")
    dr.admm_solve(plan, dev_tensor(g, dr.F32), u_alone, _params(spec))
    gh = g.astype(np.float32)
    uh = np.zeros((nz, N, N, m), dtype=np.float32)
    d = dr.job_desc(N, N, nz, N, theta, t, basis, m, nt, flag, _params(spec), gh, uh)
    d32 = dr.job_desc(N, N, nz, N, theta, t, basis, m, nt, dr.F32, _params(spec), gh, np.zeros_like(uh))
    assert dr.job_device_bytes(d32) - dr.job_device_bytes(d) >= 2 * 2 * 4 * nt * N * N * nz
    srv = dr.Server(device=0, budget_bytes=1 << 34, slots=1)
    r = srv.wait(srv.submit(d), timeout_s=300.0)
    srv.close()
    assert r["rc"] == dr.DR_OK and r["state"] == dr.JOB_DONE
    np.testing.assert_array_equal(uh.astype(np.float64), host_values(u_alone))
