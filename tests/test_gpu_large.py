"""The large mixed-precision volume at full size: 64 slices of 1024^2, 1024
bins, K = 6000 projections over 20 half-turns, m = 16 Legendre -- the
benchmark's workload, on plans autotuned exactly as the benchmark's solver
tunes them (the variants and launch configurations it then runs).  The
oracle cannot process the whole volume in seconds, so the GPU outputs are
checked on samples it can compute one by one: the forward on 12 projections
of 2 slices (each projection's oracle value depends only on u of its slice),
the adjoint on one slice with all 6000 projections (data zero on the other
slices, whose output must then be exactly zero).  FP32 storage must meet
1e-5 (relative L2 and every element against the largest); BF16 storage with
FP32 accumulation is checked against the oracle fed the same bf16-rounded
inputs (1e-3 after the same rounding of the output, 2^-8 end to end)."""
import numpy as np
import pytest

import oracle
from paper_1809_09725_gb300 import dynrecon as dr
from paper_1809_09725_gb300 import synth

from _common import assert_close, host_values, to_bf16_f64

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

W = synth.WORKLOADS["ellipsoids1024"]
SLICES = [5, 41]
ADJ_SLICE = 41
PROJ = [0, 1, 299, 300, 1234, 2999, 3000, 3001, 4500, 5555, 5998, 5999]


@pytest.fixture(scope="module", params=[dr.F32, dr.BF16], ids=["f32", "bf16"])
def tuned_plan(request):
    theta, t = W.geometry()
    plan = dr.Plan(W.N, W.N, W.nz, W.ns, theta, t, W.basis, W.m, W.nt, request.param)
    plan.autotune()
    info = plan.info()
    assert info["tuned"] == 1 and info["unique_angles"] == 300 and info["max_group"] == 20
    # the fold pays on this geometry (20 projections per distinct angle)
    assert info["fwd_variant"] in (dr.FOLD, dr.FOLD2) and info["adj_variant"] == dr.FOLD
    yield request.param, plan, theta, t
    plan.close()
    torch.cuda.empty_cache()


def _sample_fwd(u_full, theta, t, k_idx):
    """Oracle forward restricted to selected projections and slices."""
    Phi = oracle.basis_table(W.basis, W.m, t[k_idx])
    out = []
    for z in SLICES:
        out.append(oracle.dyn_fwd(u_full[z:z + 1], theta[k_idx], Phi, W.ns)[0])
    return np.stack(out)


def test_large_volume_forward_samples(tuned_plan):
    prec, plan, theta, t = tuned_plan
    sd = getattr(torch, plan.storage_dtype)
    u = torch.randn((W.nz, W.N, W.N, W.m), generator=torch.Generator().manual_seed(7), dtype=torch.float32)
    u = u.to(sd).cuda()
    g = torch.empty(plan.g_shape(), dtype=sd, device="cuda")
    dr.dyn_radon_fwd(plan, u, g)
    plan.sync()
    u_sl = np.zeros((W.nz, W.N, W.N, W.m))
    for z in SLICES:
        u_sl[z] = host_values(u[z])
    ref = _sample_fwd(u_sl, theta, t, np.array(PROJ))
    got = np.stack([host_values(g[z][PROJ]) for z in SLICES])
    del u, g
    if prec == dr.F32:
        assert_close(got, ref, 1e-5)
    else:
        assert_close(got, to_bf16_f64(ref), 1e-3)
        assert_close(got, ref, 2.0 ** -8)


def test_large_volume_adjoint_slice(tuned_plan):
    prec, plan, theta, t = tuned_plan
    sd = getattr(torch, plan.storage_dtype)
    rng = synth.rng_for(1025)
    gz = rng.standard_normal((1, W.K, W.ns))
    gz = gz.astype(np.float32).astype(np.float64) if prec == dr.F32 else to_bf16_f64(gz)
    g = torch.zeros(plan.g_shape(), dtype=sd, device="cuda")
    g[ADJ_SLICE] = torch.from_numpy(gz[0]).to(sd).cuda()
    u = torch.full(plan.u_shape(), float("nan"), dtype=sd, device="cuda")
    dr.dyn_radon_adj(plan, g, u)
    plan.sync()
    got = host_values(u[ADJ_SLICE])
    others = [host_values(u[z]) for z in (0, ADJ_SLICE - 1, ADJ_SLICE + 1, W.nz - 1)]
    del u, g
    P = oracle.Problem(W.N, W.N, 1, W.ns, theta, t, W.basis, W.m, W.nt)
    ref = P.adj(gz)[0]
    for o in others:
        assert np.all(o == 0.0)
    if prec == dr.F32:
        assert_close(got, ref, 1e-5)
    else:
        assert_close(got, to_bf16_f64(ref), 1e-3)
        assert_close(got, ref, 2.0 ** -8)
