"""The large mixed-precision volume at full size: 64 slices of 1024^2, 1024
bins, K = 6000 projections over 20 half-turns, m = 16 Legendre.  The oracle
cannot process the whole volume in seconds, so the GPU outputs are checked
on samples it can compute one by one: the forward on 12 projections of 2
slices (each projection's oracle value depends only on u of its slice), the
adjoint on a 1-slice sub-volume with all 6000 projections.  FP32 storage
must meet 1e-5; BF16 storage with FP32 accumulation is checked against the
oracle fed the same bf16-rounded inputs (1e-3 after the same rounding of the
output, 2^-8 end to end)."""
import numpy as np
import pytest

import oracle
from paper_1809_09725_gb300 import dynrecon as dr
from paper_1809_09725_gb300 import synth

from _common import dev_tensor, host_values, rel, to_bf16_f64

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

W = synth.WORKLOADS["ellipsoids1024"]
SLICES = [5, 41]
PROJ = [0, 1, 299, 300, 1234, 2999, 3000, 3001, 4500, 5555, 5998, 5999]


def _sample_fwd(u_full, theta, t, k_idx):
    """Oracle forward restricted to selected projections and slices."""
    Phi = oracle.basis_table(W.basis, W.m, t[k_idx])
    out = []
    for z in SLICES:
        out.append(oracle.dyn_fwd(u_full[z:z + 1], theta[k_idx], Phi, W.ns)[0])
    return np.stack(out)


@pytest.mark.parametrize("prec", [dr.F32, dr.BF16])
def test_large_volume_forward_samples(prec):
    theta, t = W.geometry()
    plan = dr.Plan(W.N, W.N, W.nz, W.ns, theta, t, W.basis, W.m, W.nt, prec)
    u = torch.randn((W.nz, W.N, W.N, W.m), generator=torch.Generator().manual_seed(7), dtype=torch.float32)
    u = u.to(getattr(torch, plan.storage_dtype)).cuda()
    g = torch.empty(plan.g_shape(), dtype=getattr(torch, plan.storage_dtype), device="cuda")
    dr.dyn_radon_fwd(plan, u, g)
    plan.sync()
    u_sl = np.zeros((W.nz, W.N, W.N, W.m))
    for z in SLICES:
        u_sl[z] = host_values(u[z])
    ref = _sample_fwd(u_sl, theta, t, np.array(PROJ))
    got = np.stack([host_values(g[z][PROJ]) for z in SLICES])
    if prec == dr.F32:
        assert rel(got, ref) <= 1e-5
    else:
        assert rel(got, to_bf16_f64(ref)) <= 1e-3
        assert rel(got, ref) <= 2.0 ** -8


@pytest.mark.parametrize("prec", [dr.F32, dr.BF16])
def test_large_volume_adjoint_subvolume(prec):
    theta, t = W.geometry()
    nz = 1
    plan = dr.Plan(W.N, W.N, nz, W.ns, theta, t, W.basis, W.m, W.nt, prec)
    rng = synth.rng_for(1025)
    g = rng.standard_normal((nz, W.K, W.ns))
    if prec == dr.F32:
        g = g.astype(np.float32).astype(np.float64)
    else:
        g = to_bf16_f64(g)
    u = torch.empty(plan.u_shape(), dtype=getattr(torch, plan.storage_dtype), device="cuda")
    dr.dyn_radon_adj(plan, dev_tensor(g, prec), u)
    plan.sync()
    P = oracle.Problem(W.N, W.N, nz, W.ns, theta, t, W.basis, W.m, W.nt)
    ref = P.adj(g)
    got = host_values(u)
    if prec == dr.F32:
        assert rel(got, ref) <= 1e-5
    else:
        assert rel(got, to_bf16_f64(ref)) <= 1e-3
        assert rel(got, ref) <= 2.0 ** -8
