"""dyn_radon_adj_noalloc: the back-projection for callers that may not
allocate device memory (inside a stream capture, or under a no-allocation
policy), with its folded data in the library's fixed 8 MiB device array.

Its output must equal the ordinary entry point's (dyn_radon_adj, half-turn
fold variant) within the FP32 operator tolerance used elsewhere (1e-5
relative L2), on two calls in a row: the second call reuses the array the
first one left behind.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1809_09725_gb300 import dynrecon as dr
from paper_1809_09725_gb300 import synth

from _common import dev_tensor, host_values, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _plan_and_data():
    # 2 slices of 64^2, 256 projections over 4 half-turns (64 distinct angles), m = 8
    theta, t = synth.scan(256, 4, mod_pi=True)
    plan = dr.Plan(64, 64, 2, 64, theta, t, dr.FOURIER, 8, 4, dr.F32)
    plan.set_variant(dr.FOLD, dr.FOLD)
    return plan


def test_noalloc_adjoint_equals_adjoint_on_two_calls():
    import __graft_entry__
    __graft_entry__.build()
    plan = _plan_and_data()
    rng = synth.rng_for(777)
    for call, beta in enumerate((0.0, 0.5)):
        g = dev_tensor(rng.standard_normal(plan.g_shape()), dr.F32)
        u0 = rng.standard_normal(plan.u_shape())
        u_ref = dev_tensor(u0, dr.F32)
        u_new = dev_tensor(u0, dr.F32)
        dr.dyn_radon_adj(plan, g, u_ref, beta=beta)
        dr.dyn_radon_adj_noalloc(plan, g, u_new, beta=beta)
        plan.sync()
        assert rel(host_values(u_new), host_values(u_ref)) <= 1e-5, call


def test_noalloc_rejects_problems_larger_than_its_array():
    # 16 slices of 256^2, 180 distinct angles, m = 8: 35 MB of folded data > 8 MiB
    w = synth.WORKLOADS["ellipsoids256"]
    theta, t = w.geometry()
    plan = dr.Plan(w.N, w.N, w.nz, w.ns, theta, t, w.basis, w.m, w.nt, dr.F32)
    g = torch.zeros(plan.g_shape(), dtype=torch.float32, device="cuda")
    u = torch.zeros(plan.u_shape(), dtype=torch.float32, device="cuda")
    with pytest.raises(dr.DynreconError) as err:
        dr.dyn_radon_adj_noalloc(plan, g, u)
    assert "8388608" in str(err.value)
