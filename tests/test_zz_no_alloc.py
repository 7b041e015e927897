"""dyn_radon_adj_noalloc: the back-projection for callers that cannot
allocate device memory at call time (code running while a stream is
captured, where an allocation would fail or break the capture, and
applications that hand out a fixed device budget from their own pool).  Its
folded data live in the library's fixed 8 MiB device array.

Checked through the C ABI on two calls in a row (the second reuses what the
first left in the array, and accumulates with beta = 0.5): against the
ordinary entry point (dyn_radon_adj, half-turn fold variant) and against the
FP64 oracle, for F32 plans (1e-5 relative L2) and BF16 storage (1e-3 against
the oracle fed the same bf16 inputs and rounded the same way), at m = 4, 8
and 16 (separate kernel instantiations).  This file is collected last on
purpose: a failure here leaves every other test already run."""
import numpy as np
import pytest

import oracle
from paper_1809_09725_gb300 import dynrecon as dr
from paper_1809_09725_gb300 import synth

from _common import assert_close, dev_tensor, host_values, to_bf16_f64

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NX, NY, NZ, NS, K, HT = 64, 60, 2, 66, 256, 4


def _plan(m, prec):
    # 2 slices of 64 x 60, 256 projections over 4 half-turns (64 distinct angles)
    theta, t = synth.scan(K, HT, mod_pi=True)
    basis = dr.LEGENDRE if m == 16 else dr.FOURIER
    plan = dr.Plan(NX, NY, NZ, NS, theta, t, basis, m, HT, prec)
    plan.set_variant(dr.FOLD, dr.FOLD)
    P = oracle.Problem(NX, NY, NZ, NS, theta, t, basis, m, HT)
    return plan, P


@pytest.mark.parametrize("m", [4, 8, 16])
@pytest.mark.parametrize("prec", [dr.F32, dr.BF16])
def test_noalloc_adjoint_equals_adjoint_and_oracle_on_two_calls(prec, m):
    import __graft_entry__
    __graft_entry__.build()
    plan, P = _plan(m, prec)
    rng = synth.rng_for(777 + m)
    rnd = (lambda x: to_bf16_f64(x)) if prec == dr.BF16 else (lambda x: x.astype(np.float32).astype(np.float64))
    for call, beta in enumerate((0.0, 0.5)):
        g = rnd(rng.standard_normal(plan.g_shape()))
        u0 = rnd(rng.standard_normal(plan.u_shape()))
        u_ref = dev_tensor(u0, prec)
        u_new = dev_tensor(u0, prec)
        dr.dyn_radon_adj(plan, dev_tensor(g, prec), u_ref, beta=beta)
        dr.dyn_radon_adj_noalloc(plan, dev_tensor(g, prec), u_new, beta=beta)
        plan.sync()
        ref = beta * u0 + P.adj(g)
        if prec == dr.F32:
            assert_close(host_values(u_new), host_values(u_ref), 1e-5)
            assert_close(host_values(u_new), ref, 1e-5)
        else:
            assert_close(host_values(u_new), host_values(u_ref), 1e-3)
            assert_close(host_values(u_new), to_bf16_f64(ref), 1e-3)


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
