"""The C ABI library builds, loads and exports every entry point that
include/dynrecon.h declares (no compute calls: runs without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dynrecon.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1809_09725_gb300 import dynrecon
    return dynrecon.load()


def test_header_lists_the_entry_points():
    names = _declared()
    for n in ("dyn_radon_fwd", "dyn_radon_adj", "tv4d_prox", "admm_solve", "dr_plan_create"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1809_09725_gb300 import dynrecon
    for name in _declared():
        assert hasattr(lib, name), name
    assert sorted(dynrecon.EXPORTS) == _declared()


def test_version_string(lib):
    assert lib.dr_version().decode().startswith("dynrecon")


def test_oracle_and_library_share_no_code():
    """The oracle is plain C in oracle/, the product is CUDA in the package:
    neither includes or imports the other."""
    osrc = open(os.path.join(ROOT, "oracle", "dynrecon_oracle.c")).read()
    assert "#include \"" not in osrc
    csrc = os.path.join(ROOT, "paper_1809_09725_gb300", "csrc")
    for f in os.listdir(csrc):
        assert "oracle" not in open(os.path.join(csrc, f)).read().lower(), f
    for f in ("dynrecon.py", "__init__.py", "build.py"):
        txt = open(os.path.join(ROOT, "paper_1809_09725_gb300", f)).read()
        assert "import oracle" not in txt and "from oracle" not in txt, f


def test_job_admission_estimate_is_host_only_and_monotone(lib):
    """dr_job_device_bytes is plain host arithmetic (callable without a GPU):
    it grows with the volume, the projection count and the precision."""
    import numpy as np
    from paper_1809_09725_gb300 import dynrecon as dr

    def est(nz=2, K=100, prec=dr.F32, algo=dr.ADMM_CG, N=64, m=4):
        theta = np.linspace(0, 3, K)
        t = np.linspace(0, 0.99, K)
        dt = np.float64 if prec == dr.F64 else np.float32
        g = np.zeros((nz, K, N), dtype=dt)
        u = np.zeros((nz, N, N, m), dtype=dt)
        prm = dr.SolveParams()
        lib.dr_solve_params_default(prm)
        prm.algo = algo
        return dr.job_device_bytes(dr.job_desc(N, N, nz, N, theta, t, dr.FOURIER, m, 4, prec, prm, g, u))

    base = est()
    assert base > 0
    assert est(nz=4) > 1.8 * base - 4 * (1 << 20)
    assert est(K=400) > est(K=100)
    assert est(prec=dr.F64) > base
    assert est(m=16) > base
    # a 16 x 256^2, 1800-projection, m = 8 job needs well under 2 GB
    assert est(nz=16, K=1800, N=256, m=8) < 2 * 1024 ** 3


def test_slab_estimate_lets_the_largest_serving_job_fit(lib):
    """The largest job of the serving mix (2048^2 x 128 slices, K = 7200,
    m = 32, 20 frames, BF16) needs several hundred GB with its whole volume on
    the device, but streamed in slabs it fits a 150 GB budget; the slab
    estimate grows with the slab thickness (host arithmetic only)."""
    import numpy as np
    from paper_1809_09725_gb300 import dynrecon as dr

    K = 7200
    theta = np.linspace(0.0, 20 * np.pi, K, endpoint=False)
    t = np.arange(K) / K
    prm = dr.SolveParams()
    lib.dr_solve_params_default(prm)
    prm.algo, prm.iters = dr.CHAMBOLLE_POCK, 30
    d = dr.JobDesc()
    d.nx = d.ny = d.ns = 2048
    d.nz, d.K, d.m, d.nt, d.prec, d.basis = 128, K, 32, 20, dr.BF16, dr.FOURIER
    d.params = prm
    budget = 150 * 10 ** 9
    assert dr.job_device_bytes(d) > 3 * budget
    sizes = [dr.job_slab_device_bytes(d, s) for s in (1, 2, 4, 8, 16)]
    assert all(a < b for a, b in zip(sizes, sizes[1:]))
    assert sizes[3] < budget  # slabs of 8 slices


def test_host_side_argument_checks_without_a_gpu(lib):
    """Entry points reject missing arguments on the host, before any CUDA
    call: a NULL plan, a resume request without a state buffer; the solver
    defaults keep checkpointing off."""
    import ctypes
    from paper_1809_09725_gb300 import dynrecon as dr
    assert lib.dr_plan_state_bytes(None, dr.ADMM_CG) == 0
    assert lib.dr_plan_wait_selftest(None, 0.1) == dr.DR_EINVAL
    assert lib.tv4d_normal(None, None, None, 1.0, 0.0) == dr.DR_EINVAL
    p = dr.SolveParams()
    lib.dr_solve_params_default(ctypes.byref(p))
    assert not p.state and p.resume == 0
    assert (p.algo, p.iters, p.n_cg) == (dr.ADMM_CG, 20, 4)
    assert lib.admm_solve(None, None, None, ctypes.byref(p)) == dr.DR_EINVAL
    assert "NULL" in lib.dr_last_error().decode()
