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
