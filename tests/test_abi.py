"""The C-ABI library builds, loads and exports every symbol include/ddp.h declares
(no compute calls: these run without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ddp():
    from paper_1601_04587_gb300 import build
    build.build()
    import paper_1601_04587_gb300 as m
    return m


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "ddp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ddp_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary_calls():
    names = declared_symbols()
    for required in ["ddp_load_gauge", "ddp_set_domain", "ddp_solve_propagator", "ddp_series_terms",
                     "ddp_contract", "ddp_solve_batch", "ddp_submit", "ddp_poll"]:
        assert required in names


def test_library_exports_every_declared_symbol(ddp):
    lib = ddp.lib()
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_error_strings(ddp):
    assert ddp.error_string(ddp.DDP_OK) == "ok"
    assert "converge" in ddp.error_string(ddp.DDP_ERR_NOT_CONVERGED)
    assert ddp.error_string(99) == "unknown status"


def test_create_rejects_missing_device(ddp):
    # without a GPU (or with an out-of-range ordinal) creation fails cleanly
    with pytest.raises(ddp.DDPError):
        ddp.ddp_create(1 << 20)


def test_binding_has_no_cpu_fallback():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_1601_04587_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "liboracle" not in src, f
