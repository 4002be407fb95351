"""The C ABI library builds for sm_103a, loads, and exports every function
declared in include/lbm.h (no compute call: this runs without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2503_07898_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("lbm_grid_create_dense", "lbm_grid_create_sparse", "lbm_set_boundary",
                 "lbm_init_equilibrium", "lbm_step", "lbm_get_moments", "lbm_conservation"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(lbm_[a-z0-9_]+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_loads_and_binds_every_symbol(libpath):
    from paper_2503_07898_gb300 import binding
    lib = binding.load()
    for n in declared_functions():
        assert hasattr(lib, n)
    assert binding.lbm_last_error() == ""
