"""The C-ABI library builds for sm_103a and exports every symbol include/eot.h declares
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "eot.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(eot_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2504_02067_gb300 import buildlib
    return buildlib.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("eot_create", "eot_destroy", "eot_marginals", "eot_hvp", "eot_newton_solve",
              "eot_solve", "eot_backward", "eot_params_default", "eot_status_string"):
        assert f in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (eot_[a-z_0-9]+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing


def test_library_loads_and_binding_matches(libpath):
    from paper_2504_02067_gb300 import binding
    L = binding.load_library(libpath)
    for f in declared_functions():
        assert hasattr(L, f)
    for f in binding.EXPORTS:
        assert f in declared_functions()
    # pure host calls (no device work)
    p = L.eot_params_default()
    assert p.gamma_i == 16.0 and p.gamma_f == 4096.0 and p.p == 1.5 and p.w_r == 0.45
    assert L.eot_status_string(3) == b"EOT_ERR_CG_MAXITER"
    assert ctypes.sizeof(binding.EotProblem) == 88
    assert ctypes.sizeof(binding.EotParams) == 72
    assert ctypes.sizeof(binding.EotStats) == 112
