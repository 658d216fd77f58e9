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
              "eot_solve", "eot_backward", "eot_params_default", "eot_status_string", "eot_value",
              "eot_plan_argmax", "eot_plan_support", "eot_solve_batched", "eot_round"):
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
    for code, name in binding.STATUS_NAMES.items():
        assert L.eot_status_string(code) == name.encode()
    assert ctypes.sizeof(binding.EotProblem) == 88
    assert ctypes.sizeof(binding.EotParams) == 88
    assert ctypes.sizeof(binding.EotStats) == 136


def test_struct_layouts_match_the_header(tmp_path):
    """Every field offset of the ctypes structures equals the C compiler's offsetof
    for the structures of include/eot.h (the binding marshals them by layout)."""
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    from paper_2504_02067_gb300 import binding
    structs = {"eot_problem": binding.EotProblem, "eot_params": binding.EotParams,
               "eot_stats": binding.EotStats, "eot_stage_record": binding.EotStageRecord}
    lines = []
    for cname, cls in structs.items():
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in cls._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "eot.h"\nint main(void) {\n'
                   + "\n".join(lines) + "\n  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        parts = line.split()
        if len(parts) == 3:
            got[(parts[0], parts[1])] = int(parts[2])
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_status_codes_match_the_header(tmp_path):
    """The binding's status names carry the header's enum values, including the
    bounded-device-wait status EOT_ERR_DEVICE_TIMEOUT."""
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    from paper_2504_02067_gb300 import binding
    src = tmp_path / "codes.c"
    src.write_text('#include <stdio.h>\n#include "eot.h"\nint main(void) {\n'
                   + "\n".join('  printf("%s %%d\\n", (int)%s);' % (nm, nm)
                               for nm in binding.STATUS_NAMES.values())
                   + "\n  return 0;\n}\n")
    exe = tmp_path / "codes"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = {out[k]: int(out[k + 1]) for k in range(0, len(out), 2)}
    for code, name in binding.STATUS_NAMES.items():
        assert got[name] == code
    assert got["EOT_ERR_DEVICE_TIMEOUT"] == 10
