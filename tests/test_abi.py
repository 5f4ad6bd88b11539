"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/flexrt.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re
import subprocess

import paper_2409_04521_gb300 as F

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "flexrt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(flexrt_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("flexrt_create", "flexrt_add_sources", "flexrt_step", "flexrt_get_fields",
                     "flexrt_get_budget", "flexrt_destroy", "flexrt_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    path = F.library_path()
    F.lib()  # builds if needed and loads
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    L = ctypes.CDLL(path)
    for n in declared_functions():
        assert hasattr(L, n)


def test_invalid_arguments_rejected_without_gpu_work():
    L = F.lib()
    assert L.flexrt_create(None, None, None, None, None, None, None) != 0
    assert L.flexrt_step(None, 1.0) != 0
    assert L.flexrt_get_budget(None, None) != 0


def test_default_options():
    o = F.default_options()
    assert o.l_max == 12 and o.n_ray_min == 3.0 and o.eps_term == 1e-10 and o.chem_iters == 5
