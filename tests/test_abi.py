"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every entry point declared in include/amg.h (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2006_16147_gb300 import build
    return build.build()


def _declared():
    txt = open(os.path.join(ROOT, "include", "amg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(amg_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_boundary():
    names = _declared()
    for must in ("amg_setup", "amg_solve", "amg_free", "amg_vcycle", "amg_hierarchy_info"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (amg_\w+)", out))
    assert set(_declared()) <= exported


def test_binding_names_match_header():
    from paper_2006_16147_gb300 import amg
    assert set(amg.EXPORTED) <= set(_declared())


def test_no_gpu_calls_needed_for_options(libpath):
    from paper_2006_16147_gb300 import amg
    o = amg.amg_options_default()
    assert (o.sweeps, o.max_coarse, o.pre, o.post, o.omega, o.precision) == (3, 200, 1, 1, 1.0, 0)


def test_struct_layouts_match_c():
    # compile a tiny C probe of the header's struct sizes and offsets on the host
    from paper_2006_16147_gb300 import amg
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "amg.h"
int main(void){
 printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(amg_csr), sizeof(amg_options), offsetof(amg_options, omega),
        offsetof(amg_options, stream), sizeof(amg_solve_info), sizeof(amg_hier_info),
        offsetof(amg_options, keep_sweeps), offsetof(amg_options, profile), offsetof(amg_hier_info, opc),
        offsetof(amg_options, min_ratio), offsetof(amg_hier_info, device_bytes));
 return 0;}
'''
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "probe")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        got = [int(v) for v in subprocess.check_output([exe]).split()]
    want = [ctypes.sizeof(amg.amg_csr), ctypes.sizeof(amg.amg_options), amg.amg_options.omega.offset,
            amg.amg_options.stream.offset, ctypes.sizeof(amg.amg_solve_info), ctypes.sizeof(amg.amg_hier_info),
            amg.amg_options.keep_sweeps.offset, amg.amg_options.profile.offset, amg.amg_hier_info.opc.offset,
            amg.amg_options.min_ratio.offset, amg.amg_hier_info.device_bytes.offset]
    assert got == want
