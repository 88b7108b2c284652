"""CPU checks of the C ABI boundary (no GPU, no compute calls).

* libdsoa.so builds for sm_103a, loads, and exports every function that
  include/dsoa.h declares.
* The ctypes mirrors of the argument structs in paper_1810_11765_gb300.dsoa have the
  size and field offsets that gcc gives the C declarations of include/dsoa_apps.h.
* Argument validation that happens on the host returns error codes.
"""
import ctypes
import os
import re
import subprocess

import pytest

from conftest import ROOT

INCLUDE = os.path.join(ROOT, "include")


@pytest.fixture(scope="module")
def lib():
    from paper_1810_11765_gb300 import build, dsoa
    build.build()
    return dsoa.load()


def declared_functions():
    names = []
    for h in ("dsoa.h",):
        src = open(os.path.join(INCLUDE, h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:int|const char\*)\s+(dsoa_\w+)\s*\(", src, flags=re.M)
    return names


def test_every_declared_function_is_exported(lib):
    from paper_1810_11765_gb300 import dsoa
    names = declared_functions()
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", dsoa.lib_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (dsoa_\w+)", out))
    assert set(names) <= exported
    assert set(names) == set(dsoa.ABI_FUNCTIONS)


def test_error_strings(lib):
    assert lib.dsoa_error_string(0) == b"ok"
    assert lib.dsoa_error_string(-4) == b"heap too small"


def test_host_side_argument_checks(lib):
    out = ctypes.c_void_p()
    assert lib.dsoa_heap_create(16, None, ctypes.byref(out)) == -1
    assert lib.dsoa_heap_create_from(None, 1 << 20, None, ctypes.byref(out)) == -1
    assert lib.dsoa_register_type(None, None, 0, None) == -1
    assert lib.dsoa_graph_destroy(None) == -1
    assert lib.dsoa_count(None, 0, None) == -1


PROBE = r"""
#include <stdio.h>
#include <stddef.h>
#include "dsoa_apps.h"
#define S(T) printf(#T " size %zu\n", sizeof(T));
#define O(T, f) printf(#T " " #f " %zu\n", offsetof(T, f));
int main(void) {
  S(dsoa_micro_args) O(dsoa_micro_args, round) O(dsoa_micro_args, x_out) O(dsoa_micro_args, stats)
  O(dsoa_micro_args, handles_out)
  S(dsoa_micro_stats) O(dsoa_micro_stats, sum_x)
  S(dsoa_inst) O(dsoa_inst, seed) O(dsoa_inst, t) O(dsoa_inst, state)
  S(dsoa_gol_args) O(dsoa_gol_args, n_inst) O(dsoa_gol_args, alive_type)
  S(dsoa_wator_args) O(dsoa_wator_args, shark_type)
  S(dsoa_traffic_args) O(dsoa_traffic_args, seed) O(dsoa_traffic_args, car_type)
  S(dsoa_nbody_args) O(dsoa_nbody_args, seed) O(dsoa_nbody_args, n_ids) O(dsoa_nbody_args, G)
  O(dsoa_nbody_args, vscale) O(dsoa_nbody_args, body_type) O(dsoa_nbody_args, flags)
  return 0;
}
"""


def test_ctypes_layouts_match_c_headers(tmp_path):
    from paper_1810_11765_gb300 import dsoa as D
    src = tmp_path / "probe.c"
    src.write_text(PROBE)
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c11", "-I" + INCLUDE, str(src), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    py = {"dsoa_micro_args": D.MicroArgs, "dsoa_micro_stats": D.MicroStats, "dsoa_inst": D.Inst,
          "dsoa_gol_args": D.GolArgs, "dsoa_wator_args": D.WatorArgs,
          "dsoa_traffic_args": D.TrafficArgs, "dsoa_nbody_args": D.NBodyArgs}
    n = 0
    for ln in lines:
        if not ln:
            continue
        parts = ln.split()
        cls = py[parts[0]]
        if parts[1] == "size":
            assert ctypes.sizeof(cls) == int(parts[2]), ln
        else:
            assert getattr(cls, parts[1]).offset == int(parts[2]), ln
        n += 1
    assert n >= 15


def test_user_method_library_builds_against_the_public_headers(lib, tmp_path):
    """A user library of do-all methods (tests/user_method.cu) compiles for
    sm_103a from include/ alone, links against libdsoa and exports its launchers;
    it needs dsoa_register_method, which libdsoa exports."""
    from paper_1810_11765_gb300 import build
    out = tmp_path / "libuser_methods.so"
    r = subprocess.run([build._nvcc(), *build.ARCH, "-O3", "-std=c++17", "-I", INCLUDE, "-shared",
                        "-Xcompiler", "-fPIC", "-cudart", "shared", "-o", str(out),
                        os.path.join(ROOT, "tests", "user_method.cu"), "-L", build.OUT, "-ldsoa"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    syms = subprocess.run(["nm", "-D", str(out)], capture_output=True, text=True).stdout
    for name in ("user_scale", "user_spawn", "user_mark"):
        assert re.search(rf" T {name}$", syms, flags=re.M), name
    assert re.search(r" U dsoa_register_method$", syms, flags=re.M)
    assert hasattr(lib, "dsoa_register_method")
