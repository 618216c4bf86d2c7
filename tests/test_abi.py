"""Host-side checks of the C ABI (no GPU needed): the library builds, loads,
and exports every entry point include/dgamp_ct.h declares, and the binding's
structs match the header's layout."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dgamp_ct.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dgamp_ct_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1609_04661_gb300 import build, binding
    build.build()
    return C.CDLL(binding.LIB_PATH)


def test_library_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert len(names) >= 15
    for nm in names:
        assert hasattr(lib, nm), f"{nm} declared in dgamp_ct.h but not exported"


def test_binding_lists_every_declared_symbol():
    from paper_1609_04661_gb300 import binding
    assert sorted(binding.EXPORTS) == _declared_functions()


def test_struct_layouts_match_header(lib, tmp_path):
    import shutil
    import subprocess
    from paper_1609_04661_gb300 import binding
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "dgamp_ct.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(dgamp_ct_geometry),'
                    ' sizeof(dgamp_ct_options), sizeof(dgamp_ct_stats), offsetof(dgamp_ct_options, seed),'
                    ' offsetof(dgamp_ct_options, use_graph), offsetof(dgamp_ct_stats, tau_x_floored),'
                    ' offsetof(dgamp_ct_options, tv_metric), sizeof(dgamp_ct_fan_geometry),'
                    ' offsetof(dgamp_ct_fan_geometry, det_spacing), sizeof(dgamp_ct_tuning),'
                    ' offsetof(dgamp_ct_tuning, pj_band), offsetof(dgamp_ct_tuning, pj_waves));'
                    'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [C.sizeof(binding.Geometry), C.sizeof(binding.Options), C.sizeof(binding.Stats),
            binding.Options.seed.offset, binding.Options.use_graph.offset,
            binding.Stats.tau_x_floored.offset, binding.Options.tv_metric.offset,
            C.sizeof(binding.FanGeometry), binding.FanGeometry.det_spacing.offset, C.sizeof(binding.Tuning),
            binding.Tuning.pj_band.offset, binding.Tuning.pj_waves.offset]
    assert got == want
    o = binding.Options()
    assert lib.dgamp_ct_default_options(C.byref(o)) == 0
    assert (o.k_tv, o.c_tv, o.eps_rel, o.onsager, o.use_graph) == (20, 3.0, 1e-3, 1, 1)


def test_argument_errors_need_no_device(lib):
    from paper_1609_04661_gb300 import binding
    f = lib.dgamp_ct_plan
    f.restype = C.c_int
    h = C.c_void_p()
    assert f(None, None, C.byref(h)) == -1
    g = binding.Geometry(1, 10, 10, None)          # n < 2
    assert f(C.byref(g), None, C.byref(h)) == -1
    o = binding.Options()
    lib.dgamp_ct_default_options(C.byref(o))
    o.eps_rel = -1.0
    g = binding.Geometry(16, 10, 24, None)
    assert f(C.byref(g), C.byref(o), C.byref(h)) == -1
    lib.dgamp_ct_strerror.restype = C.c_char_p
    assert lib.dgamp_ct_strerror(-3) == b"out of device memory"
    assert lib.dgamp_ct_solve(None, None, C.c_double(1.0), 1, None, None, None, None) == -1
    # fan beam: a source inside the image's circumscribed circle (plus margin)
    # or a zero bin pitch is refused before any device call
    fp = lib.dgamp_ct_plan_fan
    fp.restype = C.c_int
    assert fp(None, None, C.byref(h)) == -1
    for sd, dd, du in [(12.0, 100.0, 1.0), (100.0, 13.0, 1.0), (100.0, 100.0, 0.0), (2e8, 100.0, 1.0)]:
        fg = binding.FanGeometry(binding.Geometry(16, 10, 24, None), sd, dd, du)
        assert fp(C.byref(fg), None, C.byref(h)) == -1
